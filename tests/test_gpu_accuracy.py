"""Statistical accuracy of the observables: the FP32 filter, the plain FP64 form and the
FP64 oracle sample the same distribution (Sec. 3.5.2 FFBS, Sec. 3.5.4 Gibbs; the
estimators of Sec. 4).

Each side runs independent chains (disjoint seeds), discards a burn-in, and averages every
observable per chain over the measured sweeps; the chains' spread gives the standard
error, so autocorrelation within a chain does not bias it.  Sides that run the same
Markov kernel from the same start share the law of every sweep, so they agree whether or
not the burn-in reached equilibrium; different kernels are compared after a long one.  For every observable and
every pair of sides the test forms z = (a - b) / sqrt(se_a^2 + se_b^2).  Under a correct
sampler each z is a standard normal draw: the test asserts |z| < 4.5 for all of them (a
gross-bias guard), that no more of them exceed 2 than a binomial count with
P(|z| > 2) = 0.0455 allows at the 99.9% level (the 2-sigma criterion: a bias of a few
sigma in any observable pushes its z values past 2), and that the FP32 and FP64 standard
errors agree within 20% (equal accuracy per sweep).  Run with `-s` to print the table of
means, standard errors and z values.

The particle density is conserved by every move, so it must equal the filling exactly.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

NAMES = ("double_occ", "m2", "ekin", "s_pipi", "c_10")
P2 = 0.0455  # P(|z| > 2) for a standard normal z


def two_sigma_limit(n, alpha=1e-3):
    """Largest count of |z| > 2 among n standard normal z values that a binomial law
    (n, P2) exceeds with probability below alpha."""
    from scipy.stats import binom

    k = 0
    while binom.sf(k, n, P2) >= alpha:
        k += 1
    return k


def check_two_sigma(zs):
    zs = np.abs(np.asarray(zs, dtype=float))
    n2, lim = int((zs > 2.0).sum()), two_sigma_limit(len(zs))
    print(f"|z| > 2: {n2} of {len(zs)} (binomial 99.9% limit {lim})")
    assert n2 <= lim, (n2, lim, sorted(zs)[-5:])


def gpu_side(L, params, prec, seeds, burn, meas, block=0, local=False, perm=False, signed=False):
    """Per-chain means of the library's estimators after `burn` discarded sweeps.  block:
    FFBS blocks of that many slices; local: every FFBS sweep followed by a local-update
    sweep (both measure); perm: pair-swap permutation updates (sign-reweighted).  With
    signed, returns the per-chain means of sign x observable and of the sign instead."""
    from paper_2510_13866_gb300 import Lattice

    t, U, beta, dtau, fill = params
    lat = Lattice(L, list(seeds), precision=prec)
    lat.set_params(t, U, beta, dtau, fill)
    if block:
        lat.set_block(block)
    if perm:
        lat.set_permutations(True)

    def run(n):
        if local:
            for _ in range(n // 2):
                lat.sweep(1)
                lat.local_sweep(1)
        else:
            lat.sweep(n)

    run(burn)
    lat.measure(reset=True)
    run(meas)
    obs = lat.measure()
    lat.close()
    assert all(o["n_samples"] == meas for o in obs)
    assert all(o["n_degenerate"] == 0 and o["n_nonpositive"] == 0 for o in obs)
    dens = np.array([o["density"] for o in obs])
    rows = np.array([[o["double_occ"], o["m2"], o["ekin"], o["s_pipi"], o["Cr"][1]] for o in obs])
    if signed:
        sg = np.array([o["mean_sign"] for o in obs])
        return rows * sg[:, None], sg
    assert all(o["mean_sign"] == 1.0 for o in obs)
    return dens, rows


def oracle_side(L, params, seeds, burn, meas):
    """Per-chain means of the oracle's estimators: the sums of `oracle.measure` over the
    M slices and N sites, divided as the library's read-out divides them."""
    t, U, beta, dtau, fill = params
    N = L * L
    kpp = L // 2 + L * (L // 2)
    dens, rows = [], []
    for sd in seeds:
        ch = oracle.Chain(L, t, U, beta, dtau, fill, sd)
        for _ in range(burn):
            ch.sweep()
        acc = np.zeros(6)
        for _ in range(meas):
            r = ch.sweep()
            m = oracle.measure(L, ch.M, r["hist"])
            MN = ch.M * N
            acc += [m["n"] / MN, m["d"] / MN, m["m2"] / MN, -(t / beta) * r["links"].sum() / N,
                    m["Sk"][kpp] / (4 * ch.M), m["Cr"][1] / (4 * ch.M)]
        acc /= meas
        dens.append(acc[0])
        rows.append(acc[1:])
    return np.array(dens), np.array(rows)


def mean_se(rows):
    return rows.mean(axis=0), rows.std(axis=0, ddof=1) / np.sqrt(len(rows))


@pytest.mark.parametrize("L,params,n_gpu,n_orc,burn,meas", [
    (4, (1.0, 4.0, 2.0, 0.1, 1.0), 1024, 48, 100, 400),   # the plain-method case: L=4, U=4, beta=2, M=20
    (6, (1.0, 8.0, 2.0, 0.1, 0.5), 1024, 24, 100, 300),   # quarter filling, odd worldline count, U=8
])
def test_fp32_fp64_and_oracle_agree_statistically(L, params, n_gpu, n_orc, burn, meas):
    fill = params[4]
    d32, r32 = gpu_side(L, params, "fp32", range(10_000, 10_000 + n_gpu), burn, meas)
    d64, r64 = gpu_side(L, params, "fp64", range(20_000, 20_000 + n_gpu), burn, meas)
    dor, ror = oracle_side(L, params, range(30_000, 30_000 + n_orc), burn, meas)
    for d in (d32, d64, dor):
        assert np.allclose(d, fill, rtol=0, atol=1e-12)
    sides = {"fp32": mean_se(r32), "fp64": mean_se(r64), "oracle": mean_se(ror)}
    print(f"\nL={L} (t, U, beta, dtau, filling)={params}: GPU {n_gpu} chains per precision, "
          f"oracle {n_orc} chains, {burn} + {meas} sweeps each")
    print(f"{'observable':>11} | {'fp32 mean':>12} {'se':>9} | {'fp64 mean':>12} {'se':>9} | "
          f"{'oracle mean':>12} {'se':>9} | z32-64  z32-orc  z64-orc")
    worst = 0.0
    allz = []
    for j, name in enumerate(NAMES):
        m32, m64, mor = (sides[k][0][j] for k in ("fp32", "fp64", "oracle"))
        s32, s64, sor = (sides[k][1][j] for k in ("fp32", "fp64", "oracle"))
        z = [(m32 - m64) / np.hypot(s32, s64), (m32 - mor) / np.hypot(s32, sor), (m64 - mor) / np.hypot(s64, sor)]
        allz += z
        worst = max(worst, *map(abs, z))
        print(f"{name:>11} | {m32:12.6f} {s32:9.2e} | {m64:12.6f} {s64:9.2e} | {mor:12.6f} {sor:9.2e} | "
              + "  ".join(f"{v:+6.2f}" for v in z))
        assert all(abs(v) < 4.5 for v in z), (name, z)
        assert 0.8 < s32 / s64 < 1.25, (name, s32, s64)
    print(f"largest |z| = {worst:.2f}")
    check_two_sigma(allz)


def table(title, sides, names, ref=None):
    """Print means, errors and z values of every side against `ref` (default: all pairs);
    returns the largest |z|."""
    keys = list(sides)
    pairs = [(a, b) for i, a in enumerate(keys) for b in keys[i + 1:]] if ref is None else \
        [(ref, b) for b in keys if b != ref]
    print("\n" + title)
    print(f"{'observable':>11} | " + " | ".join(f"{k:>10} mean {'se':>9}" for k in keys) + " | "
          + "  ".join(f"z {a}-{b}" for a, b in pairs))
    worst = 0.0
    allz = []
    for j, name in enumerate(names):
        z = [(sides[a][0][j] - sides[b][0][j]) / np.hypot(sides[a][1][j], sides[b][1][j]) for a, b in pairs]
        allz += z
        worst = max(worst, *map(abs, z))
        print(f"{name:>11} | " + " | ".join(f"{sides[k][0][j]:15.6f} {sides[k][1][j]:9.2e}" for k in keys)
              + " | " + "  ".join(f"{v:+6.2f}" for v in z))
        assert all(abs(v) < 4.5 for v in z), (name, z)
    print(f"largest |z| = {worst:.2f}")
    check_two_sigma(allz)
    return worst


def test_update_schemes_share_the_stationary_law():
    """Closed-loop FFBS, FFBS in blocks with held ends (Sec. 3.5.2) and FFBS sweeps
    interleaved with local link moves (Sec. 3.5.1) are different Markov kernels with the
    same stationary law: their equilibrium observables agree (FP32, 1024 chains each,
    disjoint seeds, at the plain-method case L=4, U=4, beta=2, M=20).  Short blocks move a
    worldline slowly: from the static start, the double occupancy of B=3 chains reaches its
    equilibrium only after about 300 sweeps (B=2: more than 500), and interleaved local
    sweeps halve the FFBS sweeps, so every scheme discards 4000."""
    L, params, n, burn, meas = 4, (1.0, 4.0, 2.0, 0.1, 1.0), 1024, 4000, 1000
    sides = {}
    for name, kw, base in (("closed", {}, 40_000), ("B=5", {"block": 5}, 50_000),
                           ("+local", {"local": True}, 60_000), ("B=3+local", {"block": 3, "local": True}, 70_000)):
        d, r = gpu_side(L, params, "fp32", range(base, base + n), burn, meas, **kw)
        assert np.allclose(d, params[4], rtol=0, atol=1e-12)
        sides[name] = mean_se(r)
    table(f"L={L} {params}: update schemes, {n} FP32 chains each, {burn} + {meas} sweeps", sides, NAMES,
          ref="closed")


def oracle_perm_side(L, params, seeds, burn, meas):
    """Per-chain means of sign x estimator and of the sign, from the oracle's sweeps with
    pair-swap permutation updates (Eq. reweight: <O> = <sgn O> / <sgn>)."""
    t, U, beta, dtau, fill = params
    N = L * L
    kpp = L // 2 + L * (L // 2)
    num, den = [], []
    for sd in seeds:
        ch = oracle.Chain(L, t, U, beta, dtau, fill, sd)
        for _ in range(burn):
            ch.perm_sweep()
        acc, sg = np.zeros(5), 0.0
        for _ in range(meas):
            r = ch.perm_sweep()
            m = oracle.measure(L, ch.M, r["hist"])
            MN = ch.M * N
            acc += r["sign"] * np.array([m["d"] / MN, m["m2"] / MN, -(t / beta) * r["links"].sum() / N,
                                         m["Sk"][kpp] / (4 * ch.M), m["Cr"][1] / (4 * ch.M)])
            sg += r["sign"]
        num.append(acc / meas)
        den.append(sg / meas)
    return np.array(num), np.array(den)


def ratio_se(num, den):
    """<sgn O> / <sgn> over independent chains and its delta-method standard error; the
    mean sign with its error is appended as the last entry."""
    n = len(den)
    R = num.mean(axis=0) / den.mean()
    resid = num - R[None, :] * den[:, None]
    se = resid.std(axis=0, ddof=1) / np.sqrt(n) / abs(den.mean())
    return (np.append(R, den.mean()), np.append(se, den.std(ddof=1) / np.sqrt(n)))


def test_permutation_observables_agree_statistically():
    """Sign-reweighted observables and the mean sign with pair-swap permutation updates
    (Sec. 3.5.3): FP32, FP64 and the oracle agree.  L=6 with two worldlines per spin at
    beta=0.5, where swaps are frequent (0.3 per sweep) and the mean sign is about 0.6."""
    L, params, n_gpu, n_orc, burn, meas = 6, (1.0, 4.0, 0.5, 0.1, 1.0 / 9.0), 1024, 128, 100, 400
    sides = {}
    for prec, base in (("fp32", 80_000), ("fp64", 90_000)):
        num, den = gpu_side(L, params, prec, range(base, base + n_gpu), burn, meas, perm=True, signed=True)
        sides[prec] = ratio_se(num, den)
    sides["oracle"] = ratio_se(*oracle_perm_side(L, params, range(100_000, 100_000 + n_orc), burn, meas))
    assert 0.3 < sides["fp32"][0][-1] < 0.9
    table(f"L={L} {params} with permutation updates: GPU {n_gpu} chains per precision, oracle {n_orc} "
          f"chains, {burn} + {meas} sweeps", sides, NAMES + ("mean_sign",))
