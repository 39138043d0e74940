"""Statistical accuracy of the observables: the FP32 filter, the plain FP64 form and the
FP64 oracle sample the same distribution (Sec. 3.5.2 FFBS, Sec. 3.5.4 Gibbs; the
estimators of Sec. 4).

Each side runs independent chains (disjoint seeds), discards a burn-in, and averages every
observable per chain over the measured sweeps; the chains' spread gives the standard
error, so autocorrelation within a chain does not bias it.  For every observable and
every pair of sides the test forms z = (a - b) / sqrt(se_a^2 + se_b^2).  Under a correct
sampler each z is a standard normal draw: the test asserts |z| < 4.5 for all of them and
that the FP32 and FP64 standard errors agree within 20% (equal accuracy per sweep).  Run
with `-s` to print the table of means, standard errors and z values.

The particle density is conserved by every move, so it must equal the filling exactly.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

NAMES = ("double_occ", "m2", "ekin", "s_pipi", "c_10")


def gpu_side(L, params, prec, seeds, burn, meas):
    from paper_2510_13866_gb300 import Lattice

    t, U, beta, dtau, fill = params
    lat = Lattice(L, list(seeds), precision=prec)
    lat.set_params(t, U, beta, dtau, fill)
    lat.sweep(burn)
    lat.measure(reset=True)
    lat.sweep(meas)
    obs = lat.measure()
    lat.close()
    assert all(o["n_samples"] == meas for o in obs)
    assert all(o["n_degenerate"] == 0 and o["n_nonpositive"] == 0 for o in obs)
    dens = np.array([o["density"] for o in obs])
    rows = np.array([[o["double_occ"], o["m2"], o["ekin"], o["s_pipi"], o["Cr"][1]] for o in obs])
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
    for j, name in enumerate(NAMES):
        m32, m64, mor = (sides[k][0][j] for k in ("fp32", "fp64", "oracle"))
        s32, s64, sor = (sides[k][1][j] for k in ("fp32", "fp64", "oracle"))
        z = [(m32 - m64) / np.hypot(s32, s64), (m32 - mor) / np.hypot(s32, sor), (m64 - mor) / np.hypot(s64, sor)]
        worst = max(worst, *map(abs, z))
        print(f"{name:>11} | {m32:12.6f} {s32:9.2e} | {m64:12.6f} {s64:9.2e} | {mor:12.6f} {sor:9.2e} | "
              + "  ".join(f"{v:+6.2f}" for v in z))
        assert all(abs(v) < 4.5 for v in z), (name, z)
        assert 0.8 < s32 / s64 < 1.25, (name, s32, s64)
    print(f"largest |z| = {worst:.2f}")
