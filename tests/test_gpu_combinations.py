"""48 seeded random combinations of the sweep's options against the FP64 oracle, through the
C ABI: lattice size (warp and wide kernels), worldline count, number of slices, U of
either sign (Hirsch or Gaussian field), FFBS blocks, permutation updates, the stencil
convolution, precision, and ragged batches mixing all of these per chain.

Every case runs two sweeps on the GPU and in the oracle from the same seeds, then (if no
chain has met a CDF edge) one local-update sweep.  Per chain:
the anchor, the permutation and its sign, the filter log-weights (1e-5 relative in FP32,
1e-12 in FP64), and the worldlines in draw order, which must agree up to a first
difference at a draw whose uniform lies within the tolerance of a CDF edge; after a
sweep with no such difference the fields must agree as well.  A chain stops being
compared after its first difference, since the two samplers then follow different paths.

The FFT convolution resolves a message only to about eps log2(N) of its largest value
(eps = 2^-24 in FP32, 2^-53 in FP64), so the log-weight of a unit whose end site carries
a small share of the final message, kappa = max_y alpha(y) / alpha(x_end), is known only
to about eps kappa per block.  Strong Gaussian fields (U < 0 with large |U| dtau) reach
kappa = 1e4 to 1e15 within two sweeps.  The library reports an error estimate per
log-weight (hqmc_logw_error: eps log2(N) len kappa per block, with its own kappa) and
counts those above the tolerance (hqmc_obs.n_inexact).  Under a Gaussian field the message
can concentrate more at interior slices than at the end, so there the library sums, over
the unit's positions i, the mean of max_y alpha_i(y) / alpha_i(x_i) given the site x_{i+1}
it has just drawn (times a calibration factor in FP64), instead of taking len times the
end's.  Every log-weight it does not flag must meet the plain tolerance; a flagged one must
lie within its estimate; and on a single-block unit the library's kappa must be the one the
oracle's messages give (for a Gaussian field, along the GPU's drawn path).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err
from test_gpu_perm import unit_mismatches

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
EPS = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
# the library's calibration factor of the sampled part of a Gaussian-field estimate
GAUSS_FACTOR = {"fp32": 1.0, "fp64": 32.0}
SIZES = (2, 3, 4, 6, 8, 12, 16, 24, 32, 48)


def draw_cases(n=48, seed=2510):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        chains = []
        for _ in range(3 if k % 4 == 3 else 1):
            L = int(rng.choice(SIZES))
            N = L * L
            big = L >= 24  # the oracle's direct convolution costs N^2 per slice
            nsig = int(rng.integers(1, (8 if big else N) + 1))
            dtau = float(rng.choice([0.05, 0.1, 0.125, 0.2, 0.25]))
            M = int(rng.integers(1, (10 if big else 24) + 1))
            U = float(rng.choice([-4.0, 2.0, 4.0, 8.0]))
            block = int(rng.integers(1, M + 1)) if rng.random() < 0.4 else 0
            chains.append((L, (1.0, U, M * dtau, dtau, 2.0 * nsig / N), block))
        perm = bool(rng.random() < 0.35)
        prec = "fp64" if rng.random() < 0.4 and all(c[0] <= 32 for c in chains) else "fp32"
        # the stencil (|d| <= 6) is the exact circulant for L <= 13 and is not built for
        # the wide kernel
        stencil = bool(rng.random() < 0.25 and all(c[0] <= 12 for c in chains))
        out.append((chains, perm, prec, stencil))
    return out


CASES = draw_cases()

# |log-weight error| / the library's estimate, per precision and convolution, gathered by the
# random combinations and summarised by the last test of this file
RATIOS = {}


def slice_potentials(orc):
    """W [2][M][N] of the oracle chain's current fields (Hirsch: exp(+-lambda s) by spin;
    Gaussian: exp(a sigma) for both spins)."""
    if orc.gauss:
        w = np.exp(oracle.gauss_coupling(orc.U, orc.dtau) * orc.sigma)
        return np.stack([w, w])
    lam = oracle.lam(orc.U, orc.dtau)
    return np.stack([np.exp(lam * orc.s), np.exp(-lam * orc.s)])


def unit_kappa(orc, W, a, block, sg, p):
    """Sum over the blocks of worldline p's unit of max_y alpha_end(y) / alpha_end(x_end),
    with the held sites read from the chain after the sweep (they do not move)."""
    L, M, N = orc.L, orc.M, orc.N
    g, _ = oracle.g_table(L, orc.t, orc.dtau)
    G = np.fft.fft2(np.outer(g, g))
    q = orc.perm[sg, p]
    vp = np.where(np.arange(M) < a, orc.x[sg, q], orc.x[sg, p])
    vp[a] = orc.x[sg, q, a]
    B = block if 0 < block < M else M
    kap = 0.0
    for b in range(0, M, B):
        l0, ln = (a + b) % M, min(B, M - b)
        xs = orc.x[sg, p, a] if b == 0 else vp[l0]
        xe = vp[(l0 + ln) % M]
        _, f = oracle.filter_block(L, M, g, W[sg], l0, ln, int(xs), int(xe), want_f=True)
        al = np.real(np.fft.ifft2(np.fft.fft2(f[(l0 + ln - 1) % M].reshape(L, L)) * G)).reshape(-1)
        kap += al.max() / max(al[xe], 1e-300)
    return kap


def unit_kappa_sum(orc, W, a, sg, p, x_new, factor):
    """Gaussian-field form for a closed single-block unit, from the oracle's messages at the
    sites x_new the GPU drew: factor * sum over positions i = 1..M-1 of
    max_y alpha_i(y) sum_y W_i(y) G(x_{i+1} - y) / sum_y f_i(y) G(x_{i+1} - y) (the mean of
    max alpha_i / alpha_i(x_i) given x_{i+1}), plus the end's max alpha_M / alpha_M(x_M)."""
    L, M, N = orc.L, orc.M, orc.N
    g, _ = oracle.g_table(L, orc.t, orc.dtau)
    G = np.fft.fft2(np.outer(g, g))
    xa = int(x_new[sg, p, a])
    _, f = oracle.filter_block(L, M, g, W[sg], a, M, xa, xa, want_f=True)
    ys = np.arange(N)

    def gcol(x):  # G(x - y) for every y
        return g[(x % L - ys % L) % L] * g[(x // L - ys // L) % L]

    tot = 0.0
    for i in range(1, M):
        li = (a + i) % M
        fi, wi = f[li], W[sg][li]
        gx = gcol(int(x_new[sg, p, (a + i + 1) % M]))
        tot += (fi / wi).max() * (wi @ gx) / max(fi @ gx, 1e-300)
    al = np.real(np.fft.ifft2(np.fft.fft2(f[(a + M - 1) % M].reshape(L, L)) * G)).reshape(-1)
    return factor * tot + al.max() / max(al[xa], 1e-300)


def case_id(case):
    chains, perm, prec, stencil = case
    parts = [f"L{L}M{round(p[2] / p[3])}n{round(p[4] * L * L / 2)}U{p[1]:g}" + (f"B{b}" if b else "")
             for L, p, b in chains]
    return "-".join(parts) + ("-perm" if perm else "") + f"-{prec}" + ("-stencil" if stencil else "")


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_random_combination_matches_oracle(case):
    from paper_2510_13866_gb300 import HQMCError, Lattice

    chains, perm, prec, stencil = case
    tol = TOL[prec]
    seeds = [101 + 7 * c for c in range(len(chains))]
    lat = Lattice([c[0] for c in chains], seeds, precision=prec)
    for c, (L, params, block) in enumerate(chains):
        lat.set_params(*params, chain=c)
        if block:
            lat.set_block(block, chain=c)
    if stencil:
        lat.set_conv("stencil")
    if perm and min(round(p[2] / p[3]) for _, p, _ in chains) < 2:
        # documented: a swap at tau = beta needs two distinct slices around it
        with pytest.raises(HQMCError) as err:
            lat.set_permutations(True)
            lat.sweep(1)
        assert err.value.code == -6  # HQMC_ERR_UNSUPPORTED
        lat.close()
        return
    if perm:
        lat.set_permutations(True)
    orcs = [oracle.Chain(L, *params, sd) for (L, params, _), sd in zip(chains, seeds)]
    live = [True] * len(chains)
    for k in range(2):
        logw = lat.sweep(1, logw=True)
        lerr = lat.logw_error()
        nflag = [o["n_inexact"] for o in lat.measure(reset=True)]
        for c, ((L, params, block), orc) in enumerate(zip(chains, orcs)):
            if not live[c]:
                continue
            W = slice_potentials(orc)  # the fields this sweep filters with
            if perm:
                ref = orc.perm_sweep(want_margin=True, block=block)
                p_gpu, sign = lat.get_perm(c)
                if not np.array_equal(p_gpu, orc.perm):
                    # a swap decision within 1e-12 of its acceptance ratio
                    assert np.any(ref["margin_perm"] < 1e-12), (k, c)
                    live[c] = False
                    continue
                assert sign == orc.sign, (k, c)
            else:
                ref = orc.sweep(want_margin=True, block=block)
            s, x, a, sw = lat.get_state(c)
            assert sw == k + 1 and a == ref["anchor"], (k, c)
            err = rel_err(logw[c], ref["logw"])
            flagged = ~(lerr[c] <= tol * np.maximum(1.0, np.abs(logw[c])))
            ok = np.isfinite(lerr[c]) & np.isfinite(ref["logw"]) & (lerr[c] > 0)
            RATIOS.setdefault((prec, stencil, params[1] < 0), []).extend(
                (np.abs(logw[c] - ref["logw"])[ok] / lerr[c][ok]).tolist())
            assert nflag[c] == int(flagged.sum()), (k, c, nflag[c], int(flagged.sum()))
            for sg, p in zip(*np.nonzero(err > tol)):
                # beyond the plain tolerance only where the library flags the log-weight, and
                # then within its own estimate
                assert flagged[sg, p], (k, c, sg, p, err[sg, p], lerr[c][sg, p])
                absdiff = abs(logw[c][sg, p] - ref["logw"][sg, p])
                assert absdiff <= max(lerr[c][sg, p], tol * max(1.0, abs(ref["logw"][sg, p]))), \
                    (k, c, sg, p, absdiff, lerr[c][sg, p])
            if stencil or (0 < block < orc.M):
                continue
            for sg, p in zip(*np.nonzero(flagged)):
                if not np.isfinite(lerr[c][sg, p]):
                    continue  # a non-positive end value (counted in n_nonpositive as well)
                # one block of M slices: the estimate is eps log2(N) M kappa with the library's
                # own kappa, which must be the oracle's where the end value is resolved at all
                # (kappa well below 1 / eps)
                kap_gpu = lerr[c][sg, p] / (EPS[prec] * np.log2(orc.N) * orc.M)
                if orc.gauss:
                    if perm:
                        continue  # the unit's path crosses worldlines at the permuted boundary
                    kap = unit_kappa_sum(orc, W, a, sg, p, x, GAUSS_FACTOR[prec]) / orc.M
                else:
                    kap = unit_kappa(orc, W, a, block, sg, p)
                if kap < 1e-3 / EPS[prec]:
                    assert 0.5 < kap_gpu / kap < 2.0, (k, c, sg, p, kap_gpu, kap)
            if perm:
                firsts, bad = unit_mismatches(x, orc.x, ref["margin"], a, orc.M, orc.perm, tol, block)
            else:
                _, firsts, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, tol, block=block)
            assert not bad, (k, c, bad[:3])
            if firsts:
                live[c] = False
                continue
            if orc.gauss:
                assert np.allclose(lat.get_sigma(c), orc.sigma, rtol=0, atol=1e-12), (k, c)
            else:
                assert np.array_equal(s, orc.s), (k, c)
    if all(live):
        # then a local-update sweep (Sec. 3.5.1) from the shared state: both sides form the
        # acceptance ratio in FP64, so a worldline may differ only where one of its
        # decisions lay within 1e-12 of the ratio
        lat.local_sweep(1)
        for c, orc in enumerate(orcs):
            ref = orc.local_sweep(want_margin=True)
            s, x, _, sw = lat.get_state(c)
            assert sw == 3, c
            bad = [(sg, p) for sg in range(2) for p in range(orc.Nsig)
                   if not np.array_equal(x[sg, p], orc.x[sg, p]) and not np.any(ref["margin"][sg, p] < 1e-12)]
            assert not bad, (c, bad[:3])
            if np.array_equal(x, orc.x):
                if orc.gauss:
                    assert np.allclose(lat.get_sigma(c), orc.sigma, rtol=0, atol=1e-12), c
                else:
                    assert np.array_equal(s, orc.s), c
    lat.close()


def test_autotune_keeps_results_with_every_option():
    """The CTA-shape autotuner times throwaway copies that carry the context's blocks,
    permutation updates and convolution form, and leaves the chains untouched: a context
    tuned after one sweep continues bit for bit like one that was never tuned."""
    from paper_2510_13866_gb300 import Lattice

    Ls = [8, 12, 12, 6]
    pars = [(1.0, 4.0, 1.0, 0.1, 1.0), (1.0, -4.0, 0.8, 0.1, 0.5), (1.0, 2.0, 1.2, 0.1, 0.25),
            (1.0, 8.0, 0.5, 0.1, 1.0)]
    blocks = [3, 0, 5, 2]

    def make():
        lat = Lattice(Ls, [60, 61, 62, 63], precision="fp32")
        for c, (p, b) in enumerate(zip(pars, blocks)):
            lat.set_params(*p, chain=c)
            if b:
                lat.set_block(b, chain=c)
        lat.set_permutations(True)
        lat.set_conv("stencil")
        return lat

    ref = make()
    lw_ref = ref.sweep(3, logw=True)
    st_ref = [(ref.get_state(c), ref.get_perm(c)) for c in range(len(Ls))]
    sig_ref = ref.get_sigma(1)
    ref.close()

    lat = make()
    lat.sweep(2)
    lat.autotune(trial_sweeps=2)
    assert all(lat.get_state(c)[3] == 2 for c in range(len(Ls)))
    lw = lat.sweep(1, logw=True)
    for c in range(len(Ls)):
        assert np.array_equal(lw[c], lw_ref[c]), c
        (s, x, a, sw), (perm, sign) = lat.get_state(c), lat.get_perm(c)
        (s0, x0, a0, sw0), (perm0, sign0) = st_ref[c]
        assert np.array_equal(s, s0) and np.array_equal(x, x0) and a == a0 and sw == sw0 == 3, c
        assert np.array_equal(perm, perm0) and sign == sign0, c
    assert np.array_equal(lat.get_sigma(1), sig_ref)
    lat.close()


def test_zz_error_estimate_calibration():
    """Distribution of |log-weight error| / estimate over the random combinations above (run
    with -s to print it).  The FP32 FFT filter's errors stay within their estimate (for
    Hirsch fields eps log2(N) len kappa with the end concentration standing in for every
    slice's; for Gaussian fields the concentrations at the drawn sites summed).  FP64 is
    printed, not bounded."""
    if not RATIOS:
        pytest.skip("the random combinations did not run in this session")
    print()
    for (prec, stencil, gauss), r in sorted(RATIOS.items()):
        r = np.asarray(r)
        print(f"{prec} {'stencil' if stencil else 'fft':>7} {'U<0' if gauss else 'U>=0':>4}: {len(r):5d} log-weights, "
              f"error / estimate: median {np.median(r):.3g}, 99th percentile {np.percentile(r, 99):.3g}, "
              f"max {r.max():.3g}")
    fp32_fft = [np.asarray(r) for (prec, st, _), r in RATIOS.items() if prec == "fp32" and not st]
    if fp32_fft:
        assert np.concatenate(fp32_fft).max() <= 1.0, np.concatenate(fp32_fft).max()
