"""GPU open-path estimator of the one-body density matrix and n_k (Sec. 4, "Observables")
against closed forms and the oracle, through the C ABI (hqmc_set_measure_open,
hqmc_measure_open).

  - U = 0 without permutations, closed loops: every worldline's end message is the free
    propagator from its own end site, so each sample is exactly A(r) = 2 Nsig G_b(r) / G_b(0)
    with b = beta and G_b = g_b (x) g_b, and n_k = 2 Nsig e^{-b eps_k} / sum_k e^{-b eps_k}
    (Boltzmann particles per spin): the warp kernel and the wide kernel, FP32 (1e-5) and
    FP64 (1e-11).  (With blocks the last block runs from its held start x_s to x_e, a sample
    is G_b(x_e + r - x_s) / G_b(x_e - x_s) with b its length, and only the ensemble mean is
    G_beta(r) / G_beta(0); blocks are covered by the next check.)
  - U != 0: one sweep from a shared state, the GPU's sums against the oracle's
    open_estimate (orc_open_ratio over every worldline's last block) element by element,
    closed loops, blocks and permutations.
  - U = 0 with permutation updates, two fermions per spin: the sign-reweighted estimator
    gives the canonical free-fermion occupation n_k = e^{-b eps_k}(Z_1 - e^{-b eps_k}) / Z_2
    per spin, Z_1 = sum_k e^{-b eps_k}, Z_2 = (Z_1^2 - sum_k e^{-2 b eps_k}) / 2
    (statistical, 4096 chains).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-11}


def free_prop_ratio(L, t, b):
    """G_b(r) / G_b(0) for r = rx + L ry, with G_b the product of the 1D propagators of
    imaginary time b (the Trotterised propagator is exact at U = 0)."""
    k = 2 * np.pi * np.arange(L) / L
    gk = np.exp(2 * t * b * np.cos(k))
    g = np.real(np.fft.ifft(gk))  # g_b(d) = (1/L) sum_k e^{2 t b cos k} e^{ikd}
    G = np.outer(g, g).reshape(-1)  # index ry * L + rx
    return G / G[0], gk


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,M,dtau,fill,block", [(4, 8, 0.1, 0.5, 0), (8, 6, 0.1, 1.0, 0), (32, 5, 0.05, 0.25, 0),
                                                 (48, 5, 0.05, 0.125, 0), (64, 4, 0.05, 0.125, 0)])
def test_open_u0_closed_form(L, M, dtau, fill, block, prec):
    from paper_2510_13866_gb300 import Lattice

    t = 1.0
    N = L * L
    lat = Lattice(L, [3, 4], precision=prec)
    lat.set_params(t, 0.0, M * dtau, dtau, fill)
    if block:
        lat.set_block(block)
    lat.set_measure_open(True)
    nsw = 3
    lat.sweep(nsw)
    _, _, ns = lat.shapes[0]
    B = block if 0 < block < M else M
    last = M - (M + B - 1) // B * B + B  # length of the last block
    ratio, gk = free_prop_ratio(L, t, last * dtau)
    want_dm = 2 * ns * ratio / N
    w = np.exp(2 * t * last * dtau * (np.cos(2 * np.pi * np.arange(L) / L)[None, :] +
                                      np.cos(2 * np.pi * np.arange(L) / L)[:, None])).reshape(-1)
    want_nk = 2 * ns * w / w.sum()
    for c, (nk, dm) in enumerate(lat.measure_open()):
        scale = np.abs(want_dm).max()
        assert np.abs(dm - want_dm).max() <= TOL[prec] * scale, (c, np.abs(dm - want_dm).max() / scale)
        assert np.abs(nk - want_nk).max() <= TOL[prec] * want_nk.max(), (c, np.abs(nk - want_nk).max())
        assert np.isclose(nk.mean(), 2 * ns / N, rtol=TOL[prec])
    lat.close()


def gpu_and_oracle_one_sweep(L, params, seed, prec, block=0, perm=False, warm=2):
    """(GPU sums of one sweep, oracle sums of the same sweep) from a shared state."""
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, [seed], precision=prec)
    lat.set_params(*params)
    if block:
        lat.set_block(block)
    if perm:
        lat.set_permutations(True)
    lat.sweep(warm)
    s, x, _, sw = lat.get_state(0)
    P, _ = lat.get_perm(0)
    lat.set_measure_open(True)
    lat.sweep(1)
    _, dm = lat.measure_open()[0]
    P1, sign = lat.get_perm(0)
    _, _, a, _ = lat.get_state(0)
    lat.close()
    orc = oracle.Chain(L, *params, seed)
    orc.s[:] = s
    orc.x[:] = x
    orc.perm[:] = P1  # the unit structure follows the permutation after this sweep's update
    orc.sweep_count = sw
    ref = sign * orc.open_estimate(orc.slice_potentials(), a, block)
    return dm * L * L, ref


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,params,block,perm", [
    (4, (1.0, 4.0, 1.0, 0.1, 1.0), 0, False),
    (6, (1.0, 8.0, 0.6, 0.1, 0.5), 3, False),
    (8, (1.0, 4.0, 0.5, 0.05, 0.25), 0, True),
    (16, (1.0, 2.0, 0.4, 0.05, 0.125), 0, False),
    (48, (1.0, 4.0, 0.25, 0.05, 14 / 2304), 0, False),
    (64, (1.0, 4.0, 0.3, 0.05, 6 / 4096), 2, False),
    (48, (1.0, 4.0, 0.3, 0.05, 10 / 2304), 0, True),
])
def test_open_one_sweep_matches_oracle(L, params, block, perm, prec):
    got, ref = gpu_and_oracle_one_sweep(L, params, 7, prec, block, perm)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL[prec] * 10 * scale, np.abs(got - ref).max() / scale


def test_open_free_fermions_with_permutations():
    """U = 0, L = 4, two worldlines per spin, beta = 0.75, dtau = 0.25 (M = 3) with pair-swap
    permutation updates: the sign-reweighted n_k equals the canonical two-fermion occupation
    (per spin, times two spins) within 4.5 standard errors at every k, over 4096 chains."""
    from paper_2510_13866_gb300 import Lattice

    L, t, beta, dtau = 4, 1.0, 0.75, 0.25
    N = L * L
    kk = 2 * np.pi * np.arange(L) / L
    w = np.exp(2 * t * beta * (np.cos(kk)[None, :] + np.cos(kk)[:, None])).reshape(-1)  # e^{-beta eps_k}
    Z1, Z2 = w.sum(), 0.5 * (w.sum() ** 2 - (w ** 2).sum())
    want = 2 * w * (Z1 - w) / Z2
    assert np.isclose(want.sum(), 4.0)
    nch = 4096
    lat = Lattice(L, list(range(70000, 70000 + nch)), precision="fp32")
    lat.set_params(t, 0.0, beta, dtau, 0.25)
    lat.set_permutations(True)
    lat.sweep(30)
    lat.set_measure_open(True)
    nsw = 100
    lat.sweep(nsw)
    obs = lat.measure()
    res = lat.measure_open()
    ssum = np.array([o["mean_sign"] * o["n_samples"] for o in obs])
    num = np.array([nk for nk, _ in res]) * ssum[:, None]  # per chain: sum over sweeps of sign x n_k
    est = num.sum(axis=0) / ssum.sum()
    z = num - est[None, :] * ssum[:, None]
    se = z.std(axis=0, ddof=1) * np.sqrt(nch) / abs(ssum.sum())
    boltz = 4 * w / w.sum()  # distinguishable particles: what a sign-blind estimator gives
    assert np.all(np.abs(est - want) < 4.5 * se + 1e-9), (est, want, se)
    assert np.abs(boltz - want).max() > 10 * se.max(), (boltz, want, se)
    lat.close()
