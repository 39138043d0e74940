"""The FFBS filter with its line convolutions as a direct periodic stencil (the
truncated-stencil comparison) on the GPU, against the FP64 oracle, through the C ABI.

The stencil applies g(d) for |d| <= 6: for L <= 13 that is the exact circulant, and the
tolerances are the closed loop's (log-weights 1e-5 FP32, 1e-12 FP64; paths identical up
to a first draw within the tolerance of a CDF edge).  For larger L the dropped weight,
tail = sum over 6 < |d| of g(d) / sum_d g(d), bounds the relative change of each slice's
message, so the FP64 log-weight tolerance is max(1e-12, 4 M tail).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def tail(L, t, dtau):
    g, _ = oracle.g_table(L, t, dtau)
    d = np.minimum(np.arange(L), L - np.arange(L))
    return g[d > 6].sum() / g.sum()


def make(L, seeds, prec, params):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, seeds, precision=prec)
    lat.set_params(*params)
    lat.set_conv("stencil")
    return lat


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,params", [
    (3, (1.0, 2.0, 0.6, 0.1, 4 / 9)),
    (4, (1.0, 4.0, 1.0, 0.1, 1.0)),
    (6, (1.0, 4.0, 1.1, 0.1, 0.5)),
    (8, (1.0, 6.0, 1.3, 0.1, 0.75)),
    (12, (1.0, 4.0, 0.7, 0.1, 0.5)),
    (16, (1.0, 4.0, 0.5, 0.05, 1.0)),
    (24, (1.0, 8.0, 0.4, 0.05, 1.0)),
    (32, (1.0, 4.0, 0.45, 0.05, 1.0)),
])
def test_stencil_sweep_parity(prec, L, params):
    t, U, beta, dtau, fill = params
    lat = make(L, [7, 8], prec, params)
    logw = lat.sweep(1, logw=True)
    orc0 = oracle.Chain(L, *params, 7)
    tol = max(TOL[prec], 4 * orc0.M * tail(L, t, dtau))
    assert tol <= 1e-5
    for c in range(2):
        orc = oracle.Chain(L, *params, int(lat.seeds[c]))
        ref = orc.sweep(want_margin=True)
        s, x, a, _ = lat.get_state(c)
        assert a == ref["anchor"]
        assert rel_err(logw[c], ref["logw"]).max() <= tol, (c, rel_err(logw[c], ref["logw"]).max())
        _, firsts, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, max(tol, TOL[prec]))
        assert not bad, bad[:3]
    lat.close()


def test_stencil_has_no_degenerate_draws_at_low_temperature():
    """L = 32, U = 4, beta = 8, dtau = 0.05 (M = 160), half filling, 8 chains, 3 sweeps: the
    stencil filter's small values are sums of non-negative terms, so no draw meets an
    all-zero CDF and every amplitude at the held site is positive."""
    lat = make(32, list(range(8)), "fp32", (1.0, 4.0, 8.0, 0.05, 1.0))
    lat.sweep(3)
    for o in lat.measure():
        assert o["n_degenerate"] == 0 and o["n_nonpositive"] == 0
    lat.close()


def test_stencil_matches_fft_at_full_size():
    """L = 32, t=1, U=4, beta=4, dtau=0.05 (M = 80), 64 chains: the stencil and FFT filters
    give log-weights within 1e-5 of each other and of the oracle (first worldline of each
    spin of chain 0)."""
    from paper_2510_13866_gb300 import Lattice

    params = (1.0, 4.0, 4.0, 0.05, 1.0)
    a = make(32, list(range(64)), "fp32", params)
    b = Lattice(32, list(range(64)), precision="fp32")
    b.set_params(*params)
    la, lb = a.sweep(1, logw=True), b.sweep(1, logw=True)
    for c in range(64):
        assert rel_err(la[c], lb[c]).max() <= 2e-5
    orc = oracle.Chain(32, *params, 0)
    ref = orc.sweep(want_margin=True, nwl_limit=1)
    assert rel_err(la[0][:, :1], ref["logw"][:, :1]).max() <= 1e-5
    a.close()
    b.close()


def test_stencil_rejects_wide_lattices():
    from paper_2510_13866_gb300 import HQMCError, Lattice

    lat = Lattice(48, [0], precision="fp32")
    lat.set_params(1.0, 4.0, 0.2, 0.05, 0.5)
    with pytest.raises(HQMCError):
        lat.set_conv("stencil")
    lat.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stencil_with_blocks_and_permutations(prec):
    """The stencil form in the general work-unit instantiation: L = 8 (the exact 8-tap
    circulant), blocks of 3 slices, permutation updates; two sweeps against the oracle's
    permuted block sweep (log-weights, permutations, held sites)."""
    params = (1.0, 4.0, 1.0, 0.25, 0.5)  # M = 4
    lat = make(8, [5], prec, params)
    lat.set_block(3)
    lat.set_permutations(True)
    orc = oracle.Chain(8, *params, 5)
    for k in range(2):
        logw = lat.sweep(1, logw=True)[0]
        ref = orc.perm_sweep(want_margin=True, block=3)
        perm, sign = lat.get_perm(0)
        if not np.array_equal(perm, orc.perm):
            assert np.any(ref["margin_perm"] < 1e-12)
            break
        assert sign == orc.sign
        assert rel_err(logw, ref["logw"]).max() <= TOL[prec], k
        _, x, a, _ = lat.get_state(0)
        if prec == "fp64":
            assert np.array_equal(x, orc.x), k
        elif not np.array_equal(x, orc.x):
            break  # an FP32 draw at a CDF edge: the chains part here
    lat.close()
