"""Block FFBS (Sec. 3.5.2: a block of slices resampled with its two end sites held) on the
GPU against the FP64 oracle, through the C ABI.

With block length B < M the loop is cut at the anchor a into blocks a, a+B, a+2B, ...
(the last one shorter when B does not divide M); every block's interior is drawn given
its held ends, and the sweep's log-weight is the sum of the blocks'.  Tolerances as for
the closed loop: log-weights 1e-5 (FP32) / 1e-12 (FP64) relative to max(1, |log Z|);
paths identical within each block up to a first draw within the tolerance of a CDF
edge; held sites identical; the field identical wherever the occupancies agree.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def make(Ls, seeds, prec, params, B):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(Ls, seeds, precision=prec)
    lat.set_params(*params)
    lat.set_block(B)
    return lat


def occupancy(x, M, N):
    n = np.zeros((2, M, N), dtype=np.int64)
    for sg in range(2):
        for p in range(x.shape[1]):
            np.add.at(n[sg], (np.arange(M), x[sg, p]), 1)
    return n


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,params,B", [
    (4, (1.0, 4.0, 1.0, 0.1, 1.0), 1),       # M = 10: every slice held, nothing drawn
    (4, (1.0, 4.0, 1.0, 0.1, 1.0), 2),       # M = 10: 5 blocks of 2
    (6, (1.0, 4.0, 1.1, 0.1, 0.5), 4),       # M = 11: blocks 4, 4, 3
    (3, (1.0, 2.0, 0.6, 0.1, 4 / 9), 5),     # M = 6: blocks 5, 1
    (8, (1.0, 6.0, 1.3, 0.1, 0.75), 3),      # M = 13: odd and even block lengths
    (16, (1.0, 4.0, 0.5, 0.05, 1.0), 7),     # M = 10: blocks 7, 3
    (32, (1.0, 4.0, 0.45, 0.05, 1.0), 4),    # M = 9: blocks 4, 4, 1
    (8, (1.0, -4.0, 1.0, 0.1, 1.0), 3),      # U < 0, Gaussian field: blocks 3, 3, 3, 1
])
def test_block_sweep_parity(prec, L, params, B):
    lat = make(L, [7, 8], prec, params, B)
    logw = lat.sweep(1, logw=True)
    draws = 0
    for c in range(2):
        orc = oracle.Chain(L, *params, int(lat.seeds[c]))
        before = orc.x.copy()
        ref = orc.sweep(want_margin=True, block=B)
        s, x, a, _ = lat.get_state(c)
        assert a == ref["anchor"]
        assert rel_err(logw[c], ref["logw"]).max() <= TOL[prec]
        d, firsts, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, TOL[prec], block=B)
        assert not bad, bad[:3]
        draws += d
        if prec == "fp64":
            assert firsts == 0
        held = [(a + k) % orc.M for k in range(0, orc.M, B)]
        assert np.array_equal(x[:, :, held], before[:, :, held])
        same = np.all(occupancy(x, orc.M, L * L) == ref["hist"], axis=0)
        if orc.gauss:
            assert np.allclose(lat.get_sigma(c)[same], orc.sigma[same], rtol=0, atol=1e-12)
        else:
            assert np.array_equal(s[same], orc.s[same])
    if B == 1:
        assert draws == 0
    lat.close()


def test_block_length_m_or_more_is_the_closed_loop():
    """B = M, B > M and B = 0 give the same bits (FP32, L = 16, three sweeps)."""
    params = (1.0, 4.0, 1.0, 0.05, 1.0)  # M = 20
    outs = []
    for B in (0, 20, 57):
        lat = make(16, [3, 4], "fp32", params, B)
        lw = [lat.sweep(1, logw=True) for _ in range(3)]
        outs.append((np.stack(lw), [lat.get_state(c) for c in range(2)]))
        lat.close()
    for lw, st in outs[1:]:
        assert np.array_equal(lw, outs[0][0])
        for c in range(2):
            for u, v in zip(st[c], outs[0][1][c]):
                assert np.array_equal(np.asarray(u), np.asarray(v))


def test_fp64_block_chain_tracks_the_oracle():
    """L = 4, U = 4, beta = 2, dtau = 0.1 (M = 20), B = 6 (blocks 6, 6, 6, 2): the FP64 GPU
    chain and the oracle agree for 60 sweeps (log-weights 1e-12, paths, field), and
    the kinetic energy accumulated from the block links matches the oracle's (FP32 link
    table and per-pair sums on both precisions: 1e-5)."""
    params = (1.0, 4.0, 2.0, 0.1, 1.0)
    lat = make(4, [0], "fp64", params, 6)
    orc = oracle.Chain(4, *params, 0)
    links = 0.0
    for k in range(60):
        lw = lat.sweep(1, logw=True)[0]
        ref = orc.sweep(block=6)
        links += ref["links"].sum()
        assert rel_err(lw, ref["logw"]).max() <= 1e-12, k
    s, x, _, sw = lat.get_state(0)
    assert sw == 60 and np.array_equal(x, orc.x) and np.array_equal(s, orc.s)
    m = lat.measure()[0]
    assert m["n_samples"] == 60
    assert m["ekin"] == pytest.approx(-(params[0] / params[2]) * links / (60 * 16), rel=1e-5)  # FP32 link table
    lat.close()


def test_per_chain_block_lengths_in_a_ragged_batch():
    """Chains of different sizes in one context, each with its own block length."""
    from paper_2510_13866_gb300 import Lattice

    Ls = [8, 12, 16, 24]
    pars = [(1.0, 4.0, 0.8, 0.1, 1.0), (1.0, 2.0, 0.7, 0.1, 0.5), (1.0, 4.0, 0.5, 0.05, 0.875),
            (1.0, 8.0, 0.3, 0.05, 1.0)]
    Bs = [3, 0, 4, 2]
    seeds = [40, 41, 42, 43]
    lat = Lattice(Ls, seeds, precision="fp32")
    for c, (p, B) in enumerate(zip(pars, Bs)):
        lat.set_params(*p, chain=c)
        lat.set_block(B, chain=c)
    logw = lat.sweep(1, logw=True)
    for c, (p, B) in enumerate(zip(pars, Bs)):
        orc = oracle.Chain(Ls[c], *p, seeds[c])
        ref = orc.sweep(want_margin=True, block=B)
        _, x, a, _ = lat.get_state(c)
        assert a == ref["anchor"]
        assert rel_err(logw[c], ref["logw"]).max() <= 1e-5
        _, _, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, 1e-5, block=B)
        assert not bad, bad[:3]
    lat.close()


@pytest.mark.parametrize("L,params,B,nwl", [
    (48, (1.0, 4.0, 0.3, 0.05, 0.5), 4, 8),     # M = 6: blocks 4, 2
    (64, (1.0, 4.0, 0.25, 0.05, 1.0), 2, 4),    # M = 5: blocks 2, 2, 1
    (128, (1.0, 4.0, 0.2, 0.05, 0.125), 3, 2),  # M = 4: blocks 3, 1
])
def test_wide_block_parity(L, params, B, nwl):
    lat = make(L, [13], "fp32", params, B)
    logw = lat.sweep(1, logw=True)
    orc = oracle.Chain(L, *params, 13)
    ref = orc.sweep(want_margin=True, nwl_limit=nwl, block=B)
    _, x, a, _ = lat.get_state(0)
    assert a == ref["anchor"]
    assert rel_err(logw[0][:, :nwl], ref["logw"][:, :nwl]).max() <= 1e-5
    _, _, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, 1e-5, nwl=nwl, block=B)
    assert not bad, bad[:3]
    lat.close()


def test_block_headline_size_holds_block_ends():
    """L = 32, t=1, U=4, beta=4, dtau=0.05 (M = 80), half filling, 64 chains, B = 16, in
    the benchmark's launch configuration: every held site keeps its value, the log-weights
    are finite, and the first worldline of each spin of chain 0 matches the oracle."""
    params = (1.0, 4.0, 4.0, 0.05, 1.0)
    lat = make(32, list(range(64)), "fp32", params, 16)
    before = [lat.get_state(c)[1] for c in range(64)]
    logw = lat.sweep(1, logw=True)
    for c in range(64):
        _, x, a, _ = lat.get_state(c)
        held = [(a + k) % 80 for k in range(0, 80, 16)]
        assert np.array_equal(x[:, :, held], before[c][:, :, held])
        assert np.all(np.isfinite(logw[c]))
    orc = oracle.Chain(32, *params, 0)
    ref = orc.sweep(want_margin=True, nwl_limit=1, block=16)
    _, x, a, _ = lat.get_state(0)
    assert rel_err(logw[0][:, :1], ref["logw"][:, :1]).max() <= 1e-5
    _, _, bad = path_mismatches(x, orc.x, ref["margin"], a, 80, 1e-5, nwl=1, block=16)
    assert not bad, bad[:3]
    lat.close()


def test_set_block_rejects_bad_arguments():
    from paper_2510_13866_gb300 import HQMCError, Lattice

    lat = Lattice(8, [0], precision="fp32")
    with pytest.raises(HQMCError):
        lat.set_block(-1)
    with pytest.raises(HQMCError):
        lat.set_block(2, chain=3)
    lat.close()


def test_block_units_are_bitwise_independent_of_the_launch():
    """The blocks of a pair run as separate work units in any order; the partial
    log-weights are summed in block order, so graph replay, plain launches, persistent
    and one-group-per-unit grids and different CTA shapes give the same bits."""
    params = (1.0, 4.0, 2.0, 0.05, 1.0)  # M = 40, B = 6: blocks 6 x 6, 4
    outs = []
    for mode in [dict(use_graph=True, persistent=True, warps_per_cta=4),
                 dict(use_graph=False, persistent=False, warps_per_cta=1),
                 dict(use_graph=True, persistent=True, warps_per_cta=8)]:
        lat = make([16, 8, 16], [1, 2, 3], "fp32", params, 6)
        lat.set_launch(**mode)
        lw = [lat.sweep(1, logw=True) for _ in range(3)]
        outs.append((lw, [lat.get_state(c)[:2] for c in range(3)]))
        lat.close()
    for lw, st in outs[1:]:
        for k in range(3):
            for c in range(3):
                assert np.array_equal(lw[k][c], outs[0][0][k][c])
        for c in range(3):
            assert np.array_equal(st[c][0], outs[0][1][c][0])
            assert np.array_equal(st[c][1], outs[0][1][c][1])


def test_set_block_midway_keeps_the_chain():
    """Changing B between sweeps re-lays the context out but keeps fields, worldlines
    and the sweep counter: the chain continues exactly as a fresh context restored from
    the same state with that B."""
    params = (1.0, 4.0, 1.0, 0.05, 1.0)  # M = 20
    a = make(8, [5], "fp32", params, 0)
    a.sweep(3)
    s, x, _, sw = a.get_state(0)
    a.set_block(7)
    a.sweep(2)
    b = make(8, [5], "fp32", params, 7)
    b.set_state(0, s=s, x=x, sweeps=sw)
    b.sweep(2)
    for u, v in zip(a.get_state(0), b.get_state(0)):
        assert np.array_equal(np.asarray(u), np.asarray(v))
    a.close()
    b.close()
