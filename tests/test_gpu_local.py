"""Local link updates (Sec. 3.5.1, Eq. Rlocal in the position basis) on the GPU against the
FP64 oracle, through the C ABI.

Both sides form R in FP64 from their own propagator tables, so a decision u < R can differ
only where the oracle's u lies within 1e-12 of R; then that worldline is not compared
further.  Everywhere else the paths, the accepted-move counts, the occupancy and the
Gibbs fields after the sweep are identical.  Each case starts both sides from the same
state (the oracle's, after one FFBS sweep, copied into the context).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def make(L, seeds, prec, params):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, seeds, precision=prec)
    lat.set_params(*params)
    return lat


def start(lat, c, orc):
    lat.set_state(c, s=None if orc.gauss else orc.s, x=orc.x, sweeps=orc.sweep_count)
    if orc.gauss:
        lat.set_sigma(c, orc.sigma)


def compare_paths(x_gpu, x_orc, margin):
    """Worldlines must agree unless one of their decisions was within RTOL of its edge."""
    bad = []
    for sg in range(2):
        for p in range(x_gpu.shape[1]):
            if not np.array_equal(x_gpu[sg, p], x_orc[sg, p]) and not np.any(margin[sg, p] < RTOL):
                bad.append((sg, p))
    return bad


def occupancy(x, M, N):
    n = np.zeros((2, M, N), dtype=np.int64)
    for sg in range(2):
        for p in range(x.shape[1]):
            np.add.at(n[sg], (np.arange(M), x[sg, p]), 1)
    return n


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,params", [
    (4, (1.0, 4.0, 1.0, 0.1, 1.0)),       # M = 10
    (3, (1.0, 2.0, 0.6, 0.1, 4 / 9)),     # M = 6
    (6, (1.0, 4.0, 1.1, 0.1, 0.5)),       # M = 11: a third colour
    (4, (1.0, 4.0, 0.1, 0.1, 1.0)),       # M = 1: the slice is its own neighbour
    (4, (1.0, 4.0, 0.2, 0.1, 1.0)),       # M = 2
    (8, (1.0, -4.0, 0.8, 0.1, 1.0)),      # U < 0, Gaussian field
    (16, (2.0, 4.0, 0.5, 0.25, 1.0)),     # t dtau = 0.5: many moves accepted
    (32, (1.0, 4.0, 0.45, 0.05, 1.0)),    # M = 9
])
def test_local_sweep_parity(prec, L, params):
    lat = make(L, [7, 8], prec, params)
    orcs = []
    for c in range(2):
        orc = oracle.Chain(L, *params, int(lat.seeds[c]))
        orc.sweep()
        start(lat, c, orc)
        orcs.append(orc)
    lat.local_sweep(1)
    obs = lat.measure()
    for c, orc in enumerate(orcs):
        ref = orc.local_sweep(want_margin=True)
        s, x, _, sw = lat.get_state(c)
        assert sw == 2
        bad = compare_paths(x, orc.x, ref["margin"])
        assert not bad, bad[:3]
        if np.array_equal(x, orc.x):
            assert obs[c]["n_local_accepted"] == ref["accepted"]
            assert np.array_equal(occupancy(x, orc.M, L * L), ref["hist"])
            if orc.gauss:
                assert np.allclose(lat.get_sigma(c), orc.sigma, rtol=0, atol=1e-12)
            else:
                assert np.array_equal(s, orc.s)
    lat.close()


def test_local_and_ffbs_sweeps_interleave_with_the_oracle():
    """FP64, L = 4, U = 4, beta = 2 (M = 20): 20 rounds of (two local sweeps, one FFBS
    sweep) on the GPU and in the oracle agree: FFBS log-weights 1e-12, paths, fields,
    the sweep counter, the accepted moves and the kinetic energy of the link sums (FP32
    link table on both precisions: 1e-5)."""
    params = (1.0, 4.0, 2.0, 0.1, 1.0)
    lat = make(4, [3], "fp64", params)
    orc = oracle.Chain(4, *params, 3)
    acc = 0
    links = 0.0
    for k in range(20):
        lat.local_sweep(2)
        for _ in range(2):
            r = orc.local_sweep()
            acc += r["accepted"]
            links += r["links"].sum()
        lw = lat.sweep(1, logw=True)[0]
        ref = orc.sweep()
        links += ref["links"].sum()
        assert rel_err(lw, ref["logw"]).max() <= 1e-12, k
    s, x, _, sw = lat.get_state(0)
    assert sw == 60 and np.array_equal(x, orc.x) and np.array_equal(s, orc.s)
    m = lat.measure()[0]
    assert m["n_samples"] == 60
    assert m["n_local_accepted"] == acc > 0
    assert m["ekin"] == pytest.approx(-(params[0] / params[2]) * links / (60 * 16), rel=1e-5)
    lat.close()


def test_local_sweep_full_size():
    """L = 32, t=1, U=4, beta=4, dtau=0.05 (M = 80), half filling, 64 chains: one local
    sweep; chains 0 and 63 start from the oracle's state after one FFBS sweep and are
    compared in full (the other chains from their initial state)."""
    params = (1.0, 4.0, 4.0, 0.05, 1.0)
    lat = make(32, list(range(64)), "fp32", params)
    orcs = {}
    for c in (0, 63):
        orc = oracle.Chain(32, *params, c)
        orc.sweep()
        start(lat, c, orc)
        orcs[c] = orc
    lat.local_sweep(1)
    obs = lat.measure()
    for c, orc in orcs.items():
        ref = orc.local_sweep(want_margin=True)
        _, x, _, _ = lat.get_state(c)
        assert not compare_paths(x, orc.x, ref["margin"])
        if np.array_equal(x, orc.x):
            assert obs[c]["n_local_accepted"] == ref["accepted"]
    lat.close()


def test_local_sweep_wide_lattice():
    """L = 48 (the wide-lattice class): local moves need no FFT, same parity."""
    params = (1.0, 4.0, 0.3, 0.05, 0.5)
    lat = make(48, [5], "fp32", params)
    lat.local_sweep(2)
    orc = oracle.Chain(48, *params, 5)
    orc.local_sweep()
    ref = orc.local_sweep(want_margin=True)
    _, x, _, sw = lat.get_state(0)
    assert sw == 2
    assert not compare_paths(x, orc.x, ref["margin"])
    lat.close()
