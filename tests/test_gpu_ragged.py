"""The 256-chain ragged batch (L in {8,12,16,24,32,48}, beta in {2,4,6}, U in {2,4,8},
filling in {0.5, 0.875, 1}, dtau = 0.05, drawn per chain from Philox key (1, 0)) in one
context, one CUDA-graph replay per sweep, and the CTA-shape autotuner."""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu


def test_ragged_256_chains_sampled_parity():
    from paper_2510_13866_gb300 import Lattice
    from paper_2510_13866_gb300.workloads import ragged

    work = ragged(256)
    lat = Lattice([w[0] for w in work], [w[2] for w in work], precision="fp32")
    for c, (_, p, _) in enumerate(work):
        lat.set_params(*p, chain=c)
    logw = lat.sweep(1, logw=True)
    for c in range(256):
        assert np.all(np.isfinite(logw[c]))
    # one chain of every size against the oracle, a few worldlines per spin
    seen = {}
    for c, (L, p, _) in enumerate(work):
        seen.setdefault(L, c)
    for L, c in sorted(seen.items()):
        _, p, seed = work[c]
        k = 4 if L <= 16 else 2
        orc = oracle.Chain(L, *p, seed)
        ref = orc.sweep(want_margin=True, nwl_limit=k)
        s, x, a, _ = lat.get_state(c)
        assert a == ref["anchor"]
        assert rel_err(logw[c][:, :k], ref["logw"][:, :k]).max() <= 1e-5, L
        _, _, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, 1e-5, nwl=k)
        assert not bad, (L, bad[:3])
    lat.close()


def test_autotune_keeps_results_and_state(tmp_path):
    from paper_2510_13866_gb300 import Lattice

    Ls = [8, 16, 16, 32]
    pars = [(1.0, 4.0, 1.0, 0.05, 1.0), (1.0, 2.0, 0.5, 0.05, 0.875), (1.0, 4.0, 0.5, 0.05, 1.0),
            (1.0, 8.0, 0.4, 0.05, 0.5)]

    def make():
        lat = Lattice(Ls, [40, 41, 42, 43], precision="fp32")
        for c, p in enumerate(pars):
            lat.set_params(*p, chain=c)
        return lat

    ref = make()
    lw_ref = ref.sweep(2, logw=True)
    st_ref = [ref.get_state(c) for c in range(4)]
    ref.close()

    lat = make()
    lat.sweep(1)
    cache = str(tmp_path / "tune.json")
    chosen = lat.autotune(trial_sweeps=2, cache=cache)
    assert set(chosen) == {8, 16, 32} and all(w in (1, 2, 4, 8) for w in chosen.values())
    assert lat.get_state(0)[3] == 1  # the context's own chains were not advanced
    lw = lat.sweep(1, logw=True)
    for c in range(4):
        assert np.array_equal(lw[c], lw_ref[c])
        got = lat.get_state(c)
        assert np.array_equal(got[0], st_ref[c][0]) and np.array_equal(got[1], st_ref[c][1])
    lat.close()
    # the cache is reused without timing again
    lat2 = make()
    assert lat2.autotune(cache=cache) == chosen
    lat2.close()
