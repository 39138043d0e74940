"""The Gibbs/measure kernel handles a group of slices per CTA (hqmc_set_slice_launch; 0
picks about 1024 sites per CTA).  The group size changes only the order in which S(k)'s
FP64 partial sums meet: fields, worldlines, log-weights and the integer observables must
be identical for every group size, and S(k) equal to FP64 rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run(L, M, group, U=4.0, seeds=(3, 4, 5)):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice([L] * len(seeds), list(seeds), precision="fp32")
    lat.set_params(1.0, U, M * 0.05, 0.05, 1.0)
    lat.set_slice_launch(group)
    lw = [lat.sweep(1, logw=True) for _ in range(3)]
    st = [lat.get_state(c) for c in range(len(seeds))]
    sig = [lat.get_sigma(c) for c in range(len(seeds))] if U < 0 else None
    obs = lat.measure()
    lat.close()
    return lw, st, sig, obs


@pytest.mark.parametrize("L,M,U", [(8, 40, 4.0), (8, 37, -4.0), (12, 21, 4.0), (16, 24, 4.0), (48, 8, 4.0)])
def test_slice_group_changes_only_rounding(L, M, U):
    ref = run(L, M, 1, U)
    for group in (0, 2, 5, 16):
        lw, st, sig, obs = run(L, M, group, U)
        for k in range(3):
            for c in range(len(lw[k])):
                assert np.array_equal(lw[k][c], ref[0][k][c]), (group, k, c)
        for c in range(len(st)):
            assert np.array_equal(st[c][0], ref[1][c][0]) and np.array_equal(st[c][1], ref[1][c][1]), (group, c)
            if sig is not None:
                assert np.array_equal(sig[c], ref[2][c]), (group, c)
            for key in ("density", "double_occ", "m2", "n_samples"):
                assert obs[c][key] == ref[3][c][key], (group, c, key)
            assert np.allclose(obs[c]["Sk"], ref[3][c]["Sk"], rtol=1e-12, atol=1e-12), (group, c)
