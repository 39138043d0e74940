"""Edge cases of the sweep on the GPU against the FP64 oracle, through the C ABI: a single
worldline per spin, a full band (N_sigma = N), a single slice (M = 1), two slices, zero
sweeps, and the largest lattice of the register kernel with an odd worldline count."""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def run(L, params, prec, seeds=(3,), sweeps=1):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, list(seeds), precision=prec)
    lat.set_params(*params)
    for k in range(sweeps):
        logw = lat.sweep(1, logw=True)
        for c, sd in enumerate(seeds):
            orc = run.orcs.setdefault((L, params, prec, sd), oracle.Chain(L, *params, sd))
            ref = orc.sweep(want_margin=True)
            s, x, a, sw = lat.get_state(c)
            assert sw == k + 1 and a == ref["anchor"]
            assert rel_err(logw[c], ref["logw"]).max() <= TOL[prec]
            _, firsts, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, TOL[prec])
            assert not bad, bad[:3]
            if firsts:
                lat.close()
                return
            assert np.array_equal(s, orc.s)
    lat.close()


run.orcs = {}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,params", [
    (8, (1.0, 4.0, 1.0, 0.1, 2.0 / 64.0)),   # one worldline per spin (a pair with a shadow)
    (4, (1.0, 4.0, 1.0, 0.1, 2.0)),          # full band: N_sigma = N = 16
    (4, (1.0, 4.0, 0.1, 0.1, 1.0)),          # M = 1: the loop is the anchor slice alone
    (6, (1.0, 4.0, 0.2, 0.1, 1.0)),          # M = 2
    (32, (1.0, 4.0, 0.3, 0.05, 2.0 * 3.0 / 1024.0)),  # L = 32, three worldlines per spin
])
def test_edge_sweeps(prec, L, params):
    run.orcs.clear()
    run(L, params, prec, seeds=(3, 4), sweeps=3)


def test_zero_sweeps_leave_the_state():
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(8, [1], precision="fp32")
    lat.set_params(1.0, 4.0, 1.0, 0.1, 1.0)
    lat.sweep(2)
    before = lat.get_state(0)
    lat.sweep(0)
    lat.local_sweep(0)
    after = lat.get_state(0)
    for u, v in zip(before, after):
        assert np.array_equal(np.asarray(u), np.asarray(v))
    lat.close()


def test_fp64_fft_floor_far_from_the_peak():
    """The FFT filter's rounding is relative to the message's peak.  An FP64 context takes a
    log-potential v = 25 at one site on every slice (0 elsewhere) through
    hqmc_log_weight_grad, with one worldline per spin held four steps away in x and y, where
    the final message is about 1e-10 of its peak (kappa = peak / end value).  Against the
    dense transfer product (scipy expm, non-negative sums, the same construction the oracle
    is pinned to) the log-weight error stays within 4 eps log2(N) M kappa per worldline; the
    measured error is printed."""
    import math

    import scipy.linalg as sla
    import torch

    from paper_2510_13866_gb300 import Lattice

    L, M, dtau = 8, 8, 0.1
    N = L * L
    lat = Lattice(L, [5], precision="fp64")
    lat.set_params(1.0, 4.0, M * dtau, dtau, 2.0 / N)  # one worldline per spin
    xa = 4 + L * 4
    lat.set_state(0, s=np.ones((M, N), dtype=np.int8), x=np.full((2, 1, M), xa, dtype=np.int32))
    v = np.zeros((2, M, N))
    v[:, :, 0] = 25.0
    lz, _, _ = lat.log_weight_grad(v=torch.from_numpy(v.ravel()).cuda(), want_dv=False)
    lat.close()

    A = np.zeros((N, N))
    for iy in range(L):
        for ix in range(L):
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                A[ix + L * iy, (ix + dx) % L + L * ((iy + dy) % L)] += 1.0
    G = sla.expm(1.0 * dtau * A)
    w = np.zeros(N)
    w[xa] = 1.0
    for l in range(M):
        w = G @ (np.exp(v[0, l]) * w)
    kappa = w.max() / w[xa]
    ref = 2.0 * math.log(w[xa])
    err = abs(lz[0] - ref)
    bound = 2 * 4 * 2.0 ** -53 * math.log2(N) * M * kappa
    print(f"\nkappa {kappa:.3g}: FP64 FFT log-weight error {err:.3g} (bound {bound:.3g}, eps kappa "
          f"{2.0 ** -53 * kappa:.3g})")
    assert kappa > 1e9
    assert err <= bound
