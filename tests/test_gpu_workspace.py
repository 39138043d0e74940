"""Device memory of a context (hqmc_workspace_size, hqmc_attach_workspace) and the failure of
an allocation, as errors the host reads, never as a fault:

  - a context on a caller-owned (torch) buffer and one that allocates its own give the same
    bits;
  - a buffer smaller than hqmc_workspace_size is refused with HQMC_ERR_NOMEM and a
    misaligned one with HQMC_ERR_ARG, leaving the context usable;
  - a context whose layout cannot fit the device (about 335 GB of histograms) fails its
    first sweep with HQMC_ERR_NOMEM, and a small context runs normally afterwards.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run(torch_memory):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(8, [7, 8], precision="fp32", torch_memory=torch_memory)
    lat.set_params(1.0, 4.0, 1.0, 0.05, 1.0)
    lw = [lat.sweep(1, logw=True) for _ in range(3)]
    st = [lat.get_state(c) for c in range(2)]
    lat.close()
    return lw, st


def test_caller_owned_and_library_memory_agree():
    a, b = run(True), run(False)
    for k in range(3):
        for c in range(2):
            assert np.array_equal(a[0][k][c], b[0][k][c])
    for c in range(2):
        assert np.array_equal(a[1][c][0], b[1][c][0]) and np.array_equal(a[1][c][1], b[1][c][1])


def test_attach_refuses_small_and_misaligned_buffers():
    import torch

    from paper_2510_13866_gb300 import Lattice
    from paper_2510_13866_gb300.hqmc import lib

    lat = Lattice(8, [3], precision="fp32", torch_memory=False)
    lat.set_params(1.0, 4.0, 1.0, 0.05, 1.0)
    n = lat.workspace_size()
    buf = torch.empty(n + 512, dtype=torch.uint8, device="cuda:0")
    p = (buf.data_ptr() + 255) // 256 * 256
    assert lib().hqmc_attach_workspace(lat._ctx, C.c_void_p(p), n - 256) == -2  # HQMC_ERR_NOMEM
    assert lib().hqmc_attach_workspace(lat._ctx, C.c_void_p(p + 16), n) == -1  # HQMC_ERR_ARG
    assert lib().hqmc_attach_workspace(lat._ctx, C.c_void_p(p), n) == 0
    lw = lat.sweep(2, logw=True)
    assert all(np.all(np.isfinite(w)) for w in lw)
    lat.close()
    del buf


def test_allocation_failure_is_an_error():
    from paper_2510_13866_gb300 import HQMCError, Lattice

    # 256 chains of L = 128 at M = 10000: the two int32 histograms alone are 2 M N 4 B =
    # 1.3 GB per chain, beyond the device; cudaMalloc refuses the request
    lat = Lattice(128, list(range(256)), precision="fp32", torch_memory=False)
    lat.set_params(1.0, 4.0, 500.0, 0.05, 0.125)
    with pytest.raises(HQMCError) as err:
        lat.sweep(1)
    assert err.value.code == -2  # HQMC_ERR_NOMEM
    lat.close()
    lw = run(False)[0]
    assert all(np.all(np.isfinite(w)) for w in lw[0])
