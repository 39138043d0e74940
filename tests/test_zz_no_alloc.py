"""hqmc_ffbs_noalloc, the FFBS entry point that allocates no device memory, against the
context path (hqmc_sweep) that owns its workspace.

Callers that cannot call cudaMalloc (another framework's pool, a pre-reserved arena,
allocation-free loops) pass only their own inputs and outputs; the entry point takes
its scratch from a static device array.  Two calls in a row must reproduce the FFBS
of two consecutive context sweeps: the same paths and log-weights within the
log-weight tolerance of the other tests (1e-5 relative in FP32, 1e-12 in FP64).
This file is collected last so a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.mark.parametrize("prec,L,beta,fill", [("fp32", 16, 1.0, 1.0), ("fp64", 8, 0.8, 0.875), ("fp32", 12, 0.5, 0.875)])
def test_noalloc_matches_context_on_two_calls(prec, L, beta, fill):
    import torch

    from paper_2510_13866_gb300 import Lattice, hqmc

    t, U, dtau, seed = 1.0, 4.0, 0.05, 17
    lat = Lattice(L, [seed], precision=prec)
    lat.set_params(t, U, beta, dtau, fill)
    s0, x0, _, sw0 = lat.get_state(0)
    assert sw0 == 0
    lw1 = lat.sweep(1, logw=True)[0].ravel()
    s1, x1, _, _ = lat.get_state(0)
    lw2 = lat.sweep(1, logw=True)[0].ravel()
    _, x2, _, _ = lat.get_state(0)
    _, M, Ns = lat.shapes[0]
    lat.close()

    lib = hqmc.lib()
    stream = torch.cuda.current_stream()
    s_dev = torch.from_numpy(s0.copy()).cuda()
    x_dev = torch.from_numpy(x0.copy()).cuda()
    lw_dev = torch.zeros(2 * Ns, dtype=torch.float64, device="cuda")
    p = hqmc.HQMC_FP64 if prec == "fp64" else hqmc.HQMC_FP32

    def call(sweep):
        rc = lib.hqmc_ffbs_noalloc(L, M, Ns, t, U, dtau, seed, sweep, C.c_void_p(s_dev.data_ptr()),
                                   C.c_void_p(x_dev.data_ptr()), C.c_void_p(lw_dev.data_ptr()), p,
                                   C.c_void_p(stream.cuda_stream))
        assert rc == 0, hqmc.ERRORS.get(rc, rc)
        torch.cuda.synchronize()
        return x_dev.cpu().numpy(), lw_dev.cpu().numpy()

    x_a, lw_a = call(0)
    assert np.array_equal(x_a, x1)
    assert (np.abs(lw_a - lw1) / np.maximum(1.0, np.abs(lw1))).max() <= TOL[prec]

    s_dev.copy_(torch.from_numpy(s1))  # the field after the context's Gibbs step
    x_b, lw_b = call(1)
    assert np.array_equal(x_b, x2)
    assert (np.abs(lw_b - lw2) / np.maximum(1.0, np.abs(lw2))).max() <= TOL[prec]


def test_noalloc_rejects_what_does_not_fit_and_bad_input():
    import torch

    from paper_2510_13866_gb300 import hqmc

    lib = hqmc.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L, M, Ns = 32, 4000, 512  # slot of 32 MB does not fit the 32 MiB scratch
    s_dev = torch.ones(8, dtype=torch.int8, device="cuda")
    x_dev = torch.zeros(8, dtype=torch.int32, device="cuda")
    lw_dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptrs = [C.c_void_p(a.data_ptr()) for a in (s_dev, x_dev, lw_dev)]
    assert lib.hqmc_ffbs_noalloc(L, M, Ns, 1.0, 4.0, 0.05, 0, 0, *ptrs, 0, stream) == -8
    # out-of-range site index is caught before the FFBS kernel runs
    L, M, Ns = 4, 3, 2
    s_dev = torch.ones(M * L * L, dtype=torch.int8, device="cuda")
    x_dev = torch.full((2 * Ns * M,), 99, dtype=torch.int32, device="cuda")
    lw_dev = torch.zeros(2 * Ns, dtype=torch.float64, device="cuda")
    ptrs = [C.c_void_p(a.data_ptr()) for a in (s_dev, x_dev, lw_dev)]
    assert lib.hqmc_ffbs_noalloc(L, M, Ns, 1.0, 4.0, 0.1, 0, 0, *ptrs, 0, stream) == -1


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_leaves_a_wide_context_launchable(prec):
    """A context whose CTAs carry 8 worldline groups needs the FFBS kernel's shared-memory
    limit of that shape; a no-allocation call in between (4 warps per CTA) must not lower
    it, so the context's next sweep still runs and matches a context that never saw it."""
    import torch

    from paper_2510_13866_gb300 import Lattice, hqmc

    L, t, U, beta, dtau, seed = 32, 1.0, 4.0, 0.4, 0.05, 5
    ref = Lattice(L, [seed], precision=prec)
    ref.set_params(t, U, beta, dtau, 0.25)
    ref.set_class_launch(L, 8)
    ref.sweep(1)
    lw_ref = ref.sweep(1, logw=True)[0]
    ref.close()

    lat = Lattice(L, [seed], precision=prec)
    lat.set_params(t, U, beta, dtau, 0.25)
    lat.set_class_launch(L, 8)
    lat.sweep(1)
    s, x, _, _ = lat.get_state(0)
    _, M, Ns = lat.shapes[0]
    lib = hqmc.lib()
    stream = torch.cuda.current_stream()
    s_dev = torch.from_numpy(s.copy()).cuda()
    x_dev = torch.from_numpy(x.copy()).cuda()
    lw_dev = torch.zeros(2 * Ns, dtype=torch.float64, device="cuda")
    p = hqmc.HQMC_FP64 if prec == "fp64" else hqmc.HQMC_FP32
    rc = lib.hqmc_ffbs_noalloc(L, M, Ns, t, U, dtau, seed, 1, C.c_void_p(s_dev.data_ptr()),
                               C.c_void_p(x_dev.data_ptr()), C.c_void_p(lw_dev.data_ptr()), p,
                               C.c_void_p(stream.cuda_stream))
    assert rc == 0, hqmc.ERRORS.get(rc, rc)
    lw = lat.sweep(1, logw=True)[0]  # raised HQMC_ERR_CUDA when the limit had been lowered
    lat.close()
    assert np.array_equal(lw, lw_ref)
