"""Attractive U < 0 with the continuous Gaussian field (Sec. 3.5.5) on the GPU, against
the FP64 oracle, through the C ABI.

W = exp(a sigma) for both spins, a = sqrt(|U| dtau); Gibbs sigma ~ N(a (n - 1/2), 1) with
Box-Muller draws from the uniforms of j = 2x, 2x+1.  Tolerances as for U > 0: log-weights
1e-5 (FP32) / 1e-12 (FP64) relative to max(1, |log Z|); paths identical except at a draw
within the tolerance of a CDF edge; the field identical (to FP64 rounding of the
transcendental functions, 1e-12) wherever both sides saw the same occupancy.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def make(L, seeds, prec, params):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, seeds, precision=prec)
    lat.set_params(*params)
    return lat


def occupancy(x, M, N):
    n = np.zeros((2, M, N), dtype=np.int64)
    for sg in range(2):
        for p in range(x.shape[1]):
            np.add.at(n[sg], (np.arange(M), x[sg, p]), 1)
    return n


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_initial_gauss_field_matches_oracle(prec):
    params = (1.0, -4.0, 0.8, 0.1, 1.0)
    lat = make(6, [3, 9], prec, params)
    for c in range(2):
        orc = oracle.Chain(6, *params, int(lat.seeds[c]))
        assert np.allclose(lat.get_sigma(c), orc.sigma, rtol=0, atol=1e-12)
        _, x, _, _ = lat.get_state(c)
        assert np.array_equal(x, orc.x)
    lat.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,beta,dtau,fill,U", [
    (4, 1.0, 0.1, 1.0, -4.0), (3, 0.6, 0.1, 4 / 9, -2.0), (8, 1.0, 0.1, 0.75, -6.0),
    (16, 0.5, 0.05, 1.0, -4.0), (32, 0.5, 0.05, 1.0, -8.0)])
def test_first_sweep_parity_attractive(prec, L, beta, dtau, fill, U):
    params = (1.0, U, beta, dtau, fill)
    lat = make(L, [5, 6], prec, params)
    logw = lat.sweep(1, logw=True)
    for c in range(2):
        orc = oracle.Chain(L, *params, int(lat.seeds[c]))
        ref = orc.sweep(want_margin=True)
        _, x, a, _ = lat.get_state(c)
        assert a == ref["anchor"]
        assert rel_err(logw[c], ref["logw"]).max() <= TOL[prec]
        _, firsts, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, TOL[prec])
        assert not bad, bad[:3]
        if prec == "fp64":
            assert firsts == 0
        n_gpu = occupancy(x, orc.M, L * L)
        same = np.all(n_gpu == ref["hist"], axis=0)
        assert np.allclose(lat.get_sigma(c)[same], orc.sigma[same], rtol=0, atol=1e-12)
    lat.close()


def test_fp64_attractive_tracks_the_oracle():
    """L=4, U=-4, beta=2, dtau=0.1, half filling: the FP64 GPU chain and the oracle chain
    agree for 100 sweeps (log-weights 1e-12, paths and field)."""
    params = (1.0, -4.0, 2.0, 0.1, 1.0)
    lat = make(4, [0], "fp64", params)
    orc = oracle.Chain(4, *params, 0)
    for k in range(100):
        lw = lat.sweep(1, logw=True)[0]
        ref = orc.sweep()
        assert rel_err(lw, ref["logw"]).max() <= 1e-12, k
    _, x, _, sw = lat.get_state(0)
    assert sw == 100 and np.array_equal(x, orc.x)
    assert np.allclose(lat.get_sigma(0), orc.sigma, rtol=0, atol=1e-9)
    lat.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("L,nwl", [(48, 6), (64, 4)])
def test_wide_attractive_parity(L, nwl, prec):
    params = (1.0, -4.0, 0.2, 0.05, 1.0)
    lat = make(L, [12], prec, params)
    logw = lat.sweep(1, logw=True)
    orc = oracle.Chain(L, *params, 12)
    ref = orc.sweep(want_margin=True, nwl_limit=nwl)
    _, x, a, _ = lat.get_state(0)
    assert a == ref["anchor"]
    assert rel_err(logw[0][:, :nwl], ref["logw"][:, :nwl]).max() <= TOL[prec]
    _, _, bad = path_mismatches(x, orc.x, ref["margin"], a, orc.M, TOL[prec], nwl=nwl)
    assert not bad, bad[:3]
    lat.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_adjoint_attractive_matches_oracle(prec, tol):
    """d log Z / d v (v = a sigma) and d log Z / d t of a U < 0 chain against the oracle's
    forward-backward pass given the same log-potential."""
    params = (1.0, -4.0, 0.8, 0.1, 1.0)
    L = 8
    lat = make(L, [2], prec, params)
    lat.sweep(2)
    lat.set_checkpoint(0, bf16=False)
    lz, dv, dt = lat.log_weight_grad()
    _, M, _ = lat.shapes[0]
    orc = oracle.Chain(L, *params, 2)
    _, x, _, _ = lat.get_state(0)
    orc.x[:] = x
    a = oracle.gauss_coupling(params[1], params[3])
    sig = lat.get_sigma(0)
    v = np.stack([a * sig, a * sig])
    rz, rdv, rdt = orc.grad(v)
    assert abs(lz[0] - rz) <= (1e-5 if prec == "fp32" else 1e-10) * abs(rz)
    got = dv.double().cpu().numpy().reshape(2, M, L * L)
    assert np.abs(got - rdv).max() <= tol * max(1.0, np.abs(rdv).max())
    assert abs(dt[0] - rdt) <= tol * max(1.0, abs(rdt))
    lat.close()


def test_sigma_roundtrip_and_resume_are_exact():
    params = (1.0, -3.0, 0.6, 0.1, 1.0)
    a = make(8, [4], "fp32", params)
    a.sweep(4)
    s, x, _, sw = a.get_state(0)
    sig = a.get_sigma(0)
    a.sweep(3)
    ref_x, ref_sig = a.get_state(0)[1], a.get_sigma(0)
    b = make(8, [4], "fp32", params)
    b.set_state(0, x=x, sweeps=sw)
    b.set_sigma(0, sig)
    assert np.array_equal(b.get_sigma(0), sig)
    b.sweep(3)
    assert np.array_equal(b.get_state(0)[1], ref_x)
    assert np.array_equal(b.get_sigma(0), ref_sig)
    from paper_2510_13866_gb300 import HQMCError

    with pytest.raises(HQMCError):
        b.set_params(1.0, 4.0, 0.6, 0.1, 1.0)  # the field type is fixed once the state exists
    a.close()
    b.close()
