"""Pins of the oracle's open-path estimator of the one-body density matrix (Sec. 4,
"Observables": n_k = (1/N) sum_{ij sigma} e^{ik(r_i - r_j)} <c^dag_j c_i> needs the weight of
paths that do not close).

The FFBS filter of a unit, read at every end site y instead of the held end x_e, gives the
weights of the open configurations; E[alpha_end(x_e + r) / alpha_end(x_e)] over the
closed ensemble is the open/closed weight ratio, and its sum over worldlines and spins is
A(r) = sum_x sum_sigma <c^dag_{x+r} c_x>.  The pins do not use the oracle's own filter:
  - U = 0: the ratio is G_beta(r) / G_beta(0) with G_beta = expm(t beta A) (scipy), for
    any path (closed form);
  - U != 0: a dense product of the slice transfer matrices G diag(W_l) (scipy expm);
  - one up and one down worldline: the exact Trotterised open/closed ratio
    Tr(P_r^T T^M) / Tr(T^M) of the N^2-state transfer matrix with the Hirsch field summed
    out, against the sampled estimator (statistical).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from test_oracle_pins import dense_G, lattice_adjacency


def shift_index(L, x, r):
    rx, ry = r % L, r // L
    return (x % L + rx) % L + L * ((x // L + ry) % L)


@pytest.mark.parametrize("L,M,dtau", [(3, 4, 0.25), (4, 6, 0.1), (6, 5, 0.2)])
def test_open_ratio_u0_closed_form(orc, L, M, dtau):
    N = L * L
    t = 1.0
    g, _ = orc.g_table(L, t, dtau)
    W = np.ones((M, N))
    Gb = sla.expm(t * M * dtau * lattice_adjacency(L))
    rng = np.random.default_rng(3)
    for _ in range(4):
        xs, l0 = int(rng.integers(N)), int(rng.integers(M))
        ratio = orc.open_ratio(L, M, g, W, l0, M, xs, xs)
        want = np.array([Gb[shift_index(L, xs, r), xs] for r in range(N)]) / Gb[xs, xs]
        assert np.allclose(ratio, want, rtol=1e-11, atol=1e-13), np.abs(ratio - want).max()


@pytest.mark.parametrize("L,M,B,dtau,U", [(3, 5, 3, 0.2, 4.0), (4, 6, 6, 0.1, 8.0), (4, 7, 2, 0.25, 2.0)])
def test_open_ratio_dense_transfer(orc, L, M, B, dtau, U):
    N = L * L
    t = 1.0
    g, _ = orc.g_table(L, t, dtau)
    rng = np.random.default_rng(11)
    lam = orc.lam(U, dtau)
    s = rng.choice([-1, 1], size=(M, N))
    W = np.exp(lam * s)
    G = dense_G(L, t, dtau)
    for _ in range(3):
        l0, xs, xe = int(rng.integers(M)), int(rng.integers(N)), int(rng.integers(N))
        v = np.zeros(N)
        v[xs] = 1.0
        for i in range(B):
            v = G @ (W[(l0 + i) % M] * v)
        want = np.array([v[shift_index(L, xe, r)] for r in range(N)]) / v[xe]
        got = orc.open_ratio(L, M, g, W, l0, B, xs, xe)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-13), np.abs(got / want - 1).max()


def exact_open_two_particle(L, t, U, dtau, M):
    """2 Tr(P_r^T T^M) / Tr(T^M) for one up and one down worldline: T = (G (x) G) V with the
    summed Hirsch weight V (exp(dtau U) apart, 1 together) at the source state, and P_r the
    displacement of the up particle's end by r (the cut sits after a propagation, before a
    potential, as in the filter)."""
    N = L * L
    G = dense_G(L, t, dtau)
    GG = np.kron(G, G)
    same = np.array([1.0 if (i // N) == (i % N) else 0.0 for i in range(N * N)])
    V = np.where(same > 0, 1.0, math.exp(dtau * U))
    T = GG * V[None, :]
    TM = np.linalg.matrix_power(T, M)
    Z = np.trace(TM)
    out = np.zeros(N)
    for r in range(N):
        acc = 0.0
        for j in range(N * N):
            xu, xd = j // N, j % N
            acc += TM[shift_index(L, xu, r) * N + xd, j]
        out[r] = 2.0 * acc / Z  # the down worldline contributes the same by symmetry
    return out


def test_open_estimator_two_particle_exact(orc):
    """The sampled estimator (FFBS + Gibbs chain, closed loops) against the exact ratio."""
    L, U, beta, dtau = 3, 8.0, 1.0, 0.25
    M = 4
    want = exact_open_two_particle(L, 1.0, U, dtau, M)
    assert want[0] == pytest.approx(2.0)
    ch = orc.Chain(L=L, t=1.0, U=U, beta=beta, dtau=dtau, filling=2.0 / (L * L), seed=9)
    samples = []
    for k in range(40000):
        a = int(math.floor(orc.uniform(ch.seed, ch.sweep_count, 2, 0, 0) * M))
        a = min(a, M - 1)
        est = ch.open_estimate(ch.slice_potentials(), a)
        out = ch.sweep()
        assert out["anchor"] == a
        if k >= 500:
            samples.append(est)
    x = np.array(samples)
    nb = 20
    b = x[: len(x) // nb * nb].reshape(nb, -1, x.shape[1]).mean(axis=1)
    m, se = b.mean(axis=0), b.std(axis=0, ddof=1) / math.sqrt(nb)
    assert np.allclose(x[:, 0], 2.0, rtol=1e-14)
    z = (m - want) / np.maximum(se, 1e-12)
    assert np.all(np.abs(z[1:]) < 4.5), (m, want, se)
    # the displaced weight is smaller than the closed one, and not trivially zero; the
    # interaction moves it by many standard errors from the free value (a check of power)
    free = exact_open_two_particle(L, 1.0, 0.0, dtau, M)
    assert np.all(np.abs(free[1:] - want[1:]) > 6 * se[1:]), (free, want, se)
    assert np.all(want[1:] < 2.0) and want[1:].min() > 0.01
