"""Trotter-order pin of the oracle's discretisation (Sec. 5, the O(beta dtau^2) splitting
error of the Trotter/Strang factorisation of Eq. trotter).

For one up and one down worldline the Hubbard model is an N^2-state problem that is
solved exactly in continuous imaginary time: H = K (x) 1 + 1 (x) K + U [x_up = x_dn],
K = -t (nearest-neighbour adjacency), by scipy's matrix exponential.  The oracle's
discretisation of the same problem is built from the oracle's own tables -- the 1D
propagator g(d) and its t-derivative (orc_g_table) and the Hirsch coupling lambda
(orc_lambda), whose field sum gives cosh(lambda m) per site -- as a transfer matrix
over M = beta / dtau slices.  Its double occupancy and its kinetic energy (the
oracle's link estimator -(t/beta) sum d/dt log G, in expectation -(t/beta) d log Z/dt)
must approach the exact values with an error that falls by about 4x per halving of
dtau.  A dropped Trotter factor, a wrong lambda or a first-order split would show as
a ratio near 2 or a non-vanishing error.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from test_oracle_pins import lattice_adjacency


def exact_continuum(L, t, U, beta):
    N = L * L
    A = lattice_adjacency(L)
    I = np.eye(N)
    Kt = -t * (np.kron(A, I) + np.kron(I, A))
    same = np.array([1.0 if (i // N) == (i % N) else 0.0 for i in range(N * N)])
    H = Kt + U * np.diag(same)
    R = sla.expm(-beta * H)
    Z = np.trace(R)
    D = np.trace(np.diag(same) @ R) / Z / N
    Ekin = np.trace(Kt @ R) / Z / N
    return D, Ekin


def trotter_from_oracle(orc, L, t, U, beta, dtau):
    N = L * L
    M = int(round(beta / dtau))
    g, dg = orc.g_table(L, t, dtau)
    lam = orc.lam(U, dtau)
    ix = np.arange(N) % L
    iy = np.arange(N) // L
    dx = (ix[None, :] - ix[:, None]) % L
    dy = (iy[None, :] - iy[:, None]) % L
    G = g[dx] * g[dy]                     # <x'|exp(-dtau K)|x>, separable
    dG = dg[dx] * g[dy] + g[dx] * dg[dy]  # its t-derivative
    GG = np.kron(G, G)
    dGG = np.kron(dG, G) + np.kron(G, dG)
    same = np.array([1.0 if (i // N) == (i % N) else 0.0 for i in range(N * N)])
    # summed Hirsch field: prod_x cosh(lambda m_x) = cosh(lambda)^2 apart, 1 together
    V = np.where(same > 0, 1.0, math.cosh(lam) ** 2)
    T = GG * V[None, :]
    TM1 = np.linalg.matrix_power(T, M - 1)
    Z = np.trace(TM1 @ T)
    D = np.trace(TM1 @ (GG * (V * same)[None, :])) / Z / N
    dZ = M * np.trace(TM1 @ (dGG * V[None, :]))
    Ekin = -(t / beta) * dZ / Z / N
    return D, Ekin


@pytest.mark.parametrize("L,U,beta", [(3, 4.0, 1.0), (3, 8.0, 0.5), (4, 2.0, 1.0)])
def test_trotter_error_is_second_order(orc, L, U, beta):
    t = 1.0
    D_ex, E_ex = exact_continuum(L, t, U, beta)
    dts = [beta / 8, beta / 16, beta / 32, beta / 64]
    res = [trotter_from_oracle(orc, L, t, U, beta, d) for d in dts]
    for k, ex in ((0, D_ex), (1, E_ex)):
        err = [r[k] - ex for r in res]
        ratios = [err[i] / err[i + 1] for i in range(len(err) - 1)]
        # second order: 4 per halving, approached as dtau -> 0 (a first-order split gives 2)
        assert all(3.5 < q < 4.5 for q in ratios), (k, err, ratios)
        assert abs(ratios[-1] - 4.0) < 0.05, (k, ratios)
        # Richardson extrapolation of the two finest steps removes the dtau^2 term
        rich = (4 * res[-1][k] - res[-2][k]) / 3
        assert abs(rich - ex) < 0.05 * abs(err[-1]), (k, rich, ex, err[-1])


def test_trotter_limit_u0_is_exact_for_the_propagator(orc):
    """At U = 0 the split is exact (K alone), so every dtau gives the continuum answer."""
    L, t, beta = 3, 1.0, 1.0
    D_ex, E_ex = exact_continuum(L, t, 0.0, beta)
    for dtau in (0.5, 0.25, 0.1):
        D, E = trotter_from_oracle(orc, L, t, 0.0, beta, dtau)
        assert abs(D - D_ex) < 1e-12 and abs(E - E_ex) < 1e-11, (dtau, D - D_ex, E - E_ex)
