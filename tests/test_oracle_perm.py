"""Pins of the oracle's permutation updates (Sec. 3.5.3: worldlines reconnected at
tau = beta by pair swaps, sampled with |w| and reweighted by sgn P, Eq. reweight).

Independent sources: total path weights from scipy's matrix exponential, enumeration of
a unit's interior paths, and the closed forms of non-interacting worldlines: with U = 0
and two worldlines of one spin, the sum over paths of the weight with P = identity is
Tr(T)^2 and with the swap Tr(T^2), T = exp(beta t A); the fermionic partition function is
their half-difference.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from test_oracle_pins import lattice_adjacency, ring_adjacency

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def total_weight(G, W, X, P):
    """prod_p prod_l W_l(x_l^p) G(x_{l+1}^p - x_l^p) with x_M^p = x_0^{P(p)}."""
    n, M = X.shape
    w = 1.0
    for p in range(n):
        for l in range(M):
            nxt = X[p, l + 1] if l + 1 < M else X[P[p], 0]
            w *= W[l, X[p, l]] * G[X[p, l], nxt]
    return w


def test_perm_ratio_is_the_weight_ratio():
    L, t, dtau, M = 4, 1.0, 0.4, 3
    N = L * L
    G = sla.expm(t * dtau * lattice_adjacency(L))
    g = sla.expm(t * dtau * ring_adjacency(L))[0]
    rng = np.random.default_rng(5)
    W = rng.uniform(0.3, 2.0, size=(M, N))
    for _ in range(20):
        X = rng.integers(0, N, size=(4, M))
        P = rng.permutation(4)
        p, q = rng.choice(4, size=2, replace=False)
        P2 = P.copy()
        P2[p], P2[q] = P[q], P[p]
        want = total_weight(G, W, X, P2) / total_weight(G, W, X, P)
        got = oracle.perm_ratio(L, g, int(X[p, M - 1]), int(X[q, M - 1]), int(X[P[p], 0]), int(X[P[q], 0]))
        assert got == pytest.approx(want, rel=1e-12)


def test_unit_log_weight_under_a_permutation_by_enumeration():
    """L = 3, M = 3, two worldlines per spin: the log-weight of the unit of p (slice a of p
    to slice a of P(p), under the permutation the sweep's FFBS ran with) is the log of the
    sum over its interior sites of prod W G, enumerated; slice a is held."""
    L, t, U, beta, dtau = 3, 1.0, 3.0, 0.6, 0.2
    N = L * L
    ch = oracle.Chain(L, t, U, beta, dtau, 4.0 / 9.0, 17)
    M = ch.M
    assert M == 3 and ch.Nsig == 2
    ch.perm[:] = [[1, 0], [1, 0]]
    ch.sign = 1
    rng = np.random.default_rng(1)
    ch.x[:] = rng.integers(0, N, size=ch.x.shape)
    x0, s0 = ch.x.copy(), ch.s.copy()
    G = sla.expm(t * dtau * lattice_adjacency(L))
    lam = ch.lam
    out = ch.perm_sweep()
    a = out["anchor"]
    for sg in range(2):
        W = np.exp((1.0 if sg == 0 else -1.0) * lam * s0.astype(np.float64))
        P = ch.perm[sg]
        for p in range(2):
            start, end = x0[sg, p, a], x0[sg, P[p], a]
            tot = 0.0
            for mid in itertools.product(range(N), repeat=M - 1):
                seq = [start, *mid, end]
                w = 1.0
                for i in range(M):
                    w *= W[(a + i) % M, seq[i]] * G[seq[i], seq[i + 1]]
                tot += w
            assert out["logw"][sg, p] == pytest.approx(np.log(tot), rel=1e-12)
        assert np.array_equal(ch.x[sg, :, a], x0[sg, :, a])


def free_two_worldlines(L, t, beta):
    """Closed forms for two U = 0 worldlines of one spin: P(swap), E[sgn P] and
    d log Z_F / dt with Z_F = (Tr(T)^2 - Tr(T^2)) / 2, T = exp(beta t A)."""
    A = lattice_adjacency(L)

    def traces(tt):
        T = sla.expm(beta * tt * A)
        return np.trace(T), np.trace(T @ T)

    a, b = traces(t)
    p_swap = b / (a * a + b)
    e_sgn = (a * a - b) / (a * a + b)
    h = 1e-5

    def zf(tt):
        ta, tb = traces(tt)
        return (ta * ta - tb) / 2

    dlogzf = (np.log(zf(t + h)) - np.log(zf(t - h))) / (2 * h)
    return p_swap, e_sgn, dlogzf


@pytest.mark.parametrize("with_local,block,dtau", [(False, 0, 0.25), (True, 0, 0.25), (False, 2, 0.125)])
def test_free_worldlines_sample_the_fermionic_closed_forms(with_local, block, dtau):
    """U = 0, L = 3, two worldlines per spin, t = 1, beta = 0.5, where P(swap) = 0.22 and
    E[sgn] = 0.57 per spin (the closed forms hold at any dtau, since G^M = exp(beta t A)).
    Independent chains (30 sweeps each: closed-loop FFBS at M = 2, optionally each sweep
    followed by a local sweep, or FFBS in blocks of 2 slices at M = 4) give P(swap) and
    E[sgn] per spin within 4 standard errors of Tr(T^2)/(Tr(T)^2 + Tr(T^2)) and its
    companion; without local sweeps, the sign-reweighted link estimator of one spin,
    E[sgn sum links] / E[sgn], lies within 4 standard errors of d log Z_F / dt."""
    L, t, beta = 3, 1.0, 0.5
    p_swap, e_sgn, dlogzf = free_two_worldlines(L, t, beta)
    swapped, sg_links, sgns = [], [], []
    for seed in range(800):
        ch = oracle.Chain(L, t, 0.0, beta, dtau, 4.0 / 9.0, 1000 + seed)
        for _ in range(30):
            out = ch.perm_sweep(block=block)
            if with_local:
                ch.local_sweep()
        for sg in range(2):
            sw = int(ch.perm[sg, 0] == 1)
            sgn = -1.0 if sw else 1.0
            swapped.append(sw)
            sgns.append(sgn)
            sg_links.append(sgn * out["links"][sg].sum())
    swapped = np.array(swapped, dtype=float)
    n = swapped.size
    se = np.sqrt(p_swap * (1 - p_swap) / n)
    assert abs(swapped.mean() - p_swap) < 4 * se, (swapped.mean(), p_swap, se)
    sgns = np.array(sgns)
    assert abs(sgns.mean() - e_sgn) < 4 * 2 * se
    if not with_local:
        num, den = np.array(sg_links), sgns
        est = num.mean() / den.mean()
        z = num - est * den
        se_r = z.std(ddof=1) / np.sqrt(n) / abs(den.mean())
        assert se_r < 0.05 * abs(dlogzf)
        assert abs(est - dlogzf) < 4 * se_r, (est, dlogzf, se_r)


def test_perm_sweep_sign_is_the_parity_of_the_permutations():
    """The chain's sign is the product of the two permutations' parities after every
    sweep (L = 4, U = 4, four worldlines per spin)."""
    ch = oracle.Chain(4, 1.0, 4.0, 1.0, 0.25, 0.5, 3)
    swaps = 0
    for _ in range(40):
        swaps += ch.perm_sweep()["swaps"]
        par = 1
        for sg in range(2):
            P = ch.perm[sg]
            assert sorted(P) == list(range(ch.Nsig))
            seen = set()
            for i in range(ch.Nsig):
                if i in seen:
                    continue
                j, ln = i, 0
                while j not in seen:
                    seen.add(j)
                    j = P[j]
                    ln += 1
                par *= (-1) ** (ln - 1)
        assert ch.sign == par
    assert swaps > 0


def test_perm_sweep_with_the_identity_kept_is_the_plain_sweep():
    """With no swap accepted the permuted sweep is the plain FFBS sweep: an oracle chain
    whose swaps are all rejected (t dtau small, distant last/first sites) follows the plain
    chain exactly."""
    params = (1.0, 4.0, 0.6, 0.1, 1.0)
    a = oracle.Chain(4, *params, 9)
    b = oracle.Chain(4, *params, 9)
    for _ in range(5):
        ra = a.sweep()
        rb = b.perm_sweep()
        if rb["swaps"]:
            break
        assert np.array_equal(a.x, b.x) and np.array_equal(a.s, b.s)
        assert np.allclose(ra["logw"], rb["logw"], rtol=1e-14, atol=0)
