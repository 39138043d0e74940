"""Pins of the oracle's local link update (Sec. 3.5.1, Eq. Rlocal, read in the position
basis: x_l moves one lattice step with its neighbours x_{l-1}, x_{l+1} held, accepted
with probability min(1, R), R the ratio of the path weights prod_l W_l(x_l) G(x_{l+1}-x_l)).

Independent sources: path weights from scipy's matrix exponential of the hopping matrix,
the exact stationary law of one worldline (enumerated), and independent samples drawn by
the sampler itself compared with that law by a chi-square test.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as ss

import oracle
from test_oracle_pins import lattice_adjacency, ring_adjacency

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def path_weight(G, W, path):
    """prod_l W_l(x_l) G(x_{l+1} - x_l) of a closed path (G the dense N x N propagator)."""
    M = len(path)
    w = 1.0
    for l in range(M):
        w *= W[l, path[l]] * G[path[l], path[(l + 1) % M]]
    return w


def test_local_step_moves_one_lattice_bond():
    for L in (2, 3, 5):
        A = lattice_adjacency(L)
        for x in range(L * L):
            targets = [oracle.local_step(L, x, d) for d in range(4)]
            for y in targets:
                assert A[x, y] > 0  # a nearest neighbour on the torus
            if L >= 3:
                assert len(set(targets)) == 4
            # +x/-x and +y/-y undo each other (symmetric proposal)
            assert oracle.local_step(L, targets[0], 1) == x
            assert oracle.local_step(L, targets[2], 3) == x


def test_local_colors_separate_neighbouring_slices():
    for M in range(1, 12):
        cols = [oracle.local_color(M, l) for l in range(M)]
        assert set(cols) <= {0, 1, 2}
        if M >= 2:
            for l in range(M):
                if M > 1 and (l + 1) % M != l:
                    assert cols[l] != cols[(l + 1) % M] or M == 1


@pytest.mark.parametrize("M", [1, 2, 5])
def test_local_ratio_is_the_path_weight_ratio(M):
    """R from the oracle equals w(X')/w(X) for every slice and step, with G = expm(t dtau A)
    and random positive slice potentials (both spins of the Hirsch form and general W)."""
    L, t, dtau = 4, 1.0, 0.3
    N = L * L
    G = sla.expm(t * dtau * lattice_adjacency(L))
    g = sla.expm(t * dtau * ring_adjacency(L))[0]
    rng = np.random.default_rng(M)
    W = rng.uniform(0.2, 3.0, size=(M, N))
    for _ in range(4):
        path = list(rng.integers(0, N, size=M))
        w0 = path_weight(G, W, path)
        for l in range(M):
            for d in range(4):
                xnew = oracle.local_step(L, path[l], d)
                p2 = list(path)
                p2[l] = xnew
                want = path_weight(G, W, p2) / w0
                got = oracle.local_ratio(L, M, g, W[l], path[(l - 1) % M], path[l], path[(l + 1) % M], xnew)
                assert got == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_local_sweep_kernel_leaves_the_path_law_invariant(M):
    """Exact one-sweep transition matrix of one worldline (L = 3, all 9^M paths), built
    from the oracle's ratio and colour schedule: the exact path law pi ~ prod W G is
    stationary, and every single-slice kernel satisfies detailed balance."""
    L, t, dtau = 3, 1.0, 0.7
    N = L * L
    G = sla.expm(t * dtau * lattice_adjacency(L))
    g = sla.expm(t * dtau * ring_adjacency(L))[0]
    rng = np.random.default_rng(10 + M)
    W = rng.uniform(0.3, 2.5, size=(M, N))
    paths = list(itertools.product(range(N), repeat=M))
    index = {p: i for i, p in enumerate(paths)}
    pi = np.array([path_weight(G, W, p) for p in paths])
    pi /= pi.sum()
    T = np.eye(len(paths))
    for c in range(3):
        for l in range(M):
            if oracle.local_color(M, l) != c:
                continue
            K = np.zeros((len(paths), len(paths)))
            for i, p in enumerate(paths):
                for d in range(4):
                    xnew = oracle.local_step(L, p[l], d)
                    R = oracle.local_ratio(L, M, g, W[l], p[(l - 1) % M], p[l], p[(l + 1) % M], xnew)
                    a = min(1.0, R)
                    q = list(p)
                    q[l] = xnew
                    K[i, index[tuple(q)]] += 0.25 * a
                    K[i, i] += 0.25 * (1.0 - a)
            flow = pi[:, None] * K
            assert np.allclose(flow, flow.T, rtol=1e-10, atol=1e-15)
            T = T @ K
    assert np.allclose(pi @ T, pi, rtol=1e-10, atol=1e-14)
    assert np.allclose(T.sum(axis=1), 1.0)


def test_local_sweep_follows_its_rule():
    """Every decision of one oracle local sweep (L = 4, U = 4, M = 7) is reproduced from
    its documented uniforms (phase 4, j = 2l for the step, 2l+1 for the acceptance), the
    colour order and the ratio; the Gibbs step afterwards is the FFBS sweep's."""
    L, U, dtau = 4, 4.0, 0.1
    ch = oracle.Chain(L, 1.0, U, 0.7, dtau, 1.0, 21)
    ch.sweep()  # move away from the static start
    M, N, Ns = ch.M, ch.N, ch.Nsig
    s0, x0, sw = ch.s.copy(), ch.x.copy(), ch.sweep_count
    lam = ch.lam
    g, _ = oracle.g_table(L, 1.0, dtau)
    out = ch.local_sweep(want_margin=True)
    x = x0.copy()
    acc = 0
    for sg in range(2):
        W = np.exp((1.0 if sg == 0 else -1.0) * lam * s0.astype(np.float64))
        for p in range(Ns):
            wl = sg * Ns + p
            for c in range(3):
                for l in range(M):
                    if oracle.local_color(M, l) != c:
                        continue
                    u0 = oracle.uniform(21, sw, 4, wl, 2 * l)
                    u1 = oracle.uniform(21, sw, 4, wl, 2 * l + 1)
                    xnew = oracle.local_step(L, x[sg, p, l], min(3, int(u0 * 4)))
                    R = oracle.local_ratio(L, M, g, W[l], x[sg, p, (l - 1) % M], x[sg, p, l],
                                           x[sg, p, (l + 1) % M], xnew)
                    if u1 < R:
                        x[sg, p, l] = xnew
                        acc += 1
    assert np.array_equal(x, ch.x)
    assert acc == out["accepted"] > 0
    hist = np.zeros((2, M, N), dtype=np.int64)
    for sg in range(2):
        for p in range(Ns):
            np.add.at(hist[sg], (np.arange(M), x[sg, p]), 1)
    assert np.array_equal(hist, out["hist"])
    m = hist[0] - hist[1]
    for l in range(M):
        for xx in range(N):
            u = oracle.uniform(21, sw, 1, l, xx)
            assert ch.s[l, xx] == (1 if u < 1.0 / (1.0 + np.exp(-2.0 * lam * m[l, xx])) else -1)


def test_local_sampler_draws_the_exact_law():
    """Independent chains (U = 0, L = 3, one worldline per spin, t dtau = 1, M = 3) run 25
    local sweeps from the static start; their final paths are independent draws whose
    displacement pairs (x1-x0, x2-x1) must follow the exact law pi ~ prod G (chi-square)."""
    L, t, beta, dtau = 3, 1.0, 3.0, 1.0
    N = L * L
    G = sla.expm(t * dtau * lattice_adjacency(L))
    paths = list(itertools.product(range(N), repeat=3))
    pi = np.array([path_weight(G, np.ones((3, N)), p) for p in paths])
    pi /= pi.sum()

    def disp(a, b):
        return ((b % L - a % L) % L) + L * ((b // L - a // L) % L)

    want = np.zeros((N, N))
    for p, w in zip(paths, pi):
        want[disp(p[0], p[1]), disp(p[1], p[2])] += w
    counts = np.zeros((N, N))
    for seed in range(1500):
        ch = oracle.Chain(L, t, 0.0, beta, dtau, 2.0 / 9.0, seed)
        for _ in range(25):
            ch.local_sweep()
        for sg in range(2):
            p = ch.x[sg, 0]
            counts[disp(p[0], p[1]), disp(p[1], p[2])] += 1
    n = counts.sum()
    chi2, pval = ss.chisquare(counts.ravel(), want.ravel() * n)
    assert pval > 1e-4, (chi2, pval)
