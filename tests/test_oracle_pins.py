"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what it pins and the independent source: a library routine
(numpy's Philox, scipy's matrix exponential), brute-force enumeration, a closed
form, or an invariant.  Every function in oracle/hqmc_oracle.c is covered here.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def ring_adjacency(L):
    A = np.zeros((L, L))
    for i in range(L):
        A[i, (i + 1) % L] += 1.0
        A[i, (i - 1) % L] += 1.0
    return A


def lattice_adjacency(L):
    N = L * L
    A = np.zeros((N, N))
    for iy in range(L):
        for ix in range(L):
            x = ix + L * iy
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                A[x, (ix + dx) % L + L * ((iy + dy) % L)] += 1.0
    return A


def dense_G(L, t, dtau):
    """exp(-dtau K) with K = -t * (nearest-neighbour adjacency), by scipy's expm."""
    return sla.expm(t * dtau * lattice_adjacency(L))


# --------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al., SC'11) against numpy.random.Philox
# --------------------------------------------------------------------------
def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([2**64 - 1] * 4, [2**64 - 1] * 2)]
    for _ in range(200):
        cases.append((rng.integers(0, 2**64, 4, dtype=np.uint64, endpoint=False).tolist(),
                      rng.integers(0, 2**64, 2, dtype=np.uint64, endpoint=False).tolist()))
    for ctr, key in cases:
        # numpy advances its 256-bit counter before each block, so start it one below.
        c_int = sum(int(c) << (64 * k) for k, c in enumerate(ctr))
        bg = np.random.Philox(counter=(c_int - 1) % 2**256, key=sum(int(k) << (64 * i) for i, k in enumerate(key)))
        ref = bg.random_raw(4)
        got = orc.philox4x64_10(ctr, key)
        assert np.array_equal(ref, got), (ctr, key)


def test_uniform_counter_layout(orc):
    """u(seed, sweep, phase, i, j) is word j&3 of Philox((j>>2, i, phase, sweep), (seed, 0))."""
    for seed, sweep, phase, i, j in [(0, 0, 0, 0, 0), (5, 17, 1, 79, 1023), (63, 2**64 - 1, 3, 3, 6),
                                     (2**40 + 3, 499, 2, 0, 0), (1, 2, 0, 1023, 77)]:
        c_int = (j >> 2) | (i << 64) | (phase << 128) | (sweep << 192)
        bg = np.random.Philox(counter=(c_int - 1) % 2**256, key=seed)
        w = int(bg.random_raw(4)[j & 3])
        assert orc.uniform(seed, sweep, phase, i, j) == (w >> 11) / 2.0**53


# --------------------------------------------------------------------------
# Propagator against scipy's matrix exponential of the hopping matrix
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,t,dtau", [(2, 1.0, 0.1), (3, 1.0, 0.5), (4, 1.0, 0.1), (8, 0.7, 0.05),
                                      (12, 1.0, 0.05), (32, 1.0, 0.05)])
def test_g_table_is_exp_of_hopping(orc, L, t, dtau):
    g, dg = orc.g_table(L, t, dtau)
    A = ring_adjacency(L)
    E = sla.expm(t * dtau * A)
    # the plain DFT sum of L unit-size terms carries ~L*eps absolute rounding
    tol = 4e-16 * L
    assert np.allclose(g, E[0], rtol=1e-12, atol=tol)
    # d/dt exp(t dtau A) = dtau A exp(t dtau A)
    assert np.allclose(dg, (dtau * A @ E)[0], rtol=1e-12, atol=tol)


@pytest.mark.parametrize("L", [3, 4])
def test_separable_G_is_2d_exp(orc, L):
    t, dtau = 1.0, 0.3
    g, _ = orc.g_table(L, t, dtau)
    G = dense_G(L, t, dtau)
    N = L * L
    for x in range(N):
        for y in range(N):
            d = ((y % L - x % L) % L, (y // L - x // L) % L)
            assert abs(G[x, y] - g[d[0]] * g[d[1]]) < 1e-13


def test_hirsch_identity(orc):
    """(1/2) sum_s exp(lambda s (nu - nd)) is proportional to exp(-dtau U (nu-1/2)(nd-1/2))."""
    for U, dtau in [(4.0, 0.05), (4.0, 0.1), (8.0, 0.05), (2.0, 0.25)]:
        lam = orc.lam(U, dtau)
        ratios = []
        for nu, nd in itertools.product((0, 1), repeat=2):
            lhs = 0.5 * (math.exp(lam * (nu - nd)) + math.exp(-lam * (nu - nd)))
            rhs = math.exp(-dtau * U * (nu - 0.5) * (nd - 0.5))
            ratios.append(lhs / rhs)
        assert max(ratios) - min(ratios) < 1e-13 * max(ratios)
    assert orc.lam(0.0, 0.1) == 0.0


# --------------------------------------------------------------------------
# Forward filter
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,beta,dtau", [(4, 2.0, 0.1), (8, 4.0, 0.25), (5, 1.0, 0.125)])
def test_filter_u0_closed_form(orc, L, beta, dtau):
    """At U=0, Z_p = <x|exp(-beta K)|x> = (exp(beta t A_ring))[0,0]^2 (no Trotter error)."""
    M = orc.n_slices(beta, dtau)
    g, _ = orc.g_table(L, 1.0, dtau)
    W = np.ones((M, L * L))
    ref = 2.0 * math.log(sla.expm(beta * ring_adjacency(L))[0, 0])
    for a, xa in [(0, 0), (M - 1, L * L - 1), (M // 2, 3)]:
        lz = orc.filter_logz(L, M, g, W, a, xa)
        assert abs(lz - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("L,M,dtau,U", [(3, 5, 0.3, 4.0), (4, 6, 0.1, 4.0), (4, 7, 0.2, 8.0), (6, 4, 0.05, 2.0)])
def test_filter_matches_dense_transfer_product(orc, L, M, dtau, U):
    """Z_p = e_xa^T prod_i [G diag(W_{a+i})] e_xa with G from scipy expm."""
    rng = np.random.default_rng(L * 100 + M)
    N = L * L
    G = dense_G(L, 1.0, dtau)
    g, _ = orc.g_table(L, 1.0, dtau)
    lam = orc.lam(U, dtau)
    for sigma in (1.0, -1.0):
        s = rng.choice([-1, 1], size=(M, N))
        W = np.exp(sigma * lam * s)
        for a, xa in [(0, 0), (M - 1, N - 1), (2, N // 2)]:
            v = np.zeros(N)
            v[xa] = 1.0
            for i in range(M):
                v = G @ (W[(a + i) % M] * v)
            ref = math.log(v[xa])
            lz = orc.filter_logz(L, M, g, W, a, xa)
            assert abs(lz - ref) <= 1e-12 * max(1.0, abs(ref))


def test_filter_keeps_relative_accuracy_far_from_the_peak(orc):
    """A potential that pulls the message onto one site (W = e^25 there, 1 elsewhere) leaves
    a loop anchored four steps away in x and y with a weight about 1e-10 of the peak.  The
    oracle's direct convolution sums non-negative terms, so its log-weight still matches
    the dense transfer product (scipy expm, also non-negative sums) to 1e-12 relative: the
    oracle has no rounding floor relative to the peak, which makes it the reference for the
    FFT path's floor."""
    L, dtau = 8, 0.1
    N = L * L
    G = dense_G(L, 1.0, dtau)
    g, _ = orc.g_table(L, 1.0, dtau)
    sink, xa = 0, 4 + L * 4
    for M in (4, 6, 8):
        W = np.ones((M, N))
        W[:, sink] = math.exp(25.0)
        v = np.zeros(N)
        v[xa] = 1.0
        for i in range(M):
            v = G @ (W[i] * v)
        kappa = v.max() / v[xa]
        assert kappa > 1e9
        ref = math.log(v[xa])
        lz = orc.filter_logz(L, M, g, W, 0, xa)
        assert abs(lz - ref) <= 1e-12 * max(1.0, abs(ref)), (M, kappa, lz, ref)


def _enumerate_paths(L, M, g, W, a, xa):
    """All closed paths with x_a held: returns (paths [P][M], weights [P])."""
    N = L * L
    interior = [(a + i) % M for i in range(1, M)]
    paths, weights = [], []
    for combo in itertools.product(range(N), repeat=M - 1):
        x = [0] * M
        x[a] = xa
        for l, site in zip(interior, combo):
            x[l] = site
        w = 1.0
        for l in range(M):
            y0, y1 = x[l], x[(l + 1) % M]
            d = ((y1 % L - y0 % L) % L, (y1 // L - y0 // L) % L)
            w *= W[l][y0] * g[d[0]] * g[d[1]]
        paths.append(tuple(x))
        weights.append(w)
    return paths, np.array(weights)


def test_filter_and_backward_vs_enumeration(orc):
    """Brute force over all 9^3 interior paths (L=3, M=4): log Z and the FFBS path law (chi^2)."""
    L, M, dtau, U = 3, 4, 0.5, 4.0
    N = L * L
    g, _ = orc.g_table(L, 1.0, dtau)
    lam = orc.lam(U, dtau)
    rng = np.random.default_rng(3)
    s = rng.choice([-1, 1], size=(M, N))
    W = np.exp(lam * s)
    a, xa = 1, 4
    paths, w = _enumerate_paths(L, M, g, W, a, xa)
    ref = math.log(w.sum())
    lz, f = orc.filter_logz(L, M, g, W, a, xa, want_f=True)
    assert abs(lz - ref) < 1e-12 * abs(ref)
    prob = w / w.sum()
    index = {p: k for k, p in enumerate(paths)}
    counts = np.zeros(len(paths))
    n = 30000
    x0 = np.full(M, xa, dtype=np.int32)
    for sweep in range(n):
        xp, _ = orc.backward(L, M, g, f, a, 11, sweep, 0, x0)
        counts[index[tuple(int(v) for v in xp)]] += 1
    expected = prob * n
    big = expected >= 5
    chi2 = (((counts - expected) ** 2) / expected)[big].sum()
    rest_o, rest_e = counts[~big].sum(), expected[~big].sum()
    chi2 += (rest_o - rest_e) ** 2 / max(rest_e, 1e-9)
    dof = big.sum()
    # p < 1e-6 threshold: chi2 > dof + 5.3 sqrt(2 dof)
    assert chi2 < dof + 5.3 * math.sqrt(2 * dof), (chi2, dof)


def test_block_filter_and_backward_vs_enumeration(orc):
    """A block {l0 : l0+B} with both end sites held (Sec. 3.5.2): brute force over all 9^2
    interior paths (L=3, B=3 inside M=5, wrapping past slice M-1): log Z of the block and
    the law of the drawn interior (chi^2)."""
    L, M, B, dtau, U = 3, 5, 3, 0.5, 4.0
    N = L * L
    g, _ = orc.g_table(L, 1.0, dtau)
    lam = orc.lam(U, dtau)
    rng = np.random.default_rng(5)
    W = np.exp(lam * rng.choice([-1, 1], size=(M, N)))
    l0, xs, xe = 3, 2, 7  # slices 3, 4, 0 and the held site at slice 1
    inner = [(l0 + i) % M for i in range(1, B)]
    paths, weights = [], []
    for combo in itertools.product(range(N), repeat=B - 1):
        x = {l0: xs, (l0 + B) % M: xe}
        x.update(zip(inner, combo))
        w = 1.0
        for i in range(B):
            l = (l0 + i) % M
            y0, y1 = x[l], x[(l + 1) % M]
            w *= W[l][y0] * g[(y1 % L - y0 % L) % L] * g[(y1 // L - y0 // L) % L]
        paths.append(combo)
        weights.append(w)
    weights = np.array(weights)
    lz, f = orc.filter_block(L, M, g, W, l0, B, xs, xe, want_f=True)
    assert abs(lz - math.log(weights.sum())) < 1e-12 * abs(math.log(weights.sum()))
    prob = weights / weights.sum()
    index = {p: k for k, p in enumerate(paths)}
    counts = np.zeros(len(paths))
    n = 20000
    x0 = np.zeros(M, dtype=np.int32)
    x0[l0], x0[(l0 + B) % M] = xs, xe
    for sweep in range(n):
        xp, margin = orc.backward_block(L, M, g, f, l0, B, 17, sweep, 0, x0)
        assert xp[l0] == xs and xp[(l0 + B) % M] == xe  # the ends are held
        counts[index[tuple(int(xp[l]) for l in inner)]] += 1
    expected = prob * n
    big = expected >= 5
    chi2 = (((counts - expected) ** 2) / expected)[big].sum()
    rest_o, rest_e = counts[~big].sum(), expected[~big].sum()
    chi2 += (rest_o - rest_e) ** 2 / max(rest_e, 1e-9)
    dof = big.sum()
    assert chi2 < dof + 5.3 * math.sqrt(2 * dof), (chi2, dof)


def test_sweep_block_equals_loop_when_block_covers_it(orc):
    """B >= M is the closed-loop FFBS from the anchor: identical chains."""
    a = orc.Chain(L=4, t=1.0, U=4.0, beta=1.0, dtau=0.1, filling=1.0, seed=8)
    b = orc.Chain(L=4, t=1.0, U=4.0, beta=1.0, dtau=0.1, filling=1.0, seed=8)
    for _ in range(3):
        ra, rb = a.sweep(), b.sweep(block=10)
        assert np.array_equal(ra["logw"], rb["logw"])
    assert np.array_equal(a.x, b.x) and np.array_equal(a.s, b.s)


def test_backward_inverse_cdf_rule(orc):
    """The drawn site is the smallest y with u*S < C(y) (row-major), checked by hand."""
    L, M = 3, 3
    g, _ = orc.g_table(L, 1.0, 0.7)
    rng = np.random.default_rng(5)
    f = rng.random((M, L * L))
    a, seed, sweep, wl = 0, 9, 4, 2
    x0 = np.array([4, 0, 0], dtype=np.int32)
    xp, margin = orc.backward(L, M, g, f, a, seed, sweep, wl, x0)
    nxt = int(x0[0])
    for l in (2, 1):
        p = np.array([f[l, y] * g[(nxt % L - y % L) % L] * g[(nxt // L - y // L) % L] for y in range(L * L)])
        u = orc.uniform(seed, sweep, 0, wl, l)
        C = np.cumsum(p)
        pick = int(np.argmax(u * C[-1] < C))
        assert xp[l] == pick
        nxt = pick


def test_t0_static_paths(orc):
    """t = 0: G = identity, the path cannot move and Z_p = prod_l W_l(x_a)."""
    ch = orc.Chain(L=4, t=0.0, U=4.0, beta=1.0, dtau=0.1, filling=1.0, seed=3)
    x_before = ch.x.copy()
    s_before = ch.s.copy()
    out = ch.sweep()
    assert np.array_equal(ch.x, x_before)
    lam = ch.lam
    for sg, sigma in enumerate((1.0, -1.0)):
        for p in range(ch.Nsig):
            xa = x_before[sg, p, 0]
            ref = sum(sigma * lam * s_before[l, xa] for l in range(ch.M))
            assert abs(out["logw"][sg, p] - ref) < 1e-12 * max(1.0, abs(ref))


# --------------------------------------------------------------------------
# Initial state
# --------------------------------------------------------------------------
def test_initial_state(orc):
    ch = orc.Chain(L=4, t=1.0, U=4.0, beta=2.0, dtau=0.1, filling=1.0, seed=0)
    L, N = 4, 16
    up = ch.x[0, :, 0]
    dn = ch.x[1, :, 0]
    assert all(((x % L) + (x // L)) % 2 == 0 for x in up)
    assert all(((x % L) + (x // L)) % 2 == 1 for x in dn)
    assert sorted(up.tolist()) == up.tolist() and len(set(up.tolist())) == N // 2
    assert np.all(ch.x == ch.x[:, :, :1])  # static in time
    # s from phase 3: +1 iff u < 1/2
    for l in (0, 5, 19):
        for x in (0, 7, 15):
            u = orc.uniform(0, 2**64 - 1, 3, l, x)
            assert ch.s[l, x] == (1 if u < 0.5 else -1)
    frac = (ch.s == 1).mean()
    assert 0.4 < frac < 0.6


# --------------------------------------------------------------------------
# Gibbs conditional
# --------------------------------------------------------------------------
def test_gibbs_conditional_frequencies(orc):
    """Empirical P(s=+1 | m) over many sweeps equals (1 + tanh(lambda m))/2."""
    ch = orc.Chain(L=2, t=1.0, U=8.0, beta=0.5, dtau=0.25, filling=1.0, seed=21)
    lam = ch.lam
    tally = {}
    for _ in range(6000):
        out = ch.sweep()
        m = out["hist"][0] - out["hist"][1]
        for mv, sv in zip(m.ravel(), ch.s.ravel()):
            c = tally.setdefault(int(mv), [0, 0])
            c[0] += 1
            c[1] += sv == 1
    for mv, (n, k) in tally.items():
        if n < 200:
            continue
        p = (1 + math.tanh(lam * mv)) / 2
        assert abs(k / n - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-12, (mv, n, k, p)


# --------------------------------------------------------------------------
# Whole sweep: exact two-particle (1 up + 1 down) transfer matrix
# --------------------------------------------------------------------------
def two_particle_exact(L, t, U, dtau, M):
    """Exact Trotterised Z, double occupancy per site and kinetic energy per site for
    one up and one down worldline (no same-spin exchange exists, so P = identity is exact).
    U > 0: summing the Hirsch field gives prod_x cosh(lambda m_x) = exp(dtau U) if apart,
    1 if together.  U < 0: integrating the Gaussian field gives prod_x exp(a^2 (n_x - 1/2)^2 / 2),
    a^2 = |U| dtau, which is exp(|U| dtau) more when together than apart."""
    N = L * L

    def logZ_and_D(tt):
        G = sla.expm(tt * dtau * lattice_adjacency(L))
        GG = np.kron(G, G)  # index x_up * N + x_dn
        same = np.array([1.0 if (i // N) == (i % N) else 0.0 for i in range(N * N)])
        if U >= 0:
            V = np.where(same > 0, 1.0, math.exp(dtau * U))
        else:
            V = np.where(same > 0, math.exp(-dtau * U), 1.0)
        T = GG * V[None, :]
        TM = np.linalg.matrix_power(T, M)
        Z = np.trace(TM)
        TM1 = np.linalg.matrix_power(T, M - 1)
        Zsame = np.trace(TM1 @ (GG * (V * same)[None, :]))
        return math.log(Z), Zsame / Z / N

    lz, D = logZ_and_D(t)
    h = 1e-5
    dlz = (logZ_and_D(t + h)[0] - logZ_and_D(t - h)[0]) / (2 * h)
    beta = M * dtau
    ekin = -(t / beta) * dlz / N
    return D, ekin


def _batch_stats(x, nb=20):
    x = np.asarray(x)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


def test_sweep_two_particle_exact(orc):
    """FFBS + Gibbs composition against the exact two-particle answer (D and E_kin)."""
    L, U, dtau, beta = 3, 4.0, 0.25, 1.0
    M = 4
    filling = 2.0 / (L * L)  # Nsig = 1
    D_ex, E_ex = two_particle_exact(L, 1.0, U, dtau, M)
    ch = orc.Chain(L=L, t=1.0, U=U, beta=beta, dtau=dtau, filling=filling, seed=5)
    Ds, Es = [], []
    for k in range(24000):
        out = ch.sweep()
        if k < 500:
            continue
        m = orc.measure(L, M, out["hist"], want_fields=False)
        Ds.append(m["d"] / (M * L * L))
        Es.append(-(1.0 / beta) * out["links"].sum() / (L * L))
    dm, de = _batch_stats(Ds)
    em, ee = _batch_stats(Es)
    assert abs(dm - D_ex) < 4.5 * de + 1e-4, (dm, de, D_ex)
    assert abs(em - E_ex) < 4.5 * ee + 1e-4, (em, ee, E_ex)


@pytest.mark.parametrize("block", [2, 3])
def test_sweep_two_particle_exact_blocks(orc, block):
    """Block FFBS (B < M, block ends held) + Gibbs still samples the exact two-particle
    measure: D and E_kin against the transfer matrix (M = 4).  (B = 1 has no interior
    slice: it moves no worldline and is not ergodic.)"""
    L, U, dtau, beta = 3, 4.0, 0.25, 1.0
    M = 4
    D_ex, E_ex = two_particle_exact(L, 1.0, U, dtau, M)
    ch = orc.Chain(L=L, t=1.0, U=U, beta=beta, dtau=dtau, filling=2.0 / (L * L), seed=9 + block)
    Ds, Es = [], []
    for k in range(24000):
        out = ch.sweep(block=block)
        if k < 500:
            continue
        m = orc.measure(L, M, out["hist"], want_fields=False)
        Ds.append(m["d"] / (M * L * L))
        Es.append(-(1.0 / beta) * out["links"].sum() / (L * L))
    dm, de = _batch_stats(Ds)
    em, ee = _batch_stats(Es)
    assert abs(dm - D_ex) < 4.5 * de + 1e-4, (dm, de, D_ex)
    assert abs(em - E_ex) < 4.5 * ee + 1e-4, (em, ee, E_ex)


def test_sweep_two_particle_exact_attractive(orc):
    """U < 0 with the Gaussian field: FFBS + Gaussian Gibbs against the exact two-particle
    double occupancy and kinetic energy (the field integrated out in closed form)."""
    L, U, dtau, beta = 3, -4.0, 0.25, 1.0
    M = 4
    filling = 2.0 / (L * L)
    D_ex, E_ex = two_particle_exact(L, 1.0, U, dtau, M)
    ch = orc.Chain(L=L, t=1.0, U=U, beta=beta, dtau=dtau, filling=filling, seed=6)
    Ds, Es = [], []
    for k in range(24000):
        out = ch.sweep()
        if k < 500:
            continue
        m = orc.measure(L, M, out["hist"], want_fields=False)
        Ds.append(m["d"] / (M * L * L))
        Es.append(-(1.0 / beta) * out["links"].sum() / (L * L))
    dm, de = _batch_stats(Ds)
    em, ee = _batch_stats(Es)
    assert abs(dm - D_ex) < 4.5 * de + 1e-4, (dm, de, D_ex)
    assert abs(em - E_ex) < 4.5 * ee + 1e-4, (em, ee, E_ex)


@pytest.mark.parametrize("block,with_local", [(2, False), (0, True), (3, True)])
def test_sweep_two_particle_exact_attractive_blocks_and_local(orc, block, with_local):
    """U < 0 (Gaussian field) with FFBS in blocks and/or every FFBS sweep followed by a
    local-update sweep: the composition still samples the exact two-particle measure
    (D and E_kin against the transfer matrix with the field integrated out)."""
    L, U, dtau, beta = 3, -4.0, 0.25, 1.0
    M = 4
    D_ex, E_ex = two_particle_exact(L, 1.0, U, dtau, M)
    ch = orc.Chain(L=L, t=1.0, U=U, beta=beta, dtau=dtau, filling=2.0 / (L * L), seed=20 + block)
    Ds, Es = [], []
    for k in range(24000):
        out = ch.local_sweep() if with_local and k % 2 else ch.sweep(block=block)
        if k < 500:
            continue
        m = orc.measure(L, M, out["hist"], want_fields=False)
        Ds.append(m["d"] / (M * L * L))
        Es.append(-(1.0 / beta) * out["links"].sum() / (L * L))
    dm, de = _batch_stats(Ds)
    em, ee = _batch_stats(Es)
    assert abs(dm - D_ex) < 4.5 * de + 1e-4, (dm, de, D_ex)
    assert abs(em - E_ex) < 4.5 * ee + 1e-4, (em, ee, E_ex)


def test_box_muller_normal(orc):
    """Box-Muller output of independent uniforms is standard normal (Kolmogorov-Smirnov)."""
    from scipy import stats

    rng = np.random.default_rng(11)
    u = rng.random((20000, 2))
    z = np.array([orc.normal(a, b) for a, b in u])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert orc.normal(0.0, 0.0) == 0.0  # 1 - u1 = 1: radius zero


def test_gauss_conditional_moments(orc):
    """Gaussian Gibbs: sigma | paths ~ N(a (n - 1/2), 1) (Eq. gaussCond), a = sqrt(|U| dtau)."""
    ch = orc.Chain(L=4, t=1.0, U=-6.0, beta=0.5, dtau=0.1, filling=1.0, seed=3)
    a = math.sqrt(6.0 * 0.1)
    assert abs(orc.gauss_coupling(-6.0, 0.1) - a) < 1e-15
    buckets = {}
    for _ in range(400):
        out = ch.sweep()
        n = out["hist"][0] + out["hist"][1]
        for nv, sv in zip(n.ravel(), ch.sigma.ravel()):
            buckets.setdefault(int(nv), []).append(sv - a * (nv - 0.5))
    for nv, r in buckets.items():
        if len(r) < 500:
            continue
        r = np.asarray(r)
        assert abs(r.mean()) < 5 / math.sqrt(len(r)), (nv, r.mean())
        assert abs(r.var() - 1.0) < 5 * math.sqrt(2.0 / len(r)), (nv, r.var())


def test_sweep_u0_kinetic_energy(orc):
    """U = 0, distinguishable worldlines: E_kin per particle = sum eps e^{-beta eps} / sum e^{-beta eps}."""
    L, beta, dtau = 4, 2.0, 0.1
    ks = 2 * np.pi * np.arange(L) / L
    eps = np.array([-2 * (math.cos(a) + math.cos(b)) for a in ks for b in ks])
    w = np.exp(-beta * eps)
    e_ref = (eps * w).sum() / w.sum()
    ch = orc.Chain(L=L, t=1.0, U=0.0, beta=beta, dtau=dtau, filling=1.0, seed=2)
    Es = []
    for k in range(1500):
        out = ch.sweep()
        if k >= 100:
            Es.append(-(1.0 / beta) * out["links"].sum() / (2 * ch.Nsig))
    em, ee = _batch_stats(Es)
    assert abs(em - e_ref) < 4.5 * ee + 1e-3, (em, ee, e_ref)


def test_joint_stationarity_enumeration(orc):
    """Whole joint state (paths and field) on L=2, M=2, 1 up + 1 down: the empirical
    marginals of a long chain match pi, computed by enumerating all 2^8 * 16 * 16 states."""
    L, M, U, dtau = 2, 2, 6.0, 0.5
    N = L * L
    g, _ = orc.g_table(L, 1.0, dtau)
    lam = orc.lam(U, dtau)

    def G(x0, x1):
        return g[(x1 % L - x0 % L) % L] * g[(x1 // L - x0 // L) % L]

    paths = list(itertools.product(range(N), repeat=M))
    wpath = np.array([np.prod([G(p[l], p[(l + 1) % M]) for l in range(M)]) for p in paths])
    fields = np.array(list(itertools.product((-1, 1), repeat=M * N))).reshape(-1, M, N)
    # pi(pu, pd, s) = w(pu) w(pd) prod_l exp(lam s[l, pu_l]) exp(-lam s[l, pd_l])
    P = len(paths)
    Wu = np.array([[np.prod([math.exp(lam * f[l, p[l]]) for l in range(M)]) for p in paths] for f in fields])
    Wd = np.array([[np.prod([math.exp(-lam * f[l, p[l]]) for l in range(M)]) for p in paths] for f in fields])
    joint = Wu[:, :, None] * Wd[:, None, :] * wpath[None, :, None] * wpath[None, None, :]
    joint /= joint.sum()
    # marginal of (x_up at slice 0, x_dn at slice 0) and of s[0,0]
    m_xx = np.zeros((N, N))
    for iu, pu in enumerate(paths):
        for idn, pd in enumerate(paths):
            m_xx[pu[0], pd[0]] += joint[:, iu, idn].sum()
    p_s00 = joint[fields[:, 0, 0] == 1].sum()
    ch = orc.Chain(L=L, t=1.0, U=U, beta=M * dtau, dtau=dtau, filling=0.5, seed=77)
    cnt = np.zeros((N, N))
    s00 = []
    n = 40000
    for k in range(n + 200):
        ch.sweep()
        if k >= 200:
            cnt[ch.x[0, 0, 0], ch.x[1, 0, 0]] += 1
            s00.append(ch.s[0, 0] == 1)
    emp = cnt / n
    # batch means for s00; multinomial bound (inflated for autocorrelation) for x
    sm, se = _batch_stats(np.array(s00, dtype=float))
    assert abs(sm - p_s00) < 4.5 * se + 2e-3, (sm, se, p_s00)
    err = np.abs(emp - m_xx)
    tol = 6 * np.sqrt(m_xx * (1 - m_xx) / n) * 3 + 2e-3
    assert np.all(err < tol), (emp, m_xx)


# --------------------------------------------------------------------------
# Forward-backward marginals and d log Z / dt
# --------------------------------------------------------------------------
def test_marginals_vs_enumeration(orc):
    L, M, dtau = 3, 4, 0.4
    N = L * L
    g, dg = orc.g_table(L, 1.0, dtau)
    rng = np.random.default_rng(8)
    v = rng.normal(0, 0.5, size=(M, N))
    x0 = 2
    paths, w = _enumerate_paths(L, M, g, np.exp(v), 0, x0)
    lz, marg, dt = orc.marginals(L, M, g, dg, v, x0)
    assert abs(lz - math.log(w.sum())) < 1e-12 * abs(math.log(w.sum()))
    ref = np.zeros((M, N))
    for p, wk in zip(paths, w):
        for l in range(M):
            ref[l, p[l]] += wk
    ref /= w.sum()
    assert np.allclose(marg, ref, atol=1e-13)
    assert np.allclose(marg.sum(axis=1), 1.0, atol=1e-13)
    # d log Z / dt by enumeration: sum over paths w * sum_links d/dt log G
    dlog = []
    for p in paths:
        acc = 0.0
        for l in range(M):
            y0, y1 = p[l], p[(l + 1) % M]
            dx, dy = (y1 % L - y0 % L) % L, (y1 // L - y0 // L) % L
            acc += dg[dx] / g[dx] + dg[dy] / g[dy]
        dlog.append(acc)
    ref_dt = (w * np.array(dlog)).sum() / w.sum()
    assert abs(dt - ref_dt) < 1e-11 * max(1, abs(ref_dt))


def test_grad_finite_differences(orc):
    """d log Z/dt and d log Z/dv against FP64 central differences (h = 1e-6)."""
    L, M, dtau = 4, 6, 0.2
    N = L * L
    rng = np.random.default_rng(4)
    v = rng.normal(0, 0.4, size=(M, N))
    x0 = 5
    h = 1e-6

    def lz(t, vv):
        g, dg = orc.g_table(L, t, dtau)
        return orc.marginals(L, M, g, dg, vv, x0)

    z0, marg, dt = lz(1.0, v)
    fd = (lz(1.0 + h, v)[0] - lz(1.0 - h, v)[0]) / (2 * h)
    assert abs(fd - dt) < 1e-6 * max(1, abs(dt))
    for l, x in [(1, 5), (3, 6), (5, 0), (2, 15)]:
        vp, vm = v.copy(), v.copy()
        vp[l, x] += h
        vm[l, x] -= h
        fdv = (lz(1.0, vp)[0] - lz(1.0, vm)[0]) / (2 * h)
        assert abs(fdv - marg[l, x]) < 1e-7


def test_chain_grad_sums(orc):
    ch = orc.Chain(L=4, t=1.0, U=4.0, beta=0.6, dtau=0.1, filling=0.5, seed=9)
    ch.sweep()
    lz, dv, dt = ch.grad()
    # marginals of every worldline sum to one per slice: sum_x dv = Nsig
    assert np.allclose(dv.sum(axis=2), ch.Nsig, atol=1e-11)
    # slice 0 is the anchor: dv[sigma, 0] is the occupancy of the anchors
    for sg in range(2):
        occ = np.bincount(ch.x[sg, :, 0], minlength=16)
        assert np.allclose(dv[sg, 0], occ, atol=1e-12)


# --------------------------------------------------------------------------
# Observables
# --------------------------------------------------------------------------
def test_measure_definitions(orc):
    rng = np.random.default_rng(12)
    L, M = 6, 3
    N = L * L
    hist = rng.integers(0, 3, size=(2, M, N)).astype(np.int32)
    out = orc.measure(L, M, hist)
    nu, nd = hist[0].astype(float), hist[1].astype(float)
    m = nu - nd
    assert out["n"] == (nu + nd).sum() and out["d"] == (nu * nd).sum() and out["m2"] == (m * m).sum()
    Sk = np.zeros(N)
    Cr = np.zeros(N)
    for l in range(M):
        mf = np.fft.fft2(m[l].reshape(L, L))  # [iy, ix] -> k index kx + L ky
        Sk += (np.abs(mf) ** 2).ravel() / N
        Cr += np.real(np.fft.ifft2(np.abs(mf) ** 2)).ravel() / N
    assert np.allclose(out["Sk"], Sk, rtol=1e-12, atol=1e-10)
    assert np.allclose(out["Cr"], Cr, rtol=1e-12, atol=1e-10)
