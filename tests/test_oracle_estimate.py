"""The identity behind the Gaussian-field log-weight error estimate, by exact enumeration on a
small lattice with the oracle's propagator (no GPU).

For a unit from x_s at position 0 to the held end x_e at position len, with forward messages
alpha_i (the weight of the paths from x_s that reach y at position i, before W_i) and backward
messages beta_i (the weight of the paths from y at position i to x_e, W_i included), the
sampler draws x_i from the posterior alpha_i beta_i / <alpha_i, beta_i>.  Then

  E_post[ max alpha_i / alpha_i(x_i) ] = max alpha_i sum_y beta_i(y) / <alpha_i, beta_i>,

the factor by which an error of size max alpha_i at slice i reaches alpha_end(x_e); and the
backward sampler's conditional mean given the next site,

  E[ max alpha_i / alpha_i(x_i) | x_{i+1} = z ] = max alpha_i sum_y W_i(y) G(z - y) / S_i(z),
  S_i(z) = sum_y f_i(y) G(z - y),  f_i = W_i alpha_i,

averages over the posterior of x_{i+1} to the same value.  The kernels sum the second form
over the drawn path.
"""
import numpy as np

import oracle


def setup(L=3, M=6, dtau=0.25, seed=11):
    N = L * L
    g, _ = oracle.g_table(L, 1.0, dtau)
    ys = np.arange(N)
    G = g[(ys[:, None] % L - ys[None, :] % L) % L] * g[(ys[:, None] // L - ys[None, :] // L) % L]
    rng = np.random.default_rng(seed)
    W = np.exp(1.5 * rng.standard_normal((M, N)))  # a strong positive potential per slice
    return N, G, W


def messages(N, G, W, xs, xe):
    M = W.shape[0]
    alpha = [None] * (M + 1)
    a = np.zeros(N)
    a[xs] = 1.0
    alpha[0] = a
    for i in range(M):
        alpha[i + 1] = G @ (W[i] * alpha[i])
    beta = [None] * (M + 1)
    b = np.zeros(N)
    b[xe] = 1.0
    beta[M] = b
    for i in range(M - 1, -1, -1):
        beta[i] = W[i] * (G.T @ beta[i + 1])
    return alpha, beta


def test_posterior_mean_of_the_concentration():
    N, G, W = setup()
    M = W.shape[0]
    alpha, beta = messages(N, G, W, 0, 4)
    Z = alpha[M][4]
    for i in range(1, M):
        a, b = alpha[i], beta[i]
        assert np.isclose(a @ b, Z, rtol=1e-12)  # every slice carries the same total
        post = a * b / Z
        lhs = post @ (a.max() / a)
        rhs = a.max() * b.sum() / Z
        assert np.isclose(lhs, rhs, rtol=1e-12), (i, lhs, rhs)


def test_conditional_mean_given_the_next_site_has_the_same_mean():
    N, G, W = setup(L=4, M=5, dtau=0.2, seed=5)
    M = W.shape[0]
    alpha, beta = messages(N, G, W, 3, 9)
    Z = alpha[M][9]
    for i in range(1, M):
        a = alpha[i]
        f = W[i] * a
        post_next = alpha[i + 1] * beta[i + 1] / Z  # the posterior of x_{i+1}
        # the sampler's conditional p(x_i = y | x_{i+1} = z) ~ f(y) G(z - y)
        S = G @ f                     # S(z) = sum_y G(z, y) f(y)
        cond = a.max() * (G @ W[i]) / S  # its mean of max a / a(x_i)
        direct = np.array([(f * G[z]) @ (a.max() / a) / S[z] for z in range(N)])
        assert np.allclose(cond, direct, rtol=1e-12)
        assert np.isclose(post_next @ cond, a.max() * beta[i].sum() / Z, rtol=1e-12), i
