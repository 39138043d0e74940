/*
 * hqmc_oracle.c -- plain FP64 CPU oracle for the worldline FFBS + Hirsch-Gibbs sweep
 * of arXiv 2510.13866 ("FFT-Accelerated Auxiliary Variable MCMC for Fermionic
 * Lattice Models").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU path computes.  It is called only from tests/, from the smoke check
 * and from the benchmark's CPU-baseline leg.  The product path never links, loads
 * or calls it, and it shares no code, header or table generator with the CUDA
 * library: every table below is computed here from its definition.
 *
 * Conventions (one line each; where the paper is silent or garbled, each states the
 * reading taken):
 *   site index      x = ix + L*iy on an L x L torus, N = L*L.
 *   slices          l = 0..M-1, M = beta/dtau; a worldline closes: x_M == x_0 (Sec. 3.1).
 *   propagator      g(d) = (1/L) sum_j exp(2 t dtau cos(2 pi j/L)) cos(2 pi j d/L),
 *                   G(dx,dy) = g(dx) g(dy) = <x+d| exp(-dtau K) |x>, the
 *                   real-space form of the kinetic factors D(k)D(k') of Eq. (Tkk)
 *                   with eps_k = -2t sum_a cos k_a (Sec. 3.3).
 *   slice potential W_{l,sigma}(x) = exp(sigma * lambda * s_{x l}), sigma=+1 (up), -1 (down),
 *                   cosh(lambda) = exp(dtau U / 2)  (Hirsch transformation, Eq. hirsch).
 *   target          pi(X, s) ~ prod_{sigma,p,l} W_{l sigma}(x_l) G(x_{l+1} - x_l), s uniform.
 *   forward filter  alpha <- G * (W_l . alpha), Eq. (ffbsFwd) in the position basis.
 *   backward draw   P(x_l | x_{l+1}) ~ f_l(x_l) G(x_{l+1} - x_l)   (Sec. 3.5.2).
 *   Gibbs           P(s = +1 | paths) = (1 + tanh(lambda m)) / 2, m = n_up - n_dn (Sec. 3.5.4).
 *   random numbers  Philox4x64-10 of Salmon, Moraes, Dror and Shaw (SC'11), key (seed, 0),
 *                   counter (j >> 2, i, phase, sweep), output word j & 3, u = (w >> 11) 2^-53.
 *                   phase 0: FFBS draw, i = sigma*Nsig + p, j = l
 *                   phase 1: Gibbs draw, i = l, j = x
 *                   phase 2: anchor slice, i = 0, j = 0
 *                   phase 3: initial field, sweep = 2^64 - 1, i = l, j = x
 *                   phase 4: local link update, i = sigma*Nsig + p, j = 2l (step), 2l+1 (accept)
 *                   phase 5: permutation update, i = sigma, j = 0 (pairing), 1 + k (pair k)
 *   permutations    perm[sigma][p] = P(p): worldline p's slice M-1 links to slice 0 of
 *                   worldline P(p) (x_M^{(p)} = x_0^{(P(p))}, Sec. 3.5.3); the identity
 *                   closes every worldline on itself.  The sampled weight is |w|; the
 *                   sign sgn(P_up) sgn(P_dn) reweights observables (Eq. reweight).
 *
 * Every function that has no independent pin in tests/ says "parity unpinned" here;
 * at present every function is pinned (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

int orc_num_threads(void);

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", */
/* SC'11): ten rounds of a 64x64->128 multiply S-box with a Weyl key schedule.  */
/* ------------------------------------------------------------------------- */
static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(M0, c[0], &hi0, &lo0);
        orc_mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* One uniform in [0,1) for stream (seed, sweep, phase, i, j). */
double orc_uniform(uint64_t seed, uint64_t sweep, uint64_t phase, uint64_t i, uint64_t j)
{
    uint64_t ctr[4] = {j >> 2, i, phase, sweep}, key[2] = {seed, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    return (double)(w[j & 3] >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------- */
/* Model constants                                                            */
/* ------------------------------------------------------------------------- */

/* lambda with cosh(lambda) = exp(dtau U / 2) (Hirsch transformation, Eq. hirsch). */
double orc_lambda(double U, double dtau)
{
    return acosh(exp(0.5 * dtau * U));
}

/* 1D propagator g(d) and its t-derivative, written out from the definition
 * exp(-dtau K) with eps_k = -2t cos k (Sec. 3.3, item 1). */
void orc_g_table(int L, double t, double dtau, double *g, double *dg)
{
    for (int d = 0; d < L; ++d) {
        double s = 0.0, ds = 0.0;
        for (int j = 0; j < L; ++j) {
            double ck = cos(2.0 * ORC_PI * j / L);
            double e = exp(2.0 * t * dtau * ck);
            double ph = cos(2.0 * ORC_PI * (double)j * (double)d / L);
            s += e * ph;
            ds += 2.0 * dtau * ck * e * ph;
        }
        g[d] = s / L;
        if (dg) dg[d] = ds / L;
    }
}

static inline int orc_wrap(int v, int L) { v %= L; return v < 0 ? v + L : v; }

static inline int omp_in_parallel_safe(void)
{
#ifdef _OPENMP
    return omp_in_parallel();
#else
    return 1;
#endif
}

/* G(y - x) for sites x, y. */
static inline double orc_G(const double *g, int L, int x, int y)
{
    int dx = orc_wrap((y % L) - (x % L), L), dy = orc_wrap((y / L) - (x / L), L);
    return g[dx] * g[dy];
}

/* dG/dt(y - x) = g'(dx) g(dy) + g(dx) g'(dy). */
static inline double orc_dG(const double *g, const double *dg, int L, int x, int y)
{
    int dx = orc_wrap((y % L) - (x % L), L), dy = orc_wrap((y / L) - (x / L), L);
    return dg[dx] * g[dy] + g[dx] * dg[dy];
}

/* out(y) = sum_x K(y - x) in(x): direct periodic convolution, O(N^2).  Large lattices
 * split the output sites over threads when no outer loop is parallel (each out(y) is
 * still one sequential sum, so the result does not depend on the thread count). */
static void orc_conv(int L, const double *g, const double *in, double *out)
{
    int N = L * L;
#pragma omp parallel for schedule(static) if (N >= 1024 && !omp_in_parallel_safe())
    for (int y = 0; y < N; ++y) {
        double acc = 0.0;
        for (int x = 0; x < N; ++x) acc += orc_G(g, L, x, y) * in[x];
        out[y] = acc;
    }
}

static void orc_conv_dG(int L, const double *g, const double *dg, const double *in, double *out)
{
    int N = L * L;
#pragma omp parallel for schedule(static) if (N >= 1024 && !omp_in_parallel_safe())
    for (int y = 0; y < N; ++y) {
        double acc = 0.0;
        for (int x = 0; x < N; ++x) acc += orc_dG(g, dg, L, x, y) * in[x];
        out[y] = acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Initial state                                                              */
/* ------------------------------------------------------------------------- */

/* Site of worldline p of spin sigma at the start: up particles fill sublattice A
 * ((ix+iy) even) in row-major order, then sublattice B; down particles fill B then A. */
int orc_initial_site(int L, int sigma, int p)
{
    int N = L * L, k = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int want = (sigma == 0) ? pass : 1 - pass; /* parity class to take in this pass */
        for (int x = 0; x < N; ++x) {
            if (((x % L) + (x / L)) % 2 != want) continue;
            if (k == p) return x;
            ++k;
        }
    }
    return -1;
}

/* s[l*N + x] = +-1 from phase 3; x[((sigma*Nsig)+p)*M + l] = static worldline. */
void orc_init_state(int L, int M, int Nsig, uint64_t seed, int8_t *s, int32_t *xpath)
{
    int N = L * L;
    for (int l = 0; l < M; ++l)
        for (int x = 0; x < N; ++x)
            s[l * N + x] = orc_uniform(seed, UINT64_MAX, 3, (uint64_t)l, (uint64_t)x) < 0.5 ? 1 : -1;
    for (int sg = 0; sg < 2; ++sg)
        for (int p = 0; p < Nsig; ++p) {
            int site = orc_initial_site(L, sg, p);
            for (int l = 0; l < M; ++l) xpath[((size_t)sg * Nsig + p) * M + l] = site;
        }
}

/* ------------------------------------------------------------------------- */
/* Forward filter and backward sampling (Sec. 3.5.2, Eq. ffbsFwd)             */
/* ------------------------------------------------------------------------- */

/* Forward filter over the block of B slices l0, l0+1, ..., l0+B-1 (mod M) with the
 * worldline held at x_{l0} = xs and x_{l0+B} = xe (Sec. 3.5.2: "a block {l0 : l1} with
 * fixed endpoints").  alpha_{l0} = delta_{xs}; f_l = W_l . alpha_l is stored (if f_store)
 * at f_store[l]; alpha is sum-normalised after every step.  Returns
 * log sum over block paths of prod W G = sum log c + log alpha_{l0+B}(xe). */
double orc_filter_block(int L, int M, const double *g, const double *W, int l0, int B, int xs, int xe,
                        double *f_store)
{
    int N = L * L;
    double *alpha = calloc(N, sizeof(double)), *f = malloc(N * sizeof(double)),
           *nxt = malloc(N * sizeof(double));
    double logZ = 0.0;
    alpha[xs] = 1.0;
    for (int i = 0; i < B; ++i) {
        int l = (l0 + i) % M;
        for (int x = 0; x < N; ++x) f[x] = W[(size_t)l * N + x] * alpha[x];
        if (f_store) memcpy(f_store + (size_t)l * N, f, N * sizeof(double));
        orc_conv(L, g, f, nxt);
        double c = 0.0;
        for (int x = 0; x < N; ++x) c += nxt[x];
        for (int x = 0; x < N; ++x) alpha[x] = nxt[x] / c;
        logZ += log(c);
    }
    logZ += log(alpha[xe]);
    free(alpha); free(f); free(nxt);
    return logZ;
}

/* Open-path weights of a block (Sec. 4, "Observables": n_k needs <c^dag_j c_i>, the weight
 * of paths that do not close).  The block's filter from xs gives alpha_{l0+B}(y) = the sum
 * over block paths from xs ending at y instead of at the held xe; its ratio to the closed
 * value alpha_{l0+B}(xe) is the weight ratio of the configuration whose path is cut at
 * slice l0+B and displaced there by r, against the closed one.  Writes
 * ratio[rx + L ry] = alpha_{l0+B}(xe + (rx, ry)) / alpha_{l0+B}(xe) (periodic) and returns
 * the block's log-weight. */
double orc_open_ratio(int L, int M, const double *g, const double *W, int l0, int B, int xs, int xe,
                      double *ratio)
{
    int N = L * L;
    double *alpha = calloc(N, sizeof(double)), *f = malloc(N * sizeof(double)),
           *nxt = malloc(N * sizeof(double));
    double logZ = 0.0;
    alpha[xs] = 1.0;
    for (int i = 0; i < B; ++i) {
        int l = (l0 + i) % M;
        for (int x = 0; x < N; ++x) f[x] = W[(size_t)l * N + x] * alpha[x];
        orc_conv(L, g, f, nxt);
        double c = 0.0;
        for (int x = 0; x < N; ++x) c += nxt[x];
        for (int x = 0; x < N; ++x) alpha[x] = nxt[x] / c;
        logZ += log(c);
    }
    int ex = xe % L, ey = xe / L;
    for (int ry = 0; ry < L; ++ry)
        for (int rx = 0; rx < L; ++rx)
            ratio[rx + L * ry] = alpha[orc_wrap(ex + rx, L) + L * orc_wrap(ey + ry, L)] / alpha[xe];
    logZ += log(alpha[xe]);
    free(alpha); free(f); free(nxt);
    return logZ;
}

/* Forward filter of the closed loop of one worldline anchored at slice a, site xa:
 * the block of all M slices with both ends at xa. */
double orc_filter(int L, int M, const double *g, const double *W, int a, int xa, double *f_store)
{
    return orc_filter_block(L, M, g, W, a, M, xa, xa, f_store);
}

/* Backward sampling of the block's interior given the stored f_l and x_{l0+B} (already in
 * xpath): for i = B-1..1, l = (l0+i) mod M, draw x_l from p(y) ~ f_l(y) G(x_{l+1} - y) by
 * the row-major inverse CDF, the smallest y with u*S < C(y).  margin[l] (optional)
 * receives the distance from u*S to the nearer edge of the chosen CDF interval, over S. */
void orc_backward_block(int L, int M, const double *g, const double *f_store, int l0, int B,
                        uint64_t seed, uint64_t sweep, uint64_t wl, int32_t *xpath, double *margin)
{
    int N = L * L;
    double *p = malloc(N * sizeof(double));
    for (int i = B - 1; i >= 1; --i) {
        int l = (l0 + i) % M, next = xpath[(l + 1) % M];
        double S = 0.0;
        for (int y = 0; y < N; ++y) {
            p[y] = f_store[(size_t)l * N + y] * orc_G(g, L, y, next);
            S += p[y];
        }
        double u = orc_uniform(seed, sweep, 0, wl, (uint64_t)l);
        double target = u * S, C = 0.0, Cprev = 0.0;
        int pick = -1;
        for (int y = 0; y < N; ++y) {
            Cprev = C;
            C += p[y];
            if (target < C) { pick = y; break; }
        }
        if (pick < 0) { pick = next; Cprev = C = target; } /* S == 0: degenerate, stay */
        xpath[l] = pick;
        if (margin) {
            double m1 = target - Cprev, m2 = C - target;
            margin[l] = (S > 0.0) ? (m1 < m2 ? m1 : m2) / S : 0.0;
        }
    }
    if (margin) margin[l0 % M] = INFINITY; /* the block's start is held, not drawn */
    free(p);
}

/* Backward sampling of the closed loop anchored at slice a. */
void orc_backward(int L, int M, const double *g, const double *f_store, int a,
                  uint64_t seed, uint64_t sweep, uint64_t wl, int32_t *xpath, double *margin)
{
    orc_backward_block(L, M, g, f_store, a, M, seed, sweep, wl, xpath, margin);
}

/* ------------------------------------------------------------------------- */
/* One sweep of one chain: anchor, FFBS of every worldline, occupancy, Gibbs.  */
/* ------------------------------------------------------------------------- */

/* Inputs/outputs:
 *   s      [M][N] int8 +-1, updated by the Gibbs step.
 *   xpath  [2][Nsig][M] int32 site indices, updated by FFBS.
 *   logw   [2][Nsig] filter log-weights computed with the field before Gibbs (nullable).
 *   hist   [2][M][N] int32 occupancy of the new paths (nullable).
 *   margin [2][Nsig][M] CDF margins of every draw (nullable).
 *   links  [2][Nsig] sum over the M links of d/dt log G(x_{l+1} - x_l) (nullable).
 *   anchor receives the anchor slice (nullable).
 *   nwl_limit: if >= 0, only the first nwl_limit worldlines of each spin are
 *   resampled (a bounded sample for timing); the Gibbs step is then skipped.
 *   block: FFBS block length B (0 or >= M: the whole loop from the anchor); with B < M
 *   the loop is resampled block by block from the anchor, each with its ends held. 
 * Worldlines are independent given s, so they are processed in parallel. */
/* FFBS of every worldline (the first nwl of each spin) given the slice potentials
 * W [2][M][N] (spin-major): anchor, filter, backward draw, link sums. */
static double orc_link_sum(int L, int M, const double *g, const double *dg, const int32_t *xp, int next0);

/* perm (nullable: the identity) [2][Nsig]: with a permutation, the unit of worldline p is
 * the stretch from slice a of p to slice a of P(p): slices a+1..M-1 of p, then 0..a-1 of
 * P(p), with the ends x_a^{(p)} and x_a^{(P(p))} held (with P = identity, the closed loop
 * of p).  The units partition every slice but a, so they are independent given the slice-a
 * sites.  Unit p draws with the uniforms of worldline p.  margin and the drawn sites go to
 * the owning worldline. */
static int orc_ffbs_all(int L, int M, int Nsig, const double *g, const double *dg, const double *W,
                        uint64_t seed, uint64_t sweep, int32_t *xpath, double *logw, double *margin,
                        double *links, int *anchor, int nwl, int block, const int32_t *perm)
{
    int B = (block > 0 && block < M) ? block : M;
    int nblk = (M + B - 1) / B;
    int N = L * L;
    int a = (int)floor(orc_uniform(seed, sweep, 2, 0, 0) * M);
    if (a >= M) a = M - 1;
    if (anchor) *anchor = a;
    int total = 2 * nwl;
    /* worldlines in parallel when there are enough of them; otherwise the convolution
     * itself runs in parallel over output sites */
#pragma omp parallel for schedule(dynamic, 1) if (total >= 2 * orc_num_threads())
    for (int k = 0; k < total; ++k) {
        int sg = k / nwl, p = k % nwl;
        uint64_t wl = (uint64_t)sg * Nsig + p;
        uint64_t wq = (uint64_t)sg * Nsig + (perm ? perm[wl] : p);
        int32_t *xp = xpath + wl * M, *xq = xpath + wq * M;
        double *fst = malloc((size_t)M * N * sizeof(double));
        /* the unit's sites by slice: p from a on, P(p) before a; at a itself the end site
         * x_a^{(P(p))}, which the last interior draw conditions on */
        int32_t *vp = malloc(M * sizeof(int32_t));
        double *vm = margin ? malloc(M * sizeof(double)) : NULL;
        for (int l = 0; l < M; ++l) vp[l] = (l < a) ? xq[l] : xp[l];
        vp[a] = xq[a];
        /* blocks a, a+B, a+2B, ... (the last one may be shorter), resampled in turn with
         * their end sites held; the log-weight is the sum of the blocks' */
        double lz = 0.0;
        for (int b = 0; b < nblk; ++b) {
            int l0 = (a + b * B) % M, len = (b + 1) * B <= M ? B : M - b * B;
            int xs = (b == 0) ? xp[a] : vp[l0], xe = vp[(l0 + len) % M];
            lz += orc_filter_block(L, M, g, W + (size_t)sg * M * N, l0, len, xs, xe, fst);
            orc_backward_block(L, M, g, fst, l0, len, seed, sweep, wl, vp, vm);
        }
        for (int l = 0; l < M; ++l) {
            if (l == a) continue;
            if (l < a) xq[l] = vp[l];
            else xp[l] = vp[l];
            if (vm) margin[((l < a) ? wq : wl) * M + l] = vm[l];
        }
        if (vm) margin[wl * M + a] = INFINITY; /* slice a is held */
        if (logw) logw[wl] = lz;
        free(fst);
        free(vp);
        free(vm);
    }
    /* link sums of the final paths (a second pass: a worldline's early slices belong to
     * another unit) */
    if (links)
        for (int k = 0; k < total; ++k) {
            int sg = k / nwl, p = k % nwl;
            uint64_t wl = (uint64_t)sg * Nsig + p;
            uint64_t wq = (uint64_t)sg * Nsig + (perm ? perm[wl] : p);
            links[wl] = orc_link_sum(L, M, g, dg, xpath + wl * M, xpath[wq * M]);
        }
    return a;
}

/* Kinetic estimator of one worldline: sum over its M links of
 * d/dt log G(x_{l+1} - x_l) = g'(dx)/g(dx) + g'(dy)/g(dy), the last link going to next0
 * (its own x_0 when closed on itself, x_0 of P(p) with a permutation). */
static double orc_link_sum(int L, int M, const double *g, const double *dg, const int32_t *xp, int next0)
{
    double acc = 0.0;
    for (int l = 0; l < M; ++l) {
        int x0 = xp[l], x1 = (l + 1 < M) ? xp[l + 1] : next0;
        int dx = orc_wrap((x1 % L) - (x0 % L), L), dy = orc_wrap((x1 / L) - (x0 / L), L);
        acc += dg[dx] / g[dx] + dg[dy] / g[dy];
    }
    return acc;
}

/* Occupancy histogram [2][M][N] of the current worldlines. */
static void orc_histogram(int L, int M, int Nsig, const int32_t *xpath, int32_t *n)
{
    int N = L * L;
    memset(n, 0, (size_t)2 * M * N * sizeof(int32_t));
    for (int sg = 0; sg < 2; ++sg)
        for (int p = 0; p < Nsig; ++p)
            for (int l = 0; l < M; ++l)
                n[((size_t)sg * M + l) * N + xpath[((size_t)sg * Nsig + p) * M + l]] += 1;
}

/* Hirsch-Gibbs step (Sec. 3.5.4): every field from its factorised conditional
 * P(s = +1 | paths) = 1 / (1 + exp(-2 lambda m)), m = n_up - n_dn, phase-1 uniform. */
static void orc_gibbs_hirsch(int L, int M, double lam, uint64_t seed, uint64_t sweep, const int32_t *n, int8_t *s)
{
    int N = L * L;
    for (int l = 0; l < M; ++l)
        for (int x = 0; x < N; ++x) {
            int m = n[(size_t)l * N + x] - n[((size_t)M + l) * N + x];
            double pplus = 1.0 / (1.0 + exp(-2.0 * lam * m));
            double u = orc_uniform(seed, sweep, 1, (uint64_t)l, (uint64_t)x);
            s[(size_t)l * N + x] = (u < pplus) ? 1 : -1;
        }
}

/* Hirsch slice potentials W [2][M][N] = exp(sigma lambda s), sigma = +1 up, -1 down. */
static double *orc_hirsch_W(int L, int M, double lam, const int8_t *s)
{
    int N = L * L;
    double *W = malloc((size_t)2 * M * N * sizeof(double));
    for (int sg = 0; sg < 2; ++sg) {
        double sigma = sg == 0 ? 1.0 : -1.0;
        for (int l = 0; l < M; ++l)
            for (int x = 0; x < N; ++x)
                W[((size_t)sg * M + l) * N + x] = exp(sigma * lam * s[(size_t)l * N + x]);
    }
    return W;
}

int orc_sweep(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed, uint64_t sweep,
              int8_t *s, int32_t *xpath, double *logw, int32_t *hist, double *margin,
              double *links, int *anchor, int nwl_limit, int block)
{
    int N = L * L;
    double lam = orc_lambda(U, dtau);
    double *g = malloc(L * sizeof(double)), *dg = malloc(L * sizeof(double));
    orc_g_table(L, t, dtau, g, dg);
    double *W = orc_hirsch_W(L, M, lam, s);
    int nwl = (nwl_limit >= 0 && nwl_limit < Nsig) ? nwl_limit : Nsig;
    orc_ffbs_all(L, M, Nsig, g, dg, W, seed, sweep, xpath, logw, margin, links, anchor, nwl, block, NULL);
    if (nwl_limit < 0 || nwl_limit >= Nsig) {
        int32_t *n = hist ? hist : malloc((size_t)2 * M * N * sizeof(int32_t));
        orc_histogram(L, M, Nsig, xpath, n);
        orc_gibbs_hirsch(L, M, lam, seed, sweep, n, s);
        if (!hist) free(n);
    }
    free(g); free(dg); free(W);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Attractive U < 0: continuous Gaussian field (Sec. 3.5.5, Eq. gaussHS,      */
/* Eq. gaussCond).  Reading: a = sqrt(|U| dtau) and the shift n - 1/2 of the   */
/* main text (the appendix's sqrt(|U| dtau / 2)(n - 1) does not reproduce     */
/* exp(|U| dtau n_up n_dn)).  Every worldline, of either spin, sees            */
/* W_l(x) = exp(a sigma_{x,l}); the factor exp(-a sigma / 2) and the Gaussian  */
/* belong to the field's own weight.                                          */
/* ------------------------------------------------------------------------- */

/* Standard normal from two uniforms in [0,1) by the Box-Muller transform (Box and
 * Muller, 1958): z = sqrt(-2 ln(1 - u1)) cos(2 pi u2). */
double orc_normal(double u1, double u2)
{
    return sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * ORC_PI * u2);
}

/* a = sqrt(|U| dtau). */
double orc_gauss_coupling(double U, double dtau)
{
    return sqrt(fabs(U) * dtau);
}

/* Initial field: sigma[l][x] standard normal from phase 3 (sweep 2^64-1), j = 2x, 2x+1. */
void orc_init_sigma(int L, int M, uint64_t seed, double *sigma)
{
    int N = L * L;
    for (int l = 0; l < M; ++l)
        for (int x = 0; x < N; ++x)
            sigma[(size_t)l * N + x] = orc_normal(orc_uniform(seed, UINT64_MAX, 3, (uint64_t)l, 2 * (uint64_t)x),
                                                  orc_uniform(seed, UINT64_MAX, 3, (uint64_t)l, 2 * (uint64_t)x + 1));
}

/* Gaussian Gibbs step (Eq. gaussCond): sigma_{x,l} ~ N(a (n_up + n_dn - 1/2), 1), the
 * normal from the phase-1 uniforms of j = 2x, 2x+1. */
static void orc_gibbs_gauss(int L, int M, double a, uint64_t seed, uint64_t sweep, const int32_t *n, double *sigma)
{
    int N = L * L;
    for (int l = 0; l < M; ++l)
        for (int x = 0; x < N; ++x) {
            int nt = n[(size_t)l * N + x] + n[((size_t)M + l) * N + x];
            double u1 = orc_uniform(seed, sweep, 1, (uint64_t)l, 2 * (uint64_t)x);
            double u2 = orc_uniform(seed, sweep, 1, (uint64_t)l, 2 * (uint64_t)x + 1);
            sigma[(size_t)l * N + x] = a * (nt - 0.5) + orc_normal(u1, u2);
        }
}

/* Gaussian-field slice potentials W [2][M][N] = exp(a sigma), both spins. */
static double *orc_gauss_W(int L, int M, double a, const double *sigma)
{
    int N = L * L;
    double *W = malloc((size_t)2 * M * N * sizeof(double));
    for (int sg = 0; sg < 2; ++sg)
        for (int l = 0; l < M; ++l)
            for (int x = 0; x < N; ++x)
                W[((size_t)sg * M + l) * N + x] = exp(a * sigma[(size_t)l * N + x]);
    return W;
}

/* One sweep with the Gaussian field: FFBS as in orc_sweep with W = exp(a sigma) for both
 * spins, then sigma_{x,l} ~ N(a (n_up + n_dn - 1/2), 1), drawn from phase 1 with
 * j = 2x, 2x+1. */
int orc_sweep_gauss(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed, uint64_t sweep,
                    double *sigma, int32_t *xpath, double *logw, int32_t *hist, double *margin,
                    double *links, int *anchor, int nwl_limit, int block)
{
    int N = L * L;
    double a = orc_gauss_coupling(U, dtau);
    double *g = malloc(L * sizeof(double)), *dg = malloc(L * sizeof(double));
    orc_g_table(L, t, dtau, g, dg);
    double *W = orc_gauss_W(L, M, a, sigma);
    int nwl = (nwl_limit >= 0 && nwl_limit < Nsig) ? nwl_limit : Nsig;
    orc_ffbs_all(L, M, Nsig, g, dg, W, seed, sweep, xpath, logw, margin, links, anchor, nwl, block, NULL);
    if (nwl_limit < 0 || nwl_limit >= Nsig) {
        int32_t *n = hist ? hist : malloc((size_t)2 * M * N * sizeof(int32_t));
        orc_histogram(L, M, Nsig, xpath, n);
        orc_gibbs_gauss(L, M, a, seed, sweep, n, sigma);
        if (!hist) free(n);
    }
    free(g); free(dg); free(W);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Local link update (Sec. 3.5.1, Eq. Rlocal), read in the position basis: the */
/* momentum-space ratio's kinetic factors become the propagators G to the two  */
/* held neighbours and its potential factors become W_l at the old and new     */
/* site.  One site x_l of one worldline moves by one lattice step e (uniform   */
/* over +x, -x, +y, -y, a symmetric proposal) with x_{l-1}, x_{l+1} held, and  */
/* is accepted with probability min(1, R) (Metropolis).                        */
/* ------------------------------------------------------------------------- */

/* The site one lattice step from x: dir 0 = +x, 1 = -x, 2 = +y, 3 = -y. */
int orc_local_step(int L, int x, int dir)
{
    int ix = x % L, iy = x / L;
    if (dir == 0) ix = orc_wrap(ix + 1, L);
    else if (dir == 1) ix = orc_wrap(ix - 1, L);
    else if (dir == 2) iy = orc_wrap(iy + 1, L);
    else iy = orc_wrap(iy - 1, L);
    return ix + L * iy;
}

/* R of moving slice l of a worldline from x to xnew, given the slice potential Wl [N] and
 * the held neighbours xm = x_{l-1}, xn = x_{l+1}:
 *   R = G(xnew - xm) W_l(xnew) G(xn - xnew) / (G(x - xm) W_l(x) G(xn - x)).
 * M = 1 (the slice is its own neighbour, the link G(0) does not change): R = W(xnew)/W(x). */
double orc_local_ratio(int L, int M, const double *g, const double *Wl, int xm, int x, int xn, int xnew)
{
    if (M == 1) return Wl[xnew] / Wl[x];
    double num = orc_G(g, L, xm, xnew) * Wl[xnew] * orc_G(g, L, xnew, xn);
    double den = orc_G(g, L, xm, x) * Wl[x] * orc_G(g, L, x, xn);
    return num / den;
}

/* Colour of slice l: slices of one colour are never neighbours in imaginary time, so
 * their updates are independent given the rest (even l, odd l, and l = M-1 alone when
 * M is odd). */
int orc_local_color(int M, int l)
{
    return (M % 2 == 1 && l == M - 1) ? 2 : l % 2;
}

/* One local sweep of every worldline given W [2][M][N]: colours 0, 1, 2 in turn, every
 * slice of the colour of every worldline proposed once.  With a permutation perm
 * (nullable: the identity), slice 0 of p follows slice M-1 of P^{-1}(p) and slice M-1 of p
 * precedes slice 0 of P(p); those are of other colours (M >= 2), so one colour's moves stay
 * independent.  Uniforms: phase 4, i = sigma Nsig + p, j = 2l for the step
 * (dir = floor(4u)) and j = 2l + 1 for the acceptance (accept iff u < R).  margin[wl][l]
 * (optional) receives |u - R| (INFINITY when R >= 1: always accepted).  Returns the
 * number of accepted moves. */
static long long orc_local_all(int L, int M, int Nsig, const double *g, const double *dg, const double *W,
                               uint64_t seed, uint64_t sweep, int32_t *xpath, double *margin, double *links,
                               const int32_t *perm)
{
    int N = L * L;
    long long accepted = 0;
    int32_t *pinv = malloc((size_t)2 * Nsig * sizeof(int32_t));
    for (int k = 0; k < 2 * Nsig; ++k) pinv[k] = k % Nsig;
    if (perm)
        for (int k = 0; k < 2 * Nsig; ++k) pinv[(k / Nsig) * Nsig + perm[k]] = k % Nsig;
    for (int c = 0; c < 3; ++c) {
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : accepted) if (2 * Nsig >= 2 * orc_num_threads())
        for (int k = 0; k < 2 * Nsig; ++k) {
            int sg = k / Nsig;
            uint64_t wl = (uint64_t)k;
            int32_t *xp = xpath + wl * M;
            const int32_t *xprev = xpath + ((uint64_t)sg * Nsig + pinv[k]) * M;
            const int32_t *xnext = xpath + ((uint64_t)sg * Nsig + (perm ? perm[k] : k % Nsig)) * M;
            for (int l = 0; l < M; ++l) {
                if (orc_local_color(M, l) != c) continue;
                int xm = (l > 0) ? xp[l - 1] : xprev[M - 1], x = xp[l], xn = (l + 1 < M) ? xp[l + 1] : xnext[0];
                double u0 = orc_uniform(seed, sweep, 4, wl, 2 * (uint64_t)l);
                double u1 = orc_uniform(seed, sweep, 4, wl, 2 * (uint64_t)l + 1);
                int dir = (int)(u0 * 4.0);
                if (dir > 3) dir = 3;
                int xnew = orc_local_step(L, x, dir);
                double R = orc_local_ratio(L, M, g, W + ((size_t)sg * M + l) * N, xm, x, xn, xnew);
                if (margin) margin[wl * M + l] = (R >= 1.0) ? INFINITY : fabs(u1 - R);
                if (u1 < R) {
                    xp[l] = xnew;
                    ++accepted;
                }
            }
        }
    }
    if (links)
        for (int k = 0; k < 2 * Nsig; ++k) {
            uint64_t wq = (uint64_t)(k / Nsig) * Nsig + (perm ? perm[k] : k % Nsig);
            links[k] = orc_link_sum(L, M, g, dg, xpath + (uint64_t)k * M, xpath[wq * M]);
        }
    free(pinv);
    return accepted;
}

/* One local-update sweep of one chain: local moves of every worldline (above), occupancy,
 * then the same Gibbs step as the FFBS sweep (Hirsch for U >= 0 with s; Gaussian for
 * U < 0 with sigma).  Outputs as in orc_sweep; *accepted receives the accepted moves. */
int orc_sweep_local(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed, uint64_t sweep,
                    int8_t *s, double *sigma, int32_t *xpath, int32_t *hist, double *margin, double *links,
                    long long *accepted, const int32_t *perm)
{
    int N = L * L;
    double *g = malloc(L * sizeof(double)), *dg = malloc(L * sizeof(double));
    orc_g_table(L, t, dtau, g, dg);
    double lam = U < 0.0 ? 0.0 : orc_lambda(U, dtau), a = orc_gauss_coupling(U, dtau);
    double *W = U < 0.0 ? orc_gauss_W(L, M, a, sigma) : orc_hirsch_W(L, M, lam, s);
    long long acc = orc_local_all(L, M, Nsig, g, dg, W, seed, sweep, xpath, margin, links, perm);
    if (accepted) *accepted = acc;
    int32_t *n = hist ? hist : malloc((size_t)2 * M * N * sizeof(int32_t));
    orc_histogram(L, M, Nsig, xpath, n);
    if (U < 0.0) orc_gibbs_gauss(L, M, a, seed, sweep, n, sigma);
    else orc_gibbs_hirsch(L, M, lam, seed, sweep, n, s);
    if (!hist) free(n);
    free(g); free(dg); free(W);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Permutation updates (Sec. 3.5.3): reconnect worldlines at tau = beta.  A   */
/* pair swap exchanges the successors of two worldlines p, q of one spin,      */
/* P'(p) = P(q), P'(q) = P(p); only the two links across tau = beta change.   */
/* Sampling |w|, it is accepted with probability min(1, R); each accepted swap */
/* flips sgn(P), which reweights observables (Eq. reweight).                  */
/* ------------------------------------------------------------------------- */

/* R of the swap, from the last sites xlp = x_{M-1}^{(p)}, xlq = x_{M-1}^{(q)} and the
 * successors' first sites a0 = x_0^{(P(p))}, b0 = x_0^{(P(q))}:
 *   R = G(b0 - xlp) G(a0 - xlq) / (G(a0 - xlp) G(b0 - xlq)). */
double orc_perm_ratio(int L, const double *g, int xlp, int xlq, int a0, int b0)
{
    return (orc_G(g, L, xlp, b0) * orc_G(g, L, xlq, a0)) / (orc_G(g, L, xlp, a0) * orc_G(g, L, xlq, b0));
}

/* One permutation update of both spins.  Pairing: rotation r = floor(u Nsig) (phase 5,
 * i = sigma, j = 0) and the disjoint pairs (2k + r, 2k + 1 + r) mod Nsig, k < Nsig/2 (a
 * state-independent choice, each swap its own inverse, so the proposal is symmetric;
 * over the rotations every adjacent transposition is proposed, which generates every
 * permutation).  Pair k is accepted iff u < R (phase 5, i = sigma, j = 1 + k).
 * margin (optional) [2][Nsig/2] receives |u - R| (INFINITY when R >= 1).  Returns the
 * accepted swaps; *sign flips with each. */
static long long orc_perm_update(int L, int M, int Nsig, const double *g, uint64_t seed, uint64_t sweep,
                                 const int32_t *xpath, int32_t *perm, int *sign, double *margin)
{
    long long acc = 0;
    int npr = Nsig / 2;
    for (int sg = 0; sg < 2; ++sg) {
        if (npr == 0) continue;
        int r = (int)floor(orc_uniform(seed, sweep, 5, (uint64_t)sg, 0) * Nsig);
        if (r >= Nsig) r = Nsig - 1;
        int32_t *P = perm + (size_t)sg * Nsig;
        const int32_t *X = xpath + (size_t)sg * Nsig * M;
        for (int k = 0; k < npr; ++k) {
            int p = (2 * k + r) % Nsig, q = (2 * k + 1 + r) % Nsig;
            double R = orc_perm_ratio(L, g, X[(size_t)p * M + M - 1], X[(size_t)q * M + M - 1],
                                      X[(size_t)P[p] * M], X[(size_t)P[q] * M]);
            double u = orc_uniform(seed, sweep, 5, (uint64_t)sg, 1 + (uint64_t)k);
            if (margin) margin[(size_t)sg * npr + k] = (R >= 1.0) ? INFINITY : fabs(u - R);
            if (u < R) {
                int t = P[p];
                P[p] = P[q];
                P[q] = t;
                *sign = -*sign;
                ++acc;
            }
        }
    }
    return acc;
}

/* One sweep with permutations: the permutation update (above), then FFBS of every
 * worldline's unit under the new permutation (orc_ffbs_all), the occupancy and the Gibbs
 * step of the chain's field type.  perm [2][Nsig] and *sign are updated in place;
 * *swaps receives the accepted swaps; margin_perm [2][Nsig/2] (nullable).  Other outputs
 * as in orc_sweep (logw per unit). */
int orc_sweep_perm(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed, uint64_t sweep,
                   int8_t *s, double *sigma, int32_t *xpath, int32_t *perm, int *sign, double *logw,
                   int32_t *hist, double *margin, double *margin_perm, double *links, int *anchor, int block,
                   long long *swaps)
{
    int N = L * L;
    double *g = malloc(L * sizeof(double)), *dg = malloc(L * sizeof(double));
    orc_g_table(L, t, dtau, g, dg);
    double lam = U < 0.0 ? 0.0 : orc_lambda(U, dtau), a = orc_gauss_coupling(U, dtau);
    double *W = U < 0.0 ? orc_gauss_W(L, M, a, sigma) : orc_hirsch_W(L, M, lam, s);
    long long acc = orc_perm_update(L, M, Nsig, g, seed, sweep, xpath, perm, sign, margin_perm);
    if (swaps) *swaps = acc;
    orc_ffbs_all(L, M, Nsig, g, dg, W, seed, sweep, xpath, logw, margin, links, anchor, Nsig, block, perm);
    int32_t *n = hist ? hist : malloc((size_t)2 * M * N * sizeof(int32_t));
    orc_histogram(L, M, Nsig, xpath, n);
    if (U < 0.0) orc_gibbs_gauss(L, M, a, seed, sweep, n, sigma);
    else orc_gibbs_hirsch(L, M, lam, seed, sweep, n, s);
    if (!hist) free(n);
    free(g); free(dg); free(W);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Forward-backward marginals and d log Z / dt of one worldline (adjoint of   */
/* Eq. ffbsFwd).  Anchor slice 0, site x0.  v is [M][N] log-potential.         */
/* ------------------------------------------------------------------------- */
double orc_marginals(int L, int M, const double *g, const double *dg, const double *v, int x0,
                     double *marg, double *dlogZ_dt)
{
    int N = L * L;
    double *F = malloc((size_t)M * N * sizeof(double));
    double *alpha = calloc(N, sizeof(double)), *tmp = malloc(N * sizeof(double));
    double *b = calloc(N, sizeof(double)), *H = malloc(N * sizeof(double)),
           *Hd = malloc(N * sizeof(double));
    double logZ = 0.0;
    alpha[x0] = 1.0;
    for (int l = 0; l < M; ++l) {
        for (int x = 0; x < N; ++x) F[(size_t)l * N + x] = exp(v[(size_t)l * N + x]) * alpha[x];
        orc_conv(L, g, F + (size_t)l * N, tmp);
        double c = 0.0;
        for (int x = 0; x < N; ++x) c += tmp[x];
        for (int x = 0; x < N; ++x) alpha[x] = tmp[x] / c;
        logZ += log(c);
    }
    logZ += log(alpha[x0]);
    /* backward messages: b_M = delta_{x0}; H_l = G * b_{l+1}; b_l = W_l H_l */
    b[x0] = 1.0;
    double dt = 0.0;
    for (int l = M - 1; l >= 0; --l) {
        orc_conv(L, g, b, H);       /* G is even, so correlation == convolution */
        orc_conv_dG(L, g, dg, b, Hd);
        double z = 0.0, zd = 0.0;
        for (int x = 0; x < N; ++x) {
            z += F[(size_t)l * N + x] * H[x];
            zd += F[(size_t)l * N + x] * Hd[x];
        }
        if (marg)
            for (int x = 0; x < N; ++x) marg[(size_t)l * N + x] = F[(size_t)l * N + x] * H[x] / z;
        dt += zd / z;
        double c = 0.0;
        for (int x = 0; x < N; ++x) { b[x] = exp(v[(size_t)l * N + x]) * H[x]; c += b[x]; }
        for (int x = 0; x < N; ++x) b[x] /= c;
    }
    if (dlogZ_dt) *dlogZ_dt = dt;
    free(F); free(alpha); free(tmp); free(b); free(H); free(Hd);
    return logZ;
}

/* Whole-chain gradient: logZ = sum over worldlines, each anchored at slice 0 on
 * its current site; dv[sigma][l][x] = sum_p marginal; v defaults to sigma*lambda*s. */
double orc_chain_grad(int L, int M, int Nsig, double t, double U, double dtau, const int8_t *s,
                      const double *v_in, const int32_t *xpath, double *dv, double *dlogZ_dt)
{
    int N = L * L;
    double lam = orc_lambda(U, dtau);
    double *g = malloc(L * sizeof(double)), *dg = malloc(L * sizeof(double));
    orc_g_table(L, t, dtau, g, dg);
    double *v = malloc((size_t)2 * M * N * sizeof(double));
    for (int sg = 0; sg < 2; ++sg)
        for (size_t k = 0; k < (size_t)M * N; ++k)
            v[(size_t)sg * M * N + k] = v_in ? v_in[(size_t)sg * M * N + k]
                                             : (sg == 0 ? 1.0 : -1.0) * lam * s[k];
    if (dv) memset(dv, 0, (size_t)2 * M * N * sizeof(double));
    double total = 0.0, dtt = 0.0;
    int nw = 2 * Nsig;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total, dtt)
    for (int k = 0; k < nw; ++k) {
        int sg = k / Nsig;
        double *marg = malloc((size_t)M * N * sizeof(double)), d = 0.0;
        total += orc_marginals(L, M, g, dg, v + (size_t)sg * M * N, xpath[(size_t)k * M], marg, &d);
        dtt += d;
        if (dv) {
#pragma omp critical
            for (size_t q = 0; q < (size_t)M * N; ++q) dv[(size_t)sg * M * N + q] += marg[q];
        }
        free(marg);
    }
    if (dlogZ_dt) *dlogZ_dt = dtt;
    free(g); free(dg); free(v);
    return total;
}

/* ------------------------------------------------------------------------- */
/* Observables of one configuration (Sec. 4, "Observables"), summed over       */
/* slices.  hist is [2][M][N]; out receives                                    */
/*   out[0] = sum n_up + n_dn, out[1] = sum n_up n_dn, out[2] = sum m^2        */
/* and Sk[k] = sum_l |m^(k)|^2 / N with m^(k) = sum_x m(x) e^{-i k.x},          */
/* Cr[r] = sum_l sum_x m(x) m(x + r) / N, both on the N-point grid.            */
/* ------------------------------------------------------------------------- */
void orc_measure(int L, int M, const int32_t *hist, double *out, double *Sk, double *Cr)
{
    int N = L * L;
    double sn = 0, sd = 0, sm = 0;
    int *m = malloc(N * sizeof(int));
    if (Sk) memset(Sk, 0, N * sizeof(double));
    if (Cr) memset(Cr, 0, N * sizeof(double));
    for (int l = 0; l < M; ++l) {
        for (int x = 0; x < N; ++x) {
            int nu = hist[(size_t)l * N + x], nd = hist[((size_t)M + l) * N + x];
            sn += nu + nd; sd += (double)nu * nd;
            m[x] = nu - nd; sm += (double)m[x] * m[x];
        }
        if (Sk)
            for (int k = 0; k < N; ++k) {
                int kx = k % L, ky = k / L;
                double re = 0.0, im = 0.0;
                for (int x = 0; x < N; ++x) {
                    double ph = -2.0 * ORC_PI * ((double)kx * (x % L) + (double)ky * (x / L)) / L;
                    re += m[x] * cos(ph); im += m[x] * sin(ph);
                }
                Sk[k] += (re * re + im * im) / N;
            }
        if (Cr)
            for (int r = 0; r < N; ++r) {
                int rx = r % L, ry = r / L;
                double acc = 0.0;
                for (int x = 0; x < N; ++x) {
                    int y = orc_wrap(x % L + rx, L) + L * orc_wrap(x / L + ry, L);
                    acc += (double)m[x] * m[y];
                }
                Cr[r] += acc / N;
            }
    }
    out[0] = sn; out[1] = sd; out[2] = sm;
    free(m);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
