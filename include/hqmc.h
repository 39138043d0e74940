/*
 * hqmc.h -- C ABI of the GB300 (sm_103a) worldline sampler for the 2D repulsive
 * Hubbard model of arXiv 2510.13866, "FFT-Accelerated Auxiliary Variable MCMC for
 * Fermionic Lattice Models".
 *
 * One sweep of a chain is
 *   1. an anchor slice a drawn per chain,
 *   2. forward-filtering backward-sampling (FFBS) of every worldline with its
 *      position at slice a held (Sec. 3.5.2, Eq. ffbsFwd and the backward
 *      conditional that follows it),
 *   3. the factorised Gibbs resample of every Hirsch field s_{x,l}
 *      (Sec. 3.5.4: P(s=+1 | paths) = (1 + tanh(lambda m)) / 2, m = n_up - n_dn),
 *   4. accumulation of the observables of Sec. 4 from the new occupations.
 *
 * Conventions used by every entry point:
 *   - site x = ix + L*iy on an L x L torus, N = L*L; slices l = 0..M-1, M = beta/dtau.
 *   - the forward filter runs in the position basis: alpha <- G * (W_l . alpha)
 *     with G(d) = <x+d| exp(-dtau K) |x> (the kinetic factors D(k) of Eq. Tkk,
 *     eps_k = -2t (cos kx + cos ky)) and W_{l,sigma}(x) = exp(sigma lambda s_{x,l}),
 *     sigma = +1 for up, -1 for down, cosh(lambda) = exp(dtau U / 2) (Eq. hirsch).
 *   - worldlines close on themselves (permutation = identity); log-weights leave out
 *     every constant of the Hirsch identity and the field prior 2^{-NM}.
 *   - random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, 0),
 *     counter (j >> 2, i, phase, sweep), word j & 3, u = (word >> 11) * 2^-53;
 *     phase 0 = FFBS draw (i = sigma*Nsig + p, j = l), 1 = Gibbs (i = l, j = x),
 *     2 = anchor (i = j = 0), 3 = initial field (sweep = 2^64-1, i = l, j = x).
 *   - "packed over chains" means chain 0's block, then chain 1's, ... with no padding.
 *
 * Errors: every int-returning call returns HQMC_OK (0) or a negative HQMC_ERR_* code;
 * hqmc_strerror gives its text and hqmc_last_error_detail the context's last message.
 * A context is bound to one device and one CUDA stream; it is not thread safe.
 */
#ifndef HQMC_H
#define HQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hqmc_ctx hqmc_ctx;

/* arithmetic of the forward filter and backward sampler */
#define HQMC_FP32 0 /* FP32 FFT and convolution; FP64 only for log Z and the Gibbs ratios */
#define HQMC_FP64 1 /* every step in FP64 (the plain comparison form) */

#define HQMC_OK 0
#define HQMC_ERR_ARG (-1)         /* invalid argument (see each call) */
#define HQMC_ERR_NOMEM (-2)       /* device allocation failed or workspace too small */
#define HQMC_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define HQMC_ERR_TIMEOUT (-4)     /* reserved: no kernel of this library waits on a flag, a peer or a
                                   * barrier it does not own, so no call returns it today */
#define HQMC_ERR_STATE (-5)       /* call out of order (e.g. sweep before set_params) */
#define HQMC_ERR_UNSUPPORTED (-6) /* lattice size or mode not built into this library */
#define HQMC_ERR_NUMERIC (-7)     /* a draw met an all-zero CDF or log Z met a non-positive amplitude */
#define HQMC_ERR_SCRATCH (-8)     /* the problem does not fit hqmc_ffbs_noalloc's static scratch */

/* Observables of one chain, averaged over slices and over the sweeps accumulated
 * since the last reset (Sec. 4, "Observables").  Per-site quantities. */
typedef struct {
    int64_t n_samples; /* sweeps accumulated */
    double density;    /* <n_up + n_dn> */
    double double_occ; /* D = <n_up n_dn> */
    double m2;         /* <(n_up - n_dn)^2> = 4 <(S^z)^2> */
    double ekin;       /* -(t/beta) <sum over links d/dt log G(x_{l+1} - x_l)> / N */
    double s_pipi;     /* S(k) at k = (pi, pi) (nearest grid point for odd L) */
    /* FFBS diagnostics since the last reset (not errors; a sweep continues):
     * n_degenerate   draws whose CDF was all zero (the worldline keeps its site at that
     *                slice) plus forward slices with a non-finite normaliser -- in FP32 this
     *                happens where a path sits in a region whose true weight lies below the
     *                FFT's rounding floor (about 1e-7 of the slice maximum);
     * n_nonpositive  filter amplitudes alpha_M(x_a) <= 0 (that log-weight is not finite). */
    int64_t n_degenerate;
    int64_t n_nonpositive;
    int64_t n_local_accepted; /* local link moves accepted (hqmc_local_sweep) since the last reset */
    /* With permutations (hqmc_set_permutations) the sampled weight is |w| and every average
     * above is sign-reweighted, <O> = sum(O s) / sum(s) over the measured sweeps with
     * s = sgn(P_up) sgn(P_dn) (Eq. reweight); without them s = +1. */
    double mean_sign;         /* sum(s) / n_samples */
    int64_t n_perm_accepted;  /* permutation swaps accepted since the last reset */
    /* filter log-weights (one per worldline and sweep since the last reset) whose error
     * estimate (hqmc_logw_error) exceeds the precision's tolerance, 1e-5 (FP32) or 1e-12
     * (FP64) of max(1, |log Z|); such a log-weight may be less accurate than that. */
    int64_t n_inexact;
} hqmc_obs;

/* Create a context for n_chains independent chains on CUDA device `device`.
 *   L[c]      linear size of chain c's lattice; 2 <= L[c] and L[c] must be one of the
 *             sizes built into the library (hqmc_supported_L), else HQMC_ERR_UNSUPPORTED:
 *             2, 3, 4, 6, 8, 12, 16, 24, 32 (a warp group per worldline pair) and 48, 64,
 *             128 (a thread per line of each worldline), all in both precisions and for
 *             every entry point.
 *   seeds[c]  Philox key of chain c.
 *   precision HQMC_FP32 or HQMC_FP64.
 * *out receives the context (caller frees it with hqmc_destroy).  No device memory is
 * allocated here.  Errors: HQMC_ERR_ARG (null pointers, n_chains < 1, bad precision),
 * HQMC_ERR_UNSUPPORTED, HQMC_ERR_CUDA (device cannot be selected). */
int hqmc_init_lattice(hqmc_ctx **out, int n_chains, const int *L, const uint64_t *seeds,
                      int precision, int device);

/* Model parameters of chain `chain` (-1 = all chains): hopping t >= 0, U (finite),
 * inverse temperature beta and slice dtau with beta/dtau an integer M (within 1e-9),
 * filling with filling*N/2 a positive integer Nsig (worldlines per spin, 2 Nsig <= 2N).
 * U >= 0 uses the discrete Hirsch field s = +-1 (Sec. 3.5.4): W = exp(sigma lambda s),
 * cosh lambda = exp(dtau U / 2).  U < 0 uses the continuous Gaussian field of Sec. 3.5.5
 * (Eq. gaussHS): W = exp(a sigma_{x,l}) for both spins, a = sqrt(|U| dtau), and the Gibbs
 * step draws sigma ~ N(a (n_up + n_dn - 1/2), 1) (Eq. gaussCond; reading: the main text's
 * a and shift, which reproduce exp(|U| dtau n_up n_dn); the appendix's sqrt(|U| dtau / 2)
 * and n - 1 do not).  Gaussian draws: Box-Muller from the uniforms of j = 2x and 2x+1.
 * Before the first sweep any parameter may change; afterwards only t, U and (beta,
 * dtau) at fixed M may change, and U keeps its sign (M, Nsig and the field type fix the
 * state), else HQMC_ERR_STATE.  Errors: HQMC_ERR_ARG, HQMC_ERR_UNSUPPORTED. */
int hqmc_set_params(hqmc_ctx *ctx, int chain, double t, double U, double beta, double dtau,
                    double filling);

/* FFBS block length B of one chain (chain = -1: all chains).  B = 0, or B >= M, resamples
 * each worldline as the closed loop of M slices from the anchor slice a with x_a held
 * (the default).  1 <= B < M resamples it block by block (Sec. 3.5.2, a block of slices
 * with fixed endpoints): the blocks start at a, a+B, a+2B, ... (mod M), the last one
 * ends at a and may be shorter, and each block's interior slices are drawn given its two
 * end sites, which keep their current values.  The sweep's log-weight of a worldline is
 * then the sum over its blocks of log sum_{paths inside} prod W G, each block's filter
 * started from delta at its first site and read at its last.  The blocks of a worldline
 * pair are independent work units of the FFBS launch (they share no slice but the held
 * ends), so a long loop spreads over many SMs; the partial log-weights are summed in
 * block order, which gives the same bits as resampling the blocks one after another.
 * Both kernels (L <= 32 and wide) and both precisions take it; the no-allocation entry
 * point always uses B = M.  A change of B re-lays the context out at its next use as
 * described at hqmc_set_class_launch (state kept, observable accumulators restart, an
 * attached workspace must be attached again).  Errors: HQMC_ERR_ARG (chain out of range,
 * B < 0), HQMC_ERR_CUDA. */
int hqmc_set_block(hqmc_ctx *ctx, int chain, int B);

/* Storage of the filter's f_l = W_l . alpha_l for the backward pass of the wide kernel
 * (L >= 48, FP32 context; L <= 32 and FP64 always stream):
 *   HQMC_FSTORE_STREAM  every f_l in FP32 (the default; 8 N bytes per particle-slice
 *                       written and read back)
 *   HQMC_FSTORE_BF16    f_l kept only every `stride` positions of the FFBS block (0 =
 *                       ceil(sqrt(longest block))), as BF16 (8 significant bits; the
 *                       normaliser exponent is not needed to sample); the backward pass
 *                       recomputes each stride-long segment in FP32 from its checkpoint into
 *                       a per-CTA buffer and samples from it.  f then carries the BF16
 *                       rounding (relative 2^-9) propagated through the segment, so draws can
 *                       differ from the streamed form where a uniform lies that close to a
 *                       CDF edge; log-weights come from the forward pass and are unchanged.
 *                       Memory per resident worldline drops from M N to about
 *                       (M / stride) N / 2 + stride N floats; the recompute doubles the FFT
 *                       work of the filter.
 *   HQMC_FSTORE_F32     the same with FP32 checkpoints: the recompute is exact, so every draw
 *                       equals the streamed form's (a check of the recompute path).
 * A change re-lays the context out at its next use as described at hqmc_set_class_launch.
 * Errors: HQMC_ERR_ARG, HQMC_ERR_UNSUPPORTED (checkpoints in an FP64 context), HQMC_ERR_CUDA. */
#define HQMC_FSTORE_STREAM 0
#define HQMC_FSTORE_BF16 1
#define HQMC_FSTORE_F32 2
int hqmc_set_ffbs_storage(hqmc_ctx *ctx, int kind, int stride);

/* CUDA stream (a cudaStream_t passed as void*) on which every later call is ordered;
 * NULL = the legacy default stream.  Changing it drops the captured sweep graph. */
int hqmc_set_stream(hqmc_ctx *ctx, void *stream);

/* Launch configuration: use_graph = replay one captured CUDA graph per sweep;
 * persistent = size the FFBS grid to the resident capacity (each worldline group
 * loops over pairs) instead of one group per pair; warps_per_cta in {1,2,4,8}
 * (0 = default).  Takes effect at the next sweep; a change of grid or shape re-lays
 * the context out as described at hqmc_set_class_launch.  Errors: HQMC_ERR_ARG. */
int hqmc_set_launch(hqmc_ctx *ctx, int use_graph, int persistent, int warps_per_cta);

/* Slices of one chain handled by one CTA of the Gibbs/measure kernel.  Up to L = 12 (the
 * context's largest lattice) the CTA handles its slices together, every loop running over
 * (slice, site) of the group, so a small lattice still fills the CTA; beyond, it handles them
 * one after another.  0 (the default) picks what measured fastest on GB300: 16 slices up to
 * L = 12 (fewer when the grid would hold under two CTAs per SM), then 4 up to L = 16, 2 up
 * to L = 48 and 1 above.  The grouped form caps the value by the shared memory the group
 * needs.  The fields, paths and integer sums do not depend
 * on it; S(k) may differ by FP64 rounding.  Errors: HQMC_ERR_ARG (outside 0..1024). */
int hqmc_set_slice_launch(hqmc_ctx *ctx, int slices_per_cta);

/* Warps per CTA of the FFBS kernel for the chains of lattice size L only (0 = the
 * context default); wide sizes (L > 32, one CTA per pair) have a fixed shape and ignore
 * it.  A change of shape re-lays the context out at its next use: fields, worldlines and
 * the sweep counter are kept, observable accumulators restart, and a workspace attached
 * by the caller must be attached again (hqmc_workspace_size gives the new size).
 * Errors: HQMC_ERR_ARG (no chain of size L, bad shape), HQMC_ERR_CUDA. */
int hqmc_set_class_launch(hqmc_ctx *ctx, int L, int warps_per_cta);

/* Effective warps per CTA for size L (0 for wide sizes).  Errors: HQMC_ERR_ARG. */
int hqmc_get_class_launch(hqmc_ctx *ctx, int L, int *warps_per_cta);

/* Autotuner of the CTA shape: for every register-line lattice size in the context, time
 * trial_sweeps sweeps of a temporary copy of that size's chains (same parameters, seeds
 * and precision; its own cudaMalloc'd workspace, destroyed afterwards) with 1, 2, 4 and
 * 8 warps per CTA, and keep the fastest with hqmc_set_class_launch.  The context's own
 * chains are not advanced.  Launch shapes give bitwise-identical results; only speed
 * changes.  *n_tuned (nullable) receives the number of sizes tuned.
 * Errors: HQMC_ERR_ARG, HQMC_ERR_STATE (no params), HQMC_ERR_NOMEM, HQMC_ERR_CUDA. */
int hqmc_autotune(hqmc_ctx *ctx, int trial_sweeps, int *n_tuned);

/* Device memory the context needs (state + scratch), in bytes, for the current
 * parameters and launch configuration.  Errors: HQMC_ERR_STATE before set_params. */
int hqmc_workspace_size(hqmc_ctx *ctx, size_t *bytes);

/* Hand the context a caller-owned device buffer of at least hqmc_workspace_size bytes,
 * 256-byte aligned; the caller keeps it alive until hqmc_destroy or the next attach.
 * Without an attached buffer the context allocates its own with cudaMalloc at the
 * first sweep.  Attaching re-initialises the chain state (fields and worldlines).
 * Errors: HQMC_ERR_ARG (null, misaligned), HQMC_ERR_NOMEM (too small). */
int hqmc_attach_workspace(hqmc_ctx *ctx, void *dev_ptr, size_t bytes);

/* Run n_sweeps >= 0 sweeps on the context's stream.  logw_out (nullable, host) receives
 * the FP64 filter log-weights log Z_p of the LAST sweep, packed over chains as
 * [2][Nsig] (spin-major), where Z_p = sum over closed paths of worldline p with its
 * anchor-slice position held of prod_l W_l(x_l) G(x_{l+1} - x_l), evaluated with the
 * field before that sweep's Gibbs step.  The call blocks until the sweeps finish.
 * Numerical degeneracies are counted (hqmc_obs.n_degenerate, n_nonpositive), not raised.
 * Errors: HQMC_ERR_STATE (no params), HQMC_ERR_NOMEM, HQMC_ERR_CUDA. */
int hqmc_sweep(hqmc_ctx *ctx, int n_sweeps, double *logw_out);

/* Error estimates of the log-weights of the last sweep, written to err_out (host, packed
 * like hqmc_sweep's logw_out).  The power-of-two normaliser is exact, so the error of a
 * block's log-weight is that of its end value alpha_end(x_end).  An FFT leaves every site
 * of a slice with a rounding error of about eps log2(N) of the slice's largest value, so a
 * site that ends kappa = max_y alpha_end(y) / alpha_end(x_end) times below the largest
 * carries about eps log2(N) kappa from each slice.  The estimate of a block of len slices
 * is eps log2(N) len kappa for a Hirsch field (eps = 2^-24 in FP32, 2^-53 in FP64; the end
 * concentration stands in for every slice's).  A strong Gaussian field concentrates the
 * message more inside the block than at its end, so for a Gaussian field it is
 * eps log2(N) (c sum_i E[max_y alpha_i(y) / alpha_i(x_i) | x_{i+1}] + kappa) over the block's
 * interior positions i, given the sites x_{i+1} the sweep drew (over the posterior of the
 * path these terms have the mean that carries slice i's rounding to the log-weight), with
 * the calibration factor c = 1 in FP32 and 32 in FP64.  The estimates of a worldline's
 * blocks are summed.  With HQMC_CONV_STENCIL every
 * output is a sum of non-negative terms that keeps its own relative accuracy and kappa is
 * replaced by 1.  A non-positive end value gives +inf.  Worldlines whose estimate exceeds
 * the precision's tolerance are counted in hqmc_obs.n_inexact; where this matters (strong
 * fields concentrate the message, kappa of 1e4 and beyond) the stencil form gives the
 * accurate value.  The estimate is calibrated, not a bound: against a direct O(N^2)
 * convolution, FP32 errors stayed below 0.73 of it.
 * Errors: HQMC_ERR_ARG, HQMC_ERR_STATE (no sweep yet), HQMC_ERR_CUDA. */
int hqmc_logw_error(hqmc_ctx *ctx, double *err_out);

/* Run n_sweeps >= 0 local-update sweeps (Sec. 3.5.1, Eq. Rlocal, read in the position
 * basis) on the context's stream, as an alternative or a complement to the FFBS sweep.
 * One sweep proposes, for every worldline and slice l once, a move of x_l by one lattice
 * step (+x, -x, +y, -y, uniform) with x_{l-1} and x_{l+1} held, accepted with probability
 * min(1, R), R = G(x'-x_{l-1}) W_l(x') G(x_{l+1}-x') / [G(x-x_{l-1}) W_l(x) G(x_{l+1}-x)]
 * in FP64 (M = 1: R = W_l(x')/W_l(x)).  Slices are visited by colour: even l, odd l, then
 * l = M-1 alone when M is odd (slices of one colour are never neighbours).  Uniforms:
 * Philox phase 4, i = sigma Nsig + p, j = 2l (step, floor(4u)) and 2l + 1 (accept iff
 * u < R).  Then the same Gibbs step and observable accumulation as hqmc_sweep; the sweep
 * counter advances.  Accepted moves are counted per chain (hqmc_obs.n_local_accepted).
 * Plain launches (no graph).  Errors: HQMC_ERR_ARG, HQMC_ERR_STATE, HQMC_ERR_CUDA. */
int hqmc_local_sweep(hqmc_ctx *ctx, int n_sweeps);

/* Permutation updates at tau = beta (Sec. 3.5.3).  on = 1: every later hqmc_sweep first
 * proposes, for each chain and spin, pair swaps of successors P'(p) = P(q), P'(q) = P(p)
 * over the disjoint pairs (2k + r, 2k + 1 + r) mod Nsig, k < Nsig/2, with the rotation
 * r = floor(u Nsig) (Philox phase 5, i = sigma, j = 0), each accepted iff u < R (phase 5,
 * j = 1 + k), R = G(x_0^{P(q)} - x_{M-1}^p) G(x_0^{P(p)} - x_{M-1}^q) /
 * [G(x_0^{P(p)} - x_{M-1}^p) G(x_0^{P(q)} - x_{M-1}^q)] in FP64; each accepted swap flips
 * the chain's sign.  The FFBS of the sweep then runs every worldline's unit from slice a of
 * p to slice a of P(p) (slices a+1..M-1 of p, then 0..a-1 of P(p), both slice-a sites
 * held), local sweeps link slice M-1 of p to slice 0 of P(p), and the observables are
 * sign-reweighted (hqmc_obs).  The permutation starts at the identity and is kept when
 * the updates are turned off again.  The adjoint then returns HQMC_ERR_UNSUPPORTED.
 * Errors: HQMC_ERR_STATE (set_params missing), HQMC_ERR_UNSUPPORTED (a chain with M < 2). */
int hqmc_set_permutations(hqmc_ctx *ctx, int on);

/* Line convolutions of the FFBS forward filter (a comparison of two ways to apply the
 * separable propagator G = g (x) g):
 *   HQMC_CONV_FFT      half-length real FFTs with a spectral mix (the default);
 *   HQMC_CONV_STENCIL  the direct periodic stencil out[x] = sum_{|d|<=R} g(d) v[x-d] with
 *                      R = min(6, (L-1)/2) (and the d = L/2 term once for even L <= 12):
 *                      the exact circulant for L <= 13, beyond it g truncated at |d| = 6,
 *                      which drops a relative weight below 2 sum_{d>6} g(d) / sum_d g(d)
 *                      per slice (about 3e-13 at t dtau = 0.05).  Sums of non-negative
 *                      terms keep small filter values accurate where the FFT leaves a
 *                      rounding floor.
 * Applies to L <= 32 (both precisions); the adjoint keeps its FFT.
 * Errors: HQMC_ERR_ARG, HQMC_ERR_UNSUPPORTED (a chain with L > 32). */
#define HQMC_CONV_FFT 0
#define HQMC_CONV_STENCIL 1
int hqmc_set_conv(hqmc_ctx *ctx, int kind);

/* The permutations of chain c, perm [2][Nsig] (host, int32: perm[sigma][p] = P(p)), and
 * sign = sgn(P_up) sgn(P_dn); either may be NULL.  hqmc_set_perm overwrites them (each row
 * must be a permutation of 0..Nsig-1; the sign follows from the parities).
 * Errors: HQMC_ERR_ARG, HQMC_ERR_STATE, HQMC_ERR_CUDA. */
int hqmc_get_perm(hqmc_ctx *ctx, int chain, int32_t *perm, int *sign);
int hqmc_set_perm(hqmc_ctx *ctx, int chain, const int32_t *perm);

/* Read the accumulated observables.  out: host array [n_chains] (nullable).
 * Sk, Cr (nullable, host) receive per chain the spin structure factor
 * S(k) = (1/N) sum_{ij} e^{ik(r_i-r_j)} <S^z_i S^z_j> on the N-point grid k = kx + L ky
 * (k_a = 2 pi k_a / L) and C(r) = <S^z_0 S^z_r> at r = rx + L ry, packed over chains.
 * reset != 0 zeroes the accumulators after reading.  Errors: HQMC_ERR_STATE, _CUDA. */
int hqmc_measure(hqmc_ctx *ctx, hqmc_obs *out, double *Sk, double *Cr, int reset);

/* Open-path estimator of the one-body density matrix and the momentum distribution (Sec. 4,
 * "Observables": n_k = (1/N) sum_{i,j,sigma} e^{ik.(r_i - r_j)} <c^dag_{j sigma} c_{i sigma}>).
 * Closed worldlines carry no off-diagonal element, but the FFBS filter of a unit already
 * holds the weights of the open ones: its end message alpha_end(y) sums the unit's paths
 * that end at y instead of at the held end x_e, so alpha_end(x_e + r) / alpha_end(x_e) is
 * the weight of the configuration cut at x_e and displaced there by r, relative to the
 * closed one; over the sampled (closed) ensemble its mean is that ratio of partition sums
 * (reading of this library: the Rao-Blackwellised displacement estimator).  on = 1: every
 * later sweep adds, for the last block of every worldline's unit, sign x alpha_end(x_e + r)
 * / alpha_end(x_e) to a per-chain sum over r = rx + L ry (N values; the sign is the
 * permutation sign with hqmc_set_permutations, else +1).  This costs 2 N FP64 atomics per
 * worldline pair and sweep.  Turning it on or off drops the captured sweep graph and
 * restarts every observable accumulator (as hqmc_measure with reset).
 * Errors: HQMC_ERR_ARG, HQMC_ERR_CUDA. */
int hqmc_set_measure_open(hqmc_ctx *ctx, int on);

/* Read the open-path estimator (hqmc_set_measure_open must be on): per chain, packed over
 * chains, N values each (host arrays, nullable):
 *   nk[k]  n_k = (1/N) sum_r cos(k.r) A(r), k = kx + L ky, k_a = 2 pi k_a / L, spin-summed
 *          (the mean of n_k over k is the density n)
 *   dm[r]  A(r) / N = (1/N) sum_x sum_sigma <c^dag_{x+r} c_x>, r = rx + L ry (dm[0] = n)
 * with A(r) the accumulated sum divided by the sum of signs since the last reset.
 * Errors: HQMC_ERR_STATE (estimator off or no state), HQMC_ERR_CUDA. */
int hqmc_measure_open(hqmc_ctx *ctx, double *nk, double *dm);

/* Checkpoint format of hqmc_log_weight_grad's reverse pass.  The forward pass keeps
 * F_l = W_l . alpha_l only every `stride` slices (0 = ceil(sqrt M)) and the reverse pass
 * recomputes each stride-long segment from its checkpoint.
 *   HQMC_CKPT_BF16  (FP32 context) checkpoints as BF16 with the slice's power-of-two
 *                   exponent; recomputed F carries the BF16 rounding (relative 2^-9)
 *   HQMC_CKPT_FULL  checkpoints in the context's own precision (exact recompute)
 * The FP64 context always keeps FP64 checkpoints.  Errors: HQMC_ERR_ARG. */
#define HQMC_CKPT_BF16 0
#define HQMC_CKPT_FULL 1
int hqmc_set_checkpoint(hqmc_ctx *ctx, int stride, int kind);

/* Log-weight of the current worldlines with every worldline anchored at slice 0 on its
 * current site, and its gradient (the adjoint of the forward filter of Eq. ffbsFwd):
 *   logZ[c]      = sum_{sigma,p} log Z_p                                      (host [n_chains])
 *   dlogZ_dv     = d logZ / d v_{l,sigma}(x), v = log W, i.e. the summed
 *                  forward-backward site marginals, device [2][M][N] per chain packed
 *                  over chains, element type float (FP32 context) or double (FP64)
 *   dlogZ_dt[c]  = d logZ / d t                                              (host [n_chains])
 * v (nullable, device, same type and layout as dlogZ_dv) replaces log W = sigma lambda s.
 * Any output pointer may be NULL; dlogZ_dv is zeroed by the call before accumulation
 * (FP32 atomics: the summation order over worldlines is not fixed).  The reverse pass
 * checkpoints as set by hqmc_set_checkpoint (default: every ceil(sqrt M) slices, BF16 with
 * a per-slice exponent in an FP32 context).  The first call allocates the context's
 * adjoint scratch with cudaMalloc (freed by hqmc_destroy).  Blocks until done.
 * Errors: HQMC_ERR_STATE, HQMC_ERR_NOMEM, HQMC_ERR_CUDA, HQMC_ERR_NUMERIC. */
int hqmc_log_weight_grad(hqmc_ctx *ctx, const void *v, double *logZ, void *dlogZ_dv,
                         double *dlogZ_dt);

/* Shape of chain c: L, M (slices), Nsig (worldlines per spin).  Errors: HQMC_ERR_ARG. */
int hqmc_chain_shape(hqmc_ctx *ctx, int chain, int *L, int *M, int *Nsig);

/* Copy chain c's state to host buffers (each nullable):
 *   s [M][N] int8 (+1/-1; zeros for a U < 0 chain, whose field is read with
 *   hqmc_get_sigma), x [2][Nsig][M] int32 sites, anchor = last anchor slice
 *   (-1 before the first sweep), sweeps = sweeps done.  Errors: HQMC_ERR_STATE, _CUDA. */
int hqmc_get_state(hqmc_ctx *ctx, int chain, int8_t *s, int32_t *x, int *anchor,
                   uint64_t *sweeps);

/* Gaussian field sigma [M][N] (doubles) of a U < 0 chain, to or from host memory; setting
 * it recomputes the chain's slice potentials.  Errors: HQMC_ERR_ARG (null, a U >= 0
 * chain, non-finite values), HQMC_ERR_STATE, HQMC_ERR_CUDA. */
int hqmc_get_sigma(hqmc_ctx *ctx, int chain, double *sigma);
int hqmc_set_sigma(hqmc_ctx *ctx, int chain, const double *sigma);

/* Overwrite chain c's field and worldlines (layouts as in hqmc_get_state; sites must be
 * in [0, N), s in {-1, +1}); sweeps (if non-NULL) sets the sweep counter of the whole
 * context (used for checkpoint/resume: a restored context reproduces the draws).
 * Errors: HQMC_ERR_ARG, HQMC_ERR_STATE, HQMC_ERR_CUDA. */
int hqmc_set_state(hqmc_ctx *ctx, int chain, const int8_t *s, const int32_t *x,
                   const uint64_t *sweeps);

/* Per-phase device timing.  max_sweeps > 0 turns it on: later sweeps launch without
 * a graph and record CUDA events around the FFBS launches (on the streams they run on)
 * and around the Gibbs/measure kernel, for up to max_sweeps sweeps; 0 turns it off.
 * Errors: HQMC_ERR_ARG, HQMC_ERR_CUDA. */
int hqmc_set_profiling(hqmc_ctx *ctx, int max_sweeps);

/* Sum over the recorded sweeps of the FFBS and the Gibbs/measure device times (ms)
 * and the number of sweeps recorded; clears the record.  Errors: HQMC_ERR_STATE, _CUDA. */
int hqmc_profile_read(hqmc_ctx *ctx, double *ffbs_ms, double *slice_ms, int *n_sweeps);

/* FFBS of one chain's worldlines that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running inside another framework's memory pool that forbids
 * untracked device allocations, processes whose device memory is already claimed by a
 * pre-reserved arena, or loops that must not pay an allocation's implicit device
 * synchronisation.  It runs the same forward filter and backward sampler as
 * hqmc_sweep (the FFBS step only: no Gibbs step, no observables) and takes every
 * intermediate from one static device array of 32 MiB built into the library, which
 * every device that loads the library keeps until the process exits.
 *
 *   L, M, Nsig      lattice size (a built size, L <= 32), slices, worldlines per spin
 *   t, U, dtau      model parameters as in hqmc_set_params, but U >= 0 only (the discrete
 *                   Hirsch field; U < 0 is HQMC_ERR_ARG)
 *   seed, sweep     Philox key and sweep index: the call draws what sweep number `sweep`
 *                   of a context chain with this seed draws in its FFBS, provided that
 *                   chain runs the context defaults -- the closed loop (no hqmc_set_block),
 *                   HQMC_CONV_FFT and no permutation ever used; a chain with blocks, the
 *                   stencil or permutations draws differently
 *   s               device, [M][N] int8 field (+1/-1), read only
 *   x               device, [2][Nsig][M] int32 sites, read and overwritten with the new paths
 *   logw            device, [2][Nsig] double, receives the filter log-weights
 *   precision       HQMC_FP32 or HQMC_FP64
 *   stream          cudaStream_t (as void*) the work is ordered on; the call blocks until done
 *
 * The caller owns s, x and logw.  Scratch needed: the fixed part (tables, the packed
 * field, 16-bit worldlines, a [2][M][N] int32 histogram; about 6 B per site-slice plus
 * 4 B per worldline-slice) plus at least one slot of M*N*8 bytes (16 for FP64); a problem
 * that does not fit 32 MiB is rejected with HQMC_ERR_SCRATCH.  Fewer slots than pairs
 * only lowers parallelism.  Every call looks up the array's device address in the current
 * device's context (cudaGetSymbolAddress).  All calls share the one array and each call
 * re-initialises what must start at zero; calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Errors: HQMC_ERR_ARG (null pointers, sizes, U < 0, or s/x values out of range; x and
 * logw are then untouched), HQMC_ERR_UNSUPPORTED, HQMC_ERR_SCRATCH, HQMC_ERR_CUDA,
 * HQMC_ERR_NUMERIC.  HQMC_ERR_NUMERIC (a draw met an all-zero CDF, where the worldline
 * kept its site, or a log-weight met a non-positive amplitude) is reported after the
 * sweep: x and logw then already hold that sweep's outputs. */
int hqmc_ffbs_noalloc(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed,
                      uint64_t sweep, const int8_t *s, int32_t *x, double *logw, int precision,
                      void *stream);

/* Measured FP32 fused multiply-add throughput of GPU `device` in TFLOP/s, written to
 * *tflops (host): the denominator of the FFBS kernels' ALU roofline.  packed = 1 times the
 * packed f32x2 instruction (FFMA2, 4 flops) that the line FFTs use, packed = 0 the scalar
 * FFMA (2 flops).  One wave of CTAs on every SM runs independent FMA chains; the best of
 * five timed launches counts.  Takes a few ms; allocates and frees a small buffer and a
 * stream of its own, and restores the current device.  Errors: HQMC_ERR_ARG (null
 * pointer, packed not 0 or 1), HQMC_ERR_CUDA. */
int hqmc_fp32_peak(int device, int packed, double *tflops);

/* Measured FP64 fused multiply-add throughput of GPU `device` in TFLOP/s (DFMA, 2 flops),
 * written to *tflops (host): the denominator of the plain FP64 form's ALU roofline.  Same
 * loop structure, launch and ownership as hqmc_fp32_peak.  Errors: HQMC_ERR_ARG (null
 * pointer), HQMC_ERR_CUDA. */
int hqmc_fp64_peak(int device, double *tflops);

/* Lattice sizes built into this library: writes up to cap entries, returns the count. */
int hqmc_supported_L(int *out, int cap);

/* Release the context and any memory it allocated itself (not an attached workspace). */
void hqmc_destroy(hqmc_ctx *ctx);

/* Static text for an HQMC_* code. */
const char *hqmc_strerror(int code);

/* Last error message recorded on this context ("" if none); valid until the next call. */
const char *hqmc_last_error_detail(hqmc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HQMC_H */
