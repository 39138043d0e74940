// internal.h -- device-side data layout shared by the host runtime and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace hqmc {

constexpr int kMaxL = 128;
constexpr int kPTab = 64;  // P(s=+1 | m) tabulated for |m| <= kPTab, computed beyond

// Per-chain tables, computed on the host in FP64 at set_params.
struct ChainTab {
    double ghat_d[kMaxL];  // e^{2 t dtau cos(2 pi k / L)} / L          (1D kernel in k-space)
    double g_d[kMaxL];     // g(d) = <x+d| e^{dtau t A} |x> in 1D        (real-space kernel)
    double h_d[kMaxL];     // d/dt log g(d)
    float ghat_f[kMaxL];
    float g_f[kMaxL];
    float h_f[kMaxL];
    double dghat_d[kMaxL]; // d/dt ghat(k)
    float dghat_f[kMaxL];
    // line-convolution constants of the half-length real FFT (even L): alpha_k, beta_k
    // interleaved for k = 0..L/2-1; odd L: ghat(k) for k = 0..L-1
    double mix_d[kMaxL];
    float mix_f[kMaxL];
    double mixd_d[kMaxL];  // the same for the kernel d g / dt (adjoint)
    float mixd_f[kMaxL];
    double pplus[2 * kPTab + 1];  // 1 / (1 + e^{-2 lambda m}), m = -kPTab..kPTab
};

// Per-chain shape, parameters and offsets into the context's device arrays.
struct ChainDev {
    int L, N, M, Nsig;
    int npair;  // pairs per spin = ceil(Nsig / 2)
    int wpl;    // 32-bit words per lattice line of the bit-packed field
    uint64_t seed;
    double lam;       // Hirsch lambda
    double w_plus[2]; // W for s = +1, spin up / down: e^{+lambda}, e^{-lambda}
    double w_minus[2];
    double t, beta;
    int block;          // FFBS block length B (0 or >= M: the closed loop from the anchor)
    long long lwp_off;  // double offset of per-block log-weight partials [2 Nsig][nblk] (nblk > 1)
    long long done_off; // unsigned offset of per-pair finished-block counters [2 npair] (nblk > 1)
    int gauss;          // 1: U < 0, continuous Gaussian field sigma, W = exp(gcoup sigma), both spins
    double gcoup;       // sqrt(|U| dtau)
    long long g_off;    // element offset of sigma [M][N] (doubles); W at 2 g_off: rows [M][L][L]
                        // (iy-major) then columns [M][L][L] (ix-major), context precision
    long long s_off;    // word offset of the field: rows [M][L][wpl] then cols [M][L][wpl]
    long long x_off;    // int16 offset of worldlines [2][Nsig][M]
    long long h_off;    // int32 offset of the occupancy histogram [2][M][N]
    long long logw_off; // double offset of log-weights [2][Nsig]
    long long v_off;    // element offset of [2][M][N] gradient arrays
    long long meas_off; // offset into the measurement arrays (N per chain)
    long long perm_off; // int offset of the permutation P [2][Nsig] then its inverse [2][Nsig]
};

// Per-chain measurement accumulators (device, zeroed at reset).
struct MeasAcc {
    unsigned long long n_sum;   // sum over slices, sites of n_up + n_dn
    unsigned long long d_sum;   // sum n_up n_dn
    unsigned long long m2_sum;  // sum m^2
    unsigned long long samples; // sweeps accumulated
    double link_sum;            // sum over worldlines and links of d/dt log G
    unsigned long long degenerate;   // FFBS draws that met an all-zero CDF (the site was kept)
                                     // and forward slices with a non-finite normaliser
    unsigned long long nonpositive;  // filter amplitudes alpha_M(x_a) <= 0 (log-weight invalid)
    unsigned long long local_accepted;  // accepted local link moves
    long long sign_sum;                 // sum over measured sweeps of sgn(P_up) sgn(P_dn)
    unsigned long long perm_accepted;   // accepted permutation swaps
    unsigned long long inexact;         // filter log-weights whose error estimate exceeds the
                                        // precision's tolerance (logw_err_estimate)
};
// The sums n_sum, d_sum, m2_sum, link_sum and S(k) are weighted by the sweep's sign
// (two's complement in the unsigned counters); with permutations off the sign is +1.

struct DevState {
    const ChainDev *chains;
    const ChainTab *tabs;
    uint32_t *sbits;     // bit-packed fields (bit 1 = s +1)
    int16_t *x;          // worldlines
    int *hist;           // occupancy histogram (zero between sweeps)
    double *logw;        // filter log-weights of the last sweep
    int *anchor;         // per chain
    MeasAcc *meas;       // per chain
    double *sk;          // per chain N: sum of |m^(k)|^2 / N
    unsigned long long *dens;  // per chain N: sum of n_up + n_dn per site (kept for diagnostics)
    unsigned long long *sweep; // device sweep counter
    unsigned *status;    // error bits
    double *gsig;        // Gaussian fields sigma (U < 0 chains)
    void *gw;            // their slice potentials W = exp(a sigma), rows then columns
    int gw_f64;          // W stored as double (FP64 context) or float
    double *logw_part;   // per-block log-weight partials of block FFBS
    double *logw_err;    // error estimates of the log-weights of the last sweep (as logw)
    double *logw_err_part;  // their per-block partials (as logw_part)
    unsigned *blk_done;  // per-pair counters of finished blocks (zero between sweeps)
    int *perm;           // permutations at tau = beta and their inverses (perm_off per chain)
    unsigned *parity;    // per chain: bit 0 = parity of P_up P_dn (sign -1 when set)
    double *open_acc;    // per chain N (nullable: off): sum over sweeps, spins and worldlines of
                         // sign x alpha_end(x_e + r) / alpha_end(x_e) (open-path estimator)
};

// Blocks of the FFBS loop of a chain: length B (0 or >= M: one block of M slices) and count.
__host__ __device__ inline int ffbs_block_len(int block, int M) { return (block > 0 && block < M) ? block : M; }
__host__ __device__ inline int ffbs_nblk(int block, int M) {
    const int B = ffbs_block_len(block, M);
    return (M + B - 1) / B;
}

// device status bits (no kernel of this library waits on a flag, a peer or a barrier it does
// not own, so there is no timeout bit)
enum : unsigned { kStatusDegenerate = 1u, kStatusNonPositive = 2u };

// One launch of the FFBS kernel covers the chains of one lattice size.  Its work units are
// (worldline pair, block) with the blocks of one pair independent given their held ends.
struct FfbsLaunch {
    const int *class_chains;   // chain ids of this class
    const int *class_unit_off; // [nclass + 1] prefix sums of 2 npair nblk
    int nclass;
    int total_units;
    int len_max;               // longest block in the class (scratch slot size, slices)
    void *scratch;             // slots of len_max * L * L complex values
    long long slot_elems;      // elements per group slot (f storage, then len_max maxima)
    unsigned *next_unit;       // work counter: groups take units in order (zeroed per launch)
    int stencil;               // line convolutions by the periodic stencil instead of the FFT
    int general;               // some chain has FFBS blocks B < M, or the context has used
                               // permutations: the general work-unit instantiation runs
    // wide kernel, FP32: f kept only every ckpt_K positions (0: every f streamed), as BF16
    // (ckpt_bf16) or FP32 checkpoints at the start of a worldline's slot; the backward pass
    // recomputes each segment into the buffer at seg_off (elements) of the slot
    int ckpt_K;
    int ckpt_bf16;
    long long seg_off;
    int gauss;                 // some chain of the class has a Gaussian field (U < 0)
};

// One launch of the adjoint kernel covers the chains of one lattice size.
struct GradLaunch {
    const int *class_chains;
    const int *class_pair_off;
    int nclass;
    int total_pairs;
    int K;                     // checkpoint stride (slices)
    int ckpt_bf16;             // 1: checkpoints as BF16 pairs, 0: in the context precision
    void *ckpt;                // per group: [nseg][N] checkpoint elements, then [nseg][2] int exponents
    long long ckpt_bytes;      // bytes per group
    long long ckpt_exp_off;    // byte offset of the exponents within a group's block
    void *seg;                 // per group: [K][N] recomputed F_l (context precision pairs)
    long long seg_elems;       // pair elements per group
    const void *v;             // optional log-potential, [2][M][N] per chain (nullable)
    void *dv;                  // d log Z / d v, same layout (nullable), zeroed by the caller
    double *logz;              // [chain], zeroed by the caller
    double *dt;                // [chain], zeroed by the caller
    unsigned *next_pair;       // work counter, zeroed by the caller
};

// Launchers (defined in the per-precision translation units).
cudaError_t launch_ffbs(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid,
                        int warps_per_cta, cudaStream_t stream);
int ffbs_groups_per_warp(int L);
size_t ffbs_smem_bytes(int L, bool fp64, int warps_per_cta);
cudaError_t ffbs_occupancy(int L, bool fp64, int warps_per_cta, int *blocks_per_sm);
bool ffbs_supported(int L);

cudaError_t launch_init_state(const DevState &st, int nchains, cudaStream_t stream);
cudaError_t launch_slice(const DevState &st, int nchains, int max_M, int max_L, int slices_per_cta,
                         bool measure, cudaStream_t stream);
cudaError_t configure_slice(int max_L, int S);
int slice_group(int max_L, int requested, long long work_slices, int num_sms);
void host_chain_table(int L, double t, double U, double dtau, ChainTab &tb, double *lam);
cudaError_t launch_advance(const DevState &st, cudaStream_t stream);
// local link updates: the largest (worldline, slice) count of one colour of a chain, and
// one launch over every chain for one colour (0, 1, 2)
int local_max_units(int M, int Nsig);
cudaError_t launch_local(const DevState &st, int nchains, int max_units, int color, cudaStream_t stream);
// one permutation update (pair swaps at tau = beta) of every chain and spin
cudaError_t launch_perm(const DevState &st, int nchains, int max_pairs, cudaStream_t stream);

__device__ __forceinline__ int chain_sign(const DevState &st, int c) { return (st.parity[c] & 1u) ? -1 : 1; }
cudaError_t launch_gauss_w(const DevState &st, int chain, int M, int N, cudaStream_t stream);
// observables read-out: S(k) and C(r) of every chain; tmp holds 2 N doubles per chain
cudaError_t launch_readout(const DevState &st, int nchains, int max_N, double *cr_out,
                           double *sk_out, double *tmp, cudaStream_t stream);
// n_k and the one-body density matrix of every chain from the open-path sums
cudaError_t launch_readout_open(const DevState &st, int nchains, int max_N, double *nk_out,
                                double *dm_out, double *tmp, cudaStream_t stream);

}  // namespace hqmc
