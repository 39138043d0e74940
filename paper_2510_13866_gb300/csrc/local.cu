// local.cu -- local link updates of every worldline (Sec. 3.5.1, Eq. Rlocal), read in
// the position basis: slice l of a worldline moves one lattice step e (uniform over +x,
// -x, +y, -y) with its neighbours x_{l-1}, x_{l+1} held, accepted with probability
// min(1, R),
//     R = G(x' - x_{l-1}) W_l(x') G(x_{l+1} - x') / [G(x - x_{l-1}) W_l(x) G(x_{l+1} - x)],
// a handful of table lookups per move.  Slices of one colour (even l; odd l; l = M-1 alone
// when M is odd) are never neighbours in imaginary time, so one launch per colour updates
// all of them at once: one thread per (chain, worldline, slice of the colour).  The
// occupancy histogram and the kinetic link sums of the final paths are fused in.  With a
// permutation P at tau = beta, slice 0 of p follows slice M-1 of P^{-1}(p) and slice M-1
// of p precedes slice 0 of P(p) (other colours when M >= 2).
//
// The permutation update (Sec. 3.5.3) is here too: pair swaps of successors,
// P'(p) = P(q), P'(q) = P(p), accepted with probability min(1, R),
//     R = G(x_0^{P(q)} - x_{M-1}^p) G(x_0^{P(p)} - x_{M-1}^q)
//         / [G(x_0^{P(p)} - x_{M-1}^p) G(x_0^{P(q)} - x_{M-1}^q)],
// over disjoint pairs (2k + r, 2k + 1 + r) mod Nsig with a random rotation r, one thread
// per pair; every accepted swap flips the chain's sign.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace hqmc {

namespace {

constexpr int kLocalThreads = 256;

__host__ __device__ inline int local_color(int M, int l) { return (M % 2 == 1 && l == M - 1) ? 2 : l % 2; }
// slices of colour c
__host__ __device__ inline int local_count(int M, int c) {
    if (M % 2 == 0) return c == 2 ? 0 : M / 2;
    return c == 2 ? 1 : (M - 1) / 2;
}

__device__ __forceinline__ int wrapd(int d, int L) { return d < 0 ? d + L : d; }

// G(b - a) = g(dx) g(dy), FP64
__device__ __forceinline__ double G2(const double *g, int L, int a, int b) {
    return g[wrapd(b % L - a % L, L)] * g[wrapd(b / L - a / L, L)];
}

// W_l(x) of worldline spin sg (Hirsch bit or Gaussian field), FP64
__device__ __forceinline__ double slice_w(const DevState &st, const ChainDev &cd, int sg, int l, int x) {
    const int L = cd.L;
    if (cd.gauss) return exp(cd.gcoup * st.gsig[cd.g_off + (long long)l * cd.N + x]);
    const int ix = x % L, iy = x / L;
    const uint32_t w = st.sbits[cd.s_off + ((long long)l * L + iy) * cd.wpl + (ix >> 5)];
    return ((w >> (ix & 31)) & 1u) ? cd.w_plus[sg] : cd.w_minus[sg];
}

// d/dt log G(b - a) from the FP32 link table (as the FFBS kernels)
__device__ __forceinline__ float link_h(const float *h, int L, int a, int b) {
    return h[wrapd(b % L - a % L, L)] + h[wrapd(b / L - a / L, L)];
}

__global__ void __launch_bounds__(kLocalThreads) local_kernel(DevState st, int color) {
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N, M = cd.M, Nsig = cd.Nsig;
    const int cnt = local_count(M, color);
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = u < 2LL * Nsig * cnt;
    float ek = 0.f;
    bool accepted = false;
    if (act) {
        const ChainTab &tb = st.tabs[c];
        const int wl = int(u / cnt), k = int(u % cnt);
        const int l = color == 2 ? M - 1 : 2 * k + color;
        const int sg = wl / Nsig, p = wl - sg * Nsig;
        const int16_t *xspin = st.x + cd.x_off + (long long)sg * Nsig * M;
        int16_t *xp = st.x + cd.x_off + (long long)wl * M;
        const int lm = l == 0 ? M - 1 : l - 1, ln = l + 1 == M ? 0 : l + 1;
        const int *P = st.perm + cd.perm_off + sg * Nsig, *Pinv = P + 2 * Nsig;
        const int xm = l == 0 ? xspin[(long long)Pinv[p] * M + lm] : xp[lm];
        const int xn = l + 1 == M ? xspin[(long long)P[p] * M] : xp[ln];
        const int x = xp[l];
        // uniforms: phase 4, i = worldline, j = 2l (step) and 2l + 1 (acceptance)
        const u64x4 w4 = philox4x64_10((uint64_t)(l >> 1), (uint64_t)wl, 4, *st.sweep, cd.seed, 0);
        const double u0 = u53((l & 1) ? w4.v[2] : w4.v[0]), u1 = u53((l & 1) ? w4.v[3] : w4.v[1]);
        int dir = int(u0 * 4.0);
        if (dir > 3) dir = 3;
        int ix = x % L, iy = x / L;
        if (dir == 0) ix = ix + 1 == L ? 0 : ix + 1;
        else if (dir == 1) ix = ix == 0 ? L - 1 : ix - 1;
        else if (dir == 2) iy = iy + 1 == L ? 0 : iy + 1;
        else iy = iy == 0 ? L - 1 : iy - 1;
        const int xnew = ix + L * iy;
        const double *g = tb.g_d;
        double R;
        if (M == 1) {
            // closed on itself (permutations need M >= 2): the link G(0) stays
            R = slice_w(st, cd, sg, l, xnew) / slice_w(st, cd, sg, l, x);
        } else {
            const double num = G2(g, L, xm, xnew) * slice_w(st, cd, sg, l, xnew) * G2(g, L, xnew, xn);
            const double den = G2(g, L, xm, x) * slice_w(st, cd, sg, l, x) * G2(g, L, x, xn);
            R = num / den;
        }
        accepted = u1 < R;
        const int xf = accepted ? xnew : x;
        if (accepted) xp[l] = int16_t(xf);
        atomicAdd(st.hist + cd.h_off + ((long long)sg * M + l) * N + xf, 1);
        // kinetic links whose other end is already final (a lower colour); M = 1: the self link
        const float *h = tb.h_f;
        if (M == 1) {
            ek = link_h(h, L, xf, xf);
        } else {
            if (local_color(M, lm) < color) ek += link_h(h, L, xm, xf);
            if (local_color(M, ln) < color) ek += link_h(h, L, xf, xn);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ek += __shfl_xor_sync(0xffffffffu, ek, o);
    const unsigned nacc = __popc(__ballot_sync(0xffffffffu, accepted));
    if ((threadIdx.x & 31) == 0) {
        if (ek != 0.f) atomicAdd(&st.meas[c].link_sum, double(ek) * chain_sign(st, c));
        if (nacc) atomicAdd(&st.meas[c].local_accepted, (unsigned long long)nacc);
    }
}

__global__ void __launch_bounds__(kLocalThreads) perm_kernel(DevState st) {
    const int c = blockIdx.y, sg = blockIdx.z;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, M = cd.M, Nsig = cd.Nsig, npr = Nsig / 2;
    const uint64_t sweep = *st.sweep;
    // pairing rotation (phase 5, i = sigma, j = 0)
    int r = int(u53(philox4x64_10(0, (uint64_t)sg, 5, sweep, cd.seed, 0).v[0]) * Nsig);
    if (r >= Nsig) r = Nsig - 1;
    int *P = st.perm + cd.perm_off + sg * Nsig, *Pinv = P + 2 * Nsig;
    const int16_t *X = st.x + cd.x_off + (long long)sg * Nsig * M;
    const double *g = st.tabs[c].g_d;
    unsigned cnt = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npr; k += gridDim.x * blockDim.x) {
        int p = 2 * k + r, q = 2 * k + 1 + r;
        if (p >= Nsig) p -= Nsig;
        if (q >= Nsig) q -= Nsig;
        const int Pp = P[p], Pq = P[q];
        const int xlp = X[(long long)p * M + M - 1], xlq = X[(long long)q * M + M - 1];
        const int a0 = X[(long long)Pp * M], b0 = X[(long long)Pq * M];
        const double R = (G2(g, L, xlp, b0) * G2(g, L, xlq, a0)) / (G2(g, L, xlp, a0) * G2(g, L, xlq, b0));
        // pair k: phase 5, i = sigma, j = 1 + k
        const u64x4 w4 = philox4x64_10((uint64_t)((1 + k) >> 2), (uint64_t)sg, 5, sweep, cd.seed, 0);
        const int wsel = (1 + k) & 3;
        const double u = u53(wsel == 0 ? w4.v[0] : wsel == 1 ? w4.v[1] : wsel == 2 ? w4.v[2] : w4.v[3]);
        if (u < R) {
            P[p] = Pq;
            P[q] = Pp;
            Pinv[Pq] = p;
            Pinv[Pp] = q;
            ++cnt;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) {
        atomicAdd(&st.meas[c].perm_accepted, (unsigned long long)cnt);
        if (cnt & 1u) atomicXor(&st.parity[c], 1u);
    }
}

}  // namespace

cudaError_t launch_perm(const DevState &st, int nchains, int max_pairs, cudaStream_t stream) {
    if (max_pairs <= 0) return cudaSuccess;
    const dim3 grid(std::min((max_pairs + kLocalThreads - 1) / kLocalThreads, 64), nchains, 2);
    perm_kernel<<<grid, kLocalThreads, 0, stream>>>(st);
    return cudaGetLastError();
}

int local_max_units(int M, int Nsig) {
    int m = 0;
    for (int c = 0; c < 3; ++c) m = std::max(m, 2 * Nsig * local_count(M, c));
    return m;
}

cudaError_t launch_local(const DevState &st, int nchains, int max_units, int color, cudaStream_t stream) {
    if (max_units <= 0) return cudaSuccess;
    const dim3 grid((max_units + kLocalThreads - 1) / kLocalThreads, nchains);
    local_kernel<<<grid, kLocalThreads, 0, stream>>>(st, color);
    return cudaGetLastError();
}

}  // namespace hqmc
