// ffbs.cuh -- forward-filtering backward-sampling of worldline pairs (Sec. 3.5.2).
//
// A group of L lanes (L <= 32) owns one pair of same-spin worldlines of one chain;
// the two are the real and imaginary parts of one complex L x L array, since the
// propagator G and the slice potential W are real (they never mix the parts).
// Each lane holds one lattice line in registers.  One slice of the forward filter
//     alpha_{l+1} = G * (W_l . alpha_l)            (Eq. ffbsFwd, position basis)
// is a line convolution along the in-register direction (FFT, multiply by the 1D
// kernel g^, inverse FFT), one transpose through shared memory, and the same along
// the other direction: G = g (x) g is separable, so the layout simply alternates
// between slices and only one transpose per slice is needed.  The message is
// renormalised by an exact power of two after every slice; the exponents are summed
// as integers, so the running log-normaliser is exact and log Z is formed in FP64.
// f_l = W_l . alpha_l is written to a per-group scratch slot (column-major), and the
// backward pass reads it back slice by slice to draw
//     x_l ~ max(f_l(y), 0) G(x_{l+1} - y)
// by the row-major inverse CDF with a Philox uniform, fusing the occupancy histogram
// and the kinetic-energy link sum.
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace hqmc {

template <int L>
struct FfbsGeo {
    static_assert(L >= 2 && L <= 32, "register-line FFBS covers L <= 32");
    static constexpr int GW = (L <= 4) ? 4 : (L <= 8) ? 8 : (L <= 16) ? 16 : 32;  // lanes per group
    static constexpr int GPW = 32 / GW;                                          // groups per warp
    static constexpr int BUF = L * (L + 1);  // transpose buffer (padded rows), complex elements
};

// comparison value for "u*S < C(y)" when C is held in T: round u*S down to T,
// so that  t < C  <=>  rd(t) < C  for every C representable in T.
template <typename T>
__device__ __forceinline__ T cmp_value(double t);
template <>
__device__ __forceinline__ float cmp_value<float>(double t) { return __double2float_rd(t); }
template <>
__device__ __forceinline__ double cmp_value<double>(double t) { return t; }

template <typename T>
__device__ __forceinline__ const T *tab_ghat(const ChainTab &tb);
template <>
__device__ __forceinline__ const float *tab_ghat<float>(const ChainTab &tb) { return tb.ghat_f; }
template <>
__device__ __forceinline__ const double *tab_ghat<double>(const ChainTab &tb) { return tb.ghat_d; }
template <typename T>
__device__ __forceinline__ const T *tab_g(const ChainTab &tb);
template <>
__device__ __forceinline__ const float *tab_g<float>(const ChainTab &tb) { return tb.g_f; }
template <>
__device__ __forceinline__ const double *tab_g<double>(const ChainTab &tb) { return tb.g_d; }

// pick element r of a register array with a runtime index (no local-memory spill)
template <int L, typename T>
__device__ __forceinline__ cplx<T> reg_select(const cplx<T> (&v)[L], int r) {
    cplx<T> o = v[0];
#pragma unroll
    for (int k = 1; k < L; ++k)
        if (k == r) o = v[k];
    return o;
}

template <typename T, int L>
__global__ void ffbs_kernel(DevState st, FfbsLaunch fl) {
    using G = FfbsGeo<L>;
    constexpr int N = L * L;
    constexpr int GW = G::GW;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GW;  // lane within the group = line index
    const int gw = lane / GW;  // group within the warp
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (gw * GW));
    const bool active = gl < L;
    const int wpc = blockDim.x >> 5;
    cplx<T> *buf = reinterpret_cast<cplx<T> *>(smem_raw) + (warp * G::GPW + gw) * G::BUF;
    const long long gid = ((long long)blockIdx.x * wpc + warp) * G::GPW + gw;
    const long long ngroups = (long long)gridDim.x * wpc * G::GPW;
    cplx<T> *slot = reinterpret_cast<cplx<T> *>(fl.scratch) + gid * fl.slot_elems;
    const uint64_t sweep = *st.sweep;

    for (long long q = gid; q < fl.total_pairs; q += ngroups) {
        // ---- locate the pair: chain, spin, worldlines ----
        int lo = 0, hi = fl.nclass - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (fl.class_pair_off[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        const int c = fl.class_chains[lo];
        const ChainDev &cd = st.chains[c];
        const ChainTab &tb = st.tabs[c];
        const int M = cd.M, Nsig = cd.Nsig;
        const int rr = int(q - fl.class_pair_off[lo]);
        const int sg = rr / cd.npair, kp = rr % cd.npair;
        const int p0 = 2 * kp, p1 = 2 * kp + 1;
        const bool has1 = p1 < Nsig;
        const uint64_t wl0 = (uint64_t)sg * Nsig + p0, wl1 = (uint64_t)sg * Nsig + p1;
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * cd.wpl;
        int16_t *xp0 = st.x + cd.x_off + (long long)wl0 * M;
        int16_t *xp1 = st.x + cd.x_off + (long long)wl1 * M;

        // 1D kernel in k-space (already divided by L), k = 0..L/2
        T gh[L / 2 + 1];
        {
            const T *src = tab_ghat<T>(tb);
#pragma unroll
            for (int k = 0; k <= L / 2; ++k) gh[k] = src[k];
        }

        // ---- anchor slice (phase 2) ----
        const u64x4 ua = philox4x64_10(0, 0, 2, sweep, cd.seed, 0);
        int a = int(u53(ua.v[0]) * M);
        if (a >= M) a = M - 1;
        if (rr == 0 && gl == 0) st.anchor[c] = a;
        const int xa0 = xp0[a];
        const int xa1 = has1 ? int(xp1[a]) : xa0;  // a missing partner shadows worldline 0
        const int ax0 = xa0 % L, ay0 = xa0 / L, ax1 = xa1 % L, ay1 = xa1 / L;

        // ---- forward filter ----
        cplx<T> v[L];
        {
            // f_a = W_a(x_a) delta_{x_a}, layout R: lane = iy, register = ix
            const uint32_t w = active ? srow[((long long)a * L + gl) * cd.wpl] : 0u;
#pragma unroll
            for (int r = 0; r < L; ++r) {
                const T wv = ((w >> r) & 1u) ? wp : wm;
                v[r].x = (gl == ay0 && r == ax0) ? wv : T(0);
                v[r].y = (gl == ay1 && r == ax1) ? wv : T(0);
            }
        }
        int esum0 = 0, esum1 = 0;
        T fin0 = T(0), fin1 = T(0);
        int l = a;
        for (int i = 0; i < M; ++i) {
            const bool layC = (i & 1) != 0;  // layout of f_l: R (lane = iy) or C (lane = ix)
            if (i >= 1 && active) {
                cplx<T> *dst = slot + (long long)i * N;
                if (!layC) {
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[r * L + gl] = v[r];
                } else {
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[gl * L + r] = v[r];
                }
            }
            conv_line<L, T>(v, gh);
            __syncwarp(gmask);
            if (active) {
#pragma unroll
                for (int r = 0; r < L; ++r) buf[r * (L + 1) + gl] = v[r];
            }
            __syncwarp(gmask);
            if (active) {
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = buf[gl * (L + 1) + r];
            }
            conv_line<L, T>(v, gh);
            // v = alpha_{l+1} (scale 2^{-esum}) in the other layout
            T s0 = T(0), s1 = T(0);
            if (active) {
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    s0 += v[r].x;
                    s1 += v[r].y;
                }
            }
            s0 = group_sum<GW>(s0, gmask);
            s1 = group_sum<GW>(s1, gmask);
            const int l1 = (l + 1 == M) ? 0 : l + 1;
            if (i < M - 1) {
                int e0 = 0, e1 = 0;
                if (s0 > T(0) && s0 < T(1e30)) e0 = fbits<T>::exponent(s0);
                else if (gl == 0) atomicOr(st.status, kStatusDegenerate);
                if (s1 > T(0) && s1 < T(1e30)) e1 = fbits<T>::exponent(s1);
                esum0 += e0;
                esum1 += e1;
                const T sc0 = fbits<T>::pow2(-e0), sc1 = fbits<T>::pow2(-e1);
                const T a0 = wp * sc0, b0 = wm * sc0, a1 = wp * sc1, b1 = wm * sc1;
                // new layout is C (lane = ix) when i is even
                const uint32_t *wsrc = layC ? srow : scol;
                const uint32_t w = active ? wsrc[((long long)l1 * L + gl) * cd.wpl] : 0u;
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    const bool up = (w >> r) & 1u;
                    v[r].x *= up ? a0 : b0;
                    v[r].y *= up ? a1 : b1;
                }
            } else {
                // alpha_M(x_a): final layout is C if M is odd
                const bool finC = (M & 1) != 0;
                const int own0 = finC ? ax0 : ay0, reg0 = finC ? ay0 : ax0;
                const int own1 = finC ? ax1 : ay1, reg1 = finC ? ay1 : ax1;
                const T c0 = reg_select<L, T>(v, reg0).x;
                const T c1 = reg_select<L, T>(v, reg1).y;
                fin0 = __shfl_sync(gmask, c0, own0, GW);
                fin1 = __shfl_sync(gmask, c1, own1, GW);
            }
            l = l1;
        }
        if (gl == 0) {
            const double ln2 = 0.69314718055994530942;
            const double lz0 = double(esum0) * ln2 + log(double(fin0));
            st.logw[cd.logw_off + wl0] = lz0;
            if (!(fin0 > T(0))) atomicOr(st.status, kStatusNonPositive);
            if (has1) {
                st.logw[cd.logw_off + wl1] = double(esum1) * ln2 + log(double(fin1));
                if (!(fin1 > T(0))) atomicOr(st.status, kStatusNonPositive);
            }
        }

        // ---- backward sampling ----
        // doubled real-space table g2[j] = g(j mod L), j in [0, 2L), in this group's buffer
        __syncwarp(gmask);
        T *g2 = reinterpret_cast<T *>(buf);
        {
            const T *src = tab_g<T>(tb);
            for (int j = gl; j < 2 * L; j += GW) g2[j] = src[j < L ? j : j - L];
        }
        __syncwarp(gmask);
        const float *hl = tb.h_f;
        int cur0 = xa0, cur1 = xa1;
        float ek0 = 0.f, ek1 = 0.f;
        int *hist_s = st.hist + cd.h_off + (long long)sg * M * N;
        if (gl == 0) {
            atomicAdd(hist_s + (long long)a * N + xa0, 1);
            if (has1) atomicAdd(hist_s + (long long)a * N + xa1, 1);
        }
        int cached = -1;
        uint64_t words[4] = {0, 0, 0, 0};
        for (int i = M - 1; i >= 1; --i) {
            int lb = a + i;
            if (lb >= M) lb -= M;
            // uniforms of this slice for both worldlines (lanes 0 and 1 compute, then share)
            const int grp = lb >> 2;
            if (grp != cached) {
                const u64x4 w4 = philox4x64_10((uint64_t)grp, (gl & 1) ? wl1 : wl0, 0, sweep, cd.seed, 0);
#pragma unroll
                for (int k = 0; k < 4; ++k) words[k] = w4.v[k];
                cached = grp;
            }
            uint64_t myw = words[0];
#pragma unroll
            for (int k = 1; k < 4; ++k)
                if ((lb & 3) == k) myw = words[k];
            const double u0 = u53(__shfl_sync(gmask, myw, 0, GW));
            const double u1 = u53(__shfl_sync(gmask, myw, 1, GW));

            // f_l row gl (lane = iy), p(y) = max(f, 0) G(x_{l+1} - y), in-lane prefix
            const cplx<T> *srcf = slot + (long long)i * N;
            const int cx0 = cur0 % L, cy0 = cur0 / L, cx1 = cur1 % L, cy1 = cur1 / L;
            T rt0 = T(0), rt1 = T(0);
            if (active) {
                const T gy0 = g2[gl - cy0 + L], gy1 = g2[gl - cy1 + L];
#pragma unroll
                for (int ix = 0; ix < L; ++ix) {
                    const cplx<T> f = srcf[ix * L + gl];
                    const T q0 = (f.x > T(0) ? f.x : T(0)) * (gy0 * g2[ix - cx0 + L]);
                    const T q1 = (f.y > T(0) ? f.y : T(0)) * (gy1 * g2[ix - cx1 + L]);
                    rt0 += q0;
                    rt1 += q1;
                    v[ix].x = rt0;  // inclusive in-row prefix
                    v[ix].y = rt1;
                }
            }
            // inclusive scan of row totals over the group's lanes
            T in0 = rt0, in1 = rt1;
#pragma unroll
            for (int o = 1; o < GW; o <<= 1) {
                const T t0 = __shfl_up_sync(gmask, in0, o, GW);
                const T t1 = __shfl_up_sync(gmask, in1, o, GW);
                if (gl >= o) {
                    in0 += t0;
                    in1 += t1;
                }
            }
            T ex0 = __shfl_up_sync(gmask, in0, 1, GW), ex1 = __shfl_up_sync(gmask, in1, 1, GW);
            if (gl == 0) {
                ex0 = T(0);
                ex1 = T(0);
            }
            const T S0 = __shfl_sync(gmask, in0, L - 1, GW);
            const T S1 = __shfl_sync(gmask, in1, L - 1, GW);
            const T t0 = cmp_value<T>(u0 * double(S0));
            const T t1 = cmp_value<T>(u1 * double(S1));
            // first site of this row with t < ex + prefix and a positive increment
            int cand0 = -1, last0 = -1, cand1 = -1, last1 = -1;
            if (active) {
                T pv0 = T(0), pv1 = T(0);
#pragma unroll
                for (int ix = 0; ix < L; ++ix) {
                    const bool inc0 = v[ix].x > pv0, inc1 = v[ix].y > pv1;
                    if (inc0) {
                        last0 = ix;
                        if (cand0 < 0 && t0 < ex0 + v[ix].x) cand0 = ix;
                    }
                    if (inc1) {
                        last1 = ix;
                        if (cand1 < 0 && t1 < ex1 + v[ix].y) cand1 = ix;
                    }
                    pv0 = v[ix].x;
                    pv1 = v[ix].y;
                }
            }
            int nxt0, nxt1;
            {
                const unsigned b0 = __ballot_sync(gmask, cand0 >= 0) & gmask;
                const unsigned b1 = __ballot_sync(gmask, cand1 >= 0) & gmask;
                const unsigned f0 = __ballot_sync(gmask, last0 >= 0) & gmask;
                const unsigned f1 = __ballot_sync(gmask, last1 >= 0) & gmask;
                const int base = gw * GW;
                int row0, row1, col0, col1;
                if (b0) {
                    row0 = __ffs(b0) - 1 - base;
                    col0 = __shfl_sync(gmask, cand0, row0, GW);
                } else {
                    row0 = f0 ? 31 - __clz(f0) - base : -1;
                    col0 = row0 >= 0 ? __shfl_sync(gmask, last0, row0 < 0 ? 0 : row0, GW) : -1;
                }
                if (b1) {
                    row1 = __ffs(b1) - 1 - base;
                    col1 = __shfl_sync(gmask, cand1, row1, GW);
                } else {
                    row1 = f1 ? 31 - __clz(f1) - base : -1;
                    col1 = row1 >= 0 ? __shfl_sync(gmask, last1, row1 < 0 ? 0 : row1, GW) : -1;
                }
                if (row0 < 0 || !(S0 > T(0))) {
                    nxt0 = cur0;  // all-zero CDF: stay and report
                    if (gl == 0) atomicOr(st.status, kStatusDegenerate);
                } else {
                    nxt0 = col0 + L * row0;
                }
                if (row1 < 0 || !(S1 > T(0))) {
                    nxt1 = cur1;
                    if (gl == 0 && has1) atomicOr(st.status, kStatusDegenerate);
                } else {
                    nxt1 = col1 + L * row1;
                }
            }
            if (gl == 0) {
                // link x_l -> x_{l+1}
                ek0 += hl[(cx0 - nxt0 % L + L) % L] + hl[(cy0 - nxt0 / L + L) % L];
                xp0[lb] = int16_t(nxt0);
                atomicAdd(hist_s + (long long)lb * N + nxt0, 1);
                if (has1) {
                    ek1 += hl[(cx1 - nxt1 % L + L) % L] + hl[(cy1 - nxt1 / L + L) % L];
                    xp1[lb] = int16_t(nxt1);
                    atomicAdd(hist_s + (long long)lb * N + nxt1, 1);
                }
            }
            cur0 = nxt0;
            cur1 = nxt1;
        }
        if (gl == 0) {
            // link x_a -> x_{a+1}
            ek0 += hl[(cur0 % L - ax0 + L) % L] + hl[(cur0 / L - ay0 + L) % L];
            if (has1) ek1 += hl[(cur1 % L - ax1 + L) % L] + hl[(cur1 / L - ay1 + L) % L];
            atomicAdd(&st.meas[c].link_sum, double(ek0) + (has1 ? double(ek1) : 0.0));
        }
        __syncwarp(gmask);
    }
}

template <typename T, int L>
size_t ffbs_smem_bytes_t(int warps_per_cta) {
    using G = FfbsGeo<L>;
    return size_t(warps_per_cta) * G::GPW * G::BUF * sizeof(cplx<T>);
}

}  // namespace hqmc
