// ffbs.cuh -- forward-filtering backward-sampling of worldline pairs (Sec. 3.5.2).
//
// A group of GW >= L lanes owns one pair of same-spin worldlines of one chain; the two
// travel together as the .x/.y components of a two-worldline vector (FP32: one packed
// f32x2 instruction per operation on the pair).  Each lane holds one lattice line in
// registers.  One slice of the forward filter
//     alpha_{l+1} = G * (W_l . alpha_l)            (Eq. ffbsFwd, position basis)
// is a line convolution along the in-register direction, one transpose through shared
// memory, and the same along the other direction: G = g (x) g is separable, so the
// layout simply alternates between slices and one transpose per slice suffices.  A line
// convolution of the real lines is two half-length complex FFTs with a pairwise
// spectral mix between them (conv_line in device_common.cuh).  The message is
// renormalised by an exact power of two after every slice; the exponents are summed as
// integers, so the running log-normaliser is exact and log Z is formed in FP64.
//
// f_l = W_l . alpha_l is streamed to a per-group scratch slot with coalesced 16-byte
// stores.  The backward pass prefetches each slice into shared memory with asynchronous
// copies while the previous slice is being sampled, and draws
//     x_l ~ max(f_l(y), 0) G(x_{l+1} - y)
// by the row-major inverse CDF with a Philox uniform, fusing the occupancy histogram
// and the kinetic-energy link sum.
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace hqmc {

template <typename T, int L>
struct FfbsGeo {
    static_assert(L >= 2 && L <= 32, "register-line FFBS covers L <= 32");
    using V = vec2_t<T>;
    static constexpr int GW = (L <= 4) ? 4 : (L <= 8) ? 8 : (L <= 16) ? 16 : 32;  // lanes per group
    static constexpr int GPW = 32 / GW;                                          // groups per warp
    // elements per 16-byte chunk of the f slot (odd L in FP32: 8-byte chunks of one element)
    static constexpr int CH = (sizeof(T) == 4 && L % 2 == 0) ? 2 : 1;
    static constexpr int CHB = CH * int(sizeof(V));                                // chunk bytes
    static constexpr int LP = L + CH;                                              // transpose pitch
    static constexpr size_t XBUF = size_t(L) * LP * sizeof(V);
    static constexpr size_t a16(size_t v) { return (v + 15) & ~size_t(15); }
    static constexpr size_t MIXB = a16(size_t(L) * sizeof(V));
    static constexpr size_t G2B = a16(size_t(2 * L) * sizeof(T));
    static constexpr size_t WXB = a16(size_t(L) * sizeof(V));
    static constexpr size_t RBB = a16(size_t(2 * L) * sizeof(V));  // crossing rows of both worldlines
    static constexpr size_t METAB = 32;  // the work unit's block bookkeeping
    static constexpr size_t HLB = a16(size_t(L) * sizeof(float));  // link table d/dt log g
    static constexpr size_t GROUP_BYTES = XBUF + MIXB + G2B + WXB + RBB + METAB + HLB;
};

// Target u*S of an inverse-CDF draw from the Philox word w, in the CDF's precision.
// FP64: u = (w >> 11) 2^-53 and t = u*S.  FP32: u truncated to its leading 24 fraction
// bits, u24 = (w >> 40) 2^-24 (exact in FP32, |u - u24| < 2^-24), and t = u24*S rounded
// down, so no FP64 instruction enters the per-slice loop; the perturbation of u is far
// below the draw tolerance of the FP32 path.
template <typename T>
__device__ __forceinline__ T draw_target(uint64_t w, T S);
template <>
__device__ __forceinline__ float draw_target<float>(uint64_t w, float S) {
    const float u24 = float(uint32_t(w >> 40)) * 0x1.0p-24f;
    return __fmul_rd(u24, S);
}
template <>
__device__ __forceinline__ double draw_target<double>(uint64_t w, double S) { return u53(w) * S; }

template <typename T>
__device__ __forceinline__ const T *tab_mix(const ChainTab &tb);
template <>
__device__ __forceinline__ const float *tab_mix<float>(const ChainTab &tb) { return tb.mix_f; }
template <>
__device__ __forceinline__ const double *tab_mix<double>(const ChainTab &tb) { return tb.mix_d; }
template <typename T>
__device__ __forceinline__ const T *tab_g(const ChainTab &tb);
template <>
__device__ __forceinline__ const float *tab_g<float>(const ChainTab &tb) { return tb.g_f; }
template <>
__device__ __forceinline__ const double *tab_g<double>(const ChainTab &tb) { return tb.g_d; }

// Slice potential of a Gaussian-field chain (U < 0): W_l(ix, iy) from the row array
// (lines = y, iy-major) or the column array (lines = x, ix-major), context precision.
template <typename T>
__device__ __forceinline__ const T *gauss_line(const DevState &st, const ChainDev &cd, bool cols, int l, int line) {
    return static_cast<const T *>(st.gw) + 2 * cd.g_off + (cols ? (long long)cd.M * cd.N : 0) +
           (long long)l * cd.N + (long long)line * cd.L;
}

// v[r] *= W_l(line, r) (s0, s1): one line of a Gaussian-field chain's slice potential
template <typename T, int L, typename V>
__device__ __forceinline__ void mul_gauss_line(V (&v)[L], const T *w, T s0, T s1) {
    if constexpr (sizeof(T) == 4 && L % 4 == 0) {
#pragma unroll
        for (int j = 0; j < L / 4; ++j) {
            const float4 q = reinterpret_cast<const float4 *>(w)[j];
            v[4 * j] = vmul(v[4 * j], V{q.x * s0, q.x * s1});
            v[4 * j + 1] = vmul(v[4 * j + 1], V{q.y * s0, q.y * s1});
            v[4 * j + 2] = vmul(v[4 * j + 2], V{q.z * s0, q.z * s1});
            v[4 * j + 3] = vmul(v[4 * j + 3], V{q.w * s0, q.w * s1});
        }
    } else {
#pragma unroll
        for (int r = 0; r < L; ++r) v[r] = vmul(v[r], V{w[r] * s0, w[r] * s1});
    }
}

// pick element r of a register array with a runtime index (no local-memory spill)
template <int L, typename V>
__device__ __forceinline__ V reg_select(const V (&v)[L], int r) {
    V o = v[0];
#pragma unroll
    for (int k = 1; k < L; ++k)
        if (k == r) o = v[k];
    return o;
}

template <typename V>
__device__ __forceinline__ V vmax0(V a) {
    return {a.x > 0 ? a.x : decltype(a.x)(0), a.y > 0 ? a.y : decltype(a.y)(0)};
}

// chunk c of an f slot (CH consecutive elements of one writer lane)
template <typename T, int L>
__device__ __forceinline__ void store_chunk(vec2_t<T> *dst, int c, const vec2_t<T> *e) {
    using G = FfbsGeo<T, L>;
    if constexpr (G::CH == 2) {
        reinterpret_cast<float4 *>(dst)[c] = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
    } else {
        dst[c] = e[0];
    }
}

template <typename T, int L>
__device__ __forceinline__ void async_chunk(vec2_t<T> *sdst, int sc, const vec2_t<T> *gsrc, int gc) {
    using G = FfbsGeo<T, L>;
    if constexpr (G::CHB == 16) cp_async16(sdst + size_t(sc) * G::CH, gsrc + size_t(gc) * G::CH);
    else cp_async8(sdst + sc, gsrc + gc);
}

// GAUSS: the class holds Gaussian-field chains (U < 0): their slice potentials are read from
// the W arrays and their log-weight estimate sums the concentration of every position along
// the drawn path; the Hirsch-only instantiation carries none of that code.
// STN: line convolutions by the periodic stencil (stencil_store) instead of the FFT.
// BLK: the general work units -- FFBS blocks B < M and/or a permutation at tau = beta (the
// closed-loop instantiation carries none of that bookkeeping).  With a permutation P the
// unit of worldline p runs from slice a of p to slice a of P(p): its positions at or past
// the wrap (a + offset >= M) are slices of worldline P(p).
template <typename T, int L, bool BLK, bool STN, bool GAUSS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) ffbs_kernel(DevState st, FfbsLaunch fl) {
    using G = FfbsGeo<T, L>;
    using V = vec2_t<T>;
    constexpr int N = L * L;
    constexpr int GW = G::GW, CH = G::CH, LP = G::LP;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GW;  // lane within the group = line index
    const int gw = lane / GW;  // group within the warp
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (gw * GW));
    const bool active = gl < L;
    const int wpc = blockDim.x >> 5;
    unsigned char *gsm = smem_raw + size_t(warp * G::GPW + gw) * G::GROUP_BYTES;
    V *xbuf = reinterpret_cast<V *>(gsm);
    V *mix = reinterpret_cast<V *>(gsm + G::XBUF);
    T *g2 = reinterpret_cast<T *>(gsm + G::XBUF + G::MIXB);
    V *wx = reinterpret_cast<V *>(gsm + G::XBUF + G::MIXB + G::G2B);
    V *rb = reinterpret_cast<V *>(gsm + G::XBUF + G::MIXB + G::G2B + G::WXB);  // [2][L]
    // bookkeeping of the current unit (b, nblk, pair, l0, l0+len, first position past the
    // wrap, successors of both worldlines), parked in shared memory across the forward loop
    // instead of in registers
    volatile int *meta = reinterpret_cast<volatile int *>(gsm + G::XBUF + G::MIXB + G::G2B + G::WXB + G::RBB);
    float *hsm = reinterpret_cast<float *>(gsm + G::XBUF + G::MIXB + G::G2B + G::WXB + G::RBB + G::METAB);
    const long long gid = ((long long)blockIdx.x * wpc + warp) * G::GPW + gw;
    const long long ngroups = (long long)gridDim.x * wpc * G::GPW;
    V *slot = reinterpret_cast<V *>(fl.scratch) + gid * fl.slot_elems;
    const uint64_t sweep = *st.sweep;

    // work units (pair, block) are taken from a work counter (classes list their chains by
    // decreasing block length, so the longest units go first and the tail is short)
    (void)ngroups;
    for (;;) {
        unsigned qn = 0;
        if (gl == 0) qn = atomicAdd(fl.next_unit, 1u);
        const long long q = (long long)__shfl_sync(gmask, qn, 0, GW);
        if (q >= fl.total_units) break;
        // ---- locate the pair: chain, spin, worldlines ----
        int lo = 0, hi = fl.nclass - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (fl.class_unit_off[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        const int c = fl.class_chains[lo];
        const ChainDev &cd = st.chains[c];
        const ChainTab &tb = st.tabs[c];
        const int M = cd.M, Nsig = cd.Nsig;
        // unit = (pair, block): the blocks of a pair are independent given their held ends
        const int ru = int(q - fl.class_unit_off[lo]);
        int sg, kp, len, a_keep = 0;
        {
            const int Bk = BLK ? ffbs_block_len(cd.block, M) : M, nblk = BLK ? ffbs_nblk(cd.block, M) : 1;
            const int rr = BLK ? ru / nblk : ru, b = BLK ? ru - rr * nblk : 0;
            sg = rr / cd.npair;
            kp = rr % cd.npair;
            // block b of the blocks of Bk slices from the anchor a, a+Bk, a+2Bk, ... (the
            // last may be shorter), resampled with its two end sites held; the log-weight
            // is the sum of the blocks'.  Bk = M is the closed loop with both ends at x_a.
            const u64x4 ua = philox4x64_10(0, 0, 2, sweep, cd.seed, 0);  // anchor (phase 2)
            int a = int(u53(ua.v[0]) * M);
            if (a >= M) a = M - 1;
            if (ru == 0 && gl == 0) st.anchor[c] = a;
            int l0 = a + b * Bk;
            if (l0 >= M) l0 -= M;
            len = (b + 1) * Bk <= M ? Bk : M - b * Bk;
            const int le = (l0 + len >= M) ? l0 + len - M : l0 + len;
            if constexpr (BLK) {
                __syncwarp(gmask);
                if (gl == 0) {
                    const int *P = st.perm + cd.perm_off + sg * Nsig;
                    meta[0] = b;
                    meta[1] = nblk;
                    meta[2] = rr;
                    meta[3] = l0;
                    meta[4] = le;
                    meta[5] = M - a - b * Bk;  // block positions >= this lie past the wrap
                    meta[6] = P[2 * kp];
                    meta[7] = (2 * kp + 1 < Nsig) ? P[2 * kp + 1] : P[2 * kp];
                }
            } else {
                a_keep = a;  // the closed loop starts and ends at the anchor
                (void)le;
            }
        }
        auto first_slice = [&]() { if constexpr (BLK) return int(meta[3]); else return a_keep; };
        auto end_slice = [&]() { if constexpr (BLK) return int(meta[4]); else return a_keep; };
        // the sites of both worldlines at block position i (slice l): past the wrap they
        // are the successors' (general units only)
        int16_t *xspin = st.x + cd.x_off + (long long)sg * Nsig * M;
        auto owner0 = [&](int i) -> int16_t * {
            if constexpr (BLK) return xspin + (long long)(i >= meta[5] ? meta[6] : 2 * kp) * M;
            else return xspin + (long long)(2 * kp) * M;
        };
        auto owner1 = [&](int i) -> int16_t * {
            if constexpr (BLK) return xspin + (long long)(i >= meta[5] ? meta[7] : 2 * kp + 1) * M;
            else return xspin + (long long)(2 * kp + 1) * M;
        };
        const int p0 = 2 * kp, p1 = 2 * kp + 1;
        const bool has1 = p1 < Nsig;
        const uint64_t wl0 = (uint64_t)sg * Nsig + p0, wl1 = (uint64_t)sg * Nsig + p1;
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * cd.wpl;

        // line-convolution constants and the doubled real-space kernel g2[j] = g(j mod L)
        __syncwarp(gmask);
        {
            const T *src = tab_mix<T>(tb);
            for (int j = gl; j < L; j += GW) mix[j] = vsplat(src[j]);
            const T *gs = tab_g<T>(tb);
            for (int j = gl; j < 2 * L; j += GW) g2[j] = gs[j < L ? j : j - L];
            for (int j = gl; j < L; j += GW) hsm[j] = tb.h_f[j];
        }
        __syncwarp(gmask);

        // ---- forward filter ----
        __syncwarp(gmask);
        const int l0 = first_slice();
        V v[L];
        {
            // the held end sites are re-read where they are used (short live ranges)
            const int xs0 = owner0(0)[l0];
            const int xs1 = has1 ? int(owner1(0)[l0]) : xs0;  // a missing partner shadows worldline 0
            const int sx0 = xs0 % L, sy0 = xs0 / L, sx1 = xs1 % L, sy1 = xs1 / L;
            // f_{l0} = W_{l0}(x_{l0}) delta_{x_{l0}}, layout R: lane = iy, register = ix
            T wv0, wv1;
            if (GAUSS && cd.gauss) {
                wv0 = gauss_line<T>(st, cd, false, l0, sy0)[sx0];
                wv1 = gauss_line<T>(st, cd, false, l0, sy1)[sx1];
            } else {
                wv0 = ((srow[((long long)l0 * L + sy0) * cd.wpl + (sx0 >> 5)] >> (sx0 & 31)) & 1u) ? wp : wm;
                wv1 = ((srow[((long long)l0 * L + sy1) * cd.wpl + (sx1 >> 5)] >> (sx1 & 31)) & 1u) ? wp : wm;
            }
#pragma unroll
            for (int r = 0; r < L; ++r) {
                v[r].x = (gl == sy0 && r == sx0) ? wv0 : T(0);
                v[r].y = (gl == sy1 && r == sx1) ? wv1 : T(0);
            }
        }
        int esum0 = 0, esum1 = 0;
        T fin0 = T(0), fin1 = T(0);
        T top0 = T(0), top1 = T(0);  // largest value of the final message (kappa = top / fin)
        // Gaussian-field units keep max_y alpha_i(y) of every interior position i (at the
        // scale of the stored f_i) after the unit's f slices, for the backward pass
        V *aux = slot + (long long)fl.len_max * N;
        int l = l0;
        for (int i = 0; i < len; ++i) {
            // the next slice's field bits (Hirsch chains), loaded before this slice's
            // convolutions so that their latency is hidden behind them
            uint32_t wnext = 0u;
            if (!(GAUSS && cd.gauss) && active && i < len - 1) {
                const int ln1 = (l + 1 == M) ? 0 : l + 1;
                wnext = ((i & 1) ? srow : scol)[((long long)ln1 * L + gl) * cd.wpl];
            }
            // f_l of slice i, in the writer's layout: chunk j*L + lane holds registers CH*j..
            if (i >= 1 && active) {
                V *dst = slot + (long long)i * N;
#pragma unroll
                for (int j = 0; j < L / CH; ++j) store_chunk<T, L>(dst, j * L + gl, &v[CH * j]);
            }
            if constexpr (STN) {
                // the lane's own row of the transpose buffer back into registers
                auto read_row = [&]() {
                    const V *src = xbuf + gl * LP;
                    if constexpr (CH == 2) {
#pragma unroll
                        for (int j = 0; j < L / 2; ++j) {
                            const float4 c4 = reinterpret_cast<const float4 *>(src)[j];
                            v[2 * j] = make_float2(c4.x, c4.y);
                            v[2 * j + 1] = make_float2(c4.z, c4.w);
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < L; ++p) v[p] = src[p];
                    }
                };
                // stencil along the register direction, written straight into the transpose
                // (lane p, register r -> lane r, register p) ...
                __syncwarp(gmask);
                if (active) stencil_store<L>(v, g2, xbuf + gl, LP);
                __syncwarp(gmask);
                if (active) {
                    read_row();
                    // ... and along the other direction into the lane's own row of the
                    // transpose buffer (read only by this lane)
                    stencil_store<L>(v, g2, xbuf + gl * LP, 1);
                    read_row();
                }
            } else {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                conv_line<L>(v, mix);
                if (h == 0) {
                    // transpose: lane p, register r  ->  lane r, register p
                    __syncwarp(gmask);
                    if (active) {
#pragma unroll
                        for (int r = 0; r < L; ++r) xbuf[r * LP + gl] = v[r];
                    }
                    __syncwarp(gmask);
                    if (active) {
                        const V *src = xbuf + gl * LP;
                        if constexpr (CH == 2) {
#pragma unroll
                            for (int j = 0; j < L / 2; ++j) {
                                const float4 c4 = reinterpret_cast<const float4 *>(src)[j];
                                v[2 * j] = make_float2(c4.x, c4.y);
                                v[2 * j + 1] = make_float2(c4.z, c4.w);
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < L; ++p) v[p] = src[p];
                        }
                    }
                }
            }
            }
            // v = alpha_{l+1} (scale 2^{-esum}) in the other layout
            V s = vzero(v[0]);
            if (active) {
                // pairwise (tree) sum: short dependency chains
                V part[(L + 1) / 2];
#pragma unroll
                for (int r = 0; r < L / 2; ++r) part[r] = vadd(v[2 * r], v[2 * r + 1]);
                if constexpr (L % 2) part[L / 2] = v[L - 1];
#pragma unroll
                for (int w = 1; w < (L + 1) / 2; w <<= 1)
#pragma unroll
                    for (int r = 0; r + w < (L + 1) / 2; r += 2 * w) part[r] = vadd(part[r], part[r + w]);
                s = part[0];
            }
            T s0 = group_sum<GW>(s.x, gmask);
            T s1 = group_sum<GW>(s.y, gmask);
            const int l1 = (l + 1 == M) ? 0 : l + 1;
            if (i < len - 1) {
                int e0 = 0, e1 = 0;
                if (s0 > T(0) && s0 < T(1e30)) e0 = fbits<T>::exponent(s0);
                else if (gl == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
                if (s1 > T(0) && s1 < T(1e30)) e1 = fbits<T>::exponent(s1);
                esum0 += e0;
                esum1 += e1;
                const T sc0 = fbits<T>::pow2(-e0), sc1 = fbits<T>::pow2(-e1);
                const V A = {wp * sc0, wp * sc1}, B = {wm * sc0, wm * sc1};
                // the new layout is C (lane = ix) when i is even: the field by columns
                if (GAUSS && cd.gauss) {
                    {
                        // v = alpha of position i + 1
                        V mx = vzero(v[0]);
#pragma unroll
                        for (int r = 0; r < L; ++r) {
                            mx.x = v[r].x > mx.x ? v[r].x : mx.x;
                            mx.y = v[r].y > mx.y ? v[r].y : mx.y;
                        }
                        const T m0 = group_max<GW>(mx.x, gmask), m1 = group_max<GW>(mx.y, gmask);
                        if (gl == 0) aux[i + 1] = V{m0 * sc0, m1 * sc1};
                    }
                    if (active) mul_gauss_line<T, L>(v, gauss_line<T>(st, cd, (i & 1) == 0, l1, gl), sc0, sc1);
                } else {
                    const uint32_t w = wnext;
#pragma unroll
                    for (int r = 0; r < L; ++r) v[r] = vmul(v[r], ((w >> r) & 1u) ? A : B);
                }
            } else {
                // alpha_{l0+len}(x_{l0+len}): final layout is C if len is odd
                const bool finC = (len & 1) != 0;
                const int le = end_slice();
                const int xe0 = owner0(len)[le];
                const int xe1 = has1 ? int(owner1(len)[le]) : xe0;
                const int ex0 = xe0 % L, ey0 = xe0 / L, ex1 = xe1 % L, ey1 = xe1 / L;
                const int own0 = finC ? ex0 : ey0, reg0 = finC ? ey0 : ex0;
                const int own1 = finC ? ex1 : ey1, reg1 = finC ? ey1 : ex1;
                const T c0 = reg_select<L>(v, reg0).x;
                const T c1 = reg_select<L>(v, reg1).y;
                fin0 = __shfl_sync(gmask, c0, own0, GW);
                fin1 = __shfl_sync(gmask, c1, own1, GW);
                V mx = vzero(v[0]);
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    mx.x = v[r].x > mx.x ? v[r].x : mx.x;
                    mx.y = v[r].y > mx.y ? v[r].y : mx.y;
                }
                top0 = group_max<GW>(mx.x, gmask);
                top1 = group_max<GW>(mx.y, gmask);
                // open-path estimator (one-body density matrix, for n_k): the last block's end
                // message read at every site, relative to the held end, sign-weighted
                const bool last_blk = BLK ? (int(meta[0]) == int(meta[1]) - 1) : true;
                if (st.open_acc && last_blk && active) {
                    double *acc = st.open_acc + cd.meas_off;
                    const T sgn = T(chain_sign(st, c));
                    const T i0 = fin0 > T(0) ? sgn / fin0 : T(0), i1 = (has1 && fin1 > T(0)) ? sgn / fin1 : T(0);
#pragma unroll
                    for (int r = 0; r < L; ++r) {
                        const int x = finC ? gl : r, y = finC ? r : gl;
                        const int d0 = (x - ex0 + L) % L + L * ((y - ey0 + L) % L);
                        const int d1 = (x - ex1 + L) % L + L * ((y - ey1 + L) % L);
                        if (i0 != T(0)) atomicAdd(acc + d0, double(v[r].x * i0));
                        if (i1 != T(0)) atomicAdd(acc + d1, double(v[r].y * i1));
                    }
                }
            }
            l = l1;
        }
        // the unit's log-weights and their error estimates; Hirsch units book them after the
        // forward pass, Gaussian-field units after the backward pass, which supplies kin
        auto book = [&](double kin0, double kin1) {
            if (gl != 0) return;
            // log-weight of the block; with several blocks, the pair's last finished block
            // sums the partials in block order (the same bits whichever finishes last)
            const double ln2 = 0.69314718055994530942;
            const double part0 = double(esum0) * ln2 + log(double(fin0));
            const double part1 = double(esum1) * ln2 + log(double(fin1));
            if (!(fin0 > T(0))) atomicAdd(&st.meas[c].nonpositive, 1ull);
            if (has1 && !(fin1 > T(0))) atomicAdd(&st.meas[c].nonpositive, 1ull);
            const double inf = __longlong_as_double(0x7ff0000000000000LL);
            // Hirsch units: len x the end concentration; Gaussian units: the conditional means
            // of the concentration over positions 1 .. len-1 given the drawn next sites (kin,
            // from the backward pass; calibration factor in FP64), plus the end's
            const double kap0 = double(top0) / double(fin0), kap1 = double(top1) / double(fin1);
            const double err0 = !(fin0 > T(0)) ? inf
                                : (GAUSS && cd.gauss) ? logw_err_estimate<T>(gauss_sum_factor<T>() * kin0 + kap0, STN ? len : 1, L, STN)
                                           : logw_err_estimate<T>(kap0, len, L, STN);
            const double err1 = !(fin1 > T(0)) ? inf
                                : (GAUSS && cd.gauss) ? logw_err_estimate<T>(gauss_sum_factor<T>() * kin1 + kap1, STN ? len : 1, L, STN)
                                           : logw_err_estimate<T>(kap1, len, L, STN);
            // a log-weight whose estimate exceeds the tolerance is counted (hqmc_obs.n_inexact)
            auto flag = [&](double lwv, double e) {
                if (!(e <= logw_tolerance<T>() * fmax(1.0, fabs(lwv)))) atomicAdd(&st.meas[c].inexact, 1ull);
            };
            double *lw = st.logw + cd.logw_off;
            double *le = st.logw_err + cd.logw_off;
            const int b = BLK ? int(meta[0]) : 0, nblk = BLK ? int(meta[1]) : 1, rr = BLK ? int(meta[2]) : 0;
            if (!BLK || nblk == 1) {
                lw[wl0] = part0;
                le[wl0] = err0;
                flag(part0, err0);
                if (has1) {
                    lw[wl1] = part1;
                    le[wl1] = err1;
                    flag(part1, err1);
                }
            } else {
                double *lp = st.logw_part + cd.lwp_off;
                double *ep = st.logw_err_part + cd.lwp_off;
                lp[wl0 * nblk + b] = part0;
                ep[wl0 * nblk + b] = err0;
                if (has1) {
                    lp[wl1 * nblk + b] = part1;
                    ep[wl1 * nblk + b] = err1;
                }
                __threadfence();
                unsigned *done = st.blk_done + cd.done_off + rr;
                if (atomicAdd(done, 1u) == unsigned(nblk - 1)) {
                    __threadfence();
                    double s0 = 0.0, s1 = 0.0, e0 = 0.0, e1 = 0.0;
                    for (int k = 0; k < nblk; ++k) {
                        s0 += __ldcg(lp + wl0 * nblk + k);
                        e0 += __ldcg(ep + wl0 * nblk + k);
                        if (has1) {
                            s1 += __ldcg(lp + wl1 * nblk + k);
                            e1 += __ldcg(ep + wl1 * nblk + k);
                        }
                    }
                    lw[wl0] = s0;
                    le[wl0] = e0;
                    flag(s0, e0);
                    if (has1) {
                        lw[wl1] = s1;
                        le[wl1] = e1;
                        flag(s1, e1);
                    }
                    *done = 0u;  // ready for the next sweep
                }
            }
        };
        if (!(GAUSS && cd.gauss)) book(0.0, 0.0);

        // ---- backward sampling ----
        // slice i of the slot -> xbuf: R slices (i even) chunk-for-chunk, C slices (i odd)
        // into rows of pitch L+1 chunks so that the row-wise reads below are conflict-free
        auto prefetch = [&](int i) {
            if (active) {
                const V *src = slot + (long long)i * N;
                const int pitch = (i & 1) ? L + 1 : L;
#pragma unroll
                for (int j = 0; j < L / CH; ++j) async_chunk<T, L>(xbuf, j * pitch + gl, src, j * L + gl);
            }
            cp_async_commit();
        };
        __syncwarp(gmask);
        if (len > 1) prefetch(len - 1);
        const float *hl = hsm;  // the link sums read the table from shared memory
        int *hist_s = st.hist + cd.h_off + (long long)sg * M * N;
        float ek0 = 0.f, ek1 = 0.f;
        const int le = end_slice();
        const int xs0 = owner0(0)[l0];
        const int xs1 = has1 ? int(owner1(0)[l0]) : xs0;
        const int sx0 = xs0 % L, sy0 = xs0 / L, sx1 = xs1 % L, sy1 = xs1 / L;
        int cur0 = owner0(len)[le];
        int cur1 = has1 ? int(owner1(len)[le]) : cur0;
        if (gl == 0) {
            atomicAdd(hist_s + (long long)l0 * N + xs0, 1);
            if (has1) atomicAdd(hist_s + (long long)l0 * N + xs1, 1);
        }
        int cached = -1;
        uint64_t wd0 = 0, wd1 = 0, wd2 = 0, wd3 = 0;
        // Gaussian-field units: sum over positions i of E[max_y alpha_i(y) / alpha_i(x_i) | x_{i+1}]
        // = max alpha_i sum_y W_i(y) G(x_{i+1} - y) / S_i, S_i = sum_y f_i(y) G(x_{i+1} - y) the
        // draw's total.  Under the unit's posterior its mean is max alpha_i sum_y beta_i(y) /
        // <alpha_i, beta_i> (beta_i the backward message from the held end): the factor by which
        // a rounding error of the size of max alpha_i at slice i reaches the log-weight.
        T kin0 = T(0), kin1 = T(0);
        for (int i = len - 1; i >= 1; --i) {
            int lb = l0 + i;
            if (lb >= M) lb -= M;
            // row gl of f_l (lane = iy, register = ix)
            cp_async_wait_all();
            __syncwarp(gmask);
            if (active) {
                if ((i & 1) == 0) {
#pragma unroll
                    for (int j = 0; j < L / CH; ++j) {
                        if constexpr (CH == 2) {
                            const float4 c4 = reinterpret_cast<const float4 *>(xbuf)[j * L + gl];
                            v[2 * j] = make_float2(c4.x, c4.y);
                            v[2 * j + 1] = make_float2(c4.z, c4.w);
                        } else {
                            v[j] = xbuf[j * L + gl];
                        }
                    }
                } else {
                    const V *src = xbuf + (gl / CH) * (L + 1) * CH + gl % CH;
#pragma unroll
                    for (int ix = 0; ix < L; ++ix) v[ix] = src[ix * CH];
                }
            }
            __syncwarp(gmask);
            if (i > 1) prefetch(i - 1);

            // uniforms of this slice for both worldlines: one Philox call per lane fills the
            // words of GW/2 groups of four slices at once (lane 2k + w: group k of the block,
            // worldline w), then the slice's two words are shared from their lanes
            constexpr int PG = GW / 2;
            const int grp = lb >> 2, blk = grp / PG;
            if (blk != cached) {
                const u64x4 w4 = philox4x64_10((uint64_t)(blk * PG + (gl >> 1)), (gl & 1) ? wl1 : wl0, 0, sweep,
                                               cd.seed, 0);
                wd0 = w4.v[0];
                wd1 = w4.v[1];
                wd2 = w4.v[2];
                wd3 = w4.v[3];
                cached = blk;
            }
            const int wsel = lb & 3, src = 2 * (grp - blk * PG);
            const uint64_t myw = wsel == 0 ? wd0 : wsel == 1 ? wd1 : wsel == 2 ? wd2 : wd3;
            const uint64_t uw0 = __shfl_sync(gmask, myw, src, GW);
            const uint64_t uw1 = __shfl_sync(gmask, myw, src + 1, GW);

            // p(y) = max(f, 0) g(ix - cx) g(iy - cy): x-weights shared through wx
            const int cx0 = cur0 % L, cy0 = cur0 / L, cx1 = cur1 % L, cy1 = cur1 / L;
            if (active) wx[gl] = V{g2[gl - cx0 + L], g2[gl - cx1 + L]};
            __syncwarp(gmask);
            V gy = vzero(v[0]);
            if (active) gy = V{g2[gl - cy0 + L], g2[gl - cy1 + L]};
            V P = vzero(v[0]);
            if (active) {
#pragma unroll
                for (int ix = 0; ix < L; ++ix) {
                    P = vfma(vmax0(v[ix]), vmul(wx[ix], gy), P);
                    v[ix] = P;  // inclusive in-row prefix
                }
            }
            // inclusive scan of row totals over the group's lanes
            T in0 = P.x, in1 = P.y;
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
            if constexpr (GAUSS) {
                if (cd.gauss) {
                    // sum_y W_i(y) G(x_{i+1} - y) over row gl of W (the same field for both spins)
                    V Q = vzero(v[0]);
                    if (active) {
                        const T *wrow = gauss_line<T>(st, cd, false, lb, gl);
#pragma unroll 4
                        for (int ix = 0; ix < L; ++ix) Q = vfma(vsplat(wrow[ix]), wx[ix], Q);
                        Q = vmul(Q, gy);
                    }
                    const T q0 = group_sum<GW>(Q.x, gmask), q1 = group_sum<GW>(Q.y, gmask);
                    const V am = __ldcg(aux + i);
                    const T inf = T(1) / T(0);
                    kin0 += S0 > T(0) ? am.x * q0 / S0 : inf;
                    kin1 += S1 > T(0) ? am.y * q1 / S1 : inf;
                }
            }
            const T t0 = draw_target<T>(uw0, S0);
            const T t1 = draw_target<T>(uw1, S1);
            // the row that holds the crossing (the first row whose total exceeds what remains
            // of u*S), then in it the first column whose prefix does: the crossing row's
            // prefixes go through shared memory, one column per lane
            const T r0 = t0 - ex0, r1 = t1 - ex1;
            int nxt0, nxt1;
            {
                const int base = gw * GW;
                const unsigned b0 = __ballot_sync(gmask, active && t0 >= ex0 && P.x > r0) & gmask;
                const unsigned b1 = __ballot_sync(gmask, active && t1 >= ex1 && P.y > r1) & gmask;
                int row0 = b0 ? __ffs(b0) - 1 - base : -1;
                int row1 = b1 ? __ffs(b1) - 1 - base : -1;
                auto put_row = [&](V *d) {
                    if constexpr (CH == 2) {
#pragma unroll
                        for (int j = 0; j < L / 2; ++j)
                            reinterpret_cast<float4 *>(d)[j] =
                                make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
                    } else {
#pragma unroll
                        for (int j = 0; j < L; ++j) d[j] = v[j];
                    }
                };
                if (active && gl == row0) put_row(rb);
                if (active && gl == row1) put_row(rb + L);
                __syncwarp(gmask);
                const T q0 = __shfl_sync(gmask, r0, row0 < 0 ? 0 : row0, GW);
                const T q1 = __shfl_sync(gmask, r1, row1 < 0 ? 0 : row1, GW);
                const unsigned c0 = __ballot_sync(gmask, active && row0 >= 0 && rb[gl].x > q0) & gmask;
                const unsigned c1 = __ballot_sync(gmask, active && row1 >= 0 && rb[L + gl].y > q1) & gmask;
                __syncwarp(gmask);
                int col0 = c0 ? __ffs(c0) - 1 - base : 0;
                int col1 = c1 ? __ffs(c1) - 1 - base : 0;
                if (row0 < 0 || row1 < 0) {
                    // u*S at or beyond the rounded total: the last site with a positive weight
                    int last0 = -1, last1 = -1;
                    if (active) {
                        V pv = vzero(v[0]);
#pragma unroll
                        for (int ix = 0; ix < L; ++ix) {
                            if (v[ix].x > pv.x) last0 = ix;
                            if (v[ix].y > pv.y) last1 = ix;
                            pv = v[ix];
                        }
                    }
                    const unsigned f0 = __ballot_sync(gmask, last0 >= 0) & gmask;
                    const unsigned f1 = __ballot_sync(gmask, last1 >= 0) & gmask;
                    const int lr0 = f0 ? 31 - __clz(f0) - base : -1;
                    const int lr1 = f1 ? 31 - __clz(f1) - base : -1;
                    const int lc0 = __shfl_sync(gmask, last0, lr0 < 0 ? 0 : lr0, GW);
                    const int lc1 = __shfl_sync(gmask, last1, lr1 < 0 ? 0 : lr1, GW);
                    if (row0 < 0) {
                        row0 = lr0;
                        col0 = lc0;
                    }
                    if (row1 < 0) {
                        row1 = lr1;
                        col1 = lc1;
                    }
                }
                if (row0 < 0 || !(S0 > T(0))) {
                    nxt0 = cur0;  // all-zero CDF: stay and report
                    if (gl == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
                } else {
                    nxt0 = col0 + L * row0;
                }
                if (row1 < 0 || !(S1 > T(0))) {
                    nxt1 = cur1;
                    if (gl == 0 && has1) atomicAdd(&st.meas[c].degenerate, 1ull);
                } else {
                    nxt1 = col1 + L * row1;
                }
            }
            if (gl == 0) {
                // link x_l -> x_{l+1}
                ek0 += hl[(cx0 - nxt0 % L + L) % L] + hl[(cy0 - nxt0 / L + L) % L];
                owner0(i)[lb] = int16_t(nxt0);
                atomicAdd(hist_s + (long long)lb * N + nxt0, 1);
                if (has1) {
                    ek1 += hl[(cx1 - nxt1 % L + L) % L] + hl[(cy1 - nxt1 / L + L) % L];
                    owner1(i)[lb] = int16_t(nxt1);
                    atomicAdd(hist_s + (long long)lb * N + nxt1, 1);
                }
            }
            cur0 = nxt0;
            cur1 = nxt1;
        }
        if constexpr (GAUSS) {
            if (cd.gauss) book(double(kin0), double(kin1));
        }
        if (gl == 0) {
            // link x_{l0} -> x_{l0+1}
            ek0 += hl[(cur0 % L - sx0 + L) % L] + hl[(cur0 / L - sy0 + L) % L];
            if (has1) ek1 += hl[(cur1 % L - sx1 + L) % L] + hl[(cur1 / L - sy1 + L) % L];
            double eks = double(ek0) + (has1 ? double(ek1) : 0.0);
            if constexpr (BLK) eks *= chain_sign(st, c);  // sign-weighted with permutations
            atomicAdd(&st.meas[c].link_sum, eks);
        }
        __syncwarp(gmask);
    }
}

template <typename T, int L>
size_t ffbs_smem_bytes_t(int warps_per_cta) {
    using G = FfbsGeo<T, L>;
    return size_t(warps_per_cta) * G::GPW * G::GROUP_BYTES;
}

}  // namespace hqmc
