// ffbs_wide.cuh -- forward-filtering backward-sampling (Sec. 3.5.2) for lattices wider
// than a warp: L in {48, 64, 128}, FP32 and FP64.
//
// One thread owns one lattice line of one worldline and holds it in registers as plain
// scalars (L values).  A CTA holds WPC worldlines of one spin (WPC = 2 at L = 48, where
// two worldlines fill three warps exactly; WPC = 1 otherwise), with thread t serving
// worldline t % WPC, line t / WPC.  A slice of the forward filter
//     alpha_{l+1} = G * (W_l . alpha_l)                     (Eq. ffbsFwd, position basis)
// is the line convolution of every line in registers (conv_line_1fft: a half-length complex
// FFT, the spectral mix of a real line, and the same FFT code again for the inverse), one
// transpose per worldline through shared memory, and the line convolution along the other
// direction; the layout alternates between slices.  In FP32 the complex adds and subtracts
// take a value's (re, im) as one f32x2 operand; products that cross the halves stay scalar.
// No thread shares a line with another, so the FFT needs no cross-thread exchange: the only
// data movement is the transpose.  A line per thread keeps the register count low enough
// for two 128-thread CTAs per SM at L = 128.
//
// Reductions over a worldline's lines (normaliser, maximum, row-total scan) are shuffles
// over the lanes of one worldline (offsets WPC .. 16) and a fixed-order sum of the warps'
// partials, so results do not depend on scheduling.
//
// f_l = W_l . alpha_l is streamed to the worldline's slot in 16-byte chunks (chunk j of
// line p at j*L + p, coalesced over the lines); the backward pass prefetches each slice
// into shared memory with cp.async and samples x_l ~ max(f_l(y), 0) G(x_{l+1} - y) by the
// row-major inverse CDF, one row per thread.
#pragma once

#include <cuda_bf16.h>

#include "ffbs.cuh"

namespace hqmc {

template <typename T, int L>
struct WideGeo {
    static constexpr int WPC = (L % 32 == 0) ? 1 : 2;  // worldlines per CTA
    static constexpr int NT = WPC * L;                    // threads: one per (worldline, line)
    static constexpr int NW = NT / 32;
    static constexpr int CH = int(16 / sizeof(T));        // elements per 16-byte chunk
    static constexpr int LP = L + 1;                      // transpose pitch (elements)
    static constexpr size_t a16(size_t v) { return (v + 15) & ~size_t(15); }
    // per worldline: the transpose buffer, also the prefetch buffer of one f slice
    static constexpr size_t XTR = size_t(L) * LP * sizeof(T);
    static constexpr size_t XPF = size_t(L / CH) * (L + 1) * 16;
    static constexpr size_t XB = a16(XTR > XPF ? XTR : XPF);
    static constexpr size_t MIXB = a16(size_t(2 * L) * sizeof(T));  // (al, -al, be, -be) per k
    static constexpr size_t G2B = a16(size_t(2 * L) * sizeof(T));
    static constexpr size_t WXB = a16(size_t(WPC) * L * sizeof(T));
    static constexpr size_t HLB = a16(size_t(L) * sizeof(float));
    static constexpr size_t REDB = a16(size_t(2 * NW * WPC + 4 * WPC) * sizeof(T));
    static constexpr size_t IB = 64;  // work unit, crossings, fallbacks, end exponents
    static constexpr size_t UB = a16(size_t(WPC) * 8);
    static constexpr size_t BYTES = WPC * XB + MIXB + G2B + WXB + HLB + REDB + IB + UB;
    // resident CTAs per SM the register budget is sized for
    static constexpr int MINB = sizeof(T) == 4 ? (L == 128 ? 2 : L == 64 ? 8 : 6) : (L == 128 ? 1 : 2);
    static_assert(L % 4 == 0 && NT % 32 == 0 && NT <= 256, "wide geometry");
    static_assert(XB >= XPF, "prefetch buffer");
};

// 16-byte moves between a register array (elements k .. k + 16/sizeof(T) - 1, constant k
// after unrolling) and memory, without taking the array's address
template <int K, int L>
__device__ __forceinline__ float4 pack16(const float (&v)[L]) { return make_float4(v[K], v[K + 1], v[K + 2], v[K + 3]); }
template <int K, int L>
__device__ __forceinline__ double2 pack16(const double (&v)[L]) { return make_double2(v[K], v[K + 1]); }
template <int K, int L>
__device__ __forceinline__ void unpack16(float (&v)[L], float4 c) {
    v[K] = c.x;
    v[K + 1] = c.y;
    v[K + 2] = c.z;
    v[K + 3] = c.w;
}
template <int K, int L>
__device__ __forceinline__ void unpack16(double (&v)[L], double2 c) {
    v[K] = c.x;
    v[K + 1] = c.y;
}
template <typename T>
using chunk16_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// Checkpoints of f (FP32 filters with f kept every K positions): checkpoint s of a
// worldline's slot holds f of position s K in the writer's layout, BF16 (16-byte chunk j
// of line p at j*L + p holds elements 8j .. 8j+7) or FP32 (as the streamed slices).
template <int L>
__device__ __forceinline__ void store_ckpt(const float (&v)[L], float *slot, int s, int bf16, int p) {
    constexpr int N = L * L;
    if (bf16) {
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(slot) + (long long)s * N);
        static_for<0, L / 8>([&](auto JI) {
            constexpr int j = decltype(JI)::value;
            const __nv_bfloat162 a = __floats2bfloat162_rn(v[8 * j], v[8 * j + 1]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[8 * j + 2], v[8 * j + 3]);
            const __nv_bfloat162 c = __floats2bfloat162_rn(v[8 * j + 4], v[8 * j + 5]);
            const __nv_bfloat162 d = __floats2bfloat162_rn(v[8 * j + 6], v[8 * j + 7]);
            unsigned ua, ub, uc, ud;
            memcpy(&ua, &a, 4);
            memcpy(&ub, &b, 4);
            memcpy(&uc, &c, 4);
            memcpy(&ud, &d, 4);
            dst[j * L + p] = make_uint4(ua, ub, uc, ud);
        });
    } else {
        float4 *dst = reinterpret_cast<float4 *>(slot + (long long)s * N);
        static_for<0, L / 4>([&](auto JI) {
            constexpr int j = decltype(JI)::value;
            dst[j * L + p] = pack16<4 * j>(v);
        });
    }
}
template <int L>
__device__ __forceinline__ void load_ckpt(float (&v)[L], const float *slot, int s, int bf16, int p) {
    constexpr int N = L * L;
    if (bf16) {
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(slot) + (long long)s * N);
        static_for<0, L / 8>([&](auto JI) {
            constexpr int j = decltype(JI)::value;
            const uint4 q = src[j * L + p];
            __nv_bfloat162 ba, bb, bc, bd;
            memcpy(&ba, &q.x, 4);
            memcpy(&bb, &q.y, 4);
            memcpy(&bc, &q.z, 4);
            memcpy(&bd, &q.w, 4);
            const float2 a = __bfloat1622float2(ba);
            const float2 b = __bfloat1622float2(bb);
            const float2 c = __bfloat1622float2(bc);
            const float2 d = __bfloat1622float2(bd);
            unpack16<8 * j>(v, make_float4(a.x, a.y, b.x, b.y));
            unpack16<8 * j + 4>(v, make_float4(c.x, c.y, d.x, d.y));
        });
    } else {
        const float4 *src = reinterpret_cast<const float4 *>(slot + (long long)s * N);
        static_for<0, L / 4>([&](auto JI) {
            constexpr int j = decltype(JI)::value;
            unpack16<4 * j>(v, src[j * L + p]);
        });
    }
}

// sum and maximum over the lanes of this thread's worldline (lanes lane % WPC == w) of
// one warp; every such lane gets the result
template <int WPC, typename T>
__device__ __forceinline__ T wl_warp_sum(T v) {
#pragma unroll
    for (int o = WPC; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int WPC, typename T>
__device__ __forceinline__ T wl_warp_max(T v) {
#pragma unroll
    for (int o = WPC; o < 32; o <<= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// CKPT: f kept every fl.ckpt_K positions and recomputed per segment in the backward pass
// (FP32 only); the streaming instantiation carries none of that code.  GAUSS: the class
// holds Gaussian-field chains (U < 0), whose potentials are read from the sigma field's
// tables and whose log-weight estimate is summed in the backward pass; the Hirsch-only
// instantiation carries none of that code.
template <typename T, int L, bool CKPT, bool GAUSS>
__global__ void __launch_bounds__(WideGeo<T, L>::NT, WideGeo<T, L>::MINB) ffbs_wide_kernel(DevState st, FfbsLaunch fl) {
    using G = WideGeo<T, L>;
    constexpr int WPC = G::WPC, NT = G::NT, NW = G::NW, CH = G::CH, LP = G::LP, N = L * L;
    constexpr int NCH = N / CH;  // 16-byte chunks per slice of one worldline
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sp = smem_raw;
    T *xbuf_all = reinterpret_cast<T *>(sp);
    sp += WPC * G::XB;
    T *mix = reinterpret_cast<T *>(sp);
    sp += G::MIXB;
    T *g2 = reinterpret_cast<T *>(sp);
    sp += G::G2B;
    T *wx_all = reinterpret_cast<T *>(sp);
    sp += G::WXB;
    float *hl = reinterpret_cast<float *>(sp);
    sp += G::HLB;
    T *wred = reinterpret_cast<T *>(sp);  // [NW][WPC] sums, [NW][WPC] maxima, [WPC] x 4 end values
    T *wmx = wred + NW * WPC;
    T *endv = wmx + NW * WPC;             // [WPC] end value, [WPC] top, [WPC] spare
    sp += G::REDB;
    int *ibuf = reinterpret_cast<int *>(sp);  // [0] unit, [1 + w] crossing, [5 + w] fallback, [9 + w] esum
    sp += G::IB;
    uint64_t *ubuf = reinterpret_cast<uint64_t *>(sp);  // [WPC] uniforms of the slice

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = tid % WPC;  // worldline of the CTA
    const int p = tid / WPC;  // line (forward), row (backward)
    T *xb = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(xbuf_all) + w * G::XB);
    T *wx = wx_all + w * L;
    const uint64_t sweep = *st.sweep;
    T *slot = reinterpret_cast<T *>(fl.scratch) + (long long)blockIdx.x * fl.slot_elems +
              (long long)w * (fl.slot_elems / WPC);

    // per-worldline sum and maximum over the CTA (fixed order: deterministic)
    auto wl_sum = [&](T v) -> T {
        v = wl_warp_sum<WPC>(v);
        __syncthreads();
        if (lane < WPC) wred[warp * WPC + lane] = v;
        __syncthreads();
        T r = wred[w];
#pragma unroll
        for (int k = 1; k < NW; ++k) r += wred[k * WPC + w];
        return r;
    };

    for (;;) {
        __syncthreads();
        if (tid == 0) ibuf[0] = int(atomicAdd(fl.next_unit, 1u));
        __syncthreads();
        const long long q = ibuf[0];
        if (q >= fl.total_units) break;
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
        const int ngrp = (Nsig + WPC - 1) / WPC;  // worldline groups per spin
        // unit = (group, block): the blocks of a group are independent given their held ends
        const int Bk = ffbs_block_len(cd.block, M), nblk = ffbs_nblk(cd.block, M);
        const int ru = int(q - fl.class_unit_off[lo]);
        const int rr = ru / nblk, b = ru - rr * nblk;
        const int sg = rr / ngrp, kg = rr % ngrp;
        const int pw0 = WPC * kg;
        const int nwl = (pw0 + WPC <= Nsig) ? WPC : Nsig - pw0;  // worldlines present in the group
        const bool has = w < nwl;
        const int pw = has ? pw0 + w : pw0;  // a missing worldline shadows the first (never written)
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const int wpl = cd.wpl;
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * wpl;
        // with a permutation P the unit of p runs from slice a of p to slice a of P(p): its
        // block positions at or past the wrap are slices of the successor (the identity:
        // the closed loop)
        int16_t *xspin = st.x + cd.x_off + (long long)sg * Nsig * M;
        const int qsucc = st.perm[cd.perm_off + sg * Nsig + pw];

        for (int j = tid; j < L; j += NT) {
            // conv_line_1fft's table: al_k, -al_k, be_k, -be_k from the interleaved al_k, be_k
            const T m = tab_mix<T>(tb)[j];
            mix[2 * j] = m;
            mix[2 * j + 1] = -m;
            hl[j] = tb.h_f[j];
        }
        for (int j = tid; j < 2 * L; j += NT) g2[j] = tab_g<T>(tb)[j < L ? j : j - L];

        const u64x4 ua = philox4x64_10(0, 0, 2, sweep, cd.seed, 0);
        int a = int(u53(ua.v[0]) * M);
        if (a >= M) a = M - 1;
        if (ru == 0 && tid == 0) st.anchor[c] = a;

        // block b of Bk slices from the anchor, resampled with its two end sites held
        // (Bk = M: the closed loop); the log-weight is the sum of the blocks'
        int l0 = a + b * Bk;
        if (l0 >= M) l0 -= M;
        const int len = (b + 1) * Bk <= M ? Bk : M - b * Bk;
        const int le = (l0 + len >= M) ? l0 + len - M : l0 + len;
        const int wi = M - a - b * Bk;  // block positions >= wi lie past the wrap
        auto owner = [&](int i) { return xspin + (long long)(i >= wi ? qsucc : pw) * M; };
        __syncthreads();

        // ---- forward filter ----
        T v[L];
        {
            const int xs = owner(0)[l0];
            const int sx = xs % L, sy = xs / L;
            T wv;
            if (GAUSS && cd.gauss) wv = gauss_line<T>(st, cd, false, l0, sy)[sx];
            else wv = ((srow[((long long)l0 * L + sy) * wpl + (sx >> 5)] >> (sx & 31)) & 1u) ? wp : wm;
#pragma unroll
            for (int r = 0; r < L; ++r) v[r] = (has && p == sy && r == sx) ? wv : T(0);
        }
        int esum = 0;
        // the slice of block position i (positions run from the block start l0)
        auto slice_of = [&](int i) {
            int s_ = l0 + i;
            return s_ >= M ? s_ - M : s_;
        };
        // f of position i (in the writer's layout: chunk j*L + p holds registers CH*j..) to
        // 16-byte chunks at dst
        auto put_f = [&](T *dst_base) {
            chunk16_t<T> *dst = reinterpret_cast<chunk16_t<T> *>(dst_base);
            static_for<0, L / CH>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                dst[j * L + p] = pack16<CH * j>(v);
            });
        };
        // G * v: both line directions with the transpose between them (the layout flips),
        // then the worldline's sum of the new message
        auto conv_sum = [&]() -> T {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                conv_line_1fft<L>(v, mix);
                if (h == 0) {
                    // transpose: line p, register r  ->  line r, register p
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < L; ++r) xb[r * LP + p] = v[r];
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < L; ++r) v[r] = xb[p * LP + r];
                }
            }
            T part[L / 2];
#pragma unroll
            for (int r = 0; r < L / 2; ++r) part[r] = v[2 * r] + v[2 * r + 1];
#pragma unroll
            for (int d = 1; d < L / 2; d <<= 1)
#pragma unroll
                for (int r = 0; r + d < L / 2; r += 2 * d) part[r] += part[r + d];
            return wl_sum(part[0]);
        };
        // v = alpha of position i + 1 (layout of parity i + 1)  ->  f of position i + 1:
        // renormalise by 2^-e and multiply by W of its slice; returns e
        auto renorm_w = [&](int i, T s, bool count) -> int {
            int e = 0;
            if (s > T(0) && s < T(1e30)) e = fbits<T>::exponent(s);
            else if (count && has && p == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
            const T sc = fbits<T>::pow2(-e);
            const int l1 = slice_of(i + 1);
            // the new layout is C (lines = x) when i is even: the field by columns
            if (GAUSS && cd.gauss) {
                const T *wl_ = gauss_line<T>(st, cd, (i & 1) == 0, l1, p);
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= wl_[r] * sc;
            } else {
                uint32_t wb[L / 32 + (L % 32 ? 1 : 0)];
                const uint32_t *bsrc = ((i & 1) ? srow : scol) + ((long long)l1 * L + p) * wpl;
#pragma unroll
                for (int k = 0; k < L / 32 + (L % 32 ? 1 : 0); ++k) wb[k] = bsrc[k];
                const T A = wp * sc, B = wm * sc;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= ((wb[r >> 5] >> (r & 31)) & 1u) ? A : B;
            }
            return e;
        };
        const int K = CKPT ? fl.ckpt_K : 0;  // 0: every f streamed; else f kept every K positions
        // Gaussian-field units keep max_y alpha_i(y) of every interior position i (at the
        // scale of the stored f_i) after the worldline's f storage, for the backward pass
        T *aux = slot + (fl.slot_elems / WPC - fl.len_max);
        for (int i = 0; i < len; ++i) {
            if (has) {
                if (K == 0) {
                    if (i >= 1) put_f(slot + (long long)i * N);
                } else if (i % K == 0) {
                    if constexpr (CKPT && sizeof(T) == 4) store_ckpt<L>(v, slot, i / K, fl.ckpt_bf16, p);
                }
            }
            const T s = conv_sum();
            if (i < len - 1) {
                T top = T(0);
                if (GAUSS && cd.gauss) {
                    // v = alpha of position i + 1: its largest value over the worldline
                    T mx = T(0);
#pragma unroll
                    for (int r = 0; r < L; ++r) mx = v[r] > mx ? v[r] : mx;
                    mx = wl_warp_max<WPC>(mx);
                    if (lane < WPC) wmx[warp * WPC + lane] = mx;
                    __syncthreads();
                    top = wmx[w];
                    for (int k = 1; k < NW; ++k) top = wmx[k * WPC + w] > top ? wmx[k * WPC + w] : top;
                }
                const int e = renorm_w(i, s, true);
                esum += e;
                if ((GAUSS && cd.gauss) && has && p == 0) aux[i + 1] = top * fbits<T>::pow2(-e);
            } else {
                // alpha_{l0+len}(x_{l0+len}): the final layout is C if len is odd; its
                // largest value gives kappa = top / end
                const bool finC = (len & 1) != 0;
                const int xe = owner(len)[le];
                const int ex = xe % L, ey = xe / L;
                const int own = finC ? ex : ey, reg = finC ? ey : ex;
                T mx = T(0);
#pragma unroll
                for (int r = 0; r < L; ++r) mx = v[r] > mx ? v[r] : mx;
                mx = wl_warp_max<WPC>(mx);
                if (lane < WPC) wmx[warp * WPC + lane] = mx;
                if (p == own) endv[w] = reg_select<L>(v, reg);
                __syncthreads();
                // open-path estimator (one-body density matrix, for n_k): the last block's end
                // message read at every site, relative to the held end, sign-weighted
                if (st.open_acc && b == nblk - 1 && has) {
                    const T fin = endv[w];
                    if (fin > T(0)) {
                        double *acc = st.open_acc + cd.meas_off;
                        const T inv = T(chain_sign(st, c)) / fin;
#pragma unroll
                        for (int r = 0; r < L; ++r) {
                            const int x = finC ? p : r, y = finC ? r : p;
                            atomicAdd(acc + (x - ex + L) % L + L * ((y - ey + L) % L), double(v[r] * inv));
                        }
                    }
                }
                if (tid < WPC) {
                    T top = wmx[tid];
                    for (int k = 1; k < NW; ++k) top = wmx[k * WPC + tid] > top ? wmx[k * WPC + tid] : top;
                    endv[WPC + tid] = top;
                }
                if (p == 0) ibuf[9 + w] = esum;
                __syncthreads();
            }
        }
        // the unit's log-weights and their error estimates (endv[3 WPC + k]: the Gaussian-field
        // sum of worldline k from the backward pass); Hirsch units book them after the forward
        // pass, Gaussian-field units after the backward pass
        auto book = [&]() {
            if (tid != 0) return;
            // log-weights of the block; with several blocks, the group's last finished block
            // sums the partials in block order (the same bits whichever finishes last)
            const double ln2 = 0.69314718055994530942;
            const double inf = __longlong_as_double(0x7ff0000000000000LL);
            double part[WPC], err[WPC];
            for (int k = 0; k < nwl; ++k) {
                const T fin = endv[k], top = endv[WPC + k];
                part[k] = double(ibuf[9 + k]) * ln2 + log(double(fin));
                // Hirsch units: len x the end concentration; Gaussian units: the conditional
                // means of the concentration over positions 1 .. len-1 given the drawn next
                // sites (calibration factor in FP64), plus the end's
                const double kap = double(top) / double(fin);
                err[k] = !(fin > T(0)) ? inf
                         : (GAUSS && cd.gauss) ? logw_err_estimate<T>(gauss_sum_factor<T>() * double(endv[3 * WPC + k]) + kap, 1, L, false)
                                    : logw_err_estimate<T>(kap, len, L, false);
                if (!(fin > T(0))) atomicAdd(&st.meas[c].nonpositive, 1ull);
            }
            auto flag = [&](double lwv, double e) {
                if (!(e <= logw_tolerance<T>() * fmax(1.0, fabs(lwv)))) atomicAdd(&st.meas[c].inexact, 1ull);
            };
            double *lw = st.logw + cd.logw_off;
            double *le_ = st.logw_err + cd.logw_off;
            const uint64_t wl0 = (uint64_t)sg * Nsig + pw0;
            if (nblk == 1) {
                for (int k = 0; k < nwl; ++k) {
                    lw[wl0 + k] = part[k];
                    le_[wl0 + k] = err[k];
                    flag(part[k], err[k]);
                }
            } else {
                double *lp = st.logw_part + cd.lwp_off;
                double *ep = st.logw_err_part + cd.lwp_off;
                for (int k = 0; k < nwl; ++k) {
                    lp[(wl0 + k) * nblk + b] = part[k];
                    ep[(wl0 + k) * nblk + b] = err[k];
                }
                __threadfence();
                unsigned *done = st.blk_done + cd.done_off + rr;
                if (atomicAdd(done, 1u) == unsigned(nblk - 1)) {
                    __threadfence();
                    for (int k = 0; k < nwl; ++k) {
                        double s0 = 0.0, e0 = 0.0;
                        for (int kb = 0; kb < nblk; ++kb) {
                            s0 += __ldcg(lp + (wl0 + k) * nblk + kb);
                            e0 += __ldcg(ep + (wl0 + k) * nblk + kb);
                        }
                        lw[wl0 + k] = s0;
                        le_[wl0 + k] = e0;
                        flag(s0, e0);
                    }
                    *done = 0u;  // ready for the next sweep
                }
            }
        };
        if (!(GAUSS && cd.gauss)) book();

        // ---- backward sampling ----
        // slice i of the slots -> xbuf: R slices (i even) chunk for chunk, C slices (i odd)
        // into rows of pitch L+1 chunks so that the row-wise reads below are conflict-free
        // f of position i: the streamed slice, or with checkpoints the recomputed segment
        // buffer after the checkpoint region (slot position i % K)
        auto f_src = [&](const T *wslot, int i) {
            return K == 0 ? wslot + (long long)i * N : wslot + fl.seg_off + (long long)(i % K) * N;
        };
        auto prefetch = [&](int i) {
            const bool C = (i & 1) != 0;
            for (int ch = tid; ch < WPC * NCH; ch += NT) {
                const int ww = ch / NCH, k = ch - ww * NCH;
                const int qq = k / L, line = k - qq * L;
                const float4 *src = reinterpret_cast<const float4 *>(
                    f_src(slot + (long long)(ww - w) * (fl.slot_elems / WPC), i));
                float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(xbuf_all) + ww * G::XB);
                cp_async16(dst + (C ? qq * (L + 1) + line : k), src + k);
            }
            cp_async_commit();
        };
        // recompute positions s K .. min(len, s K + K) - 1 from checkpoint s into the segment
        // buffer, in FP32 (the same slice steps as the forward filter)
        auto recompute = [&](int sgi) {
            if constexpr (CKPT && sizeof(T) == 4) {
                const int i0 = sgi * K, i1 = min(len, i0 + K);
                load_ckpt<L>(v, slot, sgi, fl.ckpt_bf16, p);
                if (!has) {
#pragma unroll
                    for (int r = 0; r < L; ++r) v[r] = T(0);
                }
                put_f(slot + fl.seg_off);
                for (int i = i0; i < i1 - 1; ++i) {
                    const T s_ = conv_sum();
                    renorm_w(i, s_, false);
                    put_f(slot + fl.seg_off + (long long)(i + 1 - i0) * N);
                }
            }
        };
        __syncthreads();
        if (len > 1 && K == 0) prefetch(len - 1);
        int cur_seg = -1;
        const int xs = owner(0)[l0];
        const int sx = xs % L, sy = xs / L;
        int cur = owner(len)[le];
        int *hist_s = st.hist + cd.h_off + (long long)sg * M * N;
        if (has && p == 0) atomicAdd(hist_s + (long long)l0 * N + xs, 1);
        float ek = 0.f;
        int cached = -1;
        uint64_t wd0 = 0, wd1 = 0, wd2 = 0, wd3 = 0;
        // Gaussian-field units: sum over positions i of E[max_y alpha_i(y) / alpha_i(x_i) | x_{i+1}]
        // = max alpha_i sum_y W_i(y) G(x_{i+1} - y) / S_i, S_i = sum_y f_i(y) G(x_{i+1} - y) the
        // draw's total.  Under the unit's posterior its mean is max alpha_i sum_y beta_i(y) /
        // <alpha_i, beta_i> (beta_i the backward message from the held end): the factor by which
        // a rounding error of the size of max alpha_i at slice i reaches the log-weight.
        T kin = T(0);
        for (int i = len - 1; i >= 1; --i) {
            int lb = l0 + i;
            if (lb >= M) lb -= M;
            if (CKPT && K != 0 && i / K != cur_seg) {
                // entering a new segment: no copy is in flight here (the previous position
                // did not prefetch across the boundary); its writes are visible after the barrier
                cur_seg = i / K;
                __syncthreads();
                recompute(cur_seg);
                __syncthreads();
                prefetch(i);
            }
            cp_async_wait_all();
            __syncthreads();
            // row p of f_l (x = 0 .. L-1)
            T f[L];
            if ((i & 1) == 0) {
                const chunk16_t<T> *src = reinterpret_cast<const chunk16_t<T> *>(xb);
                static_for<0, L / CH>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    unpack16<CH * j>(f, src[j * L + p]);
                });
            } else {
                const T *src = xb + (p / CH) * (L + 1) * CH + (p % CH);
#pragma unroll
                for (int x = 0; x < L; ++x) f[x] = src[x * CH];
            }
            // uniforms of this slice: warp 0 fills the words of 32/WPC groups of four slices
            // at once (lane = group * WPC + worldline); the slice's owners publish theirs
            constexpr int PG = 32 / WPC;
            const int grp = lb >> 2, blk = grp / PG;
            if (warp == 0 && blk != cached) {
                const int gw = lane % WPC;
                const uint64_t wlg = (uint64_t)sg * Nsig + (pw0 + gw < Nsig ? pw0 + gw : pw0);
                const u64x4 w4 = philox4x64_10((uint64_t)(blk * PG + lane / WPC), wlg, 0, sweep, cd.seed, 0);
                wd0 = w4.v[0];
                wd1 = w4.v[1];
                wd2 = w4.v[2];
                wd3 = w4.v[3];
                cached = blk;
            }
            const int wsel = lb & 3, src = WPC * (grp - blk * PG);
            if (warp == 0 && lane >= src && lane < src + WPC)
                ubuf[lane - src] = wsel == 0 ? wd0 : wsel == 1 ? wd1 : wsel == 2 ? wd2 : wd3;
            const int cx = cur % L, cy = cur / L;
            __syncthreads();
            if (i > 1 && (K == 0 || (i - 1) / K == cur_seg)) prefetch(i - 1);
            wx[p] = g2[p - cx + L];
            if (tid < 2 * WPC) ibuf[1 + (tid < WPC ? tid : 4 + tid - WPC)] = tid < WPC ? 0x7fffffff : -1;
            __syncthreads();
            // p(y) = max(f, 0) g(ix - cx) g(iy - cy): inclusive in-row prefix
            T P = T(0);
            {
                const T gy = g2[p - cy + L];
#pragma unroll
                for (int x = 0; x < L; ++x) {
                    const T fx = f[x] > T(0) ? f[x] : T(0);
                    P = vfma(fx, wx[x] * gy, P);
                    f[x] = P;
                }
            }
            // exclusive offsets over the rows of this worldline: a scan over the lanes of
            // the worldline (offsets WPC, 2 WPC, ...), then the earlier warps' totals
            T inc = P;
#pragma unroll
            for (int o = WPC; o < 32; o <<= 1) {
                const T t0 = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t0;
            }
            if (lane >= 32 - WPC) wred[warp * WPC + (lane - (32 - WPC))] = inc;
            __syncthreads();
            T base = T(0), Stot = T(0);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const T t0 = wred[k * WPC + w];
                if (k < warp) base += t0;
                Stot += t0;
            }
            const T ex = base + inc - P;
            const T t = draw_target<T>(ubuf[w], Stot);
            if (GAUSS && cd.gauss) {
                // sum_y W_i(y) G(x_{i+1} - y): row p of W against the x-weights
                const T *wrow = gauss_line<T>(st, cd, false, lb, p);
                T Q = T(0);
#pragma unroll 4
                for (int x = 0; x < L; ++x) Q = vfma(wrow[x], wx[x], Q);
                const T qs = wl_sum(Q * g2[p - cy + L]);
                if (has && p == 0) kin += Stot > T(0) ? __ldcg(aux + i) * qs / Stot : T(1) / T(0);
            }
            const T rem = t - ex;
            if (has) {
                int n = 0;
#pragma unroll
                for (int x = 0; x < L; ++x) n += (f[x] <= rem) ? 1 : 0;
                if (t >= ex && n < L) atomicMin(&ibuf[1 + w], p * 256 + n);
            }
            __syncthreads();
            int win = ibuf[1 + w];
            bool miss = false;
            for (int k = 0; k < nwl; ++k) miss |= ibuf[1 + k] == 0x7fffffff;
            if (miss) {
                // u*S at or beyond the rounded total: the last site with a positive weight
                if (has) {
                    int last = -1;
                    T pv = T(0);
#pragma unroll
                    for (int x = 0; x < L; ++x) {
                        if (f[x] > pv) last = x;
                        pv = f[x];
                    }
                    if (last >= 0) atomicMax(&ibuf[5 + w], p * 256 + last);
                }
                __syncthreads();
                if (win == 0x7fffffff) win = ibuf[5 + w];
            }
            // an absent worldline (odd count) keeps its shadow site, so that its threads
            // index the propagator tables within bounds on the next slice
            int nxt = cur;
            if (has) {
                const int col = win & 255, row = win >> 8;
                if (win < 0 || !(Stot > T(0)) || col >= L || row >= L) {
                    if (p == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
                } else {
                    nxt = col + L * row;
                }
            }
            if (has && p == 0) {
                ek += hl[(cx - nxt % L + L) % L] + hl[(cy - nxt / L + L) % L];
                owner(i)[lb] = int16_t(nxt);
                atomicAdd(hist_s + (long long)lb * N + nxt, 1);
            }
            cur = nxt;
        }
        if (GAUSS && cd.gauss) {
            if (has && p == 0) endv[3 * WPC + w] = kin;
            __syncthreads();
            book();
        }
        if (has && p == 0) {
            // link x_{l0} -> x_{l0+1}
            ek += hl[(cur % L - sx + L) % L] + hl[(cur / L - sy + L) % L];
            atomicAdd(&st.meas[c].link_sum, double(ek) * chain_sign(st, c));
        }
    }
}

#define HQMC_WIDE_SIZES(X) X(48) X(64) X(128)

// host side, per Gaussian flag: raise the kernels' shared-memory limits and return the
// residency of the streaming instantiation; launch the class's instantiation (the limit is
// raised beforehand, never during stream capture)
template <typename T, int L, bool G>
cudaError_t wide_occ(int *blocks) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t e = raise_smem_limit(ffbs_wide_kernel<T, L, true, G>, WideGeo<T, L>::BYTES);
        if (e != cudaSuccess) return e;
    }
    auto k = ffbs_wide_kernel<T, L, false, G>;
    cudaError_t e = raise_smem_limit(k, WideGeo<T, L>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, WideGeo<T, L>::NT, WideGeo<T, L>::BYTES);
}

template <bool G>
cudaError_t wide_occ_dispatch(int L, bool fp64, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return fp64 ? wide_occ<double, n, G>(blocks) : wide_occ<float, n, G>(blocks);
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <bool G>
cudaError_t wide_launch_dispatch(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n)                                                                                           \
    case n:                                                                                                    \
        if (fp64)                                                                                              \
            ffbs_wide_kernel<double, n, false, G><<<grid, WideGeo<double, n>::NT, WideGeo<double, n>::BYTES, s>>>(st, fl); \
        else if (fl.ckpt_K > 0)                                                                               \
            ffbs_wide_kernel<float, n, true, G><<<grid, WideGeo<float, n>::NT, WideGeo<float, n>::BYTES, s>>>(st, fl);     \
        else                                                                                                   \
            ffbs_wide_kernel<float, n, false, G><<<grid, WideGeo<float, n>::NT, WideGeo<float, n>::BYTES, s>>>(st, fl);    \
        return cudaGetLastError();
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hqmc
