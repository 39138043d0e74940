// ffbs_big.cuh -- forward-filtering backward-sampling (Sec. 3.5.2) for lattices wider
// than a warp: L in {48, 64, 128}, FP32.
//
// One CTA owns one pair of same-spin worldlines (the .x/.y halves of float2, packed
// f32x2 arithmetic as in ffbs_kernel).  S threads hold one lattice line (S = 1 for
// L <= 64, S = 2 for L = 128), E = L/S elements each, in registers.  A slice of the
// forward filter alpha_{l+1} = G * (W_l . alpha_l) (Eq. ffbsFwd) is a line convolution
// along the in-register direction, one transpose through shared memory and a line
// convolution along the other direction, exactly as in the warp-wide kernel; the
// reductions (normaliser, row scan, crossing search) are block-wide.
//
// Line convolution with S = 2: the half-length complex FFT of size n = L/2 is split by
// decimation in time over the two threads (thread s holds z_{s + 2j}): each thread
// transforms its n/2 values, the odd thread applies W_n^k, and one exchange with the
// partner thread (shfl_xor 1) completes the radix-2 stage, leaving thread s with the
// spectral block [s n/2, (s+1) n/2).  The spectral mix pairs k with n-k, which lies in
// the partner's block at the mirrored register, so one more exchange feeds it; the
// inverse runs the same steps backwards.
//
// f_l is streamed to the CTA's slot in the same 16-byte chunk format as ffbs_kernel
// (chunk (position pair, line)); the backward pass prefetches each slice into shared
// memory with cp.async and samples x_l ~ max(f_l(y), 0) G(x_{l+1} - y) by the row-major
// inverse CDF, each thread scanning E consecutive sites of one row.
#pragma once

#include "ffbs.cuh"

namespace hqmc {

template <int L>
struct BigGeo {
    // threads per lattice line: two at L = 48 (three full warps per pair, 119 registers,
    // five CTAs per SM) and L = 128 (the line does not fit one thread); one at L = 64,
    // where the pair split over 128 threads measured 26% slower than 64 threads
    static constexpr int S = (L == 48 || L > 64) ? 2 : 1;
    static constexpr int E = L / S;                      // line elements per thread
    static constexpr int NT = ((L * S + 31) / 32) * 32;  // threads per CTA (one pair)
    static constexpr int NW = NT / 32;
    // resident CTAs per SM the register budget is sized for (L = 64: six CTAs of two warps
    // at 168 registers measured 2% faster than four at 235)
    static constexpr int MINB = (L == 48) ? 5 : (L == 64) ? 6 : 1;
    static constexpr int n = L / 2;                      // half-length complex FFT size
    static constexpr int m = n / S;                      // per-thread FFT size
    static constexpr int LP = (S == 2) ? L + 4 : L + 2;  // transpose pitch (elements)
    static constexpr size_t XBUF = size_t(L) * LP * 8;   // also holds (L/2)(L+1) 16-byte chunks
    static constexpr size_t MIXB = size_t(L) * 8;
    static constexpr size_t G2B = size_t(2 * L) * 4;
    static constexpr size_t WXB = size_t(L) * 8;
    static constexpr size_t TOTB = size_t(NT) * 8;       // per-thread totals / exclusive offsets
    static constexpr size_t RED = 16 * 8 + 64;           // warp partials and a few ints
    static constexpr size_t BYTES = XBUF + MIXB + G2B + WXB + 2 * TOTB + RED;
    static_assert(L % 4 == 0 && (S == 1 || m % 1 == 0), "line split");
    static_assert(XBUF >= size_t(L / 2) * (L + 1) * 16, "prefetch buffer");
};

// position in its line of register e of a thread that holds half s of the line
template <int L>
__device__ __forceinline__ int big_pos(int e, int s) {
    if constexpr (BigGeo<L>::S == 1) return e;
    else return 4 * (e >> 1) + 2 * s + (e & 1);
}

// word and bit of register e's site in its line's bit-packed field row/column
template <int L>
__device__ __forceinline__ int big_word(int e) {
    if constexpr (BigGeo<L>::S == 1) return e >> 5;
    else return e >> 4;
}
template <int L>
__device__ __forceinline__ int big_bit(int e, int s) {
    if constexpr (BigGeo<L>::S == 1) return e & 31;
    else return ((4 * (e >> 1)) & 31) + 2 * s + (e & 1);
}

// twiddle W_n^{+-k} for the odd thread of a split line, identity for the even one
template <int SGN, int K, int NN>
__device__ __forceinline__ cvec<float2> split_twiddle(cvec<float2> v, bool odd) {
    constexpr int k = ((K % NN) + NN) % NN;
    if constexpr (k == 0) {
        return v;
    } else {
        constexpr float c = float(ct::cos2pi(k, NN));
        constexpr float sn = float(SGN * ct::sin2pi(k, NN));
        const float cc = odd ? c : 1.f, ss = odd ? sn : 0.f;
        return {vfma(v.re, vsplat(cc), vmul(v.im, vsplat(-ss))), vfma(v.re, vsplat(ss), vmul(v.im, vsplat(cc)))};
    }
}

__device__ __forceinline__ float2 shfl_x1(float2 a) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, 1), __shfl_xor_sync(0xffffffffu, a.y, 1));
}

// line convolution of one thread's share of a line (see the file comment)
template <int L>
__device__ __forceinline__ void big_conv(float2 (&v)[BigGeo<L>::E], const float2 *mix, int s) {
    using B = BigGeo<L>;
    if constexpr (B::S == 1) {
        conv_line<L>(v, mix);
    } else {
        constexpr int n = B::n, m = B::m;
        const bool odd = s != 0;
        cvec<float2> z[m];
#pragma unroll
        for (int j = 0; j < m; ++j) z[j] = {v[2 * j], v[2 * j + 1]};
        fft<m, -1>(z);
        static_for<0, m>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            z[k] = split_twiddle<-1, k, n>(z[k], odd);
        });
#pragma unroll
        for (int k = 0; k < m; ++k) {
            const cvec<float2> pz = {shfl_x1(z[k].re), shfl_x1(z[k].im)};
            z[k] = odd ? cv_sub(pz, z[k]) : cv_add(z[k], pz);  // block s of the spectrum
        }
        // spectral mix: partner of index k + m s is n - k - m s: the mirrored register
        // (m - k) of the partner thread, or the value itself at k = 0
        cvec<float2> pm[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            const cvec<float2> src = z[(m - k) % m];
            pm[k] = {shfl_x1(src.re), shfl_x1(src.im)};
        }
        pm[0] = z[0];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            float2 al, be;
            load_mix(mix, k + m * s, al, be);
            const cvec<float2> zk = z[k];
            z[k] = {vfma(zk.re, al, vmul(pm[k].im, be)), vfma(zk.im, al, vmul(pm[k].re, be))};
        }
        // inverse: radix-2 across the pair, conjugate twiddle, per-thread inverse FFT
#pragma unroll
        for (int k = 0; k < m; ++k) {
            const cvec<float2> pz = {shfl_x1(z[k].re), shfl_x1(z[k].im)};
            z[k] = odd ? cv_sub(pz, z[k]) : cv_add(z[k], pz);
        }
        static_for<0, m>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            z[k] = split_twiddle<+1, k, n>(z[k], odd);
        });
        fft<m, +1>(z);
#pragma unroll
        for (int j = 0; j < m; ++j) {
            v[2 * j] = z[j].re;
            v[2 * j + 1] = z[j].im;
        }
    }
}

template <int L>
__global__ void __launch_bounds__(BigGeo<L>::NT, BigGeo<L>::MINB) ffbs_big_kernel(DevState st, FfbsLaunch fl) {
    using B = BigGeo<L>;
    using V = float2;
    using T = float;
    constexpr int S = B::S, E = B::E, NT = B::NT, NW = B::NW, LP = B::LP, N = L * L;
    constexpr int NCH = N / 2;  // 16-byte chunks per slice
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *xbuf = reinterpret_cast<V *>(smem_raw);
    V *mix = reinterpret_cast<V *>(smem_raw + B::XBUF);
    T *g2 = reinterpret_cast<T *>(smem_raw + B::XBUF + B::MIXB);
    V *wx = reinterpret_cast<V *>(smem_raw + B::XBUF + B::MIXB + B::G2B);
    V *tot = reinterpret_cast<V *>(smem_raw + B::XBUF + B::MIXB + B::G2B + B::WXB);
    V *exk = tot + NT;
    V *wred = exk + NT;                             // [16]
    int *ibuf = reinterpret_cast<int *>(wred + 16);  // [16]
    uint64_t *ubuf = reinterpret_cast<uint64_t *>(ibuf + 8);  // [2] (16-byte aligned: wred 128 B)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = tid / S, s = tid % S;  // forward: line p, half s
    const bool active = p < L;
    // backward: row rb, half hb; k = rb*S + hb is the row-major order of the thread's sites
    const int hb = tid / L, rb = tid % L;
    const bool bact = tid < L * S;
    V *slot = reinterpret_cast<V *>(fl.scratch) + (long long)blockIdx.x * fl.slot_elems;
    const uint64_t sweep = *st.sweep;

    // block-wide sum of a pair (every thread gets it)
    auto block_sum = [&](V v) -> V {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        __syncthreads();
        if (lane == 0) wred[warp] = v;
        __syncthreads();
        V r = wred[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = vadd(r, wred[w]);
        return r;
    };
    // bits of line `line` of slice l: rows (lines = y) or columns (lines = x)
    auto load_bits = [&](const uint32_t *base, int l, int line, uint32_t (&wb)[(L + 31) / 32], int wpl) {
#pragma unroll
        for (int w = 0; w < (L + 31) / 32; ++w) wb[w] = base[((long long)l * L + line) * wpl + w];
    };

    // work units (pair, block) are taken from a work counter, longest blocks first
    for (;;) {
        __syncthreads();
        if (tid == 0) ibuf[4] = int(atomicAdd(fl.next_unit, 1u));
        __syncthreads();
        const long long q = ibuf[4];
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
        // unit = (pair, block): the blocks of a pair are independent given their held ends
        const int Bk = ffbs_block_len(cd.block, M), nblk = ffbs_nblk(cd.block, M);
        const int ru = int(q - fl.class_unit_off[lo]);
        const int rr = ru / nblk, b = ru - rr * nblk;
        const int sg = rr / cd.npair, kp = rr % cd.npair;
        const int p0 = 2 * kp, p1 = 2 * kp + 1;
        const bool has1 = p1 < Nsig;
        const uint64_t wl0 = (uint64_t)sg * Nsig + p0, wl1 = (uint64_t)sg * Nsig + p1;
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const int wpl = cd.wpl;
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * wpl;
        // with a permutation P the unit of p runs from slice a of p to slice a of P(p): its
        // block positions at or past the wrap are slices of the successors q0 = P(p0),
        // q1 = P(p1) (the identity: the closed loops)
        int16_t *xspin = st.x + cd.x_off + (long long)sg * Nsig * M;
        const int *Pp = st.perm + cd.perm_off + sg * Nsig;
        const int q0 = Pp[p0], q1 = has1 ? Pp[p1] : q0;

        __syncthreads();
        for (int j = tid; j < L; j += NT) mix[j] = vsplat(tb.mix_f[j]);
        for (int j = tid; j < 2 * L; j += NT) g2[j] = tb.g_f[j < L ? j : j - L];
        if (tid == 0) {
            ibuf[0] = 0x7fffffff;
            ibuf[1] = 0x7fffffff;
        }
        __syncthreads();

        const u64x4 ua = philox4x64_10(0, 0, 2, sweep, cd.seed, 0);
        int a = int(u53(ua.v[0]) * M);
        if (a >= M) a = M - 1;
        if (ru == 0 && tid == 0) st.anchor[c] = a;

        // block b of Bk slices from the anchor, resampled with its two end sites held
        // (Bk = M: the closed loop); the log-weight is the sum of the blocks'
        const float *hl = tb.h_f;
        int *hist_s = st.hist + cd.h_off + (long long)sg * M * N;
        float ek0 = 0.f, ek1 = 0.f;
        int l0 = a + b * Bk;
        if (l0 >= M) l0 -= M;
        const int len = (b + 1) * Bk <= M ? Bk : M - b * Bk;
        const int le = (l0 + len >= M) ? l0 + len - M : l0 + len;
        const int wi = M - a - b * Bk;  // block positions >= wi lie past the wrap
        auto owner0 = [&](int i) { return xspin + (long long)(i >= wi ? q0 : p0) * M; };
        auto owner1 = [&](int i) { return xspin + (long long)(i >= wi ? q1 : p1) * M; };

        // ---- forward filter ----
        __syncthreads();
        V v[E];
        {
            const int xs0 = owner0(0)[l0];
            const int xs1 = has1 ? int(owner1(0)[l0]) : xs0;
            const int sx0 = xs0 % L, sy0 = xs0 / L, sx1 = xs1 % L, sy1 = xs1 / L;
            T wv0, wv1;
            if (cd.gauss) {
                wv0 = gauss_line<T>(st, cd, false, l0, sy0)[sx0];
                wv1 = gauss_line<T>(st, cd, false, l0, sy1)[sx1];
            } else {
                wv0 = ((srow[((long long)l0 * L + sy0) * wpl + (sx0 >> 5)] >> (sx0 & 31)) & 1u) ? wp : wm;
                wv1 = ((srow[((long long)l0 * L + sy1) * wpl + (sx1 >> 5)] >> (sx1 & 31)) & 1u) ? wp : wm;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int pos = big_pos<L>(e, s);
                v[e].x = (active && p == sy0 && pos == sx0) ? wv0 : T(0);
                v[e].y = (active && p == sy1 && pos == sx1) ? wv1 : T(0);
            }
        }
        int esum0 = 0, esum1 = 0;
        T fin0 = T(0), fin1 = T(0);
        int l = l0;
        for (int i = 0; i < len; ++i) {
            if (i >= 1 && active) {
                float4 *dst = reinterpret_cast<float4 *>(slot + (long long)i * N);
#pragma unroll
                for (int j = 0; j < E / 2; ++j)
                    dst[(S * j + s) * L + p] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
            }
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                big_conv<L>(v, mix, s);
                if (h == 0) {
                    __syncthreads();
                    if (active) {
#pragma unroll
                        for (int e = 0; e < E; ++e) xbuf[big_pos<L>(e, s) * LP + p] = v[e];
                    }
                    __syncthreads();
                    if (active) {
                        const V *src = xbuf + p * LP;
#pragma unroll
                        for (int j = 0; j < E / 2; ++j) {
                            const float4 c4 = *reinterpret_cast<const float4 *>(src + big_pos<L>(2 * j, s));
                            v[2 * j] = make_float2(c4.x, c4.y);
                            v[2 * j + 1] = make_float2(c4.z, c4.w);
                        }
                    }
                }
            }
            V sm = vzero(v[0]);
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) sm = vadd(sm, v[e]);
            }
            const V tsum = block_sum(sm);
            const T s0 = tsum.x, s1 = tsum.y;
            const int l1 = (l + 1 == M) ? 0 : l + 1;
            if (i < len - 1) {
                int e0 = 0, e1 = 0;
                if (s0 > T(0) && s0 < T(1e30)) e0 = fbits<T>::exponent(s0);
                else if (tid == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
                if (s1 > T(0) && s1 < T(1e30)) e1 = fbits<T>::exponent(s1);
                esum0 += e0;
                esum1 += e1;
                const T sc0 = fbits<T>::pow2(-e0), sc1 = fbits<T>::pow2(-e1);
                const V A = {wp * sc0, wp * sc1}, Bv = {wm * sc0, wm * sc1};
                if (active && cd.gauss) {
                    const T *w = gauss_line<T>(st, cd, (i & 1) == 0, l1, p);
#pragma unroll
                    for (int j = 0; j < E / 2; ++j) {
                        const float2 q = *reinterpret_cast<const float2 *>(w + big_pos<L>(2 * j, s));
                        v[2 * j] = vmul(v[2 * j], V{q.x * sc0, q.x * sc1});
                        v[2 * j + 1] = vmul(v[2 * j + 1], V{q.y * sc0, q.y * sc1});
                    }
                } else if (active) {
                    uint32_t wb[(L + 31) / 32];
                    load_bits((i & 1) ? srow : scol, l1, p, wb, wpl);
#pragma unroll
                    for (int e = 0; e < E; ++e) v[e] = vmul(v[e], ((wb[big_word<L>(e)] >> big_bit<L>(e, s)) & 1u) ? A : Bv);
                }
            } else {
                // alpha_{l0+len}(x_{l0+len}): final layout is C (lines = x) if len is odd
                const bool finC = (len & 1) != 0;
                const int xe0 = owner0(len)[le];
                const int xe1 = has1 ? int(owner1(len)[le]) : xe0;
                const int ex0 = xe0 % L, ey0 = xe0 / L, ex1 = xe1 % L, ey1 = xe1 / L;
                const int own0 = finC ? ex0 : ey0, pos0 = finC ? ey0 : ex0;
                const int own1 = finC ? ex1 : ey1, pos1 = finC ? ey1 : ex1;
                if (active) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int pos = big_pos<L>(e, s);
                        if (p == own0 && pos == pos0) wred[8].x = v[e].x;
                        if (p == own1 && pos == pos1) wred[8].y = v[e].y;
                    }
                }
                __syncthreads();
                fin0 = wred[8].x;
                fin1 = wred[8].y;
            }
            l = l1;
        }
        if (tid == 0) {
            // log-weight of the block; with several blocks, the pair's last finished block
            // sums the partials in block order (the same bits whichever finishes last)
            const double ln2 = 0.69314718055994530942;
            const double part0 = double(esum0) * ln2 + log(double(fin0));
            const double part1 = double(esum1) * ln2 + log(double(fin1));
            if (!(fin0 > T(0))) atomicAdd(&st.meas[c].nonpositive, 1ull);
            if (has1 && !(fin1 > T(0))) atomicAdd(&st.meas[c].nonpositive, 1ull);
            double *lw = st.logw + cd.logw_off;
            if (nblk == 1) {
                lw[wl0] = part0;
                if (has1) lw[wl1] = part1;
            } else {
                double *lp = st.logw_part + cd.lwp_off;
                lp[wl0 * nblk + b] = part0;
                if (has1) lp[wl1 * nblk + b] = part1;
                __threadfence();
                unsigned *done = st.blk_done + cd.done_off + rr;
                if (atomicAdd(done, 1u) == unsigned(nblk - 1)) {
                    __threadfence();
                    double s0 = 0.0, s1 = 0.0;
                    for (int k = 0; k < nblk; ++k) {
                        s0 += __ldcg(lp + wl0 * nblk + k);
                        if (has1) s1 += __ldcg(lp + wl1 * nblk + k);
                    }
                    lw[wl0] = s0;
                    if (has1) lw[wl1] = s1;
                    *done = 0u;  // ready for the next sweep
                }
            }
        }

        // ---- backward sampling ----
        auto prefetch = [&](int i) {
            const float4 *src = reinterpret_cast<const float4 *>(slot + (long long)i * N);
            float4 *dst = reinterpret_cast<float4 *>(xbuf);
            const bool C = (i & 1) != 0;
            for (int ch = tid; ch < NCH; ch += NT) {
                const int qq = ch / L, line = ch % L;
                cp_async16(dst + (C ? qq * (L + 1) + line : ch), src + ch);
            }
            cp_async_commit();
        };
        __syncthreads();
        if (len > 1) prefetch(len - 1);
        const int xs0 = owner0(0)[l0];
        const int xs1 = has1 ? int(owner1(0)[l0]) : xs0;
        const int sx0 = xs0 % L, sy0 = xs0 / L, sx1 = xs1 % L, sy1 = xs1 / L;
        int cur0 = owner0(len)[le];
        int cur1 = has1 ? int(owner1(len)[le]) : cur0;
        if (tid == 0) {
            atomicAdd(hist_s + (long long)l0 * N + xs0, 1);
            if (has1) atomicAdd(hist_s + (long long)l0 * N + xs1, 1);
        }
        int cached = -1;
        uint64_t wd0 = 0, wd1 = 0, wd2 = 0, wd3 = 0;
        for (int i = len - 1; i >= 1; --i) {
            int lb = l0 + i;
            if (lb >= M) lb -= M;
            cp_async_wait_all();
            __syncthreads();
            // this thread's E sites of row rb, from column hb*E
            V f[E];
            if (bact) {
                if ((i & 1) == 0) {
                    const float4 *src = reinterpret_cast<const float4 *>(xbuf);
#pragma unroll
                    for (int j = 0; j < E / 2; ++j) {
                        const float4 c4 = src[((hb * E) / 2 + j) * L + rb];
                        f[2 * j] = make_float2(c4.x, c4.y);
                        f[2 * j + 1] = make_float2(c4.z, c4.w);
                    }
                } else {
                    const V *src = xbuf + (rb / 2) * (L + 1) * 2 + (rb & 1);
#pragma unroll
                    for (int e = 0; e < E; ++e) f[e] = src[(hb * E + e) * 2];
                }
            }
            // uniforms of this slice: the first warp's 32 threads fill the words of 16 groups
            // of four slices at once (thread 2k + w: group k of the block, worldline w); the
            // slice's two threads publish theirs.  Then the x-weights of both worldlines.
            constexpr int PG = 16;
            const int grp = lb >> 2, blk = grp / PG;
            if (tid < 2 * PG && blk != cached) {
                const u64x4 w4 = philox4x64_10((uint64_t)(blk * PG + (tid >> 1)), (tid & 1) ? wl1 : wl0, 0, sweep,
                                               cd.seed, 0);
                wd0 = w4.v[0];
                wd1 = w4.v[1];
                wd2 = w4.v[2];
                wd3 = w4.v[3];
                cached = blk;
            }
            const int wsel = lb & 3, src = 2 * (grp - blk * PG);
            if (tid >= src && tid < src + 2) ubuf[tid - src] = wsel == 0 ? wd0 : wsel == 1 ? wd1 : wsel == 2 ? wd2 : wd3;
            const int cx0 = cur0 % L, cy0 = cur0 / L, cx1 = cur1 % L, cy1 = cur1 / L;
            __syncthreads();
            if (i > 1) prefetch(i - 1);
            for (int j = tid; j < L; j += NT) wx[j] = V{g2[j - cx0 + L], g2[j - cx1 + L]};
            if (tid == 0) {
                ibuf[0] = 0x7fffffff;
                ibuf[1] = 0x7fffffff;
                ibuf[2] = -1;
                ibuf[3] = -1;
            }
            __syncthreads();
            V P = vzero(wx[0]);
            if (bact) {
                const V gy = V{g2[rb - cy0 + L], g2[rb - cy1 + L]};
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    P = vfma(vmax0(f[e]), vmul(wx[hb * E + e], gy), P);
                    f[e] = P;
                }
            }
            // exclusive offsets in row-major order k = rb*S + hb
            const int k = bact ? rb * S + hb : tid;
            tot[k] = bact ? P : vzero(P);
            __syncthreads();
            V inc = tot[tid];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float t0 = __shfl_up_sync(0xffffffffu, inc.x, o);
                const float t1 = __shfl_up_sync(0xffffffffu, inc.y, o);
                if (lane >= o) {
                    inc.x += t0;
                    inc.y += t1;
                }
            }
            if (lane == 31) wred[warp] = inc;
            __syncthreads();
            V base = vzero(inc), Stot = vzero(inc);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (w < warp) base = vadd(base, wred[w]);
                Stot = vadd(Stot, wred[w]);
            }
            exk[tid] = vsub(vadd(base, inc), tot[tid]);
            __syncthreads();
            const V ex = exk[k];
            const T t0 = draw_target<T>(ubuf[0], Stot.x);
            const T t1 = draw_target<T>(ubuf[1], Stot.y);
            const T r0 = t0 - ex.x, r1 = t1 - ex.y;
            int n0 = 0, n1 = 0;
            if (bact) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    n0 += (f[e].x <= r0) ? 1 : 0;
                    n1 += (f[e].y <= r1) ? 1 : 0;
                }
                if (t0 >= ex.x && n0 < E) atomicMin(&ibuf[0], k * 256 + n0);
                if (t1 >= ex.y && n1 < E) atomicMin(&ibuf[1], k * 256 + n1);
            }
            __syncthreads();
            int win0 = ibuf[0], win1 = ibuf[1];
            if (win0 == 0x7fffffff || win1 == 0x7fffffff) {
                // u*S at or beyond the rounded total: the last site with a positive weight
                if (bact) {
                    int last0 = -1, last1 = -1;
                    V pv = vzero(f[0]);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (f[e].x > pv.x) last0 = e;
                        if (f[e].y > pv.y) last1 = e;
                        pv = f[e];
                    }
                    if (last0 >= 0) atomicMax(&ibuf[2], k * 256 + last0);
                    if (last1 >= 0) atomicMax(&ibuf[3], k * 256 + last1);
                }
                __syncthreads();
                if (win0 == 0x7fffffff) win0 = ibuf[2];
                if (win1 == 0x7fffffff) win1 = ibuf[3];
            }
            int nxt0, nxt1;
            if (win0 < 0 || !(Stot.x > T(0))) {
                nxt0 = cur0;
                if (tid == 0) atomicAdd(&st.meas[c].degenerate, 1ull);
            } else {
                const int kk = win0 >> 8, col = (kk % S) * E + (win0 & 255);
                nxt0 = col + L * (kk / S);
            }
            if (win1 < 0 || !(Stot.y > T(0))) {
                nxt1 = cur1;
                if (tid == 0 && has1) atomicAdd(&st.meas[c].degenerate, 1ull);
            } else {
                const int kk = win1 >> 8, col = (kk % S) * E + (win1 & 255);
                nxt1 = col + L * (kk / S);
            }
            if (tid == 0) {
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
        if (tid == 0) {
            // link x_{l0} -> x_{l0+1}
            ek0 += hl[(cur0 % L - sx0 + L) % L] + hl[(cur0 / L - sy0 + L) % L];
            if (has1) ek1 += hl[(cur1 % L - sx1 + L) % L] + hl[(cur1 / L - sy1 + L) % L];
            atomicAdd(&st.meas[c].link_sum, (double(ek0) + (has1 ? double(ek1) : 0.0)) * chain_sign(st, c));
        }
    }
}

}  // namespace hqmc
