// grad.cuh -- log-weight of the current worldlines and its adjoint: the hand-written
// reverse pass of the forward filter (Eq. ffbsFwd, Sec. 3.5.2) giving
//     d log Z / d v_{l,sigma}(x)  (v = log W: the forward-backward site marginals)
//     d log Z / d t
// for every worldline anchored at slice 0 on its current site x0.
//
// With F_l = W_l . alpha_l, alpha_{l+1} = G * F_l, Z = alpha_M(x0), the backward messages
// are b_M = delta_{x0}, H_l = G * b_{l+1} (G is even, so correlation = convolution),
// b_l = W_l . H_l, and Z = <F_l, H_l> for every l.  Hence
//     d log Z / d v_l(x) = F_l(x) H_l(x) / Z,
//     d log Z / d t      = sum_l <F_l, (dG/dt) * b_{l+1}> / Z.
// Every message is renormalised by a power of two per slice; the ratios above are
// scale-free, so no normaliser needs to be carried in the reverse pass.
//
// Memory: the forward pass keeps F_l only every K slices (K = ceil(sqrt M) by default),
// in BF16 with the slice's power-of-two exponent (FP32 context) or in the context's own
// precision; the reverse pass recomputes each K-slice segment into a per-group buffer
// (L2-resident) and walks it backwards.  One group of lanes owns a pair of same-spin
// worldlines, as in the FFBS kernel; dG/dt * b shares the line spectra of G * b:
//   x lines:  Z = DFT(b);  A = IDFT(mix_g Z),  Ad = IDFT(mix_dg Z)      (one transpose each)
//   y lines:  ZA = DFT(A), ZAd = DFT(Ad);  H = IDFT(mix_g ZA),
//             D = IDFT(mix_g ZAd + mix_dg ZA)                       (= dG/dt * b)
#pragma once

#include <cuda_bf16.h>

#include "ffbs.cuh"

namespace hqmc {

template <typename T, int L>
struct GradGeo {
    using F = FfbsGeo<T, L>;
    using V = vec2_t<T>;
    static constexpr size_t XBUF = F::XBUF;
    static constexpr size_t MIXB = F::MIXB;
    static constexpr size_t GROUP_BYTES = XBUF + 2 * MIXB;
};

template <typename T>
__device__ __forceinline__ const T *tab_mixd(const ChainTab &tb);
template <>
__device__ __forceinline__ const float *tab_mixd<float>(const ChainTab &tb) { return tb.mixd_f; }
template <>
__device__ __forceinline__ const double *tab_mixd<double>(const ChainTab &tb) { return tb.mixd_d; }

template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ void atomic_add_t(T *p, T v) { atomicAdd(p, v); }

// four FP32 reductions into one 16-byte aligned global address (sm_90 and later)
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

template <typename T, int L>
__global__ void __launch_bounds__(128) grad_kernel(DevState st, GradLaunch gk) {
    using G = GradGeo<T, L>;
    using FG = FfbsGeo<T, L>;
    using V = vec2_t<T>;
    constexpr int N = L * L;
    constexpr int GW = FG::GW, LP = FG::LP, CH = FG::CH, KS = line_spec<L>::K;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GW, gw = lane / GW;
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (gw * GW));
    const bool active = gl < L;
    const int wpc = blockDim.x >> 5;
    unsigned char *gsm = smem_raw + size_t(warp * FG::GPW + gw) * G::GROUP_BYTES;
    V *xbuf = reinterpret_cast<V *>(gsm);
    V *mixg = reinterpret_cast<V *>(gsm + G::XBUF);
    V *mixdg = reinterpret_cast<V *>(gsm + G::XBUF + G::MIXB);
    const long long gid = ((long long)blockIdx.x * wpc + warp) * FG::GPW + gw;
    const long long ngroups = (long long)gridDim.x * wpc * FG::GPW;
    unsigned char *ck = reinterpret_cast<unsigned char *>(gk.ckpt) + gid * gk.ckpt_bytes;
    V *seg = reinterpret_cast<V *>(gk.seg) + gid * gk.seg_elems;
    const T *vlog_all = reinterpret_cast<const T *>(gk.v);
    T *dv_all = reinterpret_cast<T *>(gk.dv);
    const int K = gk.K;

    // transpose through shared memory: lane p, register r  ->  lane r, register p
    auto transpose = [&](V (&v)[L]) {
        __syncwarp(gmask);
        if (active) {
#pragma unroll
            for (int r = 0; r < L; ++r) xbuf[r * LP + gl] = v[r];
        }
        __syncwarp(gmask);
        if (active) {
            const V *src = xbuf + gl * LP;
#pragma unroll
            for (int p = 0; p < L; ++p) v[p] = src[p];
        }
    };

    (void)ngroups;
    for (;;) {
        unsigned qn = 0;
        if (gl == 0) qn = atomicAdd(gk.next_pair, 1u);
        const long long q = (long long)__shfl_sync(gmask, qn, 0, GW);
        if (q >= gk.total_pairs) break;
        int lo = 0, hi = gk.nclass - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (gk.class_pair_off[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        const int c = gk.class_chains[lo];
        const ChainDev &cd = st.chains[c];
        const ChainTab &tb = st.tabs[c];
        const int M = cd.M, Nsig = cd.Nsig;
        const int rr = int(q - gk.class_pair_off[lo]);
        const int sg = rr / cd.npair, kp = rr % cd.npair;
        const int p0 = 2 * kp, p1 = 2 * kp + 1;
        const bool has1 = p1 < Nsig;
        const uint64_t wl0 = (uint64_t)sg * Nsig + p0, wl1 = (uint64_t)sg * Nsig + p1;
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * cd.wpl;
        const T *vlog = vlog_all ? vlog_all + cd.v_off + (long long)sg * M * N : nullptr;
        T *dvp = dv_all ? dv_all + cd.v_off + (long long)sg * M * N : nullptr;
        // vector reductions need every slice's row start 16-byte aligned
        const bool dv_v4 = dvp && (N % 4 == 0) && (reinterpret_cast<uintptr_t>(dvp) & 15) == 0;
        const int x00 = st.x[cd.x_off + (long long)wl0 * M];
        const int x01 = has1 ? int(st.x[cd.x_off + (long long)wl1 * M]) : x00;
        const int ax0 = x00 % L, ay0 = x00 / L, ax1 = x01 % L, ay1 = x01 / L;

        __syncwarp(gmask);
        {
            const T *src = tab_mix<T>(tb), *srcd = tab_mixd<T>(tb);
            for (int j = gl; j < L; j += GW) {
                mixg[j] = vsplat(src[j]);
                mixdg[j] = vsplat(srcd[j]);
            }
        }
        __syncwarp(gmask);

        // site of register r of this lane in the layout of slice l (R: lane = iy, C: lane = ix)
        auto site = [&](int l, int r) { return (l & 1) ? gl + L * r : r + L * gl; };
        // v <- v . W_l . (s0, s1)  (slice l's layout)
        auto mul_w = [&](V (&v)[L], int l, T s0, T s1) {
            if (!active) return;
            if (vlog) {
                const T *vl = vlog + (long long)l * N;
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    const T w = exp_t<T>(vl[site(l, r)]);
                    v[r] = vmul(v[r], V{w * s0, w * s1});
                }
            } else if (cd.gauss) {
                mul_gauss_line<T, L>(v, gauss_line<T>(st, cd, (l & 1) != 0, l, gl), s0, s1);
            } else {
                const uint32_t *wsrc = (l & 1) ? scol : srow;
                const uint32_t w = wsrc[((long long)l * L + gl) * cd.wpl];
                const V A = {wp * s0, wp * s1}, B = {wm * s0, wm * s1};
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = vmul(v[r], ((w >> r) & 1u) ? A : B);
            }
        };
        auto sums = [&](const V (&v)[L], T &s0, T &s1) {
            V s = vzero(v[0]);
            if (active) {
#pragma unroll
                for (int r = 0; r < L; ++r) s = vadd(s, v[r]);
            }
            s0 = group_sum<GW>(s.x, gmask);
            s1 = group_sum<GW>(s.y, gmask);
        };
        auto pow2_of = [&](T s, int &e) -> T {
            e = 0;
            if (s > T(0) && s < T(1e30)) e = fbits<T>::exponent(s);
            else if (gl == 0) atomicOr(st.status, kStatusDegenerate);
            return fbits<T>::pow2(-e);
        };
        // one slice of G * v: x lines (in registers), transpose, y lines; layout flips
        auto conv2 = [&](V (&v)[L]) {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                conv_line<L>(v, mixg);
                if (h == 0) transpose(v);
            }
        };
        auto ck_store = [&](int s, const V (&v)[L], int e0, int e1) {
            if (gk.ckpt_bf16) {
                __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(ck) + (long long)s * N;
                if (active) {
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[r * L + gl] = __floats2bfloat162_rn(float(v[r].x), float(v[r].y));
                }
            } else {
                V *dst = reinterpret_cast<V *>(ck) + (long long)s * N;
                if (active) {
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[r * L + gl] = v[r];
                }
            }
            if (gl == 0) {
                int *ex = reinterpret_cast<int *>(ck + gk.ckpt_exp_off) + 2 * s;
                ex[0] = e0;
                ex[1] = e1;
            }
        };
        auto ck_load = [&](int s, V (&v)[L]) {
            if (!active) return;
            if (gk.ckpt_bf16) {
                const __nv_bfloat162 *src = reinterpret_cast<const __nv_bfloat162 *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    const float2 f = __bfloat1622float2(src[r * L + gl]);
                    v[r] = V{T(f.x), T(f.y)};
                }
            } else {
                const V *src = reinterpret_cast<const V *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = src[r * L + gl];
            }
        };

        // ---- forward filter from slice 0, F_l kept every K slices ----
        V f[L];
#pragma unroll
        for (int r = 0; r < L; ++r) {
            f[r].x = (gl == ay0 && r == ax0) ? T(1) : T(0);
            f[r].y = (gl == ay1 && r == ax1) ? T(1) : T(0);
        }
        mul_w(f, 0, T(1), T(1));
        int esum0 = 0, esum1 = 0;
        T fin0 = T(1), fin1 = T(1);
        for (int l = 0; l < M; ++l) {
            if (l % K == 0) ck_store(l / K, f, esum0, esum1);
            conv2(f);
            T s0, s1;
            sums(f, s0, s1);
            if (l < M - 1) {
                int e0, e1;
                const T sc0 = pow2_of(s0, e0), sc1 = pow2_of(s1, e1);
                esum0 += e0;
                esum1 += e1;
                mul_w(f, l + 1, sc0, sc1);
            } else {
                const bool finC = (M & 1) != 0;
                const int own0 = finC ? ax0 : ay0, reg0 = finC ? ay0 : ax0;
                const int own1 = finC ? ax1 : ay1, reg1 = finC ? ay1 : ax1;
                const T c0 = reg_select<L>(f, reg0).x;
                const T c1 = reg_select<L>(f, reg1).y;
                fin0 = __shfl_sync(gmask, c0, own0, GW);
                fin1 = __shfl_sync(gmask, c1, own1, GW);
            }
        }
        if (gl == 0) {
            const double ln2 = 0.69314718055994530942;
            double lz = double(esum0) * ln2 + log(double(fin0));
            if (!(fin0 > T(0))) atomicOr(st.status, kStatusNonPositive);
            if (has1) {
                lz += double(esum1) * ln2 + log(double(fin1));
                if (!(fin1 > T(0))) atomicOr(st.status, kStatusNonPositive);
            }
            atomicAdd(&gk.logz[c], lz);
        }

        // ---- reverse pass ----
        // b_M = delta_{x0}, laid out so that G * b lands in the layout of F_{M-1}
        V b[L];
        {
            const bool bC = (M & 1) != 0;
#pragma unroll
            for (int r = 0; r < L; ++r) {
                b[r].x = (bC ? (gl == ax0 && r == ay0) : (gl == ay0 && r == ax0)) ? T(1) : T(0);
                b[r].y = (bC ? (gl == ax1 && r == ay1) : (gl == ay1 && r == ax1)) ? T(1) : T(0);
            }
        }
        // d log Z / dt: per-slice ratios in the context precision, compensated (Kahan) sums
        // (no FP64 instruction per slice in the FP32 context)
        T dts0 = T(0), dtc0 = T(0), dts1 = T(0), dtc1 = T(0);
        auto kahan = [](T &sum, T &comp, T v) {
            const T y = v - comp;
            const T t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        };
        const int nseg = (M + K - 1) / K;
        for (int s = nseg - 1; s >= 0; --s) {
            const int lb = s * K, le = min(M, lb + K);
            // recompute F_lb .. F_{le-1} into the segment buffer (same lane, same slots)
            ck_load(s, f);
            for (int l = lb; l < le; ++l) {
                if (active) {
                    V *dst = seg + (long long)(l - lb) * N;
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[r * L + gl] = f[r];
                }
                if (l < le - 1) {
                    conv2(f);
                    T s0, s1;
                    sums(f, s0, s1);
                    int e0, e1;
                    const T sc0 = pow2_of(s0, e0), sc1 = pow2_of(s1, e1);
                    mul_w(f, l + 1, sc0, sc1);
                }
            }
            for (int l = le - 1; l >= lb; --l) {
                // H = G * b and D = dG/dt * b (both end in the layout of F_l)
                V d[L];
                {
                    cvec<V> z[KS], zd[KS];
                    line_fwd<L>(b, z);
                    spec_mix<L, false>(zd, z, mixdg);
                    spec_mix_inplace<L>(z, mixg);
                    line_inv<L>(z, b);
                    line_inv<L>(zd, d);
                }
                transpose(b);
                transpose(d);
                {
                    cvec<V> z[KS], zd[KS];
                    line_fwd<L>(b, z);
                    line_fwd<L>(d, zd);
                    spec_mix_inplace<L>(zd, mixg);
                    spec_mix<L, true>(zd, z, mixdg);
                    spec_mix_inplace<L>(z, mixg);
                    line_inv<L>(z, b);   // H
                    line_inv<L>(zd, d);  // D
                }
                // F_l from the segment buffer
                if (active) {
                    const V *src = seg + (long long)(l - lb) * N;
#pragma unroll
                    for (int r = 0; r < L; ++r) f[r] = src[r * L + gl];
                }
                V zf = vzero(b[0]), zdf = vzero(b[0]);
                if (active) {
#pragma unroll
                    for (int r = 0; r < L; ++r) {
                        zf = vfma(f[r], b[r], zf);
                        zdf = vfma(f[r], d[r], zdf);
                    }
                }
                const T z0 = group_sum<GW>(zf.x, gmask), z1 = group_sum<GW>(zf.y, gmask);
                const T zd0 = group_sum<GW>(zdf.x, gmask), zd1 = group_sum<GW>(zdf.y, gmask);
                if (!(z0 > T(0)) || (has1 && !(z1 > T(0)))) {
                    if (gl == 0) atomicOr(st.status, kStatusNonPositive);
                }
                kahan(dts0, dtc0, zd0 / z0);
                kahan(dts1, dtc1, zd1 / z1);
                if (dvp && active) {
                    const T iz0 = T(1) / z0, iz1 = has1 ? T(1) / z1 : T(0);
                    T *dvl = dvp + (long long)l * N;
                    bool done = false;
                    if constexpr (sizeof(T) == 4 && L % 4 == 0) {
                        // even slices: the lane's L sites are contiguous (site r + L gl), so
                        // they go out as 16-byte vector reductions, one L2 sector each
                        if (!(l & 1) && dv_v4) {
                            T *q = dvl + L * gl;
#pragma unroll
                            for (int r = 0; r < L; r += 4) {
                                const V m0 = vmul(f[r], b[r]), m1 = vmul(f[r + 1], b[r + 1]);
                                const V m2 = vmul(f[r + 2], b[r + 2]), m3 = vmul(f[r + 3], b[r + 3]);
                                red_add_v4(q + r, m0.x * iz0 + m0.y * iz1, m1.x * iz0 + m1.y * iz1,
                                           m2.x * iz0 + m2.y * iz1, m3.x * iz0 + m3.y * iz1);
                            }
                            done = true;
                        }
                    }
                    if (!done) {
#pragma unroll
                        for (int r = 0; r < L; ++r) {
                            const V m = vmul(f[r], b[r]);
                            atomic_add_t<T>(dvl + site(l, r), m.x * iz0 + m.y * iz1);
                        }
                    }
                }
                // b_l = W_l . H_l, renormalised
                mul_w(b, l, T(1), T(1));
                T s0, s1;
                sums(b, s0, s1);
                int e0, e1;
                const T sc0 = pow2_of(s0, e0), sc1 = pow2_of(s1, e1);
                const V sc = {sc0, sc1};
#pragma unroll
                for (int r = 0; r < L; ++r) b[r] = vmul(b[r], sc);
            }
        }
        if (gl == 0) atomicAdd(&gk.dt[c], double(dts0) + (has1 ? double(dts1) : 0.0));
        __syncwarp(gmask);
    }
    (void)CH;
}

template <typename T, int L>
size_t grad_smem_bytes_t(int warps_per_cta) {
    return size_t(warps_per_cta) * FfbsGeo<T, L>::GPW * GradGeo<T, L>::GROUP_BYTES;
}

}  // namespace hqmc
