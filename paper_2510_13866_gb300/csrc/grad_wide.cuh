// grad_wide.cuh -- log-weight of the current worldlines and its adjoint (the reverse pass of
// the forward filter, Eq. ffbsFwd of Sec. 3.5.2) for lattices wider than a warp: L in
// {48, 64, 128}, FP32 and FP64.  The quantities and the checkpoint scheme are those of
// grad.cuh: every worldline anchored at slice 0 on its current site,
//     d log Z / d v_l(x) = F_l(x) H_l(x) / Z,      Z = <F_l, H_l> for every l,
//     d log Z / d t      = sum_l <F_l, (dG/dt) * b_{l+1}> / Z,
// with F_l = W_l . alpha_l, H_l = G * b_{l+1}, b_l = W_l . H_l, b_M = delta_{x0}; F kept
// every K slices (BF16 or the context precision) and each K-slice segment recomputed.
//
// One thread owns one lattice line of one worldline, as in the wide FFBS kernel
// (ffbs_wide.cuh), and holds one message line at a time.  The t-derivative needs no second
// message: G = exp(t dtau A) with A the lattice adjacency (g(d) is the d-th element of
// exp(t dtau A) on a ring, G = g (x) g), so dG/dt = dtau A G and
//     <F_l, (dG/dt) * b_{l+1}> = dtau <F_l, A H_l>,
// the sum over each site's four neighbours of H_l: the two along the thread's line are in
// its registers, the two across lines come from a copy of H_l in shared memory.
#pragma once

#include <cuda_bf16.h>

#include "ffbs_wide.cuh"
#include "grad.cuh"

namespace hqmc {

template <typename T, int L>
__global__ void __launch_bounds__(WideGeo<T, L>::NT, WideGeo<T, L>::MINB) grad_wide_kernel(DevState st, GradLaunch gk) {
    using G = WideGeo<T, L>;
    constexpr int WPC = G::WPC, NT = G::NT, NW = G::NW, CH = G::CH, LP = G::LP, N = L * L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sp = smem_raw;
    T *xbuf_all = reinterpret_cast<T *>(sp);
    sp += WPC * G::XB;
    T *mix = reinterpret_cast<T *>(sp);
    sp += G::MIXB;
    sp += G::G2B + G::WXB + G::HLB;  // (layout shared with the FFBS kernel; unused here)
    T *wred = reinterpret_cast<T *>(sp);
    T *endv = wred + 2 * NW * WPC;
    sp += G::REDB;
    int *ibuf = reinterpret_cast<int *>(sp);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = tid % WPC, p = tid / WPC;
    T *xb = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(xbuf_all) + w * G::XB);
    unsigned char *ck = reinterpret_cast<unsigned char *>(gk.ckpt) + (long long)blockIdx.x * gk.ckpt_bytes +
                        (long long)w * (gk.ckpt_bytes / WPC);
    T *seg = reinterpret_cast<T *>(gk.seg) + (long long)blockIdx.x * gk.seg_elems + (long long)w * (gk.seg_elems / WPC);
    const T *vlog_all = reinterpret_cast<const T *>(gk.v);
    T *dv_all = reinterpret_cast<T *>(gk.dv);
    const int K = gk.K;

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
        if (tid == 0) ibuf[0] = int(atomicAdd(gk.next_pair, 1u));
        __syncthreads();
        const long long q = ibuf[0];
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
        const int ngrp = (Nsig + WPC - 1) / WPC;
        const int rr = int(q - gk.class_pair_off[lo]);
        const int sg = rr / ngrp, kg = rr % ngrp;
        const int pw0 = WPC * kg;
        const int nwl = (pw0 + WPC <= Nsig) ? WPC : Nsig - pw0;
        const bool has = w < nwl;
        const int pw = has ? pw0 + w : pw0;
        const T wp = T(cd.w_plus[sg]), wm = T(cd.w_minus[sg]);
        const uint32_t *srow = st.sbits + cd.s_off;
        const uint32_t *scol = srow + (long long)M * L * cd.wpl;
        const T *vlog = vlog_all ? vlog_all + cd.v_off + (long long)sg * M * N : nullptr;
        T *dvp = dv_all ? dv_all + cd.v_off + (long long)sg * M * N : nullptr;
        const int x0 = st.x[cd.x_off + ((long long)sg * Nsig + pw) * M];
        const int ax = x0 % L, ay = x0 / L;
        const T dtau = T(cd.beta / M);

        for (int j = tid; j < L; j += NT) {
            const T m = tab_mix<T>(tb)[j];  // (al, -al, be, -be) per k for conv_line_1fft
            mix[2 * j] = m;
            mix[2 * j + 1] = -m;
        }
        __syncthreads();

        // site of register r of line p in the layout of slice l (R: line = y, C: line = x)
        auto site = [&](int l, int r) { return (l & 1) ? p + L * r : r + L * p; };
        T v[L];
        // v <- v . W_l . sc  (slice l's layout)
        auto mul_w = [&](int l, T sc) {
            if (vlog) {
                const T *vl = vlog + (long long)l * N;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= exp_t<T>(vl[site(l, r)]) * sc;
            } else if (cd.gauss) {
                const T *wl_ = gauss_line<T>(st, cd, (l & 1) != 0, l, p);
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= wl_[r] * sc;
            } else {
                uint32_t wb[L / 32 + (L % 32 ? 1 : 0)];
                const uint32_t *bsrc = ((l & 1) ? scol : srow) + ((long long)l * L + p) * cd.wpl;
#pragma unroll
                for (int k = 0; k < L / 32 + (L % 32 ? 1 : 0); ++k) wb[k] = bsrc[k];
                const T A = wp * sc, B = wm * sc;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= ((wb[r >> 5] >> (r & 31)) & 1u) ? A : B;
            }
        };
        // v <- G * v (the layout flips)
        auto conv = [&]() {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                conv_line_1fft<L>(v, mix);
                if (h == 0) {
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < L; ++r) xb[r * LP + p] = v[r];
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < L; ++r) v[r] = xb[p * LP + r];
                }
            }
        };
        auto line_sum = [&]() -> T {
            T s = T(0);
#pragma unroll
            for (int r = 0; r < L; ++r) s += v[r];
            return wl_sum(s);
        };
        auto pow2_of = [&](T s, int &e) -> T {
            e = 0;
            if (s > T(0) && s < T(1e30)) e = fbits<T>::exponent(s);
            else if (has && p == 0) atomicOr(st.status, kStatusDegenerate);
            return fbits<T>::pow2(-e);
        };
        // checkpoint s of this worldline: F of slice s K (BF16 or the context precision)
        auto ck_store = [&](int s) {
            if (!has) return;
            if (gk.ckpt_bf16) {
                __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) dst[r * L + p] = __float2bfloat16_rn(float(v[r]));
            } else {
                T *dst = reinterpret_cast<T *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) dst[r * L + p] = v[r];
            }
        };
        auto ck_load = [&](int s) {
            if (gk.ckpt_bf16) {
                const __nv_bfloat16 *src = reinterpret_cast<const __nv_bfloat16 *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = T(__bfloat162float(src[r * L + p]));
            } else {
                const T *src = reinterpret_cast<const T *>(ck) + (long long)s * N;
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = src[r * L + p];
            }
            if (!has) {
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = T(0);
            }
        };

        // ---- forward filter from slice 0, F_l kept every K slices ----
#pragma unroll
        for (int r = 0; r < L; ++r) v[r] = (has && p == ay && r == ax) ? T(1) : T(0);
        mul_w(0, T(1));
        int esum = 0;
        for (int l = 0; l < M; ++l) {
            if (l % K == 0) ck_store(l / K);
            conv();
            const T s = line_sum();
            if (l < M - 1) {
                int e;
                const T sc = pow2_of(s, e);
                esum += e;
                mul_w(l + 1, sc);
            } else {
                // alpha_M(x0): the final layout is C if M is odd
                const bool finC = (M & 1) != 0;
                const int own = finC ? ax : ay, reg = finC ? ay : ax;
                if (p == own) endv[w] = reg_select<L>(v, reg);
                if (p == 0) ibuf[9 + w] = esum;  // each worldline's own exponent sum
                __syncthreads();
            }
        }
        if (tid == 0) {
            const double ln2 = 0.69314718055994530942;
            double lz = 0.0;
            for (int k = 0; k < nwl; ++k) {
                lz += double(ibuf[9 + k]) * ln2 + log(double(endv[k]));
                if (!(endv[k] > T(0))) atomicOr(st.status, kStatusNonPositive);
            }
            atomicAdd(&gk.logz[c], lz);
        }

        // ---- reverse pass ----
        // b_M = delta_{x0}, laid out so that G * b lands in the layout of F_{M-1}
        {
            const bool bC = (M & 1) != 0;
#pragma unroll
            for (int r = 0; r < L; ++r) v[r] = (has && (bC ? (p == ax && r == ay) : (p == ay && r == ax))) ? T(1) : T(0);
        }
        T dts = T(0), dtc = T(0);  // compensated sum of the per-slice ratios (thread p = 0)
        const int nseg = (M + K - 1) / K;
        for (int s = nseg - 1; s >= 0; --s) {
            const int lb = s * K, lend = min(M, lb + K);
            // recompute F_lb .. F_{lend-1} into the segment buffer; b waits in the buffer's
            // spare slice (one message line per thread stays in registers)
            {
                T *park = seg + (long long)K * N;  // one spare slice after the segment
#pragma unroll
                for (int r = 0; r < L; ++r) park[r * L + p] = v[r];
                ck_load(s);
                T *dst0 = seg;
#pragma unroll
                for (int r = 0; r < L; ++r) dst0[r * L + p] = v[r];
                for (int l = lb; l < lend - 1; ++l) {
                    conv();
                    const T sm = line_sum();
                    int e;
                    const T sc = pow2_of(sm, e);
                    mul_w(l + 1, sc);
                    T *dst = seg + (long long)(l + 1 - lb) * N;
#pragma unroll
                    for (int r = 0; r < L; ++r) dst[r * L + p] = v[r];
                }
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] = park[r * L + p];
            }
            for (int l = lend - 1; l >= lb; --l) {
                conv();  // v = H_l = G * b_{l+1}, in the layout of F_l
                // H_l's lines in shared memory for the neighbours across lines
                __syncthreads();
#pragma unroll
                for (int r = 0; r < L; ++r) xb[p * LP + r] = v[r];
                __syncthreads();
                const T *F = seg + (long long)(l - lb) * N;
                const int pm = (p == 0) ? L - 1 : p - 1, pp = (p == L - 1) ? 0 : p + 1;
                T z = T(0), zd = T(0);
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    const T f = F[r * L + p];
                    const T nb = v[(r + L - 1) % L] + v[(r + 1) % L] + xb[pm * LP + r] + xb[pp * LP + r];
                    z = vfma(f, v[r], z);
                    zd = vfma(f, nb, zd);
                }
                const T Z = wl_sum(z), ZD = wl_sum(zd);
                if (has && !(Z > T(0)) && p == 0) atomicOr(st.status, kStatusNonPositive);
                if (has && p == 0) {
                    const T y = dtau * ZD / Z - dtc;
                    const T t = dts + y;
                    dtc = (t - dts) - y;
                    dts = t;
                }
                if (dvp && has) {
                    const T iz = T(1) / Z;
                    T *dvl = dvp + (long long)l * N;
#pragma unroll
                    for (int r = 0; r < L; ++r) atomic_add_t<T>(dvl + site(l, r), F[r * L + p] * v[r] * iz);
                }
                // b_l = W_l . H_l, renormalised
                mul_w(l, T(1));
                const T sm = line_sum();
                int e;
                const T sc = pow2_of(sm, e);
#pragma unroll
                for (int r = 0; r < L; ++r) v[r] *= sc;
            }
        }
        if (has && p == 0) atomicAdd(&gk.dt[c], double(dts));
    }
    (void)CH;
}

}  // namespace hqmc
