// slice.cu -- site-parallel kernels: the Hirsch-field Gibbs resample fused with the
// observable accumulation (Sec. 3.5.4 and Sec. 4), state initialisation, the sweep
// counter and the observable read-out.
#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "internal.h"

namespace hqmc {

namespace {

constexpr int kSliceThreads = 256;
constexpr int kSkSmemMaxN = 4096;  // S(k) summed over the CTA's slices in shared memory up
                                   // to L = 64; beyond, each slice adds to global memory

// Block-wide sum of an unsigned 64-bit value into *dst (one atomic per block).
__device__ void block_add_u64(unsigned long long v, unsigned long long *dst, unsigned long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    __syncthreads();
    if (ln == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        if (s) atomicAdd(dst, s);
    }
}

struct SliceSmem {
    size_t rows, red, pp, ms, x1, vb, tw, sk, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// byte offsets of the slice kernel's shared arrays for lattice size L and S slices handled
// together: per slice the field bits by rows and columns, the slice's m and its row DFT,
// and (grouped form) its |m^(k)|^2 before the sum over the group's slices
__host__ __device__ inline SliceSmem slice_smem_layout(int L, int wpl, int S, bool grouped) {
    const size_t N = size_t(L) * L, K1 = size_t(L) / 2 + 1;
    SliceSmem s{};
    s.rows = 0;
    s.red = align16(s.rows + size_t(S) * 2 * size_t(L) * wpl * 4);
    s.pp = align16(s.red + 32 * 8);
    s.ms = align16(s.pp + (2 * kPTab + 1) * 8);
    s.x1 = align16(s.ms + size_t(S) * N * 4);
    s.vb = align16(s.x1 + size_t(S) * K1 * L * 8);
    s.tw = align16(s.vb + (grouped ? size_t(S) * K1 * L * 8 : 0));
    s.sk = align16(s.tw + size_t(L) * 8);
    s.total = N <= size_t(kSkSmemMaxN) ? align16(s.sk + N * 8) : s.sk;
    return s;
}

constexpr size_t kSliceSmemBudget = 200 * 1024;
constexpr int kGroupMaxL = 12;  // the grouped form up to this lattice size

// Gaussian field (U < 0): standard normal by the Box-Muller transform from the two
// uniforms of j = 2x and 2x+1: z = sqrt(-2 ln(1 - u1)) cos(2 pi u2), in FP64.
__device__ __forceinline__ double box_muller(uint64_t w1, uint64_t w2) {
    const double u1 = u53(w1), u2 = u53(w2);
    return sqrt(-2.0 * log(1.0 - u1)) * cospi(2.0 * u2);
}

// sigma_{x,l} and its slice potential W = exp(a sigma) in both layouts
__device__ __forceinline__ void put_gauss(const DevState &st, const ChainDev &cd, int l, int x, double sig) {
    const int L = cd.L, N = cd.N;
    const int ix = x % L, iy = x / L;
    st.gsig[cd.g_off + (long long)l * N + x] = sig;
    const double w = exp(cd.gcoup * sig);
    const long long rw = 2 * cd.g_off + (long long)l * N + iy * L + ix;
    const long long cw = 2 * cd.g_off + (long long)cd.M * N + (long long)l * N + ix * L + iy;
    if (st.gw_f64) {
        static_cast<double *>(st.gw)[rw] = w;
        static_cast<double *>(st.gw)[cw] = w;
    } else {
        static_cast<float *>(st.gw)[rw] = float(w);
        static_cast<float *>(st.gw)[cw] = float(w);
    }
}

}  // namespace

// Sequential form (lattices above kGroupMaxL): one CTA per (chain, group of
// slices_per_cta slices), the slices one after another through the same shared arrays.
// For every site of a slice:
//   m = n_up - n_dn;  s = +1 iff u < P(s=+1|m) = 1/(1+exp(-2 lambda m))  (FP64 compare),
// written bit-packed by rows and by columns; the histogram is cleared for the next
// sweep.  With `measure`, the slice's n, n_up n_dn, m^2 and |m^(k)|^2/N are added to
// the chain's accumulators (m^ by a direct separable DFT in FP32).
__global__ void __launch_bounds__(kSliceThreads) slice_kernel(DevState st, int slices_per_cta, int measure) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N, M = cd.M, wpl = cd.wpl;
    const int l_begin = blockIdx.x * slices_per_cta;
    if (l_begin >= M) return;
    const int l_end = min(M, l_begin + slices_per_cta);
    const uint64_t sweep = *st.sweep;
    const double lam = cd.lam;
    const ChainTab &tb = st.tabs[c];

    const bool do_sk = measure != 0;
    const bool sk_smem = N <= kSkSmemMaxN;
    const SliceSmem lay = slice_smem_layout(L, wpl, 1, false);
    uint32_t *rows = reinterpret_cast<uint32_t *>(smem_raw + lay.rows);  // [L][wpl]
    uint32_t *cols = rows + L * wpl;                                     // [L][wpl]
    unsigned long long *red = reinterpret_cast<unsigned long long *>(smem_raw + lay.red);
    double *pp = reinterpret_cast<double *>(smem_raw + lay.pp);         // P(s=+1 | m), |m| <= kPTab
    float *ms = reinterpret_cast<float *>(smem_raw + lay.ms);            // [N] m of the slice
    float2 *x1 = reinterpret_cast<float2 *>(smem_raw + lay.x1);          // [N] row DFT
    float2 *tw = reinterpret_cast<float2 *>(smem_raw + lay.tw);          // [L] e^{-2 pi i j / L}
    double *skacc = reinterpret_cast<double *>(smem_raw + lay.sk);       // [N]

    for (int k = threadIdx.x; k < 2 * L * wpl; k += blockDim.x) rows[k] = 0u;
    for (int k = threadIdx.x; k < 2 * kPTab + 1; k += blockDim.x) pp[k] = tb.pplus[k];
    if (do_sk) {
        for (int j = threadIdx.x; j < L; j += blockDim.x) {
            float s, co;
            sincospif(2.0f * float(j) / float(L), &s, &co);
            tw[j] = make_float2(co, -s);
        }
        if (sk_smem)
            for (int k = threadIdx.x; k < N; k += blockDim.x) skacc[k] = 0.0;
    }
    __syncthreads();

    unsigned long long n_acc = 0, d_acc = 0, m2_acc = 0;
    int *hu_base = st.hist + cd.h_off;
    int *hd_base = hu_base + (long long)M * N;
    uint32_t *srow_g = st.sbits + cd.s_off;
    uint32_t *scol_g = srow_g + (long long)M * L * wpl;

    for (int l = l_begin; l < l_end; ++l) {
        int *hu = hu_base + (long long)l * N;
        int *hd = hd_base + (long long)l * N;
        if (cd.gauss) {
            // Gaussian field: sigma ~ N(a (n_up + n_dn - 1/2), 1), uniforms j = 2x, 2x+1
            const int npairs = (N + 1) >> 1;
            for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
                const u64x4 w4 = philox4x64_10((uint64_t)pr, (uint64_t)l, 1, sweep, cd.seed, 0);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int x = 2 * pr + j;
                    if (x >= N) break;
                    const int nu = hu[x], nd = hd[x];
                    hu[x] = 0;
                    hd[x] = 0;
                    const int m = nu - nd;
                    put_gauss(st, cd, l, x, cd.gcoup * (double(nu + nd) - 0.5) + box_muller(w4.v[2 * j], w4.v[2 * j + 1]));
                    if (measure) {
                        n_acc += (unsigned long long)(nu + nd);
                        d_acc += (unsigned long long)(nu * nd);
                        m2_acc += (unsigned long long)(m * m);
                        if (do_sk) ms[x] = float(m);
                    }
                }
            }
        }
        const int nquads = cd.gauss ? 0 : (N + 3) >> 2;
        // whole quads of 16-byte aligned counts move as one vector load and one store
        const bool vec = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(hu) | reinterpret_cast<uintptr_t>(hd)) & 15) == 0;
        for (int qd = threadIdx.x; qd < nquads; qd += blockDim.x) {
            const u64x4 w4 = philox4x64_10((uint64_t)qd, (uint64_t)l, 1, sweep, cd.seed, 0);
            int nuq[4], ndq[4];
            if (vec) {
                const int4 a = reinterpret_cast<const int4 *>(hu)[qd], b = reinterpret_cast<const int4 *>(hd)[qd];
                reinterpret_cast<int4 *>(hu)[qd] = make_int4(0, 0, 0, 0);
                reinterpret_cast<int4 *>(hd)[qd] = make_int4(0, 0, 0, 0);
                nuq[0] = a.x; nuq[1] = a.y; nuq[2] = a.z; nuq[3] = a.w;
                ndq[0] = b.x; ndq[1] = b.y; ndq[2] = b.z; ndq[3] = b.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int x = 4 * qd + j;
                    nuq[j] = x < N ? hu[x] : 0;
                    ndq[j] = x < N ? hd[x] : 0;
                    if (x < N) {
                        hu[x] = 0;
                        hd[x] = 0;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = 4 * qd + j;
                if (x >= N) break;
                const int nu = nuq[j], nd = ndq[j];
                const int m = nu - nd;
                const double pplus = (m >= -kPTab && m <= kPTab) ? pp[m + kPTab]
                                                                  : 1.0 / (1.0 + exp(-2.0 * lam * m));
                const bool up = u53(w4.v[j]) < pplus;
                const int ix = x % L, iy = x / L;
                if (up) {
                    atomicOr(&rows[iy * wpl + (ix >> 5)], 1u << (ix & 31));
                    atomicOr(&cols[ix * wpl + (iy >> 5)], 1u << (iy & 31));
                }
                if (measure) {
                    n_acc += (unsigned long long)(nu + nd);
                    d_acc += (unsigned long long)(nu * nd);
                    m2_acc += (unsigned long long)(m * m);
                    if (do_sk) ms[x] = float(m);
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < (cd.gauss ? 0 : L * wpl); k += blockDim.x) {
            srow_g[(long long)l * L * wpl + k] = rows[k];
            scol_g[(long long)l * L * wpl + k] = cols[k];
        }
        // S(k) of a real field: m^(-k) = conj(m^(k)), so only kx = 0..L/2 is transformed and
        // |m^(L - kx, L - ky)|^2 = |m^(kx, ky)|^2 fills the other half
        const int K1 = L / 2 + 1;  // kx = 0 .. L/2
        if (do_sk) {
            // x1[iy][kx] = sum_ix m[iy][ix] e^{-2 pi i kx ix / L}
            for (int o = threadIdx.x; o < K1 * L; o += blockDim.x) {
                const int kx = o % K1, iy = o / K1;
                float re = 0.f, im = 0.f;
                int ph = 0;
                for (int ix = 0; ix < L; ++ix) {
                    const float mv = ms[iy * L + ix];
                    re += mv * tw[ph].x;
                    im += mv * tw[ph].y;
                    ph += kx;
                    if (ph >= L) ph -= L;
                }
                x1[o] = make_float2(re, im);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * L * wpl; k += blockDim.x) rows[k] = 0u;
        if (do_sk) {
            // m^[ky][kx] = sum_iy x1[iy][kx] e^{-2 pi i ky iy / L};  S += |m^|^2 / N
            for (int o = threadIdx.x; o < K1 * L; o += blockDim.x) {
                const int kx = o % K1, ky = o / K1;
                float re = 0.f, im = 0.f;
                int ph = 0;
                for (int iy = 0; iy < L; ++iy) {
                    const float2 a = x1[iy * K1 + kx], w = tw[ph];
                    re += a.x * w.x - a.y * w.y;
                    im += a.x * w.y + a.y * w.x;
                    ph += ky;
                    if (ph >= L) ph -= L;
                }
                const double v = double(re * re + im * im) / double(N);
                const int k = ky * L + kx;
                const bool mirror = kx > 0 && 2 * kx < L;
                const int km = (ky == 0 ? 0 : L - ky) * L + (L - kx);
                if (sk_smem) {
                    skacc[k] += v;
                    if (mirror) skacc[km] += v;
                } else {
                    atomicAdd(&st.sk[cd.meas_off + k], v * chain_sign(st, c));
                    if (mirror) atomicAdd(&st.sk[cd.meas_off + km], v * chain_sign(st, c));
                }
            }
        }
        __syncthreads();
    }
    if (measure) {
        // sums weighted by the sweep's sign sgn(P_up) sgn(P_dn) (Eq. reweight; +1 without
        // permutations), negative contributions in two's complement
        const int sgn = chain_sign(st, c);
        auto wsum = [&](unsigned long long v) { return sgn > 0 ? v : 0ull - v; };
        MeasAcc &acc = st.meas[c];
        block_add_u64(wsum(n_acc), &acc.n_sum, red);
        block_add_u64(wsum(d_acc), &acc.d_sum, red);
        block_add_u64(wsum(m2_acc), &acc.m2_sum, red);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicAdd(&acc.samples, 1ull);
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc.sign_sum), (unsigned long long)(long long)sgn);
        }
        if (do_sk && sk_smem)
            for (int k = threadIdx.x; k < N; k += blockDim.x) atomicAdd(&st.sk[cd.meas_off + k], skacc[k] * sgn);
    }
}

// Grouped form (lattices up to kGroupMaxL): one CTA per (chain, group of S consecutive
// slices), the slices handled together: every loop below runs over (slice, item) of the
// whole group, so a small lattice still fills the CTA's threads.  For every site of a slice:
//   m = n_up - n_dn;  s = +1 iff u < P(s=+1|m) = 1/(1+exp(-2 lambda m))  (FP64 compare),
// written bit-packed by rows and by columns; the histogram is cleared for the next
// sweep.  With `measure`, the slice's n, n_up n_dn, m^2 and |m^(k)|^2/N are added to
// the chain's accumulators (m^ by a direct separable DFT in FP32; each k sums the group's
// slices in slice order).
__global__ void __launch_bounds__(kSliceThreads) slice_group_kernel(DevState st, int S, int measure) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N, M = cd.M, wpl = cd.wpl;
    const int l_begin = blockIdx.x * S;
    if (l_begin >= M) return;
    const int ns = min(M, l_begin + S) - l_begin;  // slices of this CTA
    const uint64_t sweep = *st.sweep;
    const double lam = cd.lam;
    const ChainTab &tb = st.tabs[c];
    const int K1 = L / 2 + 1;  // kx = 0 .. L/2

    const bool do_sk = measure != 0;
    const bool sk_smem = N <= kSkSmemMaxN;
    const SliceSmem lay = slice_smem_layout(L, wpl, S, true);
    uint32_t *rows = reinterpret_cast<uint32_t *>(smem_raw + lay.rows);  // [S][2][L][wpl]
    unsigned long long *red = reinterpret_cast<unsigned long long *>(smem_raw + lay.red);
    double *pp = reinterpret_cast<double *>(smem_raw + lay.pp);         // P(s=+1 | m), |m| <= kPTab
    float *ms = reinterpret_cast<float *>(smem_raw + lay.ms);            // [S][N] m of the slices
    float2 *x1 = reinterpret_cast<float2 *>(smem_raw + lay.x1);          // [S][L][K1] row DFTs
    float2 *tw = reinterpret_cast<float2 *>(smem_raw + lay.tw);          // [L] e^{-2 pi i j / L}
    double *skacc = reinterpret_cast<double *>(smem_raw + lay.sk);       // [N]
    const int bits = 2 * L * wpl;  // words of one slice's rows and columns

    for (int k = threadIdx.x; k < ns * bits; k += blockDim.x) rows[k] = 0u;
    for (int k = threadIdx.x; k < 2 * kPTab + 1; k += blockDim.x) pp[k] = tb.pplus[k];
    if (do_sk) {
        for (int j = threadIdx.x; j < L; j += blockDim.x) {
            float sn, co;
            sincospif(2.0f * float(j) / float(L), &sn, &co);
            tw[j] = make_float2(co, -sn);
        }
        if (sk_smem)
            for (int k = threadIdx.x; k < N; k += blockDim.x) skacc[k] = 0.0;
    }
    __syncthreads();

    unsigned long long n_acc = 0, d_acc = 0, m2_acc = 0;
    int *hu_base = st.hist + cd.h_off;
    int *hd_base = hu_base + (long long)M * N;
    uint32_t *srow_g = st.sbits + cd.s_off;
    uint32_t *scol_g = srow_g + (long long)M * L * wpl;

    if (cd.gauss) {
        // Gaussian field: sigma ~ N(a (n_up + n_dn - 1/2), 1), uniforms j = 2x, 2x+1
        const int npairs = (N + 1) >> 1;
        for (int it = threadIdx.x; it < ns * npairs; it += blockDim.x) {
            const int sl = it / npairs, pr = it - sl * npairs, l = l_begin + sl;
            int *hu = hu_base + (long long)l * N;
            int *hd = hd_base + (long long)l * N;
            const u64x4 w4 = philox4x64_10((uint64_t)pr, (uint64_t)l, 1, sweep, cd.seed, 0);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int x = 2 * pr + j;
                if (x >= N) break;
                const int nu = hu[x], nd = hd[x];
                hu[x] = 0;
                hd[x] = 0;
                const int m = nu - nd;
                put_gauss(st, cd, l, x, cd.gcoup * (double(nu + nd) - 0.5) + box_muller(w4.v[2 * j], w4.v[2 * j + 1]));
                if (measure) {
                    n_acc += (unsigned long long)(nu + nd);
                    d_acc += (unsigned long long)(nu * nd);
                    m2_acc += (unsigned long long)(m * m);
                    if (do_sk) ms[sl * N + x] = float(m);
                }
            }
        }
    } else {
        const int nquads = (N + 3) >> 2;
        for (int it = threadIdx.x; it < ns * nquads; it += blockDim.x) {
            const int sl = it / nquads, qd = it - sl * nquads, l = l_begin + sl;
            int *hu = hu_base + (long long)l * N;
            int *hd = hd_base + (long long)l * N;
            uint32_t *rw = rows + sl * bits, *cl = rw + L * wpl;
            const u64x4 w4 = philox4x64_10((uint64_t)qd, (uint64_t)l, 1, sweep, cd.seed, 0);
            // whole quads of 16-byte aligned counts move as one vector load and one store
            const bool vec = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(hu) | reinterpret_cast<uintptr_t>(hd)) & 15) == 0;
            int nuq[4], ndq[4];
            if (vec) {
                const int4 a4 = reinterpret_cast<const int4 *>(hu)[qd], b4 = reinterpret_cast<const int4 *>(hd)[qd];
                reinterpret_cast<int4 *>(hu)[qd] = make_int4(0, 0, 0, 0);
                reinterpret_cast<int4 *>(hd)[qd] = make_int4(0, 0, 0, 0);
                nuq[0] = a4.x; nuq[1] = a4.y; nuq[2] = a4.z; nuq[3] = a4.w;
                ndq[0] = b4.x; ndq[1] = b4.y; ndq[2] = b4.z; ndq[3] = b4.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int x = 4 * qd + j;
                    nuq[j] = x < N ? hu[x] : 0;
                    ndq[j] = x < N ? hd[x] : 0;
                    if (x < N) {
                        hu[x] = 0;
                        hd[x] = 0;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = 4 * qd + j;
                if (x >= N) break;
                const int nu = nuq[j], nd = ndq[j];
                const int m = nu - nd;
                const double pplus = (m >= -kPTab && m <= kPTab) ? pp[m + kPTab]
                                                                  : 1.0 / (1.0 + exp(-2.0 * lam * m));
                const bool up = u53(w4.v[j]) < pplus;
                const int ix = x % L, iy = x / L;
                if (up) {
                    atomicOr(&rw[iy * wpl + (ix >> 5)], 1u << (ix & 31));
                    atomicOr(&cl[ix * wpl + (iy >> 5)], 1u << (iy & 31));
                }
                if (measure) {
                    n_acc += (unsigned long long)(nu + nd);
                    d_acc += (unsigned long long)(nu * nd);
                    m2_acc += (unsigned long long)(m * m);
                    if (do_sk) ms[sl * N + x] = float(m);
                }
            }
        }
    }
    __syncthreads();
    if (!cd.gauss) {
        for (int k = threadIdx.x; k < ns * L * wpl; k += blockDim.x) {
            const int sl = k / (L * wpl), kk = k - sl * (L * wpl);
            const long long off = (long long)(l_begin + sl) * L * wpl + kk;
            srow_g[off] = rows[sl * bits + kk];
            scol_g[off] = rows[sl * bits + L * wpl + kk];
        }
    }
    // S(k) of a real field: m^(-k) = conj(m^(k)), so only kx = 0..L/2 is transformed and
    // |m^(L - kx, L - ky)|^2 = |m^(kx, ky)|^2 fills the other half
    if (do_sk) {
        // x1[sl][iy][kx] = sum_ix m[sl][iy][ix] e^{-2 pi i kx ix / L}
        for (int o = threadIdx.x; o < ns * K1 * L; o += blockDim.x) {
            const int sl = o / (K1 * L), r = o - sl * (K1 * L);
            const int kx = r % K1, iy = r / K1;
            const float *msl = ms + sl * N + iy * L;
            float re = 0.f, im = 0.f;
            int ph = 0;
            for (int ix = 0; ix < L; ++ix) {
                const float mv = msl[ix];
                re += mv * tw[ph].x;
                im += mv * tw[ph].y;
                ph += kx;
                if (ph >= L) ph -= L;
            }
            x1[o] = make_float2(re, im);
        }
        __syncthreads();
        // m^[ky][kx] = sum_iy x1[iy][kx] e^{-2 pi i ky iy / L} for every (slice, k) of the
        // group, |m^|^2 / N into vb; then S += the group's slices summed in slice order by the
        // thread that owns k
        double *vb = reinterpret_cast<double *>(smem_raw + lay.vb);
        for (int o = threadIdx.x; o < ns * K1 * L; o += blockDim.x) {
            const int sl = o / (K1 * L), r = o - sl * (K1 * L);
            const int kx = r % K1, ky = r / K1;
            const float2 *xs = x1 + sl * (K1 * L);
            float re = 0.f, im = 0.f;
            int ph = 0;
            for (int iy = 0; iy < L; ++iy) {
                const float2 a = xs[iy * K1 + kx], w = tw[ph];
                re += a.x * w.x - a.y * w.y;
                im += a.x * w.y + a.y * w.x;
                ph += ky;
                if (ph >= L) ph -= L;
            }
            vb[o] = double(re * re + im * im) / double(N);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < K1 * L; o += blockDim.x) {
            const int kx = o % K1, ky = o / K1;
            double v = 0.0;
            for (int sl = 0; sl < ns; ++sl) v += vb[sl * (K1 * L) + o];
            const int k = ky * L + kx;
            const bool mirror = kx > 0 && 2 * kx < L;
            const int km = (ky == 0 ? 0 : L - ky) * L + (L - kx);
            if (sk_smem) {
                skacc[k] += v;
                if (mirror) skacc[km] += v;
            } else {
                atomicAdd(&st.sk[cd.meas_off + k], v * chain_sign(st, c));
                if (mirror) atomicAdd(&st.sk[cd.meas_off + km], v * chain_sign(st, c));
            }
        }
        __syncthreads();
    }
    if (measure) {
        // sums weighted by the sweep's sign sgn(P_up) sgn(P_dn) (Eq. reweight; +1 without
        // permutations), negative contributions in two's complement
        const int sgn = chain_sign(st, c);
        auto wsum = [&](unsigned long long v) { return sgn > 0 ? v : 0ull - v; };
        MeasAcc &acc = st.meas[c];
        block_add_u64(wsum(n_acc), &acc.n_sum, red);
        block_add_u64(wsum(d_acc), &acc.d_sum, red);
        block_add_u64(wsum(m2_acc), &acc.m2_sum, red);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicAdd(&acc.samples, 1ull);
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc.sign_sum), (unsigned long long)(long long)sgn);
        }
        if (do_sk && sk_smem)
            for (int k = threadIdx.x; k < N; k += blockDim.x) atomicAdd(&st.sk[cd.meas_off + k], skacc[k] * sgn);
    }
}

// Slices per CTA for the context's largest lattice: `requested` (> 0), or with 0 the fastest
// measured on GB300 (Gibbs/measure ms per sweep): up to L = 12 the grouped form with 16
// slices (L = 8, M = 1024, 32 chains: 0.138 against 0.244 for the sequential form's best);
// beyond, the sequential form with 4 slices at L <= 16, 2 at L <= 48 and 1 above (0.182
// ms at L = 16, 0.178 at L = 32, 0.526 at L = 64).  Any value is capped by shared memory.
// The automatic grouped choice also leaves at least two CTAs per SM (work_slices = chains x
// the longest M): one L = 8 chain of M = 1024 takes 3 slices per CTA, not 16.
int slice_group(int max_L, int requested, long long work_slices, int num_sms) {
    const int wpl = (max_L + 31) / 32;
    const bool grouped = max_L <= kGroupMaxL;
    int S = requested > 0 ? requested : grouped ? 16 : max_L <= 16 ? 4 : max_L <= 48 ? 2 : 1;
    if (requested <= 0 && grouped && num_sms > 0)
        S = int(std::max(1LL, std::min<long long>(S, work_slices / (2LL * num_sms))));
    if (grouped)
        while (S > 1 && slice_smem_layout(max_L, wpl, S, true).total > kSliceSmemBudget) --S;
    return S;
}

static size_t slice_smem(int max_L, int S) {
    const int wpl = (max_L + 31) / 32;
    return max_L <= kGroupMaxL ? slice_smem_layout(max_L, wpl, S, true).total
                               : slice_smem_layout(max_L, wpl, 1, false).total;
}

cudaError_t configure_slice(int max_L, int S) {
    auto k = max_L <= kGroupMaxL ? slice_group_kernel : slice_kernel;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(slice_smem(max_L, S)));
}

cudaError_t launch_slice(const DevState &st, int nchains, int max_M, int max_L, int S, bool measure,
                         cudaStream_t stream) {
    const size_t sm = slice_smem(max_L, S);
    dim3 grid((max_M + S - 1) / S, nchains);
    if (max_L <= kGroupMaxL) slice_group_kernel<<<grid, kSliceThreads, sm, stream>>>(st, S, measure ? 1 : 0);
    else slice_kernel<<<grid, kSliceThreads, sm, stream>>>(st, S, measure ? 1 : 0);
    return cudaGetLastError();
}

// Initial state: s from Philox phase 3 (sweep = 2^64 - 1), +1 iff u < 1/2;
// worldline p of the up spin on the p-th site of sublattice A ((ix+iy) even, row-major)
// then of sublattice B, the down spin on B then A; every slice the same site.
__global__ void init_fields_kernel(DevState st) {
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N, M = cd.M, wpl = cd.wpl;
    uint32_t *srow = st.sbits + cd.s_off, *scol = srow + (long long)M * L * wpl;
    for (int l = blockIdx.x; l < M; l += gridDim.x) {
        for (int k = threadIdx.x; k < L * wpl; k += blockDim.x) {
            srow[(long long)l * L * wpl + k] = 0u;
            scol[(long long)l * L * wpl + k] = 0u;
        }
    }
    __syncthreads();
    if (cd.gauss) {
        // standard normal sigma from phase 3 (sweep 2^64-1), uniforms j = 2x, 2x+1
        for (int l = blockIdx.x; l < M; l += gridDim.x)
            for (int x = threadIdx.x; x < N; x += blockDim.x) {
                const u64x4 w4 = philox4x64_10((uint64_t)(x >> 1), (uint64_t)l, 3, ~0ull, cd.seed, 0);
                const int j = 2 * (x & 1);
                put_gauss(st, cd, l, x, box_muller(w4.v[j], w4.v[j + 1]));
            }
        return;
    }
    for (int l = blockIdx.x; l < M; l += gridDim.x) {
        for (int x = threadIdx.x; x < N; x += blockDim.x) {
            const u64x4 w4 = philox4x64_10((uint64_t)(x >> 2), (uint64_t)l, 3, ~0ull, cd.seed, 0);
            if (u53(w4.v[x & 3]) < 0.5) {
                const int ix = x % L, iy = x / L;
                atomicOr(&srow[((long long)l * L + iy) * wpl + (ix >> 5)], 1u << (ix & 31));
                atomicOr(&scol[((long long)l * L + ix) * wpl + (iy >> 5)], 1u << (iy & 31));
            }
        }
    }
}

__global__ void init_paths_kernel(DevState st) {
    const int c = blockIdx.x;
    const ChainDev &cd = st.chains[c];
    const int sg = threadIdx.x;  // 0 up, 1 down
    if (sg > 1) return;
    const int L = cd.L, N = cd.N, M = cd.M;
    int p = 0;
    for (int pass = 0; pass < 2 && p < cd.Nsig; ++pass) {
        const int want = (sg == 0) ? pass : 1 - pass;
        for (int x = 0; x < N && p < cd.Nsig; ++x) {
            if (((x % L) + (x / L)) % 2 != want) continue;
            int16_t *xp = st.x + cd.x_off + ((long long)sg * cd.Nsig + p) * M;
            for (int l = 0; l < M; ++l) xp[l] = int16_t(x);
            ++p;
        }
    }
    if (sg == 0) st.anchor[c] = -1;
}

cudaError_t launch_init_state(const DevState &st, int nchains, cudaStream_t stream) {
    init_fields_kernel<<<dim3(1, nchains), 256, 0, stream>>>(st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    init_paths_kernel<<<nchains, 32, 0, stream>>>(st);
    return cudaGetLastError();
}

__global__ void advance_kernel(DevState st) { *st.sweep += 1ull; }

// W = exp(a sigma) again for chain c (after a change of a)
__global__ void gauss_w_kernel(DevState st, int c) {
    const ChainDev &cd = st.chains[c];
    const long long MN = (long long)cd.M * cd.N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < MN; k += (long long)gridDim.x * blockDim.x)
        put_gauss(st, cd, int(k / cd.N), int(k % cd.N), st.gsig[cd.g_off + k]);
}

cudaError_t launch_gauss_w(const DevState &st, int chain, int M, int N, cudaStream_t stream) {
    const long long MN = (long long)M * N;
    gauss_w_kernel<<<int(std::min<long long>((MN + 255) / 256, 1024)), 256, 0, stream>>>(st, chain);
    return cudaGetLastError();
}

cudaError_t launch_advance(const DevState &st, cudaStream_t stream) {
    advance_kernel<<<1, 1, 0, stream>>>(st);
    return cudaGetLastError();
}

// C(r) = (1/N) sum_k cos(k.r) S(k) with S(k) = sk[k] / (4 samples M) (S^z = m/2), by
// separable passes (O(N L) per chain instead of O(N^2)):
//   A[ky][rx] = sum_kx S(kx, ky) cos(2 pi kx rx / L),  B[ky][rx] = sum_kx S(kx, ky) sin(...),
//   C(rx, ry) = (1/N) sum_ky A[ky][rx] cos(2 pi ky ry / L) - B[ky][rx] sin(2 pi ky ry / L).
// Phases are reduced mod L before the trigonometric call, so every factor is exact to
// rounding.  Sums are sign-reweighted (divided by the sum of signs, the sample count
// without permutations).
// src (nullable): per-chain input in place of the accumulated |m(k)|^2 (the open-path sums
// for n_k, which take the same separable transform with k and r exchanged)
__global__ void readout_rows_kernel(DevState st, const double *src, double *tmp) {
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N;
    const double *sk = (src ? src : st.sk) + cd.meas_off;
    double *A = tmp + 2 * cd.meas_off, *B = A + N;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < N; o += gridDim.x * blockDim.x) {
        const int rx = o % L, ky = o / L;
        double a = 0.0, b = 0.0;
        int ph = 0;
        for (int kx = 0; kx < L; ++kx) {
            double sn, cs;
            sincospi(2.0 * double(ph) / double(L), &sn, &cs);
            a += sk[ky * L + kx] * cs;
            b += sk[ky * L + kx] * sn;
            ph += rx;
            if (ph >= L) ph -= L;
        }
        A[o] = a;
        B[o] = b;
    }
}

__global__ void readout_cols_kernel(DevState st, const double *tmp, double *cr_out, double *sk_out) {
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N;
    const long long ns = st.meas[c].sign_sum;
    const double norm = ns ? 1.0 / (4.0 * double(ns) * cd.M) : 0.0;
    const double *sk = st.sk + cd.meas_off;
    const double *A = tmp + 2 * cd.meas_off, *B = A + N;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        const int rx = r % L, ry = r / L;
        double acc = 0.0;
        int ph = 0;
        for (int ky = 0; ky < L; ++ky) {
            double sn, cs;
            sincospi(2.0 * double(ph) / double(L), &sn, &cs);
            acc += A[ky * L + rx] * cs - B[ky * L + rx] * sn;
            ph += ry;
            if (ph >= L) ph -= L;
        }
        cr_out[cd.meas_off + r] = acc * norm / N;
        sk_out[cd.meas_off + r] = sk[r] * norm;
    }
}

cudaError_t launch_readout(const DevState &st, int nchains, int max_N, double *cr_out, double *sk_out,
                           double *tmp, cudaStream_t stream) {
    dim3 grid((max_N + 255) / 256, nchains);
    readout_rows_kernel<<<grid, 256, 0, stream>>>(st, nullptr, tmp);
    readout_cols_kernel<<<grid, 256, 0, stream>>>(st, tmp, cr_out, sk_out);
    return cudaGetLastError();
}

// n_k = (1/N) sum_r cos(k.r) A(r) and the one-body density matrix per site A(r) / N, from the
// open-path sums A(r) = sum over sweeps of sign x sum_{sigma,p} alpha_end(x_e + r) / alpha_end(x_e),
// divided by the sum of signs (Sec. 4, "Observables"; the paper's n_k with
// sum_x <c^dag_{x+r} c_x> = A(r)): the same two separable passes as C(r)
__global__ void readout_open_cols_kernel(DevState st, const double *tmp, double *nk_out, double *dm_out) {
    const int c = blockIdx.y;
    const ChainDev &cd = st.chains[c];
    const int L = cd.L, N = cd.N;
    const long long ns = st.meas[c].sign_sum;
    const double norm = ns ? 1.0 / (double(ns) * N) : 0.0;
    const double *A = tmp + 2 * cd.meas_off, *B = A + N;
    const double *acc = st.open_acc + cd.meas_off;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const int kx = k % L, ky = k / L;
        double s = 0.0;
        int ph = 0;
        for (int ry = 0; ry < L; ++ry) {
            double sn, cs;
            sincospi(2.0 * double(ph) / double(L), &sn, &cs);
            s += A[ry * L + kx] * cs - B[ry * L + kx] * sn;
            ph += ky;
            if (ph >= L) ph -= L;
        }
        nk_out[cd.meas_off + k] = s * norm;
        dm_out[cd.meas_off + k] = acc[k] * norm;
    }
}

cudaError_t launch_readout_open(const DevState &st, int nchains, int max_N, double *nk_out, double *dm_out,
                                double *tmp, cudaStream_t stream) {
    dim3 grid((max_N + 255) / 256, nchains);
    readout_rows_kernel<<<grid, 256, 0, stream>>>(st, st.open_acc, tmp);
    readout_open_cols_kernel<<<grid, 256, 0, stream>>>(st, tmp, nk_out, dm_out);
    return cudaGetLastError();
}

}  // namespace hqmc
