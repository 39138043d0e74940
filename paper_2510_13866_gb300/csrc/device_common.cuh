// device_common.cuh -- two-worldline vector arithmetic, a register-resident complex FFT
// over those vectors, Philox4x64-10, and small warp helpers shared by the sm_103a kernels
// of this library.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace hqmc {

// ---------------------------------------------------------------------------------
// Two same-spin worldlines travel together through the filter: component .x belongs to
// one, .y to the other.  The propagator and the slice potential are real, so every
// operation of the filter acts on both components alike.  In FP32 that is one packed
// f32x2 instruction (FADD2 / FMUL2 / FFMA2, sm_100 and later) for the pair.
// ---------------------------------------------------------------------------------
template <typename T>
struct vec2_of;
template <>
struct vec2_of<float> {
    using type = float2;
};
template <>
struct vec2_of<double> {
    using type = double2;
};
template <typename T>
using vec2_t = typename vec2_of<T>::type;

// packed FP32 pair arithmetic (FADD2 / FMUL2 / FFMA2; subtraction as PTX sub.rn.f32x2)
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// the pair is assembled from and split into its two f32 halves inside the asm, so no
// value is reinterpreted through a pointer of another type (which would break when the
// compiler keeps the pair in local memory)
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 vsplat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsplat(double s) { return make_double2(s, s); }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }

// One worldline per thread: the same operations on plain scalars (the FMA pipe does the
// same work per flop as with the packed pair; only the issue count differs).
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vzero(float) { return 0.f; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vzero(double) { return 0.0; }

// a constant broadcast to the element type V (a pair or a scalar)
template <typename V>
struct splat_t;
template <>
struct splat_t<float2> {
    __device__ static float2 of(float s) { return make_float2(s, s); }
};
template <>
struct splat_t<double2> {
    __device__ static double2 of(double s) { return make_double2(s, s); }
};
template <>
struct splat_t<float> {
    __device__ static float of(float s) { return s; }
};
template <>
struct splat_t<double> {
    __device__ static double of(double s) { return s; }
};
template <typename V, typename S>
__device__ __forceinline__ V splat(S s) { return splat_t<V>::of(s); }

// (alpha_k, beta_k) broadcast pairs of conv_line's spectral mix, read from shared memory
// at every use (a volatile load: kept out of registers across the slice loop, where
// they would cost L registers)
__device__ __forceinline__ void load_mix(const float2 *mix, int k, float2 &al, float2 &be) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(mix + 2 * k));
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(al.x), "=f"(al.y), "=f"(be.x), "=f"(be.y) : "r"(a));
}
__device__ __forceinline__ void load_mix(const double2 *mix, int k, double2 &al, double2 &be) {
    al = mix[2 * k];
    be = mix[2 * k + 1];
}
__device__ __forceinline__ float2 load_mix1(const float2 *mix, int k) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(mix + k));
    float2 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(a));
    return r;
}
__device__ __forceinline__ double2 load_mix1(const double2 *mix, int k) { return mix[k]; }
// scalar tables (one worldline per thread): alpha_k, beta_k interleaved, or gh_k / L
__device__ __forceinline__ void load_mix(const float *mix, int k, float &al, float &be) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(mix + 2 * k));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(al), "=f"(be) : "r"(a));
}
__device__ __forceinline__ void load_mix(const double *mix, int k, double &al, double &be) {
    al = mix[2 * k];
    be = mix[2 * k + 1];
}
__device__ __forceinline__ float load_mix1(const float *mix, int k) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(mix + k));
    float r;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a));
    return r;
}
__device__ __forceinline__ double load_mix1(const double *mix, int k) { return mix[k]; }

// complex number whose real and imaginary parts are two-worldline vectors
template <typename V>
struct cvec {
    V re, im;
};

// One FP32 worldline per thread: a complex add or subtract takes (re, im) as one f32x2
// pair (one FADD2).  Products that cross the halves (re with im) stay scalar: packed forms
// that swapped the two halves of a pair gave results that depended on register allocation
// and differed between identical runs on sm_103a.
__device__ __forceinline__ float2 pk(const cvec<float> &a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ cvec<float> upk(float2 v) { return {v.x, v.y}; }

template <typename V>
__device__ __forceinline__ cvec<V> cv_add(cvec<V> a, cvec<V> b) {
    if constexpr (std::is_same<V, float>::value) return upk(__fadd2_rn(pk(a), pk(b)));
    else return {vadd(a.re, b.re), vadd(a.im, b.im)};
}
template <typename V>
__device__ __forceinline__ cvec<V> cv_sub(cvec<V> a, cvec<V> b) {
    if constexpr (std::is_same<V, float>::value) return upk(vsub(pk(a), pk(b)));
    else return {vsub(a.re, b.re), vsub(a.im, b.im)};
}
// multiply by +i (SGN > 0) or -i
template <int SGN, typename V>
__device__ __forceinline__ cvec<V> cv_muli(cvec<V> a) {
    // i (re, im) = (-im, re), -i (re, im) = (im, -re)
    if constexpr (SGN > 0) return {vsub(vzero(a.im), a.im), a.re};
    else return {a.im, vsub(vzero(a.re), a.re)};
}

// ---------------------------------------------------------------------------------
// compile-time cos/sin of 2 pi k / n: octant reduction in integers, then a Taylor
// series on [0, pi/4] (error below 1e-20), evaluated by the compiler.
// ---------------------------------------------------------------------------------
namespace ct {
constexpr double kPi = 3.141592653589793238462643383279502884;
__host__ __device__ constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / double((2 * n) * (2 * n + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / double((2 * n - 1) * (2 * n));
        sum += term;
    }
    return sum;
}
// angle 2 pi k / n = (pi/4) * (8k/n): octant o = floor(8k/n), phi = (pi/4) f/n
__host__ __device__ constexpr double cos2pi(int k, int n) {
    k = ((k % n) + n) % n;
    long long r = 8LL * k;
    int o = int(r / n);
    double f = double(r - (long long)o * n);
    double phi = (kPi / 4) * f / n, cphi = (kPi / 4) * (double(n) - f) / n;
    switch (o) {
        case 0: return taylor_cos(phi);
        case 1: return taylor_sin(cphi);
        case 2: return -taylor_sin(phi);
        case 3: return -taylor_cos(cphi);
        case 4: return -taylor_cos(phi);
        case 5: return -taylor_sin(cphi);
        case 6: return taylor_sin(phi);
        default: return taylor_cos(cphi);
    }
}
__host__ __device__ constexpr double sin2pi(int k, int n) {
    k = ((k % n) + n) % n;
    long long r = 8LL * k;
    int o = int(r / n);
    double f = double(r - (long long)o * n);
    double phi = (kPi / 4) * f / n, cphi = (kPi / 4) * (double(n) - f) / n;
    switch (o) {
        case 0: return taylor_sin(phi);
        case 1: return taylor_cos(cphi);
        case 2: return taylor_cos(phi);
        case 3: return taylor_sin(cphi);
        case 4: return -taylor_sin(phi);
        case 5: return -taylor_cos(cphi);
        case 6: return -taylor_cos(phi);
        default: return -taylor_sin(cphi);
    }
}
}  // namespace ct

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

template <typename V>
struct scalar_of;
template <>
struct scalar_of<float2> {
    using type = float;
};
template <>
struct scalar_of<double2> {
    using type = double;
};
template <>
struct scalar_of<float> {
    using type = float;
};
template <>
struct scalar_of<double> {
    using type = double;
};

// v * exp(SGN * 2 pi i K / NN), with the trivial angles done without multiplies
template <int SGN, int K, int NN, typename V>
__device__ __forceinline__ cvec<V> twiddle(cvec<V> v) {
    using T = typename scalar_of<V>::type;
    constexpr int k = ((K % NN) + NN) % NN;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (2 * k == NN) {
        if constexpr (std::is_same<V, float>::value) return upk(__fmul2_rn(pk(v), make_float2(-1.f, -1.f)));
        else return {vsub(vzero(v.re), v.re), vsub(vzero(v.im), v.im)};
    } else if constexpr (4 * k == NN) {
        return cv_muli<SGN>(v);
    } else if constexpr (4 * k == 3 * NN) {
        return cv_muli<-SGN>(v);
    } else {
        constexpr T c = T(ct::cos2pi(k, NN));
        constexpr T s = T(SGN * ct::sin2pi(k, NN));
        // (re + i im)(c + i s) = (c re - s im) + i (s re + c im)
        return {vfma(v.re, splat<V>(c), vmul(v.im, splat<V>(-s))), vfma(v.re, splat<V>(s), vmul(v.im, splat<V>(c)))};
    }
}

// small DFTs of the mixed-radix decomposition (natural order in and out)
template <int SGN, typename V>
__device__ __forceinline__ void dft2(cvec<V> &a0, cvec<V> &a1) {
    cvec<V> t = a0;
    a0 = cv_add(t, a1);
    a1 = cv_sub(t, a1);
}
template <int SGN, typename V>
__device__ __forceinline__ void dft3(cvec<V> &a0, cvec<V> &a1, cvec<V> &a2) {
    using T = typename scalar_of<V>::type;
    constexpr T h = T(-0.5);
    constexpr T s = T(SGN * 0.86602540378443864676372317075293618);
    cvec<V> sum = cv_add(a1, a2), dif = cv_sub(a1, a2);
    cvec<V> base, rot;
    if constexpr (std::is_same<V, float>::value) {
        base = upk(__ffma2_rn(pk(sum), make_float2(h, h), pk(a0)));
    } else {
        base = {vfma(sum.re, splat<V>(h), a0.re), vfma(sum.im, splat<V>(h), a0.im)};
    }
    rot = {vmul(dif.im, splat<V>(-s)), vmul(dif.re, splat<V>(s))};  // i s (a1 - a2)
    a0 = cv_add(a0, sum);
    a1 = cv_add(base, rot);
    a2 = cv_sub(base, rot);
}
template <int SGN, typename V>
__device__ __forceinline__ void dft4(cvec<V> &a0, cvec<V> &a1, cvec<V> &a2, cvec<V> &a3) {
    const cvec<V> s02 = cv_add(a0, a2), d02 = cv_sub(a0, a2);
    const cvec<V> s13 = cv_add(a1, a3), d13 = cv_sub(a1, a3);
    a0 = cv_add(s02, s13);
    a2 = cv_sub(s02, s13);
    // a1 = d02 + (SGN i) d13, a3 = d02 - (SGN i) d13, with the rotation folded into add/sub
    if constexpr (SGN > 0) {
        a1 = {vsub(d02.re, d13.im), vadd(d02.im, d13.re)};
        a3 = {vadd(d02.re, d13.im), vsub(d02.im, d13.re)};
    } else {
        a1 = {vadd(d02.re, d13.im), vsub(d02.im, d13.re)};
        a3 = {vsub(d02.re, d13.im), vadd(d02.im, d13.re)};
    }
}

template <int N>
__host__ __device__ constexpr int first_radix() {
    return (N % 4 == 0 && N > 4) ? 4 : (N % 2 == 0 ? 2 : 3);
}

// In-place DFT of N register values, X[k] = sum_n a[n] exp(SGN 2 pi i n k / N),
// unnormalised, by recursive decimation in time (N = R * Ms, R in {2, 3, 4}).
template <int N, int SGN, typename V>
__device__ __forceinline__ void fft(cvec<V> (&a)[N]) {
    if constexpr (N == 1) {
    } else if constexpr (N == 2) {
        dft2<SGN>(a[0], a[1]);
    } else if constexpr (N == 3) {
        dft3<SGN>(a[0], a[1], a[2]);
    } else if constexpr (N == 4) {
        dft4<SGN>(a[0], a[1], a[2], a[3]);
    } else {
        constexpr int R = first_radix<N>();
        constexpr int Ms = N / R;
        static_assert(R * Ms == N, "radix");
        cvec<V> sub[R][Ms];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < Ms; ++m) sub[r][m] = a[R * m + r];
#pragma unroll
        for (int r = 0; r < R; ++r) fft<Ms, SGN>(sub[r]);
        static_for<0, Ms>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            cvec<V> t[R];
            t[0] = sub[0][k];
            static_for<1, R>([&](auto RI) {
                constexpr int r = decltype(RI)::value;
                t[r] = twiddle<SGN, r * k, N>(sub[r][k]);
            });
            if constexpr (R == 2) dft2<SGN>(t[0], t[1]);
            else if constexpr (R == 3) dft3<SGN>(t[0], t[1], t[2]);
            else dft4<SGN>(t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int q = 0; q < R; ++q) a[k + Ms * q] = t[q];
        });
    }
}

// Building blocks of conv_line with the spectrum exposed, for passes that apply more
// than one line kernel to the same line (the adjoint applies g and dg/dt):
//   line_fwd: spectrum of the line (even L: DFT_n of the packed line, odd L: DFT_L)
//   spec_mix: out = mix(in), or out += mix(in) with ACC (out must not alias in)
//   line_inv: the line whose spectrum is z (the 1/n or 1/L factor is in the mix)
template <int L>
struct line_spec {
    static constexpr int K = (L % 2 == 0) ? L / 2 : L;
};

template <int L, typename V>
__device__ __forceinline__ void line_fwd(const V (&v)[L], cvec<V> (&z)[line_spec<L>::K]) {
    if constexpr (L % 2 == 0) {
#pragma unroll
        for (int m = 0; m < L / 2; ++m) z[m] = {v[2 * m], v[2 * m + 1]};
    } else {
#pragma unroll
        for (int m = 0; m < L; ++m) z[m] = {v[m], vzero(v[m])};
    }
    fft<line_spec<L>::K, -1>(z);
}

template <int L, typename V>
__device__ __forceinline__ void line_inv(cvec<V> (&z)[line_spec<L>::K], V (&v)[L]) {
    fft<line_spec<L>::K, +1>(z);
    if constexpr (L % 2 == 0) {
#pragma unroll
        for (int m = 0; m < L / 2; ++m) {
            v[2 * m] = z[m].re;
            v[2 * m + 1] = z[m].im;
        }
    } else {
#pragma unroll
        for (int m = 0; m < L; ++m) v[m] = z[m].re;
    }
}

template <int L, bool ACC, typename V>
__device__ __forceinline__ void spec_mix(cvec<V> (&out)[line_spec<L>::K], const cvec<V> (&in)[line_spec<L>::K],
                                         const V *mix) {
    if constexpr (L % 2 == 0) {
        constexpr int n = L / 2;
        static_for<0, n>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            constexpr int kp = (n - k) % n;
            V al, be;
            load_mix(mix, k, al, be);
            const V re = vfma(in[k].re, al, vmul(in[kp].im, be));
            const V im = vfma(in[k].im, al, vmul(in[kp].re, be));
            if constexpr (ACC) out[k] = {vadd(out[k].re, re), vadd(out[k].im, im)};
            else out[k] = {re, im};
        });
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const V w = load_mix1(mix, k);
            if constexpr (ACC) out[k] = {vfma(in[k].re, w, out[k].re), vfma(in[k].im, w, out[k].im)};
            else out[k] = {vmul(in[k].re, w), vmul(in[k].im, w)};
        }
    }
}

// in-place spectral mix (even L: the pairs (k, n-k) are read before either is written)
template <int L, typename V>
__device__ __forceinline__ void spec_mix_inplace(cvec<V> (&z)[line_spec<L>::K], const V *mix) {
    if constexpr (L % 2 == 0) {
        constexpr int n = L / 2;
        static_for<0, n>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            constexpr int kp = (n - k) % n;
            if constexpr (k == kp) {
                V al, be;
                load_mix(mix, k, al, be);
                const cvec<V> zk = z[k];
                z[k] = {vfma(zk.re, al, vmul(zk.im, be)), vfma(zk.im, al, vmul(zk.re, be))};
            } else if constexpr (k < kp) {
                V a0, b0, a1, b1;
                load_mix(mix, k, a0, b0);
                load_mix(mix, kp, a1, b1);
                const cvec<V> zk = z[k], zp = z[kp];
                z[k] = {vfma(zk.re, a0, vmul(zp.im, b0)), vfma(zk.im, a0, vmul(zp.re, b0))};
                z[kp] = {vfma(zp.re, a1, vmul(zk.im, b1)), vfma(zp.im, a1, vmul(zk.re, b1))};
            }
        });
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const V w = load_mix1(mix, k);
            z[k] = {vmul(z[k].re, w), vmul(z[k].im, w)};
        }
    }
}

// Periodic convolution of one lattice line of both worldlines with the even real line
// kernel g: v <- g * v.
//
// Even L: the line is packed as n = L/2 complex values z_m = v_{2m} + i v_{2m+1}.  With
// Z = DFT_n(z), the half-spectrum identities of a real DFT give the packed transform of
// the convolved line directly as
//     Z'_k = alpha_k Z_k + i beta_k conj(Z_{(n-k) mod n})
// with theta_k = 2 pi k / L, P_k = (gh_k + gh_{k+n}) / 2, Q_k = (gh_k - gh_{k+n}) / 2,
//     alpha_k = (P_k - Q_k sin theta_k) / n,   beta_k = Q_k cos theta_k / n,
// gh the L-point DFT of g; then z' = IDFT_n(Z') unpacks to the convolved line.  Two
// half-size complex FFTs per line, all arithmetic on two-worldline vectors.
// Odd L: full-size complex DFT of the real line, multiply by gh_k / L, inverse DFT.
// `mix` holds alpha_k, beta_k interleaved (even L) or gh_k / L (odd L), each already
// broadcast to both components.
template <int L, typename V>
__device__ __forceinline__ void conv_line(V (&v)[L], const V *mix) {
    cvec<V> z[line_spec<L>::K];
    line_fwd<L>(v, z);
    spec_mix_inplace<L>(z, mix);
    line_inv<L>(z, v);
}

// Line convolution of ONE worldline's line (scalar elements, even L) with a single FFT body:
// the inverse transform is conj(FFT(conj Z')), so both passes run the same forward FFT code
// (half the code of conv_line, which keeps the instruction cache warm at large L).  The
// spectral mix writes conj(Z') directly:
//     conj(Z'_k) = (al_k, -al_k) . Z_k + (be_k, -be_k) . (Im Z_{n-k}, Re Z_{n-k})
// with mixc[4k .. 4k+3] = (al_k, -al_k, be_k, -be_k) (al, be as in conv_line); the last
// conjugation is the sign of the odd elements.
template <int L, typename T>
__device__ __forceinline__ void conv_line_1fft(T (&v)[L], const T *mixc) {
    static_assert(L % 2 == 0, "even lines");
    constexpr int n = L / 2;
    cvec<T> z[n];
#pragma unroll
    for (int m = 0; m < n; ++m) z[m] = {v[2 * m], v[2 * m + 1]};
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        fft<n, -1>(z);
        if (pass == 0) {
            static_for<0, n>([&](auto KI) {
                constexpr int k = decltype(KI)::value;
                constexpr int kp = (n - k) % n;
                auto mixk = [&](const cvec<T> &zk, const cvec<T> &zp, int kk) -> cvec<T> {
                    T a, na, b, nb;
                    if constexpr (std::is_same<T, float>::value) {
                        const float4 c4 = reinterpret_cast<const float4 *>(mixc)[kk];
                        a = c4.x;
                        na = c4.y;
                        b = c4.z;
                        nb = c4.w;
                    } else {
                        a = mixc[4 * kk];
                        na = mixc[4 * kk + 1];
                        b = mixc[4 * kk + 2];
                        nb = mixc[4 * kk + 3];
                    }
                    return {fma(zk.re, a, zp.im * b), fma(zk.im, na, zp.re * nb)};
                };
                if constexpr (k == kp) {
                    z[k] = mixk(z[k], z[k], k);
                } else if constexpr (k < kp) {
                    const cvec<T> zk = z[k], zp = z[kp];
                    z[k] = mixk(zk, zp, k);
                    z[kp] = mixk(zp, zk, kp);
                }
            });
        }
    }
#pragma unroll
    for (int m = 0; m < n; ++m) {
        v[2 * m] = z[m].re;
        v[2 * m + 1] = -z[m].im;
    }
}

// The same line convolution as a direct periodic stencil, out[x] = sum_d g(d) v[x - d]
// over |d| <= R, R = min(kStencilR, (L-1)/2), with the d = L/2 term once for even
// L <= 2 kStencilR: the exact circulant up to L = 2 kStencilR + 1, beyond it g truncated
// at |d| = kStencilR (the comparison of a truncated separable stencil with the FFT).
// Every output is a sum of non-negative terms for non-negative input, so small values
// keep their relative accuracy instead of sitting on an FFT rounding floor.  g holds
// g(0..L-1) as scalars (shared memory).  The outputs go to dst[x * stride] (shared
// memory) as they are formed, so the input line is the only array held in registers.
constexpr int kStencilR = 6;
template <int L, typename V, typename T>
__device__ __forceinline__ void stencil_store(const V (&v)[L], const T *g, V *dst, int stride) {
    constexpr int R = ((L - 1) / 2 < kStencilR) ? (L - 1) / 2 : kStencilR;
    constexpr bool half = (L % 2 == 0) && (L / 2 <= kStencilR);
    V tap[R + 2];
#pragma unroll
    for (int d = 0; d <= R; ++d) tap[d] = vsplat(g[d]);
    if constexpr (half) tap[R + 1] = vsplat(g[L / 2]);
#pragma unroll
    for (int x = 0; x < L; ++x) {
        V acc = vmul(tap[0], v[x]);
#pragma unroll
        for (int d = 1; d <= R; ++d) acc = vfma(tap[d], vadd(v[(x - d + L) % L], v[(x + d) % L]), acc);
        if constexpr (half) acc = vfma(tap[R + 1], v[(x + L / 2) % L], acc);
        dst[x * stride] = acc;
    }
}

// ---------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), key (seed, 0)
// ---------------------------------------------------------------------------------
struct u64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return {{c0, c1, c2, c3}};
}

__device__ __forceinline__ double u53(uint64_t w) { return double(w >> 11) * 0x1.0p-53; }

// ---------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------
template <typename T>
struct fbits;
template <>
struct fbits<float> {
    // exponent e with 2^e <= v < 2^(e+1) for a positive normal v
    __device__ static int exponent(float v) { return int((__float_as_uint(v) >> 23) & 0xffu) - 127; }
    __device__ static float pow2(int e) { return __uint_as_float(uint32_t(e + 127) << 23); }
};
template <>
struct fbits<double> {
    __device__ static int exponent(double v) {
        return int((uint64_t(__double_as_longlong(v)) >> 52) & 0x7ffull) - 1023;
    }
    __device__ static double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
};

template <int W, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
    return v;
}
template <int W, typename T>
__device__ __forceinline__ T group_max(T v, unsigned mask) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        const T u = __shfl_xor_sync(mask, v, o, W);
        v = u > v ? u : v;
    }
    return v;
}

// Tolerance of a filter log-weight, relative to max(1, |log Z|), in the precision of the
// filter: 1e-5 for FP32, 1e-12 for FP64.
template <typename T>
__host__ __device__ constexpr double logw_tolerance() { return sizeof(T) == 4 ? 1e-5 : 1e-12; }

// Error estimate of one block's filter log-weight log alpha_end(x_end) + (sum of exponents) ln 2.
// The exponent sum is exact.  The FFT leaves every site of a slice with a rounding error of
// about eps log2(N) of the slice's largest value, so a site that ends kappa times below the
// largest, kappa = max_y alpha_end(y) / alpha_end(x_end), carries a relative error of about
// eps log2(N) kappa from each slice: eps log2(N) len kappa for a block of len slices, the end
// concentration standing in for every slice's (Hirsch fields).  The stencil form sums
// non-negative terms, so every site keeps its own relative accuracy and kappa is replaced by
// 1.  eps = 2^-24 (FP32), 2^-53 (FP64).  A non-positive end value gives +inf.  Against the
// oracle's direct convolution (48 random combinations and an equilibrated L = 32 state) the
// FP32 errors stay below 0.73 of it.  Gaussian-field units pass the sum over their slices
// of a one-sample estimate of each slice's concentration (gauss_sum_factor below) plus the
// end's, with len = 1.
template <typename T>
__device__ __forceinline__ double logw_err_estimate(double kappa, int len, int L, bool stencil) {
    const double eps = sizeof(T) == 4 ? 0x1.0p-24 : 0x1.0p-53;
    const double log2n = 2.0 * log2(double(L));
    const double k = stencil ? 1.0 : kappa;
    return eps * log2n * double(len > 0 ? len : 1) * k;
}

// Calibration factor of the sampled part of the Gaussian-field estimate.  FP64 flags only
// strongly concentrated units (the tolerance is 1e-12 against eps = 1.1e-16), where the
// one-sample conditional mean of each slice's concentration spreads most: over 1108 FP64
// log-weights of the random combinations the error reached 20.7 times the unscaled sum
// (99th percentile 5.7), while FP32 stayed below 0.3 of it.
template <typename T>
__host__ __device__ constexpr double gauss_sum_factor() { return sizeof(T) == 4 ? 1.0 : 32.0; }

// Ampere-style asynchronous global -> shared copies (16 or 8 bytes per lane).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace hqmc
