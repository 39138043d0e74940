// device_common.cuh -- register-resident complex FFT of one lattice line, Philox4x64-10,
// and small warp helpers shared by the sm_103a kernels of this library.
#pragma once

#include <cstdint>
#include <type_traits>

namespace hqmc {

// ---------------------------------------------------------------------------------
// complex value of one lattice line element; .x and .y carry two worldlines of the
// same spin (the propagator and the slice potential are real, so the two never mix)
// ---------------------------------------------------------------------------------
template <typename T>
struct cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.x * s, a.y * s}; }
// multiply by +i or -i
template <int SGN, typename T>
__device__ __forceinline__ cplx<T> cmul_i(cplx<T> a) {
    if constexpr (SGN > 0) return {-a.y, a.x};
    else return {a.y, -a.x};
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

// v * exp(SGN * 2 pi i K / NN), with the trivial angles done without multiplies
template <int SGN, int K, int NN, typename T>
__device__ __forceinline__ cplx<T> twiddle(cplx<T> v) {
    constexpr int k = ((K % NN) + NN) % NN;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (2 * k == NN) {
        return {-v.x, -v.y};
    } else if constexpr (4 * k == NN) {
        return cmul_i<SGN>(v);
    } else if constexpr (4 * k == 3 * NN) {
        return cmul_i<-SGN>(v);
    } else {
        constexpr T c = T(ct::cos2pi(k, NN));
        constexpr T s = T(SGN * ct::sin2pi(k, NN));
        return {v.x * c - v.y * s, v.x * s + v.y * c};
    }
}

// small DFTs of the mixed-radix decomposition (natural order in and out)
template <int SGN, typename T>
__device__ __forceinline__ void dft2(cplx<T> &a0, cplx<T> &a1) {
    cplx<T> t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}
template <int SGN, typename T>
__device__ __forceinline__ void dft3(cplx<T> &a0, cplx<T> &a1, cplx<T> &a2) {
    constexpr T h = T(-0.5);
    constexpr T s = T(SGN * 0.86602540378443864676372317075293618);
    cplx<T> sum = cadd(a1, a2), dif = csub(a1, a2);
    cplx<T> base = {a0.x + h * sum.x, a0.y + h * sum.y};
    cplx<T> rot = {-s * dif.y, s * dif.x};  // i s (a1 - a2)
    a0 = cadd(a0, sum);
    a1 = cadd(base, rot);
    a2 = csub(base, rot);
}
template <int SGN, typename T>
__device__ __forceinline__ void dft4(cplx<T> &a0, cplx<T> &a1, cplx<T> &a2, cplx<T> &a3) {
    cplx<T> s02 = cadd(a0, a2), d02 = csub(a0, a2);
    cplx<T> s13 = cadd(a1, a3), d13 = cmul_i<SGN>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

template <int N>
__host__ __device__ constexpr int first_radix() {
    return (N % 4 == 0 && N > 4) ? 4 : (N % 2 == 0 ? 2 : 3);
}

// In-place DFT of N register values, X[k] = sum_n a[n] exp(SGN 2 pi i n k / N),
// unnormalised, by recursive decimation in time (N = R * Ms, R in {2, 3, 4}).
template <int N, int SGN, typename T>
__device__ __forceinline__ void fft(cplx<T> (&a)[N]) {
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
        cplx<T> sub[R][Ms];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < Ms; ++m) sub[r][m] = a[R * m + r];
#pragma unroll
        for (int r = 0; r < R; ++r) fft<Ms, SGN>(sub[r]);
        static_for<0, Ms>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            cplx<T> t[R];
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

// Periodic convolution of one line with the even real kernel whose DFT is gh[k]
// (gh already divided by N): a <- IDFT(gh . DFT(a)).  gh holds k = 0..N/2.
template <int N, typename T>
__device__ __forceinline__ void conv_line(cplx<T> (&a)[N], const T (&gh)[N / 2 + 1]) {
    fft<N, -1>(a);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const T w = gh[k <= N / 2 ? k : N - k];
        a[k].x *= w;
        a[k].y *= w;
    }
    fft<N, +1>(a);
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

}  // namespace hqmc
