// peak.cu -- measured FP32 and FP64 fused multiply-add throughput of the current GPU: the
// denominators of the ALU rooflines of the FFBS kernels (their FFT and pointwise arithmetic
// is packed f32x2, FFMA2/FMUL2/FADD2) and of the plain FP64 form.
//
// Every thread runs kChains independent dependency chains of fused multiply-adds, so the
// FMA pipe never waits on a result.  The grid is one wave of kCtasPerSm resident CTAs of
// 256 threads on every SM.  The multiplier and addend come from the launch arguments and
// the chains' sums are stored, so nothing folds at compile time.  Each packed instruction
// counts 4 flops (two lanes of multiply-add), a scalar one 2.  The best of five timed
// launches, after one untimed, is reported.
#include <cuda_runtime.h>

#include "../../include/hqmc.h"

namespace hqmc {
namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kIters = 8192;
constexpr int kCtasPerSm = 4;

__global__ void __launch_bounds__(kThreads, kCtasPerSm) fma2_loop(float2 *out, float2 a, float2 b, int iters) {
    float2 acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = make_float2(float(threadIdx.x + j), float(blockIdx.x - j));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc[j] = __ffma2_rn(acc[j], a, b);
    }
    float2 s = acc[0];
#pragma unroll
    for (int j = 1; j < kChains; ++j) s = __fadd2_rn(s, acc[j]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) fma_loop(float *out, float a, float b, int iters) {
    float acc[2 * kChains];
#pragma unroll
    for (int j = 0; j < 2 * kChains; ++j) acc[j] = float(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 2 * kChains; ++j) acc[j] = fmaf(acc[j], a, b);
    }
    float s = acc[0];
#pragma unroll
    for (int j = 1; j < 2 * kChains; ++j) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) dfma_loop(double *out, double a, double b, int iters) {
    double acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = double(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc[j] = fma(acc[j], a, b);
    }
    double s = acc[0];
#pragma unroll
    for (int j = 1; j < kChains; ++j) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of five timed launches (after one untimed) of `launch` on a private stream, in ms
template <typename F>
int best_ms(F launch, float *out_ms) {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HQMC_OK;
    float best = -1.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = HQMC_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, st);
            launch(st);
            cudaEventRecord(e1, st);
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = HQMC_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best < 0.f || ms < best)) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc == HQMC_OK && !(best > 0.f)) rc = HQMC_ERR_CUDA;
    *out_ms = best;
    return rc;
}

}  // namespace
}  // namespace hqmc

#pragma GCC visibility push(default)
extern "C" {

int hqmc_fp32_peak(int device, int packed, double *tflops) {
    using namespace hqmc;
    if (!tflops || (packed != 0 && packed != 1)) return HQMC_ERR_ARG;
    *tflops = 0.0;
    int prev = 0, sms = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return HQMC_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = kCtasPerSm * (sms > 0 ? sms : 1);
    const size_t n = size_t(grid) * kThreads;
    void *buf = nullptr;
    float ms = 0.f;
    int rc = cudaMalloc(&buf, n * sizeof(float2)) == cudaSuccess ? HQMC_OK : HQMC_ERR_CUDA;
    if (rc == HQMC_OK)
        rc = best_ms(
            [&](cudaStream_t st) {
                if (packed)
                    fma2_loop<<<grid, kThreads, 0, st>>>(static_cast<float2 *>(buf), make_float2(0.999999f, 0.999998f),
                                                         make_float2(1e-6f, 2e-6f), kIters);
                else
                    fma_loop<<<grid, kThreads, 0, st>>>(static_cast<float *>(buf), 0.999999f, 1e-6f, kIters);
            },
            &ms);
    // per thread: kIters x kChains packed FMAs (4 flops) or kIters x 2 kChains scalar (2)
    if (rc == HQMC_OK) *tflops = double(n) * kIters * kChains * 4.0 / (double(ms) * 1e-3) / 1e12;
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    return rc;
}

int hqmc_fp64_peak(int device, double *tflops) {
    using namespace hqmc;
    if (!tflops) return HQMC_ERR_ARG;
    *tflops = 0.0;
    int prev = 0, sms = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return HQMC_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = kCtasPerSm * (sms > 0 ? sms : 1);
    const size_t n = size_t(grid) * kThreads;
    constexpr int iters = kIters / 8;  // the FP64 pipe is far slower: keep a launch near 10 ms
    void *buf = nullptr;
    float ms = 0.f;
    int rc = cudaMalloc(&buf, n * sizeof(double)) == cudaSuccess ? HQMC_OK : HQMC_ERR_CUDA;
    if (rc == HQMC_OK)
        rc = best_ms([&](cudaStream_t st) { dfma_loop<<<grid, kThreads, 0, st>>>(static_cast<double *>(buf), 0.999999, 1e-6, iters); },
                     &ms);
    if (rc == HQMC_OK) *tflops = double(n) * iters * kChains * 2.0 / (double(ms) * 1e-3) / 1e12;
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    return rc;
}

}  // extern "C"
#pragma GCC visibility pop
