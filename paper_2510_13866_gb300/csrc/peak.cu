// peak.cu -- measured FP32 fused multiply-add throughput of the current GPU: the
// denominator of the FFBS kernels' ALU roofline (their FFT and pointwise arithmetic is
// packed f32x2, FFMA2/FMUL2/FADD2).
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

}  // namespace
}  // namespace hqmc

#pragma GCC visibility push(default)
extern "C" {

int hqmc_fp32_peak(int device, int packed, double *tflops) {
    using namespace hqmc;
    if (!tflops || (packed != 0 && packed != 1)) return HQMC_ERR_ARG;
    *tflops = 0.0;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return HQMC_ERR_CUDA;
    int sms = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void *buf = nullptr;
    int rc = HQMC_OK;
    const int grid = [&] {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        return kCtasPerSm * (sms > 0 ? sms : 1);
    }();
    const size_t n = size_t(grid) * kThreads;
    float best_ms = -1.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&buf, n * sizeof(float2)) != cudaSuccess) {
        rc = HQMC_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 6 && rc == HQMC_OK; ++rep) {
            cudaEventRecord(e0, st);
            if (packed)
                fma2_loop<<<grid, kThreads, 0, st>>>(static_cast<float2 *>(buf), make_float2(0.999999f, 0.999998f),
                                                     make_float2(1e-6f, 2e-6f), kIters);
            else
                fma_loop<<<grid, kThreads, 0, st>>>(static_cast<float *>(buf), 0.999999f, 1e-6f, kIters);
            cudaEventRecord(e1, st);
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = HQMC_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best_ms < 0.f || ms < best_ms)) best_ms = ms;  // the first launch warms up
        }
    }
    if (rc == HQMC_OK && best_ms > 0.f) {
        // per thread: kIters x kChains packed FMAs (4 flops) or kIters x 2 kChains scalar (2)
        const double flops = double(n) * kIters * kChains * 4.0;
        *tflops = flops / (double(best_ms) * 1e-3) / 1e12;
    } else if (rc == HQMC_OK) {
        rc = HQMC_ERR_CUDA;
    }
    if (buf) cudaFree(buf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    return rc;
}

}  // extern "C"
#pragma GCC visibility pop
