// noalloc.cu -- forward-filtering backward-sampling of one chain without any device
// allocation: every intermediate (tables, bit-packed field, 16-bit worldlines, the
// occupancy histogram and the per-group f_l slots) lives in one file-scope
// __device__ array of fixed size.  The FFBS kernel itself is the library's usual one.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "../../include/hqmc.h"
#include "internal.h"

namespace hqmc {
cudaError_t launch_ffbs_f32(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t launch_ffbs_f64(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t ffbs_occupancy_f32(int L, int wpc, int *blocks);
cudaError_t ffbs_occupancy_f64(int L, int wpc, int *blocks);
}  // namespace hqmc

using namespace hqmc;

namespace {

// Size of the static scratch.  Every device that loads this library holds it until
// the process exits, so it is kept modest.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr unsigned kStatusBadInput = 8u;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct StaticLayout {
    size_t cd, tab, cls, sbits, x, hist, meas, anchor, sweep, status, lerr, slots, fixed;
};

StaticLayout layout_for(int L, int M, int Nsig) {
    StaticLayout s{};
    const size_t N = size_t(L) * L, wpl = size_t(L + 31) / 32;
    size_t o = 0;
    s.cd = o;
    o = align256(o + sizeof(ChainDev));
    s.tab = o;
    o = align256(o + sizeof(ChainTab));
    s.cls = o;
    o = align256(o + 4 * sizeof(int));
    s.sbits = o;
    o = align256(o + 2 * size_t(M) * L * wpl * 4);
    s.x = o;
    o = align256(o + 2 * size_t(Nsig) * M * 2);
    s.hist = o;
    o = align256(o + 2 * size_t(M) * N * 4);
    s.meas = o;
    o = align256(o + sizeof(MeasAcc));
    s.anchor = o;
    o = align256(o + sizeof(int));
    s.sweep = o;
    o = align256(o + 8);
    s.status = o;
    o = align256(o + 8);
    s.lerr = o;  // error estimates of the log-weights (the kernel writes them; not returned)
    o = align256(o + 2 * size_t(Nsig) * 8);
    s.slots = o;
    s.fixed = o;
    return s;
}

// Writes the chain descriptor, tables and launch arrays; clears what must start at zero.
__global__ void static_setup_kernel(unsigned char *base, StaticLayout lay, ChainDev cd, ChainTab tab,
                                    unsigned long long sweep) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        *reinterpret_cast<ChainDev *>(base + lay.cd) = cd;
        int *cls = reinterpret_cast<int *>(base + lay.cls);
        cls[0] = 0;                // chain id
        cls[1] = 0;                // pair offsets [0, 2*npair]
        cls[2] = 2 * cd.npair;
        cls[3] = 0;                // work counter of the FFBS launch
        *reinterpret_cast<int *>(base + lay.anchor) = -1;
        *reinterpret_cast<unsigned long long *>(base + lay.sweep) = sweep;
        *reinterpret_cast<unsigned *>(base + lay.status) = 0u;
        MeasAcc z{};
        *reinterpret_cast<MeasAcc *>(base + lay.meas) = z;
    }
    // the table is copied word by word by the whole block
    const unsigned *src = reinterpret_cast<const unsigned *>(&tab);
    unsigned *dst = reinterpret_cast<unsigned *>(base + lay.tab);
    for (int k = tid; k < int(sizeof(ChainTab) / 4); k += blockDim.x) dst[k] = src[k];
}

// int8 field [M][N] -> bit-packed rows and columns; int32 worldlines -> int16.
// Any value out of range sets kStatusBadInput (the FFBS kernel is then not launched).
__global__ void static_pack_kernel(unsigned char *base, StaticLayout lay, int L, int M, int Nsig,
                                   const int8_t *s, const int32_t *x) {
    const int N = L * L, wpl = (L + 31) / 32;
    uint32_t *rows = reinterpret_cast<uint32_t *>(base + lay.sbits);
    uint32_t *cols = rows + size_t(M) * L * wpl;
    int16_t *x16 = reinterpret_cast<int16_t *>(base + lay.x);
    unsigned *status = reinterpret_cast<unsigned *>(base + lay.status);
    const long long nwords = (long long)M * L * wpl;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // one thread per word: rows word (l, iy, w) covers ix = 32w .. 32w+31
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nwords; k += stride) {
        const int w = int(k % wpl), line = int((k / wpl) % L), l = int(k / ((long long)wpl * L));
        uint32_t rw = 0u, cw = 0u;
        for (int b = 0; b < 32; ++b) {
            const int o = 32 * w + b;
            if (o >= L) break;
            const int8_t vr = s[(size_t)l * N + o + (size_t)L * line];  // (ix = o, iy = line)
            const int8_t vc = s[(size_t)l * N + line + (size_t)L * o];  // (ix = line, iy = o)
            if ((vr != 1 && vr != -1) || (vc != 1 && vc != -1)) atomicOr(status, kStatusBadInput);
            rw |= (vr == 1 ? 1u : 0u) << b;
            cw |= (vc == 1 ? 1u : 0u) << b;
        }
        rows[k] = rw;
        cols[k] = cw;
    }
    const long long nx = 2LL * Nsig * M;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nx; k += stride) {
        const int32_t v = x[k];
        if (v < 0 || v >= N) {
            atomicOr(status, kStatusBadInput);
            x16[k] = 0;
        } else {
            x16[k] = int16_t(v);
        }
    }
}

__global__ void static_unpack_kernel(const unsigned char *base, StaticLayout lay, long long nx, int32_t *x) {
    const int16_t *x16 = reinterpret_cast<const int16_t *>(base + lay.x);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nx; k += (long long)gridDim.x * blockDim.x)
        x[k] = x16[k];
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" int hqmc_ffbs_noalloc(int L, int M, int Nsig, double t, double U, double dtau, uint64_t seed,
                                 uint64_t sweep, const int8_t *s, int32_t *x, double *logw, int precision,
                                 void *stream) {
    if (!s || !x || !logw) return HQMC_ERR_ARG;
    if (precision != HQMC_FP32 && precision != HQMC_FP64) return HQMC_ERR_ARG;
    if (L < 2 || L > 32 || M < 1 || M > 32767 || Nsig < 1 || Nsig > L * L) return HQMC_ERR_ARG;
    if (!ffbs_supported(L)) return HQMC_ERR_UNSUPPORTED;
    if (!(t >= 0.0) || !(U >= 0.0) || !(dtau > 0.0)) return HQMC_ERR_ARG;
    const bool f64 = precision == HQMC_FP64;
    const StaticLayout lay = layout_for(L, M, Nsig);
    const size_t slot = size_t(M) * L * L * (f64 ? 16 : 8);
    if (lay.fixed + slot > kStaticScratchBytes) return HQMC_ERR_SCRATCH;

    // the static array's device address in the current device's context, looked up on
    // every call (the host-side name of the array is not a device address, and a cached
    // address would go stale after a device reset reloads the module)
    unsigned char *base = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HQMC_ERR_CUDA;
        }
        base = static_cast<unsigned char *>(p);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    ChainDev cd{};
    ChainTab tab;
    double lam = 0.0;
    host_chain_table(L, t, U, dtau, tab, &lam);
    cd.L = L;
    cd.N = L * L;
    cd.M = M;
    cd.Nsig = Nsig;
    cd.npair = (Nsig + 1) / 2;
    cd.wpl = (L + 31) / 32;
    cd.seed = seed;
    cd.lam = lam;
    cd.w_plus[0] = std::exp(lam);
    cd.w_minus[0] = std::exp(-lam);
    cd.w_plus[1] = std::exp(-lam);
    cd.w_minus[1] = std::exp(lam);
    cd.t = t;
    cd.beta = M * dtau;

    // launch shape: as many worldline groups as the remaining scratch holds slots for
    int wpc = 4;
    const int gpw = ffbs_groups_per_warp(L);
    const long long max_groups = (long long)((kStaticScratchBytes - lay.fixed) / slot);
    while (wpc > 1 && max_groups < (long long)wpc * gpw) wpc >>= 1;
    const int gpc = wpc * gpw;
    const long long total_pairs = 2LL * cd.npair;
    long long grid = (total_pairs + gpc - 1) / gpc;
    const long long grid_cap = max_groups / gpc;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) return HQMC_ERR_SCRATCH;
    // resident CTAs per SM (this also raises the kernel's shared-memory limit to the
    // launch's needs): the grid need not exceed one resident wave, since groups take
    // pairs from a work counter
    int bps = 0, nsm = 0, dev = 0;
    cudaError_t e = f64 ? ffbs_occupancy_f64(L, wpc, &bps) : ffbs_occupancy_f32(L, wpc, &bps);
    if (e != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HQMC_ERR_CUDA;
    const long long wave = (long long)std::max(1, bps) * std::max(1, nsm);
    if (grid > wave) grid = wave;

    static_setup_kernel<<<1, 256, 0, st>>>(base, lay, cd, tab, (unsigned long long)sweep);
    if (cudaGetLastError() != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaMemsetAsync(base + lay.hist, 0, 2 * size_t(M) * L * L * 4, st) != cudaSuccess) return HQMC_ERR_CUDA;
    static_pack_kernel<<<152, 256, 0, st>>>(base, lay, L, M, Nsig, s, x);
    if (cudaGetLastError() != cudaSuccess) return HQMC_ERR_CUDA;
    unsigned status = 0;
    if (cudaMemcpyAsync(&status, base + lay.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HQMC_ERR_CUDA;
    if (status & kStatusBadInput) return HQMC_ERR_ARG;

    DevState ds{};
    ds.chains = reinterpret_cast<const ChainDev *>(base + lay.cd);
    ds.tabs = reinterpret_cast<const ChainTab *>(base + lay.tab);
    ds.sbits = reinterpret_cast<uint32_t *>(base + lay.sbits);
    ds.x = reinterpret_cast<int16_t *>(base + lay.x);
    ds.hist = reinterpret_cast<int *>(base + lay.hist);
    ds.logw = logw;
    ds.anchor = reinterpret_cast<int *>(base + lay.anchor);
    ds.meas = reinterpret_cast<MeasAcc *>(base + lay.meas);
    ds.sk = nullptr;
    ds.dens = nullptr;
    ds.sweep = reinterpret_cast<unsigned long long *>(base + lay.sweep);
    ds.status = reinterpret_cast<unsigned *>(base + lay.status);
    ds.logw_err = reinterpret_cast<double *>(base + lay.lerr);
    FfbsLaunch fl{};
    fl.class_chains = reinterpret_cast<const int *>(base + lay.cls);
    fl.class_unit_off = fl.class_chains + 1;  // the closed loop: one unit per pair
    fl.nclass = 1;
    fl.total_units = int(total_pairs);
    fl.len_max = M;
    fl.scratch = base + lay.slots;
    fl.slot_elems = (long long)M * L * L;
    fl.next_unit = reinterpret_cast<unsigned *>(base + lay.cls) + 3;
    e = f64 ? launch_ffbs_f64(L, ds, fl, int(grid), wpc, st) : launch_ffbs_f32(L, ds, fl, int(grid), wpc, st);
    if (e != cudaSuccess) return HQMC_ERR_CUDA;
    const long long nx = 2LL * Nsig * M;
    static_unpack_kernel<<<152, 256, 0, st>>>(base, lay, nx, x);
    if (cudaGetLastError() != cudaSuccess) return HQMC_ERR_CUDA;
    MeasAcc acc{};
    if (cudaMemcpyAsync(&status, base + lay.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HQMC_ERR_CUDA;
    if (cudaMemcpyAsync(&acc, base + lay.meas, sizeof(MeasAcc), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HQMC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HQMC_ERR_CUDA;
    if (status || acc.degenerate || acc.nonpositive) return HQMC_ERR_NUMERIC;
    return HQMC_OK;
}
#pragma GCC visibility pop
