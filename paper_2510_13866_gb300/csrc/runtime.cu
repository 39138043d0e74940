// runtime.cu -- host side of the C ABI declared in include/hqmc.h: parameter validation,
// FP64 tables, device layout, workspace, CUDA-graph capture of one sweep, read-outs.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hqmc.h"
#include "internal.h"

namespace hqmc {
cudaError_t launch_ffbs_f32(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t launch_ffbs_f64(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t ffbs_occupancy_f32(int L, int wpc, int *blocks);
cudaError_t ffbs_occupancy_f64(int L, int wpc, int *blocks);
cudaError_t launch_ffbs_f32g(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t launch_ffbs_f64g(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s);
cudaError_t ffbs_occupancy_f32g(int L, int wpc, int *blocks);
cudaError_t ffbs_occupancy_f64g(int L, int wpc, int *blocks);
size_t ffbs_smem_f32(int L, int wpc);
size_t ffbs_smem_f64(int L, int wpc);
cudaError_t launch_grad_f32(int L, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s);
cudaError_t launch_grad_f64(int L, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s);
cudaError_t grad_occupancy_f32(int L, int *blocks);
cudaError_t grad_occupancy_f64(int L, int *blocks);
constexpr int kGradWarpsHost = 4;  // warps per CTA of the adjoint kernel (fixed)

cudaError_t launch_ffbs_wide(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s);
cudaError_t launch_grad_wide(int L, bool fp64, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s);
cudaError_t grad_wide_occupancy(int L, bool fp64, int *blocks);
cudaError_t ffbs_wide_occupancy(int L, bool fp64, int *blocks);
bool ffbs_wide_supported(int L);
int ffbs_wide_wpc(int L);

// register-line sizes (one warp-group per pair) and wide sizes (one thread per line of
// each worldline, one or two worldlines per CTA); both precisions
static const int kSizes[] = {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 128};

bool ffbs_supported(int L) {
    for (int s : kSizes)
        if (s == L && s <= 32) return true;
    return false;
}
static bool is_big(int L) { return L > 32; }
int ffbs_groups_per_warp(int L) { return L <= 4 ? 8 : L <= 8 ? 4 : L <= 16 ? 2 : 1; }
}  // namespace hqmc

using namespace hqmc;

namespace {

struct HostChain {
    int L = 0, N = 0, M = 0, Nsig = 0;
    uint64_t seed = 0;
    double t = 0, U = 0, beta = 0, dtau = 0, filling = 0;
    int block = 0;  // FFBS block length (0: the closed loop)
    bool set = false;
};

struct LClass {
    int L = 0;
    std::vector<int> chains;
    std::vector<int> pair_off;  // prefix sums of the adjoint's work units per chain: 2 npair
                                // (L <= 32), 2 ceil(Nsig / WPC) worldline groups (wide)
    std::vector<int> unit_off;  // prefix sums of 2*npair*nblk (FFBS work units: pair, block)
    int total_pairs = 0;
    int total_units = 0;
    int M_max = 0;
    int len_max = 0;            // longest FFBS block (scratch slot, slices)
    int grid = 0;          // CTAs launched
    long long groups = 0;  // worldline groups launched
    size_t scratch_off = 0;
    size_t scratch_bytes = 0;
    // wide classes with f checkpoints (FP32): every K positions, the segment buffer at
    // seg_off of a worldline's slot of wl_elems floats (ckpt_K = 0: every f streamed)
    int ckpt_K = 0;
    long long seg_off = 0, wl_elems = 0;
    // FFBS slot per group, in the kernel's elements (pairs for L <= 32, scalars of the CTA's
    // worldlines for wide): the f storage of each worldline, then len_max per-position maxima
    // of the forward messages (Gaussian-field units), padded to whole 16-byte chunks
    long long slot_elems = 0;
    size_t cls_off = 0;    // device offset of the class arrays
};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct hqmc_ctx {
    int device = 0;
    int precision = HQMC_FP32;
    int nchains = 0;
    std::vector<HostChain> ch;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev;
    bool use_graph = true, persistent = true;
    int wpc = 0;
    int slices_per_cta = 0;  // Gibbs/measure kernel: slices handled by one CTA (0: automatic)
    bool perm_on = false;    // permutation updates at tau = beta in every sweep
    int conv = HQMC_CONV_FFT;  // line convolutions of the FFBS: FFT or periodic stencil
    bool perm_used = false;  // a permutation other than the identity may be in the state
    int num_sms = 0;
    std::string err;

    // device layout (valid when `ready`)
    bool ready = false;       // layout built and state initialised
    bool started = false;     // a sweep has run
    bool own_mem = false;
    unsigned char *base = nullptr;
    size_t bytes = 0;
    unsigned char *attached = nullptr;
    size_t attached_bytes = 0;
    std::vector<ChainDev> cdev;
    std::vector<LClass> classes;
    DevState st{};
    size_t off_cr = 0, off_sko = 0, off_rd = 0, off_open = 0, total_N = 0;
    bool open_on = false;  // open-path estimator (one-body density matrix, n_k) accumulated
    int fstore = HQMC_FSTORE_STREAM;  // storage of f for the backward pass (wide sizes, FP32)
    int fstride = 0;                  // checkpoint stride (0: ceil(sqrt(longest block)))
    long long total_wl = 0;
    double *d_cr = nullptr, *d_sko = nullptr, *d_rd = nullptr;
    uint64_t sweeps_host = 0;

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    // per-size CTA shape (warps per CTA) chosen by hqmc_set_class_launch / hqmc_autotune
    std::vector<std::pair<int, int>> class_wpc;
    // state kept across a re-layout (launch shape change): restored by the next prepare()
    bool pending_restore = false;
    std::vector<uint32_t> keep_bits;
    std::vector<int16_t> keep_x;
    std::vector<double> keep_sig;
    std::vector<int> keep_perm;
    std::vector<unsigned> keep_parity;
    unsigned long long keep_sweep = 0;
    bool keep_started = false;

    // adjoint: checkpoint stride (0 = ceil(sqrt M)) and format, context-owned scratch
    int ckpt_stride = 0;
    int ckpt_kind = HQMC_CKPT_BF16;
    unsigned char *grad_mem = nullptr;
    size_t grad_bytes = 0;
    long long total_v = 0;

    // per-phase timing: events [4 * slot]: ffbs start, ffbs end, slice start, slice end
    int prof_max = 0, prof_n = 0;
    std::vector<cudaEvent_t> prof_ev;
};

namespace {

int fail(hqmc_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(hqmc_ctx *c, cudaError_t e, const char *where) {
    return fail(c, HQMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HQMC_CUDA(ctx, call)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// 1D ring propagator g(d) = [exp(z A)]_{0d}, A = ring adjacency, by its Taylor series
// applied to a unit vector: every term is non-negative, so each entry is accurate to
// rounding even where it is tiny.
void ring_propagator(int L, double z, std::vector<double> &g) {
    std::vector<double> term(L, 0.0), nxt(L, 0.0);
    g.assign(L, 0.0);
    term[0] = 1.0;
    g[0] = 1.0;
    for (int n = 1; n < 2000; ++n) {
        double mx = 0.0;
        for (int d = 0; d < L; ++d) {
            const double v = term[(d + L - 1) % L] + term[(d + 1) % L];
            nxt[d] = v * z / n;
            mx = std::max(mx, nxt[d]);
        }
        term.swap(nxt);
        for (int d = 0; d < L; ++d) g[d] += term[d];
        if (n > 2 * L + 8 && mx < 1e-300) break;
        if (mx == 0.0) break;
    }
}

void build_tab(const HostChain &h, ChainTab &tb, double lam) {
    std::memset(&tb, 0, sizeof(tb));
    const int L = h.L;
    const double z = h.t * h.dtau;
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < L; ++k) {
        const double ck = std::cos(two_pi * k / L);
        const double gh = std::exp(2.0 * z * ck);
        tb.ghat_d[k] = gh / L;
        tb.ghat_f[k] = float(gh / L);
        tb.dghat_d[k] = 2.0 * h.dtau * ck * gh / L;
        tb.dghat_f[k] = float(tb.dghat_d[k]);
    }
    // spectral mix of conv_line: with n = L/2, P = (gh_k + gh_{k+n})/2, Q = (gh_k - gh_{k+n})/2,
    // alpha_k = (P - Q sin(2 pi k/L)) / n and beta_k = Q cos(2 pi k/L) / n (gh unnormalised)
    // (mixd: the same for d gh / dt = 2 dtau cos(2 pi k/L) gh_k)
    auto ghk = [&](double th) { return std::exp(2.0 * z * std::cos(th)); };
    auto dghk = [&](double th) { return 2.0 * h.dtau * std::cos(th) * std::exp(2.0 * z * std::cos(th)); };
    if (L % 2 == 0) {
        const int n = L / 2;
        for (int k = 0; k < n; ++k) {
            const double th = two_pi * k / L, th2 = th + 0.5 * two_pi;
            const double P = 0.5 * (ghk(th) + ghk(th2)), Q = 0.5 * (ghk(th) - ghk(th2));
            tb.mix_d[2 * k] = (P - Q * std::sin(th)) / n;
            tb.mix_d[2 * k + 1] = Q * std::cos(th) / n;
            const double Pd = 0.5 * (dghk(th) + dghk(th2)), Qd = 0.5 * (dghk(th) - dghk(th2));
            tb.mixd_d[2 * k] = (Pd - Qd * std::sin(th)) / n;
            tb.mixd_d[2 * k + 1] = Qd * std::cos(th) / n;
        }
    } else {
        for (int k = 0; k < L; ++k) {
            tb.mix_d[k] = ghk(two_pi * k / L) / L;
            tb.mixd_d[k] = dghk(two_pi * k / L) / L;
        }
    }
    for (int k = 0; k < L; ++k) {
        tb.mix_f[k] = float(tb.mix_d[k]);
        tb.mixd_f[k] = float(tb.mixd_d[k]);
    }
    std::vector<double> g;
    ring_propagator(L, z, g);
    for (int d = 0; d < L; ++d) {
        tb.g_d[d] = g[d];
        tb.g_f[d] = float(g[d]);
        // d/dt exp(t dtau A) = dtau A exp(t dtau A)  =>  g'(d) = dtau (g(d-1) + g(d+1))
        const double dg = h.dtau * (g[(d + L - 1) % L] + g[(d + 1) % L]);
        const double hv = g[d] > 0.0 ? dg / g[d] : 0.0;
        tb.h_d[d] = hv;
        tb.h_f[d] = float(hv);
    }
    for (int m = -kPTab; m <= kPTab; ++m) tb.pplus[m + kPTab] = 1.0 / (1.0 + std::exp(-2.0 * lam * m));
}

double hirsch_lambda(double U, double dtau) { return std::acosh(std::exp(0.5 * dtau * U)); }

}  // namespace

namespace hqmc {
// Tables and lambda of one chain, for entry points that do not own a context.
void host_chain_table(int L, double t, double U, double dtau, ChainTab &tb, double *lam) {
    HostChain h;
    h.L = L;
    h.N = L * L;
    h.t = t;
    h.U = U;
    h.dtau = dtau;
    *lam = hirsch_lambda(U, dtau);
    build_tab(h, tb, *lam);
}
}  // namespace hqmc

namespace {

int check_params(hqmc_ctx *c, int L, double t, double U, double beta, double dtau, double filling, int *M,
                 int *Nsig) {
    if (!(t >= 0.0) || !std::isfinite(t)) return fail(c, HQMC_ERR_ARG, "t must be finite and >= 0");
    if (!std::isfinite(U)) return fail(c, HQMC_ERR_ARG, "U must be finite");
    if (!(beta > 0.0) || !(dtau > 0.0) || !std::isfinite(beta) || !std::isfinite(dtau))
        return fail(c, HQMC_ERR_ARG, "beta and dtau must be positive");
    const double mr = beta / dtau;
    const long long m = llround(mr);
    if (m < 1 || std::fabs(double(m) * dtau - beta) > 1e-9 * std::max(1.0, beta))
        return fail(c, HQMC_ERR_ARG, "beta/dtau must be an integer");
    if (m > 32767) return fail(c, HQMC_ERR_ARG, "too many slices");
    const double ns = filling * L * L / 2.0;
    const long long n = llround(ns);
    if (!(filling > 0.0) || std::fabs(ns - double(n)) > 1e-9 || n < 1 || n > (long long)L * L)
        return fail(c, HQMC_ERR_ARG, "filling*N/2 must be an integer in [1, N]");
    *M = int(m);
    *Nsig = int(n);
    return HQMC_OK;
}

void drop_graph(hqmc_ctx *c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
}

void free_layout(hqmc_ctx *c) {
    drop_graph(c);
    if (c->own_mem && c->base) cudaFree(c->base);
    c->base = nullptr;
    c->own_mem = false;
    c->ready = false;
}

int occupancy(hqmc_ctx *c, int L, int wpc, int *blocks) {
    cudaError_t e = is_big(L) ? ffbs_wide_occupancy(L, c->precision == HQMC_FP64, blocks)
                    : c->precision == HQMC_FP64 ? ffbs_occupancy_f64(L, wpc, blocks)
                                                : ffbs_occupancy_f32(L, wpc, blocks);
    if (e == cudaSuccess && !is_big(L)) {
        // the Gaussian-field instantiations get their limits too; the grid follows the
        // smaller residency of the two
        int bg = 0;
        e = c->precision == HQMC_FP64 ? ffbs_occupancy_f64g(L, wpc, &bg) : ffbs_occupancy_f32g(L, wpc, &bg);
        if (e == cudaSuccess && bg > 0) *blocks = std::min(*blocks, bg);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy");
    if (*blocks < 1) *blocks = 1;
    return HQMC_OK;
}

// chains x the longest M: the Gibbs/measure kernel's work in slices
long long slice_work(const hqmc_ctx *c) {
    int max_M = 0;
    for (auto &d : c->cdev) max_M = std::max(max_M, d.M);
    return (long long)c->nchains * max_M;
}

int default_wpc(hqmc_ctx *c, int L) {
    for (auto &kv : c->class_wpc)
        if (kv.first == L && kv.second > 0) return kv.second;
    if (c->wpc > 0) return c->wpc;
    return c->precision == HQMC_FP64 ? 4 : 4;
}

// Compute the device layout (offsets) and its size; fills c->classes, c->cdev.
int plan_layout(hqmc_ctx *c, size_t *total) {
    const int nc = c->nchains;
    for (int i = 0; i < nc; ++i)
        if (!c->ch[i].set) return fail(c, HQMC_ERR_STATE, "set_params has not been called for every chain");
    const bool f64 = c->precision == HQMC_FP64;
    c->cdev.assign(nc, ChainDev{});
    // classes by L
    c->classes.clear();
    for (int i = 0; i < nc; ++i) {
        auto it = std::find_if(c->classes.begin(), c->classes.end(), [&](const LClass &k) { return k.L == c->ch[i].L; });
        if (it == c->classes.end()) {
            c->classes.push_back(LClass{});
            c->classes.back().L = c->ch[i].L;
            it = c->classes.end() - 1;
        }
        it->chains.push_back(i);
    }
    // within a size class the chains with the longest FFBS blocks (M, or B < M) go first:
    // groups take work units in this order from the class's work counter, which keeps the
    // tail of a launch short
    auto blen = [&](int i) { return ffbs_block_len(c->ch[i].block, c->ch[i].M); };
    for (auto &k : c->classes)
        std::stable_sort(k.chains.begin(), k.chains.end(), [&](int x, int y) { return blen(x) > blen(y); });
    size_t off = 0;
    auto take = [&](size_t b) {
        off = round_up(off, 256);
        const size_t o = off;
        off += b;
        return o;
    };
    const size_t o_chains = take(sizeof(ChainDev) * nc);
    const size_t o_tabs = take(sizeof(ChainTab) * nc);
    long long sb = 0, xb = 0, hb = 0, lb = 0, vb = 0, mb = 0, gb = 0, pb = 0, db = 0, qb = 0;
    for (int i = 0; i < nc; ++i) {
        const HostChain &h = c->ch[i];
        ChainDev &d = c->cdev[i];
        d.L = h.L;
        d.N = h.N;
        d.M = h.M;
        d.Nsig = h.Nsig;
        d.npair = (h.Nsig + 1) / 2;
        d.wpl = (h.L + 31) / 32;
        d.seed = h.seed;
        d.lam = hirsch_lambda(h.U, h.dtau);
        d.w_plus[0] = std::exp(d.lam);
        d.w_minus[0] = std::exp(-d.lam);
        d.w_plus[1] = std::exp(-d.lam);
        d.w_minus[1] = std::exp(d.lam);
        d.t = h.t;
        d.beta = h.beta;
        d.gauss = h.U < 0.0 ? 1 : 0;
        d.block = h.block;
        const int nblk = ffbs_nblk(h.block, h.M);
        d.lwp_off = pb;
        d.done_off = db;
        d.perm_off = qb;
        qb += 4LL * h.Nsig;  // P [2][Nsig], then P^{-1} [2][Nsig]
        if (nblk > 1) {
            pb += 2LL * h.Nsig * nblk;
            db += 2LL * h.Nsig;  // one counter per work group: a pair (L <= 32) or fewer worldlines
        }
        d.gcoup = std::sqrt(std::fabs(h.U) * h.dtau);
        d.g_off = gb;
        if (d.gauss) gb += ((long long)h.M * h.N + 3) / 4 * 4;  // 16-byte aligned W lines
        d.s_off = sb;
        sb += 2LL * h.M * h.L * d.wpl;
        d.x_off = xb;
        xb += 2LL * h.Nsig * h.M;
        d.h_off = hb;
        hb += 2LL * h.M * h.N;
        d.logw_off = lb;
        lb += 2LL * h.Nsig;
        d.v_off = vb;
        vb += 2LL * h.M * h.N;
        d.meas_off = mb;
        mb += h.N;
    }
    c->total_N = size_t(mb);
    c->total_wl = lb;
    c->total_v = vb;
    const size_t o_s = take(size_t(sb) * 4);
    const size_t o_x = take(size_t(xb) * 2);
    const size_t o_h = take(size_t(hb) * 4);
    const size_t o_l = take(size_t(lb) * 8);
    const size_t o_a = take(size_t(nc) * 4);
    const size_t o_m = take(sizeof(MeasAcc) * nc);
    const size_t o_sk = take(size_t(mb) * 8);
    const size_t o_dn = take(size_t(mb) * 8);
    const size_t o_sw = take(8);
    const size_t o_stt = take(8);
    const size_t o_gs = take(size_t(gb) * 8);
    const size_t o_gw = take(size_t(gb) * 2 * (f64 ? 8 : 4));
    const size_t o_lp = take(size_t(pb) * 8);
    const size_t o_le = take(size_t(lb) * 8);
    const size_t o_lep = take(size_t(pb) * 8);
    const size_t o_bd = take(size_t(db) * 4);
    const size_t o_pm = take(size_t(qb) * 4);
    const size_t o_par = take(size_t(nc) * 4);
    c->off_cr = take(size_t(mb) * 8);
    c->off_sko = take(size_t(mb) * 8);
    c->off_rd = take(size_t(mb) * 16);  // read-out passes: 2 N doubles per chain
    c->off_open = take(size_t(mb) * 8);  // open-path sums: N doubles per chain
    // classes
    for (auto &k : c->classes) {
        k.pair_off.assign(1, 0);
        k.unit_off.assign(1, 0);
        k.M_max = 0;
        k.len_max = 0;
        for (int ci : k.chains) {
            const ChainDev &d = c->cdev[ci];
            const int gw = is_big(k.L) ? ffbs_wide_wpc(k.L) : 2;
            k.pair_off.push_back(k.pair_off.back() + 2 * ((d.Nsig + gw - 1) / gw));
            // FFBS work units (group, block); a group is a worldline pair, or for the wide
            // kernel the worldlines one CTA holds
            const int wg = is_big(k.L) ? ffbs_wide_wpc(k.L) : 2;
            const int ngrp = (d.Nsig + wg - 1) / wg;
            k.unit_off.push_back(k.unit_off.back() + 2 * ngrp * ffbs_nblk(d.block, d.M));
            k.M_max = std::max(k.M_max, d.M);
            k.len_max = std::max(k.len_max, ffbs_block_len(d.block, d.M));
        }
        k.total_pairs = k.pair_off.back();
        k.total_units = k.unit_off.back();
        // [chains][pair_off][work counter][unit_off]
        k.cls_off = take(sizeof(int) * (k.chains.size() + k.pair_off.size() + 1 + k.unit_off.size()));
    }
    // FFBS grid and scratch per class
    for (auto &k : c->classes) {
        const int wpc = default_wpc(c, k.L);
        const int gpc = is_big(k.L) ? 1 : wpc * ffbs_groups_per_warp(k.L);  // wide lattices: one pair per CTA
        const int need = (k.total_units + gpc - 1) / gpc;
        int grid = need;
        if (c->persistent) {
            int bps = 1;
            int rc = occupancy(c, k.L, wpc, &bps);
            if (rc) return rc;
            // every class may fill the GPU: groups take pairs from a work counter, so
            // concurrent classes share the SMs dynamically
            const int cap = std::max(1, bps * c->num_sms);
            grid = std::min(need, cap);
        }
        k.grid = std::max(1, grid);
        k.groups = (long long)k.grid * gpc;
        // f slots: a worldline pair per group (L <= 32), or the CTA's worldlines (wide)
        const long long N = (long long)k.L * k.L;
        // elements per 16-byte chunk: pairs of FP32 (one for odd L, whose chunks are 8 bytes),
        // FP64 pairs, wide scalars
        const long long ch = is_big(k.L) ? (f64 ? 2 : 4) : (f64 || (k.L & 1)) ? 1 : 2;
        const long long aux = (k.len_max + ch - 1) / ch * ch;
        long long per_wl = (long long)k.len_max * N;
        k.ckpt_K = 0;
        if (is_big(k.L) && !f64 && c->fstore != HQMC_FSTORE_STREAM) {
            // checkpoints every K positions (BF16: two per float) then a K-slice segment
            const int K = c->fstride > 0 ? std::min(c->fstride, k.len_max)
                                         : std::max(1, int(std::ceil(std::sqrt(double(k.len_max)))));
            const long long nseg = (k.len_max + K - 1) / K;
            k.ckpt_K = K;
            k.seg_off = (c->fstore == HQMC_FSTORE_BF16) ? nseg * N / 2 : nseg * N;
            k.wl_elems = k.seg_off + (long long)K * N;
            per_wl = k.wl_elems;
        }
        k.slot_elems = (per_wl + aux) * (is_big(k.L) ? ffbs_wide_wpc(k.L) : 1);
        const size_t elem = is_big(k.L) ? (f64 ? 8 : 4) : (f64 ? 16 : 8);
        k.scratch_bytes = size_t(k.groups) * size_t(k.slot_elems) * elem;
        k.scratch_off = take(k.scratch_bytes);
    }
    *total = round_up(off, 256);
    // keep the offsets for binding
    c->st = DevState{};
    c->st.chains = reinterpret_cast<const ChainDev *>(o_chains);
    c->st.tabs = reinterpret_cast<const ChainTab *>(o_tabs);
    c->st.sbits = reinterpret_cast<uint32_t *>(o_s);
    c->st.x = reinterpret_cast<int16_t *>(o_x);
    c->st.hist = reinterpret_cast<int *>(o_h);
    c->st.logw = reinterpret_cast<double *>(o_l);
    c->st.anchor = reinterpret_cast<int *>(o_a);
    c->st.meas = reinterpret_cast<MeasAcc *>(o_m);
    c->st.sk = reinterpret_cast<double *>(o_sk);
    c->st.dens = reinterpret_cast<unsigned long long *>(o_dn);
    c->st.sweep = reinterpret_cast<unsigned long long *>(o_sw);
    c->st.status = reinterpret_cast<unsigned *>(o_stt);
    c->st.gsig = reinterpret_cast<double *>(o_gs);
    c->st.gw = reinterpret_cast<void *>(o_gw);
    c->st.gw_f64 = f64 ? 1 : 0;
    c->st.logw_part = reinterpret_cast<double *>(o_lp);
    c->st.logw_err = reinterpret_cast<double *>(o_le);
    c->st.logw_err_part = reinterpret_cast<double *>(o_lep);
    c->st.blk_done = reinterpret_cast<unsigned *>(o_bd);
    c->st.perm = reinterpret_cast<int *>(o_pm);
    c->st.parity = reinterpret_cast<unsigned *>(o_par);
    return HQMC_OK;
}

template <typename P>
P rebase(P p, unsigned char *base) {
    return reinterpret_cast<P>(base + reinterpret_cast<size_t>(p));
}

// Plan, bind memory (attached or owned), upload tables and initialise the state.
int prepare(hqmc_ctx *c) {
    if (c->ready) return HQMC_OK;
    HQMC_CUDA(c, cudaSetDevice(c->device));
    size_t need = 0;
    int rc = plan_layout(c, &need);
    if (rc) return rc;
    if (c->attached) {
        if (c->attached_bytes < need) return fail(c, HQMC_ERR_NOMEM, "attached workspace too small");
        c->base = c->attached;
        c->own_mem = false;
    } else {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, HQMC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        c->base = static_cast<unsigned char *>(p);
        c->own_mem = true;
    }
    c->bytes = need;
    DevState &s = c->st;
    s.chains = rebase(s.chains, c->base);
    s.tabs = rebase(s.tabs, c->base);
    s.sbits = rebase(s.sbits, c->base);
    s.x = rebase(s.x, c->base);
    s.hist = rebase(s.hist, c->base);
    s.logw = rebase(s.logw, c->base);
    s.anchor = rebase(s.anchor, c->base);
    s.meas = rebase(s.meas, c->base);
    s.sk = rebase(s.sk, c->base);
    s.dens = rebase(s.dens, c->base);
    s.sweep = rebase(s.sweep, c->base);
    s.status = rebase(s.status, c->base);
    s.gsig = rebase(s.gsig, c->base);
    s.gw = rebase(s.gw, c->base);
    s.logw_part = rebase(s.logw_part, c->base);
    s.logw_err = rebase(s.logw_err, c->base);
    s.logw_err_part = rebase(s.logw_err_part, c->base);
    s.blk_done = rebase(s.blk_done, c->base);
    s.perm = rebase(s.perm, c->base);
    s.parity = rebase(s.parity, c->base);
    c->d_cr = reinterpret_cast<double *>(c->base + c->off_cr);
    s.open_acc = c->open_on ? reinterpret_cast<double *>(c->base + c->off_open) : nullptr;
    c->d_sko = reinterpret_cast<double *>(c->base + c->off_sko);
    c->d_rd = reinterpret_cast<double *>(c->base + c->off_rd);
    cudaStream_t st = c->stream;
    HQMC_CUDA(c, cudaMemsetAsync(c->base, 0, need, st));
    std::vector<ChainTab> tabs(c->nchains);
    for (int i = 0; i < c->nchains; ++i) build_tab(c->ch[i], tabs[i], c->cdev[i].lam);
    HQMC_CUDA(c, cudaMemcpyAsync((void *)s.chains, c->cdev.data(), sizeof(ChainDev) * c->nchains, cudaMemcpyHostToDevice, st));
    HQMC_CUDA(c, cudaMemcpyAsync((void *)s.tabs, tabs.data(), sizeof(ChainTab) * c->nchains, cudaMemcpyHostToDevice, st));
    for (auto &k : c->classes) {
        std::vector<int> buf(k.chains);
        buf.insert(buf.end(), k.pair_off.begin(), k.pair_off.end());
        buf.push_back(0);  // work counter
        buf.insert(buf.end(), k.unit_off.begin(), k.unit_off.end());
        HQMC_CUDA(c, cudaMemcpyAsync(c->base + k.cls_off, buf.data(), sizeof(int) * buf.size(), cudaMemcpyHostToDevice, st));
    }
    // kernel attributes are set here, outside any stream capture
    for (auto &k : c->classes) {
        int bps = 0;
        rc = occupancy(c, k.L, default_wpc(c, k.L), &bps);
        if (rc) return rc;
    }
    {
        int max_L = 0;
        for (auto &d : c->cdev) max_L = std::max(max_L, d.L);
        HQMC_CUDA(c, configure_slice(max_L, slice_group(max_L, c->slices_per_cta, slice_work(c), c->num_sms)));
    }
    {
        // permutations start at the identity (and so do their inverses); parity 0 = sign +1
        std::vector<int> ident;
        for (auto &d : c->cdev)
            for (int r = 0; r < 4; ++r)
                for (int p = 0; p < d.Nsig; ++p) ident.push_back(p);
        if (!ident.empty())
            HQMC_CUDA(c, cudaMemcpyAsync(s.perm, ident.data(), ident.size() * 4, cudaMemcpyHostToDevice, st));
        HQMC_CUDA(c, cudaStreamSynchronize(st));
    }
    cudaError_t e = launch_init_state(s, c->nchains, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "init_state");
    HQMC_CUDA(c, cudaStreamSynchronize(st));
    c->sweeps_host = 0;
    c->ready = true;
    c->started = false;
    if (c->pending_restore) {
        HQMC_CUDA(c, cudaMemcpy(c->st.sbits, c->keep_bits.data(), c->keep_bits.size() * 4, cudaMemcpyHostToDevice));
        HQMC_CUDA(c, cudaMemcpy(c->st.x, c->keep_x.data(), c->keep_x.size() * 2, cudaMemcpyHostToDevice));
        HQMC_CUDA(c, cudaMemcpy(c->st.sweep, &c->keep_sweep, 8, cudaMemcpyHostToDevice));
        if (!c->keep_perm.empty()) {
            HQMC_CUDA(c, cudaMemcpy(c->st.perm, c->keep_perm.data(), c->keep_perm.size() * 4, cudaMemcpyHostToDevice));
            HQMC_CUDA(c, cudaMemcpy(c->st.parity, c->keep_parity.data(), c->keep_parity.size() * 4, cudaMemcpyHostToDevice));
        }
        if (!c->keep_sig.empty()) {
            HQMC_CUDA(c, cudaMemcpy(c->st.gsig, c->keep_sig.data(), c->keep_sig.size() * 8, cudaMemcpyHostToDevice));
            for (int i = 0; i < c->nchains; ++i)
                if (c->cdev[i].gauss) {
                    cudaError_t e = launch_gauss_w(c->st, i, c->cdev[i].M, c->cdev[i].N, c->stream);
                    if (e != cudaSuccess) return cuda_fail(c, e, "gauss_w");
                }
            HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
        }
        c->sweeps_host = c->keep_sweep;
        c->started = c->keep_started;
        c->pending_restore = false;
    }
    return HQMC_OK;
}

// Keep the chain state (fields, worldlines, sweep counter) on the host and release the
// layout; the next prepare() lays the context out again and restores it.  Observable
// accumulators restart from zero.
int stash_state(hqmc_ctx *c) {
    if (!c->ready) {
        free_layout(c);
        return HQMC_OK;
    }
    size_t sb = 0, xb = 0;
    for (auto &d : c->cdev) {
        sb += 2ull * d.M * d.L * d.wpl;
        xb += 2ull * d.Nsig * d.M;
    }
    c->keep_bits.resize(sb);
    c->keep_x.resize(xb);
    long long gtot = 0;
    for (auto &d : c->cdev)
        if (d.gauss) gtot = std::max(gtot, d.g_off + ((long long)d.M * d.N + 3) / 4 * 4);
    c->keep_sig.resize(size_t(gtot));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (gtot) HQMC_CUDA(c, cudaMemcpy(c->keep_sig.data(), c->st.gsig, size_t(gtot) * 8, cudaMemcpyDeviceToHost));
    HQMC_CUDA(c, cudaMemcpy(c->keep_bits.data(), c->st.sbits, sb * 4, cudaMemcpyDeviceToHost));
    HQMC_CUDA(c, cudaMemcpy(c->keep_x.data(), c->st.x, xb * 2, cudaMemcpyDeviceToHost));
    HQMC_CUDA(c, cudaMemcpy(&c->keep_sweep, c->st.sweep, 8, cudaMemcpyDeviceToHost));
    size_t pb = 0;
    for (auto &d : c->cdev) pb += 4ull * d.Nsig;
    c->keep_perm.resize(pb);
    c->keep_parity.resize(c->cdev.size());
    if (pb) HQMC_CUDA(c, cudaMemcpy(c->keep_perm.data(), c->st.perm, pb * 4, cudaMemcpyDeviceToHost));
    HQMC_CUDA(c, cudaMemcpy(c->keep_parity.data(), c->st.parity, c->keep_parity.size() * 4, cudaMemcpyDeviceToHost));
    c->keep_started = c->started;
    c->pending_restore = true;
    free_layout(c);
    return HQMC_OK;
}

// NVTX range for the host-side enqueue of one phase (no-ops unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int enqueue_sweep(hqmc_ctx *c, cudaStream_t st, bool capture) {
    NvtxRange sweep_range("hqmc sweep");
    const bool f64 = c->precision == HQMC_FP64;
    const int nk = int(c->classes.size());
    const bool prof = !capture && c->prof_max > 0 && c->prof_n < c->prof_max;
    cudaEvent_t *pe = prof ? &c->prof_ev[4 * size_t(c->prof_n)] : nullptr;
    if (prof) HQMC_CUDA(c, cudaEventRecord(pe[0], st));
    // permutation update at tau = beta before the FFBS of the sweep (Sec. 3.5.3)
    if (c->perm_on) {
        NvtxRange r("hqmc permutations");
        int max_pairs = 0;
        for (auto &d : c->cdev) max_pairs = std::max(max_pairs, d.Nsig / 2);
        cudaError_t e = launch_perm(c->st, c->nchains, max_pairs, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "perm launch");
    }
    // fork: class k > 0 on aux stream k-1
    if (nk > 1) {
        while ((int)c->aux.size() < nk - 1) {
            cudaStream_t s;
            HQMC_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            c->aux.push_back(s);
        }
        while ((int)c->ev.size() < 2 * nk) {
            cudaEvent_t e;
            HQMC_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->ev.push_back(e);
        }
        HQMC_CUDA(c, cudaEventRecord(c->ev[0], st));
        for (int k = 1; k < nk; ++k) HQMC_CUDA(c, cudaStreamWaitEvent(c->aux[k - 1], c->ev[0], 0));
    }
    (void)capture;
    for (int k = 0; k < nk; ++k) {
        NvtxRange r("hqmc ffbs class");
        LClass &cl = c->classes[k];
        FfbsLaunch fl{};
        int *cls = reinterpret_cast<int *>(c->base + cl.cls_off);
        const size_t n = cl.chains.size();
        fl.class_chains = cls;
        fl.nclass = int(n);
        fl.next_unit = reinterpret_cast<unsigned *>(cls + n + (n + 1));
        fl.class_unit_off = cls + n + (n + 1) + 1;
        fl.total_units = cl.total_units;
        fl.len_max = cl.len_max;
        fl.general = (cl.total_units != cl.total_pairs || c->perm_used) ? 1 : 0;
        fl.stencil = (c->conv == HQMC_CONV_STENCIL && !is_big(cl.L)) ? 1 : 0;
        fl.scratch = c->base + cl.scratch_off;
        fl.slot_elems = cl.slot_elems;
        fl.ckpt_K = cl.ckpt_K;
        fl.ckpt_bf16 = c->fstore == HQMC_FSTORE_BF16 ? 1 : 0;
        fl.seg_off = cl.seg_off;
        cudaStream_t s = k == 0 ? st : c->aux[k - 1];
        HQMC_CUDA(c, cudaMemsetAsync(fl.next_unit, 0, sizeof(unsigned), s));
        const int wpc = default_wpc(c, cl.L);
        fl.gauss = 0;
        for (int ci : cl.chains) fl.gauss |= c->cdev[ci].gauss;
        cudaError_t e = is_big(cl.L) ? launch_ffbs_wide(cl.L, f64, c->st, fl, cl.grid, s)
                        : f64 ? (fl.gauss ? launch_ffbs_f64g(cl.L, c->st, fl, cl.grid, wpc, s)
                                          : launch_ffbs_f64(cl.L, c->st, fl, cl.grid, wpc, s))
                              : (fl.gauss ? launch_ffbs_f32g(cl.L, c->st, fl, cl.grid, wpc, s)
                                          : launch_ffbs_f32(cl.L, c->st, fl, cl.grid, wpc, s));
        if (e != cudaSuccess) return cuda_fail(c, e, "ffbs launch");
    }
    if (nk > 1) {
        for (int k = 1; k < nk; ++k) {
            HQMC_CUDA(c, cudaEventRecord(c->ev[k], c->aux[k - 1]));
            HQMC_CUDA(c, cudaStreamWaitEvent(st, c->ev[k], 0));
        }
    }
    if (prof) HQMC_CUDA(c, cudaEventRecord(pe[1], st));
    int max_M = 0;
    for (auto &d : c->cdev) max_M = std::max(max_M, d.M);
    if (prof) HQMC_CUDA(c, cudaEventRecord(pe[2], st));
    int max_L = 0;
    for (auto &d : c->cdev) max_L = std::max(max_L, d.L);
    const int sgroup = slice_group(max_L, c->slices_per_cta, slice_work(c), c->num_sms);
    nvtxRangePushA("hqmc gibbs+measure");
    cudaError_t e = launch_slice(c->st, c->nchains, max_M, max_L, sgroup, true, st);
    nvtxRangePop();
    if (e != cudaSuccess) return cuda_fail(c, e, "slice launch");
    if (prof) {
        HQMC_CUDA(c, cudaEventRecord(pe[3], st));
        ++c->prof_n;
    }
    e = launch_advance(c->st, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "advance launch");
    return HQMC_OK;
}

int check_status(hqmc_ctx *c) {
    unsigned stt = 0;
    HQMC_CUDA(c, cudaMemcpyAsync(&stt, c->st.status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (stt) {
        HQMC_CUDA(c, cudaMemsetAsync(c->st.status, 0, sizeof(unsigned), c->stream));
        return fail(c, HQMC_ERR_NUMERIC,
                    (stt & kStatusDegenerate) ? "a draw met an all-zero CDF" : "log Z met a non-positive amplitude");
    }
    return HQMC_OK;
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

const char *hqmc_strerror(int code) {
    switch (code) {
        case HQMC_OK: return "ok";
        case HQMC_ERR_ARG: return "invalid argument";
        case HQMC_ERR_NOMEM: return "out of device memory";
        case HQMC_ERR_CUDA: return "CUDA runtime error";
        case HQMC_ERR_TIMEOUT: return "device wait timed out";
        case HQMC_ERR_STATE: return "call out of order";
        case HQMC_ERR_UNSUPPORTED: return "unsupported lattice size or mode";
        case HQMC_ERR_NUMERIC: return "numerical degeneracy";
        case HQMC_ERR_SCRATCH: return "problem exceeds the static scratch of hqmc_ffbs_noalloc";
        default: return "unknown error";
    }
}

const char *hqmc_last_error_detail(hqmc_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int hqmc_supported_L(int *out, int cap) {
    int n = 0;
    for (int s : kSizes) {
        if (out && n < cap) out[n] = s;
        ++n;
    }
    return n;
}

int hqmc_init_lattice(hqmc_ctx **out, int n_chains, const int *L, const uint64_t *seeds, int precision, int device) {
    if (!out || !L || !seeds || n_chains < 1) return HQMC_ERR_ARG;
    if (precision != HQMC_FP32 && precision != HQMC_FP64) return HQMC_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n_chains; ++i) {
        if (L[i] < 2) return HQMC_ERR_ARG;
        const bool ok = ffbs_supported(L[i]) || ffbs_wide_supported(L[i]);
        if (!ok) return HQMC_ERR_UNSUPPORTED;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return HQMC_ERR_CUDA;
    }
    hqmc_ctx *c = new hqmc_ctx();
    c->device = device;
    c->precision = precision;
    c->nchains = n_chains;
    c->ch.resize(n_chains);
    for (int i = 0; i < n_chains; ++i) {
        c->ch[i].L = L[i];
        c->ch[i].N = L[i] * L[i];
        c->ch[i].seed = seeds[i];
    }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return HQMC_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return HQMC_ERR_CUDA;
    }
    c->own_stream = true;
    if (precision == HQMC_FP64) {
        c->use_graph = false;
        c->persistent = false;
    }
    *out = c;
    return HQMC_OK;
}

int hqmc_set_params(hqmc_ctx *c, int chain, double t, double U, double beta, double dtau, double filling) {
    if (!c) return HQMC_ERR_ARG;
    if (chain < -1 || chain >= c->nchains) return fail(c, HQMC_ERR_ARG, "chain index out of range");
    const int lo = chain < 0 ? 0 : chain, hi = chain < 0 ? c->nchains : chain + 1;
    for (int i = lo; i < hi; ++i) {
        int M = 0, Ns = 0;
        int rc = check_params(c, c->ch[i].L, t, U, beta, dtau, filling, &M, &Ns);
        if (rc) return rc;
        if (c->ready && (M != c->ch[i].M || Ns != c->ch[i].Nsig))
            return fail(c, HQMC_ERR_STATE, "M and Nsig are fixed once the state exists");
        if (c->ready && ((U < 0.0) != (c->ch[i].U < 0.0)))
            return fail(c, HQMC_ERR_STATE, "the field type (Hirsch for U >= 0, Gaussian for U < 0) is fixed once the state exists");
    }
    for (int i = lo; i < hi; ++i) {
        HostChain &h = c->ch[i];
        int M = 0, Ns = 0;
        check_params(c, h.L, t, U, beta, dtau, filling, &M, &Ns);
        h.t = t;
        h.U = U;
        h.beta = beta;
        h.dtau = dtau;
        h.filling = filling;
        h.M = M;
        h.Nsig = Ns;
        h.set = true;
    }
    if (c->ready) {
        // refresh per-chain tables and constants in place (shape unchanged)
        for (int i = lo; i < hi; ++i) {
            ChainDev &d = c->cdev[i];
            d.lam = hirsch_lambda(c->ch[i].U, c->ch[i].dtau);
            d.w_plus[0] = std::exp(d.lam);
            d.w_minus[0] = std::exp(-d.lam);
            d.w_plus[1] = std::exp(-d.lam);
            d.w_minus[1] = std::exp(d.lam);
            d.t = c->ch[i].t;
            d.beta = c->ch[i].beta;
            d.gcoup = std::sqrt(std::fabs(c->ch[i].U) * c->ch[i].dtau);
            ChainTab tb;
            build_tab(c->ch[i], tb, d.lam);
            HQMC_CUDA(c, cudaMemcpyAsync((void *)(c->st.chains + i), &d, sizeof(ChainDev), cudaMemcpyHostToDevice, c->stream));
            HQMC_CUDA(c, cudaMemcpyAsync((void *)(c->st.tabs + i), &tb, sizeof(ChainTab), cudaMemcpyHostToDevice, c->stream));
            if (d.gauss) {
                cudaError_t e = launch_gauss_w(c->st, i, d.M, d.N, c->stream);
                if (e != cudaSuccess) return cuda_fail(c, e, "gauss_w");
            }
        }
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HQMC_OK;
}

int hqmc_set_block(hqmc_ctx *c, int chain, int B) {
    if (!c) return HQMC_ERR_ARG;
    if (chain < -1 || chain >= c->nchains) return fail(c, HQMC_ERR_ARG, "chain index out of range");
    if (B < 0) return fail(c, HQMC_ERR_ARG, "block length must be >= 0");
    const int lo = chain < 0 ? 0 : chain, hi = chain < 0 ? c->nchains : chain + 1;
    bool changed = false;
    for (int i = lo; i < hi; ++i) {
        changed = changed || c->ch[i].block != B;
        c->ch[i].block = B;
    }
    // the work-unit tables, partial sums and scratch depend on the blocks: lay the context
    // out again at its next use, keeping the state
    if (changed) return stash_state(c);
    return HQMC_OK;
}

int hqmc_set_conv(hqmc_ctx *c, int kind) {
    if (!c || (kind != HQMC_CONV_FFT && kind != HQMC_CONV_STENCIL)) return HQMC_ERR_ARG;
    if (kind == HQMC_CONV_STENCIL)
        for (auto &h : c->ch)
            if (is_big(h.L)) return fail(c, HQMC_ERR_UNSUPPORTED, "the stencil form covers L <= 32");
    c->conv = kind;
    drop_graph(c);
    return HQMC_OK;
}

int hqmc_set_permutations(hqmc_ctx *c, int on) {
    if (!c) return HQMC_ERR_ARG;
    if (on) {
        for (auto &h : c->ch) {
            if (!h.set) return fail(c, HQMC_ERR_STATE, "set_params has not been called for every chain");
            if (h.M < 2) return fail(c, HQMC_ERR_UNSUPPORTED, "permutation updates need M >= 2");
        }
        c->perm_used = true;
    }
    c->perm_on = on != 0;
    drop_graph(c);  // the captured sweep changes
    return HQMC_OK;
}

int hqmc_get_perm(hqmc_ctx *c, int chain, int32_t *perm, int *sign) {
    if (!c || chain < 0 || chain >= c->nchains) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    if (perm)
        HQMC_CUDA(c, cudaMemcpyAsync(perm, c->st.perm + d.perm_off, 2ull * d.Nsig * 4, cudaMemcpyDeviceToHost, c->stream));
    unsigned par = 0;
    HQMC_CUDA(c, cudaMemcpyAsync(&par, c->st.parity + chain, 4, cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sign) *sign = (par & 1u) ? -1 : 1;
    return HQMC_OK;
}

int hqmc_set_perm(hqmc_ctx *c, int chain, const int32_t *perm) {
    if (!c || !perm || chain < 0 || chain >= c->nchains) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    const int Ns = d.Nsig;
    std::vector<int> buf(4ull * Ns);
    unsigned par = 0;
    for (int sg = 0; sg < 2; ++sg) {
        std::vector<char> seen(Ns, 0);
        for (int p = 0; p < Ns; ++p) {
            const int q = perm[sg * Ns + p];
            if (q < 0 || q >= Ns || seen[q]) return fail(c, HQMC_ERR_ARG, "not a permutation of the worldlines");
            seen[q] = 1;
            buf[sg * Ns + p] = q;
            buf[2 * Ns + sg * Ns + q] = p;
        }
        // parity: (length - 1) summed over the cycles
        std::vector<char> vis(Ns, 0);
        for (int p = 0; p < Ns; ++p) {
            if (vis[p]) continue;
            int len = 0;
            for (int j = p; !vis[j]; j = perm[sg * Ns + j]) {
                vis[j] = 1;
                ++len;
            }
            par ^= unsigned(len - 1) & 1u;
        }
    }
    if (Ns > 0) {
        c->perm_used = true;
        drop_graph(c);
        HQMC_CUDA(c, cudaMemcpyAsync(c->st.perm + d.perm_off, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice, c->stream));
    }
    HQMC_CUDA(c, cudaMemcpyAsync(c->st.parity + chain, &par, 4, cudaMemcpyHostToDevice, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HQMC_OK;
}

int hqmc_set_ffbs_storage(hqmc_ctx *c, int kind, int stride) {
    if (!c) return HQMC_ERR_ARG;
    if (kind != HQMC_FSTORE_STREAM && kind != HQMC_FSTORE_BF16 && kind != HQMC_FSTORE_F32)
        return fail(c, HQMC_ERR_ARG, "unknown storage kind");
    if (stride < 0) return fail(c, HQMC_ERR_ARG, "stride must be >= 0");
    if (kind != HQMC_FSTORE_STREAM && c->precision == HQMC_FP64)
        return fail(c, HQMC_ERR_UNSUPPORTED, "checkpoints of f are built for the FP32 filter");
    const bool changed = kind != c->fstore || stride != c->fstride;
    c->fstore = kind;
    c->fstride = stride;
    // the scratch layout depends on it: lay out again at the next use, keeping the state
    if (changed) return stash_state(c);
    return HQMC_OK;
}

int hqmc_set_stream(hqmc_ctx *c, void *stream) {
    if (!c) return HQMC_ERR_ARG;
    drop_graph(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->own_stream = false;
    c->stream = static_cast<cudaStream_t>(stream);
    if (!c->stream) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return HQMC_ERR_CUDA;
        c->own_stream = true;
    }
    return HQMC_OK;
}

int hqmc_set_launch(hqmc_ctx *c, int use_graph, int persistent, int warps_per_cta) {
    if (!c) return HQMC_ERR_ARG;
    if (warps_per_cta != 0 && warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(c, HQMC_ERR_ARG, "warps_per_cta must be 0, 1, 2, 4 or 8");
    const bool relayout = (bool(persistent) != c->persistent) || (warps_per_cta != c->wpc);
    c->use_graph = use_graph != 0;
    c->persistent = persistent != 0;
    c->wpc = warps_per_cta;
    drop_graph(c);
    // the scratch size depends on the grid: lay out again at the next use, keeping the state
    if (relayout) return stash_state(c);
    return HQMC_OK;
}

int hqmc_set_slice_launch(hqmc_ctx *c, int slices_per_cta) {
    if (!c || slices_per_cta < 0 || slices_per_cta > 1024) return HQMC_ERR_ARG;
    c->slices_per_cta = slices_per_cta;
    drop_graph(c);
    if (c->ready) {
        // the kernel's shared memory follows the group size (set here, outside any capture)
        int max_L = 0;
        for (auto &d : c->cdev) max_L = std::max(max_L, d.L);
        HQMC_CUDA(c, configure_slice(max_L, slice_group(max_L, c->slices_per_cta, slice_work(c), c->num_sms)));
    }
    return HQMC_OK;
}

int hqmc_set_class_launch(hqmc_ctx *c, int L, int warps_per_cta) {
    if (!c) return HQMC_ERR_ARG;
    if (warps_per_cta != 0 && warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(c, HQMC_ERR_ARG, "warps_per_cta must be 0, 1, 2, 4 or 8");
    bool found = false;
    for (auto &h : c->ch) found = found || h.L == L;
    if (!found) return fail(c, HQMC_ERR_ARG, "no chain of this lattice size");
    const int before = default_wpc(c, L);
    bool set = false;
    for (auto &kv : c->class_wpc)
        if (kv.first == L) {
            kv.second = warps_per_cta;
            set = true;
        }
    if (!set) c->class_wpc.push_back({L, warps_per_cta});
    drop_graph(c);
    if (default_wpc(c, L) != before) return stash_state(c);
    return HQMC_OK;
}

int hqmc_get_class_launch(hqmc_ctx *c, int L, int *warps_per_cta) {
    if (!c || !warps_per_cta) return HQMC_ERR_ARG;
    *warps_per_cta = L > 32 ? 0 : default_wpc(c, L);
    return HQMC_OK;
}

int hqmc_autotune(hqmc_ctx *c, int trial_sweeps, int *n_tuned) {
    if (!c || trial_sweeps < 1) return HQMC_ERR_ARG;
    for (auto &h : c->ch)
        if (!h.set) return fail(c, HQMC_ERR_STATE, "set_params has not been called for every chain");
    std::vector<int> sizes;
    for (auto &h : c->ch)
        if (h.L <= 32 && std::find(sizes.begin(), sizes.end(), h.L) == sizes.end()) sizes.push_back(h.L);
    int tuned = 0;
    for (int L : sizes) {
        // a throwaway context with this size's chains: same parameters, seeds and precision
        std::vector<int> Ls;
        std::vector<uint64_t> seeds;
        std::vector<const HostChain *> hs;
        for (auto &h : c->ch)
            if (h.L == L) {
                Ls.push_back(h.L);
                seeds.push_back(h.seed);
                hs.push_back(&h);
            }
        hqmc_ctx *t = nullptr;
        int rc = hqmc_init_lattice(&t, int(Ls.size()), Ls.data(), seeds.data(), c->precision, c->device);
        if (rc) return fail(c, rc, "autotune: temporary context");
        for (size_t i = 0; i < hs.size(); ++i) {
            rc = hqmc_set_params(t, int(i), hs[i]->t, hs[i]->U, hs[i]->beta, hs[i]->dtau, hs[i]->filling);
            if (!rc) rc = hqmc_set_block(t, int(i), hs[i]->block);
            if (rc) break;
        }
        // the trial runs the kernel instantiation the context itself runs
        if (!rc) rc = hqmc_set_conv(t, c->conv);
        if (!rc && c->perm_used) rc = hqmc_set_permutations(t, c->perm_on ? 1 : 0);
        if (!rc && c->perm_used && !c->perm_on) t->perm_used = true;
        int best = 0;
        float best_ms = 0.f;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = HQMC_ERR_CUDA;
        for (int w : {1, 2, 4, 8}) {
            if (rc) break;
            rc = hqmc_set_launch(t, c->use_graph ? 1 : 0, c->persistent ? 1 : 0, w);
            if (!rc) rc = hqmc_sweep(t, 2, nullptr);  // warm-up (and graph capture)
            if (rc) break;
            cudaEventRecord(e0, t->stream);
            rc = hqmc_sweep(t, trial_sweeps, nullptr);
            cudaEventRecord(e1, t->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = HQMC_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!rc && (best == 0 || ms < best_ms)) {
                best = w;
                best_ms = ms;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        const std::string detail = t->err;
        hqmc_destroy(t);
        if (rc) return fail(c, rc, "autotune: " + detail);
        rc = hqmc_set_class_launch(c, L, best);
        if (rc) return rc;
        ++tuned;
    }
    if (n_tuned) *n_tuned = tuned;
    return HQMC_OK;
}

int hqmc_workspace_size(hqmc_ctx *c, size_t *bytes) {
    if (!c || !bytes) return HQMC_ERR_ARG;
    size_t need = 0;
    DevState keep = c->st;
    auto keep_cdev = c->cdev;
    auto keep_cls = c->classes;
    int rc = plan_layout(c, &need);
    if (c->ready) {
        c->st = keep;
        c->cdev = keep_cdev;
        c->classes = keep_cls;
    }
    if (rc) return rc;
    *bytes = need;
    return HQMC_OK;
}

int hqmc_attach_workspace(hqmc_ctx *c, void *dev_ptr, size_t bytes) {
    if (!c || !dev_ptr) return HQMC_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) return fail(c, HQMC_ERR_ARG, "workspace must be 256-byte aligned");
    free_layout(c);  // a stashed state (after a launch-shape change) is restored by prepare()
    c->attached = static_cast<unsigned char *>(dev_ptr);
    c->attached_bytes = bytes;
    size_t need = 0;
    int rc = plan_layout(c, &need);
    if (rc) return rc;
    if (bytes < need) {
        c->attached = nullptr;
        c->attached_bytes = 0;
        return fail(c, HQMC_ERR_NOMEM, "workspace smaller than hqmc_workspace_size");
    }
    return prepare(c);
}

int hqmc_sweep(hqmc_ctx *c, int n_sweeps, double *logw_out) {
    if (!c || n_sweeps < 0) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    HQMC_CUDA(c, cudaSetDevice(c->device));
    if (c->use_graph && c->prof_max == 0 && !c->exec && n_sweeps > 0) {
        HQMC_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_sweep(c, c->stream, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        c->graph = g;
        e = cudaGraphInstantiate(&c->exec, g, 0);
        if (e != cudaSuccess) {
            drop_graph(c);
            return cuda_fail(c, e, "graph instantiate");
        }
    }
    const bool graph = c->use_graph && c->prof_max == 0;
    for (int i = 0; i < n_sweeps; ++i) {
        if (graph) {
            HQMC_CUDA(c, cudaGraphLaunch(c->exec, c->stream));
        } else {
            rc = enqueue_sweep(c, c->stream, false);
            if (rc) return rc;
        }
    }
    c->sweeps_host += n_sweeps;
    if (n_sweeps > 0) c->started = true;
    if (logw_out)
        HQMC_CUDA(c, cudaMemcpyAsync(logw_out, c->st.logw, sizeof(double) * c->total_wl, cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

int hqmc_logw_error(hqmc_ctx *c, double *err_out) {
    if (!c || !err_out) return HQMC_ERR_ARG;
    if (!c->ready || !c->started) return fail(c, HQMC_ERR_STATE, "no sweep has run");
    HQMC_CUDA(c, cudaSetDevice(c->device));
    HQMC_CUDA(c, cudaMemcpyAsync(err_out, c->st.logw_err, sizeof(double) * c->total_wl, cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HQMC_OK;
}

int hqmc_local_sweep(hqmc_ctx *c, int n_sweeps) {
    if (!c || n_sweeps < 0) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    HQMC_CUDA(c, cudaSetDevice(c->device));
    int max_units = 0, max_M = 0, max_L = 0;
    for (auto &d : c->cdev) {
        max_units = std::max(max_units, local_max_units(d.M, d.Nsig));
        max_M = std::max(max_M, d.M);
        max_L = std::max(max_L, d.L);
    }
    for (int i = 0; i < n_sweeps; ++i) {
        for (int color = 0; color < 3; ++color) {
            cudaError_t e = launch_local(c->st, c->nchains, max_units, color, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "local launch");
        }
        cudaError_t e = launch_slice(c->st, c->nchains, max_M, max_L, slice_group(max_L, c->slices_per_cta, slice_work(c), c->num_sms), true,
                                     c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "slice launch");
        e = launch_advance(c->st, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "advance launch");
    }
    c->sweeps_host += n_sweeps;
    if (n_sweeps > 0) c->started = true;
    return check_status(c);
}

int hqmc_measure(hqmc_ctx *c, hqmc_obs *out, double *Sk, double *Cr, int reset) {
    if (!c) return HQMC_ERR_ARG;
    if (!c->ready) return fail(c, HQMC_ERR_STATE, "no state yet");
    int max_N = 0;
    for (auto &d : c->cdev) max_N = std::max(max_N, d.N);
    cudaError_t e = launch_readout(c->st, c->nchains, max_N, c->d_cr, c->d_sko, c->d_rd, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "readout");
    std::vector<MeasAcc> acc(c->nchains);
    HQMC_CUDA(c, cudaMemcpyAsync(acc.data(), c->st.meas, sizeof(MeasAcc) * c->nchains, cudaMemcpyDeviceToHost, c->stream));
    if (Sk) HQMC_CUDA(c, cudaMemcpyAsync(Sk, c->d_sko, 8 * c->total_N, cudaMemcpyDeviceToHost, c->stream));
    if (Cr) HQMC_CUDA(c, cudaMemcpyAsync(Cr, c->d_cr, 8 * c->total_N, cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> skh(c->total_N);
    HQMC_CUDA(c, cudaMemcpyAsync(skh.data(), c->d_sko, 8 * c->total_N, cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (out) {
        for (int i = 0; i < c->nchains; ++i) {
            const ChainDev &d = c->cdev[i];
            // sign-reweighted averages (Eq. reweight): the sums are sign-weighted and divided
            // by the sum of signs, which equals the sample count without permutations
            const double ns = double(acc[i].sign_sum);
            const double denom = ns * d.M * d.N;
            hqmc_obs &o = out[i];
            o.n_samples = (int64_t)acc[i].samples;
            o.density = denom != 0 ? double((long long)acc[i].n_sum) / denom : 0.0;
            o.double_occ = denom != 0 ? double((long long)acc[i].d_sum) / denom : 0.0;
            o.m2 = denom != 0 ? double((long long)acc[i].m2_sum) / denom : 0.0;
            o.ekin = ns != 0 ? -(c->ch[i].t / c->ch[i].beta) * acc[i].link_sum / (ns * d.N) : 0.0;
            o.mean_sign = acc[i].samples ? ns / double(acc[i].samples) : 1.0;
            o.n_perm_accepted = (int64_t)acc[i].perm_accepted;
            const int kh = d.L / 2;
            o.s_pipi = skh[d.meas_off + kh + d.L * kh];
            o.n_degenerate = (int64_t)acc[i].degenerate;
            o.n_nonpositive = (int64_t)acc[i].nonpositive;
            o.n_local_accepted = (int64_t)acc[i].local_accepted;
            o.n_inexact = (int64_t)acc[i].inexact;
        }
    }
    if (reset) {
        HQMC_CUDA(c, cudaMemsetAsync(c->st.meas, 0, sizeof(MeasAcc) * c->nchains, c->stream));
        HQMC_CUDA(c, cudaMemsetAsync(c->st.sk, 0, 8 * c->total_N, c->stream));
        HQMC_CUDA(c, cudaMemsetAsync(c->base + c->off_open, 0, 8 * c->total_N, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HQMC_OK;
}

int hqmc_set_measure_open(hqmc_ctx *c, int on) {
    if (!c) return HQMC_ERR_ARG;
    c->open_on = on != 0;
    drop_graph(c);  // the captured sweep holds the device state by value
    if (c->ready) {
        HQMC_CUDA(c, cudaSetDevice(c->device));
        c->st.open_acc = c->open_on ? reinterpret_cast<double *>(c->base + c->off_open) : nullptr;
        // every accumulator restarts, so that the open-path sums and the sign sum cover the
        // same sweeps
        HQMC_CUDA(c, cudaMemsetAsync(c->st.meas, 0, sizeof(MeasAcc) * c->nchains, c->stream));
        HQMC_CUDA(c, cudaMemsetAsync(c->st.sk, 0, 8 * c->total_N, c->stream));
        HQMC_CUDA(c, cudaMemsetAsync(c->base + c->off_open, 0, 8 * c->total_N, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HQMC_OK;
}

int hqmc_measure_open(hqmc_ctx *c, double *nk, double *dm) {
    if (!c) return HQMC_ERR_ARG;
    if (!c->ready || !c->open_on) return fail(c, HQMC_ERR_STATE, "the open-path estimator is off");
    HQMC_CUDA(c, cudaSetDevice(c->device));
    int max_N = 0;
    for (auto &d : c->cdev) max_N = std::max(max_N, d.N);
    // the read-out uses the S(k) / C(r) output arrays as its destination
    cudaError_t e = launch_readout_open(c->st, c->nchains, max_N, c->d_cr, c->d_sko, c->d_rd, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "open readout");
    if (nk) HQMC_CUDA(c, cudaMemcpyAsync(nk, c->d_cr, 8 * c->total_N, cudaMemcpyDeviceToHost, c->stream));
    if (dm) HQMC_CUDA(c, cudaMemcpyAsync(dm, c->d_sko, 8 * c->total_N, cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HQMC_OK;
}

int hqmc_chain_shape(hqmc_ctx *c, int chain, int *L, int *M, int *Nsig) {
    if (!c || chain < 0 || chain >= c->nchains) return HQMC_ERR_ARG;
    if (L) *L = c->ch[chain].L;
    if (M) *M = c->ch[chain].M;
    if (Nsig) *Nsig = c->ch[chain].Nsig;
    return HQMC_OK;
}

int hqmc_get_state(hqmc_ctx *c, int chain, int8_t *s, int32_t *x, int *anchor, uint64_t *sweeps) {
    if (!c || chain < 0 || chain >= c->nchains) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    if (s && d.gauss) std::memset(s, 0, size_t(d.M) * d.N);
    if (s && !d.gauss) {
        std::vector<uint32_t> bits(size_t(d.M) * d.L * d.wpl);
        HQMC_CUDA(c, cudaMemcpyAsync(bits.data(), c->st.sbits + d.s_off, bits.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int l = 0; l < d.M; ++l)
            for (int iy = 0; iy < d.L; ++iy)
                for (int ix = 0; ix < d.L; ++ix) {
                    const uint32_t w = bits[(size_t(l) * d.L + iy) * d.wpl + (ix >> 5)];
                    s[size_t(l) * d.N + ix + d.L * iy] = ((w >> (ix & 31)) & 1u) ? 1 : -1;
                }
    }
    if (x) {
        std::vector<int16_t> xs(2ull * d.Nsig * d.M);
        HQMC_CUDA(c, cudaMemcpyAsync(xs.data(), c->st.x + d.x_off, xs.size() * 2, cudaMemcpyDeviceToHost, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
        for (size_t k = 0; k < xs.size(); ++k) x[k] = xs[k];
    }
    if (anchor) {
        HQMC_CUDA(c, cudaMemcpyAsync(anchor, c->st.anchor + chain, 4, cudaMemcpyDeviceToHost, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (sweeps) {
        unsigned long long sw = 0;
        HQMC_CUDA(c, cudaMemcpyAsync(&sw, c->st.sweep, 8, cudaMemcpyDeviceToHost, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
        *sweeps = sw;
    }
    return HQMC_OK;
}

int hqmc_get_sigma(hqmc_ctx *c, int chain, double *sigma) {
    if (!c || chain < 0 || chain >= c->nchains || !sigma) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    if (!d.gauss) return fail(c, HQMC_ERR_ARG, "chain has the Hirsch field (U >= 0): use hqmc_get_state");
    HQMC_CUDA(c, cudaMemcpyAsync(sigma, c->st.gsig + d.g_off, sizeof(double) * d.M * d.N, cudaMemcpyDeviceToHost, c->stream));
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HQMC_OK;
}

int hqmc_set_sigma(hqmc_ctx *c, int chain, const double *sigma) {
    if (!c || chain < 0 || chain >= c->nchains || !sigma) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    if (!d.gauss) return fail(c, HQMC_ERR_ARG, "chain has the Hirsch field (U >= 0): use hqmc_set_state");
    for (long long k = 0; k < (long long)d.M * d.N; ++k)
        if (!std::isfinite(sigma[k])) return fail(c, HQMC_ERR_ARG, "field values must be finite");
    HQMC_CUDA(c, cudaMemcpyAsync(c->st.gsig + d.g_off, sigma, sizeof(double) * d.M * d.N, cudaMemcpyHostToDevice, c->stream));
    cudaError_t e = launch_gauss_w(c->st, chain, d.M, d.N, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "gauss_w");
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HQMC_OK;
}

int hqmc_set_state(hqmc_ctx *c, int chain, const int8_t *s, const int32_t *x, const uint64_t *sweeps) {
    if (!c || chain < 0 || chain >= c->nchains) return HQMC_ERR_ARG;
    int rc = prepare(c);
    if (rc) return rc;
    const ChainDev &d = c->cdev[chain];
    if (s && d.gauss) return fail(c, HQMC_ERR_ARG, "chain has the Gaussian field (U < 0): use hqmc_set_sigma");
    if (s) {
        std::vector<uint32_t> rows(size_t(d.M) * d.L * d.wpl, 0u), cols(rows.size(), 0u);
        for (int l = 0; l < d.M; ++l)
            for (int iy = 0; iy < d.L; ++iy)
                for (int ix = 0; ix < d.L; ++ix) {
                    const int8_t v = s[size_t(l) * d.N + ix + d.L * iy];
                    if (v != 1 && v != -1) return fail(c, HQMC_ERR_ARG, "field values must be +1 or -1");
                    if (v == 1) {
                        rows[(size_t(l) * d.L + iy) * d.wpl + (ix >> 5)] |= 1u << (ix & 31);
                        cols[(size_t(l) * d.L + ix) * d.wpl + (iy >> 5)] |= 1u << (iy & 31);
                    }
                }
        HQMC_CUDA(c, cudaMemcpyAsync(c->st.sbits + d.s_off, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, c->stream));
        HQMC_CUDA(c, cudaMemcpyAsync(c->st.sbits + d.s_off + rows.size(), cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (x) {
        std::vector<int16_t> xs(2ull * d.Nsig * d.M);
        for (size_t k = 0; k < xs.size(); ++k) {
            if (x[k] < 0 || x[k] >= d.N) return fail(c, HQMC_ERR_ARG, "site index out of range");
            xs[k] = int16_t(x[k]);
        }
        HQMC_CUDA(c, cudaMemcpyAsync(c->st.x + d.x_off, xs.data(), xs.size() * 2, cudaMemcpyHostToDevice, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (sweeps) {
        unsigned long long sw = *sweeps;
        HQMC_CUDA(c, cudaMemcpyAsync(c->st.sweep, &sw, 8, cudaMemcpyHostToDevice, c->stream));
        HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
        c->sweeps_host = sw;
    }
    return HQMC_OK;
}

int hqmc_set_checkpoint(hqmc_ctx *c, int stride, int kind) {
    if (!c) return HQMC_ERR_ARG;
    if (stride < 0) return fail(c, HQMC_ERR_ARG, "checkpoint stride must be >= 0");
    if (kind != HQMC_CKPT_BF16 && kind != HQMC_CKPT_FULL) return fail(c, HQMC_ERR_ARG, "unknown checkpoint kind");
    c->ckpt_stride = stride;
    c->ckpt_kind = kind;
    return HQMC_OK;
}

int hqmc_log_weight_grad(hqmc_ctx *c, const void *v, double *logZ, void *dlogZ_dv, double *dlogZ_dt) {
    if (!c) return HQMC_ERR_ARG;
    if (c->perm_used) return fail(c, HQMC_ERR_UNSUPPORTED, "the adjoint is of closed loops; permutations are in use");
    int rc = prepare(c);
    if (rc) return rc;
    HQMC_CUDA(c, cudaSetDevice(c->device));
    const bool f64 = c->precision == HQMC_FP64;
    const bool bf16 = !f64 && c->ckpt_kind == HQMC_CKPT_BF16;
    const size_t vsz = f64 ? 16 : 8;             // one element of a worldline pair
    const size_t tsz = f64 ? 8 : 4;              // one element of v / dv
    struct Plan {
        int K, nseg, grid;
        long long groups;
        size_t ck_bytes, ck_exp_off, seg_elems, off;
    };
    std::vector<Plan> plans(c->classes.size());
    const size_t head = size_t(c->nchains) * 16 + c->classes.size() * 4;  // logz, dt per chain; counters
    size_t off = round_up(head, 256);
    for (size_t k = 0; k < c->classes.size(); ++k) {
        const LClass &cl = c->classes[k];
        Plan &p = plans[k];
        const int M = cl.M_max;
        p.K = c->ckpt_stride > 0 ? std::min(c->ckpt_stride, M) : std::max(1, int(std::ceil(std::sqrt(double(M)))));
        p.nseg = (M + p.K - 1) / p.K;
        const size_t N = size_t(cl.L) * cl.L;
        if (is_big(cl.L)) {
            // wide: one CTA per group of WPC worldlines; per worldline the checkpoints (BF16 or
            // the context precision) and a segment of K slices plus a spare one for b
            const int wpc = ffbs_wide_wpc(cl.L);
            p.ck_exp_off = 0;
            p.ck_bytes = size_t(wpc) * round_up(size_t(p.nseg) * N * (bf16 ? 2 : tsz), 256);
            p.seg_elems = size_t(wpc) * (size_t(p.K) + 1) * N;
            int bps = 1;
            cudaError_t e = grad_wide_occupancy(cl.L, f64, &bps);
            if (e != cudaSuccess) return cuda_fail(c, e, "grad occupancy");
            bps = std::max(1, bps);
            p.grid = std::max(1, std::min(cl.total_pairs, bps * c->num_sms));
            p.groups = p.grid;
            p.off = off;
            off = round_up(off + size_t(p.groups) * (p.ck_bytes + p.seg_elems * tsz), 256);
            continue;
        }
        p.ck_exp_off = round_up(size_t(p.nseg) * N * (bf16 ? 4 : vsz), 16);
        p.ck_bytes = round_up(p.ck_exp_off + size_t(p.nseg) * 8, 256);
        p.seg_elems = size_t(p.K) * N;
        int bps = 1;
        cudaError_t e = f64 ? grad_occupancy_f64(cl.L, &bps) : grad_occupancy_f32(cl.L, &bps);
        if (e != cudaSuccess) return cuda_fail(c, e, "grad occupancy");
        bps = std::max(1, bps);
        const int gpc = kGradWarpsHost * ffbs_groups_per_warp(cl.L);
        const int need = (cl.total_pairs + gpc - 1) / gpc;
        p.grid = std::max(1, std::min(need, bps * c->num_sms));
        p.groups = (long long)p.grid * gpc;
        p.off = off;
        off = round_up(off + size_t(p.groups) * (p.ck_bytes + p.seg_elems * vsz), 256);
    }
    if (off > c->grad_bytes) {
        if (c->grad_mem) cudaFree(c->grad_mem);
        c->grad_mem = nullptr;
        c->grad_bytes = 0;
        void *m = nullptr;
        cudaError_t e = cudaMalloc(&m, off);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, HQMC_ERR_NOMEM, std::string("cudaMalloc (adjoint scratch): ") + cudaGetErrorString(e));
        }
        c->grad_mem = static_cast<unsigned char *>(m);
        c->grad_bytes = off;
    }
    cudaStream_t st = c->stream;
    double *d_logz = reinterpret_cast<double *>(c->grad_mem);
    double *d_dt = d_logz + c->nchains;
    unsigned *d_next = reinterpret_cast<unsigned *>(d_dt + c->nchains);
    HQMC_CUDA(c, cudaMemsetAsync(d_logz, 0, head, st));
    if (dlogZ_dv) HQMC_CUDA(c, cudaMemsetAsync(dlogZ_dv, 0, size_t(c->total_v) * tsz, st));
    for (size_t k = 0; k < c->classes.size(); ++k) {
        const LClass &cl = c->classes[k];
        const Plan &p = plans[k];
        GradLaunch gk{};
        gk.class_chains = reinterpret_cast<const int *>(c->base + cl.cls_off);
        gk.class_pair_off = gk.class_chains + cl.chains.size();
        gk.nclass = int(cl.chains.size());
        gk.total_pairs = cl.total_pairs;
        gk.K = p.K;
        gk.ckpt_bf16 = bf16 ? 1 : 0;
        gk.ckpt = c->grad_mem + p.off;
        gk.ckpt_bytes = (long long)p.ck_bytes;
        gk.ckpt_exp_off = (long long)p.ck_exp_off;
        gk.seg = c->grad_mem + p.off + size_t(p.groups) * p.ck_bytes;
        gk.seg_elems = (long long)p.seg_elems;
        gk.v = v;
        gk.dv = dlogZ_dv;
        gk.logz = d_logz;
        gk.dt = d_dt;
        gk.next_pair = d_next + k;
        cudaError_t e = is_big(cl.L) ? launch_grad_wide(cl.L, f64, c->st, gk, p.grid, st)
                        : f64        ? launch_grad_f64(cl.L, c->st, gk, p.grid, st)
                                     : launch_grad_f32(cl.L, c->st, gk, p.grid, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "grad launch");
    }
    std::vector<double> h(2 * size_t(c->nchains));
    HQMC_CUDA(c, cudaMemcpyAsync(h.data(), d_logz, h.size() * 8, cudaMemcpyDeviceToHost, st));
    HQMC_CUDA(c, cudaStreamSynchronize(st));
    if (logZ) std::memcpy(logZ, h.data(), size_t(c->nchains) * 8);
    if (dlogZ_dt) std::memcpy(dlogZ_dt, h.data() + c->nchains, size_t(c->nchains) * 8);
    return check_status(c);
}

int hqmc_set_profiling(hqmc_ctx *c, int max_sweeps) {
    if (!c || max_sweeps < 0) return HQMC_ERR_ARG;
    for (auto e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_max = 0;
    c->prof_n = 0;
    if (max_sweeps > 0) {
        c->prof_ev.resize(4 * size_t(max_sweeps));
        for (auto &e : c->prof_ev) HQMC_CUDA(c, cudaEventCreate(&e));
        c->prof_max = max_sweeps;
    }
    return HQMC_OK;
}

int hqmc_profile_read(hqmc_ctx *c, double *ffbs_ms, double *slice_ms, int *n_sweeps) {
    if (!c) return HQMC_ERR_ARG;
    if (c->prof_max == 0) return fail(c, HQMC_ERR_STATE, "profiling is off");
    HQMC_CUDA(c, cudaStreamSynchronize(c->stream));
    double fs = 0.0, ss = 0.0;
    for (int i = 0; i < c->prof_n; ++i) {
        float a = 0.f, b = 0.f;
        HQMC_CUDA(c, cudaEventElapsedTime(&a, c->prof_ev[4 * i], c->prof_ev[4 * i + 1]));
        HQMC_CUDA(c, cudaEventElapsedTime(&b, c->prof_ev[4 * i + 2], c->prof_ev[4 * i + 3]));
        fs += a;
        ss += b;
    }
    if (ffbs_ms) *ffbs_ms = fs;
    if (slice_ms) *slice_ms = ss;
    if (n_sweeps) *n_sweeps = c->prof_n;
    c->prof_n = 0;
    return HQMC_OK;
}

void hqmc_destroy(hqmc_ctx *c) {
    if (!c) return;
    for (auto e : c->prof_ev) cudaEventDestroy(e);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_layout(c);
    if (c->grad_mem) cudaFree(c->grad_mem);
    for (auto s : c->aux) cudaStreamDestroy(s);
    for (auto e : c->ev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
#pragma GCC visibility pop
