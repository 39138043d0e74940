"""Python binding of the hqmc C ABI (include/hqmc.h): argument marshalling only.

Every step of a sweep runs in the CUDA kernels of libhqmc.so; PyTorch supplies the
device memory (the context's workspace is a torch uint8 tensor) and the stream.
There is no CPU fallback: if the library cannot be loaded this module raises.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhqmc.so")

HQMC_FP32, HQMC_FP64 = 0, 1
HQMC_CKPT_BF16, HQMC_CKPT_FULL = 0, 1
ERRORS = {
    -1: "HQMC_ERR_ARG", -2: "HQMC_ERR_NOMEM", -3: "HQMC_ERR_CUDA", -4: "HQMC_ERR_TIMEOUT",
    -5: "HQMC_ERR_STATE", -6: "HQMC_ERR_UNSUPPORTED", -7: "HQMC_ERR_NUMERIC", -8: "HQMC_ERR_SCRATCH",
}

# every entry point declared in include/hqmc.h, with its ctypes signature
_vp, _i, _d, _sz, _u64 = C.c_void_p, C.c_int, C.c_double, C.c_size_t, C.c_uint64
SIGNATURES = {
    "hqmc_init_lattice": (_i, [C.POINTER(_vp), _i, _vp, _vp, _i, _i]),
    "hqmc_set_params": (_i, [_vp, _i, _d, _d, _d, _d, _d]),
    "hqmc_set_block": (_i, [_vp, _i, _i]),
    "hqmc_set_ffbs_storage": (_i, [_vp, _i, _i]),
    "hqmc_set_stream": (_i, [_vp, _vp]),
    "hqmc_set_launch": (_i, [_vp, _i, _i, _i]),
    "hqmc_set_slice_launch": (_i, [_vp, _i]),
    "hqmc_set_class_launch": (_i, [_vp, _i, _i]),
    "hqmc_get_class_launch": (_i, [_vp, _i, _vp]),
    "hqmc_autotune": (_i, [_vp, _i, _vp]),
    "hqmc_workspace_size": (_i, [_vp, C.POINTER(_sz)]),
    "hqmc_attach_workspace": (_i, [_vp, _vp, _sz]),
    "hqmc_sweep": (_i, [_vp, _i, _vp]),
    "hqmc_logw_error": (_i, [_vp, _vp]),
    "hqmc_local_sweep": (_i, [_vp, _i]),
    "hqmc_set_permutations": (_i, [_vp, _i]),
    "hqmc_set_conv": (_i, [_vp, _i]),
    "hqmc_get_perm": (_i, [_vp, _i, _vp, _vp]),
    "hqmc_set_perm": (_i, [_vp, _i, _vp]),
    "hqmc_measure": (_i, [_vp, _vp, _vp, _vp, _i]),
    "hqmc_set_measure_open": (_i, [_vp, _i]),
    "hqmc_measure_open": (_i, [_vp, _vp, _vp]),
    "hqmc_set_checkpoint": (_i, [_vp, _i, _i]),
    "hqmc_log_weight_grad": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "hqmc_chain_shape": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hqmc_get_state": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "hqmc_set_state": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hqmc_get_sigma": (_i, [_vp, _i, _vp]),
    "hqmc_set_sigma": (_i, [_vp, _i, _vp]),
    "hqmc_set_profiling": (_i, [_vp, _i]),
    "hqmc_profile_read": (_i, [_vp, _vp, _vp, _vp]),
    "hqmc_ffbs_noalloc": (_i, [_i, _i, _i, _d, _d, _d, _u64, _u64, _vp, _vp, _vp, _i, _vp]),
    "hqmc_supported_L": (_i, [_vp, _i]),
    "hqmc_fp32_peak": (_i, [_i, _i, C.POINTER(_d)]),
    "hqmc_fp64_peak": (_i, [_i, C.POINTER(_d)]),
    "hqmc_destroy": (None, [_vp]),
    "hqmc_strerror": (C.c_char_p, [_i]),
    "hqmc_last_error_detail": (C.c_char_p, [_vp]),
}


class HQMCError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__(f"{ERRORS.get(code, code)}: {detail}")


class Obs(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("density", C.c_double), ("double_occ", C.c_double),
                ("m2", C.c_double), ("ekin", C.c_double), ("s_pipi", C.c_double),
                ("n_degenerate", C.c_int64), ("n_nonpositive", C.c_int64), ("n_local_accepted", C.c_int64),
                ("mean_sign", C.c_double), ("n_perm_accepted", C.c_int64), ("n_inexact", C.c_int64)]


_lib = None


def lib():
    """Load libhqmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2510_13866_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def supported_L():
    n = lib().hqmc_supported_L(None, 0)
    buf = (C.c_int * n)()
    lib().hqmc_supported_L(buf, n)
    return list(buf)


def fp32_peak(device=0, packed=True):
    """Measured FP32 fused multiply-add throughput (TFLOP/s) of `device`: packed f32x2
    (FFMA2, as the line FFTs run) or scalar FFMA."""
    out = C.c_double(0.0)
    rc = lib().hqmc_fp32_peak(int(device), int(bool(packed)), C.byref(out))
    if rc != 0:
        raise HQMCError(rc, "hqmc_fp32_peak")
    return out.value


def fp64_peak(device=0):
    """Measured FP64 fused multiply-add throughput (TFLOP/s) of `device`."""
    out = C.c_double(0.0)
    rc = lib().hqmc_fp64_peak(int(device), C.byref(out))
    if rc != 0:
        raise HQMCError(rc, "hqmc_fp64_peak")
    return out.value


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Lattice:
    """A batch of independent chains (one hqmc context) on one CUDA device."""

    def __init__(self, L, seeds, precision="fp32", device=0, torch_memory=True):
        import torch

        self._torch = torch
        Ls = [int(L)] * len(seeds) if np.isscalar(L) else [int(v) for v in L]
        if len(Ls) != len(seeds):
            raise ValueError("one L per seed")
        self.Ls = np.array(Ls, dtype=np.int32)
        self.seeds = np.array(seeds, dtype=np.uint64)
        self.n_chains = len(Ls)
        self.precision = HQMC_FP64 if precision in ("fp64", HQMC_FP64) else HQMC_FP32
        self.device = device
        self.torch_memory = torch_memory
        self._ws = None
        self._ctx = C.c_void_p()
        self._check(lib().hqmc_init_lattice(C.byref(self._ctx), self.n_chains, _ptr(self.Ls),
                                            _ptr(self.seeds), self.precision, device), ctx=False)
        stream = torch.cuda.current_stream(device)
        self._check(lib().hqmc_set_stream(self._ctx, C.c_void_p(stream.cuda_stream)))
        self.shapes = None
        self.params = None
        # (t, U, beta, dtau, filling) of every chain as last set, so that a change of t
        # alone (log_weight) keeps each chain's own U, beta, dtau and filling
        self.chain_params = [None] * self.n_chains

    # -- helpers -----------------------------------------------------------
    def _check(self, rc, ctx=True):
        if rc != 0:
            detail = lib().hqmc_last_error_detail(self._ctx).decode() if ctx and self._ctx else ""
            raise HQMCError(rc, detail)

    def close(self):
        if self._ctx:
            lib().hqmc_destroy(self._ctx)
            self._ctx = C.c_void_p()
        self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration -----------------------------------------------------
    def set_params(self, t, U, beta, dtau, filling, chain=-1):
        self._check(lib().hqmc_set_params(self._ctx, chain, t, U, beta, dtau, filling))
        p = (float(t), float(U), float(beta), float(dtau), float(filling))
        if chain == -1:
            self.params = p
            self.chain_params = [p] * self.n_chains
        else:
            self.chain_params[int(chain)] = p
            self.params = p if all(q == p for q in self.chain_params) else None
        self.shapes = None

    def set_block(self, B, chain=-1):
        """FFBS block length (0 or >= M: the closed loop from the anchor; 1 <= B < M:
        blocks from the anchor with both end sites held)."""
        self._check(lib().hqmc_set_block(self._ctx, int(chain), int(B)))
        if self.torch_memory and self._ws is not None:
            self._attach()

    def set_ffbs_storage(self, kind="stream", stride=0):
        """Storage of f for the wide kernel's backward pass: "stream" (every slice, FP32),
        "bf16" or "f32" checkpoints every `stride` positions (0: ceil(sqrt M)) with the
        segments recomputed."""
        self._check(lib().hqmc_set_ffbs_storage(self._ctx, {"stream": 0, "bf16": 1, "f32": 2}[kind], int(stride)))
        if self.torch_memory and self._ws is not None:
            self._attach()

    def set_checkpoint(self, stride=0, bf16=True):
        """Checkpoint stride of the adjoint's reverse pass (0 = ceil(sqrt M)) and format
        (BF16 with a per-slice exponent, or the context's own precision)."""
        self._check(lib().hqmc_set_checkpoint(self._ctx, int(stride), HQMC_CKPT_BF16 if bf16 else HQMC_CKPT_FULL))

    def set_launch(self, use_graph=True, persistent=True, warps_per_cta=0):
        self._check(lib().hqmc_set_launch(self._ctx, int(use_graph), int(persistent), int(warps_per_cta)))
        if self.torch_memory and self._ws is not None:
            self._attach()

    def set_slice_launch(self, slices_per_cta):
        self._check(lib().hqmc_set_slice_launch(self._ctx, int(slices_per_cta)))

    def set_class_launch(self, L, warps_per_cta):
        self._check(lib().hqmc_set_class_launch(self._ctx, int(L), int(warps_per_cta)))
        if self.torch_memory and self._ws is not None:
            self._attach()

    def class_launch(self, L):
        w = C.c_int(0)
        self._check(lib().hqmc_get_class_launch(self._ctx, int(L), C.byref(w)))
        return w.value

    def autotune(self, trial_sweeps=3, cache=None):
        """CTA shape per lattice size, timed by the library on throwaway copies of the chains
        (hqmc_autotune).  With `cache` (a JSON path) the choice is keyed by GPU, precision,
        size, slices and pair count, read from the file when present and written back."""
        import json

        key_of = {}
        for L in sorted(set(int(v) for v in self.Ls)):
            if L > 32:
                continue
            shp = [s for s, l in zip(self._shapes(), self.Ls) if l == L]
            Mmax = max(M for _, M, _ in shp)
            pairs = sum(2 * ((ns + 1) // 2) for _, _, ns in shp)
            name = self._torch.cuda.get_device_name(self.device)
            key_of[L] = f"{name}|{'fp64' if self.precision == HQMC_FP64 else 'fp32'}|L={L}|M={Mmax}|pairs={pairs}"
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if all(k in table for k in key_of.values()):
            for L, k in key_of.items():
                self.set_class_launch(L, table[k])
            return {L: table[k] for L, k in key_of.items()}
        n = C.c_int(0)
        self._check(lib().hqmc_autotune(self._ctx, int(trial_sweeps), C.byref(n)))
        if self.torch_memory and self._ws is not None:
            self._attach()
        chosen = {L: self.class_launch(L) for L in key_of}
        if cache:
            table.update({key_of[L]: w for L, w in chosen.items()})
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return chosen

    def workspace_size(self):
        n = C.c_size_t(0)
        self._check(lib().hqmc_workspace_size(self._ctx, C.byref(n)))
        return n.value

    def _attach(self):
        n = self.workspace_size()
        if self._ws is None or self._ws.numel() < n:
            self._ws = self._torch.empty(n + 256, dtype=self._torch.uint8, device=f"cuda:{self.device}")
        p = self._ws.data_ptr()
        p = (p + 255) // 256 * 256
        self._check(lib().hqmc_attach_workspace(self._ctx, C.c_void_p(p), n))

    def prepare(self):
        """Bind device memory (torch-allocated) and initialise the chain state."""
        if self.torch_memory and self._ws is None:
            self._attach()
        self._shapes()

    def _shapes(self):
        if self.shapes is None:
            out = []
            for c in range(self.n_chains):
                L, M, Ns = C.c_int(), C.c_int(), C.c_int()
                self._check(lib().hqmc_chain_shape(self._ctx, c, C.byref(L), C.byref(M), C.byref(Ns)))
                out.append((L.value, M.value, Ns.value))
            self.shapes = out
        return self.shapes

    # -- the path ----------------------------------------------------------
    def sweep(self, n=1, logw=False):
        """Run n sweeps; with logw=True return the last sweep's log-weights, a list of
        [2, Nsig] arrays per chain."""
        self.prepare()
        buf = None
        if logw:
            total = sum(2 * ns for _, _, ns in self.shapes)
            buf = np.zeros(total, dtype=np.float64)
        self._check(lib().hqmc_sweep(self._ctx, int(n), _ptr(buf)))
        if not logw:
            return None
        out, o = [], 0
        for _, _, ns in self.shapes:
            out.append(buf[o:o + 2 * ns].reshape(2, ns))
            o += 2 * ns
        return out

    def logw_error(self):
        """Error estimates of the last sweep's log-weights (hqmc_logw_error), a list of
        [2, Nsig] arrays per chain like sweep(logw=True)."""
        self.prepare()
        total = sum(2 * ns for _, _, ns in self.shapes)
        buf = np.zeros(total, dtype=np.float64)
        self._check(lib().hqmc_logw_error(self._ctx, _ptr(buf)))
        out, o = [], 0
        for _, _, ns in self.shapes:
            out.append(buf[o:o + 2 * ns].reshape(2, ns))
            o += 2 * ns
        return out

    def local_sweep(self, n=1):
        """Run n local-update sweeps (single-slice Metropolis moves of every worldline,
        then the Gibbs step and observables)."""
        self.prepare()
        self._check(lib().hqmc_local_sweep(self._ctx, int(n)))

    def set_conv(self, kind):
        """Line convolutions of the FFBS filter: "fft" (default) or "stencil"."""
        self._check(lib().hqmc_set_conv(self._ctx, {"fft": 0, "stencil": 1}[kind]))

    def set_permutations(self, on=True):
        """Pair-swap permutation updates at tau = beta in every sweep (sign-reweighted
        observables)."""
        self._check(lib().hqmc_set_permutations(self._ctx, int(bool(on))))

    def get_perm(self, chain):
        """(perm [2, Nsig] int32 with perm[sigma, p] = P(p), sign) of one chain."""
        self.prepare()
        _, _, Ns = self.shapes[chain]
        perm = np.zeros((2, Ns), dtype=np.int32)
        sign = C.c_int(0)
        self._check(lib().hqmc_get_perm(self._ctx, chain, _ptr(perm), C.byref(sign)))
        return perm, sign.value

    def set_perm(self, chain, perm):
        self.prepare()
        _, _, Ns = self.shapes[chain]
        pa = np.ascontiguousarray(perm, dtype=np.int32).reshape(2, Ns)
        self._check(lib().hqmc_set_perm(self._ctx, chain, _ptr(pa)))

    def measure(self, reset=False):
        self.prepare()
        obs = (Obs * self.n_chains)()
        totN = sum(L * L for L, _, _ in self.shapes)
        sk = np.zeros(totN)
        cr = np.zeros(totN)
        self._check(lib().hqmc_measure(self._ctx, obs, _ptr(sk), _ptr(cr), int(bool(reset))))
        res, o = [], 0
        for c, (L, _, _) in enumerate(self.shapes):
            N = L * L
            ob = obs[c]
            res.append(dict(n_samples=ob.n_samples, density=ob.density, double_occ=ob.double_occ, m2=ob.m2,
                            ekin=ob.ekin, s_pipi=ob.s_pipi, n_degenerate=ob.n_degenerate,
                            n_nonpositive=ob.n_nonpositive, n_local_accepted=ob.n_local_accepted,
                            mean_sign=ob.mean_sign, n_perm_accepted=ob.n_perm_accepted, n_inexact=ob.n_inexact,
                            Sk=sk[o:o + N].copy(), Cr=cr[o:o + N].copy()))
            o += N
        return res

    def set_measure_open(self, on=True):
        """Accumulate the open-path estimator of the one-body density matrix (for n_k) in
        every later sweep; restarts the observable accumulators."""
        self._check(lib().hqmc_set_measure_open(self._ctx, int(bool(on))))

    def measure_open(self):
        """Per chain (n_k [N], one-body density matrix per site [N]) from the open-path sums
        since the last reset (hqmc_measure_open)."""
        self.prepare()
        totN = sum(L * L for L, _, _ in self.shapes)
        nk = np.zeros(totN)
        dm = np.zeros(totN)
        self._check(lib().hqmc_measure_open(self._ctx, _ptr(nk), _ptr(dm)))
        out, o = [], 0
        for L, _, _ in self.shapes:
            out.append((nk[o:o + L * L].copy(), dm[o:o + L * L].copy()))
            o += L * L
        return out

    def get_state(self, chain):
        self.prepare()
        L, M, Ns = self.shapes[chain]
        s = np.zeros((M, L * L), dtype=np.int8)
        x = np.zeros((2, Ns, M), dtype=np.int32)
        a = C.c_int(0)
        sw = C.c_uint64(0)
        self._check(lib().hqmc_get_state(self._ctx, chain, _ptr(s), _ptr(x), C.byref(a), C.byref(sw)))
        return s, x, a.value, sw.value

    def set_state(self, chain, s=None, x=None, sweeps=None):
        self.prepare()
        L, M, Ns = self.shapes[chain]
        sa = None if s is None else np.ascontiguousarray(s, dtype=np.int8).reshape(M, L * L)
        xa = None if x is None else np.ascontiguousarray(x, dtype=np.int32).reshape(2, Ns, M)
        sw = None if sweeps is None else C.byref(C.c_uint64(int(sweeps)))
        self._check(lib().hqmc_set_state(self._ctx, chain, _ptr(sa), _ptr(xa), sw))

    def get_sigma(self, chain):
        """Gaussian field [M][N] of a U < 0 chain."""
        self.prepare()
        L, M, _ = self.shapes[chain]
        sig = np.zeros((M, L * L))
        self._check(lib().hqmc_get_sigma(self._ctx, chain, _ptr(sig)))
        return sig

    def set_sigma(self, chain, sigma):
        self.prepare()
        L, M, _ = self.shapes[chain]
        sig = np.ascontiguousarray(sigma, dtype=np.float64).reshape(M, L * L)
        self._check(lib().hqmc_set_sigma(self._ctx, chain, _ptr(sig)))

    def set_profiling(self, max_sweeps):
        self._check(lib().hqmc_set_profiling(self._ctx, int(max_sweeps)))

    def profile_read(self):
        """(FFBS ms summed, Gibbs/measure ms summed, sweeps recorded)."""
        f, s, n = C.c_double(), C.c_double(), C.c_int()
        self._check(lib().hqmc_profile_read(self._ctx, C.byref(f), C.byref(s), C.byref(n)))
        return f.value, s.value, n.value

    def log_weight_grad(self, v=None, want_dv=True):
        """(logZ [chains], dlogZ/dv packed [sum 2 M N] torch tensor, dlogZ/dt [chains])."""
        torch = self._torch
        self.prepare()
        dt = torch.float64 if self.precision == HQMC_FP64 else torch.float32
        tot = sum(2 * M * L * L for L, M, _ in self.shapes)
        dv = torch.zeros(tot, dtype=dt, device=f"cuda:{self.device}") if want_dv else None
        vp = None
        if v is not None:
            if v.dtype != dt or not v.is_cuda or v.numel() != tot:
                raise ValueError("v must be a contiguous CUDA tensor of the context's dtype, packed [2][M][N] per chain")
            v = v.contiguous()
            vp = C.c_void_p(v.data_ptr())
        lz = np.zeros(self.n_chains)
        ddt = np.zeros(self.n_chains)
        self._check(lib().hqmc_log_weight_grad(self._ctx, vp, _ptr(lz),
                                               None if dv is None else C.c_void_p(dv.data_ptr()), _ptr(ddt)))
        return lz, dv, ddt


def _log_weight_function():
    import torch

    class LogWeight(torch.autograd.Function):
        """log Z of every chain (worldlines anchored at slice 0 on their current sites) as a
        function of the log-potential v (packed [2][M][N] per chain) and the hopping t.

        The forward and the adjoint both run in libhqmc.so (one hqmc_log_weight_grad
        call); backward only scales the saved per-chain gradients by the incoming ones."""

        @staticmethod
        def forward(ctx, lat, v, t):
            tv = float(t)
            if any(p is None for p in lat.chain_params):
                raise ValueError("set_params first (for every chain)")
            # only t changes: every chain keeps its own U, beta, dtau and filling
            for c, p in enumerate(list(lat.chain_params)):
                if p[0] != tv:
                    lat.set_params(tv, *p[1:], chain=c)
            lz, dv, dt = lat.log_weight_grad(v=v.detach(), want_dv=True)
            sizes = [2 * M * L * L for L, M, _ in lat.shapes]
            ctx.save_for_backward(dv)
            ctx.sizes = sizes
            ctx.dt = torch.as_tensor(dt, dtype=torch.float64)
            ctx.t_shape = t.shape if torch.is_tensor(t) else None
            return torch.as_tensor(lz, dtype=torch.float64, device=v.device)

        @staticmethod
        def backward(ctx, g):
            (dv,) = ctx.saved_tensors
            rep = torch.repeat_interleave(g.to(dv.dtype), torch.as_tensor(ctx.sizes, device=g.device))
            gv = dv * rep
            gt = None
            if ctx.t_shape is not None:
                gt = (g.detach().cpu() * ctx.dt).sum().to(torch.float64).reshape(ctx.t_shape)
            return None, gv, gt

    return LogWeight


_LW = None


def log_weight(lat, v, t):
    """Differentiable log Z per chain: torch.autograd sees v (device tensor of the context's
    dtype, packed [2][M][N] per chain) and t (a 0-d CPU tensor)."""
    global _LW
    if _LW is None:
        _LW = _log_weight_function()
    return _LW.apply(lat, v, t)
