"""FP64 CPU oracle for the worldline FFBS + Hirsch-Gibbs sweep (arXiv 2510.13866).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports this package.

numpy wrappers over oracle/hqmc_oracle.c (ctypes).  Layouts:
  s      [M][N] int8 (+1/-1), site x = ix + L*iy
  xpath  [2][Nsig][M] int32
  hist   [2][M][N] int32
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i, u64, vp = C.c_double, C.c_int, C.c_uint64, C.c_void_p
        L.orc_philox4x64_10.argtypes = [vp, vp, vp]
        L.orc_uniform.argtypes = [u64, u64, u64, u64, u64]
        L.orc_uniform.restype = d
        L.orc_lambda.argtypes = [d, d]
        L.orc_lambda.restype = d
        L.orc_g_table.argtypes = [i, d, d, vp, vp]
        L.orc_initial_site.argtypes = [i, i, i]
        L.orc_initial_site.restype = i
        L.orc_init_state.argtypes = [i, i, i, u64, vp, vp]
        L.orc_filter.argtypes = [i, i, vp, vp, i, i, vp]
        L.orc_filter.restype = d
        L.orc_backward.argtypes = [i, i, vp, vp, i, u64, u64, u64, vp, vp]
        L.orc_filter_block.argtypes = [i, i, vp, vp, i, i, i, i, vp]
        L.orc_filter_block.restype = d
        L.orc_open_ratio.argtypes = [i, i, vp, vp, i, i, i, i, vp]
        L.orc_open_ratio.restype = d
        L.orc_backward_block.argtypes = [i, i, vp, vp, i, i, u64, u64, u64, vp, vp]
        L.orc_sweep.argtypes = [i, i, i, d, d, d, u64, u64, vp, vp, vp, vp, vp, vp, vp, i, i]
        L.orc_sweep.restype = i
        L.orc_marginals.argtypes = [i, i, vp, vp, vp, i, vp, vp]
        L.orc_marginals.restype = d
        L.orc_chain_grad.argtypes = [i, i, i, d, d, d, vp, vp, vp, vp, vp]
        L.orc_chain_grad.restype = d
        L.orc_measure.argtypes = [i, i, vp, vp, vp, vp]
        L.orc_normal.argtypes = [d, d]
        L.orc_normal.restype = d
        L.orc_gauss_coupling.argtypes = [d, d]
        L.orc_gauss_coupling.restype = d
        L.orc_init_sigma.argtypes = [i, i, u64, vp]
        L.orc_sweep_gauss.argtypes = [i, i, i, d, d, d, u64, u64, vp, vp, vp, vp, vp, vp, vp, i, i]
        L.orc_sweep_gauss.restype = i
        L.orc_num_threads.restype = i
        L.orc_local_step.argtypes = [i, i, i]
        L.orc_local_step.restype = i
        L.orc_local_ratio.argtypes = [i, i, vp, vp, i, i, i, i]
        L.orc_local_ratio.restype = d
        L.orc_local_color.argtypes = [i, i]
        L.orc_local_color.restype = i
        L.orc_sweep_local.argtypes = [i, i, i, d, d, d, u64, u64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_sweep_local.restype = i
        L.orc_perm_ratio.argtypes = [i, vp, i, i, i, i]
        L.orc_perm_ratio.restype = d
        L.orc_sweep_perm.argtypes = [i, i, i, d, d, d, u64, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i, vp]
        L.orc_sweep_perm.restype = i
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def uniform(seed, sweep, phase, i, j):
    return lib().orc_uniform(seed, sweep, phase, i, j)


def lam(U, dtau):
    return lib().orc_lambda(U, dtau)


def g_table(L, t, dtau):
    g = np.zeros(L)
    dg = np.zeros(L)
    lib().orc_g_table(L, t, dtau, _p(g), _p(dg))
    return g, dg


def n_slices(beta, dtau):
    M = int(round(beta / dtau))
    if M < 1 or abs(M * dtau - beta) > 1e-9 * max(1.0, beta):
        raise ValueError("beta/dtau must be an integer")
    return M


def n_sigma(L, filling):
    v = filling * L * L / 2
    n = int(round(v))
    if abs(v - n) > 1e-9 or n < 1:
        raise ValueError("filling*N/2 must be a positive integer")
    return n


def initial_site(L, sigma, p):
    return lib().orc_initial_site(L, sigma, p)


def normal(u1, u2):
    return lib().orc_normal(u1, u2)


def gauss_coupling(U, dtau):
    return lib().orc_gauss_coupling(U, dtau)


class Chain:
    """One Markov chain's state in the oracle.  U >= 0: Hirsch field s (int8 +-1);
    U < 0: continuous Gaussian field sigma (float64)."""

    def __init__(self, L, t, U, beta, dtau, filling, seed):
        self.L, self.t, self.U, self.beta, self.dtau = L, t, U, beta, dtau
        self.N = L * L
        self.M = n_slices(beta, dtau)
        self.Nsig = n_sigma(L, filling)
        self.seed = seed
        self.sweep_count = 0
        self.gauss = U < 0
        self.s = np.zeros((self.M, self.N), dtype=np.int8)
        self.x = np.zeros((2, self.Nsig, self.M), dtype=np.int32)
        lib().orc_init_state(L, self.M, self.Nsig, seed, _p(self.s), _p(self.x))
        # permutation at tau = beta (identity: every worldline closes on itself) and its sign
        self.perm = np.tile(np.arange(self.Nsig, dtype=np.int32), (2, 1))
        self.sign = 1
        self.sigma = None
        if self.gauss:
            self.sigma = np.zeros((self.M, self.N))
            lib().orc_init_sigma(L, self.M, seed, _p(self.sigma))

    @property
    def lam(self):
        return lam(self.U, self.dtau)

    def sweep(self, want_margin=False, nwl_limit=-1, block=0):
        """One sweep; returns a dict with logw, hist, anchor, links (and margin)."""
        M, N, Ns = self.M, self.N, self.Nsig
        logw = np.full((2, Ns), np.nan)
        hist = np.zeros((2, M, N), dtype=np.int32)
        margin = np.full((2, Ns, M), np.nan) if want_margin else None
        links = np.full((2, Ns), np.nan)
        anchor = C.c_int(-1)
        if self.gauss:
            lib().orc_sweep_gauss(self.L, M, Ns, self.t, self.U, self.dtau, self.seed, self.sweep_count,
                                  _p(self.sigma), _p(self.x), _p(logw), _p(hist), _p(margin), _p(links),
                                  C.byref(anchor), nwl_limit, block)
        else:
            lib().orc_sweep(self.L, M, Ns, self.t, self.U, self.dtau, self.seed, self.sweep_count,
                            _p(self.s), _p(self.x), _p(logw), _p(hist), _p(margin), _p(links),
                            C.byref(anchor), nwl_limit, block)
        self.sweep_count += 1
        out = dict(logw=logw, hist=hist, anchor=anchor.value, links=links)
        if want_margin:
            out["margin"] = margin
        return out

    def local_sweep(self, want_margin=False):
        """One local-update sweep (Eq. Rlocal in the position basis, then Gibbs); returns
        a dict with hist, links, accepted (and margin)."""
        M, N, Ns = self.M, self.N, self.Nsig
        hist = np.zeros((2, M, N), dtype=np.int32)
        margin = np.full((2, Ns, M), np.nan) if want_margin else None
        links = np.full((2, Ns), np.nan)
        acc = C.c_longlong(0)
        lib().orc_sweep_local(self.L, M, Ns, self.t, self.U, self.dtau, self.seed, self.sweep_count,
                              _p(self.s), _p(self.sigma), _p(self.x), _p(hist), _p(margin), _p(links),
                              C.byref(acc), _p(self.perm))
        self.sweep_count += 1
        out = dict(hist=hist, links=links, accepted=acc.value)
        if want_margin:
            out["margin"] = margin
        return out

    def perm_sweep(self, want_margin=False, block=0):
        """One sweep with permutations: pair-swap update at tau = beta, FFBS of every
        worldline's unit under the new permutation, Gibbs.  Returns a dict with logw (per
        unit), hist, anchor, links, swaps, sign (and margin, margin_perm)."""
        M, N, Ns = self.M, self.N, self.Nsig
        logw = np.full((2, Ns), np.nan)
        hist = np.zeros((2, M, N), dtype=np.int32)
        margin = np.full((2, Ns, M), np.nan) if want_margin else None
        mperm = np.full((2, max(1, Ns // 2)), np.nan) if want_margin else None
        links = np.full((2, Ns), np.nan)
        anchor = C.c_int(-1)
        sign = C.c_int(self.sign)
        swaps = C.c_longlong(0)
        lib().orc_sweep_perm(self.L, M, Ns, self.t, self.U, self.dtau, self.seed, self.sweep_count,
                             _p(self.s), _p(self.sigma), _p(self.x), _p(self.perm), C.byref(sign), _p(logw),
                             _p(hist), _p(margin), _p(mperm), _p(links), C.byref(anchor), block, C.byref(swaps))
        self.sign = sign.value
        self.sweep_count += 1
        out = dict(logw=logw, hist=hist, anchor=anchor.value, links=links, swaps=swaps.value, sign=self.sign)
        if want_margin:
            out["margin"] = margin
            out["margin_perm"] = mperm
        return out

    def slice_potentials(self):
        """W [2][M][N] of the current fields: Hirsch exp(+-lambda s) by spin, or Gaussian
        exp(a sigma) for both spins."""
        if self.gauss:
            w = np.exp(gauss_coupling(self.U, self.dtau) * self.sigma)
            return np.stack([w, w])
        lm = lam(self.U, self.dtau)
        return np.stack([np.exp(lm * self.s), np.exp(-lm * self.s)])

    def open_estimate(self, W, a, block=0):
        """Sum over every worldline of its unit's last-block open-path ratios (orc_open_ratio),
        [N] indexed by the displacement r = rx + L ry of the end: the per-sweep sample of
        sum_x sum_sigma <c^dag_{x+r} c_x> (Sec. 4, "Observables", n_k), for the fields W the
        sweep filters with, its anchor a, the current permutation and the held sites."""
        L, M, N = self.L, self.M, self.N
        g, _ = g_table(L, self.t, self.dtau)
        B = block if 0 < block < M else M
        nblk = (M + B - 1) // B
        acc = np.zeros(N)
        for sg in range(2):
            for p in range(self.Nsig):
                q = self.perm[sg, p]
                vp = np.where(np.arange(M) < a, self.x[sg, q], self.x[sg, p])
                vp[a] = self.x[sg, q, a]
                l0 = (a + (nblk - 1) * B) % M
                ln = M - (nblk - 1) * B
                xs = self.x[sg, p, a] if nblk == 1 else vp[l0]
                acc += open_ratio(L, M, g, W[sg], l0, ln, int(xs), int(vp[(l0 + ln) % M]))
        return acc

    def grad(self, v=None):
        """(logZ, dlogZ/dv [2][M][N], dlogZ/dt) with every worldline anchored at slice 0."""
        dv = np.zeros((2, self.M, self.N))
        dt = C.c_double(0.0)
        vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        lz = lib().orc_chain_grad(self.L, self.M, self.Nsig, self.t, self.U, self.dtau,
                                  _p(self.s), _p(vv), _p(self.x), _p(dv), C.byref(dt))
        return lz, dv, dt.value


def filter_logz(L, M, g, W, a, xa, want_f=False):
    W = np.ascontiguousarray(W, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    f = np.zeros((M, L * L)) if want_f else None
    lz = lib().orc_filter(L, M, _p(g), _p(W), a, xa, _p(f))
    return (lz, f) if want_f else lz


def filter_block(L, M, g, W, l0, B, xs, xe, want_f=False):
    W = np.ascontiguousarray(W, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    f = np.zeros((M, L * L)) if want_f else None
    lz = lib().orc_filter_block(L, M, _p(g), _p(W), l0, B, xs, xe, _p(f))
    return (lz, f) if want_f else lz


def open_ratio(L, M, g, W, l0, B, xs, xe):
    """alpha_end(xe + r) / alpha_end(xe) [N] (r = rx + L ry) of the block's filter from xs."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(L * L)
    lib().orc_open_ratio(L, M, _p(g), _p(W), l0, B, xs, xe, _p(out))
    return out


def backward_block(L, M, g, f, l0, B, seed, sweep, wl, xpath):
    xp = np.ascontiguousarray(xpath, dtype=np.int32).copy()
    margin = np.zeros(M)
    lib().orc_backward_block(L, M, _p(np.ascontiguousarray(g, dtype=np.float64)),
                             _p(np.ascontiguousarray(f, dtype=np.float64)), l0, B, seed, sweep, wl,
                             _p(xp), _p(margin))
    return xp, margin


def backward(L, M, g, f, a, seed, sweep, wl, xpath):
    xp = np.ascontiguousarray(xpath, dtype=np.int32).copy()
    margin = np.zeros(M)
    lib().orc_backward(L, M, _p(np.ascontiguousarray(g, dtype=np.float64)),
                       _p(np.ascontiguousarray(f, dtype=np.float64)), a, seed, sweep, wl,
                       _p(xp), _p(margin))
    return xp, margin


def perm_ratio(L, g, xlp, xlq, a0, b0):
    return lib().orc_perm_ratio(L, _p(np.ascontiguousarray(g, dtype=np.float64)), xlp, xlq, a0, b0)


def local_step(L, x, direction):
    return lib().orc_local_step(L, x, direction)


def local_ratio(L, M, g, Wl, xm, x, xn, xnew):
    return lib().orc_local_ratio(L, M, _p(np.ascontiguousarray(g, dtype=np.float64)),
                                 _p(np.ascontiguousarray(Wl, dtype=np.float64)), xm, x, xn, xnew)


def local_color(M, l):
    return lib().orc_local_color(M, l)


def marginals(L, M, g, dg, v, x0):
    v = np.ascontiguousarray(v, dtype=np.float64)
    marg = np.zeros((M, L * L))
    dt = C.c_double(0.0)
    lz = lib().orc_marginals(L, M, _p(np.ascontiguousarray(g)), _p(np.ascontiguousarray(dg)),
                             _p(v), x0, _p(marg), C.byref(dt))
    return lz, marg, dt.value


def measure(L, M, hist, want_fields=True):
    hist = np.ascontiguousarray(hist, dtype=np.int32)
    out = np.zeros(3)
    Sk = np.zeros(L * L) if want_fields else None
    Cr = np.zeros(L * L) if want_fields else None
    lib().orc_measure(L, M, _p(hist), _p(out), _p(Sk), _p(Cr))
    return dict(n=out[0], d=out[1], m2=out[2], Sk=Sk, Cr=Cr)


def num_threads():
    return lib().orc_num_threads()
