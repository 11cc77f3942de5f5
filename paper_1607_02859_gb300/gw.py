"""Thin ctypes binding of libgw.so (include/gw.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device arrays are torch tensors (complex64 for the FP32 and
tensor-core precisions, complex128 for FP64); host arrays are numpy.  The
stream is torch's current CUDA stream.  There is no CPU fallback: if libgw.so
is missing, loading raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgw.so")

FP64, FP32, F16X3, BF16X3 = 0, 1, 2, 3
PREC = {"fp64": FP64, "fp32": FP32, "f16x3": F16X3, "bf16x3": BF16X3}
CT, ST, IST = 0, 1, 2
STATUS = {0: "GW_OK", 1: "GW_ERR_ARG", 2: "GW_ERR_SHAPE", 3: "GW_ERR_OOM", 4: "GW_ERR_CUDA",
          5: "GW_ERR_NUMERIC", 6: "GW_ERR_TIMEOUT", 7: "GW_ERR_UNSUPPORTED"}

# every symbol declared in include/gw.h
EXPORTS = ["gw_ctx_create", "gw_ctx_destroy", "gw_last_error", "gw_ctx_launches", "gw_ctx_scratch_bytes", "gw_ctx_reserve",
           "gw_ctx_set_timing", "gw_ctx_kernel_stats", "gw_version", "gw_g_set", "gw_coulomb_sqrt", "gw_fit_transform", "gw_green_tau", "gw_chi0_rtau",
           "gw_chi0_rtau_fused", "gw_rr_to_GG_fft", "gw_tau_to_omega", "gw_screen_W", "gw_sigma_diag",
           "gw_chi0_omega", "gw_rr_to_GG_fft_noalloc", "gw_workspace_size", "gw_screen_W_refine", "gw_chi0_omega_kmesh", "gw_sigma_diag_kmesh",
           "gw_chi0_plan_create", "gw_chi0_plan_launch", "gw_chi0_plan_status", "gw_chi0_plan_destroy",
           "gw_sigma_matrix", "gw_qp_energies", "gw_invert_transform", "gw_sigma_to_tau", "gw_mp2_grids",
           "gw_zgemm_sliced", "gw_batch_plan", "gw_batch_launch", "gw_batch_wait", "gw_batch_destroy",
           "gw_chi0_omega_pw", "gw_sigma_diag_pw", "gw_chi0_omega_kmesh_pw"]


class GwError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.message = message


class Grid(ct.Structure):
    _fields_ = [("n", ct.c_int * 3), ("lattice", ct.c_double * 9)]


class BatchSystem(ct.Structure):
    _fields_ = [("grid", Grid), ("n_b", ct.c_int), ("n_occ", ct.c_int), ("eps_h", ct.POINTER(ct.c_double)),
                ("mu", ct.c_double), ("n", ct.c_int), ("tau_h", ct.POINTER(ct.c_double)),
                ("omega_h", ct.POINTER(ct.c_double)), ("C_h", ct.POINTER(ct.c_double)),
                ("S_h", ct.POINTER(ct.c_double)), ("Cinv_h", ct.POINTER(ct.c_double)), ("n_chi", ct.c_int),
                ("gvec_h", ct.POINTER(ct.c_int32)), ("fft_index_h", ct.POINTER(ct.c_int32)), ("n_n", ct.c_int),
                ("bands_h", ct.POINTER(ct.c_int32)), ("r_block", ct.c_int), ("refine_iters", ct.c_int),
                ("psi", ct.c_void_p), ("chi_w", ct.c_void_p), ("w_tau", ct.c_void_p)]


_P = ct.c_void_p
_I = ct.c_int
_D = ct.c_double
_DP = ct.POINTER(ct.c_double)
_IP = ct.POINTER(ct.c_int32)
_G = ct.POINTER(Grid)

_SIGS = {
    "gw_ctx_create": (_I, [_I, ct.POINTER(_P)]),
    "gw_ctx_destroy": (_I, [_P]),
    "gw_last_error": (ct.c_char_p, [_P]),
    "gw_ctx_launches": (ct.c_ulonglong, [_P]),
    "gw_ctx_scratch_bytes": (ct.c_size_t, [_P]),
    "gw_ctx_reserve": (ct.c_int, [_P, ct.c_size_t]),
    "gw_version": (_I, []),
    "gw_ctx_set_timing": (_I, [_P, _I]),
    "gw_ctx_kernel_stats": (_I, [_P, ct.c_char_p, ct.POINTER(ct.c_ulonglong), _DP, _DP, ct.POINTER(ct.c_int)]),
    "gw_g_set": (_I, [_G, _I, _IP, _IP]),
    "gw_coulomb_sqrt": (_I, [_G, _IP, _I, _DP]),
    "gw_fit_transform": (_I, [_I, _DP, _DP, _D, _D, _I, _D, _DP, _DP, _DP, _DP]),
    "gw_green_tau": (_I, [_P, _G, _I, _I, _P, _DP, _D, _D, _I, _I, _I, _P, _P, _P]),
    "gw_chi0_rtau": (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    "gw_chi0_rtau_fused": (_I, [_P, _G, _I, _I, _P, _DP, _D, _D, _I, _I, _I, _P, _P]),
    "gw_rr_to_GG_fft": (_I, [_P, _G, _I, _I, _I, _IP, _I, _I, _I, _P, _P, _P]),
    "gw_rr_to_GG_fft_noalloc": (_I, [_G, _I, _I, _I, _IP, _I, _I, _I, _P, _P, _P]),
    "gw_workspace_size": (_I, [_G, _I, _I, _I, _I, _I, _I, _I, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t),
                               ct.POINTER(ct.c_size_t)]),
    "gw_tau_to_omega": (_I, [_P, _I, _I, _DP, ct.c_size_t, _I, _P, _P, _P]),
    "gw_screen_W": (_I, [_P, _G, _I, _IP, _I, _I, _P, _P, _DP, _P]),
    "gw_screen_W_refine": (_I, [_P, _G, _I, _IP, _I, _I, _I, _P, _P, _DP, _P]),
    "gw_chi0_plan_create": (_I, [_P, _G, _I, _I, _DP, ct.c_double, _I, _DP, _DP, _I, _IP, _I, _I, ct.POINTER(_P)]),
    "gw_chi0_plan_launch": (_I, [_P, _P, _P, _P]),
    "gw_chi0_plan_status": (_I, [_P, _P]),
    "gw_chi0_plan_destroy": (_I, [_P]),
    "gw_sigma_diag_kmesh": (_I, [_P, _G, _IP, _I, _I, _P, _DP, ct.c_double, _IP, _I, _I, _DP, _DP, _DP, _DP, _P, _I,
                                 _IP, _I, _DP, _P, _DP, _I, _P, _P]),
    "gw_chi0_omega_kmesh": (_I, [_P, _G, _IP, _I, _I, _P, _DP, ct.c_double, _I, _DP, _DP, _I, _IP, _I, _I, _P, _P]),
    "gw_chi0_omega_kmesh_pw": (_I, [_P, _G, _IP, _I, _I, _P, _DP, ct.c_double, _I, _DP, _DP, _I, _IP, _I, _IP, _I,
                                    _P, _P]),
    "gw_sigma_diag": (_I, [_P, _G, _I, _I, _P, _DP, _D, _IP, _I, _I, _DP, _DP, _DP, _DP, _P, _I, _IP, _I,
                           _DP, _DP, _DP, _I, _DP, _P]),
    "gw_chi0_omega": (_I, [_P, _G, _I, _I, _P, _DP, _D, _I, _DP, _DP, _I, _IP, _I, _I, _P, _P]),
    "gw_chi0_omega_pw": (_I, [_P, _G, _I, _I, _P, _DP, _D, _I, _DP, _DP, _I, _IP, _I, _IP, _I, _P, _P]),
    "gw_sigma_diag_pw": (_I, [_P, _G, _I, _I, _P, _DP, _D, _IP, _I, _I, _DP, _DP, _DP, _DP, _P, _I, _IP, _I, _IP,
                              _I, _DP, _DP, _DP, _I, _DP, _P]),
    "gw_sigma_matrix": (_I, [_P, _G, _I, _I, _P, _DP, _D, _IP, _I, _I, _DP, _DP, _DP, _DP, _P, _I, _IP, _I,
                             _DP, _DP, _P]),
    "gw_qp_energies": (_I, [_P, _I, _I, _DP, _DP, _DP, _D, _DP, _I, _DP, _DP, _DP, _DP, _DP, _DP, _P]),
    "gw_invert_transform": (_I, [_I, _DP, _DP]),
    "gw_mp2_grids": (_I, [_I, _D, _D, _DP, _DP, _DP, _DP, _DP]),
    "gw_zgemm_sliced": (_I, [_P, _I, _I, _I, _P, ct.c_long, _P, ct.c_long, _P, ct.c_long, _I, _P]),
    "gw_batch_plan": (_I, [_P, _I, ct.POINTER(BatchSystem), _I, ct.POINTER(_P)]),
    "gw_batch_launch": (_I, [_P, _P]),
    "gw_batch_wait": (_I, [_P, _I, _DP, ct.POINTER(ct.c_int)]),
    "gw_batch_destroy": (_I, [_P]),
    "gw_sigma_to_tau": (_I, [_P, _I, _I, _I, _DP, _DP, _DP, _DP, _P]),
}

_lib = None


def lib():
    """Load libgw.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgw.so not built: run paper_1607_02859_gb300/build.py (or __graft_entry__.build())")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_IP)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _check(st, ctx=None):
    if st != 0:
        msg = lib().gw_last_error(ctx.handle if ctx is not None else None)
        raise GwError(st, msg.decode() if msg else "")


def make_grid(n, lattice) -> Grid:
    g = Grid()
    for d in range(3):
        g.n[d] = int(n[d])
    lat = np.asarray(lattice, dtype=np.float64).reshape(9)
    for i in range(9):
        g.lattice[i] = float(lat[i])
    return g


def prec_of(p):
    return PREC[p] if isinstance(p, str) else int(p)


def cdtype(prec):
    import torch
    return torch.complex128 if prec_of(prec) == FP64 else torch.complex64


class Context:
    """A libgw context bound to one CUDA device."""

    def __init__(self, device=0):
        h = _P()
        _check(lib().gw_ctx_create(int(device), ct.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().gw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(lib().gw_ctx_launches(self.handle))

    @property
    def scratch_bytes(self) -> int:
        return int(lib().gw_ctx_scratch_bytes(self.handle))

    def reserve(self, nbytes: int):
        """Grow the scratch arena to at least nbytes now (synchronises the device when it grows)."""
        _check(lib().gw_ctx_reserve(self.handle, int(nbytes)), self)

    FAMILIES = ("green_tc", "cgemm_tc", "cgemm_simt", "row_fft", "col_fft", "col_line_ct", "sigma_contract", "ct",
                "cgemm_exact", "row_pw")

    def set_timing(self, enabled: bool):
        _check(lib().gw_ctx_set_timing(self.handle, 1 if enabled else 0), self)

    def kernel_stats(self):
        """{family: (launches, ms, work, work_is_bytes)} since timing was enabled."""
        out = {}
        for fam in self.FAMILIES:
            n = ct.c_ulonglong(0)
            ms = ct.c_double(0)
            w = ct.c_double(0)
            b = ct.c_int(0)
            _check(lib().gw_ctx_kernel_stats(self.handle, fam.encode(), ct.byref(n), ct.byref(ms), ct.byref(w),
                                             ct.byref(b)), self)
            out[fam] = (int(n.value), float(ms.value), float(w.value), bool(b.value))
        return out


# ------------------------------------------------------------------ host setup

def g_set(grid: Grid, n_chi: int):
    gv = np.zeros((n_chi, 3), dtype=np.int32)
    idx = np.zeros(n_chi, dtype=np.int32)
    _check(lib().gw_g_set(ct.byref(grid), int(n_chi), _ip(gv), _ip(idx)))
    return gv, idx


def coulomb_sqrt(grid: Grid, gvec):
    gv = _i32(gvec)
    out = np.zeros(len(gv), dtype=np.float64)
    _check(lib().gw_coulomb_sqrt(ct.byref(grid), _ip(gv), len(gv), _dp(out)))
    return out


def fit_transform(tau, omega, x_min, x_max, n_x=4000, ridge=1e-6):
    tau = _f64(tau)
    omega = _f64(omega)
    n = len(tau)
    C = np.zeros((n, n))
    S = np.zeros((n, n))
    Ci = np.zeros((n, n))
    err = np.zeros(2)
    _check(lib().gw_fit_transform(n, _dp(tau), _dp(omega), float(x_min), float(x_max), int(n_x), float(ridge),
                                  _dp(C), _dp(S), _dp(Ci), _dp(err)))
    return {"C": C, "S": S, "Cinv": Ci, "Sinv": invert_transform(S), "fit_err_cos": err[0], "fit_err_sin": err[1]}


def mp2_grids(n, x_min, x_max):
    """Optimised imaginary-time and frequency grids (gw_mp2_grids)."""
    tau = np.zeros(int(n))
    om = np.zeros(int(n))
    al = np.zeros(int(n))
    sg = np.zeros(int(n))
    err = np.zeros(2)
    _check(lib().gw_mp2_grids(int(n), float(x_min), float(x_max), _dp(tau), _dp(om), _dp(al), _dp(sg), _dp(err)))
    return {"tau": tau, "omega": om, "alpha": al, "sigma": sg, "err_time": float(err[0]),
            "err_frequency": float(err[1])}


def invert_transform(M):
    """Inverse of a transform matrix (Eqs. INV_CT_FFT, INV_ST_FFT), FP64 on the host."""
    M = _f64(M)
    n = M.shape[0]
    out = np.zeros((n, n))
    _check(lib().gw_invert_transform(n, _dp(M), _dp(out)))
    return out


def workspace_size(grid, n_b, n_occ, n, n_chi, n_n, prec, r_block=0):
    """(chi0_omega, screen_W, sigma_diag) scratch bytes of the context arena."""
    a, s, g = ct.c_size_t(0), ct.c_size_t(0), ct.c_size_t(0)
    _check(lib().gw_workspace_size(ct.byref(grid), int(n_b), int(n_occ), int(n), int(n_chi), int(n_n), prec_of(prec),
                                   int(r_block), ct.byref(a), ct.byref(s), ct.byref(g)))
    return int(a.value), int(s.value), int(g.value)


# ------------------------------------------------------------------ device calls

def _stream():
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, name, prec=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if prec is not None and t.dtype != cdtype(prec):
        raise ValueError("%s must be %s for this precision" % (name, cdtype(prec)))
    return ct.c_void_p(t.data_ptr())


def green_tau(ctx, grid, psi, eps, n_occ, mu, tau, r0, n_rows, prec, g_occ=None, g_unocc=None):
    p = prec_of(prec)
    eps = _f64(eps)
    _check(lib().gw_green_tau(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p), _dp(eps),
                              float(mu), float(tau), int(r0), int(n_rows), p, _dev(g_occ, "g_occ", p),
                              _dev(g_unocc, "g_unocc", p), _stream()), ctx)


def chi0_rtau(ctx, g_occ, g_unocc, chi, prec):
    p = prec_of(prec)
    n_rows, n_cols = g_occ.shape
    _check(lib().gw_chi0_rtau(ctx.handle, n_rows, n_cols, p, _dev(g_occ, "g_occ", p), _dev(g_unocc, "g_unocc", p),
                              _dev(chi, "chi", p), _stream()), ctx)


def chi0_rtau_fused(ctx, grid, psi, eps, n_occ, mu, tau, r0, n_rows, prec, chi):
    p = prec_of(prec)
    eps = _f64(eps)
    _check(lib().gw_chi0_rtau_fused(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p),
                                    _dp(eps), float(mu), float(tau), int(r0), int(n_rows), p, _dev(chi, "chi", p),
                                    _stream()), ctx)


def rr_to_GG_fft(ctx, grid, direction, stage, fft_index, prec, r0, n_rows, inp, out):
    p = prec_of(prec)
    idx = _i32(fft_index)
    _check(lib().gw_rr_to_GG_fft(ctx.handle, ct.byref(grid), int(direction), int(stage), len(idx), _ip(idx), p,
                                 int(r0), int(n_rows), _dev(inp, "in", p), _dev(out, "out", p), _stream()), ctx)


def rr_to_GG_fft_noalloc(grid, direction, stage, fft_index, prec, r0, n_rows, inp, out):
    """gw_rr_to_GG_fft with its index maps in the library's fixed device array:
    for callers that may not allocate device memory (no context needed)."""
    p = prec_of(prec)
    idx = _i32(fft_index)
    _check(lib().gw_rr_to_GG_fft_noalloc(ct.byref(grid), int(direction), int(stage), len(idx), _ip(idx), p, int(r0),
                                         int(n_rows), _dev(inp, "in", p), _dev(out, "out", p), _stream()))


def zgemm_sliced(ctx, A, B, C, levels=5):
    """C = A B for complex128 device matrices, FP64-class accuracy on the tensor cores."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    if K2 != K or tuple(C.shape) != (M, N):
        raise ValueError("shapes do not match")
    for t in (A, B, C):
        if t.dtype != torch.complex128 or not t.is_cuda or t.stride(1) != 1:
            raise ValueError("complex128 device matrices with unit column stride needed")
    _check(lib().gw_zgemm_sliced(ctx.handle, int(M), int(N), int(K), ct.c_void_p(A.data_ptr()), int(A.stride(0)),
                                 ct.c_void_p(B.data_ptr()), int(B.stride(0)), ct.c_void_p(C.data_ptr()),
                                 int(C.stride(0)), int(levels), _stream()), ctx)


def tau_to_omega(ctx, kind, M, inp, out, prec):
    p = prec_of(prec)
    M = _f64(M)
    n = M.shape[0]
    elems = inp.numel() // n
    _check(lib().gw_tau_to_omega(ctx.handle, int(kind), n, _dp(M), elems, p, _dev(inp, "in", p),
                                 _dev(out, "out", p), _stream()), ctx)


def screen_W(ctx, grid, gvec, prec, chi_w, w_w, resid=True, refine=0):
    """W~(i omega) from chi0(i omega); refine > 0 adds that many FP64 refinement
    steps per frequency (gw_screen_W_refine).  Returns the residuals or None."""
    p = prec_of(prec)
    gv = _i32(gvec)
    n_omega = chi_w.shape[0]
    res = np.zeros(n_omega) if resid else None
    if refine:
        _check(lib().gw_screen_W_refine(ctx.handle, ct.byref(grid), len(gv), _ip(gv), n_omega, p, int(refine),
                                        _dev(chi_w, "chi_w", p), _dev(w_w, "w_w", p), _dp(res), _stream()), ctx)
    else:
        _check(lib().gw_screen_W(ctx.handle, ct.byref(grid), len(gv), _ip(gv), n_omega, p, _dev(chi_w, "chi_w", p),
                                 _dev(w_w, "w_w", p), _dp(res), _stream()), ctx)
    return res


def sigma_diag(ctx, grid, psi, eps, n_occ, mu, bands, tau, omega, C, S, w_tau, fft_index, prec, w_real=None):
    p = prec_of(prec)
    eps = _f64(eps)
    bands = _i32(bands)
    tau = _f64(tau)
    omega = _f64(omega)
    C = _f64(C)
    S = _f64(S)
    idx = _i32(fft_index)
    n = len(tau)
    n_n = len(bands)
    s_tau = np.zeros((2, n_n, n))
    s_iw = np.zeros((n_n, n), dtype=np.complex128)
    wr = None if w_real is None else _f64(w_real)
    n_real = 0 if wr is None else len(wr)
    s_re = np.zeros((n_n, max(n_real, 1)), dtype=np.complex128)
    st = lib().gw_sigma_diag(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p), _dp(eps),
                             float(mu), _ip(bands), n_n, n, _dp(tau), _dp(omega), _dp(C), _dp(S),
                             _dev(w_tau, "w_tau", p), len(idx), _ip(idx), p, _dp(s_tau),
                             s_iw.ctypes.data_as(_DP), _dp(wr), n_real,
                             s_re.ctypes.data_as(_DP) if n_real else None, _stream())
    _check(st, ctx)
    out = {"sigma_unocc": s_tau[0], "sigma_occ": s_tau[1], "sigma_iw": s_iw}
    if n_real:
        out["sigma_real"] = s_re
    return out


def sigma_diag_pw(ctx, grid, psi, eps, n_occ, mu, bands, tau, omega, C, S, w_tau, fft_index, pw_index, prec,
                  w_real=None):
    """gw_sigma_diag with G through its plane-wave form (gw_sigma_diag_pw); same outputs as sigma_diag."""
    p = prec_of(prec)
    bands = _i32(bands)
    tau = _f64(tau)
    idx = _i32(fft_index)
    pw = _i32(pw_index)
    n = len(tau)
    n_n = len(bands)
    s_tau = np.zeros((2, n_n, n))
    s_iw = np.zeros((n_n, n), dtype=np.complex128)
    wr = None if w_real is None else _f64(w_real)
    n_real = 0 if wr is None else len(wr)
    s_re = np.zeros((n_n, max(n_real, 1)), dtype=np.complex128)
    _check(lib().gw_sigma_diag_pw(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p),
                                  _dp(_f64(eps)), float(mu), _ip(bands), n_n, n, _dp(tau), _dp(_f64(omega)),
                                  _dp(_f64(C)), _dp(_f64(S)), _dev(w_tau, "w_tau", p), len(idx), _ip(idx), len(pw),
                                  _ip(pw), p, _dp(s_tau), s_iw.ctypes.data_as(_DP), _dp(wr), n_real,
                                  s_re.ctypes.data_as(_DP) if n_real else None, _stream()), ctx)
    out = {"sigma_unocc": s_tau[0], "sigma_occ": s_tau[1], "sigma_iw": s_iw}
    if n_real:
        out["sigma_real"] = s_re
    return out


def sigma_matrix(ctx, grid, psi, eps, n_occ, mu, bands, tau, omega, C, S, w_tau, fft_index, prec):
    """Full self-energy matrix over the listed bands (gw_sigma_matrix): a dict with
    sigma_unocc, sigma_occ [n_n][n_n][n] and sigma_iw [n_n][n_n][n], complex."""
    p = prec_of(prec)
    bands = _i32(bands)
    tau = _f64(tau)
    idx = _i32(fft_index)
    n = len(tau)
    n_n = len(bands)
    s_tau = np.zeros((2, n_n, n_n, n), dtype=np.complex128)
    s_iw = np.zeros((n_n, n_n, n), dtype=np.complex128)
    st = lib().gw_sigma_matrix(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p),
                               _dp(_f64(eps)), float(mu), _ip(bands), n_n, n, _dp(tau), _dp(_f64(omega)),
                               _dp(_f64(C)), _dp(_f64(S)), _dev(w_tau, "w_tau", p), len(idx), _ip(idx), p,
                               s_tau.ctypes.data_as(_DP), s_iw.ctypes.data_as(_DP), _stream())
    _check(st, ctx)
    return {"sigma_unocc": s_tau[0], "sigma_occ": s_tau[1], "sigma_iw": s_iw}


def sigma_to_tau(ctx, sigma_iw, Cinv, Sinv):
    """(Sigma_unocc(tau), Sigma_occ(-tau)) from Sigma(i omega) (gw_sigma_to_tau):
    [n_n][n] -> two real [n_n][n] arrays, or [n_n][n_n][n] -> two complex [n_n][n_n][n]."""
    sig = np.ascontiguousarray(sigma_iw, dtype=np.complex128)
    matrix = sig.ndim == 3
    n_n, n = sig.shape[0], sig.shape[-1]
    if matrix and sig.shape[1] != n_n:
        raise ValueError("a matrix Sigma must be [n_n][n_n][n]")
    out = np.zeros((2,) + sig.shape, dtype=np.complex128 if matrix else np.float64)
    _check(lib().gw_sigma_to_tau(ctx.handle, n_n, n, int(matrix), _dp(_f64(Cinv)), _dp(_f64(Sinv)),
                                 sig.ctypes.data_as(_DP), out.ctypes.data_as(_DP), _stream()), ctx)
    return out[0], out[1]


def qp_energies(ctx, omega, sigma_iw, eps, mu, vstat, w=None):
    """Linearised QP energies and spectral functions (gw_qp_energies): a dict with
    e_qp, z [n_n], sigma_eps, dsigma [n_n] complex and, if w is given, spectral [n_n][len(w)]."""
    omega = _f64(omega)
    sig = np.ascontiguousarray(np.atleast_2d(sigma_iw), dtype=np.complex128)
    n_n, n = sig.shape
    eps = _f64(np.atleast_1d(eps))
    vstat = _f64(np.atleast_1d(vstat))
    if len(omega) != n or len(eps) != n_n or len(vstat) != n_n:
        raise ValueError("sizes of omega, sigma_iw, eps and vstat disagree")
    wv = None if w is None else _f64(w)
    n_w = 0 if wv is None else len(wv)
    e = np.zeros(n_n)
    z = np.zeros(n_n)
    se = np.zeros(n_n, dtype=np.complex128)
    ds = np.zeros(n_n, dtype=np.complex128)
    sp = np.zeros((n_n, max(n_w, 1)))
    st = lib().gw_qp_energies(ctx.handle, n_n, n, _dp(omega), sig.ctypes.data_as(_DP), _dp(eps), float(mu),
                              _dp(vstat), n_w, _dp(wv), _dp(e), _dp(z), se.ctypes.data_as(_DP),
                              ds.ctypes.data_as(_DP), sp.ctypes.data_as(_DP) if n_w else None, _stream())
    _check(st, ctx)
    out = {"e_qp": e, "z": z, "sigma_eps": se, "dsigma": ds}
    if n_w:
        out["spectral"] = sp
    return out


def chi0_omega(ctx, grid, psi, eps, n_occ, mu, tau, C, fft_index, prec, chi_w, r_block=0):
    p = prec_of(prec)
    eps = _f64(eps)
    tau = _f64(tau)
    C = _f64(C)
    idx = _i32(fft_index)
    _check(lib().gw_chi0_omega(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p), _dp(eps),
                               float(mu), len(tau), _dp(tau), _dp(C), len(idx), _ip(idx), p, int(r_block),
                               _dev(chi_w, "chi_w", p), _stream()), ctx)


def chi0_omega_pw(ctx, grid, psi, eps, n_occ, mu, tau, C, fft_index, pw_index, prec, chi_w):
    """chi0(G,G',i omega) with G through its plane-wave form (gw_chi0_omega_pw);
    pw_index: FFT positions of the plane waves spanning the orbitals."""
    p = prec_of(prec)
    idx = _i32(fft_index)
    pw = _i32(pw_index)
    _check(lib().gw_chi0_omega_pw(ctx.handle, ct.byref(grid), psi.shape[0], int(n_occ), _dev(psi, "psi", p),
                                  _dp(_f64(eps)), float(mu), len(tau), _dp(_f64(tau)), _dp(_f64(C)), len(idx), _ip(idx),
                                  len(pw), _ip(pw), p, _dev(chi_w, "chi_w", p), _stream()), ctx)


def chi0_omega_kmesh(ctx, grid, nk, psi_k, eps_k, n_occ, mu, tau, C, gvec, prec, chi_w, r_block=0):
    """chi0_q(G,G',i omega) for every q of a Gamma-centred k mesh (gw_chi0_omega_kmesh).
    psi_k: device [N_k][N_b][N_r]; eps_k [N_k][N_b]; gvec [n_chi][3]; chi_w [N_k][n][n_chi][n_chi]."""
    p = prec_of(prec)
    nkv = _i32(nk)
    eps_k = _f64(eps_k)
    tau = _f64(tau)
    C = _f64(C)
    gv = _i32(gvec)
    _check(lib().gw_chi0_omega_kmesh(ctx.handle, ct.byref(grid), _ip(nkv), psi_k.shape[1], int(n_occ),
                                     _dev(psi_k, "psi_k", p), _dp(eps_k), float(mu), len(tau), _dp(tau), _dp(C),
                                     len(gv), _ip(gv), p, int(r_block), _dev(chi_w, "chi_w", p), _stream()), ctx)


def chi0_omega_kmesh_pw(ctx, grid, nk, psi_k, eps_k, n_occ, mu, tau, C, gvec, pw_index, prec, chi_w):
    """chi0_q(G,G',i omega) on a Gamma-centred k mesh with G_k through its plane-wave
    form (gw_chi0_omega_kmesh_pw).  psi_k: device [N_k][N_b][N_r]; pw_index: cell
    FFT positions of the plane waves spanning every exp(-i k.r) psi_nk; the rest as
    chi0_omega_kmesh."""
    p = prec_of(prec)
    nkv = _i32(nk)
    eps_k = _f64(eps_k)
    tau = _f64(tau)
    C = _f64(C)
    gv = _i32(gvec)
    pw = _i32(pw_index)
    _check(lib().gw_chi0_omega_kmesh_pw(ctx.handle, ct.byref(grid), _ip(nkv), psi_k.shape[1], int(n_occ),
                                        _dev(psi_k, "psi_k", p), _dp(eps_k), float(mu), len(tau), _dp(tau), _dp(C),
                                        len(gv), _ip(gv), len(pw), _ip(pw), p, _dev(chi_w, "chi_w", p), _stream()), ctx)


class Chi0Plan:
    """gw_chi0_plan: the chi0 chain set up once; launch() issues only kernels
    (no host-device copy, no synchronisation), so it can be captured in a CUDA
    graph.  Plans of one Context share its scratch arena: launch them in order."""

    def __init__(self, ctx, grid, n_b, eps, n_occ, mu, tau, C, fft_index, prec, r_block=0):
        self.ctx = ctx
        self.prec = prec
        self.n = len(tau)
        self._keep = (grid, _f64(eps), _f64(tau), _f64(C), _i32(fft_index))
        h = _P()
        _check(lib().gw_chi0_plan_create(ctx.handle, ct.byref(grid), int(n_b), int(n_occ), _dp(self._keep[1]),
                                         float(mu), self.n, _dp(self._keep[2]), _dp(self._keep[3]),
                                         len(self._keep[4]), _ip(self._keep[4]), prec_of(prec), int(r_block),
                                         ct.byref(h)), ctx)
        self.handle = h

    def launch(self, psi, chi_w):
        p = prec_of(self.prec)
        _check(lib().gw_chi0_plan_launch(self.handle, _dev(psi, "psi", p), _dev(chi_w, "chi_w", p), _stream()),
               self.ctx)

    def status(self):
        _check(lib().gw_chi0_plan_status(self.handle, _stream()), self.ctx)

    def close(self):
        if self.handle:
            lib().gw_chi0_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sigma_diag_kmesh(ctx, grid, nk, psi_k, eps_k, n_occ, mu, bands_k, tau, omega, C, S, w_tau, gvec, prec,
                     w_real=None):
    """Sigma_nk for (band, k index) pairs on a k mesh (gw_sigma_diag_kmesh); w_tau [N_k][n][n_chi][n_chi]."""
    p = prec_of(prec)
    nkv = _i32(nk)
    bk = _i32(np.asarray(bands_k).reshape(-1, 2))
    tau = _f64(tau)
    n = len(tau)
    n_n = bk.shape[0]
    s_tau = np.zeros((2, n_n, n))
    s_iw = np.zeros((n_n, n), dtype=np.complex128)
    wr = None if w_real is None else _f64(w_real)
    n_real = 0 if wr is None else len(wr)
    s_re = np.zeros((n_n, max(n_real, 1)), dtype=np.complex128)
    gv = _i32(gvec)
    _check(lib().gw_sigma_diag_kmesh(ctx.handle, ct.byref(grid), _ip(nkv), psi_k.shape[1], int(n_occ),
                                     _dev(psi_k, "psi_k", p), _dp(_f64(eps_k)), float(mu), _ip(bk), n_n, n, _dp(tau),
                                     _dp(_f64(omega)), _dp(_f64(C)), _dp(_f64(S)), _dev(w_tau, "w_tau", p), len(gv),
                                     _ip(gv), p, _dp(s_tau), s_iw.ctypes.data_as(_DP), _dp(wr), n_real,
                                     s_re.ctypes.data_as(_DP) if n_real else None, _stream()), ctx)
    out = {"sigma_unocc": s_tau[0], "sigma_occ": s_tau[1], "sigma_iw": s_iw}
    if n_real:
        out["sigma_real"] = s_re
    return out


class Batch:
    """Many systems through the whole hot path in one CUDA-graph launch
    (gw_batch_plan / gw_batch_launch / gw_batch_wait).  Each system is a dict
    with grid, psi (device), eps, n_occ, mu, tau, omega, C, S, Cinv, gvec,
    fft_index, bands, chi_w and w_tau (device work arrays) and optionally
    r_block and refine.  The host arrays are kept alive by the object."""

    def __init__(self, ctx, systems, prec):
        self.ctx = ctx
        self.prec = prec_of(prec)
        self._keep = []
        arr = (BatchSystem * len(systems))()
        self.shapes = []
        for i, s in enumerate(systems):
            eps, tau, om = _f64(s["eps"]), _f64(s["tau"]), _f64(s["omega"])
            C, S, Ci = _f64(s["C"]), _f64(s["S"]), _f64(s["Cinv"])
            gv, fi, bands = _i32(s["gvec"]), _i32(s["fft_index"]), _i32(s["bands"])
            self._keep += [eps, tau, om, C, S, Ci, gv, fi, bands]
            b = arr[i]
            b.grid = s["grid"]
            b.n_b = s["psi"].shape[0]
            b.n_occ = int(s["n_occ"])
            b.eps_h, b.mu, b.n = _dp(eps), float(s["mu"]), len(tau)
            b.tau_h, b.omega_h, b.C_h, b.S_h, b.Cinv_h = _dp(tau), _dp(om), _dp(C), _dp(S), _dp(Ci)
            b.n_chi, b.gvec_h, b.fft_index_h = len(fi), _ip(gv), _ip(fi)
            b.n_n, b.bands_h = len(bands), _ip(bands)
            b.r_block, b.refine_iters = int(s.get("r_block", 0)), int(s.get("refine", 0))
            b.psi = _dev(s["psi"], "psi", self.prec)
            b.chi_w = _dev(s["chi_w"], "chi_w", self.prec)
            b.w_tau = _dev(s["w_tau"], "w_tau", self.prec)
            self.shapes.append((len(bands), len(tau)))
        self._arr = arr
        h = ct.c_void_p()
        _check(lib().gw_batch_plan(ctx.handle, len(systems), arr, self.prec, ct.byref(h)), ctx)
        self.handle = h

    def launch(self):
        _check(lib().gw_batch_launch(self.handle, _stream()), self.ctx)

    def wait(self, timeout_ms=-1):
        """(list of Sigma_nn(i omega) arrays [n_n][n], list of per-system status)."""
        tot = sum(a * b for a, b in self.shapes)
        buf = np.zeros(2 * tot)
        st = (ct.c_int * len(self.shapes))()
        rc = lib().gw_batch_wait(self.handle, int(timeout_ms), _dp(buf), st)
        if rc not in (0, 5):           # numeric failures are reported per system
            _check(rc, self.ctx)
        z = buf[0::2] + 1j * buf[1::2]
        out, o = [], 0
        for a, b in self.shapes:
            out.append(z[o:o + a * b].reshape(a, b))
            o += a * b
        return out, list(st)

    def close(self):
        if getattr(self, "handle", None):
            lib().gw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
