"""ctypes binding of libls_gb300.so (C ABI of include/ls.h).

Argument marshalling only: geometry / option structs, the host n^2 callback,
torch tensors passed as raw device pointers with torch's current CUDA stream.
The library must have been built (``build_library()`` or ``__graft_entry__.build()``);
loading fails loudly otherwise -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LS_FP64, LS_MIXED, LS_MIXED32 = 0, 1, 2   # LS_MIXED32: solves only (complex64 Arnoldi vectors too)
_SHAPES = {"disc": 0, "kite": 1, "star": 2}
_STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "no convergence",
           5: "device wait timed out", 6: "unsupported"}


def lib_path() -> str:
    return os.path.join(_PKG, "_lib", "libls_gb300.so")


def build_library(verbose: bool = False) -> str:
    from . import build as _b
    return _b.build(verbose=verbose)


class LSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("shape", C.c_int), ("params", C.c_double * 8), ("collar_w", C.c_double),
                ("n1", C.c_int), ("n2", C.c_int), ("tau0", C.c_double), ("tau1", C.c_double),
                ("h", C.c_double), ("cart_x0", C.c_double), ("cart_y0", C.c_double),
                ("cart_nx", C.c_int), ("cart_ny", C.c_int)]


class Options(C.Structure):
    _fields_ = [("Q", C.c_int), ("p", C.c_int), ("R_a", C.c_double), ("R_b", C.c_double),
                ("R_cart", C.c_double), ("M", C.c_int), ("N_tau", C.c_int), ("q_polar", C.c_int),
                ("n_rho", C.c_int), ("n_theta", C.c_int), ("chi_s0", C.c_double),
                ("box_x0", C.c_double), ("box_y0", C.c_double), ("H", C.c_double),
                ("L", C.c_int), ("N_eq", C.c_int), ("n_fb", C.c_int), ("n_coll", C.c_int),
                ("rcond", C.c_double), ("rcond_mixed", C.c_double), ("n_threads", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("N", C.c_int64), ("n_collar", C.c_int64), ("n_cart", C.c_int64), ("nnz_near", C.c_int64),
                ("L", C.c_int), ("N_eq", C.c_int), ("n_es", C.c_int), ("n_loc", C.c_int), ("n_fb", C.c_int),
                ("fft_M", C.c_int), ("n_cells_occupied", C.c_int), ("plan_seconds", C.c_double),
                ("device_bytes", C.c_int64), ("stage_seconds", C.c_double * 4)]


def _info_dict(info):
    d = {f: getattr(info, f) for f, _ in PlanInfo._fields_}
    d["stage_seconds"] = {k: float(v) for k, v in zip(("nodes", "near", "accel", "device"), info.stage_seconds)}
    return d


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("residual", C.c_double),
                ("seconds", C.c_double)]


class TuneReport(C.Structure):
    _fields_ = [("nrhs", C.c_int), ("conv_cols64", C.c_int), ("conv_cols32", C.c_int), ("group32", C.c_int),
                ("near_cuda32", C.c_int), ("n_candidates", C.c_int), ("local_cuda32", C.c_int),
                ("proj_cuda32", C.c_int), ("fft_radix32", C.c_int),
                ("ms64_default", C.c_double),
                ("ms64_best", C.c_double), ("ms32_default", C.c_double), ("ms32_best", C.c_double)]


N2FN = C.CFUNCTYPE(C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)

_lib = None
_SIGS = {
    "ls_plan_create": ([C.POINTER(Geometry), N2FN, C.c_void_p, C.c_double, C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "ls_plan_info": ([C.c_void_p, C.POINTER(PlanInfo)]),
    "ls_plan_nodes": ([C.c_void_p, C.c_void_p, C.c_void_p]),
    "ls_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "ls_solve": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                  C.POINTER(SolveInfo), C.c_void_p]),
    "ls_farfield": ([C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "ls_plan_destroy": ([C.c_void_p]),
    "ls_status_string": ([C.c_int]),
    "ls_last_error": ([C.c_void_p]),
    "ls_host_plan_create": ([C.POINTER(Geometry), N2FN, C.c_void_p, C.c_double, C.POINTER(Options),
                            C.POINTER(C.c_void_p)]),
    "ls_host_plan_sizes": ([C.c_void_p, C.c_void_p]),
    "ls_host_plan_nodes": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ls_host_plan_near": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ls_host_plan_accel": ([C.c_void_p] + [C.c_void_p] * 8),
    "ls_host_plan_destroy": ([C.c_void_p]),
    "ls_host_accel3_create": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_double, C.c_int,
                              C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_void_p)]),
    "ls_host_accel3_sizes": ([C.c_void_p, C.c_void_p]),
    "ls_host_accel3_get": ([C.c_void_p] + [C.c_void_p] * 9),
    "ls_host_accel3_destroy": ([C.c_void_p]),
    "ls_host_ball3_create": ([C.c_void_p, C.POINTER(C.c_void_p)]),
    "ls_host_ball3_sizes": ([C.c_void_p, C.c_void_p]),
    "ls_host_ball3_nodes": ([C.c_void_p] + [C.c_void_p] * 6),
    "ls_host_ball3_destroy": ([C.c_void_p]),
    "ls_host_ball3_row": ([C.c_void_p, C.c_double, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ls_host_ball3_near": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                            C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    "ls_host_ball3_near_get": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ls_interior_window3": ([C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                             C.c_double, C.c_void_p, C.POINTER(C.c_int)]),
    "ls_set_stage_timing": ([C.c_void_p, C.c_int]),
    "ls_apply_noalloc": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ls_check_cells": ([C.POINTER(Geometry), N2FN, C.c_void_p, C.c_double, C.POINTER(Options), C.c_void_p]),
    "ls_get_stage_times": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "ls_plan_device_status": ([C.c_void_p]),
    "ls_set_wait_limit": ([C.c_void_p, C.c_int]),
    "ls_measure_peaks": ([C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ls_plan_autotune": ([C.c_void_p, C.c_int, C.POINTER(TuneReport)]),
    "ls_plan_set_variants": ([C.c_void_p, C.POINTER(TuneReport)]),
    "ls_plan_create3": ([C.c_void_p, C.c_void_p, N2FN, C.c_void_p, C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ls_batch_create": ([C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "ls_batch_offsets": ([C.c_void_p, C.c_void_p]),
    "ls_batch_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ls_batch_solve": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int,
                        C.POINTER(SolveInfo), C.c_void_p, C.c_void_p]),
    "ls_batch_destroy": ([C.c_void_p]),
    "ls_batch_last_error": ([C.c_void_p]),
}
EXPORTED = tuple(_SIGS)


def load_library(path: str | None = None):
    """Load libls_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise LSError(6, f"{p} is missing: build it with paper_1509_05063_gb300.build_library()")
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_char_p if name in ("ls_status_string", "ls_last_error", "ls_batch_last_error") else C.c_int
    if path is None:
        _lib = lib
    return lib


def _check(st: int, handle=None, batch=False):
    if st != 0:
        msg = ""
        if _lib is not None:
            msg = (_lib.ls_batch_last_error if batch else _lib.ls_last_error)(handle).decode()
        raise LSError(st, msg)


def geometry_from(wl) -> Geometry:
    g = Geometry()
    g.dim = 2
    g.shape = _SHAPES[wl.shape]
    for i, v in enumerate(wl.shape_params):
        g.params[i] = float(v)
    g.collar_w, g.n1, g.n2, g.tau0, g.tau1 = wl.collar_w, wl.n1, wl.n2, wl.tau0, wl.tau1
    g.h, g.cart_x0, g.cart_y0, g.cart_nx, g.cart_ny = wl.h, wl.cart_x0, wl.cart_y0, wl.cart_nx, wl.cart_ny
    return g


def options_from(wl, n_threads: int = 0, rcond: float = 0.0, rcond_mixed: float = 0.0) -> Options:
    o = Options()
    for f in ("Q", "p", "R_a", "R_b", "R_cart", "M", "N_tau", "q_polar", "n_rho", "n_theta", "chi_s0",
              "box_x0", "box_y0", "H", "L", "N_eq", "n_fb", "n_coll"):
        setattr(o, f, getattr(wl, f))
    o.rcond, o.rcond_mixed, o.n_threads = rcond, rcond_mixed, n_threads
    return o


def _n2_callback(n2, dim: int = 2):
    def cb(n, xy, out, ctx):
        try:
            pts = np.ctypeslib.as_array(xy, shape=(n, dim))
            vals = np.asarray(n2(pts), dtype=np.float64).reshape(n)
            np.ctypeslib.as_array(out, shape=(n,))[:] = vals
            return 0
        except Exception:  # the C side reports the failure
            return 1
    return N2FN(cb)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def check_cells(wl, n2, n_threads: int = 0):
    """ls_check_cells: validity and streamed near-field size of a cell layout.
    Returns a dict, or None when the layout is not usable (reason in 'error')."""
    load_library()
    out = np.zeros(7)
    cb = _n2_callback(n2)
    st = _lib.ls_check_cells(C.byref(geometry_from(wl)), cb, None, float(wl.kappa),
                             C.byref(options_from(wl, n_threads)), out.ctypes.data)
    if st != 0:
        return {"ok": False, "error": _lib.ls_last_error(None).decode()}
    return {"ok": True, "N": int(out[0]), "cells": int(out[1]), "block_entries": int(out[2]), "M": int(out[3]),
            "L": int(out[4]), "box_x0": float(out[5]), "box_y0": float(out[6])}


class Plan:
    """A device plan (ls_plan_create).  n2: callable mapping (n, 2) points to n^2 values."""

    def __init__(self, wl, n2, n_threads: int = 0, rcond: float = 0.0, rcond_mixed: float = 0.0):
        load_library()
        self.wl = wl
        self.kappa = float(wl.kappa)
        self._cb = _n2_callback(n2)
        h = C.c_void_p()
        st = _lib.ls_plan_create(C.byref(geometry_from(wl)), self._cb, None, self.kappa,
                                 C.byref(options_from(wl, n_threads, rcond, rcond_mixed)), C.byref(h))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        self._h = h
        info = PlanInfo()
        _check(_lib.ls_plan_info(self._h, C.byref(info)), self._h)
        self.info = _info_dict(info)
        self.N = int(info.N)

    def nodes(self):
        xy = np.zeros((self.N, 2))
        canon = np.zeros(self.N, np.int64)
        _check(_lib.ls_plan_nodes(self._h, xy.ctypes.data, canon.ctypes.data), self._h)
        return xy, canon

    def apply(self, u, out=None, prec: int = LS_FP64, stream=None):
        """A u for torch tensors on the GPU: complex128 (LS_FP64) or complex64
        (LS_MIXED), shape (N,) or (nrhs, N)."""
        import torch
        want = torch.complex128 if prec == LS_FP64 else torch.complex64
        if u.dtype != want or not u.is_cuda or not u.is_contiguous():
            raise LSError(1, f"u must be a contiguous CUDA {want} tensor")
        nrhs = 1 if u.dim() == 1 else u.shape[0]
        if u.shape[-1] != self.N:
            raise LSError(1, "length mismatch")
        if out is None:
            out = torch.empty_like(u)
        _check(_lib.ls_apply(self._h, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()), nrhs, prec,
                             _stream(stream)), self._h)
        return out

    def solve(self, uinc, u0=None, tol: float = 1e-10, max_iter: int = 500, restart: int = 100,
              prec: int = LS_FP64, stream=None):
        import torch
        if uinc.dtype != torch.complex128 or not uinc.is_cuda or not uinc.is_contiguous():
            raise LSError(1, "uinc must be a contiguous CUDA complex128 tensor")
        nrhs = 1 if uinc.dim() == 1 else uinc.shape[0]
        u = torch.zeros_like(uinc) if u0 is None else u0.clone()
        info = SolveInfo()
        st = _lib.ls_solve(self._h, C.c_void_p(uinc.data_ptr()), C.c_void_p(u.data_ptr()), nrhs, tol, max_iter,
                           restart, prec, C.byref(info), _stream(stream))
        res = {f: getattr(info, f) for f, _ in SolveInfo._fields_}
        if st not in (0, 4):
            _check(st, self._h)
        res["converged"] = st == 0
        return u, res

    def farfield(self, u, dirs, stream=None):
        import torch
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
        nrhs = 1 if u.dim() == 1 else u.shape[0]
        A = torch.empty((nrhs, len(dirs)), dtype=torch.complex128, device=u.device)
        _check(_lib.ls_farfield(self._h, C.c_void_p(u.data_ptr()), nrhs, dirs.ctypes.data, len(dirs),
                                C.c_void_p(A.data_ptr()), _stream(stream)), self._h)
        return A

    def apply_noalloc(self, u, out, prec: int = LS_FP64, stream=None):
        """A u for ONE right-hand side through ls_apply_noalloc: the library
        allocates nothing; its work arrays sit in a fixed device array shared by
        all calls (see include/ls.h).  out must be preallocated like u."""
        import torch
        want = torch.complex128 if prec == LS_FP64 else torch.complex64
        for t in (u, out):
            if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != self.N:
                raise LSError(1, f"u and out must be contiguous CUDA {want} tensors of length N")
        _check(_lib.ls_apply_noalloc(self._h, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()), prec,
                                     _stream(stream)), self._h)
        return out

    def device_status(self):
        """Raise LSError (status 5) if a device-side wait timed out since the last check."""
        _check(_lib.ls_plan_device_status(self._h), self._h)

    def autotune(self, nrhs: int = 16):
        """Time the apply's kernel variants on this plan's GPU and keep the
        fastest (ls_plan_autotune): lattice column-pass width (FP64 and
        complex64), complex64 right-hand-side group, tensor or CUDA cores
        for the near field, the local coefficients and the projection, and
        the complex64 lattice FFT's radix (16 or 4).
        Returns the choice and the default / best milliseconds."""
        r = TuneReport()
        _check(_lib.ls_plan_autotune(self._h, int(nrhs), C.byref(r)), self._h)
        return {f: getattr(r, f) for f, _ in TuneReport._fields_}

    def set_variants(self, conv_cols64: int = 1, conv_cols32: int = 1, group32: int = 16, near_cuda32: int = 0,
                     local_cuda32: int = 0, proj_cuda32: int = 0, fft_radix32: int = 16, **_ignored):
        """Set the kernel variants (ls_plan_set_variants); accepts a dict
        returned by autotune() as keyword arguments."""
        r = TuneReport(conv_cols64=int(conv_cols64), conv_cols32=int(conv_cols32), group32=int(group32),
                       near_cuda32=int(near_cuda32), local_cuda32=int(local_cuda32), proj_cuda32=int(proj_cuda32),
                       fft_radix32=int(fft_radix32))
        _check(_lib.ls_plan_set_variants(self._h, C.byref(r)), self._h)

    def set_wait_limit(self, polls: int):
        """Polls per device-side wait of the tensor-core near field (0: every wait gives up)."""
        _check(_lib.ls_set_wait_limit(self._h, int(polls)), self._h)

    def set_stage_timing(self, enable: bool):
        _check(_lib.ls_set_stage_timing(self._h, int(enable)), self._h)

    def stage_times(self, prec: int = LS_FP64):
        ms = np.zeros(5)
        calls = np.zeros(1, np.int64)
        _check(_lib.ls_get_stage_times(self._h, prec, ms.ctypes.data, calls.ctypes.data), self._h)
        return ms, int(calls[0])

    def close(self):
        if getattr(self, "_h", None):
            _lib.ls_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPlan:
    """Host-only plan construction (ls_host_plan_*): nodes, near-field CSR and
    accelerator matrices as numpy arrays.  No GPU needed."""

    def __init__(self, wl, n2, n_threads: int = 0, rcond: float = 0.0):
        load_library()
        self.wl = wl
        cb = _n2_callback(n2)
        h = C.c_void_p()
        st = _lib.ls_host_plan_create(C.byref(geometry_from(wl)), cb, None, float(wl.kappa),
                                      C.byref(options_from(wl, n_threads, rcond)), C.byref(h))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        self._h = h
        sz = np.zeros(8, np.int64)
        _check(_lib.ls_host_plan_sizes(h, sz.ctypes.data))
        self.N, self.nnz, self.nocc, self.n_es, self.nfb2, self.n_loc, self.M, self.P_len = map(int, sz)

    def nodes(self):
        xy = np.zeros((self.N, 2))
        canon = np.zeros(self.N, np.int64)
        wfac = np.zeros(self.N)
        _check(_lib.ls_host_plan_nodes(self._h, xy.ctypes.data, canon.ctypes.data, wfac.ctypes.data))
        return xy, canon, wfac

    def near(self):
        import scipy.sparse as sp
        rowptr = np.zeros(self.N + 1, np.int64)
        col = np.zeros(self.nnz, np.int32)
        val = np.zeros(self.nnz, np.complex128)
        _check(_lib.ls_host_plan_near(self._h, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data))
        return sp.csr_matrix((val, col, rowptr), shape=(self.N, self.N))

    def accel(self):
        occ = np.zeros(self.nocc, np.int32)
        P_off = np.zeros(self.nocc + 1, np.int64)
        P = np.zeros(self.P_len, np.complex128)
        Bp = np.zeros((self.nfb2, self.n_loc), np.complex128)
        BT = np.zeros((9, self.nfb2, self.n_es), np.complex128)
        Phi = np.zeros((self.N, self.nfb2), np.complex128)
        G = np.zeros((self.M, self.M), np.complex128)
        D = np.zeros((self.M, self.M), np.complex128)
        _check(_lib.ls_host_plan_accel(self._h, occ.ctypes.data, P_off.ctypes.data, P.ctypes.data, Bp.ctypes.data,
                                       BT.ctypes.data, Phi.ctypes.data, G.ctypes.data, D.ctypes.data))
        return dict(occ=occ, P_off=P_off, P=P, Bpinv=Bp, BT=BT, Phi=Phi, Gtab=G, Dtab=D)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ls_host_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostAccel3:
    """Host-only setup of the 3-D accelerator (ls_host_accel3_*) for a node set
    xyz (N, 3) with factors wfac = w m omega; the matrices as numpy arrays."""

    def __init__(self, xyz, wfac, kappa: float, box0, H: float, L: int, N_eq: int, p: int = 0,
                 m_coll: int = 0, rcond: float = 0.0, n_threads: int = 0):
        load_library()
        xyz = np.ascontiguousarray(xyz, np.float64)
        wfac = np.ascontiguousarray(wfac, np.float64)
        b0 = np.ascontiguousarray(box0, np.float64)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or wfac.shape != (xyz.shape[0],) or b0.shape != (3,):
            raise ValueError("xyz must be (N, 3), wfac (N,), box0 (3,)")
        h = C.c_void_p()
        st = _lib.ls_host_accel3_create(xyz.ctypes.data, wfac.ctypes.data, xyz.shape[0], float(kappa),
                                        b0.ctypes.data, float(H), int(L), int(N_eq), int(p), int(m_coll),
                                        float(rcond), int(n_threads), C.byref(h))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        self._h = h
        sz = np.zeros(7, np.int64)
        _check(_lib.ls_host_accel3_sizes(h, sz.ctypes.data))
        self.nocc, self.n_es, self.nb, self.n_loc, self.M, self.P_len, self.N = map(int, sz)

    def get(self):
        occ = np.zeros(self.nocc, np.int32)
        P_off = np.zeros(self.nocc + 1, np.int64)
        order = np.zeros(self.N, np.int64)
        P = np.zeros(self.P_len, np.complex128)
        Bp = np.zeros((self.nb, self.n_loc), np.complex128)
        BT = np.zeros((27, self.nb, self.n_es), np.complex128)
        Phi = np.zeros((self.N, self.nb), np.complex128)
        G = np.zeros((self.M,) * 3, np.complex128)
        D = np.zeros((self.M,) * 3, np.complex128)
        _check(_lib.ls_host_accel3_get(self._h, occ.ctypes.data, P_off.ctypes.data, order.ctypes.data, P.ctypes.data,
                                       Bp.ctypes.data, BT.ctypes.data, Phi.ctypes.data, G.ctypes.data, D.ctypes.data))
        return dict(occ=occ, P_off=P_off, order=order, P=P, Bpinv=Bp, BT=BT, Phi=Phi, Gtab=G, Dtab=D)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ls_host_accel3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ball3Params(C.Structure):
    _fields_ = [("a", C.c_double), ("w", C.c_double), ("n_f", C.c_int), ("n_s", C.c_int), ("Q", C.c_int),
                ("delta", C.c_double), ("h", C.c_double), ("tau0", C.c_double), ("tau1", C.c_double)]


class Rules3Params(C.Structure):
    _fields_ = [("R", C.c_double), ("p", C.c_int), ("q", C.c_int), ("n_rho", C.c_int), ("n_mu", C.c_int),
                ("n_phi", C.c_int), ("rc", C.c_double), ("rs", C.c_double), ("n_sig", C.c_int), ("n_th", C.c_int),
                ("chi_s0", C.c_double)]


class HostBall3:
    """Host-only 3-D ball discretisation (ls_host_ball3_*): nodes, weights,
    partitions of unity and grid indices as numpy arrays."""

    def __init__(self, a=1.0, w=0.5, n_f=17, n_s=9, Q=5, delta=0.25, h=0.1, tau0=0.3, tau1=0.95):
        load_library()
        prm = Ball3Params(float(a), float(w), int(n_f), int(n_s), int(Q), float(delta), float(h), float(tau0),
                          float(tau1))
        hd = C.c_void_p()
        st = _lib.ls_host_ball3_create(C.byref(prm), C.byref(hd))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        self._h = hd
        sz = np.zeros(4, np.int64)
        _check(_lib.ls_host_ball3_sizes(hd, sz.ctypes.data))
        self.N, self.n_shell, self.n_cart, self.grid_m = map(int, sz)

    def nodes(self):
        x = np.zeros((self.N, 3))
        w = np.zeros(self.N)
        om = np.zeros(self.N)
        psi = np.zeros(self.N)
        face = np.zeros(self.N, np.int8)
        grid = np.zeros((self.N, 3), np.int32)
        _check(_lib.ls_host_ball3_nodes(self._h, x.ctypes.data, w.ctypes.data, om.ctypes.data, psi.ctypes.data,
                                        face.ctypes.data, grid.ctypes.data))
        return dict(x=x, w=w, omega=om, psi=psi, face=face, grid=grid)

    @staticmethod
    def _rules(rules):
        if rules is None:
            return None
        d = dict(R=3.0, p=5, q=3, n_rho=16, n_mu=16, n_phi=32, rc=6.0, rs=6.0, n_sig=20, n_th=32, chi_s0=0.1)
        d.update(rules)
        return Rules3Params(**d)

    def near(self, kappa: float, box0, H: float, L: int, rows=None, rules: dict | None = None, n_threads: int = 0,
             stencils_only: bool = False):
        """Adjacent part of the 3-D operator over the listed rows (ls_host_ball3_near) as a
        scipy CSR matrix (len(rows) x N); stencils_only: the singular parts and the sparse
        -eta w omega G correction only."""
        import scipy.sparse as sp
        prm = self._rules(rules)
        b0 = np.ascontiguousarray(box0, np.float64)
        r = None if rows is None else np.ascontiguousarray(rows, np.int64)
        nnz = C.c_int64()
        st = _lib.ls_host_ball3_near(self._h, float(kappa), C.byref(prm) if prm is not None else None,
                                     b0.ctypes.data, float(H), int(L), None if r is None else r.ctypes.data,
                                     0 if r is None else len(r), int(bool(stencils_only)), int(n_threads),
                                     C.byref(nnz))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        n_rows = self.N if r is None else len(r)
        rowptr = np.zeros(n_rows + 1, np.int64)
        col = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value, np.complex128)
        _check(_lib.ls_host_ball3_near_get(self._h, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data))
        return sp.csr_matrix((val, col, rowptr), shape=(n_rows, self.N))

    def row(self, kappa: float, q: int, rules: dict | None = None):
        """Row q of the 3-D operator K (ls_host_ball3_row) and the cut-off values eta."""
        prm = self._rules(rules)
        row = np.zeros(self.N, np.complex128)
        eta = np.zeros(self.N)
        st = _lib.ls_host_ball3_row(self._h, float(kappa), C.byref(prm) if prm is not None else None, int(q),
                                    row.ctypes.data, eta.ctypes.data)
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        return row, eta

    def close(self):
        if getattr(self, "_h", None):
            _lib.ls_host_ball3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Accel3Params(C.Structure):
    _fields_ = [("box0", C.c_double * 3), ("H", C.c_double), ("L", C.c_int), ("N_eq", C.c_int), ("p", C.c_int),
                ("m_coll", C.c_int), ("rcond", C.c_double), ("n_threads", C.c_int)]


class Plan3(Plan):
    """A 3-D device plan of a penetrable ball (ls_plan_create3): ball and rule
    parameters as in HostBall3, n2: callable mapping (n, 3) points to n^2,
    the cube-cell box (corner box0, side H, L per axis) and the accelerator's
    N_eq, local-expansion degree p (0: 2 N_eq + 1) and fit truncation.
    apply / solve / farfield (3-D directions) as for Plan."""

    def __init__(self, n2, kappa: float, box0, H: float, L: int, N_eq: int, ball: dict | None = None,
                 rules: dict | None = None, p: int = 0, m_coll: int = 0, rcond: float = 0.0, n_threads: int = 0):
        load_library()
        b = dict(a=1.0, w=0.5, n_f=17, n_s=9, Q=5, delta=0.25, h=0.1, tau0=0.3, tau1=0.95)
        b.update(ball or {})
        prm = Ball3Params(float(b["a"]), float(b["w"]), int(b["n_f"]), int(b["n_s"]), int(b["Q"]), float(b["delta"]),
                          float(b["h"]), float(b["tau0"]), float(b["tau1"]))
        ru = HostBall3._rules(rules)
        acc = Accel3Params((C.c_double * 3)(*[float(v) for v in box0]), float(H), int(L), int(N_eq), int(p),
                           int(m_coll), float(rcond), int(n_threads))
        self.wl = None
        self.kappa = float(kappa)
        self._cb = _n2_callback(n2, dim=3)
        h = C.c_void_p()
        st = _lib.ls_plan_create3(C.byref(prm), C.byref(ru) if ru is not None else None, self._cb, None,
                                  self.kappa, C.byref(acc), C.byref(h))
        if st != 0:
            raise LSError(st, _lib.ls_last_error(None).decode())
        self._h = h
        info = PlanInfo()
        _check(_lib.ls_plan_info(self._h, C.byref(info)), self._h)
        self.info = _info_dict(info)
        self.N = int(info.N)

    def nodes(self):
        xyz = np.zeros((self.N, 3))
        canon = np.zeros(self.N, np.int64)
        _check(_lib.ls_plan_nodes(self._h, xyz.ctypes.data, canon.ctypes.data), self._h)
        return xyz, canon

    def farfield(self, u, dirs, stream=None):
        import torch
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        nrhs = 1 if u.dim() == 1 else u.shape[0]
        A = torch.empty((nrhs, len(dirs)), dtype=torch.complex128, device=u.device)
        _check(_lib.ls_farfield(self._h, C.c_void_p(u.data_ptr()), nrhs, dirs.ctypes.data, len(dirs),
                                C.c_void_p(A.data_ptr()), _stream(stream)), self._h)
        return A


def measure_peaks():
    """Measured FP64 FMA and TF32 tensor-core (tcgen05) throughput of the
    current GPU in TFLOP/s: {"fp64": ..., "tf32": ...} (ls_measure_peaks)."""
    load_library()
    f64, t32 = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ls_measure_peaks(C.byref(f64), C.byref(t32)))
    return {"fp64": f64.value, "tf32": t32.value}


def interior_window3(kappa, h, R=3.0, p=5, q=3, n_rho=16, n_mu=16, n_phi=32, chi_s0=0.1):
    """Window (2 Wn + 1)^3 of the 3-D interior singular rule (ls_interior_window3)."""
    load_library()
    Wn = C.c_int()
    args = (float(kappa), float(h), float(R), int(p), int(q), int(n_rho), int(n_mu), int(n_phi), float(chi_s0))
    st = _lib.ls_interior_window3(*args, None, C.byref(Wn))
    if st != 0:
        raise LSError(st, _lib.ls_last_error(None).decode())
    win = np.zeros((2 * Wn.value + 1,) * 3, np.complex128)
    _check(_lib.ls_interior_window3(*args, win.ctypes.data, C.byref(Wn)))
    return win, Wn.value


class Batch:
    """A multi-instance batch (ls_batch_create) over existing Plans.  Vectors are
    the instances' node vectors concatenated in plan order (offsets[i] ..
    offsets[i + 1]); the plans must outlive the batch."""

    def __init__(self, plans):
        load_library()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = C.c_void_p()
        st = _lib.ls_batch_create(arr, len(self.plans), C.byref(h))
        if st != 0:
            raise LSError(st, _lib.ls_batch_last_error(None).decode())
        self._h = h
        off = np.zeros(len(self.plans) + 1, np.int64)
        _check(_lib.ls_batch_offsets(self._h, off.ctypes.data), self._h, batch=True)
        self.offsets = off
        self.N = int(off[-1])

    def split(self, v):
        """Views of the instances' parts of a concatenated vector."""
        return [v[..., int(a):int(b)] for a, b in zip(self.offsets[:-1], self.offsets[1:])]

    def apply(self, u, out=None, prec: int = LS_FP64, stream=None):
        import torch
        want = torch.complex128 if prec == LS_FP64 else torch.complex64
        if u.dtype != want or not u.is_cuda or not u.is_contiguous() or u.numel() != self.N:
            raise LSError(1, f"u must be a contiguous CUDA {want} tensor of length {self.N}")
        if out is None:
            out = torch.empty_like(u)
        _check(_lib.ls_batch_apply(self._h, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()), prec,
                                   _stream(stream)), self._h, batch=True)
        return out

    def solve(self, uinc, u0=None, tol: float = 1e-10, max_iter: int = 500, restart: int = 100,
              prec: int = LS_FP64, stream=None):
        import torch
        if uinc.dtype != torch.complex128 or not uinc.is_cuda or not uinc.is_contiguous() or uinc.numel() != self.N:
            raise LSError(1, f"uinc must be a contiguous CUDA complex128 tensor of length {self.N}")
        u = torch.zeros_like(uinc) if u0 is None else u0.clone()
        info = SolveInfo()
        per = (SolveInfo * len(self.plans))()
        st = _lib.ls_batch_solve(self._h, C.c_void_p(uinc.data_ptr()), C.c_void_p(u.data_ptr()), tol, max_iter,
                                 restart, prec, C.byref(info), per, _stream(stream))
        res = {f: getattr(info, f) for f, _ in SolveInfo._fields_}
        if st not in (0, 4):
            _check(st, self._h, batch=True)
        res["converged"] = st == 0
        res["per_instance"] = [{f: getattr(p, f) for f, _ in SolveInfo._fields_} for p in per]
        return u, res

    def close(self):
        if getattr(self, "_h", None):
            _lib.ls_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
