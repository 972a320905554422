"""Thin Python binding of libslrf.so (include/slrf.h), argument marshalling only.

Every step of the eigensolver runs in the library's CUDA kernels; this module
only converts Python objects (numpy arrays on the host, torch CUDA tensors on
the device) into the pointers and sizes of the C ABI.  There is no fallback:
if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

# ---------------------------------------------------------------- constants
OK, EINVAL, ENOMEM, EBUDGET, ECUDA, ETIMEOUT = 0, 1, 2, 3, 4, 5
NOT_CONVERGED, STAGNATION, BREAKDOWN, SUBSPACE_TOO_SMALL, CHOLQR_FAIL, PENDING = 6, 7, 8, 9, 10, 11
PREC_FP64, PREC_MIXED = 0, 1
KRYLOV_COCG, KRYLOV_BICGSTAB = 0, 1
PRECOND_NONE, PRECOND_JACOBI, PRECOND_MG, PRECOND_AUTO, PRECOND_ILU = 0, 1, 2, 3, 4
SPMM_AUTO, SPMM_ROWGROUP, SPMM_STAGED, SPMM_NODEBLOCK, SPMM_SELL = 0, 1, 2, 3, 4
RULE_MIDPOINT, RULE_GAUSS_LEGENDRE, RULE_GAUSS_CHEBYSHEV, RULE_SLRF = 0, 1, 2, 3
RULES = {"midpoint": 0, "gauss_legendre": 1, "gauss_chebyshev": 2, "slrf": 3}
MAX_POLES = 16
NKERNEL_CLASSES = 15
MG_MAX_LEVELS = 16


class slrf_pencil(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("a_val", C.c_void_p), ("b_val", C.c_void_p), ("on_device", C.c_int32)]


class slrf_filter(C.Structure):
    _fields_ = [("n_poles", C.c_int32), ("sigma_re", C.POINTER(C.c_double)), ("sigma_im", C.POINTER(C.c_double)),
                ("w_re", C.POINTER(C.c_double)), ("w_im", C.POINTER(C.c_double))]


class slrf_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("krylov", C.c_int32), ("precond", C.c_int32),
                ("inner_maxit", C.c_int32), ("inner_tol", C.c_double), ("lock_tol", C.c_double),
                ("check_every", C.c_int32), ("eig_refine", C.c_int32), ("mem_budget", C.c_int64),
                ("profile", C.c_int32), ("spmm_rows", C.c_int32), ("gram_ozaki", C.c_int32),
                ("mg_nu", C.c_int32), ("mg_cycle", C.c_int32), ("mg_coarse", C.c_int32), ("mg_block", C.c_int32),
                ("mg_omega", C.c_double), ("mg_theta", C.c_double), ("mg_shift_limit", C.c_double),
                ("stagnation_window", C.c_int32),
                ("profile_mask", C.c_uint32), ("spmm_kernel", C.c_int32), ("mg_exact", C.c_int32),
                ("ilu_sweeps", C.c_int32), ("ilu_tri_sweeps", C.c_int32), ("sell_c", C.c_int32),
                ("sell_sigma", C.c_int32), ("mg_exact_tc", C.c_int32), ("mg_n_null", C.c_int32),
                ("mg_near_null", C.c_void_p)]


class slrf_report(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("n_wanted", C.c_int32), ("n_conv", C.c_int32),
                ("status_detail", C.c_int32), ("max_resid", C.c_double), ("max_resid_ax", C.c_double),
                ("krylov_iters", C.c_int64), ("spmv", C.c_int64), ("iters_per_pole", C.c_double * MAX_POLES),
                ("kernel_launches", C.c_int64), ("ms_total", C.c_double), ("ms_krylov", C.c_double),
                ("ms_rr", C.c_double), ("k_launches", C.c_int64 * NKERNEL_CLASSES),
                ("k_ms", C.c_double * NKERNEL_CLASSES), ("k_bytes", C.c_double * NKERNEL_CLASSES),
                ("k_flops", C.c_double * NKERNEL_CLASSES), ("mg_levels", C.c_int32), ("krylov_fp64", C.c_int32),
                ("spmm_kernel", C.c_int32)]

    def as_dict(self, lib=None) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("k_") and k != "iters_per_pole"}
        d["iters_per_pole"] = list(self.iters_per_pole)
        names = [class_name(i, lib) for i in range(NKERNEL_CLASSES)]
        d["kernels"] = {names[i]: {"launches": int(self.k_launches[i]), "ms": float(self.k_ms[i]),
                                   "bytes": float(self.k_bytes[i]), "flops": float(self.k_flops[i])}
                        for i in range(NKERNEL_CLASSES) if self.k_launches[i]}
        return d


class slrf_request(C.Structure):
    _fields_ = [("pencil", slrf_pencil), ("filter", slrf_filter), ("gamma", C.c_double), ("L", C.c_int32),
                ("V0", C.c_void_p), ("tol", C.c_double), ("max_outer", C.c_int32), ("opts", slrf_opts)]


_P = C.c_void_p
_SIGNATURES = {
    "slrf_status_str": (C.c_char_p, [C.c_int]),
    "slrf_last_error": (C.c_char_p, []),
    "slrf_kernel_class_name": (C.c_char_p, [C.c_int32]),
    "slrf_opts_default": (C.c_int, [C.POINTER(slrf_opts)]),
    "slrf_create": (C.c_int, [C.POINTER(_P), C.POINTER(slrf_pencil), C.POINTER(slrf_opts), _P]),
    "slrf_set_opts": (C.c_int, [_P, C.POINTER(slrf_opts)]),
    "slrf_destroy": (None, [_P]),
    "slrf_filter_apply": (C.c_int, [_P, C.POINTER(slrf_filter), _P, C.c_int64, C.c_int32, _P, C.c_int64,
                                    C.POINTER(slrf_report)]),
    "slrf_subspace_iterate": (C.c_int, [_P, C.POINTER(slrf_filter), C.c_double, C.c_int32, _P, C.c_int64,
                                        C.c_double, C.c_int32, _P, _P, C.c_int64, _P, C.POINTER(C.c_int32),
                                        C.POINTER(slrf_report)]),
    "slrf_subspace_iterate_host": (C.c_int, [_P, C.POINTER(slrf_filter), C.c_double, C.c_int32, _P, C.c_int64,
                                             C.c_double, C.c_int32, _P, _P, C.c_int64, _P, C.POINTER(C.c_int32),
                                             C.POINTER(slrf_report)]),
    "slrf_shifted_spmm": (C.c_int, [_P, C.POINTER(slrf_filter), C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]),
    "slrf_precond_apply": (C.c_int, [_P, C.POINTER(slrf_filter), C.c_int32, C.c_int32, C.c_int32, _P, _P, _P,
                                     C.POINTER(C.c_int32)]),
    "slrf_spmm_ab": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64]),
    "slrf_gram": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _P, C.c_int64, _P]),
    "slrf_syev": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "slrf_rayleigh_ritz": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _P, _P, C.c_int64, _P]),
    "slrf_design_poles": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "slrf_filter_eval": (C.c_int, [C.POINTER(slrf_filter), C.POINTER(C.c_double), C.c_int64,
                                   C.POINTER(C.c_double)]),
    "slrf_batch_iterate": (C.c_int, [C.c_int32, C.POINTER(_P), C.POINTER(slrf_filter), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int32), C.POINTER(_P), C.POINTER(C.c_int64), C.c_double,
                                     C.c_int32, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_int64), C.POINTER(_P),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int), C.POINTER(slrf_report), C.c_int32]),
    "slrf_request_bytes": (C.c_int64, [C.POINTER(slrf_request)]),
    "slrf_server_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int64]),
    "slrf_server_submit": (C.c_int, [_P, C.POINTER(slrf_request), C.POINTER(C.c_int64)]),
    "slrf_server_poll": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P, C.POINTER(C.c_int32),
                                   C.POINTER(slrf_report), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "slrf_server_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]),
    "slrf_server_destroy": (None, [_P]),
    "slrf_gram_noalloc": (C.c_int, [C.c_int64, C.c_int32, _P, C.c_int64, _P, C.c_int64, _P, _P]),
    "slrf_noalloc_last_error": (C.c_char_p, []),
    "slrf_fma_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), _P]),
    "slrf_release_cached_memory": (C.c_int, [C.c_int32]),
    "slrf_tall_product": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64]),
    "slrf_mg_describe": (C.c_int, [C.POINTER(slrf_pencil), C.POINTER(slrf_opts), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double), _P, _P, _P]),
    "slrf_mg_transfer": (C.c_int, [C.POINTER(slrf_pencil), C.POINTER(slrf_opts), C.c_int32, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double), _P, _P, _P]),
}

_lib = None


def load(path: str | None = None):
    """Load libslrf.so (built in-tree by ``_build.build_library``); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libslrf.so not found at {path}: run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == _build.LIB:
        _lib = lib
    return lib


def class_name(i, lib=None):
    lib = lib or load()
    s = lib.slrf_kernel_class_name(i)
    return s.decode() if s else None


class SlrfError(RuntimeError):
    def __init__(self, status, where=""):
        lib = load()
        msg = lib.slrf_status_str(status).decode()
        extra = lib.slrf_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra else ""))
        self.status = status


def _check(status, where, allowed=(OK,)):
    if status not in allowed:
        raise SlrfError(status, where)
    return status


def default_opts(**kw) -> slrf_opts:
    """Library defaults with the given fields replaced.  ``mg_near_null`` takes
    an (n, k) array (the near-null space of A for the multigrid aggregation);
    the options object keeps it alive and sets ``mg_n_null`` = k."""
    o = slrf_opts()
    load().slrf_opts_default(C.byref(o))
    for k, v in kw.items():
        _set_opt(o, k, v)
    return o


def _set_opt(o: slrf_opts, k: str, v):
    if not hasattr(o, k):
        raise KeyError(k)
    if k == "mg_near_null" and v is not None and not isinstance(v, int):
        arr = np.ascontiguousarray(v, dtype=np.float64)
        if arr.ndim != 2:
            raise ValueError("mg_near_null must be an (n, k) array")
        o._near_null = arr
        o.mg_near_null = arr.ctypes.data
        o.mg_n_null = arr.shape[1]
        return
    setattr(o, k, v)


class Filter:
    """N upper-half-plane poles and weights (conjugates implied)."""

    def __init__(self, sigma, w):
        sigma = np.asarray(sigma, dtype=complex).ravel()
        w = np.asarray(w, dtype=complex).ravel()
        if sigma.shape != w.shape or not 1 <= sigma.size <= MAX_POLES:
            raise ValueError("need 1..16 poles with one weight each")
        self.sigma = sigma
        self.w = w
        self._arr = [np.ascontiguousarray(a, dtype=np.float64) for a in (sigma.real, sigma.imag, w.real, w.imag)]
        dp = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in self._arr]
        self.c = slrf_filter(sigma.size, *dp)

    @property
    def n_poles(self):
        return self.sigma.size


def design_poles(rule: str, N: int, gamma: float, alpha: float = 1.0, beta: float = 0.01) -> Filter:
    """Pole/weight set from the library's host designer (quadrature rule or SLRF)."""
    out = [np.zeros(N) for _ in range(4)]
    ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in out]
    _check(load().slrf_design_poles(RULES[rule], N, alpha, beta, gamma, *ptrs), "slrf_design_poles")
    return Filter(out[0] + 1j * out[1], out[2] + 1j * out[3])


def filter_eval(f: Filter, x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    out = np.zeros_like(x)
    _check(load().slrf_filter_eval(C.byref(f.c), x.ctypes.data_as(C.POINTER(C.c_double)), x.size,
                                   out.ctypes.data_as(C.POINTER(C.c_double))), "slrf_filter_eval")
    return out


def fma_peak(precision: int = PREC_MIXED, stream=None) -> float:
    """Measured FP32 (PREC_MIXED) or FP64 (PREC_FP64) FMA throughput, flop/s."""
    v = C.c_double()
    _check(load().slrf_fma_peak(precision, C.byref(v), _stream_ptr(stream)), "slrf_fma_peak")
    return v.value


def release_cached_memory(device: int = 0) -> None:
    """Return the unused part of the library's device memory pool (memory
    released by destroyed handles, kept for later handles) to the driver."""
    _check(load().slrf_release_cached_memory(device), "slrf_release_cached_memory")


def mg_describe(pencil, opts: slrf_opts | None = None, coarse: bool = False) -> dict:
    """Multigrid hierarchy of a host pencil (built on the host by the library).

    Returns level sizes and stored entries, the setup time and, with
    ``coarse=True``, the coarsest pencil (dense) and its eigenvalues."""
    lib = load()
    keep = [np.ascontiguousarray(pencil.row_ptr, dtype=np.int32),
            np.ascontiguousarray(pencil.col_idx, dtype=np.int32),
            np.ascontiguousarray(pencil.a_val, dtype=np.float64),
            np.ascontiguousarray(pencil.b_val, dtype=np.float64)]
    p = slrf_pencil(int(pencil.n), int(keep[1].size), *[a.ctypes.data for a in keep], 0)
    o = opts or default_opts()
    nl = C.c_int32()
    ln = (C.c_int64 * MG_MAX_LEVELS)()
    lz = (C.c_int64 * MG_MAX_LEVELS)()
    ms = C.c_double()
    _check(lib.slrf_mg_describe(C.byref(p), C.byref(o), C.byref(nl), ln, lz, C.byref(ms), None, None, None),
           "slrf_mg_describe")
    out = {"levels": [int(ln[i]) for i in range(nl.value)], "nnz": [int(lz[i]) for i in range(nl.value)],
           "setup_ms": ms.value}
    if coarse:
        nc = out["levels"][-1]
        lam = np.zeros(nc)
        Ac = np.zeros((nc, nc))
        Bc = np.zeros((nc, nc))
        _check(lib.slrf_mg_describe(C.byref(p), C.byref(o), C.byref(nl), ln, lz, C.byref(ms),
                                    lam.ctypes.data_as(C.c_void_p), Ac.ctypes.data_as(C.c_void_p),
                                    Bc.ctypes.data_as(C.c_void_p)), "slrf_mg_describe")
        out.update(coarse_lambda=lam, coarse_A=Ac, coarse_B=Bc)
    return out


def mg_transfer(pencil, level: int, opts: slrf_opts | None = None):
    """Prolongator P_level of the host-built multigrid hierarchy as
    (ptr, col, val, n_rows, n_cols) CSR arrays, and rho_level, the spectral
    radius of diag(A_l)^{-1} A_l that scales the level's Jacobi damping."""
    lib = load()
    keep = [np.ascontiguousarray(pencil.row_ptr, dtype=np.int32),
            np.ascontiguousarray(pencil.col_idx, dtype=np.int32),
            np.ascontiguousarray(pencil.a_val, dtype=np.float64),
            np.ascontiguousarray(pencil.b_val, dtype=np.float64)]
    p = slrf_pencil(int(pencil.n), int(keep[1].size), *[a.ctypes.data for a in keep], 0)
    o = opts or default_opts()
    nr, nc, nz, rho = C.c_int32(), C.c_int32(), C.c_int64(), C.c_double()
    _check(lib.slrf_mg_transfer(C.byref(p), C.byref(o), level, C.byref(nr), C.byref(nc), C.byref(nz), C.byref(rho),
                                None, None, None), "slrf_mg_transfer")
    ptr = np.zeros(nr.value + 1, np.int32)
    col = np.zeros(nz.value, np.int32)
    val = np.zeros(nz.value)
    _check(lib.slrf_mg_transfer(C.byref(p), C.byref(o), level, C.byref(nr), C.byref(nc), C.byref(nz), C.byref(rho),
                                ptr.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
                                val.ctypes.data_as(C.c_void_p)), "slrf_mg_transfer")
    return (ptr, col, val, nr.value, nc.value), rho.value


def _dptr(t, dtype_name="float64"):
    """Device pointer of a contiguous torch CUDA tensor (row-major)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a torch CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Handle:
    """An slrf handle: the pencil on the device plus workspace, bound to a stream."""

    def __init__(self, pencil, opts: slrf_opts | None = None, stream=None):
        self.lib = load()
        self.n = int(pencil.n)
        self._keep = [np.ascontiguousarray(pencil.row_ptr, dtype=np.int32),
                      np.ascontiguousarray(pencil.col_idx, dtype=np.int32),
                      np.ascontiguousarray(pencil.a_val, dtype=np.float64),
                      np.ascontiguousarray(pencil.b_val, dtype=np.float64)]
        p = slrf_pencil(self.n, int(self._keep[1].size), *[a.ctypes.data for a in self._keep], 0)
        self.opts = opts or default_opts()
        self._stream = stream
        h = C.c_void_p()
        _check(self.lib.slrf_create(C.byref(h), C.byref(p), C.byref(self.opts), _stream_ptr(stream)), "slrf_create")
        self.h = h
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.slrf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **kw):
        for k, v in kw.items():
            _set_opt(self.opts, k, v)
        _check(self.lib.slrf_set_opts(self.h, C.byref(self.opts)), "slrf_set_opts")

    # ---- hot path ----------------------------------------------------------
    def filter_apply(self, f: Filter, V, U=None, allowed=(OK, NOT_CONVERGED)):
        import torch
        m = V.shape[1]
        if U is None:
            U = torch.empty_like(V)
        rep = slrf_report()
        st = self.lib.slrf_filter_apply(self.h, C.byref(f.c), _dptr(V), V.stride(0), m, _dptr(U), U.stride(0),
                                        C.byref(rep))
        _check(st, "slrf_filter_apply", allowed)
        return U, st, rep

    def subspace_iterate(self, f: Filter, gamma: float, V0, tol=1e-8, max_outer=50, theta=None, X=None,
                         resid=None, allowed=(OK, NOT_CONVERGED, SUBSPACE_TOO_SMALL, STAGNATION)):
        import torch
        L = V0.shape[1]
        dev = V0.device
        theta = torch.empty(L, dtype=torch.float64, device=dev) if theta is None else theta
        X = torch.empty_like(V0) if X is None else X
        resid = torch.empty(L, dtype=torch.float64, device=dev) if resid is None else resid
        nconv = C.c_int32(0)
        rep = slrf_report()
        st = self.lib.slrf_subspace_iterate(self.h, C.byref(f.c), gamma, L, _dptr(V0), V0.stride(0), tol,
                                            max_outer, _dptr(theta), _dptr(X), X.stride(0), _dptr(resid),
                                            C.byref(nconv), C.byref(rep))
        _check(st, "slrf_subspace_iterate", allowed)
        return theta, X, resid, nconv.value, st, rep

    def subspace_iterate_host(self, f: Filter, gamma: float, V0: np.ndarray, tol=1e-8, max_outer=50,
                              allowed=(OK, NOT_CONVERGED, SUBSPACE_TOO_SMALL, STAGNATION),
                              theta=None, X=None, resid=None):
        """Host-buffer solve.  theta (L), X (n x L) and resid (L) may be given
        as C-contiguous float64 arrays (e.g. in pinned memory, which the
        device-to-host copy of X reads fastest); else they are allocated."""
        V0 = np.ascontiguousarray(V0, dtype=np.float64)
        n, L = V0.shape

        def out(a, shape):
            if a is None:
                return np.zeros(shape)
            if a.shape != shape or a.dtype != np.float64 or not a.flags.c_contiguous or not a.flags.writeable:
                raise ValueError(f"output array must be a writable C-contiguous float64 array of shape {shape}")
            return a
        theta, X, resid = out(theta, (L,)), out(X, (n, L)), out(resid, (L,))
        nconv = C.c_int32(0)
        rep = slrf_report()
        st = self.lib.slrf_subspace_iterate_host(self.h, C.byref(f.c), gamma, L, V0.ctypes.data, L, tol, max_outer,
                                                 theta.ctypes.data, X.ctypes.data, L, resid.ctypes.data,
                                                 C.byref(nconv), C.byref(rep))
        _check(st, "slrf_subspace_iterate_host", allowed)
        return theta, X, resid, nconv.value, st, rep

    # ---- individual steps -------------------------------------------------
    def shifted_spmm(self, f: Filter, P, m, ldp, prec=PREC_MIXED, Q=None, mu=None):
        import torch
        Q = torch.empty_like(P) if Q is None else Q
        _check(self.lib.slrf_shifted_spmm(self.h, C.byref(f.c), prec, m, ldp, _dptr(P), _dptr(Q),
                                          _dptr(mu) if mu is not None else None), "slrf_shifted_spmm")
        return Q

    def precond_apply(self, f: Filter, R, m, ldp, prec=PREC_MIXED, Z=None, mu=None):
        """Z_j = C_j R_j (the Krylov preconditioner of every pole) in the block
        layout of shifted_spmm; returns (Z, multigrid levels used)."""
        import torch
        Z = torch.zeros_like(R) if Z is None else Z
        lv = C.c_int32()
        _check(self.lib.slrf_precond_apply(self.h, C.byref(f.c), prec, m, ldp, _dptr(R), _dptr(Z),
                                           _dptr(mu) if mu is not None else None, C.byref(lv)),
               "slrf_precond_apply")
        return Z, lv.value

    def spmm_ab(self, X, want_a=True, want_b=True):
        import torch
        m = X.shape[1]
        Y = torch.empty_like(X) if want_a else None
        Z = torch.empty_like(X) if want_b else None
        _check(self.lib.slrf_spmm_ab(self.h, m, _dptr(X), X.stride(0), _dptr(Y) if Y is not None else None, m,
                                     _dptr(Z) if Z is not None else None, m), "slrf_spmm_ab")
        return Y, Z

    def gram(self, X, Y):
        import torch
        m = X.shape[1]
        G = torch.empty((m, m), dtype=torch.float64, device=X.device)
        _check(self.lib.slrf_gram(self.h, m, _dptr(X), X.stride(0), _dptr(Y), Y.stride(0), _dptr(G)), "slrf_gram")
        return G

    def tall_product(self, A, B):
        """C = A B for A (n x k, n = the pencil's size) and B (k x m), device FP64."""
        import torch
        C = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=A.device)
        _check(self.lib.slrf_tall_product(self.h, A.shape[1], B.shape[1], _dptr(A), A.stride(0), _dptr(B),
                                          B.stride(0), _dptr(C), C.stride(0)), "slrf_tall_product")
        return C

    def syev(self, S):
        import torch
        m = S.shape[0]
        lam = torch.empty(m, dtype=torch.float64, device=S.device)
        Q = torch.empty_like(S)
        _check(self.lib.slrf_syev(self.h, m, _dptr(S), _dptr(lam), _dptr(Q)), "slrf_syev")
        return lam, Q

    def rayleigh_ritz(self, U, allowed=(OK,)):
        import torch
        m = U.shape[1]
        theta = torch.empty(m, dtype=torch.float64, device=U.device)
        X = torch.empty_like(U)
        resid = torch.empty(m, dtype=torch.float64, device=U.device)
        st = self.lib.slrf_rayleigh_ritz(self.h, m, _dptr(U), U.stride(0), _dptr(theta), _dptr(X), X.stride(0),
                                         _dptr(resid))
        _check(st, "slrf_rayleigh_ritz", allowed)
        return theta, X, resid


# ---------------------------------------------------------------- many problems
def batch_iterate(handles, filters, gammas, V0s, tol=1e-8, max_outer=50, n_threads=0):
    """Solve independent problems concurrently (one handle, i.e. one stream, each).

    handles: list of Handle; filters: list of Filter; gammas: floats; V0s: list
    of torch CUDA tensors (n_i x L_i).  Returns a list of
    (theta, X, resid, n_conv, status, report) per problem.
    """
    import torch
    k = len(handles)
    lib = load()
    torch.cuda.synchronize()   # inputs written on torch's stream must be complete
    hs = (C.c_void_p * k)(*[h.h for h in handles])
    fs = (slrf_filter * k)(*[f.c for f in filters])
    gam = (C.c_double * k)(*gammas)
    Ls = (C.c_int32 * k)(*[v.shape[1] for v in V0s])
    outs = [(torch.empty(v.shape[1], dtype=torch.float64, device=v.device), torch.empty_like(v),
             torch.empty(v.shape[1], dtype=torch.float64, device=v.device)) for v in V0s]
    v0p = (C.c_void_p * k)(*[v.data_ptr() for v in V0s])
    ldv = (C.c_int64 * k)(*[v.stride(0) for v in V0s])
    thp = (C.c_void_p * k)(*[o[0].data_ptr() for o in outs])
    xp = (C.c_void_p * k)(*[o[1].data_ptr() for o in outs])
    ldx = (C.c_int64 * k)(*[o[1].stride(0) for o in outs])
    rp = (C.c_void_p * k)(*[o[2].data_ptr() for o in outs])
    nconv = (C.c_int32 * k)()
    st = (C.c_int * k)()
    reps = (slrf_report * k)()
    lib.slrf_batch_iterate(k, hs, fs, gam, Ls, v0p, ldv, tol, max_outer, thp, xp, ldx, rp, nconv, st, reps,
                           n_threads)
    torch.cuda.synchronize()
    return [(outs[i][0], outs[i][1], outs[i][2], nconv[i], st[i], reps[i]) for i in range(k)]


class Server:
    """Request server (include/slrf.h slrf_server_*): host inputs, host outputs."""

    def __init__(self, n_workers=2, mem_budget=0):
        self.lib = load()
        s = C.c_void_p()
        _check(self.lib.slrf_server_create(C.byref(s), n_workers, int(mem_budget)), "slrf_server_create")
        self.s = s
        self._keep = {}

    def request(self, pencil, f: Filter, gamma, V0, tol=1e-8, max_outer=50, opts=None):
        arrs = [np.ascontiguousarray(pencil.row_ptr, dtype=np.int32), np.ascontiguousarray(pencil.col_idx, dtype=np.int32),
                np.ascontiguousarray(pencil.a_val, dtype=np.float64), np.ascontiguousarray(pencil.b_val, dtype=np.float64),
                np.ascontiguousarray(V0, dtype=np.float64)]
        r = slrf_request(slrf_pencil(int(pencil.n), int(arrs[1].size), *[x.ctypes.data for x in arrs[:4]], 0), f.c,
                         float(gamma), int(V0.shape[1]), arrs[4].ctypes.data, float(tol), int(max_outer),
                         opts or default_opts())
        return r, arrs

    def bytes(self, req):
        return self.lib.slrf_request_bytes(C.byref(req[0]))

    def submit(self, pencil, f: Filter, gamma, V0, tol=1e-8, max_outer=50, opts=None):
        req = self.request(pencil, f, gamma, V0, tol, max_outer, opts)
        t = C.c_int64()
        _check(self.lib.slrf_server_submit(self.s, C.byref(req[0]), C.byref(t)), "slrf_server_submit")
        self._keep[t.value] = (int(pencil.n), int(V0.shape[1]))
        return t.value

    def poll(self, ticket, wait=True):
        n, L = self._keep[ticket]
        theta, X, resid = np.zeros(L), np.zeros((n, L)), np.zeros(L)
        nconv, lat, res = C.c_int32(), C.c_double(), C.c_int()
        rep = slrf_report()
        st = self.lib.slrf_server_poll(self.s, ticket, 1 if wait else 0, theta.ctypes.data, X.ctypes.data,
                                       resid.ctypes.data, C.byref(nconv), C.byref(rep), C.byref(lat), C.byref(res))
        if st == PENDING:
            return None
        _check(st, "slrf_server_poll")
        del self._keep[ticket]
        return theta, X, resid, nconv.value, res.value, rep, lat.value

    def stats(self):
        q, r, f, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self.lib.slrf_server_stats(self.s, C.byref(q), C.byref(r), C.byref(f), C.byref(b))
        return {"queued": q.value, "running": r.value, "finished": f.value, "bytes_in_use": b.value}

    def close(self):
        if getattr(self, "s", None):
            self.lib.slrf_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
