"""Thin Python binding of libtucker.so (include/tucker.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Tensors are torch tensors
(device memory and the current CUDA stream come from torch); numpy arrays are accepted for host
inputs.  Nothing is computed in Python: if the CUDA library is missing or no GPU is visible the
calls raise, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_int32, c_int64, c_uint32, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtucker.so")

TUCKER_OK, TUCKER_EINVAL, TUCKER_ENOMEM, TUCKER_ECUDA = 0, -1, -2, -3
TUCKER_EEMPTY, TUCKER_ETIMEOUT, TUCKER_EINTERNAL, TUCKER_ENOTCONV = -4, -5, -6, -7
TUCKER_FP64, TUCKER_MIXED = 0, 1
TUCKER_HOST, TUCKER_DEVICE = 0, 1


class tucker_coo(Structure):
    _fields_ = [("dims", c_int64 * 3), ("nnz", c_int64), ("idx", c_void_p * 3),
                ("val", c_void_p), ("where", c_int32)]


class tucker_opts(Structure):
    _fields_ = [("precision", c_int32), ("tol", c_double), ("max_iter", c_int32),
                ("init", c_void_p * 3), ("init_where", c_int32), ("stream", c_void_p),
                ("flags", c_uint32)]


class tucker_result(Structure):
    _fields_ = [("G", c_void_p), ("U", c_void_p * 3), ("fit_history", c_void_p),
                ("where", c_int32), ("fit", c_double), ("iters", c_int32),
                ("rank_deficient", c_int32)]


class TuckerError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        lib = _lib()
        msg = lib.tucker_strerror(status).decode()
        detail = lib.tucker_last_error_detail().decode()
        super().__init__(f"{what}: {msg} ({status})" + (f" [{detail}]" if detail else ""))


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "tucker_tensor_create": (c_int32, [POINTER(tucker_coo), c_void_p, POINTER(c_void_p)]),
    "tucker_tensor_destroy": (c_int32, [c_void_p]),
    "tucker_tensor_info": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_double)]),
    "tucker_hosvd": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_hooi": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_sp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_mp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_strerror": (c_char_p, [c_int32]),
    "tucker_last_error_detail": (c_char_p, []),
    "tucker_ordering": (c_int32, [c_void_p, c_int32, c_int32, c_int32, POINTER(c_int64), c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "tucker_unfolding_gram": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    "tucker_ttmc": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                              c_void_p]),
    "tucker_slice_proj": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                                    c_void_p]),
    "tucker_gram": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    "tucker_eig_topk": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                  c_void_p]),
    "tucker_core": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_void_p,
                              POINTER(c_double), c_void_p]),
}


def _lib():
    """Loads libtucker.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_0711_2023_gb300.build.build() (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int, what: str):
    if status != TUCKER_OK:
        raise TuckerError(status, what)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the Tucker library runs on a CUDA GPU; none is visible")
    return torch


def _stream():
    return c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dptr(t):
    return c_void_p(t.data_ptr())


def _dev_f64(a):
    """A contiguous float64 CUDA tensor holding `a` (torch or numpy)."""
    torch = _torch()
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    return a.to(device="cuda", dtype=torch.float64).contiguous()


def _J(J):
    return (c_int32 * 3)(*[int(j) for j in J])


class Tensor:
    """Owning wrapper of a tucker_tensor handle (device copy of a COO tensor)."""

    def __init__(self, handle, dims):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)

    def close(self):
        if self.handle:
            _lib().tucker_tensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return tucker_tensor_info(self)


def tucker_tensor_create(idx, val, dims) -> Tensor:
    """idx: int32 [3, nnz] and val: float64 [nnz], either both CUDA tensors (device path) or
    numpy arrays / CPU tensors (copied from host memory by the library)."""
    torch = _torch()
    lib = _lib()
    coo = tucker_coo()
    for a in range(3):
        coo.dims[a] = int(dims[a])
    keep = []
    if isinstance(idx, torch.Tensor) and idx.is_cuda:
        idx_t = idx.to(torch.int32).contiguous()
        val_t = val.to(torch.float64).contiguous()
        keep += [idx_t, val_t]
        coo.nnz = int(val_t.numel())
        for a in range(3):
            coo.idx[a] = idx_t[a].data_ptr() if coo.nnz else None
        coo.val = val_t.data_ptr() if coo.nnz else None
        coo.where = TUCKER_DEVICE
    else:
        idx_h = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        val_h = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
        keep += [idx_h, val_h]
        coo.nnz = int(val_h.shape[0])
        for a in range(3):
            coo.idx[a] = idx_h[a].ctypes.data if coo.nnz else None
        coo.val = val_h.ctypes.data if coo.nnz else None
        coo.where = TUCKER_HOST
    h = c_void_p()
    _check(lib.tucker_tensor_create(ctypes.byref(coo), _stream(), ctypes.byref(h)),
           "tucker_tensor_create")
    return Tensor(h, dims)


def tucker_tensor_destroy(X: Tensor):
    X.close()


def tucker_strerror(status: int) -> str:
    return _lib().tucker_strerror(int(status)).decode()


def tucker_last_error_detail() -> str:
    return _lib().tucker_last_error_detail().decode()


def tucker_tensor_info(X: Tensor):
    nnz, n2 = c_int64(), c_double()
    _check(_lib().tucker_tensor_info(X.handle, ctypes.byref(nnz), ctypes.byref(n2)),
           "tucker_tensor_info")
    return int(nnz.value), float(n2.value)


def _opts(precision, tol, max_iter, init):
    o = tucker_opts()
    o.precision = TUCKER_MIXED if precision in ("mixed", TUCKER_MIXED) else TUCKER_FP64
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.init_where = TUCKER_DEVICE
    o.stream = _stream().value
    o.flags = 0
    keep = []
    if init is not None:
        for a in range(3):
            if init[a] is not None:
                t = _dev_f64(init[a])
                keep.append(t)
                o.init[a] = t.data_ptr()
    return o, keep


def _run(fn_name, X: Tensor, J, precision, tol, max_iter, init):
    torch = _torch()
    o, keep = _opts(precision, tol, max_iter, init)
    G = torch.empty(tuple(int(j) for j in J), dtype=torch.float64, device="cuda")
    U = [torch.empty((X.dims[a], int(J[a])), dtype=torch.float64, device="cuda") for a in range(3)]
    fh = torch.empty(max(1, int(max_iter)), dtype=torch.float64, device="cuda")
    r = tucker_result()
    r.G = G.data_ptr()
    for a in range(3):
        r.U[a] = U[a].data_ptr()
    r.fit_history = fh.data_ptr()
    r.where = TUCKER_DEVICE
    _check(getattr(_lib(), fn_name)(X.handle, _J(J), ctypes.byref(o), ctypes.byref(r)), fn_name)
    iters = int(r.iters)
    return dict(G=G, U=U, fit=float(r.fit), iters=iters,
                fit_history=fh[:iters].cpu().numpy().tolist(), rank_deficient=int(r.rank_deficient))


def tucker_hosvd(X: Tensor, J, precision="fp64"):
    return _run("tucker_hosvd", X, J, precision, 0.0, 1, None)


def tucker_hooi(X: Tensor, J, tol=1e-4, max_iter=50, precision="fp64", init=None):
    return _run("tucker_hooi", X, J, precision, tol, max_iter, init)


def tucker_sp(X: Tensor, J, C_raw, tol=1e-4, max_iter=50, precision="fp64"):
    return _run("tucker_sp", X, J, precision, tol, max_iter, [None, None, C_raw])


def tucker_mp(X: Tensor, J, tol=1e-4, max_iter=50, precision="fp64"):
    return _run("tucker_mp", X, J, precision, tol, max_iter, None)


# ---- step entry points -------------------------------------------------------------------------

def tucker_ordering(X: Tensor, n, m, o):
    """Copies ordering (n, m, o) to host numpy arrays."""
    lib = _lib()
    F = c_int64()
    _check(lib.tucker_ordering(X.handle, n, m, o, ctypes.byref(F), None, None, None, None, None,
                               TUCKER_HOST), "tucker_ordering")
    nnz, _ = tucker_tensor_info(X)
    F = int(F.value)
    root_ptr = np.zeros(X.dims[n] + 1, dtype=np.int64)
    fiber_idx = np.zeros(max(F, 1), dtype=np.int32)
    fiber_ptr = np.zeros(F + 1, dtype=np.int64)
    leaf_idx = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=np.float64)
    _check(lib.tucker_ordering(X.handle, n, m, o, None, root_ptr.ctypes.data,
                               fiber_idx.ctypes.data, fiber_ptr.ctypes.data, leaf_idx.ctypes.data,
                               val.ctypes.data, TUCKER_HOST), "tucker_ordering")
    return dict(root_ptr=root_ptr, fiber_idx=fiber_idx[:F], fiber_ptr=fiber_ptr,
                leaf_idx=leaf_idx[:nnz], val=val[:nnz], nfibers=F)


def tucker_unfolding_gram(X: Tensor, n):
    torch = _torch()
    M = torch.empty((X.dims[n], X.dims[n]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_unfolding_gram(X.handle, n, _dptr(M), _stream()), "tucker_unfolding_gram")
    return M


def _others(n):
    return [a for a in range(3) if a != n]


def tucker_ttmc(X: Tensor, n, Um, Uo):
    torch = _torch()
    m, o = _others(n)
    Um, Uo = _dev_f64(Um), _dev_f64(Uo)
    Y = torch.empty((X.dims[n], Um.shape[1] * Uo.shape[1]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_ttmc(X.handle, n, _dptr(Um), Um.shape[1], _dptr(Uo), Uo.shape[1],
                              _dptr(Y), _stream()), "tucker_ttmc")
    return Y


def tucker_slice_proj(X: Tensor, n, m, Um):
    torch = _torch()
    o = 3 - n - m
    Um = _dev_f64(Um)
    Y = torch.empty((X.dims[n], X.dims[o] * Um.shape[1]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_slice_proj(X.handle, n, m, _dptr(Um), Um.shape[1], _dptr(Y), _stream()),
           "tucker_slice_proj")
    return Y


def tucker_gram(Y1, Y2=None):
    torch = _torch()
    Y1 = _dev_f64(Y1)
    rows = Y1.shape[0]
    M = torch.empty((rows, rows), dtype=torch.float64, device="cuda")
    if Y2 is not None:
        Y2 = _dev_f64(Y2)
    _check(_lib().tucker_gram(_dptr(Y1), Y1.shape[1], _dptr(Y2) if Y2 is not None else None,
                              Y2.shape[1] if Y2 is not None else 0, rows, _dptr(M), _stream()),
           "tucker_gram")
    return M


def tucker_eig_topk(M, J, U0=None):
    torch = _torch()
    M = _dev_f64(M)
    n = M.shape[0]
    U = torch.empty((n, int(J)), dtype=torch.float64, device="cuda")
    lam = torch.empty(int(J), dtype=torch.float64, device="cuda")
    U0p = None
    if U0 is not None:
        U0 = _dev_f64(U0)
        U0p = _dptr(U0)
    _check(_lib().tucker_eig_topk(_dptr(M), n, int(J), U0p, _dptr(U), _dptr(lam), _stream()),
           "tucker_eig_topk")
    return U, lam


def tucker_core(X: Tensor, A, B, C):
    torch = _torch()
    A, B, C = _dev_f64(A), _dev_f64(B), _dev_f64(C)
    J = (A.shape[1], B.shape[1], C.shape[1])
    G = torch.empty(J, dtype=torch.float64, device="cuda")
    g2 = c_double()
    _check(_lib().tucker_core(X.handle, _dptr(A), _dptr(B), _dptr(C), _J(J), _dptr(G),
                              ctypes.byref(g2), _stream()), "tucker_core")
    return G, float(g2.value)


def header_functions(header_path=None):
    """Names of the functions declared in include/tucker.h (for export checks)."""
    import re
    path = header_path or os.path.join(os.path.dirname(HERE), "include", "tucker.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tucker_[a-z0-9_]+)\s*\(", text)))
