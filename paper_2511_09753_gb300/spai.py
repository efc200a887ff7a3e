"""Python binding of libspai.so (ctypes; argument marshalling only).

Every numeric step runs in the library's CUDA kernels; this module converts
numpy arrays / torch CUDA tensors to pointers and codes to exceptions.  If
the shared library is missing the import of a handle fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspai.so")

SPAI_FP64, SPAI_MIXED = 0, 1
SPAI_MR, SPAI_LOMR, SPAI_CG = 0, 1, 2
SPAI_DROP_NONE, SPAI_DROP_TOPK_COL, SPAI_DROP_TOPK_COL_DIAG = 0, 1, 2
PREC_NONE, PREC_JACOBI, PREC_SPAI, PREC_SPAI_SYM = 0, 1, 2, 3
METHODS = {"mr": SPAI_MR, "lomr": SPAI_LOMR, "cg": SPAI_CG,
           "mr_pi": 3, "lomr_pi": 4, "cg_pi": 5}  # Section 5's forms with Pi = diag(A)^{-1}

OK, CONVERGED_EARLY, LOMR_FALLBACK, PCG_MAXIT, PCG_BREAKDOWN = 0, 1, 2, 3, 4
ERR_CAPACITY = -8

EXPORTED = ["spai_validate_csr", "spai_status_string", "spai_create", "spai_destroy", "spai_reset",
            "spai_set_stream", "spai_run", "spai_mr", "spai_lomr", "spai_cg",
            "spai_residual_norm", "spai_get_nnz", "spai_get_M", "spai_set_M", "spai_apply",
            "pcg_solve", "spai_save_state", "spai_load_state", "spai_set_timing",
            "spai_get_stats", "spai_true_residual_noalloc", "spai_create_batched",
            "spai_batch_info", "spai_batch_history", "spai_batch_residual_norms",
            "spai_batch_get_M", "pcg_solve_block", "spai_set_pcg_prec", "spai_sym_lanczos",
            "spai_fixed_pattern", "spai_fpmr_create", "spai_fpmr_forward", "spai_fpmr_backward",
            "spai_fpmr_info", "spai_fpmr_destroy", "spai_autotune", "spai_drop_global",
            "spai_drop_heuristic", "spai_run_global", "spai_fpmr_set_method"]


class SpaiError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


class _Opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("cap_factor", C.c_double)]


class _Hist(C.Structure):
    _fields_ = [("resnorm", C.c_void_p), ("coef", C.c_void_p), ("iters_done", C.c_int),
                ("flags", C.c_int), ("nnz", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("colpass_launches", C.c_int64), ("colpass_bytes", C.c_int64),
                ("colpass_ms", C.c_double), ("pcg_launches", C.c_int64),
                ("other_launches", C.c_int64), ("spgemm_columns", C.c_int64),
                ("colpass_r_bytes", C.c_int64), ("colpass_steady_launches", C.c_int64)]


_lib = None
_lib_path = LIB_PATH


def use_library(path: str) -> None:
    """Bind to another build of the same library (the profiling build
    libspai_phase.so) instead of libspai.so; call before the first load()."""
    global _lib_path
    if _lib is not None and path != _lib_path:
        raise RuntimeError("the library is already loaded")
    _lib_path = path


def load():
    """Load libspai.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_lib_path):
        raise RuntimeError(f"libspai.so not built ({_lib_path}); run paper_2511_09753_gb300.build")
    lib = C.CDLL(_lib_path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "spai_validate_csr": (i32, [i64, i64, vp, vp, vp, i32]),
        "spai_status_string": (C.c_char_p, [i32]),
        "spai_create": (i32, [C.POINTER(vp), i64, i64, vp, vp, vp, i32, C.POINTER(_Opts), vp]),
        "spai_destroy": (i32, [vp]),
        "spai_reset": (i32, [vp]),
        "spai_set_stream": (i32, [vp, vp]),
        "spai_run": (i32, [vp, i32, i32, i32, C.POINTER(_Hist)]),
        "spai_mr": (i32, [vp, i32, i32, C.POINTER(_Hist)]),
        "spai_lomr": (i32, [vp, i32, i32, C.POINTER(_Hist)]),
        "spai_cg": (i32, [vp, i32, i32, C.POINTER(_Hist)]),
        "spai_residual_norm": (i32, [vp, C.POINTER(dbl)]),
        "spai_get_nnz": (i32, [vp, C.POINTER(i64)]),
        "spai_get_M": (i32, [vp, C.POINTER(i64), vp, vp, vp, i32]),
        "spai_set_M": (i32, [vp, vp, vp, vp, i32]),
        "spai_apply": (i32, [vp, vp, vp, i32, i64]),
        "pcg_solve": (i32, [vp, vp, vp, i32, dbl, i32, i32, i32, C.POINTER(i32), C.POINTER(dbl)]),
        "pcg_solve_block": (i32, [vp, i32, vp, vp, dbl, i32, i32, i32, vp, vp, vp]),
        "spai_set_pcg_prec": (i32, [vp, i32]),
        "spai_fixed_pattern": (i32, [vp, i32]),
        "spai_fpmr_create": (i32, [C.POINTER(vp), i64, i64, vp, vp, i32, i32, vp]),
        "spai_fpmr_forward": (i32, [vp, vp, i32, C.POINTER(dbl)]),
        "spai_fpmr_backward": (i32, [vp, dbl, vp, i32]),
        "spai_fpmr_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
        "spai_fpmr_destroy": (i32, [vp]),
        "spai_fpmr_set_method": (i32, [vp, i32]),
        "spai_autotune": (i32, [vp, i32, i32, C.POINTER(dbl)]),
        "spai_drop_global": (i32, [vp, i32, i64]),
        "spai_drop_heuristic": (i32, [vp, i64]),
        "spai_run_global": (i32, [vp, i32, i32, i64, i64, C.POINTER(_Hist)]),
        "spai_sym_lanczos": (i32, [vp, i32, vp, vp, vp, C.POINTER(i32), C.POINTER(dbl),
                                   C.POINTER(dbl)]),
        "spai_save_state": (i32, [vp, vp, C.POINTER(C.c_size_t)]),
        "spai_load_state": (i32, [vp, vp, C.c_size_t]),
        "spai_set_timing": (i32, [vp, i32]),
        "spai_get_stats": (i32, [vp, C.POINTER(_Stats)]),
        "spai_true_residual_noalloc": (i32, [i64, vp, vp, vp, vp, vp, vp, vp]),
        "spai_create_batched": (i32, [C.POINTER(vp), i32, vp, vp, vp, vp, vp, C.POINTER(_Opts),
                                      vp]),
        "spai_batch_info": (i32, [vp, C.POINTER(i32), vp]),
        "spai_batch_history": (i32, [vp, vp, vp, vp]),
        "spai_batch_residual_norms": (i32, [vp, vp]),
        "spai_batch_get_M": (i32, [vp, i32, C.POINTER(i64), vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().spai_status_string(int(code)).decode()


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), (1 if a.is_cuda else 0), a
    return a.ctypes.data, 0, a


def _check_noalloc_args(n, rowptr, colind, vals, b, x, out):
    """The C entry point trusts its device pointers; a host tensor, a wrong
    dtype or a short array would make the kernel read or write out of bounds.
    Checked here, before anything is launched."""
    import torch
    n = int(n)
    named = (("rowptr", rowptr, torch.int32), ("colind", colind, torch.int32),
             ("vals", vals, torch.float64), ("b", b, torch.float64), ("x", x, torch.float64),
             ("out", out, torch.float64))
    cur = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t, dt in named:
        if not getattr(t, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, not the current device")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if 1 <= n <= (1 << 24):  # the library itself rejects other n with a status code
        if rowptr.numel() != n + 1:
            raise ValueError(f"rowptr needs n + 1 = {n + 1} entries, has {rowptr.numel()}")
        if b.numel() != n or x.numel() != n:
            raise ValueError(f"b and x need n = {n} entries")
        if colind.numel() != vals.numel():
            raise ValueError("colind and vals differ in length")
    if out.numel() < 2:
        raise ValueError("out needs 2 entries")


def true_residual_noalloc(n, rowptr, colind, vals, b, x, out, stream=None) -> int:
    """Allocation-free ||b - A x||_2 and ||b||_2 into the 2-element FP64 CUDA
    tensor `out` (all arguments contiguous CUDA tensors on the current
    device: rowptr and colind int32, vals, b, x and out float64).  For
    callers that cannot allocate device memory; see include/spai.h.  Raises
    ValueError on a bad argument before anything runs; returns the status
    code of the C call."""
    _check_noalloc_args(n, rowptr, colind, vals, b, x, out)
    return load().spai_true_residual_noalloc(int(n), rowptr.data_ptr(), colind.data_ptr(),
                                             vals.data_ptr(), b.data_ptr(), x.data_ptr(),
                                             out.data_ptr(), _stream_ptr(stream))


def validate_csr(n, rowptr, colind, vals, check_symmetry=True) -> int:
    rp, ci, va = _np(rowptr, np.int32), _np(colind, np.int32), _np(vals, np.float64)
    return load().spai_validate_csr(int(n), int(len(va)), rp.ctypes.data, ci.ctypes.data,
                                    va.ctypes.data, int(check_symmetry))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Spai:
    """Handle for one SPD matrix A (CSR, exactly symmetric).

    prec: "fp64" or "mixed" (FP32 values, FP64 reductions and coefficients).
    cap_factor: column capacity and drop cap, cap_j = floor(f * nnz(A[:, j])).
    Arrays may be numpy (host) or torch CUDA tensors (device).
    """

    def __init__(self, n, rowptr, colind, vals, prec="fp64", cap_factor=2.0, stream=None):
        self.lib = load()
        self.n = int(n)
        if hasattr(vals, "data_ptr"):
            rp, ci, va = rowptr, colind, vals
        else:
            rp, ci, va = _np(rowptr, np.int32), _np(colind, np.int32), _np(vals, np.float64)
        self.nnz = int(va.numel() if hasattr(va, "numel") else len(va))
        p_rp, dev, k1 = _ptr(rp)
        p_ci, _, k2 = _ptr(ci)
        p_va, _, k3 = _ptr(va)
        opts = _Opts(SPAI_MIXED if prec == "mixed" else SPAI_FP64, float(cap_factor))
        h = C.c_void_p()
        rc = self.lib.spai_create(C.byref(h), self.n, self.nnz, p_rp, p_ci, p_va, dev,
                                  C.byref(opts), _stream_ptr(stream))
        if rc != 0:
            raise SpaiError(rc, "spai_create")
        self.h = h
        self.prec = prec

    def close(self):
        if getattr(self, "h", None):
            self.lib.spai_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, where, ok=(OK,)):
        if rc not in ok and rc < 0:
            raise SpaiError(rc, where)
        return rc

    def run(self, method, iters, drop=True, keep_diag=False):
        """iters iterations of method; drop: the per-column hard threshold
        (keep_diag: it always keeps the column's diagonal entry).  Returns
        dict(status, done, flags, resnorm[0..iters], coef, nnz[0..iters]) with
        nnz[i] = nnz(M_i) (-1 where not recorded: past an early stop, or on a
        batched handle)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        res = np.full(iters + 1, np.nan)
        coef = np.full(2 * max(iters, 1), np.nan)
        nnz = np.full(iters + 1, -1, dtype=np.int64)
        hist = _Hist(res.ctypes.data, coef.ctypes.data, 0, 0, nnz.ctypes.data)
        rule = (SPAI_DROP_NONE if not drop else
                SPAI_DROP_TOPK_COL_DIAG if keep_diag else SPAI_DROP_TOPK_COL)
        rc = self.lib.spai_run(self.h, m, int(iters), rule, C.byref(hist))
        self._check(rc, "spai_run")
        return dict(status=rc, done=hist.iters_done, flags=hist.flags, resnorm=res,
                    coef=coef.reshape(-1, 2), nnz=nnz)

    def mr(self, iters, drop=True, keep_diag=False):
        return self.run("mr", iters, drop, keep_diag)

    def lomr(self, iters, drop=True, keep_diag=False):
        return self.run("lomr", iters, drop, keep_diag)

    def cg(self, iters, drop=True, keep_diag=False):
        return self.run("cg", iters, drop, keep_diag)

    def reset(self):
        self._check(self.lib.spai_reset(self.h), "spai_reset")

    def residual_norm(self) -> float:
        out = C.c_double()
        self._check(self.lib.spai_residual_norm(self.h, C.byref(out)), "spai_residual_norm")
        return out.value

    def nnz_M(self) -> int:
        out = C.c_int64()
        self._check(self.lib.spai_get_nnz(self.h, C.byref(out)), "spai_get_nnz")
        return out.value

    def get_M(self, out=None):
        """CSC triple (colptr int32[n+1], rowind int32[nnz], vals float64[nnz]) on the host;
        out: host arrays to fill (for example views of pinned memory), long enough."""
        nnz = C.c_int64()
        self._check(self.lib.spai_get_M(self.h, C.byref(nnz), None, None, None, 0), "spai_get_M")
        if out is not None:
            cp, ri, va = out
            if (len(cp) < self.n + 1 or len(ri) < nnz.value or len(va) < nnz.value
                    or cp.dtype != np.int32 or ri.dtype != np.int32 or va.dtype != np.float64):
                raise ValueError("get_M: out arrays too short or of the wrong dtype")
        else:
            cp = np.zeros(self.n + 1, dtype=np.int32)
            ri = np.zeros(max(nnz.value, 1), dtype=np.int32)
            va = np.zeros(max(nnz.value, 1), dtype=np.float64)
        self._check(self.lib.spai_get_M(self.h, C.byref(nnz), cp.ctypes.data, ri.ctypes.data,
                                        va.ctypes.data, 0), "spai_get_M")
        return cp, ri[:nnz.value], va[:nnz.value]

    def get_M_device(self, colptr, rowind, vals):
        """Fill device tensors (int32, int32, float64) with the CSC of M; returns nnz."""
        nnz = C.c_int64()
        self._check(self.lib.spai_get_M(self.h, C.byref(nnz), colptr.data_ptr(), rowind.data_ptr(),
                                        vals.data_ptr(), 1), "spai_get_M")
        return nnz.value

    def set_M(self, colptr, rowind, vals):
        cp, ri, va = _np(colptr, np.int32), _np(rowind, np.int32), _np(vals, np.float64)
        self._check(self.lib.spai_set_M(self.h, cp.ctypes.data, ri.ctypes.data, va.ctypes.data, 0),
                    "spai_set_M")

    def apply(self, x, y):
        """y = M x for FP64 CUDA tensors x, y of shape (n,) or (nrhs, n)."""
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        self._check(self.lib.spai_apply(self.h, x.data_ptr(), y.data_ptr(), nrhs, self.n),
                    "spai_apply")
        return y

    def pcg(self, b, x=None, rtol=1e-8, maxit=10000, precond=PREC_SPAI_SYM):
        """Vector PCG with x0 = 0; b/x numpy (host) or FP64 CUDA tensors (device)."""
        dev = hasattr(b, "data_ptr")
        if dev:
            if x is None:
                import torch
                x = torch.empty_like(b)
            pb, px = b.data_ptr(), x.data_ptr()
        else:
            b = _np(b, np.float64)
            x = np.zeros(self.n) if x is None else x
            pb, px = b.ctypes.data, x.ctypes.data
        it = C.c_int()
        rr = C.c_double()
        rc = self.lib.pcg_solve(self.h, pb, px, 1, float(rtol), int(maxit), int(precond),
                                1 if dev else 0, C.byref(it), C.byref(rr))
        self._check(rc, "pcg_solve")
        return dict(status=rc, iters=it.value, relres=rr.value, x=x)

    def _sizes(self):
        return [int(self.n)]

    def set_pcg_prec(self, prec):
        """Products inside PCG in "fp64" (default) or "mixed" (FP32 values,
        FP32 operand copies; FP64 vectors, dots and scalars)."""
        self._check(self.lib.spai_set_pcg_prec(self.h, SPAI_MIXED if prec == "mixed" else SPAI_FP64),
                    "spai_set_pcg_prec")

    def pcg_block(self, B, rtol=1e-8, maxit=10000, precond=PREC_SPAI_SYM, nrhs=None, x=None):
        """Block PCG: up to 32 independent recurrences per matrix of the handle.

        B: a list with one (nrhs, n_m) host array per matrix, or one flat FP64
        CUDA tensor in the library layout (matrix after matrix, vector after
        vector; give nrhs).  Returns dict(status, iters, statuses, relres, x),
        the per-recurrence arrays shaped (nmat, nrhs); x in the form of B.
        """
        sizes = self._sizes()
        dev = hasattr(B, "data_ptr")
        if dev:
            R = int(nrhs)
            if x is None:
                import torch
                x = torch.empty_like(B)
            pb, px = B.data_ptr(), x.data_ptr()
        else:
            R = int(np.asarray(B[0]).shape[0])
            flat = np.concatenate([_np(np.asarray(b).reshape(R, n), np.float64).ravel()
                                   for b, n in zip(B, sizes)])
            xf = np.zeros_like(flat)
            pb, px = flat.ctypes.data, xf.ctypes.data
        k = len(sizes)
        it = np.zeros(k * R, dtype=np.int32)
        st = np.zeros(k * R, dtype=np.int32)
        rr = np.zeros(k * R)
        rc = self.lib.pcg_solve_block(self.h, R, pb, px, float(rtol), int(maxit), int(precond),
                                      1 if dev else 0, it.ctypes.data, st.ctypes.data,
                                      rr.ctypes.data)
        self._check(rc, "pcg_solve_block")
        if not dev:
            x, o = [], 0
            for n in sizes:
                x.append(xf[o:o + R * n].reshape(R, n))
                o += R * n
        return dict(status=rc, iters=it.reshape(k, R), statuses=st.reshape(k, R),
                    relres=rr.reshape(k, R), x=x)

    def autotune(self, method, iters=10):
        """Pick the fastest launch shape for `method` (times `iters` iterations after
        `iters` untimed ones; resets M); returns ms per iteration."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        out = C.c_double()
        self._check(self.lib.spai_autotune(self.h, m, int(iters), C.byref(out)), "spai_autotune")
        return out.value

    def drop_global(self, m, which="M"):
        """Keep the m largest-|v| entries of M (or of P) over the whole matrix."""
        self._check(self.lib.spai_drop_global(self.h, 0 if which == "M" else 1, int(m)),
                    "spai_drop_global")

    def run_global(self, method, iters, m_dir, m_M):
        """MR, LOMR or CG (or their Pi forms) with global dropping inside every
        iteration (see spai_run_global)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        res = np.full(iters + 1, np.nan)
        coef = np.full(2 * max(iters, 1), np.nan)
        hist = _Hist(res.ctypes.data, coef.ctypes.data, 0, 0, None)
        rc = self.lib.spai_run_global(self.h, m, int(iters), int(m_dir), int(m_M), C.byref(hist))
        self._check(rc, "spai_run_global")
        return dict(status=rc, done=hist.iters_done, flags=hist.flags, resnorm=res,
                    coef=coef.reshape(-1, 2))

    def drop_heuristic(self, m):
        """Appendix A: symmetrise M, drop round-off entries, then by score to m entries."""
        self._check(self.lib.spai_drop_heuristic(self.h, int(m)), "spai_drop_heuristic")

    def fixed_pattern(self, k):
        """M := the best approximate inverse on supp(A^k) (column least squares)."""
        self._check(self.lib.spai_fixed_pattern(self.h, int(k)), "spai_fixed_pattern")

    def sym_spectrum(self, steps=200, v0=None, seed=0):
        """Lanczos on (M + M^T)/2 from v0 (default: standard normal draws from
        default_rng(seed)); returns dict(lmin, lmax, alpha, beta, steps)."""
        if v0 is None:
            v0 = np.random.default_rng(seed).standard_normal(int(self.n))
        v0 = _np(v0, np.float64)
        a = np.zeros(steps)
        b = np.zeros(steps)
        k = C.c_int()
        lo = C.c_double()
        hi = C.c_double()
        self._check(self.lib.spai_sym_lanczos(self.h, int(steps), v0.ctypes.data, a.ctypes.data,
                                              b.ctypes.data, C.byref(k), C.byref(lo), C.byref(hi)),
                    "spai_sym_lanczos")
        return dict(lmin=lo.value, lmax=hi.value, alpha=a[:k.value], beta=b[:k.value],
                    steps=k.value)

    def save_state(self) -> bytes:
        n = C.c_size_t()
        self._check(self.lib.spai_save_state(self.h, None, C.byref(n)), "spai_save_state")
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.spai_save_state(self.h, buf, C.byref(n)), "spai_save_state")
        return buf.raw[:n.value]

    def load_state(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        self._check(self.lib.spai_load_state(self.h, buf, len(data)), "spai_load_state")

    def set_timing(self, on=True):
        self._check(self.lib.spai_set_timing(self.h, int(bool(on))), "spai_set_timing")

    def stats(self):
        s = _Stats()
        self._check(self.lib.spai_get_stats(self.h, C.byref(s)), "spai_get_stats")
        return {k: getattr(s, k) for k, _ in _Stats._fields_}


class SpaiBatch(Spai):
    """Many SPD matrices solved together (block-diagonal, per-matrix coefficients).

    mats: list of (n, rowptr, colind, vals) host CSR triples.
    """

    def __init__(self, mats, prec="fp64", cap_factor=2.0, stream=None):
        self.lib = load()
        k = len(mats)
        self.nmat = k
        ns = np.array([m[0] for m in mats], dtype=np.int64)
        arrs = [(_np(m[1], np.int32), _np(m[2], np.int32), _np(m[3], np.float64)) for m in mats]
        nnz = np.array([len(a[2]) for a in arrs], dtype=np.int64)
        rps = (C.c_void_p * k)(*[a[0].ctypes.data for a in arrs])
        cis = (C.c_void_p * k)(*[a[1].ctypes.data for a in arrs])
        vas = (C.c_void_p * k)(*[a[2].ctypes.data for a in arrs])
        opts = _Opts(SPAI_MIXED if prec == "mixed" else SPAI_FP64, float(cap_factor))
        h = C.c_void_p()
        rc = self.lib.spai_create_batched(C.byref(h), k, ns.ctypes.data, nnz.ctypes.data, rps, cis,
                                          vas, C.byref(opts), _stream_ptr(stream))
        if rc != 0:
            raise SpaiError(rc, "spai_create_batched")
        self.h = h
        self.prec = prec
        self.ns = ns
        self.n = int(self._total_n())

    def _total_n(self):
        # padded block-diagonal size: each matrix rounded up to 256
        return int(sum((int(x) + 255) // 256 * 256 for x in self.ns))

    def run(self, method, iters, drop=True, keep_diag=False):
        r = super().run(method, iters, drop, keep_diag)
        res = np.full(self.nmat * (iters + 1), np.nan)
        done = np.zeros(self.nmat, dtype=np.int32)
        flags = np.zeros(self.nmat, dtype=np.int32)
        self._check(self.lib.spai_batch_history(self.h, res.ctypes.data, done.ctypes.data,
                                                flags.ctypes.data), "spai_batch_history")
        r["resnorm_each"] = res.reshape(self.nmat, iters + 1)
        r["done_each"] = done
        r["flags_each"] = flags
        return r

    def _sizes(self):
        return [int(x) for x in self.ns]

    def batch_info(self):
        """Sizes of the matrices of the batch (without padding)."""
        nm = C.c_int()
        ns = np.zeros(self.nmat, dtype=np.int64)
        self._check(self.lib.spai_batch_info(self.h, C.byref(nm), ns.ctypes.data),
                    "spai_batch_info")
        return [int(x) for x in ns[:nm.value]]

    def residual_norms(self):
        out = np.zeros(self.nmat)
        self._check(self.lib.spai_batch_residual_norms(self.h, out.ctypes.data),
                    "spai_batch_residual_norms")
        return out

    def get_M_of(self, m):
        nnz = C.c_int64()
        self._check(self.lib.spai_batch_get_M(self.h, int(m), C.byref(nnz), None, None, None),
                    "spai_batch_get_M")
        n = int(self.ns[m])
        cp = np.zeros(n + 1, dtype=np.int32)
        ri = np.zeros(max(nnz.value, 1), dtype=np.int32)
        va = np.zeros(max(nnz.value, 1), dtype=np.float64)
        self._check(self.lib.spai_batch_get_M(self.h, int(m), C.byref(nnz), cp.ctypes.data,
                                              ri.ctypes.data, va.ctypes.data), "spai_batch_get_M")
        return cp, ri[:nnz.value], va[:nnz.value]


class FixedPatternMR:
    """K fixed-pattern MR (or, method="lomr", LOMR) steps on supp(A) and the
    gradient of ||I - A M_K||_F^2 with respect to A's stored values (see
    spai_fpmr_* in include/spai.h)."""

    def __init__(self, n, rowptr, colind, K, prec="fp64", stream=None, method="mr"):
        self.lib = load()
        rp, ci = _np(rowptr, np.int32), _np(colind, np.int32)
        h = C.c_void_p()
        rc = self.lib.spai_fpmr_create(C.byref(h), int(n), len(ci), rp.ctypes.data, ci.ctypes.data,
                                       int(K), SPAI_MIXED if prec == "mixed" else SPAI_FP64,
                                       _stream_ptr(stream))
        if rc != 0:
            raise SpaiError(rc, "spai_fpmr_create")
        self.h, self.n, self.nnz, self.K = h, int(n), len(ci), int(K)
        if method != "mr":
            rc = self.lib.spai_fpmr_set_method(self.h, METHODS[method])
            if rc != 0:
                self.close()
                raise SpaiError(rc, "spai_fpmr_set_method")

    def _ptr(self, a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr(), 1 if a.is_cuda else 0
        return a.ctypes.data, 0

    def forward(self, vals) -> float:
        if not hasattr(vals, "data_ptr"):
            vals = _np(vals, np.float64)
        p, dev = self._ptr(vals)
        loss = C.c_double()
        rc = self.lib.spai_fpmr_forward(self.h, p, dev, C.byref(loss))
        if rc != 0:
            raise SpaiError(rc, "spai_fpmr_forward")
        return loss.value

    def backward(self, dloss=1.0, out=None):
        if out is None:
            out = np.zeros(self.nnz)
        p, dev = self._ptr(out)
        rc = self.lib.spai_fpmr_backward(self.h, float(dloss), p, dev)
        if rc != 0:
            raise SpaiError(rc, "spai_fpmr_backward")
        return out

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self.lib.spai_fpmr_info(self.h, C.byref(a), C.byref(b), C.byref(c))
        return dict(nnz_t=a.value, list_entries=b.value, launches=c.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.spai_fpmr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fpmr_loss(vals, fpmr):
    """||I - A M_K||_F^2 as a differentiable function of A's values (an FP64
    CUDA tensor in CSR order) through torch.autograd."""
    import torch

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v):
            loss = fpmr.forward(v.detach().contiguous())
            return torch.tensor(loss, dtype=torch.float64, device=v.device)

        @staticmethod
        def backward(ctx, g):
            out = torch.empty(fpmr.nnz, dtype=torch.float64, device=g.device)
            fpmr.backward(float(g.item()), out)
            return out

    return _F.apply(vals)
