"""CPU oracle for the SPAI methods (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It compiles ``spai_oracle.c`` with gcc
(``-O2 -ffp-contract=off``) into ``oracle/_build/liboracle.so`` and, with
``-fopenmp`` added, into ``oracle/_build/liboracle_omp.so`` (the loops over
columns and PCG rows shared among threads; the same bits as the serial
build), and wraps them with ctypes.  It imports nothing from the product
package.

Method definitions followed (Venkovic & Anzt): MR = Algorithm 1, CG =
Algorithm 3 (Def. 1, Prop. 2), LOMR = Algorithm 4 (Def. 2, Theorem 3), hard
thresholding = Sec. 6.1 Eq. (6.2) applied per column, explicit residual =
Sec. 6.2.  The C file's header lists every reading taken where the paper is
silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spai_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

MR, LOMR, CG = 0, 1, 2
MR_PI, LOMR_PI, CG_PI = 3, 4, 5  # Section 5's forms with Pi = diag(A)^{-1} (Algorithms 5, 8, 7)
METHODS = {"mr": MR, "lomr": LOMR, "cg": CG, "mr_pi": MR_PI, "lomr_pi": LOMR_PI, "cg_pi": CG_PI}
FLAG_CONVERGED, FLAG_FALLBACK, FLAG_NONFINITE = 1, 2, 4
DROP_NONE, DROP_TOPK, DROP_DIRECTIONS = 0, 1, 2


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library (idempotent); omp=True builds the
    OpenMP one."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if omp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    if omp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(omp: bool = False):
    with _lock:
        if omp in _libs:
            return _libs[omp]
        lib = C.CDLL(build(omp=omp))
        p_i32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        p_f64 = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.orc_new.restype = C.c_void_p
        lib.orc_new.argtypes = [C.c_int, p_i32, p_i32, p_f64, C.c_int, C.c_double]
        lib.orc_free.argtypes = [C.c_void_p]
        lib.orc_run.restype = C.c_int
        lib.orc_run.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, p_f64, p_f64, C.c_void_p,
                                C.POINTER(C.c_int)]
        lib.orc_set_keep_diag.argtypes = [C.c_void_p, C.c_int]
        lib.orc_nnz.restype = C.c_int64
        lib.orc_nnz.argtypes = [C.c_void_p, C.c_int]
        lib.orc_get.argtypes = [C.c_void_p, C.c_int, p_i32, p_i32, p_f64]
        lib.orc_set_M.restype = C.c_int
        lib.orc_set_M.argtypes = [C.c_void_p, p_i32, p_i32, p_f64]
        lib.orc_spgemm_count.restype = C.c_int64
        lib.orc_spgemm_count.argtypes = [C.c_void_p]
        lib.orc_residual_norm.restype = C.c_double
        lib.orc_residual_norm.argtypes = [C.c_void_p]
        lib.orc_column_residual.restype = C.c_int
        lib.orc_column_residual.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        lib.orc_product_column.restype = C.c_int
        lib.orc_product_column.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]
        lib.orc_drop_column.restype = C.c_int
        lib.orc_drop_column.argtypes = [C.c_int, p_i32, p_f64, C.c_int, C.c_int]
        lib.orc_fixsum.restype = C.c_double
        lib.orc_fixsum.argtypes = [p_f64, C.c_int64]
        lib.orc_pairwise.restype = C.c_double
        lib.orc_pairwise.argtypes = [p_f64, C.c_int64]
        lib.orc_pcg.restype = C.c_int
        lib.orc_pcg.argtypes = [C.c_int, p_i32, p_i32, p_f64, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, p_f64, C.c_double, C.c_int, p_f64,
                                C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int]
        lib.orc_lanczos.restype = C.c_int
        lib.orc_lanczos.argtypes = [C.c_int, p_i32, p_i32, p_f64, p_f64, C.c_int, p_f64, p_f64]
        _libs[omp] = lib
        return lib


def pairwise(t) -> float:
    """Balanced pairwise sum over t zero-padded to a power of two."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    return _load().orc_pairwise(t, len(t))


def fixsum(t) -> float:
    """Order-free sum used for column inner products (128-bit fixed point
    anchored at the largest term, rounded once)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    return _load().orc_fixsum(t, len(t))


class Oracle:
    """Sparse-iterate state (M, P, Z) for one SPD matrix A.

    ``mixed=True`` emulates the FP32-value / FP64-reduction arithmetic
    exactly; ``cap_factor`` sets cap_j = floor(f * nnz(A[:, j])) in [1, n].
    M starts at diag(A)^{-1}.  ``omp=True`` uses the OpenMP build (all
    threads OpenMP is given; the same results bit for bit).
    """

    def __init__(self, n, rowptr, colind, vals, mixed=False, cap_factor=2.0, omp=False):
        self.lib = _load(omp)
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.vals = np.ascontiguousarray(vals, dtype=np.float64)
        self.mixed = bool(mixed)
        self.h = self.lib.orc_new(self.n, self.rowptr, self.colind, self.vals, int(mixed),
                                  float(cap_factor))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_free(h)
            self.h = None

    def run(self, method, iters, drop=DROP_TOPK):
        """Returns dict(done, resnorm[0..iters], coef[iters][2], nnz[0..iters],
        flags); nnz[i] = nnz(M_i), the iterate whose residual resnorm[i] is
        (-1 past an early stop)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        res = np.full(iters + 1, np.nan)
        coef = np.full(2 * max(iters, 1), np.nan)
        nnz = np.full(iters + 1, -1, dtype=np.int64)
        flags = C.c_int(0)
        done = self.lib.orc_run(self.h, m, int(iters), int(drop), res, coef, nnz.ctypes.data,
                                C.byref(flags))
        return dict(done=done, resnorm=res, coef=coef.reshape(-1, 2), nnz=nnz, flags=flags.value)

    def set_keep_diag(self, on=True):
        """Every later per-column drop keeps the column's diagonal entry
        (Appendix A: the diagonal is never dropped); it counts toward cap_j."""
        self.lib.orc_set_keep_diag(self.h, 1 if on else 0)

    def get(self, which=0):
        """CSC (colptr, rowind, vals) of M (0), P (1) or Z (2)."""
        nnz = self.lib.orc_nnz(self.h, which)
        cp = np.zeros(self.n + 1, dtype=np.int32)
        ri = np.zeros(max(nnz, 1), dtype=np.int32)
        va = np.zeros(max(nnz, 1), dtype=np.float64)
        self.lib.orc_get(self.h, which, cp, ri, va)
        return cp, ri[:nnz], va[:nnz]

    def get_M(self):
        return self.get(0)

    def set_M(self, colptr, rowind, vals):
        self.lib.orc_set_M(self.h, np.ascontiguousarray(colptr, dtype=np.int32),
                           np.ascontiguousarray(rowind, dtype=np.int32),
                           np.ascontiguousarray(vals, dtype=np.float64))

    def spgemm_count(self):
        return self.lib.orc_spgemm_count(self.h)

    def residual_norm(self):
        return self.lib.orc_residual_norm(self.h)

    def product_column(self, rows, vals):
        """A x for one column x (sorted rows) with the method's arithmetic."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        L = self.lib.orc_product_column(self.h, len(rows), rows.ctypes.data, vals.ctypes.data,
                                        None, None)
        orow = np.zeros(max(L, 1), dtype=np.int32)
        oval = np.zeros(max(L, 1), dtype=np.float64)
        self.lib.orc_product_column(self.h, len(rows), rows.ctypes.data, vals.ctypes.data,
                                    orow.ctypes.data, oval.ctypes.data)
        return orow[:L], oval[:L]

    def column_residual(self, j):
        L = self.lib.orc_column_residual(self.h, int(j), None, None)
        rows = np.zeros(max(L, 1), dtype=np.int32)
        vals = np.zeros(max(L, 1), dtype=np.float64)
        self.lib.orc_column_residual(self.h, int(j), rows.ctypes.data, vals.ctypes.data)
        return rows[:L], vals[:L]


def drop_column(rows, vals, cap, keep_row=-1):
    """Hard-threshold one row-sorted column to ``cap`` entries (Sec. 6.1, per
    column); row ``keep_row`` (>= 0) is kept whenever present."""
    rows = np.array(rows, dtype=np.int32)
    vals = np.array(vals, dtype=np.float64)
    L = _load().orc_drop_column(len(rows), rows, vals, int(cap), int(keep_row))
    return rows[:L], vals[:L]


def pcg(n, rowptr, colind, vals, b, rtol=1e-8, maxit=10000, precond=0, M=None, mixed=False,
        omp=False):
    """Vector PCG with x0 = 0; precond 0 none, 1 Jacobi, 2 SPAI M, 3 symmetric
    part (M + M^T)/2 of the SPAI (M given as a CSC triple).  mixed: products
    with A and with M (or its symmetric part) in FP32 values (FP32 operand
    copy, FP32 fma chain); vectors, inner products and scalars in FP64.

    Returns dict(iters, status (0 conv / 1 maxit / 2 breakdown), relres, x).
    omp=True: the OpenMP build (the same results bit for bit).
    """
    lib = _load(omp)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64)
    st = C.c_int(0)
    rr = C.c_double(0.0)
    keep = []
    if precond in (2, 3):
        cp, ri, mv = (np.ascontiguousarray(M[0], dtype=np.int32),
                      np.ascontiguousarray(M[1], dtype=np.int32),
                      np.ascontiguousarray(M[2], dtype=np.float64))
        keep = [cp, ri, mv]
        args = (cp.ctypes.data, ri.ctypes.data, mv.ctypes.data)
    else:
        args = (None, None, None)
    it = lib.orc_pcg(int(n), rowptr, colind, vals, int(precond), *args, b, float(rtol), int(maxit),
                     x, C.byref(st), C.byref(rr), 1 if mixed else 0)
    del keep
    return dict(iters=it, status=st.value, relres=rr.value, x=x)


def lanczos(n, M, v0, steps):
    """Lanczos on the symmetric part (M + M^T)/2 of M (CSC triple) from v0:
    returns dict(alpha, beta, steps, lmin, lmax), the extremal eigenvalues of
    the tridiagonal T from scipy's tridiagonal eigensolver."""
    from scipy.linalg import eigvalsh_tridiagonal
    lib = _load()
    cp, ri, mv = (np.ascontiguousarray(M[0], dtype=np.int32), np.ascontiguousarray(M[1], dtype=np.int32),
                  np.ascontiguousarray(M[2], dtype=np.float64))
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    a = np.zeros(max(steps, 1))
    b = np.zeros(max(steps, 1))
    k = lib.orc_lanczos(int(n), cp, ri, mv, v0, int(steps), a, b)
    ev = eigvalsh_tridiagonal(a[:k], b[:k - 1]) if k > 1 else a[:k]
    return dict(alpha=a[:k], beta=b[:k], steps=k, lmin=float(ev[0]), lmax=float(ev[-1]))


def pattern_power(n, rowptr, colind, k):
    """supp(A^k e_j) for every column j (sorted row lists); A's pattern is
    symmetric, so column j's neighbours are row j's columns."""
    pats = []
    for j in range(n):
        seen = {j}
        front = [j]
        for _ in range(k):
            nxt = []
            for u in front:
                for c in colind[rowptr[u]:rowptr[u + 1]]:
                    c = int(c)
                    if c not in seen:
                        seen.add(c)
                        nxt.append(c)
            front = nxt
        pats.append(sorted(seen))
    return pats


def fixed_pattern_spai(n, rowptr, colind, vals, k):
    """The best approximate inverse on a prescribed pattern (the paper's
    Exp. 09 / Figs. 1-2): column j of M minimises ||e_j - A m_j||_2 over
    supp(m_j) = supp(A^k e_j), solved as a dense least-squares problem on
    the rows A touches.  Returns M as a CSC triple."""
    A = np.zeros((n, n))
    for i in range(n):
        A[i, colind[rowptr[i]:rowptr[i + 1]]] = vals[rowptr[i]:rowptr[i + 1]]
    pats = pattern_power(n, rowptr, colind, k)
    cp = [0]
    ri, va = [], []
    for j, J in enumerate(pats):
        B = A[:, J]
        rows = np.nonzero(np.any(B != 0.0, axis=1))[0]
        e = (rows == j).astype(np.float64)
        m = np.linalg.lstsq(B[rows], e, rcond=None)[0]
        ri.extend(J)
        va.extend(m.tolist())
        cp.append(len(ri))
    return (np.array(cp, dtype=np.int32), np.array(ri, dtype=np.int32), np.array(va))
