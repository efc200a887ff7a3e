"""Seeded synthetic SPD operators and right-hand sides.

This module is the only code shared by the CPU oracle tests and the CUDA
path.  It builds input matrices and vectors and holds none of the SPAI
method's arithmetic.  Every generator returns a CSR triple
``(rowptr int32, colind int32, vals float64)`` with rows sorted by column
index and an exactly symmetric value array, plus ``n``.

The paper's test matrices (SuiteSparse and the authors' own collection,
Section 7, Table 3) are not available here; these stencil operators stand
in for them.  They are SPD, with n from 1e3 to 1e6 and 5 to 9 nonzeros per
row, which brackets the paper's nnz/n range at its lower end.

Recipes
-------
* ``laplacian_2d_5pt(N)``: stencil [-1,-1,4,-1,-1] on an N x N grid of
  interior nodes, Dirichlet boundary eliminated, no h^2 scaling.
* ``varcoef_3d_7pt(N, sigma, ell, seed)``: node permeability kappa = exp(g)
  on an (N+2)^3 grid that includes the Dirichlet boundary layer; g is a
  stationary Gaussian field with covariance sigma^2 exp(-r^2 / (2 ell^2))
  (white noise from ``default_rng(seed)`` convolved by FFT with a Gaussian
  of std ell/sqrt(2) on a periodic box padded by ceil(3 ell) per side, then
  shifted and scaled to empirical mean 0 and std sigma).  Each grid edge
  carries the harmonic mean 2 k_a k_b / (k_a + k_b) of its end nodes; the
  diagonal is the sum of all incident edge coefficients, including edges to
  boundary nodes; off-diagonals are minus the edge coefficient.
* ``varcoef_2d_5pt``: the same construction in two dimensions.
* ``aniso_2d_9pt(N, eps, theta)``: diffusion tensor R(theta) diag(1, eps)
  R(theta)^T discretised with the 9-point stencil (centre 2a+2c, E/W -a,
  N/S -c, NE/SW -b/2, NW/SE +b/2) where a = cos^2 + eps sin^2,
  c = sin^2 + eps cos^2, b = (1 - eps) sin cos.  b^2 < a c makes it SPD.
* ``rhs_uniform(n, seed)``: ``default_rng(seed).uniform(-1, 1, n)``.
"""
from __future__ import annotations

import math

import numpy as np


def _assemble(n: int, offsets, coef_cols):
    """Assemble CSR from per-offset value columns.

    ``offsets`` must be sorted ascending (so rows come out column-sorted);
    ``coef_cols[t]`` is a float64 array of length n holding the entry of each
    row at column ``row + offsets[t]`` or NaN where that entry is absent.
    """
    vals = np.stack(coef_cols, axis=1)              # (n, W)
    rows = np.arange(n, dtype=np.int64)[:, None]
    cols = rows + np.asarray(offsets, dtype=np.int64)[None, :]
    mask = ~np.isnan(vals)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[mask].astype(np.int32)
    v = vals[mask].astype(np.float64)
    return rowptr.astype(np.int32), colind, v


def laplacian_2d_5pt(N: int):
    n = N * N
    idx = np.arange(n)
    x = idx % N
    y = idx // N
    nan = np.full(n, np.nan)
    south = np.where(y > 0, -1.0, nan)
    west = np.where(x > 0, -1.0, nan)
    east = np.where(x < N - 1, -1.0, nan)
    north = np.where(y < N - 1, -1.0, nan)
    centre = np.full(n, 4.0)
    rp, ci, v = _assemble(n, [-N, -1, 0, 1, N], [south, west, centre, east, north])
    return n, rp, ci, v


def laplacian_1d(n: int):
    nan = np.full(n, np.nan)
    idx = np.arange(n)
    left = np.where(idx > 0, -1.0, nan)
    right = np.where(idx < n - 1, -1.0, nan)
    rp, ci, v = _assemble(n, [-1, 0, 1], [left, np.full(n, 2.0), right])
    return n, rp, ci, v


def gaussian_field(shape, sigma: float, ell: float, seed: int) -> np.ndarray:
    """Stationary Gaussian field, squared-exponential covariance (see module doc)."""
    pad = int(math.ceil(3.0 * ell))
    big = tuple(s + 2 * pad for s in shape)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(big)
    s = ell / math.sqrt(2.0)
    freqs = [np.fft.fftfreq(m) for m in big]
    # Fourier transform of a unit-mass Gaussian kernel of std s (grid units)
    k2 = np.zeros(big)
    for ax, f in enumerate(freqs):
        sh = [1] * len(big)
        sh[ax] = -1
        k2 = k2 + (f.reshape(sh) ** 2)
    kern_hat = np.exp(-2.0 * (math.pi ** 2) * (s ** 2) * k2)
    g = np.fft.ifftn(np.fft.fftn(w) * kern_hat).real
    sl = tuple(slice(pad, pad + m) for m in shape)
    g = g[sl]
    g = g - g.mean()
    g = g * (sigma / g.std())
    return g


def _harm(a, b):
    return 2.0 * a * b / (a + b)


def varcoef_3d_7pt(N: int, sigma: float = 1.5, ell: float = 8.0, seed: int = 0):
    kap = np.exp(gaussian_field((N + 2, N + 2, N + 2), sigma, ell, seed))  # [z, y, x]
    c = kap[1:-1, 1:-1, 1:-1]
    ex_p = _harm(c, kap[1:-1, 1:-1, 2:])
    ex_m = _harm(c, kap[1:-1, 1:-1, :-2])
    ey_p = _harm(c, kap[1:-1, 2:, 1:-1])
    ey_m = _harm(c, kap[1:-1, :-2, 1:-1])
    ez_p = _harm(c, kap[2:, 1:-1, 1:-1])
    ez_m = _harm(c, kap[:-2, 1:-1, 1:-1])
    diag = (ex_p + ex_m + ey_p + ey_m + ez_p + ez_m).ravel()
    n = N ** 3
    idx = np.arange(n)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    nan = np.full(n, np.nan)
    zm = np.where(z > 0, -ez_m.ravel(), nan)
    ym = np.where(y > 0, -ey_m.ravel(), nan)
    xm = np.where(x > 0, -ex_m.ravel(), nan)
    xp = np.where(x < N - 1, -ex_p.ravel(), nan)
    yp = np.where(y < N - 1, -ey_p.ravel(), nan)
    zp = np.where(z < N - 1, -ez_p.ravel(), nan)
    rp, ci, v = _assemble(n, [-N * N, -N, -1, 0, 1, N, N * N], [zm, ym, xm, diag, xp, yp, zp])
    return n, rp, ci, v


def varcoef_2d_5pt(N: int, sigma: float = 1.5, ell: float = 8.0, seed: int = 0):
    kap = np.exp(gaussian_field((N + 2, N + 2), sigma, ell, seed))  # [y, x]
    c = kap[1:-1, 1:-1]
    ex_p = _harm(c, kap[1:-1, 2:])
    ex_m = _harm(c, kap[1:-1, :-2])
    ey_p = _harm(c, kap[2:, 1:-1])
    ey_m = _harm(c, kap[:-2, 1:-1])
    diag = (ex_p + ex_m + ey_p + ey_m).ravel()
    n = N * N
    idx = np.arange(n)
    x = idx % N
    y = idx // N
    nan = np.full(n, np.nan)
    ym = np.where(y > 0, -ey_m.ravel(), nan)
    xm = np.where(x > 0, -ex_m.ravel(), nan)
    xp = np.where(x < N - 1, -ex_p.ravel(), nan)
    yp = np.where(y < N - 1, -ey_p.ravel(), nan)
    rp, ci, v = _assemble(n, [-N, -1, 0, 1, N], [ym, xm, diag, xp, yp])
    return n, rp, ci, v


def varcoef_grid(dims, sigma: float = 1.5, ell: float = 8.0, seed: int = 0):
    """Variable-coefficient diffusion on a rectangular 2-D (ny, nx) or 3-D
    (nz, ny, nx) grid, same construction as varcoef_3d_7pt / varcoef_2d_5pt."""
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    kap = np.exp(gaussian_field(tuple(m + 2 for m in dims), sigma, ell, seed))
    inner = tuple(slice(1, -1) for _ in range(d))
    c = kap[inner]
    n = int(np.prod(dims))
    idx = np.arange(n).reshape(dims)
    strides = [int(np.prod(dims[a + 1:])) for a in range(d)]
    nan = np.full(n, np.nan)
    cols_m, cols_p, diag = [], [], np.zeros(dims)
    for a in range(d):
        sl_p = list(inner)
        sl_m = list(inner)
        sl_p[a] = slice(2, None)
        sl_m[a] = slice(None, -2)
        ep = _harm(c, kap[tuple(sl_p)])
        em = _harm(c, kap[tuple(sl_m)])
        diag = diag + ep + em
        coord = (idx // strides[a]) % dims[a]
        cols_m.append(np.where(coord.ravel() > 0, -em.ravel(), nan))
        cols_p.append(np.where(coord.ravel() < dims[a] - 1, -ep.ravel(), nan))
    offsets = [-strides[a] for a in range(d)] + [0] + [strides[a] for a in reversed(range(d))]
    cols = cols_m + [diag.ravel()] + list(reversed(cols_p))
    order = np.argsort(offsets)
    rp, ci, v = _assemble(n, [offsets[k] for k in order], [cols[k] for k in order])
    return n, rp, ci, v


def batch_uneven(count: int = 64, nmin: float = 1e3, nmax: float = 6.4e4, seed: int = 0,
                 sigma: float = 1.5, ell: float = 8.0):
    """Batch of variable-coefficient operators with n log-uniform in
    [nmin, nmax] (drawn from default_rng(seed)), alternating 2-D 5-point and
    3-D 7-point grids, matrix k using field seed 1000 + k."""
    rng = np.random.default_rng(seed)
    targets = np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))
    mats = []
    for k, t in enumerate(targets):
        if k % 2 == 0:
            nx = max(2, int(round(math.sqrt(t))))
            ny = max(2, int(round(t / nx)))
            dims = (ny, nx)
        else:
            nx = max(2, int(round(t ** (1.0 / 3.0))))
            ny = nx
            nz = max(2, int(round(t / (nx * ny))))
            dims = (nz, ny, nx)
        mats.append(varcoef_grid(dims, sigma, ell, 1000 + k))
    return mats


def aniso_2d_9pt(N: int, eps: float = 1e-3, theta: float = math.pi / 6):
    cs, sn = math.cos(theta), math.sin(theta)
    a = cs * cs + eps * sn * sn
    c = sn * sn + eps * cs * cs
    b = (1.0 - eps) * sn * cs
    n = N * N
    idx = np.arange(n)
    x = idx % N
    y = idx // N
    nan = np.full(n, np.nan)
    has_w, has_e = x > 0, x < N - 1
    has_s, has_n = y > 0, y < N - 1
    sw = np.where(has_s & has_w, -b / 2, nan)
    s_ = np.where(has_s, -c, nan)
    se = np.where(has_s & has_e, b / 2, nan)
    w_ = np.where(has_w, -a, nan)
    ce = np.full(n, 2 * a + 2 * c)
    e_ = np.where(has_e, -a, nan)
    nw = np.where(has_n & has_w, b / 2, nan)
    n_ = np.where(has_n, -c, nan)
    ne = np.where(has_n & has_e, -b / 2, nan)
    rp, ci, v = _assemble(n, [-N - 1, -N, -N + 1, -1, 0, 1, N - 1, N, N + 1],
                          [sw, s_, se, w_, ce, e_, nw, n_, ne])
    return n, rp, ci, v


def random_spd_banded(n: int, bw: int, seed: int, diag_shift: float = 0.5):
    """Small random SPD matrix A = L L^T + shift I with banded lower factor L.

    Used only by tests (tiny n): L has unit-ish diagonal and uniform(0,1)
    off-diagonals within the band, in the spirit of the paper's custom
    A = L L^T matrices (Section 7).
    """
    rng = np.random.default_rng(seed)
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = rng.uniform(0.5, 1.5)
        for j in range(max(0, i - bw), i):
            L[i, j] = rng.uniform(0.0, 1.0) * 0.5
    A = L @ L.T + diag_shift * np.eye(n)
    A = 0.5 * (A + A.T)
    return dense_to_csr(A)


def dense_to_csr(A: np.ndarray):
    n = A.shape[0]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        cols.append(nz)
        vals.append(A[i, nz])
        rowptr[i + 1] = rowptr[i] + len(nz)
    return n, rowptr, np.concatenate(cols).astype(np.int32), np.concatenate(vals).astype(np.float64)


def csr_to_dense(n, rowptr, colind, vals) -> np.ndarray:
    A = np.zeros((n, n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            A[i, colind[e]] = vals[e]
    return A


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


# Named workloads with the sizes the benchmark configurations use.
WORKLOADS = {
    "lap2d_32": dict(gen="laplacian_2d_5pt", args=dict(N=32), cap_factor=2.0, iters=20),
    "varcoef3d_64": dict(gen="varcoef_3d_7pt", args=dict(N=64, sigma=1.5, ell=8.0, seed=0),
                         cap_factor=3.0, iters=50),
    "aniso2d_1024": dict(gen="aniso_2d_9pt", args=dict(N=1024, eps=1e-3, theta=math.pi / 6),
                         cap_factor=2.0, iters=100),
}


def make(name: str):
    w = WORKLOADS[name]
    return globals()[w["gen"]](**w["args"])
