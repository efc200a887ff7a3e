"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a dense
brute-force minimiser, a closed form, a theorem of the paper, scipy, or a
fixture printed in the paper.  No GPU.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_2511_09753_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_from_csc(n, cp, ri, va):
    M = np.zeros((n, n))
    for j in range(n):
        M[ri[cp[j]:cp[j + 1]], j] = va[cp[j]:cp[j + 1]]
    return M


def frob(X, Y):
    return float(np.sum(X * Y))


def tiny_spd(n=10, seed=3):
    return I.random_spd_banded(n, 2, seed)


def lap2d(N):
    return I.laplacian_2d_5pt(N)


# ------------------------------------------------------------- summation

def test_pairwise_exact_on_integers_and_close_to_fsum():
    rng = np.random.default_rng(0)
    t = rng.integers(-1000, 1000, 777).astype(np.float64)
    assert O.pairwise(t) == float(t.sum())
    x = rng.standard_normal(1000) * np.exp(rng.uniform(-20, 20, 1000))
    exact = math.fsum(x)
    bound = 10 * np.finfo(float).eps * np.sum(np.abs(x))  # log2(1024) levels
    assert abs(O.pairwise(x) - exact) <= bound
    assert O.pairwise([]) == 0.0
    assert O.pairwise([3.5]) == 3.5


def test_pairwise_tree_shape():
    # (a+b)+(c+0) differs from ((a+b)+c) for these values: pins the tree shape
    a, b, c = 1.0, 1e-16, 1e-16
    assert O.pairwise([a, b, c]) == (a + b) + (c + 0.0)
    assert O.pairwise([1e16, 1.0, -1e16, 1.0]) == (1e16 + 1.0) + (-1e16 + 1.0)


def test_fixsum_is_the_correctly_rounded_exact_sum():
    # within 2^58 of the largest term nothing is truncated, so the result is
    # the exact sum rounded once -- which math.fsum also computes
    rng = np.random.default_rng(2)
    for trial in range(300):
        L = int(rng.integers(1, 400))
        x = rng.standard_normal(L) * np.exp2(rng.integers(-50, 0, L))
        if trial % 3 == 0:
            x = np.concatenate([x, -x[: L // 2]])  # heavy cancellation
        assert O.fixsum(x) == math.fsum(x)
        assert O.fixsum(rng.permutation(x)) == O.fixsum(x)     # order free
    assert O.fixsum([]) == 0.0
    assert O.fixsum([1.0, -1.0]) == 0.0
    assert O.fixsum([2.0 ** 1000, 1.0]) == 2.0 ** 1000          # tiny term truncated
    big = [1e300, -1e300, 3.0]
    assert O.fixsum(big) == 0.0                                  # 3 is below 2^(E-110)


# ------------------------------------------------------------- dropping

def brute_drop(rows, vals, cap):
    if len(rows) <= cap:
        return list(rows), list(vals)
    order = sorted(range(len(rows)), key=lambda e: (-abs(vals[e]), rows[e]))[:cap]
    order.sort(key=lambda e: rows[e])
    return [rows[e] for e in order], [vals[e] for e in order]


def test_drop_matches_brute_force_with_ties():
    rng = np.random.default_rng(1)
    for trial in range(200):
        L = int(rng.integers(1, 60))
        rows = np.sort(rng.choice(1000, L, replace=False))
        vals = rng.choice([-0.5, -0.25, 0.25, 0.5, 1.0, 3.0], L) * rng.choice([1.0, 1.0, 0.999], L)
        cap = int(rng.integers(1, 40))
        r1, v1 = O.drop_column(rows, vals, cap)
        r2, v2 = brute_drop(list(rows), list(vals), cap)
        assert list(r1) == r2 and list(v1) == v2


def test_drop_hand_made_tie():
    # four equal magnitudes (the 5-point Laplacian's R_0 pattern): keep the
    # largest, then the smallest row indices among the ties
    r, v = O.drop_column([1, 3, 5, 7, 9], [0.25, -0.25, 0.5, 0.25, -0.25], 3)
    assert list(r) == [1, 3, 5] and list(v) == [0.25, -0.25, 0.5]


# ------------------------------------------------ SpGEMM / residual vs scipy

def test_column_residual_matches_scipy():
    n, rp, ci, v = I.varcoef_3d_7pt(8, seed=5)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    o.run("lomr", 3)
    cp, ri, va = o.get_M()
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    M = sp.csc_matrix((va, ri, cp), shape=(n, n))
    R = (sp.identity(n) - A @ M).tocsc()
    R.eliminate_zeros()
    for j in range(0, n, 7):
        rows, vals = o.column_residual(j)
        col = R[:, j].toarray().ravel()
        nz = np.nonzero(col)[0]
        assert set(rows) <= set(nz) | set(rows)
        np.testing.assert_allclose(vals, col[rows], rtol=1e-13, atol=1e-15)
        # every structurally produced nonzero of scipy is in the oracle's column
        big = nz[np.abs(col[nz]) > 1e-14]
        assert set(big) <= set(rows)


# ---------------------------------------------- MR: line minimiser (Eq. 2.6)

def test_mr_step_is_exact_line_minimiser():
    n, rp, ci, v = tiny_spd(10)
    A = I.csr_to_dense(n, rp, ci, v)
    for drop, capf in [(O.DROP_NONE, 1e9), (O.DROP_DIRECTIONS, 1.0)]:
        o = O.Oracle(n, rp, ci, v, cap_factor=capf)
        M0 = dense_from_csc(n, *o.get_M())
        R0 = np.eye(n) - A @ M0
        if drop == O.DROP_NONE:
            P = R0
        else:  # brute-force per-column drop of R0 to cap_j = nnz(A[:, j])
            P = np.zeros_like(R0)
            for j in range(n):
                nz = np.nonzero(R0[:, j])[0]
                rr, vv = brute_drop(list(nz), list(R0[nz, j]), int(np.count_nonzero(A[:, j])))
                P[rr, j] = vv
        AP = A @ P
        alpha = np.linalg.lstsq(AP.reshape(-1, 1), R0.reshape(-1), rcond=None)[0][0]
        o.run("mr", 1, drop=drop)
        M1 = dense_from_csc(n, *o.get_M())
        np.testing.assert_allclose(M1, M0 + alpha * P, rtol=0, atol=1e-13)


# --------------------------------------- LOMR: 2-D minimiser (Thm 3, Eq. 4.7)

def test_lomr_step_is_exact_2d_minimiser_and_beats_mr():
    n, rp, ci, v = tiny_spd(9, seed=7)
    A = I.csr_to_dense(n, rp, ci, v)
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    o.run("lomr", 2, drop=O.DROP_NONE)
    for _ in range(4):
        M1 = dense_from_csc(n, *o.get_M())
        Pm = dense_from_csc(n, *o.get(1))  # P_{i-1}
        R1 = np.eye(n) - A @ M1
        B = np.stack([(A @ R1).ravel(), (A @ Pm).ravel()], axis=1)
        d, g = np.linalg.lstsq(B, R1.ravel(), rcond=None)[0]
        expect = M1 + d * R1 + g * Pm
        # one-dimensional MR step from the same iterate
        AR = A @ R1
        a = frob(R1, AR) / frob(AR, AR)
        mr_norm = np.linalg.norm(np.eye(n) - A @ (M1 + a * R1))
        r = o.run("lomr", 1, drop=O.DROP_NONE)
        M2 = dense_from_csc(n, *o.get_M())
        np.testing.assert_allclose(M2, expect, rtol=0, atol=1e-12)
        lomr_norm = np.linalg.norm(np.eye(n) - A @ M2)
        assert lomr_norm <= mr_norm * (1 + 1e-12)  # Eq. (4.3)
        assert r["resnorm"][1] <= r["resnorm"][0] * (1 + 1e-12)


# ------------------------------------ MR: norm identity and rate (Theorem 1)

def test_mr_norm_identity_and_rate_bound():
    N = 6
    n, rp, ci, v = lap2d(N)
    A = I.csr_to_dense(n, rp, ci, v)
    lam_min = min(4 - 2 * math.cos(j * math.pi / (N + 1)) - 2 * math.cos(k * math.pi / (N + 1))
                  for j in range(1, N + 1) for k in range(1, N + 1))
    assert abs(lam_min - np.linalg.eigvalsh(A)[0]) < 1e-12
    C = math.sqrt(1 - lam_min ** 2 / float(np.sum(v * v)))  # tr(A^2) = sum a_ij^2
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    prev = None
    for i in range(25):
        M = dense_from_csc(n, *o.get_M())
        R = np.eye(n) - A @ M
        r = o.run("mr", 1, drop=O.DROP_NONE)
        nr0, nr1 = r["resnorm"][0], r["resnorm"][1]
        assert abs(nr0 - np.linalg.norm(R)) <= 1e-12 * nr0
        alpha = r["coef"][0, 0]
        # ||R_{i+1}||^2 = ||R_i||^2 - alpha_i (A R_i, R_i)
        np.testing.assert_allclose(nr1 ** 2, nr0 ** 2 - alpha * frob(A @ R, R), rtol=1e-11)
        assert nr1 <= C * nr0 * (1 + 1e-12)
        if prev is not None:
            assert nr0 <= prev * (1 + 1e-14)
        prev = nr1


def test_mr_rate_bound_random_spd():
    n, rp, ci, v = tiny_spd(12, seed=11)
    A = I.csr_to_dense(n, rp, ci, v)
    lam = np.linalg.eigvalsh(A)
    C = math.sqrt(1 - lam[0] ** 2 / np.trace(A @ A))
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    r = o.run("mr", 40, drop=O.DROP_NONE)
    res = r["resnorm"]
    assert np.all(res[1:] <= C * res[:-1] * (1 + 1e-12))


# ----------------------------- Pi-preconditioned forms (Algorithms 5, 7, 8)

@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_pi_forms_reduce_to_plain_forms_on_power_of_two_diagonals(method, mixed):
    """With Pi = diag(A)^{-1} = I / 2^k every Pi scaling is exact, so Z = Pi R
    ranks, drops and combines like R, the weighted inner products are the
    plain ones scaled by powers of two, and the iterates are bitwise those of
    the plain method; step coefficients carry the factor 2^k where the
    algebra says (MR and CG alpha, LOMR delta)."""
    for (n, rp, ci, v), scale in ((lap2d(12), 4.0), (I.laplacian_1d(50), 2.0)):
        plain = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=2.0)
        pre = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=2.0)
        a = plain.run(method, 7)
        b = pre.run(method + "_pi", 7)
        assert a["done"] == b["done"] == 7
        assert np.array_equal(a["resnorm"], b["resnorm"])
        for x, y in zip(plain.get_M(), pre.get_M()):
            assert np.array_equal(x, y)
        np.testing.assert_array_equal(b["coef"][:, 0], scale * a["coef"][:, 0])
        np.testing.assert_array_equal(b["coef"][:, 1], a["coef"][:, 1])


def _pi_dense(A):
    return np.diag(1.0 / np.diag(A))


def test_pi_mr_step_is_the_weighted_line_minimiser():
    """Algorithm 5, no dropping: alpha minimises (R - a A Z, Pi (R - a A Z))
    over a, with Z = Pi R; the Pi-weighted residual never grows."""
    n, rp, ci, v = I.varcoef_grid((4, 5), seed=9)
    A = I.csr_to_dense(n, rp, ci, v)
    Pi = _pi_dense(A)
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    prev = None
    for _ in range(6):
        M = dense_from_csc(n, *o.get_M())
        R = np.eye(n) - A @ M
        Z = Pi @ R
        AZ = A @ Z
        alpha = frob(AZ, Pi @ R) / frob(AZ, Pi @ AZ)
        o.run("mr_pi", 1, drop=O.DROP_NONE)
        M1 = dense_from_csc(n, *o.get_M())
        np.testing.assert_allclose(M1, M + alpha * Z, rtol=0, atol=1e-13)
        R1 = np.eye(n) - A @ M1
        w = frob(R1, Pi @ R1)
        if prev is not None:
            assert w <= prev * (1 + 1e-12)
        prev = w


def test_pi_lomr_step_is_the_weighted_2d_minimiser():
    """Algorithm 8, no dropping: (delta, gamma) minimise the Pi-weighted
    norm of R - d A Z - g A P_{i-1} (its 2x2 normal equations)."""
    n, rp, ci, v = I.varcoef_grid((3, 4), seed=5)
    A = I.csr_to_dense(n, rp, ci, v)
    Pi = _pi_dense(A)
    W = np.sqrt(np.diag(Pi))[:, None]
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    o.run("lomr_pi", 2, drop=O.DROP_NONE)
    for _ in range(4):
        M1 = dense_from_csc(n, *o.get_M())
        Pm = dense_from_csc(n, *o.get(1))
        R1 = np.eye(n) - A @ M1
        Z = Pi @ R1
        B = np.stack([(W * (A @ Z)).ravel(), (W * (A @ Pm)).ravel()], axis=1)
        d, g = np.linalg.lstsq(B, (W * R1).ravel(), rcond=None)[0]
        o.run("lomr_pi", 1, drop=O.DROP_NONE)
        M2 = dense_from_csc(n, *o.get_M())
        np.testing.assert_allclose(M2, M1 + d * Z + g * Pm, rtol=0, atol=1e-12)


def test_pi_cg_orthogonality():
    """Algorithm 7, no dropping: (R_i, Pi R_j) = 0 and (P_i, A P_j) = 0 for
    i != j (the preconditioned counterparts of Eqs. 3.4 and 3.6)."""
    n, rp, ci, v = I.varcoef_grid((3, 4), seed=2)
    A = I.csr_to_dense(n, rp, ci, v)
    Pi = _pi_dense(A)
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    Rs, Ps = [], []
    Rs.append(np.eye(n) - A @ dense_from_csc(n, *o.get_M()))
    o.run("cg_pi", 0, drop=O.DROP_NONE)
    Ps.append(dense_from_csc(n, *o.get(1)))
    np.testing.assert_allclose(Ps[0], Pi @ Rs[0], rtol=0, atol=1e-15)
    for _ in range(5):
        o.run("cg_pi", 1, drop=O.DROP_NONE)
        Rs.append(np.eye(n) - A @ dense_from_csc(n, *o.get_M()))
        Ps.append(dense_from_csc(n, *o.get(1)))
    scale = frob(Rs[0], Pi @ Rs[0])
    for i in range(1, len(Rs)):
        for j in range(i):
            assert abs(frob(Rs[i], Pi @ Rs[j])) <= 1e-10 * scale
            assert abs(frob(Ps[i], A @ Ps[j])) <= 1e-9 * scale * 10


# ------------------------------------------- CG: Prop. 2 and Theorem 5

def test_cg_orthogonality():
    n, rp, ci, v = tiny_spd(10, seed=5)
    A = I.csr_to_dense(n, rp, ci, v)
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    Rs, Ps = [], []
    M = dense_from_csc(n, *o.get_M())
    Rs.append(np.eye(n) - A @ M)
    o.run("cg", 0, drop=O.DROP_NONE)
    Ps.append(dense_from_csc(n, *o.get(1)))
    for i in range(5):
        o.run("cg", 1, drop=O.DROP_NONE)
        M = dense_from_csc(n, *o.get_M())
        Rs.append(np.eye(n) - A @ M)
        Ps.append(dense_from_csc(n, *o.get(1)))
    scale = np.linalg.norm(Rs[0]) ** 2
    for i in range(1, len(Rs)):
        for j in range(i):
            assert abs(frob(Rs[i], Rs[j])) <= 1e-10 * scale          # Eq. (3.4)
            assert abs(frob(Rs[i], Ps[j])) <= 1e-10 * scale          # Eq. (3.5)
            assert abs(frob(Ps[i], A @ Ps[j])) <= 1e-9 * scale * 10  # Eq. (3.6)


def test_cg_finite_termination_distinct_eigenvalues():
    rng = np.random.default_rng(4)
    n = 9
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.array([1.0, 1.0, 1.0, 3.0, 3.0, 3.0, 7.0, 7.0, 7.0])
    A = Q @ np.diag(lam) @ Q.T
    A = 0.5 * (A + A.T)
    n, rp, ci, v = I.dense_to_csr(A)
    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    r = o.run("cg", 3, drop=O.DROP_NONE)
    M = dense_from_csc(n, *o.get_M())
    assert np.abs(M - np.linalg.inv(A)).max() < 1e-10                 # Theorem 5
    assert r["resnorm"][3] < 1e-10 * r["resnorm"][0]


def test_cg_error_bound():
    n, rp, ci, v = lap2d(5)
    A = I.csr_to_dense(n, rp, ci, v)
    Ainv = np.linalg.inv(A)
    lam = np.linalg.eigvalsh(A)
    kap = lam[-1] / lam[0]
    q = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)

    def anorm(E):
        return math.sqrt(max(np.trace(E.T @ A @ E), 0.0))

    o = O.Oracle(n, rp, ci, v, cap_factor=1e9)
    e0 = anorm(Ainv - dense_from_csc(n, *o.get_M()))
    for i in range(1, 12):
        o.run("cg", 1, drop=O.DROP_NONE)
        ei = anorm(Ainv - dense_from_csc(n, *o.get_M()))
        assert ei <= math.sqrt(n) * q ** i * e0 * (1 + 1e-9) + 1e-13  # Eq. (3.10)


# ------------------------------------------------------- special cases

def test_diagonal_matrix_stops_cleanly():
    n = 7
    A = np.diag(np.arange(1.0, n + 1))
    n, rp, ci, v = I.dense_to_csr(A)
    for m in ("mr", "lomr", "cg"):
        o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
        r = o.run(m, 5)
        assert r["resnorm"][0] == 0.0
        assert r["flags"] & O.FLAG_CONVERGED
        assert r["done"] == 0


def test_constant_diagonal_step0_matches_closed_form():
    # A = 4 I - L (5-point Laplacian): M0 = I/4, R0 = L/4 exactly, whose
    # Frobenius norm is sqrt(#offdiag)/4
    n, rp, ci, v = lap2d(6)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    r = o.run("mr", 1)
    offdiag = len(v) - n
    assert r["resnorm"][0] == math.sqrt(offdiag) / 4


# ------------------------------------------- Table 2 operation counts

def test_table2_spgemm_counts():
    table = {}
    with open(os.path.join(GOLDEN, "table2_spgemm_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, c = line.split()
                table[k] = int(c)
    n, rp, ci, v = lap2d(8)
    K = 6
    for m, key in (("mr", "MR"), ("cg", "CG"), ("lomr", "LOMR")):
        o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
        base = o.spgemm_count()
        r = o.run(m, K)
        assert r["done"] == K
        used = o.spgemm_count() - base
        # MR/LOMR add one final residual product; CG one initial residual
        assert used == table[key] * K + 1


# --------------------------------------------------------------- PCG

def test_pcg_matches_scipy_cg_counts():
    n, rp, ci, v = lap2d(20)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    b = I.rhs_uniform(n, 0)
    for precond in (0, 1):
        res = O.pcg(n, rp, ci, v, b, rtol=1e-8, precond=precond)
        count = [0]

        def cb(xk):
            count[0] += 1
        Minv = None if precond == 0 else sp.diags(1.0 / A.diagonal())
        x, info = spla.cg(A, b, rtol=1e-8, atol=0.0, M=Minv, callback=cb, maxiter=10000)
        assert info == 0 and res["status"] == 0
        assert abs(res["iters"] - count[0]) <= 1
        assert res["relres"] < 2e-8
        np.testing.assert_allclose(res["x"], x, rtol=1e-6, atol=1e-8)


def test_pcg_exact_inverse_and_jacobi_as_matrix():
    n, rp, ci, v = lap2d(8)
    A = I.csr_to_dense(n, rp, ci, v)
    b = I.rhs_uniform(n, 0)
    Ainv = np.linalg.inv(A)
    cp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ri = np.tile(np.arange(n, dtype=np.int32), n)
    res = O.pcg(n, rp, ci, v, b, precond=2, M=(cp, ri, Ainv.T.ravel().copy()))
    assert res["iters"] == 1 and res["relres"] < 1e-12
    d = np.arange(n + 1, dtype=np.int32)
    jac = O.pcg(n, rp, ci, v, b, precond=2, M=(d, d[:-1].copy(), 1.0 / np.diag(A)))
    assert jac["iters"] == O.pcg(n, rp, ci, v, b, precond=1)["iters"]
    sym = O.pcg(n, rp, ci, v, b, precond=3, M=(d, d[:-1].copy(), 1.0 / np.diag(A)))
    assert sym["iters"] == jac["iters"]


def test_mixed_pcg_first_step_is_exact_on_integer_data():
    """With values and operands exact in FP32 and every FP32 product and sum
    exact (small integers), the FP32-values products equal the FP64 ones, so
    one mixed iteration reproduces one FP64 iteration bit for bit."""
    n, rp, ci, v = I.laplacian_1d(40)          # entries 2 and -1
    b = np.arange(1.0, n + 1.0) % 7.0 - 3.0      # small integers
    d = np.arange(n + 1, dtype=np.int32)
    half = (d, d[:-1].copy(), np.full(n, 0.5))  # M = I / 2, exact in FP32
    for precond, M in ((0, None), (2, half), (3, half)):
        a = O.pcg(n, rp, ci, v, b, maxit=1, precond=precond, M=M, mixed=True)
        f = O.pcg(n, rp, ci, v, b, maxit=1, precond=precond, M=M)
        assert a["iters"] == f["iters"] == 1 and a["status"] == f["status"] == 1
        assert np.array_equal(a["x"], f["x"])


def test_mixed_pcg_tracks_fp64_pcg():
    """FP32-values products perturb each product by FP32 rounding only: the
    iteration count stays within 2 % of the FP64 solve and x within FP32
    accuracy of it, while the results do differ (the rounding is applied)."""
    n, rp, ci, v = lap2d(32)
    b = I.rhs_uniform(n, 0)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    o.run("mr", 20)
    M = o.get_M()
    for precond in (1, 3):
        f = O.pcg(n, rp, ci, v, b, rtol=1e-8, precond=precond, M=M)
        a = O.pcg(n, rp, ci, v, b, rtol=1e-8, precond=precond, M=M, mixed=True)
        assert f["status"] == a["status"] == 0
        assert abs(a["iters"] - f["iters"]) <= max(1, 0.02 * f["iters"])
        assert not np.array_equal(a["x"], f["x"])
        assert np.linalg.norm(a["x"] - f["x"]) <= 1e-5 * np.linalg.norm(f["x"])
        assert a["relres"] < 1e-5


# ------------------------------------------------------- mixed precision

def test_mixed_emulation_tracks_fp64():
    n, rp, ci, v = I.varcoef_3d_7pt(10, seed=2)
    r64 = O.Oracle(n, rp, ci, v, cap_factor=3.0)
    r32 = O.Oracle(n, rp, ci, v, cap_factor=3.0, mixed=True)
    a = r64.run("lomr", 10)
    b = r32.run("lomr", 10)
    assert abs(b["resnorm"][-1] - a["resnorm"][-1]) <= 1e-4 * a["resnorm"][-1]
    cp, ri, va = r32.get_M()
    assert np.all(va.astype(np.float32).astype(np.float64) == va)


def test_continuation_equals_single_run():
    n, rp, ci, v = lap2d(10)
    for m in ("mr", "lomr", "cg"):
        a = O.Oracle(n, rp, ci, v, cap_factor=2.0)
        a.run(m, 7)
        a.run(m, 5)
        b = O.Oracle(n, rp, ci, v, cap_factor=2.0)
        b.run(m, 12)
        for x, y in zip(a.get_M(), b.get_M()):
            assert np.array_equal(x, y)


# ------------------------------------------------- definiteness diagnostics

def test_lanczos_extremes_match_dense_eigenvalues_of_sym_part():
    """After enough steps the extremal Ritz values are the extremal
    eigenvalues of S = (M + M^T)/2 (dense eigvalsh), and the recurrence
    tridiagonalises S: V^T S V = T for the Lanczos basis of a short run."""
    n, rp, ci, v = I.varcoef_grid((6, 7), seed=4)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    o.run("mr", 6)
    cp, ri, mv = o.get_M()
    M = dense_from_csc(n, cp, ri, mv)
    S = 0.5 * (M + M.T)
    ev = np.linalg.eigvalsh(S)
    v0 = np.random.default_rng(0).standard_normal(n)
    r = O.lanczos(n, (cp, ri, mv), v0, 3 * n)
    assert abs(r["lmin"] - ev[0]) <= 1e-10 * abs(ev).max()
    assert abs(r["lmax"] - ev[-1]) <= 1e-10 * abs(ev).max()
    # three-term recurrence, rebuilt densely from the oracle's coefficients
    k = 8
    r8 = O.lanczos(n, (cp, ri, mv), v0, k)
    V = np.zeros((n, k + 1))
    V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = S @ V[:, j] - r8["alpha"][j] * V[:, j] - (r8["beta"][j - 1] * V[:, j - 1] if j else 0)
        V[:, j + 1] = w / r8["beta"][j]
    T = np.diag(r8["alpha"]) + np.diag(r8["beta"][:-1], 1) + np.diag(r8["beta"][:-1], -1)
    np.testing.assert_allclose(V[:, :k].T @ S @ V[:, :k], T, atol=1e-10)


def test_lanczos_on_diagonal_and_indefinite_sym_parts():
    """Diagonal M: T's eigenvalues are M's distinct entries (one per
    Krylov dimension); a symmetric part with a negative eigenvalue is seen
    as lmin < 0."""
    n = 6
    d = np.array([3.0, -1.0, 2.0, 5.0, 0.5, 4.0])
    cp = np.arange(n + 1, dtype=np.int32)
    ri = np.arange(n, dtype=np.int32)
    r = O.lanczos(n, (cp, ri, d), np.ones(n), n)
    assert r["steps"] == n
    np.testing.assert_allclose(sorted(np.linalg.eigvalsh(
        np.diag(r["alpha"]) + np.diag(r["beta"][:-1], 1) + np.diag(r["beta"][:-1], -1))),
        sorted(d), rtol=0, atol=1e-12)
    assert r["lmin"] < 0 and abs(r["lmin"] + 1.0) < 1e-12 and abs(r["lmax"] - 5.0) < 1e-12
    # a nonsymmetric M: only its symmetric part counts
    A = np.array([[2.0, 1.0], [-1.0, 2.0]])   # sym part = 2 I
    r2 = O.lanczos(2, (np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                       A.T.ravel().copy()), np.array([1.0, 0.3]), 2)
    assert abs(r2["alpha"][0] - 2.0) <= 1e-15 and r2["beta"][0] <= 1e-15
    assert abs(r2["lmin"] - 2.0) <= 1e-14 and abs(r2["lmax"] - 2.0) <= 1e-14


def test_fixed_pattern_spai_pins():
    """k = 0 gives m_jj = a_jj / ||A e_j||^2; a pattern that covers every
    row gives A^{-1}; each column's residual is orthogonal to A's columns on
    its pattern (the normal equations)."""
    n, rp, ci, v = I.varcoef_grid((4, 5), seed=3)
    A = I.csr_to_dense(n, rp, ci, v)
    cp, ri, va = O.fixed_pattern_spai(n, rp, ci, v, 0)
    assert np.array_equal(ri, np.arange(n))
    np.testing.assert_allclose(va, np.diag(A) / np.sum(A * A, axis=0), rtol=1e-14)
    cp, ri, va = O.fixed_pattern_spai(n, rp, ci, v, n)
    np.testing.assert_allclose(dense_from_csc(n, cp, ri, va), np.linalg.inv(A), rtol=0, atol=1e-12)
    for k in (1, 2, 3):
        cp, ri, va = O.fixed_pattern_spai(n, rp, ci, v, k)
        M = dense_from_csc(n, cp, ri, va)
        pats = O.pattern_power(n, rp, ci, k)
        for j in range(n):
            J = pats[j]
            assert list(ri[cp[j]:cp[j + 1]]) == J
            res = np.eye(n)[:, j] - A @ M[:, j]
            np.testing.assert_allclose(A[:, J].T @ res, 0.0, atol=1e-13)
    # A^k patterns: the 5-point stencil reaches 1, 5, 13, 25 rows in the interior
    n2, rp2, ci2, v2 = I.laplacian_2d_5pt(12)
    sizes = [len(O.pattern_power(n2, rp2, ci2, k)[5 * 12 + 5]) for k in range(4)]
    assert sizes == [1, 5, 13, 25]


# ------------------------------------------ differentiation (fixed pattern)

def test_fpmr_gradient_k0_closed_form():
    """K = 0: L = sum_{r != s} (a_rs / a_ss)^2, so dL/da_rs = 2 a_rs / a_ss^2
    off the diagonal and dL/da_ss = -2 sum_{r != s} a_rs^2 / a_ss^3."""
    from oracle import fpmr
    n, rp, ci, v = I.varcoef_grid((4, 5), seed=2)
    loss, g = fpmr.gradient(n, rp, ci, v, 0)
    A = I.csr_to_dense(n, rp, ci, v)
    d = np.diag(A)
    off = A - np.diag(d)
    assert abs(loss - float(np.sum((off / d[None, :]) ** 2))) <= 1e-12 * loss
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            s = ci[e]
            want = 2 * v[e] / d[s] ** 2 if i != s else -2 * np.sum(off[:, s] ** 2) / d[s] ** 3
            assert abs(g[e] - want) <= 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("K", [1, 3, 10])
def test_fpmr_gradient_matches_central_differences(K):
    """Central differences (h = 1e-6, relative to each entry) on 50 entries
    of A treated as independent values."""
    from oracle import fpmr
    n, rp, ci, v = I.varcoef_3d_7pt(6, seed=4)
    loss, g = fpmr.gradient(n, rp, ci, v, K)
    rng = np.random.default_rng(K)
    for e in rng.choice(len(v), 50, replace=False):
        h = 1e-6 * abs(v[e])
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        fd = (fpmr.forward(n, rp, ci, vp, K) - fpmr.forward(n, rp, ci, vm, K)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(abs(g).max(), 1e-300), (e, fd, g[e])


@pytest.mark.parametrize("K", [1, 3, 10])
def test_fplomr_gradient_matches_central_differences(K):
    """Fixed-pattern LOMR (Algorithm 4 / Theorem 3 on supp(A)): the hand-written
    adjoint against central differences (h = 1e-6 relative) on 50 entries."""
    from oracle import fpmr
    n, rp, ci, v = I.varcoef_3d_7pt(6, seed=4)
    loss, g = fpmr.gradient_lomr(n, rp, ci, v, K)
    rng = np.random.default_rng(100 + K)
    for e in rng.choice(len(v), 50, replace=False):
        h = 1e-6 * abs(v[e])
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        fd = (fpmr.forward_lomr(n, rp, ci, vp, K) - fpmr.forward_lomr(n, rp, ci, vm, K)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(abs(g).max(), 1e-300), (e, fd, g[e])


def test_fplomr_first_step_is_the_mr_step():
    """With P_{-1} = 0 the first LOMR step is the MR step (Algorithm 4), so one
    step of each gives the same loss and gradient; later LOMR steps reach a
    loss no larger than MR's from the same iterate (Eq. 4.3): checked from
    M_1 on by a step of each."""
    from oracle import fpmr
    n, rp, ci, v = I.varcoef_grid((5, 6), seed=8)
    l1, g1 = fpmr.gradient_lomr(n, rp, ci, v, 1)
    l2, g2 = fpmr.gradient(n, rp, ci, v, 1)
    assert abs(l1 - l2) <= 1e-13 * l2
    np.testing.assert_allclose(g1, g2, rtol=1e-10, atol=1e-12 * abs(g2).max())
    _, st = fpmr.forward_lomr(n, rp, ci, v, 2, keep=True)
    assert not st["coefs"][1][2]  # a genuine 2-D step
    assert fpmr.forward_lomr(n, rp, ci, v, 2) <= fpmr.forward(n, rp, ci, v, 2) * (1 + 1e-12)


# ------------------------------------------ global dropping (Sec. 6.1, App. A)

def test_hard_threshold_global_cap_brute_force():
    from oracle import dropping as D
    n, rp, ci, v = lap2d(6)
    o = O.Oracle(n, rp, ci, v, cap_factor=3.0)
    o.run("mr", 3)
    cp, ri, va = o.get_M()
    for m in (n, 2 * n, len(va) - 3, len(va) + 5):
        k = D.hard_threshold(n, (cp, ri, va), m)
        ent = sorted((-abs(va[e]), j, ri[e]) for j in range(n) for e in range(cp[j], cp[j + 1]))
        want = sorted((j, r) for _, j, r in ent[:m])
        got = sorted((j, int(k[1][e])) for j in range(n) for e in range(k[0][j], k[0][j + 1]))
        assert got == want


def test_heuristic_scores_are_the_exact_single_drop_change():
    """Eq. 430: dropping one entry m_kl changes ||R||_F^2 by
    m_kl^2 ||A e_k||^2 + 2 m_kl (A R)_kl; the heuristic drops the entries
    of smallest change and keeps the diagonal."""
    from oracle import dropping as D
    n, rp, ci, v = I.varcoef_grid((5, 6), seed=1)
    A = I.csr_to_dense(n, rp, ci, v)
    o = O.Oracle(n, rp, ci, v, cap_factor=3.0)
    o.run("lomr", 4)
    Mc = o.get_M()
    M = dense_from_csc(n, *Mc)
    S = 0.5 * (M + M.T)
    S[np.abs(S) < 2.0 ** -53] = 0.0
    R = np.eye(n) - A @ S
    base = np.sum(R * R)
    nz = [(k, l) for k in range(n) for l in range(n) if S[k, l] != 0 and k != l]
    change = {}
    for (k, l) in nz:
        S2 = S.copy()
        S2[k, l] = 0.0
        R2 = np.eye(n) - A @ S2
        change[(k, l)] = np.sum(R2 * R2) - base
        pred = S[k, l] ** 2 * np.sum(A[:, k] ** 2) + 2 * S[k, l] * (A @ R)[k, l]
        assert abs(change[(k, l)] - pred) <= 1e-10 * max(1.0, base)
    m = len(nz) + n - 25
    out = D.heuristic(n, rp, ci, v, Mc, m)
    Mo = dense_from_csc(n, *out)
    assert np.all(np.diag(Mo) == np.diag(S))               # diagonal kept
    order = sorted(change, key=lambda kl: (change[kl], kl[1], kl[0]))
    assert change[order[25]] - change[order[24]] > 1e-9 * max(1.0, base)  # no near-tie at the cut
    assert set((k, l) for (k, l) in nz if Mo[k, l] == 0) == set(order[:25])
    # entries that stay keep the symmetrised values
    keep = Mo != 0
    assert np.array_equal(Mo[keep], S[keep])


def test_global_mr_flow_step_is_the_line_minimiser_of_the_thresholded_direction():
    """One iteration of MR with global dropping: alpha_0 minimises
    ||R_0 - a A P_0||_F for P_0 the brute-force top-m_dir of R_0 (MR) or of
    Pi R_0 (MR_SPD, weighted norm), and the final history entry is the
    dense ||I - A M_1||_F of the returned M."""
    from oracle import dropping as D
    n, rp, ci, v = I.varcoef_grid((5, 6), seed=4)
    A = I.csr_to_dense(n, rp, ci, v)
    d = np.diag(A)
    R0 = np.eye(n) - A @ np.diag(1.0 / d)
    for use_pi in (False, True):
        X = np.diag(1.0 / d) @ R0 if use_pi else R0
        ent = sorted((-abs(X[r, j]), j, r) for j in range(n) for r in range(n) if X[r, j] != 0)
        m_dir = len(ent) // 3
        P = np.zeros_like(X)
        for _, j, r in ent[:m_dir]:
            P[r, j] = X[r, j]
        AP = A @ P
        W = np.diag(1.0 / d) if use_pi else np.eye(n)
        alpha = np.sum(R0 * (W @ AP)) / np.sum(AP * (W @ AP))
        out = D.run_global_mr(n, rp, ci, v, 1, m_dir, 10 ** 9, use_pi=use_pi)
        assert out["done"] == 1
        assert abs(out["coef"][0] - alpha) <= 1e-12 * abs(alpha)
        M1 = dense_from_csc(n, *out["M"])
        np.testing.assert_allclose(out["resnorm"][-1], np.linalg.norm(np.eye(n) - A @ M1),
                                   rtol=1e-12)


def _top(X, m):
    """Brute-force global hard threshold: the m entries of largest |x|
    (ties: smaller column, then smaller row)."""
    n = X.shape[0]
    ent = sorted((-abs(X[r, j]), j, r) for j in range(n) for r in range(n) if X[r, j] != 0)
    P = np.zeros_like(X)
    for _, j, r in ent[:m]:
        P[r, j] = X[r, j]
    return P


def test_global_lomr_flow_steps_are_the_2d_minimisers():
    """LOMR with global dropping: (delta_0, gamma_0) = (the line minimiser of
    ||R_0 - d A Z_0||_W, 0) for Z_0 the brute-force top-m_dir of (Pi) R_0, and
    (delta_1, gamma_1) minimise ||R_1 - A (d Z_1 + g P_0)||_W (Theorem 3) with
    P_0 the top-m_dir of delta_0 Z_0 and R_1 the dense residual of the
    returned M_1; W = I (LOMR) or Pi (LOMR_SPD)."""
    from oracle import dropping as D
    n, rp, ci, v = I.varcoef_grid((5, 6), seed=4)
    A = I.csr_to_dense(n, rp, ci, v)
    d = np.diag(A)
    R0 = np.eye(n) - A @ np.diag(1.0 / d)
    m_dir, m_M = 2 * len(v) // 3, 10 ** 9
    for use_pi in (False, True):
        Wd = 1.0 / d if use_pi else np.ones(n)
        ip = lambda X, Y: np.sum(X * (Wd[:, None] * Y))
        Z0 = _top(np.diag(1.0 / d) @ R0 if use_pi else R0, m_dir)
        U = A @ Z0
        d0 = ip(U, R0) / ip(U, U)
        one = D.run_global_lomr(n, rp, ci, v, 1, m_dir, m_M, use_pi=use_pi)
        assert one["done"] == 1
        assert abs(one["coef"][0, 0] - d0) <= 1e-12 * abs(d0) and one["coef"][0, 1] == 0.0
        M1 = dense_from_csc(n, *one["M"])
        # M_1 = the heuristic (here: symmetrisation) of M_0 + S_0, S_0 = delta_0 Z_0
        T = np.diag(1.0 / d) + d0 * Z0
        np.testing.assert_allclose(M1, 0.5 * (T + T.T), rtol=0, atol=1e-14)
        R1 = np.eye(n) - A @ M1
        np.testing.assert_allclose(one["resnorm"][-1], np.linalg.norm(R1), rtol=1e-12)
        P0 = _top(d0 * Z0, m_dir)
        Z1 = _top(np.diag(1.0 / d) @ R1 if use_pi else R1, m_dir)
        U, V = A @ Z1, A @ P0
        G = np.array([[ip(U, U), ip(U, V)], [ip(U, V), ip(V, V)]])
        dg = np.linalg.solve(G, [ip(U, R1), ip(V, R1)])
        two = D.run_global_lomr(n, rp, ci, v, 2, m_dir, m_M, use_pi=use_pi)
        assert two["done"] == 2
        np.testing.assert_allclose(two["coef"][1], dg, rtol=1e-9)


def test_global_cg_flow_coefficients_match_dense_cg():
    """CG with global dropping: alpha_0 = (R_0, Pi R_0) / (P_0, A P_0) for P_0
    the top-m_dir of (Pi) R_0; beta_0 = (R_1, Pi R_1) / (R_0, Pi R_0) with R_1
    the dense residual of the returned M_1; alpha_1 from P_1 = the top-m_dir
    of (Pi) R_1 + beta_0 P_0 (Algorithms 3 and 7; Pi = I for plain CG)."""
    from oracle import dropping as D
    n, rp, ci, v = I.varcoef_grid((5, 6), seed=4)
    A = I.csr_to_dense(n, rp, ci, v)
    d = np.diag(A)
    R0 = np.eye(n) - A @ np.diag(1.0 / d)
    m_dir, m_M = 2 * len(v) // 3, 10 ** 9
    for use_pi in (False, True):
        Pi = np.diag(1.0 / d) if use_pi else np.eye(n)
        P0 = _top(Pi @ R0, m_dir)
        rz0 = np.sum(R0 * (Pi @ R0))
        a0 = rz0 / np.sum(P0 * (A @ P0))
        one = D.run_global_cg(n, rp, ci, v, 1, m_dir, m_M, use_pi=use_pi)
        assert one["done"] == 1
        M1 = dense_from_csc(n, *one["M"])
        T = np.diag(1.0 / d) + a0 * P0  # M_1 = the heuristic (symmetrisation) of M_0 + alpha_0 P_0
        np.testing.assert_allclose(M1, 0.5 * (T + T.T), rtol=0, atol=1e-14)
        R1 = np.eye(n) - A @ M1
        rz1 = np.sum(R1 * (Pi @ R1))
        np.testing.assert_allclose(one["coef"][0], [a0, rz1 / rz0], rtol=1e-12)
        np.testing.assert_allclose(one["resnorm"], [np.linalg.norm(R0), np.linalg.norm(R1)],
                                   rtol=1e-12)
        P1 = _top(Pi @ R1 + (rz1 / rz0) * P0, m_dir)
        a1 = rz1 / np.sum(P1 * (A @ P1))
        two = D.run_global_cg(n, rp, ci, v, 2, m_dir, m_M, use_pi=use_pi)
        assert two["done"] == 2
        np.testing.assert_allclose(two["coef"][1, 0], a1, rtol=1e-10)


# ---------------------------------------- exact arithmetic of the products

def _round_f32(q):
    """The float32 nearest to the rational q (ties to even), as a float."""
    from fractions import Fraction
    if q == 0:
        return 0.0
    neg, q = q < 0, abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    qe = max(e - 23, -149)  # 24-bit significand; subnormal quantum 2^-149
    scaled = q / Fraction(2) ** qe
    k = scaled.numerator // scaled.denominator
    rem = scaled - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    x = float(Fraction(k) * Fraction(2) ** qe)
    return -x if neg else x


def test_product_column_is_the_exact_rounded_fma_chain():
    """A X_j, both precisions, against an independent construction: each
    fma of the ascending-k chain acc = fma(a_rk, x_k, acc) evaluated exactly
    on rationals and rounded once to FP64 or FP32 (the fixed order of the
    product chain; the mixed path rounds A's values to FP32 first)."""
    from fractions import Fraction
    n, rp, ci, v = I.varcoef_grid((7, 8), seed=21)
    rng = np.random.default_rng(3)
    for mixed in (False, True):
        o = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=4.0)
        av = [float(np.float32(x)) for x in v] if mixed else list(v)
        rnd = _round_f32 if mixed else (lambda q: float(q))
        for trial in range(6):
            rows = np.sort(rng.choice(n, size=9, replace=False))
            vals = rng.standard_normal(9) * 10.0 ** rng.integers(-3, 4, 9)
            if mixed:
                vals = vals.astype(np.float32).astype(np.float64)
            want = {}
            for k, x in zip(rows.tolist(), vals.tolist()):  # ascending k
                for q in range(rp[k], rp[k + 1]):
                    r = int(ci[q])
                    want[r] = rnd(Fraction(av[q]) * Fraction(x) + Fraction(want.get(r, 0.0)))
            gr, gv = o.product_column(rows, vals)
            exp = sorted((r, x) for r, x in want.items() if x != 0.0)
            assert gr.tolist() == [r for r, _ in exp]
            assert gv.tolist() == [x for _, x in exp]


def test_column_residual_is_exact_chain_then_one_rounding():
    """R_j = e_j - A M_j: the exact-rational fma chain of A M_j, then 1 - s on
    the diagonal rounded once to the value type and -s elsewhere, exact
    zeros removed (supp holds nonzeros only, Sec. 6.1), for the stored M after
    a few MR steps."""
    from fractions import Fraction
    n, rp, ci, v = I.varcoef_grid((6, 7), seed=22)
    for mixed in (False, True):
        o = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=3.0)
        o.run("mr", 3)
        cp, ri, mv = o.get_M()
        av = [float(np.float32(x)) for x in v] if mixed else list(v)
        rnd = _round_f32 if mixed else (lambda q: float(q))
        for j in range(0, n, 5):
            acc = {}
            for k, x in zip(ri[cp[j]:cp[j + 1]].tolist(), mv[cp[j]:cp[j + 1]].tolist()):
                for q in range(rp[k], rp[k + 1]):
                    r = int(ci[q])
                    acc[r] = rnd(Fraction(av[q]) * Fraction(x) + Fraction(acc.get(r, 0.0)))
            want = {r: -x for r, x in acc.items()}
            want[j] = rnd(Fraction(1) - Fraction(acc.get(j, 0.0)))
            exp = sorted((r, x) for r, x in want.items() if x != 0.0)
            gr, gv = o.column_residual(j)
            assert gr.tolist() == [r for r, _ in exp]
            assert gv.tolist() == [x for _, x in exp]


def _cols(X):
    cp, ri, va = X
    return [dict(zip(ri[cp[j]:cp[j + 1]].tolist(), va[cp[j]:cp[j + 1]].tolist()))
            for j in range(len(cp) - 1)]


def test_update_combinations_are_single_roundings():
    """The iterate updates in their fixed rounding order, checked entry by entry against exact
    rational arithmetic: MR and CG M+ = fl(m + alpha p); CG P+ = fl(r + beta p);
    LOMR S = fl(delta z + fl(gamma p)), P = S, M+ = fl(m + s), each rounded
    once to FP64 (then once more to FP32 on the mixed path), exact zeros
    removed (no dropping here, so nothing else changes the entries)."""
    from fractions import Fraction
    n, rp, ci, v = I.varcoef_grid((6, 5), seed=23)

    def f64(q):
        return float(q)

    for mixed in (False, True):
        rv = (lambda x: float(np.float32(x))) if mixed else (lambda x: x)

        def comb(c, y, x):  # fl(x + c y), one FP64 rounding, then the value type
            return rv(f64(Fraction(c) * Fraction(y) + Fraction(x)))

        for method in ("mr", "cg", "lomr"):
            o = O.Oracle(n, rp, ci, v, mixed=mixed, cap_factor=float(n))
            o.run(method, 1, drop=O.DROP_NONE)
            M1, P1 = _cols(o.get(0)), _cols(o.get(1))
            r = o.run(method, 1, drop=O.DROP_NONE)  # continues the recurrence
            M2, P2, Z2 = _cols(o.get(0)), _cols(o.get(1)), _cols(o.get(2))
            c0, c1 = r["coef"][0]
            for j in range(n):
                if method == "mr":  # M2 = M1 + alpha_1 P_1 (P_1 = R_1 now in P2)
                    want = {k: comb(c0, P2[j].get(k, 0.0), M1[j].get(k, 0.0))
                            for k in set(M1[j]) | set(P2[j])}
                    got = M2[j]
                elif method == "cg":  # M2 = M1 + alpha_1 P_1 with the P of the first call
                    want = {k: comb(c0, P1[j].get(k, 0.0), M1[j].get(k, 0.0))
                            for k in set(M1[j]) | set(P1[j])}
                    got = M2[j]
                else:  # LOMR: S_1 = delta Z_1 + gamma P_0 (P1), P2 = S_1, M2 = M1 + S_1
                    S = {}
                    for k in set(Z2[j]) | set(P1[j]):
                        g = c1 * P1[j].get(k, 0.0)  # FP64 product, rounded
                        S[k] = rv(f64(Fraction(c0) * Fraction(Z2[j].get(k, 0.0)) + Fraction(g)))
                    S = {k: x for k, x in S.items() if x != 0.0}
                    assert P2[j] == S
                    want = {k: rv(f64(Fraction(M1[j].get(k, 0.0)) + Fraction(S.get(k, 0.0))))
                            for k in set(M1[j]) | set(S)}
                    got = M2[j]
                want = {k: x for k, x in want.items() if x != 0.0}
                assert got == want, (method, mixed, j)
