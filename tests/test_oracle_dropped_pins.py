"""Pins of the oracle's dropped-direction branches (Sec. 6.1 applied per column).

With per-column hard thresholding the directions are Z_i = D(R_i) (LOMR),
P_i = D(S_i) (LOMR), P_0 = D(R_0) and P_{i+1} = D(R_{i+1} + beta P_i) (CG);
M is dropped too under the full rule.  Each test below rebuilds every step
of the oracle's run from its state before the step with dense numpy algebra
and a brute-force per-column drop (full sort by (|v| descending, row
ascending), then truncation), and checks:

- LOMR (Algorithm 4, Theorem 3): (delta_i, gamma_i) minimise
  ||R_i - A (d Z_i + g P_{i-1})||_F over the span of the DROPPED Z_i and
  the stored P_{i-1} (the 2-D least-squares problem solved densely), and
  Z_i, P_i, M_{i+1} are the brute-force drops of R_i, S_i and M_i + S_i;
- CG (Algorithm 3, Prop. 2 ratios): alpha_i = ||R_i||^2 / (P_i, A P_i) with
  the dropped P_i, beta_i = ||R_{i+1}||^2 / ||R_i||^2, and M_{i+1}, P_{i+1}
  are the brute-force drops of M_i + alpha P_i and R_{i+1} + beta P_i;
- MR and LOMR never increase ||R||_F when only the directions are dropped
  (Eq. 2.6 and Theorem 3: the step is a least-squares minimiser over a span
  that contains 0, so ||R_{i+1}|| <= ||R_i||).

The residual columns R_i are read from the oracle's column residual, whose
arithmetic is pinned bit for bit against exact rational fma chains in
``test_oracle_pins.py``; the combinations are rebuilt with one exact
rational rounding each, so the dropped patterns are compared exactly,
including the tie-heavy 2-D Laplacian.  Each test also checks that it would
catch the plausible slips (U formed from the undropped R, alpha from the
undropped direction): those give coefficients far from the oracle's.
No GPU.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2511_09753_gb300 import inputs as I


def _caps(n, rp, f):
    """cap_j = floor(f * nnz(A[:, j])) clamped to [1, n] (A symmetric)."""
    lens = np.diff(np.asarray(rp))
    return [int(min(max(np.floor(f * L), 1), n)) for L in lens]


def _brute_drop(col, cap):
    """Keep the cap entries of largest |v|, ties to the smaller row."""
    if len(col) <= cap:
        return dict(col)
    keep = sorted(col, key=lambda r: (-abs(col[r]), r))[:cap]
    return {r: col[r] for r in keep}


def _cols(X):
    cp, ri, va = X
    return [dict(zip(ri[cp[j]:cp[j + 1]].tolist(), va[cp[j]:cp[j + 1]].tolist()))
            for j in range(len(cp) - 1)]


def _dense(cols, n):
    D = np.zeros((n, n))
    for j, c in enumerate(cols):
        for r, x in c.items():
            D[r, j] = x
    return D


def _residual_cols(o, n):
    out = []
    for j in range(n):
        rows, vals = o.column_residual(j)
        out.append(dict(zip(rows.tolist(), vals.tolist())))
    return out


def _fl(q):
    return float(q)  # Fraction -> nearest double (ties to even)


def _nz(d):
    return {k: x for k, x in d.items() if x != 0.0}


CASES = [
    ("random_spd", lambda: I.random_spd_banded(12, 3, seed=11), 1.0),
    ("laplacian_ties", lambda: I.laplacian_2d_5pt(4), 0.5),
    ("varcoef", lambda: I.varcoef_grid((4, 4), seed=9), 0.8),
]


@pytest.mark.parametrize("name,make,f", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("drop", [O.DROP_DIRECTIONS, O.DROP_TOPK], ids=["dirs", "topk"])
def test_lomr_dropped_steps_are_2d_minimisers_over_the_dropped_span(name, make, f, drop):
    n, rp, ci, v = make()
    A = I.csr_to_dense(n, rp, ci, v)
    caps = _caps(n, rp, f)
    o = O.Oracle(n, rp, ci, v, cap_factor=f)
    Pprev = [dict() for _ in range(n)]  # P_{-1} = 0
    slip_gap = 0.0
    dropped_any = False
    for i in range(6):
        M = _cols(o.get(0))
        R = _residual_cols(o, n)
        Z = [_brute_drop(R[j], caps[j]) for j in range(n)]
        dropped_any |= any(len(Z[j]) < len(R[j]) for j in range(n))
        Rd, Zd, Pd = _dense(R, n), _dense(Z, n), _dense(Pprev, n)
        U, V = A @ Zd, A @ Pd
        if i == 0:
            d_ref, g_ref = np.sum(U * Rd) / np.sum(U * U), 0.0
        else:
            B = np.stack([U.ravel(), V.ravel()], axis=1)
            d_ref, g_ref = np.linalg.lstsq(B, Rd.ravel(), rcond=None)[0]
        # the slip "U = A R instead of A D(R)" gives other coefficients
        Us = A @ Rd
        if i == 0:
            d_s = np.sum(Us * Rd) / np.sum(Us * Us)
        else:
            d_s = np.linalg.lstsq(np.stack([Us.ravel(), V.ravel()], axis=1), Rd.ravel(),
                                  rcond=None)[0][0]
        slip_gap = max(slip_gap, abs(d_s - d_ref) / abs(d_ref))

        r = o.run("lomr", 1, drop=drop)
        assert r["done"] == 1 and not (r["flags"] & O.FLAG_FALLBACK)
        d, g = r["coef"][0]
        # the coefficients, to within the 2x2 system's conditioning ...
        cond = 1.0 if i == 0 else np.linalg.cond(B.T @ B)
        tol = 1e-13 * cond * max(abs(d_ref), abs(g_ref))
        assert abs(d - d_ref) <= tol and abs(g - g_ref) <= tol, (i, d, d_ref, g, g_ref)
        # ... and the objective they reach, which is the dense minimum
        obj = lambda dd, gg: float(np.sum((Rd - dd * U - gg * V) ** 2))
        assert obj(d, g) - obj(d_ref, g_ref) <= 1e-13 * float(np.sum(Rd * Rd))
        assert r["resnorm"][0] == pytest.approx(np.linalg.norm(Rd), rel=1e-13)
        # Z_i, P_i = D(S_i), M_{i+1} = D(M_i + S_i) (reading: S = fl(d z + fl(g p)))
        Zo, Po, Mo = _cols(o.get(2)), _cols(o.get(1)), _cols(o.get(0))
        for j in range(n):
            assert Zo[j] == Z[j], (i, j)
            S = _nz({k: _fl(Fraction(d) * Fraction(Z[j].get(k, 0.0))
                            + Fraction(g * Pprev[j].get(k, 0.0)))
                     for k in set(Z[j]) | set(Pprev[j])})
            assert Po[j] == _brute_drop(S, caps[j]), (i, j)
            Mp = _nz({k: _fl(Fraction(M[j].get(k, 0.0)) + Fraction(S.get(k, 0.0)))
                      for k in set(M[j]) | set(S)})
            if drop == O.DROP_TOPK:
                Mp = _brute_drop(Mp, caps[j])
            assert Mo[j] == Mp, (i, j)
        if drop == O.DROP_DIRECTIONS:  # Theorem 3: the minimiser over a span containing 0
            assert r["resnorm"][1] <= r["resnorm"][0] * (1 + 1e-13)
        Pprev = Po
    assert dropped_any
    assert slip_gap > 1e-6  # the check above tells the dropped Z from the full R


@pytest.mark.parametrize("name,make,f", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("drop", [O.DROP_DIRECTIONS, O.DROP_TOPK], ids=["dirs", "topk"])
def test_cg_dropped_steps_follow_algorithm_3_with_dropped_directions(name, make, f, drop):
    n, rp, ci, v = make()
    A = I.csr_to_dense(n, rp, ci, v)
    caps = _caps(n, rp, f)
    o = O.Oracle(n, rp, ci, v, cap_factor=f)
    R = _residual_cols(o, n)
    o.run("cg", 0, drop=drop)  # sets P_0 = D(R_0)
    P = _cols(o.get(1))
    assert P == [_brute_drop(R[j], caps[j]) for j in range(n)]
    slip_gap = 0.0
    Xu = _dense(R, n)  # the direction before its drop
    for i in range(6):
        M = _cols(o.get(0))
        Rd, Pd = _dense(R, n), _dense(P, n)
        rr = float(np.sum(Rd * Rd))
        a_ref = rr / np.sum(Pd * (A @ Pd))
        a_slip = rr / np.sum(Xu * (A @ Xu))  # the slip: alpha from the undropped direction
        slip_gap = max(slip_gap, abs(a_slip - a_ref) / abs(a_ref))
        r = o.run("cg", 1, drop=drop)
        assert r["done"] == 1
        a, b = r["coef"][0]
        assert abs(a - a_ref) <= 1e-12 * abs(a_ref), (i, a, a_ref)
        Mo = _cols(o.get(0))
        for j in range(n):
            Mp = _nz({k: _fl(Fraction(a) * Fraction(P[j].get(k, 0.0)) + Fraction(M[j].get(k, 0.0)))
                      for k in set(M[j]) | set(P[j])})
            if drop == O.DROP_TOPK:
                Mp = _brute_drop(Mp, caps[j])
            assert Mo[j] == Mp, (i, j)
        R1 = _residual_cols(o, n)
        rr1 = float(np.sum(_dense(R1, n) ** 2))
        assert abs(b - rr1 / rr) <= 1e-12 * (rr1 / rr), (i, b, rr1 / rr)
        assert r["resnorm"][1] == pytest.approx(np.sqrt(rr1), rel=1e-13)
        Po = _cols(o.get(1))
        Xs = []
        for j in range(n):
            X = _nz({k: _fl(Fraction(b) * Fraction(P[j].get(k, 0.0)) + Fraction(R1[j].get(k, 0.0)))
                     for k in set(R1[j]) | set(P[j])})
            assert Po[j] == _brute_drop(X, caps[j]), (i, j)
            Xs.append(X)
        R, P, Xu = R1, Po, _dense(Xs, n)
    assert slip_gap > 1e-6


@pytest.mark.parametrize("method", ["mr", "lomr"])
@pytest.mark.parametrize("name,make,f", CASES, ids=[c[0] for c in CASES])
def test_direction_only_dropping_never_increases_the_residual(method, name, make, f):
    """Eq. 2.6 (MR) and Theorem 3 (LOMR): with M kept whole, each step
    minimises ||R - A S|| over a span that contains S = 0."""
    n, rp, ci, v = make()
    o = O.Oracle(n, rp, ci, v, cap_factor=f)
    r = o.run(method, 25, drop=O.DROP_DIRECTIONS)
    h = r["resnorm"][: r["done"] + 1]
    assert r["done"] >= 10
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-13)), h
    assert h[-1] < 0.9 * h[0]


def test_mr_dropped_direction_steps_match_brute_force():
    """MR (Algorithm 1) with P_i = D(R_i): several consecutive steps, each
    alpha the dense line minimiser along the brute-force dropped P_i, and
    M_{i+1} = D(M_i + alpha P_i) entry for entry."""
    n, rp, ci, v = I.laplacian_2d_5pt(4)
    A = I.csr_to_dense(n, rp, ci, v)
    f = 0.5
    caps = _caps(n, rp, f)
    o = O.Oracle(n, rp, ci, v, cap_factor=f)
    for i in range(6):
        M = _cols(o.get(0))
        R = _residual_cols(o, n)
        P = [_brute_drop(R[j], caps[j]) for j in range(n)]
        Rd, Pd = _dense(R, n), _dense(P, n)
        AP = A @ Pd
        a_ref = np.sum(Rd * AP) / np.sum(AP * AP)
        r = o.run("mr", 1, drop=O.DROP_TOPK)
        a = r["coef"][0, 0]
        assert abs(a - a_ref) <= 1e-12 * abs(a_ref)
        assert _cols(o.get(1)) == P
        Mo = _cols(o.get(0))
        for j in range(n):
            Mp = _nz({k: _fl(Fraction(a) * Fraction(P[j].get(k, 0.0)) + Fraction(M[j].get(k, 0.0)))
                      for k in set(M[j]) | set(P[j])})
            assert Mo[j] == _brute_drop(Mp, caps[j]), (i, j)


def _brute_drop_keep(col, cap, keep_row):
    """The drop with the column's diagonal always kept (it counts toward the
    cap): the diagonal, then the cap - 1 largest |v| of the other rows."""
    if len(col) <= cap:
        return dict(col)
    if keep_row not in col:
        return _brute_drop(col, cap)
    rest = {r: x for r, x in col.items() if r != keep_row}
    out = _brute_drop(rest, cap - 1) if cap > 1 else {}
    out[keep_row] = col[keep_row]
    return out


def test_drop_column_keep_diag_brute_force():
    rng = np.random.default_rng(7)
    for trial in range(300):
        L = int(rng.integers(1, 50))
        rows = np.sort(rng.choice(200, L, replace=False))
        vals = rng.choice([-0.5, -0.25, 0.25, 0.5, 1.0, 3.0, 1e-3], L) * rng.choice([1.0, 0.999], L)
        cap = int(rng.integers(1, 30))
        keep = int(rows[rng.integers(0, L)]) if trial % 4 else 999  # 999: absent
        r1, v1 = O.drop_column(rows, vals, cap, keep_row=keep)
        want = _brute_drop_keep(dict(zip(rows.tolist(), vals.tolist())), cap, keep)
        assert dict(zip(r1.tolist(), v1.tolist())) == want
    # the smallest entry survives when it is the diagonal
    r, v = O.drop_column([1, 3, 5], [5.0, -1e-9, 4.0], 2, keep_row=3)
    assert list(r) == [1, 3] and list(v) == [5.0, -1e-9]


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_keep_diag_steps_match_brute_force(method):
    """With keep_diag every per-column drop (of M and of the directions)
    keeps row j of column j: one LOMR/MR/CG step rebuilt densely with that
    drop equals the oracle's, and M's diagonal never vanishes."""
    n, rp, ci, v = I.varcoef_grid((4, 4), seed=9)
    A = I.csr_to_dense(n, rp, ci, v)
    f = 0.6
    caps = _caps(n, rp, f)
    o = O.Oracle(n, rp, ci, v, cap_factor=f)
    o.set_keep_diag(True)
    if method == "cg":
        o.run("cg", 0)
    for i in range(4):
        M = _cols(o.get(0))
        R = _residual_cols(o, n)
        Pprev = _cols(o.get(1))
        r = o.run(method, 1)
        a, g = r["coef"][0]
        Mo, Po = _cols(o.get(0)), _cols(o.get(1))
        for j in range(n):
            if method == "mr":
                P = _brute_drop_keep(R[j], caps[j], j)
                assert Po[j] == P
                Mp = _nz({k: _fl(Fraction(a) * Fraction(P.get(k, 0.0)) + Fraction(M[j].get(k, 0.0)))
                          for k in set(M[j]) | set(P)})
            elif method == "cg":
                Mp = _nz({k: _fl(Fraction(a) * Fraction(Pprev[j].get(k, 0.0))
                                 + Fraction(M[j].get(k, 0.0)))
                          for k in set(M[j]) | set(Pprev[j])})
            else:
                Z = _brute_drop_keep(R[j], caps[j], j)
                assert _cols(o.get(2))[j] == Z
                S = _nz({k: _fl(Fraction(a) * Fraction(Z.get(k, 0.0))
                                + Fraction(g * Pprev[j].get(k, 0.0)))
                         for k in set(Z) | set(Pprev[j])})
                assert Po[j] == _brute_drop_keep(S, caps[j], j)
                Mp = _nz({k: _fl(Fraction(M[j].get(k, 0.0)) + Fraction(S.get(k, 0.0)))
                          for k in set(M[j]) | set(S)})
            assert Mo[j] == _brute_drop_keep(Mp, caps[j], j), (i, j)
            assert j in Mo[j]
        assert r["nnz"][0] == sum(len(c) for c in M)
        assert r["nnz"][1] == sum(len(c) for c in Mo)


@pytest.mark.parametrize("method", ["mr", "lomr", "cg"])
def test_nnz_history_counts_the_iterates(method):
    """nnz[i] is nnz(M_i) of the iterate whose residual resnorm[i] records:
    checked against the iterate exported after each single step."""
    n, rp, ci, v = I.laplacian_2d_5pt(6)
    o = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    o2 = O.Oracle(n, rp, ci, v, cap_factor=2.0)
    r = o.run(method, 5)
    seen = [int(o2.get(0)[0][-1])]
    for i in range(5):
        o2.run(method, 1)
        seen.append(int(o2.get(0)[0][-1]))
    assert list(r["nnz"]) == seen
    assert seen[0] == n and seen[-1] > seen[1] > n
