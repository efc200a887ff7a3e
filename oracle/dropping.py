"""Oracle for the paper's global dropping operators (test infrastructure).

Hard thresholding with a global density cap (Sec. 6.1, Eq. 6.2 / 445):
when |supp(X)| > m, keep the m entries of largest |x|; ties go to the
smaller (column, row) position.

The dropping heuristic for the main iterate (Appendix A):
  1. M := (M + M^T) / 2  (s_kl = 0.5 (m_kl + m_lk) in FP64, rounded to the
     value type; exact zeros dropped);
  2. drop the off-diagonal entries with |m_kl| < u, u the unit round-off of
     the value type (2^-53 for FP64, 2^-24 for FP32 values);
  3. if |supp(M)| > m, drop the |supp(M)| - m off-diagonal entries of
     smallest score s_kl = m_kl^2 ||A e_k||^2 + 2 m_kl (A R)_kl, R = I - A M
     (Eq. 435 with the m^2 reading of Eq. 430: the change of ||R||_F^2 when
     that entry alone is dropped); ties go to the smaller (column, row)
     position, the diagonal is always kept.
Arithmetic of the scores (shared with the kernels by definition): R's
columns as the method computes them (an fma chain over ascending k in the
value type, R = 1 - s on the diagonal, -s elsewhere), ||A e_k||^2 and
(A R)_kl as FP64 fma chains over ascending column of row k of A, and
s = fma(2 m, ar, (m m) nrm) in FP64.
"""
import numpy as np


def _csc_cols(cp, ri, va):
    return [(ri[cp[j]:cp[j + 1]].astype(np.int64), va[cp[j]:cp[j + 1]].astype(np.float64))
            for j in range(len(cp) - 1)]


def _to_csc(n, cols):
    cp = [0]
    ri, va = [], []
    for j in range(n):
        r, v = cols[j]
        o = np.argsort(r, kind="stable")
        ri.extend(r[o].tolist())
        va.extend(v[o].tolist())
        cp.append(len(ri))
    return np.array(cp, np.int32), np.array(ri, np.int32), np.array(va, np.float64)


def hard_threshold(n, M, m):
    """Keep the m entries of largest |x| (ties: smaller (column, row))."""
    cols = _csc_cols(*M)
    ent = [(-abs(v), j, r) for j, (rr, vv) in enumerate(cols) for r, v in zip(rr, vv)]
    if len(ent) <= m:
        return M
    ent.sort()
    keep = set((j, r) for _, j, r in ent[:m])
    out = []
    for j, (rr, vv) in enumerate(cols):
        sel = np.array([(j, int(r)) in keep for r in rr], dtype=bool)
        out.append((rr[sel], vv[sel]))
    return _to_csc(n, out)


def _fma(a, b, c):
    """Correctly rounded FP64 fma via exact rationals."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def heuristic(n, rowptr, colind, vals, M, m, mixed=False):
    """Appendix A's three steps on M (CSC triple); returns the new M."""
    av = np.array([float(np.float32(x)) for x in vals]) if mixed else np.asarray(vals, np.float64)
    u = 2.0 ** -24 if mixed else 2.0 ** -53
    cols = _csc_cols(*M)
    dense = {}
    for j, (rr, vv) in enumerate(cols):
        for r, v in zip(rr, vv):
            dense[(int(r), j)] = float(v)
    keys = set(dense) | set((j, r) for (r, j) in dense)
    sym = {}
    for (r, j) in keys:
        s = 0.5 * (dense.get((r, j), 0.0) + dense.get((j, r), 0.0))
        if mixed:
            s = float(np.float32(s))
        if s != 0.0 and (r == j or abs(s) >= u):
            sym[(r, j)] = s
    newcols = [[] for _ in range(n)]
    for (r, j), s in sym.items():
        newcols[j].append((r, s))
    cols2 = []
    for j in range(n):
        lst = sorted(newcols[j])
        cols2.append((np.array([a for a, _ in lst], np.int64), np.array([b for _, b in lst])))
    if len(sym) <= m:
        return _to_csc(n, cols2)
    nrm = np.zeros(n)
    for k in range(n):
        acc = 0.0
        for q in range(rowptr[k], rowptr[k + 1]):
            acc = _fma(av[q], av[q], acc)
        nrm[k] = acc
    from oracle import Oracle
    o = Oracle(n, rowptr, colind, vals, mixed=mixed, cap_factor=float(n))
    o.set_M(*_to_csc(n, cols2))
    scores = []
    for j in range(n):
        rr, rv = o.column_residual(j)
        R = dict(zip(rr.tolist(), rv.tolist()))
        for r, x in zip(*cols2[j]):
            r = int(r)
            if r == j:
                continue
            ar = 0.0
            for q in range(rowptr[r], rowptr[r + 1]):
                ar = _fma(av[q], R.get(int(colind[q]), 0.0), ar)
            s = _fma(2.0 * x, ar, (x * x) * nrm[r])
            scores.append((s, j, r))
    ndiag = sum(1 for (r, j) in sym if r == j)
    ndrop = len(sym) - max(m, ndiag)
    scores.sort()
    drop = set((j, r) for _, j, r in scores[:ndrop])
    out = []
    for j in range(n):
        rr, vv = cols2[j]
        sel = np.array([(j, int(r)) not in drop for r in rr], dtype=bool)
        out.append((rr[sel], vv[sel]))
    return _to_csc(n, out)


def _rv(x, mixed):
    return float(np.float32(x)) if mixed else float(x)


def run_global_mr(n, rowptr, colind, vals, iters, m_dir, m_M, mixed=False, use_pi=False):
    """MR (Algorithm 1) or MR_SPD (Algorithm 5, Pi = diag(A)^{-1}) with the
    paper's global dropping placed as in its Experiment 05: every iteration
    takes R_i = I - A M_i, the direction P_i = (Pi) R_i hard-thresholded to the
    m_dir largest entries over the whole matrix, alpha_i from that P_i (the
    coefficient arithmetic of the column pass), M_i + alpha_i P_i (union, FP64
    fma rounded once), then the Appendix A heuristic with density cap m_M.
    Returns dict(M, resnorm, coef, done)."""
    import math
    from oracle import Oracle, fixsum, pairwise
    o = Oracle(n, rowptr, colind, vals, mixed=mixed, cap_factor=float(n))
    M = o.get_M()
    diag = np.zeros(n)
    for i in range(n):
        for q in range(rowptr[i], rowptr[i + 1]):
            if colind[q] == i:
                diag[i] = vals[q]
    pi = 1.0 / diag
    res, coef = [], []
    done = 0

    def residuals(Mc):
        o.set_M(*Mc)
        R = [o.column_residual(j) for j in range(n)]
        rr = pairwise([fixsum(np.asarray(v) * np.asarray(v)) for _, v in R])
        return R, rr

    for _ in range(iters):
        R, rr = residuals(M)
        res.append(math.sqrt(rr))
        if rr == 0.0:
            break
        cols = []
        for j, (rr_, rv_) in enumerate(R):
            if use_pi:
                z = [(int(r), _rv(pi[r] * v, mixed)) for r, v in zip(rr_, rv_)]
                z = [(r, v) for r, v in z if v != 0.0]
                cols.append((np.array([r for r, _ in z], np.int64), np.array([v for _, v in z])))
            else:
                cols.append((np.asarray(rr_, np.int64), np.asarray(rv_, np.float64)))
        P = hard_threshold(n, _to_csc(n, cols), m_dir)
        rq_p, qq_p = [], []
        for j in range(n):
            pr = P[1][P[0][j]:P[0][j + 1]]
            pv = P[2][P[0][j]:P[0][j + 1]]
            qr, qv = o.product_column(pr, pv)
            Rj = dict(zip(R[j][0].tolist(), R[j][1].tolist()))
            if use_pi:
                t1 = [(Rj[r] * q) * pi[r] for r, q in zip(qr.tolist(), qv.tolist()) if r in Rj]
                t2 = [(q * q) * pi[r] for r, q in zip(qr.tolist(), qv.tolist())]
            else:
                t1 = [Rj[r] * q for r, q in zip(qr.tolist(), qv.tolist()) if r in Rj]
                t2 = [q * q for q in qv.tolist()]
            rq_p.append(fixsum(np.array(t1)))
            qq_p.append(fixsum(np.array(t2)))
        rq, qq = pairwise(rq_p), pairwise(qq_p)
        if qq == 0.0:
            break
        alpha = rq / qq
        coef.append(alpha)
        newcols = []
        for j in range(n):
            a = dict(zip(M[1][M[0][j]:M[0][j + 1]].tolist(), M[2][M[0][j]:M[0][j + 1]].tolist()))
            b = dict(zip(P[1][P[0][j]:P[0][j + 1]].tolist(), P[2][P[0][j]:P[0][j + 1]].tolist()))
            rows = sorted(set(a) | set(b))
            vv = [_rv(_fma(alpha, b.get(r, 0.0), a.get(r, 0.0)), mixed) for r in rows]
            keep = [(r, v) for r, v in zip(rows, vv) if v != 0.0]
            newcols.append((np.array([r for r, _ in keep], np.int64), np.array([v for _, v in keep])))
        M = heuristic(n, rowptr, colind, vals, _to_csc(n, newcols), m_M, mixed=mixed)
        done += 1
    if done == iters:
        _, rr = residuals(M)
        res.append(math.sqrt(rr))
    return dict(M=M, resnorm=np.array(res), coef=np.array(coef), done=done)


# ---------------------------------------------------------------------------
# LOMR and CG with the same global dropping inside every iteration.  Columns
# are held as {row: value} dicts; inner products are the column pass's
# (exact terms x*y, or (x*y)*pi_k with Pi, summed by fixsum per column and
# pairwise over columns).

def _dicts(X):
    cp, ri, va = X
    return [dict(zip(ri[cp[j]:cp[j + 1]].tolist(), va[cp[j]:cp[j + 1]].tolist()))
            for j in range(len(cp) - 1)]


def _csc(n, cols):
    out = []
    for c in cols:
        rows = sorted(r for r, v in c.items() if v != 0.0)
        out.append((np.array(rows, np.int64), np.array([c[r] for r in rows])))
    return _to_csc(n, out)


def _inner(cols_x, cols_y, w=None):
    """sum_j (X_j, Y_j) (weighted by w = diag(Pi) when given)."""
    from oracle import fixsum, pairwise
    parts = []
    for x, y in zip(cols_x, cols_y):
        rows = [r for r in x if r in y]
        t = [(x[r] * y[r]) * w[r] if w is not None else x[r] * y[r] for r in rows]
        parts.append(fixsum(np.array(t)))
    return pairwise(parts)


def _setup(n, rowptr, colind, vals, mixed):
    from oracle import Oracle
    o = Oracle(n, rowptr, colind, vals, mixed=mixed, cap_factor=float(n))
    diag = np.zeros(n)
    for i in range(n):
        for q in range(rowptr[i], rowptr[i + 1]):
            if colind[q] == i:
                diag[i] = vals[q]
    return o, 1.0 / diag


def _residual(o, n, M):
    """R = I - A M column by column (the method's arithmetic) as dicts."""
    o.set_M(*M)
    out = []
    for j in range(n):
        r, v = o.column_residual(j)
        out.append(dict(zip(r.tolist(), v.tolist())))
    return out


def _product(o, n, X):
    """A X_j for every column (the method's arithmetic) as dicts."""
    out = []
    for c in X:
        rows = sorted(c)
        r, v = o.product_column(np.array(rows, np.int64), np.array([c[k] for k in rows]))
        out.append(dict(zip(r.tolist(), v.tolist())))
    return out


def _scaled(R, pi, use_pi, mixed):
    """(Pi) R, rounded to the value type, exact zeros removed."""
    if not use_pi:
        return [dict(c) for c in R]
    return [{r: _rv(pi[r] * v, mixed) for r, v in c.items() if _rv(pi[r] * v, mixed) != 0.0}
            for c in R]


def run_global_lomr(n, rowptr, colind, vals, iters, m_dir, m_M, mixed=False, use_pi=False):
    """LOMR (Algorithm 4; LOMR_SPD, Algorithm 8, with Pi = diag(A)^{-1}) with
    global dropping in every iteration: Z_i = the m_dir largest entries of
    (Pi) R_i over the whole matrix; delta_i, gamma_i minimise over
    span{A Z_i, A P_{i-1}} (Theorem 3; the paper does not treat a singular
    2x2 system, so an MR step is taken when c <= 64 eps uu vv or vv = 0);
    S_i = delta_i Z_i + gamma_i P_{i-1};
    P_i = the m_dir largest entries of S_i; M_{i+1} = Appendix A's heuristic
    of M_i + S_i with density cap m_M.  Returns dict(M, resnorm, coef, done,
    fallback)."""
    import math
    o, pi = _setup(n, rowptr, colind, vals, mixed)
    w = pi if use_pi else None
    M = o.get_M()
    P = [dict() for _ in range(n)]  # P_{-1} = 0
    res, coef = [], []
    done, fallback = 0, False
    eps = 2.220446049250313e-16
    for i in range(iters):
        R = _residual(o, n, M)
        rr = _inner(R, R)
        res.append(math.sqrt(rr))
        if rr == 0.0:
            break
        Z = _dicts(hard_threshold(n, _csc(n, _scaled(R, pi, use_pi, mixed)), m_dir))
        U, V = _product(o, n, Z), _product(o, n, P)
        uu, vv, uv = _inner(U, U, w), _inner(V, V, w), _inner(U, V, w)
        ur, vr = _inner(U, R, w), _inner(V, R, w)
        if uu == 0.0:
            break
        t1, t2 = uu * vv, uv * uv
        c = t1 - t2
        if vv == 0.0 or c <= (64.0 * eps) * t1:
            delta, gamma = ur / uu, 0.0
            fallback |= vv != 0.0
        else:
            delta, gamma = (vv * ur - uv * vr) / c, (uu * vr - uv * ur) / c
        if not (math.isfinite(delta) and math.isfinite(gamma)):
            break
        coef.append((delta, gamma))
        S = []
        for z, p in zip(Z, P):
            S.append({r: _rv(_fma(delta, z.get(r, 0.0), gamma * p.get(r, 0.0)), mixed)
                      for r in set(z) | set(p)})
        S = [{r: v for r, v in s.items() if v != 0.0} for s in S]
        T = []
        for m, s in zip(_dicts(M), S):
            T.append({r: _rv(m.get(r, 0.0) + s.get(r, 0.0), mixed) for r in set(m) | set(s)})
        P = _dicts(hard_threshold(n, _csc(n, S), m_dir))
        M = heuristic(n, rowptr, colind, vals, _csc(n, T), m_M, mixed=mixed)
        done += 1
    if done == iters:
        R = _residual(o, n, M)
        res.append(math.sqrt(_inner(R, R)))
    return dict(M=M, resnorm=np.array(res), coef=np.array(coef).reshape(-1, 2), done=done,
                fallback=fallback)


def run_global_cg(n, rowptr, colind, vals, iters, m_dir, m_M, mixed=False, use_pi=False):
    """CG on the Frobenius inner product (Algorithm 3; Algorithm 7 with
    Pi = diag(A)^{-1}) with global dropping in every iteration:
    P_0 = the m_dir largest entries of (Pi) R_0; alpha_i = (R_i, (Pi) R_i) /
    (P_i, A P_i); M_{i+1} = Appendix A's heuristic of M_i + alpha_i P_i with
    density cap m_M; R_{i+1} = I - A M_{i+1}; beta_i = (R_{i+1}, (Pi) R_{i+1})
    / (R_i, (Pi) R_i); P_{i+1} = the m_dir largest entries of
    (Pi) R_{i+1} + beta_i P_i.  Returns dict(M, resnorm, coef, done)."""
    import math
    o, pi = _setup(n, rowptr, colind, vals, mixed)
    w = pi if use_pi else None
    M = o.get_M()
    R = _residual(o, n, M)
    rr = _inner(R, R)
    res, coef = [math.sqrt(rr)], []
    rz = _inner(R, R, w) if use_pi else rr
    P = _dicts(hard_threshold(n, _csc(n, _scaled(R, pi, use_pi, mixed)), m_dir))
    done = 0
    for i in range(iters):
        if rz == 0.0:
            break
        Q = _product(o, n, P)
        pq = _inner(P, Q)
        if pq == 0.0:
            break
        alpha = rz / pq
        if not math.isfinite(alpha):
            break
        T = []
        for m, p in zip(_dicts(M), P):
            T.append({r: _rv(_fma(alpha, p.get(r, 0.0), m.get(r, 0.0)), mixed) for r in set(m) | set(p)})
        M = heuristic(n, rowptr, colind, vals, _csc(n, T), m_M, mixed=mixed)
        R = _residual(o, n, M)
        rr1 = _inner(R, R)
        res.append(math.sqrt(rr1))
        rz1 = _inner(R, R, w) if use_pi else rr1
        beta = rz1 / rz
        coef.append((alpha, beta))
        done += 1
        if rz1 == 0.0:
            break
        Zs = _scaled(R, pi, use_pi, mixed)
        C = []
        for z, p in zip(Zs, P):
            C.append({r: _rv(_fma(beta, p.get(r, 0.0), z.get(r, 0.0)), mixed) for r in set(z) | set(p)})
        P = _dicts(hard_threshold(n, _csc(n, C), m_dir))
        rz = rz1
    return dict(M=M, resnorm=np.array(res), coef=np.array(coef).reshape(-1, 2), done=done)
