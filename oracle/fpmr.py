"""Oracle for differentiating fixed-pattern MR (test infrastructure only).

K steps of MR on the fixed pattern S = supp(A) (Algorithm 1 with the
direction restricted to S):
    M_0 = diag(A)^{-1};  R_i = I - A M_i;  P_i = mask_S(R_i);  Q_i = A P_i;
    alpha_i = (R_i, Q_i)_F / (Q_i, Q_i)_F;  M_{i+1} = M_i + alpha_i P_i;
    L = ||I - A M_K||_F^2,
with the stored values of A as independent entries, and its gradient by
reverse-mode differentiation of those steps (adjoints written out by hand,
FP64, scipy.sparse products).  The gradient form of the objective,
d||I - A M||^2 / dM = -2 A^T R, is the paper's Eq. (gradient) in Sec. 3.
"""
import numpy as np
import scipy.sparse as sp


def _mask(X, S):
    """X restricted to the pattern of S (a 0/1 CSR of the same shape)."""
    return X.multiply(S).tocsr()


def forward(n, rowptr, colind, vals, K, keep=False):
    A = sp.csr_matrix((np.asarray(vals, dtype=np.float64), colind, rowptr), shape=(n, n))
    S = sp.csr_matrix((np.ones(len(vals)), colind, rowptr), shape=(n, n))
    I = sp.identity(n, format="csr")
    M = sp.diags(1.0 / A.diagonal()).tocsr()
    Ms, alphas = [M], []
    for _ in range(K):
        R = (I - A @ M).tocsr()
        P = _mask(R, S)
        Q = (A @ P).tocsr()
        num = R.multiply(Q).sum()
        den = Q.multiply(Q).sum()
        alpha = num / den
        M = (M + alpha * P).tocsr()
        Ms.append(M)
        alphas.append((alpha, num, den))
    R = (I - A @ M).tocsr()
    loss = float(R.multiply(R).sum())
    if keep:
        return loss, dict(A=A, S=S, I=I, Ms=Ms, alphas=alphas)
    return loss


def gradient(n, rowptr, colind, vals, K):
    """(loss, dL/d vals) with dL/dvals in A's CSR order."""
    loss, st = forward(n, rowptr, colind, vals, K, keep=True)
    A, S, I, Ms, alphas = st["A"], st["S"], st["I"], st["Ms"], st["alphas"]
    dA = sp.csr_matrix((n, n))
    R = (I - A @ Ms[K]).tocsr()
    dR = 2.0 * R
    dA = dA - _mask(dR @ Ms[K].T, S)
    dM = -_mask(A.T @ dR, S)
    for i in range(K - 1, -1, -1):
        M = Ms[i]
        alpha, num, den = alphas[i]
        R = (I - A @ M).tocsr()
        P = _mask(R, S)
        Q = (A @ P).tocsr()
        dP = alpha * dM
        dalpha = dM.multiply(P).sum()
        dnum = dalpha / den
        dden = -dalpha * alpha / den
        dR = dnum * Q
        dQ = dnum * R + 2.0 * dden * Q
        dA = dA + _mask(dQ @ P.T, S)
        dP = dP + _mask(A.T @ dQ, S)
        dR = dR + dP
        dA = dA - _mask(dR @ M.T, S)
        dM = dM - _mask(A.T @ dR, S)
    d = A.diagonal()
    dA = dA - sp.diags(dM.diagonal() / (d * d))
    dA = _mask(dA.tocsr(), S)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    out = np.asarray(dA[rows, np.asarray(colind)]).ravel()
    return loss, out


# ------------------------------------------------- fixed-pattern LOMR
# K steps of LOMR (Algorithm 4, the 2-D minimiser of Theorem 3) on the fixed
# pattern S = supp(A):
#   M_0 = diag(A)^{-1};  P_{-1} = 0;  R_i = I - A M_i;  Z_i = mask_S(R_i);
#   U = A Z_i;  V = A P_{i-1};  uu, vv, uv, ur, vr the Frobenius products;
#   c = uu vv - uv^2;  delta = (vv ur - uv vr) / c,  gamma = (uu vr - uv ur) / c,
#   or the MR step delta = ur / uu, gamma = 0 when vv = 0 (i = 0) or
#   c <= 64 eps uu vv (the library's fallback);
#   S_i = delta Z_i + gamma P_{i-1};  M_{i+1} = M_i + S_i;  P_i = S_i;
#   L = ||I - A M_K||_F^2.
# Every M_i, P_i lives on S, so no dropping is needed.

_EPS = 2.220446049250313e-16


def _fro(X, Y):
    return float(X.multiply(Y).sum())


def _lomr_coef(uu, vv, uv, ur, vr):
    """(delta, gamma, mr_step) of one LOMR step."""
    c = uu * vv - uv * uv
    if vv == 0.0 or c <= 64.0 * _EPS * (uu * vv):
        return ur / uu, 0.0, True
    return (vv * ur - uv * vr) / c, (uu * vr - uv * ur) / c, False


def forward_lomr(n, rowptr, colind, vals, K, keep=False):
    A = sp.csr_matrix((np.asarray(vals, dtype=np.float64), colind, rowptr), shape=(n, n))
    S = sp.csr_matrix((np.ones(len(vals)), colind, rowptr), shape=(n, n))
    I = sp.identity(n, format="csr")
    M = sp.diags(1.0 / A.diagonal()).tocsr()
    P = sp.csr_matrix((n, n))
    Ms, Ps, coefs = [M], [P], []
    for _ in range(K):
        R = (I - A @ M).tocsr()
        Z = _mask(R, S)
        U = (A @ Z).tocsr()
        V = (A @ P).tocsr()
        d, g, mr = _lomr_coef(_fro(U, U), _fro(V, V), _fro(U, V), _fro(U, R), _fro(V, R))
        St = (d * Z + g * P).tocsr()
        M = (M + St).tocsr()
        P = St
        Ms.append(M)
        Ps.append(P)
        coefs.append((d, g, mr))
    R = (I - A @ M).tocsr()
    loss = float(R.multiply(R).sum())
    if keep:
        return loss, dict(A=A, S=S, I=I, Ms=Ms, Ps=Ps, coefs=coefs)
    return loss


def gradient_lomr(n, rowptr, colind, vals, K):
    """(loss, dL/d vals) of K fixed-pattern LOMR steps, reverse mode written
    out by hand: for step i, with dS = dM_{i+1} + dP_i,
      d(delta) = (dS, Z), d(gamma) = (dS, P_{i-1}), dZ = delta dS,
      dP_{i-1} = gamma dS;  the products' adjoints from the derivatives of
      delta = (vv ur - uv vr)/c and gamma = (uu vr - uv ur)/c (or of
      delta = ur/uu on an MR step);  dU = 2 duu U + duv V + dur R,
      dV = 2 dvv V + duv U + dvr R, dR = dur U + dvr V;  then through
      U = A Z, V = A P_{i-1}, Z = mask_S(R), R = I - A M_i."""
    loss, st = forward_lomr(n, rowptr, colind, vals, K, keep=True)
    A, S, I, Ms, Ps, coefs = st["A"], st["S"], st["I"], st["Ms"], st["Ps"], st["coefs"]
    R = (I - A @ Ms[K]).tocsr()
    dR = 2.0 * R
    dA = -_mask(dR @ Ms[K].T, S)
    dM = -_mask(A.T @ dR, S)
    dPn = sp.csr_matrix((n, n))  # adjoint of P_i as the next step's P_{i-1}
    for i in range(K - 1, -1, -1):
        M, Pp = Ms[i], Ps[i]
        d, g, mr = coefs[i]
        R = (I - A @ M).tocsr()
        Z = _mask(R, S)
        U = (A @ Z).tocsr()
        V = (A @ Pp).tocsr()
        uu, vv, uv, ur, vr = _fro(U, U), _fro(V, V), _fro(U, V), _fro(U, R), _fro(V, R)
        dS = (dM + dPn).tocsr()
        dd = _fro(dS, Z)
        dg = _fro(dS, Pp)
        dZ = d * dS
        dPp = g * dS
        if mr:
            duu, dvv, duv, dur, dvr = -dd * d / uu, 0.0, 0.0, dd / uu, 0.0
        else:
            c = uu * vv - uv * uv
            duu = (dd * (-d * vv) + dg * (vr - g * vv)) / c
            dvv = (dd * (ur - d * uu) + dg * (-g * uu)) / c
            duv = (dd * (-vr + 2.0 * d * uv) + dg * (-ur + 2.0 * g * uv)) / c
            dur = (dd * vv - dg * uv) / c
            dvr = (-dd * uv + dg * uu) / c
        dU = 2.0 * duu * U + duv * V + dur * R
        dV = 2.0 * dvv * V + duv * U + dvr * R
        dRi = dur * U + dvr * V
        dA = dA + _mask(dU @ Z.T, S) + _mask(dV @ Pp.T, S)
        dZ = dZ + _mask(A.T @ dU, S)
        dPp = dPp + _mask(A.T @ dV, S)
        dRi = dRi + dZ
        dA = dA - _mask(dRi @ M.T, S)
        dM = dM - _mask(A.T @ dRi, S)
        dPn = dPp
    d = A.diagonal()
    dA = dA - sp.diags(dM.diagonal() / (d * d))
    dA = _mask(dA.tocsr(), S)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    out = np.asarray(dA[rows, np.asarray(colind)]).ravel()
    return loss, out
