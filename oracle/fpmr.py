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
