"""CPU tile low-rank (TLR) reference -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. V: Sigma is split into nb x nb tiles (the last one ragged); diagonal tiles
stay dense and every off-diagonal tile (i, j), i > j, is replaced by U_ij V_ij^T
keeping the singular values above an absolute threshold eps (rank k_ij varies
per tile).  The paper leaves the TLR Cholesky itself to its citations; this is
the plain right-looking tile algorithm on that format, written step by step:

  for k = 0 .. nt-1:
      D_k  <- chol(D_k)                               dense POTRF
      V_ik <- D_k^{-1} V_ik            (i > k)        TRSM: L_ik = U_ik (D_k^{-1} V_ik)^T
      D_i  <- D_i - U_ik (V_ik^T V_ik) U_ik^T (i > k) SYRK
      A_ij <- trunc_eps([U_ij, -U_ik W][V_ij, U_jk]^T),  W = V_ik^T V_jk   (i > j > k)

trunc_eps recompresses through QR of both factors and an SVD of the small
core, keeping singular values > eps (the same absolute rule as the initial
compression).  log|Sigma| = 2 sum log diag(D_k) and z^T Sigma^{-1} z = ||L^{-1} z||^2
follow from tile forward substitution (eq. 1).

Points are first put in Morton (Z-curve) order so that tiles are spatially
compact; the likelihood does not depend on the order (tested).

Pins: tests/test_oracle_tlr.py (eps = 0 equals dense, nt = 1 equals dense,
rank/threshold rule against numpy SVD, solves against dense triangular solves).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from . import dense as DN


def morton_permutation(x, y, bits: int = 16) -> np.ndarray:
    """Indices that sort points along the Z-order curve of their bounding square.

    Coordinates are scaled by the larger side of the bounding box, quantised to
    2^bits levels per axis and bit-interleaved (x in even bits, y in odd bits);
    ties keep the original order.
    """
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    x0, y0 = x.min(), y.min()
    ext = max(x.max() - x0, y.max() - y0)
    scale = (2 ** bits) / ext if ext > 0 else 0.0
    top = 2 ** bits - 1
    qx = np.minimum(np.floor((x - x0) * scale), top).astype(np.uint64)
    qy = np.minimum(np.floor((y - y0) * scale), top).astype(np.uint64)
    key = np.zeros(len(x), dtype=np.uint64)
    for b in range(bits):
        key |= ((qx >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((qy >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return np.argsort(key, kind="stable")


def _trunc(U, V, eps):
    """Truncated SVD of U V^T keeping singular values > eps: returns (U s, V)."""
    if U.shape[1] == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    X, s, Yt = np.linalg.svd(Ru @ Rv.T)
    k = int(np.sum(s > eps))
    return Qu @ (X[:, :k] * s[:k]), Qv @ Yt[:k].T


class TLRMatrix:
    """Lower-triangular TLR storage: dense D[i], low-rank (U[i,j], V[i,j]) for i > j."""

    def __init__(self, n, nb):
        self.n, self.nb = n, nb
        self.nt = (n + nb - 1) // nb
        self.D = [None] * self.nt
        self.U = {}
        self.V = {}
        self.max_rank = 0

    def rows(self, i):
        return slice(i * self.nb, min((i + 1) * self.nb, self.n))

    def ranks(self):
        return {ij: u.shape[1] for ij, u in self.U.items()}


def compress(S: np.ndarray, nb: int, eps: float) -> TLRMatrix:
    """Sec. V: tile S and replace each off-diagonal tile by its eps-truncated SVD."""
    n = S.shape[0]
    T = TLRMatrix(n, nb)
    for i in range(T.nt):
        T.D[i] = S[T.rows(i), T.rows(i)].copy()
        for j in range(i):
            A = S[T.rows(i), T.rows(j)]
            Uf, s, Vt = np.linalg.svd(A, full_matrices=False)
            k = int(np.sum(s > eps))
            T.U[i, j] = Uf[:, :k] * s[:k]
            T.V[i, j] = Vt[:k].T.copy()
    return T


def cholesky(T: TLRMatrix, eps: float) -> TLRMatrix:
    """Right-looking TLR Cholesky in place (see module docstring)."""
    nt = T.nt
    for k in range(nt):
        T.D[k] = sl.cholesky(T.D[k], lower=True)
        for i in range(k + 1, nt):
            T.V[i, k] = sl.solve_triangular(T.D[k], T.V[i, k], lower=True)
        for i in range(k + 1, nt):
            U, V = T.U[i, k], T.V[i, k]
            T.D[i] = T.D[i] - U @ (V.T @ V) @ U.T
        for i in range(k + 2, nt):
            for j in range(k + 1, i):
                W = T.V[i, k].T @ T.V[j, k]
                Up = np.hstack([T.U[i, j], -T.U[i, k] @ W])
                Vp = np.hstack([T.V[i, j], T.U[j, k]])
                T.U[i, j], T.V[i, j] = _trunc(Up, Vp, eps)
                T.max_rank = max(T.max_rank, T.U[i, j].shape[1])
    return T


def forward_solve(T: TLRMatrix, z: np.ndarray) -> np.ndarray:
    """y = L^{-1} z by tile forward substitution on the TLR factor."""
    y = np.array(z, dtype=np.float64, copy=True)
    for i in range(T.nt):
        r = y[T.rows(i)]
        for j in range(i):
            r = r - T.U[i, j] @ (T.V[i, j].T @ y[T.rows(j)])
        y[T.rows(i)] = sl.solve_triangular(T.D[i], r, lower=True)
    return y


def backward_solve(T: TLRMatrix, y: np.ndarray) -> np.ndarray:
    """x = L^{-T} y by tile backward substitution on the TLR factor."""
    x = np.array(y, dtype=np.float64, copy=True)
    for i in range(T.nt - 1, -1, -1):
        r = x[T.rows(i)]
        for k in range(i + 1, T.nt):
            r = r - T.V[k, i] @ (T.U[k, i].T @ x[T.rows(k)])
        x[T.rows(i)] = sl.solve_triangular(T.D[i], r, lower=True, trans="T")
    return x


def logdet(T: TLRMatrix) -> float:
    return float(2.0 * np.sum(np.concatenate([np.log(np.diag(D)) for D in T.D])))


def factor(x, y, theta, nb, eps, order=True):
    """Morton-order, generate, compress and factor; returns (T, perm)."""
    perm = morton_permutation(x, y) if order else np.arange(len(x))
    xs, ys = np.asarray(x)[perm], np.asarray(y)[perm]
    T = compress(DN.covariance(xs, ys, theta), nb, eps)
    return cholesky(T, eps), perm


def loglik(x, y, z, theta, nb, eps, order=True):
    """Eq. 1 on the TLR factor; returns (l, log|Sigma|, quad, T)."""
    T, perm = factor(x, y, theta, nb, eps, order)
    n = len(z)
    w = forward_solve(T, np.asarray(z)[perm])
    ld = logdet(T)
    quad = float(w @ w)
    ll = -0.5 * n * np.log(2.0 * np.pi) - 0.5 * ld - 0.5 * quad
    return ll, ld, quad, T


def krige(x_obs, y_obs, z_obs, x_new, y_new, theta, nb, eps):
    """Eq. 4 with Sigma_22^{-1} z_obs from the TLR factor (forward + backward)."""
    T, perm = factor(x_obs, y_obs, theta, nb, eps)
    a = backward_solve(T, forward_solve(T, np.asarray(z_obs)[perm]))
    S12 = DN.covariance(x_new, y_new, theta, np.asarray(x_obs)[perm], np.asarray(y_obs)[perm])
    return S12 @ a
