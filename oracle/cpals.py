"""CP-ALS (Algorithm 1) in FP64 numpy on top of the C oracle's MTTKRP --
TEST INFRASTRUCTURE (see the package docstring).

Per sweep and per mode n (Algorithm 1):
  V   = Hadamard product of the Grams A_k^T A_k, k != n
  M   = MTTKRP of mode n (Eq. 1), FP64
  A_n = M V^+  (Cholesky solve of the symmetric V; eigen-pseudo-inverse when
                a Cholesky pivot is <= R * eps * max_i V_ii, i.e. V is not
                numerically positive definite)
Readings added to Algorithm 1, which states neither: after each update the
columns of A_n are scaled to unit 2-norm and the norms kept as lambda; the
fit after a sweep is 1 - ||X - Xhat|| / ||X|| with ||Xhat||^2 from the Grams
and <X, Xhat> from the last mode's M.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def gram(A: np.ndarray) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    return A.T @ A


def pd_tolerance(V: np.ndarray) -> float:
    """Smallest Cholesky pivot accepted as positive: R * eps * max_i V_ii.
    A pivot at or below it means V is treated as not positive definite
    (numerically singular or indefinite) and the pseudo-inverse is used."""
    V = np.asarray(V, dtype=np.float64)
    return V.shape[0] * np.finfo(np.float64).eps * max(float(np.max(np.diag(V))), 0.0)


def cholesky_lower(V: np.ndarray):
    """Right-looking Cholesky V = L L^T of symmetric V, in the order of the
    textbook algorithm: pivot j, scale column j below it, update the trailing
    lower triangle. Returns L, or None as soon as a pivot is <= pd_tolerance(V)."""
    V = np.asarray(V, dtype=np.float64)
    R = V.shape[0]
    tol = pd_tolerance(V)
    L = np.tril(V).copy()
    for j in range(R):
        d = L[j, j]
        if not d > tol:
            return None
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] /= L[j, j]
        # trailing update of the lower triangle: L[i,k] -= L[i,j] L[k,j], k <= i
        L[j + 1:, j + 1:] -= np.tril(np.outer(L[j + 1:, j], L[j + 1:, j]))
    return L


def pinv_sym(V: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse of symmetric V from its eigen-decomposition
    V = Q diag(w) Q^T: V^+ = Q diag(w^+) Q^T, where w^+ = 1/w for
    |w| > max|w| * R * eps and 0 otherwise."""
    V = np.asarray(V, dtype=np.float64)
    w, Q = np.linalg.eigh(V)
    cut = np.max(np.abs(w)) * V.shape[0] * np.finfo(np.float64).eps
    keep = np.abs(w) > cut
    winv = np.zeros_like(w)
    winv[keep] = 1.0 / w[keep]
    return (Q * winv) @ Q.T


def solve_right(M: np.ndarray, V: np.ndarray) -> Tuple[np.ndarray, int]:
    """A = M V^+ for symmetric V (the update of Algorithm 1). If every
    Cholesky pivot of V exceeds pd_tolerance(V), A solves A V = M by forward
    and back substitution with L (info 0); otherwise A = M pinv_sym(V)
    (info 1)."""
    M = np.asarray(M, dtype=np.float64)
    L = cholesky_lower(V)
    if L is not None:
        Y = np.linalg.solve(L, M.T)          # L Y = M^T
        return np.linalg.solve(L.T, Y).T, 0  # L^T Z = Y, A = Z^T
    return M @ pinv_sym(V), 1


def fit_of(normX2: float, lam: np.ndarray, grams: Sequence[np.ndarray], M_last: np.ndarray,
           A_last: np.ndarray) -> float:
    V = np.ones_like(grams[0])
    for G in grams:
        V = V * G
    normXhat2 = float(lam @ V @ lam)
    inner = float(np.sum(lam * np.sum(M_last * A_last, axis=0)))
    resid2 = max(normX2 + normXhat2 - 2.0 * inner, 0.0)
    return 1.0 - np.sqrt(resid2) / np.sqrt(normX2)


def cp_als(coords, vals, dims, factors0: Sequence[np.ndarray], iters: int
           ) -> Tuple[List[np.ndarray], np.ndarray, List[float]]:
    from . import mttkrp  # the C oracle

    N = len(dims)
    A = [np.array(f, dtype=np.float64, copy=True) for f in factors0]
    R = A[0].shape[1]
    lam = np.ones(R)
    G = [gram(a) for a in A]
    x = np.asarray(vals, dtype=np.float64)
    normX2 = float(x @ x)
    fits: List[float] = []
    for _ in range(int(iters)):
        M = None
        for n in range(N):
            V = np.ones((R, R))
            for k in range(N):
                if k != n:
                    V = V * G[k]
            M, _ = mttkrp(coords, x, dims, A, n)
            An, _ = solve_right(M, V)
            lam = np.linalg.norm(An, axis=0)
            lam_safe = np.where(lam == 0, 1.0, lam)
            An = An / lam_safe
            A[n] = An
            G[n] = gram(An)
        fits.append(fit_of(normX2, lam, G, M, A[N - 1]))
    return A, lam, fits
