"""CP-ALS (Algorithm 1) in FP64 numpy on top of the C oracle's MTTKRP --
TEST INFRASTRUCTURE (see the package docstring).

Per sweep and per mode n (Algorithm 1):
  V   = Hadamard product of the Grams A_k^T A_k, k != n
  M   = MTTKRP of mode n (Eq. 1), FP64
  A_n = M V^+  (Cholesky solve of the symmetric V; eigen-pseudo-inverse when
                V is not positive definite)
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


def solve_right(M: np.ndarray, V: np.ndarray) -> np.ndarray:
    """A = M V^+ for symmetric V."""
    try:
        L = np.linalg.cholesky(V)
        Y = np.linalg.solve(L, M.T)          # L Y = M^T
        return np.linalg.solve(L.T, Y).T     # L^T Z = Y, A = Z^T
    except np.linalg.LinAlgError:
        w, Q = np.linalg.eigh(V)
        cut = np.max(np.abs(w)) * V.shape[0] * np.finfo(np.float64).eps
        winv = np.where(np.abs(w) > cut, 1.0 / np.where(w == 0, 1.0, w), 0.0)
        return M @ (Q * winv) @ Q.T


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
            An = solve_right(M, V)
            lam = np.linalg.norm(An, axis=0)
            lam_safe = np.where(lam == 0, 1.0, lam)
            An = An / lam_safe
            A[n] = An
            G[n] = gram(An)
        fits.append(fit_of(normX2, lam, G, M, A[N - 1]))
    return A, lam, fits
