"""Dense symmetric-definite eigensolver written out from the mathematics --
TEST INFRASTRUCTURE.

An independent check of the oracle's reduced eigensolve (Fig. 2 step 4,
Eqs. 6 and 8: A_Q Phi = eps B_Q Phi with B_Q-orthonormal Phi) and of the whole
loop on tiny pencils.  It calls no LAPACK routine, so a mistake in how the
oracle uses LAPACK (or in LAPACK's driver selection) cannot hide behind it.

  * B = L L^T by the Cholesky recurrence (plain loops);
  * C = L^{-1} A L^{-T} by forward substitution on both sides;
  * C = V diag(eps) V^T by the cyclic Jacobi method: sweeps over every
    off-diagonal pair (p, q) in row order, each pair annihilated by the plane
    rotation whose tangent t solves t^2 + 2 tau t - 1 = 0,
    tau = (c_qq - c_pp) / (2 c_pq), taking the root of smaller magnitude;
  * Phi = L^{-T} V, so that Phi^T B Phi = V^T V = I and A Phi = B Phi diag(eps).

Loops are plain Python over pairs with numpy row/column updates: fine for the
tiny sizes (N <= a few hundred) it is used at.
"""

from __future__ import annotations

import math

import numpy as np


class JacobiNoConvergence(RuntimeError):
    """The sweep cap was reached before the off-diagonal part vanished."""


def rotation(app: float, aqq: float, apq: float):
    """(c, s) of the plane rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s)
    for which (J^T A J)_pq = 0: with t = s / c the condition
    (c^2 - s^2) a_pq + c s (a_pp - a_qq) = 0 becomes t^2 + 2 tau t - 1 = 0."""
    tau = (aqq - app) / (2.0 * apq)
    sgn = 1.0 if tau >= 0.0 else -1.0
    t = sgn / (abs(tau) + math.sqrt(1.0 + tau * tau))
    c = 1.0 / math.sqrt(1.0 + t * t)
    return c, t * c


def off_norm(A: np.ndarray) -> float:
    """Frobenius norm of the off-diagonal part."""
    return float(np.sqrt(max(0.0, (A * A).sum() - (np.diag(A) ** 2).sum())))


def jacobi_symmetric(S: np.ndarray, max_sweeps: int = 60):
    """All eigenpairs of a real symmetric matrix: (eigenvalues ascending,
    orthonormal eigenvectors as columns).  A pair is rotated unless its entry
    is already negligible: |a_pq| <= u sqrt(|a_pp a_qq|) (u = 2^-52, the
    criterion that keeps every eigenvalue accurate to its own scale) or
    |a_pq| <= 1e-3 u ||A||_F; the iteration ends after a sweep with no
    rotation."""
    A = np.array(S, dtype=np.float64, copy=True)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    A = 0.5 * (A + A.T)
    V = np.eye(n)
    u = 2.0 ** -52
    floor = 1e-3 * u * float(np.sqrt((A * A).sum()))
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if abs(apq) <= u * math.sqrt(abs(A[p, p] * A[q, q])) or abs(apq) <= floor:
                    continue
                rotated = True
                c, s = rotation(A[p, p], A[q, q], apq)
                rp, rq = A[p, :].copy(), A[q, :].copy()          # A <- J^T A
                A[p, :] = c * rp - s * rq
                A[q, :] = s * rp + c * rq
                cp, cq = A[:, p].copy(), A[:, q].copy()          # A <- A J
                A[:, p] = c * cp - s * cq
                A[:, q] = s * cp + c * cq
                vp, vq = V[:, p].copy(), V[:, q].copy()          # V <- V J
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    else:
        raise JacobiNoConvergence(f"off-diagonal norm {off_norm(A):.3e} after {max_sweeps} sweeps")
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def cholesky_lower(B: np.ndarray) -> np.ndarray:
    """L with B = L L^T (B symmetric positive definite): column by column,
    l_jj = sqrt(b_jj - sum_k<j l_jk^2), l_ij = (b_ij - sum_k<j l_ik l_jk) / l_jj."""
    n = B.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        d = B[j, j] - float(L[j, :j] @ L[j, :j])
        if not d > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (B[i, j] - float(L[i, :j] @ L[j, :j])) / L[j, j]
    return L


def forward_substitute(L: np.ndarray, R: np.ndarray) -> np.ndarray:
    """L^{-1} R for lower triangular L, row by row."""
    X = np.zeros_like(R, dtype=np.float64)
    for i in range(L.shape[0]):
        X[i] = (R[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def back_substitute_transposed(L: np.ndarray, R: np.ndarray) -> np.ndarray:
    """L^{-T} R for lower triangular L (L^T is upper triangular), last row first."""
    n = L.shape[0]
    X = np.zeros_like(R, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        X[i] = (R[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X


def jacobi_generalized_eigh(A: np.ndarray, B: np.ndarray, max_sweeps: int = 60):
    """Eigenpairs of A phi = eps B phi (A symmetric, B s.p.d.) with
    B-orthonormal phi: eigenvalues ascending and Phi (columns)."""
    A = 0.5 * (np.asarray(A, dtype=np.float64) + np.asarray(A, dtype=np.float64).T)
    B = 0.5 * (np.asarray(B, dtype=np.float64) + np.asarray(B, dtype=np.float64).T)
    L = cholesky_lower(B)
    C = forward_substitute(L, forward_substitute(L, A).T)      # L^{-1} A L^{-T}
    eps, V = jacobi_symmetric(C, max_sweeps=max_sweeps)
    Phi = back_substitute_transposed(L, V)
    return eps, Phi
