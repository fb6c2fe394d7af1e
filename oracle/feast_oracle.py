"""FEAST oracle: each function restates one passage of Polizzi, arXiv:0901.2665.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  float64 /
complex128 throughout; library primitives (sparse products, dense LU solves,
the LAPACK symmetric-definite eigensolver) serve as single steps, with no
blocking, fusion or reordering beyond the paper's own steps.

Readings of the paper taken here (the paper is silent or garbled on them):
  * RHS of the node solves is B*Y, with Y random in loop 1 and Y = X from the
    previous loop afterwards (Sec. III.B (i) sets Y = BX for the refinement).
  * Q carries the minus sign of Eq. 15 / Fig. 2 step 2 literally.
  * Convergence: relative change of the in-interval trace between consecutive
    loops, |t_k - t_{k-1}| <= tol * sum |lambda_m|, with an unchanged count;
    loop 1 never stops (Sec. III.B (i), Sec. IV.A).
  * B_Q counts as not s.p.d. when its smallest eigenvalue is <= 1e-14 times
    its largest (Sec. III.B (ii)).
  * The in-interval test is closed: lmin <= lambda <= lmax (Fig. 2 step 5).
  * Outputs are sorted ascending with the in-interval pairs first.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from workloads import STENCIL_OFFSETS


class BQNotSPD(RuntimeError):
    """B_Q = Q^T B Q lost positive definiteness: M0 too large (Sec. III.B (ii))."""


# ----------------------------------------------------------------------------
# Quadrature (Fig. 2 caption; Eqs. 13-14)
# ----------------------------------------------------------------------------

def _legendre_and_derivative(n: int, x: float):
    p_prev, p = 1.0, x
    for k in range(1, n):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    return p, dp


def gauss_legendre(Ne: int):
    """Ne-point Gauss-Legendre nodes x_e and weights w_e on [-1, 1].

    Newton iteration on the Legendre polynomial P_Ne from the classical
    starting points cos(pi (i - 1/4) / (Ne + 1/2)); weights
    w = 2 / ((1 - x^2) P'_Ne(x)^2).  Ordered as the paper prints the Ne=8 table
    (Fig. 2 caption): x_1 < x_3 < ... positive, x_{2i} = -x_{2i-1}; for odd Ne
    the zero node comes first."""
    if Ne < 1:
        raise ValueError("Ne must be >= 1")
    pos = []
    for i in range(1, Ne // 2 + 1):
        x = math.cos(math.pi * (i - 0.25) / (Ne + 0.5))
        for _ in range(100):
            p, dp = _legendre_and_derivative(Ne, x)
            dx = p / dp
            x -= dx
            if abs(dx) < 1e-17:
                break
        p, dp = _legendre_and_derivative(Ne, x)
        pos.append((x, 2.0 / ((1.0 - x * x) * dp * dp)))
    pos.sort()
    xs, ws = [], []
    if Ne % 2 == 1:
        _, dp = _legendre_and_derivative(Ne, 0.0)
        xs.append(0.0)
        ws.append(2.0 / (dp * dp))
    for x, w in pos:
        xs += [x, -x]
        ws += [w, w]
    return np.array(xs), np.array(ws)


def contour_points(lmin: float, lmax: float, Ne: int):
    """Nodes on the upper half circle C+ around [lmin, lmax] (Eqs. 13-14):
    r = (lmax - lmin)/2, theta_e = -(pi/2)(x_e - 1), Z_e = (lmax+lmin)/2 + r e^{i theta_e}.
    Returns (x, w, theta, Z, r)."""
    x, w = gauss_legendre(Ne)
    r = (lmax - lmin) / 2.0
    theta = -(math.pi / 2.0) * (x - 1.0)
    Z = (lmax + lmin) / 2.0 + r * np.exp(1j * theta)
    return x, w, theta, Z, r


def filter_value(lam, lmin: float, lmax: float, Ne: int):
    """Scalar rational filter that step 2 applies to an eigenvalue lam:
    with G(Z) = (Z B - A)^{-1} = X (Z - Lambda)^{-1} X^T on B-orthonormal X,
    Eq. 15 gives Q = X f(Lambda) X^T (B Y) with
    f(lam) = -sum_e (w_e / 2) Re{ r e^{i theta_e} / (Z_e - lam) }."""
    _, w, theta, Z, r = contour_points(lmin, lmax, Ne)
    lam = np.asarray(lam, dtype=np.float64)
    terms = (w / 2.0) * (r * np.exp(1j * theta) / (Z - lam[..., None])).real
    return -terms.sum(axis=-1)


# ----------------------------------------------------------------------------
# Operators (Eq. 2): assembled sparse matrices from the 27-point coefficients
# ----------------------------------------------------------------------------

def assemble(coef27: np.ndarray, nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Sparse matrix whose row i holds coef27[s, i] at column i + off(s)."""
    N = nx * ny * nz
    idx = np.arange(N, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols, vals = [], [], []
    for s, (dx, dy, dz) in enumerate(STENCIL_OFFSETS):
        ok = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
              & (iz + dz >= 0) & (iz + dz < nz))
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + nx * (dy + ny * dz))
        vals.append(coef27[s, ok])
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return M.tocsr()


def norm1(M: sp.spmatrix) -> float:
    """Matrix 1-norm: largest absolute column sum."""
    return float(abs(M).sum(axis=0).max())


# ----------------------------------------------------------------------------
# Step 2: node solves (Z_e B - A) Q_e = B Y and the quadrature sum (Eq. 15)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class BlockTridiagFactor:
    """Block Gaussian elimination of a block-tridiagonal matrix over its
    z-layers: S_1 = D_1, S_i = D_i - L_i S_{i-1}^{-1} U_{i-1}, with each dense
    S_i held as a partially pivoted LU factorisation (LAPACK getrf)."""
    n: int
    nb: int
    lower: list      # L_i = M[layer i, layer i-1], i >= 1
    upper: list      # U_i = M[layer i, layer i+1], i < nb-1
    lu: list         # getrf factors of S_i

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        n, nb = self.n, self.nb
        g = [None] * nb
        g[0] = rhs[0:n]
        for i in range(1, nb):
            g[i] = rhs[i * n:(i + 1) * n] - self.lower[i] @ sla.lu_solve(self.lu[i - 1], g[i - 1])
        x = [None] * nb
        x[nb - 1] = sla.lu_solve(self.lu[nb - 1], g[nb - 1])
        for i in range(nb - 2, -1, -1):
            x[i] = sla.lu_solve(self.lu[i], g[i] - self.upper[i] @ x[i + 1])
        return np.concatenate(x, axis=0)


def block_tridiag_factor(M: sp.csr_matrix, n: int, nb: int) -> BlockTridiagFactor:
    """Factor M (N = n*nb, couplings only between neighbouring layers)."""
    M = M.tocsr()

    def blk(i, j):
        return M[i * n:(i + 1) * n, j * n:(j + 1) * n].toarray()

    lower = [None] + [blk(i, i - 1) for i in range(1, nb)]
    upper = [blk(i, i + 1) for i in range(nb - 1)] + [None]
    lu = []
    S = blk(0, 0)
    lu.append(sla.lu_factor(S, check_finite=False))
    for i in range(1, nb):
        S = blk(i, i) - lower[i] @ sla.lu_solve(lu[i - 1], upper[i - 1])
        lu.append(sla.lu_factor(S, check_finite=False))
    return BlockTridiagFactor(n, nb, lower, upper, lu)


def quadrature_subspace(A: sp.csr_matrix, B: sp.csr_matrix, RHS: np.ndarray,
                        lmin: float, lmax: float, Ne: int, n: int, nb: int,
                        factors=None):
    """Fig. 2 step 2: Q = 0; for each node solve (Z_e B - A) Q_e = RHS and
    accumulate Q = Q - (w_e/2) Re{ r e^{i theta_e} Q_e } (Eq. 15), nodes in the
    order e = 1..Ne.  ``factors`` caches the node factorisations so that they
    are computed once for all refinement loops (Sec. V (ii)).
    Returns (Q, factors)."""
    _, w, theta, Z, r = contour_points(lmin, lmax, Ne)
    if factors is None:
        factors = [block_tridiag_factor((Z[e] * B - A).astype(np.complex128), n, nb) for e in range(Ne)]
    Q = np.zeros(RHS.shape, dtype=np.float64)
    for e in range(Ne):
        Qe = factors[e].solve(RHS.astype(np.complex128))
        Q = Q - (w[e] / 2.0) * (r * np.exp(1j * theta[e]) * Qe).real
    return Q, factors


# ----------------------------------------------------------------------------
# Steps 3-5: Rayleigh-Ritz (Eqs. 6-9)
# ----------------------------------------------------------------------------

def rayleigh_ritz(Q: np.ndarray, A: sp.csr_matrix, B: sp.csr_matrix):
    """A_Q = Q^T A Q, B_Q = Q^T B Q (Eq. 7); solve A_Q Phi = eps B_Q Phi with
    B_Q-orthonormal Phi (Eq. 6, LAPACK sygvd); lambda = eps (Eq. 8) ascending,
    X = Q Phi (Eq. 9).  Raises BQNotSPD when B_Q is not positive definite."""
    AQ = Q.T @ (A @ Q)
    BQ = Q.T @ (B @ Q)
    AQ = 0.5 * (AQ + AQ.T)   # symmetric in exact arithmetic
    BQ = 0.5 * (BQ + BQ.T)
    d = np.linalg.eigvalsh(BQ)
    if not (d[0] > 1e-14 * d[-1]):
        raise BQNotSPD(f"B_Q eigenvalue ratio {d[0] / d[-1]:.3e}")
    eps, Phi = sla.eigh(AQ, BQ)
    return eps, Q @ Phi, AQ, BQ


def residuals(A: sp.csr_matrix, B: sp.csr_matrix, lam: np.ndarray, X: np.ndarray):
    """Per column: ||A x - lam B x||_1 / (||A||_1 ||x||_1) and the paper's
    ||A x - lam B x||_1 / ||A x||_1 (Table I caption)."""
    AX = A @ X
    R = AX - (B @ X) * lam[None, :]
    rn = np.abs(R).sum(axis=0)
    xn = np.abs(X).sum(axis=0)
    axn = np.abs(AX).sum(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return rn / (norm1(A) * xn), rn / axn


# ----------------------------------------------------------------------------
# The outer loop (Fig. 2 steps 1-6, Sec. III.B (i))
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class FeastResult:
    lam: np.ndarray          # (M0,) ascending, in-interval first
    X: np.ndarray            # (N, M0)
    resid: np.ndarray        # (M0,) ||Ax - lam Bx||_1 / (||A||_1 ||x||_1)
    resid_paper: np.ndarray  # (M0,) ||Ax - lam Bx||_1 / ||Ax||_1
    m_found: int
    loops: int
    converged: bool
    trace_history: list
    rel_change_history: list


def feast(op, lmin: float, lmax: float, M0: int, Ne: int, Y: np.ndarray,
          tol: float = 1e-12, max_loops: int = 20) -> FeastResult:
    """FEAST for a real symmetric A and s.p.d. B given as 27-point layered
    operators (``op`` has nx, ny, nz, A27, B27).  Y (N x M0) is the start
    block (Fig. 2 step 1)."""
    nx, ny, nz = op.nx, op.ny, op.nz
    n, nb = nx * ny, nz
    A = assemble(op.A27, nx, ny, nz)
    B = assemble(op.B27, nx, ny, nz)
    Ycur = np.array(Y, dtype=np.float64)
    factors = None
    prev_trace, prev_count = None, None
    traces, changes = [], []
    converged = False
    for loop in range(1, max_loops + 1):
        RHS = B @ Ycur                                                   # Y = B X (Sec. III.B (i))
        Q, factors = quadrature_subspace(A, B, RHS, lmin, lmax, Ne, n, nb, factors)   # step 2
        eps, X, _, _ = rayleigh_ritz(Q, A, B)                            # steps 3-5
        inside = (eps >= lmin) & (eps <= lmax)
        count = int(inside.sum())
        trace = float(eps[inside].sum())                                 # step 6
        scale = float(np.abs(eps[inside]).sum())
        traces.append(trace)
        if prev_trace is not None:
            change = abs(trace - prev_trace) / scale if scale > 0 else 0.0
            changes.append(change)
            if count == prev_count and change <= tol:
                converged = True
        Ycur = X
        if converged:
            break
        prev_trace, prev_count = trace, count
    order = np.concatenate([np.flatnonzero(inside), np.flatnonzero(~inside)])
    lam = eps[order]
    X = X[:, order]
    r1, rp = residuals(A, B, lam, X)
    return FeastResult(lam, X, r1, rp, count, loop, converged, traces, changes)


# ----------------------------------------------------------------------------
# Complex Hermitian A (Sec. III.A, Eqs. 10 and 12)
# ----------------------------------------------------------------------------

def quadrature_subspace_hermitian(A: sp.csr_matrix, B: sp.csr_matrix, RHS: np.ndarray,
                                  lmin: float, lmax: float, Ne: int, n: int, nb: int,
                                  factors=None):
    """Eq. 12: Q = -sum_e (w_e r / 4) (e^{i theta_e} G(Z_e) + e^{-i theta_e}
    G^dagger(Z_e)) RHS, with G(Z) = (Z B - A)^{-1} and, A being Hermitian,
    G^dagger(Z) = G(conj Z) (Sec. III.A); each node solves at Z_e and at its
    conjugate, accumulated in the order e = 1..Ne.  ``factors`` caches the
    2 Ne factorisations.  Returns (Q, factors)."""
    _, w, theta, Z, r = contour_points(lmin, lmax, Ne)
    if factors is None:
        factors = [(block_tridiag_factor((Z[e] * B - A).astype(np.complex128), n, nb),
                    block_tridiag_factor((np.conj(Z[e]) * B - A).astype(np.complex128), n, nb))
                   for e in range(Ne)]
    Q = np.zeros(RHS.shape, dtype=np.complex128)
    for e in range(Ne):
        Ge = factors[e][0].solve(RHS.astype(np.complex128))
        Gd = factors[e][1].solve(RHS.astype(np.complex128))
        Q = Q - (w[e] * r / 4.0) * (np.exp(1j * theta[e]) * Ge + np.exp(-1j * theta[e]) * Gd)
    return Q, factors


def rayleigh_ritz_hermitian(Q: np.ndarray, A: sp.csr_matrix, B: sp.csr_matrix):
    """Steps 3-5 for complex Q: A_Q = Q^H A Q, B_Q = Q^H B Q (Hermitian), the
    Hermitian-definite pencil by LAPACK (hegvd), X = Q Phi; the same
    definiteness test as the real case."""
    AQ = Q.conj().T @ (A @ Q)
    BQ = Q.conj().T @ (B @ Q)
    AQ = 0.5 * (AQ + AQ.conj().T)   # Hermitian in exact arithmetic
    BQ = 0.5 * (BQ + BQ.conj().T)
    d = np.linalg.eigvalsh(BQ)
    if not (d[0] > 1e-14 * d[-1]):
        raise BQNotSPD(f"B_Q eigenvalue ratio {d[0] / d[-1]:.3e}")
    eps, Phi = sla.eigh(AQ, BQ)
    return eps, Q @ Phi, AQ, BQ


def feast_hermitian(op, lmin: float, lmax: float, M0: int, Ne: int, Y: np.ndarray,
                    tol: float = 1e-12, max_loops: int = 20) -> FeastResult:
    """FEAST for a complex Hermitian A (``op.A27`` complex) and a real s.p.d.
    B: the loop of ``feast`` with Y, Q, X and Phi complex and the contour sum
    of Eq. 12 in step 2 (Sec. III.B, the changes listed for Hermitian A)."""
    nx, ny, nz = op.nx, op.ny, op.nz
    n, nb = nx * ny, nz
    A = assemble(op.A27, nx, ny, nz)
    B = assemble(op.B27, nx, ny, nz)
    Ycur = np.array(Y, dtype=np.complex128)
    factors = None
    prev_trace, prev_count = None, None
    traces, changes = [], []
    converged = False
    for loop in range(1, max_loops + 1):
        RHS = B @ Ycur
        Q, factors = quadrature_subspace_hermitian(A, B, RHS, lmin, lmax, Ne, n, nb, factors)
        eps, X, _, _ = rayleigh_ritz_hermitian(Q, A, B)
        inside = (eps >= lmin) & (eps <= lmax)
        count = int(inside.sum())
        trace = float(eps[inside].sum())
        scale = float(np.abs(eps[inside]).sum())
        traces.append(trace)
        if prev_trace is not None:
            change = abs(trace - prev_trace) / scale if scale > 0 else 0.0
            changes.append(change)
            if count == prev_count and change <= tol:
                converged = True
        Ycur = X
        if converged:
            break
        prev_trace, prev_count = trace, count
    order = np.concatenate([np.flatnonzero(inside), np.flatnonzero(~inside)])
    lam = eps[order]
    X = X[:, order]
    r1, rp = residuals(A, B, lam, X)
    return FeastResult(lam, X, r1, rp, count, loop, converged, traces, changes)


# ----------------------------------------------------------------------------
# Independent checks used to pin the oracle
# ----------------------------------------------------------------------------

def dense_generalized_eigh(op):
    """All eigenpairs of the dense pencil (A, B) via LAPACK (tiny N only)."""
    A = assemble(op.A27, op.nx, op.ny, op.nz).toarray()
    B = assemble(op.B27, op.nx, op.ny, op.nz).toarray()
    return sla.eigh(A, B)


def inertia_count(op, sigma: float) -> int:
    """Number of eigenvalues of the pencil (A, B) below sigma, i.e. the number
    of negative eigenvalues of A - sigma B (Sylvester's law of inertia, B s.p.d.).
    Block elimination over the z-layers: the inertia of a block-tridiagonal
    symmetric matrix is the sum of the inertias of its successive Schur
    complements S_i = D_i - L_i S_{i-1}^{-1} L_i^T (Haynsworth additivity)."""
    nx, ny, nz = op.nx, op.ny, op.nz
    n = nx * ny
    Mreal = (assemble(op.A27, nx, ny, nz) - sigma * assemble(op.B27, nx, ny, nz)).tocsr()

    def blk(i, j):
        return Mreal[i * n:(i + 1) * n, j * n:(j + 1) * n].toarray()

    neg = 0
    S = blk(0, 0)
    for i in range(nz):
        if i > 0:
            L = blk(i, i - 1)
            S = blk(i, i) - L @ np.linalg.solve(S_prev, L.T)
        S = 0.5 * (S + S.T)
        neg += int((np.linalg.eigvalsh(S) < 0).sum())
        S_prev = S
    return neg


def closed_form_eigenvalues_v0(nx: int, ny: int, nz: int) -> np.ndarray:
    """All eigenvalues (ascending) of A = K/2, B = M at V = 0 for the Q1
    operator with spacing h = 1/(nx+1): lambda_ijk = (mu_i(nx) + mu_j(ny) + mu_k(nz))/2,
    mu_k(m) = (6/h^2)(1 - cos t)/(2 + cos t), t = k pi/(m+1).  Sine vectors
    diagonalise K1 = (1/h) tridiag(-1,2,-1) (eigenvalue (2 - 2cos t)/h) and
    M1 = (h/6) tridiag(1,4,1) (eigenvalue h(4 + 2cos t)/6), so every Kronecker
    term of K is mu times M on the tensor-product sine basis."""
    h = 1.0 / (nx + 1)

    def mu(m):
        t = np.arange(1, m + 1) * math.pi / (m + 1)
        return (6.0 / h ** 2) * (1.0 - np.cos(t)) / (2.0 + np.cos(t))

    lam = 0.5 * (mu(nx)[:, None, None] + mu(ny)[None, :, None] + mu(nz)[None, None, :])
    return np.sort(lam.ravel())
