"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed Gauss-Legendre table (Fig. 2 caption), exactness of Gauss quadrature,
closed forms of the contour filter, the V = 0 tensor-product spectrum, the
spectral form of Q from a dense pencil eigendecomposition, LAPACK/SuperLU on
tiny inputs, a Jacobi generalized eigensolver written from the mathematics
(oracle/jacobi.py, itself pinned to closed forms), hand-computed residuals and
norms (Table I caption), Sylvester inertia and the k-fold multiplicity
construction of Sec. IV.B.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle
import workloads
from conftest import GOLDEN


def _paper_gl8():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gl8_paper.txt")) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[2])) for r in rows}


# ---------------------------------------------------------------- quadrature

def test_gl8_matches_paper_table():
    """Fig. 2 caption: the printed Ne = 8 nodes/weights (15 digits)."""
    x, w = oracle.gauss_legendre(8)
    tab = _paper_gl8()
    for i, (xp, wp) in tab.items():
        assert abs(x[i - 1] - xp) < 2e-15, (i, x[i - 1], xp)
        assert abs(w[i - 1] - wp) < 2e-15
        assert x[i] == -x[i - 1] and w[i] == w[i - 1]   # x_{2i} = -x_{2i-1}


@pytest.mark.parametrize("Ne", [1, 2, 3, 4, 5, 8, 12, 16])
def test_gauss_legendre_exact_on_polynomials(Ne):
    """An Ne-point Gauss rule integrates x^k exactly for k <= 2 Ne - 1."""
    x, w = oracle.gauss_legendre(Ne)
    assert len(x) == Ne and np.all(np.abs(x) < 1)
    for k in range(2 * Ne):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # and not for k = 2 Ne (the rule has degree exactly 2 Ne - 1)
    assert abs(np.dot(w, x ** (2 * Ne)) - 2.0 / (2 * Ne + 1)) > 1e-12


def test_contour_points_on_upper_half_circle():
    """Eqs. 13-14: Z_e = c + r e^{i theta_e}, theta_e in (0, pi)."""
    lmin, lmax = 3.0, 11.0
    x, w, theta, Z, r = oracle.contour_points(lmin, lmax, 8)
    assert r == 4.0
    assert np.allclose(np.abs(Z - 7.0), 4.0, atol=1e-14, rtol=0)
    assert np.all(Z.imag > 0) and np.all((theta > 0) & (theta < math.pi))
    assert np.allclose(theta, (math.pi / 2) * (1 - x))


def test_filter_closed_forms():
    """The rational filter of Eq. 15: f = -1 at the centre (each node term
    reduces to w_e/2), f(c + r t) + f(c + r/t) = -1 (so -1/2 at both ends),
    f symmetric about the centre, small far outside the interval."""
    lmin, lmax = -2.0, 6.0
    c, r = 2.0, 4.0
    f = lambda lam: oracle.filter_value(np.array([lam]), lmin, lmax, 8)[0]  # noqa: E731
    assert abs(f(c) + 1.0) < 1e-15
    assert abs(f(lmin) + 0.5) < 1e-14 and abs(f(lmax) + 0.5) < 1e-14
    for d in (0.3, 1.7, 3.9, 5.0, 9.0):
        assert abs(f(c + d) - f(c - d)) < 1e-14
    # inversion through the circle: with u = e^{i theta} on the unit circle,
    # Re{u/(u - t)} + Re{u/(u - 1/t)} = 1 for real t != 0, so summing the node
    # terms with sum_e w_e = 2 gives f(c + r t) + f(c + r/t) = -1 exactly
    for t in (0.2, 0.5, 0.9, -0.7, 1.3, -3.0):
        assert abs(f(c + r * t) + f(c + r / t) + 1.0) < 1e-13
    assert abs(f(c + 2 * r)) < 1e-4 and abs(f(c + 3 * r)) < 1e-6


# ---------------------------------------------------------------- operators

def test_v0_spectrum_closed_form_matches_dense_pencil():
    """Assembled Q1 operator at V = 0 vs the tensor-product closed form: two
    independent derivations of the same spectrum."""
    for (nx, ny, nz) in [(3, 4, 5), (5, 5, 3), (2, 3, 7)]:
        op = workloads.q1_operator(nx, ny, nz)
        lam = oracle.dense_generalized_eigh(op)[0]
        cf = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
        assert np.allclose(lam, cf, rtol=1e-12, atol=0)


def test_operator_symmetric_and_B_spd():
    op = workloads.q1_operator(4, 3, 5, workloads.gaussian_potential(4, 7, 4, 3, 5))
    A = oracle.assemble(op.A27, 4, 3, 5).toarray()
    B = oracle.assemble(op.B27, 4, 3, 5).toarray()
    assert np.abs(A - A.T).max() < 1e-14 and np.abs(B - B.T).max() < 1e-15
    assert np.linalg.eigvalsh(B).min() > 0


# ---------------------------------------------------------------- step 2

def _tiny():
    op = workloads.q1_operator(4, 3, 6, workloads.gaussian_potential(3, 11, 4, 3, 6))
    A = oracle.assemble(op.A27, 4, 3, 6)
    B = oracle.assemble(op.B27, 4, 3, 6)
    return op, A, B


def test_block_tridiag_solve_matches_sparse_lu():
    """Node solve (Fig. 2 step 2) vs SuperLU on the assembled complex matrix,
    and its residual via the independent sparse product."""
    op, A, B = _tiny()
    rng = np.random.default_rng(3)
    Z = 30.0 + 4.5j
    M = (Z * B - A).astype(np.complex128)
    rhs = rng.standard_normal((op.N, 5))
    fac = oracle.block_tridiag_factor(M, op.n, op.nz)
    q = fac.solve(rhs.astype(np.complex128))
    ref = spla.splu(M.tocsc()).solve(rhs.astype(np.complex128))
    assert np.abs(q - ref).max() / np.abs(ref).max() < 1e-12
    assert np.abs(M @ q - rhs).max() / np.abs(rhs).max() < 1e-12


def test_quadrature_matches_spectral_form():
    """Eq. 15 on a tiny pencil equals Q = X f(Lambda) X^T RHS, with X, Lambda
    from the dense LAPACK pencil solve and f the scalar filter."""
    op, A, B = _tiny()
    lam, X = oracle.dense_generalized_eigh(op)
    lmin, lmax = lam[2] - 0.3, 0.5 * (lam[7] + lam[8])
    rhs = np.random.default_rng(5).standard_normal((op.N, 4))
    Q, _ = oracle.quadrature_subspace(A, B, rhs, lmin, lmax, 8, op.n, op.nz)
    f = oracle.filter_value(lam, lmin, lmax, 8)
    Qref = X @ (f[:, None] * (X.T @ rhs))
    assert np.abs(Q - Qref).max() / np.abs(Qref).max() < 1e-12


# ---------------------------------------------------------------- steps 3-5

def test_rayleigh_ritz_2x2_closed_form():
    """Steps 3-5 of the oracle on a 2 x 2 pencil with an invertible,
    non-orthogonal Q.  A full-rank Q makes A_Q, B_Q congruent to A, B (Eq. 7),
    so the Ritz values are the pencil's eigenvalues: by hand,
    det(A - e B) = (2 - 2e)(3 - e) - (1 - e/2)^2 = 1.75 e^2 - 7 e + 5, with
    roots (7 -+ sqrt(14)) / 3.5.  X = Q Phi must be B-orthonormal (Eq. 9) and
    satisfy A X = B X diag(eps) exactly (Eq. 2)."""
    import scipy.sparse as sp
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    B = np.array([[2.0, 0.5], [0.5, 1.0]])
    Q = np.array([[1.0, 2.0], [0.5, -1.0]])
    roots = np.array([(7.0 - math.sqrt(14.0)) / 3.5, (7.0 + math.sqrt(14.0)) / 3.5])
    eps, X, AQ, BQ = oracle.rayleigh_ritz(Q, sp.csr_matrix(A), sp.csr_matrix(B))
    assert np.allclose(eps, roots, rtol=1e-14, atol=0)
    assert np.abs(X.T @ B @ X - np.eye(2)).max() < 1e-14
    assert np.abs(A @ X - B @ X * eps[None, :]).max() < 1e-14
    # a plausible slip, B_Q = Q^T Q (B dropped from Eq. 7), breaks the pin
    wrong = np.sort(np.real(np.linalg.eigvals(np.linalg.solve(Q.T @ Q, Q.T @ A @ Q))))
    assert np.abs(wrong - roots).max() > 1e-2


def test_reduced_eigensolve_matches_jacobi():
    """The oracle's step 4 (LAPACK sygvd inside rayleigh_ritz) against the
    Jacobi solver written from the mathematics, on the A_Q, B_Q that
    rayleigh_ritz itself forms from a tiny Q1 pencil and a random block."""
    import scipy.sparse as sp  # noqa: F401
    op = workloads.q1_operator(4, 3, 5, workloads.gaussian_potential(3, 21, 4, 3, 5))
    A = oracle.assemble(op.A27, 4, 3, 5)
    B = oracle.assemble(op.B27, 4, 3, 5)
    Q = np.random.default_rng(8).standard_normal((op.N, 12))
    eps, X, AQ, BQ = oracle.rayleigh_ritz(Q, A, B)
    ej, Pj = oracle.jacobi_generalized_eigh(AQ, BQ)
    assert np.abs(eps - ej).max() <= 1e-12 * np.abs(ej).max()
    # same Ritz vectors up to sign (the eigenvalues here are simple)
    Xj = Q @ Pj
    for c in range(12):
        s = np.sign(Xj[:, c] @ (B @ X[:, c]))
        assert np.abs(s * Xj[:, c] - X[:, c]).max() <= 1e-9 * np.abs(X[:, c]).max()


# ---------------------------------------------------------------- Jacobi (independent eigensolver)

def test_jacobi_2x2_closed_form():
    """A symmetric 2 x 2 matrix [[a, b], [b, c]] has the eigenvalues
    (a + c)/2 -+ sqrt(((a - c)/2)^2 + b^2)."""
    for a, b, c in [(2.0, 1.0, -3.0), (1.0, 1e-9, 1.0), (5.0, -4.0, 5.0), (0.0, 2.0, 0.0)]:
        w, V = oracle.jacobi_symmetric(np.array([[a, b], [b, c]]))
        d = math.sqrt(((a - c) / 2) ** 2 + b * b)
        assert np.allclose(w, [(a + c) / 2 - d, (a + c) / 2 + d], rtol=1e-15, atol=1e-15)
        assert np.abs(V.T @ V - np.eye(2)).max() < 1e-15


def test_jacobi_generalized_v0_closed_form():
    """The Jacobi solver on the assembled V = 0 pencil reproduces the
    tensor-product closed form, with B-orthonormal eigenvectors."""
    for (nx, ny, nz) in [(3, 4, 5), (2, 3, 7)]:
        op = workloads.q1_operator(nx, ny, nz)
        A = oracle.assemble(op.A27, nx, ny, nz).toarray()
        B = oracle.assemble(op.B27, nx, ny, nz).toarray()
        eps, Phi = oracle.jacobi_generalized_eigh(A, B)
        cf = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
        assert np.allclose(eps, cf, rtol=1e-12, atol=0)
        assert np.abs(Phi.T @ B @ Phi - np.eye(op.N)).max() < 1e-12
        assert np.abs(A @ Phi - B @ Phi * eps[None, :]).max() < 1e-12 * np.abs(A).max()


def test_jacobi_generalized_matches_lapack_dense_pencil():
    """Jacobi and LAPACK (the oracle's dense reference) on pencils with a
    potential: eigenvalue by eigenvalue to 1e-12."""
    for (nx, ny, nz, G, seed) in [(5, 4, 6, 3, 17), (3, 3, 8, 4, 2)]:
        op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
        A = oracle.assemble(op.A27, nx, ny, nz).toarray()
        B = oracle.assemble(op.B27, nx, ny, nz).toarray()
        ej, _ = oracle.jacobi_generalized_eigh(A, B)
        el = oracle.dense_generalized_eigh(op)[0]
        assert np.allclose(ej, el, rtol=1e-12, atol=0)


def test_feast_matches_jacobi_on_tiny_pencil():
    """The whole oracle loop (Fig. 2) against the from-scratch Jacobi
    eigensolve of the dense pencil: the M lowest eigenvalues to 1e-12, the
    eigenvectors through their B-projectors (all simple here)."""
    op = workloads.q1_operator(5, 4, 6, workloads.gaussian_potential(3, 17, 5, 4, 6))
    A = oracle.assemble(op.A27, 5, 4, 6)
    B = oracle.assemble(op.B27, 5, 4, 6)
    ej, Pj = oracle.jacobi_generalized_eigh(A.toarray(), B.toarray())
    M = 7
    lmin, lmax = ej[0] - 0.5 * (ej[M] - ej[M - 1]), 0.5 * (ej[M - 1] + ej[M])
    res = oracle.feast(op, lmin, lmax, 12, 8, workloads.random_Y(op.N, 12, 5), tol=1e-12)
    assert res.converged and res.m_found == M
    assert np.allclose(res.lam[:M], ej[:M], rtol=1e-12, atol=0)
    for c in range(M):
        x, xj = res.X[:, c], Pj[:, c]
        assert np.abs(x * (xj @ (B @ x)) - xj * (xj @ (B @ xj))).max() <= 1e-9 * np.abs(xj).max()


def test_jacobi_pins_catch_planted_mistakes(monkeypatch):
    """A wrong rotation -- the sign of s flipped, or tau with its sign
    reversed -- no longer annihilates a_pq: the 2 x 2 closed form fails or the
    sweeps never end."""
    import oracle.jacobi as jac
    S = np.array([[2.0, 1.0], [1.0, -3.0]])
    d = math.sqrt(2.5 ** 2 + 1.0)
    want = [-0.5 - d, -0.5 + d]
    orig = jac.rotation

    def flipped(app, aqq, apq):
        c, s = orig(app, aqq, apq)
        return c, -s

    def tau_reversed(app, aqq, apq):
        return orig(aqq, app, apq)

    for bad in (flipped, tau_reversed):
        monkeypatch.setattr(jac, "rotation", bad)
        try:
            w, _ = jac.jacobi_symmetric(S, max_sweeps=20)
            assert not np.allclose(w, want, rtol=1e-12), bad.__name__
        except jac.JacobiNoConvergence:
            pass
    monkeypatch.setattr(jac, "rotation", orig)
    w, _ = jac.jacobi_symmetric(S, max_sweeps=20)
    assert np.allclose(w, want, rtol=1e-14)


# ---------------------------------------------------------------- residuals (Table I caption)

def test_norm1_closed_forms():
    """||M||_1 = largest absolute column sum: 6 for [[1, -2], [3, 4]] (its
    infinity norm is 7, its 2-norm 5.12); and for the Q1 operator at V = 0,
    A = K/2 has the interior column 8h/3 in absolute sum (centre 4h/3, 12
    edge neighbours -h/12, 8 corners -h/24, faces 0)."""
    import scipy.sparse as sp
    assert oracle.norm1(sp.csr_matrix(np.array([[1.0, -2.0], [3.0, 4.0]]))) == 6.0
    for g in [(3, 3, 3), (4, 5, 6), (7, 3, 4)]:
        op = workloads.q1_operator(*g)
        h = 1.0 / (g[0] + 1)
        assert abs(oracle.norm1(oracle.assemble(op.A27, *g)) - 8.0 * h / 3.0) < 1e-15


def _resid_case():
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[3.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]]))
    B = sp.csr_matrix(np.diag([2.0, 1.0, 1.0]))
    X = np.array([[1.0, 1.0, 1.0], [0.0, 1.0, -1.0], [0.0, 0.0, 2.0]])
    lam = np.array([1.0, 2.0, 0.5])
    # by hand, ||A||_1 = 4 (columns 4, 4, 3):
    #   x = (1, 0, 0),  l = 1:   A x - l B x = (1, -1, 0),      ||.||_1 = 2,    ||x||_1 = 1, ||A x||_1 = 4
    #   x = (1, 1, 0),  l = 2:   A x - l B x = (-2, -1, -1),    ||.||_1 = 4,    ||x||_1 = 2, ||A x||_1 = 4
    #   x = (1, -1, 2), l = 1/2: A x - l B x = (3, -4.5, 4),    ||.||_1 = 11.5, ||x||_1 = 4, ||A x||_1 = 14
    want = np.array([2.0 / 4.0, 4.0 / 8.0, 11.5 / 16.0])
    want_paper = np.array([2.0 / 4.0, 4.0 / 4.0, 11.5 / 14.0])
    return A, B, X, lam, want, want_paper


def test_residuals_hand_computed():
    """Both residual forms on a 3 x 3 pencil with planted non-eigenvectors."""
    A, B, X, lam, want, want_paper = _resid_case()
    r1, rp = oracle.residuals(A, B, lam, X)
    assert np.allclose(r1, want, rtol=1e-15, atol=0)
    assert np.allclose(rp, want_paper, rtol=1e-15, atol=0)
    # invariant under scaling of x
    r1s, rps = oracle.residuals(A, B, lam, X * np.array([3.0, -0.25, 7.0])[None, :])
    assert np.allclose(r1s, want, rtol=1e-15) and np.allclose(rps, want_paper, rtol=1e-15)


def test_residual_pins_catch_planted_mistakes(monkeypatch):
    """Plausible slips in the residual formulas each miss the hand values:
    the 2-norm for ||x||, the 2-norm or Frobenius norm for ||A||, B dropped,
    the two denominators swapped."""
    import numpy.linalg as la
    import oracle.feast_oracle as fo
    A, B, X, lam, want, want_paper = _resid_case()
    Ad = A.toarray()
    # the oracle with ||A||_1 replaced by the 2-norm / Frobenius norm
    for bad_norm in (lambda M: float(la.norm(M.toarray(), 2)), lambda M: float(la.norm(M.toarray(), "fro"))):
        monkeypatch.setattr(fo, "norm1", bad_norm)
        r1, _ = fo.residuals(A, B, lam, X)
        assert not np.allclose(r1, want, rtol=1e-6)
    monkeypatch.setattr(fo, "norm1", oracle.norm1)
    R = Ad @ X - (B.toarray() @ X) * lam[None, :]
    rn = np.abs(R).sum(axis=0)
    # ||x||_2 in place of ||x||_1
    assert not np.allclose(rn / (4.0 * la.norm(X, axis=0)), want, rtol=1e-6)
    # B dropped: A x - l x
    rn_noB = np.abs(Ad @ X - X * lam[None, :]).sum(axis=0)
    assert not np.allclose(rn_noB / (4.0 * np.abs(X).sum(axis=0)), want, rtol=1e-6)
    # denominators swapped between the two forms
    assert not np.allclose(rn / np.abs(Ad @ X).sum(axis=0), want, rtol=1e-6)
    assert not np.allclose(rn / (4.0 * np.abs(X).sum(axis=0)), want_paper, rtol=1e-6)


# ---------------------------------------------------------------- full loop

def _interval(intervals, key):
    iv = intervals[key]
    return iv["lmin"], iv["lmax"], iv["M"]


def test_feast_v0_matches_closed_form(intervals):
    """cfg 10x10x20 at V = 0: the M eigenvalues equal the tensor-product closed
    form to 1e-12 relative; the count equals the inertia count."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(0, zero_potential=True)
    lmin, lmax, M = _interval(intervals, "q1_10x10x20/v0")
    res = oracle.feast(op, lmin, lmax, wl.M0, wl.Ne, workloads.random_Y(op.N, wl.M0, 1000), tol=wl.tol)
    cf = oracle.closed_form_eigenvalues_v0(10, 10, 20)
    assert res.converged and res.m_found == M
    assert np.allclose(res.lam[:M], cf[:M], rtol=1e-12, atol=0)
    assert res.resid[:M].max() < 1e-12
    assert oracle.inertia_count(op, lmax) - oracle.inertia_count(op, lmin) == M


@pytest.mark.parametrize("seed", [0, 3])
def test_feast_matches_dense_pencil(intervals, seed):
    """cfg 10x10x20 with a Gaussian potential: eigenvalues vs the dense LAPACK
    pencil to 1e-12; X B-orthonormal (Eq. 9 / Sec. III.A); residual <= 1e-10;
    the trace change falls loop over loop (Table II behaviour)."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(seed)
    lmin, lmax, M = _interval(intervals, f"q1_10x10x20/seed{seed}")
    res = oracle.feast(op, lmin, lmax, wl.M0, wl.Ne, workloads.random_Y(op.N, wl.M0, 1000 + seed), tol=wl.tol)
    lam = oracle.dense_generalized_eigh(op)[0]
    assert res.m_found == M and res.converged
    assert np.allclose(res.lam[:M], lam[:M], rtol=1e-12, atol=0)
    B = oracle.assemble(op.B27, 10, 10, 20)
    X = res.X[:, :M]
    assert np.abs(X.T @ (B @ X) - np.eye(M)).max() < 1e-12
    assert res.resid[:M].max() < 1e-10
    ch = res.rel_change_history
    assert all(b < a for a, b in zip(ch, ch[1:])) or ch[-1] < 1e-13
    # Courant-Fischer: Ritz values of any subspace are >= the true ones
    assert np.all(res.lam[:M] >= lam[:M] - 1e-12 * np.abs(lam[:M]))


def test_inertia_count_matches_dense_eigenvalues():
    op = workloads.q1_operator(4, 5, 6, workloads.gaussian_potential(5, 2, 4, 5, 6))
    lam = oracle.dense_generalized_eigh(op)[0]
    for sigma in (lam[0] - 1.0, 0.5 * (lam[3] + lam[4]), 0.5 * (lam[40] + lam[41]), lam[-1] + 1):
        assert oracle.inertia_count(op, sigma) == int((lam < sigma).sum())


def test_full_size_brackets_are_consistent(intervals):
    """The stored brackets of sampled eigenvalues of the 32 x 32 x 400
    workload (bisection on the inertia count above) are tight, ordered, inside
    the certified interval and inside the coarser brackets stored with it,
    and their end counts straddle their index."""
    with open(os.path.join(GOLDEN, "fullsize_brackets.json")) as f:
        fb = json.load(f)
    iv = intervals[fb["key"]]
    coarse = iv["brackets"]
    prev = -math.inf
    for k in sorted(fb["brackets"], key=int):
        b = fb["brackets"][k]
        assert 0 < b["hi"] - b["lo"] <= fb["rel_width"] * abs(b["hi"]) <= 1e-11 * abs(b["hi"])
        assert b["nu_lo"] <= int(k) - 1 < int(k) <= b["nu_hi"]
        assert iv["lmin"] <= b["lo"] and b["hi"] <= iv["lmax"] and b["lo"] >= prev
        if k in coarse:
            assert coarse[k][0] <= b["lo"] and b["hi"] <= coarse[k][1]
        prev = b["hi"]
    assert {"1", str(iv["M"])} <= set(fb["brackets"])


def test_k_copies_give_k_fold_multiplicity():
    """Sec. IV.B, k(N, M): block-diagonal copies make every eigenvalue k-fold
    and FEAST finds k M pairs in the unchanged interval."""
    blk = workloads.q1_operator(4, 4, 5, workloads.gaussian_potential(3, 9, 4, 4, 5))
    lam1 = oracle.dense_generalized_eigh(blk)[0]
    M = 6
    lmin, lmax = lam1[0] - 0.5, 0.5 * (lam1[M - 1] + lam1[M])
    k = 2
    rep = workloads.replicate_z(blk, k)
    res = oracle.feast(rep, lmin, lmax, 16, 8, workloads.random_Y(rep.N, 16, 77), tol=1e-12)
    assert res.m_found == k * M
    got = np.sort(res.lam[:k * M]).reshape(M, k)
    assert np.allclose(got, np.repeat(lam1[:M, None], k, axis=1), rtol=1e-11, atol=0)


def test_bq_not_spd_when_m0_too_large():
    """Sec. III.B (ii): far more vectors than eigenvalues in a narrow interval
    drive B_Q's smallest eigenvalue below the 1e-14 ratio."""
    op = workloads.q1_operator(5, 5, 6)
    lam = oracle.closed_form_eigenvalues_v0(5, 5, 6)
    lmin, lmax = lam[0] - 0.1, 0.5 * (lam[0] + lam[1])
    with pytest.raises(oracle.BQNotSPD):
        oracle.feast(op, lmin, lmax, 60, 8, workloads.random_Y(op.N, 60, 1), tol=1e-12)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle (on the CPU) and check that a pin
    fails for each: a dropped 1/2 in Eq. 15, a wrong contour centre in Eq. 14,
    a dropped factor r, the imaginary instead of the real part.  (Reflecting
    the nodes to the lower half circle is not a mistake for real symmetric A:
    G(conj Z) = conj G(Z) leaves the real part of Eq. 15 unchanged.)"""
    op, A, B = _tiny()
    lam, X = oracle.dense_generalized_eigh(op)
    lmin, lmax = lam[2] - 0.3, 0.5 * (lam[7] + lam[8])
    rhs = np.random.default_rng(5).standard_normal((op.N, 4))
    f = oracle.filter_value(lam, lmin, lmax, 8)
    Qref = X @ (f[:, None] * (X.T @ rhs))
    import oracle.feast_oracle as fo

    def err_with(patched_contour=None, part="real", scale=2.0):
        orig = fo.contour_points

        def contour(lmin_, lmax_, Ne_):
            x, w, th, Z, r = orig(lmin_, lmax_, Ne_)
            if patched_contour:
                return patched_contour(x, w, th, Z, r)
            return x, w, th, Z, r
        monkeypatch.setattr(fo, "contour_points", contour)
        try:
            Q, _ = fo.quadrature_subspace(A, B, rhs, lmin, lmax, 8, op.n, op.nz)
        finally:
            monkeypatch.setattr(fo, "contour_points", orig)
        return np.abs(Q - Qref).max() / np.abs(Qref).max()

    assert err_with() < 1e-12
    # dropped 1/2: weights doubled
    assert err_with(lambda x, w, th, Z, r: (x, 2 * w, th, Z, r)) > 1e-3
    # centre taken as (lmax - lmin)/2 instead of (lmax + lmin)/2 in Eq. 14
    assert err_with(lambda x, w, th, Z, r: (x, w, th, Z - (lmax + lmin) / 2 + r, r)) > 1e-3
    # factor r dropped from Eq. 15
    assert err_with(lambda x, w, th, Z, r: (x, w, th, Z, 1.0)) > 1e-3
    # rotated phase (e^{i theta} -> i e^{i theta} picks the imaginary part)
    assert err_with(lambda x, w, th, Z, r: (x, w, th + math.pi / 2, Z, r)) > 1e-3


# ---------------------------------------------------------------- learned start (CPU reference)

def test_mlp_backward_matches_finite_differences():
    """The reference MLP's backward pass against central differences of its
    loss (float64, no rounding)."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    sizes = [7, 12, 12, 12, 9]
    params = mlp.init_params(sizes, 1)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((5, 7))
    target = rng.standard_normal((5, 9))
    weights = rng.uniform(0.5, 1.5, 9)
    out, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, out, target, weights)
    eps = 1e-6
    for k in range(len(params)):
        W, b = params[k]
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += eps
            Wm[i, j] -= eps
            lp = mlp.loss(mlp.forward([(Wp, b) if q == k else params[q] for q in range(len(params))], x)[0],
                          target, weights)
            lm = mlp.loss(mlp.forward([(Wm, b) if q == k else params[q] for q in range(len(params))], x)[0],
                          target, weights)
            assert abs((lp - lm) / (2 * eps) - grads[k][0][i, j]) < 1e-7
        bp, bm = b.copy(), b.copy()
        bp[0] += eps
        bm[0] -= eps
        lp = mlp.loss(mlp.forward([(W, bp) if q == k else params[q] for q in range(len(params))], x)[0], target, weights)
        lm = mlp.loss(mlp.forward([(W, bm) if q == k else params[q] for q in range(len(params))], x)[0], target, weights)
        assert abs((lp - lm) / (2 * eps) - grads[k][1][0]) < 1e-7


def test_sine_basis_orthonormal_and_projection_is_adjoint():
    """The discrete sine vectors diagonalise tridiag(-1,2,-1) (a closed form:
    eigenvalue 2 - 2 cos(p pi/(m+1))), are orthonormal, and `project` is the
    adjoint (and on its range the inverse) of `expand`."""
    from oracle import mlp
    m = 11
    S = mlp.sine_basis(m, m)
    assert np.abs(S.T @ S - np.eye(m)).max() < 1e-13
    T = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    lam = 2 - 2 * np.cos(np.arange(1, m + 1) * math.pi / (m + 1))
    assert np.abs(T @ S - S * lam[None, :]).max() < 1e-13
    rng = np.random.default_rng(2)
    nx, ny, nz, c, px, py = 6, 5, 3, 4, 3, 2
    coef = rng.standard_normal((nz, c, px * py))
    X = rng.standard_normal((nx * ny * nz, c))
    Y = mlp.expand(coef, nx, ny, nz, px, py)
    assert abs(np.sum(Y * X) - np.sum(coef * mlp.project(X, nx, ny, nz, px, py))) < 1e-12
    assert np.abs(mlp.project(Y, nx, ny, nz, px, py) - coef).max() < 1e-13


def test_bf16_rounding_nearest_even():
    from oracle import mlp
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-40], dtype=np.float32)
    r = mlp.round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                                             # 1 + 2^-8 is a tie: even is 1.0
    assert r[2] == 1.0 + 2 ** -7                                   # above the tie rounds up
    assert r[3] == -2.5


# ---------------------------------------------------------------- Hermitian A (Eqs. 10, 12)

def _tiny_hermitian(flux=0.4, gauge_seed=None, gauge_B=False):
    real = workloads.q1_operator(5, 4, 6, workloads.gaussian_potential(3, 17, 5, 4, 6))
    return real, workloads.peierls_operator(real, flux=flux, gauge_seed=gauge_seed, gauge_B=gauge_B)


def test_peierls_operator_is_hermitian():
    _, op = _tiny_hermitian(flux=0.4, gauge_seed=3)
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz).toarray()
    assert np.abs(A.imag).max() > 1e-3                      # genuinely complex
    assert np.abs(A - A.conj().T).max() < 1e-15 * np.abs(A).max()


def test_hermitian_quadrature_matches_spectral_form():
    """Eq. 12 on a tiny Hermitian pencil equals Q = X f(Lambda) X^H RHS with
    the real filter f of Eq. 15 (G(Z) = X (Z - Lambda)^{-1} X^H, and the two
    terms of Eq. 12 add to twice the real part)."""
    _, op = _tiny_hermitian()
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz)
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    lam, X = sla.eigh(A.toarray(), B.toarray())
    lmin, lmax = lam[1] - 0.3, 0.5 * (lam[6] + lam[7])
    rhs = workloads.random_Y_complex(op.N, 3, 41)
    Q, _ = oracle.quadrature_subspace_hermitian(A, B, rhs, lmin, lmax, 8, op.n, op.nz)
    f = oracle.filter_value(lam, lmin, lmax, 8)
    Qref = X @ (f[:, None] * (X.conj().T @ rhs))
    assert np.abs(Q - Qref).max() / np.abs(Qref).max() < 1e-12


def test_hermitian_formula_reduces_to_the_real_one():
    """For real A and real Y, Eq. 12 gives the real subspace of Eq. 15."""
    real, op = _tiny_hermitian(flux=0.0)
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz)
    Ar = oracle.assemble(real.A27, real.nx, real.ny, real.nz)
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    lam = oracle.dense_generalized_eigh(real)[0]
    lmin, lmax = lam[0] - 0.5, 0.5 * (lam[5] + lam[6])
    rhs = np.random.default_rng(43).standard_normal((op.N, 4))
    Qh, _ = oracle.quadrature_subspace_hermitian(A, B, rhs, lmin, lmax, 8, op.n, op.nz)
    Qr, _ = oracle.quadrature_subspace(Ar, B, rhs, lmin, lmax, 8, op.n, op.nz)
    assert np.abs(Qh.imag).max() < 1e-13 * np.abs(Qr).max()
    assert np.abs(Qh.real - Qr).max() < 1e-12 * np.abs(Qr).max()


def test_feast_hermitian_matches_dense_pencil():
    """A uniform field (flux 0.4 per plaquette) and a potential: the Hermitian
    loop finds the eigenvalues of the dense Hermitian pencil to 1e-12 with
    B-orthonormal eigenvectors (X^H B X = I) and residuals <= 1e-10."""
    _, op = _tiny_hermitian(flux=0.4)
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz)
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    M = 6
    lmin, lmax = lam[0] - 0.5 * (lam[M] - lam[M - 1]), 0.5 * (lam[M - 1] + lam[M])
    res = oracle.feast_hermitian(op, lmin, lmax, 10, 8, workloads.random_Y_complex(op.N, 10, 1001), tol=1e-12)
    assert res.converged and res.m_found == M
    assert np.allclose(res.lam[:M], lam[:M], rtol=1e-12, atol=0)
    X = res.X[:, :M]
    assert np.abs(X.conj().T @ (B @ X) - np.eye(M)).max() < 1e-12
    assert res.resid[:M].max() < 1e-10


def test_feast_hermitian_is_gauge_invariant():
    """A pure gauge transformation D^H (A, B) D, D = diag(exp(i chi)), leaves
    the spectrum unchanged: the Hermitian loop on the transformed pencil finds
    the eigenvalues of the real pencil (closed interval as for the real loop)."""
    real, op = _tiny_hermitian(flux=0.0, gauge_seed=5, gauge_B=True)
    lam = oracle.dense_generalized_eigh(real)[0]
    M = 6
    lmin, lmax = lam[0] - 0.5 * (lam[M] - lam[M - 1]), 0.5 * (lam[M - 1] + lam[M])
    res = oracle.feast_hermitian(op, lmin, lmax, 10, 8, workloads.random_Y_complex(op.N, 10, 1002), tol=1e-12)
    assert res.converged and res.m_found == M
    assert np.allclose(res.lam[:M], lam[:M], rtol=1e-12, atol=0)


def test_hermitian_pin_catches_planted_mistakes():
    """Each plausible slip in Eq. 12 breaks the spectral-form pin: the G^dagger
    term dropped (and the first doubled), the weight 1/4 read as 1/2, the
    conjugate node replaced by Z_e itself."""
    _, op = _tiny_hermitian()
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz)
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    lam, X = sla.eigh(A.toarray(), B.toarray())
    lmin, lmax = lam[1] - 0.3, 0.5 * (lam[6] + lam[7])
    rhs = workloads.random_Y_complex(op.N, 2, 47)
    f = oracle.filter_value(lam, lmin, lmax, 8)
    Qref = X @ (f[:, None] * (X.conj().T @ rhs))
    _, w, theta, Z, r = oracle.contour_points(lmin, lmax, 8)

    def solve(z):
        return sla.solve((z * B - A).toarray(), rhs)

    wrong = {
        "no adjoint term": sum(-(w[e] * r / 2.0) * np.exp(1j * theta[e]) * solve(Z[e]) for e in range(8)),
        "weight 1/2": sum(-(w[e] * r / 2.0) * (np.exp(1j * theta[e]) * solve(Z[e])
                                               + np.exp(-1j * theta[e]) * solve(np.conj(Z[e]))) for e in range(8)),
        "Z for conj Z": sum(-(w[e] * r / 4.0) * (np.exp(1j * theta[e]) + np.exp(-1j * theta[e])) * solve(Z[e])
                            for e in range(8)),
    }
    for name, Q in wrong.items():
        assert np.abs(Q - Qref).max() / np.abs(Qref).max() > 1e-3, name


def test_stored_oracle_eigenvalues_are_consistent():
    """The stored converged oracle runs (make_oracle_eigenvalues.py) lie inside
    their certified intervals, ascending, with the certified count, residuals
    <= 1e-10 and the first loop never the last (Fig. 2 step 6)."""
    with open(os.path.join(GOLDEN, "oracle_eigenvalues.json")) as f:
        gold = json.load(f)
    with open(os.path.join(GOLDEN, "batch_intervals.json")) as f:
        bivs = json.load(f)
    with open(os.path.join(GOLDEN, "learned_intervals.json")) as f:
        livs = json.load(f)
    assert {"batch/45", "batch/46", "learned/10000"} <= set(gold)
    for key, g in gold.items():
        kind, ident = key.split("/")
        iv = (bivs if kind == "batch" else livs)[ident]
        lam = np.array(g["lam"])
        assert g["m_found"] == len(lam) == iv["M"] == iv["inertia_lmax"] - iv["inertia_lmin"]
        assert np.all(np.diff(lam) >= 0) and iv["lmin"] <= lam[0] and lam[-1] <= iv["lmax"]
        assert g["resid_max"] <= 1e-10 and g["loops"] >= 2
