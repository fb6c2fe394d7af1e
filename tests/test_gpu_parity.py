"""Parity of the CUDA path (through the C-ABI) with the CPU oracle on the same
seeded inputs.  Sizes span several tiles of every kernel plus ragged tails
(layer sizes 100 and 132 against 32-wide sweep panels and 64-wide tiles;
subspace widths 16, 24, 33).

Tolerances: the plain FP64 path must give node solutions within 1e-10 of the
oracle relative to max |Q_e| (condition of Z_e B - A up to ~1e4 times the
rounding of an unpivoted elimination), eigenvalues within 1e-10 relative and
residuals <= 1e-10 (the stated eigenpair targets).
"""

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


def cm(a):
    """numpy (N, k) -> CUDA tensor holding it column-major."""
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def back(t):
    """CUDA tensor (k, N) column-major -> numpy (N, k)."""
    return t.cpu().numpy().T


def dev_op(op):
    A = torch.from_numpy(op.A27).cuda()
    B = torch.from_numpy(op.B27).cuda()
    return F().make_operator(op.nx, op.ny, op.nz, A, B), (A, B)


GRIDS = [(10, 10, 20, 8, 0), (12, 11, 9, 5, 4), (7, 5, 6, 3, 2)]


@pytest.mark.parametrize("nx,ny,nz,G,seed", GRIDS)
@pytest.mark.parametrize("k", [1, 16, 33])
def test_stencil_apply_matches_oracle(nx, ny, nz, G, seed, k):
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    X = np.random.default_rng(seed).standard_normal((op.N, k))
    h = F().Handle()
    for C27 in (op.A27, op.B27):
        Y = torch.zeros((k, op.N), dtype=torch.float64, device="cuda")
        h.feast_stencil_apply(nx, ny, nz, torch.from_numpy(C27).cuda(), cm(X), Y, k)
        ref = oracle.assemble(C27, nx, ny, nz) @ X
        assert np.abs(back(Y) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny,nz,G,seed", GRIDS)
def test_node_solve_fp64_matches_oracle(nx, ny, nz, G, seed):
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, lam[min(12, len(lam) - 1)]
    _, _, _, Z, _ = oracle.contour_points(lmin, lmax, 8)
    k = 24
    RHS = np.random.default_rng(seed + 1).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    h = F().Handle()
    for z in (Z[0], Z[7]):   # a node near the middle and the one closest to the real axis
        Qe = torch.zeros((k, op.N), dtype=torch.complex128, device="cuda")
        h.feast_node_solve(dop, complex(z), cm(RHS), Qe, k)
        ref = oracle.block_tridiag_factor((z * B - A).astype(np.complex128), op.n, nz).solve(
            RHS.astype(np.complex128))
        got = back(Qe)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny,nz,G,seed", GRIDS[:2])
def test_quadrature_fp64_matches_oracle(nx, ny, nz, G, seed):
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, 0.5 * (lam[9] + lam[10])
    k = 16
    RHS = np.random.default_rng(seed + 2).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    Q = torch.zeros((k, op.N), dtype=torch.float64, device="cuda")
    F().Handle().feast_quadrature(dop, lmin, lmax, 8, cm(RHS), Q, k)
    ref, _ = oracle.quadrature_subspace(A, B, RHS, lmin, lmax, 8, op.n, nz)
    assert np.abs(back(Q) - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("m", [1, 2, 16, 33, 64, 128])
@pytest.mark.parametrize("bcond", [1e3, 1e8])
def test_reduced_eig_matches_lapack(m, bcond):
    """Step 4 vs the oracle's LAPACK routine.  The pencil's eigenvalues are
    determined only to ~eps cond(B_Q) ||A_Q||, so with cond 1e3 they must agree
    to 1e-10 of the largest; for cond 1e8 the test checks the backward error
    and the B_Q-orthonormality (Eq. 9) instead."""
    rng = np.random.default_rng(m)
    U = np.linalg.qr(rng.standard_normal((m, m)))[0]
    BQ = U @ np.diag(np.logspace(0, -np.log10(bcond), m)) @ U.T
    S = rng.standard_normal((m, m))
    AQ = S + S.T
    eps = torch.zeros(m, dtype=torch.float64, device="cuda")
    Phi = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    F().Handle().feast_reduced_eig(cm(AQ), cm(BQ), m, eps, Phi)
    import scipy.linalg as sla
    ref = sla.eigh(AQ, BQ)[0]            # the oracle's step 4 routine
    e = eps.cpu().numpy()
    P = back(Phi)
    assert np.all(np.diff(e) >= 0)
    if bcond <= 1e3:
        assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max()
    # normalised backward error ||A P - B P E|| / ((||A|| + |eps| ||B||) ||P||);
    # LAPACK's own is ~1e-16 here
    R = AQ @ P - BQ @ P * e[None, :]
    scale = (np.abs(AQ).max() + np.abs(e).max() * np.abs(BQ).max()) * np.abs(P).max()
    assert np.abs(R).max() <= 1e-14 * scale
    assert np.abs(P.T @ BQ @ P - np.eye(m)).max() <= max(1e-10, 1e3 * 2.2e-16 * bcond)


def test_reduced_eig_singular_bq_reported():
    """A B_Q of rank m/2 is rejected (Sec. III.B (ii))."""
    m = 32
    rng = np.random.default_rng(9)
    V = rng.standard_normal((m, m // 2))
    BQ = V @ V.T
    AQ = np.eye(m)
    eps = torch.zeros(m, dtype=torch.float64, device="cuda")
    Phi = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    st = F().Handle().feast_reduced_eig(cm(AQ), cm(BQ), m, eps, Phi, allow=(F().FEAST_ERR_BQ_NOT_SPD,))
    assert st == F().FEAST_ERR_BQ_NOT_SPD


def _compare_feast(res_gpu_lam, X_gpu, m_gpu, loops_gpu, ref, op, M):
    assert m_gpu == ref.m_found == M
    lam = res_gpu_lam[:M]
    assert np.abs(lam - ref.lam[:M]).max() <= 1e-10 * np.abs(ref.lam[:M]).max()
    assert abs(loops_gpu - ref.loops) <= 1
    # eigenvectors: compare B-projectors onto each cluster of close eigenvalues
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    Xg, Xo = X_gpu[:, :M], ref.X[:, :M]
    assert np.abs(Xg.T @ (B @ Xg) - np.eye(M)).max() <= 1e-10
    i = 0
    while i < M:
        j = i + 1
        while j < M and abs(ref.lam[j] - ref.lam[i]) < 1e-8 * abs(ref.lam[i]):
            j += 1
        Pg = Xg[:, i:j] @ (Xg[:, i:j].T @ (B @ Xo[:, i:j]))
        assert np.abs(Pg - Xo[:, i:j]).max() <= 1e-8 * np.abs(Xo[:, i:j]).max()
        i = j


@pytest.mark.parametrize("nx,ny,nz,G,seed", GRIDS)
@pytest.mark.parametrize("k", [1, 7, 40])
def test_residuals_match_oracle_elementwise(nx, ny, nz, G, seed, k):
    """Both residual forms of the Table I caption, column by column, against
    the oracle's on the same seeded pairs (random vectors, so every residual is
    O(1) and its relative rounding error ~1e-15)."""
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    rng = np.random.default_rng(100 + seed)
    X = rng.standard_normal((op.N, k))
    lam = rng.uniform(5.0, 60.0, k)
    dop, keep = dev_op(op)
    r1 = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
    rp = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
    F().Handle().feast_residuals(dop, cm(lam), cm(X), k, r1, rp)
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    ref1, refp = oracle.residuals(A, B, lam, X)
    assert np.all(np.abs(r1.cpu().numpy() - ref1) <= 1e-12 * ref1)
    assert np.all(np.abs(rp.cpu().numpy() - refp) <= 1e-12 * refp)


def test_residuals_of_converged_pairs_match_oracle():
    """Converged eigenpairs of the oracle's loop: the residuals are rounding
    noise (~1e-16), so the two computations must agree to a small multiple of
    the unit roundoff in the normalised units of each form."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(4)
    lam_d, Xd = oracle.dense_generalized_eigh(op)
    k = 12
    lam, X = lam_d[:k], Xd[:, :k]
    dop, keep = dev_op(op)
    r1 = torch.zeros(k, dtype=torch.float64, device="cuda")
    rp = torch.zeros(k, dtype=torch.float64, device="cuda")
    F().Handle().feast_residuals(dop, cm(lam), cm(X), k, r1, rp)
    ref1, refp = oracle.residuals(oracle.assemble(op.A27, 10, 10, 20), oracle.assemble(op.B27, 10, 10, 20), lam, X)
    assert ref1.max() < 1e-13 and refp.max() < 1e-13
    assert np.abs(r1.cpu().numpy() - ref1).max() <= 2e-15
    assert np.abs(rp.cpu().numpy() - refp).max() <= 2e-14


@pytest.mark.parametrize("key,seed,zero", [("q1_10x10x20/v0", 0, True)] +
                         [(f"q1_10x10x20/seed{s}", s, False) for s in range(5)])
def test_feast_solve_fp64_matches_oracle(intervals, key, seed, zero):
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(seed, zero_potential=zero)
    iv = intervals[key]
    Y = workloads.random_Y(op.N, wl.M0, 1000 + seed)
    ref = oracle.feast(op, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, Y, tol=wl.tol)
    dop, keep = dev_op(op)
    lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
    resid = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    h = F().Handle()
    r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, cm(Y), lam, X, resid, allow=())
    _compare_feast(lam.cpu().numpy(), back(X), r.m_found, r.loops, ref, op, iv["M"])
    assert resid.cpu().numpy()[:iv["M"]].max() <= 1e-10
    assert r.info.resid_max <= 1e-10
    # residuals of the GPU eigenpairs recomputed by the oracle; the solve's own
    # residual output agrees with them pair by pair (both are rounding noise
    # here, so the agreement is absolute in the normalised units)
    r1, _ = oracle.residuals(oracle.assemble(op.A27, 10, 10, 20), oracle.assemble(op.B27, 10, 10, 20),
                             lam.cpu().numpy(), back(X))
    assert r1[:iv["M"]].max() <= 1e-10
    assert np.abs(resid.cpu().numpy()[:iv["M"]] - r1[:iv["M"]]).max() <= 2e-15
    if zero:
        cf = oracle.closed_form_eigenvalues_v0(10, 10, 20)
        assert np.abs(lam.cpu().numpy()[:iv["M"]] - cf[:iv["M"]]).max() <= 1e-10 * cf[iv["M"] - 1]


def test_feast_host_buffers_equal_device_buffers(intervals):
    """The end-to-end call with host arrays gives bit-identical results."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(2)
    iv = intervals["q1_10x10x20/seed2"]
    Y = workloads.random_Y(op.N, wl.M0, 1002)
    h = F().Handle()
    lam_h = np.zeros(wl.M0)
    X_h = np.zeros((wl.M0, op.N))
    res_h = np.zeros(wl.M0)
    hop = F().make_operator(op.nx, op.ny, op.nz, op.A27, op.B27)
    r1 = h.feast_solve(hop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, np.ascontiguousarray(Y.T), lam_h, X_h,
                       res_h, allow=())
    dop, keep = dev_op(op)
    lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
    r2 = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, cm(Y), lam, X, None, allow=())
    assert r1.m_found == r2.m_found and r1.loops == r2.loops
    assert np.array_equal(lam_h, lam.cpu().numpy())
    assert np.array_equal(X_h, X.cpu().numpy())


def test_feast_random_start_equals_explicit_splitmix_block(intervals):
    """Y0 = NULL draws the SplitMix64 block of the handle's seed on the device."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(1)
    iv = intervals["q1_10x10x20/seed1"]
    dop, keep = dev_op(op)
    h = F().Handle(seed=4242)
    out = []
    for Y0 in (None, cm(workloads.random_Y(op.N, wl.M0, 4242))):
        lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
        X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
        h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, Y0, lam, X, allow=())
        out.append((lam.cpu().numpy(), X.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_bq_not_spd_reported():
    """Sec. III.B (ii): the oracle raises BQNotSPD on this case; so must the GPU."""
    op = workloads.q1_operator(5, 5, 6)
    lam = oracle.closed_form_eigenvalues_v0(5, 5, 6)
    lmin, lmax = lam[0] - 0.1, 0.5 * (lam[0] + lam[1])
    Y = workloads.random_Y(op.N, 60, 1)
    with pytest.raises(oracle.BQNotSPD):
        oracle.feast(op, lmin, lmax, 60, 8, Y, tol=1e-12)
    dop, keep = dev_op(op)
    lam_d = torch.zeros(60, dtype=torch.float64, device="cuda")
    X = torch.zeros((60, op.N), dtype=torch.float64, device="cuda")
    with pytest.raises(F().FeastError) as ei:
        F().Handle().feast_solve(dop, lmin, lmax, 60, 8, 1e-12, cm(Y), lam_d, X, allow=())
    assert ei.value.status == F().FEAST_ERR_BQ_NOT_SPD


def test_argument_errors():
    op = workloads.q1_operator(4, 4, 4)
    dop, keep = dev_op(op)
    h = F().Handle()
    lam = torch.zeros(8, dtype=torch.float64, device="cuda")
    X = torch.zeros((8, op.N), dtype=torch.float64, device="cuda")
    for args in [(5.0, 1.0, 8, 8), (1.0, 5.0, 0, 8), (1.0, 5.0, 200, 8), (1.0, 5.0, 8, 0)]:
        with pytest.raises(F().FeastError) as ei:
            h.feast_solve(dop, args[0], args[1], args[2], args[3], 1e-12, None, lam, X, allow=())
        assert ei.value.status == F().FEAST_ERR_ARG
