"""FEAST for a complex Hermitian A on the GPU (Sec. III.A; Eqs. 10 and 12)
against the oracle's Hermitian loop (oracle.feast_hermitian) on the same
seeded complex start blocks.

Operators: the real Q1 operators with Peierls phases on their couplings
(workloads.peierls_operator): a uniform field along z gives a genuinely
complex Hermitian A; a pure gauge transformation of both A and B (complex B)
leaves the spectrum of the real pencil.  Tolerances are those of the real
path: eigenvalues 1e-10 relative, residuals <= 1e-10, X^H B X = I.
"""

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


def ccm(a):
    """numpy complex (N, k) -> CUDA complex128 tensor holding it column-major."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.complex128).T)).cuda()


def cback(t):
    return t.cpu().numpy().T


def dev_hop(op):
    A = torch.from_numpy(np.ascontiguousarray(op.A27.astype(np.complex128))).cuda()
    B = torch.from_numpy(np.ascontiguousarray(np.asarray(op.B27).astype(np.complex128))).cuda()
    return F().make_operator(op.nx, op.ny, op.nz, A, B), (A, B)


def _hermitian(nx, ny, nz, G, seed, flux=0.4, gauge_seed=None, gauge_B=False):
    real = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    return real, workloads.peierls_operator(real, flux=flux, gauge_seed=gauge_seed, gauge_B=gauge_B)


def _solve(op, lmin, lmax, M0, Y, Ne=8, tol=1e-12, seed=1000):
    dop, keep = dev_hop(op)
    lam = torch.zeros(M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((M0, op.N), dtype=torch.complex128, device="cuda")
    resid = torch.zeros(M0, dtype=torch.float64, device="cuda")
    h = F().Handle(seed=seed)
    r = h.feast_solve_hermitian(dop, lmin, lmax, M0, Ne, tol, None if Y is None else ccm(Y), lam, X, resid,
                                allow=())
    return r, lam.cpu().numpy(), cback(X), resid.cpu().numpy()


def _interval(lam, M):
    return lam[0] - 0.5 * (lam[M] - lam[M - 1]), 0.5 * (lam[M - 1] + lam[M])


@pytest.mark.parametrize("grid", [(5, 4, 6, 3, 17), (12, 11, 9, 5, 4), (7, 9, 10, 4, 8)])
def test_hermitian_feast_matches_oracle(grid):
    nx, ny, nz, G, seed = grid
    _, op = _hermitian(nx, ny, nz, G, seed, flux=0.35)
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    lam_d = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    M, M0 = 7, 12
    lmin, lmax = _interval(lam_d, M)
    Y = workloads.random_Y_complex(op.N, M0, 300 + seed)
    ref = oracle.feast_hermitian(op, lmin, lmax, M0, 8, Y, tol=1e-12)
    r, lam, X, resid = _solve(op, lmin, lmax, M0, Y)
    assert r.m_found == ref.m_found == M
    assert abs(r.loops - ref.loops) <= 1
    assert np.abs(lam[:M] - ref.lam[:M]).max() <= 1e-10 * np.abs(ref.lam[:M]).max()
    assert np.abs(lam[:M] - lam_d[:M]).max() <= 1e-10 * np.abs(lam_d[:M]).max()
    Xg, Xo = X[:, :M], ref.X[:, :M]
    assert np.abs(Xg.conj().T @ (B @ Xg) - np.eye(M)).max() <= 1e-10
    # eigenvectors through the B-projectors of clusters of close eigenvalues
    i = 0
    while i < M:
        j = i + 1
        while j < M and abs(ref.lam[j] - ref.lam[i]) < 1e-8 * abs(ref.lam[i]):
            j += 1
        Pg = Xg[:, i:j] @ (Xg[:, i:j].conj().T @ (B @ Xo[:, i:j]))
        assert np.abs(Pg - Xo[:, i:j]).max() <= 1e-8 * np.abs(Xo[:, i:j]).max()
        i = j
    # residuals: bounded, and equal to the oracle's recomputation pair by pair
    r1, rp = oracle.residuals(A, B, lam[:M], Xg)
    assert r1.max() <= 1e-10 and resid[:M].max() <= 1e-10
    assert np.abs(resid[:M] - r1).max() <= 2e-15
    assert r.info.resid_paper_max <= 1e-10


def test_hermitian_gauge_transformed_pencil_keeps_real_spectrum():
    """D^H (A, B) D with D = diag(exp(i chi)) (complex A and B): the GPU finds
    the eigenvalues of the real pencil (Sec. III.A allows Hermitian A; the
    phases cancel in the spectrum)."""
    real, op = _hermitian(6, 5, 7, 4, 2, flux=0.0, gauge_seed=5, gauge_B=True)
    lam_r = oracle.dense_generalized_eigh(real)[0]
    M, M0 = 6, 10
    lmin, lmax = _interval(lam_r, M)
    r, lam, X, resid = _solve(op, lmin, lmax, M0, workloads.random_Y_complex(op.N, M0, 77))
    assert r.m_found == M
    assert np.abs(lam[:M] - lam_r[:M]).max() <= 1e-10 * np.abs(lam_r[:M]).max()
    assert resid[:M].max() <= 1e-10


def test_hermitian_real_operator_matches_real_path(intervals):
    """At zero field the Hermitian path on the real 10 x 10 x 20 operator gives
    the eigenvalues of the real FP64 path (and of the oracle) to 1e-10."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    real = wl.operator(2)
    op = workloads.peierls_operator(real, flux=0.0)
    iv = intervals["q1_10x10x20/seed2"]
    M = iv["M"]
    r, lam, X, resid = _solve(op, iv["lmin"], iv["lmax"], wl.M0, None)
    ref = oracle.feast(real, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, workloads.random_Y(real.N, wl.M0, 1002), tol=1e-12)
    assert r.m_found == ref.m_found == M
    assert np.abs(lam[:M] - ref.lam[:M]).max() <= 1e-10 * np.abs(ref.lam[:M]).max()
    assert resid[:M].max() <= 1e-10


def test_hermitian_random_start_equals_explicit_block():
    """Y0 = NULL draws u(seed) + i u(seed + 1) on the device, the block of
    workloads.random_Y_complex: both runs are bit-identical."""
    _, op = _hermitian(5, 4, 6, 3, 17, flux=0.35)
    A = oracle.assemble(op.A27, 5, 4, 6).toarray()
    B = oracle.assemble(op.B27, 5, 4, 6).toarray()
    lam_d = sla.eigh(A, B, eigvals_only=True)
    lmin, lmax = _interval(lam_d, 5)
    out = []
    for Y in (None, workloads.random_Y_complex(op.N, 9, 4242)):
        r, lam, X, resid = _solve(op, lmin, lmax, 9, Y, seed=4242)
        out.append((lam, X))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_hermitian_argument_errors():
    _, op = _hermitian(4, 4, 4, 2, 1)
    dop, keep = dev_hop(op)
    lam = torch.zeros(8, dtype=torch.float64, device="cuda")
    X = torch.zeros((8, op.N), dtype=torch.complex128, device="cuda")
    h = F().Handle()
    for args in [(5.0, 1.0, 8, 8), (1.0, 5.0, 0, 8), (1.0, 5.0, 65, 8), (1.0, 5.0, 8, 0)]:
        with pytest.raises(F().FeastError) as ei:
            h.feast_solve_hermitian(dop, args[0], args[1], args[2], args[3], 1e-12, None, lam, X, allow=())
        assert ei.value.status == F().FEAST_ERR_ARG
    # host arrays are refused
    Ah, Bh = op.A27.astype(np.complex128), op.B27.astype(np.complex128)
    hop = F().make_operator(op.nx, op.ny, op.nz, Ah, Bh)
    with pytest.raises(F().FeastError) as ei:
        h.feast_solve_hermitian(hop, 1.0, 50.0, 8, 8, 1e-12, None, lam, X, allow=())
    assert ei.value.status == F().FEAST_ERR_ARG
