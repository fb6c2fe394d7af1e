"""The experiments of the paper beyond the single solve, on the GPU path:

- other contour node counts (Table III: Ne = 4 and 16 beside 8), against the
  oracle run with the same Ne;
- the k(N, M) replica construction of Sec. IV.B: k uncoupled copies make every
  eigenvalue exactly k-fold and FEAST finds k M pairs;
- a sequence of close problems (Sec. IV.C, Fig. 3): a potential changed in
  small steps, each solve started from the previous subspace, needs fewer
  refinement loops than a random start and finds the same eigenpairs.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import back, cm, dev_op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


def _prec(name):
    return F().FEAST_PREC_MIXED if name == "mixed" else F().FEAST_PREC_FP64


# Sec. III.B (ii): M0 has an upper limit beyond which B_Q is not positive
# definite.  With 16 nodes the filter is so sharp that the components of the
# M0 - M extra directions fall below the definiteness threshold of the reduced
# problem from the second loop on for M0 >= 12 on this workload (the oracle
# raises BQNotSPD), so that case runs with M0 = 11.
SWEEP_M0 = {4: 16, 16: 11}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("Ne", [4, 16])
def test_node_count_sweep_matches_oracle(intervals, Ne, precision):
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(3)
    iv = intervals["q1_10x10x20/seed3"]
    M0 = SWEEP_M0[Ne]
    Y = workloads.random_Y(op.N, M0, 1003)
    ref = oracle.feast(op, iv["lmin"], iv["lmax"], M0, Ne, Y, tol=wl.tol)
    dop, keep = dev_op(op)
    lam = torch.zeros(M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((M0, op.N), dtype=torch.float64, device="cuda")
    h = F().Handle(precision=_prec(precision))
    r = h.feast_solve(dop, iv["lmin"], iv["lmax"], M0, Ne, wl.tol, cm(Y), lam, X, None, allow=())
    M = iv["M"]
    assert r.m_found == ref.m_found == M
    got = lam.cpu().numpy()[:M]
    assert np.abs(got - ref.lam[:M]).max() <= 1e-10 * np.abs(ref.lam[:M]).max()
    assert abs(r.loops - ref.loops) <= 1
    assert r.info.resid_max <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_k_copies_give_k_fold_eigenvalues(precision):
    # 8x8 cross section: n = 64 also takes the TMA-staged sweep update
    blk = workloads.q1_operator(8, 8, 6, workloads.gaussian_potential(4, 21, 8, 8, 6))
    lam1 = oracle.dense_generalized_eigh(blk)[0]
    M, k = 8, 3
    lmin, lmax = lam1[0] - 0.5 * (lam1[M] - lam1[M - 1]), 0.5 * (lam1[M - 1] + lam1[M])
    rep = workloads.replicate_z(blk, k)
    M0 = 40
    dop, keep = dev_op(rep)
    lam = torch.zeros(M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((M0, rep.N), dtype=torch.float64, device="cuda")
    h = F().Handle(precision=_prec(precision))
    r = h.feast_solve(dop, lmin, lmax, M0, 8, 1e-12, None, lam, X, None, allow=())
    assert r.m_found == k * M
    got = np.sort(lam.cpu().numpy()[:k * M]).reshape(M, k)
    assert np.abs(got - lam1[:M, None]).max() <= 1e-10 * lam1[M - 1]
    assert r.info.resid_max <= 1e-10
    # the k copies of each eigenvector span the k decoupled slabs: B-orthonormal
    B = oracle.assemble(rep.B27, rep.nx, rep.ny, rep.nz)
    Xg = back(X)[:, :k * M]
    assert np.abs(Xg.T @ (B @ Xg) - np.eye(k * M)).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_started_sequence_of_close_problems(intervals, precision):
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    base = workloads.gaussian_potential(wl.gaussians, 0, wl.nx, wl.ny, wl.nz)
    iv = intervals["q1_10x10x20/seed0"]
    M, M0 = iv["M"], wl.M0
    h = F().Handle(precision=_prec(precision))
    lam = torch.zeros(M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((M0, wl.N), dtype=torch.float64, device="cuda")
    Xprev = None
    for t in range(4):
        pot = dataclasses.replace(base, amps=base.amps * (1.0 + 0.002 * t))
        op = workloads.q1_operator(wl.nx, wl.ny, wl.nz, pot)
        ref = np.sort(oracle.dense_generalized_eigh(op)[0])
        inside = ref[(ref >= iv["lmin"]) & (ref <= iv["lmax"])]
        dop, keep = dev_op(op)
        r_rand = h.feast_solve(dop, iv["lmin"], iv["lmax"], M0, wl.Ne, wl.tol, None, lam, X, None, allow=())
        if Xprev is not None:
            r = h.feast_solve(dop, iv["lmin"], iv["lmax"], M0, wl.Ne, wl.tol, Xprev, lam, X, None, allow=())
            assert r.loops < r_rand.loops, (t, r.loops, r_rand.loops)
        else:
            r = r_rand
        assert r.m_found == len(inside) == M
        assert np.abs(lam.cpu().numpy()[:M] - inside).max() <= 1e-10 * np.abs(inside).max()
        assert r.info.resid_max <= 1e-10
        Xprev = X.clone()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_interval_slicing_gives_the_union(precision):
    """Sec. V, level (i): adjacent slices of an interval are independent
    problems (here one batched call); together they find exactly the
    eigenpairs of the whole interval, none twice."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(1)
    lam = np.sort(oracle.dense_generalized_eigh(op)[0])
    M = 12
    cuts = [0, 4, 8, 12]   # slices of 4 eigenvalues each, cut at midpoints
    lo = [lam[0] - 0.5 * (lam[M] - lam[M - 1]) if a == 0 else 0.5 * (lam[a - 1] + lam[a]) for a in cuts[:-1]]
    hi = [0.5 * (lam[b - 1] + lam[b]) for b in cuts[1:]]
    # M0 = 7: with M0 = 8 the middle slice's B_Q fails the definiteness test
    # (Sec. III.B (ii)) in the oracle too, its eighth direction being filtered
    # to ~1e-7
    M0 = 7
    dop, keep = dev_op(op)
    n_sl = len(lo)
    lams = [torch.zeros(M0, dtype=torch.float64, device="cuda") for _ in range(n_sl)]
    Xs = [torch.zeros((M0, op.N), dtype=torch.float64, device="cuda") for _ in range(n_sl)]
    res = [torch.zeros(M0, dtype=torch.float64, device="cuda") for _ in range(n_sl)]
    h = F().Handle(precision=_prec(precision))
    st, mf, loops, sts = h.feast_solve_batched([dop] * n_sl, lo, hi, [M0] * n_sl, 8, 1e-12, None, lams, Xs, res)
    found = np.sort(np.concatenate([lams[i].cpu().numpy()[:mf[i]] for i in range(n_sl)]))
    assert list(mf) == [4, 4, 4]
    assert np.abs(found - lam[:M]).max() <= 1e-10 * lam[M - 1]
    assert max(float(res[i][:mf[i]].max()) for i in range(n_sl)) <= 1e-10


def test_inexact_inner_solves_still_converge(intervals):
    """Sec. IV.C: with node solves accurate only to 1e-3 (the first mixed
    solve, at most one refinement step) and a trace tolerance of 1e-8, FEAST still converges:
    the eigenvalues to about the square of the solve error, the residuals to
    about the solve error."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(0)
    iv = intervals["q1_10x10x20/seed0"]
    lam = np.sort(oracle.dense_generalized_eigh(op)[0])
    M = iv["M"]
    dop, keep = dev_op(op)
    lamd = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
    resid = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    h = F().Handle(precision=F().FEAST_PREC_MIXED, ir_tol=1e-3, ir_early=False)
    r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, 1e-8, None, lamd, X, resid, allow=())
    assert r.m_found == M
    assert r.info.ir_steps_max <= 1
    assert np.abs(lamd.cpu().numpy()[:M] - lam[:M]).max() <= 1e-5 * lam[M - 1]
    assert resid.cpu().numpy()[:M].max() <= 1e-3



# ---------------------------------------------------------------- iterative inner solves (Sec. IV.C)

def _cocg_handle(tol, **kw):
    return F().Handle(inner_solver=F().FEAST_INNER_COCG, inner_tol=tol, **kw)


@pytest.mark.parametrize("tol", [1e-3, 1e-10])
def test_cocg_node_solve_meets_its_tolerance(tol):
    """The iterative inner solver (Jacobi-preconditioned COCG) on a ragged
    grid, at the node nearest the middle of the contour and the one closest to
    the real axis: every column's residual ||(Z B - A) q - b||_2 / ||b||_2,
    recomputed by the oracle's sparse product, meets the tolerance, and q is
    within (tolerance x condition) of the oracle's direct block solve."""
    nx, ny, nz = 12, 11, 9
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(5, 4, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, lam[12]
    _, _, _, Z, _ = oracle.contour_points(lmin, lmax, 8)
    k = 24
    RHS = np.random.default_rng(11).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    h = _cocg_handle(tol)
    for z in (Z[0], Z[7]):
        Qe = torch.zeros((k, op.N), dtype=torch.complex128, device="cuda")
        info = h.feast_node_solve(dop, complex(z), cm(RHS), Qe, k)
        assert info.inner_iters_max > 0 and info.inner_rel_max <= tol
        q = back(Qe)
        M = (z * B - A).astype(np.complex128)
        rel = np.linalg.norm(M @ q - RHS, axis=0) / np.linalg.norm(RHS, axis=0)
        assert rel.max() <= 1.5 * tol, (z, rel.max())
        ref = oracle.block_tridiag_factor(M, op.n, nz).solve(RHS.astype(np.complex128))
        assert np.abs(q - ref).max() <= max(3e4 * tol, 1e-12) * np.abs(ref).max()


def test_iterative_inner_solves_example_iii(intervals):
    """Sec. IV.C settings: inner systems solved iteratively to a relative
    residual of 1e-3, trace tolerance 1e-8.  FEAST still finds every pair of
    the interval, the eigenvalues to well below the inner tolerance (1e-5
    relative against the dense pencil) and residuals in the paper's range
    (<= 1e-3)."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(0)
    iv = intervals["q1_10x10x20/seed0"]
    lam = np.sort(oracle.dense_generalized_eigh(op)[0])
    M = iv["M"]
    dop, keep = dev_op(op)
    lamd = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
    resid = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    h = _cocg_handle(1e-3)
    r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, 1e-8, None, lamd, X, resid, allow=())
    assert r.m_found == M and r.info.factor_flops == 0
    assert 0 < r.info.inner_iters_max < 5000 and r.info.inner_rel_max <= 1e-3
    assert np.abs(lamd.cpu().numpy()[:M] - lam[:M]).max() <= 1e-5 * lam[M - 1]
    assert resid.cpu().numpy()[:M].max() <= 1e-3
    # the residuals the solve reports are the oracle's, pair by pair
    r1, _ = oracle.residuals(oracle.assemble(op.A27, 10, 10, 20), oracle.assemble(op.B27, 10, 10, 20),
                             lamd.cpu().numpy()[:M], back(X)[:, :M])
    assert np.abs(resid.cpu().numpy()[:M] - r1).max() <= 1e-12 * r1.max()


def test_iterative_inner_solves_warm_sequence():
    """Fig. 3 in miniature: a potential changed in small steps, inner systems
    solved iteratively (to 1e-4 here; at 1e-3 the inexact solves perturb
    the trace from loop to loop by about the 1e-8 tolerance on a problem this
    small, so the loop count turns noisy), trace tolerance 1e-8.  Every
    problem yields the dense pencil's eigenvalues to 1e-5 from a random start
    and from the previous problem's subspace; the warm start's first loop is
    at least ten times closer to the converged trace, and it needs no more
    loops than the random start."""
    nx, ny, nz, M, M0 = 8, 8, 12, 8, 14
    base = workloads.gaussian_potential(6, 21, nx, ny, nz)
    h = _cocg_handle(1e-4)
    Xprev = None
    for t in range(4):
        pot = dataclasses.replace(base, amps=base.amps * (1.0 + 0.01 * t))
        op = workloads.q1_operator(nx, ny, nz, pot)
        lam = oracle.dense_generalized_eigh(op)[0]
        if t == 0:
            lmin, lmax = lam[0] - 0.5 * (lam[M] - lam[M - 1]), 0.5 * (lam[M - 1] + lam[M])
        inside = (lam >= lmin) & (lam <= lmax)
        ref = lam[inside]
        m_in = int(inside.sum())
        dop, keep = dev_op(op)
        first_err, loops, Xout = {}, {}, {}
        for start in ("random", "warm"):
            if start == "warm" and Xprev is None:
                continue
            lamd = torch.zeros(M0, dtype=torch.float64, device="cuda")
            X = torch.zeros((M0, op.N), dtype=torch.float64, device="cuda")
            r = h.feast_solve(dop, lmin, lmax, M0, 8, 1e-8, Xprev if start == "warm" else None, lamd, X, allow=())
            assert r.m_found == m_in, (t, start)
            got = lamd.cpu().numpy()[:m_in]
            assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), (t, start)
            first_err[start] = abs(r.info.trace[0] - ref.sum()) / np.abs(ref).sum()
            loops[start] = r.loops
            Xout[start] = X.clone()
        if "warm" in first_err:
            assert first_err["warm"] <= 0.1 * first_err["random"], (t, first_err)
            assert loops["warm"] <= loops["random"], (t, loops)
        Xprev = Xout.get("warm", Xout["random"])
