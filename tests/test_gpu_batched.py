"""Batched solves (many independent instances of uneven size, Sec. V
parallelism level (i)) through feast_solve_batched: every instance must match
the oracle at the eigenpair gates and be bit-identical to its own
feast_solve (same kernels, deterministic), for both precisions."""

import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import back, cm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (nx, ny, nz, M0, M, potential seed): layer sizes 64/90/144/42/81, ragged
SPECS = [(8, 8, 12, 16, 9, 31), (10, 9, 15, 24, 15, 32), (12, 12, 7, 16, 10, 33), (7, 6, 20, 12, 7, 34),
         (9, 9, 9, 20, 12, 35)]


def _instances():
    out = []
    for nx, ny, nz, M0, M, seed in SPECS:
        op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(4, seed, nx, ny, nz))
        lam = oracle.dense_generalized_eigh(op)[0]
        lmin = lam[0] - 0.5 * (lam[M] - lam[M - 1])
        lmax = 0.5 * (lam[M - 1] + lam[M])
        Y = workloads.random_Y(op.N, M0, 500 + seed)
        out.append((op, lmin, lmax, M0, M, Y))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_matches_oracle_and_single_solves(precision):
    import paper_0901_2665_gb300 as F
    prec = F.FEAST_PREC_MIXED if precision == "mixed" else F.FEAST_PREC_FP64
    inst = _instances()
    keep, ops, lo, hi, m0s, Ys, lams, Xs, res = [], [], [], [], [], [], [], [], []
    for op, lmin, lmax, M0, M, Y in inst:
        A = torch.from_numpy(op.A27).cuda()
        B = torch.from_numpy(op.B27).cuda()
        keep += [A, B]
        ops.append(F.make_operator(op.nx, op.ny, op.nz, A, B))
        lo.append(lmin)
        hi.append(lmax)
        m0s.append(M0)
        Ys.append(cm(Y))
        lams.append(torch.zeros(M0, dtype=torch.float64, device="cuda"))
        Xs.append(torch.zeros((M0, op.N), dtype=torch.float64, device="cuda"))
        res.append(torch.zeros(M0, dtype=torch.float64, device="cuda"))
    h = F.Handle(precision=prec)
    st, mf, lp, sts = h.feast_solve_batched(ops, lo, hi, m0s, 8, 1e-12, Ys, lams, Xs, res, workers=3)
    assert st == F.FEAST_OK and (sts == 0).all()
    for i, (op, lmin, lmax, M0, M, Y) in enumerate(inst):
        ref = oracle.feast(op, lmin, lmax, M0, 8, Y, tol=1e-12)
        lam = lams[i].cpu().numpy()
        assert mf[i] == ref.m_found == M
        assert np.abs(lam[:M] - ref.lam[:M]).max() <= 1e-10 * np.abs(ref.lam[:M]).max()
        assert res[i].cpu().numpy()[:M].max() <= 1e-10
        # identical to the single-instance call
        lam1 = torch.zeros(M0, dtype=torch.float64, device="cuda")
        X1 = torch.zeros((M0, op.N), dtype=torch.float64, device="cuda")
        r1 = h.feast_solve(ops[i], lmin, lmax, M0, 8, 1e-12, Ys[i], lam1, X1, allow=())
        assert r1.m_found == mf[i] and r1.loops == lp[i]
        assert torch.equal(lam1, lams[i]) and torch.equal(X1, Xs[i])


def test_batched_reports_failing_instance():
    """A failing instance (B_Q not s.p.d.) is reported in its status while the
    others still succeed."""
    import paper_0901_2665_gb300 as F
    inst = _instances()[:2]
    bad = workloads.q1_operator(5, 5, 6)
    lamb = oracle.closed_form_eigenvalues_v0(5, 5, 6)
    keep, ops, lo, hi, m0s, lams, Xs = [], [], [], [], [], [], []
    cases = [(op, lmin, lmax, M0) for op, lmin, lmax, M0, M, Y in inst]
    cases.append((bad, lamb[0] - 0.1, 0.5 * (lamb[0] + lamb[1]), 60))
    for op, lmin, lmax, M0 in cases:
        A = torch.from_numpy(op.A27).cuda()
        B = torch.from_numpy(op.B27).cuda()
        keep += [A, B]
        ops.append(F.make_operator(op.nx, op.ny, op.nz, A, B))
        lo.append(lmin)
        hi.append(lmax)
        m0s.append(M0)
        lams.append(torch.zeros(M0, dtype=torch.float64, device="cuda"))
        Xs.append(torch.zeros((M0, op.N), dtype=torch.float64, device="cuda"))
    h = F.Handle()
    st, mf, lp, sts = h.feast_solve_batched(ops, lo, hi, m0s, 8, 1e-12, None, lams, Xs, None, workers=2,
                                            raise_on_error=False)
    assert st == F.FEAST_ERR_BQ_NOT_SPD
    assert list(sts) == [F.FEAST_OK, F.FEAST_OK, F.FEAST_ERR_BQ_NOT_SPD]
    assert "instance 2" in h.last_error()
