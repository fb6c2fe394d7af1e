"""The full-size 32 x 32 x 400 workload (N = 409,600, the 100 lowest
eigenpairs, M0 = 128, Ne = 8) solved on the mixed path exactly as the
benchmark times it: one handle on the current stream, the library's seeded
random start, three solves so that the third replays its factorisation and
its whole loop from CUDA graphs; and once on the plain FP64 path.

The oracle cannot run FEAST at this size within a test, so the results are
checked against what it computes one by one, and against properties that
hold at any size:
- the pair count equals nu(lmax) - nu(lmin) = 100 from the oracle's inertia
  count (Sylvester's law, stored in intervals.json);
- sampled eigenvalues (k = 1, 50, 100) lie within 1e-10 relative of their
  brackets [lo, hi] from bisection on the same inertia count
  (fullsize_brackets.json, hi - lo <= 1e-11 hi);
- every eigenvalue lies in the interval, ascending;
- every residual ||Ax - lambda Bx||_1 / (||A||_1 ||x||_1), recomputed by the
  oracle's sparse product, is <= 1e-10 (the GPU's own report too);
- X^T B X = I on the 100 pairs, to 1e-9: the reduced eigensolve makes Phi
  B_Q-orthonormal to about eps cond(B_Q), and B_Q holds the 28 filtered
  directions beyond the interval down to f(lambda)^2 ~ 1e-7 of the others.
The same grid at V = 0 is checked against the closed-form spectrum.
"""

import json
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
KEY, NAME, START_SEED = "q1_32x32x400/seed0", "q1_32x32x400_fp64", 1000


def _solve(op, lmin, lmax, M0, Ne, tol, solves, precision="mixed"):
    """Solve `solves` times on one handle (the benchmark's form); returns the
    last result with lambda (M0,), X (N x M0) and the reported residuals."""
    import paper_0901_2665_gb300 as F

    A27 = torch.from_numpy(op.A27).cuda()
    B27 = torch.from_numpy(op.B27).cuda()
    dop = F.make_operator(op.nx, op.ny, op.nz, A27, B27)
    lam = torch.zeros(M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((M0, op.N), dtype=torch.float64, device="cuda")
    resid = torch.zeros(M0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    prec = F.FEAST_PREC_MIXED if precision == "mixed" else F.FEAST_PREC_FP64
    h = F.Handle(precision=prec, seed=START_SEED, stream=stream.cuda_stream)
    for _ in range(solves):
        r = h.feast_solve(dop, lmin, lmax, M0, Ne, tol, None, lam, X, resid, allow=())
    torch.cuda.synchronize()
    h.close()
    return r, lam.cpu().numpy(), X.cpu().numpy().T, resid.cpu().numpy()


def _check_pairs(op, lmin, lmax, lg, Xg, rg):
    """Properties every computed pair must have, checked on the CPU with the
    oracle's sparse operators."""
    assert np.all(np.diff(lg) >= 0) and lg[0] >= lmin and lg[-1] <= lmax
    assert rg.max() <= 1e-10
    A = oracle.assemble(op.A27, op.nx, op.ny, op.nz)
    B = oracle.assemble(op.B27, op.nx, op.ny, op.nz)
    r1, _ = oracle.residuals(A, B, lg, Xg)
    assert r1.max() <= 1e-10, r1.max()
    G = Xg.T @ (B @ Xg)
    assert np.abs(G - np.eye(len(lg))).max() <= 1e-9


def test_full_size_workload_as_benchmarked(intervals):
    wl = workloads.WORKLOADS[NAME]
    iv = intervals[KEY]
    with open(os.path.join(GOLDEN, "fullsize_brackets.json")) as f:
        brackets = json.load(f)["brackets"]
    op = wl.operator(0)
    M = iv["M"]
    r, lam, X, resid = _solve(op, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, 3)
    # the third solve replays its loop as one CUDA graph (device-side loop conditions)
    assert r.info.loop_graphs == 1
    assert r.m_found == M == iv["inertia_lmax"] - iv["inertia_lmin"]
    assert r.info.resid_max <= 1e-10
    lg = lam[:M]
    for k, b in brackets.items():
        x = lg[int(k) - 1]
        assert b["lo"] - 1e-10 * abs(x) <= x <= b["hi"] + 1e-10 * abs(x), (k, x, b)
    _check_pairs(op, iv["lmin"], iv["lmax"], lg, X[:, :M], resid[:M])


def test_full_size_workload_plain_fp64_path(intervals):
    """The plain FP64 path (complex128 block factors and solves, the baseline
    the other forms are compared with) on the same full-size workload, with
    the same oracle checks: count against the inertia certificate, the
    bracketed eigenvalues, every residual and B-orthonormality."""
    wl = workloads.WORKLOADS[NAME]
    iv = intervals[KEY]
    with open(os.path.join(GOLDEN, "fullsize_brackets.json")) as f:
        brackets = json.load(f)["brackets"]
    op = wl.operator(0)
    M = iv["M"]
    r, lam, X, resid = _solve(op, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, 1, precision="fp64")
    assert r.m_found == M == iv["inertia_lmax"] - iv["inertia_lmin"]
    assert r.info.resid_max <= 1e-10
    lg = lam[:M]
    for k, b in brackets.items():
        x = lg[int(k) - 1]
        assert b["lo"] - 1e-10 * abs(x) <= x <= b["hi"] + 1e-10 * abs(x), (k, x, b)
    _check_pairs(op, iv["lmin"], iv["lmax"], lg, X[:, :M], resid[:M])


def test_full_size_zero_potential_matches_closed_form():
    """The same grid at V = 0: all 100 eigenvalues against the tensor-product
    closed form, element by element, to 1e-10 relative.  The interval follows
    the midpoint reading of the certified intervals (lambda_100 = 47.408 and
    lambda_101 = 48.165 are 0.76 apart; the closed form gives the count)."""
    wl = workloads.WORKLOADS[NAME]
    op = wl.operator(0, zero_potential=True)
    cf = oracle.closed_form_eigenvalues_v0(op.nx, op.ny, op.nz)
    M = wl.M
    lmax = 0.5 * (cf[M - 1] + cf[M])
    lmin = cf[0] - 0.5 * (cf[M] - cf[M - 1])
    assert int(((cf >= lmin) & (cf <= lmax)).sum()) == M
    r, lam, X, resid = _solve(op, lmin, lmax, wl.M0, wl.Ne, wl.tol, 1)
    assert r.m_found == M
    assert np.abs(lam[:M] - cf[:M]).max() <= 1e-10 * np.abs(cf[:M]).max()
    _check_pairs(op, lmin, lmax, lam[:M], X[:, :M], resid[:M])
