"""Parity of the mixed-precision path (complex64 tensor-core factors and
solves, FP64 iterative refinement) with the CPU oracle.

The refinement stops when ||R||_F <= 1e-12 ||RHS||_F for every node, so the
node solutions must satisfy that bound when their residual is recomputed by
the oracle's own sparse product, and agree with the oracle's FP64 solution to
within the forward error that bound allows (condition number of Z_e B - A up
to ~1e4 here: 1e-8 relative).  Eigenpairs must meet the same gates as the FP64
path: eigenvalues within 1e-10 relative, residuals <= 1e-10.
"""

import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import GRIDS, _compare_feast, back, cm, dev_op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


# cross sections with n a multiple of 64 take the TMA-staged sweep update:
# 16x12 (n = 192: three panels, a ragged second row tile), 16x16 (n = 256)
GRIDS_TMA = [(16, 12, 7, 4, 5), (16, 16, 5, 4, 6)]


@pytest.mark.parametrize("nx,ny,nz,G,seed", GRIDS + GRIDS_TMA)
@pytest.mark.parametrize("k", [5, 24])
def test_node_solve_mixed_matches_oracle(nx, ny, nz, G, seed, k):
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, lam[min(12, len(lam) - 1)]
    _, _, _, Z, _ = oracle.contour_points(lmin, lmax, 8)
    RHS = np.random.default_rng(seed + 11).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    h = F().Handle(precision=F().FEAST_PREC_MIXED)
    for z in (Z[0], Z[7]):
        Qe = torch.zeros((k, op.N), dtype=torch.complex128, device="cuda")
        info = h.feast_node_solve(dop, complex(z), cm(RHS), Qe, k, precision=F().FEAST_PREC_MIXED)
        got = back(Qe)
        M = (z * B - A).astype(np.complex128)
        res = np.linalg.norm(M @ got - RHS) / np.linalg.norm(RHS)
        assert res <= 1e-12, res
        assert info.ir_resid_max <= 1e-12 and info.ir_steps_max >= 1
        ref = oracle.block_tridiag_factor(M, op.n, nz).solve(RHS.astype(np.complex128))
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_node_solve_mixed_full_cross_section_matches_oracle():
    """The 32 x 32 cross-section of the full-size workload (n = 1024: sixteen
    64-wide panels, eight 128-row tiles) with its 128 right-hand sides."""
    nx, ny, nz, G, seed, k = 32, 32, 3, 4, 7, 128
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, lam[40]
    _, _, _, Z, _ = oracle.contour_points(lmin, lmax, 8)
    RHS = np.random.default_rng(seed + 11).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    h = F().Handle(precision=F().FEAST_PREC_MIXED)
    for z in (Z[0], Z[3]):
        Qe = torch.zeros((k, op.N), dtype=torch.complex128, device="cuda")
        info = h.feast_node_solve(dop, complex(z), cm(RHS), Qe, k, precision=F().FEAST_PREC_MIXED)
        got = back(Qe)
        M = (z * B - A).astype(np.complex128)
        res = np.linalg.norm(M @ got - RHS) / np.linalg.norm(RHS)
        assert res <= 1e-12, res
        ref = oracle.block_tridiag_factor(M, op.n, nz).solve(RHS.astype(np.complex128))
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


SOLVE_TILES = ["16x4", "32x4", "64x3", "64x4"]


@pytest.mark.parametrize("nx,ny,nz,k", [(32, 32, 3, 128), (16, 12, 5, 100)])
def test_node_solve_mixed_every_solve_tile(monkeypatch, nx, ny, nz, k):
    """Every built configuration of the solve GEMM (complex columns per CTA
    tile x pipeline stages; the autotuner picks one by timing) solves to the
    same bar: 32x32 (eight full row tiles) and 16x12 (a ragged row
    tile; 100 columns: a ragged column tile at every width)."""
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(4, 3, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, lam[20]
    _, _, _, Z, _ = oracle.contour_points(lmin, lmax, 8)
    RHS = np.random.default_rng(k).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    z = Z[1]
    M = (z * B - A).astype(np.complex128)
    ref = oracle.block_tridiag_factor(M, op.n, nz).solve(RHS.astype(np.complex128))
    dop, keep = dev_op(op)
    h = F().Handle(precision=F().FEAST_PREC_MIXED)
    for tile in SOLVE_TILES:
        monkeypatch.setenv("FEAST_SOLVE_TILE", tile)
        Qe = torch.zeros((k, op.N), dtype=torch.complex128, device="cuda")
        info = h.feast_node_solve(dop, complex(z), cm(RHS), Qe, k, precision=F().FEAST_PREC_MIXED)
        got = back(Qe)
        res = np.linalg.norm(M @ got - RHS) / np.linalg.norm(RHS)
        assert res <= 1e-12, (tile, res)
        assert info.ir_resid_max <= 1e-12, tile
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), tile
    h.close()


def test_quadrature_mixed_matches_oracle():
    nx, ny, nz, G, seed = GRIDS[0]
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, 0.5 * (lam[9] + lam[10])
    k = 16
    RHS = np.random.default_rng(seed + 2).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    Q = torch.zeros((k, op.N), dtype=torch.float64, device="cuda")
    F().Handle().feast_quadrature(dop, lmin, lmax, 8, cm(RHS), Q, k, precision=F().FEAST_PREC_MIXED)
    ref, _ = oracle.quadrature_subspace(A, B, RHS, lmin, lmax, 8, op.n, nz)
    assert np.abs(back(Q) - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("nz", [1, 2, 3, 4, 7])
def test_quadrature_mixed_every_layer_count(nz):
    """Eq. 15 over few layers: the middle layer alone, chains of unequal
    length and the last layer of each chain, whose shares come from the
    product epilogue rather than a backward coupling -- every layer's share
    is added exactly once."""
    nx, ny, G, seed = 12, 11, 5, 4
    op = workloads.q1_operator(nx, ny, nz, workloads.gaussian_potential(G, seed, nx, ny, nz))
    lam = oracle.closed_form_eigenvalues_v0(nx, ny, nz)
    lmin, lmax = lam[0] - 3.0, 0.5 * (lam[5] + lam[6])
    k = 12
    RHS = np.random.default_rng(nz).standard_normal((op.N, k))
    A = oracle.assemble(op.A27, nx, ny, nz)
    B = oracle.assemble(op.B27, nx, ny, nz)
    dop, keep = dev_op(op)
    Q = torch.zeros((k, op.N), dtype=torch.float64, device="cuda")
    F().Handle().feast_quadrature(dop, lmin, lmax, 8, cm(RHS), Q, k, precision=F().FEAST_PREC_MIXED)
    ref, _ = oracle.quadrature_subspace(A, B, RHS, lmin, lmax, 8, op.n, nz)
    assert np.abs(back(Q) - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("key,seed,zero", [("q1_10x10x20/v0", 0, True)] +
                         [(f"q1_10x10x20/seed{s}", s, False) for s in range(5)])
def test_feast_solve_mixed_matches_oracle(intervals, key, seed, zero):
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(seed, zero_potential=zero)
    iv = intervals[key]
    Y = workloads.random_Y(op.N, wl.M0, 1000 + seed)
    ref = oracle.feast(op, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, Y, tol=wl.tol)
    dop, keep = dev_op(op)
    lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
    resid = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
    h = F().Handle(precision=F().FEAST_PREC_MIXED)
    r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, cm(Y), lam, X, resid, allow=())
    _compare_feast(lam.cpu().numpy(), back(X), r.m_found, r.loops, ref, op, iv["M"])
    assert resid.cpu().numpy()[:iv["M"]].max() <= 1e-10
    assert r.info.ir_resid_max <= 1e-12


def test_graph_replayed_sweeps_match_direct_launches(intervals):
    """The node-solve sweeps run from captured CUDA graphs (the first solve of
    a handle; the second runs its whole loop as one graph); with kernel timing
    on they are launched one by one.  All give the same result bit for bit."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(2)
    iv = intervals["q1_10x10x20/seed2"]
    Y = workloads.random_Y(op.N, wl.M0, 1002)
    dop, keep = dev_op(op)
    runs = []
    for profile in (False, True):
        h = F().Handle(precision=F().FEAST_PREC_MIXED, profile=profile)
        for _ in range(2):
            lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
            X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
            r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, cm(Y), lam, X, None, allow=())
            runs.append((profile, lam.cpu().numpy(), back(X), (r.info.sweep_graphs, r.info.loop_graphs), r.m_found))
        h.close()
    graphed = [x for x in runs if not x[0]]
    direct = [x for x in runs if x[0]]
    assert graphed[0][3][0] > 0 and graphed[0][3][1] == 0 and graphed[1][3][1] == 1
    assert all(x[3] == (0, 0) for x in direct)
    for g in graphed + direct[1:]:
        assert g[4] == direct[0][4] == iv["M"]
        np.testing.assert_array_equal(g[1], direct[0][1])
        np.testing.assert_array_equal(g[2], direct[0][2])


@pytest.mark.parametrize("key,seed,early", [("q1_10x10x20/seed1", 1, True), ("q1_10x10x20/seed4", 4, False)])
def test_device_loop_graph_equals_host_loop(intervals, key, seed, early):
    """The same solve three times on one handle: the first runs the loop from
    the host, the second captures it as one CUDA graph whose loop conditions
    (the refinement of every node solve and the trace test) are decided on
    the device, the third replays that graph.  The kernels and decisions are
    the same, so eigenvalues, eigenvectors, loop counts and the trace history
    are bit-identical; and they match the oracle."""
    wl = workloads.WORKLOADS["q1_10x10x20_fp64"]
    op = wl.operator(seed)
    iv = intervals[key]
    dop, keep = dev_op(op)
    h = F().Handle(precision=F().FEAST_PREC_MIXED, seed=1000 + seed, ir_early=early)
    out = []
    for rep in range(3):
        lam = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
        X = torch.zeros((wl.M0, op.N), dtype=torch.float64, device="cuda")
        resid = torch.zeros(wl.M0, dtype=torch.float64, device="cuda")
        r = h.feast_solve(dop, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, wl.tol, None, lam, X, resid, allow=())
        out.append((r, lam.cpu().numpy(), back(X), resid.cpu().numpy()))
    assert [o[0].info.loop_graphs for o in out] == [0, 1, 1]
    r0, lam0, X0, res0 = out[0]
    for r, lam, X, res in out[1:]:
        assert r.m_found == r0.m_found and r.loops == r0.loops
        assert np.array_equal(lam, lam0) and np.array_equal(X, X0) and np.array_equal(res, res0)
        assert list(r.info.trace[:r.loops]) == list(r0.info.trace[:r0.loops])
        assert r.info.ir_steps_max == r0.info.ir_steps_max
    ref = oracle.feast(op, iv["lmin"], iv["lmax"], wl.M0, wl.Ne, workloads.random_Y(op.N, wl.M0, 1000 + seed),
                       tol=wl.tol)
    _compare_feast(lam0, X0, r0.m_found, r0.loops, ref, op, iv["M"])
