"""The learned-start network's GPU kernels against the CPU reference
(oracle/mlp.py): forward output, loss and every gradient with the bfloat16
rounding points emulated on the CPU; the sine-basis expansion and projection;
and that Adam steps reduce the loss.

Tolerances: the GPU accumulates in fp32 and evaluates SiLU with the fast
exponential; a value that lands next to a bfloat16 rounding boundary can round
one unit (2^-8) differently, so gradients agree to 1e-2 relative in Frobenius
norm (typically ~1e-4) and the loss to 1e-4.
"""

import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


def _net(sizes, seed):
    params = mlp.init_params(sizes, seed)
    rng = np.random.default_rng(seed + 1)
    return [(W.astype(np.float32).astype(np.float64), (rng.standard_normal(b.shape) * 0.1).astype(np.float32)
             .astype(np.float64)) for W, b in params]


def _upload(net, params):
    for k, (W, b) in enumerate(params):
        net.feast_mlp_set_layer(k, np.ascontiguousarray(W, dtype=np.float32), np.ascontiguousarray(b, dtype=np.float32))


@pytest.mark.parametrize("B", [200, 256])
def test_mlp_gradients_match_reference(B):
    sizes = [10, 128, 128, 128, 256]
    params = _net(sizes, 3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((B, 10)).astype(np.float32)
    T = rng.standard_normal((B, 256)).astype(np.float32)
    w = rng.uniform(0.25, 1.0, 256).astype(np.float32)
    net = F().Mlp(10, 128, 256, 256)
    _upload(net, params)
    out = torch.zeros((B, 256), dtype=torch.float32, device="cuda")
    net.feast_mlp_forward(torch.from_numpy(X).cuda(), B, out)
    ref_out, cache = mlp.forward(params, X.astype(np.float64), bf16=True)
    assert np.abs(out.cpu().numpy() - ref_out).max() <= 2e-2 * np.abs(ref_out).max()
    loss = net.feast_mlp_train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(w).cuda(),
                                    B, 0.0)
    ref_loss = mlp.loss(ref_out, T.astype(np.float64), w.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    grads = mlp.backward(params, cache, ref_out, T.astype(np.float64), w.astype(np.float64), bf16=True)
    for k, (gW_ref, gb_ref) in enumerate(grads):
        gW = np.zeros(gW_ref.shape, dtype=np.float32)
        gb = np.zeros(gb_ref.shape, dtype=np.float32)
        net.feast_mlp_get_layer(k, gW=gW, gb=gb)
        assert np.linalg.norm(gW - gW_ref) <= 1e-2 * np.linalg.norm(gW_ref), k
        assert np.linalg.norm(gb - gb_ref) <= 1e-2 * np.linalg.norm(gb_ref), k


def test_mlp_adam_first_step_is_sign_step():
    """Adam's first step with zero moments moves every parameter by
    -lr * g / (|g| + eps), i.e. -lr * sign(g) wherever |g| >> eps; checked
    against the reference gradients where their sign is not in doubt."""
    sizes = [10, 128, 128, 128, 256]
    params = _net(sizes, 8)
    rng = np.random.default_rng(9)
    B, lr = 256, 1e-3
    X = rng.standard_normal((B, 10)).astype(np.float32)
    T = rng.standard_normal((B, 256)).astype(np.float32)
    w = np.ones(256, dtype=np.float32)
    net = F().Mlp(10, 128, 256, B)
    _upload(net, params)
    net.feast_mlp_train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(w).cuda(), B, lr)
    ref_out, cache = mlp.forward(params, X.astype(np.float64), bf16=True)
    grads = mlp.backward(params, cache, ref_out, T.astype(np.float64), w.astype(np.float64), bf16=True)
    for k, ((W0, b0), (gW, gb)) in enumerate(zip(params, grads)):
        W1 = np.zeros(W0.shape, dtype=np.float32)
        b1 = np.zeros(b0.shape, dtype=np.float32)
        net.feast_mlp_get_layer(k, W=W1, b=b1)
        for p0, p1, g in ((W0, W1, gW), (b0, b1, gb)):
            sure = np.abs(g) > 0.05 * np.abs(g).max()
            step = (p1 - p0)[sure]
            assert sure.sum() > 0
            assert np.allclose(step, -lr * np.sign(g[sure]), rtol=1e-3, atol=2e-6), k


def test_mlp_adam_steps_reduce_loss():
    """A smooth target (tanh of a linear map of the input) is fitted: 200 Adam
    steps cut the loss by more than 5x."""
    sizes = [10, 128, 128, 128, 128]
    params = _net(sizes, 5)
    rng = np.random.default_rng(6)
    B = 384
    Xh = rng.standard_normal((B, 10))
    R = rng.standard_normal((10, 128)) / np.sqrt(10)
    X = torch.from_numpy(Xh.astype(np.float32)).cuda()
    T = torch.from_numpy(np.tanh(Xh @ R).astype(np.float32)).cuda()
    w = torch.ones(128, dtype=torch.float32, device="cuda")
    net = F().Mlp(10, 128, 128, B)
    _upload(net, params)
    first = net.feast_mlp_train_step(X, T, w, B, 2e-3)
    for _ in range(200):
        last = net.feast_mlp_train_step(X, T, w, B, 2e-3)
    assert np.isfinite(last) and last < 0.2 * first


def test_sine_expand_and_project_match_reference():
    rng = np.random.default_rng(7)
    nx, ny, nz, M0, px, py = 12, 9, 5, 6, 4, 3
    coef = rng.standard_normal((nz, M0, px * py)).astype(np.float32)
    Y = torch.zeros((M0, nx * ny * nz), dtype=torch.float64, device="cuda")
    F().feast_sine_expand(torch.from_numpy(coef).cuda(), nx, ny, nz, M0, px, py, Y)
    ref = mlp.expand(coef.astype(np.float64), nx, ny, nz, px, py)
    assert np.abs(Y.cpu().numpy().T - ref).max() <= 1e-5 * np.abs(ref).max()
    X = rng.standard_normal((nx * ny * nz, M0))
    C = torch.zeros((nz, M0, px * py), dtype=torch.float32, device="cuda")
    F().feast_sine_project(torch.from_numpy(np.ascontiguousarray(X.T)).cuda(), nx, ny, nz, M0, px, py, C)
    refc = mlp.project(X, nx, ny, nz, px, py)
    assert np.abs(C.cpu().numpy() - refc).max() <= 1e-4 * np.abs(refc).max()


def test_trained_network_saves_a_loop_on_held_out_instances():
    """The committed network (trained on 2000 converged instances of the
    24x24x100 family) starts FEAST on held-out instances whose intervals the
    oracle certified: same eigenvalues and residual gate as the random start,
    one refinement loop fewer at trace tolerance 1e-10, and the eigenvalues
    of the learned start equal the oracle's converged FEAST (stored for one
    instance) to 1e-10."""
    import json
    import os

    import paper_0901_2665_gb300 as F
    from paper_0901_2665_gb300 import learned as L

    with open(os.path.join(os.path.dirname(__file__), "golden", "learned_intervals.json")) as f:
        ivs = json.load(f)
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_eigenvalues.json")) as f:
        gold = json.load(f)
    assert ivs
    net = L.load_weights()
    h = F.Handle(precision=F.FEAST_PREC_MIXED)
    compared = 0
    for key in sorted(ivs):
        iv = ivs[key]
        op = L.operator(iv["seed"])
        A = torch.from_numpy(op.A27).cuda()
        B = torch.from_numpy(op.B27).cuda()
        dop = F.make_operator(op.nx, op.ny, op.nz, A, B)
        lam = torch.zeros(L.M0, dtype=torch.float64, device="cuda")
        X = torch.zeros((L.M0, op.N), dtype=torch.float64, device="cuda")
        r0, _ = L.solve(h, dop, iv["lmin"], iv["lmax"], None, lam, X, torch, tol=1e-10)
        lam0 = lam.cpu().numpy()[:iv["M"]].copy()
        r1, _, used = L.learned_solve(h, net, iv["seed"], dop, iv["lmin"], iv["lmax"], lam, X, torch, tol=1e-10)
        lam1 = lam.cpu().numpy()[:iv["M"]]
        assert used == F.FEAST_OK, key
        assert r0.m_found == r1.m_found == iv["M"], key
        assert np.abs(lam1 - lam0).max() <= 1e-10 * np.abs(lam0).max(), key
        assert r0.info.resid_max <= 1e-10 and r1.info.resid_max <= 1e-10, key
        assert r1.loops < r0.loops, (key, r0.loops, r1.loops)
        g = gold.get(f"learned/{iv['seed']}")
        if g is not None:
            # the learned start's eigenvalues against the oracle's own FEAST
            ref = np.array(g["lam"])
            assert g["m_found"] == iv["M"]
            assert np.abs(lam1 - ref).max() <= 1e-10 * np.abs(ref).max(), key
            compared += 1
    assert compared >= 1
