"""Learned initial subspace for FEAST (form 4): data, training and use.

A family of instances shares a Q1 grid (24x24x100) and 16 Gaussian potential
terms whose (x, y) centres are fixed for the family; each instance draws the
z-centre, width and amplitude of every term (48 scalars).  The network maps
per-layer features -- those 48 scalars (terms ordered by z-centre, fixed
affine scaling), the search interval and the layer position -- to the
coefficients of the start block Y on the layer's 8x8 separable sine basis.

Training target.  FEAST needs only the span of the wanted eigenvectors, so the
loss must not depend on their signs or on the basis chosen inside the span.
The target is therefore the spectral projector (the density matrix of Eq. 3,
restricted to the sine basis) applied to a fixed probe block: with U an
orthonormal basis of the coefficient vectors of the M wanted Ritz vectors and
S fixed seeded probes, columns c < M hold sqrt(D/M) U U^T s_c (D = nz*px*py)
and columns c >= M hold s_c itself, which keeps Y of full rank M0 (the start
block of an ideal filter, Eq. 15, applied to the probes).

The network, the projection onto the basis and the expansion run in the
library's kernels; this module marshals arrays, orders the calls and prepares
the training labels (a QR of a D x M matrix per instance, on the host: data
preparation, not part of a solve).  A learned start that FEAST rejects (B_Q not
positive definite, a failed reduced eigensolve or pivot, a non-finite block)
falls back to the random start.
"""

from __future__ import annotations

import dataclasses
import os
import time

import numpy as np

import workloads

from . import FEAST_ERR_BQ_NOT_SPD, FEAST_ERR_JACOBI, FEAST_ERR_NONFINITE, FEAST_ERR_PIVOT, FEAST_OK, \
    FEAST_PREC_MIXED, FeastError, Handle, Mlp, feast_sine_project, make_operator

NX, NY, NZ = 24, 24, 100
GAUSSIANS = 16
M, M0, NE = 40, 64, 8
PX = PY = 8
IN_DIM = 3 * GAUSSIANS + 3
WIDTH = 512
OUT_DIM = M0 * PX * PY
FAMILY_XY_SEED = 4
PROBE_SEED = 77
D = NZ * PX * PY
TOL = 1e-12
FALLBACK = (FEAST_ERR_BQ_NOT_SPD, FEAST_ERR_JACOBI, FEAST_ERR_PIVOT, FEAST_ERR_NONFINITE)


def potential(seed: int):
    return workloads.gaussian_potential(GAUSSIANS, seed, NX, NY, NZ, fixed_xy_seed=FAMILY_XY_SEED)


def operator(seed: int) -> workloads.Operator:
    return workloads.q1_operator(NX, NY, NZ, potential(seed))


def features(seed: int, lmin: float, lmax: float) -> np.ndarray:
    """(NZ, IN_DIM) float32 features of every layer of instance `seed`."""
    pot = potential(seed)
    _, Lx, _, Lz = workloads.box_lengths(NX, NY, NZ)
    order = np.argsort(pot.centres[:, 2])
    cz = pot.centres[order, 2] / Lz * 2.0 - 1.0
    w = (pot.sigmas[order] / Lx - 0.2) / 0.1
    a = pot.amps[order] + 1.0
    inst = np.concatenate([cz, w, a, [(lmin - 30.0) / 20.0, (lmax - 30.0) / 20.0]])
    z = (np.arange(NZ) + 1.0) / (NZ + 1.0) * 2.0 - 1.0
    return np.concatenate([np.repeat(inst[None, :], NZ, axis=0), z[:, None]], axis=1).astype(np.float32)


def loss_weights() -> np.ndarray:
    """Projector columns weigh 1; the probe columns (a constant target) 1/4."""
    w = np.full((M0, PX * PY), 0.25, dtype=np.float32)
    w[:M] = 1.0
    return w.ravel()


def probes() -> np.ndarray:
    """Fixed probe block S (D x M0) of standard normal entries in coefficient
    space (row l*PX*PY + pq), so that targets have entries of unit size."""
    return np.random.default_rng(PROBE_SEED).standard_normal((D, M0))


def to_columns(coef: np.ndarray) -> np.ndarray:
    """(NZ, M0', PX*PY) layer-major coefficients -> (D, M0') columns."""
    return coef.transpose(0, 2, 1).reshape(D, coef.shape[1])


def to_layers(cols: np.ndarray) -> np.ndarray:
    """(D, M0') columns -> (NZ, M0' * PX*PY) rows of the network's output."""
    return cols.reshape(NZ, PX * PY, cols.shape[1]).transpose(0, 2, 1).reshape(NZ, -1)


def subspace_target(coef_wanted: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Target rows (NZ, M0*PX*PY) for the wanted Ritz vectors' coefficients
    coef_wanted (NZ, M, PX*PY): projector columns, then probe columns."""
    U, _ = np.linalg.qr(to_columns(coef_wanted.astype(np.float64)))
    T = np.concatenate([np.sqrt(D / M) * (U @ (U.T @ S[:, :M])), S[:, M:]], axis=1)
    return to_layers(T).astype(np.float32)


def subspace_sines(pred_rows: np.ndarray, U: np.ndarray):
    """Largest and mean sine of the principal angles between span(U) (D x M,
    orthonormal) and the span of all M0 predicted columns."""
    P = to_columns(pred_rows.reshape(NZ, M0, PX * PY).astype(np.float64))
    Qp, _ = np.linalg.qr(P)
    c = np.clip(np.linalg.svd(U.T @ Qp, compute_uv=False), 0.0, 1.0)
    s = np.sqrt(1.0 - c ** 2)
    return float(s.max()), float(s.mean())


def wide_interval(seed: int):
    """An interval that surely starts below the spectrum and holds more than M
    eigenvalues (the V = 0 spectrum shifted by the potential's minimum)."""
    h = 1.0 / (NX + 1)
    ix, iy, iz = workloads.grid_index(NX, NY, NZ)
    vmin = float(potential(seed)((ix + 1) * h, (iy + 1) * h, (iz + 1) * h).min())

    def mu(m):
        t = np.arange(1, m + 1) * np.pi / (m + 1)
        return (6.0 / h ** 2) * (1.0 - np.cos(t)) / (2.0 + np.cos(t))

    lam0 = np.sort((0.5 * (mu(NX)[:, None, None] + mu(NY)[None, :, None] + mu(NZ)[None, None, :])).ravel())
    return float(lam0[0] + vmin - 1.0), float(lam0[M + 3])


@dataclasses.dataclass
class Sample:
    seed: int
    lmin: float
    lmax: float
    feats: np.ndarray       # (NZ, IN_DIM)
    coef: np.ndarray        # (NZ, M0 * PX * PY) targets
    U: np.ndarray           # (D, M) orthonormal basis of the wanted coefficients
    trunc: float            # largest sine of a wanted vector to the sine basis


def generate(seeds, torch, workers: int = 4, log=None):
    """Converged FEAST subspaces for `seeds` (mixed precision, batched), their
    lowest-M intervals and projector targets."""
    dev = torch.device("cuda")
    h = Handle(precision=FEAST_PREC_MIXED)
    S = probes()
    out = []
    chunk = 16
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        keep, ops, lo, hi, m0s, lams, Xs = [], [], [], [], [], [], []
        for s in part:
            op = operator(s)
            A = torch.from_numpy(op.A27).to(dev)
            B = torch.from_numpy(op.B27).to(dev)
            keep += [A, B]
            ops.append(make_operator(NX, NY, NZ, A, B))
            l0, l1 = wide_interval(s)
            lo.append(l0)
            hi.append(l1)
            m0s.append(M0)
            lams.append(torch.zeros(M0, dtype=torch.float64, device=dev))
            Xs.append(torch.zeros((M0, op.N), dtype=torch.float64, device=dev))
        st, mf, lp, sts = h.feast_solve_batched(ops, lo, hi, m0s, NE, TOL, None, lams, Xs, None, workers=workers,
                                                raise_on_error=False)
        for i, s in enumerate(part):
            if sts[i] != FEAST_OK or mf[i] <= M:
                continue
            # in-interval pairs come first, ascending: columns 0..M-1 are the lowest M
            inside = lams[i].cpu().numpy()[:mf[i]]
            lmin = float(inside[0] - 0.5 * (inside[M] - inside[M - 1]))
            lmax = float(0.5 * (inside[M - 1] + inside[M]))
            coef = torch.zeros((NZ, M0, PX * PY), dtype=torch.float32, device=dev)
            feast_sine_project(Xs[i], NX, NY, NZ, M0, PX, PY, coef)
            C = coef.cpu().numpy()[:, :M, :]
            xn = np.linalg.norm(Xs[i][:M].cpu().numpy(), axis=1)
            cn = np.sqrt((C.astype(np.float64) ** 2).sum(axis=(0, 2)))
            trunc = float(np.sqrt(np.clip(1.0 - (cn / xn) ** 2, 0.0, 1.0)).max())
            U, _ = np.linalg.qr(to_columns(C.astype(np.float64)))
            out.append(Sample(s, lmin, lmax, features(s, lmin, lmax), subspace_target(C, S), U, trunc))
        if log:
            log(f"generated {len(out)} / {c0 + len(part)}")
    h.close()
    return out


def init_params(seed: int):
    """W ~ N(0, 1/fan_in), b = 0 for the four layers (numpy, host)."""
    rng = np.random.default_rng(seed)
    sizes = [IN_DIM, WIDTH, WIDTH, WIDTH, OUT_DIM]
    return [((rng.standard_normal((fo, fi)) / np.sqrt(fi)).astype(np.float32), np.zeros(fo, dtype=np.float32))
            for fi, fo in zip(sizes[:-1], sizes[1:])]


def predict_rows(net: Mlp, samples, torch) -> np.ndarray:
    """Network output rows (n, NZ, OUT_DIM) for the samples' features."""
    dev = torch.device("cuda")
    per = max(1, net_capacity(net) // NZ)
    out = np.zeros((len(samples), NZ, OUT_DIM), dtype=np.float32)
    for b0 in range(0, len(samples), per):
        part = samples[b0:b0 + per]
        x = torch.from_numpy(np.concatenate([s.feats for s in part])).to(dev)
        y = torch.zeros((len(part) * NZ, OUT_DIM), dtype=torch.float32, device=dev)
        net.feast_mlp_forward(x, len(part) * NZ, y)
        out[b0:b0 + len(part)] = y.cpu().numpy().reshape(len(part), NZ, OUT_DIM)
    return out


def net_capacity(net: Mlp) -> int:
    return net.max_batch


def validate(net: Mlp, samples, torch):
    """Mean over samples of the largest and of the mean principal-angle sine
    between the wanted coefficient space and the predicted span."""
    pred = predict_rows(net, samples, torch)
    r = np.array([subspace_sines(p, s.U) for p, s in zip(pred, samples)])
    return float(r[:, 0].mean()), float(r[:, 1].mean())


def train_network(samples, torch, epochs: int = 40, batch_instances: int = 32, lr: float = 1e-3, lr_end: float = 1e-5,
                  seed: int = 0, val=None, val_every: int = 10, log=None):
    """Trains a fresh network on `samples` with the library's kernels (Adam with
    a cosine learning-rate decay, minibatches of whole instances gathered on
    the host).  Returns (net, per-epoch losses, validation history)."""
    dev = torch.device("cuda")
    X = np.stack([s.feats for s in samples])          # (n, NZ, IN_DIM)
    T = np.stack([s.coef for s in samples])           # (n, NZ, OUT_DIM)
    wd = torch.from_numpy(loss_weights()).to(dev)
    rows = batch_instances * NZ
    net = Mlp(IN_DIM, WIDTH, OUT_DIM, rows)
    for k, (W, b) in enumerate(init_params(seed)):
        net.feast_mlp_set_layer(k, W, b)
    rng = np.random.default_rng(seed + 1)
    losses, history = [], []
    n = len(samples)
    steps_per_epoch = (n + batch_instances - 1) // batch_instances
    total = epochs * steps_per_epoch
    step = 0
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n, batch_instances):
            idx = np.sort(perm[b0:b0 + batch_instances])
            a = lr_end + 0.5 * (lr - lr_end) * (1.0 + np.cos(np.pi * step / total))
            xb = torch.from_numpy(np.ascontiguousarray(X[idx].reshape(-1, IN_DIM))).to(dev)
            tb = torch.from_numpy(np.ascontiguousarray(T[idx].reshape(-1, OUT_DIM))).to(dev)
            tot += net.feast_mlp_train_step(xb, tb, wd, len(idx) * NZ, a) * len(idx)
            step += 1
        losses.append(tot / n)
        msg = f"epoch {ep}: loss {losses[-1]:.4e}"
        if val is not None and ((ep + 1) % val_every == 0 or ep == epochs - 1):
            vmax, vmean = validate(net, val, torch)
            history.append(dict(epoch=ep, loss=losses[-1], sin_max=vmax, sin_mean=vmean))
            msg += f"  held-out sin(angle) max {vmax:.3e} mean {vmean:.3e}"
        if log:
            log(msg)
    return net, losses, history


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "learned_start_24x24x100.npz")


def save_weights(net: Mlp, path: str):
    """The four layers as an .npz: W_k as bfloat16 bit patterns (uint16, the
    values the forward kernels read), b_k in fp32."""
    sizes = [IN_DIM, WIDTH, WIDTH, WIDTH, OUT_DIM]
    arrs = {}
    for k in range(4):
        W = np.zeros((sizes[k + 1], sizes[k]), dtype=np.float32)
        b = np.zeros(sizes[k + 1], dtype=np.float32)
        net.feast_mlp_get_layer(k, W=W, b=b)
        u = W.view(np.uint32).astype(np.uint64)
        arrs[f"W{k}"] = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)   # nearest even
        arrs[f"b{k}"] = b
    np.savez_compressed(path, **arrs)


def load_weights(path: str = WEIGHTS, max_batch: int = NZ) -> Mlp:
    z = np.load(path)
    net = Mlp(IN_DIM, WIDTH, OUT_DIM, max_batch)
    for k in range(4):
        W = z[f"W{k}"]
        if W.dtype == np.uint16:
            W = (W.astype(np.uint32) << 16).view(np.float32)
        net.feast_mlp_set_layer(k, np.ascontiguousarray(W, dtype=np.float32), np.ascontiguousarray(z[f"b{k}"]))
    return net


def solve(h: Handle, op_dev, lmin, lmax, Y0, lam, X, torch, tol=TOL):
    """FEAST from start block Y0 (None = random); returns (result, seconds)."""
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = h.feast_solve(op_dev, lmin, lmax, M0, NE, tol, Y0, lam, X)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t


def learned_solve(h: Handle, net: Mlp, seed: int, op_dev, lmin, lmax, lam, X, torch, tol=TOL):
    """FEAST from the network's start block, falling back to the random start
    when FEAST rejects that block.  Returns (result, seconds, fallback status
    or FEAST_OK when the learned block was used)."""
    dev = torch.device("cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    Y = torch.empty((M0, NX * NY * NZ), dtype=torch.float64, device=dev)
    used = FEAST_OK
    try:
        net.feast_predict_Y(torch.from_numpy(features(seed, lmin, lmax)).to(dev), NX, NY, NZ, M0, PX, PY, Y)
        r = h.feast_solve(op_dev, lmin, lmax, M0, NE, tol, Y, lam, X)
    except FeastError as ex:
        if ex.status not in FALLBACK:
            raise
        used = ex.status
        r = h.feast_solve(op_dev, lmin, lmax, M0, NE, tol, None, lam, X)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t, used


def evaluate(h: Handle, net: Mlp, samples, torch, tols=(1e-10, TOL)):
    """Per held-out instance and stopping tolerance: loops, time and residual
    of the random and the learned start, and whether both found the same
    eigenvalues."""
    dev = torch.device("cuda")
    rows = []
    for smp in samples:
        op = operator(smp.seed)
        A = torch.from_numpy(op.A27).to(dev)
        B = torch.from_numpy(op.B27).to(dev)
        dop = make_operator(NX, NY, NZ, A, B)
        lam = torch.zeros(M0, dtype=torch.float64, device=dev)
        X = torch.zeros((M0, op.N), dtype=torch.float64, device=dev)
        solve(h, dop, smp.lmin, smp.lmax, None, lam, X, torch)          # warm caches and tuner
        for tol in tols:
            r0, t_rand = solve(h, dop, smp.lmin, smp.lmax, None, lam, X, torch, tol)
            lam_rand = lam.cpu().numpy()[:r0.m_found].copy()
            r1, t_learn, used = learned_solve(h, net, smp.seed, dop, smp.lmin, smp.lmax, lam, X, torch, tol)
            lam_learn = lam.cpu().numpy()[:r1.m_found].copy()
            same = r0.m_found == r1.m_found and np.abs(lam_rand - lam_learn).max() <= 1e-10 * np.abs(lam_rand).max()
            rows.append(dict(seed=smp.seed, tol=tol, m=r1.m_found, loops_random=r0.loops, loops_learned=r1.loops,
                             t_random=t_rand, t_learned=t_learn, resid_random=r0.info.resid_max,
                             resid_learned=r1.info.resid_max, fallback_status=int(used),
                             same_eigenvalues=bool(same)))
    return rows


def summarise(rows, tol):
    r = [x for x in rows if x["tol"] == tol]
    return dict(tol=tol, n=len(r),
                mean_loops_random=float(np.mean([x["loops_random"] for x in r])),
                mean_loops_learned=float(np.mean([x["loops_learned"] for x in r])),
                mean_t_random=float(np.mean([x["t_random"] for x in r])),
                mean_t_learned=float(np.mean([x["t_learned"] for x in r])),
                all_same=all(x["same_eigenvalues"] for x in r),
                max_resid_random=float(max(x["resid_random"] for x in r)),
                max_resid_learned=float(max(x["resid_learned"] for x in r)),
                fallbacks=sum(x["fallback_status"] != FEAST_OK for x in r))


def main():
    """Train on `--train` seeds, evaluate on `--eval` held-out seeds (loops and
    time to solution with the learned start against the random start)."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--epochs", default="40", help="comma-separated: one network per entry")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--out", default="learned_results.json")
    ap.add_argument("--weights", default=None)
    args = ap.parse_args()
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f}s] {m}", flush=True)  # noqa: E731
    train = generate(list(range(args.train)), torch, workers=args.workers, log=log)
    evalset = generate(list(range(10000, 10000 + args.eval)), torch, workers=args.workers)
    t_gen = time.time() - t0
    log(f"truncation sine: train max {max(s.trunc for s in train):.3e}, mean {np.mean([s.trunc for s in train]):.3e}")
    best = None
    runs = []
    for ep in [int(e) for e in args.epochs.split(",")]:
        t1 = time.time()
        net, losses, history = train_network(train, torch, epochs=ep, batch_instances=args.batch, lr=args.lr,
                                             val=evalset, log=log)
        runs.append(dict(epochs=ep, first_loss=losses[0], final_loss=losses[-1], train_s=time.time() - t1,
                         validation=history, losses=losses))
        if best is None or history[-1]["sin_mean"] < best[1]:
            best = (net, history[-1]["sin_mean"], ep)
    net = best[0]
    if args.weights:
        save_weights(net, args.weights)
    h = Handle(precision=FEAST_PREC_MIXED)
    rows = evaluate(h, net, evalset, torch)
    summary = dict(train=len(train), eval=len(evalset), lr=args.lr, batch=args.batch, gen_s=t_gen, chosen_epochs=best[2],
                   trunc_max=max(s.trunc for s in train + evalset),
                   runs=[{k: v for k, v in r.items() if k != "losses"} for r in runs],
                   by_tol=[summarise(rows, t) for t in sorted({x["tol"] for x in rows})])
    with open(args.out, "w") as f:
        json.dump(dict(summary=summary, rows=rows, runs=runs), f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
