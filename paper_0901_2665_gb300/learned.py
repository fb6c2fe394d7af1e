"""Learned initial subspace for FEAST (form 4): data, training and use.

A family of instances shares a Q1 grid (24x24x100) and 16 Gaussian potential
terms whose (x, y) centres are fixed for the family; each instance draws the
z-centre, width and amplitude of every term (48 scalars).  The network maps
per-layer features -- those 48 scalars (terms ordered by z-centre, fixed
affine scaling), the search interval and the layer position -- to the
coefficients of the start block Y on the layer's 8x8 separable sine basis.

Training targets are FEAST's own converged Ritz vectors (sign-normalised,
projected on the basis by the library's projection kernel).  The network, the
projection and the expansion all run in the library's kernels; this module
only marshals arrays and orders the calls.  A learned start that fails (B_Q
not positive definite, or a non-finite block) falls back to the random start.
"""

from __future__ import annotations

import dataclasses
import time

import numpy as np

import workloads

from . import FEAST_ERR_BQ_NOT_SPD, FEAST_ERR_JACOBI, FEAST_ERR_PIVOT, FEAST_OK, FEAST_PREC_MIXED, FeastError, \
    Handle, Mlp, feast_sine_project, make_operator

NX, NY, NZ = 24, 24, 100
GAUSSIANS = 16
M, M0, NE = 40, 64, 8
PX = PY = 8
IN_DIM = 3 * GAUSSIANS + 3
WIDTH = 512
OUT_DIM = M0 * PX * PY
FAMILY_XY_SEED = 4
TOL = 1e-12


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
    """Columns of the lowest M pairs weigh 1, the others 1/4."""
    w = np.full((M0, PX * PY), 0.25, dtype=np.float32)
    w[:M] = 1.0
    return w.ravel()


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


def generate(seeds, torch, workers: int = 4, log=None):
    """Converged FEAST subspaces for `seeds` (mixed precision, batched), their
    lowest-M intervals and sine-basis targets."""
    dev = torch.device("cuda")
    h = Handle(precision=FEAST_PREC_MIXED)
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
            lam = lams[i].cpu().numpy()
            inside = np.sort(lam[:mf[i]])
            lmin = float(inside[0] - 0.5 * (inside[M] - inside[M - 1]))
            lmax = float(0.5 * (inside[M - 1] + inside[M]))
            coef = torch.zeros((NZ, M0, PX * PY), dtype=torch.float32, device=dev)
            feast_sine_project(Xs[i], NX, NY, NZ, M0, PX, PY, coef)
            C = coef.cpu().numpy()
            # sign: the largest coefficient of every column positive
            flat = C.transpose(1, 0, 2).reshape(M0, -1)
            sgn = np.sign(flat[np.arange(M0), np.abs(flat).argmax(axis=1)])
            C = C * sgn[None, :, None]
            out.append(Sample(s, lmin, lmax, features(s, lmin, lmax), C.reshape(NZ, -1).astype(np.float32)))
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


def train_network(samples, torch, epochs: int = 40, batch_instances: int = 32, lr: float = 1e-3, seed: int = 0,
                  log=None):
    """Trains a fresh network on `samples` with the library's kernels (Adam,
    minibatches of whole instances, gathered on the host).  Returns
    (net, target scale, per-epoch losses)."""
    dev = torch.device("cuda")
    X = np.stack([s.feats for s in samples])          # (n, NZ, IN_DIM)
    T = np.stack([s.coef for s in samples])           # (n, NZ, OUT_DIM)
    scale = float(np.sqrt(np.mean(T ** 2)))
    T = (T / scale).astype(np.float32)
    wd = torch.from_numpy(loss_weights()).to(dev)
    rows = batch_instances * NZ
    net = Mlp(IN_DIM, WIDTH, OUT_DIM, rows)
    for k, (W, b) in enumerate(init_params(seed)):
        net.feast_mlp_set_layer(k, W, b)
    rng = np.random.default_rng(seed + 1)
    losses = []
    n = len(samples)
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n, batch_instances):
            idx = perm[b0:b0 + batch_instances]
            xb = torch.from_numpy(np.ascontiguousarray(X[idx].reshape(-1, IN_DIM))).to(dev)
            tb = torch.from_numpy(np.ascontiguousarray(T[idx].reshape(-1, OUT_DIM))).to(dev)
            tot += net.feast_mlp_train_step(xb, tb, wd, len(idx) * NZ, lr) * len(idx)
        losses.append(tot / n)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return net, scale, losses


def solve(h: Handle, op_dev, lmin, lmax, Y0, lam, X, torch):
    """FEAST from start block Y0 (None = random); returns (result, seconds)."""
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = h.feast_solve(op_dev, lmin, lmax, M0, NE, TOL, Y0, lam, X)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t


def learned_solve(h: Handle, net: Mlp, seed: int, op_dev, lmin, lmax, lam, X, torch):
    """FEAST from the network's start block, falling back to the random start
    when that block is unusable (FEAST rejects a degenerate or non-finite start
    through B_Q, the Jacobi sweeps or a pivot).  Returns (result, seconds, used_learned)."""
    dev = torch.device("cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    Y = torch.zeros((M0, NX * NY * NZ), dtype=torch.float64, device=dev)
    net.feast_predict_Y(torch.from_numpy(features(seed, lmin, lmax)).to(dev), NX, NY, NZ, M0, PX, PY, Y)
    used = True
    try:
        r = h.feast_solve(op_dev, lmin, lmax, M0, NE, TOL, Y, lam, X)
    except FeastError as ex:
        if ex.status not in (FEAST_ERR_BQ_NOT_SPD, FEAST_ERR_JACOBI, FEAST_ERR_PIVOT):
            raise
        used = False
        r = h.feast_solve(op_dev, lmin, lmax, M0, NE, TOL, None, lam, X)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t, used


def main():
    """Train on `--train` seeds, evaluate on `--eval` held-out seeds (loops and
    time to solution with the learned start against the random start)."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--out", default="learned_results.json")
    args = ap.parse_args()
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f}s] {m}", flush=True)  # noqa: E731
    train = generate(list(range(args.train)), torch, workers=args.workers, log=log)
    t_gen = time.time() - t0
    net, scale, losses = train_network(train, torch, epochs=args.epochs, log=log)
    t_train = time.time() - t0 - t_gen
    evalset = generate(list(range(10000, 10000 + args.eval)), torch, workers=args.workers)
    dev = torch.device("cuda")
    h = Handle(precision=FEAST_PREC_MIXED)
    rows = []
    for smp in evalset:
        op = operator(smp.seed)
        A = torch.from_numpy(op.A27).to(dev)
        B = torch.from_numpy(op.B27).to(dev)
        dop = make_operator(NX, NY, NZ, A, B)
        lam = torch.zeros(M0, dtype=torch.float64, device=dev)
        X = torch.zeros((M0, op.N), dtype=torch.float64, device=dev)
        solve(h, dop, smp.lmin, smp.lmax, None, lam, X, torch)          # warm caches and tuner
        r0, t_rand = solve(h, dop, smp.lmin, smp.lmax, None, lam, X, torch)
        lam_rand = lam.cpu().numpy()[:r0.m_found].copy()
        r1, t_learn, used = learned_solve(h, net, smp.seed, dop, smp.lmin, smp.lmax, lam, X, torch)
        lam_learn = lam.cpu().numpy()[:r1.m_found].copy()
        same = r0.m_found == r1.m_found and np.abs(lam_rand - lam_learn).max() <= 1e-10 * np.abs(lam_rand).max()
        rows.append(dict(seed=smp.seed, m=r1.m_found, loops_random=r0.loops, loops_learned=r1.loops,
                         t_random=t_rand, t_learned=t_learn, resid_random=r0.info.resid_max,
                         resid_learned=r1.info.resid_max, used_learned=used, same_eigenvalues=bool(same)))
    summary = dict(train=len(train), eval=len(rows), epochs=args.epochs, final_loss=losses[-1],
                   first_loss=losses[0], gen_s=t_gen, train_s=t_train,
                   mean_loops_random=float(np.mean([r["loops_random"] for r in rows])),
                   mean_loops_learned=float(np.mean([r["loops_learned"] for r in rows])),
                   mean_t_random=float(np.mean([r["t_random"] for r in rows])),
                   mean_t_learned=float(np.mean([r["t_learned"] for r in rows])),
                   all_same=all(r["same_eigenvalues"] for r in rows),
                   max_resid_learned=float(max(r["resid_learned"] for r in rows)),
                   fallbacks=sum(not r["used_learned"] for r in rows))
    with open(args.out, "w") as f:
        json.dump(dict(summary=summary, rows=rows, losses=losses), f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
