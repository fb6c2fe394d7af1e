"""Write tests/golden/intervals.json: the search interval of every synthetic
workload instance, certified by the oracle's inertia count.

Reading of "an interval enclosing the lowest M eigenvalues, with margins at
midpoints between neighbours": lmax = (lambda_M + lambda_{M+1})/2 and
lmin = lambda_1 - (lambda_{M+1} - lambda_M)/2.  The eigenvalues come from the
dense LAPACK pencil solve for small N, else from multisection on the oracle's
inertia count nu(sigma) = #{lambda < sigma}.  Each interval is certified by
nu(lmax) - nu(lmin) = M.  Calls only ``oracle`` and ``workloads``.

    python tests/golden/make_intervals.py [name ...]
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "intervals.json")

# (key, workload name, potential seed or None for V=0)
INSTANCES = [
    ("q1_10x10x20/v0", "q1_10x10x20_fp64", None),
] + [
    (f"q1_10x10x20/seed{s}", "q1_10x10x20_fp64", s) for s in range(5)
] + [
    ("q1_24x24x100/seed0", "q1_24x24x100_fp64", 0),
    ("q1_32x32x400/seed0", "q1_32x32x400_fp64", 0),
]

_OP_CACHE = {}


def _op(name, seed):
    key = (name, seed)
    if key not in _OP_CACHE:
        wl = workloads.WORKLOADS[name]
        _OP_CACHE[key] = wl.operator(0 if seed is None else seed, zero_potential=seed is None)
    return _OP_CACHE[key]


def _count(args):
    name, seed, sigma = args
    return sigma, oracle.inertia_count(_op(name, seed), sigma)


def _multisection(name, seed, M, pool, log):
    """Bracket lambda_1, lambda_M, lambda_{M+1} by multisection on nu(sigma)."""
    wl = workloads.WORKLOADS[name]
    lam0 = oracle.closed_form_eigenvalues_v0(wl.nx, wl.ny, wl.nz)
    op = _op(name, seed)
    # generous bracket: the potential only lowers the spectrum, by at most
    # -sum of amplitudes; widen by 10% on both sides and verify the counts
    lo0 = lam0[0] - 2.0 * wl.gaussians - 1.0
    hi0 = lam0[M] * 1.1 + 1.0
    # the V = 0 spectrum shifted by the potential's range gives likely brackets
    ix, iy, iz = workloads.grid_index(wl.nx, wl.ny, wl.nz)
    h = 1.0 / (wl.nx + 1)
    pot = workloads.gaussian_potential(wl.gaussians, seed, wl.nx, wl.ny, wl.nz)
    vmin = float(pot((ix + 1) * h, (iy + 1) * h, (iz + 1) * h).min())
    guesses = [lam0[0] + vmin - 0.1, lam0[0] + 0.01, lam0[M - 1] + vmin - 0.1,
               lam0[M] + 0.01, lam0[M] + 0.5 * vmin]
    pts = [lo0, hi0] + guesses
    known = dict(pool.map(_count, [(name, seed, s) for s in pts]))
    assert known[lo0] == 0 and known[hi0] >= M + 1, (known, lo0, hi0)
    targets = [1, M, M + 1]

    def bracket(k):
        # lambda_k in [lo, hi): nu(lo) <= k-1 < k <= nu(hi)
        lo = max(s for s, c in known.items() if c <= k - 1)
        hi = min(s for s, c in known.items() if c >= k)
        return lo, hi

    rnd = 0
    while True:
        rnd += 1
        br = {k: bracket(k) for k in targets}
        gap_lo = br[M + 1][0] - br[M][1]
        width_ok = {k: (br[k][1] - br[k][0]) <= max(0.02 * gap_lo, 1e-9) for k in targets}
        if gap_lo > 0 and all(width_ok.values()):
            break
        if br[M] == br[M + 1] and br[M][1] - br[M][0] < 1e-9 * abs(br[M][1]):
            raise RuntimeError("lambda_M and lambda_M+1 coincide; extend M")
        pts = []
        todo = [k for k in targets if not (gap_lo > 0 and width_ok[k])]
        per = max(1, (os.cpu_count() or 8) // len(todo))
        for k in todo:
            lo, hi = br[k]
            pts += [lo + (hi - lo) * (j + 1) / (per + 1) for j in range(per)]
        pts = sorted(set(pts) - set(known))
        known.update(dict(pool.map(_count, [(name, seed, s) for s in pts])))
        log(f"  round {rnd}: {len(pts)} counts; brackets "
            + ", ".join(f"l{k}=[{br[k][0]:.6f},{br[k][1]:.6f})" for k in targets))
    br = {k: bracket(k) for k in targets}
    mid = {k: 0.5 * (br[k][0] + br[k][1]) for k in targets}
    return mid[1], mid[M], mid[M + 1], br


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    log = lambda s: print(s, flush=True)  # noqa: E731
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 8) as pool:
        for key, name, seed in INSTANCES:
            if names and key not in names:
                continue
            wl = workloads.WORKLOADS[name]
            M = wl.M
            t0 = time.time()
            op = _op(name, seed)
            if wl.N <= 5000:
                lam = oracle.dense_generalized_eigh(op)[0]
                l1, lM, lM1 = lam[0], lam[M - 1], lam[M]
                method = "dense LAPACK pencil eigenvalues"
                brackets = None
            else:
                l1, lM, lM1, br = _multisection(name, seed, M, pool, log)
                method = "multisection on the oracle inertia count"
                brackets = {str(k): list(v) for k, v in br.items()}
            lmax = 0.5 * (lM + lM1)
            lmin = l1 - 0.5 * (lM1 - lM)
            c_lo = dict(pool.map(_count, [(name, seed, lmin)]))[lmin]
            c_hi = dict(pool.map(_count, [(name, seed, lmax)]))[lmax]
            assert c_hi - c_lo == M, (c_lo, c_hi, M)
            data[key] = dict(workload=name, seed=seed, M=M, lmin=lmin, lmax=lmax,
                             lambda_1=l1, lambda_M=lM, lambda_M1=lM1,
                             inertia_lmin=c_lo, inertia_lmax=c_hi, method=method,
                             brackets=brackets)
            log(f"{key}: [{lmin:.10f}, {lmax:.10f}] M={M} certified ({time.time() - t0:.0f} s)")
            with open(OUT, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
