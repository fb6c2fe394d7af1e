"""Write tests/golden/learned_intervals.json: search intervals of held-out
instances of the learned-start family, certified by the oracle's inertia.

The family: Q1 grid 24x24x100, 16 Gaussian terms whose (x, y) centres come
from the fixed seed 4 and whose z-centre, width and amplitude come from the
instance seed.  The interval holds the lowest M = 40 eigenvalues with margins
at midpoints between neighbours: lmax = (lambda_M + lambda_{M+1})/2,
lmin = lambda_1 - (lambda_{M+1} - lambda_M)/2, the three eigenvalues
bracketed by multisection on nu(sigma) = #{lambda < sigma} and the count
certified by nu(lmax) - nu(lmin) = M.  Calls only ``oracle`` and ``workloads``.

    python tests/golden/make_learned_intervals.py [seed ...]
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

OUT = os.path.join(HERE, "learned_intervals.json")
NX, NY, NZ, GAUSSIANS, XY_SEED, M = 24, 24, 100, 16, 4, 40
SEEDS = [10000, 10001, 10002]

_OPS = {}


def _op(seed):
    if seed not in _OPS:
        pot = workloads.gaussian_potential(GAUSSIANS, seed, NX, NY, NZ, fixed_xy_seed=XY_SEED)
        _OPS[seed] = workloads.q1_operator(NX, NY, NZ, pot)
    return _OPS[seed]


def _count(args):
    seed, sigma = args
    return sigma, oracle.inertia_count(_op(seed), sigma)


def _bracket(known, k):
    lo = max(s for s, c in known.items() if c <= k - 1)
    hi = min(s for s, c in known.items() if c >= k)
    return lo, hi


def intervals(seed, pool, log):
    lam0 = oracle.closed_form_eigenvalues_v0(NX, NY, NZ)
    h = 1.0 / (NX + 1)
    ix, iy, iz = workloads.grid_index(NX, NY, NZ)
    pot = workloads.gaussian_potential(GAUSSIANS, seed, NX, NY, NZ, fixed_xy_seed=XY_SEED)
    vmin = float(pot((ix + 1) * h, (iy + 1) * h, (iz + 1) * h).min())
    # the potential lowers the V = 0 spectrum by at most |min V|
    lo0, hi0 = lam0[0] + vmin - 1.0, lam0[M] + 1.0
    known = dict(pool.map(_count, [(seed, s) for s in np.linspace(lo0, hi0, 16)]))
    assert known[lo0] == 0 and known[hi0] >= M + 1, known
    targets = [1, M, M + 1]
    per = max(1, (os.cpu_count() or 8) // 3)
    for rnd in range(60):
        br = {k: _bracket(known, k) for k in targets}
        gap = br[M + 1][0] - br[M][1]
        if gap > 0 and all(br[k][1] - br[k][0] <= max(0.02 * gap, 1e-9) for k in targets):
            break
        pts = []
        for k in targets:
            lo, hi = br[k]
            if not (gap > 0 and hi - lo <= max(0.02 * gap, 1e-9)):
                pts += [lo + (hi - lo) * (j + 1) / (per + 1) for j in range(per)]
        known.update(dict(pool.map(_count, [(seed, s) for s in sorted(set(pts) - set(known))])))
        log(f"  seed {seed} round {rnd}: " + ", ".join(f"l{k}=[{br[k][0]:.6f},{br[k][1]:.6f})" for k in targets))
    else:
        raise RuntimeError("multisection did not separate lambda_M and lambda_M+1")
    mid = {k: 0.5 * sum(_bracket(known, k)) for k in targets}
    lmax = 0.5 * (mid[M] + mid[M + 1])
    lmin = mid[1] - 0.5 * (mid[M + 1] - mid[M])
    c = dict(pool.map(_count, [(seed, lmin), (seed, lmax)]))
    assert c[lmax] - c[lmin] == M, c
    return dict(seed=seed, M=M, lmin=lmin, lmax=lmax, inertia_lmin=c[lmin], inertia_lmax=c[lmax])


def main(seeds):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    log = lambda s: print(s, flush=True)  # noqa: E731
    with mp.get_context("spawn").Pool(os.cpu_count() or 8) as pool:
        for seed in seeds:
            t0 = time.time()
            data[str(seed)] = intervals(seed, pool, log)
            log(f"seed {seed}: {data[str(seed)]} ({time.time() - t0:.0f} s)")
            with open(OUT, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or SEEDS)
