"""Write tests/golden/oracle_eigenvalues.json: the eigenpairs that the CPU
oracle's FEAST loop (Fig. 2, Eqs. 13-15, Rayleigh-Ritz Eqs. 6-9) converges to
on instances too large to run inside a test:

  * batch/<i>: instances of the 64-instance batched workload
    (workloads.batch_instances, intervals certified in batch_intervals.json);
  * learned/<seed>: held-out instances of the learned-start family (24x24x100,
    16 Gaussians with (x, y) centres from the fixed seed 4; intervals
    certified in learned_intervals.json).

Each entry holds the in-interval eigenvalues (ascending), the count, the loop
count, the largest in-interval residual of both forms, and the start block's
seed (workloads.random_Y(N, M0, y_seed)).  Trace tolerance 1e-12, Ne = 8.
Calls only ``oracle`` and ``workloads``.

    python tests/golden/make_oracle_eigenvalues.py [key ...]
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

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "oracle_eigenvalues.json")
BATCH = [45, 46]                 # 24x24x72 (M0 = 32) and 16x16x347 (M0 = 128)
LEARNED = [10000]
LEARNED_GRID, LEARNED_GAUSSIANS, LEARNED_XY_SEED, LEARNED_M0 = (24, 24, 100), 16, 4, 64
NE, TOL = 8, 1e-12


def _job(key):
    kind, ident = key.split("/")
    ident = int(ident)
    if kind == "batch":
        bi = workloads.batch_instances(64)[ident]
        iv = json.load(open(os.path.join(HERE, "batch_intervals.json")))[str(ident)]
        op, M0, y_seed = bi.operator(), bi.M0, 500 + ident
    else:
        nx, ny, nz = LEARNED_GRID
        pot = workloads.gaussian_potential(LEARNED_GAUSSIANS, ident, nx, ny, nz, fixed_xy_seed=LEARNED_XY_SEED)
        op = workloads.q1_operator(nx, ny, nz, pot)
        iv = json.load(open(os.path.join(HERE, "learned_intervals.json")))[str(ident)]
        M0, y_seed = LEARNED_M0, 900 + ident % 1000
    t0 = time.time()
    res = oracle.feast(op, iv["lmin"], iv["lmax"], M0, NE, workloads.random_Y(op.N, M0, y_seed), tol=TOL)
    m = res.m_found
    assert res.converged and m == iv["M"], (key, m, iv["M"])
    return key, {"nx": op.nx, "ny": op.ny, "nz": op.nz, "M0": M0, "Ne": NE, "tol": TOL, "y_seed": y_seed,
                 "lmin": iv["lmin"], "lmax": iv["lmax"], "m_found": m, "loops": res.loops,
                 "lam": [float(x) for x in res.lam[:m]], "resid_max": float(res.resid[:m].max()),
                 "resid_paper_max": float(res.resid_paper[:m].max()), "seconds": round(time.time() - t0, 1)}


def main():
    keys = sys.argv[1:] or [f"batch/{i}" for i in BATCH] + [f"learned/{s}" for s in LEARNED]
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    with mp.get_context("spawn").Pool(min(len(keys), os.cpu_count() or 1)) as pool:
        for key, entry in pool.imap_unordered(_job, keys):
            out[key] = entry
            print(f"{key}: {entry['m_found']} pairs, {entry['loops']} loops, {entry['seconds']} s", flush=True)
            with open(OUT, "w") as f:
                json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
