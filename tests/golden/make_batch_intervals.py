"""Write tests/golden/batch_intervals.json: search intervals of the batched
workload (workloads.batch_instances), each enclosing about 0.75*M0
eigenvalues, with the count certified by the oracle's inertia.

Reading of "an interval enclosing ~0.75*M0 eigenvalues": the potential only
lowers the V = 0 spectrum lambda0 by at most |min V|, so
lmin = lambda0_1 + min V - 1 lies below the spectrum (certified: count 0) and
lmax = lambda0_T + min V / 2 with T = round(0.75*M0) encloses about T
eigenvalues; the exact number M = nu(lmax) - nu(lmin) is recorded.  If M
falls outside [0.6, 0.9]*M0, lmax moves by a quarter of the potential range
and is counted again.  Calls only `oracle` and `workloads`.

    python tests/golden/make_batch_intervals.py [count]
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "batch_intervals.json")


def one(inst):
    op = inst.operator()
    lam0 = oracle.closed_form_eigenvalues_v0(inst.nx, inst.ny, inst.nz)
    h = 1.0 / (inst.nx + 1)
    ix, iy, iz = workloads.grid_index(inst.nx, inst.ny, inst.nz)
    pot = workloads.gaussian_potential(inst.gaussians, inst.potential_seed, inst.nx, inst.ny, inst.nz)
    vmin = float(pot((ix + 1) * h, (iy + 1) * h, (iz + 1) * h).min())
    T = int(round(0.75 * inst.M0))
    lmin = float(lam0[0] + vmin - 1.0)
    c_lo = oracle.inertia_count(op, lmin)
    while c_lo != 0:
        lmin -= 2.0
        c_lo = oracle.inertia_count(op, lmin)
    lmax = float(lam0[T - 1] + 0.5 * vmin)
    counts = []
    for _ in range(4):
        M = oracle.inertia_count(op, lmax) - c_lo
        counts.append((lmax, M))
        if 0.6 * inst.M0 <= M <= 0.9 * inst.M0:
            break
        lmax += (0.25 * abs(vmin) + 0.1) * (1 if M < 0.6 * inst.M0 else -1)
    return dict(index=inst.index, nx=inst.nx, ny=inst.ny, nz=inst.nz, M0=inst.M0,
                potential_seed=inst.potential_seed, lmin=lmin, lmax=lmax, M=M,
                inertia_lmin=c_lo, inertia_lmax=M + c_lo, tries=counts)


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    insts = workloads.batch_instances(count)
    # largest first so the pool stays busy
    order = sorted(insts, key=lambda b: -(b.nx * b.ny) ** 3 * b.nz)
    data = {}
    with mp.get_context("spawn").Pool(os.cpu_count() or 8) as pool:
        for res in pool.imap_unordered(one, order):
            data[str(res["index"])] = res
            print(f"instance {res['index']}: {res['nx']}x{res['ny']}x{res['nz']} M0={res['M0']} "
                  f"[{res['lmin']:.6f}, {res['lmax']:.6f}] M={res['M']}", flush=True)
            with open(OUT, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
