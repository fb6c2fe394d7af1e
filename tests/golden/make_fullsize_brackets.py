"""Write tests/golden/fullsize_brackets.json: tight brackets of sampled
eigenvalues of the 32 x 32 x 400 Q1 workload (seed 0), from the oracle's
inertia count alone.

nu(sigma) = #{lambda < sigma} (Sylvester's law of inertia on A - sigma B,
evaluated by the oracle's block elimination over the z-layers).  For each
sampled index k the script bisects on nu until lambda_k lies in [lo, hi] with
nu(lo) <= k - 1 < k <= nu(hi) and hi - lo <= 1e-11 |hi|.  The starting
brackets are the certified interval ends and the coarse brackets stored in
intervals.json by make_intervals.py (also written by the oracle).  The
full-size GPU test checks its eigenvalues against these brackets.  Calls only
``oracle`` and ``workloads``.

    python tests/golden/make_fullsize_brackets.py
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "fullsize_brackets.json")
KEY, NAME, SEED = "q1_32x32x400/seed0", "q1_32x32x400_fp64", 0
SAMPLES = (1, 50, 100)
REL_WIDTH = 1e-11


def main():
    iv = json.load(open(os.path.join(HERE, "intervals.json")))[KEY]
    op = workloads.WORKLOADS[NAME].operator(SEED)
    # exact counts nu(sigma): the certified interval ends, then every bisection point
    known = {iv["lmin"]: iv["inertia_lmin"], iv["lmax"]: iv["inertia_lmax"]}
    coarse = iv.get("brackets") or {}   # per k: nu(lo) <= k - 1 < k <= nu(hi)
    counts = 0
    out = {"key": KEY, "workload": NAME, "seed": SEED, "rel_width": REL_WIDTH,
           "method": "bisection on the oracle inertia count", "brackets": {}}
    for k in SAMPLES:
        lo = max(s for s, c in known.items() if c <= k - 1)
        hi = min(s for s, c in known.items() if c >= k)
        if str(k) in coarse:
            lo, hi = max(lo, coarse[str(k)][0]), min(hi, coarse[str(k)][1])
        t0 = time.time()
        while hi - lo > REL_WIDTH * abs(hi):
            mid = 0.5 * (lo + hi)
            c = oracle.inertia_count(op, mid)
            counts += 1
            known[mid] = c
            if c >= k:
                hi = mid
            else:
                lo = mid
            print(f"  lambda_{k}: [{lo:.15g}, {hi:.15g}] width {hi - lo:.3e}", flush=True)
        # the exact counts at both ends, recorded for the reader
        for s in (lo, hi):
            if s not in known:
                known[s] = oracle.inertia_count(op, s)
                counts += 1
        nu_lo, nu_hi = known[lo], known[hi]
        assert nu_lo <= k - 1 < k <= nu_hi, (k, nu_lo, nu_hi)
        out["brackets"][str(k)] = {"lo": lo, "hi": hi, "nu_lo": nu_lo, "nu_hi": nu_hi}
        print(f"lambda_{k} in [{lo:.15g}, {hi:.15g}] ({time.time() - t0:.0f} s)", flush=True)
        out["inertia_counts"] = counts
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
