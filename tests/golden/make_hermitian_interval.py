"""Write tests/golden/hermitian_interval.json: the search interval of the
Hermitian benchmark workload (a 16 x 16 x 40 Q1 operator, 8 Gaussian terms,
seed 11, with Peierls phases of a uniform field of 0.3 flux quanta per
plaquette along z: workloads.peierls_operator), enclosing its lowest 24
eigenvalues with margins at midpoints between neighbours
(lmax = (l_M + l_{M+1}) / 2, lmin = l_1 - (l_{M+1} - l_M) / 2), and those 24
eigenvalues, from the dense Hermitian pencil of the oracle (LAPACK).  Calls
only ``oracle`` and ``workloads``.

    python tests/golden/make_hermitian_interval.py
"""

from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "hermitian_interval.json")
NX, NY, NZ, GAUSSIANS, SEED, FLUX, M = 16, 16, 40, 8, 11, 0.3, 24


def main():
    real = workloads.q1_operator(NX, NY, NZ, workloads.gaussian_potential(GAUSSIANS, SEED, NX, NY, NZ))
    op = workloads.peierls_operator(real, flux=FLUX)
    lam = oracle.dense_generalized_eigh(op)[0]
    out = {"nx": NX, "ny": NY, "nz": NZ, "gaussians": GAUSSIANS, "seed": SEED, "flux": FLUX, "M": M,
           "lmin": float(lam[0] - 0.5 * (lam[M] - lam[M - 1])), "lmax": float(0.5 * (lam[M - 1] + lam[M])),
           "lam": [float(x) for x in lam[:M + 1]], "method": "dense Hermitian pencil (LAPACK) of the oracle"}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(out["lmin"], out["lmax"])


if __name__ == "__main__":
    main()
