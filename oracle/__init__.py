"""CPU FP64 oracle of FEAST (Polizzi, arXiv:0901.2665) -- TEST INFRASTRUCTURE.

Plain, slow, obviously correct restatement of the paper's method (Fig. 2 with
Eqs. 13-15, Rayleigh-Ritz Eqs. 6-9, refinement Sec. III.B (i)) in numpy/scipy
float64/complex128, and a dense Jacobi generalized eigensolver written from
the mathematics (``jacobi.py``, no LAPACK) that checks it on tiny pencils.
It shares no code with the CUDA library and imports nothing from it.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may import it; the product path never does.
"""

from .feast_oracle import (  # noqa: F401
    BQNotSPD,
    FeastResult,
    assemble,
    block_tridiag_factor,
    closed_form_eigenvalues_v0,
    contour_points,
    dense_generalized_eigh,
    feast,
    feast_hermitian,
    filter_value,
    gauss_legendre,
    inertia_count,
    norm1,
    quadrature_subspace,
    quadrature_subspace_hermitian,
    rayleigh_ritz,
    rayleigh_ritz_hermitian,
    residuals,
)
from .jacobi import (  # noqa: F401
    JacobiNoConvergence,
    cholesky_lower,
    jacobi_generalized_eigh,
    jacobi_symmetric,
)
