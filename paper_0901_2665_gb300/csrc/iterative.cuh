// Iterative (COCG, Jacobi-preconditioned) node solves (internal interface).
#pragma once

#include "common.cuh"

namespace feast {

struct CocgStats {
  int iterations = 0;     // iterations run (every column of every node)
  double rel_max = 0.0;   // largest final ||r|| / ||b|| of a column
};

// Device bytes of the work space cocg_solve needs for Ne nodes and k right-hand sides.
size_t cocg_work_bytes(Grid g, int Ne, int k);

// X_e (Ne x N x k complex, col-major per node) = (Z_e B - A)^{-1} RHS to
// ||r||_2 <= tol ||b||_2 per column, by preconditioned COCG; k <= 128.
// Returns nullptr on success, else a static message; a breakdown sets
// DEV_PIVOT in *status.
const char* cocg_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                       const double* RHS, cplx* X, int k, double tol, int max_iter, void* work, int* status,
                       CocgStats* stats);

// Q = sum_e Re{coef_e X_e} over the nodes in order e = 1..Ne (Eq. 15).
void quadrature_from_solutions(cudaStream_t s, long long N, int k, int Ne, const cplx* coef, const cplx* X,
                               double* Q);

}  // namespace feast
