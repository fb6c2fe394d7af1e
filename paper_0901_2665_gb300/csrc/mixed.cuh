// Mixed-precision node factor-and-solve: complex64 block inverses computed and
// applied on the tcgen05 tensor cores, FP64-residual iterative refinement of
// every node solution (internal interface).
#pragma once

#include "common.cuh"

namespace feast {

struct MixedSolveStats {
  int steps_max = 0;        // most refinement steps taken by one node solve
  double resid_max = 0.0;   // worst final relative residual ||R||_F / ||RHS||_F
};

struct MixedWork {
  void* bufs[20] = {};
  size_t sizes[20] = {};
  int nz_factored = 0, ne_factored = 0;   // shape of the factors held
  int bemb_k = 0;                         // right-hand sides the RHS operand was zeroed for
  cudaStream_t side = nullptr;            // lookahead stream of the factorisation
  cudaEvent_t ev_narrow = nullptr, ev_side = nullptr;
  void release();
};

// Both return nullptr on success, else a static error message.
const char* mixed_factor(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, int* status);
const char* mixed_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                        MixedWork& w, const double* RHS, cplx* G, int k, double ir_tol, int ir_max,
                        MixedSolveStats* stats, int* status);

}  // namespace feast
