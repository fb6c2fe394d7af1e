// Mixed-precision node factor-and-solve: complex64 block inverses computed and
// applied on the tcgen05 tensor cores, FP64-residual iterative refinement of
// every node solution (internal interface).
#pragma once

#include "common.cuh"

namespace feast {

struct MixedSolveStats {
  int steps_max = 0;        // most refinement steps taken by one node solve
  double resid_max = 0.0;   // worst final relative residual ||R||_F / ||RHS||_F
  long long graph_sweeps = 0;   // pairs of sweeps run from a captured CUDA graph
};

// Instantiated CUDA graphs of the node-solve sweeps (one forward and one
// backward sweep over all layers, ~4 launches a layer), keyed by everything
// the captured launches depend on; least recently used entry replaced.  A
// key is captured the second time it is seen (a capture and instantiation
// cost more than one direct run, so one-off shapes stay direct).
constexpr int kSweepGraphs = 8;
constexpr int kSweepKey = 20;
struct SweepGraphCache {
  cudaGraphExec_t exec[kSweepGraphs] = {};
  unsigned long long key[kSweepGraphs][kSweepKey] = {};
  unsigned long long used[kSweepGraphs] = {};
  unsigned long long clock = 0;
  unsigned long long seen[kSweepGraphs][kSweepKey] = {};   // keys run once, directly
  int seen_next = 0;
};

struct MixedWork {
  void* bufs[20] = {};
  size_t sizes[20] = {};
  int nz_factored = 0, ne_factored = 0;   // shape of the factors held
  int bemb_k = 0;                         // right-hand sides the RHS operand was zeroed for
  cudaStream_t side = nullptr;            // lookahead stream of the factorisation
  cudaEvent_t ev_narrow = nullptr, ev_side = nullptr;
  SweepGraphCache graphs;
  bool use_graphs = true;                      // off for the workers of a batched call (one-off instances)
  cudaStream_t cap = nullptr;                  // non-blocking stream that captures (the caller's may be the legacy one)
  cudaGraphExec_t factor_graph = nullptr;      // the captured factorisation
  unsigned long long factor_key[kSweepKey] = {};
  unsigned long long factor_seen[kSweepKey] = {};   // last factorisation run directly
  long long factor_launches = 0;               // kernels in it
  long long factor_replays = 0;
  void release();
};

// Both return nullptr on success, else a static error message.
const char* mixed_factor(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, int* status);
// Solves (Z_e B - A) Q_e = RHS for every node e to the refinement tolerance.
// G (nullable): receives Q_e (Ne x N x k complex128).  Qp (nullable):
// receives the node shares Re{coef_e Q_e} of the quadrature sum (Eq. 15,
// Ne x N x k real), accumulated in the backward-sweep epilogue.
const char* mixed_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                        MixedWork& w, const double* RHS, cplx* G, double* Qp, const cplx* coef, int k, double ir_tol,
                        int ir_max, MixedSolveStats* stats, int* status);

}  // namespace feast
