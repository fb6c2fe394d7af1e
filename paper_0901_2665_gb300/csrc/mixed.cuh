// Mixed-precision node factor-and-solve: complex64 block inverses computed and
// applied on the tcgen05 tensor cores, FP64-residual iterative refinement of
// every node solution (internal interface).
#pragma once

#include <functional>

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
constexpr int kLoopKey = 48;
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

// Device-side state of a solve whose refinement loops (Fig. 2 steps 2-6 and
// the refinement of every node solve) run inside one CUDA graph with
// device-side loop conditions.
struct LoopState {
  int loop;             // loops started (1-based once running)
  int ir_step;          // refinement steps of the current loop's node solves
  int count, prev_count;
  int converged;        // trace test met in a loop refined to ir_tol
  int fail;             // 1: refinement cap reached, 2: a non-finite residual
  int ir_steps_max;
  int ir_steps_total;   // refinement steps of all loops
  double trace, prev_trace;
  double ir_target;     // refinement target of the current loop
  double ir_resid_max;  // largest relative residual at which a node solve run to ir_tol stopped
  double trace_hist[64], change_hist[64];
};

// Fixed parameters of such a graph.
#ifndef FEAST_EARLY_TOL1
#define FEAST_EARLY_TOL1 1e-4
#endif
// Refinement targets of loops 1 and 2 from a random start (options.ir_early):
// their subspaces are still far from converged, so their solves need less
// accuracy (never below options.ir_tol).
__host__ __device__ constexpr double early_tol(int loop) { return loop == 1 ? FEAST_EARLY_TOL1 : 1e-8; }

struct LoopParams {
  double lmin, lmax, tol, ir_tol;
  int early;            // loosened refinement targets in loops 1 and 2
  int max_loops, ir_max, M0;
};

// The steps of a loop outside the node solves, launched on the stream given.
struct LoopHooks {
  std::function<void(cudaStream_t)> rhs;       // RHS = B Y
  std::function<void(cudaStream_t)> quad_rr;   // Q from the quadrature shares; Rayleigh-Ritz -> eps, X
  std::function<void(cudaStream_t)> next_y;    // Y = X
};

struct MixedWork {
  void* bufs[20] = {};
  size_t sizes[20] = {};
  int nz_factored = 0, ne_factored = 0;   // shape of the factors held
  int bemb_k = 0;                         // right-hand sides the RHS operand was zeroed for
  // row layouts (n, row stride) the solve operands were zeroed for: the
  // split-pair rows must read zeros past 2n in a ragged last block
  long long fr_layout = -1, bemb_layout = -1;
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
  cudaStream_t cap2 = nullptr, cap3 = nullptr; // streams that capture the bodies of loop nodes
  cudaGraphExec_t loop_graph = nullptr;        // the captured loop of a solve
  unsigned long long loop_key[kLoopKey] = {};
  unsigned long long loop_seen[kLoopKey] = {};
  long long loop_replays = 0;
  long long loop_outer_launches = 0, loop_inner_launches = 0;   // kernels of one loop body, one refinement step
  void release();
};

// Both return nullptr on success, else a static error message.
const char* mixed_factor(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, int* status);
// Allocates the work buffers and sets the kernel attributes of a node solve
// of k right-hand sides (factors in place), as mixed_solve does first.
const char* mixed_solve_prepare(cudaStream_t s, Grid g, int Ne, int k, MixedWork& w, int* status);
// Solves (Z_e B - A) Q_e = RHS for every node e to the refinement tolerance.
// G (nullable): receives Q_e (Ne x N x k complex128).  Qp (nullable):
// receives the node shares Re{coef_e Q_e} of the quadrature sum (Eq. 15,
// Ne x N x k real), accumulated in the backward-sweep epilogue.
const char* mixed_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                        MixedWork& w, const double* RHS, cplx* G, double* Qp, const cplx* coef, int k, double ir_tol,
                        int ir_max, MixedSolveStats* stats, int* status);

// The loop of a mixed-precision solve (factors in place, Y set) as one CUDA
// graph with device-side conditions: a WHILE node over the FEAST loops whose
// body holds the node solves with a nested WHILE node over their refinement
// steps, the quadrature and Rayleigh-Ritz hooks, and the trace test; the
// state ends in *st.  key: everything the captured launches depend on.  The
// graph is captured the second time a key is seen and replayed afterwards;
// returns "not captured" (nothing launched) when the caller must run the
// host-driven loop instead, nullptr once the graph ran, else an error.
const char* mixed_loop(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                       MixedWork& w, const double* RHS, double* Qp, const cplx* coef, int k, const LoopParams& lp,
                       const double* eps, LoopState* st, const LoopHooks& hooks, const unsigned long long* key,
                       int* status);
extern const char* const kNotCaptured;

// Self-test of the bounded waits of the pipelined kernels: one thread waits,
// through the same bounded-wait helper, on an mbarrier that nothing
// completes and gives up after `polls` polls (1 .. kSelftestMaxPolls),
// recording DEV_TIMEOUT in *status; the kernel then returns normally.
constexpr long long kSelftestMaxPolls = 1LL << 26;
void selftest_wait(cudaStream_t s, long long polls, int* status);

}  // namespace feast
