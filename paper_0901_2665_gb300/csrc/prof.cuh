// Kernel accounting: a launch counter (always on) and, when enabled, CUDA
// event pairs around selected kernels, accumulated per kernel class.  Event
// pairs live in a ring; when it fills, the host waits for the oldest pair
// (which completed long ago in stream order) and folds it into the totals, so
// timing never stalls the device queue.  Process-global; single host thread.
#pragma once

#include <cuda_runtime.h>

namespace feast {
namespace prof {

enum Cls {
  SWEEP_GEMM = 0,   // tcgen05 trailing update of the block sweep (wide: all but the next panel's tile)
  SOLVE_GEMM = 1,   // tcgen05 block-solve product S' g
  PINV = 2,         // 64 x 64 panel inversion
  PANEL_T = 3,      // T = L Pinv and GEMM operand packing
  SCHUR = 4,        // Schur complements through the layer couplings
  COUPLE = 5,       // layer couplings of the solve sweeps
  RESIDUAL = 6,     // FP64 refinement residual
  FP64_SOLVE = 7,   // plain FP64 path: factor and solve kernels
  FF_RESIDUAL = 8,  // incremental refinement residual in double-float
  SWEEP_NARROW = 9, // the same update on the next panel's column tile only (critical path)
  NCLS = 10
};

void set_enabled(bool on);
bool enabled();
void begin(cudaStream_t s, int cls);
void end(cudaStream_t s, int cls);
// Algorithmic work (flops) of the kernels of a class, added at launch.
void add_work(int cls, double flops);
// Waits for every recorded pair, adds the totals into ms/count/work, clears them.
void collect(double* ms, long long* count, double* work = nullptr);
void count_launch(int n = 1);
long long launches();

}  // namespace prof
}  // namespace feast
