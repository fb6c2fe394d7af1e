// Mixed-precision node solves (see mixed.cuh).
#include "mixed.cuh"

namespace feast {

void MixedWork::release() {
  for (int i = 0; i < 16; ++i) {
    if (bufs[i]) cudaFree(bufs[i]);
    bufs[i] = nullptr;
    sizes[i] = 0;
  }
}

const char* mixed_factor(cudaStream_t, Grid, int, const cplx*, const double*, const double*, MixedWork&, int*) {
  return "mixed-precision path not available in this build";
}

const char* mixed_solve(cudaStream_t, Grid, int, const cplx*, const double*, const double*, MixedWork&,
                        const double*, cplx*, int, double, int, MixedSolveStats*, int*) {
  return "mixed-precision path not available in this build";
}

}  // namespace feast
