// 27-point stencil products, layer couplings of the node systems and the
// quadrature sum (Fig. 2 steps 2, 3, 6; Eq. 15).
#include "kernels.cuh"
#include "prof.cuh"

namespace feast {

namespace {

constexpr int kColsPerThread = 16;

// Y[:, c] = C X[:, c].  One thread per row, kColsPerThread columns per thread
// so the 27 coefficients of the row are read once per column group.
__global__ void __launch_bounds__(256) k_stencil_apply(Grid g, const double* __restrict__ C27,
                                                       const double* __restrict__ X, long long ldx,
                                                       double* __restrict__ Y, long long ldy, int k) {
  const long long N = g.N();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
  double c[27];
  long long off[27];
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
    const bool ok = ix + dx >= 0 && ix + dx < nx && iy + dy >= 0 && iy + dy < ny && iz + dz >= 0 &&
                    iz + dz < nz;
    c[s] = ok ? C27[(long long)s * N + i] : 0.0;
    off[s] = ok ? (long long)dx + (long long)nx * (dy + (long long)ny * dz) : 0;
  }
  const int c0 = blockIdx.y * kColsPerThread;
  const int c1 = min(k, c0 + kColsPerThread);
  for (int col = c0; col < c1; ++col) {
    const double* x = X + (long long)col * ldx + i;
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < 27; ++s) acc = fma(c[s], x[off[s]], acc);
    Y[(long long)col * ldy + i] = acc;
  }
}

__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

__global__ void k_random_block(long long total, uint64_t seed, double* Y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    Y[t] = splitmix_uniform(seed, (uint64_t)t);
}

__global__ void k_stencil_norm1(Grid g, const double* __restrict__ A27, double* out) {
  const long long N = g.N();
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < 27; ++j) s += fabs(A27[(long long)j * N + i]);
    m = fmax(m, s);
  }
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // single block launch: plain store
    out[0] = red[0];
  }
}

// G_e[layer i][p, m] = RHS[layer i][p, m] + sum_{dz=-1 slots} M_e[p, a] Tmp_e[a, m]
__global__ void __launch_bounds__(256) k_couple_forward(Grid g, int layer, const cplx* __restrict__ Z,
                                                        const double* __restrict__ A27,
                                                        const double* __restrict__ B27,
                                                        const double* __restrict__ RHS,
                                                        const cplx* __restrict__ Tmp, long long sT,
                                                        cplx* __restrict__ G, long long sG, int k) {
  const int n = g.n();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int e = blockIdx.z;
  const long long N = g.N();
  const long long row = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const cplx z = Z[e];
  cplx c[9];
  int off[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    const int s = t;  // dz = -1 slots are 0..8
    const bool ok = px + dx >= 0 && px + dx < g.nx && py + dy >= 0 && py + dy < g.ny;
    const double a = ok ? A27[(long long)s * N + row] : 0.0;
    const double b = ok ? B27[(long long)s * N + row] : 0.0;
    c[t] = cplx{z.re * b - a, z.im * b};
    off[t] = ok ? p + dx + g.nx * dy : p;
  }
  const cplx* T = Tmp + e * sT;
  cplx* Ge = G + e * sG;
  const int c0 = blockIdx.y * kColsPerThread, c1 = min(k, c0 + kColsPerThread);
  for (int m = c0; m < c1; ++m) {
    cplx acc = cplx{RHS[(long long)m * N + row], 0.0};
#pragma unroll
    for (int t = 0; t < 9; ++t) cfma(acc, c[t], T[(long long)m * n + off[t]]);
    Ge[(long long)m * N + row] = acc;
  }
}

// Tmp_e[p, m] = G_e[layer i][p, m] - sum_{dz=+1 slots} M_e[p, a] G_e[layer i+1][a, m]
// (for the top layer the sum is empty and Tmp_e = G_e[layer i])
__global__ void __launch_bounds__(256) k_couple_backward(Grid g, int layer, const cplx* __restrict__ Z,
                                                         const double* __restrict__ A27,
                                                         const double* __restrict__ B27,
                                                         const cplx* __restrict__ G, long long sG,
                                                         cplx* __restrict__ Tmp, long long sT, int k) {
  const int n = g.n();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int e = blockIdx.z;
  const long long N = g.N();
  const long long row = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const bool has_next = layer + 1 < g.nz;  // the top layer has no upper coupling
  const cplx z = Z[e];
  cplx c[9];
  long long off[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    const int s = 18 + t;  // dz = +1 slots are 18..26
    const bool ok = has_next && px + dx >= 0 && px + dx < g.nx && py + dy >= 0 && py + dy < g.ny;
    const double a = ok ? A27[(long long)s * N + row] : 0.0;
    const double b = ok ? B27[(long long)s * N + row] : 0.0;
    c[t] = cplx{z.re * b - a, z.im * b};
    off[t] = ok ? (long long)n + dx + g.nx * dy : 0;
  }
  const cplx* Ge = G + e * sG;
  cplx* T = Tmp + e * sT;
  const int c0 = blockIdx.y * kColsPerThread, c1 = min(k, c0 + kColsPerThread);
  for (int m = c0; m < c1; ++m) {
    const cplx* col = Ge + (long long)m * N + row;
    cplx acc = col[0];
    cplx u = cplx{0.0, 0.0};
#pragma unroll
    for (int t = 0; t < 9; ++t) cfma(u, c[t], col[off[t]]);
    T[(long long)m * n + p] = csub(acc, u);
  }
}

// Q[t] = sum_e Qp[e][t], nodes in order e = 1..Ne (a fixed summation order,
// so the result does not depend on the launch schedule).
__global__ void k_quadrature_node_sum(long long total, int Ne, const double* __restrict__ Qp, long long sQ,
                                 double* __restrict__ Q) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = 0; e < Ne; ++e) acc += Qp[e * sQ + t];
    Q[t] = acc;
  }
}

__global__ void k_rhs_to_complex(long long rows, int k, const double* __restrict__ RHS, long long ldr,
                                 cplx* __restrict__ G, long long ldg, long long sG) {
  const long long total = rows * k;
  const int e = blockIdx.y;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % rows, m = t / rows;
    G[e * sG + m * ldg + r] = cplx{RHS[m * ldr + r], 0.0};
  }
}

int grid1d(long long total, int block) {
  long long b = (total + block - 1) / block;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void stencil_apply(cudaStream_t s, Grid g, const double* C27, const double* X, long long ldx, double* Y,
                   long long ldy, int k) {
  if (g.N() == 0 || k == 0) return;
  dim3 grid(cdiv(g.N(), 256), cdiv(k, kColsPerThread));
  k_stencil_apply<<<grid, 256, 0, s>>>(g, C27, X, ldx, Y, ldy, k);
  prof::count_launch();
}

void random_block(cudaStream_t s, long long N, int k, uint64_t seed, double* Y) {
  long long total = N * k;
  if (total == 0) return;
  k_random_block<<<grid1d(total, 256), 256, 0, s>>>(total, seed, Y);
  prof::count_launch();
}

void stencil_norm1(cudaStream_t s, Grid g, const double* A27, double* out) {
  k_stencil_norm1<<<1, 256, 0, s>>>(g, A27, out);
  prof::count_launch();
}

void couple_forward(cudaStream_t s, Grid g, int layer, int Ne, const cplx* Z, const double* A27,
                    const double* B27, const double* RHS, const cplx* Tmp, long long sT, cplx* G,
                    long long sG, int k) {
  dim3 grid(cdiv(g.n(), 256), cdiv(k, kColsPerThread), Ne);
  k_couple_forward<<<grid, 256, 0, s>>>(g, layer, Z, A27, B27, RHS, Tmp, sT, G, sG, k);
  prof::count_launch();
}

void couple_backward(cudaStream_t s, Grid g, int layer, int Ne, const cplx* Z, const double* A27,
                     const double* B27, const cplx* G, long long sG, cplx* Tmp, long long sT, int k) {
  dim3 grid(cdiv(g.n(), 256), cdiv(k, kColsPerThread), Ne);
  k_couple_backward<<<grid, 256, 0, s>>>(g, layer, Z, A27, B27, G, sG, Tmp, sT, k);
  prof::count_launch();
}

void quadrature_sum(cudaStream_t s, long long N, int k, int Ne, const double* Qp, long long sQ, double* Q) {
  long long total = N * k;
  if (total == 0) return;
  k_quadrature_node_sum<<<grid1d(total, 256), 256, 0, s>>>(total, Ne, Qp, sQ, Q);
  prof::count_launch();
}

void rhs_to_complex(cudaStream_t s, long long rows, int k, int Ne, const double* RHS, long long ldr,
                    cplx* G, long long ldg, long long sG) {
  long long total = rows * k;
  if (total == 0) return;
  dim3 grid(grid1d(total, 256), Ne);
  k_rhs_to_complex<<<grid, 256, 0, s>>>(rows, k, RHS, ldr, G, ldg, sG);
  prof::count_launch();
}

}  // namespace feast
