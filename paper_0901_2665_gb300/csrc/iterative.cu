// Iterative inner solver for the node systems (Fig. 2 step 2 without a
// factorisation).  Sec. IV.C solves the inner systems of FEAST "using an
// iterative method with preconditioner" to a modest relative residual (1e-3),
// with the trace tolerance kept at 1e-8, and Sec. V notes that iterative
// solvers avoid the memory of direct ones.
//
// M_e = Z_e B - A is complex symmetric (A, B real symmetric), so the solver is
// the conjugate orthogonal conjugate gradient method (COCG: CG with the
// bilinear form x^T y in place of x^H y, van der Vorst and Melissen, IEEE
// Trans. Magn. 26, 1990) with the Jacobi preconditioner D_e = diag(M_e),
// which keeps the preconditioned operator complex symmetric:
//   x = 0, r = b, z = D^{-1} r, p = z, rho = r^T z
//   repeat:  q = M p,  alpha = rho / p^T q,  x += alpha p,  r -= alpha q,
//            stop the column when ||r||_2 <= tol ||b||_2,
//            z = D^{-1} r,  rho' = r^T z,  p = z + (rho'/rho) p,  rho = rho'.
// Every node and every right-hand side carries its own scalars; all of them
// advance together in each launch (grid z = node), converged columns are
// frozen.  FP64 throughout.  Column sums are formed per block of rows and then
// summed in block order, so the result does not depend on the schedule.
#include <algorithm>
#include <cmath>
#include <vector>

#include "iterative.cuh"
#include "prof.cuh"

namespace feast {

namespace {

constexpr int kCgRows = 128;                 // grid rows per block
constexpr int kCgThreads = 256;              // two column groups
constexpr int kCgGroups = kCgThreads / kCgRows;
constexpr size_t kCgSmem = sizeof(cplx) * 27 * kCgRows;

struct CgDims {
  int nx, ny, nz, n, k, Ne;
  long long N;
  int nblk;
};

__device__ __forceinline__ cplx cbil(cplx a, cplx b) { return cmul(a, b); }   // a b (no conjugate)

// Coefficients c_s(i) = (Z_e B - A)[i, i + off(s)] of the block's rows (0 outside the grid).
__device__ void cg_stage(const CgDims& d, cplx z, const double* __restrict__ A27, const double* __restrict__ B27,
                         long long i0, cplx* csm) {
  for (int t = threadIdx.x; t < 27 * kCgRows; t += blockDim.x) {
    const int s = t / kCgRows, r = t % kCgRows;
    const long long i = i0 + r;
    cplx c{0.0, 0.0};
    if (i < d.N) {
      const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
      const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
      if (ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 && iz + dz < d.nz) {
        const double a = A27[(long long)s * d.N + i], b = B27[(long long)s * d.N + i];
        c = cplx{z.re * b - a, z.im * b};
      }
    }
    csm[t] = c;
  }
}

// Adds v into the block's column sum `col[m]` (warp reduction, then one
// shared-memory atomic per warp); every lane of the warp has the same m.
__device__ __forceinline__ void col_add(cplx* col, int m, cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_down_sync(0xffffffffu, v.re, o);
    v.im += __shfl_down_sync(0xffffffffu, v.im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&col[m].re, v.re);
    atomicAdd(&col[m].im, v.im);
  }
}

// x = 0, r = b, z = D^{-1} r, p = z; partials of r^T z (slot 0) and
// ||b||^2 (slot 1, real part) per (node, block, column).
__global__ void __launch_bounds__(kCgThreads) k_cg_init(CgDims d, const cplx* __restrict__ Z,
                                                        const double* __restrict__ A27,
                                                        const double* __restrict__ B27,
                                                        const double* __restrict__ RHS, cplx* __restrict__ X,
                                                        cplx* __restrict__ R, cplx* __restrict__ Zv,
                                                        cplx* __restrict__ P, cplx* __restrict__ part) {
  __shared__ cplx col[2][128];
  const int e = blockIdx.y, tid = threadIdx.x;
  const long long i0 = (long long)blockIdx.x * kCgRows;
  for (int t = tid; t < 2 * 128; t += kCgThreads) col[t / 128][t % 128] = cplx{0.0, 0.0};
  __syncthreads();
  const cplx z = Z[e];
  const int r = tid % kCgRows, g = tid / kCgRows;
  const long long i = i0 + r;
  const long long sG = d.N * d.k;
  cplx dinv{0.0, 0.0};
  if (i < d.N) dinv = cinv(cplx{z.re * B27[13 * d.N + i] - A27[13 * d.N + i], z.im * B27[13 * d.N + i]});
  for (int m = g; m < d.k; m += kCgGroups) {
    cplx rz{0.0, 0.0}, bb{0.0, 0.0};
    if (i < d.N) {
      const long long at = e * sG + (long long)m * d.N + i;
      const double b = RHS[(long long)m * d.N + i];
      const cplx rv{b, 0.0};
      const cplx zv = cmul(dinv, rv);
      X[at] = cplx{0.0, 0.0};
      R[at] = rv;
      Zv[at] = zv;
      P[at] = zv;
      rz = cbil(rv, zv);
      bb = cplx{b * b, 0.0};
    }
    col_add(col[0], m, rz);
    col_add(col[1], m, bb);
  }
  __syncthreads();
  for (int m = tid; m < d.k; m += kCgThreads) {
    cplx* o = part + (((long long)e * d.nblk + blockIdx.x) * d.k + m) * 2;
    o[0] = col[0][m];
    o[1] = col[1][m];
  }
}

// q = M_e p for the live columns; partials of p^T q (slot 0).
__global__ void __launch_bounds__(kCgThreads) k_cg_apply(CgDims d, const cplx* __restrict__ Z,
                                                         const double* __restrict__ A27,
                                                         const double* __restrict__ B27,
                                                         const cplx* __restrict__ P, cplx* __restrict__ Qv,
                                                         cplx* __restrict__ part, const int* __restrict__ done) {
  extern __shared__ cplx csm[];
  __shared__ cplx col[128];
  const int e = blockIdx.y, tid = threadIdx.x;
  const long long i0 = (long long)blockIdx.x * kCgRows;
  for (int t = tid; t < 128; t += kCgThreads) col[t] = cplx{0.0, 0.0};
  cg_stage(d, Z[e], A27, B27, i0, csm);
  __syncthreads();
  const int r = tid % kCgRows, g = tid / kCgRows;
  const long long i = i0 + r;
  const long long sG = d.N * d.k;
  int off[27];
  {
    const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
#pragma unroll
    for (int s = 0; s < 27; ++s) {
      const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
      const bool ok = i < d.N && ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 &&
                      iz + dz < d.nz;
      off[s] = ok ? dx + d.nx * (dy + d.ny * dz) : 0;
    }
  }
  for (int m = g; m < d.k; m += kCgGroups) {
    if (done[e * d.k + m]) continue;   // uniform over the column group's warps
    cplx pq{0.0, 0.0};
    if (i < d.N) {
      const cplx* p = P + e * sG + (long long)m * d.N + i;
      cplx acc{0.0, 0.0};
#pragma unroll
      for (int s = 0; s < 27; ++s) cfma(acc, csm[s * kCgRows + r], p[off[s]]);
      Qv[e * sG + (long long)m * d.N + i] = acc;
      pq = cbil(p[0], acc);
    }
    col_add(col, m, pq);
  }
  __syncthreads();
  for (int m = tid; m < d.k; m += kCgThreads) part[(((long long)e * d.nblk + blockIdx.x) * d.k + m) * 2] = col[m];
}

// alpha = rho / p^T q for the live columns (block sums in order); a zero or
// non-finite denominator (breakdown) ends the column with its status set.
__global__ void k_cg_alpha(CgDims d, const cplx* __restrict__ part, const cplx* __restrict__ rho,
                           cplx* __restrict__ alpha, int* __restrict__ done, int* __restrict__ status) {
  const int e = blockIdx.x;
  for (int m = threadIdx.x; m < d.k; m += blockDim.x) {
    const int id = e * d.k + m;
    if (done[id]) {
      alpha[id] = cplx{0.0, 0.0};
      continue;
    }
    cplx s{0.0, 0.0};
    for (int b = 0; b < d.nblk; ++b) s = cadd(s, part[(((long long)e * d.nblk + b) * d.k + m) * 2]);
    const double mag = fabs(s.re) + fabs(s.im);
    if (!(mag > 0.0) || !isfinite(mag)) {
      alpha[id] = cplx{0.0, 0.0};
      done[id] = 2;
      atomicExch(status, (int)DEV_PIVOT);
      continue;
    }
    alpha[id] = cmul(rho[id], cinv(s));
  }
}

// x += alpha p, r -= alpha q, z = D^{-1} r; partials of r^T z (slot 0) and
// ||r||^2 (slot 1, real part).
__global__ void __launch_bounds__(kCgThreads) k_cg_update(CgDims d, const cplx* __restrict__ Z,
                                                          const double* __restrict__ A27,
                                                          const double* __restrict__ B27,
                                                          const cplx* __restrict__ alpha, cplx* __restrict__ X,
                                                          cplx* __restrict__ R, cplx* __restrict__ Zv,
                                                          const cplx* __restrict__ P, const cplx* __restrict__ Qv,
                                                          cplx* __restrict__ part, const int* __restrict__ done) {
  __shared__ cplx col[2][128];
  const int e = blockIdx.y, tid = threadIdx.x;
  const long long i0 = (long long)blockIdx.x * kCgRows;
  for (int t = tid; t < 2 * 128; t += kCgThreads) col[t / 128][t % 128] = cplx{0.0, 0.0};
  __syncthreads();
  const cplx z = Z[e];
  const int r = tid % kCgRows, g = tid / kCgRows;
  const long long i = i0 + r;
  const long long sG = d.N * d.k;
  cplx dinv{0.0, 0.0};
  if (i < d.N) dinv = cinv(cplx{z.re * B27[13 * d.N + i] - A27[13 * d.N + i], z.im * B27[13 * d.N + i]});
  for (int m = g; m < d.k; m += kCgGroups) {
    if (done[e * d.k + m]) continue;
    cplx rz{0.0, 0.0}, rr{0.0, 0.0};
    if (i < d.N) {
      const long long at = e * sG + (long long)m * d.N + i;
      const cplx a = alpha[e * d.k + m];
      cplx x = X[at], rv = R[at];
      cfma(x, a, P[at]);
      cfma(rv, cneg(a), Qv[at]);
      const cplx zv = cmul(dinv, rv);
      X[at] = x;
      R[at] = rv;
      Zv[at] = zv;
      rz = cbil(rv, zv);
      rr = cplx{rv.re * rv.re + rv.im * rv.im, 0.0};
    }
    col_add(col[0], m, rz);
    col_add(col[1], m, rr);
  }
  __syncthreads();
  for (int m = tid; m < d.k; m += kCgThreads) {
    cplx* o = part + (((long long)e * d.nblk + blockIdx.x) * d.k + m) * 2;
    o[0] = col[0][m];
    o[1] = col[1][m];
  }
}

// rho' = r^T z, ||r||; a column whose ||r|| <= tol ||b|| is done, else
// beta = rho'/rho.  first: only rho and ||b|| (after k_cg_init).
__global__ void k_cg_beta(CgDims d, const cplx* __restrict__ part, cplx* __restrict__ rho, cplx* __restrict__ beta,
                          double* __restrict__ bnorm2, double* __restrict__ rel, int* __restrict__ done,
                          double tol, int first) {
  const int e = blockIdx.x;
  for (int m = threadIdx.x; m < d.k; m += blockDim.x) {
    const int id = e * d.k + m;
    if (done[id]) {
      beta[id] = cplx{0.0, 0.0};
      continue;
    }
    cplx rz{0.0, 0.0};
    double rr = 0.0;
    for (int b = 0; b < d.nblk; ++b) {
      const cplx* o = part + (((long long)e * d.nblk + b) * d.k + m) * 2;
      rz = cadd(rz, o[0]);
      rr += o[1].re;
    }
    if (first) {
      bnorm2[id] = rr;
      rel[id] = rr > 0.0 ? 1.0 : 0.0;
      rho[id] = rz;
      if (!(rr > 0.0)) done[id] = 1;   // a zero right-hand side: x = 0
      continue;
    }
    const double rl = sqrt(rr / bnorm2[id]);
    rel[id] = rl;
    if (rl <= tol) {
      done[id] = 1;
      beta[id] = cplx{0.0, 0.0};
      continue;
    }
    beta[id] = cmul(rz, cinv(rho[id]));
    rho[id] = rz;
  }
}

// p = z + beta p for the live columns
__global__ void k_cg_direction(CgDims d, const cplx* __restrict__ beta, const cplx* __restrict__ Zv,
                               cplx* __restrict__ P, const int* __restrict__ done) {
  const int e = blockIdx.y;
  const long long total = d.N * d.k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / d.N);
    if (done[e * d.k + m]) continue;
    const long long at = e * total + t;
    cplx p = Zv[at];
    cfma(p, beta[e * d.k + m], P[at]);
    P[at] = p;
  }
}

__global__ void k_quadrature_from_solutions(long long total, int Ne, const cplx* __restrict__ coef,
                                            const cplx* __restrict__ X, double* __restrict__ Q) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = 0; e < Ne; ++e) {
      const cplx v = X[e * total + t];
      const cplx c = coef[e];
      acc += c.re * v.re - c.im * v.im;
    }
    Q[t] = acc;
  }
}

template <class T>
T* carve(char*& p, size_t count) {
  T* out = reinterpret_cast<T*>(p);
  p += ((sizeof(T) * count + 255) / 256) * 256;
  return out;
}

}  // namespace

size_t cocg_work_bytes(Grid g, int Ne, int k) {
  const long long N = g.N();
  const long long nblk = (N + kCgRows - 1) / kCgRows;
  const size_t vec = sizeof(cplx) * (size_t)Ne * N * k;
  const size_t sc = sizeof(cplx) * (size_t)Ne * k;
  return 4 * ((vec + 255) / 256 * 256) + sizeof(cplx) * 2 * (size_t)Ne * nblk * k + 4 * (sc + 256) +
         2 * (sizeof(double) * Ne * k + 256) + (sizeof(int) * Ne * k + 256) + 4096;
}

const char* cocg_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                       const double* RHS, cplx* X, int k, double tol, int max_iter, void* work, int* status,
                       CocgStats* stats) {
  CgDims d{g.nx, g.ny, g.nz, g.n(), k, Ne, g.N(), 0};
  d.nblk = (int)((d.N + kCgRows - 1) / kCgRows);
  if (k > 128) return "iterative inner solver: at most 128 right-hand sides";
  char* p = static_cast<char*>(work);
  const size_t vec = (size_t)Ne * d.N * k;
  cplx* R = carve<cplx>(p, vec);
  cplx* Zv = carve<cplx>(p, vec);
  cplx* P = carve<cplx>(p, vec);
  cplx* Qv = carve<cplx>(p, vec);
  cplx* part = carve<cplx>(p, 2 * (size_t)Ne * d.nblk * k);
  cplx* rho = carve<cplx>(p, (size_t)Ne * k);
  cplx* alpha = carve<cplx>(p, (size_t)Ne * k);
  cplx* beta = carve<cplx>(p, (size_t)Ne * k);
  double* bn2 = carve<double>(p, (size_t)Ne * k);
  double* rel = carve<double>(p, (size_t)Ne * k);
  int* done = carve<int>(p, (size_t)Ne * k);
  static PerDevice<cudaError_t> attr;
  if (attr.get([] { return cudaFuncSetAttribute(k_cg_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCgSmem); },
               cudaErrorInvalidDevice) != cudaSuccess)
    return "iterative inner solver: attribute rejected";
  const dim3 rgrid(d.nblk, Ne);
  const int cb = std::min(1024, std::max(32, ((k + 31) / 32) * 32));
  const dim3 vgrid((unsigned)std::min<long long>(4096, (d.N * k + 255) / 256), Ne);
  // apply + update: 108 + 16 FP64 flops per complex entry (FMA = 2), counted per iteration
  const double it_flops = 248.0 * (double)d.N * k * Ne;
  cudaMemsetAsync(done, 0, sizeof(int) * Ne * k, s);
  k_cg_init<<<rgrid, kCgThreads, 0, s>>>(d, Z, A27, B27, RHS, X, R, Zv, P, part);
  k_cg_beta<<<Ne, cb, 0, s>>>(d, part, rho, beta, bn2, rel, done, tol, 1);
  prof::count_launch(2);
  std::vector<int> hd((size_t)Ne * k);
  int it = 0;
  bool all = false;
  for (it = 1; it <= max_iter; ++it) {
    prof::begin(s, prof::FP64_SOLVE);
    prof::add_work(prof::FP64_SOLVE, it_flops);
    k_cg_apply<<<rgrid, kCgThreads, kCgSmem, s>>>(d, Z, A27, B27, P, Qv, part, done);
    k_cg_alpha<<<Ne, cb, 0, s>>>(d, part, rho, alpha, done, status);
    k_cg_update<<<rgrid, kCgThreads, 0, s>>>(d, Z, A27, B27, alpha, X, R, Zv, P, Qv, part, done);
    k_cg_beta<<<Ne, cb, 0, s>>>(d, part, rho, beta, bn2, rel, done, tol, 0);
    k_cg_direction<<<vgrid, 256, 0, s>>>(d, beta, Zv, P, done);
    prof::end(s, prof::FP64_SOLVE);
    prof::count_launch(5);
    if (it % 8 == 0 || it == max_iter) {
      if (cudaMemcpyAsync(hd.data(), done, sizeof(int) * Ne * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return "iterative inner solver: device error";
      all = true;
      for (int v : hd) all = all && v != 0;
      if (all) break;
    }
  }
  if (stats) {
    std::vector<double> hr((size_t)Ne * k);
    cudaMemcpyAsync(hr.data(), rel, sizeof(double) * Ne * k, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    stats->iterations = std::min(it, max_iter);
    stats->rel_max = 0.0;
    for (double v : hr) stats->rel_max = std::max(stats->rel_max, v);
  }
  if (!all) return "iterative inner solver did not reach its tolerance";
  return nullptr;
}

void quadrature_from_solutions(cudaStream_t s, long long N, int k, int Ne, const cplx* coef, const cplx* X,
                               double* Q) {
  const long long total = N * k;
  if (total == 0) return;
  k_quadrature_from_solutions<<<(unsigned)std::min<long long>(152 * 32, (total + 255) / 256), 256, 0, s>>>(
      total, Ne, coef, X, Q);
  prof::count_launch();
}

}  // namespace feast
