// Double-float versions of the FP64 products of a loop for the mixed path:
// the right-hand side B Y, the operator products A Q and B Q, the Gram
// matrices Q^T (A Q) and Q^T (B Q) of Rayleigh-Ritz (Eqs. 7) and the Ritz
// vectors X = Q Phi (Eq. 9).
//
// A double-float number is an unevaluated sum hi + lo of two fp32 values
// (about 48 significant bits).  Each product of two of them keeps the
// leading product exactly (one FMA gives its rounding error, Dekker) plus the
// two cross terms (lo*lo, ~2^-48 relative, is dropped); sums are compensated
// by TwoSum (Knuth) with the error terms collected in the low word and the
// pair renormalised every few steps.  On GB300 the FP64 pipe runs at 1/64 of
// the FP32 rate, so about a dozen fp32 instructions per product still run
// several times faster than one FP64 FMA.  The long Gram sums are cut into
// chunks of kGramRowsDf rows whose partial results are added in FP64 in a
// fixed order, which keeps the accumulated rounding at the FP64 kernels'
// level.  The reduced eigensolve and the final residuals stay in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kernels.cuh"
#include "prof.cuh"

namespace feast {

namespace {

constexpr int kDfTile = 64;         // Gram / tall-GEMM tile (64 x 64 outputs per CTA, 4 x 4 per thread)
constexpr int kGramRowsDf = 512;    // rows per Gram partial sum
constexpr int kDfColsPerThread = 16;

// rounding-explicit intrinsics throughout: the compiler must not contract a
// product into a following sum, which would break the exact error terms

__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// p + e = a b up to the dropped a.lo b.lo
__device__ __forceinline__ void df_prod(float2 a, float2 b, float& p, float& e) {
  p = __fmul_rn(a.x, b.x);
  e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
}

// (s, c) += p + e: TwoSum of the leading parts, errors into c
__device__ __forceinline__ void df_acc(float& s, float& c, float p, float e) {
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) <- Fast2Sum(s, c): |c| back below half an ulp of s
__device__ __forceinline__ void df_renorm(float& s, float& c) {
  const float h = __fadd_rn(s, c);
  c = __fsub_rn(c, __fsub_rn(h, s));
  s = h;
}

__global__ void k_split_df(long long total, const double* __restrict__ X, float2* __restrict__ Y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    Y[t] = df_split(X[t]);
}

// Y = C X for a 27-point operator (C27 slot-major FP64, split once per row),
// X double-float N x k (column stride ldx); Y double-float or FP64.
template <class OutT>
__global__ void __launch_bounds__(256, 2) k_stencil_apply_df(Grid g, const double* __restrict__ C27,
                                                          const float2* __restrict__ X, long long ldx,
                                                          OutT* __restrict__ Y, long long ldy, int k) {
  const long long N = g.N();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
  float2 c[27];
  int off[27];   // neighbour offsets: |dx + nx (dy + ny dz)| <= 1 + nx + nx ny
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
    const bool ok = ix + dx >= 0 && ix + dx < nx && iy + dy >= 0 && iy + dy < ny && iz + dz >= 0 &&
                    iz + dz < nz;
    c[s] = df_split(ok ? C27[(long long)s * N + i] : 0.0);
    off[s] = ok ? dx + nx * (dy + ny * dz) : 0;
  }
  const int c0 = blockIdx.y * kDfColsPerThread;
  const int c1 = min(k, c0 + kDfColsPerThread);
  for (int col = c0; col < c1; ++col) {
    const float2* x = X + (long long)col * ldx + i;
    float s = 0.f, cc = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      float p, e;
      df_prod(c[t], x[off[t]], p, e);
      df_acc(s, cc, p, e);
      if (t % 9 == 8) df_renorm(s, cc);
    }
    if constexpr (std::is_same<OutT, double>::value)
      Y[(long long)col * ldy + i] = (double)s + (double)cc;
    else
      Y[(long long)col * ldy + i] = make_float2(s, cc);
  }
}

// Partial Gram sums P_z[a, b] = sum over the rows of chunk z of X[r, a] Y[r, b]
// (double-float products and sums, the chunk's result in FP64); with sym only
// the tiles on and above the diagonal.
__global__ void __launch_bounds__(256) k_gram_partial_df(long long N, int k1, int k2, const float2* __restrict__ X,
                                                         const float2* __restrict__ Y, double* __restrict__ partial,
                                                         int sym) {
  constexpr int BK = 16;
  __shared__ float2 Xs[BK][kDfTile + 1];
  __shared__ float2 Ys[BK][kDfTile + 1];
  int ta = blockIdx.x, tb = blockIdx.y;
  if (sym) {   // upper-triangle tile number -> (ta <= tb)
    int t = blockIdx.x;
    tb = 0;
    while (t > tb) {
      t -= tb + 1;
      ++tb;
    }
    ta = t;
  }
  const int a0 = ta * kDfTile, b0 = tb * kDfTile;
  const long long r0 = (long long)blockIdx.z * kGramRowsDf;
  const long long r1 = min(N, r0 + kGramRowsDf);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float s[4][4] = {}, c[4][4] = {};
  for (long long rb = r0; rb < r1; rb += BK) {
    for (int t = tid; t < BK * kDfTile; t += 256) {
      const int rr = t % BK, col = t / BK;
      const long long r = rb + rr;
      Xs[rr][col] = (r < r1 && a0 + col < k1) ? X[(long long)(a0 + col) * N + r] : make_float2(0.f, 0.f);
      Ys[rr][col] = (r < r1 && b0 + col < k2) ? Y[(long long)(b0 + col) * N + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < BK; ++rr) {
      float2 xa[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = Xs[rr][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yb[j] = Ys[rr][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float p, e;
          df_prod(xa[i], yb[j], p, e);
          df_acc(s[i][j], c[i][j], p, e);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) df_renorm(s[i][j], c[i][j]);
    __syncthreads();
  }
  double* P = partial + (long long)blockIdx.z * k1 * k2;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 16 * i;
    if (a >= k1) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx + 16 * j;
      if (b < k2) P[a + (long long)b * k1] = (double)s[i][j] + (double)c[i][j];
    }
  }
}

// out = sum over chunks in chunk order; with sym the entries below the
// diagonal tiles are read from their mirror images
__global__ void k_gram_reduce_df(int nchunks, int k1, int total, const double* __restrict__ partial,
                                 double* __restrict__ out, int sym) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int src = t;
  if (sym) {
    const int a = t % k1, b = t / k1;
    if (a / kDfTile > b / kDfTile) src = b + a * k1;
  }
  double acc = 0.0;
  for (int c = 0; c < nchunks; ++c) acc += partial[(long long)c * total + src];
  out[t] = acc;
}

// C[r, c] = sum_j Q[r, j] P[j, c] (Q double-float N x m, P FP64 m x k split
// as it is staged, C FP64); 64 rows x 64 cols per CTA.
__global__ void __launch_bounds__(256) k_gemm_tall_df(long long N, int m, int k, const float2* __restrict__ Q,
                                                      const double* __restrict__ P, double* __restrict__ C) {
  constexpr int BK = 16;
  __shared__ float2 Qs[BK][kDfTile + 1];
  __shared__ float2 Ps[BK][kDfTile + 1];
  const long long r0 = (long long)blockIdx.x * kDfTile;
  const int c0 = blockIdx.y * kDfTile;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float s[4][4] = {}, c[4][4] = {};
  for (int kb = 0; kb < m; kb += BK) {
    for (int t = tid; t < BK * kDfTile; t += 256) {
      const int row = t % kDfTile, kk = t / kDfTile;
      const long long r = r0 + row;
      Qs[kk][row] = (r < N && kb + kk < m) ? Q[(long long)(kb + kk) * N + r] : make_float2(0.f, 0.f);
    }
    for (int t = tid; t < BK * kDfTile; t += 256) {
      const int kk = t % BK, col = t / BK;
      Ps[kk][col] = df_split((kb + kk < m && c0 + col < k) ? P[(long long)(c0 + col) * m + kb + kk] : 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float2 q[4], p[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = Qs[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) p[j] = Ps[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float pp, e;
          df_prod(q[i], p[j], pp, e);
          df_acc(s[i][j], c[i][j], pp, e);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) df_renorm(s[i][j], c[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long r = r0 + tx + 16 * i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = c0 + ty + 16 * j;
      if (cc < k) C[(long long)cc * N + r] = (double)s[i][j] + (double)c[i][j];
    }
  }
}

}  // namespace

void split_df(cudaStream_t s, long long total, const double* X, float2* Y) {
  const long long blocks = std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 32));
  k_split_df<<<(unsigned)blocks, 256, 0, s>>>(total, X, Y);
  prof::count_launch();
}

void stencil_apply_df(cudaStream_t s, Grid g, const double* C27, const float2* X, long long ldx, float2* Y,
                      long long ldy, int k) {
  if (k <= 0) return;
  dim3 grid(cdiv(g.N(), 256), cdiv(k, kDfColsPerThread));
  k_stencil_apply_df<float2><<<grid, 256, 0, s>>>(g, C27, X, ldx, Y, ldy, k);
  prof::count_launch();
}

void stencil_apply_df(cudaStream_t s, Grid g, const double* C27, const float2* X, long long ldx, double* Y,
                      long long ldy, int k) {
  if (k <= 0) return;
  dim3 grid(cdiv(g.N(), 256), cdiv(k, kDfColsPerThread));
  k_stencil_apply_df<double><<<grid, 256, 0, s>>>(g, C27, X, ldx, Y, ldy, k);
  prof::count_launch();
}

long long gram_partial_elems_df(long long N, int k1, int k2) {
  return (long long)cdiv(N, kGramRowsDf) * k1 * k2;
}

void gram_df(cudaStream_t s, long long N, int k1, int k2, const float2* X, const float2* Y, double* partial,
             double* out, bool symmetric) {
  const int nchunks = cdiv(N, kGramRowsDf);
  const bool sym = symmetric && k1 == k2;
  const int nt = cdiv(k1, kDfTile);
  dim3 grid = sym ? dim3(nt * (nt + 1) / 2, 1, nchunks) : dim3(nt, cdiv(k2, kDfTile), nchunks);
  k_gram_partial_df<<<grid, 256, 0, s>>>(N, k1, k2, X, Y, partial, sym ? 1 : 0);
  prof::count_launch();
  const int total = k1 * k2;
  k_gram_reduce_df<<<cdiv(total, 256), 256, 0, s>>>(nchunks, k1, total, partial, out, sym ? 1 : 0);
  prof::count_launch();
}

void gemm_tall_df(cudaStream_t s, long long N, int m, int k, const float2* Q, const double* P, double* C) {
  dim3 grid(cdiv(N, kDfTile), cdiv(k, kDfTile));
  k_gemm_tall_df<<<grid, 256, 0, s>>>(N, m, k, Q, P, C);
  prof::count_launch();
}

}  // namespace feast
