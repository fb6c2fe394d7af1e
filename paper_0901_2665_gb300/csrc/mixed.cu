// Mixed-precision node factor-and-solve (Fig. 2 step 2 in complex64 on the
// tensor cores, refined to FP64 accuracy).
//
// Factor: the same unpivoted block elimination as the FP64 path (Schur
// complements through the layer couplings, symmetric block sweep inversion
// S'_i = -S_i^{-1}), carried in fp32 complex.  The sweep's trailing updates
// S[i, j] -= sum_k T[i, k] L[j, k] (panel width 64) run as one real TF32 GEMM
// on tcgen05 through the real embedding
//   [Ur | Ui] = [Tr | Ti] [[Lr^T, Li^T], [-Li^T, Lr^T]],
// and so do the block solves t = S' g.  Storage of S'_i is "row-split": row p
// holds the n real parts, then the n imaginary parts, so a row is directly
// the K-major A operand [Sr | Si] of the solve GEMM.
//
// Solve: forward/backward sweeps in complex64 (TF32 products, fp32
// accumulation) give a correction d = M~^{-1} R; FP64 iterative refinement
// Q_e += d, R = RHS - (Z_e B - A) Q_e repeats until ||R||/||RHS|| <= ir_tol
// for every node.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mixed.cuh"
#include "tc_gemm.cuh"

namespace feast {

namespace {

constexpr int kPanel = 64;   // sweep panel width (complex columns)
constexpr int kRowsPerPanelCta = 128;

struct f2 {
  float x, y;
};
__device__ __forceinline__ f2 f2mul(f2 a, f2 b) { return f2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ void f2fma(f2& acc, f2 a, f2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ f2 f2inv(f2 a) {
  if (fabsf(a.x) >= fabsf(a.y)) {
    float r = a.y / a.x, d = a.x + a.y * r;
    return f2{1.0f / d, -r / d};
  }
  float r = a.x / a.y, d = a.x * r + a.y;
  return f2{r / d, -1.0f / d};
}

// coefficient of M_e = Z_e B - A at stencil slot s of grid row `row`
__device__ __forceinline__ f2 mcoef(const double* A27, const double* B27, long long N, int s, long long row, cplx z) {
  const double a = A27[(long long)s * N + row], b = B27[(long long)s * N + row];
  return f2{(float)(z.re * b - a), (float)(z.im * b)};
}

// ------------------------------------------------------------------ layout
struct Dims {
  int nx, ny, nz, n, Ne;
  long long N;
  int ldF;       // floats per row-split row (>= 2n, multiple of 32)
  int nblk64;    // ceil(n / 64)
  int k;         // right-hand sides
  int CB;        // complex columns per solve-GEMM tile
  int nblkCB;    // ceil(k / CB)
  int ldB;       // floats per embedded RHS row
};

// ------------------------------------------------------------------ Schur
// T1[a, q] = sum_b S'[a, b] C[q, b] (row-split, fp32)
__global__ void __launch_bounds__(256) k_mx_schur1(Dims d, int layer, const cplx* __restrict__ Z,
                                                   const double* __restrict__ A27, const double* __restrict__ B27,
                                                   const float* __restrict__ F, float* __restrict__ T1) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y, e = blockIdx.z;
  if (q >= d.n) return;
  const long long rowq = (long long)layer * d.n + q;
  const int qx = q % d.nx, qy = q / d.nx;
  const cplx z = Z[e];
  const float* S = F + (((long long)e * d.nz + layer - 1) * d.n + a) * d.ldF;
  f2 acc{0.f, 0.f};
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    if (qx + dx < 0 || qx + dx >= d.nx || qy + dy < 0 || qy + dy >= d.ny) continue;
    const int b = q + dx + d.nx * dy;
    f2fma(acc, f2{S[b], S[d.n + b]}, mcoef(A27, B27, d.N, t, rowq, z));
  }
  float* out = T1 + ((long long)e * d.n + a) * d.ldF;
  out[q] = acc.x;
  out[d.n + q] = acc.y;
}

// S_i[p, q] = D_i[p, q] + sum_a C[p, a] T1[a, q] -> F (layer i)
__global__ void __launch_bounds__(256) k_mx_schur2(Dims d, int layer, const cplx* __restrict__ Z,
                                                   const double* __restrict__ A27, const double* __restrict__ B27,
                                                   const float* __restrict__ T1, float* __restrict__ F) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y, e = blockIdx.z;
  if (q >= d.n) return;
  const long long rowp = (long long)layer * d.n + p;
  const int px = p % d.nx, py = p / d.nx;
  const cplx z = Z[e];
  f2 acc{0.f, 0.f};
  const int ddx = (q % d.nx) - px, ddy = (q / d.nx) - py;
  if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) acc = mcoef(A27, B27, d.N, 9 + (ddy + 1) * 3 + (ddx + 1), rowp, z);
  if (layer > 0) {
    const float* T = T1 + (long long)e * d.n * d.ldF;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dx = t % 3 - 1, dy = t / 3 - 1;
      if (px + dx < 0 || px + dx >= d.nx || py + dy < 0 || py + dy >= d.ny) continue;
      const float* Trow = T + (long long)(p + dx + d.nx * dy) * d.ldF;
      f2fma(acc, mcoef(A27, B27, d.N, t, rowp, z), f2{Trow[q], Trow[d.n + q]});
    }
  }
  float* out = F + (((long long)e * d.nz + layer) * d.n + p) * d.ldF;
  out[q] = acc.x;
  out[d.n + q] = acc.y;
}

// ------------------------------------------------------------------ panel
// For panel K = [k0, k0+bw) of node e: Pinv = S[K,K]^{-1} (fp32 unpivoted
// sweep, redundantly per CTA), then for this CTA's 128 rows i:
//   T[i, :] = S[i, K] Pinv,  L[i, :] = S[i, K]
// and the GEMM operands Aop = [Tr | Ti] (row i) and Bop (embedded L, rows in
// blocks of 64 complex columns: 64 rows [Lr, -Li] then 64 rows [Li, Lr]),
// rounded to TF32.  Chunk 0 also stores Pinv.
__global__ void __launch_bounds__(256) k_mx_panel(Dims d, int layer, int k0, int bw, const float* __restrict__ F,
                                                  float* __restrict__ Aop, float* __restrict__ Bop,
                                                  f2* __restrict__ Tc, f2* __restrict__ PinvOut, int* status) {
  extern __shared__ f2 psm[];
  f2* P = psm;                               // 64 x 65
  f2* Ls = psm + kPanel * (kPanel + 1);      // 128 x 65
  f2* fac = Ls + kRowsPerPanelCta * (kPanel + 1);   // 64
  __shared__ f2 piv_inv;
  __shared__ int bad;
  const int e = blockIdx.y;
  const int r0 = blockIdx.x * kRowsPerPanelCta;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int n = d.n;
  const float* Fl = F + ((long long)e * d.nz + layer) * n * d.ldF;
  if (tid == 0) bad = 0;
  for (int t = tid; t < kPanel * kPanel; t += nth) {
    const int i = t / kPanel, j = t % kPanel;
    f2 v{(i == j) ? 1.f : 0.f, 0.f};
    if (i < bw && j < bw) {
      const float* row = Fl + (long long)(k0 + i) * d.ldF;
      v = f2{row[k0 + j], row[n + k0 + j]};
    }
    P[i * (kPanel + 1) + j] = v;
  }
  for (int t = tid; t < kRowsPerPanelCta * kPanel; t += nth) {
    const int r = t / kPanel, m = t % kPanel;
    const int i = r0 + r;
    f2 v{0.f, 0.f};
    if (i < n && m < bw) {
      const float* row = Fl + (long long)i * d.ldF;
      v = f2{row[k0 + m], row[n + k0 + m]};
    }
    Ls[r * (kPanel + 1) + m] = v;
  }
  __syncthreads();
  // unpivoted sweep of P: after all pivots P = -P0^{-1}
  for (int kk = 0; kk < kPanel; ++kk) {
    if (tid == 0) {
      const f2 dv = P[kk * (kPanel + 1) + kk];
      const float mag = fabsf(dv.x) + fabsf(dv.y);
      if (!(mag > 0.f) || !isfinite(mag)) bad = 1;
      piv_inv = (mag > 0.f) ? f2inv(dv) : f2{0.f, 0.f};
    }
    __syncthreads();
    const f2 inv = piv_inv;
    for (int i = tid; i < kPanel; i += nth) fac[i] = f2mul(P[i * (kPanel + 1) + kk], inv);
    __syncthreads();
    for (int t = tid; t < kPanel * kPanel; t += nth) {
      const int i = t / kPanel, j = t % kPanel;
      if (i == kk || j == kk) continue;
      f2 v = P[i * (kPanel + 1) + j];
      const f2 u = f2mul(fac[i], P[kk * (kPanel + 1) + j]);
      v.x -= u.x;
      v.y -= u.y;
      P[i * (kPanel + 1) + j] = v;
    }
    __syncthreads();
    for (int t = tid; t < kPanel; t += nth) {
      if (t != kk) {
        P[t * (kPanel + 1) + kk] = fac[t];
        P[kk * (kPanel + 1) + t] = f2mul(P[kk * (kPanel + 1) + t], inv);
      }
    }
    if (tid == 0) P[kk * (kPanel + 1) + kk] = f2{-inv.x, -inv.y};
    __syncthreads();
  }
  // Pinv = -P
  if (blockIdx.x == 0)
    for (int t = tid; t < kPanel * kPanel; t += nth) {
      const f2 v = P[(t / kPanel) * (kPanel + 1) + t % kPanel];
      PinvOut[(long long)e * kPanel * kPanel + t] = f2{-v.x, -v.y};
    }
  // T = L Pinv for the 128 rows; one (row, 8-column group) per thread-iteration
  for (int t = tid; t < kRowsPerPanelCta * (kPanel / 8); t += nth) {
    const int r = t / (kPanel / 8), cg = (t % (kPanel / 8)) * 8;
    const int i = r0 + r;
    f2 acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = f2{0.f, 0.f};
    for (int m = 0; m < kPanel; ++m) {
      const f2 l = Ls[r * (kPanel + 1) + m];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const f2 pv = P[m * (kPanel + 1) + cg + c];
        f2fma(acc[c], l, f2{-pv.x, -pv.y});
      }
    }
    if (i < n) {
      float* arow = Aop + ((long long)e * n + i) * (2 * kPanel);
      f2* trow = Tc + ((long long)e * n + i) * kPanel;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        arow[cg + c] = tc::to_tf32(acc[c].x);
        arow[kPanel + cg + c] = tc::to_tf32(acc[c].y);
        trow[cg + c] = acc[c];
      }
      // embedded L rows for complex column j = i
      const long long brow = ((long long)e * d.nblk64 + i / 64) * 128 + (i % 64);
      float* bre = Bop + brow * (2 * kPanel);
      float* bim = Bop + (brow + 64) * (2 * kPanel);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const f2 l = Ls[r * (kPanel + 1) + cg + c];
        bre[cg + c] = tc::to_tf32(l.x);
        bre[kPanel + cg + c] = tc::to_tf32(-l.y);
        bim[cg + c] = tc::to_tf32(l.y);
        bim[kPanel + cg + c] = tc::to_tf32(l.x);
      }
    }
  }
  if (tid == 0 && bad) atomicExch(status, (int)DEV_PIVOT);
}

// ------------------------------------------------------------------ epilogues
// Sweep trailing update on tile (rows tm*128.., complex columns tn*64..).
struct SweepEpi {
  float* F;        // row-split storage of the layer being swept, node stride sF floats
  long long sF;
  int ldF, n, k0, bw, last;
  const f2* Tc;    // n x 64 per node
  const f2* Pinv;  // 64 x 64 per node
  __device__ void operator()(int e, int tm, int tn, int row, uint32_t taddr) const {
    const int i = tm * tc::kBlockM + row;
    float* Frow = F + e * sF + (long long)i * ldF;
    const f2* T = Tc + (long long)e * n * kPanel;
    const f2* Pi = Pinv + (long long)e * kPanel * kPanel;
    const bool inI = i >= k0 && i < k0 + bw;
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 16) {
      float re[16], im[16];
      tc::tmem_ld16(taddr + c0, re);
      tc::tmem_ld16(taddr + 64 + c0, im);
      if (i >= n) continue;
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int j = tn * 64 + c0 + t;
        if (j >= n) continue;
        const bool inJ = j >= k0 && j < k0 + bw;
        float vr, vi;
        if (!inI && !inJ) {
          vr = Frow[j] - re[t];
          vi = Frow[n + j] - im[t];
        } else if (inI && !inJ) {
          const f2 v = T[(long long)j * kPanel + (i - k0)];
          vr = v.x;
          vi = v.y;
        } else if (!inI && inJ) {
          const f2 v = T[(long long)i * kPanel + (j - k0)];
          vr = v.x;
          vi = v.y;
        } else {
          const f2 v = Pi[(i - k0) * kPanel + (j - k0)];
          vr = -v.x;
          vi = -v.y;
        }
        if (last) {
          vr = tc::to_tf32(vr);
          vi = tc::to_tf32(vi);
        }
        Frow[j] = vr;
        Frow[n + j] = vi;
      }
    }
  }
};

// Solve product: out[m*ldo + p] = alpha * (S' g)[p, m] (complex64).
template <int CB>
struct SolveEpi {
  f2* out;
  long long sOut, ldo;
  int n, k;
  float alpha;
  __device__ void operator()(int e, int tm, int tn, int row, uint32_t taddr) const {
    const int p = tm * tc::kBlockM + row;
    f2* o = out + e * sOut;
#pragma unroll 1
    for (int c0 = 0; c0 < CB; c0 += 16) {
      float re[16], im[16];
      tc::tmem_ld16(taddr + c0, re);
      tc::tmem_ld16(taddr + CB + c0, im);
      if (p >= n) continue;
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int m = tn * CB + c0 + t;
        if (c0 + t < CB && m < k) o[(long long)m * ldo + p] = f2{alpha * re[t], alpha * im[t]};
      }
    }
  }
};

// ------------------------------------------------------------------ couplings
// Writes the embedded, TF32-rounded RHS rows of complex column m.
__device__ __forceinline__ void write_emb(const Dims& d, float* Bemb, int e, int p, int m, f2 g) {
  const long long blk = (long long)e * d.nblkCB + m / d.CB;
  const long long rre = blk * 2 * d.CB + (m % d.CB);
  float* re_row = Bemb + rre * d.ldB;
  float* im_row = Bemb + (rre + d.CB) * d.ldB;
  re_row[p] = tc::to_tf32(g.x);
  re_row[d.n + p] = tc::to_tf32(-g.y);
  im_row[p] = tc::to_tf32(g.y);
  im_row[d.n + p] = tc::to_tf32(g.x);
}

// forward: g_i = R_i + C_i t (t = S'_{i-1} g_{i-1}; absent for layer 0)
// R is the real RHS (Rreal) or the complex64 residual of node e (Rc).
__global__ void __launch_bounds__(256) k_mx_couple_fwd(Dims d, int layer, const cplx* __restrict__ Z,
                                                       const double* __restrict__ A27, const double* __restrict__ B27,
                                                       const double* __restrict__ Rreal, const f2* __restrict__ Rc,
                                                       const f2* __restrict__ Tout, f2* __restrict__ Gc,
                                                       float* __restrict__ Bemb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.z;
  if (p >= d.n) return;
  const long long row = (long long)layer * d.n + p;
  const int px = p % d.nx, py = p / d.nx;
  const cplx z = Z[e];
  f2 c[9];
  int off[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    const bool ok = layer > 0 && px + dx >= 0 && px + dx < d.nx && py + dy >= 0 && py + dy < d.ny;
    c[t] = ok ? mcoef(A27, B27, d.N, t, row, z) : f2{0.f, 0.f};
    off[t] = ok ? p + dx + d.nx * dy : p;
  }
  const long long sG = d.N * d.k;
  const f2* T = Tout + (long long)e * d.n * d.k;
  const int m0 = blockIdx.y * 16, m1 = min(d.k, m0 + 16);
  for (int m = m0; m < m1; ++m) {
    f2 g = Rc ? Rc[e * sG + (long long)m * d.N + row] : f2{(float)Rreal[(long long)m * d.N + row], 0.f};
    if (layer > 0) {
#pragma unroll
      for (int t = 0; t < 9; ++t) f2fma(g, c[t], T[(long long)m * d.n + off[t]]);
    }
    Gc[e * sG + (long long)m * d.N + row] = g;
    write_emb(d, Bemb, e, p, m, g);
  }
}

// backward: s_i = g_i - U_i x_{i+1} (U_i = M[i, i+1], empty on the top layer)
__global__ void __launch_bounds__(256) k_mx_couple_bwd(Dims d, int layer, const cplx* __restrict__ Z,
                                                       const double* __restrict__ A27, const double* __restrict__ B27,
                                                       const f2* __restrict__ Gc, float* __restrict__ Bemb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.z;
  if (p >= d.n) return;
  const long long row = (long long)layer * d.n + p;
  const int px = p % d.nx, py = p / d.nx;
  const bool has_next = layer + 1 < d.nz;
  const cplx z = Z[e];
  f2 c[9];
  long long off[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    const bool ok = has_next && px + dx >= 0 && px + dx < d.nx && py + dy >= 0 && py + dy < d.ny;
    c[t] = ok ? mcoef(A27, B27, d.N, 18 + t, row, z) : f2{0.f, 0.f};
    off[t] = ok ? (long long)d.n + dx + d.nx * dy : 0;
  }
  const long long sG = d.N * d.k;
  const int m0 = blockIdx.y * 16, m1 = min(d.k, m0 + 16);
  for (int m = m0; m < m1; ++m) {
    const f2* col = Gc + e * sG + (long long)m * d.N + row;
    f2 s = col[0];
    f2 u{0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 9; ++t) f2fma(u, c[t], col[off[t]]);
    s.x -= u.x;
    s.y -= u.y;
    write_emb(d, Bemb, e, p, m, s);
  }
}

// ------------------------------------------------------------------ refinement
// Q_e (complex128) = (first ? 0 : Q_e) + d_e (complex64)
__global__ void k_mx_accumulate(long long total, int first, const f2* __restrict__ Gc, cplx* __restrict__ Q,
                                const int* __restrict__ active) {
  const int e = blockIdx.y;
  if (!active[e]) return;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const f2 v = Gc[e * total + t];
    if (first) {
      Q[e * total + t] = cplx{(double)v.x, (double)v.y};
    } else {
      cplx q = Q[e * total + t];
      q.re += v.x;
      q.im += v.y;
      Q[e * total + t] = q;
    }
  }
}

constexpr int kResBlock = 256;
constexpr int kResCols = 16;

// R_e = RHS - (Z_e B - A) Q_e in FP64; stores R as complex64 and per-block
// partial sums of |R|^2 (and |RHS|^2 for node 0).
__global__ void __launch_bounds__(kResBlock) k_mx_residual(Dims d, const cplx* __restrict__ Z,
                                                           const double* __restrict__ A27,
                                                           const double* __restrict__ B27,
                                                           const double* __restrict__ RHS,
                                                           const cplx* __restrict__ Q, f2* __restrict__ Rc,
                                                           double* __restrict__ partial, const int* __restrict__ active) {
  const int e = blockIdx.z;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (active[e] && i < d.N) {
    const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
    const cplx z = Z[e];
    cplx c[27];
    long long off[27];
#pragma unroll
    for (int s = 0; s < 27; ++s) {
      const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
      const bool ok = ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 &&
                      iz + dz < d.nz;
      const double a = ok ? A27[(long long)s * d.N + i] : 0.0;
      const double b = ok ? B27[(long long)s * d.N + i] : 0.0;
      c[s] = cplx{z.re * b - a, z.im * b};
      off[s] = ok ? (long long)dx + (long long)d.nx * (dy + (long long)d.ny * dz) : 0;
    }
    const long long sG = d.N * d.k;
    const int m0 = blockIdx.y * kResCols, m1 = min(d.k, m0 + kResCols);
    for (int m = m0; m < m1; ++m) {
      const cplx* q = Q + e * sG + (long long)m * d.N + i;
      const double b = RHS[(long long)m * d.N + i];
      cplx acc = cplx{b, 0.0};
#pragma unroll
      for (int s = 0; s < 27; ++s) {
        const cplx v = q[off[s]];
        acc.re -= c[s].re * v.re - c[s].im * v.im;
        acc.im -= c[s].re * v.im + c[s].im * v.re;
      }
      Rc[e * sG + (long long)m * d.N + i] = f2{(float)acc.re, (float)acc.im};
      rr += acc.re * acc.re + acc.im * acc.im;
      bb += b * b;
    }
  }
  __shared__ double red[2][kResBlock];
  red[0][threadIdx.x] = rr;
  red[1][threadIdx.x] = bb;
  __syncthreads();
  for (int w = kResBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long nblk = (long long)gridDim.x * gridDim.y;
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partial[(long long)e * nblk * 2 + 2 * b] = red[0][0];
    partial[(long long)e * nblk * 2 + 2 * b + 1] = red[1][0];
  }
}

// rel[e] = sqrt(sum |R|^2 / sum |RHS|^2), blocks summed in order
__global__ void k_mx_resnorm(int Ne, long long nblk, const double* __restrict__ partial, double* __restrict__ rel,
                             const int* __restrict__ active) {
  const int e = blockIdx.x;
  double s0 = 0.0, s1 = 0.0;
  for (long long b = threadIdx.x; b < nblk; b += blockDim.x) {
    s0 += partial[(long long)e * nblk * 2 + 2 * b];
    s1 += partial[(long long)e * nblk * 2 + 2 * b + 1];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) rel[e] = active[e] ? (red[1][0] > 0 ? sqrt(red[0][0] / red[1][0]) : 0.0) : 0.0;
}

// ------------------------------------------------------------------ host helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D fp32 tensor map: `inner` elements per row (row stride ld floats), `rows`
// rows, box 32 x box_rows, 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* map, const float* base, long long inner, long long rows, long long ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, class Epi>
cudaError_t launch_tc(cudaStream_t s, dim3 grid, const CUtensorMap& a, const CUtensorMap& b, tc::Geom geo,
                      const Epi& epi, int* status) {
  constexpr size_t smem = tc::Smem<BN>::kBytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc::k_tc_gemm<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tc::k_tc_gemm<BN, Epi><<<grid, tc::kThreads, smem, s>>>(a, b, geo, epi, status);
  return cudaGetLastError();
}

enum Buf { B_F = 0, B_T1, B_AOP, B_BOP, B_TC, B_PINV, B_GC, B_RC, B_BEMB, B_TOUT, B_PART, B_REL, B_ACTIVE, B_COUNT };

bool ensure(MixedWork& w, int idx, size_t bytes, cudaStream_t s, bool zero = false) {
  if (w.sizes[idx] >= bytes && w.bufs[idx]) {
    if (zero) cudaMemsetAsync(w.bufs[idx], 0, bytes, s);
    return true;
  }
  if (w.bufs[idx]) cudaFree(w.bufs[idx]);
  w.bufs[idx] = nullptr;
  w.sizes[idx] = 0;
  if (cudaMalloc(&w.bufs[idx], bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  w.sizes[idx] = bytes;
  if (zero) cudaMemsetAsync(w.bufs[idx], 0, bytes, s);
  return true;
}

template <class T>
T* buf(MixedWork& w, int idx) {
  return static_cast<T*>(w.bufs[idx]);
}

Dims make_dims(Grid g, int Ne, int k) {
  Dims d;
  d.nx = g.nx;
  d.ny = g.ny;
  d.nz = g.nz;
  d.n = g.n();
  d.Ne = Ne;
  d.N = g.N();
  d.ldF = ((2 * d.n + 31) / 32) * 32;
  d.nblk64 = (d.n + 63) / 64;
  d.k = k;
  d.CB = k <= 8 ? 8 : (k <= 16 ? 16 : (k <= 32 ? 32 : 64));
  d.nblkCB = (k + d.CB - 1) / d.CB;
  d.ldB = d.ldF;
  return d;
}

}  // namespace

void MixedWork::release() {
  for (int i = 0; i < 16; ++i) {
    if (bufs[i]) cudaFree(bufs[i]);
    bufs[i] = nullptr;
    sizes[i] = 0;
  }
  nz_factored = 0;
}

const char* mixed_factor(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, int* status) {
  Dims d = make_dims(g, Ne, 1);
  if (!encode_fn()) return "cuTensorMapEncodeTiled is not available from the driver";
  const size_t fbytes = sizeof(float) * (size_t)Ne * d.nz * d.n * d.ldF;
  if (!ensure(w, B_F, fbytes, s)) return "out of device memory (mixed factors)";
  if (!ensure(w, B_T1, sizeof(float) * (size_t)Ne * d.n * d.ldF, s)) return "out of device memory (schur scratch)";
  if (!ensure(w, B_AOP, sizeof(float) * (size_t)Ne * d.n * 2 * kPanel, s, true)) return "out of device memory";
  if (!ensure(w, B_BOP, sizeof(float) * (size_t)Ne * d.nblk64 * 128 * 2 * kPanel, s, true)) return "out of device memory";
  if (!ensure(w, B_TC, sizeof(f2) * (size_t)Ne * d.n * kPanel, s)) return "out of device memory";
  if (!ensure(w, B_PINV, sizeof(f2) * (size_t)Ne * kPanel * kPanel, s)) return "out of device memory";
  // The row-split padding [2n, ldF) is never read (the tensor maps stop at 2n).
  float* F = buf<float>(w, B_F);
  float* Aop = buf<float>(w, B_AOP);
  float* Bop = buf<float>(w, B_BOP);
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, Aop, 2 * kPanel, (long long)Ne * d.n, 2 * kPanel, 128)) return "tensor map (Aop) rejected";
  if (!make_map(&tmB, Bop, 2 * kPanel, (long long)Ne * d.nblk64 * 128, 2 * kPanel, 128))
    return "tensor map (Bop) rejected";
  const size_t panel_smem = sizeof(f2) * ((size_t)kPanel * (kPanel + 1) + (size_t)kRowsPerPanelCta * (kPanel + 1) + kPanel);
  static bool panel_attr = false;
  if (!panel_attr) {
    cudaFuncSetAttribute(k_mx_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem);
    panel_attr = true;
  }
  const long long sF = (long long)d.nz * d.n * d.ldF;
  for (int layer = 0; layer < d.nz; ++layer) {
    if (layer > 0)
      k_mx_schur1<<<dim3(cdiv(d.n, 256), d.n, Ne), 256, 0, s>>>(d, layer, Z, A27, B27, F, buf<float>(w, B_T1));
    k_mx_schur2<<<dim3(cdiv(d.n, 256), d.n, Ne), 256, 0, s>>>(d, layer, Z, A27, B27, buf<float>(w, B_T1), F);
    for (int k0 = 0; k0 < d.n; k0 += kPanel) {
      const int bw = d.n - k0 < kPanel ? d.n - k0 : kPanel;
      k_mx_panel<<<dim3(cdiv(d.n, kRowsPerPanelCta), Ne), 256, panel_smem, s>>>(
          d, layer, k0, bw, F, Aop, Bop, buf<f2>(w, B_TC), buf<f2>(w, B_PINV), status);
      SweepEpi epi{F + (long long)layer * d.n * d.ldF, sF, d.ldF, d.n, k0, bw, k0 + kPanel >= d.n,
                   buf<f2>(w, B_TC), buf<f2>(w, B_PINV)};
      tc::Geom geo{0, d.n, 0, d.nblk64 * 128, (2 * kPanel) / tc::kBlockK};
      cudaError_t err = launch_tc<128>(s, dim3(d.nblk64, cdiv(d.n, 128), Ne), tmA, tmB, geo, epi, status);
      if (err != cudaSuccess) return "tcgen05 sweep-update launch failed";
    }
  }
  w.nz_factored = d.nz;
  w.ne_factored = Ne;
  return nullptr;
}

namespace {

template <int CB>
const char* solve_sweeps(cudaStream_t s, const Dims& d, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, const double* Rreal, const f2* Rc, int* status) {
  float* F = buf<float>(w, B_F);
  f2* Gc = buf<f2>(w, B_GC);
  f2* Tout = buf<f2>(w, B_TOUT);
  float* Bemb = buf<float>(w, B_BEMB);
  CUtensorMap tmF, tmB;
  if (!make_map(&tmF, F, 2 * d.n, (long long)d.Ne * d.nz * d.n, d.ldF, 128)) return "tensor map (factors) rejected";
  if (!make_map(&tmB, Bemb, 2 * d.n, (long long)d.Ne * d.nblkCB * 2 * CB, d.ldB, 2 * CB))
    return "tensor map (rhs) rejected";
  const int nk = (2 * d.n + tc::kBlockK - 1) / tc::kBlockK;
  const dim3 cgrid(cdiv(d.n, 256), cdiv(d.k, 16), d.Ne);
  const dim3 ggrid(d.nblkCB, cdiv(d.n, 128), d.Ne);
  // forward sweep
  k_mx_couple_fwd<<<cgrid, 256, 0, s>>>(d, 0, Z, A27, B27, Rreal, Rc, Tout, Gc, Bemb);
  for (int i = 1; i < d.nz; ++i) {
    SolveEpi<CB> epi{Tout, (long long)d.n * d.k, d.n, d.n, d.k, 1.0f};
    tc::Geom geo{(i - 1) * d.n, d.nz * d.n, 0, d.nblkCB * 2 * CB, nk};
    if (launch_tc<2 * CB>(s, ggrid, tmF, tmB, geo, epi, status) != cudaSuccess) return "tcgen05 solve launch failed";
    k_mx_couple_fwd<<<cgrid, 256, 0, s>>>(d, i, Z, A27, B27, Rreal, Rc, Tout, Gc, Bemb);
  }
  // backward sweep: x_i overwrites g_i
  for (int i = d.nz - 1; i >= 0; --i) {
    k_mx_couple_bwd<<<cgrid, 256, 0, s>>>(d, i, Z, A27, B27, Gc, Bemb);
    SolveEpi<CB> epi{Gc + (long long)i * d.n, d.N * d.k, d.N, d.n, d.k, -1.0f};
    tc::Geom geo{i * d.n, d.nz * d.n, 0, d.nblkCB * 2 * CB, nk};
    if (launch_tc<2 * CB>(s, ggrid, tmF, tmB, geo, epi, status) != cudaSuccess) return "tcgen05 solve launch failed";
  }
  return nullptr;
}

const char* solve_once(cudaStream_t s, const Dims& d, const cplx* Z, const double* A27, const double* B27,
                       MixedWork& w, const double* Rreal, const f2* Rc, int* status) {
  switch (d.CB) {
    case 8: return solve_sweeps<8>(s, d, Z, A27, B27, w, Rreal, Rc, status);
    case 16: return solve_sweeps<16>(s, d, Z, A27, B27, w, Rreal, Rc, status);
    case 32: return solve_sweeps<32>(s, d, Z, A27, B27, w, Rreal, Rc, status);
    default: return solve_sweeps<64>(s, d, Z, A27, B27, w, Rreal, Rc, status);
  }
}

}  // namespace

const char* mixed_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                        MixedWork& w, const double* RHS, cplx* G, int k, double ir_tol, int ir_max,
                        MixedSolveStats* stats, int* status) {
  Dims d = make_dims(g, Ne, k);
  if (w.nz_factored != d.nz || w.ne_factored != Ne) return "mixed solve called without matching factors";
  const long long sG = d.N * k;
  if (!ensure(w, B_GC, sizeof(f2) * (size_t)Ne * sG, s)) return "out of device memory (node sweeps)";
  if (!ensure(w, B_RC, sizeof(f2) * (size_t)Ne * sG, s)) return "out of device memory (residuals)";
  if (!ensure(w, B_TOUT, sizeof(f2) * (size_t)Ne * d.n * k, s)) return "out of device memory";
  const size_t bemb = sizeof(float) * (size_t)Ne * d.nblkCB * 2 * d.CB * d.ldB;
  // rows of columns >= k and the padding stay zero; re-zero when the shape changes
  const bool shape_changed = w.sizes[B_BEMB] != bemb || w.bemb_k != k;
  if (!ensure(w, B_BEMB, bemb, s, shape_changed)) return "out of device memory";
  w.bemb_k = k;
  const dim3 rgrid(cdiv(d.N, kResBlock), cdiv(k, kResCols), Ne);
  const long long nblk = (long long)rgrid.x * rgrid.y;
  if (!ensure(w, B_PART, sizeof(double) * 2 * (size_t)Ne * nblk, s)) return "out of device memory";
  if (!ensure(w, B_REL, sizeof(double) * Ne, s)) return "out of device memory";
  if (!ensure(w, B_ACTIVE, sizeof(int) * Ne, s)) return "out of device memory";
  std::vector<int> active(Ne, 1);
  cudaMemcpyAsync(w.bufs[B_ACTIVE], active.data(), sizeof(int) * Ne, cudaMemcpyHostToDevice, s);
  std::vector<double> rel(Ne, 0.0), final_rel(Ne, 0.0);
  const int acc_blocks = (int)std::min<long long>(4096, (sG + 255) / 256);
  // first solve: Q_e = M~^{-1} RHS
  if (const char* m = solve_once(s, d, Z, A27, B27, w, RHS, nullptr, status)) return m;
  k_mx_accumulate<<<dim3(acc_blocks, Ne), 256, 0, s>>>(sG, 1, buf<f2>(w, B_GC), G, buf<int>(w, B_ACTIVE));
  int steps = 0;
  for (;;) {
    k_mx_residual<<<rgrid, kResBlock, 0, s>>>(d, Z, A27, B27, RHS, G, buf<f2>(w, B_RC), buf<double>(w, B_PART),
                                              buf<int>(w, B_ACTIVE));
    k_mx_resnorm<<<Ne, 256, 0, s>>>(Ne, nblk, buf<double>(w, B_PART), buf<double>(w, B_REL), buf<int>(w, B_ACTIVE));
    int st = 0;
    cudaMemcpyAsync(rel.data(), w.bufs[B_REL], sizeof(double) * Ne, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return "device error during refinement";
    if (st != 0) return nullptr;   // the caller reports the device status
    bool any = false;
    for (int e = 0; e < Ne; ++e) {
      if (!active[e]) continue;
      if (!std::isfinite(rel[e])) return "non-finite residual in the refinement";
      final_rel[e] = rel[e];
      if (rel[e] <= ir_tol) active[e] = 0;
      else any = true;
    }
    if (!any) break;
    if (steps >= ir_max) return "iterative refinement did not reach the tolerance";
    cudaMemcpyAsync(w.bufs[B_ACTIVE], active.data(), sizeof(int) * Ne, cudaMemcpyHostToDevice, s);
    if (const char* m = solve_once(s, d, Z, A27, B27, w, nullptr, buf<f2>(w, B_RC), status)) return m;
    k_mx_accumulate<<<dim3(acc_blocks, Ne), 256, 0, s>>>(sG, 0, buf<f2>(w, B_GC), G, buf<int>(w, B_ACTIVE));
    ++steps;
  }
  if (stats) {
    stats->steps_max = std::max(stats->steps_max, steps);
    for (int e = 0; e < Ne; ++e) stats->resid_max = std::max(stats->resid_max, final_rel[e]);
  }
  return nullptr;
}

}  // namespace feast
