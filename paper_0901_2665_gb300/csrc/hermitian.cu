// FEAST for a complex Hermitian A (Sec. III.A: "A is real symmetric or
// Hermitian"; Sec. III.B, Eqs. 10 and 12), FP64.
//
// With A Hermitian and B Hermitian positive definite, G(Z) = (Z B - A)^{-1}
// satisfies G(conj Z) = G(Z)^dagger (Sec. III.B), and the contour sum becomes
// Eq. 12:
//   Q = -sum_e (w_e r / 4) (e^{i theta_e} G(Z_e) + e^{-i theta_e} G(conj Z_e)) Y,
// with Y, Q complex.  Each of the 2 Ne shifts Z_e, conj Z_e is a "node" of
// the batched kernels (grid z = node).
//
// Node systems.  M = Z B - A is no longer complex symmetric (M^T = Z B^T - A^T
// and A^T = conj A), so the block elimination over the z-layers keeps both
// couplings: L_i = M[layer i, layer i-1] (the dz = -1 stencil slots of the
// rows of layer i) and U_i = M[layer i, layer i+1] (the dz = +1 slots):
//   S_1 = D_1,  S_i = D_i - L_i S_{i-1}^{-1} U_{i-1}.
// It exists without pivoting: the Hermitian part of M times -i, Im(Z) B, is
// definite (positive at Z_e, negative at conj Z_e), and so is it for every
// leading block and Schur complement, which are therefore nonsingular.  Each
// S_i is inverted in place by the (general) block sweep operator with panel
// width 32: sweeping panel K maps
//   S[K,K] -> -P^{-1},  S[K,j] -> P^{-1} S[K,j],  S[i,K] -> S[i,K] P^{-1},
//   S[i,j] -> S[i,j] - S[i,K] P^{-1} S[K,j]        (P = S[K,K]),
// and sweeping every panel leaves S'_i = -S_i^{-1}.  Then S_i = D_i + L_i S'_{i-1} U_{i-1}
// and the solve is
//   forward   g_1 = b_1,  g_i = b_i + L_i (S'_{i-1} g_{i-1}),
//   backward  x_nb = -S'_nb g_nb,  x_i = -S'_i (g_i - U_i x_{i+1}).
//
// Rayleigh-Ritz (Eqs. 6-9 with Q complex): A_Q = Q^H A Q, B_Q = Q^H B Q, the
// Hermitian-definite reduced problem by a two-stage complex Jacobi on one CTA
// (B_Q = U D U^H; C = D^{-1/2} U^H A_Q U D^{-1/2} = W E W^H; Phi = U D^{-1/2} W),
// X = Q Phi.  Each Jacobi rotation first turns the phase of a_pq away
// (a_pq = |a_pq| e^{i phi}) and then applies the real rotation of the modulus.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hermitian.cuh"
#include "prof.cuh"

namespace feast {

namespace {

constexpr int kHPanel = 32;   // sweep panel width

__device__ __forceinline__ cplx cconj(cplx a) { return cplx{a.re, -a.im}; }
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// (Z B - A)[row, row + off(s)] (0 outside the grid, as the operator stores it)
__device__ __forceinline__ cplx hcoef(const HermOp& o, cplx z, int s, long long row) {
  const long long N = o.g.N();
  const cplx a = o.A27[(long long)s * N + row];
  const cplx b = o.B27[(long long)s * N + row];
  return cplx{z.re * b.re - z.im * b.im - a.re, z.re * b.im + z.im * b.re - a.im};
}

// ---- Schur complement, pass 1: T1[a, q] = sum_b S'[a, b] U[b, q] with
// U = M[layer i-1, layer i]: U[b, q] is the dz = +1 coefficient of row
// (i-1, b) towards (i, q), nonzero for q - b in the 3 x 3 in-plane stencil.
__global__ void __launch_bounds__(256) k_h_schur1(HermOp o, int layer, const cplx* __restrict__ Z,
                                                  const cplx* __restrict__ Sprev, long long sS, cplx* __restrict__ T1,
                                                  long long sT) {
  const Grid g = o.g;
  const int n = g.n();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y, e = blockIdx.z;
  if (q >= n) return;
  const int qx = q % g.nx, qy = q / g.nx;
  const cplx z = Z[e];
  const cplx* S = Sprev + e * sS + (long long)a * n;
  cplx acc{0.0, 0.0};
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;   // q = b + (dx, dy)
    const int bx = qx - dx, by = qy - dy;
    if (bx < 0 || bx >= g.nx || by < 0 || by >= g.ny) continue;
    const int b = bx + g.nx * by;
    cfma(acc, S[b], hcoef(o, z, 18 + t, (long long)(layer - 1) * n + b));
  }
  T1[e * sT + (long long)a * n + q] = acc;
}

// ---- pass 2: S_i[p, q] = D_i[p, q] + sum_a L[p, a] T1[a, q]
__global__ void __launch_bounds__(256) k_h_schur2(HermOp o, int layer, int has_prev, const cplx* __restrict__ Z,
                                                  const cplx* __restrict__ T1, long long sT, cplx* __restrict__ S,
                                                  long long sS) {
  const Grid g = o.g;
  const int n = g.n();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y, e = blockIdx.z;
  if (q >= n) return;
  const long long rowp = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const cplx z = Z[e];
  cplx acc{0.0, 0.0};
  const int ddx = (q % g.nx) - px, ddy = (q / g.nx) - py;
  if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) acc = hcoef(o, z, 9 + (ddy + 1) * 3 + (ddx + 1), rowp);
  if (has_prev) {
    const cplx* T = T1 + e * sT;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dx = t % 3 - 1, dy = t / 3 - 1;
      if (px + dx < 0 || px + dx >= g.nx || py + dy < 0 || py + dy >= g.ny) continue;
      cfma(acc, hcoef(o, z, t, rowp), T[(long long)(p + dx + g.nx * dy) * n + q]);
    }
  }
  S[e * sS + (long long)p * n + q] = acc;
}

// ---- Gauss-Jordan sweep of the bw x bw diagonal panel P = S[K, K] (one CTA
// per node, one entry per thread): Pinv = P^{-1}.
__global__ void __launch_bounds__(1024) k_h_panel_invert(const cplx* __restrict__ Sall, long long sS, int n, int k0,
                                                         int bw, cplx* __restrict__ PinvAll, int* status) {
  __shared__ cplx P[kHPanel][kHPanel + 1];
  __shared__ cplx piv_inv;
  __shared__ int bad;
  const int e = blockIdx.x;
  const cplx* S = Sall + e * sS;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  const int i = tid / kHPanel, j = tid % kHPanel;
  if (i < bw && j < bw) P[i][j] = S[(long long)(k0 + i) * n + k0 + j];
  __syncthreads();
  for (int kk = 0; kk < bw; ++kk) {
    if (tid == 0) {
      const cplx d = P[kk][kk];
      const double mag = fabs(d.re) + fabs(d.im);
      if (!(mag > 0.0) || !isfinite(mag)) bad = 1;
      piv_inv = mag > 0.0 ? cinv(d) : cplx{0.0, 0.0};
    }
    __syncthreads();
    const cplx inv = piv_inv;
    const bool mine = i < bw && j < bw;
    cplx upd{0.0, 0.0};
    if (mine && i != kk && j != kk) upd = cmul(cmul(P[i][kk], inv), P[kk][j]);
    __syncthreads();
    if (mine && i != kk && j != kk) P[i][j] = csub(P[i][j], upd);
    __syncthreads();
    if (mine && i == kk && j != kk) P[kk][j] = cmul(inv, P[kk][j]);
    if (mine && j == kk && i != kk) P[i][kk] = cmul(P[i][kk], inv);
    __syncthreads();
    if (tid == 0) P[kk][kk] = cneg(inv);
    __syncthreads();
  }
  cplx* Pinv = PinvAll + (long long)e * kHPanel * kHPanel;
  if (i < bw && j < bw) Pinv[i * kHPanel + j] = cneg(P[i][j]);
  if (tid == 0 && bad) atomicExch(status, (int)DEV_PIVOT);
}

// ---- panel operands, one thread per index r < n:
//   Tc[r, c] = (S[r, K] Pinv)[c],  Lr[r, c] = S[k0 + c, r],  Tr[r, c] = (Pinv S[K, r])[c]
__global__ void __launch_bounds__(128) k_h_panel_T(const cplx* __restrict__ Sall, long long sS, int n, int k0, int bw,
                                                   const cplx* __restrict__ PinvAll, cplx* __restrict__ Tc,
                                                   cplx* __restrict__ Lr, cplx* __restrict__ Tr) {
  __shared__ cplx Pi[kHPanel][kHPanel];
  const int e = blockIdx.y;
  const cplx* Pinv = PinvAll + (long long)e * kHPanel * kHPanel;
  for (int t = threadIdx.x; t < kHPanel * kHPanel; t += blockDim.x) Pi[t / kHPanel][t % kHPanel] = Pinv[t];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const cplx* S = Sall + e * sS;
  const long long base = ((long long)e * n + r) * kHPanel;
  cplx v[kHPanel];
  // Tc from the panel's column part S[r, K]
#pragma unroll
  for (int m = 0; m < kHPanel; ++m) v[m] = m < bw ? S[(long long)r * n + k0 + m] : cplx{0.0, 0.0};
  for (int c = 0; c < bw; ++c) {
    cplx a{0.0, 0.0};
#pragma unroll
    for (int m = 0; m < kHPanel; ++m)
      if (m < bw) cfma(a, v[m], Pi[m][c]);
    Tc[base + c] = a;
  }
  // Tr and Lr from the row part S[K, r]
#pragma unroll
  for (int m = 0; m < kHPanel; ++m) v[m] = m < bw ? S[(long long)(k0 + m) * n + r] : cplx{0.0, 0.0};
  for (int c = 0; c < bw; ++c) {
    cplx b{0.0, 0.0};
#pragma unroll
    for (int m = 0; m < kHPanel; ++m)
      if (m < bw) cfma(b, Pi[c][m], v[m]);
    Tr[base + c] = b;
  }
#pragma unroll
  for (int c = 0; c < kHPanel; ++c)
    if (c < bw) Lr[base + c] = v[c];
}

// ---- trailing update of the sweep on 64 x 64 tiles:
//   i, j outside K:  S[i, j] -= sum_c Tc[i, c] Lr[j, c]
//   i in K, j not:   S[i, j]  = Tr[j, i - k0]
//   j in K, i not:   S[i, j]  = Tc[i, j - k0]
//   both in K:       S[i, j]  = -Pinv[i - k0, j - k0]
__global__ void __launch_bounds__(256) k_h_sweep_update(cplx* __restrict__ Sall, long long sS, int n, int k0, int bw,
                                                        const cplx* __restrict__ TcAll, const cplx* __restrict__ LrAll,
                                                        const cplx* __restrict__ TrAll,
                                                        const cplx* __restrict__ PinvAll) {
  constexpr int BM = 64, BK = 16;
  __shared__ cplx Ts[BK][BM];
  __shared__ cplx Ls[BK][BM];
  const int e = blockIdx.z;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const cplx* Tc = TcAll + (long long)e * n * kHPanel;
  const cplx* Lr = LrAll + (long long)e * n * kHPanel;
  const cplx* Tr = TrAll + (long long)e * n * kHPanel;
  cplx acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = cplx{0.0, 0.0};
  for (int kb = 0; kb < bw; kb += BK) {
    for (int t = tid; t < BM * BK; t += 256) {
      const int row = t / BK, kk = t % BK;
      const bool okk = kb + kk < bw;
      Ts[kk][row] = (i0 + row < n && okk) ? Tc[(long long)(i0 + row) * kHPanel + kb + kk] : cplx{0.0, 0.0};
      Ls[kk][row] = (j0 + row < n && okk) ? Lr[(long long)(j0 + row) * kHPanel + kb + kk] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Ts[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Ls[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
  cplx* S = Sall + e * sS;
  const cplx* Pinv = PinvAll + (long long)e * kHPanel * kHPanel;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= n) continue;
    const bool inI = i >= k0 && i < k0 + bw;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= n) continue;
      const bool inJ = j >= k0 && j < k0 + bw;
      cplx* dst = S + (long long)i * n + j;
      if (!inI && !inJ) *dst = csub(*dst, acc[r][c]);
      else if (inI && !inJ) *dst = Tr[(long long)j * kHPanel + (i - k0)];
      else if (!inI && inJ) *dst = Tc[(long long)i * kHPanel + (j - k0)];
      else *dst = cneg(Pinv[(i - k0) * kHPanel + (j - k0)]);
    }
  }
}

// ---- C_e = alpha S_e X_e: S n x n row-major (general), X, C n x k column-major
__global__ void __launch_bounds__(256) k_h_gemm(int n, int k, double alpha, const cplx* __restrict__ Sall, long long sS,
                                                const cplx* __restrict__ Xall, long long ldx, long long sX,
                                                cplx* __restrict__ Call, long long ldc, long long sC) {
  constexpr int BM = 64, BN = 32, BK = 16;
  __shared__ cplx As[BK][BM];
  __shared__ cplx Bs[BK][BN];
  const int e = blockIdx.z;
  const int p0 = blockIdx.y * BM, m0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const cplx* S = Sall + e * sS;
  const cplx* X = Xall + e * sX;
  cplx acc[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = cplx{0.0, 0.0};
  for (int kb = 0; kb < n; kb += BK) {
    for (int t = tid; t < BM * BK; t += 256) {
      const int row = t / BK, kk = t % BK;
      As[kk][row] = (p0 + row < n && kb + kk < n) ? S[(long long)(p0 + row) * n + kb + kk] : cplx{0.0, 0.0};
    }
    for (int t = tid; t < BN * BK; t += 256) {
      const int col = t / BK, kk = t % BK;
      Bs[kk][col] = (m0 + col < k && kb + kk < n) ? X[(long long)(m0 + col) * ldx + kb + kk] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[4], b[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
      b[0] = Bs[kk][tx];
      b[1] = Bs[kk][tx + 16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        cfma(acc[r][0], a[r], b[0]);
        cfma(acc[r][1], a[r], b[1]);
      }
    }
    __syncthreads();
  }
  cplx* C = Call + e * sC;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + ty + 16 * r;
    if (p >= n) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int m = m0 + tx + 16 * c;
      if (m < k) C[(long long)m * ldc + p] = cplx{alpha * acc[r][c].re, alpha * acc[r][c].im};
    }
  }
}

// ---- layer couplings of the sweeps (one thread per row p and column m):
// forward:  G_e[layer i] = RHS[layer i] + L_i Tmp_e
__global__ void __launch_bounds__(256) k_h_couple_fwd(HermOp o, int layer, const cplx* __restrict__ Z,
                                                      const cplx* __restrict__ RHS, const cplx* __restrict__ Tmp,
                                                      long long sT, cplx* __restrict__ G, long long sG, int k) {
  const Grid g = o.g;
  const int n = g.n();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y, e = blockIdx.z;
  if (p >= n || m >= k) return;
  const long long N = g.N();
  const long long row = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const cplx z = Z[e];
  cplx acc = RHS[(long long)m * N + row];
  const cplx* T = Tmp + e * sT + (long long)m * n;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    if (px + dx < 0 || px + dx >= g.nx || py + dy < 0 || py + dy >= g.ny) continue;
    cfma(acc, hcoef(o, z, t, row), T[p + dx + g.nx * dy]);
  }
  G[e * sG + (long long)m * N + row] = acc;
}

// backward: Tmp_e = G_e[layer i] - U_i G_e[layer i+1]
__global__ void __launch_bounds__(256) k_h_couple_bwd(HermOp o, int layer, const cplx* __restrict__ Z,
                                                      const cplx* __restrict__ G, long long sG, cplx* __restrict__ Tmp,
                                                      long long sT, int k) {
  const Grid g = o.g;
  const int n = g.n();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y, e = blockIdx.z;
  if (p >= n || m >= k) return;
  const long long N = g.N();
  const long long row = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const cplx z = Z[e];
  const cplx* col = G + e * sG + (long long)m * N + row;
  cplx u{0.0, 0.0};
  if (layer + 1 < g.nz) {
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dx = t % 3 - 1, dy = t / 3 - 1;
      if (px + dx < 0 || px + dx >= g.nx || py + dy < 0 || py + dy >= g.ny) continue;
      cfma(u, hcoef(o, z, 18 + t, row), col[n + dx + g.nx * dy]);
    }
  }
  Tmp[e * sT + (long long)m * n + p] = csub(col[0], u);
}

__global__ void k_h_copy_layer(const cplx* __restrict__ RHS, long long N, int n, int k, cplx* __restrict__ G,
                               long long sG) {
  const int e = blockIdx.y;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * k;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % n, m = t / n;
    G[e * sG + m * N + r] = RHS[m * N + r];
  }
}

// ---- Q = sum_e coef_e X_e in node order (Eq. 12: complex coefficients)
__global__ void k_h_quadrature(long long total, int nodes, const cplx* __restrict__ coef, const cplx* __restrict__ X,
                               cplx* __restrict__ Q) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    cplx acc{0.0, 0.0};
    for (int e = 0; e < nodes; ++e) cfma(acc, coef[e], X[e * total + t]);
    Q[t] = acc;
  }
}

// ---- Y = C X for a complex 27-point operator C, X and Y complex N x k
__global__ void __launch_bounds__(256) k_h_stencil(Grid g, const cplx* __restrict__ C27, const cplx* __restrict__ X,
                                                   cplx* __restrict__ Y, int k) {
  const long long N = g.N();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (i >= N || m >= k) return;
  const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.n());
  const cplx* x = X + (long long)m * N;
  cplx acc{0.0, 0.0};
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
    if (ix + dx < 0 || ix + dx >= g.nx || iy + dy < 0 || iy + dy >= g.ny || iz + dz < 0 || iz + dz >= g.nz) continue;
    cfma(acc, C27[(long long)s * N + i], x[i + dx + g.nx * (dy + (long long)g.ny * dz)]);
  }
  Y[(long long)m * N + i] = acc;
}

// ---- Gram: out (k x k) = X^H Y over row chunks, partial per chunk; deterministic
constexpr int kHGramRows = 4096;
__global__ void __launch_bounds__(256) k_h_gram_partial(long long N, int k, const cplx* __restrict__ X,
                                                        const cplx* __restrict__ Y, cplx* __restrict__ partial) {
  constexpr int T = 32, BK = 16;
  __shared__ cplx Xs[BK][T + 1];
  __shared__ cplx Ys[BK][T + 1];
  const int a0 = blockIdx.x * T, b0 = blockIdx.y * T;
  const long long r0 = (long long)blockIdx.z * kHGramRows, r1 = min(N, r0 + kHGramRows);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  cplx acc[2][2] = {};
  for (long long rb = r0; rb < r1; rb += BK) {
    for (int t = tid; t < BK * T; t += 256) {
      const int rr = t % BK, c = t / BK;
      const long long r = rb + rr;
      Xs[rr][c] = (r < r1 && a0 + c < k) ? X[(long long)(a0 + c) * N + r] : cplx{0.0, 0.0};
      Ys[rr][c] = (r < r1 && b0 + c < k) ? Y[(long long)(b0 + c) * N + r] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < BK; ++rr)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) cfma_conj(acc[i][j], Xs[rr][ty + 16 * i], Ys[rr][tx + 16 * j]);
    __syncthreads();
  }
  cplx* P = partial + (long long)blockIdx.z * k * k;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < k && b < k) P[a + (long long)b * k] = acc[i][j];
    }
}

__global__ void k_h_gram_reduce(int nchunks, int total, const cplx* __restrict__ partial, cplx* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  cplx s{0.0, 0.0};
  for (int c = 0; c < nchunks; ++c) s = cadd(s, partial[(long long)c * total + t]);
  out[t] = s;
}

// ---- C (N x k) = Q (N x m) P (m x k), complex, column-major
__global__ void __launch_bounds__(256) k_h_gemm_tall(long long N, int m, int k, const cplx* __restrict__ Q,
                                                     const cplx* __restrict__ P, cplx* __restrict__ C) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r >= N || c >= k) return;
  cplx acc{0.0, 0.0};
  for (int j = 0; j < m; ++j) cfma(acc, Q[(long long)j * N + r], P[(long long)c * m + j]);
  C[(long long)c * N + r] = acc;
}

// ---- complex Hermitian Jacobi on one CTA (matrix in shared memory, ld m+1;
// accumulated rotations to V, column-major m x m in global memory).  Round-robin
// ordering as in the real kernel; a pair is skipped when |a_pq| <= 1e-15
// sqrt(|a_pp a_qq|) or <= abs_tol.  Returns the sweeps used or -1.
__device__ int hjacobi_block(cplx* As, int m, cplx* V, double* cs, cplx* ph, int* pq, int* flag, double abs_tol,
                             int max_sweeps) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ld = m + 1;
  const int mp = m + (m & 1);
  const int npairs = mp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int step = 0; step < mp - 1; ++step) {
      for (int kq = tid; kq < npairs; kq += nth) {
        int p, q;
        if (kq == 0) {
          p = mp - 1;
          q = step;
        } else {
          p = (step + kq) % (mp - 1);
          q = (step - kq + (mp - 1)) % (mp - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        cplx e{1.0, 0.0};
        if (q < m) {
          const cplx apq = As[p * ld + q];
          const double mag = hypot(apq.re, apq.im);
          const double app = As[p * ld + p].re, aqq = As[q * ld + q].re;
          if (mag > 1e-15 * sqrt(fabs(app)) * sqrt(fabs(aqq)) && mag > abs_tol && mag > 1e-300) {
            e = cplx{apq.re / mag, apq.im / mag};
            const double tau = (aqq - app) / (2.0 * mag);
            const double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            *flag = 1;
          }
        }
        pq[2 * kq] = p;
        pq[2 * kq + 1] = q;
        cs[2 * kq] = c;
        cs[2 * kq + 1] = s;
        ph[kq] = e;
      }
      __syncthreads();
      // rows: row p <- c row_p - s e row_q, row q <- s row_p + c e row_q
      for (int t = tid; t < npairs * m; t += nth) {
        const int kq = t / m, j = t % m;
        const int p = pq[2 * kq], q = pq[2 * kq + 1];
        const double s = cs[2 * kq + 1];
        if (q >= m || s == 0.0) continue;
        const double c = cs[2 * kq];
        const cplx e = ph[kq];
        const cplx ap = As[p * ld + j], aq = As[q * ld + j];
        const cplx eq = cmul(e, aq);
        As[p * ld + j] = cplx{c * ap.re - s * eq.re, c * ap.im - s * eq.im};
        As[q * ld + j] = cplx{s * ap.re + c * eq.re, s * ap.im + c * eq.im};
      }
      __syncthreads();
      // columns (and V): col p <- c col_p - s conj(e) col_q, col q <- s col_p + c conj(e) col_q
      for (int t = tid; t < npairs * m; t += nth) {
        const int kq = t / m, i = t % m;
        const int p = pq[2 * kq], q = pq[2 * kq + 1];
        const double s = cs[2 * kq + 1];
        if (q >= m || s == 0.0) continue;
        const double c = cs[2 * kq];
        const cplx ec = cconj(ph[kq]);
        const cplx ap = As[i * ld + p], aq = cmul(ec, As[i * ld + q]);
        As[i * ld + p] = cplx{c * ap.re - s * aq.re, c * ap.im - s * aq.im};
        As[i * ld + q] = cplx{s * ap.re + c * aq.re, s * ap.im + c * aq.im};
        const cplx vp = V[(long long)p * m + i], vq = cmul(ec, V[(long long)q * m + i]);
        V[(long long)p * m + i] = cplx{c * vp.re - s * vq.re, c * vp.im - s * vq.im};
        V[(long long)q * m + i] = cplx{s * vp.re + c * vq.re, s * vp.im + c * vq.im};
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) return sweep + 1;
  }
  return -1;
}

// Two-stage Hermitian-definite reduced eigensolve (one CTA), m <= 64.
// work: U, W, T (m*m complex each).  eps ascending, Phi column-major.
__global__ void __launch_bounds__(1024) k_h_reduced_eig(int m, const cplx* __restrict__ AQ, const cplx* __restrict__ BQ,
                                                        double* __restrict__ eps, cplx* __restrict__ Phi,
                                                        cplx* __restrict__ work, int* status) {
  extern __shared__ cplx hsm[];
  const int ld = m + 1;
  cplx* As = hsm;                                           // m*(m+1)
  cplx* ph = As + m * ld;                                   // m/2+2
  double* cs = reinterpret_cast<double*>(ph + (m / 2 + 2));  // 2*(m/2+2)
  double* dsc = cs + 2 * (m / 2 + 2);                       // m
  double* ev = dsc + m;                                     // m
  int* pq = reinterpret_cast<int*>(ev + m);                 // 2*(m/2+2)
  int* flag = pq + 2 * (m / 2 + 2);
  cplx* U = work;
  cplx* W = work + (long long)m * m;
  cplx* T = work + 2LL * m * m;
  const int tid = threadIdx.x, nth = blockDim.x;
  // stage 1: B_Q (Hermitian part), U = I
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    const cplx a = BQ[i + (long long)j * m], b = cconj(BQ[j + (long long)i * m]);
    As[i * ld + j] = cplx{0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
    U[t] = cplx{i == j ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  const int sw = hjacobi_block(As, m, U, cs, ph, pq, flag, 0.0, 40);
  __shared__ double dmm[2];
  if (tid == 0) {
    double dmin = As[0].re, dmax = As[0].re;
    for (int i = 1; i < m; ++i) {
      dmin = fmin(dmin, As[i * ld + i].re);
      dmax = fmax(dmax, As[i * ld + i].re);
    }
    dmm[0] = dmin;
    dmm[1] = dmax;
  }
  __syncthreads();
  if (!(dmm[0] > 1e-14 * dmm[1])) {
    if (tid == 0) atomicExch(status, (int)DEV_BQ_NOT_SPD);
    return;
  }
  if (sw < 0) {
    if (tid == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  for (int i = tid; i < m; i += nth) dsc[i] = 1.0 / sqrt(As[i * ld + i].re);
  __syncthreads();
  // C = D^{-1/2} U^H A_Q U D^{-1/2}
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    const cplx a = AQ[i + (long long)j * m], b = cconj(AQ[j + (long long)i * m]);
    As[i * ld + j] = cplx{0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += nth) {   // T = A_Q U (col-major)
    const int i = t % m, j = t / m;
    cplx s{0.0, 0.0};
    for (int l = 0; l < m; ++l) cfma(s, As[i * ld + l], U[(long long)j * m + l]);
    T[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += nth) {   // As = D^{-1/2} U^H T D^{-1/2}
    const int i = t % m, j = t / m;
    cplx s{0.0, 0.0};
    for (int l = 0; l < m; ++l) cfma_conj(s, U[(long long)i * m + l], T[(long long)j * m + l]);
    As[i * ld + j] = cplx{s.re * dsc[i] * dsc[j], s.im * dsc[i] * dsc[j]};
  }
  __syncthreads();
  double fro2 = 0.0;
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    W[t] = cplx{i == j ? 1.0 : 0.0, 0.0};
    if (i < j) {
      const cplx a = As[i * ld + j], b = cconj(As[j * ld + i]);
      const cplx v{0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
      As[i * ld + j] = v;
      As[j * ld + i] = cconj(v);
    } else if (i == j) {
      As[i * ld + i] = cplx{As[i * ld + i].re, 0.0};
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int t = 0; t < m * m; ++t) {
      const cplx v = As[(t % m) * ld + t / m];
      fro2 += v.re * v.re + v.im * v.im;
    }
    dmm[0] = sqrt(fro2);
  }
  __syncthreads();
  const int sw2 = hjacobi_block(As, m, W, cs, ph, pq, flag, 2.0 * 2.220446049250313e-16 * dmm[0], 40);
  if (sw2 < 0) {
    if (tid == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  for (int i = tid; i < m; i += nth) ev[i] = As[i * ld + i].re;
  __syncthreads();
  // Phi = U D^{-1/2} W, columns at their ascending rank
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    const double ej = ev[j];
    int rank = 0;
    for (int l = 0; l < m; ++l) rank += (ev[l] < ej) || (ev[l] == ej && l < j);
    cplx s{0.0, 0.0};
    for (int l = 0; l < m; ++l) {
      const cplx u = U[(long long)l * m + i];
      cfma(s, cplx{u.re * dsc[l], u.im * dsc[l]}, W[(long long)j * m + l]);
    }
    Phi[i + (long long)rank * m] = s;
    if (i == 0) eps[rank] = ej;
  }
}

// ---- residual norms (Table I caption), complex vectors: per column j,
// out[3j] = ||A x - l B x||_1, out[3j+1] = ||x||_1, out[3j+2] = ||A x||_1 (moduli)
__global__ void __launch_bounds__(256) k_h_residual_norms(long long N, const cplx* __restrict__ AX,
                                                          const cplx* __restrict__ BX, const double* __restrict__ lam,
                                                          const cplx* __restrict__ X, double* __restrict__ out) {
  const int j = blockIdx.x;
  const double l = lam[j];
  double r = 0.0, xn = 0.0, an = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    const cplx ax = AX[(long long)j * N + i], bx = BX[(long long)j * N + i], x = X[(long long)j * N + i];
    r += hypot(ax.re - l * bx.re, ax.im - l * bx.im);
    xn += hypot(x.re, x.im);
    an += hypot(ax.re, ax.im);
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = r;
  red[1][threadIdx.x] = xn;
  red[2][threadIdx.x] = an;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[3 * j + threadIdx.x] = red[threadIdx.x][0];
}

// ||A||_1 of a Hermitian 27-point operator = max_i sum_s |A27[s][i]| (single block)
__global__ void k_h_norm1(long long N, const cplx* __restrict__ A27, double* out) {
  double mx = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < 27; ++t) s += hypot(A27[(long long)t * N + i].re, A27[(long long)t * N + i].im);
    mx = fmax(mx, s);
  }
  __shared__ double red[256];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

__global__ void k_h_residual_finish(int k, const double* __restrict__ norms, const double* __restrict__ normA,
                                    double* __restrict__ resid, double* __restrict__ resid_paper) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  if (resid) resid[j] = norms[3 * j] / (normA[0] * norms[3 * j + 1]);
  if (resid_paper) resid_paper[j] = norms[3 * j] / norms[3 * j + 2];
}

__global__ void k_h_permute(long long N, int k, const int* __restrict__ perm, const cplx* __restrict__ src,
                            cplx* __restrict__ dst) {
  const long long total = N * k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % N, j = t / N;
    dst[t] = src[(long long)perm[j] * N + r];
  }
}

__device__ __forceinline__ double h_uniform(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// Y(row, col) = u(seed, col N + row) + i u(seed + 1, col N + row)
__global__ void k_h_random(long long total, uint64_t seed, cplx* __restrict__ Y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    Y[t] = cplx{h_uniform(seed, (uint64_t)t), h_uniform(seed + 1ULL, (uint64_t)t)};
}

unsigned grid1(long long total) { return (unsigned)std::max<long long>(1, std::min<long long>(152 * 32, (total + 255) / 256)); }

}  // namespace

size_t herm_factor_bytes(Grid g, int nodes) {
  const long long n = g.n();
  return sizeof(cplx) * ((size_t)nodes * g.nz * n * n + (size_t)nodes * n * n + 3 * (size_t)nodes * n * kHPanel +
                         (size_t)nodes * kHPanel * kHPanel) + 1024;
}

void herm_factor(cudaStream_t s, const HermOp& o, int nodes, const cplx* Z, cplx* work, int* status) {
  const Grid g = o.g;
  const int n = g.n(), nb = g.nz;
  const long long nn = (long long)n * n;
  const long long sF = (long long)nb * nn;
  cplx* F = work;
  cplx* T1 = F + (size_t)nodes * sF;
  cplx* Tc = T1 + (size_t)nodes * nn;
  cplx* Lr = Tc + (size_t)nodes * n * kHPanel;
  cplx* Tr = Lr + (size_t)nodes * n * kHPanel;
  cplx* Pinv = Tr + (size_t)nodes * n * kHPanel;
  for (int i = 0; i < nb; ++i) {
    cplx* Si = F + (long long)i * nn;
    if (i > 0) k_h_schur1<<<dim3(cdiv(n, 256), n, nodes), 256, 0, s>>>(o, i, Z, Si - nn, sF, T1, nn);
    k_h_schur2<<<dim3(cdiv(n, 256), n, nodes), 256, 0, s>>>(o, i, i > 0, Z, T1, nn, Si, sF);
    prof::count_launch(i > 0 ? 2 : 1);
    for (int k0 = 0; k0 < n; k0 += kHPanel) {
      const int bw = std::min(kHPanel, n - k0);
      k_h_panel_invert<<<nodes, kHPanel * kHPanel, 0, s>>>(Si, sF, n, k0, bw, Pinv, status);
      k_h_panel_T<<<dim3(cdiv(n, 128), nodes), 128, 0, s>>>(Si, sF, n, k0, bw, Pinv, Tc, Lr, Tr);
      k_h_sweep_update<<<dim3(cdiv(n, 64), cdiv(n, 64), nodes), 256, 0, s>>>(Si, sF, n, k0, bw, Tc, Lr, Tr, Pinv);
      prof::count_launch(3);
    }
  }
}

void herm_solve(cudaStream_t s, const HermOp& o, int nodes, const cplx* Z, const cplx* work, const cplx* RHS, cplx* G,
                cplx* Tmp, int k) {
  const Grid g = o.g;
  const int n = g.n(), nb = g.nz;
  const long long N = g.N(), nn = (long long)n * n, sF = (long long)nb * nn;
  const long long sG = N * k, sT = (long long)n * k;
  const cplx* F = work;
  k_h_copy_layer<<<dim3(grid1((long long)n * k), nodes), 256, 0, s>>>(RHS, N, n, k, G, sG);
  const dim3 cg(cdiv(n, 256), k, nodes);
  const dim3 gg(cdiv(k, 32), cdiv(n, 64), nodes);
  for (int i = 1; i < nb; ++i) {
    k_h_gemm<<<gg, 256, 0, s>>>(n, k, 1.0, F + (long long)(i - 1) * nn, sF, G + (long long)(i - 1) * n, N, sG, Tmp, n,
                                sT);
    k_h_couple_fwd<<<cg, 256, 0, s>>>(o, i, Z, RHS, Tmp, sT, G, sG, k);
  }
  for (int i = nb - 1; i >= 0; --i) {
    k_h_couple_bwd<<<cg, 256, 0, s>>>(o, i, Z, G, sG, Tmp, sT, k);
    k_h_gemm<<<gg, 256, 0, s>>>(n, k, -1.0, F + (long long)i * nn, sF, Tmp, n, sT, G + (long long)i * n, N, sG);
  }
  prof::count_launch(1 + 2 * (nb - 1) + 2 * nb);
}

void herm_quadrature(cudaStream_t s, long long N, int k, int nodes, const cplx* coef, const cplx* G, cplx* Q) {
  k_h_quadrature<<<grid1(N * k), 256, 0, s>>>(N * k, nodes, coef, G, Q);
  prof::count_launch();
}

void herm_stencil(cudaStream_t s, Grid g, const cplx* C27, const cplx* X, cplx* Y, int k) {
  k_h_stencil<<<dim3(cdiv(g.N(), 256), k), 256, 0, s>>>(g, C27, X, Y, k);
  prof::count_launch();
}

long long herm_gram_elems(long long N, int k) { return (long long)cdiv(N, kHGramRows) * k * k; }

void herm_gram(cudaStream_t s, long long N, int k, const cplx* X, const cplx* Y, cplx* partial, cplx* out) {
  const int nchunks = cdiv(N, kHGramRows);
  k_h_gram_partial<<<dim3(cdiv(k, 32), cdiv(k, 32), nchunks), 256, 0, s>>>(N, k, X, Y, partial);
  k_h_gram_reduce<<<cdiv(k * k, 256), 256, 0, s>>>(nchunks, k * k, partial, out);
  prof::count_launch(2);
}

void herm_reduced_eig(cudaStream_t s, int m, const cplx* AQ, const cplx* BQ, double* eps, cplx* Phi, cplx* work,
                      int* status) {
  const size_t smem = sizeof(cplx) * ((size_t)m * (m + 1) + (m / 2 + 2)) + sizeof(double) * (2 * (m / 2 + 2) + 2 * m) +
                      sizeof(int) * (2 * (m / 2 + 2) + 1) + 64;
  static PerDevice<cudaError_t> attr;
  attr.get([] { return cudaFuncSetAttribute(k_h_reduced_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); },
           cudaErrorInvalidDevice);
  k_h_reduced_eig<<<1, 1024, smem, s>>>(m, AQ, BQ, eps, Phi, work, status);
  prof::count_launch();
}

void herm_gemm_tall(cudaStream_t s, long long N, int m, int k, const cplx* Q, const cplx* P, cplx* C) {
  k_h_gemm_tall<<<dim3(cdiv(N, 256), k), 256, 0, s>>>(N, m, k, Q, P, C);
  prof::count_launch();
}

void herm_residuals(cudaStream_t s, Grid g, const cplx* A27, const cplx* B27, const double* lam, const cplx* X, int k,
                    cplx* AX, cplx* BX, double* norms, double* normA, double* resid, double* resid_paper) {
  herm_stencil(s, g, A27, X, AX, k);
  herm_stencil(s, g, B27, X, BX, k);
  k_h_residual_norms<<<k, 256, 0, s>>>(g.N(), AX, BX, lam, X, norms);
  k_h_norm1<<<1, 256, 0, s>>>(g.N(), A27, normA);
  k_h_residual_finish<<<cdiv(k, 128), 128, 0, s>>>(k, norms, normA, resid, resid_paper);
  prof::count_launch(3);
}

void herm_permute(cudaStream_t s, long long N, int k, const int* perm, const cplx* src, cplx* dst) {
  k_h_permute<<<grid1(N * k), 256, 0, s>>>(N, k, perm, src, dst);
  prof::count_launch();
}

void herm_random(cudaStream_t s, long long N, int k, uint64_t seed, cplx* Y) {
  k_h_random<<<grid1(N * k), 256, 0, s>>>(N * k, seed, Y);
  prof::count_launch();
}

}  // namespace feast
