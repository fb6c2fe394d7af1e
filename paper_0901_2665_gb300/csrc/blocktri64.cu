// FP64 factor-and-solve of the node systems (Z_e B - A) Q_e = RHS (Fig. 2 step 2).
//
// M_e is block tridiagonal over the z-layers: diagonal blocks D_i (n x n, the
// in-plane 9-point part) and couplings C_i = M_e[layer i, layer i-1] (the
// dz = -1 stencil slots; by symmetry M_e[layer i-1, layer i] = C_i^T).
// Unpivoted block elimination: S_1 = D_1, S_i = D_i - C_i S_{i-1}^{-1} C_i^T.
// Each S_i is inverted in place by the symmetric block sweep operator, which
// leaves S'_i = -S_i^{-1}; so S_i = D_i + C_i S'_{i-1} C_i^T.  Every leading
// block of a complex symmetric matrix with positive definite imaginary part
// (Im(Z_e) B, Im Z_e > 0) is nonsingular, so no pivoting is needed for the
// elimination to exist.
//
// Solve with the stored S'_i:
//   forward   g_1 = b_1,  g_i = b_i + C_i (S'_{i-1} g_{i-1})
//   backward  x_nb = -S'_nb g_nb,  x_i = -S'_i (g_i - C_{i+1}^T x_{i+1})
#include "kernels.cuh"
#include "prof.cuh"

namespace feast {

namespace {

constexpr int kPanel64 = 32;   // sweep panel width of the FP64 path

// ---- Schur complement, pass 1: T1[a, q] = sum_b S'[a, b] C[q, b]  (T1 = S' C^T)
__global__ void __launch_bounds__(256) k_schur_pass1(Grid g, int layer, const cplx* __restrict__ Z,
                                                     const double* __restrict__ A27,
                                                     const double* __restrict__ B27,
                                                     const cplx* __restrict__ Sprev, long long sS,
                                                     cplx* __restrict__ T1, long long sT) {
  const int n = g.n();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  const int e = blockIdx.z;
  if (q >= n) return;
  const long long N = g.N();
  const long long rowq = (long long)layer * n + q;
  const int qx = q % g.nx, qy = q / g.nx;
  const cplx z = Z[e];
  const cplx* S = Sprev + e * sS + (long long)a * n;
  cplx acc = cplx{0.0, 0.0};
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dx = t % 3 - 1, dy = t / 3 - 1;
    if (qx + dx < 0 || qx + dx >= g.nx || qy + dy < 0 || qy + dy >= g.ny) continue;
    const double av = A27[(long long)t * N + rowq], bv = B27[(long long)t * N + rowq];
    cfma(acc, S[q + dx + g.nx * dy], cplx{z.re * bv - av, z.im * bv});
  }
  T1[e * sT + (long long)a * n + q] = acc;
}

// ---- Schur complement, pass 2: S_i[p, q] = D_i[p, q] + sum_a C[p, a] T1[a, q]
__global__ void __launch_bounds__(256) k_schur_pass2(Grid g, int layer, int has_prev,
                                                     const cplx* __restrict__ Z,
                                                     const double* __restrict__ A27,
                                                     const double* __restrict__ B27,
                                                     const cplx* __restrict__ T1, long long sT,
                                                     cplx* __restrict__ S, long long sS) {
  const int n = g.n();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  const int e = blockIdx.z;
  if (q >= n) return;
  const long long N = g.N();
  const long long rowp = (long long)layer * n + p;
  const int px = p % g.nx, py = p / g.nx;
  const cplx z = Z[e];
  cplx acc = cplx{0.0, 0.0};
  // D_i: in-plane slots (dz = 0) are 9..17
  const int ddx = (q % g.nx) - px, ddy = (q / g.nx) - py;
  if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) {
    const int s = 9 + (ddy + 1) * 3 + (ddx + 1);
    const double av = A27[(long long)s * N + rowp], bv = B27[(long long)s * N + rowp];
    acc = cplx{z.re * bv - av, z.im * bv};
  }
  if (has_prev) {
    const cplx* T = T1 + e * sT;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dx = t % 3 - 1, dy = t / 3 - 1;
      if (px + dx < 0 || px + dx >= g.nx || py + dy < 0 || py + dy >= g.ny) continue;
      const double av = A27[(long long)t * N + rowp], bv = B27[(long long)t * N + rowp];
      cfma(acc, cplx{z.re * bv - av, z.im * bv}, T[(long long)(p + dx + g.nx * dy) * n + q]);
    }
  }
  S[e * sS + (long long)p * n + q] = acc;
}

// ---- sweep of one diagonal panel P = S[K, K] (bw x bw), one CTA per node:
// scalar sweeps on every pivot give -P^{-1}; store Pinv = P^{-1}.
__global__ void __launch_bounds__(1024) k_panel_invert(cplx* __restrict__ Sall, long long sS, int n, int k0,
                                                       int bw, cplx* __restrict__ PinvAll, int* status) {
  __shared__ cplx P[kPanel64][kPanel64 + 1];
  __shared__ cplx piv_inv;
  __shared__ int bad;
  const int e = blockIdx.x;
  const cplx* S = Sall + e * sS;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int t = tid; t < bw * bw; t += blockDim.x) {
    const int i = t / bw, j = t % bw;
    P[i][j] = S[(long long)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  for (int kk = 0; kk < bw; ++kk) {
    if (tid == 0) {
      const cplx d = P[kk][kk];
      const double mag = fabs(d.re) + fabs(d.im);
      if (!(mag > 0.0) || !isfinite(mag)) bad = 1;
      piv_inv = (mag > 0.0) ? cinv(d) : cplx{0.0, 0.0};
    }
    __syncthreads();
    const cplx inv = piv_inv;
    // trailing update with the old pivot row/column (bw*bw <= blockDim.x:
    // one entry per thread)
    const int i = tid / bw, j = tid % bw;
    const bool mine = tid < bw * bw && i != kk && j != kk;
    cplx upd = cplx{0.0, 0.0};
    if (mine) upd = cmul(cmul(P[i][kk], inv), P[kk][j]);
    __syncthreads();
    if (mine) P[i][j] = csub(P[i][j], upd);
    __syncthreads();
    for (int t = tid; t < bw; t += blockDim.x) {
      if (t != kk) {
        P[t][kk] = cmul(P[t][kk], inv);
        P[kk][t] = cmul(P[kk][t], inv);
      }
    }
    __syncthreads();
    if (tid == 0) P[kk][kk] = cneg(inv);
    __syncthreads();
  }
  cplx* Pinv = PinvAll + (long long)e * kPanel64 * kPanel64;
  for (int t = tid; t < bw * bw; t += blockDim.x) {
    const int i = t / bw, j = t % bw;
    Pinv[i * kPanel64 + j] = cneg(P[i][j]);
  }
  if (tid == 0 && bad) atomicExch(status, (int)DEV_PIVOT);
}

// ---- T[i, :] = S[i, K] Pinv and L[i, :] = S[i, K] for every row i
__global__ void __launch_bounds__(128) k_panel_T(const cplx* __restrict__ Sall, long long sS, int n, int k0,
                                                 int bw, const cplx* __restrict__ PinvAll,
                                                 cplx* __restrict__ Tall, cplx* __restrict__ Lall) {
  __shared__ cplx Pi[kPanel64][kPanel64];
  const int e = blockIdx.y;
  const cplx* Pinv = PinvAll + (long long)e * kPanel64 * kPanel64;
  for (int t = threadIdx.x; t < kPanel64 * kPanel64; t += blockDim.x) Pi[t / kPanel64][t % kPanel64] = Pinv[t];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cplx* Srow = Sall + e * sS + (long long)i * n + k0;
  cplx l[kPanel64];
#pragma unroll
  for (int m = 0; m < kPanel64; ++m) l[m] = (m < bw) ? Srow[m] : cplx{0.0, 0.0};
  cplx* T = Tall + (long long)e * n * kPanel64 + (long long)i * kPanel64;
  cplx* L = Lall + (long long)e * n * kPanel64 + (long long)i * kPanel64;
  for (int c = 0; c < bw; ++c) {
    cplx acc = cplx{0.0, 0.0};
#pragma unroll
    for (int m = 0; m < kPanel64; ++m)
      if (m < bw) cfma(acc, l[m], Pi[m][c]);
    T[c] = acc;
    L[c] = l[c];
  }
}

// ---- trailing update of the sweep, 64x64 tiles:
//   i, j outside K:  S[i, j] -= sum_k T[i, k] L[j, k]
//   i in K, j not:   S[i, j]  = T[j, i - k0]
//   j in K, i not:   S[i, j]  = T[i, j - k0]
//   both in K:       S[i, j]  = -Pinv[i - k0, j - k0]
__global__ void __launch_bounds__(256) k_sweep_update(cplx* __restrict__ Sall, long long sS, int n, int k0,
                                                      int bw, const cplx* __restrict__ Tall,
                                                      const cplx* __restrict__ Lall,
                                                      const cplx* __restrict__ PinvAll) {
  constexpr int BM = 64, BK = 16;
  __shared__ cplx Ts[BK][BM];
  __shared__ cplx Ls[BK][BM];
  const int e = blockIdx.z;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const cplx* T = Tall + (long long)e * n * kPanel64;
  const cplx* L = Lall + (long long)e * n * kPanel64;
  cplx acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = cplx{0.0, 0.0};
  for (int kb = 0; kb < bw; kb += BK) {
    for (int t = tid; t < BM * BK; t += 256) {
      const int row = t / BK, kk = t % BK;
      const bool okk = kb + kk < bw;
      Ts[kk][row] = (i0 + row < n && okk) ? T[(long long)(i0 + row) * kPanel64 + kb + kk] : cplx{0.0, 0.0};
      Ls[kk][row] = (j0 + row < n && okk) ? L[(long long)(j0 + row) * kPanel64 + kb + kk] : cplx{0.0, 0.0};
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
  const cplx* Pinv = PinvAll + (long long)e * kPanel64 * kPanel64;
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
      if (!inI && !inJ) {
        *dst = csub(*dst, acc[r][c]);
      } else if (inI && !inJ) {
        *dst = T[(long long)j * kPanel64 + (i - k0)];
      } else if (!inI && inJ) {
        *dst = T[(long long)i * kPanel64 + (j - k0)];
      } else {
        *dst = cneg(Pinv[(i - k0) * kPanel64 + (j - k0)]);
      }
    }
  }
}

// ---- C = alpha * S X, S n x n (symmetric, row-major), X, C n x k col-major.
// With qp set (the backward sweep) each entry c of C is also folded into the
// node's share of the quadrature sum (Eq. 15): qp[e*sQ + m*ldq + p] = Re{coef_e c}.
__global__ void __launch_bounds__(256) k_zgemm_sym(int n, int k, double alpha, const cplx* __restrict__ Sall,
                                                   long long sS, const cplx* __restrict__ Xall, long long ldx,
                                                   long long sX, cplx* __restrict__ Call, long long ldc,
                                                   long long sC, double* __restrict__ qp, long long sQ,
                                                   long long ldq, const cplx* __restrict__ coef) {
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
  const cplx ce = qp ? coef[e] : cplx{0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + ty + 16 * r;
    if (p >= n) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int m = m0 + tx + 16 * c;
      if (m >= k) continue;
      const cplx v{alpha * acc[r][c].re, alpha * acc[r][c].im};
      C[(long long)m * ldc + p] = v;
      if (qp) qp[e * sQ + (long long)m * ldq + p] = ce.re * v.re - ce.im * v.im;
    }
  }
}

}  // namespace

void zgemm_sym(cudaStream_t s, int n, int k, int Ne, double alpha, const cplx* S, long long sS, const cplx* X,
               long long ldx, long long sX, cplx* C, long long ldc, long long sC, double* qp, long long sQ,
               long long ldq, const cplx* coef) {
  dim3 grid(cdiv(k, 32), cdiv(n, 64), Ne);
  k_zgemm_sym<<<grid, 256, 0, s>>>(n, k, alpha, S, sS, X, ldx, sX, C, ldc, sC, qp, sQ, ldq, coef);
  prof::count_launch();
}

void factor_fp64(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                 const Fp64Work& w) {
  const int n = g.n(), nb = g.nz;
  const long long nn = (long long)n * n;
  const long long sF = (long long)nb * nn;  // node stride of the factor array
  prof::begin(s, prof::FP64_SOLVE);
  prof::add_work(prof::FP64_SOLVE, 8.0 * n * (double)n * n * nb * Ne);
  for (int i = 0; i < nb; ++i) {
    prof::count_launch((i > 0 ? 2 : 1) + 3 * cdiv(n, kPanel64));
    cplx* Si = w.F + (long long)i * nn;
    if (i > 0) {
      const cplx* Sprev = w.F + (long long)(i - 1) * nn;
      k_schur_pass1<<<dim3(cdiv(n, 256), n, Ne), 256, 0, s>>>(g, i, Z, A27, B27, Sprev, sF, w.T1, nn);
    }
    k_schur_pass2<<<dim3(cdiv(n, 256), n, Ne), 256, 0, s>>>(g, i, i > 0, Z, A27, B27, w.T1, nn, Si, sF);
    for (int k0 = 0; k0 < n; k0 += kPanel64) {
      const int bw = n - k0 < kPanel64 ? n - k0 : kPanel64;
      k_panel_invert<<<Ne, 1024, 0, s>>>(Si, sF, n, k0, bw, w.Pinv, w.status);
      k_panel_T<<<dim3(cdiv(n, 128), Ne), 128, 0, s>>>(Si, sF, n, k0, bw, w.Pinv, w.T, w.L);
      k_sweep_update<<<dim3(cdiv(n, 64), cdiv(n, 64), Ne), 256, 0, s>>>(Si, sF, n, k0, bw, w.T, w.L, w.Pinv);
    }
  }
  prof::end(s, prof::FP64_SOLVE);
}

void solve_fp64(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                const cplx* F, const double* RHS, cplx* G, cplx* Tmp, int k, double* Qp, const cplx* coef) {
  const int n = g.n(), nb = g.nz;
  const long long N = g.N();
  const long long nn = (long long)n * n;
  const long long sF = (long long)nb * nn;
  const long long sG = N * k;
  const long long sT = (long long)n * k;
  // forward sweep
  rhs_to_complex(s, n, k, Ne, RHS, N, G, N, sG);
  for (int i = 1; i < nb; ++i) {
    zgemm_sym(s, n, k, Ne, 1.0, F + (long long)(i - 1) * nn, sF, G + (long long)(i - 1) * n, N, sG, Tmp, n, sT);
    couple_forward(s, g, i, Ne, Z, A27, B27, RHS, Tmp, sT, G, sG, k);
  }
  // backward sweep (x_i overwrites g_i)
  for (int i = nb - 1; i >= 0; --i) {
    couple_backward(s, g, i, Ne, Z, A27, B27, G, sG, Tmp, sT, k);
    zgemm_sym(s, n, k, Ne, -1.0, F + (long long)i * nn, sF, Tmp, n, sT, G + (long long)i * n, N, sG,
              Qp ? Qp + (long long)i * n : nullptr, sG, N, coef);
  }
}

}  // namespace feast
