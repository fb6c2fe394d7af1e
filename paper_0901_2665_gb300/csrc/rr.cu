// Rayleigh-Ritz in FP64 (Fig. 2 steps 3-5; Eqs. 6-9) and the residuals of
// Table I.
#include <cooperative_groups.h>

#include <mutex>

#include "kernels.cuh"
#include "prof.cuh"

namespace feast {

namespace {

// ---------------------------------------------------------------- Gram
constexpr int kGramTile = 64;
constexpr int kGramRows = 4096;   // rows per partial sum (split-K chunk)

// partial[chunk][a + b*k1] = sum_{r in chunk} X[r, a] Y[r, b].  With sym set
// the product is symmetric (X^T C X for a symmetric C): blockIdx.x enumerates
// only the tiles on and above the diagonal, and the reduction mirrors them.
__global__ void __launch_bounds__(256) k_gram_partial(long long N, int k1, int k2, const double* __restrict__ X,
                                                      const double* __restrict__ Y, double* __restrict__ partial,
                                                      int sym) {
  constexpr int BK = 16;
  __shared__ double Xs[BK][kGramTile + 1];
  __shared__ double Ys[BK][kGramTile + 1];
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
  const int a0 = ta * kGramTile, b0 = tb * kGramTile;
  const long long r0 = (long long)blockIdx.z * kGramRows;
  const long long r1 = min(N, r0 + kGramRows);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (long long rb = r0; rb < r1; rb += BK) {
    for (int t = tid; t < BK * kGramTile; t += 256) {
      const int rr = t % BK, c = t / BK;
      const long long r = rb + rr;
      Xs[rr][c] = (r < r1 && a0 + c < k1) ? X[(long long)(a0 + c) * N + r] : 0.0;
      Ys[rr][c] = (r < r1 && b0 + c < k2) ? Y[(long long)(b0 + c) * N + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < BK; ++rr) {
      double xa[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = Xs[rr][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yb[j] = Ys[rr][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(xa[i], yb[j], acc[i][j]);
    }
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
      if (b < k2) P[a + (long long)b * k1] = acc[i][j];
    }
  }
}

// out = sum over chunks in chunk order (deterministic); with sym the entries
// below the diagonal tiles are read from their mirror images
__global__ void k_gram_reduce(int nchunks, int k1, int total, const double* __restrict__ partial,
                              double* __restrict__ out, int sym) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int src = t;
  if (sym) {
    const int a = t % k1, b = t / k1;
    if (a / kGramTile > b / kGramTile) src = b + a * k1;
  }
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(long long)c * total + src];
  out[t] = s;
}

// ---------------------------------------------------------------- tall GEMM
// C[r, c] = sum_j Q[r, j] P[j, c]; 64 rows x 64 cols per CTA.
__global__ void __launch_bounds__(256) k_dgemm_tall(long long N, int m, int k, const double* __restrict__ Q,
                                                    const double* __restrict__ P, double* __restrict__ C) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double Qs[BK][BM + 1];
  __shared__ double Ps[BK][BN + 1];
  const long long r0 = (long long)blockIdx.x * BM;
  const int c0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (int kb = 0; kb < m; kb += BK) {
    for (int t = tid; t < BK * BM; t += 256) {
      const int row = t % BM, kk = t / BM;
      const long long r = r0 + row;
      Qs[kk][row] = (r < N && kb + kk < m) ? Q[(long long)(kb + kk) * N + r] : 0.0;
    }
    for (int t = tid; t < BK * BN; t += 256) {
      const int kk = t % BK, col = t / BK;
      Ps[kk][col] = (kb + kk < m && c0 + col < k) ? P[(long long)(c0 + col) * m + kb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double q[4], p[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = Qs[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) p[j] = Ps[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(q[i], p[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long r = r0 + tx + 16 * i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + ty + 16 * j;
      if (c < k) C[(long long)c * N + r] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------- Jacobi
// Cyclic two-sided Jacobi (Golub & Van Loan, sym.schur2 rotations) with the
// round-robin parallel ordering: in each step the m' = m + (m odd) indices are
// split into m'/2 disjoint pairs, m'-1 steps make a sweep that meets every
// pair once.  The matrix lives in shared memory (ld m+1); the accumulated
// rotations go to V (global, col-major, ld m).  Returns the sweeps used, or
// -1 when the sweep cap is hit.
__device__ int jacobi_block(double* As, int m, double* V, double* cs, int* pq, int* flag, double abs_floor,
                             int max_sweeps) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ld = m + 1;
  const int mp = m + (m & 1);
  const int npairs = mp / 2;
  double fro = 0.0;
  // scale of the matrix for the absolute threshold
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) s += As[i * ld + j] * As[i * ld + j];
    cs[2 * npairs] = sqrt(s);
  }
  __syncthreads();
  fro = cs[2 * npairs];
  // A rotation is skipped when |a_pq| <= 1e-15 sqrt(|a_pp a_qq|) (the
  // relative criterion that keeps small eigenvalues of a positive definite
  // matrix accurate to their own scale) or |a_pq| <= abs_floor * ||A||_F.
  const double abs_tol = abs_floor * fro;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int step = 0; step < mp - 1; ++step) {
      // pairs of this step and their rotations
      for (int k = tid; k < npairs; k += nth) {
        int p, q;
        if (k == 0) {
          p = mp - 1;
          q = step;
        } else {
          p = (step + k) % (mp - 1);
          q = (step - k + (mp - 1)) % (mp - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = As[p * ld + q];
          const double app = As[p * ld + p], aqq = As[q * ld + q];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app)) * sqrt(fabs(aqq)) && fabs(apq) > abs_tol &&
              fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                          : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            *flag = 1;
          }
        }
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int t = tid; t < npairs * m; t += nth) {
        const int k = t / m, j = t % m;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const double s = cs[2 * k + 1];
        if (q >= m || s == 0.0) continue;
        const double c = cs[2 * k];
        const double ap = As[p * ld + j], aq = As[q * ld + j];
        As[p * ld + j] = c * ap - s * aq;
        As[q * ld + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int t = tid; t < npairs * m; t += nth) {
        const int k = t / m, i = t % m;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const double s = cs[2 * k + 1];
        if (q >= m || s == 0.0) continue;
        const double c = cs[2 * k];
        const double ap = As[i * ld + p], aq = As[i * ld + q];
        As[i * ld + p] = c * ap - s * aq;
        As[i * ld + q] = s * ap + c * aq;
        const double vp = V[(long long)p * m + i], vq = V[(long long)q * m + i];
        V[(long long)p * m + i] = c * vp - s * vq;
        V[(long long)q * m + i] = s * vp + c * vq;
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) return sweep + 1;
  }
  return -1;
}

// Two-stage reduced eigensolve (one CTA):
//   B_Q = U diag(d) U^T           (Jacobi)
//   C   = D^{-1/2} U^T A_Q U D^{-1/2}
//   C   = W diag(eps) W^T          (Jacobi)
//   Phi = U D^{-1/2} W, eps ascending.  Phi^T B_Q Phi = I.
// work: U (m*m), W (m*m), T (m*m) doubles.
__global__ void __launch_bounds__(1024) k_reduced_eig(int m, const double* __restrict__ AQ,
                                                      const double* __restrict__ BQ, double* __restrict__ eps,
                                                      double* __restrict__ Phi, double* __restrict__ work,
                                                      int* status) {
  extern __shared__ double smem[];
  const int ld = m + 1;
  double* As = smem;                       // m*(m+1)
  double* cs = As + m * ld;                // 2*(m/2+1) + 1
  double* dsc = cs + 2 * (m / 2 + 2);      // m: D^{-1/2}
  double* ev = dsc + m;                    // m: eigenvalues of C
  int* pq = (int*)(ev + m);                // 2*(m/2+1)
  int* flag = pq + 2 * (m / 2 + 2);
  double* U = work;
  double* W = work + (long long)m * m;
  double* T = work + 2LL * m * m;
  const int tid = threadIdx.x, nth = blockDim.x;

  // ---- stage 1: B_Q
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;   // column-major input
    As[i * ld + j] = 0.5 * (BQ[i + (long long)j * m] + BQ[j + (long long)i * m]);
    U[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Stage 1 uses the purely relative criterion.  B_Q that is singular to
  // working precision keeps producing rounding-level off-diagonal entries in
  // its null directions and exhausts the sweep cap; that case is reported as
  // "not s.p.d." below through its diagonal ratio, any other cap-out as a
  // Jacobi failure.
  const int sw = jacobi_block(As, m, U, cs, pq, flag, 0.0, 40);
  __shared__ double dminmax[2];
  if (tid == 0) {
    double dmin = As[0], dmax = As[0];
    for (int i = 1; i < m; ++i) {
      dmin = fmin(dmin, As[i * ld + i]);
      dmax = fmax(dmax, As[i * ld + i]);
    }
    dminmax[0] = dmin;
    dminmax[1] = dmax;
  }
  __syncthreads();
  if (!(dminmax[0] > 1e-14 * dminmax[1])) {
    if (tid == 0) atomicExch(status, (int)DEV_BQ_NOT_SPD);
    return;
  }
  if (sw < 0) {
    if (tid == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  for (int i = tid; i < m; i += nth) dsc[i] = 1.0 / sqrt(As[i * ld + i]);
  __syncthreads();

  // ---- C = D^{-1/2} U^T A_Q U D^{-1/2}
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    As[i * ld + j] = 0.5 * (AQ[i + (long long)j * m] + AQ[j + (long long)i * m]);
  }
  __syncthreads();
  // T = A_Q U   (T col-major)
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(As[i * ld + l], U[(long long)j * m + l], s);
    T[t] = s;
  }
  __syncthreads();
  // As = D^{-1/2} U^T T D^{-1/2}
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(U[(long long)i * m + l], T[(long long)j * m + l], s);
    As[i * ld + j] = s * dsc[i] * dsc[j];
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    if (i < j) {
      const double v = 0.5 * (As[i * ld + j] + As[j * ld + i]);
      As[i * ld + j] = v;
      As[j * ld + i] = v;
    }
    W[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();

  // ---- stage 2
  // Stage 2: the Ritz values are wanted to absolute accuracy ~eps ||C||, so
  // rotations below 2 eps ||C||_F are skipped (this also bounds the sweeps
  // when C has eigenvalues near zero).
  const int sw2 = jacobi_block(As, m, W, cs, pq, flag, 2.0 * 2.220446049250313e-16, 40);
  if (sw2 < 0) {
    if (tid == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  for (int i = tid; i < m; i += nth) ev[i] = As[i * ld + i];
  __syncthreads();
  // Phi = U D^{-1/2} W, columns placed at their ascending rank
  for (int t = tid; t < m * m; t += nth) {
    const int i = t % m, j = t / m;
    const double ej = ev[j];
    int rank = 0;
    for (int l = 0; l < m; ++l) rank += (ev[l] < ej) || (ev[l] == ej && l < j);
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(U[(long long)l * m + i] * dsc[l], W[(long long)j * m + l], s);
    Phi[i + (long long)rank * m] = s;
    if (i == 0) eps[rank] = ej;
  }
}

// ---------------------------------------------------------------- Jacobi on a cluster
// The same two-stage eigensolve spread over a thread-block cluster of CL CTAs
// (8 or 16), so that CL SMs share its FP64 work: CTA r owns the rows
// i = r, r + CL, r + 2 CL, ... of the working matrix and of the accumulated
// rotations.  The rotations, their order (round-robin pairs, m' - 1 steps a
// sweep), the skip criteria and the sweep cap are those of jacobi_block.  One
// step of the sweep:
//   1. every CTA computes the rotations of all pairs from the current matrix
//      (a_pp, a_qq, a_pq read from their owners' shared memory): the same
//      IEEE operations on the same values, so every CTA holds the same (c, s)
//      without a broadcast or a barrier;
//   2. every CTA copies the partner row of each of its rows, forms its rows
//      of J^T A and then of (J^T A) J into the second buffer and applies the
//      column rotations to its rows of V; cluster barrier (after it every
//      CTA's new rows are complete and no CTA reads the old buffer any more);
//      the buffers swap.
namespace cg = cooperative_groups;

constexpr int kClThreads = 256;
constexpr int kClMinM = 32;   // smaller reduced problems stay on one CTA

struct ClLayout {
  int m, CL, R, ld, npairs;
  __device__ ClLayout(int m_, int cl) : m(m_), CL(cl) {
    R = (m + CL - 1) / CL;
    ld = m + 1;
    npairs = (m + (m & 1)) / 2;
  }
};

// shared memory of one CTA (doubles first, then ints)
__host__ __device__ inline size_t cl_smem_bytes(int m, int CL) {
  const int R = (m + CL - 1) / CL;
  const int np = (m + (m & 1)) / 2;
  return sizeof(double) * (2 * (size_t)R * (m + 1) + 3 * (size_t)R * m + 2 * (size_t)np + 5 * (size_t)m + 8) +
         sizeof(int) * (3 * (size_t)m + 8);
}

struct ClSmem {
  double *A0, *A1, *X, *P, *V, *rc, *rs, *cj, *sj, *dg, *dsc, *aux, *red;
  int *part, *isp, *rk, *flag;
  __device__ ClSmem(double* base, const ClLayout& L) {
    double* d = base;
    A0 = d; d += L.R * L.ld;
    A1 = d; d += L.R * L.ld;
    X = d; d += L.R * L.m;
    P = d; d += L.R * L.m;
    V = d; d += L.R * L.m;
    rc = d; d += L.npairs;
    rs = d; d += L.npairs;
    cj = d; d += L.m;
    sj = d; d += L.m;
    dg = d; d += L.m;
    dsc = d; d += L.m;
    aux = d; d += L.m;
    red = d; d += 8;
    int* ip = reinterpret_cast<int*>(d);
    part = ip; ip += L.m;
    isp = ip; ip += L.m;
    rk = ip; ip += L.m;
    flag = ip;
  }
};

// pair k of step `step` in the round-robin order (p < q; q >= m: no pair)
__device__ __forceinline__ void rr_pair(int k, int step, int mp, int& p, int& q) {
  if (k == 0) {
    p = mp - 1;
    q = step;
  } else {
    p = (step + k) % (mp - 1);
    q = (step - k + (mp - 1)) % (mp - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Cyclic Jacobi over the cluster on the rows in *Acur (swapped in place as the
// steps alternate buffers).  Every CTA returns the same value: the sweeps
// used, or -1 when the cap is hit.
__device__ int jacobi_cluster(cg::cluster_group& cl, const ClLayout& L, ClSmem& S, double*& Acur, double*& Anext,
                              double abs_tol, int max_sweeps) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rank = (int)cl.block_rank();
  const int m = L.m, ld = L.ld, CL = L.CL, R = L.R;
  const int mp = m + (m & 1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *S.flag = 0;
    for (int step = 0; step < mp - 1; ++step) {
      // 1. all rotations of the step, computed by every CTA
      for (int k = tid; k < L.npairs; k += nth) {
        int p, q;
        rr_pair(k, step, mp, p, q);
        double c = 1.0, sn = 0.0;
        if (q < m) {
          const double* rowp = cl.map_shared_rank(Acur, p % CL) + (p / CL) * ld;
          const double* rowq = cl.map_shared_rank(Acur, q % CL) + (q / CL) * ld;
          const double apq = rowp[q], app = rowp[p], aqq = rowq[q];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app)) * sqrt(fabs(aqq)) && fabs(apq) > abs_tol && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        S.rc[k] = c;
        S.rs[k] = sn;
      }
      __syncthreads();
      // 2. per-index rotation tables
      for (int k = tid; k < L.npairs; k += nth) {
        int p, q;
        rr_pair(k, step, mp, p, q);
        const double c = S.rc[k], sn = S.rs[k];
        if (q < m && sn != 0.0) {
          S.part[p] = q;
          S.part[q] = p;
          S.isp[p] = 1;
          S.isp[q] = 0;
          S.cj[p] = S.cj[q] = c;
          S.sj[p] = S.sj[q] = sn;
          *S.flag = 1;
        } else {
          S.part[p] = -1;
          if (q < m) S.part[q] = -1;
        }
      }
      __syncthreads();
      // 3. partner rows (current values) of this CTA's rows
      for (int t = tid; t < R * m; t += nth) {
        const int lr = t / m, j = t % m, i = lr * CL + rank;
        if (i >= m) continue;
        const int pi = S.part[i];
        if (pi >= 0) S.P[lr * m + j] = cl.map_shared_rank(Acur, pi % CL)[(pi / CL) * ld + j];
      }
      __syncthreads();
      // 4. rows: X = J^T A (this CTA's rows); V <- V J
      for (int t = tid; t < R * m; t += nth) {
        const int lr = t / m, j = t % m, i = lr * CL + rank;
        if (i >= m) continue;
        const double a = Acur[lr * ld + j];
        const int pi = S.part[i];
        double x = a;
        if (pi >= 0) {
          const double c = S.cj[i], sn = S.sj[i], pr = S.P[lr * m + j];
          x = S.isp[i] ? c * a - sn * pr : sn * pr + c * a;
        }
        S.X[lr * m + j] = x;
        const int pj = S.part[j];
        if (pj >= 0 && S.isp[j]) {
          const double c = S.cj[j], sn = S.sj[j];
          const double vp = S.V[lr * m + j], vq = S.V[lr * m + pj];
          S.V[lr * m + j] = c * vp - sn * vq;
          S.V[lr * m + pj] = sn * vp + c * vq;
        }
      }
      __syncthreads();
      // 5. columns: A' = X J into the second buffer
      for (int t = tid; t < R * m; t += nth) {
        const int lr = t / m, j = t % m, i = lr * CL + rank;
        if (i >= m) continue;
        const double x = S.X[lr * m + j];
        const int pj = S.part[j];
        double v = x;
        if (pj >= 0) {
          const double c = S.cj[j], sn = S.sj[j], xo = S.X[lr * m + pj];
          v = S.isp[j] ? c * x - sn * xo : sn * xo + c * x;
        }
        Anext[lr * ld + j] = v;
      }
      cl.sync();
      double* t = Acur;
      Acur = Anext;
      Anext = t;
    }
    __syncthreads();
    const int any = *S.flag;
    __syncthreads();
    if (!any) return sweep + 1;
  }
  return -1;
}

// diag[i] = A[i, i] for every i, read from the owners (all CTAs get all).
__device__ void cl_gather_diag(cg::cluster_group& cl, const ClLayout& L, const double* Acur, double* out) {
  for (int i = threadIdx.x; i < L.m; i += blockDim.x)
    out[i] = cl.map_shared_rank(Acur, i % L.CL)[(i / L.CL) * L.ld + i];
  cl.sync();
}

// Two-stage reduced eigensolve on a cluster (see k_reduced_eig); work as
// there: U, W, T (m*m doubles each), here row-major.  The work matrices are
// written and read by different CTAs of the launch, so their reads bypass L1
// (__ldcg) after the fence and cluster barrier that publish them.
__global__ void __launch_bounds__(kClThreads) k_reduced_eig_cluster(int m, const double* __restrict__ AQ,
                                                                    const double* __restrict__ BQ,
                                                                    double* __restrict__ eps, double* __restrict__ Phi,
                                                                    double* __restrict__ work, int* status) {
  extern __shared__ double clsmem[];
  cg::cluster_group cl = cg::this_cluster();
  const ClLayout L(m, (int)cl.num_blocks());
  ClSmem S(clsmem, L);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rank = (int)cl.block_rank();
  const int CL = L.CL, R = L.R, ld = L.ld;
  double* Ug = work;
  double* Wg = work + (long long)m * m;
  double* Tg = work + 2LL * m * m;
  double* Acur = S.A0;
  double* Anext = S.A1;

  // ---- stage 1: B_Q (symmetrised), V = I
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i >= m) continue;
    Acur[lr * ld + j] = 0.5 * (BQ[i + (long long)j * m] + BQ[j + (long long)i * m]);
    S.V[lr * m + j] = (i == j) ? 1.0 : 0.0;
  }
  cl.sync();
  const int sw = jacobi_cluster(cl, L, S, Acur, Anext, 0.0, 40);
  cl_gather_diag(cl, L, Acur, S.dg);
  double dmin = S.dg[0], dmax = S.dg[0];
  for (int i = 1; i < m; ++i) {
    dmin = fmin(dmin, S.dg[i]);
    dmax = fmax(dmax, S.dg[i]);
  }
  if (!(dmin > 1e-14 * dmax)) {
    if (tid == 0 && rank == 0) atomicExch(status, (int)DEV_BQ_NOT_SPD);
    return;
  }
  if (sw < 0) {
    if (tid == 0 && rank == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  for (int i = tid; i < m; i += nth) S.dsc[i] = 1.0 / sqrt(S.dg[i]);
  // U (row-major) to global
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i < m) Ug[(long long)i * m + j] = S.V[lr * m + j];
  }
  __threadfence();
  cl.sync();
  // ---- T = A_Q U (this CTA's rows; A_Q symmetrised into the free buffer)
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i < m) Acur[lr * ld + j] = 0.5 * (AQ[i + (long long)j * m] + AQ[j + (long long)i * m]);
  }
  __syncthreads();
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i >= m) continue;
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(Acur[lr * ld + l], __ldcg(Ug + (long long)l * m + j), s);
    Tg[(long long)i * m + j] = s;
  }
  __threadfence();
  cl.sync();
  // ---- C = D^{-1/2} U^T T D^{-1/2} (rows to the W area, then symmetrised)
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i >= m) continue;
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(__ldcg(Ug + (long long)l * m + i), __ldcg(Tg + (long long)l * m + j), s);
    Wg[(long long)i * m + j] = s * S.dsc[i] * S.dsc[j];
  }
  __threadfence();
  cl.sync();
  double fro2 = 0.0;
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i >= m) continue;
    const double v = (i == j) ? __ldcg(Wg + (long long)i * m + i)
                              : 0.5 * (__ldcg(Wg + (long long)i * m + j) + __ldcg(Wg + (long long)j * m + i));
    Acur[lr * ld + j] = v;
    S.V[lr * m + j] = (i == j) ? 1.0 : 0.0;
    fro2 += v * v;
  }
  // ||C||_F: warp sums, the CTA's sum, then the cluster's in rank order
  for (int o = 16; o > 0; o >>= 1) fro2 += __shfl_down_sync(0xffffffffu, fro2, o);
  if ((tid & 31) == 0) S.aux[tid >> 5] = fro2;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nth / 32; ++w) t += S.aux[w];
    S.red[0] = t;
  }
  cl.sync();
  double fro = 0.0;
  for (int r = 0; r < CL; ++r) fro += cl.map_shared_rank(S.red, r)[0];
  fro = sqrt(fro);
  cl.sync();
  // ---- stage 2
  const int sw2 = jacobi_cluster(cl, L, S, Acur, Anext, 2.0 * 2.220446049250313e-16 * fro, 40);
  if (sw2 < 0) {
    if (tid == 0 && rank == 0) atomicExch(status, (int)DEV_JACOBI);
    return;
  }
  cl_gather_diag(cl, L, Acur, S.dg);   // eigenvalues of C
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i < m) Wg[(long long)i * m + j] = S.V[lr * m + j];
  }
  for (int j = tid; j < m; j += nth) {
    const double ej = S.dg[j];
    int r = 0;
    for (int l = 0; l < m; ++l) r += (S.dg[l] < ej) || (S.dg[l] == ej && l < j);
    S.rk[j] = r;
  }
  __threadfence();
  cl.sync();
  // ---- Phi = U D^{-1/2} W, columns at their ascending rank
  for (int t = tid; t < R * m; t += nth) {
    const int lr = t / m, j = t % m, i = lr * CL + rank;
    if (i >= m) continue;
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(__ldcg(Ug + (long long)i * m + l) * S.dsc[l], __ldcg(Wg + (long long)l * m + j), s);
    Phi[i + (long long)S.rk[j] * m] = s;
  }
  if (rank == 0)
    for (int j = tid; j < m; j += nth) eps[S.rk[j]] = S.dg[j];
}

// ---------------------------------------------------------------- residuals
__global__ void __launch_bounds__(256) k_residual_norms(long long N, const double* __restrict__ AX,
                                                        const double* __restrict__ BX,
                                                        const double* __restrict__ lambda,
                                                        const double* __restrict__ X, double* __restrict__ out) {
  const int j = blockIdx.x;
  const double l = lambda[j];
  const double* ax = AX + (long long)j * N;
  const double* bx = BX + (long long)j * N;
  const double* x = X + (long long)j * N;
  double r = 0.0, xn = 0.0, an = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    r += fabs(ax[i] - l * bx[i]);
    xn += fabs(x[i]);
    an += fabs(ax[i]);
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

__global__ void k_residual_finish(int k, const double* __restrict__ norms, const double* __restrict__ normA,
                                  double* __restrict__ resid, double* __restrict__ resid_paper) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  if (resid) resid[j] = norms[3 * j] / (normA[0] * norms[3 * j + 1]);
  if (resid_paper) resid_paper[j] = norms[3 * j] / norms[3 * j + 2];
}

__global__ void k_permute_columns(long long N, int k, const int* __restrict__ perm, const double* __restrict__ src,
                                  double* __restrict__ dst) {
  const long long total = N * k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % N, j = t / N;
    dst[t] = src[(long long)perm[j] * N + r];
  }
}

}  // namespace

long long gram_partial_elems(long long N, int k1, int k2) {
  return (long long)cdiv(N, kGramRows) * k1 * k2;
}

void gram(cudaStream_t s, long long N, int k1, int k2, const double* X, const double* Y, double* partial,
          double* out, bool symmetric) {
  const int nchunks = cdiv(N, kGramRows);
  const bool sym = symmetric && k1 == k2;
  const int nt = cdiv(k1, kGramTile);
  dim3 grid = sym ? dim3(nt * (nt + 1) / 2, 1, nchunks) : dim3(nt, cdiv(k2, kGramTile), nchunks);
  k_gram_partial<<<grid, 256, 0, s>>>(N, k1, k2, X, Y, partial, sym ? 1 : 0);
  prof::count_launch();
  const int total = k1 * k2;
  k_gram_reduce<<<cdiv(total, 256), 256, 0, s>>>(nchunks, k1, total, partial, out, sym ? 1 : 0);
  prof::count_launch();
}

void dgemm_tall(cudaStream_t s, long long N, int m, int k, const double* Q, const double* P, double* C) {
  dim3 grid(cdiv(N, 64), cdiv(k, 64));
  k_dgemm_tall<<<grid, 256, 0, s>>>(N, m, k, Q, P, C);
  prof::count_launch();
}

// Cluster size for the reduced eigensolve: 16 CTAs where the device can
// co-schedule such a cluster (a non-portable size), else 8; 0 when neither
// launches.
int reduced_eig_cluster_size(int m) {
  static PerDevice<int> probe;   // per device: 16, else 8, else 0
  const int size = probe.get([] {
    int size16 = 0, size8 = 0;
    cudaFuncSetAttribute(k_reduced_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cl_smem_bytes(128, 8));
    cudaFuncSetAttribute(k_reduced_eig_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cl : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(kClThreads);
      cfg.dynamicSmemBytes = cl_smem_bytes(128, cl);
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_reduced_eig_cluster, &cfg) == cudaSuccess && n > 0)
        (cl == 16 ? size16 : size8) = cl;
      cudaGetLastError();
    }
    return size16 ? size16 : size8;
  }, 0);
  if (m < kClMinM) return 0;
  return size;
}

void reduced_eig(cudaStream_t s, int m, const double* AQ, const double* BQ, double* eps, double* Phi,
                 double* work, int* status) {
  if (const int cl = reduced_eig_cluster_size(m)) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = cl_smem_bytes(m, cl);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_reduced_eig_cluster, m, AQ, BQ, eps, Phi, work, status) == cudaSuccess) {
      prof::count_launch();
      return;
    }
    cudaGetLastError();   // fall through to the one-CTA kernel
  }
  const size_t smem = sizeof(double) * ((size_t)m * (m + 1) + 2 * (m / 2 + 2) + 2 * m) +
                      sizeof(int) * (2 * (m / 2 + 2) + 1);
  static PerDevice<cudaError_t> attr;
  attr.get([] { return cudaFuncSetAttribute(k_reduced_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); },
           cudaErrorInvalidDevice);
  k_reduced_eig<<<1, 1024, smem, s>>>(m, AQ, BQ, eps, Phi, work, status);
  prof::count_launch();
}

void residual_norms(cudaStream_t s, long long N, int k, const double* AX, const double* BX,
                    const double* lambda, const double* X, double* out) {
  k_residual_norms<<<k, 256, 0, s>>>(N, AX, BX, lambda, X, out);
  prof::count_launch();
}

void residual_finish(cudaStream_t s, int k, const double* norms, const double* normA, double* resid,
                     double* resid_paper) {
  k_residual_finish<<<cdiv(k, 128), 128, 0, s>>>(k, norms, normA, resid, resid_paper);
  prof::count_launch();
}

void permute_columns(cudaStream_t s, long long N, int k, const int* perm, const double* src, double* dst) {
  long long total = N * k;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_permute_columns<<<blocks, 256, 0, s>>>(N, k, perm, src, dst);
  prof::count_launch();
}

}  // namespace feast

// ---------------------------------------------------------------------------
// Allocation-free variant of the reduced eigensolve (declared in feast.h).
// Its scratch (three M0 x M0 work matrices and the device status word) is
// a file-scope device array that every GPU loading this library holds until
// the process exits; nothing is allocated per call.
#include <mutex>

#include "../../include/feast.h"

namespace {

constexpr int kNoAllocMaxM0 = 128;
constexpr int kNoAllocWork = 3 * kNoAllocMaxM0 * kNoAllocMaxM0;   // doubles of eigensolve work space
constexpr int kNoAllocDoubles = kNoAllocWork + 32;                // + the status word (and padding)

__device__ __align__(256) double g_reduced_eig_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_base[256] = {};   // device address of the array, per device ordinal

}  // namespace

extern "C" feast_status feast_reduced_eig_noalloc(const double* AQ, const double* BQ, int M0, double* eps,
                                                  double* Phi, void* cuda_stream) {
  if (M0 < 1 || M0 > kNoAllocMaxM0 || !AQ || !BQ || !eps || !Phi) return FEAST_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return FEAST_ERR_CUDA;
  }
  double* base = nullptr;
  {
    // set-up, once per device and with that device current: the host-side
    // name of the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_reduced_eig_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return FEAST_ERR_CUDA;
      }
      g_noalloc_base[dev] = static_cast<double*>(p);
    }
    base = g_noalloc_base[dev];
  }
  int* status = reinterpret_cast<int*>(base + kNoAllocWork);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the array keeps the previous call's contents: the status word must start at 0
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return FEAST_ERR_CUDA;
  }
  feast::reduced_eig(s, M0, AQ, BQ, eps, Phi, base, status);
  int st = 0;
  if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return FEAST_ERR_CUDA;
  }
  switch (st) {
    case feast::DEV_OK: return FEAST_OK;
    case feast::DEV_BQ_NOT_SPD: return FEAST_ERR_BQ_NOT_SPD;
    case feast::DEV_JACOBI: return FEAST_ERR_JACOBI;
    default: return FEAST_ERR_CUDA;
  }
}
