// Host-side launchers of the FEAST device kernels (internal interface).
#pragma once

#include "common.cuh"

namespace feast {

// ---------------------------------------------------------------- stencil.cu
// Y = C X for a 27-point coefficient array C27 ([27][N]); X, Y: N x k, col-major.
void stencil_apply(cudaStream_t s, Grid g, const double* C27, const double* X, long long ldx,
                   double* Y, long long ldy, int k);
// Splitmix64 uniform [-1,1) start block, Y(row, col) = u(seed, col*N + row).
void random_block(cudaStream_t s, long long N, int k, uint64_t seed, double* Y);
// ||A||_1 of a symmetric 27-point operator = max_i sum_s |A27[s][i]| -> *out (device).
void stencil_norm1(cudaStream_t s, Grid g, const double* A27, double* out);

// Node-batched couplings between neighbouring z-layers of M_e = Z_e B - A.
// G: Ne arrays of N x k complex (col-major, ld N, node stride sG); Tmp: Ne arrays
// of n x k complex (ld n, node stride sT); Z: Ne complex shifts (device).
// forward:  G_e[layer i] = RHS[layer i] + C_i Tmp_e       (C_i = M[i, i-1])
void couple_forward(cudaStream_t s, Grid g, int layer, int Ne, const cplx* Z, const double* A27,
                    const double* B27, const double* RHS, const cplx* Tmp, long long sT, cplx* G,
                    long long sG, int k);
// backward: Tmp_e = G_e[layer i] - U_i G_e[layer i+1]    (U_i = M[i, i+1])
void couple_backward(cudaStream_t s, Grid g, int layer, int Ne, const cplx* Z, const double* A27,
                     const double* B27, const cplx* G, long long sG, cplx* Tmp, long long sT, int k);
// Q = sum_e Qp_e in node order e = 1..Ne (Eq. 15): Qp holds the node shares
// Re{coef_e Q_e}, coef_e = -(w_e/2) r e^{i theta_e}, written by the backward
// sweeps (node stride sQ); Q: N x k.
void quadrature_sum(cudaStream_t s, long long N, int k, int Ne, const double* Qp, long long sQ, double* Q);
// Copy a real RHS into complex G (imaginary part 0) for rows [0, n) of every node.
void rhs_to_complex(cudaStream_t s, long long rows, int k, int Ne, const double* RHS, long long ldr,
                    cplx* G, long long ldg, long long sG);

// ---------------------------------------------------------------- blocktri64.cu
// FP64 factorisation of every node's block-tridiagonal M_e: for each layer i the
// swept Schur complement S'_i = -(S_i)^{-1} is stored at F + (e*nb + i)*n*n.
struct Fp64Work {
  cplx* F;       // Ne*nb*n*n
  cplx* T1;      // Ne*n*n scratch
  cplx* T;       // Ne*n*bmax panel scratch
  cplx* L;       // Ne*n*bmax
  cplx* Pinv;    // Ne*bmax*bmax
  int* status;   // device status word
};
void factor_fp64(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                 const Fp64Work& w);
// C_e = alpha * S_e X_e for symmetric n x n S (row-major), X, C: n x k complex col-major.
// qp (nullable): qp_e[m*ldq + p] = Re{coef_e C_e[p, m]} (node stride sQ).
void zgemm_sym(cudaStream_t s, int n, int k, int Ne, double alpha, const cplx* S, long long sS,
               const cplx* X, long long ldx, long long sX, cplx* C, long long ldc, long long sC,
               double* qp = nullptr, long long sQ = 0, long long ldq = 0, const cplx* coef = nullptr);
// Solve M_e G_e = RHS for all nodes with the FP64 factors; G: Ne x (N x k complex).
// Qp (nullable): the node shares Re{coef_e G_e} of Eq. 15 (Ne x N x k real),
// written by the backward sweep's products.
void solve_fp64(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                const cplx* F, const double* RHS, cplx* G, cplx* Tmp, int k, double* Qp = nullptr,
                const cplx* coef = nullptr);

// ---------------------------------------------------------------- rr.cu
// out (k1 x k2, col-major, ld k1) = X^T Y, X: N x k1, Y: N x k2 (col-major, ld N).
// partial: scratch of gram_partial_elems(N, k1, k2) doubles.  Deterministic.
long long gram_partial_elems(long long N, int k1, int k2);
// symmetric: X^T Y is symmetric (Y = C X with C symmetric, k1 == k2); only
// the tiles on and above the diagonal are computed and the rest mirrored.
void gram(cudaStream_t s, long long N, int k1, int k2, const double* X, const double* Y, double* partial,
          double* out, bool symmetric = false);
// C (N x k, ld N) = Q (N x m, ld N) * P (m x k, ld m).
void dgemm_tall(cudaStream_t s, long long N, int m, int k, const double* Q, const double* P, double* C);

// ---------------------------------------------------------------- rr_df.cu
// Double-float (hi + lo fp32 pairs) versions of the FP64 products above, for
// the mixed path (the FP64 pipe is 1/64 of the FP32 rate on this GPU).
// Y (N x k double-float) = split of X (FP64), element by element.
void split_df(cudaStream_t s, long long total, const double* X, float2* Y);
// Y = C X, C a 27-point FP64 operator, X double-float; Y double-float or FP64.
void stencil_apply_df(cudaStream_t s, Grid g, const double* C27, const float2* X, long long ldx, float2* Y,
                      long long ldy, int k);
void stencil_apply_df(cudaStream_t s, Grid g, const double* C27, const float2* X, long long ldx, double* Y,
                      long long ldy, int k);
// out (k1 x k2, FP64) = X^T Y for double-float X, Y; partial: scratch of
// gram_partial_elems_df(N, k1, k2) doubles.  Deterministic.
long long gram_partial_elems_df(long long N, int k1, int k2);
void gram_df(cudaStream_t s, long long N, int k1, int k2, const float2* X, const float2* Y, double* partial,
             double* out, bool symmetric = false);
// C (N x k, FP64) = Q (N x m, double-float) * P (m x k, FP64).
void gemm_tall_df(cudaStream_t s, long long N, int m, int k, const float2* Q, const double* P, double* C);

// Reduced generalized eigensolve A_Q Phi = eps B_Q Phi (two-stage Jacobi), m <= 128.
// work: 3*m*m doubles scratch.  Status word gets DEV_BQ_NOT_SPD / DEV_JACOBI.
void reduced_eig(cudaStream_t s, int m, const double* AQ, const double* BQ, double* eps, double* Phi,
                 double* work, int* status);
// Column norms for the residuals (Table I): for each column j of X,
// out[3j+0] = ||AX_j - l_j BX_j||_1, out[3j+1] = ||X_j||_1, out[3j+2] = ||AX_j||_1.
void residual_norms(cudaStream_t s, long long N, int k, const double* AX, const double* BX,
                    const double* lambda, const double* X, double* out);
// resid[j] = out[3j]/(normA*out[3j+1]); resid_paper[j] = out[3j]/out[3j+2] (device).
void residual_finish(cudaStream_t s, int k, const double* norms, const double* normA, double* resid,
                     double* resid_paper);
// Permute columns: dst[:, j] = src[:, perm[j]] (perm on device), N x k.
void permute_columns(cudaStream_t s, long long N, int k, const int* perm, const double* src, double* dst);

}  // namespace feast
