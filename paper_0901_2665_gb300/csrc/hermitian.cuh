// FEAST for complex Hermitian A (Eq. 12), FP64: internal interface.
#pragma once

#include "common.cuh"

namespace feast {

// A Hermitian 27-point operator: A27, B27 complex [27][N] (device), B
// Hermitian positive definite.
struct HermOp {
  Grid g;
  const cplx* A27;
  const cplx* B27;
};

// Bytes of the factor work space for `nodes` shifts.
size_t herm_factor_bytes(Grid g, int nodes);
// Block elimination of (Z_e B - A) for every shift e (grid z = shift): the
// swept complements S'_i = -S_i^{-1} land at the start of `work`.
void herm_factor(cudaStream_t s, const HermOp& o, int nodes, const cplx* Z, cplx* work, int* status);
// G_e = (Z_e B - A)^{-1} RHS with the factors in `work`; RHS N x k complex,
// G nodes x (N x k), Tmp nodes x (n x k) scratch.
void herm_solve(cudaStream_t s, const HermOp& o, int nodes, const cplx* Z, const cplx* work, const cplx* RHS, cplx* G,
                cplx* Tmp, int k);
// Q = sum_e coef_e G_e, nodes in order (Eq. 12 with complex coefficients).
void herm_quadrature(cudaStream_t s, long long N, int k, int nodes, const cplx* coef, const cplx* G, cplx* Q);
// Y = C X for a complex 27-point operator; X, Y complex N x k.
void herm_stencil(cudaStream_t s, Grid g, const cplx* C27, const cplx* X, cplx* Y, int k);
// out (k x k, col-major) = X^H Y; partial: herm_gram_elems(N, k) complex scratch.
long long herm_gram_elems(long long N, int k);
void herm_gram(cudaStream_t s, long long N, int k, const cplx* X, const cplx* Y, cplx* partial, cplx* out);
// Hermitian-definite reduced eigensolve, m <= 64; work: 3 m^2 complex.
void herm_reduced_eig(cudaStream_t s, int m, const cplx* AQ, const cplx* BQ, double* eps, cplx* Phi, cplx* work,
                      int* status);
// C (N x k) = Q (N x m) P (m x k), complex.
void herm_gemm_tall(cudaStream_t s, long long N, int m, int k, const cplx* Q, const cplx* P, cplx* C);
// Both residual forms of the Table I caption for complex eigenvectors.
void herm_residuals(cudaStream_t s, Grid g, const cplx* A27, const cplx* B27, const double* lam, const cplx* X, int k,
                    cplx* AX, cplx* BX, double* norms, double* normA, double* resid, double* resid_paper);
void herm_permute(cudaStream_t s, long long N, int k, const int* perm, const cplx* src, cplx* dst);
// Y(row, col) = u(seed, col N + row) + i u(seed + 1, col N + row), u the SplitMix64 uniform of random_block.
void herm_random(cudaStream_t s, long long N, int k, uint64_t seed, cplx* Y);

}  // namespace feast
