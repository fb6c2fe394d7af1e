/*
 * feast.h -- C-ABI of the GB300 FEAST eigensolver library (libfeast_gb300.so).
 *
 * FEAST (Polizzi, arXiv:0901.2665) finds every eigenpair (lambda, x) of the
 * generalized problem A x = lambda B x with lambda inside [lmin, lmax], for
 * real symmetric A and symmetric positive definite B (Sec. III.A, Eq. 2).
 * Each refinement loop (Fig. 2, steps 2-6):
 *   - solves the Ne complex shifted systems (Z_e B - A) Q_e = B Y with M0
 *     right-hand sides at the Gauss-Legendre nodes Z_e of the upper half
 *     circle around the interval (Eqs. 13-14);
 *   - accumulates Q = -sum_e (w_e/2) Re{ r e^{i theta_e} Q_e } (Eq. 15);
 *   - runs Rayleigh-Ritz: A_Q = Q^T A Q, B_Q = Q^T B Q, A_Q Phi = eps B_Q Phi,
 *     X = Q Phi (Eqs. 6-9);
 *   - stops on the relative change of the in-interval trace, else Y = X and
 *     the next right-hand side is B X (Sec. III.B (i)).
 *
 * Operators are 27-point layered stencils (see feast_operator).  The linear
 * systems are block tridiagonal over the z-layers and are solved by an
 * unpivoted block elimination whose diagonal blocks are inverted explicitly;
 * the inverses are computed once per node and reused by every loop
 * (Sec. V, parallelism level (ii)).
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major; N x M0 blocks have leading dimension N.
 *   - Complex arrays are interleaved (re, im) doubles.
 *   - Pointers may be host or device memory unless stated otherwise; the
 *     library inspects each pointer (cudaPointerGetAttributes) and copies host
 *     data through its own device workspace.  Step-level entry points take
 *     DEVICE pointers only.
 *   - The caller owns every buffer it passes; the handle owns its workspace
 *     and releases it in feast_destroy.
 *   - All device work is ordered on the stream given to feast_init.  Entry
 *     points that return host-visible results synchronise that stream.
 *   - Errors are returned as feast_status; no exception crosses the ABI.
 *     feast_last_error() gives a message for the last failing call.
 *   - A handle must not be used by two host threads at once.
 */
#ifndef FEAST_GB300_H
#define FEAST_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct feast_handle feast_handle;

typedef enum {
  FEAST_OK = 0,
  FEAST_ERR_ARG = 1,             /* invalid argument (sizes, interval, pointers) */
  FEAST_ERR_BQ_NOT_SPD = 2,      /* B_Q = Q^T B Q not positive definite: M0 too large
                                    for the interval (Sec. III.B (ii)) */
  FEAST_ERR_NO_CONVERGENCE = 3,  /* trace test not met within max_loops; outputs hold
                                    the last loop's pairs */
  FEAST_ERR_M0_TOO_SMALL = 4,    /* every Ritz value fell inside the interval: Fig. 2
                                    step 1 needs M0 > M; outputs hold the last loop */
  FEAST_ERR_PIVOT = 5,           /* zero or non-finite pivot in a block inversion */
  FEAST_ERR_OOM = 6,             /* device workspace allocation failed */
  FEAST_ERR_CUDA = 7,            /* CUDA runtime error */
  FEAST_ERR_TIMEOUT = 8,         /* a bounded device wait gave up */
  FEAST_ERR_JACOBI = 9,          /* reduced eigensolve did not converge */
  FEAST_ERR_NONFINITE = 10       /* a predicted start block holds a non-finite value */
} feast_status;

/* Precision of the node solves (Fig. 2 step 2).
 * FEAST_PREC_FP64: block factor and solves in FP64.
 * FEAST_PREC_MIXED: block factor and solves on the tensor cores with split
 *   bf16 pair operands (x = bf16(x) + bf16(remainder), 16 significant bits;
 *   fp32 elsewhere), refined in FP64 / double-float until each node's
 *   relative residual meets options.ir_tol; right-hand side, Gram products
 *   and Q*Phi in double-float; reduced eigensolve and final residuals in FP64. */
enum { FEAST_PREC_FP64 = 0, FEAST_PREC_MIXED = 1 };

/*
 * Layered 27-point operator on an nx x ny x nz interior grid.
 * Node id i = ix + nx*(iy + ny*iz); layer iz holds the n = nx*ny unknowns
 * [iz*n, (iz+1)*n).  A27 and B27 are [27][N] arrays of row-wise stencil
 * coefficients: slot s = (dz+1)*9 + (dy+1)*3 + (dx+1) couples row i to column
 * i + dx + nx*(dy + ny*dz) and must be 0 where that neighbour is outside the
 * grid.  A must be symmetric and B symmetric positive definite (Eq. 2); the
 * library relies on the symmetry and does not check it.
 */
typedef struct {
  int nx, ny, nz;
  const double* A27;
  const double* B27;
} feast_operator;

typedef struct {
  int max_loops;      /* refinement loop cap (default 20) */
  int precision;      /* FEAST_PREC_FP64 (default) or FEAST_PREC_MIXED */
  double ir_tol;      /* MIXED: relative residual target of each node solve (1e-12) */
  int ir_max;         /* MIXED: cap on refinement steps per node solve (default 30) */
  uint64_t seed;      /* start block when Y0 == NULL: Y(row, col) = uniform [-1, 1)
                         from SplitMix64 output col*N + row of this seed */
  int profile;        /* 1: time the main kernel classes with CUDA events (feast_info.kernel_ms) */
  int ir_early;       /* MIXED, random start (Y0 == NULL) only: 1 (default) loosens the refinement
                         target of loop 1 to 1e-4 and of loop 2 to 1e-8 (never below ir_tol); a
                         loop with a loosened target never ends the iteration.  0, or a given
                         start block: ir_tol in every loop. */
  int inner_solver;   /* FEAST_INNER_DIRECT (default): the node systems are factorised once and
                         solved by block elimination (precision selects FP64 or mixed).
                         FEAST_INNER_COCG: no factorisation; every node system is solved by the
                         Jacobi-preconditioned conjugate orthogonal CG method (FP64) to the
                         relative residual inner_tol per column -- the inexact iterative inner
                         solves of Sec. IV.C; precision and the ir_* options are then unused. */
  double inner_tol;   /* COCG: relative residual ||r||_2 / ||b||_2 of each column (default 1e-3) */
  int inner_max_iter; /* COCG: iteration cap (default 5000); reaching it fails the solve (FEAST_ERR_NO_CONVERGENCE) */
} feast_options;

enum { FEAST_INNER_DIRECT = 0, FEAST_INNER_COCG = 1 };

/* Per-solve diagnostics, valid after feast_solve (also after a failing one). */
#define FEAST_KERNEL_CLASSES 12

typedef struct {
  int loops;
  int m_found;
  double trace[64];         /* in-interval trace after each loop (first 64 loops) */
  double rel_change[64];    /* relative trace change; rel_change[0] = -1 */
  double resid_max;         /* max over in-interval pairs, ||Ax-lBx||_1/(||A||_1 ||x||_1) */
  double resid_paper_max;   /* max over in-interval pairs, ||Ax-lBx||_1/||Ax||_1 (Table I) */
  double t_factor_ms;       /* device time of the node factorisations */
  double t_solve_ms;        /* device time of all node solves (incl. refinement) */
  double t_rr_ms;           /* device time of Rayleigh-Ritz (Gram, eigensolve, X = Q Phi) */
  double t_total_ms;        /* wall time of the call */
  int ir_steps_max;         /* MIXED: most refinement steps taken by one node solve */
  double ir_resid_max;      /* MIXED: worst final relative residual of a node solve run to ir_tol */
  long long factor_flops;   /* algorithmic flops of the factorisation (8 n^3 per layer per node) */
  /* kernel accounting of the call: launches of the library's kernels, and
     with options.profile the summed device time and launch count per class:
     0 sweep-update GEMM (wide), 1 block-solve GEMM, 2 panel inversion,
     3 panel product/packing, 4 Schur complements, 5 solve couplings (work
     in bytes), 6 FP64 refinement residual, 7 FP64-path factor/solve kernels,
     8 incremental double-float refinement residual, 9 sweep-update GEMM on
     the next panel's column tile (narrow); the rest are zero */
  long long gpu_launches;
  double kernel_ms[FEAST_KERNEL_CLASSES];
  long long kernel_launches[FEAST_KERNEL_CLASSES];
  double kernel_flops[FEAST_KERNEL_CLASSES];   /* algorithmic flops of each class (complex FMA = 8 real flops;
                               a split-pair tensor-core product counts once) */
  long long sweep_graphs;   /* MIXED: forward/backward sweep pairs replayed from captured CUDA graphs
                               (0 with options.profile, which times the kernels one by one) */
  int inner_iters_max;      /* COCG: most iterations of one loop's node solves */
  double inner_rel_max;     /* COCG: largest final relative residual of a column */
  int loop_graphs;          /* 1: the refinement loops ran as one CUDA graph with device-side loop
                               conditions (see feast_solve); t_rr_ms is then -1 and t_solve_ms
                               covers the whole loop */
} feast_info;

/* Fills *opt with the defaults listed above. */
void feast_default_options(feast_options* opt);

/*
 * Creates a handle bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  opt may be NULL for
 * the defaults.  Errors: FEAST_ERR_ARG, FEAST_ERR_CUDA.
 */
feast_status feast_init(feast_handle** h, const feast_options* opt, void* cuda_stream);

/* Releases the handle and every device buffer it owns.  NULL is a no-op. */
feast_status feast_destroy(feast_handle* h);

/* Message of the last failing call on h ("" if none); valid until the next call. */
const char* feast_last_error(const feast_handle* h);

/* Copies the diagnostics of the last feast_solve into *info. */
feast_status feast_get_info(const feast_handle* h, feast_info* info);

/*
 * The eigensolver (Fig. 2).  Finds the eigenpairs of (op->A27, op->B27) in the
 * closed interval [lmin, lmax] with a subspace of M0 columns and Ne contour
 * nodes; stops when the in-interval count is unchanged and the relative trace
 * change is <= tol (loop 1 never stops).
 *   Y0      : N x M0 start block, or NULL for the seeded random block
 *             (a previous X gives a warm start: the right-hand side is B*Y0).
 *   lambda  : out, M0 Ritz values, ascending, the m_found in-interval values first.
 *   X       : out, N x M0 Ritz vectors (B-orthonormal), columns aligned with lambda.
 *   resid   : out (may be NULL), M0 residuals ||A x - l B x||_1 / (||A||_1 ||x||_1).
 *   m_found : out, number of Ritz values inside [lmin, lmax].
 *   loops   : out, refinement loops run.
 * Requirements: nx, ny, nz >= 1; 1 <= M0 <= min(N, 128); 1 <= Ne <= 64; lmin < lmax.
 * Returns FEAST_OK, or one of the codes above; on FEAST_ERR_NO_CONVERGENCE and
 * FEAST_ERR_M0_TOO_SMALL the outputs are filled.  Synchronises the stream.
 * Repeated work (MIXED precision, options.profile off): a factorisation, or a
 * pair of solve sweeps, whose shape, operator pointers and work buffers were
 * seen before on this handle is recorded once as a CUDA graph and replayed
 * into the stream on later uses (the results are the same bit for bit).  The
 * graphs hold pointers, not data: new contents at the same addresses are
 * read at replay; they are released by feast_destroy.
 */
feast_status feast_solve(feast_handle* h, const feast_operator* op, double lmin, double lmax,
                         int M0, int Ne, double tol, const double* Y0,
                         double* lambda, double* X, double* resid, int* m_found, int* loops);

/*
 * The eigensolver for a complex Hermitian A (Sec. III.A: A real symmetric or
 * Hermitian; Sec. III.B, Eqs. 10 and 12), FP64.  op->A27 and op->B27 hold
 * complex coefficients ([27][N] complex, interleaved (re, im) doubles, the
 * same slot layout as feast_operator); A must be Hermitian and B Hermitian
 * positive definite (a real B is passed with zero imaginary parts).  Step 2
 * solves at the 2 Ne shifts Z_e and conj Z_e (G(conj Z) = G(Z)^dagger) and
 * accumulates Eq. 12:
 *   Q = -sum_e (w_e r / 4) (e^{i theta_e} G(Z_e) + e^{-i theta_e} G(conj Z_e)) B Y;
 * Rayleigh-Ritz uses A_Q = Q^H A Q, B_Q = Q^H B Q and a Hermitian-definite
 * reduced eigensolve, X = Q Phi with X^H B X = I.
 *   Y0, X   : N x M0 complex (interleaved), DEVICE; Y0 may be NULL for the
 *             seeded block Y(row, col) = u(seed, col N + row) + i u(seed + 1, col N + row)
 *             (u as for feast_solve).
 *   lambda, resid, m_found, loops: as in feast_solve (host or device).
 * Requirements: 1 <= M0 <= min(N, 64); 1 <= Ne <= 32; nx*ny <= 4096; the
 * operator arrays on the device.  Returns as feast_solve does; synchronises.
 */
feast_status feast_solve_hermitian(feast_handle* h, const feast_operator* op, double lmin, double lmax, int M0,
                                   int Ne, double tol, const double* Y0, double* lambda, double* X, double* resid,
                                   int* m_found, int* loops);

/*
 * Many independent problems (Sec. V, parallelism level (i): independent
 * search intervals or instances) solved concurrently on the handle's GPU.
 * Instance i has operator ops[i], interval [lmin[i], lmax[i]] and subspace
 * M0[i]; Y0 (may be NULL, or hold NULL entries) gives start blocks; lambda[i],
 * X[i], resid[i] (resid may be NULL) receive the outputs exactly as in
 * feast_solve, as do m_found[i] and loops[i]; statuses[i] receives the
 * instance's feast_status.  Host or device pointers as in feast_solve.
 * Worker threads, each with its own stream and workspace, take the instances
 * largest first; `workers` bounds their number (0 = as many as the device
 * memory allows, at most 8).  Returns FEAST_OK when every instance
 * succeeded, else the status of the first failing instance; the handle's
 * feast_info.gpu_launches then counts every worker's kernel launches.
 * Synchronises.
 */
feast_status feast_solve_batched(feast_handle* h, int count, const feast_operator* ops, const double* lmin,
                                 const double* lmax, const int* M0, int Ne, double tol, const double* const* Y0,
                                 double* const* lambda, double* const* X, double* const* resid, int* m_found,
                                 int* loops, feast_status* statuses, int workers);

/* ---------------------------------------------------------------------------
 * Step-level entry points (DEVICE pointers only; ordered on the handle's
 * stream; they do not synchronise unless stated).
 * ------------------------------------------------------------------------- */

/*
 * Gauss-Legendre nodes and the contour (Fig. 2 caption; Eqs. 13-14), on the
 * host: x[e], w[e] (ordered as the paper's Ne = 8 table: x_1 > 0,
 * x_2 = -x_1, ...), theta[e] = -(pi/2)(x_e - 1), Z_e = (lmax+lmin)/2 + r e^{i theta_e}
 * returned as Zre/Zim.  Any output pointer may be NULL.  Host memory.
 */
feast_status feast_contour(double lmin, double lmax, int Ne, double* x, double* w,
                           double* theta, double* Zre, double* Zim);

/*
 * Y = C X for the 27-point operator C (a [27][N] coefficient array, device)
 * on the nx x ny x nz grid; X and Y are N x k column-major device arrays.
 * Used for A Q, B Q and B Y (Fig. 2 steps 2, 3, 6).
 */
feast_status feast_stencil_apply(feast_handle* h, int nx, int ny, int nz, const double* C27,
                                 const double* X, double* Y, int k);

/*
 * Node solve (Fig. 2 step 2): Qe = (Z B - A)^{-1} RHS for one complex shift
 * Z = Zre + i Zim with Zim > 0.  RHS: N x k real, Qe: N x k complex
 * (interleaved), device.  precision selects the FP64 or the mixed
 * (complex64 tensor-core factors + FP64 refinement) path.  Synchronises.
 */
feast_status feast_node_solve(feast_handle* h, const feast_operator* op, double Zre, double Zim,
                              const double* RHS, double* Qe, int k, int precision);

/*
 * Step 2 in full: Q = -sum_e (w_e/2) Re{ r e^{i theta_e} (Z_e B - A)^{-1} RHS }
 * (Eq. 15) for the Ne nodes of [lmin, lmax].  RHS, Q: N x k real, device.
 * Synchronises.
 */
feast_status feast_quadrature(feast_handle* h, const feast_operator* op, double lmin, double lmax,
                              int Ne, const double* RHS, double* Q, int k, int precision);

/*
 * Reduced eigensolve (Fig. 2 step 4; Eqs. 6, 8): A_Q Phi = eps B_Q Phi for
 * symmetric M0 x M0 A_Q and s.p.d. B_Q (column-major, device), M0 <= 128.
 * eps ascending (device, M0), Phi B_Q-orthonormal (device, M0 x M0).
 * Returns FEAST_ERR_BQ_NOT_SPD when B_Q's eigenvalue ratio is <= 1e-14.
 * Synchronises.
 */
feast_status feast_reduced_eig(feast_handle* h, const double* AQ, const double* BQ, int M0,
                               double* eps, double* Phi);

/*
 * Rayleigh-Ritz (Fig. 2 steps 3-5; Eqs. 6-9): from Q (N x M0, device) forms
 * A_Q, B_Q, solves the reduced problem and writes eps (M0, ascending) and
 * X = Q Phi (N x M0), device.  AQ/BQ (M0 x M0, device) receive the reduced
 * matrices when non-NULL.  Synchronises.
 */
feast_status feast_rayleigh_ritz(feast_handle* h, const feast_operator* op, const double* Q, int M0,
                                 double* eps, double* X, double* AQ, double* BQ);

/*
 * Residuals (Table I caption): per column m of X (N x k, device),
 * resid[m] = ||A x_m - l_m B x_m||_1 / (||A||_1 ||x_m||_1) and
 * resid_paper[m] = ||A x_m - l_m B x_m||_1 / ||A x_m||_1 (device, k each;
 * either may be NULL).  Synchronises.
 */
feast_status feast_residuals(feast_handle* h, const feast_operator* op, const double* lambda,
                             const double* X, int k, double* resid, double* resid_paper);

/* ---------------------------------------------------------------------------
 * Learned initial subspace.  The paper's refinement (Sec. III.B (i)) and its
 * warm starts over a sequence of close problems (Sec. IV.C, Fig. 3) show that
 * a good start block Y shortens the loop; here a small network predicts Y.
 * An MLP maps the features of one z-layer of an instance (in_dim <= 64
 * scalars) through three hidden layers of `width` (a multiple of 128, SiLU)
 * to out_dim = M0 * px * py coefficients: layer l's block of Y is
 *   Y[l n + ix + nx iy, c] = sum_{q<py, p<px} coef[l, c, q px + p] s_p(ix) s_q(iy),
 *   s_p(i) = sqrt(2/(m+1)) sin((p+1) pi (i+1)/(m+1)) on an axis of m nodes
 * (0-based p).  Products run on the tensor cores in BF16 with FP32
 * accumulation; parameters are FP32 and trained with Adam.  Buffers are
 * DEVICE pointers unless stated; calls are ordered on the network's stream
 * and synchronise it.
 * ------------------------------------------------------------------------- */
typedef struct feast_mlp feast_mlp;

/* Allocates a network for batches of up to max_batch rows (FEAST_ERR_ARG on
   bad sizes, FEAST_ERR_OOM).  Parameters start at zero: set them with
   feast_mlp_set_layer. */
feast_status feast_mlp_create(feast_mlp** net, int in_dim, int width, int out_dim, int max_batch, void* cuda_stream);
feast_status feast_mlp_destroy(feast_mlp* net);
/* Layer k (0..3): W (out x in, row-major, fp32) and b (out), host or device;
   resets the optimiser state. */
feast_status feast_mlp_set_layer(feast_mlp* net, int k, const float* W, const float* b);
/* Copies layer k's parameters and last gradients out (any pointer may be NULL). */
feast_status feast_mlp_get_layer(feast_mlp* net, int k, float* W, float* b, float* gW, float* gb);
/* out (B x out_dim) = network(X (B x in_dim)), row-major fp32. */
feast_status feast_mlp_forward(feast_mlp* net, const float* X, int B, float* out);
/* Loss L = sum_{r,o} weights[o] (out[r,o] - target[r,o])^2 / (2 B) of B rows,
   its gradients (kept in the network, see feast_mlp_get_layer) and, when
   lr > 0, one Adam step (beta 0.9 / 0.999, eps 1e-8).  *loss may be NULL. */
feast_status feast_mlp_train_step(feast_mlp* net, const float* X, const float* target, const float* weights, int B,
                                  float lr, double* loss);
/* Y (N x M0, column-major fp64) from coef (nz x M0 x px*py fp32), formula above. */
feast_status feast_sine_expand(const float* coef, int nx, int ny, int nz, int M0, int px, int py, double* Y,
                               void* cuda_stream);
/* The adjoint: coef[l, c, q px + p] = sum_{ix, iy} X[l n + ix + nx iy, c] s_p(ix) s_q(iy). */
feast_status feast_sine_project(const double* X, int nx, int ny, int nz, int M0, int px, int py, float* coef,
                                void* cuda_stream);
/* Y = expansion of the network's output for the nz layer features (nz x in_dim).
   FEAST_ERR_NONFINITE (Y untouched) if an output coefficient is not finite:
   the caller then starts from a random block instead. */
feast_status feast_predict_Y(feast_mlp* net, const float* features, int nx, int ny, int nz, int M0, int px, int py,
                             double* Y);

/*
 * Self-test of the bounded device waits.  Every spin-wait in the library's
 * pipelined kernels (mbarrier waits of the TMA/tcgen05 GEMMs) gives up after
 * a fixed number of polls, records a timeout in the handle's status word,
 * releases what it holds and returns, so that the CUDA context stays usable.
 * This call runs that give-up path on purpose: one thread waits, through the
 * same bounded-wait helper, on an mbarrier that nothing completes, with a
 * limit of `polls` polls (1 <= polls <= 2^26), on the handle's stream.
 *
 * Returns FEAST_ERR_TIMEOUT when the wait ran out and the kernel returned
 * (the expected outcome), FEAST_ERR_ARG for polls out of range (nothing is
 * launched), FEAST_ERR_CUDA on a launch error.  The handle stays usable.
 */
feast_status feast_selftest_wait_timeout(feast_handle* h, long long polls);

/*
 * Allocation-free reduced eigensolve.  The paper has no counterpart: this is
 * a library convenience.  It computes exactly what feast_reduced_eig computes
 * (same kernel), for callers that cannot call cudaMalloc: code that must keep
 * every device byte under its own allocator or a budget fixed at start-up
 * (a framework memory pool, a co-scheduled process with a hard memory cap),
 * and paths where an allocation's implicit synchronisation or its failure in
 * the middle of work is not acceptable.  It needs no handle.
 *
 * AQ, BQ (M0 x M0, column-major), eps (M0) and Phi (M0 x M0) are DEVICE
 * pointers owned by the caller; 1 <= M0 <= 128.  The work space (3 * 128 * 128
 * doubles plus a status word, about 385 KB) is a fixed device array inside the
 * library that every GPU which loads the library holds until the process
 * exits.  Nothing is allocated or freed per call.
 *
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress) and caches it.  Work is ordered on cuda_stream (NULL = legacy
 * default stream) and the call synchronises that stream to read the status.
 * Every call shares the one array, which keeps the last call's contents (the
 * status word is cleared at the start of each call): calls whose work overlaps
 * on the GPU, from two streams or two host threads, race on it.
 *
 * Returns FEAST_ERR_ARG for M0 outside [1, 128] or a NULL pointer (nothing is
 * launched), FEAST_ERR_BQ_NOT_SPD, FEAST_ERR_JACOBI or FEAST_ERR_CUDA as
 * feast_reduced_eig does, else FEAST_OK.
 */
feast_status feast_reduced_eig_noalloc(const double* AQ, const double* BQ, int M0, double* eps, double* Phi,
                                       void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FEAST_GB300_H */
