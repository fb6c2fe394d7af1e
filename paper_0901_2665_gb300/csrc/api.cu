// C-ABI of the FEAST GB300 library: handle, workspace and the refinement loop
// of Fig. 2 (Polizzi, arXiv:0901.2665).  All arithmetic runs in the device
// kernels; the host computes only the quadrature nodes, the in-interval count
// and the trace test on M0 scalars per loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/feast.h"
#include "hermitian.cuh"
#include "iterative.cuh"
#include "kernels.cuh"
#include "mixed.cuh"
#include "prof.cuh"

using namespace feast;

namespace {

struct FeastError {
  feast_status code;
  std::string msg;
};

[[noreturn]] void fail(feast_status code, const std::string& msg) { throw FeastError{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? FEAST_ERR_OOM : FEAST_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void ensure(size_t need, const char* name) {
    if (need <= bytes) return;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (need == 0) return;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      fail(FEAST_ERR_OOM, std::string("cudaMalloc(") + name + ", " + std::to_string(need) + " B) failed");
    }
    bytes = need;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Gauss-Legendre nodes by Newton iteration on P_Ne; ordered like the paper's
// Ne = 8 table (Fig. 2 caption): x_1 > 0 smallest positive, x_2 = -x_1, ...
void gauss_legendre(int Ne, std::vector<double>& x, std::vector<double>& w) {
  auto legendre = [Ne](double t, double& p, double& dp) {
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < Ne; ++k) {
      double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    p = (Ne == 0) ? 1.0 : p1;
    dp = Ne * (t * p1 - p0) / (t * t - 1.0);
  };
  std::vector<std::pair<double, double>> pos;
  for (int i = 1; i <= Ne / 2; ++i) {
    double t = std::cos(M_PI * (i - 0.25) / (Ne + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(t, p, dp);
      double d = p / dp;
      t -= d;
      if (std::fabs(d) < 1e-17) break;
    }
    double p, dp;
    legendre(t, p, dp);
    pos.push_back({t, 2.0 / ((1.0 - t * t) * dp * dp)});
  }
  std::sort(pos.begin(), pos.end());
  x.clear();
  w.clear();
  if (Ne % 2 == 1) {
    double p, dp;
    legendre(0.0, p, dp);
    x.push_back(0.0);
    w.push_back(2.0 / (dp * dp));
  }
  for (auto& q : pos) {
    x.push_back(q.first);
    w.push_back(q.second);
    x.push_back(-q.first);
    w.push_back(q.second);
  }
}

struct Contour {
  std::vector<double> x, w, theta;
  std::vector<cplx> Z, coef;  // coef_e = -(w_e/2) r e^{i theta_e}
  double r = 0, c = 0;
};

Contour make_contour(double lmin, double lmax, int Ne) {
  Contour ct;
  gauss_legendre(Ne, ct.x, ct.w);
  ct.r = (lmax - lmin) / 2.0;
  ct.c = (lmax + lmin) / 2.0;
  for (int e = 0; e < Ne; ++e) {
    double th = -(M_PI / 2.0) * (ct.x[e] - 1.0);
    ct.theta.push_back(th);
    ct.Z.push_back(cplx{ct.c + ct.r * std::cos(th), ct.r * std::sin(th)});
    ct.coef.push_back(cplx{-(ct.w[e] / 2.0) * ct.r * std::cos(th), -(ct.w[e] / 2.0) * ct.r * std::sin(th)});
  }
  return ct;
}

}  // namespace

struct feast_handle {
  cudaStream_t stream = nullptr;
  feast_options opt{};
  std::string err;
  feast_info info{};
  int device = 0;
  // operator copies (when the caller passes host arrays)
  DevBuf opA, opB;
  // factor and node buffers
  DevBuf F, T1, T, L, Pinv, G, Tmp, Zd, coefd, status, cgw;
  // loop buffers
  DevBuf RHS, Q, Qp, AQf, BQf, Xb, Yb, Xout, part, AQ, BQ, eps, Phi, work, norms, normA, lam_d, perm_d, resid_d,
      residp_d, loopst;
  DevBuf Qdf;   // double-float copy of Q (or of Y) for the mixed path's products
  long long loop_graph_solves = 0;   // solves whose loop ran as one CUDA graph
  MixedWork mixed;
  // Hermitian path (complex buffers)
  DevBuf hF, hG, hTmp, hRHS, hQ, hAQf, hBQf, hX, hY, hXout, hPart, hAQ, hBQ, hPhi, hWork, hZ, hCoef, hEps;
  cudaEvent_t ev[8] = {};

  void release_all() {
    for (DevBuf* b : {&opA, &opB, &F, &T1, &T, &L, &Pinv, &G, &Tmp, &Zd, &coefd, &status, &cgw, &RHS, &Q, &Qp, &AQf,
                      &BQf,
                      &Xb, &Yb, &Xout, &part, &AQ, &BQ, &eps, &Phi, &work, &norms, &normA, &lam_d, &perm_d,
                      &resid_d, &residp_d, &loopst, &Qdf, &hF, &hG, &hTmp, &hRHS, &hQ, &hAQf, &hBQf, &hX, &hY, &hXout, &hPart, &hAQ,
                      &hBQ, &hPhi, &hWork, &hZ, &hCoef, &hEps})
      b->release();
    mixed.release();
  }
};

namespace {

template <class F>
feast_status guarded(feast_handle* h, F&& body) {
  try {
    body();
    if (h) h->err.clear();
    return FEAST_OK;
  } catch (const FeastError& e) {
    if (h) h->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    return FEAST_ERR_CUDA;
  }
}

struct OpView {
  Grid g;
  const double* A27;
  const double* B27;
};

OpView device_operator(feast_handle* h, const feast_operator* op) {
  if (!op) fail(FEAST_ERR_ARG, "operator is NULL");
  if (op->nx < 1 || op->ny < 1 || op->nz < 1) fail(FEAST_ERR_ARG, "grid sizes must be >= 1");
  if (!op->A27 || !op->B27) fail(FEAST_ERR_ARG, "A27/B27 NULL");
  Grid g{op->nx, op->ny, op->nz};
  if ((long long)g.n() > 8192) fail(FEAST_ERR_ARG, "layer size nx*ny must be <= 8192");
  const size_t bytes = sizeof(double) * 27 * (size_t)g.N();
  OpView v{g, op->A27, op->B27};
  if (!is_device_ptr(op->A27)) {
    h->opA.ensure(bytes, "A27");
    ck(cudaMemcpyAsync(h->opA.p, op->A27, bytes, cudaMemcpyHostToDevice, h->stream), "copy A27");
    v.A27 = h->opA.as<double>();
  }
  if (!is_device_ptr(op->B27)) {
    h->opB.ensure(bytes, "B27");
    ck(cudaMemcpyAsync(h->opB.p, op->B27, bytes, cudaMemcpyHostToDevice, h->stream), "copy B27");
    v.B27 = h->opB.as<double>();
  }
  return v;
}

void check_status(feast_handle* h) {
  int st = 0;
  ck(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status");
  ck(cudaStreamSynchronize(h->stream), "sync");
  ck(cudaGetLastError(), "kernel launch");
  switch (st) {
    case DEV_OK: return;
    case DEV_PIVOT: fail(FEAST_ERR_PIVOT, "zero or non-finite pivot in a block inversion");
    case DEV_JACOBI: fail(FEAST_ERR_JACOBI, "Jacobi sweeps did not converge");
    case DEV_BQ_NOT_SPD: fail(FEAST_ERR_BQ_NOT_SPD, "B_Q is not positive definite (M0 too large)");
    case DEV_TIMEOUT: fail(FEAST_ERR_TIMEOUT, "bounded device wait gave up");
    default: fail(FEAST_ERR_CUDA, "unknown device status " + std::to_string(st));
  }
}

void reset_status(feast_handle* h) {
  h->status.ensure(sizeof(int) * 4, "status");
  ck(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, h->stream), "status reset");
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// Factor all Ne node matrices and keep the factors in the handle.
void factor_nodes(feast_handle* h, const OpView& op, int Ne, int precision) {
  const int n = op.g.n(), nb = op.g.nz;
  const long long nn = (long long)n * n;
  if (h->opt.inner_solver == FEAST_INNER_COCG) return;   // iterative inner solves: nothing to factor
  if (precision == FEAST_PREC_FP64) {
    h->F.ensure(sizeof(cplx) * (size_t)Ne * nb * nn, "factors");
    h->T1.ensure(sizeof(cplx) * (size_t)Ne * nn, "schur scratch");
    h->T.ensure(sizeof(cplx) * (size_t)Ne * n * 64, "panel T");
    h->L.ensure(sizeof(cplx) * (size_t)Ne * n * 64, "panel L");
    h->Pinv.ensure(sizeof(cplx) * (size_t)Ne * 64 * 64, "panel inverse");
    Fp64Work w{h->F.as<cplx>(), h->T1.as<cplx>(), h->T.as<cplx>(), h->L.as<cplx>(), h->Pinv.as<cplx>(),
               h->status.as<int>()};
    factor_fp64(h->stream, op.g, Ne, h->Zd.as<cplx>(), op.A27, op.B27, w);
  } else {
    const char* msg =
        mixed_factor(h->stream, op.g, Ne, h->Zd.as<cplx>(), op.A27, op.B27, h->mixed, h->status.as<int>());
    if (msg) fail(FEAST_ERR_CUDA, msg);
  }
}

// Solve the Ne node systems for RHS (N x k real).  G (nullable on the mixed
// path): receives the node solutions (Ne x N x k complex).  Qp (nullable):
// receives the node shares Re{coef_e Q_e} of the quadrature sum (Eq. 15),
// folded in by the backward sweeps.
void solve_nodes(feast_handle* h, const OpView& op, int Ne, int precision, const double* RHS, cplx* G, double* Qp,
                 int k, double ir_tol) {
  const int n = op.g.n();
  if (h->opt.inner_solver == FEAST_INNER_COCG) {
    // iterative inner solves (Sec. IV.C); the node shares are formed from
    // the solutions by quadrature_from_solutions instead
    if (!G) fail(FEAST_ERR_ARG, "iterative inner solves need the solution buffer");
    h->cgw.ensure(cocg_work_bytes(op.g, Ne, k), "iterative solver work space");
    CocgStats st;
    const char* msg = cocg_solve(h->stream, op.g, Ne, h->Zd.as<cplx>(), op.A27, op.B27, RHS, G, k, h->opt.inner_tol,
                                 h->opt.inner_max_iter, h->cgw.p, h->status.as<int>(), &st);
    h->info.inner_iters_max = std::max(h->info.inner_iters_max, st.iterations);
    h->info.inner_rel_max = std::max(h->info.inner_rel_max, st.rel_max);
    if (msg) {
      int dst = 0;
      cudaMemcpy(&dst, h->status.p, sizeof(int), cudaMemcpyDeviceToHost);
      fail(dst == DEV_PIVOT ? FEAST_ERR_PIVOT : FEAST_ERR_NO_CONVERGENCE, msg);
    }
    return;
  }
  if (precision == FEAST_PREC_FP64) {
    h->Tmp.ensure(sizeof(cplx) * (size_t)Ne * n * k, "solve scratch");
    if (!G) {   // the FP64 sweeps keep their layer solutions in G
      h->G.ensure(sizeof(cplx) * (size_t)Ne * op.g.N() * k, "node solutions");
      G = h->G.as<cplx>();
    }
    solve_fp64(h->stream, op.g, Ne, h->Zd.as<cplx>(), op.A27, op.B27, h->F.as<cplx>(), RHS, G, h->Tmp.as<cplx>(),
               k, Qp, h->coefd.as<cplx>());
  } else {
    MixedSolveStats st;
    const char* msg = mixed_solve(h->stream, op.g, Ne, h->Zd.as<cplx>(), op.A27, op.B27, h->mixed, RHS, G, Qp,
                                  h->coefd.as<cplx>(), k, ir_tol, h->opt.ir_max, &st, h->status.as<int>());
    if (msg) fail(FEAST_ERR_CUDA, msg);
    h->info.ir_steps_max = std::max(h->info.ir_steps_max, st.steps_max);
    if (ir_tol <= h->opt.ir_tol) h->info.ir_resid_max = std::max(h->info.ir_resid_max, st.resid_max);
    h->info.sweep_graphs += st.graph_sweeps;
  }
}

// Fig. 2 step 2 in full: the Ne node solves of RHS and the quadrature sum
// Q (Eq. 15), N x k.
void node_solves_and_quadrature(feast_handle* h, const OpView& op, int Ne, int precision, const double* RHS, int k,
                                double ir_tol, double* Q) {
  const long long N = op.g.N();
  if (h->opt.inner_solver == FEAST_INNER_COCG) {
    h->G.ensure(sizeof(cplx) * (size_t)Ne * N * k, "node solutions");
    solve_nodes(h, op, Ne, precision, RHS, h->G.as<cplx>(), nullptr, k, ir_tol);
    quadrature_from_solutions(h->stream, N, k, Ne, h->coefd.as<cplx>(), h->G.as<cplx>(), Q);
    return;
  }
  h->Qp.ensure(sizeof(double) * (size_t)Ne * N * k, "quadrature shares");
  solve_nodes(h, op, Ne, precision, RHS, nullptr, h->Qp.as<double>(), k, ir_tol);
  quadrature_sum(h->stream, N, k, Ne, h->Qp.as<double>(), N * k, Q);
}

void upload_contour(feast_handle* h, const Contour& ct) {
  const int Ne = (int)ct.Z.size();
  h->Zd.ensure(sizeof(cplx) * Ne, "Z");
  h->coefd.ensure(sizeof(cplx) * Ne, "coef");
  ck(cudaMemcpyAsync(h->Zd.p, ct.Z.data(), sizeof(cplx) * Ne, cudaMemcpyHostToDevice, h->stream), "Z");
  ck(cudaMemcpyAsync(h->coefd.p, ct.coef.data(), sizeof(cplx) * Ne, cudaMemcpyHostToDevice, h->stream), "coef");
}

// Rayleigh-Ritz on Q (device, N x M0): eps (device, M0), X (device, N x M0).
// Work space of rayleigh_ritz_dev and rhs_dev for M0 columns (allocated
// before a stream capture can start).
void rr_workspace(feast_handle* h, long long N, int M0, bool df) {
  h->AQf.ensure(sizeof(double) * N * M0, "AQ full");
  h->BQf.ensure(sizeof(double) * N * M0, "BQ full");
  h->part.ensure(sizeof(double) * std::max(gram_partial_elems(N, M0, M0), df ? gram_partial_elems_df(N, M0, M0) : 0),
                 "gram partials");
  h->AQ.ensure(sizeof(double) * M0 * M0, "A_Q");
  h->BQ.ensure(sizeof(double) * M0 * M0, "B_Q");
  h->Phi.ensure(sizeof(double) * M0 * M0, "Phi");
  h->work.ensure(sizeof(double) * 3 * M0 * M0, "eig work");
  if (df) h->Qdf.ensure(sizeof(float2) * N * M0, "double-float block");
}

// Steps 3-5 (Eqs. 6-9).  df (mixed path): the operator products, Gram
// matrices and X = Q Phi in double-float arithmetic (rr_df.cu); the reduced
// eigensolve in FP64 either way.
void rayleigh_ritz_dev(feast_handle* h, const OpView& op, const double* Q, int M0, double* eps, double* X,
                       double* AQout, double* BQout, cudaStream_t st = nullptr, bool df = false) {
  const long long N = op.g.N();
  cudaStream_t s = st ? st : h->stream;
  rr_workspace(h, N, M0, df);
  double* AQ = AQout ? AQout : h->AQ.as<double>();
  double* BQ = BQout ? BQout : h->BQ.as<double>();
  if (df) {
    float2* Qd = h->Qdf.as<float2>();
    split_df(s, N * M0, Q, Qd);
    stencil_apply_df(s, op.g, op.A27, Qd, N, h->AQf.as<float2>(), N, M0);
    stencil_apply_df(s, op.g, op.B27, Qd, N, h->BQf.as<float2>(), N, M0);
    gram_df(s, N, M0, M0, Qd, h->AQf.as<float2>(), h->part.as<double>(), AQ, true);   // Q^T (A Q), A symmetric
    gram_df(s, N, M0, M0, Qd, h->BQf.as<float2>(), h->part.as<double>(), BQ, true);
    reduced_eig(s, M0, AQ, BQ, eps, h->Phi.as<double>(), h->work.as<double>(), h->status.as<int>());
    gemm_tall_df(s, N, M0, M0, Qd, h->Phi.as<double>(), X);
    return;
  }
  stencil_apply(s, op.g, op.A27, Q, N, h->AQf.as<double>(), N, M0);
  stencil_apply(s, op.g, op.B27, Q, N, h->BQf.as<double>(), N, M0);
  gram(s, N, M0, M0, Q, h->AQf.as<double>(), h->part.as<double>(), AQ, true);   // Q^T (A Q), A symmetric
  gram(s, N, M0, M0, Q, h->BQf.as<double>(), h->part.as<double>(), BQ, true);
  reduced_eig(s, M0, AQ, BQ, eps, h->Phi.as<double>(), h->work.as<double>(), h->status.as<int>());
  dgemm_tall(s, N, M0, M0, Q, h->Phi.as<double>(), X);
}

// Step 2's right-hand side RHS = B Y (N x M0); df as in rayleigh_ritz_dev.
void rhs_dev(feast_handle* h, const OpView& op, const double* Y, int M0, double* RHS, cudaStream_t s, bool df) {
  const long long N = op.g.N();
  if (df) {
    h->Qdf.ensure(sizeof(float2) * N * M0, "double-float block");
    split_df(s, N * M0, Y, h->Qdf.as<float2>());
    stencil_apply_df(s, op.g, op.B27, h->Qdf.as<float2>(), N, RHS, N, M0);
  } else {
    stencil_apply(s, op.g, op.B27, Y, N, RHS, N, M0);
  }
}

void residuals_dev(feast_handle* h, const OpView& op, const double* lam, const double* X, int k, double* resid,
                   double* resid_paper) {
  const long long N = op.g.N();
  h->AQf.ensure(sizeof(double) * N * k, "AX");
  h->BQf.ensure(sizeof(double) * N * k, "BX");
  h->norms.ensure(sizeof(double) * 3 * k, "norms");
  h->normA.ensure(sizeof(double), "normA");
  stencil_apply(h->stream, op.g, op.A27, X, N, h->AQf.as<double>(), N, k);
  stencil_apply(h->stream, op.g, op.B27, X, N, h->BQf.as<double>(), N, k);
  residual_norms(h->stream, N, k, h->AQf.as<double>(), h->BQf.as<double>(), lam, X, h->norms.as<double>());
  stencil_norm1(h->stream, op.g, op.A27, h->normA.as<double>());
  residual_finish(h->stream, k, h->norms.as<double>(), h->normA.as<double>(), resid, resid_paper);
}

}  // namespace

extern "C" {

void feast_default_options(feast_options* opt) {
  if (!opt) return;
  opt->max_loops = 20;
  opt->precision = FEAST_PREC_FP64;
  opt->ir_tol = 1e-12;
  opt->ir_max = 30;
  opt->ir_early = 1;
  opt->seed = 1000;
  opt->profile = 0;
  opt->inner_solver = FEAST_INNER_DIRECT;
  opt->inner_tol = 1e-3;
  opt->inner_max_iter = 5000;
}

feast_status feast_init(feast_handle** out, const feast_options* opt, void* cuda_stream) {
  if (!out) return FEAST_ERR_ARG;
  *out = nullptr;
  feast_handle* h = new feast_handle();
  feast_default_options(&h->opt);
  if (opt) h->opt = *opt;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  feast_status st = guarded(h, [&] {
    if (h->opt.max_loops < 1 || h->opt.max_loops > 1000) fail(FEAST_ERR_ARG, "max_loops out of range");
    if (h->opt.precision != FEAST_PREC_FP64 && h->opt.precision != FEAST_PREC_MIXED)
      fail(FEAST_ERR_ARG, "unknown precision");
    if (h->opt.inner_solver != FEAST_INNER_DIRECT && h->opt.inner_solver != FEAST_INNER_COCG)
      fail(FEAST_ERR_ARG, "unknown inner solver");
    if (h->opt.inner_solver == FEAST_INNER_COCG && (!(h->opt.inner_tol > 0.0) || h->opt.inner_max_iter < 1))
      fail(FEAST_ERR_ARG, "inner_tol must be > 0 and inner_max_iter >= 1");
    ck(cudaGetDevice(&h->device), "cudaGetDevice");
    if (h->opt.profile) prof::set_enabled(true);
    for (auto& e : h->ev) ck(cudaEventCreate(&e), "event");
    reset_status(h);
  });
  if (st != FEAST_OK) {
    delete h;
    return st;
  }
  *out = h;
  return FEAST_OK;
}

feast_status feast_destroy(feast_handle* h) {
  if (!h) return FEAST_OK;
  cudaStreamSynchronize(h->stream);
  h->release_all();
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
  return FEAST_OK;
}

const char* feast_last_error(const feast_handle* h) { return h ? h->err.c_str() : "null handle"; }

feast_status feast_get_info(const feast_handle* h, feast_info* info) {
  if (!h || !info) return FEAST_ERR_ARG;
  *info = h->info;
  return FEAST_OK;
}

feast_status feast_contour(double lmin, double lmax, int Ne, double* x, double* w, double* theta, double* Zre,
                           double* Zim) {
  if (Ne < 1 || Ne > 64 || !(lmin < lmax)) return FEAST_ERR_ARG;
  Contour ct = make_contour(lmin, lmax, Ne);
  for (int e = 0; e < Ne; ++e) {
    if (x) x[e] = ct.x[e];
    if (w) w[e] = ct.w[e];
    if (theta) theta[e] = ct.theta[e];
    if (Zre) Zre[e] = ct.Z[e].re;
    if (Zim) Zim[e] = ct.Z[e].im;
  }
  return FEAST_OK;
}

feast_status feast_selftest_wait_timeout(feast_handle* h, long long polls) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (polls < 1 || polls > kSelftestMaxPolls) fail(FEAST_ERR_ARG, "polls must be in [1, 2^26]");
    reset_status(h);
    selftest_wait(h->stream, polls, h->status.as<int>());
    ck(cudaGetLastError(), "self-test launch");
    int st = 0;
    ck(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status");
    ck(cudaStreamSynchronize(h->stream), "sync");
    reset_status(h);   // the handle's later calls start from a clean status word
    if (st == DEV_TIMEOUT) fail(FEAST_ERR_TIMEOUT, "bounded device wait gave up (self-test)");
    if (st != DEV_OK) fail(FEAST_ERR_CUDA, "unexpected device status " + std::to_string(st));
  });
}

feast_status feast_stencil_apply(feast_handle* h, int nx, int ny, int nz, const double* C27, const double* X,
                                 double* Y, int k) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (nx < 1 || ny < 1 || nz < 1 || k < 0 || !C27 || !X || !Y) fail(FEAST_ERR_ARG, "bad stencil arguments");
    Grid g{nx, ny, nz};
    stencil_apply(h->stream, g, C27, X, g.N(), Y, g.N(), k);
    ck(cudaGetLastError(), "stencil launch");
  });
}

feast_status feast_node_solve(feast_handle* h, const feast_operator* op, double Zre, double Zim,
                              const double* RHS, double* Qe, int k, int precision) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (!(Zim > 0.0)) fail(FEAST_ERR_ARG, "Im(Z) must be > 0");
    if (k < 1 || k > 1024 || !RHS || !Qe) fail(FEAST_ERR_ARG, "bad right-hand side");
    if (precision != FEAST_PREC_FP64 && precision != FEAST_PREC_MIXED) fail(FEAST_ERR_ARG, "bad precision");
    OpView v = device_operator(h, op);
    reset_status(h);
    cplx z{Zre, Zim};
    h->Zd.ensure(sizeof(cplx), "Z");
    ck(cudaMemcpyAsync(h->Zd.p, &z, sizeof(cplx), cudaMemcpyHostToDevice, h->stream), "Z");
    h->info.ir_steps_max = 0;
    h->info.ir_resid_max = 0.0;
    h->info.inner_iters_max = 0;
    h->info.inner_rel_max = 0.0;
    factor_nodes(h, v, 1, precision);
    check_status(h);
    solve_nodes(h, v, 1, precision, RHS, reinterpret_cast<cplx*>(Qe), nullptr, k, h->opt.ir_tol);
    check_status(h);
  });
}

feast_status feast_quadrature(feast_handle* h, const feast_operator* op, double lmin, double lmax, int Ne,
                              const double* RHS, double* Q, int k, int precision) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (!(lmin < lmax) || Ne < 1 || Ne > 64 || k < 1 || !RHS || !Q) fail(FEAST_ERR_ARG, "bad arguments");
    OpView v = device_operator(h, op);
    reset_status(h);
    Contour ct = make_contour(lmin, lmax, Ne);
    upload_contour(h, ct);
    const long long N = v.g.N();
    h->info.ir_steps_max = 0;
    h->info.ir_resid_max = 0.0;
    factor_nodes(h, v, Ne, precision);
    check_status(h);
    node_solves_and_quadrature(h, v, Ne, precision, RHS, k, h->opt.ir_tol, Q);
    check_status(h);
  });
}

feast_status feast_reduced_eig(feast_handle* h, const double* AQ, const double* BQ, int M0, double* eps,
                               double* Phi) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (M0 < 1 || M0 > 128 || !AQ || !BQ || !eps || !Phi) fail(FEAST_ERR_ARG, "bad arguments");
    reset_status(h);
    h->work.ensure(sizeof(double) * 3 * M0 * M0, "eig work");
    reduced_eig(h->stream, M0, AQ, BQ, eps, Phi, h->work.as<double>(), h->status.as<int>());
    check_status(h);
  });
}

feast_status feast_rayleigh_ritz(feast_handle* h, const feast_operator* op, const double* Q, int M0,
                                 double* eps, double* X, double* AQ, double* BQ) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (M0 < 1 || M0 > 128 || !Q || !eps || !X) fail(FEAST_ERR_ARG, "bad arguments");
    OpView v = device_operator(h, op);
    reset_status(h);
    rayleigh_ritz_dev(h, v, Q, M0, eps, X, AQ, BQ);
    check_status(h);
  });
}

feast_status feast_residuals(feast_handle* h, const feast_operator* op, const double* lambda, const double* X,
                             int k, double* resid, double* resid_paper) {
  if (!h) return FEAST_ERR_ARG;
  return guarded(h, [&] {
    if (k < 1 || !lambda || !X) fail(FEAST_ERR_ARG, "bad arguments");
    OpView v = device_operator(h, op);
    residuals_dev(h, v, lambda, X, k, resid, resid_paper);
    ck(cudaStreamSynchronize(h->stream), "sync");
    ck(cudaGetLastError(), "residual kernels");
  });
}

feast_status feast_solve(feast_handle* h, const feast_operator* op, double lmin, double lmax, int M0, int Ne,
                         double tol, const double* Y0, double* lambda, double* X, double* resid, int* m_found,
                         int* loops) {
  if (!h) return FEAST_ERR_ARG;
  feast_status final_status = FEAST_OK;
  feast_status st = guarded(h, [&] {
    auto t_wall0 = std::chrono::steady_clock::now();
    h->info = feast_info{};
    if (h->opt.profile) {
      prof::set_enabled(true);
      prof::collect(nullptr, nullptr, nullptr);   // drop records of earlier calls
    } else {
      prof::set_enabled(false);
    }
    const long long launches0 = prof::launches();
    if (!(lmin < lmax) || !std::isfinite(lmin) || !std::isfinite(lmax)) fail(FEAST_ERR_ARG, "need lmin < lmax");
    if (Ne < 1 || Ne > 64) fail(FEAST_ERR_ARG, "Ne must be in [1, 64]");
    if (!lambda || !X || !m_found || !loops) fail(FEAST_ERR_ARG, "output pointer is NULL");
    if (!(tol >= 0.0)) fail(FEAST_ERR_ARG, "tol must be >= 0");
    OpView v = device_operator(h, op);
    const long long N = v.g.N();
    const int n = v.g.n();
    if (M0 < 1 || M0 > 128 || M0 > N) fail(FEAST_ERR_ARG, "M0 must be in [1, min(N, 128)]");
    const int prec = h->opt.precision;
    cudaStream_t s = h->stream;
    reset_status(h);
    Contour ct = make_contour(lmin, lmax, Ne);
    upload_contour(h, ct);

    // ---- node factorisations, once for all loops (Sec. V (ii))
    ck(cudaEventRecord(h->ev[0], s), "event");
    factor_nodes(h, v, Ne, prec);
    ck(cudaEventRecord(h->ev[1], s), "event");
    check_status(h);
    h->info.t_factor_ms = elapsed(h->ev[0], h->ev[1]);
    h->info.factor_flops =
        h->opt.inner_solver == FEAST_INNER_COCG ? 0 : (long long)8 * n * (long long)n * n * v.g.nz * Ne;

    // ---- buffers of the loop
    const size_t blk = sizeof(double) * (size_t)N * M0;
    h->RHS.ensure(blk, "RHS");
    h->Q.ensure(blk, "Q");
    h->Xb.ensure(blk, "X");
    h->Yb.ensure(blk, "Y");
    h->Xout.ensure(blk, "X out");
    h->eps.ensure(sizeof(double) * M0, "eps");
    h->lam_d.ensure(sizeof(double) * M0, "lambda");
    h->perm_d.ensure(sizeof(int) * M0, "perm");
    h->resid_d.ensure(sizeof(double) * M0, "resid");
    h->residp_d.ensure(sizeof(double) * M0, "resid paper");

    // ---- step 1: start block
    if (Y0) {
      ck(cudaMemcpyAsync(h->Yb.p, Y0, blk, is_device_ptr(Y0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
         "copy Y0");
    } else {
      random_block(s, N, M0, h->opt.seed, h->Yb.as<double>());
    }

    std::vector<double> eps(M0);
    double prev_trace = 0.0;
    int prev_count = -1;
    bool converged = false;
    int count = 0, loop = 0;
    double t_solve = 0, t_rr = 0;
    const bool early = h->opt.ir_early && !Y0 && prec == FEAST_PREC_MIXED;
    // ---- the loop as one CUDA graph with device-side conditions (mixed
    // precision, no kernel timing): steps 2-6 and every refinement decision
    // stay on the device, and the host reads the final state once
    bool device_loop = false;
    if (prec == FEAST_PREC_MIXED && !h->opt.profile && h->mixed.use_graphs &&
        h->opt.inner_solver == FEAST_INNER_DIRECT) {
      h->Qp.ensure(sizeof(double) * (size_t)Ne * N * M0, "quadrature shares");
      h->loopst.ensure(sizeof(LoopState), "loop state");
      // Rayleigh-Ritz work space, sized before a capture can start
      rr_workspace(h, N, M0, true);
      // node-solve buffers too, so that the key below is the same from the
      // first solve on
      if (const char* m = mixed_solve_prepare(s, v.g, Ne, M0, h->mixed, h->status.as<int>()))
        fail(FEAST_ERR_CUDA, m);
      const LoopParams lp{lmin, lmax, tol, h->opt.ir_tol, early ? 1 : 0, h->opt.max_loops, h->opt.ir_max, M0};
      LoopHooks hooks;
      hooks.rhs = [&](cudaStream_t st) { rhs_dev(h, v, h->Yb.as<double>(), M0, h->RHS.as<double>(), st, true); };
      hooks.quad_rr = [&](cudaStream_t st) {
        quadrature_sum(st, N, M0, Ne, h->Qp.as<double>(), N * M0, h->Q.as<double>());
        rayleigh_ritz_dev(h, v, h->Q.as<double>(), M0, h->eps.as<double>(), h->Xb.as<double>(), nullptr, nullptr, st,
                          true);
      };
      hooks.next_y = [&](cudaStream_t st) { cudaMemcpyAsync(h->Yb.p, h->Xb.p, blk, cudaMemcpyDeviceToDevice, st); };
      auto bits = [](double x) {
        unsigned long long u;
        std::memcpy(&u, &x, sizeof(u));
        return u;
      };
      auto ptr = [](const void* q) { return (unsigned long long)(uintptr_t)q; };
      unsigned long long key[kLoopKey] = {
          (unsigned long long)v.g.nx | ((unsigned long long)v.g.ny << 20) | ((unsigned long long)v.g.nz << 40),
          (unsigned long long)M0 | ((unsigned long long)Ne << 20), bits(lmin), bits(lmax), bits(tol),
          bits(h->opt.ir_tol),
          (unsigned long long)lp.early | ((unsigned long long)lp.max_loops << 8) | ((unsigned long long)lp.ir_max << 24),
          ptr(v.A27), ptr(v.B27), ptr(h->Zd.p), ptr(h->coefd.p), ptr(h->status.p), ptr(h->RHS.p), ptr(h->Q.p),
          ptr(h->Qp.p), ptr(h->Xb.p), ptr(h->Yb.p), ptr(h->eps.p), ptr(h->AQf.p), ptr(h->BQf.p), ptr(h->part.p),
          ptr(h->AQ.p), ptr(h->BQ.p), ptr(h->Phi.p), ptr(h->work.p), ptr(h->loopst.p), ptr(s), 3ULL};
      for (int i = 0; i < 16; ++i) key[28 + i] = ptr(h->mixed.bufs[i]);
      key[44] = ptr(h->Qdf.p);
      ck(cudaEventRecord(h->ev[2], s), "event");
      const char* msg = mixed_loop(s, v.g, Ne, h->Zd.as<cplx>(), v.A27, v.B27, h->mixed, h->RHS.as<double>(),
                                   h->Qp.as<double>(), h->coefd.as<cplx>(), M0, lp, h->eps.as<double>(),
                                   h->loopst.as<LoopState>(), hooks, key, h->status.as<int>());
      if (msg && msg != kNotCaptured) fail(FEAST_ERR_CUDA, msg);
      if (!msg) {
        device_loop = true;
        ck(cudaEventRecord(h->ev[4], s), "event");
        LoopState ls{};
        ck(cudaMemcpyAsync(&ls, h->loopst.p, sizeof(LoopState), cudaMemcpyDeviceToHost, s), "loop state");
        ck(cudaMemcpyAsync(eps.data(), h->eps.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "eps");
        check_status(h);
        if (ls.fail == 1) fail(FEAST_ERR_CUDA, "iterative refinement did not reach the tolerance");
        if (ls.fail == 2) fail(FEAST_ERR_CUDA, "non-finite residual in the refinement");
        loop = ls.loop;
        count = ls.count;
        converged = ls.converged != 0;
        for (int i = 0; i < std::min(loop, 64); ++i) {
          h->info.trace[i] = ls.trace_hist[i];
          h->info.rel_change[i] = ls.change_hist[i];
        }
        h->info.ir_steps_max = ls.ir_steps_max;
        h->info.ir_resid_max = ls.ir_resid_max;
        t_solve = elapsed(h->ev[2], h->ev[4]);   // the whole loop: node solves and Rayleigh-Ritz
        t_rr = -1.0;
        h->info.loop_graphs = 1;
        // the kernels the graph ran: its loop bodies and refinement steps
        prof::count_launch((int)(1 + (long long)loop * h->mixed.loop_outer_launches +
                                 (long long)ls.ir_steps_total * h->mixed.loop_inner_launches));
        ++h->loop_graph_solves;
      }
    }
    for (loop = device_loop ? loop : 1; !device_loop && loop <= h->opt.max_loops; ++loop) {

      ck(cudaEventRecord(h->ev[2], s), "event");
      // step 2: RHS = B Y, node solves, quadrature (Eq. 15)
      rhs_dev(h, v, h->Yb.as<double>(), M0, h->RHS.as<double>(), s, prec == FEAST_PREC_MIXED);
      // refinement target of this loop: loosened in loops 1 and 2 (their subspace
      // is still far from converged, so their solves need less accuracy)
      double ir_loop = h->opt.ir_tol;
      if (early && loop <= 2) ir_loop = std::max(ir_loop, early_tol(loop));
      const bool exact_loop = ir_loop <= h->opt.ir_tol;
      node_solves_and_quadrature(h, v, Ne, prec, h->RHS.as<double>(), M0, ir_loop, h->Q.as<double>());
      ck(cudaEventRecord(h->ev[3], s), "event");
      // steps 3-5: Rayleigh-Ritz
      rayleigh_ritz_dev(h, v, h->Q.as<double>(), M0, h->eps.as<double>(), h->Xb.as<double>(), nullptr, nullptr,
                        nullptr, prec == FEAST_PREC_MIXED);
      ck(cudaEventRecord(h->ev[4], s), "event");
      ck(cudaMemcpyAsync(eps.data(), h->eps.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "eps");
      check_status(h);
      t_solve += elapsed(h->ev[2], h->ev[3]);
      t_rr += elapsed(h->ev[3], h->ev[4]);
      // step 6: trace test
      count = 0;
      double trace = 0.0, scale = 0.0;
      for (int j = 0; j < M0; ++j)
        if (eps[j] >= lmin && eps[j] <= lmax) {
          ++count;
          trace += eps[j];
          scale += std::fabs(eps[j]);
        }
      if (loop - 1 < 64) {
        h->info.trace[loop - 1] = trace;
        h->info.rel_change[loop - 1] = -1.0;
      }
      if (prev_count >= 0) {
        const double change = scale > 0 ? std::fabs(trace - prev_trace) / scale : 0.0;
        if (loop - 1 < 64) h->info.rel_change[loop - 1] = change;
        if (count == prev_count && change <= tol && exact_loop) converged = true;
      }
      // Y = X: the next right-hand side is B X (a copy, so that the loop's
      // buffers keep their addresses for the captured form above)
      ck(cudaMemcpyAsync(h->Yb.p, h->Xb.p, blk, cudaMemcpyDeviceToDevice, s), "Y = X");
      if (converged) break;
      prev_trace = trace;
      prev_count = count;
    }
    if (loop > h->opt.max_loops) loop = h->opt.max_loops;

    // ---- outputs: in-interval pairs first, each group ascending
    std::vector<int> perm;
    for (int j = 0; j < M0; ++j)
      if (eps[j] >= lmin && eps[j] <= lmax) perm.push_back(j);
    for (int j = 0; j < M0; ++j)
      if (!(eps[j] >= lmin && eps[j] <= lmax)) perm.push_back(j);
    std::vector<double> lam(M0);
    for (int j = 0; j < M0; ++j) lam[j] = eps[perm[j]];
    ck(cudaMemcpyAsync(h->perm_d.p, perm.data(), sizeof(int) * M0, cudaMemcpyHostToDevice, s), "perm");
    ck(cudaMemcpyAsync(h->lam_d.p, lam.data(), sizeof(double) * M0, cudaMemcpyHostToDevice, s), "lambda");
    permute_columns(s, N, M0, h->perm_d.as<int>(), h->Yb.as<double>(), h->Xout.as<double>());
    residuals_dev(h, v, h->lam_d.as<double>(), h->Xout.as<double>(), M0, h->resid_d.as<double>(),
                  h->residp_d.as<double>());
    std::vector<double> r1(M0), rp(M0);
    ck(cudaMemcpyAsync(r1.data(), h->resid_d.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "resid");
    ck(cudaMemcpyAsync(rp.data(), h->residp_d.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "resid");
    const bool xdev = is_device_ptr(X);
    ck(cudaMemcpyAsync(X, h->Xout.p, blk, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "copy X");
    if (is_device_ptr(lambda))
      ck(cudaMemcpyAsync(lambda, h->lam_d.p, sizeof(double) * M0, cudaMemcpyDeviceToDevice, s), "copy lambda");
    if (resid) {
      if (is_device_ptr(resid))
        ck(cudaMemcpyAsync(resid, h->resid_d.p, sizeof(double) * M0, cudaMemcpyDeviceToDevice, s), "copy resid");
    }
    ck(cudaStreamSynchronize(s), "sync");
    ck(cudaGetLastError(), "kernels");
    if (!is_device_ptr(lambda)) std::memcpy(lambda, lam.data(), sizeof(double) * M0);
    if (resid && !is_device_ptr(resid)) std::memcpy(resid, r1.data(), sizeof(double) * M0);
    *m_found = count;
    *loops = loop;
    h->info.loops = loop;
    h->info.m_found = count;
    h->info.t_solve_ms = t_solve;
    h->info.t_rr_ms = t_rr;
    for (int j = 0; j < count; ++j) {
      h->info.resid_max = std::max(h->info.resid_max, r1[j]);
      h->info.resid_paper_max = std::max(h->info.resid_paper_max, rp[j]);
    }
    h->info.gpu_launches = prof::launches() - launches0;
    if (h->opt.profile) prof::collect(h->info.kernel_ms, h->info.kernel_launches, h->info.kernel_flops);
    h->info.t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_wall0).count();
    if (count >= M0) final_status = FEAST_ERR_M0_TOO_SMALL;
    else if (!converged) final_status = FEAST_ERR_NO_CONVERGENCE;
  });
  if (st != FEAST_OK) return st;
  if (final_status == FEAST_ERR_M0_TOO_SMALL)
    h->err = "every Ritz value lies inside the interval: increase M0";
  else if (final_status == FEAST_ERR_NO_CONVERGENCE)
    h->err = "trace test not met within max_loops";
  return final_status;
}

feast_status feast_solve_hermitian(feast_handle* h, const feast_operator* op, double lmin, double lmax, int M0,
                                   int Ne, double tol, const double* Y0, double* lambda, double* X, double* resid,
                                   int* m_found, int* loops) {
  if (!h) return FEAST_ERR_ARG;
  feast_status final_status = FEAST_OK;
  feast_status st = guarded(h, [&] {
    auto t_wall0 = std::chrono::steady_clock::now();
    h->info = feast_info{};
    prof::set_enabled(false);
    const long long launches0 = prof::launches();
    if (!(lmin < lmax) || !std::isfinite(lmin) || !std::isfinite(lmax)) fail(FEAST_ERR_ARG, "need lmin < lmax");
    if (Ne < 1 || Ne > 32) fail(FEAST_ERR_ARG, "Ne must be in [1, 32]");
    if (!op || !lambda || !X || !m_found || !loops) fail(FEAST_ERR_ARG, "NULL argument");
    if (!(tol >= 0.0)) fail(FEAST_ERR_ARG, "tol must be >= 0");
    if (op->nx < 1 || op->ny < 1 || op->nz < 1) fail(FEAST_ERR_ARG, "grid sizes must be >= 1");
    if (!is_device_ptr(op->A27) || !is_device_ptr(op->B27) || !is_device_ptr(X) || (Y0 && !is_device_ptr(Y0)))
      fail(FEAST_ERR_ARG, "the Hermitian solve takes device arrays for A27, B27, Y0 and X");
    const Grid g{op->nx, op->ny, op->nz};
    if (g.n() > 4096) fail(FEAST_ERR_ARG, "layer size nx*ny must be <= 4096");
    const long long N = g.N();
    if (M0 < 1 || M0 > 64 || M0 > N) fail(FEAST_ERR_ARG, "M0 must be in [1, min(N, 64)]");
    const HermOp o{g, reinterpret_cast<const cplx*>(op->A27), reinterpret_cast<const cplx*>(op->B27)};
    cudaStream_t s = h->stream;
    reset_status(h);
    // the 2 Ne shifts Z_e, conj Z_e and their coefficients in Eq. 12:
    // -(w_e r / 4) e^{i theta_e} and -(w_e r / 4) e^{-i theta_e}
    Contour ct = make_contour(lmin, lmax, Ne);
    const int nodes = 2 * Ne;
    std::vector<cplx> Zh(nodes), ch(nodes);
    for (int e = 0; e < Ne; ++e) {
      const double a = -(ct.w[e] * ct.r / 4.0);
      Zh[e] = ct.Z[e];
      Zh[Ne + e] = cplx{ct.Z[e].re, -ct.Z[e].im};
      ch[e] = cplx{a * std::cos(ct.theta[e]), a * std::sin(ct.theta[e])};
      ch[Ne + e] = cplx{a * std::cos(ct.theta[e]), -a * std::sin(ct.theta[e])};
    }
    h->hZ.ensure(sizeof(cplx) * nodes, "Z");
    h->hCoef.ensure(sizeof(cplx) * nodes, "coef");
    ck(cudaMemcpyAsync(h->hZ.p, Zh.data(), sizeof(cplx) * nodes, cudaMemcpyHostToDevice, s), "Z");
    ck(cudaMemcpyAsync(h->hCoef.p, ch.data(), sizeof(cplx) * nodes, cudaMemcpyHostToDevice, s), "coef");
    const int n = g.n();
    const size_t cblk = sizeof(cplx) * (size_t)N * M0;
    h->hF.ensure(herm_factor_bytes(g, nodes), "Hermitian factors");
    h->hG.ensure(cblk * nodes, "node solutions");
    h->hTmp.ensure(sizeof(cplx) * (size_t)nodes * n * M0, "solve scratch");
    for (DevBuf* b : {&h->hRHS, &h->hQ, &h->hAQf, &h->hBQf, &h->hX, &h->hY, &h->hXout}) b->ensure(cblk, "block");
    h->hPart.ensure(sizeof(cplx) * herm_gram_elems(N, M0), "gram partials");
    for (DevBuf* b : {&h->hAQ, &h->hBQ, &h->hPhi}) b->ensure(sizeof(cplx) * M0 * M0, "reduced");
    h->hWork.ensure(sizeof(cplx) * 3 * M0 * M0, "eig work");
    h->hEps.ensure(sizeof(double) * M0, "eps");
    h->lam_d.ensure(sizeof(double) * M0, "lambda");
    h->perm_d.ensure(sizeof(int) * M0, "perm");
    h->resid_d.ensure(sizeof(double) * M0, "resid");
    h->residp_d.ensure(sizeof(double) * M0, "resid paper");
    h->norms.ensure(sizeof(double) * 3 * M0, "norms");
    h->normA.ensure(sizeof(double), "normA");
    cplx* Zd = h->hZ.as<cplx>();

    ck(cudaEventRecord(h->ev[0], s), "event");
    herm_factor(s, o, nodes, Zd, h->hF.as<cplx>(), h->status.as<int>());
    ck(cudaEventRecord(h->ev[1], s), "event");
    check_status(h);
    h->info.t_factor_ms = elapsed(h->ev[0], h->ev[1]);
    h->info.factor_flops = (long long)8 * n * (long long)n * n * g.nz * nodes;

    if (Y0)
      ck(cudaMemcpyAsync(h->hY.p, Y0, cblk, cudaMemcpyDeviceToDevice, s), "copy Y0");
    else
      herm_random(s, N, M0, h->opt.seed, h->hY.as<cplx>());
    std::vector<double> eps(M0);
    double prev_trace = 0.0, t_solve = 0.0, t_rr = 0.0;
    int prev_count = -1, count = 0, loop = 0;
    bool converged = false;
    for (loop = 1; loop <= h->opt.max_loops; ++loop) {
      ck(cudaEventRecord(h->ev[2], s), "event");
      herm_stencil(s, g, o.B27, h->hY.as<cplx>(), h->hRHS.as<cplx>(), M0);   // RHS = B Y
      herm_solve(s, o, nodes, Zd, h->hF.as<cplx>(), h->hRHS.as<cplx>(), h->hG.as<cplx>(), h->hTmp.as<cplx>(), M0);
      herm_quadrature(s, N, M0, nodes, h->hCoef.as<cplx>(), h->hG.as<cplx>(), h->hQ.as<cplx>());   // Eq. 12
      ck(cudaEventRecord(h->ev[3], s), "event");
      herm_stencil(s, g, o.A27, h->hQ.as<cplx>(), h->hAQf.as<cplx>(), M0);
      herm_stencil(s, g, o.B27, h->hQ.as<cplx>(), h->hBQf.as<cplx>(), M0);
      herm_gram(s, N, M0, h->hQ.as<cplx>(), h->hAQf.as<cplx>(), h->hPart.as<cplx>(), h->hAQ.as<cplx>());
      herm_gram(s, N, M0, h->hQ.as<cplx>(), h->hBQf.as<cplx>(), h->hPart.as<cplx>(), h->hBQ.as<cplx>());
      herm_reduced_eig(s, M0, h->hAQ.as<cplx>(), h->hBQ.as<cplx>(), h->hEps.as<double>(), h->hPhi.as<cplx>(),
                       h->hWork.as<cplx>(), h->status.as<int>());
      herm_gemm_tall(s, N, M0, M0, h->hQ.as<cplx>(), h->hPhi.as<cplx>(), h->hX.as<cplx>());
      ck(cudaEventRecord(h->ev[4], s), "event");
      ck(cudaMemcpyAsync(eps.data(), h->hEps.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "eps");
      check_status(h);
      t_solve += elapsed(h->ev[2], h->ev[3]);
      t_rr += elapsed(h->ev[3], h->ev[4]);
      count = 0;
      double trace = 0.0, scale = 0.0;
      for (int j = 0; j < M0; ++j)
        if (eps[j] >= lmin && eps[j] <= lmax) {
          ++count;
          trace += eps[j];
          scale += std::fabs(eps[j]);
        }
      if (loop - 1 < 64) {
        h->info.trace[loop - 1] = trace;
        h->info.rel_change[loop - 1] = -1.0;
      }
      if (prev_count >= 0) {
        const double change = scale > 0 ? std::fabs(trace - prev_trace) / scale : 0.0;
        if (loop - 1 < 64) h->info.rel_change[loop - 1] = change;
        if (count == prev_count && change <= tol) converged = true;
      }
      std::swap(h->hX, h->hY);   // Y = X: the next right-hand side is B X
      if (converged) break;
      prev_trace = trace;
      prev_count = count;
    }
    if (loop > h->opt.max_loops) loop = h->opt.max_loops;
    std::vector<int> perm;
    for (int j = 0; j < M0; ++j)
      if (eps[j] >= lmin && eps[j] <= lmax) perm.push_back(j);
    for (int j = 0; j < M0; ++j)
      if (!(eps[j] >= lmin && eps[j] <= lmax)) perm.push_back(j);
    std::vector<double> lam(M0);
    for (int j = 0; j < M0; ++j) lam[j] = eps[perm[j]];
    ck(cudaMemcpyAsync(h->perm_d.p, perm.data(), sizeof(int) * M0, cudaMemcpyHostToDevice, s), "perm");
    ck(cudaMemcpyAsync(h->lam_d.p, lam.data(), sizeof(double) * M0, cudaMemcpyHostToDevice, s), "lambda");
    herm_permute(s, N, M0, h->perm_d.as<int>(), h->hY.as<cplx>(), h->hXout.as<cplx>());
    herm_residuals(s, g, o.A27, o.B27, h->lam_d.as<double>(), h->hXout.as<cplx>(), M0, h->hAQf.as<cplx>(),
                   h->hBQf.as<cplx>(), h->norms.as<double>(), h->normA.as<double>(), h->resid_d.as<double>(),
                   h->residp_d.as<double>());
    std::vector<double> r1(M0), rp(M0);
    ck(cudaMemcpyAsync(r1.data(), h->resid_d.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "resid");
    ck(cudaMemcpyAsync(rp.data(), h->residp_d.p, sizeof(double) * M0, cudaMemcpyDeviceToHost, s), "resid");
    ck(cudaMemcpyAsync(X, h->hXout.p, cblk, cudaMemcpyDeviceToDevice, s), "copy X");
    if (is_device_ptr(lambda))
      ck(cudaMemcpyAsync(lambda, h->lam_d.p, sizeof(double) * M0, cudaMemcpyDeviceToDevice, s), "copy lambda");
    if (resid && is_device_ptr(resid))
      ck(cudaMemcpyAsync(resid, h->resid_d.p, sizeof(double) * M0, cudaMemcpyDeviceToDevice, s), "copy resid");
    ck(cudaStreamSynchronize(s), "sync");
    ck(cudaGetLastError(), "kernels");
    if (!is_device_ptr(lambda)) std::memcpy(lambda, lam.data(), sizeof(double) * M0);
    if (resid && !is_device_ptr(resid)) std::memcpy(resid, r1.data(), sizeof(double) * M0);
    *m_found = count;
    *loops = loop;
    h->info.loops = loop;
    h->info.m_found = count;
    h->info.t_solve_ms = t_solve;
    h->info.t_rr_ms = t_rr;
    for (int j = 0; j < count; ++j) {
      h->info.resid_max = std::max(h->info.resid_max, r1[j]);
      h->info.resid_paper_max = std::max(h->info.resid_paper_max, rp[j]);
    }
    h->info.gpu_launches = prof::launches() - launches0;
    h->info.t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_wall0).count();
    if (count >= M0) final_status = FEAST_ERR_M0_TOO_SMALL;
    else if (!converged) final_status = FEAST_ERR_NO_CONVERGENCE;
  });
  if (st != FEAST_OK) return st;
  if (final_status == FEAST_ERR_M0_TOO_SMALL)
    h->err = "every Ritz value lies inside the interval: increase M0";
  else if (final_status == FEAST_ERR_NO_CONVERGENCE)
    h->err = "trace test not met within max_loops";
  return final_status;
}

// Device bytes one instance needs (mixed or FP64 path), for the worker count.
static double instance_bytes(const feast_operator& op, int M0, int Ne, int precision) {
  const double N = (double)op.nx * op.ny * op.nz, n = (double)op.nx * op.ny;
  const double ldF = std::ceil(2.0 * n / 32.0) * 32.0;
  const double blk = 8.0 * N * M0;
  double b = 8.0 * N * M0 * Ne + 12.0 * blk + 2.0 * 27.0 * N * 8.0;   // quadrature shares, loop blocks, operator
  if (precision == FEAST_PREC_MIXED)
    b += 4.0 * Ne * op.nz * n * ldF + 8.0 * Ne * 27.0 * N + 3.0 * 8.0 * N * M0 * Ne + 4.0 * Ne * 6.0 * n * ldF;
  else
    b += 16.0 * Ne * op.nz * n * n + 16.0 * Ne * n * n + 16.0 * N * M0 * Ne;
  return b * 1.05 + 64.0 * 1024 * 1024;
}

feast_status feast_solve_batched(feast_handle* h, int count, const feast_operator* ops, const double* lmin,
                                 const double* lmax, const int* M0, int Ne, double tol, const double* const* Y0,
                                 double* const* lambda, double* const* X, double* const* resid, int* m_found,
                                 int* loops, feast_status* statuses, int workers) {
  if (!h) return FEAST_ERR_ARG;
  if (count < 0 || (count > 0 && (!ops || !lmin || !lmax || !M0 || !lambda || !X || !m_found || !loops || !statuses)))
    return FEAST_ERR_ARG;
  if (count == 0) return FEAST_OK;
  const long long launches0 = prof::launches();
  // largest instances first
  std::vector<int> order(count);
  std::vector<double> bytes(count);
  for (int i = 0; i < count; ++i) {
    order[i] = i;
    bytes[i] = instance_bytes(ops[i], M0[i], Ne, h->opt.precision);
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return bytes[a] > bytes[b]; });
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    h->err = "cudaMemGetInfo failed";
    return FEAST_ERR_CUDA;
  }
  int K = workers > 0 ? workers : (int)std::floor(0.85 * (double)free_b / bytes[order[0]]);
  K = std::max(1, std::min({K, 8, count}));
  feast_options opt = h->opt;
  opt.profile = 0;
  const int device = h->device;
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  std::vector<std::string> errs(count);
  for (int wkr = 0; wkr < K; ++wkr) {
    pool.emplace_back([&, wkr] {
      cudaSetDevice(device);
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        for (int j; (j = next.fetch_add(1)) < count;) statuses[order[j]] = FEAST_ERR_CUDA;
        return;
      }
      feast_handle* sub = nullptr;
      if (feast_init(&sub, &opt, st) != FEAST_OK) {
        for (int j; (j = next.fetch_add(1)) < count;) statuses[order[j]] = FEAST_ERR_CUDA;
        cudaStreamDestroy(st);
        return;
      }
      // the instances are factored and swept once each: graph captures would
      // not be replayed, and the concurrent workers keep the GPU busy anyway
      sub->mixed.use_graphs = false;
      for (int j; (j = next.fetch_add(1)) < count;) {
        const int i = order[j];
        statuses[i] = feast_solve(sub, &ops[i], lmin[i], lmax[i], M0[i], Ne, tol, Y0 ? Y0[i] : nullptr, lambda[i],
                                  X[i], resid ? resid[i] : nullptr, &m_found[i], &loops[i]);
        if (statuses[i] != FEAST_OK) errs[i] = sub->err;
      }
      feast_destroy(sub);
      cudaStreamDestroy(st);
    });
  }
  for (auto& t : pool) t.join();
  h->info.gpu_launches = prof::launches() - launches0;   // every worker's launches
  for (int i = 0; i < count; ++i)
    if (statuses[i] != FEAST_OK) {
      h->err = "instance " + std::to_string(i) + ": " + errs[i];
      return statuses[i];
    }
  h->err.clear();
  return FEAST_OK;
}

}  // extern "C"
