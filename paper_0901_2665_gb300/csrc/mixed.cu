// Mixed-precision node factor-and-solve (Fig. 2 step 2 in complex64 on the
// tensor cores, refined to FP64 accuracy).
//
// Factor: the same unpivoted block elimination as the FP64 path (Schur
// complements through the layer couplings, symmetric block sweep inversion
// S'_i = -S_i^{-1}), carried in fp32 complex.  The sweep's trailing updates
// S[i, j] -= sum_k T[i, k] L[j, k] (panel width 64) run as one real GEMM
// on tcgen05 through the real embedding
//   [Ur | Ui] = [Tr | Ti] [[Lr^T, Li^T], [-Li^T, Lr^T]],
// and so do the block solves t = S' g, with both operands as split bf16
// pairs (x = x_hi + x_lo, 16 significant bits; three bf16 products each,
// the same bytes as TF32): the refinement's contraction per step is set by
// the solve's operand rounding far more than by the factor's.  Storage of
// S'_i is "row-split": row p holds the n real parts, then the n imaginary
// parts, so a row is directly the K-major A operand [Sr | Si] of the solve
// GEMM.
//
// Solve: forward/backward sweeps in complex64 (split-bf16 products, fp32
// accumulation) give a correction d = M~^{-1} R; FP64 iterative refinement
// Q_e += d, R = RHS - (Z_e B - A) Q_e repeats until ||R||/||RHS|| <= ir_tol
// for every node (the first residual in FP64, the later ones updated by the
// last correction in double-float).
//
// Launch: all Ne nodes in every kernel (grid z = node).  Without kernel
// timing, a factorisation and a pair of sweeps whose launch sequence was
// seen before on the same work space are replayed from CUDA graphs.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "mixed.cuh"
#include "prof.cuh"
#include "tc_gemm.cuh"
#include "tma.cuh"

namespace feast {

namespace {

constexpr int kPanel = 64;   // sweep panel width (complex columns)
#ifndef FEAST_PANEL_ROWS
#define FEAST_PANEL_ROWS 32
#endif
// rows per CTA of the panel product (each CTA stages the 64 x 64 inverse)
constexpr int kRowsPerPanelCta = FEAST_PANEL_ROWS;
static_assert(kRowsPerPanelCta % 8 == 0, "eight row groups of the panel product");

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

// ------------------------------------------------------------------ layout
struct Dims {
  int nx, ny, nz, n, Ne;
  long long N;
  int ldF;       // floats per row-split row (>= 2n, multiple of 32)
  int nblk64;    // ceil(n / 64)
  int k;         // right-hand sides
  int CB;        // complex columns per solve-GEMM tile
  int ST;        // pipeline stages of the solve GEMM
  int nblkCB;    // ceil(k / CB)
  int ldB;       // floats per embedded RHS row
  int K;         // middle layer of the two-ended elimination (nz - 1: one-ended)
};

// Cf[e][s][i] = (Z_e B - A)[i, i + off(s)] in complex fp32, 0 outside the grid:
// the coefficients of every node matrix, computed once per factorisation.
__global__ void k_mx_coef(Dims d, const cplx* __restrict__ Z, const double* __restrict__ A27,
                          const double* __restrict__ B27, f2* __restrict__ Cf) {
  const int e = blockIdx.y;
  const cplx z = Z[e];
  const long long total = 27LL * d.N;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / d.N);
    const long long i = t % d.N;
    const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
    const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
    const bool ok = ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 &&
                    iz + dz < d.nz;
    const double a = ok ? A27[t] : 0.0, b = ok ? B27[t] : 0.0;
    Cf[(long long)e * total + t] = ok ? f2{(float)(z.re * b - a), (float)(z.im * b)} : f2{0.f, 0.f};
  }
}

__device__ __forceinline__ f2 cf_at(const Dims& d, const f2* Cf, int e, int s, long long row) {
  return Cf[((long long)e * 27 + s) * d.N + row];
}

// Two-ended elimination.  The layers 0..k-1 are eliminated upwards from
// layer 0 (chain 0) while the layers nz-1..k+1 are eliminated downwards from
// layer nz-1 (chain 1), in the same launches; the middle layer k is then
// eliminated last with both neighbours' complements (a "twisted" block
// factorisation: the dependent chain of layer steps halves).  The kernels
// see 2 Ne virtual nodes: v < Ne is node v on chain 0, v >= Ne node v - Ne on
// chain 1.  Chain 0's previous layer is layer - 1 (couplings in the dz = -1
// slots 0..8), chain 1's is layer + 1 (slots 18..26); by the symmetry of
// M_e, the coupling back to a chain's next layer is the transpose.
// k = nz - 1 (chain 1 empty) is the plain one-ended elimination.
struct Chains {
  int Ne;          // real nodes
  int layer[2];    // layer of each chain in this step
  int rplane[2];   // ping-pong plane holding each chain's previous complement
  int wplane;      // plane written in this step
};
__device__ __forceinline__ int chain_of(const Chains& c, int v) { return v >= c.Ne ? 1 : 0; }
__device__ __forceinline__ int node_of(const Chains& c, int v) { return v >= c.Ne ? v - c.Ne : v; }
// first stencil slot of the coupling from a chain's layer to its previous layer
__device__ __forceinline__ int prev_slot(int chain) { return chain ? 18 : 0; }

// ------------------------------------------------------------------ Schur
// The fp32 working copies of S_i / S'_i live in a two-plane ping-pong buffer
// F[v][plane] per virtual node: the recursion only ever needs the previous
// layer of its chain.
// In-plane neighbour t (dx = t % 3 - 1, dy = t / 3 - 1) of grid row p as an
// offset, 0 where it falls outside the cross-section: its coupling
// coefficient is zero there, and reading the row itself keeps the load in
// bounds without a branch, so that all taps' loads are independent.
__device__ __forceinline__ int tap_offset(const Dims& d, int p, int t) {
  const int px = p % d.nx, py = p / d.nx;
  const int dx = t % 3 - 1, dy = t / 3 - 1;
  const bool ok = (dx < 0 ? px > 0 : (dx > 0 ? px + 1 < d.nx : true)) &&
                  (dy < 0 ? py > 0 : (dy > 0 ? py + 1 < d.ny : true));
  return ok ? dx + d.nx * dy : 0;
}

constexpr int kSchurRows = 8;   // rows a of S' per thread of k_mx_schur1

// T1[v][a, q] = sum_b S'[a, b] C[q, b] (row-split, fp32), C = the coupling of
// the chain's layer to its previous layer (v = blockIdx.z).  A thread takes
// column q of kSchurRows consecutive rows a and loads q's 9 coefficients once.
__global__ void __launch_bounds__(256) k_mx_schur1(Dims d, Chains ch, const f2* __restrict__ Cf,
                                                   const float* __restrict__ F, float* __restrict__ T1) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int a0 = blockIdx.y * kSchurRows, v = blockIdx.z;
  if (q >= d.n) return;
  const int c = chain_of(ch, v), e = node_of(ch, v);
  const long long rowq = (long long)ch.layer[c] * d.n + q;
  f2 cv[9];
  int b[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    cv[t] = cf_at(d, Cf, e, prev_slot(c) + t, rowq);
    b[t] = q + tap_offset(d, q, t);
  }
  for (int r = 0; r < kSchurRows; ++r) {
    const int a = a0 + r;
    if (a >= d.n) break;
    const float* S = F + (((long long)v * 2 + ch.rplane[c]) * d.n + a) * d.ldF;
    f2 acc{0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 9; ++t) f2fma(acc, f2{S[b[t]], S[d.n + b[t]]}, cv[t]);
    float* out = T1 + ((long long)v * d.n + a) * d.ldF;
    out[q] = acc.x;
    out[d.n + q] = acc.y;
  }
}

// S[p, q] = D[p, q] + sum_a C[p, a] T1[a, q] -> F (plane wplane of v), with
// C the coupling of v's layer to its previous layer (has_prev: 0 on a chain's
// first layer).  middle: v < Ne only; the middle layer takes both chains'
// contributions, C0 T1[v] + C1 T1[v + Ne] (the second when has_prev1).
// A thread takes column q of kSchur2Rows consecutive rows p: the nine taps of
// row p read T1 rows p + dx + nx dy, so per in-plane offset dy the thread
// keeps a window of the three rows p - 1, p, p + 1 and loads one new row per
// step (3 loads per output instead of 9).  A tap outside the grid has a zero
// coefficient; its window entry is T1's own (finite) value, or zero beyond
// the layer.
constexpr int kSchur2Rows = 32;
__global__ void __launch_bounds__(256) k_mx_schur2(Dims d, Chains ch, int has_prev, int middle, int has_prev1,
                                                   const f2* __restrict__ Cf, const float* __restrict__ T1,
                                                   float* __restrict__ F) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p0 = blockIdx.y * kSchur2Rows, v = blockIdx.z;
  if (q >= d.n) return;
  const int c = chain_of(ch, v), e = node_of(ch, v);
  const int n = d.n, nx = d.nx;
  const int qx = q % nx, qy = q / nx;
  const int p1 = min(n, p0 + kSchur2Rows);
  auto load = [&](const float* T, int a) {
    return (a >= 0 && a < n) ? f2{T[(long long)a * d.ldF + q], T[(long long)a * d.ldF + n + q]} : f2{0.f, 0.f};
  };
  const bool two = middle && has_prev1;
  const float* Ta = T1 + (long long)v * n * d.ldF;
  const float* Tb = T1 + (long long)(v + ch.Ne) * n * d.ldF;
  // windows w[source][dy + 1][dx + 1] = T1[p + dx + nx dy][q]
  f2 wa[3][3], wb[3][3];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int a = p0 - 1 + dx + nx * (dy - 1);   // rows p0 - 1 and p0 of band dy
      wa[dy][dx + 1] = has_prev ? load(Ta, a) : f2{0.f, 0.f};
      wb[dy][dx + 1] = two ? load(Tb, a) : f2{0.f, 0.f};
    }
  for (int p = p0; p < p1; ++p) {
    const long long rowp = (long long)ch.layer[c] * n + p;
    // slide: the windows move to rows p - 1, p, p + 1 of each band
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      wa[dy][0] = wa[dy][1];
      wa[dy][1] = wa[dy][2];
      wb[dy][0] = wb[dy][1];
      wb[dy][1] = wb[dy][2];
      const int a = p + 1 + nx * (dy - 1);
      wa[dy][2] = has_prev ? load(Ta, a) : f2{0.f, 0.f};
      wb[dy][2] = two ? load(Tb, a) : f2{0.f, 0.f};
    }
    const int px = p % nx, py = p / nx;
    f2 acc{0.f, 0.f};
    const int ddx = qx - px, ddy = qy - py;
    if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) acc = cf_at(d, Cf, e, 9 + (ddy + 1) * 3 + (ddx + 1), rowp);
    if (has_prev) {
#pragma unroll
      for (int t = 0; t < 9; ++t) f2fma(acc, cf_at(d, Cf, e, prev_slot(c) + t, rowp), wa[t / 3][t % 3]);
    }
    if (two) {
#pragma unroll
      for (int t = 0; t < 9; ++t) f2fma(acc, cf_at(d, Cf, e, prev_slot(1) + t, rowp), wb[t / 3][t % 3]);
    }
    float* out = F + (((long long)v * 2 + ch.wplane) * n + p) * d.ldF;
    out[q] = acc.x;
    out[n + q] = acc.y;
  }
}

// ------------------------------------------------------------------ panel

// In-place output of a diagonal block of the recursive inversion:
// -S[K,K]^{-1} back into the block of F and, for a block that no later step
// changes, its split bf16 pairs into the layer's solve operand Fr.
struct LeafOut {
  float* F = nullptr;
  float* Fr = nullptr;
  Chains ch{};
  int nz = 0;
};

// 1/a for complex fp32 with scaling, from approximate reciprocals (a couple
// of ulp, far below the 2^-17 of the split bf16 pairs the factors are used
// as): on the panel
// inverse's critical path every pivot waits for one of these.
__device__ __forceinline__ f2 f2inv_fast(f2 a) {
  const float rs = __fdividef(1.0f, fmaxf(fabsf(a.x), fabsf(a.y)));
  const float x = a.x * rs, y = a.y * rs;
  const float dinv = __fdividef(1.0f, x * x + y * y);
  return f2{x * dinv * rs, -y * dinv * rs};
}

// Pinv = S[K,K]^{-1} for panel K = [k0, k0+bw) of every node (one CTA per
// node): the Gauss-Jordan sweep of the 64 x 64 diagonal block (fp32, padded
// with the identity when bw < 64), one pivot at a time:
//   p = P[k,k];  P[i,j] -= P[i,k] P[k,j] / p  (i, j != k);
//   P[k,j] /= p;  P[i,k] /= p;  P[k,k] = -1/p,
// after which P = -S[K,K]^{-1}.  After each pivot the holders of the next
// pivot's row and column publish them to shared memory (double-buffered by
// pivot parity) and the holder of the next pivot publishes its reciprocal, so
// one block barrier per pivot suffices and the reciprocal is formed once.
// Every thread applies the rank-1 update to its entries, the pivot column
// through the same FMAs (its entries are cleared when published and the
// multiplier there is -1/p); the pivot row is then overwritten.  The 64 pivots
// are the kernel's critical path.
// Layout: thread t holds column j = t % 64 of the RPT consecutive rows
// h RPT + a (a < RPT), h = t / 64, so a CTA has 64 * (64 / RPT) threads.  Per
// pivot a thread reads the pivot's reciprocal, its own entry of the pivot row
// and the RPT entries of the pivot column that its rows need (a warp-wide
// broadcast, two complex values per 16-byte load), and applies RPT complex
// FMAs.  The pivot loop is unrolled within a row block so that every register
// index is a compile-time constant.  RPT = 16 (256 threads) measured fastest:
// 32 rows per thread leaves one warp per scheduler to hide every latency.
template <int RPT>
__global__ void __launch_bounds__(kPanel * (kPanel / RPT)) k_mx_pinv(Dims d, int plane, int k0, int bw,
                                                                         const float* F, f2* __restrict__ PinvOut,
                                                                         int* status, LeafOut lo) {
  constexpr int H = kPanel / RPT;   // row blocks
  static_assert(RPT % 2 == 0 && kPanel % RPT == 0, "rows per thread");
  __shared__ __align__(16) f2 rowb[2][kPanel];   // row k of P before pivot k
  __shared__ __align__(16) f2 colb[2][kPanel];   // column k of P before pivot k
  __shared__ f2 invb[2];                         // 1 / P[k, k] before pivot k
  __shared__ int bad;
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  const int j = tid % kPanel, h = tid / kPanel;
  const int n = d.n;
  const float* Fl = F + ((long long)e * 2 + plane) * n * d.ldF;
  if (tid == 0) bad = 0;
  f2 v[RPT];
#pragma unroll
  for (int a = 0; a < RPT; ++a) {
    const int i = h * RPT + a;
    f2 x{(i == j) ? 1.f : 0.f, 0.f};
    if (i < bw && j < bw) {
      const float* row = Fl + (long long)(k0 + i) * d.ldF;
      x = f2{row[k0 + j], row[n + k0 + j]};
    }
    v[a] = x;
  }
  __syncthreads();   // `bad` initialised
  // publish pivot kn = hb RPT + idx (idx a compile-time constant after
  // unrolling): its row from the row block hb, its reciprocal from its
  // holder, its column (cleared afterwards, as described above) from column kn
  auto publish = [&](int hb, int idx, int kn, int buf) {
    if (h == hb) {
      const f2 x = v[idx];
      rowb[buf][j] = x;
      if (j == kn) {
        const float mag = fabsf(x.x) + fabsf(x.y);
        const bool good = mag > 0.f && isfinite(mag);
        if (!good) bad = 1;
        invb[buf] = good ? f2inv_fast(x) : f2{0.f, 0.f};
      }
    }
    if (j == kn) {
#pragma unroll
      for (int a = 0; a < RPT; a += 2) {
        *reinterpret_cast<float4*>(&colb[buf][h * RPT + a]) = make_float4(v[a].x, v[a].y, v[a + 1].x, v[a + 1].y);
        v[a] = f2{0.f, 0.f};
        v[a + 1] = f2{0.f, 0.f};
      }
    }
  };
  publish(0, 0, 0, 0);
  __syncthreads();
#pragma unroll 1
  for (int hk = 0; hk < H; ++hk) {
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk) {
      const int k = hk * RPT + kk;
      const int b = k & 1;
      const f2 inv = invb[b];
      const f2 rki = f2mul(rowb[b][j], inv);   // P[k, j] / p
      const f2 r = (j == k) ? f2{-inv.x, -inv.y} : rki;
#pragma unroll
      for (int a = 0; a < RPT; a += 2) {
        const float4 c2 = *reinterpret_cast<const float4*>(&colb[b][h * RPT + a]);
        v[a].x = fmaf(-c2.x, r.x, v[a].x);
        v[a].x = fmaf(c2.y, r.y, v[a].x);
        v[a].y = fmaf(-c2.x, r.y, v[a].y);
        v[a].y = fmaf(-c2.y, r.x, v[a].y);
        v[a + 1].x = fmaf(-c2.z, r.x, v[a + 1].x);
        v[a + 1].x = fmaf(c2.w, r.y, v[a + 1].x);
        v[a + 1].y = fmaf(-c2.z, r.y, v[a + 1].y);
        v[a + 1].y = fmaf(-c2.w, r.x, v[a + 1].y);
      }
      // pivot row: P[k, j] = P[k, j] / p, and P[k, k] = -1 / p
      if (h == hk) v[kk] = (j == k) ? f2{-inv.x, -inv.y} : rki;
      if (k + 1 < kPanel) {
        if (kk + 1 < RPT) publish(hk, kk + 1, k + 1, b ^ 1);
        else publish(hk + 1, 0, k + 1, b ^ 1);
      }
      __syncthreads();
    }
  }
  // P holds -S[K,K]^{-1}
  if (PinvOut) {
#pragma unroll
    for (int a = 0; a < RPT; ++a) {
      const int i = h * RPT + a;
      PinvOut[(long long)e * kPanel * kPanel + i * kPanel + j] = f2{-v[a].x, -v[a].y};
    }
  }
  if (lo.F) {
    float* Fw = lo.F + ((long long)e * 2 + plane) * n * d.ldF;
    float* Frw = lo.Fr ? lo.Fr + ((long long)node_of(lo.ch, e) * lo.nz + lo.ch.layer[chain_of(lo.ch, e)]) * n * d.ldF
                       : nullptr;
#pragma unroll
    for (int a = 0; a < RPT; ++a) {
      const int i = h * RPT + a;
      if (i < bw && j < bw) {
        const long long at = (long long)(k0 + i) * d.ldF + k0 + j;
        Fw[at] = v[a].x;
        Fw[at + n] = v[a].y;
        if (Frw) {
          float* frow = Frw + (long long)(k0 + i) * d.ldF;
          tc::store_pair(frow, k0 + j, v[a].x);
          tc::store_pair(frow, n + k0 + j, v[a].y);
        }
      }
    }
  }
  if (tid == 0 && bad) atomicExch(status, (int)DEV_PIVOT);
}

#ifndef FEAST_FACTOR_RECURSIVE
#define FEAST_FACTOR_RECURSIVE 0
#endif
// 1: invert the layer complements by the recursive block inversion where it
// applies; 0 (default): the 64-column panel sweep.  Measured on the
// 32x32x400 pencil the recursion's products (long K, operands such as
// Abar B that carry no cancellation from earlier panels) lose accuracy
// against the panel sweep's rank-64 updates of partially eliminated columns:
// the refinement then needs about a third more steps, more than the factor
// saves.
constexpr bool kFactorPanelSweep = FEAST_FACTOR_RECURSIVE == 0;

#ifndef FEAST_WIDE_STAGES
#define FEAST_WIDE_STAGES 1
#endif
// pipeline stages of the wide sweep update (1: two CTAs per SM)
constexpr int kWideStages = FEAST_WIDE_STAGES;
#ifndef FEAST_NARROW_STAGES
#define FEAST_NARROW_STAGES 1
#endif
// pipeline stages of the narrow update (the next panel's column tile).  One
// stage (about 97 KB of shared memory) leaves room on its SM for a CTA of the
// concurrent wide update, which is the factor's critical path; with four the
// narrow update is 3 us faster but the wide update loses those SMs.
constexpr int kNarrowStages = FEAST_NARROW_STAGES;

#ifndef FEAST_PINV_RPT
#define FEAST_PINV_RPT 16
#endif
constexpr int kPinvRpt = FEAST_PINV_RPT;   // rows per thread of the panel inverse

#ifndef FEAST_FACTOR_KIND
#define FEAST_FACTOR_KIND 2
#endif
// Operand kind of the sweep updates (k_tc_gemm KIND): 2, split bf16 pairs
// (default); 0, TF32.
constexpr int kFactorKind = FEAST_FACTOR_KIND;
static_assert(kFactorKind == 0 || kFactorKind == 2, "sweep-update operand kind");

// K-column kcol of a sweep-update operand row, in the operand kind's layout.
__device__ __forceinline__ void store_factor_op(float* row, int kcol, float x) {
  if constexpr (kFactorKind == 2)
    tc::store_pair(row, kcol, x);
  else
    row[kcol] = tc::to_tf32(x);
}

// For panel K and this CTA's kRowsPerPanelCta rows i:  T[i, :] = S[i, K] Pinv  and
// L[i, :] = S[i, K], written as the sweep updates' GEMM operands (split bf16
// pairs, or TF32-rounded)  Aop = [Tr | Ti] (row i) and Bop (embedded L, rows
// in blocks of 64 complex columns: 64 rows [Lr, -Li] then 64 rows
// [Li, Lr]), and in fp32 as Tc.
__global__ void __launch_bounds__(256) k_mx_panel_T(Dims d, int plane, int k0, int bw, const float* __restrict__ F,
                                                    const f2* __restrict__ PinvIn, float* __restrict__ Aop,
                                                    float* __restrict__ Bop, f2* __restrict__ Tc) {
  // unpadded: the accesses below are consecutive along the second index or
  // warp-wide broadcasts, so no bank conflicts (and 32 rows fit in 48 KB)
  __shared__ f2 Ps[kPanel][kPanel];
  __shared__ f2 Ls[kRowsPerPanelCta][kPanel];
  const int e = blockIdx.y;
  const int r0 = blockIdx.x * kRowsPerPanelCta;
  const int tid = threadIdx.x;
  const int n = d.n;
  const float* Fl = F + ((long long)e * 2 + plane) * n * d.ldF;
  const f2* Pin = PinvIn + (long long)e * kPanel * kPanel;
  for (int t = tid; t < kPanel * kPanel; t += 256) Ps[t / kPanel][t % kPanel] = Pin[t];
  for (int t = tid; t < kRowsPerPanelCta * kPanel; t += 256) {
    const int r = t / kPanel, m = t % kPanel;
    const int i = r0 + r;
    f2 x{0.f, 0.f};
    if (i < n && m < bw) {
      const float* row = Fl + (long long)i * d.ldF;
      x = f2{row[k0 + m], row[n + k0 + m]};
    }
    Ls[r][m] = x;
  }
  __syncthreads();
  // thread -> columns c and c + 32, rows r0 + rq + 8q (q < kRowsPerPanelCta
  // / 8): per m two Pinv loads (32 consecutive entries a warp) and one L
  // broadcast per row feed four complex FMAs
  constexpr int kRowsPerThread = kRowsPerPanelCta / 8;
  const int c = tid % 32, rq = tid / 32;
  f2 acc[kRowsPerThread][2];
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) acc[q][0] = acc[q][1] = f2{0.f, 0.f};
#pragma unroll 8
  for (int m = 0; m < kPanel; ++m) {
    const f2 pv0 = Ps[m][c], pv1 = Ps[m][c + 32];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const f2 l = Ls[rq + 8 * q][m];
      f2fma(acc[q][0], l, pv0);
      f2fma(acc[q][1], l, pv1);
    }
  }
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int r = rq + 8 * q;
    const int i = r0 + r;
    if (i >= n) continue;
    float* arow = Aop + ((long long)e * n + i) * (2 * kPanel);
    const long long brow = ((long long)e * d.nblk64 + i / 64) * 128 + (i % 64);
    float* bre = Bop + brow * (2 * kPanel);
    float* bim = Bop + (brow + 64) * (2 * kPanel);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int cc = c + 32 * h;
      store_factor_op(arow, cc, acc[q][h].x);
      store_factor_op(arow, kPanel + cc, acc[q][h].y);
      Tc[((long long)e * n + i) * kPanel + cc] = acc[q][h];
      const f2 l = Ls[r][cc];
      store_factor_op(bre, cc, l.x);
      store_factor_op(bre, kPanel + cc, -l.y);
      store_factor_op(bim, cc, l.y);
      store_factor_op(bim, kPanel + cc, l.x);
    }
  }
}

// ------------------------------------------------------------------ epilogues
constexpr int kStageLd = tc::kBlockM + 1;   // staging row stride (floats): conflict-free both ways

// Sweep trailing update on tile (rows tm*128.., complex columns tn*64..):
//   i, j outside K:  S[i, j] -= acc[i, j]
//   i in K, j not:   S[i, j]  = T[j, i - k0]
//   j in K, i not:   S[i, j]  = T[i, j - k0]
//   both in K:       S[i, j]  = -Pinv[i - k0, j - k0]
// The last panel writes every entry of the finished S'_i, so it also stores
// the split bf16 pairs that the block solves read.
// The accumulator goes through shared memory (one half, real or imaginary,
// at a time) so that the read-modify-write of S is coalesced along rows.
struct SweepEpi {
  float* F;        // row-split fp32 working copy of the layer being swept, virtual-node stride sF floats
  long long sF;
  float* Fr;       // last panel only: split bf16 pairs of the finished S' (solve operand), node stride sFr
  long long sFr;
  int ldF, n, k0, bw;
  const f2* Tc;    // n x 64 per virtual node
  const f2* Pinv;  // 64 x 64 per virtual node
  Chains ch;       // which node and layer virtual node e is
  __device__ void operator()(int e, int tm, int tn, int row, uint32_t taddr, int ept, uint8_t* stage) const {
    float* Sg = reinterpret_cast<float*>(stage);   // 64 columns x kStageLd
    float* Fe = F + e * sF;
    float* Fre = Fr ? Fr + node_of(ch, e) * sFr + (long long)ch.layer[chain_of(ch, e)] * n * ldF : nullptr;
    const f2* T = Tc + (long long)e * n * kPanel;
    const f2* Pi = Pinv + (long long)e * kPanel * kPanel;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + half * 64 + c0, v);
#pragma unroll
        for (int t = 0; t < 16; ++t) Sg[(c0 + t) * kStageLd + row] = v[t];
      }
      tc::epilogue_sync();
      const int cc = ept % 64;
      const int j = tn * 64 + cc;
      const bool inJ = j >= k0 && j < k0 + bw;
      const bool jok = j < n;
      // rows ept/64, +2, +4, ...: 16 independent loads in flight per thread
#pragma unroll 1
      for (int base = ept / 64; base < tc::kBlockM; base += 32) {
        float cur[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int i = tm * tc::kBlockM + base + 2 * u;
          const bool inI = i >= k0 && i < k0 + bw;
          cur[u] = (jok && i < n && !inI && !inJ) ? Fe[(long long)i * ldF + half * n + j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int rr = base + 2 * u;
          const int i = tm * tc::kBlockM + rr;
          if (!jok || i >= n) continue;
          const bool inI = i >= k0 && i < k0 + bw;
          float val;
          if (!inI && !inJ) {
            val = cur[u] - Sg[cc * kStageLd + rr];
          } else if (inI && !inJ) {
            const f2 t2 = T[(long long)j * kPanel + (i - k0)];
            val = half ? t2.y : t2.x;
          } else if (!inI && inJ) {
            const f2 t2 = T[(long long)i * kPanel + (j - k0)];
            val = half ? t2.y : t2.x;
          } else {
            const f2 p2 = Pi[(i - k0) * kPanel + (j - k0)];
            val = -(half ? p2.y : p2.x);
          }
          Fe[(long long)i * ldF + half * n + j] = val;
          if (Fre) tc::store_pair(Fre + (long long)i * ldF, half * n + j, val);
        }
      }
      tc::epilogue_sync();
    }
  }
};

// The same trailing update with the read-modify-write of S staged through
// shared memory by TMA (used when n is a multiple of 64, so that a tile's 64
// complex columns never straddle the real/imaginary split of a row).  The
// epilogue threads load the CTA's S tile -- four 128-row x 32-column boxes:
// real parts of columns tn*64.. and imaginary parts n + tn*64.. -- at kernel
// start, so the load overlaps the main loop; each thread then updates its row
// in shared memory (128-byte swizzle: chunk c of row r sits at c ^ (r & 7)) and
// one thread stores the tile back with TMA (and, after the last panel, the
// solve copy as split bf16 pairs).  The 3-D maps (row, layer plane) clip every box at the
// layer's n rows.
struct SweepEpiTma {
  // the S tile goes through shared memory in two column halves of 32
  // complex columns (a real-part and an imaginary-part box of 16 KB each):
  // 32 KB instead of 64 lets three CTAs share an SM
  static constexpr size_t kTileBytes = 2 * 16384;
  static constexpr size_t kExtraSmem = kTileBytes + 64;
  CUtensorMap mapF;    // fp32 working layers: inner 2n, rows n, planes 2 per virtual node
  CUtensorMap mapFr;   // solve copy (split bf16 pairs, fp32-sized rows): inner 2n, rows n, planes Ne*nz
  int plane;           // working plane of this step
  Chains ch;           // which node and layer virtual node e is
  int nz;
  int n, k0, bw;
  int last;            // last panel: also store the solve copy
  const f2* Tc;
  const f2* Pinv;
  // box of column half hc: real parts (part 0) or imaginary parts (part 1)
  __device__ int box_x(int part, int hc, int tn) const { return part * n + tn * 64 + hc * 32; }
  __device__ void load_half(int hc, int e, int tm, int tn, uint8_t* extra, uint64_t* bar) const {
    tc::mbar_arrive_expect_tx(bar, (uint32_t)kTileBytes);
#pragma unroll
    for (int part = 0; part < 2; ++part)
      tc::tma_load_3d(extra + part * 16384, &mapF, bar, box_x(part, hc, tn), tm * tc::kBlockM, e * 2 + plane);
  }
  __device__ void prologue(int e, int tm, int tn, int ept, uint8_t* extra, int*, volatile int*) const {
    if (ept != 0) return;
    uint64_t* bar = reinterpret_cast<uint64_t*>(extra + kTileBytes);
    tc::mbar_init(bar, 1);
    tc::fence_barrier_init();
    load_half(0, e, tm, tn, extra, bar);
  }
  __device__ void run(int e, int tm, int tn, int row, uint32_t taddr, int ept, uint8_t* stage, uint8_t* extra,
                      int* status, volatile int* abort_flag) const {
    uint64_t* bar = reinterpret_cast<uint64_t*>(extra + kTileBytes);
    const f2* T = Tc + (long long)e * n * kPanel;
    const f2* Pi = Pinv + (long long)e * kPanel * kPanel;
    const int i = tm * tc::kBlockM + row;
    const bool iok = i < n;
    const bool inI = i >= k0 && i < k0 + bw;
    const int sw = row & 7;
    const bool strip = tn * 64 == k0;   // the panel's own columns: every entry is T or -Pinv
    const bool rowsK = tm * tc::kBlockM < k0 + bw && k0 < tm * tc::kBlockM + tc::kBlockM;
    // pivot rows of this tile: S[i, j] = T[j, i - k0], staged in shared
    // memory (the free pipeline stage) with coalesced loads
    f2* Ts = reinterpret_cast<f2*>(stage);   // [64 columns j][64]
    if (!strip && rowsK) {
      const float4* src = reinterpret_cast<const float4*>(T + (long long)tn * 64 * kPanel);
      float4* dstp = reinterpret_cast<float4*>(Ts);
      const int rows_avail = min(64, n - tn * 64);
      for (int t = ept; t < 64 * kPanel / 2; t += 128)
        dstp[t] = (t / (kPanel / 2) < rows_avail) ? src[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll 1
    for (int hc = 0; hc < 2; ++hc) {
      // bounded wait for this half (phase hc), also when the main loop gave
      // up, so that no copy into shared memory is in flight when the CTA exits
      bool ok = false;
      for (long long it = 0; it < tc::kWaitLimit && !ok; ++it) ok = tc::mbar_try_wait(bar, (uint32_t)hc);
      if (!ok) {
        *abort_flag = 1;
        atomicExch(status, (int)DEV_TIMEOUT);
      }
      tc::epilogue_sync();   // also: Ts staged
      if (*abort_flag) {   // uniform: read after the barrier
        if (ept == 0) tc::bulk_wait();   // the first half's stores, if any
        return;
      }
#pragma unroll 1
      for (int c0 = hc * 32; c0 < hc * 32 + 32; c0 += 16) {
        const int q0 = (c0 & 31) >> 2;
        if (strip) {
          // row i: T[i, :] (or -Pinv[i - k0, :] on the pivot rows), 16 columns at a time
          f2 val[16];
          if (iok) {
            const float4* src = reinterpret_cast<const float4*>(inI ? Pi + (long long)(i - k0) * kPanel + c0
                                                                    : T + (long long)i * kPanel + c0);
            float4 q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) q[u] = src[u];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              val[2 * u] = f2{q[u].x, q[u].y};
              val[2 * u + 1] = f2{q[u].z, q[u].w};
            }
            if (inI)
#pragma unroll
              for (int t = 0; t < 16; ++t) val[t] = f2{-val[t].x, -val[t].y};
          } else {
#pragma unroll
            for (int t = 0; t < 16; ++t) val[t] = f2{0.f, 0.f};
          }
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            float4* rowp = reinterpret_cast<float4*>(extra + part * 16384 + row * 128);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              float4 x;
              x.x = part ? val[qq * 4].y : val[qq * 4].x;
              x.y = part ? val[qq * 4 + 1].y : val[qq * 4 + 1].x;
              x.z = part ? val[qq * 4 + 2].y : val[qq * 4 + 2].x;
              x.w = part ? val[qq * 4 + 3].y : val[qq * 4 + 3].x;
              rowp[(q0 + qq) ^ sw] = x;
            }
          }
        } else {
#pragma unroll 1
          for (int part = 0; part < 2; ++part) {
            float v[16];
            tc::tmem_ld16(taddr + part * 64 + c0, v);
            float4* rowp = reinterpret_cast<float4*>(extra + part * 16384 + row * 128);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              float4 cur = rowp[(q0 + qq) ^ sw];
              float* cv = reinterpret_cast<float*>(&cur);
#pragma unroll
              for (int t4 = 0; t4 < 4; ++t4) {
                const int t = qq * 4 + t4;
                if (inI) {
                  const f2 t2 = Ts[(c0 + t) * kPanel + (i - k0)];
                  cv[t4] = part ? t2.y : t2.x;
                } else {
                  cv[t4] -= v[t];
                }
              }
              rowp[(q0 + qq) ^ sw] = cur;
            }
          }
        }
      }
      tc::fence_proxy_async_smem();
      tc::epilogue_sync();
      if (ept == 0) {
#pragma unroll
        for (int part = 0; part < 2; ++part)
          tc::tma_store_3d(&mapF, extra + part * 16384, box_x(part, hc, tn), tm * tc::kBlockM, e * 2 + plane);
        tc::bulk_commit();
        tc::bulk_wait_read();
      }
      if (last) {
        tc::epilogue_sync();   // the working-copy stores have read the half
        // each box row (32 K-columns, 16-byte chunk c at c ^ sw) becomes its
        // split bf16 pairs: chunks 0-3 the leading parts, 4-7 the trailing
#pragma unroll 1
        for (int part = 0; part < 2; ++part) {
          uint4* rowp = reinterpret_cast<uint4*>(extra + part * 16384 + row * 128);
          float x[32];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 u = rowp[c ^ sw];
            x[4 * c] = __uint_as_float(u.x);
            x[4 * c + 1] = __uint_as_float(u.y);
            x[4 * c + 2] = __uint_as_float(u.z);
            x[4 * c + 3] = __uint_as_float(u.w);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint4 h, l;
            tc::split2(x[8 * c], x[8 * c + 1], h.x, l.x);
            tc::split2(x[8 * c + 2], x[8 * c + 3], h.y, l.y);
            tc::split2(x[8 * c + 4], x[8 * c + 5], h.z, l.z);
            tc::split2(x[8 * c + 6], x[8 * c + 7], h.w, l.w);
            rowp[c ^ sw] = h;
            rowp[(4 + c) ^ sw] = l;
          }
        }
        tc::fence_proxy_async_smem();
        tc::epilogue_sync();
        if (ept == 0) {
#pragma unroll
          for (int part = 0; part < 2; ++part)
            tc::tma_store_3d(&mapFr, extra + part * 16384, box_x(part, hc, tn), tm * tc::kBlockM,
                             node_of(ch, e) * nz + ch.layer[chain_of(ch, e)]);
          tc::bulk_commit();
          tc::bulk_wait_read();
        }
      }
      if (hc == 0) {
        // the stores have read the first half (thread 0 waited above): the
        // second half reuses its shared memory
        tc::epilogue_sync();
        if (ept == 0) load_half(1, e, tm, tn, extra, bar);
      }
    }
    if (ept == 0) tc::bulk_wait();
  }
};

// fp32 -> fp64 through the bit fields (IEEE 754 binary32 -> binary64:
// exponent rebiased by 1023 - 127, mantissa shifted by 29), on the integer
// pipe: the FP64 refinement residual converts 54 values per complex entry,
// and a float-to-double conversion instruction would take an FP64-pipe slot
// each.  Exact for zero and normal numbers; an fp32 subnormal (|x| < 2^-126)
// becomes a signed zero, infinities and NaNs stay infinities and NaNs.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xFFu;
  const unsigned e64 = ex == 0xFFu ? 0x7FFu : ex + (1023u - 127u);
  const unsigned hi = (u & 0x80000000u) | (ex ? (e64 << 20) | ((u >> 3) & 0xFFFFFu) : 0u);
  const unsigned lo = ex ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// fp64 -> fp32 by truncation of the mantissa, on the integer pipe: for the
// complex64 copy of the FP64 refinement residual (whose FP64 pipe is its
// bound): the truncated value is the leading part of the resident residual
// pair, whose trailing part takes the remainder (so the pair still holds R
// to about 2^-47), and it feeds the next correction's right-hand side as
// split bf16 pairs (16 bits), where a one-ulp truncation is immaterial.  (The
// double-float residual and the couplings keep the conversion instructions:
// they are bound by instruction issue, where the integer sequence costs more.)  Magnitudes below 2^-126 become a signed
// zero, above the fp32 range an infinity; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7FFu);
  if (ex == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((hi & 0xFFFFFu) | lo ? 0x400000u : 0u));
  const int e32 = ex - (1023 - 127);
  if (e32 <= 0) return __uint_as_float(sign);
  if (e32 >= 0xFF) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e32 << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// Solve product: out[m*ldo + p] = alpha * (S' g)[p, m] (complex64); lanes are
// consecutive rows p, so the stores of a warp are contiguous.
// With qp set (the backward sweep of feast_solve / feast_quadrature) the
// epilogue also folds the layer's solution x into the node's share of the
// quadrature sum (Eq. 15):  qp[m*ldq + p] (= or +=) Re{coef_e x}  in FP64,
// coef_e = -(w_e/2) r e^{i theta_e}.  x of the first solve is Q_e itself and
// x of each refinement step is its correction, so after the last step the
// node's share is Re{coef_e Q_e}, without Q_e ever being stored.
template <int CB>
struct SolveEpi {
  f2* out;
  long long sOut, ldo;
  int n, k;
  float alpha;
  double* qp = nullptr;        // per-node quadrature partials
  long long sQ = 0, ldq = 0;   // node stride, column stride
  const cplx* coef = nullptr;  // Ne quadrature coefficients
  int qfirst = 0;              // 1: store (first solve), 0: accumulate (refinement)
  int share_chains = 3;        // chains (bit c) whose rows add their shares here
  // node_rows: out and qp belong to the real node of virtual node e, at the
  // rows of its chain's layer (the backward sweep); else out is per virtual
  // node (the forward products)
  int node_rows = 0;
  Chains ch{};
  __device__ long long base(int e, long long stride) const {
    return node_rows ? node_of(ch, e) * stride + (long long)ch.layer[chain_of(ch, e)] * n : e * stride;
  }
  // the old shares of this thread's row (a refinement step reads them back):
  // the first kPre columns are loaded while the main loop runs; a wider tile
  // loads each later group of 16 columns kPre columns ahead, inside the
  // epilogue loop, into the register slots the finished group frees
  static constexpr int kPre = CB <= 32 ? CB : 32;
  struct Pre {
    double q[kPre];
  };
  __device__ bool shares(int e) const { return qp && ((share_chains >> chain_of(ch, e)) & 1); }
  __device__ void prefetch(int e, int tm, int tn, int row, Pre& pre) const {
    const int p = tm * tc::kBlockM + row;
    const bool rd = shares(e) && !qfirst && p < n;
    const double* q = shares(e) ? qp + base(e, sQ) : nullptr;
#pragma unroll
    for (int t = 0; t < kPre; ++t) {
      const int m = tn * CB + t;
      pre.q[t] = (rd && m < k) ? q[(long long)m * ldq + p] : 0.0;
    }
  }
  __device__ void operator()(int e, int tm, int tn, int row, uint32_t taddr, int, uint8_t*, const Pre& pre) const {
    const int p = tm * tc::kBlockM + row;
    f2* o = out + base(e, sOut);
    double* q = shares(e) ? qp + base(e, sQ) : nullptr;
    const bool rd = q && !qfirst && p < n;
    cplx ce{0.0, 0.0};
    if (q) ce = coef[node_of(ch, e)];
    double ring[kPre];
#pragma unroll
    for (int t = 0; t < kPre; ++t) ring[t] = pre.q[t];
#pragma unroll
    for (int c0 = 0; c0 < CB; c0 += 16) {
      float re[16], im[16];
      tc::tmem_ld16(taddr + c0, re);
      tc::tmem_ld16(taddr + CB + c0, im);
      if (p >= n) continue;
      constexpr int kW = CB < 16 ? CB : 16;
      const int slot = c0 % kPre;
#pragma unroll
      for (int t = 0; t < kW; ++t) {
        const int m = tn * CB + c0 + t;
        if (m < k) {
          const f2 x{alpha * re[t], alpha * im[t]};
          o[(long long)m * ldo + p] = x;
          // two FP64 FMAs; the conversions run on the integer pipe
          if (q) q[(long long)m * ldq + p] = fma(ce.re, f32_to_f64(x.x), fma(-ce.im, f32_to_f64(x.y), ring[slot + t]));
        }
      }
      if (CB > kPre && c0 + kPre < CB) {
#pragma unroll
        for (int t = 0; t < kW; ++t) {
          const int m = tn * CB + c0 + kPre + t;
          ring[slot + t] = (rd && m < k) ? q[(long long)m * ldq + p] : 0.0;
        }
      }
    }
  }
};

// ------------------------------------------------------------------ recursive inversion
// The layer complement S (complex symmetric) is inverted in place by 2 x 2
// block elimination, S = [A B; B^T D] with the split at a multiple of 64:
//   Abar = -A^{-1} (recursively),        Xbar = Abar B,
//   D   <- D + Xbar^T B  (the Schur complement D - B^T A^{-1} B),
//   Sbar = -D^{-1} (recursively),        Ybar = Xbar Sbar,
//   -S^{-1} = [Abar + Ybar Xbar^T, Ybar; Ybar^T, Sbar],
// the diagonal blocks of 64 by the Gauss-Jordan sweep of k_mx_pinv.  Every
// product is a batched complex TF32 GEMM (tc::k_cgemm, C = U V^T) over the
// virtual nodes; its epilogue writes C transposed (lanes are rows of C, so
// the stores of a warp are contiguous) and/or as is, adds C^T into a
// symmetric block instead, and copies the blocks that no later step changes
// into the solve operand Fr (split bf16 pairs).  Blocks stay fp32 in F and the workspaces;
// the GEMM rounds its staged operands to TF32 (nearest).

// Destination of a row-split block: element (r, c) of batch b at
// base + b bstride + r ld + c (real part; imaginary part imoff further).
struct InvDest {
  float* base = nullptr;
  long long bstride = 0;
  int ld = 0, imoff = 0;
};

constexpr int kInvBN = 64;   // complex columns per CTA tile of the inversion GEMMs
#ifndef FEAST_INV_STAGES
#define FEAST_INV_STAGES 2
#endif
constexpr int kInvStages = FEAST_INV_STAGES;

struct InvEpi {
  InvDest t;           // C^T: element (j, i) <- C[i, j]
  InvDest r;           // C:   element (i, j) <- C[i, j]
  int add = 0;         // t += C^T instead of t = C^T
  int M = 0, N = 0;    // rows and columns of C
  // final blocks: split bf16 pair copies at offsets fr_t / fr_r (in fp32 units) of the layer's plane of
  // Fr (row stride ld_fr, imaginary parts imoff_fr further); fr == nullptr: none
  float* fr = nullptr;
  long long fr_t = -1, fr_r = -1;
  int ld_fr = 0, imoff_fr = 0;
  long long fr_plane = 0;
  Chains ch{};
  int nz = 0;
  __device__ void operator()(int b, int tm, int tn, int row, uint32_t taddr) const {
    const int i = tm * tc::kBlockM + row;
    float* frp = nullptr;
    if (fr) frp = fr + ((long long)node_of(ch, b) * nz + ch.layer[chain_of(ch, b)]) * fr_plane;
#pragma unroll 1
    for (int c0 = 0; c0 < kInvBN; c0 += 16) {
      float re[16], im[16];
      tc::cload16<kInvBN>(taddr, c0, re, im);   // warp-collective: before any exit
      const int j0 = tn * kInvBN + c0;
      if (i >= M || j0 >= N) continue;
      if (t.base) {
        float* tb = t.base + b * t.bstride + i;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int j = j0 + u;
          if (j < N) {
            float* p = tb + (long long)j * t.ld;
            float xr = re[u], xi = im[u];
            if (add) {
              xr += p[0];
              xi += p[t.imoff];
            }
            p[0] = xr;
            p[t.imoff] = xi;
            if (frp && fr_t >= 0) {
              const long long at = fr_t + (long long)j * ld_fr + i;   // row at / ld_fr, K-column at % ld_fr
              float* frow = frp + at / ld_fr * ld_fr;
              tc::store_pair(frow, (int)(at % ld_fr), xr);
              tc::store_pair(frow, (int)(at % ld_fr) + imoff_fr, xi);
            }
          }
        }
      }
      if (r.base) {
        float* p = r.base + b * r.bstride + (long long)i * r.ld + j0;
        // the solve copy's row and first K-column of this run of columns
        const long long qat = (frp && fr_r >= 0) ? fr_r + (long long)i * ld_fr + j0 : -1;
        float* qrow = qat >= 0 ? frp + qat / ld_fr * ld_fr : nullptr;
        const int qc = qat >= 0 ? (int)(qat % ld_fr) : 0;
        const uintptr_t al = reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(p + r.imoff);
        if (j0 + 16 <= N && (al & 15) == 0 && (qc & 3) == 0 && (imoff_fr & 3) == 0) {
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            *reinterpret_cast<float4*>(p + u) = make_float4(re[u], re[u + 1], re[u + 2], re[u + 3]);
            *reinterpret_cast<float4*>(p + r.imoff + u) = make_float4(im[u], im[u + 1], im[u + 2], im[u + 3]);
            if (qrow) {
              tc::store_pair4(qrow, qc + u, make_float4(re[u], re[u + 1], re[u + 2], re[u + 3]));
              tc::store_pair4(qrow, qc + imoff_fr + u, make_float4(im[u], im[u + 1], im[u + 2], im[u + 3]));
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (j0 + u < N) {
              p[u] = re[u];
              p[r.imoff + u] = im[u];
              if (qrow) {
                tc::store_pair(qrow, qc + u, re[u]);
                tc::store_pair(qrow, qc + imoff_fr + u, im[u]);
              }
            }
          }
        }
      }
    }
  }
};

// ------------------------------------------------------------------ couplings
// The nodes a sweep works on (bit e set: node e; all Ne nodes in the first
// solve, the unconverged ones in refinement steps): CTA z of every sweep
// kernel handles the node of the z-th set bit.
struct NodeList {
  int count;
  unsigned long long mask;
};

// Row of the embedded operand that holds the real parts of complex column m
// of virtual node e (the imaginary parts' row is CB further).  The
// kCoupleCols columns of a coupling thread lie in one CB block (CB is a
// multiple of kCoupleCols), so their rows are consecutive.
__device__ __forceinline__ long long emb_row(const Dims& d, int e, int m) {
  const long long blk = (long long)e * d.nblkCB + m / d.CB;
  return blk * 2 * d.CB + (m % d.CB);
}

// Writes the embedded RHS rows of the complex column whose real-part row is
// rre, as split bf16 pairs (the solve product's operand layout).
__device__ __forceinline__ void write_emb(const Dims& d, float* Bemb, long long rre, int p, f2 g) {
  float* re_row = Bemb + rre * d.ldB;
  float* im_row = Bemb + (rre + d.CB) * d.ldB;
  tc::store_pair(re_row, p, g.x);
  tc::store_pair(re_row, d.n + p, -g.y);
  tc::store_pair(im_row, p, g.y);
  tc::store_pair(im_row, d.n + p, g.x);
}

constexpr int kCoupleCols = 4;   // right-hand-side columns per thread of the coupling kernels

// forward: g = R + C t on a chain's layer, t = S'_prev g_prev the product
// of the chain's previous step (has_prev: 0 on a chain's first layer).  R is
// the real RHS (Rreal) or the complex64 residual of the node (Rc).  middle
// (chain-0 virtual nodes only): the middle layer adds both chains' products,
// C0 Tout[v] + C1 Tout[v + Ne] (the second when has_prev1).  A thread takes
// row p of kCoupleCols columns m and loads the row's taps once; CTA z
// handles the virtual node of the z-th set bit of nl.mask.  g goes to the
// node's solution column, its embedded copy to the virtual node's GEMM
// operand.
// kTwo: the middle layer with both chains' products (a second set of taps).
template <bool kTwo>
__global__ void __launch_bounds__(128) k_mx_couple_fwd(Dims d, Chains ch, int has_prev, int middle, int has_prev1,
                                                       const f2* __restrict__ Cf, const double* __restrict__ Rreal,
                                                       const f2* __restrict__ Rc, const f2* __restrict__ Tout,
                                                       f2* __restrict__ Gc, float* __restrict__ Bemb, NodeList nl,
                                                       const int* __restrict__ active) {
  tc::grid_dep_wait();   // under programmatic dependent launch: the previous product is complete
  tc::grid_dep_launch_dependents();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = blockIdx.y * kCoupleCols, v = tc::nth_set_bit(nl.mask, (int)blockIdx.z);
  if (p >= d.n) return;
  const int c = chain_of(ch, v), e = node_of(ch, v);
  if (active && !active[e]) return;   // a node the device-side refinement left out
  const long long row = (long long)ch.layer[c] * d.n + p;
  const long long sG = d.N * d.k;
  // branch-free taps: an in-plane neighbour outside the grid has a zero
  // coefficient and is read at offset 0 (the row itself) to stay in bounds
  int off[9];
  f2 c0[9], c1[kTwo ? 9 : 1];
  const bool two = kTwo && middle && has_prev1;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    off[t] = p + tap_offset(d, p, t);
    c0[t] = has_prev ? Cf[((long long)e * 27 + prev_slot(c) + t) * d.N + row] : f2{0.f, 0.f};
    if constexpr (kTwo) c1[t] = two ? Cf[((long long)e * 27 + prev_slot(1) + t) * d.N + row] : f2{0.f, 0.f};
  }
  // all columns' loads are independent: a column past k repeats column k - 1
  // (in bounds) and is not stored
  f2 g[kCoupleCols];
#pragma unroll
  for (int j = 0; j < kCoupleCols; ++j) {
    const int m = min(m0 + j, d.k - 1);
    g[j] = Rc ? Rc[e * sG + (long long)m * d.N + row] : f2{(float)Rreal[(long long)m * d.N + row], 0.f};
    if (has_prev) {
      const f2* T = Tout + ((long long)v * d.k + m) * d.n;
#pragma unroll
      for (int t = 0; t < 9; ++t) f2fma(g[j], c0[t], T[off[t]]);
    }
    if constexpr (kTwo) {
      if (two) {
        const f2* T = Tout + ((long long)(v + ch.Ne) * d.k + m) * d.n;
#pragma unroll
        for (int t = 0; t < 9; ++t) f2fma(g[j], c1[t], T[off[t]]);
      }
    }
  }
  const long long r0 = emb_row(d, v, m0);
#pragma unroll
  for (int j = 0; j < kCoupleCols; ++j) {
    if (m0 + j >= d.k) break;
    Gc[e * sG + (long long)(m0 + j) * d.N + row] = g[j];
    write_emb(d, Bemb, r0 + j, p, g[j]);
  }
}

// Where the backward sweep's quadrature shares go (Eq. 15): node e's share
// Re{coef_e x} of a layer's solution x is added (first: stored) into qp by
// the backward coupling that reads x as its x_next, on the FP64 pipe of a
// kernel that leaves it idle; the layers no later coupling reads (the last
// of each chain) take theirs in the solve product's epilogue.
struct BwdShares {
  double* qp = nullptr;        // [Ne][k][N]; nullptr: no shares
  const cplx* coef = nullptr;  // Ne quadrature coefficients
  int first = 0;               // 1: store (first solve), 0: accumulate
  int mid = -1;                // layer whose share chain 0 alone adds (the middle layer)
};

// backward: s = g - U x_next on a chain's layer, x_next the solution of the
// chain's next layer towards the middle (chain 0: layer + 1, coupled through
// the dz = +1 slots; chain 1: layer - 1, the dz = -1 slots); the embedded s
// goes to the virtual node's GEMM operand, and x_next's quadrature share to
// qs.qp (both chains read the middle layer: chain 0 adds its share).  A
// layer without a next one (the last layer of a one-ended elimination) takes
// s = g.  Threads as in the forward coupling.
__global__ void __launch_bounds__(128) k_mx_couple_bwd(Dims d, Chains ch, const f2* __restrict__ Cf,
                                                       const f2* __restrict__ Gc, float* __restrict__ Bemb,
                                                       NodeList nl, const int* __restrict__ active, BwdShares qs) {
  tc::grid_dep_wait();   // as in the forward coupling
  tc::grid_dep_launch_dependents();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = blockIdx.y * kCoupleCols, v = tc::nth_set_bit(nl.mask, (int)blockIdx.z);
  if (p >= d.n) return;
  const int c = chain_of(ch, v), e = node_of(ch, v);
  if (active && !active[e]) return;
  const int layer = ch.layer[c], next = c ? layer - 1 : layer + 1;
  const bool has_next = next >= 0 && next < d.nz;
  const long long row = (long long)layer * d.n + p;
  const long long sG = d.N * d.k;
  const long long dn = c ? -(long long)d.n : (long long)d.n;
  int off[9];
  f2 cv[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    off[t] = tap_offset(d, p, t);
    cv[t] = has_next ? Cf[((long long)e * 27 + prev_slot(1 - c) + t) * d.N + row] : f2{0.f, 0.f};
  }
  const bool share = qs.qp && has_next && (c == 0 || next != qs.mid);
  f2 sv[kCoupleCols], xn[kCoupleCols];
#pragma unroll
  for (int j = 0; j < kCoupleCols; ++j) {
    const int m = min(m0 + j, d.k - 1);   // as in the forward coupling
    const f2* col = Gc + e * sG + (long long)m * d.N + row;
    sv[j] = col[0];
    xn[j] = f2{0.f, 0.f};
    if (has_next) {
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const f2 x = col[dn + off[t]];
        sv[j].x -= cv[t].x * x.x - cv[t].y * x.y;
        sv[j].y -= cv[t].x * x.y + cv[t].y * x.x;
      }
      xn[j] = col[dn];   // x_next on this row (the centre tap)
    }
  }
  const long long r0 = emb_row(d, v, m0);
#pragma unroll
  for (int j = 0; j < kCoupleCols; ++j) {
    if (m0 + j >= d.k) break;
    write_emb(d, Bemb, r0 + j, p, sv[j]);
  }
  if (share) {
    const cplx ce = qs.coef[e];
    double* q = qs.qp + e * sG + (long long)next * d.n + p;
    double old[kCoupleCols];
#pragma unroll
    for (int j = 0; j < kCoupleCols; ++j)
      old[j] = (qs.first || m0 + j >= d.k) ? 0.0 : q[(long long)(m0 + j) * d.N];
#pragma unroll
    for (int j = 0; j < kCoupleCols; ++j) {
      if (m0 + j >= d.k) break;
      q[(long long)(m0 + j) * d.N] = fma(ce.re, (double)xn[j].x, fma(-ce.im, (double)xn[j].y, old[j]));
    }
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

#ifndef FEAST_RES_ROWS
#define FEAST_RES_ROWS 128
#endif
constexpr int kResRows = FEAST_RES_ROWS;   // grid rows per block
// Refinement targets at or above this take their first residual in
// double-float as well (its error, ~1e-12 of ||RHS||, is far below them).
constexpr double kFFirstTol = 1e-9;
constexpr int kResThreads = 256;   // two column groups per row
#ifndef FEAST_RES_COLS
#define FEAST_RES_COLS 3
#endif
constexpr int kResCols = FEAST_RES_COLS;   // columns per pass of a thread in the double-float residual
#ifndef FEAST_RES_MIN_BLOCKS
#define FEAST_RES_MIN_BLOCKS 3
#endif
constexpr int kResMinBlocks = FEAST_RES_MIN_BLOCKS;   // resident CTAs per SM the register budget allows
constexpr size_t kResSmem = sizeof(cplx) * 27 * kResRows;

// R_e = RHS - (Z_e B - A) Q_e in FP64 (108 FP64 FMAs per complex entry, the
// only FP64 arithmetic of the kernel) for the first solve's Q_e, which is its
// complex64 sweep output exactly: the block's 128 rows keep their 27
// complex coefficients in shared memory while the threads sweep the columns.
// Stores R as a double-float pair, Rc + Rlo (Rc: the complex64 leading part,
// the next correction's right-hand side; Rlo: the trailing part; together the
// start of the incremental residuals), and per-block partial sums of |R|^2 and
// |RHS|^2.
__global__ void __launch_bounds__(kResThreads) k_mx_residual(Dims d, const cplx* __restrict__ Z,
                                                             const double* __restrict__ A27,
                                                             const double* __restrict__ B27,
                                                             const double* __restrict__ RHS,
                                                             const f2* __restrict__ Q, f2* __restrict__ Rc,
                                                             f2* __restrict__ Rlo, double* __restrict__ partial,
                                                             const int* __restrict__ active,
                                                             const double* __restrict__ target) {
  extern __shared__ cplx rsm[];
  __shared__ double red[2][kResThreads];
  const int e = blockIdx.y;
  const int tid = threadIdx.x;
  if (!active[e]) return;   // block-uniform; the norm kernel ignores inactive nodes
  if (target && !(*target < kFFirstTol)) return;   // a loose target: the double-float kernel runs instead
  const long long i0 = (long long)blockIdx.x * kResRows;
  const cplx z = Z[e];
  for (int t = tid; t < 27 * kResRows; t += kResThreads) {
    const int s = t / kResRows, r = t % kResRows;
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
    rsm[t] = c;
  }
  __syncthreads();
  const int r = tid % kResRows;
  const long long i = i0 + r;
  double rr = 0.0, bb = 0.0;
  if (i < d.N) {
    const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
    int off[27];
#pragma unroll
    for (int s = 0; s < 27; ++s) {
      const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
      const bool ok = ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 &&
                      iz + dz < d.nz;
      off[s] = ok ? dx + d.nx * (dy + d.ny * dz) : 0;
    }
    const long long sG = d.N * d.k;
    for (int m = tid / kResRows; m < d.k; m += kResThreads / kResRows) {
      const f2* q = Q + e * sG + (long long)m * d.N + i;
      const double b = RHS[(long long)m * d.N + i];
      double are = b, aim = 0.0;
#pragma unroll
      for (int s = 0; s < 27; ++s) {
        const cplx c = rsm[s * kResRows + r];
        const f2 v32 = q[off[s]];
        const cplx v{f32_to_f64(v32.x), f32_to_f64(v32.y)};
        are = fma(-c.re, v.re, are);
        are = fma(c.im, v.im, are);
        aim = fma(-c.re, v.im, aim);
        aim = fma(-c.im, v.re, aim);
      }
      const float hre = f64_to_f32_trunc(are), him = f64_to_f32_trunc(aim);
      Rc[e * sG + (long long)m * d.N + i] = f2{hre, him};
      Rlo[e * sG + (long long)m * d.N + i] =
          f2{f64_to_f32_trunc(are - f32_to_f64(hre)), f64_to_f32_trunc(aim - f32_to_f64(him))};
      rr += are * are + aim * aim;
      bb += b * b;
    }
  }
  red[0][tid] = rr;
  red[1][tid] = bb;
  __syncthreads();
  for (int w = kResThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      red[0][tid] += red[0][tid + w];
      red[1][tid] += red[1][tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    partial[((long long)e * gridDim.x + blockIdx.x) * 2] = red[0][0];
    partial[((long long)e * gridDim.x + blockIdx.x) * 2 + 1] = red[1][0];
  }
}

// ---- incremental residual in double-float arithmetic
//
// After a correction delta (the complex64 solution of the previous residual,
// added exactly into Q_e in FP64) the residual moves by -(Z_e B - A) delta:
//   R <- R - (Z_e B - A) delta.
// delta is exact in fp32 and its size falls by the refinement's contraction
// each step, so the product needs about twice fp32's precision relative to
// |C| |delta|, not FP64's relative to |C| |Q|.  Each coefficient c (FP64) is
// split into c_hi + c_lo (fp32); c_hi * delta is formed exactly as a pair by
// one FMA (Dekker's product) and the 27-term sums are compensated with
// Knuth's TwoSum, i.e. the accurate dot product of Ogita, Rump and Oishi
// (SIAM J. Sci. Comput. 26, 2005) with the low coefficient part folded into the
// error term.  The rounding-explicit intrinsics keep the compiler from fusing
// the product into the sum, which would break the exact error terms.
// Knuth's TwoSum: a + b = s + err exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}

// (h, l) <- (h + l) - (ph + pl) in double-float: the leading parts by TwoSum,
// the trailing parts and its error added, then renormalised by TwoSum.
__device__ __forceinline__ void ff_sub(float& h, float& l, float ph, float pl) {
  float e1, e2;
  const float sh = two_sum(h, -ph, e1);
  const float t = __fadd_rn(__fsub_rn(l, pl), e1);
  h = two_sum(sh, t, e2);
  l = e2;
}

__device__ __forceinline__ void ff_axpy(float ch, float cl, float v, float& sh, float& sl) {
  const float p = __fmul_rn(ch, v);
  const float pe = __fmaf_rn(ch, v, -p);            // ch * v = p + pe exactly
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));   // sh + p = t + err
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, __fmaf_rn(cl, v, pe)));
}

// R <- R - (Z_e B - A) delta with R = Rc + Rlo held as a double-float pair
// (Rc, its complex64 leading part, is the next correction's right-hand side),
// partial |R|^2 per block (the |RHS|^2 partials of the first residual are
// kept).  The update itself stays in fp32 arithmetic: the FP64 pipe only
// squares the leading parts for the norm.
// kFirst: the first residual of a solve whose target is loose (>= 1e-9
// relative): R starts from RHS instead, delta is the first solution Q_e,
// and the |RHS|^2 partials are written.  The product's error, ~2^-48 kappa
// ||Q_e|| (kappa ~ 300 here), is then far below the target.
template <bool kFirst>
__global__ void __launch_bounds__(kResThreads, kResMinBlocks) k_mx_residual_inc(Dims d, const cplx* __restrict__ Z,
                                                                 const double* __restrict__ A27,
                                                                 const double* __restrict__ B27,
                                                                 const f2* __restrict__ delta, f2* __restrict__ Rc,
                                                                 f2* __restrict__ Rlo, double* __restrict__ partial,
                                                                 const int* __restrict__ active,
                                                                 const double* __restrict__ RHS,
                                                                 const double* __restrict__ target) {
  extern __shared__ float4 csm[];   // per (slot, row): Re c hi/lo, Im c hi/lo
  __shared__ double red[kResThreads];
  __shared__ double redb[kFirst ? kResThreads : 1];
  const int e = blockIdx.y;
  const int tid = threadIdx.x;
  if (!active[e]) return;
  if (kFirst && target && !(*target >= kFFirstTol)) return;   // a tight target: the FP64 kernel runs instead
  const long long i0 = (long long)blockIdx.x * kResRows;
  const cplx z = Z[e];
  for (int t = tid; t < 27 * kResRows; t += kResThreads) {
    const int s = t / kResRows, r = t % kResRows;
    const long long i = i0 + r;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < d.N) {
      const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
      const int dx = slot_dx(s), dy = slot_dy(s), dz = slot_dz(s);
      if (ix + dx >= 0 && ix + dx < d.nx && iy + dy >= 0 && iy + dy < d.ny && iz + dz >= 0 && iz + dz < d.nz) {
        const double a = A27[(long long)s * d.N + i], b = B27[(long long)s * d.N + i];
        const double cr = z.re * b - a, ci = z.im * b;
        c.x = (float)cr;
        c.y = (float)(cr - (double)c.x);
        c.z = (float)ci;
        c.w = (float)(ci - (double)c.z);
      }
    }
    csm[t] = c;
  }
  __syncthreads();
  const int r = tid % kResRows;
  const long long i = i0 + r;
  double rr = 0.0, bb = 0.0;
  if (i < d.N) {
    const int ix = (int)(i % d.nx), iy = (int)((i / d.nx) % d.ny), iz = (int)(i / d.n);
    // neighbour validity per axis; an absent neighbour has a zero coefficient
    // and is read at offset 0 (the row itself) to stay in bounds
    const bool xm = ix > 0, xp = ix + 1 < d.nx, ym = iy > 0, yp = iy + 1 < d.ny, zm = iz > 0, zp = iz + 1 < d.nz;
    const int sx = 1, sy = d.nx, sz = d.n;
    const long long sG = d.N * d.k;
    const int g = tid / kResRows;   // column group: columns g, g + 2, g + 4, ...
    constexpr int kGroups = kResThreads / kResRows;
    // kResCols columns of the group per pass, sharing each tap's coefficient
    // and offset
    for (int m = g; m < d.k; m += kResCols * kGroups) {
      const f2* v[kResCols];
      bool has[kResCols];
      const f2* v0 = delta + e * sG + (long long)m * d.N + i;
#pragma unroll
      for (int j = 0; j < kResCols; ++j) {
        has[j] = m + j * kGroups < d.k;
        v[j] = has[j] ? v0 + (long long)j * kGroups * d.N : v0;
      }
      float rh[kResCols], rl[kResCols], ih[kResCols], il[kResCols];   // Re, Im (hi, lo)
#pragma unroll
      for (int j = 0; j < kResCols; ++j) rh[j] = rl[j] = ih[j] = il[j] = 0.f;
#pragma unroll 9
      for (int s = 0; s < 27; ++s) {
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        const bool ok = (dx < 0 ? xm : (dx > 0 ? xp : true)) && (dy < 0 ? ym : (dy > 0 ? yp : true)) &&
                        (dz < 0 ? zm : (dz > 0 ? zp : true));
        const int off = ok ? dx * sx + dy * sy + dz * sz : 0;
        const float4 c = csm[s * kResRows + r];
        f2 x[kResCols];
#pragma unroll
        for (int j = 0; j < kResCols; ++j) x[j] = v[j][off];
#pragma unroll
        for (int j = 0; j < kResCols; ++j) {
          ff_axpy(c.x, c.y, x[j].x, rh[j], rl[j]);     // + Re c Re x
          ff_axpy(c.x, c.y, x[j].y, ih[j], il[j]);     // + Re c Im x
        }
#pragma unroll
        for (int j = 0; j < kResCols; ++j) {
          ff_axpy(-c.z, -c.w, x[j].y, rh[j], rl[j]);   // - Im c Im x
          ff_axpy(c.z, c.w, x[j].x, ih[j], il[j]);     // + Im c Re x
        }
      }
#pragma unroll
      for (int j = 0; j < kResCols; ++j) {
        if (!has[j]) continue;
        const int mj = m + j * kGroups;
        const long long at = e * sG + (long long)mj * d.N + i;
        f2 H, L;   // R = H + L
        if constexpr (kFirst) {
          const double b = RHS[(long long)mj * d.N + i];
          H = f2{(float)b, 0.f};
          L = f2{(float)(b - (double)H.x), 0.f};
          bb = fma(b, b, bb);
        } else {
          H = Rc[at];
          L = Rlo[at];
        }
        ff_sub(H.x, L.x, rh[j], rl[j]);
        ff_sub(H.y, L.y, ih[j], il[j]);
        Rc[at] = H;
        Rlo[at] = L;
        const double hx = H.x, hy = H.y;
        rr = fma(hx, hx, fma(hy, hy, rr));
      }
    }
  }
  red[tid] = rr;
  if constexpr (kFirst) redb[tid] = bb;
  __syncthreads();
  for (int w = kResThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      red[tid] += red[tid + w];
      if constexpr (kFirst) redb[tid] += redb[tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    partial[((long long)e * gridDim.x + blockIdx.x) * 2] = red[0];
    if constexpr (kFirst) partial[((long long)e * gridDim.x + blockIdx.x) * 2 + 1] = redb[0];
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
bool make_map(CUtensorMap* map, const float* base, long long inner, long long rows, long long ld, int box_rows) {
  return make_map_2d(map, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, inner, rows, ld, box_rows);
}

// Shared-memory attribute of a GEMM instantiation, set once per device (and
// before any stream capture: it is not a stream operation).
template <int BN, int STAGES, class Epi, int KIND = 0>
cudaError_t tc_attr() {
  constexpr size_t smem = tc::smem_bytes<BN, STAGES, Epi>();
  static PerDevice<cudaError_t> attr;
  return attr.get(
      [] {
        return cudaFuncSetAttribute(tc::k_tc_gemm<BN, STAGES, Epi, KIND>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      },
      cudaErrorInvalidDevice);
}

#ifndef FEAST_PDL
#define FEAST_PDL 1
#endif
// Launch with programmatic stream serialisation: the grid may start (and run
// its set-up up to grid_dep_wait) while the previous grid in the stream
// drains.  Used for the chains of dependent launches of the solve sweeps.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = FEAST_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int BN, int STAGES, class Epi, int KIND = 0>
cudaError_t launch_tc(cudaStream_t s, dim3 grid, const CUtensorMap& a, const CUtensorMap& b, tc::Geom geo,
                      const Epi& epi, int* status, bool pdl = false) {
  constexpr size_t smem = tc::smem_bytes<BN, STAGES, Epi>();
  if (const cudaError_t e = tc_attr<BN, STAGES, Epi, KIND>()) return e;
  if (pdl)
    return launch_pdl(tc::k_tc_gemm<BN, STAGES, Epi, KIND>, grid, dim3(tc::kThreads), smem, s, a, b, geo, epi, status);
  tc::k_tc_gemm<BN, STAGES, Epi, KIND><<<grid, tc::kThreads, smem, s>>>(a, b, geo, epi, status);
  return cudaGetLastError();
}

// Operand kind of the block-solve products (split bf16 pairs, see k_tc_gemm).
constexpr int kSolveKind = 2;

enum Buf { B_F = 0, B_T1, B_AOP, B_BOP, B_TC, B_PINV, B_GC, B_RC, B_BEMB, B_TOUT, B_PART, B_REL, B_ACTIVE, B_CF, B_FW,
           B_RLO, B_COUNT };
static_assert(B_COUNT <= 16, "MixedWork holds 16 buffers");

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

// The stream captures are recorded on: the caller's stream may be the legacy
// default stream, which cannot be captured; the graph is then launched into
// the caller's stream.
cudaStream_t capture_stream(MixedWork& w) {
  if (!w.cap && cudaStreamCreateWithFlags(&w.cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    w.cap = nullptr;
  }
  return w.cap;
}

// cfg: the solve-GEMM configuration, CB | ST << 8 (0: the default for k)
Dims make_dims(Grid g, int Ne, int k, int cfg = 0) {
  const int cb = cfg & 255, st = cfg >> 8;
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
  d.CB = cb > 0 ? cb : (k <= 8 ? 8 : (k <= 16 ? 16 : (k <= 32 ? 32 : 64)));
  d.ST = st > 0 ? st : 4;
  d.nblkCB = (k + d.CB - 1) / d.CB;
  d.ldB = d.ldF;
  // two chains need 2 Ne virtual nodes in the 64-bit node masks of the sweeps
  d.K = 2 * Ne <= 64 ? d.nz / 2 : d.nz - 1;
  return d;
}

// ---- recursive inversion: launch plan
// Workspace of recursion level L (blocks of at most cap[L] rows): Xbar and
// Xbar^T of every virtual node, row-split with row stride 2 cap[L], at float
// offset woff[L] of the buffers W and W2.
struct InvLevels {
  std::vector<int> cap;
  std::vector<long long> woff;
  long long floats = 0;   // per buffer
};

// Split of a block of s rows (s > 64): the first part is a multiple of 64.
inline int inv_split(int s) { return 64 * (((s + 63) / 64 + 1) / 2); }

InvLevels inv_levels(int n, int V) {
  InvLevels lv;
  for (int s = n; s > kPanel; s = inv_split(s)) {
    const int h = inv_split(s);
    lv.cap.push_back(h);
    lv.woff.push_back(lv.floats);
    lv.floats += (long long)V * h * 2 * h;
  }
  return lv;
}

struct InvOp {
  int leaf = 0;       // 1: diagonal block [off, off + s) by k_mx_pinv, final when fin
  int off = 0, s = 0, fin = 0;
  CUtensorMap m[4];   // U re, U im, V re, V im
  tc::CGeom geo{};
  int M = 0, N = 0;
  double flops = 0;   // per virtual node
  InvEpi epi;         // ch set per layer step
};

// The launches that invert every virtual node's plane `plane` of F in place
// (S <- -S^{-1}), final blocks also into Fr.  Returns an error or nullptr.
const char* build_inversion(const Dims& d, int V, int plane, float* F, float* Fr, float* W, float* W2,
                            const InvLevels& lv, std::vector<InvOp>& ops) {
  const long long planeF = (long long)d.n * d.ldF;
  float* Fp = F + plane * planeF;
  // F block (row0, col0, rows x cols) of every virtual node's plane: z = 2 b + plane
  auto fmap = [&](CUtensorMap* m, int row0, int col0, int rows, int cols, int box_rows) {
    const float* base = F + (long long)row0 * d.ldF + col0;
    return make_map_3d(m, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, cols, rows, 2LL * V, d.ldF, planeF, tc::kBlockK,
                       box_rows, CU_TENSOR_MAP_SWIZZLE_128B) &&
           make_map_3d(m + 1, base + d.n, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, cols, rows, 2LL * V, d.ldF, planeF,
                       tc::kBlockK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
  };
  // level-L workspace block (rows x cols from the origin): z = b
  auto wmap = [&](CUtensorMap* m, const float* Wb, int L, int rows, int cols, int box_rows) {
    const int cap = lv.cap[L];
    const float* base = Wb + lv.woff[L];
    return make_map_3d(m, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, cols, rows, V, 2LL * cap, (long long)cap * 2 * cap,
                       tc::kBlockK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B) &&
           make_map_3d(m + 1, base + cap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, cols, rows, V, 2LL * cap,
                       (long long)cap * 2 * cap, tc::kBlockK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
  };
  auto fdest = [&](int row0, int col0) {
    return InvDest{Fp + (long long)row0 * d.ldF + col0, 2 * planeF, d.ldF, d.n};
  };
  auto wdest = [&](float* Wb, int L) {
    const int cap = lv.cap[L];
    return InvDest{Wb + lv.woff[L], (long long)cap * 2 * cap, 2 * cap, cap};
  };
  auto gemm = [&](int M, int N, int K, bool u_in_f, bool v_in_f) {
    InvOp op;
    op.M = M;
    op.N = N;
    op.geo = tc::CGeom{(K + tc::kBlockK - 1) / tc::kBlockK, u_in_f ? 2 : 1, u_in_f ? plane : 0, v_in_f ? 2 : 1,
                       v_in_f ? plane : 0};
    op.flops = 8.0 * M * (double)N * K;
    op.epi.M = M;
    op.epi.N = N;
    op.epi.ld_fr = d.ldF;
    op.epi.imoff_fr = d.n;
    op.epi.fr_plane = planeF;
    op.epi.nz = d.nz;
    return op;
  };
  auto rec = [&](auto&& self, int L, int off, int s, bool fin) -> const char* {
    if (s <= kPanel) {
      InvOp op;
      op.leaf = 1;
      op.off = off;
      op.s = s;
      op.fin = fin;
      op.flops = 8.0 * s * (double)s * s;
      ops.push_back(op);
      return nullptr;
    }
    const int h = inv_split(s), t = s - h;
    if (const char* m = self(self, L + 1, off, h, false)) return m;
    {  // Xbar^T = B^T Abar -> Xbar (W, transposed) and Xbar^T (W2)
      InvOp op = gemm(t, h, h, true, true);
      if (!fmap(op.m, off + h, off, t, h, tc::kBlockM) || !fmap(op.m + 2, off, off, h, h, kInvBN))
        return "tensor map (inversion) rejected";
      op.epi.t = wdest(W, L);
      op.epi.r = wdest(W2, L);
      ops.push_back(op);
    }
    {  // D += Xbar^T B
      InvOp op = gemm(t, t, h, false, true);
      if (!wmap(op.m, W2, L, t, h, tc::kBlockM) || !fmap(op.m + 2, off + h, off, t, h, kInvBN))
        return "tensor map (inversion) rejected";
      op.epi.t = fdest(off + h, off + h);
      op.epi.add = 1;
      ops.push_back(op);
    }
    if (const char* m = self(self, L + 1, off + h, t, fin)) return m;
    {  // Ybar^T = Sbar Xbar^T -> upper-right block (transposed) and lower-left block
      InvOp op = gemm(t, h, t, true, false);
      if (!fmap(op.m, off + h, off + h, t, t, tc::kBlockM) || !wmap(op.m + 2, W, L, h, t, kInvBN))
        return "tensor map (inversion) rejected";
      op.epi.t = fdest(off, off + h);
      op.epi.r = fdest(off + h, off);
      if (fin) {
        op.epi.fr = Fr;
        op.epi.fr_t = (long long)off * d.ldF + off + h;
        op.epi.fr_r = (long long)(off + h) * d.ldF + off;
      }
      ops.push_back(op);
    }
    {  // Abar += Ybar Xbar^T
      InvOp op = gemm(h, h, t, true, false);
      if (!fmap(op.m, off, off + h, h, t, tc::kBlockM) || !wmap(op.m + 2, W, L, h, t, kInvBN))
        return "tensor map (inversion) rejected";
      op.epi.t = fdest(off, off);
      op.epi.add = 1;
      if (fin) {
        op.epi.fr = Fr;
        op.epi.fr_t = (long long)off * d.ldF + off;
      }
      ops.push_back(op);
    }
    return nullptr;
  };
  return rec(rec, 0, 0, d.n, true);
}

template <class Epi>
cudaError_t cg_attr() {
  constexpr size_t smem = tc::CSmem<kInvBN, kInvStages>::kBytes;
  static PerDevice<cudaError_t> attr;
  return attr.get(
      [] {
        return cudaFuncSetAttribute(tc::k_cgemm<kInvBN, kInvStages, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
      },
      cudaErrorInvalidDevice);
}

template <class Epi>
cudaError_t launch_cg(cudaStream_t s, dim3 grid, const CUtensorMap* m, const tc::CGeom& geo, const Epi& epi,
                      int* status) {
  constexpr size_t smem = tc::CSmem<kInvBN, kInvStages>::kBytes;
  if (const cudaError_t e = cg_attr<Epi>()) return e;
  tc::k_cgemm<kInvBN, kInvStages, Epi><<<grid, tc::kThreads, smem, s>>>(m[0], m[1], m[2], m[3], geo, epi, status);
  return cudaGetLastError();
}

}  // namespace

void MixedWork::release() {
  if (factor_graph) cudaGraphExecDestroy(factor_graph);
  factor_graph = nullptr;
  if (cap) cudaStreamDestroy(cap);
  cap = nullptr;
  for (int g = 0; g < kSweepGraphs; ++g) {
    if (graphs.exec[g]) cudaGraphExecDestroy(graphs.exec[g]);
    graphs.exec[g] = nullptr;
    graphs.used[g] = 0;
  }
  for (int i = 0; i < 16; ++i) {
    if (bufs[i]) cudaFree(bufs[i]);
    bufs[i] = nullptr;
    sizes[i] = 0;
  }
  nz_factored = 0;
  if (loop_graph) cudaGraphExecDestroy(loop_graph);
  loop_graph = nullptr;
  std::memset(loop_key, 0, sizeof(loop_key));
  std::memset(loop_seen, 0, sizeof(loop_seen));
  for (cudaStream_t* c : {&cap2, &cap3}) {
    if (*c) cudaStreamDestroy(*c);
    *c = nullptr;
  }
  if (side) cudaStreamDestroy(side);
  if (ev_narrow) cudaEventDestroy(ev_narrow);
  if (ev_side) cudaEventDestroy(ev_side);
  side = nullptr;
  ev_narrow = ev_side = nullptr;
}

const char* mixed_factor(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, int* status) {
  Dims d = make_dims(g, Ne, 1);
  if (!encode_fn()) return "cuTensorMapEncodeTiled is not available from the driver";
  const int V = 2 * Ne;   // virtual nodes (two chains)
  const size_t fbytes = sizeof(float) * (size_t)Ne * d.nz * d.n * d.ldF;
  const long long flayout = (long long)d.n << 32 | d.ldF;
  const bool f_new = w.sizes[B_F] < fbytes || !w.bufs[B_F] || w.fr_layout != flayout;
  if (!ensure(w, B_F, fbytes, s, f_new)) return "out of device memory (mixed factors)";
  w.fr_layout = flayout;
  if (!ensure(w, B_FW, sizeof(float) * (size_t)V * 2 * d.n * d.ldF, s)) return "out of device memory (working layers)";
  if (!ensure(w, B_T1, sizeof(float) * (size_t)V * d.n * d.ldF, s)) return "out of device memory (schur scratch)";
  // The recursive block inversion needs 16-byte aligned imaginary halves of
  // the row-split rows (n a multiple of 4) for its tensor maps; otherwise
  // the layers are inverted by the panel sweep.
  const bool recursive = !kFactorPanelSweep && d.n % 4 == 0 && d.n > kPanel;
  const InvLevels lv = inv_levels(d.n, V);
  // panel operands are double-buffered by panel parity (lookahead); the
  // recursive inversion keeps its workspaces Xbar and Xbar^T in the same buffers
  const size_t aop_sz = (size_t)V * d.n * 2 * kPanel;
  const size_t bop_sz = (size_t)V * d.nblk64 * 128 * 2 * kPanel;
  const size_t tc_sz = (size_t)V * d.n * kPanel;
  const size_t pinv_sz = (size_t)V * kPanel * kPanel;
  const size_t wfl = recursive ? (size_t)lv.floats : 0;
  if (!ensure(w, B_AOP, sizeof(float) * std::max(2 * aop_sz, wfl), s, true)) return "out of device memory";
  if (!ensure(w, B_BOP, sizeof(float) * std::max(2 * bop_sz, wfl), s, true)) return "out of device memory";
  if (!ensure(w, B_TC, sizeof(f2) * 2 * tc_sz, s)) return "out of device memory";
  if (!ensure(w, B_PINV, sizeof(f2) * 2 * pinv_sz, s)) return "out of device memory";
  if (!ensure(w, B_CF, sizeof(f2) * (size_t)Ne * 27 * d.N, s)) return "out of device memory (coefficients)";
  if (!w.side) {
    // highest priority: the lookahead chain is the critical path, its few
    // CTAs must not queue behind the wide update's
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (cudaStreamCreateWithPriority(&w.side, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_narrow, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_side, cudaEventDisableTiming) != cudaSuccess)
      return "could not create the lookahead stream";
  }
  cudaStream_t s2 = w.side;
  // The row-split padding [2n, ldF) is never read (the tensor maps stop at 2n).
  float* Fr = buf<float>(w, B_F);    // S'_i of every layer as split bf16 pairs (solve operand)
  float* F = buf<float>(w, B_FW);    // fp32 working layers (ping-pong per virtual node)
  f2* Cf = buf<f2>(w, B_CF);
  const int K = d.K, L0 = K, L1 = d.nz - 1 - K;   // middle layer, chain lengths
  std::vector<InvOp> inv_ops[2];
  if (recursive)
    for (int plane = 0; plane < 2; ++plane)
      if (const char* m = build_inversion(d, V, plane, F, Fr, buf<float>(w, B_AOP), buf<float>(w, B_BOP), lv,
                                          inv_ops[plane]))
        return m;
  // The launches of the factorisation (both streams).  Without kernel timing
  // they are captured once into a CUDA graph (node priorities kept, so the
  // lookahead chain still goes first) and replayed while the shape, the
  // operator and the work buffers stay the same.
  auto body = [&](cudaStream_t s) -> const char* {
    k_mx_coef<<<dim3((unsigned)std::min<long long>(4096, (27 * d.N + 255) / 256), Ne), 256, 0, s>>>(d, Z, A27, B27, Cf);
    prof::count_launch();
    float* Aop[2] = {buf<float>(w, B_AOP), buf<float>(w, B_AOP) + aop_sz};
    float* Bop[2] = {buf<float>(w, B_BOP), buf<float>(w, B_BOP) + bop_sz};
    f2* Tc[2] = {buf<f2>(w, B_TC), buf<f2>(w, B_TC) + tc_sz};
    f2* Pv[2] = {buf<f2>(w, B_PINV), buf<f2>(w, B_PINV) + pinv_sz};
    CUtensorMap tmA[2], tmB[2];
    for (int q = 0; q < 2; ++q) {
      if (!make_map(&tmA[q], Aop[q], 2 * kPanel, (long long)V * d.n, 2 * kPanel, 128)) return "tensor map (Aop) rejected";
      if (!make_map(&tmB[q], Bop[q], 2 * kPanel, (long long)V * d.nblk64 * 128, 2 * kPanel, 128))
        return "tensor map (Bop) rejected";
    }
    const long long sF = 2LL * d.n * d.ldF;
    const long long sFr = (long long)d.nz * d.n * d.ldF;
    const int npan = d.nblk64;
    // one panel step of the virtual nodes 0 .. nv-1 (all of them work on plane ch.wplane)
    auto panel = [&](cudaStream_t st, const Chains& ch, int nv, int kp) {
      const int k0 = kp * kPanel, bw = std::min(kPanel, d.n - k0), q = kp & 1;
      prof::begin(st, prof::PINV);
      prof::add_work(prof::PINV, 8.0 * kPanel * kPanel * kPanel * nv);
      k_mx_pinv<kPinvRpt><<<nv, kPanel * (kPanel / kPinvRpt), 0, st>>>(d, ch.wplane, k0, bw, F, Pv[q], status,
                                                                      LeafOut{});
      prof::end(st, prof::PINV);
      prof::begin(st, prof::PANEL_T);
      prof::add_work(prof::PANEL_T, 8.0 * d.n * kPanel * kPanel * nv);
      k_mx_panel_T<<<dim3(cdiv(d.n, kRowsPerPanelCta), nv), 256, 0, st>>>(d, ch.wplane, k0, bw, F, Pv[q], Aop[q],
                                                                        Bop[q], Tc[q]);
      prof::end(st, prof::PANEL_T);
      prof::count_launch(2);
    };
    // TMA-staged read-modify-write of S when a 64-column tile never straddles
    // the real/imaginary split of a row
    const bool tma_rmw = d.n % 64 == 0;
    CUtensorMap mapF{}, mapFr{};
    if (tma_rmw) {
      if (!make_map_3d(&mapF, F, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2LL * d.n, d.n, 2LL * V, d.ldF,
                       (long long)d.n * d.ldF, 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) ||
          !make_map_3d(&mapFr, Fr, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2LL * d.n, d.n, (long long)Ne * d.nz, d.ldF,
                       (long long)d.n * d.ldF, 32, 128, CU_TENSOR_MAP_SWIZZLE_128B))
        return "tensor map (working layers) rejected";
    }
    // trailing update of panel kp over the column tiles [base, base + count) except `skip`
    auto update = [&](cudaStream_t st, const Chains& ch, int nv, int kp, int base, int count,
                      int skip) -> cudaError_t {
      const int k0 = kp * kPanel, bw = std::min(kPanel, d.n - k0), q = kp & 1;
      const bool last = kp == npan - 1;
      tc::Geom geo{0, d.n, 0, d.nblk64 * 128, (2 * kPanel) / tc::kBlockK, base, skip};
      const int cls = base > 0 ? prof::SWEEP_NARROW : prof::SWEEP_GEMM;   // the narrow update starts at tile kp+1
      prof::begin(st, cls);
      prof::add_work(cls, 8.0 * d.n * (64.0 * count) * bw * nv);
      cudaError_t err;
      const dim3 grid(count, cdiv(d.n, 128), nv);
      if (tma_rmw) {
        SweepEpiTma epi{mapF, mapFr, ch.wplane, ch, d.nz, d.n, k0, bw, last ? 1 : 0, Tc[q], Pv[q]};
        // the narrow update (one column tile) with kNarrowStages, the wide
        // one with kWideStages (both one by default, so that their CTAs share SMs)
        err = count == 1 ? launch_tc<128, kNarrowStages, SweepEpiTma, kFactorKind>(st, grid, tmA[q], tmB[q], geo, epi, status)
                         : launch_tc<128, kWideStages, SweepEpiTma, kFactorKind>(st, grid, tmA[q], tmB[q], geo, epi,
                                                                                 status);
      } else {
        SweepEpi epi{F + (long long)ch.wplane * d.n * d.ldF, sF, last ? Fr : nullptr, sFr, d.ldF, d.n, k0, bw,
                     Tc[q], Pv[q], ch};
        err = launch_tc<128, 2, SweepEpi, kFactorKind>(st, grid, tmA[q], tmB[q], geo, epi, status);
      }
      prof::end(st, cls);
      prof::count_launch();
      return err;
    };
    // the recursive inversion of the complements of the nv virtual nodes (plane ch.wplane)
    auto invert = [&](const Chains& ch, int nv) -> const char* {
      for (const InvOp& op : inv_ops[ch.wplane]) {
        if (op.leaf) {
          prof::begin(s, prof::PINV);
          prof::add_work(prof::PINV, op.flops * nv);
          k_mx_pinv<kPinvRpt><<<nv, kPanel * (kPanel / kPinvRpt), 0, s>>>(
              d, ch.wplane, op.off, op.s, F, nullptr, status, LeafOut{F, op.fin ? Fr : nullptr, ch, d.nz});
          prof::end(s, prof::PINV);
        } else {
          InvEpi epi = op.epi;
          epi.ch = ch;
          prof::begin(s, prof::SWEEP_GEMM);
          prof::add_work(prof::SWEEP_GEMM, op.flops * nv);
          const cudaError_t err =
              launch_cg(s, dim3(cdiv(op.N, kInvBN), cdiv(op.M, tc::kBlockM), nv), op.m, op.geo, epi, status);
          prof::end(s, prof::SWEEP_GEMM);
          if (err != cudaSuccess) return "tcgen05 inversion launch failed";
        }
        prof::count_launch();
      }
      return nullptr;
    };
    // the block sweep of the complements of the nv virtual nodes (plane ch.wplane)
    auto sweep = [&](const Chains& ch, int nv) -> const char* {
      if (recursive) return invert(ch, nv);
      panel(s, ch, nv, 0);
      for (int kp = 0; kp < npan; ++kp) {
        if (kp + 1 < npan) {
          // fork: the previous wide update and this panel's inverse and
          // product (joined into s below) precede both updates of panel kp
          cudaEventRecord(w.ev_narrow, s);
          cudaStreamWaitEvent(s2, w.ev_narrow, 0);
          // the lookahead chain on the side stream: the narrow update of the
          // next panel's columns, then that panel's inverse and product ...
          if (update(s2, ch, nv, kp, kp + 1, 1, -1) != cudaSuccess) return "tcgen05 sweep-update launch failed";
          panel(s2, ch, nv, kp + 1);
          cudaEventRecord(w.ev_side, s2);
          // ... beside the wide update of the other column tiles (disjoint
          // tiles, the same panel operands)
          if (npan > 1 && update(s, ch, nv, kp, 0, npan - 1, kp + 1) != cudaSuccess)
            return "tcgen05 sweep-update launch failed";
          cudaStreamWaitEvent(s, w.ev_side, 0);
        } else {
          if (update(s, ch, nv, kp, 0, npan, -1) != cudaSuccess) return "tcgen05 sweep-update launch failed";
        }
      }
      return nullptr;
    };
    const dim3 sgrid(cdiv(d.n, 256), d.n);
    // both chains, one layer each per step
    for (int t = 0; t < L0; ++t) {
      const Chains ch{Ne, {t, d.nz - 1 - t}, {(t + 1) & 1, (t + 1) & 1}, t & 1};
      const int nv = t < L1 ? V : Ne;
      prof::begin(s, prof::SCHUR);
      prof::add_work(prof::SCHUR, (t > 0 ? 144.0 : 0.0) * d.n * (double)d.n * nv);
      if (t > 0)
        k_mx_schur1<<<dim3(sgrid.x, cdiv(d.n, kSchurRows), nv), 256, 0, s>>>(d, ch, Cf, F, buf<float>(w, B_T1));
      k_mx_schur2<<<dim3(sgrid.x, cdiv(d.n, kSchur2Rows), nv), 256, 0, s>>>(d, ch, t > 0, 0, 0, Cf,
                                                                            buf<float>(w, B_T1), F);
      prof::end(s, prof::SCHUR);
      prof::count_launch(t > 0 ? 2 : 1);
      if (const char* m = sweep(ch, nv)) return m;
    }
    // the middle layer with both chains' last complements
    {
      const Chains ch{Ne, {K, K}, {(L0 + 1) & 1, (L1 + 1) & 1}, L0 & 1};
      prof::begin(s, prof::SCHUR);
      prof::add_work(prof::SCHUR, (L0 > 0 ? 144.0 : 0.0) * (L1 > 0 ? 2.0 : 1.0) * d.n * (double)d.n * Ne);
      if (L0 > 0)
        k_mx_schur1<<<dim3(sgrid.x, cdiv(d.n, kSchurRows), L1 > 0 ? V : Ne), 256, 0, s>>>(d, ch, Cf, F,
                                                                                         buf<float>(w, B_T1));
      k_mx_schur2<<<dim3(sgrid.x, cdiv(d.n, kSchur2Rows), Ne), 256, 0, s>>>(d, ch, L0 > 0, 1, L1 > 0, Cf,
                                                                            buf<float>(w, B_T1), F);
      prof::end(s, prof::SCHUR);
      prof::count_launch(L0 > 0 ? 2 : 1);
      if (const char* m = sweep(ch, Ne)) return m;
    }
    return nullptr;
  };
  if (prof::enabled() || !w.use_graphs) {
    if (const char* m = body(s)) return m;
  } else {
    const unsigned long long key[kSweepKey] = {
        (unsigned long long)d.nx | ((unsigned long long)d.ny << 20) | ((unsigned long long)d.nz << 40),
        (unsigned long long)Ne | ((unsigned long long)d.ldF << 20),
        (unsigned long long)(uintptr_t)Z, (unsigned long long)(uintptr_t)A27, (unsigned long long)(uintptr_t)B27,
        (unsigned long long)(uintptr_t)status, (unsigned long long)(uintptr_t)w.bufs[B_F],
        (unsigned long long)(uintptr_t)w.bufs[B_FW], (unsigned long long)(uintptr_t)w.bufs[B_T1],
        (unsigned long long)(uintptr_t)w.bufs[B_AOP], (unsigned long long)(uintptr_t)w.bufs[B_BOP],
        (unsigned long long)(uintptr_t)w.bufs[B_TC], (unsigned long long)(uintptr_t)w.bufs[B_PINV],
        (unsigned long long)(uintptr_t)w.bufs[B_CF], (unsigned long long)(uintptr_t)s2, 2ULL};
    if (w.factor_graph && std::memcmp(w.factor_key, key, sizeof(key)) == 0) {
      if (cudaGraphLaunch(w.factor_graph, s) != cudaSuccess) return "factor graph launch failed";
      prof::count_launch((int)w.factor_launches);
      ++w.factor_replays;
    } else if (std::memcmp(w.factor_seen, key, sizeof(key)) != 0) {
      // first factorisation with this key: direct launches (a one-off shape
      // would pay for a capture it never replays)
      std::memcpy(w.factor_seen, key, sizeof(key));
      if (const char* m = body(s)) return m;
    } else {
      if (w.factor_graph) cudaGraphExecDestroy(w.factor_graph);
      w.factor_graph = nullptr;
      if (tc_attr<128, kWideStages, SweepEpiTma, kFactorKind>() || tc_attr<128, kNarrowStages, SweepEpiTma, kFactorKind>() ||
          tc_attr<128, 2, SweepEpi, kFactorKind>() || cg_attr<InvEpi>())
        return "tcgen05 sweep-update attribute rejected";
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      const long long launches0 = prof::launches();
      cudaStream_t cs = capture_stream(w);
      const bool capturing = cs && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      const char* msg = capturing ? body(cs) : "capture not started";
      const cudaError_t end = capturing ? cudaStreamEndCapture(cs, &graph) : cudaErrorUnknown;
      if (msg || end != cudaSuccess || !graph ||
          cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        prof::count_launch((int)(launches0 - prof::launches()));   // nothing of the capture ran
        if (capturing && msg) return msg;
        if (const char* m = body(s)) return m;   // direct launches
      } else {
        cudaGraphDestroy(graph);
        w.factor_graph = exec;
        std::memcpy(w.factor_key, key, sizeof(key));
        w.factor_launches = prof::launches() - launches0;
        if (cudaGraphLaunch(exec, s) != cudaSuccess) return "factor graph launch failed";
      }
    }
  }
  w.nz_factored = d.nz;
  w.ne_factored = Ne;
  return nullptr;
}

namespace {

// Where the backward sweep folds its solutions into the quadrature sum
// (Eq. 15): per-node partials qp (N x k, node stride N k), the coefficients,
// and whether this sweep stores (the first solve) or accumulates (a
// refinement step).  qp == nullptr: no folding.
struct QuadOut {
  double* qp;
  const cplx* coef;
  int first;
};

// One pair of sweeps of the two-ended elimination (see Chains): the forward
// sweep runs up both chains (chain 0 from layer 0, chain 1 from layer nz-1)
// to the middle layer K, whose solution x_K = -S'_K g_K starts the backward
// sweep, which then runs out along both chains.  nl: the real nodes swept.
template <int CB, int ST>
const char* solve_sweeps(cudaStream_t s, const Dims& d, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, const double* Rreal, const f2* Rc, const NodeList& nl, const QuadOut& qo,
                         int* status, const int* dactive) {
  float* F = buf<float>(w, B_F);
  f2* Gc = buf<f2>(w, B_GC);
  f2* Tout = buf<f2>(w, B_TOUT);
  float* Bemb = buf<float>(w, B_BEMB);
  const int Ne = d.Ne, V = 2 * Ne;
  CUtensorMap tmF, tmB;
  // split-pair rows: the maps span whole 128-byte blocks (a ragged last
  // block's trailing parts sit past 2n; its unused columns are zero)
  if (!make_map(&tmF, F, d.ldF, (long long)Ne * d.nz * d.n, d.ldF, 128)) return "tensor map (factors) rejected";
  if (!make_map(&tmB, Bemb, d.ldB, (long long)V * d.nblkCB * 2 * CB, d.ldB, 2 * CB))
    return "tensor map (rhs) rejected";
  const int nk = (2 * d.n + tc::kBlockK - 1) / tc::kBlockK;
  const f2* Cf = buf<f2>(w, B_CF);
  const int K = d.K, L0 = K, L1 = d.nz - 1 - K;
  // virtual nodes of a step: the swept nodes on chain 0, and on chain 1 while it has layers
  const NodeList one{nl.count, nl.mask};
  const NodeList both{2 * nl.count, nl.mask | (nl.mask << Ne)};
  tc::Geom geo0{0, d.nz * d.n, 0, d.nblkCB * 2 * CB, nk};
  geo0.split = Ne;
  geo0.active = dactive;
  // coupling work is counted in bytes: per entry the right-hand side and the
  // neighbouring solution (8 B each), g (8 B) and its embedded operand copy
  // (16 B), plus the 9 coefficients of each row
  auto couple_bytes = [&](int nv, double per_entry) { return (double)nv * d.n * ((double)d.k * per_entry + 72.0); };
  auto gemm = [&](const NodeList& vl, int layer0, int layer1, SolveEpi<CB> epi) -> bool {
    tc::Geom geo = geo0;
    geo.node_mask = vl.mask;
    geo.a_row0 = layer0 * d.n;
    geo.a_row0_hi = layer1 * d.n;
    prof::begin(s, prof::SOLVE_GEMM);
    prof::add_work(prof::SOLVE_GEMM, 8.0 * d.n * (double)d.n * d.k * vl.count);
    const bool ok =
        launch_tc<2 * CB, ST, SolveEpi<CB>, kSolveKind>(s, dim3(d.nblkCB, cdiv(d.n, 128), vl.count), tmF, tmB, geo,
                                                         epi, status, true) ==
        cudaSuccess;
    prof::end(s, prof::SOLVE_GEMM);
    return ok;
  };
  // backward products x = -S' s into the nodes' solution columns (and the
  // quadrature shares)
  // quadrature shares: in the epilogue only for the chains in share_chains
  // (the layers no later backward coupling reads), else in the couplings
  auto back_epi = [&](const Chains& ch, int share_chains) {
    SolveEpi<CB> epi{Gc, d.N * d.k, d.N, d.n, d.k, -1.0f};
    epi.node_rows = 1;
    epi.ch = ch;
    if (qo.qp && share_chains) {
      epi.qp = qo.qp;
      epi.sQ = d.N * d.k;
      epi.ldq = d.N;
      epi.coef = qo.coef;
      epi.qfirst = qo.first;
      epi.share_chains = share_chains;
    }
    return epi;
  };
  BwdShares qs;
  qs.qp = qo.qp;
  qs.coef = qo.coef;
  qs.first = qo.first;
  qs.mid = K;
  int launches = 0;
  // forward sweep: g on each chain's layer, then t = S' g for its next layer
  for (int t = 0; t < L0; ++t) {
    const Chains ch{Ne, {t, d.nz - 1 - t}, {0, 0}, 0};
    const NodeList& vl = t < L1 ? both : one;
    prof::begin(s, prof::COUPLE);
    prof::add_work(prof::COUPLE, couple_bytes(vl.count, 40.0));
    launch_pdl(k_mx_couple_fwd<false>, dim3(cdiv(d.n, 128), cdiv(d.k, kCoupleCols), vl.count), dim3(128), 0, s, d, ch,
               t > 0 ? 1 : 0, 0, 0, Cf, Rreal, Rc, Tout, Gc, Bemb, vl, dactive);
    prof::end(s, prof::COUPLE);
    SolveEpi<CB> epi{Tout, (long long)d.n * d.k, d.n, d.n, d.k, 1.0f};
    if (!gemm(vl, t, d.nz - 1 - t, epi)) return "tcgen05 solve launch failed";
    launches += 2;
  }
  // the middle layer: both chains' products meet, x_K = -S'_K g_K
  {
    const Chains ch{Ne, {K, K}, {0, 0}, 0};
    prof::begin(s, prof::COUPLE);
    prof::add_work(prof::COUPLE, couple_bytes(one.count, L1 > 0 ? 48.0 : 40.0));
    launch_pdl(k_mx_couple_fwd<true>, dim3(cdiv(d.n, 128), cdiv(d.k, kCoupleCols), one.count), dim3(128), 0, s, d,
               ch, L0 > 0 ? 1 : 0, 1, L1 > 0 ? 1 : 0, Cf, Rreal, Rc, Tout, Gc, Bemb, one, dactive);
    prof::end(s, prof::COUPLE);
    // x_K: read by the first backward coupling when there is one
    if (!gemm(one, K, K, back_epi(ch, L0 > 0 ? 0 : 1))) return "tcgen05 solve launch failed";
    launches += 2;
  }
  // backward sweep out along both chains: x overwrites g
  for (int u = 0; u < L0; ++u) {
    const Chains ch{Ne, {K - 1 - u, K + 1 + u}, {0, 0}, 0};
    const NodeList& vl = u < L1 ? both : one;
    prof::begin(s, prof::COUPLE);
    prof::add_work(prof::COUPLE, couple_bytes(vl.count, 32.0));
    launch_pdl(k_mx_couple_bwd, dim3(cdiv(d.n, 128), cdiv(d.k, kCoupleCols), vl.count), dim3(128), 0, s, d, ch, Cf,
               Gc, Bemb, vl, dactive, qs);
    prof::end(s, prof::COUPLE);
    // the last layer of each chain: no coupling reads its solution
    const int last = (u == L0 - 1 ? 1 : 0) | (u == L1 - 1 ? 2 : 0);
    if (!gemm(vl, K - 1 - u, K + 1 + u, back_epi(ch, last))) return "tcgen05 solve launch failed";
    launches += 2;
  }
  prof::count_launch(launches);
  return nullptr;
}

// ---- autotuner of the solve GEMM: tile width (complex columns per CTA
// tile) and pipeline stages, timed at the launch shape of the sweeps (both
// chains' virtual nodes, a different layer per launch).  Fewer stages can
// win: two CTAs then share an SM and overlap one's epilogue with the other's
// main loop.
template <int CB, int ST>
float time_solve_gemm(cudaStream_t s, const Dims& d0, MixedWork& w, int* status) {
  Dims d = d0;
  d.CB = CB;
  d.nblkCB = (d.k + CB - 1) / CB;
  const int V = d.K < d.nz - 1 ? 2 * d.Ne : d.Ne;
  CUtensorMap tmF, tmB;
  if (!make_map(&tmF, buf<float>(w, B_F), d.ldF, (long long)d.Ne * d.nz * d.n, d.ldF, 128)) return 1e30f;
  if (!make_map(&tmB, buf<float>(w, B_BEMB), d.ldB, (long long)V * d.nblkCB * 2 * CB, d.ldB, 2 * CB)) return 1e30f;
  const int nk = (2 * d.n + tc::kBlockK - 1) / tc::kBlockK;
  SolveEpi<CB> epi{buf<f2>(w, B_TOUT), (long long)d.n * d.k, d.n, d.n, d.k, 1.0f};
  tc::Geom geo{0, d.nz * d.n, 0, d.nblkCB * 2 * CB, nk};
  geo.split = d.Ne;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // rounds of kTuneRun back-to-back launches on successive layers, as a
  // sweep issues them; the first round warms up, the fastest later one counts
  constexpr int kTuneRun = 8, kTuneRounds = 3;
  float best = 1e30f;
  for (int round = 0; round < kTuneRounds; ++round) {
    cudaEventRecord(a, s);
    for (int r = 0; r < kTuneRun; ++r) {
      const int t = (round * kTuneRun + r) % d.nz;
      geo.a_row0 = t * d.n;
      geo.a_row0_hi = (d.nz - 1 - t) * d.n;
      launch_tc<2 * CB, ST, SolveEpi<CB>, kSolveKind>(s, dim3(d.nblkCB, cdiv(d.n, 128), V), tmF, tmB, geo, epi,
                                                      status);
    }
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (round > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  prof::count_launch(kTuneRun * kTuneRounds);
  return best;
}

std::mutex g_tune_mutex;
std::vector<std::pair<long long, int>> g_tuned;   // (n, k, Ne) key -> CB | ST << 8

constexpr int cfg_of(int cb, int st) { return cb | st << 8; }

// FEAST_SOLVE_TILE="CBxST" (e.g. 64x3) fixes the configuration of every
// solve that starts while it is set, instead of timing the candidates
// (reproducible profiles, since timings under a profiler mean nothing, and
// tests of every configuration); 0 when unset or not a built configuration.
int forced_cfg() {
  const char* env = std::getenv("FEAST_SOLVE_TILE");
  int cb = 0, st = 0;
  if (!env || std::sscanf(env, "%dx%d", &cb, &st) != 2) return 0;
  const int cfg = cfg_of(cb, st);
  const bool built = cfg == cfg_of(8, 4) || cfg == cfg_of(16, 4) || cfg == cfg_of(32, 4) || cfg == cfg_of(64, 3) ||
                     cfg == cfg_of(64, 4);
  return built ? cfg : 0;
}

int tuned_cfg(cudaStream_t s, const Dims& d, MixedWork& w, int* status) {
  if (const int cfg = forced_cfg()) return cfg;
  const long long key = ((long long)d.n << 32) ^ ((long long)d.k << 8) ^ d.Ne;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (auto& kv : g_tuned)
      if (kv.first == key) return kv.second;
  }
  int best_cfg = cfg_of(d.CB, d.ST);
  float best = 1e30f;
  auto consider = [&](int cfg, float ms) {
    if (ms < best) {
      best = ms;
      best_cfg = cfg;
    }
  };
  if (d.k <= 16) {
    consider(cfg_of(8, 4), time_solve_gemm<8, 4>(s, d, w, status));
    consider(cfg_of(16, 4), time_solve_gemm<16, 4>(s, d, w, status));
  } else {
    consider(cfg_of(16, 4), time_solve_gemm<16, 4>(s, d, w, status));
    consider(cfg_of(32, 4), time_solve_gemm<32, 4>(s, d, w, status));
    consider(cfg_of(64, 3), time_solve_gemm<64, 3>(s, d, w, status));
    consider(cfg_of(64, 4), time_solve_gemm<64, 4>(s, d, w, status));
  }
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned.push_back({key, best_cfg});
  return best_cfg;
}

const char* solve_direct(cudaStream_t s, const Dims& d, const cplx* Z, const double* A27, const double* B27,
                         MixedWork& w, const double* Rreal, const f2* Rc, const NodeList& nl, const QuadOut& qo,
                         int* status, const int* dactive = nullptr) {
  switch (cfg_of(d.CB, d.ST)) {
    case cfg_of(8, 4): return solve_sweeps<8, 4>(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status, dactive);
    case cfg_of(16, 4): return solve_sweeps<16, 4>(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status, dactive);
    case cfg_of(32, 4): return solve_sweeps<32, 4>(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status, dactive);
    case cfg_of(64, 3): return solve_sweeps<64, 3>(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status, dactive);
    case cfg_of(64, 4): return solve_sweeps<64, 4>(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status, dactive);
    default: return "solve-GEMM configuration without an instantiation";
  }
}

// One pair of sweeps.  Without kernel timing the ~4 nz launches are replayed
// from a CUDA graph captured on first use (key: shape, tile width, node mask
// and every pointer the launches read or write); a capture that fails falls
// back to direct launches.
const char* solve_once(cudaStream_t s, const Dims& d, const cplx* Z, const double* A27, const double* B27,
                       MixedWork& w, const double* Rreal, const f2* Rc, const std::vector<int>& active,
                       const QuadOut& qo, MixedSolveStats* stats, int* status) {
  NodeList nl{0, 0ULL};
  for (int e = 0; e < d.Ne; ++e)
    if (active[e]) {
      nl.mask |= 1ULL << e;
      ++nl.count;
    }
  if (nl.count == 0) return nullptr;
  if (prof::enabled() || !w.use_graphs) return solve_direct(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status);
  const unsigned long long key[kSweepKey] = {
      (unsigned long long)d.nx | ((unsigned long long)d.ny << 20) | ((unsigned long long)d.nz << 40),
      (unsigned long long)d.k | ((unsigned long long)cfg_of(d.CB, d.ST) << 20) | ((unsigned long long)d.Ne << 40),
      nl.mask,
      (unsigned long long)(uintptr_t)Rreal, (unsigned long long)(uintptr_t)Rc, (unsigned long long)(uintptr_t)Z,
      (unsigned long long)(uintptr_t)A27, (unsigned long long)(uintptr_t)B27, (unsigned long long)(uintptr_t)status,
      (unsigned long long)(uintptr_t)w.bufs[B_F], (unsigned long long)(uintptr_t)w.bufs[B_GC],
      (unsigned long long)(uintptr_t)w.bufs[B_TOUT], (unsigned long long)(uintptr_t)w.bufs[B_BEMB],
      (unsigned long long)(uintptr_t)w.bufs[B_CF], (unsigned long long)d.ldF, 1ULL,
      (unsigned long long)(uintptr_t)qo.qp, (unsigned long long)(uintptr_t)qo.coef, (unsigned long long)qo.first,
      0ULL};
  SweepGraphCache& gc = w.graphs;
  ++gc.clock;
  for (int g = 0; g < kSweepGraphs; ++g) {
    if (!gc.exec[g] || std::memcmp(gc.key[g], key, sizeof(key)) != 0) continue;
    gc.used[g] = gc.clock;
    if (cudaGraphLaunch(gc.exec[g], s) != cudaSuccess) return "sweep graph launch failed";
    prof::count_launch(4 * d.K + 2);
    if (stats) ++stats->graph_sweeps;
    return nullptr;
  }
  // first sighting of this key: run directly and remember it
  bool seen = false;
  for (int g = 0; g < kSweepGraphs && !seen; ++g) seen = std::memcmp(gc.seen[g], key, sizeof(key)) == 0;
  if (!seen) {
    std::memcpy(gc.seen[gc.seen_next], key, sizeof(key));
    gc.seen_next = (gc.seen_next + 1) % kSweepGraphs;
    return solve_direct(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status);
  }
  // second sighting: capture
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = capture_stream(w);
  if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return solve_direct(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status);
  }
  const long long launches0 = prof::launches();
  const char* msg = solve_direct(cs, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status);
  const cudaError_t end = cudaStreamEndCapture(cs, &graph);
  cudaGraphExec_t exec = nullptr;
  if (msg || end != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    prof::count_launch(launches0 - prof::launches());   // nothing of the capture ran
    if (msg) return msg;
    return solve_direct(s, d, Z, A27, B27, w, Rreal, Rc, nl, qo, status);
  }
  cudaGraphDestroy(graph);
  int slot = 0;
  for (int g = 1; g < kSweepGraphs; ++g)
    if (!gc.exec[g] || (gc.exec[slot] && gc.used[g] < gc.used[slot])) slot = g;
  if (gc.exec[slot]) cudaGraphExecDestroy(gc.exec[slot]);
  gc.exec[slot] = exec;
  std::memcpy(gc.key[slot], key, sizeof(key));
  gc.used[slot] = gc.clock;
  if (cudaGraphLaunch(exec, s) != cudaSuccess) return "sweep graph launch failed";
  if (stats) ++stats->graph_sweeps;
  return nullptr;
}

}  // namespace

// Work buffers, kernel attributes and the tuned tile width of a node solve of
// k right-hand sides; *dout: its dimensions.
static const char* solve_prepare(cudaStream_t s, Grid g, int Ne, int k, MixedWork& w, int* status, Dims* dout) {
  Dims d = make_dims(g, Ne, k);
  if (w.nz_factored != d.nz || w.ne_factored != Ne) return "mixed solve called without matching factors";
  const long long sG = d.N * k;
  if (!ensure(w, B_GC, sizeof(f2) * (size_t)Ne * sG, s)) return "out of device memory (node sweeps)";
  if (!ensure(w, B_RC, sizeof(f2) * (size_t)Ne * sG, s)) return "out of device memory (residuals)";
  // products and embedded right-hand sides are per virtual node (two chains)
  if (!ensure(w, B_TOUT, sizeof(f2) * (size_t)2 * Ne * d.n * k, s)) return "out of device memory";
  // embedded RHS operand, sized for every tile width (rows of columns >= k
  // stay zero; re-zeroed when the column count changes)
  const size_t bemb = sizeof(float) * (size_t)2 * Ne * (2 * (size_t)k + 128) * d.ldB;
  const long long blayout = (long long)d.n << 32 | d.ldB;
  const bool shape_changed = w.sizes[B_BEMB] < bemb || w.bemb_k != k || w.bemb_layout != blayout;
  if (!ensure(w, B_BEMB, bemb, s, shape_changed)) return "out of device memory";
  w.bemb_k = k;
  w.bemb_layout = blayout;
  d = make_dims(g, Ne, k, tuned_cfg(s, d, w, status));
  if (shape_changed) cudaMemsetAsync(w.bufs[B_BEMB], 0, bemb, s);
  const long long nblk = cdiv(d.N, kResRows);
  static PerDevice<cudaError_t> res_attr;
  if (res_attr.get(
          [] {
            cudaError_t e = cudaFuncSetAttribute(k_mx_residual, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kResSmem);
            if (e == cudaSuccess)
              e = cudaFuncSetAttribute(k_mx_residual_inc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kResSmem);
            if (e == cudaSuccess)
              e = cudaFuncSetAttribute(k_mx_residual_inc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kResSmem);
            return e;
          },
          cudaErrorInvalidDevice) != cudaSuccess)
    return "refinement residual attribute rejected";
  if (!ensure(w, B_PART, sizeof(double) * 2 * (size_t)Ne * nblk, s)) return "out of device memory";
  if (!ensure(w, B_REL, sizeof(double) * Ne, s)) return "out of device memory";
  if (!ensure(w, B_ACTIVE, sizeof(int) * Ne, s)) return "out of device memory";
  if (!ensure(w, B_RLO, sizeof(f2) * (size_t)Ne * sG, s)) return "out of device memory (residuals)";
  *dout = d;
  return nullptr;
}

namespace {
__global__ void k_selftest_wait(long long polls, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);   // one arrival completes phase 0: none comes
    abort_flag = 0;
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::mbar_wait_limit(&bar, 0, status, &abort_flag, polls);
}
}  // namespace

void selftest_wait(cudaStream_t s, long long polls, int* status) {
  k_selftest_wait<<<1, 32, 0, s>>>(polls, status);
  prof::count_launch();
}

const char* mixed_solve_prepare(cudaStream_t s, Grid g, int Ne, int k, MixedWork& w, int* status) {
  Dims d;
  return solve_prepare(s, g, Ne, k, w, status, &d);
}

const char* mixed_solve(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                        MixedWork& w, const double* RHS, cplx* G, double* Qp, const cplx* coef, int k, double ir_tol,
                        int ir_max, MixedSolveStats* stats, int* status) {
  Dims d;
  if (const char* m = solve_prepare(s, g, Ne, k, w, status, &d)) return m;
  const long long sG = d.N * k;
  const dim3 rgrid(cdiv(d.N, kResRows), Ne);
  const long long nblk = rgrid.x;
  std::vector<int> active(Ne, 1);
  cudaMemcpyAsync(w.bufs[B_ACTIVE], active.data(), sizeof(int) * Ne, cudaMemcpyHostToDevice, s);
  std::vector<double> rel(Ne, 0.0), final_rel(Ne, 0.0);
  const int acc_blocks = (int)std::min<long long>(4096, (sG + 255) / 256);
  // first solve: Q_e = M~^{-1} RHS
  if (const char* m = solve_once(s, d, Z, A27, B27, w, RHS, nullptr, active, QuadOut{Qp, coef, 1}, stats, status))
    return m;
  if (G) {
    k_mx_accumulate<<<dim3(acc_blocks, Ne), 256, 0, s>>>(sG, 1, buf<f2>(w, B_GC), G, buf<int>(w, B_ACTIVE));
    prof::count_launch();
  }
  int steps = 0;
  for (;;) {
    {
      int nact = 0;
      for (int e = 0; e < Ne; ++e) nact += active[e];
      if (steps == 0 && ir_tol >= kFFirstTol) {
        // a loose target: the first residual in double-float from Q_e too
        prof::begin(s, prof::FF_RESIDUAL);
        prof::add_work(prof::FF_RESIDUAL, 216.0 * (double)d.N * k * nact);
        k_mx_residual_inc<true><<<rgrid, kResThreads, kResSmem, s>>>(
            d, Z, A27, B27, buf<f2>(w, B_GC), buf<f2>(w, B_RC), buf<f2>(w, B_RLO), buf<double>(w, B_PART),
            buf<int>(w, B_ACTIVE), RHS, nullptr);
        prof::end(s, prof::FF_RESIDUAL);
      } else if (steps == 0) {
        // the first residual in FP64 from Q_e itself
        prof::begin(s, prof::RESIDUAL);
        prof::add_work(prof::RESIDUAL, 216.0 * (double)d.N * k * nact);   // 108 FP64 FMAs per complex entry
        k_mx_residual<<<rgrid, kResThreads, kResSmem, s>>>(d, Z, A27, B27, RHS, buf<f2>(w, B_GC), buf<f2>(w, B_RC),
                                                           buf<f2>(w, B_RLO), buf<double>(w, B_PART),
                                                           buf<int>(w, B_ACTIVE), nullptr);
        prof::end(s, prof::RESIDUAL);
      } else {
        // later residuals move by the last correction, in double-float
        prof::begin(s, prof::FF_RESIDUAL);
        prof::add_work(prof::FF_RESIDUAL, 216.0 * (double)d.N * k * nact);
        k_mx_residual_inc<false><<<rgrid, kResThreads, kResSmem, s>>>(
            d, Z, A27, B27, buf<f2>(w, B_GC), buf<f2>(w, B_RC), buf<f2>(w, B_RLO), buf<double>(w, B_PART),
            buf<int>(w, B_ACTIVE), nullptr, nullptr);
        prof::end(s, prof::FF_RESIDUAL);
      }
    }
    prof::count_launch(2);
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
    // only the unconverged nodes are swept again
    if (const char* m = solve_once(s, d, Z, A27, B27, w, nullptr, buf<f2>(w, B_RC), active, QuadOut{Qp, coef, 0},
                                   stats, status))
      return m;
    if (G) {
      k_mx_accumulate<<<dim3(acc_blocks, Ne), 256, 0, s>>>(sG, 0, buf<f2>(w, B_GC), G, buf<int>(w, B_ACTIVE));
      prof::count_launch();
    }
    ++steps;
  }
  if (stats) {
    stats->steps_max = std::max(stats->steps_max, steps);
    for (int e = 0; e < Ne; ++e) stats->resid_max = std::max(stats->resid_max, final_rel[e]);
  }
  return nullptr;
}

// ------------------------------------------------------------------ device-side loop

const char* const kNotCaptured = "not captured";

namespace {

// Start of a FEAST loop: the loop counter, the refinement target of the loop
// (loosened in loops 1 and 2 from a random start, as the host-driven loop
// does) and every node active again.
__global__ void k_loop_begin(LoopState* st, double ir_tol, int early, int* active, int Ne) {
  if (threadIdx.x == 0) {
    const int L = ++st->loop;
    double t = ir_tol;
    if (early && L <= 2) t = fmax(ir_tol, early_tol(L));
    st->ir_target = t;
    st->ir_step = 0;
  }
  for (int e = threadIdx.x; e < Ne; e += blockDim.x) active[e] = 1;
}

// After a residual of the node solves: a node whose relative residual meets
// the loop's target stops; the nested WHILE node runs another refinement
// step while any node is left (at most ir_max steps; then the loop fails, as
// does a non-finite residual).
__global__ void k_ir_control(LoopState* st, const double* __restrict__ rel, int* active, int Ne, int ir_max,
                             double ir_tol, cudaGraphConditionalHandle more) {
  if (threadIdx.x != 0) return;
  const double target = st->ir_target;
  int any = 0;
  for (int e = 0; e < Ne; ++e) {
    if (!active[e]) continue;
    const double r = rel[e];
    if (!isfinite(r)) {
      st->fail = 2;
      active[e] = 0;
      continue;
    }
    if (r <= target) {
      active[e] = 0;
      if (target <= ir_tol) st->ir_resid_max = fmax(st->ir_resid_max, r);
    } else {
      any = 1;
    }
  }
  if (any && st->ir_step >= ir_max) {
    st->fail = 1;
    any = 0;
  }
  st->ir_steps_max = max(st->ir_steps_max, st->ir_step);
  if (any) {
    ++st->ir_step;
    ++st->ir_steps_total;
  }
  cudaGraphSetConditional(more, any ? 1u : 0u);
}

// The trace test (Fig. 2 step 6) on the loop's Ritz values (ascending): the
// in-interval count and trace, the relative change against the previous
// loop; the outer WHILE node runs another loop unless the count is unchanged
// and the change is <= tol in a loop refined to ir_tol, the loop cap is
// reached, or a failure was recorded (refinement, or the device status word).
__global__ void k_trace_control(LoopState* st, const double* __restrict__ eps, LoopParams lp, const int* status,
                                cudaGraphConditionalHandle again) {
  if (threadIdx.x != 0) return;
  int count = 0;
  double trace = 0.0, scale = 0.0;
  for (int j = 0; j < lp.M0; ++j) {
    const double x = eps[j];
    if (x >= lp.lmin && x <= lp.lmax) {
      ++count;
      trace += x;
      scale += fabs(x);
    }
  }
  const int L = st->loop;
  if (L - 1 < 64) {
    st->trace_hist[L - 1] = trace;
    st->change_hist[L - 1] = -1.0;
  }
  if (L > 1) {
    const double change = scale > 0.0 ? fabs(trace - st->prev_trace) / scale : 0.0;
    if (L - 1 < 64) st->change_hist[L - 1] = change;
    if (count == st->prev_count && change <= lp.tol && st->ir_target <= lp.ir_tol) st->converged = 1;
  }
  st->count = count;
  st->prev_trace = trace;
  st->prev_count = count;
  const int cont = !st->converged && L < lp.max_loops && !st->fail && *status == 0;
  cudaGraphSetConditional(again, cont ? 1u : 0u);
}

__global__ void k_loop_init(LoopState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    LoopState z{};
    *st = z;
  }
}

// Adds a WHILE node on `handle` (created on the graph being captured on s) at
// the current end of that capture and returns the node's body graph; the
// work captured on s afterwards follows the node.
cudaError_t capture_while(cudaStream_t s, cudaGraphConditionalHandle handle, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edata, &ndeps);
  if (e != cudaSuccess) return e;
  if (cst != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = handle;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, edata, ndeps, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaStream_t loop_stream(cudaStream_t& c) {
  if (!c && cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c = nullptr;
  }
  return c;
}

}  // namespace

const char* mixed_loop(cudaStream_t s, Grid g, int Ne, const cplx* Z, const double* A27, const double* B27,
                       MixedWork& w, const double* RHS, double* Qp, const cplx* coef, int k, const LoopParams& lp,
                       const double* eps, LoopState* st, const LoopHooks& hooks, const unsigned long long* key,
                       int* status) {
  if (w.loop_graph && std::memcmp(w.loop_key, key, sizeof(w.loop_key)) == 0) {
    if (cudaGraphLaunch(w.loop_graph, s) != cudaSuccess) return "loop graph launch failed";
    ++w.loop_replays;
    return nullptr;
  }
  if (std::memcmp(w.loop_seen, key, sizeof(w.loop_seen)) != 0) {
    std::memcpy(w.loop_seen, key, sizeof(w.loop_seen));   // first use of the key: the host-driven loop runs
    return kNotCaptured;
  }
  // the buffers and the tile width of the shape were set by the host-driven run
  Dims d = make_dims(g, Ne, k);
  if (w.nz_factored != d.nz || w.ne_factored != Ne || !w.bufs[B_GC] || !w.bufs[B_RLO]) return kNotCaptured;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const long long tkey = ((long long)d.n << 32) ^ ((long long)d.k << 8) ^ d.Ne;
    int cfg = forced_cfg();
    if (!cfg)
      for (auto& kv : g_tuned)
        if (kv.first == tkey) cfg = kv.second;
    if (!cfg) return kNotCaptured;
    d = make_dims(g, Ne, k, cfg);
  }
  if (w.loop_graph) cudaGraphExecDestroy(w.loop_graph);
  w.loop_graph = nullptr;
  cudaStream_t cs = capture_stream(w), cs2 = loop_stream(w.cap2), cs3 = loop_stream(w.cap3);
  if (!cs || !cs2 || !cs3) return kNotCaptured;
  const dim3 rgrid(cdiv(d.N, kResRows), Ne);
  const long long nblk = rgrid.x;
  int* active = buf<int>(w, B_ACTIVE);
  const NodeList all{Ne, Ne >= 64 ? ~0ULL : ((1ULL << Ne) - 1ULL)};
  const long long launches0 = prof::launches();
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return kNotCaptured;
  const char* msg = nullptr;
  cudaError_t ce = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  bool c2 = false, c3 = false;
  if (ce == cudaSuccess) {
    k_loop_init<<<1, 1, 0, cs>>>(st);
    // conditions: `again` (another FEAST loop) starts at 1 at every launch;
    // `more` (another refinement step) is set before its node is reached
    cudaGraphConditionalHandle again = 0, more = 0;
    cudaGraph_t outer = nullptr, inner = nullptr;
    ce = cudaGraphConditionalHandleCreate(&again, graph, 1u, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) ce = capture_while(cs, again, &outer);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&more, outer, 0u, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) ce = cudaStreamBeginCaptureToGraph(cs2, outer, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    c2 = ce == cudaSuccess;
    long long n_outer0 = 0, n_inner0 = 0, n_inner1 = 0;
    if (c2) {
      n_outer0 = prof::launches();
      // one FEAST loop: B Y, the first solve of every node and its residual
      k_loop_begin<<<1, 64, 0, cs2>>>(st, lp.ir_tol, lp.early, active, Ne);
      prof::count_launch();
      hooks.rhs(cs2);
      msg = solve_direct(cs2, d, Z, A27, B27, w, RHS, nullptr, all, QuadOut{Qp, coef, 1}, status, active);
      k_mx_residual<<<rgrid, kResThreads, kResSmem, cs2>>>(d, Z, A27, B27, RHS, buf<f2>(w, B_GC), buf<f2>(w, B_RC),
                                                            buf<f2>(w, B_RLO), buf<double>(w, B_PART), active,
                                                            &st->ir_target);
      k_mx_residual_inc<true><<<rgrid, kResThreads, kResSmem, cs2>>>(
          d, Z, A27, B27, buf<f2>(w, B_GC), buf<f2>(w, B_RC), buf<f2>(w, B_RLO), buf<double>(w, B_PART), active,
          RHS, &st->ir_target);
      k_mx_resnorm<<<Ne, 256, 0, cs2>>>(Ne, nblk, buf<double>(w, B_PART), buf<double>(w, B_REL), active);
      k_ir_control<<<1, 32, 0, cs2>>>(st, buf<double>(w, B_REL), active, Ne, lp.ir_max, lp.ir_tol, more);
      prof::count_launch(4);
      // the refinement steps: a nested WHILE node
      ce = capture_while(cs2, more, &inner);
      if (ce == cudaSuccess) ce = cudaStreamBeginCaptureToGraph(cs3, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      c3 = ce == cudaSuccess;
      if (c3 && !msg) {
        n_inner0 = prof::launches();
        msg = solve_direct(cs3, d, Z, A27, B27, w, nullptr, buf<f2>(w, B_RC), all, QuadOut{Qp, coef, 0}, status,
                           active);
        k_mx_residual_inc<false><<<rgrid, kResThreads, kResSmem, cs3>>>(
            d, Z, A27, B27, buf<f2>(w, B_GC), buf<f2>(w, B_RC), buf<f2>(w, B_RLO), buf<double>(w, B_PART), active,
            nullptr, nullptr);
        k_mx_resnorm<<<Ne, 256, 0, cs3>>>(Ne, nblk, buf<double>(w, B_PART), buf<double>(w, B_REL), active);
        k_ir_control<<<1, 32, 0, cs3>>>(st, buf<double>(w, B_REL), active, Ne, lp.ir_max, lp.ir_tol, more);
        prof::count_launch(3);
        n_inner1 = prof::launches();
      }
      if (c3) {
        cudaGraph_t done = nullptr;
        const cudaError_t e3 = cudaStreamEndCapture(cs3, &done);
        if (ce == cudaSuccess) ce = e3;
      }
      if (ce == cudaSuccess && !msg) {
        hooks.quad_rr(cs2);
        k_trace_control<<<1, 1, 0, cs2>>>(st, eps, lp, status, again);
        prof::count_launch();
        hooks.next_y(cs2);
        w.loop_inner_launches = n_inner1 - n_inner0;
        w.loop_outer_launches = prof::launches() - n_outer0 - w.loop_inner_launches;
      }
      cudaGraph_t done = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cs2, &done);
      if (ce == cudaSuccess) ce = e2;
    }
    cudaGraph_t done = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(cs, &done);
    if (ce == cudaSuccess) ce = e1;
  }
  cudaGraphExec_t exec = nullptr;
  if (msg || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    prof::count_launch((int)(launches0 - prof::launches()));   // nothing of the capture ran
    if (msg) return msg;
    return kNotCaptured;
  }
  cudaGraphDestroy(graph);
  prof::count_launch((int)(launches0 - prof::launches()));
  w.loop_graph = exec;
  std::memcpy(w.loop_key, key, sizeof(w.loop_key));
  if (cudaGraphLaunch(exec, s) != cudaSuccess) return "loop graph launch failed";
  return nullptr;
}

}  // namespace feast
