// Learned initial subspace: a 4-layer MLP (width `width`, SiLU after the first
// three layers) maps per-layer features of an instance (its potential
// scalars, its search interval, the layer position) to the coefficients of
// the start block Y on a separable sine basis of that layer.  Every product
// runs on the tcgen05 tensor cores with BF16 operands and FP32 accumulation
// (kind::f16); parameters are kept in FP32 and updated by Adam.
//
// Layouts (row = sample = one layer of one instance, padded to Bp rows, a
// multiple of 128):
//   H[k]  (Bp x d_k) bf16 row-major: the input of layer k+1 (H[0] = features,
//         padded to 64 columns); the K-major A operand of the forward product
//   HT[k] (d_k x Bp) bf16: H transposed, the B operand of the weight gradient
//   W[k]  (d_{k+1} x d_k) fp32 master, Wb bf16 (forward B operand), WTb
//         (d_k x d_{k+1}) bf16 (B operand of the input gradient)
//   Z[k]  (Bp x d_k) fp32 pre-activations;  G/GT the gradient of the loss
//         with respect to the current pre-activation (fp32 row-major, and
//         bf16 row-major / transposed for the products)
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/feast.h"
#include "prof.cuh"
#include "tc_gemm.cuh"
#include "tma.cuh"

using bf16 = __nv_bfloat16;

struct feast_mlp {
  int in_dim = 0, width = 0, out_dim = 0;
  int d[5] = {};          // padded widths: d[0] = 64, d[1..3] = width, d[4] = out_dim
  int Bcap = 0;           // padded batch capacity
  cudaStream_t stream = nullptr;
  float *W[4] = {}, *b[4] = {}, *mW[4] = {}, *vW[4] = {}, *mb[4] = {}, *vb[4] = {}, *gW[4] = {}, *gb[4] = {};
  bf16 *Wb[4] = {}, *WTb[4] = {};
  bf16 *H[5] = {}, *HT[5] = {};
  float* Z[5] = {};
  float *Gf = nullptr, *Gf2 = nullptr;
  bf16 *Gb = nullptr, *GTb = nullptr, *Gb2 = nullptr, *GTb2 = nullptr;
  double* part = nullptr;
  int status_dummy = 0;
  int* status = nullptr;
  long long steps = 0;
  std::vector<void*> allocs;
};

namespace {

using feast::tc::kBlockM;

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

constexpr int kBN = 128;

// forward: Z = acc + bias; H = act(Z) in bf16, row-major and transposed
struct FwdEpi {
  const float* bias;
  float* Z;
  bf16* H;
  bf16* HT;
  int ld, Bp, act;
  __device__ void operator()(int, int tm, int tn, int row, uint32_t taddr, int, uint8_t*) const {
    const int r = tm * kBlockM + row;
#pragma unroll 1
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      float v[16];
      feast::tc::tmem_ld16(taddr + c0, v);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int col = tn * kBN + c0 + t;
        const float z = v[t] + bias[col];
        Z[(long long)r * ld + col] = z;
        if (H) {
          const bf16 h = __float2bfloat16_rn(act ? silu(z) : z);
          H[(long long)r * ld + col] = h;
          HT[(long long)col * Bp + r] = h;
        }
      }
    }
  }
};

// input gradient of layer k: G = acc * silu'(Z_prev) (fp32 and bf16 copies)
struct DhEpi {
  const float* Zp;
  float* Gf;
  bf16* Gb;
  bf16* GTb;
  int ld, Bp, B;
  __device__ void operator()(int, int tm, int tn, int row, uint32_t taddr, int, uint8_t*) const {
    const int r = tm * kBlockM + row;
#pragma unroll 1
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      float v[16];
      feast::tc::tmem_ld16(taddr + c0, v);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int col = tn * kBN + c0 + t;
        const float g = r < B ? v[t] * silu_grad(Zp[(long long)r * ld + col]) : 0.f;
        Gf[(long long)r * ld + col] = g;
        const bf16 gb = __float2bfloat16_rn(g);
        Gb[(long long)r * ld + col] = gb;
        GTb[(long long)col * Bp + r] = gb;
      }
    }
  }
};

// weight gradient: gW[o, i] = acc (rows = output features, columns = inputs)
struct DwEpi {
  float* gW;
  int ld;
  __device__ void operator()(int, int tm, int tn, int row, uint32_t taddr, int, uint8_t*) const {
    const int o = tm * kBlockM + row;
#pragma unroll 1
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      float v[16];
      feast::tc::tmem_ld16(taddr + c0, v);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int i = tn * kBN + c0 + t;
        if (i < ld) gW[(long long)o * ld + i] = v[t];
      }
    }
  }
};

template <class Epi>
cudaError_t gemm_bf16(cudaStream_t s, const bf16* A, int a_rows, const bf16* Bm, int b_rows, int K, int m_tiles,
                      int n_tiles, const Epi& epi, int* status) {
  CUtensorMap ta, tb;
  if (!feast::make_map_2d(&ta, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, K, a_rows, K, kBlockM) ||
      !feast::make_map_2d(&tb, Bm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, K, b_rows, K, kBN))
    return cudaErrorInvalidValue;
  constexpr size_t smem = feast::tc::Smem<kBN, 4>::kBytes;
  static feast::PerDevice<cudaError_t> attr;   // the opt-in is per device
  if (const cudaError_t e = attr.get(
          [] {
            return cudaFuncSetAttribute(feast::tc::k_tc_gemm<kBN, 4, Epi, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          },
          cudaErrorInvalidDevice))
    return e;
  feast::tc::Geom geo{0, 0, 0, 0, (K + 63) / 64};
  feast::tc::k_tc_gemm<kBN, 4, Epi, 1><<<dim3(n_tiles, m_tiles, 1), feast::tc::kThreads, smem, s>>>(ta, tb, geo, epi,
                                                                                                  status);
  feast::prof::count_launch();
  return cudaGetLastError();
}

// features (B x in, fp32) -> H[0] (Bp x 64) bf16 and its transpose, zero padded
__global__ void k_mlp_input(const float* __restrict__ X, int B, int in_dim, int Bp, bf16* __restrict__ H0,
                            bf16* __restrict__ H0T) {
  const long long total = (long long)Bp * 64;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / 64), c = (int)(t % 64);
    const bf16 v = __float2bfloat16_rn((r < B && c < in_dim) ? X[(long long)r * in_dim + c] : 0.f);
    H0[t] = v;
    H0T[(long long)c * Bp + r] = v;
  }
}

// output gradient of the weighted MSE L = sum w_o (out - target)^2 / (2B)
__global__ void k_mlp_loss(const float* __restrict__ out, const float* __restrict__ target,
                           const float* __restrict__ weights, int B, int Bp, int dout, float* __restrict__ Gf,
                           bf16* __restrict__ Gb, bf16* __restrict__ GTb, double* __restrict__ part) {
  double acc = 0.0;
  const long long total = (long long)Bp * dout;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / dout), o = (int)(t % dout);
    float g = 0.f;
    if (r < B) {
      const float dlt = out[t] - target[(long long)r * dout + o];
      g = weights[o] * dlt / B;
      acc += 0.5 * (double)weights[o] * dlt * dlt / B;
    }
    Gf[t] = g;
    const bf16 gb = __float2bfloat16_rn(g);
    Gb[t] = gb;
    GTb[(long long)o * Bp + r] = gb;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// gb[o] = sum_r G[r, o] (fp32, rows in order)
__global__ void k_mlp_colsum(const float* __restrict__ Gf, int Bp, int dout, float* __restrict__ gb) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= dout) return;
  float s = 0.f;
  for (int r = 0; r < Bp; ++r) s += Gf[(long long)r * dout + o];
  gb[o] = s;
}

// Adam on one parameter array; also refreshes the bf16 copies (and the
// transposed copy of a weight matrix of shape rows x cols)
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                           float c2, bf16* __restrict__ pb, bf16* __restrict__ pbT, int rows, int cols) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float gi = g[t];
    const float mi = b1 * m[t] + (1.f - b1) * gi;
    const float vi = b2 * v[t] + (1.f - b2) * gi * gi;
    m[t] = mi;
    v[t] = vi;
    const float pi = p[t] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[t] = pi;
    if (pb) {
      const bf16 q = __float2bfloat16_rn(pi);
      pb[t] = q;
      const int r = (int)(t / cols), c = (int)(t % cols);
      pbT[(long long)c * rows + r] = q;
    }
  }
}

// bf16 copies of the fp32 weights (row-major and transposed)
__global__ void k_mlp_cast(const float* __restrict__ W, int rows, int cols, int ld_in, bf16* __restrict__ Wb,
                           bf16* __restrict__ WTb, int ld_pad) {
  const long long total = (long long)rows * ld_pad;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / ld_pad), c = (int)(t % ld_pad);
    const bf16 q = __float2bfloat16_rn(c < cols ? W[(long long)r * ld_in + c] : 0.f);
    Wb[t] = q;
    WTb[(long long)c * rows + r] = q;
  }
}

// flag[0] = 1 if any of the n values is not finite
__global__ void k_mlp_finite(const float* __restrict__ v, long long n, int* __restrict__ flag) {
  bool bad = false;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(v[t]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// ---------------------------------------------------------------- sine basis
__device__ __forceinline__ float sine_vec(int p1, int i, int m) {
  // sqrt(2/(m+1)) sin(p pi (i+1)/(m+1)), p1 = p (1-based)
  return sqrtf(2.f / (m + 1)) * sinpif((float)(p1 * (i + 1)) / (float)(m + 1));
}

// Y[l n + ix + nx iy, c] = sum_{q<py, p<px} coef[l, c, q px + p] s_p(ix) s_q(iy)
__global__ void k_sine_expand(const float* __restrict__ coef, int nx, int ny, int nz, int M0, int px, int py,
                              double* __restrict__ Y) {
  const long long N = (long long)nx * ny * nz;
  const int c = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int n = nx * ny;
    const int l = (int)(i / n), ix = (int)(i % n) % nx, iy = (int)(i % n) / nx;
    const float* C = coef + ((long long)l * M0 + c) * px * py;
    float acc = 0.f;
    for (int q = 0; q < py; ++q) {
      const float sy = sine_vec(q + 1, iy, ny);
      float a = 0.f;
      for (int p = 0; p < px; ++p) a = fmaf(C[q * px + p], sine_vec(p + 1, ix, nx), a);
      acc = fmaf(a, sy, acc);
    }
    Y[(long long)c * N + i] = acc;
  }
}

// coef[l, c, q px + p] = sum_{ix, iy} X[l n + ix + nx iy, c] s_p(ix) s_q(iy)
__global__ void k_sine_project(const double* __restrict__ X, int nx, int ny, int nz, int M0, int px, int py,
                               float* __restrict__ coef) {
  extern __shared__ float xs[];
  const int l = blockIdx.x, c = blockIdx.y;
  const int n = nx * ny;
  const long long N = (long long)n * nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) xs[t] = (float)X[(long long)c * N + (long long)l * n + t];
  __syncthreads();
  for (int pq = threadIdx.x; pq < px * py; pq += blockDim.x) {
    const int p = pq % px, q = pq / px;
    float acc = 0.f;
    for (int iy = 0; iy < ny; ++iy) {
      float a = 0.f;
      for (int ix = 0; ix < nx; ++ix) a = fmaf(xs[iy * nx + ix], sine_vec(p + 1, ix, nx), a);
      acc = fmaf(a, sine_vec(q + 1, iy, ny), acc);
    }
    coef[((long long)l * M0 + c) * px * py + pq] = acc;
  }
}

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
T* dalloc(feast_mlp* net, size_t count) {
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaMemsetAsync(p, 0, count * sizeof(T), net->stream);
  net->allocs.push_back(p);
  return static_cast<T*>(p);
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

// forward pass of B rows (features already in H[0]); output in Z[4]
feast_status forward_rows(feast_mlp* net, int B) {
  const int Bp = ((B + kBlockM - 1) / kBlockM) * kBlockM;
  for (int k = 0; k < 4; ++k) {
    const int din = net->d[k], dout = net->d[k + 1];
    FwdEpi epi{net->b[k], net->Z[k + 1], k < 3 ? net->H[k + 1] : nullptr, k < 3 ? net->HT[k + 1] : nullptr, dout, Bp,
               k < 3 ? 1 : 0};
    if (gemm_bf16(net->stream, net->H[k], Bp, net->Wb[k], dout, din, Bp / kBlockM, dout / kBN, epi, net->status) !=
        cudaSuccess)
      return FEAST_ERR_CUDA;
  }
  return FEAST_OK;
}

}  // namespace

extern "C" {

feast_status feast_mlp_create(feast_mlp** out, int in_dim, int width, int out_dim, int max_batch, void* stream) {
  if (!out || in_dim < 1 || in_dim > 64 || width < 128 || width % 128 || out_dim < 128 || out_dim % 128 ||
      max_batch < 1)
    return FEAST_ERR_ARG;
  feast_mlp* net = new feast_mlp();
  net->in_dim = in_dim;
  net->width = width;
  net->out_dim = out_dim;
  net->stream = static_cast<cudaStream_t>(stream);
  net->d[0] = 64;
  net->d[1] = net->d[2] = net->d[3] = width;
  net->d[4] = out_dim;
  net->Bcap = ((max_batch + kBlockM - 1) / kBlockM) * kBlockM;
  bool ok = true;
  for (int k = 0; k < 4 && ok; ++k) {
    const size_t nw = (size_t)net->d[k + 1] * net->d[k];
    ok = (net->W[k] = dalloc<float>(net, nw)) && (net->b[k] = dalloc<float>(net, net->d[k + 1])) &&
         (net->mW[k] = dalloc<float>(net, nw)) && (net->vW[k] = dalloc<float>(net, nw)) &&
         (net->mb[k] = dalloc<float>(net, net->d[k + 1])) && (net->vb[k] = dalloc<float>(net, net->d[k + 1])) &&
         (net->gW[k] = dalloc<float>(net, nw)) && (net->gb[k] = dalloc<float>(net, net->d[k + 1])) &&
         (net->Wb[k] = dalloc<bf16>(net, nw)) && (net->WTb[k] = dalloc<bf16>(net, nw));
  }
  int dmax = std::max(width, out_dim);
  for (int k = 0; k < 5 && ok; ++k) {
    const size_t na = (size_t)net->Bcap * net->d[k];
    ok = (net->H[k] = dalloc<bf16>(net, na)) && (net->HT[k] = dalloc<bf16>(net, na)) &&
         (net->Z[k] = dalloc<float>(net, na));
  }
  ok = ok && (net->Gf = dalloc<float>(net, (size_t)net->Bcap * dmax)) &&
       (net->Gf2 = dalloc<float>(net, (size_t)net->Bcap * dmax)) &&
       (net->Gb = dalloc<bf16>(net, (size_t)net->Bcap * dmax)) &&
       (net->GTb = dalloc<bf16>(net, (size_t)net->Bcap * dmax)) &&
       (net->Gb2 = dalloc<bf16>(net, (size_t)net->Bcap * dmax)) &&
       (net->GTb2 = dalloc<bf16>(net, (size_t)net->Bcap * dmax)) && (net->part = dalloc<double>(net, 4096)) &&
       (net->status = dalloc<int>(net, 4));
  if (!ok) {
    feast_mlp_destroy(net);
    return FEAST_ERR_OOM;
  }
  *out = net;
  return FEAST_OK;
}

feast_status feast_mlp_destroy(feast_mlp* net) {
  if (!net) return FEAST_OK;
  cudaStreamSynchronize(net->stream);
  for (void* p : net->allocs) cudaFree(p);
  delete net;
  return FEAST_OK;
}

feast_status feast_mlp_set_layer(feast_mlp* net, int k, const float* W, const float* b) {
  if (!net || k < 0 || k > 3 || !W || !b) return FEAST_ERR_ARG;
  const int rows = net->d[k + 1], cols = (k == 0) ? net->in_dim : net->d[k];
  const int ldp = net->d[k];
  // the layer's fp32 master keeps the padded width (zero columns beyond the inputs)
  std::vector<float> hostW;
  const float* srcW = W;
  if (is_dev(W)) {
    hostW.resize((size_t)rows * cols);
    if (cudaMemcpy(hostW.data(), W, hostW.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return FEAST_ERR_CUDA;
    srcW = hostW.data();
  }
  std::vector<float> padded((size_t)rows * ldp, 0.f);
  for (int r = 0; r < rows; ++r) std::memcpy(&padded[(size_t)r * ldp], srcW + (size_t)r * cols, cols * sizeof(float));
  if (cudaMemcpyAsync(net->W[k], padded.data(), padded.size() * sizeof(float), cudaMemcpyHostToDevice, net->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(net->b[k], b, rows * sizeof(float), is_dev(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      net->stream) != cudaSuccess)
    return FEAST_ERR_CUDA;
  k_mlp_cast<<<blocks_for((long long)rows * ldp), 256, 0, net->stream>>>(net->W[k], rows, ldp, ldp, net->Wb[k],
                                                                       net->WTb[k], ldp);
  feast::prof::count_launch();
  cudaMemsetAsync(net->mW[k], 0, sizeof(float) * rows * ldp, net->stream);
  cudaMemsetAsync(net->vW[k], 0, sizeof(float) * rows * ldp, net->stream);
  cudaMemsetAsync(net->mb[k], 0, sizeof(float) * rows, net->stream);
  cudaMemsetAsync(net->vb[k], 0, sizeof(float) * rows, net->stream);
  net->steps = 0;
  return cudaStreamSynchronize(net->stream) == cudaSuccess ? FEAST_OK : FEAST_ERR_CUDA;
}

feast_status feast_mlp_get_layer(feast_mlp* net, int k, float* W, float* b, float* gW, float* gb) {
  if (!net || k < 0 || k > 3) return FEAST_ERR_ARG;
  const int rows = net->d[k + 1], cols = (k == 0) ? net->in_dim : net->d[k], ldp = net->d[k];
  std::vector<float> tmp((size_t)rows * ldp);
  auto get = [&](const float* src, float* dst, bool matrix) -> bool {
    if (!dst) return true;
    if (!matrix)
      return cudaMemcpy(dst, src, rows * sizeof(float), is_dev(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost) ==
             cudaSuccess;
    if (cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    std::vector<float> packed((size_t)rows * cols);
    for (int r = 0; r < rows; ++r) std::memcpy(&packed[(size_t)r * cols], &tmp[(size_t)r * ldp], cols * sizeof(float));
    return cudaMemcpy(dst, packed.data(), packed.size() * sizeof(float),
                      is_dev(dst) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost) == cudaSuccess;
  };
  if (cudaStreamSynchronize(net->stream) != cudaSuccess) return FEAST_ERR_CUDA;
  return (get(net->W[k], W, true) && get(net->b[k], b, false) && get(net->gW[k], gW, true) &&
          get(net->gb[k], gb, false))
             ? FEAST_OK
             : FEAST_ERR_CUDA;
}

feast_status feast_mlp_forward(feast_mlp* net, const float* X, int B, float* out) {
  if (!net || !X || !out || B < 1 || B > net->Bcap) return FEAST_ERR_ARG;
  const int Bp = ((B + kBlockM - 1) / kBlockM) * kBlockM;
  k_mlp_input<<<blocks_for((long long)Bp * 64), 256, 0, net->stream>>>(X, B, net->in_dim, Bp, net->H[0], net->HT[0]);
  feast::prof::count_launch();
  if (forward_rows(net, B) != FEAST_OK) return FEAST_ERR_CUDA;
  if (cudaMemcpy2DAsync(out, sizeof(float) * net->out_dim, net->Z[4], sizeof(float) * net->out_dim,
                        sizeof(float) * net->out_dim, B, cudaMemcpyDeviceToDevice, net->stream) != cudaSuccess)
    return FEAST_ERR_CUDA;
  return cudaStreamSynchronize(net->stream) == cudaSuccess ? FEAST_OK : FEAST_ERR_CUDA;
}

// Gradients of the weighted MSE of B rows (into the network's gradient
// buffers); with lr > 0 an Adam step follows.  *loss receives the loss.
feast_status feast_mlp_train_step(feast_mlp* net, const float* X, const float* target, const float* weights, int B,
                                  float lr, double* loss) {
  if (!net || !X || !target || !weights || B < 1 || B > net->Bcap) return FEAST_ERR_ARG;
  cudaStream_t s = net->stream;
  const int Bp = ((B + kBlockM - 1) / kBlockM) * kBlockM;
  k_mlp_input<<<blocks_for((long long)Bp * 64), 256, 0, s>>>(X, B, net->in_dim, Bp, net->H[0], net->HT[0]);
  feast::prof::count_launch();
  if (forward_rows(net, B) != FEAST_OK) return FEAST_ERR_CUDA;
  const int dout = net->d[4];
  const int lb = blocks_for((long long)Bp * dout);
  k_mlp_loss<<<lb, 256, 0, s>>>(net->Z[4], target, weights, B, Bp, dout, net->Gf, net->Gb, net->GTb, net->part);
  feast::prof::count_launch();
  float* Gf = net->Gf;
  bf16 *Gb = net->Gb, *GTb = net->GTb;
  float* Gf_next = net->Gf2;
  bf16 *Gb_next = net->Gb2, *GTb_next = net->GTb2;
  for (int k = 3; k >= 0; --k) {
    const int din = net->d[k], dk = net->d[k + 1];
    // weight gradient gW[o, i] = sum_r G[r, o] H_k[r, i]: A = G^T (dk x Bp), B = H_k^T (din x Bp)
    DwEpi dw{net->gW[k], din};
    if (gemm_bf16(s, GTb, dk, net->HT[k], din, Bp, dk / kBlockM, (din + kBN - 1) / kBN, dw, net->status) != cudaSuccess)
      return FEAST_ERR_CUDA;
    k_mlp_colsum<<<(dk + 255) / 256, 256, 0, s>>>(Gf, Bp, dk, net->gb[k]);
    feast::prof::count_launch();
    if (k > 0) {
      // input gradient through layer k and the activation of layer k-1:
      // A = G (Bp x dk), B = W_k^T (din x dk)
      DhEpi dh{net->Z[k], Gf_next, Gb_next, GTb_next, din, Bp, B};
      if (gemm_bf16(s, Gb, Bp, net->WTb[k], din, dk, Bp / kBlockM, din / kBN, dh, net->status) != cudaSuccess)
        return FEAST_ERR_CUDA;
      std::swap(Gf, Gf_next);
      std::swap(Gb, Gb_next);
      std::swap(GTb, GTb_next);
    }
  }
  if (lr > 0.f) {
    ++net->steps;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)net->steps), c2 = 1.f - powf(b2, (float)net->steps);
    for (int k = 0; k < 4; ++k) {
      const int rows = net->d[k + 1], cols = net->d[k];
      const long long nw = (long long)rows * cols;
      k_mlp_adam<<<blocks_for(nw), 256, 0, s>>>(net->W[k], net->gW[k], net->mW[k], net->vW[k], nw, lr, b1, b2, eps, c1,
                                               c2, net->Wb[k], net->WTb[k], rows, cols);
      k_mlp_adam<<<blocks_for(rows), 256, 0, s>>>(net->b[k], net->gb[k], net->mb[k], net->vb[k], rows, lr, b1, b2, eps,
                                                 c1, c2, nullptr, nullptr, rows, 1);
      feast::prof::count_launch(2);
    }
  }
  std::vector<double> part(lb);
  cudaMemcpyAsync(part.data(), net->part, sizeof(double) * lb, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return FEAST_ERR_CUDA;
  int st = 0;
  cudaMemcpy(&st, net->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (st != 0) return FEAST_ERR_TIMEOUT;
  if (loss) {
    double L = 0.0;
    for (double v : part) L += v;
    *loss = L;
  }
  return FEAST_OK;
}

feast_status feast_sine_expand(const float* coef, int nx, int ny, int nz, int M0, int px, int py, double* Y,
                               void* stream) {
  if (!coef || !Y || nx < 1 || ny < 1 || nz < 1 || M0 < 1 || px < 1 || py < 1 || px > nx || py > ny)
    return FEAST_ERR_ARG;
  const long long N = (long long)nx * ny * nz;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_sine_expand<<<dim3(blocks_for(N), M0), 256, 0, s>>>(coef, nx, ny, nz, M0, px, py, Y);
  feast::prof::count_launch();
  return cudaGetLastError() == cudaSuccess ? FEAST_OK : FEAST_ERR_CUDA;
}

feast_status feast_sine_project(const double* X, int nx, int ny, int nz, int M0, int px, int py, float* coef,
                                void* stream) {
  if (!coef || !X || nx < 1 || ny < 1 || nz < 1 || M0 < 1 || px < 1 || py < 1 || px > nx || py > ny ||
      nx * ny > 12000)
    return FEAST_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_sine_project<<<dim3(nz, M0), 128, sizeof(float) * nx * ny, s>>>(X, nx, ny, nz, M0, px, py, coef);
  feast::prof::count_launch();
  return cudaGetLastError() == cudaSuccess ? FEAST_OK : FEAST_ERR_CUDA;
}

feast_status feast_predict_Y(feast_mlp* net, const float* features, int nx, int ny, int nz, int M0, int px, int py,
                             double* Y) {
  if (!net || !features || !Y || nz > net->Bcap || net->out_dim != M0 * px * py) return FEAST_ERR_ARG;
  const int Bp = ((nz + kBlockM - 1) / kBlockM) * kBlockM;
  k_mlp_input<<<blocks_for((long long)Bp * 64), 256, 0, net->stream>>>(features, nz, net->in_dim, Bp, net->H[0],
                                                                      net->HT[0]);
  feast::prof::count_launch();
  if (forward_rows(net, nz) != FEAST_OK) return FEAST_ERR_CUDA;
  const long long nout = (long long)nz * net->out_dim;
  cudaMemsetAsync(net->status + 1, 0, sizeof(int), net->stream);
  k_mlp_finite<<<blocks_for(nout), 256, 0, net->stream>>>(net->Z[4], nout, net->status + 1);
  feast::prof::count_launch();
  int bad = 0;
  if (cudaMemcpyAsync(&bad, net->status + 1, sizeof(int), cudaMemcpyDeviceToHost, net->stream) != cudaSuccess ||
      cudaStreamSynchronize(net->stream) != cudaSuccess)
    return FEAST_ERR_CUDA;
  if (bad) return FEAST_ERR_NONFINITE;
  // rows of Z[4] are layers, columns (c, pq): exactly the coefficient layout
  const feast_status st = feast_sine_expand(net->Z[4], nx, ny, nz, M0, px, py, Y, net->stream);
  if (st != FEAST_OK) return st;
  return cudaStreamSynchronize(net->stream) == cudaSuccess ? FEAST_OK : FEAST_ERR_CUDA;
}

}  // extern "C"
