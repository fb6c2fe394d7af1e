// Shared device/host helpers of the FEAST GB300 library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>

namespace feast {

// Device status word written by kernels that detect a numerical failure; the
// host reads it at the next synchronisation point.
enum DevStatus : int {
  DEV_OK = 0,
  DEV_PIVOT = 1,      // zero / non-finite pivot in a block inversion
  DEV_JACOBI = 2,     // Jacobi sweeps exhausted
  DEV_BQ_NOT_SPD = 3, // B_Q eigenvalue ratio <= 1e-14
  DEV_TIMEOUT = 4,    // bounded wait gave up
};

// ---------------------------------------------------------------- complex
struct __align__(16) cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx cmake(double r, double i) { return cplx{r, i}; }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx cneg(cplx a) { return cplx{-a.re, -a.im}; }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
__host__ __device__ __forceinline__ cplx cinv(cplx a) {
  // 1/a with scaling against overflow (Smith's method)
  if (fabs(a.re) >= fabs(a.im)) {
    double r = a.im / a.re, d = a.re + a.im * r;
    return cplx{1.0 / d, -r / d};
  } else {
    double r = a.re / a.im, d = a.re * r + a.im;
    return cplx{r / d, -1.0 / d};
  }
}

// ---------------------------------------------------------------- stencil
// Slot s = (dz+1)*9 + (dy+1)*3 + (dx+1).
__host__ __device__ __forceinline__ int slot_dx(int s) { return s % 3 - 1; }
__host__ __device__ __forceinline__ int slot_dy(int s) { return (s / 3) % 3 - 1; }
__host__ __device__ __forceinline__ int slot_dz(int s) { return s / 9 - 1; }

struct Grid {
  int nx, ny, nz;
  __host__ __device__ long long N() const { return (long long)nx * ny * nz; }
  __host__ __device__ int n() const { return nx * ny; }
};

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Set-up that the CUDA runtime keeps per device (kernel attributes such as
// the dynamic shared-memory opt-in, occupancy probes): run once for each
// device ordinal, with that device current, and remember the result.  A
// process may drive several GPUs; a process-wide flag would leave every
// device but the first without the set-up.
constexpr int kMaxDevices = 64;
template <class T>
struct PerDevice {
  std::mutex mu;
  bool done[kMaxDevices] = {};
  T value[kMaxDevices] = {};
  // f() -> T runs on the first call for the current device; fail is returned
  // when the device ordinal cannot be read.
  template <class F>
  T get(F&& f, T fail) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
      cudaGetLastError();
      return fail;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      value[dev] = f();
      done[dev] = true;
    }
    return value[dev];
  }
};

}  // namespace feast
