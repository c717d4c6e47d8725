// Shared device/host helpers for libnne (complex arithmetic, launch checks).
#pragma once
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <stdint.h>
#include <math.h>

#include "../../include/nne.h"

namespace nne {

template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// |a|^2 in float64 whatever R.
template <typename R> __host__ __device__ __forceinline__ double norm2d(cx<R> a) {
  return (double)a.re * (double)a.re + (double)a.im * (double)a.im;
}
// Phase of a reflector pivot.  complex64 entries below ~1e-19 have denormal
// (few-bit) or zero float32 squares, so |x0| taken from x0.re^2 + x0.im^2 is
// wrong there, |alpha| differs from ||x|| and the reflector built from it is
// not unitary (a Clifford circuit's tensors, scaled permutations plus rounding
// noise down to 1e-24, hit this).  The phase is taken from x0 / max(|re|, |im|):
// x0 = ax0 (pr + i pi) with |pr + i pi| = 1 to rounding; (1, 0) and 0 for x0 = 0.
template <typename R, typename T>
__host__ __device__ __forceinline__ void unit_phase_of(cx<R> x0, T* pr, T* pi, T* ax0) {
  const T s = fmax(fabs((T)x0.re), fabs((T)x0.im));
  if (!(s > T(0))) {
    *pr = T(1);
    *pi = T(0);
    *ax0 = T(0);
    return;
  }
  const T a = (T)x0.re / s, b = (T)x0.im / s;
  const T r = sqrt(a * a + b * b);
  *pr = a / r;
  *pi = b / r;
  *ax0 = s * r;
}
// a += b * c
template <typename R> __host__ __device__ __forceinline__ void fma_(cx<R>& a, cx<R> b, cx<R> c) {
  a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
// a += conj(b) * c
template <typename R> __host__ __device__ __forceinline__ void fmac_(cx<R>& a, cx<R> b, cx<R> c) {
  a.re = fma(b.re, c.re, fma(b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(-b.im, c.re, a.im));
}
template <typename R> __device__ __forceinline__ cx<R> shfl_xor(cx<R> v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
}
template <typename R> __device__ __forceinline__ cx<R> shfl_idx(cx<R> v, int src) {
  return mk(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}
template <typename R> __device__ __forceinline__ cx<R> warp_sum(cx<R> v) {
  for (int m = 16; m > 0; m >>= 1) v = v + shfl_xor(v, m);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_sum_r(T v) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Matrix operation flags for the batched complex GEMM.
enum Op { OP_N = 0, OP_C = 1 };

// Strided batch descriptor: matrix b of a batch starts at ptr + b * stride (elements).
template <typename T>
struct Batched {
  T* ptr;
  long long stride;
  int ld;
};

}  // namespace nne

#define NNE_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) return nne::set_cuda_error(_e, #expr, __FILE__, __LINE__); \
  } while (0)

namespace nne {
// Kernel classes for launch accounting / event timing (nne_prof_collect).
enum ProfClass {
  K_GEMM = 0, K_SUPEROP_APPLY = 1, K_TRIDIAG = 2, K_BISECT = 3, K_INVITER = 4, K_BACKTRANSFORM = 5,
  K_QR_FACTOR = 6, K_WY = 7, K_ELEMWISE = 8, K_SWEEP_ENV = 9, K_SWEEP_OBS = 10, K_SUPEROP_BUILD = 11,
  K_FIT = 12, K_GEMM_TC = 13, K_BISECT64 = 14, PROF_CLASSES = 16
};
class ProfScope {
 public:
  // work: algorithmic flops (GEMM) or bytes (sweeps) of these launches, 0 if not tracked
  ProfScope(cudaStream_t st, int cls, int kernels = 1, double work = 0.0);
  ~ProfScope();
 private:
  cudaStream_t st_;
  int cls_;
  bool on_;
  double work_;
  cudaEvent_t a_, b_;
};
nne_status set_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (and allow non-portable cluster sizes if asked).  The limit
// only ever grows, under a lock, so launches of the same kernel with other
// sizes from other host threads stay valid.
cudaError_t ensure_kernel_smem(const void* func, size_t bytes, bool nonportable_cluster);
nne_status set_error(nne_status s, const char* fmt, ...);
}  // namespace nne
