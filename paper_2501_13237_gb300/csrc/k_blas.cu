// Batched complex GEMM (SIMT), the superoperator epilogue, and small
// elementwise / reduction kernels used by the gate step.
#include <type_traits>

#include "kernels.cuh"

namespace nne {

// C[z] = alpha * op(A[z]) * op(B[z]) + beta * C[z], row-major, M x N x K.
// op N: element (i, k) of A is A[i * lda + k]; op C: conj(A[k * lda + i]).
template <typename R, int OPA, int OPB>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K, cx<R> alpha,
                                                     const cx<R>* __restrict__ A, long long sA, int lda,
                                                     const cx<R>* __restrict__ B, long long sB, int ldb,
                                                     cx<R> beta, cx<R>* __restrict__ C, long long sC, int ldc) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ cx<R> As[BK][BM];
  __shared__ cx<R> Bs[BK][BN];
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  cx<R> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int i, k;
      if (OPA == OP_N) { k = e % BK; i = e / BK; } else { i = e % BM; k = e / BM; }
      const int gi = row0 + i, gk = k0 + k;
      cx<R> v = mk<R>(0, 0);
      if (gi < M && gk < K) v = (OPA == OP_N) ? A[(long long)gi * lda + gk] : conj(A[(long long)gk * lda + gi]);
      As[k][i] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int j, k;
      if (OPB == OP_N) { j = e % BN; k = e / BN; } else { k = e % BK; j = e / BK; }
      const int gj = col0 + j, gk = k0 + k;
      cx<R> v = mk<R>(0, 0);
      if (gj < N && gk < K) v = (OPB == OP_N) ? B[(long long)gk * ldb + gj] : conj(B[(long long)gj * ldb + gk]);
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      cx<R> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fma_(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.re != R(0) || beta.im != R(0));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = row0 + ty + 16 * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = col0 + tx + 16 * j;
      if (gj >= N) continue;
      cx<R> v = alpha * acc[i][j];
      cx<R>* c = C + (long long)gi * ldc + gj;
      if (use_beta) v = v + beta * (*c);
      *c = v;
    }
  }
}

template <typename R>
cudaError_t cgemm(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<R> alpha, const cx<R>* A,
                  long long sA, int lda, const cx<R>* B, long long sB, int ldb, cx<R> beta, cx<R>* C,
                  long long sC, int ldc, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (std::is_same<R, float>::value && tensor_cores_enabled() && gemm_tma_enabled() && M >= 128 && N >= 64 &&
      K >= 64 && cgemm_tma_available())
    return cgemm_tma(st, opA, opB, M, N, K, *reinterpret_cast<const cx<float>*>(&alpha),
                     reinterpret_cast<const cx<float>*>(A), sA, lda, reinterpret_cast<const cx<float>*>(B), sB, ldb,
                     *reinterpret_cast<const cx<float>*>(&beta), reinterpret_cast<cx<float>*>(C), sC, ldc, batch);
  if (std::is_same<R, float>::value && tensor_cores_enabled() && M >= 64 && N >= 64 && K >= 64)
    return cgemm_tc(st, opA, opB, M, N, K, *reinterpret_cast<const cx<float>*>(&alpha),
                    reinterpret_cast<const cx<float>*>(A), sA, lda, reinterpret_cast<const cx<float>*>(B), sB, ldb,
                    *reinterpret_cast<const cx<float>*>(&beta), reinterpret_cast<cx<float>*>(C), sC, ldc, batch);
  ProfScope ps(st, K_GEMM, 1, 8.0 * M * N * (double)K * batch);
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  if (opA == OP_N && opB == OP_N)
    cgemm_kernel<R, OP_N, OP_N><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc);
  else if (opA == OP_N && opB == OP_C)
    cgemm_kernel<R, OP_N, OP_C><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc);
  else if (opA == OP_C && opB == OP_N)
    cgemm_kernel<R, OP_C, OP_N><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc);
  else
    cgemm_kernel<R, OP_C, OP_C><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc);
  return cudaGetLastError();
}

// In-place superoperator on X = theta ((4 dl) x (4 dr), rows (a, s1), cols (s2, b)):
// X[a,s1',s2',b] = sum_{s1,s2} G[4 s1' + s2'][4 s1 + s2] X[a,s1,s2,b].
// One thread per (a, b) holds all 16 (s1, s2) entries.
template <typename R>
__global__ void __launch_bounds__(256) apply_superop_kernel(cx<R>* X, long long sX, int dl, int dr,
                                                             const double* __restrict__ G, long long sG) {
  __shared__ cx<R> g[256];
  const int z = blockIdx.z;
  X += z * sX;
  G += 2 * z * sG;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) g[i] = mk<R>((R)G[2 * i], (R)G[2 * i + 1]);
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)dl * dr) return;
  const int a = (int)(idx / dr), b = (int)(idx % dr);
  const long long ld = 4LL * dr;
  cx<R> t[16];
#pragma unroll
  for (int s1 = 0; s1 < 4; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) t[4 * s1 + s2] = X[(4LL * a + s1) * ld + (long long)s2 * dr + b];
#pragma unroll
  for (int u1 = 0; u1 < 4; ++u1)
#pragma unroll
    for (int u2 = 0; u2 < 4; ++u2) {
      cx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int v = 0; v < 16; ++v) fma_(acc, g[16 * (4 * u1 + u2) + v], t[v]);
      X[(4LL * a + u1) * ld + (long long)u2 * dr + b] = acc;
    }
}

template <typename R>
cudaError_t apply_superop(cudaStream_t st, cx<R>* X, long long sX, int dl, int dr, const double* G, long long sG,
                          int batch) {
  const long long work = (long long)dl * dr;
  ProfScope ps(st, K_SUPEROP_APPLY);
  dim3 grid((unsigned)((work + 255) / 256), 1, batch);
  apply_superop_kernel<R><<<grid, 256, 0, st>>>(X, sX, dl, dr, G, sG);
  return cudaGetLastError();
}

// Partial sums of |x|^2 over `count` elements per batch entry, `parts` blocks per
// entry; partial p of entry z goes to out[z * parts + p] (deterministic order).
template <typename R>
__global__ void __launch_bounds__(256) sumsq_partial_kernel(const cx<R>* X, long long sX, long long count,
                                                             double* out, int parts) {
  const int z = blockIdx.y;
  X += z * sX;
  double s = 0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < count; i += (long long)parts * 256) {
    cx<R> v = X[i];
    s += (double)v.re * v.re + (double)v.im * v.im;
  }
  s = warp_sum_r(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[z * parts + blockIdx.x] = t;
  }
}

template <typename R>
cudaError_t sumsq_partial(cudaStream_t st, const cx<R>* X, long long sX, long long count, double* out, int parts,
                          int batch) {
  ProfScope ps(st, K_ELEMWISE);
  dim3 grid(parts, batch);
  sumsq_partial_kernel<R><<<grid, 256, 0, st>>>(X, sX, count, out, parts);
  return cudaGetLastError();
}

// Gate bookkeeping per instance: kept = sum of kept parts, total = sum of total
// parts; scale[z] = 1/sqrt(kept); log_norm += log sqrt(kept); log_fid += log(kept/total).
// kept = ||C||^2 normalises the kept factor C; f = kept / total, or, when the
// discarded weight ||X - P X||^2 is given, f = (total - discarded) / total.
__global__ void finish_gate_kernel(const double* kept_parts, const double* total_parts, const double* disc_parts,
                                   int parts, int batch, double* scale, double* log_norm, double* log_fid, int* err) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= batch) return;
  double kept = 0, total = 0, disc = 0;
  for (int p = 0; p < parts; ++p) kept += kept_parts[z * parts + p];
  if (total_parts) {
    for (int p = 0; p < parts; ++p) total += total_parts[z * parts + p];
  } else {
    total = kept;
  }
  if (disc_parts)
    for (int p = 0; p < parts; ++p) disc += disc_parts[z * parts + p];
  if (!(kept > 0) || !(total > 0) || !isfinite(kept) || !isfinite(total) || !isfinite(disc)) {
    atomicExch(err, NNE_ERR_NOCONV);
    scale[z] = 1.0;
    return;
  }
  const double nrm = sqrt(kept);
  scale[z] = 1.0 / nrm;
  log_norm[z] += log(nrm);
  double f = disc_parts ? (total - disc) / total : kept / total;
  if (f > 1.0) f = 1.0;
  if (!(f > 0)) {
    atomicExch(err, NNE_ERR_NOCONV);
    return;
  }
  log_fid[z] += log(f);
}

template <typename R>
__global__ void scale_kernel(cx<R>* X, long long sX, long long count, const double* scale) {
  const int z = blockIdx.y;
  const R s = (R)scale[z];
  X += z * sX;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    X[i] = s * X[i];
}

template <typename R>
cudaError_t scale_batched(cudaStream_t st, cx<R>* X, long long sX, long long count, const double* scale, int batch) {
  ProfScope ps(st, K_ELEMWISE);
  int blocks = (int)std::min<long long>((count + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  scale_kernel<R><<<dim3(blocks, batch), 256, 0, st>>>(X, sX, count, scale);
  return cudaGetLastError();
}

// Y[z] (cols x rows) = conj(X[z])^T or X[z]^T (rows x cols), row-major both.
template <typename R, bool CONJ>
__global__ void transpose_kernel(const cx<R>* X, long long sX, int rows, int cols, int ldx, cx<R>* Y, long long sY,
                                 int ldy) {
  __shared__ cx<R> tile[32][33];
  const int z = blockIdx.z;
  X += z * sX;
  Y += z * sY;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = X[(long long)r * ldx + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) {
      cx<R> v = tile[threadIdx.x][i];
      Y[(long long)c * ldy + r] = CONJ ? conj(v) : v;
    }
  }
}

template <typename R>
cudaError_t transpose(cudaStream_t st, bool conj_, const cx<R>* X, long long sX, int rows, int cols, int ldx,
                      cx<R>* Y, long long sY, int ldy, int batch) {
  ProfScope ps(st, K_ELEMWISE);
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  dim3 block(32, 8);
  if (conj_)
    transpose_kernel<R, true><<<grid, block, 0, st>>>(X, sX, rows, cols, ldx, Y, sY, ldy);
  else
    transpose_kernel<R, false><<<grid, block, 0, st>>>(X, sX, rows, cols, ldx, Y, sY, ldy);
  return cudaGetLastError();
}

template <typename R>
__global__ void conj_inplace_kernel(cx<R>* X, long long sX, long long count) {
  X += blockIdx.y * sX;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    X[i].im = -X[i].im;
}

template <typename R>
cudaError_t conj_inplace(cudaStream_t st, cx<R>* X, long long sX, long long count, int batch) {
  ProfScope ps(st, K_ELEMWISE);
  int blocks = (int)std::min<long long>((count + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  conj_inplace_kernel<R><<<dim3(blocks, batch), 256, 0, st>>>(X, sX, count);
  return cudaGetLastError();
}

// Rows x cols identity (1 on the diagonal of the leading square block).
template <typename R>
__global__ void identity_kernel(cx<R>* X, long long sX, int rows, int cols) {
  X += blockIdx.y * sX;
  const long long count = (long long)rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    X[i] = mk<R>(r == c ? R(1) : R(0), R(0));
  }
}

template <typename R>
cudaError_t identity(cudaStream_t st, cx<R>* X, long long sX, int rows, int cols, int batch) {
  const long long count = (long long)rows * cols;
  ProfScope ps(st, K_ELEMWISE);
  int blocks = (int)std::min<long long>((count + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  identity_kernel<R><<<dim3(blocks, batch), 256, 0, st>>>(X, sX, rows, cols);
  return cudaGetLastError();
}

template <typename R>
__global__ void copy_kernel(const cx<R>* X, long long sX, cx<R>* Y, long long sY, long long count) {
  X += blockIdx.y * sX;
  Y += blockIdx.y * sY;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    Y[i] = X[i];
}

template <typename R>
cudaError_t copy_batched(cudaStream_t st, const cx<R>* X, long long sX, cx<R>* Y, long long sY, long long count,
                         int batch) {
  ProfScope ps(st, K_ELEMWISE);
  int blocks = (int)std::min<long long>((count + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  copy_kernel<R><<<dim3(blocks, batch), 256, 0, st>>>(X, sX, Y, sY, count);
  return cudaGetLastError();
}

template <typename R>
__global__ void copy2d_kernel(const cx<R>* X, long long sX, int ldx, cx<R>* Y, long long sY, int ldy, int rows,
                              int cols) {
  X += blockIdx.y * sX;
  Y += blockIdx.y * sY;
  const long long count = (long long)rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    Y[(i / cols) * ldy + i % cols] = X[(i / cols) * ldx + i % cols];
}

template <typename R>
cudaError_t copy_2d(cudaStream_t st, const cx<R>* X, long long sX, int ldx, cx<R>* Y, long long sY, int ldy, int rows,
                    int cols, int batch) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return cudaSuccess;
  ProfScope ps(st, K_ELEMWISE);
  const int blocks = (int)std::min<long long>(((long long)rows * cols + 255) / 256, 1024);
  copy2d_kernel<R><<<dim3(blocks, batch), 256, 0, st>>>(X, sX, ldx, Y, sY, ldy, rows, cols);
  return cudaGetLastError();
}

// Gauge fixing of an isometry W (n x r, ld r): column j is multiplied by
// conj(sum_i W[i][j]) / |sum_i W[i][j]| so that its column sum is real and
// non-negative (a zero sum leaves the column unchanged).
template <typename R>
__global__ void __launch_bounds__(256) fix_columns_kernel(cx<R>* Wb, long long sW, int n, int r) {
  __shared__ double red[2][8];
  const int j = blockIdx.x, z = blockIdx.y;
  cx<R>* W = Wb + z * sW;
  double sr = 0, si = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cx<R> w = W[(long long)i * r + j];
    sr += w.re;
    si += w.im;
  }
  sr = warp_sum_r(sr);
  si = warp_sum_r(si);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sr; red[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  double tr = 0, ti = 0;
  for (int w = 0; w < 8; ++w) { tr += red[0][w]; ti += red[1][w]; }
  const double a = sqrt(tr * tr + ti * ti);
  if (!(a > 0)) return;
  const cx<R> ph = mk<R>((R)(tr / a), (R)(-ti / a));
  for (int i = threadIdx.x; i < n; i += blockDim.x) W[(long long)i * r + j] = W[(long long)i * r + j] * ph;
}

template <typename R>
cudaError_t fix_columns(cudaStream_t st, cx<R>* W, long long sW, int n, int r, int batch) {
  if (r <= 0 || n <= 0) return cudaSuccess;
  ProfScope ps(st, K_ELEMWISE);
  fix_columns_kernel<R><<<dim3(r, batch), 256, 0, st>>>(W, sW, n, r);
  return cudaGetLastError();
}

// QR gauge: R_jj real and non-negative.  Q column j *= d_j, R row j *= conj(d_j),
// d_j = R_jj / |R_jj| (1 when R_jj = 0).  Q (m x k, ld k), R (k x n, ld n).
template <typename R>
__global__ void __launch_bounds__(256) fix_qr_kernel(cx<R>* Qb, long long sQ, int m, int k, cx<R>* Rb, long long sR,
                                                      int n) {
  const int j = blockIdx.x, z = blockIdx.y;
  cx<R>* Q = Qb + z * sQ;
  cx<R>* Rm = Rb + z * sR;
  const cx<R> rjj = Rm[(long long)j * n + j];
  const double a = sqrt((double)rjj.re * rjj.re + (double)rjj.im * rjj.im);
  if (!(a > 0)) return;
  const cx<R> d = mk<R>((R)(rjj.re / a), (R)(rjj.im / a));
  const cx<R> dc = conj(d);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) Q[(long long)i * k + j] = Q[(long long)i * k + j] * d;
  for (int c = j + threadIdx.x; c < n; c += blockDim.x) Rm[(long long)j * n + c] = Rm[(long long)j * n + c] * dc;
}

template <typename R>
cudaError_t fix_qr(cudaStream_t st, cx<R>* Q, long long sQ, int m, int k, cx<R>* Rm, long long sR, int n, int batch) {
  if (k <= 0) return cudaSuccess;
  ProfScope ps(st, K_ELEMWISE);
  fix_qr_kernel<R><<<dim3(k, batch), 256, 0, st>>>(Q, sQ, m, k, Rm, sR, n);
  return cudaGetLastError();
}

// Product state |b><b| on every site and instance: bond dims 1, M[0][s][0] = [s == 3 b].
template <typename R>
__global__ void product_state_kernel(int n, void* const* site, const long long* stride, const uint8_t* bits) {
  const int k = blockIdx.x, z = blockIdx.y, s = threadIdx.x;
  if (s >= 4) return;
  cx<R>* M = reinterpret_cast<cx<R>*>(site[k]) + z * stride[k];
  M[s] = mk<R>(s == 3 * (bits[k] ? 1 : 0) ? R(1) : R(0), R(0));
}

template <typename R>
cudaError_t product_state(cudaStream_t st, int n, void* const* d_site, const long long* d_stride, int n_inst,
                          const uint8_t* d_bits) {
  ProfScope ps(st, K_ELEMWISE);
  product_state_kernel<R><<<dim3(n, n_inst), 32, 0, st>>>(n, d_site, d_stride, d_bits);
  return cudaGetLastError();
}

#define NNE_INST_BLAS(R)                                                                                         \
  template cudaError_t cgemm<R>(cudaStream_t, int, int, int, int, int, cx<R>, const cx<R>*, long long, int,     \
                                const cx<R>*, long long, int, cx<R>, cx<R>*, long long, int, int);              \
  template cudaError_t apply_superop<R>(cudaStream_t, cx<R>*, long long, int, int, const double*, long long, int); \
  template cudaError_t sumsq_partial<R>(cudaStream_t, const cx<R>*, long long, long long, double*, int, int);     \
  template cudaError_t scale_batched<R>(cudaStream_t, cx<R>*, long long, long long, const double*, int);          \
  template cudaError_t transpose<R>(cudaStream_t, bool, const cx<R>*, long long, int, int, int, cx<R>*, long long, \
                                    int, int);                                                                   \
  template cudaError_t conj_inplace<R>(cudaStream_t, cx<R>*, long long, long long, int);                         \
  template cudaError_t identity<R>(cudaStream_t, cx<R>*, long long, int, int, int);                              \
  template cudaError_t copy_batched<R>(cudaStream_t, const cx<R>*, long long, cx<R>*, long long, long long, int); \
  template cudaError_t copy_2d<R>(cudaStream_t, const cx<R>*, long long, int, cx<R>*, long long, int, int, int, int); \
  template cudaError_t product_state<R>(cudaStream_t, int, void* const*, const long long*, int, const uint8_t*); \
  template cudaError_t fix_columns<R>(cudaStream_t, cx<R>*, long long, int, int, int);                          \
  template cudaError_t fix_qr<R>(cudaStream_t, cx<R>*, long long, int, int, cx<R>*, long long, int, int);

NNE_INST_BLAS(float)
NNE_INST_BLAS(double)

cudaError_t finish_gate(cudaStream_t st, const double* kept_parts, const double* total_parts, const double* disc_parts,
                        int parts, int batch, double* scale, double* log_norm, double* log_fid, int* err) {
  ProfScope ps(st, K_ELEMWISE);
  finish_gate_kernel<<<(batch + 127) / 128, 128, 0, st>>>(kept_parts, total_parts, disc_parts, parts, batch, scale,
                                                          log_norm, log_fid, err);
  return cudaGetLastError();
}

}  // namespace nne
