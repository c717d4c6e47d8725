// A block of bw <= 32 Householder reflectors in compact-WY form applied to a
// K x N block:  C <- C - V op(T) (V^H C),  op(T) = T or T^H,  V: K x bw.
//
// The product W = V^H C is bw x N with a long inner dimension K, which a
// plain tiled GEMM runs on only ceil(N / 64) CTAs per matrix.  Here it is
// split over K into S chunks: one CTA per (64 output columns, chunk, matrix)
// writes its partial product, and a second kernel sums the partials in chunk
// order (deterministic) and multiplies by op(T).  The rank-bw update of C is
// then a GEMM with inner dimension bw.
#include "kernels.cuh"

namespace nne {

constexpr int WY_B = 32;          // reflectors per block (rows of W)
constexpr int WY_SPLIT_MAX = 16;  // chunks of the inner dimension
constexpr int WY_TN = 64;         // output columns per CTA of the partial product
constexpr int WY_KS = 16;         // rows of V and C per shared-memory stage

long long wy_workspace(int N) { return (long long)(WY_SPLIT_MAX + 1) * WY_B * N; }

// Partial s of W = V^H C over rows [s * kc, min((s + 1) * kc, K)), written to
// P[z][s] (WY_B x N, rows >= bw zero).  VROWS: V is passed as V^H, row c at
// Vb + c * ldv; otherwise V is K x bw with row i at Vb + i * ldv.
template <typename R, bool VROWS>
__global__ void __launch_bounds__(256) wy_partial_kernel(const cx<R>* __restrict__ Vb, long long sV, int ldv, int bw,
                                                         int K, int N, int kc, const cx<R>* __restrict__ Cb,
                                                         long long sC, int ldc, cx<R>* __restrict__ Pb, int S) {
  __shared__ cx<R> Vs[WY_KS][WY_B + 1];   // conj(V[i][c])
  __shared__ cx<R> Cs[WY_KS][WY_TN];
  const int z = blockIdx.z, s = blockIdx.y, j0 = blockIdx.x * WY_TN;
  const cx<R>* V = Vb + z * sV;
  const cx<R>* C = Cb + z * sC;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i_begin = s * kc, i_end = min(K, i_begin + kc);
  cx<R> acc[2][4];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = mk<R>(0, 0);
  for (int i0 = i_begin; i0 < i_end; i0 += WY_KS) {
    for (int e = tid; e < WY_KS * WY_B; e += 256) {
      int k, c;
      if (VROWS) { k = e % WY_KS; c = e / WY_KS; } else { c = e % WY_B; k = e / WY_B; }
      const int gi = i0 + k;
      cx<R> v = mk<R>(0, 0);
      if (gi < i_end && c < bw) v = VROWS ? V[(long long)c * ldv + gi] : conj(V[(long long)gi * ldv + c]);
      Vs[k][c] = v;
    }
    for (int e = tid; e < WY_KS * WY_TN; e += 256) {
      const int k = e / WY_TN, j = e % WY_TN;
      const int gi = i0 + k, gj = j0 + j;
      Cs[k][j] = (gi < i_end && gj < N) ? C[(long long)gi * ldc + gj] : mk<R>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < WY_KS; ++k) {
      const cx<R> a0 = Vs[k][ty], a1 = Vs[k][ty + 16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const cx<R> b = Cs[k][tx + 16 * q];
        fma_(acc[0][q], a0, b);
        fma_(acc[1][q], a1, b);
      }
    }
    __syncthreads();
  }
  cx<R>* P = Pb + ((long long)z * S + s) * WY_B * N;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + tx + 16 * q;
      if (gj < N) P[(long long)(ty + 16 * p) * N + gj] = acc[p][q];
    }
}

// W2[z] (bw x N, ld N) = op(T[z]) * sum_s P[z][s], partials summed in order s = 0, 1, ...
template <typename R>
__global__ void __launch_bounds__(256) wy_reduce_kernel(const cx<R>* __restrict__ Pb, int S, int N, int bw,
                                                        const cx<R>* __restrict__ Tb, long long sT, int ldt,
                                                        int t_adj, cx<R>* __restrict__ W2b, long long sW2) {
  __shared__ cx<R> Ws[WY_B][WY_B + 1];
  __shared__ cx<R> Ts[WY_B][WY_B + 1];
  const int z = blockIdx.y, j0 = blockIdx.x * WY_B;
  const cx<R>* P = Pb + (long long)z * S * WY_B * N;
  const cx<R>* T = Tb + z * sT;
  cx<R>* W2 = W2b + z * sW2;
  const int tid = threadIdx.x;
  for (int e = tid; e < WY_B * WY_B; e += 256) {
    const int a = e / WY_B, b = e % WY_B;
    cx<R> t = mk<R>(0, 0);
    if (a < bw && b < bw) t = t_adj ? conj(T[(long long)b * ldt + a]) : T[(long long)a * ldt + b];
    Ts[a][b] = t;
    const int gj = j0 + b;
    cx<R> w = mk<R>(0, 0);
    if (gj < N)
      for (int s = 0; s < S; ++s) w = w + P[((long long)s * WY_B + a) * N + gj];
    Ws[a][b] = w;
  }
  __syncthreads();
  for (int e = tid; e < WY_B * WY_B; e += 256) {
    const int a = e / WY_B, j = e % WY_B;
    const int gj = j0 + j;
    if (a >= bw || gj >= N) continue;
    cx<R> acc = mk<R>(0, 0);
    for (int b = 0; b < bw; ++b) fma_(acc, Ts[a][b], Ws[b][j]);
    W2[(long long)a * N + gj] = acc;
  }
}

template <typename R>
cudaError_t wy_apply(cudaStream_t st, bool v_rows, const cx<R>* V, long long sV, int ldv, const cx<R>* T,
                     long long sT, int ldt, bool t_adj, int bw, int K, int N, cx<R>* C, long long sC, int ldc,
                     cx<R>* ws, int batch) {
  if (bw <= 0 || K <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (bw > WY_B) return cudaErrorInvalidValue;
  const int tiles = (N + WY_TN - 1) / WY_TN;
  // about four waves of partial-product CTAs, chunks of at least 64 rows
  int S = (4 * 152 + tiles * batch - 1) / (tiles * batch);
  S = std::max(1, std::min(S, std::min(WY_SPLIT_MAX, (K + 63) / 64)));
  int kc = (K + S - 1) / S;
  kc = (kc + WY_KS - 1) / WY_KS * WY_KS;
  S = (K + kc - 1) / kc;
  // workspace (batch x wy_workspace(N) elements): partials [z][s] (WY_B x N each), then W2[z] (WY_B x N)
  cx<R>* P = ws;
  cx<R>* W2 = ws + (long long)batch * WY_SPLIT_MAX * WY_B * N;
  const long long sW2 = (long long)WY_B * N;
  cudaError_t e;
  {
    ProfScope ps(st, K_WY, 2, 8.0 * bw * (double)N * K * batch);
    dim3 g1(tiles, S, batch);
    if (v_rows)
      wy_partial_kernel<R, true><<<g1, 256, 0, st>>>(V, sV, ldv, bw, K, N, kc, C, sC, ldc, P, S);
    else
      wy_partial_kernel<R, false><<<g1, 256, 0, st>>>(V, sV, ldv, bw, K, N, kc, C, sC, ldc, P, S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 g2((N + WY_B - 1) / WY_B, batch);
    wy_reduce_kernel<R><<<g2, 256, 0, st>>>(P, S, N, bw, T, sT, ldt, t_adj ? 1 : 0, W2, sW2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cgemm<R>(st, v_rows ? OP_C : OP_N, OP_N, K, N, bw, mk<R>(-1, 0), V, sV, ldv, W2, sW2, N, mk<R>(1, 0), C,
                  sC, ldc, batch);
}

template cudaError_t wy_apply<float>(cudaStream_t, bool, const cx<float>*, long long, int, const cx<float>*,
                                     long long, int, bool, int, int, int, cx<float>*, long long, int, cx<float>*, int);
template cudaError_t wy_apply<double>(cudaStream_t, bool, const cx<double>*, long long, int, const cx<double>*,
                                      long long, int, bool, int, int, int, cx<double>*, long long, int, cx<double>*,
                                      int);

}  // namespace nne
