// a1 -- fused gate+channel superoperators G = S_C (U (x) conj U) in float64
// (Sec. 2.2.1, eq. U -> C o U; two-qubit depolarizing of App. C.2.1).
// Local index s = 2 i + j for |i><j|; row 4 s1' + s2', column 4 s1 + s2.
#include "kernels.cuh"

namespace nne {

__device__ __forceinline__ void pauli(int p, cx<double> out[4]) {
  // 2x2 row-major: I, X, Y, Z
  const cx<double> z0 = mk<double>(0, 0), one = mk<double>(1, 0);
  switch (p) {
    case 0: out[0] = one; out[1] = z0; out[2] = z0; out[3] = one; break;
    case 1: out[0] = z0; out[1] = one; out[2] = one; out[3] = z0; break;
    case 2: out[0] = z0; out[1] = mk<double>(0, -1); out[2] = mk<double>(0, 1); out[3] = z0; break;
    default: out[0] = one; out[1] = z0; out[2] = z0; out[3] = mk<double>(-1, 0); break;
  }
}

// Kraus operators (4x4) of one channel kind at strength p; returns their number.
//  kind 0: two-qubit depolarizing, K0 = sqrt(1-15p/16) I, K_ab = sqrt(p/16) s_a (x) s_b
//  kind 1: amplitude damping on both qubits
//  kind 2: dephasing on both qubits
//  kind 3: single-qubit depolarizing (error probability p) on both qubits
__device__ int make_kraus(int kind, double p, cx<double> (*K)[16]) {
  cx<double> one1[4][4];   // single-qubit Kraus sets (2x2 row-major)
  double c1[4];
  int n1 = 0;
  if (kind == 0) {
    int idx = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        cx<double> pa[4], pb[4];
        pauli(a, pa);
        pauli(b, pb);
        const double c = (a == 0 && b == 0) ? sqrt(1.0 - 15.0 * p / 16.0) : sqrt(p / 16.0);
        for (int r = 0; r < 4; ++r)
          for (int q = 0; q < 4; ++q) K[idx][4 * r + q] = c * (pa[2 * (r >> 1) + (q >> 1)] * pb[2 * (r & 1) + (q & 1)]);
        ++idx;
      }
    return 16;
  }
  if (kind == 1) {
    for (int i = 0; i < 4; ++i) one1[0][i] = one1[1][i] = mk<double>(0, 0);
    one1[0][0] = mk<double>(1, 0);
    one1[0][3] = mk<double>(sqrt(1.0 - p), 0);
    one1[1][1] = mk<double>(sqrt(p), 0);
    c1[0] = c1[1] = 1.0;
    n1 = 2;
  } else if (kind == 2) {
    pauli(0, one1[0]);
    pauli(3, one1[1]);
    c1[0] = sqrt(1.0 - p);
    c1[1] = sqrt(p);
    n1 = 2;
  } else {
    for (int a = 0; a < 4; ++a) pauli(a, one1[a]);
    c1[0] = sqrt(1.0 - p);
    c1[1] = c1[2] = c1[3] = sqrt(p / 3.0);
    n1 = 4;
  }
  int idx = 0;
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n1; ++b) {
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q)
          K[idx][4 * r + q] = (c1[a] * c1[b]) * (one1[a][2 * (r >> 1) + (q >> 1)] * one1[b][2 * (r & 1) + (q & 1)]);
      ++idx;
    }
  return n1 * n1;
}

// Superoperator entry (row, col) of a Kraus set: sum_K K[i1 i2][k1 k2] conj(K[j1 j2][l1 l2]).
__device__ cx<double> superop_entry(const cx<double> (*K)[16], int nk, int row, int col) {
  const int s1 = row >> 2, s2 = row & 3, t1 = col >> 2, t2 = col & 3;
  const int i1 = s1 >> 1, j1 = s1 & 1, i2 = s2 >> 1, j2 = s2 & 1;
  const int k1 = t1 >> 1, l1 = t1 & 1, k2 = t2 >> 1, l2 = t2 & 1;
  cx<double> acc = mk<double>(0, 0);
  for (int q = 0; q < nk; ++q) {
    const cx<double> a = K[q][4 * (2 * i1 + i2) + (2 * k1 + k2)];
    const cx<double> b = K[q][4 * (2 * j1 + j2) + (2 * l1 + l2)];
    fmac_(acc, b, a);   // acc += conj(b) * a
  }
  return acc;
}

// S_noise[z] for each instance: product of the channel superoperators, depol2 first.
__global__ void __launch_bounds__(256) noise_superop_kernel(const double* rates, double* Sout) {
  __shared__ cx<double> K[16][16];
  __shared__ cx<double> S[256], T[256];
  __shared__ int nks;
  const int z = blockIdx.x, tid = threadIdx.x;
  const int row = tid >> 4, col = tid & 15;
  S[tid] = mk<double>(row == col ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int kind = 0; kind < 4; ++kind) {
    const double p = rates[4 * z + kind];
    if (p == 0.0) continue;
    if (tid == 0) nks = make_kraus(kind, p, K);
    __syncthreads();
    const int nk = nks;
    const cx<double> sc = superop_entry(K, nk, row, col);
    T[tid] = sc;
    __syncthreads();
    // S <- T S
    cx<double> acc = mk<double>(0, 0);
    for (int q = 0; q < 16; ++q) fma_(acc, T[16 * row + q], S[16 * q + col]);
    __syncthreads();
    S[tid] = acc;
    __syncthreads();
  }
  Sout[2 * (256 * z + tid)] = S[tid].re;
  Sout[2 * (256 * z + tid) + 1] = S[tid].im;
}

// G[z][g] = S_noise[z] (U_g (x) conj U_g).
__global__ void __launch_bounds__(256) gate_superop_kernel(int n_gates, const double* U, const double* Snoise,
                                                           double* G) {
  __shared__ cx<double> u[16];
  __shared__ cx<double> SU[256], SN[256];
  const int g = blockIdx.x, z = blockIdx.y, tid = threadIdx.x;
  if (tid < 16) u[tid] = mk<double>(U[32 * g + 2 * tid], U[32 * g + 2 * tid + 1]);
  SN[tid] = mk<double>(Snoise[2 * (256 * z + tid)], Snoise[2 * (256 * z + tid) + 1]);
  __syncthreads();
  const int row = tid >> 4, col = tid & 15;
  {
    const int s1 = row >> 2, s2 = row & 3, t1 = col >> 2, t2 = col & 3;
    const int i1 = s1 >> 1, j1 = s1 & 1, i2 = s2 >> 1, j2 = s2 & 1;
    const int k1 = t1 >> 1, l1 = t1 & 1, k2 = t2 >> 1, l2 = t2 & 1;
    const cx<double> a = u[4 * (2 * i1 + i2) + (2 * k1 + k2)];
    const cx<double> b = u[4 * (2 * j1 + j2) + (2 * l1 + l2)];
    SU[tid] = a * conj(b);
  }
  __syncthreads();
  cx<double> acc = mk<double>(0, 0);
  for (int q = 0; q < 16; ++q) fma_(acc, SN[16 * row + q], SU[16 * q + col]);
  const long long o = ((long long)z * n_gates + g) * 256 + tid;
  G[2 * o] = acc.re;
  G[2 * o + 1] = acc.im;
}

// Gate-dependent Pauli noise (cat-qubit, App. C.2.2; matchgate depolarizing,
// App. C.3.1): G[z][g] = S_P (U_g (x) conj U_g) with
// S_P = sum_ab p_ab (s_a (x) s_b) (x) conj(s_a (x) s_b) and
// p_ab = c0[g][ab] + lambda_z c1[g][ab] (ab = 4a + b, a on the left qubit).
// One block per (gate, level); thread (row, col) forms one entry of each factor.
__global__ void __launch_bounds__(256) pauli_superop_kernel(int n_gates, const double* U, const double* pr,
                                                            const double* lam, double* G) {
  __shared__ cx<double> u[16];
  __shared__ cx<double> sig[4][4];
  __shared__ double p[16];
  __shared__ cx<double> SU[256], SP[256];
  const int g = blockIdx.x, z = blockIdx.y, tid = threadIdx.x;
  if (tid < 16) {
    u[tid] = mk<double>(U[32 * g + 2 * tid], U[32 * g + 2 * tid + 1]);
    p[tid] = pr[32LL * g + tid] + lam[z] * pr[32LL * g + 16 + tid];
  }
  if (tid < 4) pauli(tid, sig[tid]);
  __syncthreads();
  const int row = tid >> 4, col = tid & 15;
  const int s1 = row >> 2, s2 = row & 3, t1 = col >> 2, t2 = col & 3;
  const int i1 = s1 >> 1, j1 = s1 & 1, i2 = s2 >> 1, j2 = s2 & 1;
  const int k1 = t1 >> 1, l1 = t1 & 1, k2 = t2 >> 1, l2 = t2 & 1;
  SU[tid] = u[4 * (2 * i1 + i2) + (2 * k1 + k2)] * conj(u[4 * (2 * j1 + j2) + (2 * l1 + l2)]);
  cx<double> acc = mk<double>(0, 0);
  for (int a = 0; a < 4; ++a) {
    const cx<double> fa = sig[a][2 * i1 + k1] * conj(sig[a][2 * j1 + l1]);
    for (int b = 0; b < 4; ++b) {
      const cx<double> fb = sig[b][2 * i2 + k2] * conj(sig[b][2 * j2 + l2]);
      acc = acc + p[4 * a + b] * (fa * fb);
    }
  }
  SP[tid] = acc;
  __syncthreads();
  acc = mk<double>(0, 0);
  for (int q = 0; q < 16; ++q) fma_(acc, SP[16 * row + q], SU[16 * q + col]);
  const long long o = ((long long)z * n_gates + g) * 256 + tid;
  G[2 * o] = acc.re;
  G[2 * o + 1] = acc.im;
}

cudaError_t build_pauli_superops(cudaStream_t st, int n_gates, const double* d_U, const double* d_pr, int n_inst,
                                 const double* d_lam, double* d_G) {
  if (n_gates <= 0 || n_inst <= 0) return cudaSuccess;
  ProfScope ps(st, K_SUPEROP_BUILD, 1);
  pauli_superop_kernel<<<dim3(n_gates, n_inst), 256, 0, st>>>(n_gates, d_U, d_pr, d_lam, d_G);
  return cudaGetLastError();
}

cudaError_t build_superops(cudaStream_t st, int n_gates, const double* d_U, int n_inst, const double* d_rates,
                           double* d_G, double* d_Snoise) {
  ProfScope ps(st, K_SUPEROP_BUILD, 2);
  noise_superop_kernel<<<n_inst, 256, 0, st>>>(d_rates, d_Snoise);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (n_gates > 0) gate_superop_kernel<<<dim3(n_gates, n_inst), 256, 0, st>>>(n_gates, d_U, d_Snoise, d_G);
  return cudaGetLastError();
}

}  // namespace nne
