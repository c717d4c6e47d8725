// a7 -- Pauli expectation values by transfer-matrix sweeps (Sec. 2.2.3:
// <O>_lambda from an exact contraction of the network).
//   T_P(k)[a][b] = sum_s v_P[s] M_k[a][s][b],  v_P[s] = P[j][i] for s = 2 i + j:
//   v_I = (1,0,0,1), v_X = (0,1,1,0), v_Y = (0,i,-i,0), v_Z = (1,0,0,-1).
//   L_0 = 1, L_{k+1} = L_k T_I(k);  R_n = 1, R_k = T_I(k) R_{k+1};
//   <P> = L_first T_P(first) ... T_P(last) R_{last+1} / L_n.
// Accumulation in float64; each environment is rescaled to max-abs 1 and
// its log-scale carried separately, so long chains neither overflow nor
// underflow.
#include "kernels.cuh"

namespace nne {

__device__ __forceinline__ cx<double> pvec(int p, int s) {
  // v_P[s]
  switch (p) {
    case 0: return mk<double>((s == 0 || s == 3) ? 1.0 : 0.0, 0.0);
    case 1: return mk<double>((s == 1 || s == 2) ? 1.0 : 0.0, 0.0);
    case 2: return s == 1 ? mk<double>(0, 1) : (s == 2 ? mk<double>(0, -1) : mk<double>(0, 0));
    default: return mk<double>(s == 0 ? 1.0 : (s == 3 ? -1.0 : 0.0), 0.0);
  }
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
  return t;
}

// Environment sweeps: blockIdx.x = 0 left, 1 right; one CTA per (pass, instance).
// env layout: [inst][pass][k (0..n)][max_dim] complex double; scale [inst][pass][k].
template <typename R>
__global__ void __launch_bounds__(256) env_kernel(int n, const int* dims, const void* const* site,
                                                   const long long* stride, int max_dim, double* env,
                                                   double* envscale) {
  __shared__ double red[32];
  const int pass = blockIdx.x, z = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  cx<double>* E = reinterpret_cast<cx<double>*>(env) + ((long long)z * 2 + pass) * (n + 1) * max_dim;
  double* ls = envscale + ((long long)z * 2 + pass) * (n + 1);
  if (pass == 0) {
    if (threadIdx.x == 0) { E[0] = mk<double>(1, 0); ls[0] = 0; }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const int dl = dims[k], dr = dims[k + 1];
      const cx<R>* M = reinterpret_cast<const cx<R>*>(site[k]) + z * stride[k];
      const cx<double>* Lk = E + (long long)k * max_dim;
      cx<double>* Ln = E + (long long)(k + 1) * max_dim;
      double mx = 0;
      for (int b = threadIdx.x; b < dr; b += blockDim.x) {
        cx<double> acc = mk<double>(0, 0);
        for (int a = 0; a < dl; ++a) {
          const cx<R> m0 = M[((long long)a * 4 + 0) * dr + b], m3 = M[((long long)a * 4 + 3) * dr + b];
          fma_(acc, Lk[a], mk<double>((double)m0.re + m3.re, (double)m0.im + m3.im));
        }
        Ln[b] = acc;
        mx = fmax(mx, fmax(fabs(acc.re), fabs(acc.im)));
      }
      mx = block_max(mx, red);
      const double inv = mx > 0 ? 1.0 / mx : 1.0;
      for (int b = threadIdx.x; b < dr; b += blockDim.x) Ln[b] = inv * Ln[b];
      if (threadIdx.x == 0) ls[k + 1] = ls[k] + (mx > 0 ? log(mx) : 0.0);
      __syncthreads();
    }
  } else {
    if (threadIdx.x == 0) { E[(long long)n * max_dim] = mk<double>(1, 0); ls[n] = 0; }
    __syncthreads();
    for (int k = n - 1; k >= 0; --k) {
      const int dl = dims[k], dr = dims[k + 1];
      const cx<R>* M = reinterpret_cast<const cx<R>*>(site[k]) + z * stride[k];
      const cx<double>* Rn = E + (long long)(k + 1) * max_dim;
      cx<double>* Rk = E + (long long)k * max_dim;
      double mx = 0;
      for (int a = warp; a < dl; a += nw) {
        cx<double> acc = mk<double>(0, 0);
        for (int b = lane; b < dr; b += 32) {
          const cx<R> m0 = M[((long long)a * 4 + 0) * dr + b], m3 = M[((long long)a * 4 + 3) * dr + b];
          fma_(acc, mk<double>((double)m0.re + m3.re, (double)m0.im + m3.im), Rn[b]);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
          Rk[a] = acc;
          mx = fmax(mx, fmax(fabs(acc.re), fabs(acc.im)));
        }
      }
      mx = block_max(mx, red);
      const double inv = mx > 0 ? 1.0 / mx : 1.0;
      for (int a = threadIdx.x; a < dl; a += blockDim.x) Rk[a] = inv * Rk[a];
      if (threadIdx.x == 0) ls[k] = ls[k + 1] + (mx > 0 ? log(mx) : 0.0);
      __syncthreads();
    }
  }
}

// One CTA per (observable, instance): carry S from R_{last+1} down to `first`.
template <typename R>
__global__ void __launch_bounds__(256) obs_kernel(int n, const int* dims, const void* const* site,
                                                   const long long* stride, int max_dim, const double* env,
                                                   const double* envscale, const uint8_t* paulis, const int* first,
                                                   const int* last, int n_obs, double* out) {
  extern __shared__ unsigned char smem_raw[];
  cx<double>* S = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* S2 = S + max_dim;
  __shared__ double red[32];
  __shared__ cx<double> cred[32];
  const int o = blockIdx.x, z = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const cx<double>* EL = reinterpret_cast<const cx<double>*>(env) + ((long long)z * 2 + 0) * (n + 1) * max_dim;
  const cx<double>* ER = reinterpret_cast<const cx<double>*>(env) + ((long long)z * 2 + 1) * (n + 1) * max_dim;
  const double* lsL = envscale + ((long long)z * 2 + 0) * (n + 1);
  const double* lsR = envscale + ((long long)z * 2 + 1) * (n + 1);
  const int f = first[o], l = last[o];
  double* res = out + ((long long)z * n_obs + o) * 2;
  if (f < 0) {   // identity string
    if (threadIdx.x == 0) { res[0] = 1.0; res[1] = 0.0; }
    return;
  }
  {
    const int d = dims[l + 1];
    for (int b = threadIdx.x; b < d; b += blockDim.x) S[b] = ER[(long long)(l + 1) * max_dim + b];
  }
  double lsS = lsR[l + 1];
  __syncthreads();
  for (int k = l; k >= f; --k) {
    const int dl = dims[k], dr = dims[k + 1];
    const int p = paulis[(long long)o * n + k];
    const cx<double> c0 = pvec(p, 0), c1 = pvec(p, 1), c2 = pvec(p, 2), c3 = pvec(p, 3);
    const cx<R>* M = reinterpret_cast<const cx<R>*>(site[k]) + z * stride[k];
    double mx = 0;
    for (int a = warp; a < dl; a += nw) {
      cx<double> acc = mk<double>(0, 0);
      for (int b = lane; b < dr; b += 32) {
        cx<double> t = mk<double>(0, 0);
        const cx<R>* m = M + (long long)a * 4 * dr + b;
        const cx<R> m0 = m[0], m1 = m[dr], m2 = m[2 * dr], m3 = m[3 * dr];
        fma_(t, c0, mk<double>(m0.re, m0.im));
        fma_(t, c1, mk<double>(m1.re, m1.im));
        fma_(t, c2, mk<double>(m2.re, m2.im));
        fma_(t, c3, mk<double>(m3.re, m3.im));
        fma_(acc, t, S[b]);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        S2[a] = acc;
        mx = fmax(mx, fmax(fabs(acc.re), fabs(acc.im)));
      }
    }
    mx = block_max(mx, red);
    const double inv = mx > 0 ? 1.0 / mx : 1.0;
    for (int a = threadIdx.x; a < dl; a += blockDim.x) S[a] = inv * S2[a];
    lsS += mx > 0 ? log(mx) : 0.0;
    __syncthreads();
  }
  // value = L_f . S ; trace = L_n[0]
  cx<double> acc = mk<double>(0, 0);
  for (int a = threadIdx.x; a < dims[f]; a += blockDim.x) fma_(acc, EL[(long long)f * max_dim + a], S[a]);
  acc = warp_sum(acc);
  if (lane == 0) cred[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    cx<double> v = mk<double>(0, 0);
    for (int w = 0; w < nw; ++w) v = v + cred[w];
    const cx<double> tr = EL[(long long)n * max_dim];
    const double scale = exp(lsL[f] + lsS - lsL[n]);
    const double den = tr.re * tr.re + tr.im * tr.im;
    // v / tr
    const double qr = (v.re * tr.re + v.im * tr.im) / den, qi = (v.im * tr.re - v.re * tr.im) / den;
    res[0] = qr * scale;
    res[1] = qi * scale;
  }
}

template <typename R>
cudaError_t expect_sweep(cudaStream_t st, int n, const int* d_dims, const void* const* d_site,
                         const long long* d_stride, int n_inst, int max_dim, int n_obs, const uint8_t* d_paulis,
                         const int* d_first, const int* d_last, double* d_env, double* d_envscale, double* d_out) {
  cudaError_t e;
  {
    ProfScope ps(st, K_SWEEP_ENV);
    env_kernel<R><<<dim3(2, n_inst), 256, 0, st>>>(n, d_dims, d_site, d_stride, max_dim, d_env, d_envscale);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  if (n_obs <= 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(cx<double>) * (size_t)max_dim;
  if ((e = ensure_kernel_smem((const void*)obs_kernel<R>, smem, false)) != cudaSuccess) return e;
  ProfScope ps(st, K_SWEEP_OBS);
  obs_kernel<R><<<dim3(n_obs, n_inst), 256, smem, st>>>(n, d_dims, d_site, d_stride, max_dim, d_env, d_envscale,
                                                        d_paulis, d_first, d_last, n_obs, d_out);
  return cudaGetLastError();
}

template cudaError_t expect_sweep<float>(cudaStream_t, int, const int*, const void* const*, const long long*, int, int,
                                         int, const uint8_t*, const int*, const int*, double*, double*, double*);
template cudaError_t expect_sweep<double>(cudaStream_t, int, const int*, const void* const*, const long long*, int,
                                          int, int, const uint8_t*, const int*, const int*, double*, double*, double*);

}  // namespace nne
