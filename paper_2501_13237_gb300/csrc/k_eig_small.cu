// Hermitian eigensolver pieces for matrices that fit in one cluster's shared
// memory (n <= 640 complex64 / 448 complex128 with 16 CTAs), plus the
// blocked (compact-WY) back-transformation shared by both reduction paths.
//
// Reduction: rows are spread cyclically over the CTAs of a cluster and stay
// in shared memory for the whole reduction; column j is read from its owner
// through distributed shared memory, every CTA forms the Householder vector
// redundantly (identical arithmetic, so identical results; the FP64 parts on
// one thread per CTA), the products
// p = A v are pushed to every CTA, and one more barrier closes the rank-2
// update.  Reflector j is stored conjugated as row j of Vh (n x n).
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nne {

template <typename R>
__global__ void __launch_bounds__(256) tridiag_smem_kernel(const cx<R>* Hb, long long sH, int n, R* db, cx<R>* eb,
                                                            int ldde, cx<R>* Vhb, long long sVh, int maxloc) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  const cx<R>* H = Hb + z * sH;
  R* d = db + (long long)z * ldde;
  cx<R>* e = eb + (long long)z * ldde;
  cx<R>* Vh = Vhb + z * sVh;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* Hl = reinterpret_cast<cx<R>*>(smem_raw);     // [maxloc][n] own rows
  cx<R>* vbuf = Hl + (long long)maxloc * n;           // 2 x n: column j (pushed by its owner), double-buffered
  cx<R>* w = vbuf + 2 * n;
  cx<R>* p = w + n;
  __shared__ double ks[2][16];                        // K partials pushed by every CTA
  __shared__ R dpush[2];                              // diagonal entry pushed with the column
  __shared__ double red[32];
  __shared__ cx<R> alpha_s;
  __shared__ R inv_s, twoK_s;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int nloc = n > rank ? (n - rank + CS - 1) / CS : 0;
  for (long long e2 = tid; e2 < (long long)nloc * n; e2 += nth) {
    const int li = (int)(e2 / n), c = (int)(e2 % n);
    Hl[e2] = H[(long long)(rank + li * CS) * n + c];
  }
  // every CTA of the cluster is running before anyone writes into its shared memory
  cluster.sync();
  // column 0 below the diagonal = conj(row 0 tail), pushed by the owner of row 0
  if (rank == 0) {
    for (int t = tid; t + 1 < n; t += nth) {
      const cx<R> x = conj(Hl[1 + t]);
      for (int c = 0; c < CS; ++c) *cluster.map_shared_rank(vbuf + t, c) = x;
    }
    if (tid < CS) *cluster.map_shared_rank(&dpush[0], tid) = Hl[0].re;
  }
  cluster.sync();
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1, owner = j % CS, buf = j & 1;
    cx<R>* v = vbuf + buf * n;
    const R djj = dpush[buf];
    // Householder vector (every CTA, same arithmetic).  Squared norm: per-warp
    // partials in R, combined in FP64 by one thread, which also forms alpha and
    // 1/un (FP64 is slow on this part: keep it off the other threads).
    {
      R sp = 0;
      for (int t = tid; t < m; t += nth) sp += norm2(v[t]);
      sp = warp_sum_r(sp);
      if (lane == 0) red[warp] = (double)sp;
    }
    __syncthreads();
    if (tid == 0) {
      double xn2 = 0;
      for (int w2 = 0; w2 < nw; ++w2) xn2 += red[w2];
      const cx<R> x0 = v[0];
      const double ax0 = sqrt((double)norm2(x0)), xn = sqrt(xn2);
      cx<R> alpha = mk<R>(0, 0);
      double un = 0;
      if (xn > 0) {
        const double pr = ax0 > 0 ? (double)x0.re / ax0 : 1.0, pi = ax0 > 0 ? (double)x0.im / ax0 : 0.0;
        alpha = mk<R>((R)(-xn * pr), (R)(-xn * pi));
        un = sqrt(2.0 * xn2 + 2.0 * xn * ax0);
      }
      alpha_s = alpha;
      inv_s = un > 0 ? (R)(1.0 / un) : R(0);
      if (rank == owner) { d[j] = djj; e[j] = alpha; }
    }
    __syncthreads();
    const cx<R> alpha = alpha_s;
    const R inv = inv_s;
    for (int t = tid; t < m; t += nth) {
      cx<R> u = v[t];
      if (t == 0) u = u - alpha;
      v[t] = inv * u;
    }
    __syncthreads();
    if (rank == owner) {
      cx<R>* vr = Vh + (long long)j * n + (j + 1);
      for (int t = tid; t < m; t += nth) vr[t] = conj(v[t]);
    }
    // p = A v on own rows i >= j+1, pushed to every CTA
    const int lstart = (j + 1 - rank + CS - 1) / CS;
    R kp = 0;
    for (int li = lstart + warp; li < nloc; li += nw) {
      const int i = rank + li * CS, t = i - j - 1;
      const cx<R>* row = Hl + (long long)li * n + (j + 1);
      cx<R> a0 = mk<R>(0, 0), a1 = a0, a2 = a0, a3 = a0;
      int k = lane;
      for (; k + 96 < m; k += 128) {
        fma_(a0, row[k], v[k]);
        fma_(a1, row[k + 32], v[k + 32]);
        fma_(a2, row[k + 64], v[k + 64]);
        fma_(a3, row[k + 96], v[k + 96]);
      }
      for (; k < m; k += 32) fma_(a0, row[k], v[k]);
      cx<R> acc = (a0 + a1) + (a2 + a3);
      acc = warp_sum(acc);
      if (lane < CS) *cluster.map_shared_rank(p + t, lane) = acc;
      if (lane == 0) kp += v[t].re * acc.re + v[t].im * acc.im;
    }
    if (lane == 0) red[warp] = (double)kp;
    __syncthreads();
    if (tid < CS) {
      double t = 0;
      for (int w2 = 0; w2 < nw; ++w2) t += red[w2];
      *cluster.map_shared_rank(&ks[buf][rank], tid) = t;
    }
    cluster.sync();
    if (tid == 0) {
      double K = 0;
      for (int c = 0; c < CS; ++c) K += ks[buf][c];
      twoK_s = (R)(2.0 * K);
    }
    __syncthreads();
    const R twoK = twoK_s;
    for (int t = tid; t < m; t += nth) w[t] = mk<R>(2 * p[t].re - twoK * v[t].re, 2 * p[t].im - twoK * v[t].im);
    __syncthreads();
    for (int li = lstart + warp; li < nloc; li += nw) {
      const int i = rank + li * CS, t = i - j - 1;
      cx<R>* row = Hl + (long long)li * n + (j + 1);
      const cx<R> vt = v[t], wt = w[t];
#pragma unroll 4
      for (int k = lane; k < m; k += 32) {
        cx<R> a = row[k];
        const cx<R> wk = w[k], vk = v[k];
        a.re -= vt.re * wk.re + vt.im * wk.im + wt.re * vk.re + wt.im * vk.im;
        a.im -= vt.im * wk.re - vt.re * wk.im + wt.im * vk.re - wt.re * vk.im;
        row[k] = a;
      }
    }
    // the owner of row j+1 pushes its updated tail (the next column) and diagonal
    if (j + 3 < n && rank == (j + 1) % CS) {
      __syncthreads();
      const cx<R>* rn = Hl + (long long)((j + 1) / CS) * n;
      cx<R>* vn = vbuf + (buf ^ 1) * n;
      for (int t = tid; t + j + 2 < n; t += nth) {
        const cx<R> x = conj(rn[j + 2 + t]);
        for (int c = 0; c < CS; ++c) *cluster.map_shared_rank(vn + t, c) = x;
      }
      if (tid < CS) *cluster.map_shared_rank(&dpush[buf ^ 1], tid) = rn[j + 1].re;
    }
    cluster.sync();
  }
  if (tid == 0) {
    if (n >= 2) {
      if ((n - 2) % CS == rank) d[n - 2] = Hl[(long long)((n - 2) / CS) * n + (n - 2)].re;
      if ((n - 1) % CS == rank) {
        d[n - 1] = Hl[(long long)((n - 1) / CS) * n + (n - 1)].re;
        e[n - 2] = Hl[(long long)((n - 1) / CS) * n + (n - 2)];
      }
    } else if (rank == 0) {
      d[0] = Hl[0].re;
    }
  }
}

// U[k][c] = phi_k Z[k][c] (complex from the real tridiagonal eigenvectors).
template <typename R>
__global__ void phase_scale_kernel(const R* Zb, long long sZ, const cx<R>* phib, int ldde, int n, int r, cx<R>* Ub,
                                   long long sU) {
  const int z = blockIdx.y;
  const R* Z = Zb + z * sZ;
  const cx<R>* phi = phib + (long long)z * ldde;
  cx<R>* U = Ub + z * sU;
  const long long count = (long long)n * r;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / r);
    U[i] = Z[i] * phi[k];
  }
}

// Compact-WY factors of blocks of 32 consecutive tridiagonal reflectors:
// block b (reflectors 32b .. 32b+bw-1) gives T_b with
// P_{32b} ... P_{32b+bw-1} = I - V_b T_b V_b^H, V_b^H = Vh rows 32b...
template <typename R>
__global__ void __launch_bounds__(256) wy_t_kernel(const cx<R>* Vhb, long long sVh, int n, int nref, cx<R>* Tb,
                                                    long long sT) {
  __shared__ cx<R> G[32][32];
  __shared__ cx<R> Ts[32][32];
  const int b = blockIdx.x, z = blockIdx.y;
  const cx<R>* Vh = Vhb + z * sVh;
  cx<R>* T = Tb + z * sT + (long long)b * 1024;
  const int j0 = 32 * b, bw = min(32, nref - j0);
  const int tid = threadIdx.x;
  for (int e = tid; e < 1024; e += blockDim.x) {
    const int a = e / 32, c = e % 32;
    cx<R> acc = mk<R>(0, 0);
    if (a < bw && c < bw) {
      const cx<R>* ra = Vh + (long long)(j0 + a) * n;
      const cx<R>* rc = Vh + (long long)(j0 + c) * n;
      for (int i = j0 + 1; i < n; ++i) fmac_(acc, rc[i], ra[i]);   // G[a][c] = v_a^H v_c = sum conj(v_a) v_c
      // rows hold conj(v): ra[i] = conj(v_a[i]) -> acc = sum conj(rc) ra = sum v_c conj(v_a)
    }
    G[a][c] = acc;
    Ts[a][c] = mk<R>(0, 0);
  }
  __syncthreads();
  if (tid < 32) {
    for (int i = 0; i < bw; ++i) {
      const R tau = G[i][i].re > R(0.5) ? R(2) : R(0);
      cx<R> acc = mk<R>(0, 0);
      if (tid < i)
        for (int l = tid; l < i; ++l) fma_(acc, Ts[tid][l], G[l][i]);
      __syncwarp();
      if (tid < i) Ts[tid][i] = mk<R>(-tau * acc.re, -tau * acc.im);
      if (tid == i) Ts[i][i] = mk<R>(tau, 0);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += blockDim.x) T[e] = Ts[e / 32][e % 32];
}

template <typename K, typename... Args>
static cudaError_t launch_cl(K kernel, int cs, int batch, size_t smem, cudaStream_t st, Args... args) {
  cudaError_t e = ensure_kernel_smem((const void*)kernel, smem, cs > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, batch, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr size_t SMEM_LIMIT = 220 * 1024;

// Cluster size whose shared memory holds the matrix, or 0 if none does.
template <typename R>
int smem_cluster_size(int n) {
  for (int cs = 1; cs <= 16; cs *= 2) {
    const size_t maxloc = (n + cs - 1) / cs;
    const size_t bytes = sizeof(cx<R>) * (maxloc * n + 4 * (size_t)n);
    if (bytes <= SMEM_LIMIT && (cs >= 16 || maxloc <= 64)) return cs;
  }
  return 0;
}

template <typename R>
cudaError_t tridiag_smem(cudaStream_t st, const cx<R>* H, long long sH, int n, R* d, cx<R>* e, int ldde, cx<R>* Vh,
                         long long sVh, int batch) {
  const int cs = smem_cluster_size<R>(n);
  if (cs == 0) return cudaErrorInvalidValue;
  const int maxloc = (n + cs - 1) / cs;
  const size_t smem = sizeof(cx<R>) * ((size_t)maxloc * n + 4 * (size_t)n);
  ProfScope ps(st, K_TRIDIAG, 1, 16.0 / 3.0 * (double)n * n * n * batch);   // Hermitian tridiagonalisation flops
  return launch_cl(tridiag_smem_kernel<R>, cs, batch, smem, st, H, sH, n, d, e, ldde, Vh, sVh, maxloc);
}

template <typename R>
cudaError_t backtransform_wy(cudaStream_t st, const cx<R>* Vh, long long sVh, int n, const R* Z, long long sZ,
                             const cx<R>* phi, int ldde, int r, cx<R>* U, long long sU, cx<R>* Tw, cx<R>* wy_ws,
                             int batch) {
  cudaError_t e;
  {
    ProfScope ps(st, K_BACKTRANSFORM);
    const long long count = (long long)n * r;
    int blocks = (int)std::min<long long>((count + 255) / 256, 1024);
    phase_scale_kernel<R><<<dim3(std::max(blocks, 1), batch), 256, 0, st>>>(Z, sZ, phi, ldde, n, r, U, sU);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int nref = n - 2;
  if (nref <= 0) return cudaSuccess;
  const int nb = (nref + 31) / 32;
  const long long sT = (long long)nb * 1024;
  {
    ProfScope ps(st, K_BACKTRANSFORM);
    wy_t_kernel<R><<<dim3(nb, batch), 256, 0, st>>>(Vh, sVh, n, nref, Tw, sT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int b = nb - 1; b >= 0; --b) {
    const int j0 = 32 * b, bw = std::min(32, nref - j0);
    const int r0 = j0 + 1, mb = n - r0;
    const cx<R>* Vb = Vh + (long long)j0 * n + r0;    // bw x mb, rows = conj(v)
    cx<R>* Ub = U + (long long)r0 * r;
    // U_b <- (I - V T V^H) U_b
    if ((e = wy_apply<R>(st, true, Vb, sVh, n, Tw + (long long)b * 1024, sT, 32, false, bw, mb, r, Ub, sU, r, wy_ws,
                         batch)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

#define NNE_INST_EIGS(R)                                                                                        \
  template int smem_cluster_size<R>(int);                                                                       \
  template cudaError_t tridiag_smem<R>(cudaStream_t, const cx<R>*, long long, int, R*, cx<R>*, int, cx<R>*,    \
                                       long long, int);                                                         \
  template cudaError_t backtransform_wy<R>(cudaStream_t, const cx<R>*, long long, int, const R*, long long,    \
                                           const cx<R>*, int, int, cx<R>*, long long, cx<R>*, cx<R>*, int);
NNE_INST_EIGS(float)
NNE_INST_EIGS(double)

}  // namespace nne
