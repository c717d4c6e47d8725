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
#include <map>
#include <mutex>
#include <tuple>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nne {

// Reflector of row r (the owner's own row, stored at Hl_row): x = conj of the
// row's entries right of the diagonal (the column below it, by symmetry),
// v = (x - alpha e_0) / ||x - alpha e_0||, alpha = -e^{i arg x_0} ||x||.
// Writes v to vpub, conj(v) to row r of Vh, d[r] and e[r] = alpha.  Called by
// every thread of the owning CTA; the norm is summed in R.
template <typename R>
__device__ __forceinline__ void tridiag_publish(const cx<R>* Hl_row, int n, int r, cx<R>* vpub, cx<R>* Vh, R* d,
                                                cx<R>* e, R* red, cx<R>* alpha_s, R* inv_s) {
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int m = n - r - 1;
  R sp = 0;
  for (int t = tid; t < m; t += nth) sp += norm2(Hl_row[r + 1 + t]);
  sp = warp_sum_r(sp);
  if (lane == 0) red[warp] = sp;
  __syncthreads();
  if (tid == 0) {
    R xn2 = 0;
    for (int w2 = 0; w2 < nw; ++w2) xn2 += red[w2];
    const cx<R> x0 = conj(Hl_row[r + 1]);
    R pr, pi, ax0;
    unit_phase_of(x0, &pr, &pi, &ax0);
    const R xn = sqrt(xn2);
    cx<R> alpha = mk<R>(0, 0);
    R un = 0;
    if (xn > R(0)) {
      alpha = mk<R>(-xn * pr, -xn * pi);
      un = sqrt(R(2) * xn2 + R(2) * xn * ax0);
    }
    *alpha_s = alpha;
    *inv_s = un > R(0) ? R(1) / un : R(0);
    d[r] = Hl_row[r].re;
    e[r] = alpha;
  }
  __syncthreads();
  const cx<R> alpha = *alpha_s;
  const R inv = *inv_s;
  cx<R>* vr = Vh + (long long)r * n + (r + 1);
  for (int t = tid; t < m; t += nth) {
    cx<R> u = conj(Hl_row[r + 1 + t]);
    if (t == 0) u = u - alpha;
    const cx<R> v = inv * u;
    vpub[t] = v;
    vr[t] = conj(v);
  }
}

// Householder tridiagonalisation of the Hermitian H[z] (n x n) by one
// cluster.  Rows are dealt to the CTAs cyclically and stay in shared memory.
// Column j: every CTA pulls v_j from the owner of row j, forms p = A v on
// its rows and publishes p and its share of K = v^H p; after a cluster
// barrier it pulls all of p and K, applies A <- A - v w^H - w v^H with
// w = 2p - 2Kv to its rows, and the owner of row j+1 forms and publishes
// v_{j+1}; a second barrier closes the column.  Sums run in a fixed order.
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
  cx<R>* vpub = Hl + (long long)maxloc * n;           // n: v published by the owner of the pivot row
  cx<R>* vloc = vpub + n;                             // n: this CTA's copy of v
  cx<R>* ppub = vloc + n;                             // n: p of own rows, at their offsets
  cx<R>* w = ppub + n;                                // n: w = 2p - 2Kv
  __shared__ R kpub;                                  // this CTA's share of K
  __shared__ R red[32];
  __shared__ cx<R> alpha_s;
  __shared__ R inv_s, twoK_s;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int nloc = n > rank ? (n - rank + CS - 1) / CS : 0;
  for (long long e2 = tid; e2 < (long long)nloc * n; e2 += nth) {
    const int li = (int)(e2 / n), c = (int)(e2 % n);
    Hl[e2] = H[(long long)(rank + li * CS) * n + c];
  }
  __syncthreads();
  if (n > 2 && rank == 0) tridiag_publish(Hl, n, 0, vpub, Vh, d, e, red, &alpha_s, &inv_s);
  cluster.sync();
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1, owner = j % CS;
    // pull v_j
    {
      const cx<R>* src = cluster.map_shared_rank(vpub, owner);
      for (int t = tid; t < m; t += nth) vloc[t] = src[t];
    }
    __syncthreads();
    // p = A v on own rows i > j; K share = sum Re(conj(v_t) p_t)
    const int lstart = (j + 1 - rank + CS - 1) / CS;
    R kp = 0;
    for (int li = lstart + warp; li < nloc; li += nw) {
      const int i = rank + li * CS, t = i - j - 1;
      const cx<R>* row = Hl + (long long)li * n + (j + 1);
      cx<R> a0 = mk<R>(0, 0), a1 = a0, a2 = a0, a3 = a0;
      int k = lane;
      for (; k + 96 < m; k += 128) {
        fma_(a0, row[k], vloc[k]);
        fma_(a1, row[k + 32], vloc[k + 32]);
        fma_(a2, row[k + 64], vloc[k + 64]);
        fma_(a3, row[k + 96], vloc[k + 96]);
      }
      for (; k < m; k += 32) fma_(a0, row[k], vloc[k]);
      cx<R> acc = (a0 + a1) + (a2 + a3);
      acc = warp_sum(acc);
      if (lane == 0) {
        ppub[t] = acc;
        kp += vloc[t].re * acc.re + vloc[t].im * acc.im;
      }
    }
    if (lane == 0) red[warp] = kp;
    __syncthreads();
    if (tid == 0) {
      R t = 0;
      for (int w2 = 0; w2 < nw; ++w2) t += red[w2];
      kpub = t;
    }
    cluster.sync();
    // pull p and K; w = 2p - 2Kv
    if (warp == 0) {
      R kk = lane < CS ? *cluster.map_shared_rank(&kpub, lane) : R(0);
      for (int o = 1; o < 32; o <<= 1) {
        const R other = __shfl_down_sync(0xffffffffu, kk, o);
        kk += (lane + o < 32) ? other : R(0);
      }
      if (lane == 0) twoK_s = R(2) * kk;
    }
    for (int t = tid; t < m; t += nth) w[t] = *cluster.map_shared_rank(ppub + t, (j + 1 + t) % CS);
    __syncthreads();
    {
      const R twoK = twoK_s;
      for (int t = tid; t < m; t += nth)
        w[t] = mk<R>(2 * w[t].re - twoK * vloc[t].re, 2 * w[t].im - twoK * vloc[t].im);
    }
    __syncthreads();
    for (int li = lstart + warp; li < nloc; li += nw) {
      const int i = rank + li * CS, t = i - j - 1;
      cx<R>* row = Hl + (long long)li * n + (j + 1);
      const cx<R> vt = vloc[t], wt = w[t];
#pragma unroll 4
      for (int k = lane; k < m; k += 32) {
        cx<R> a = row[k];
        const cx<R> wk = w[k], vk = vloc[k];
        a.re -= vt.re * wk.re + vt.im * wk.im + wt.re * vk.re + wt.im * vk.im;
        a.im -= vt.im * wk.re - vt.re * wk.im + wt.im * vk.re - wt.re * vk.im;
        row[k] = a;
      }
    }
    // the owner of row j+1 forms and publishes the next reflector
    if (j + 3 < n && rank == (j + 1) % CS) {
      __syncthreads();
      tridiag_publish(Hl + (long long)((j + 1) / CS) * n, n, j + 1, vpub, Vh, d, e, red, &alpha_s, &inv_s);
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

constexpr size_t SMEM_LIMIT = 224 * 1024;   // dynamic shared memory per CTA (227 KB less the static part)

template <typename R>
static size_t tridiag_smem_bytes(int n, int cs) {
  const size_t maxloc = (n + cs - 1) / cs;
  return sizeof(cx<R>) * (maxloc * n + 4 * (size_t)n);
}

// Smallest power-of-two cluster whose shared memory holds the matrix (0: none does).
template <typename R>
int smem_cluster_size(int n) {
  for (int cs = 1; cs <= 16; cs *= 2) {
    const size_t maxloc = (n + cs - 1) / cs;
    if (tridiag_smem_bytes<R>(n, cs) <= SMEM_LIMIT && (cs >= 16 || maxloc <= 64)) return cs;
  }
  return 0;
}

// Cluster size for `batch` matrices: among the sizes from smem_cluster_size(n)
// up to 16 that hold the matrix, the largest whose clusters all fit on the GPU
// at once (cudaOccupancyMaxActiveClusters); a cluster of 16 does not fit on
// every GPC, so for a batch of 8 a size of 13 or 14 can finish in one wave
// where 16 needs two.  Cached per (n, batch) and device.
template <typename R>
static int tridiag_cluster_size(int n, int batch, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(n, batch, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const int cs0 = smem_cluster_size<R>(n);
  int best = cs0, best_waves = 1 << 30;
  for (int cs = std::max(cs0, 2); cs <= 16 && cs0 > 0; ++cs) {
    const size_t smem = tridiag_smem_bytes<R>(n, cs);
    if (smem > SMEM_LIMIT) continue;
    if (ensure_kernel_smem((const void*)tridiag_smem_kernel<R>, smem, cs > 8) != cudaSuccess) continue;
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
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, (const void*)tridiag_smem_kernel<R>, &cfg) != cudaSuccess ||
        active < 1) {
      cudaGetLastError();
      continue;
    }
    const int waves = (batch + active - 1) / active;
    if (waves < best_waves || (waves == best_waves && cs > best)) {
      best_waves = waves;
      best = cs;
    }
  }
  cache[key] = best;
  return best;
}

template <typename R>
cudaError_t tridiag_smem(cudaStream_t st, const cx<R>* H, long long sH, int n, R* d, cx<R>* e, int ldde, cx<R>* Vh,
                         long long sVh, int batch) {
  if (smem_cluster_size<R>(n) == 0) return cudaErrorInvalidValue;
  const int cs = tridiag_cluster_size<R>(n, batch, st);
  const int maxloc = (n + cs - 1) / cs;
  const size_t smem = tridiag_smem_bytes<R>(n, cs);
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
