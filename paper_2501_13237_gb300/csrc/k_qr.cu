// Blocked Householder QR for tall complex matrices (m x n, row-major).
//
// Panels of 32 columns are factored by one thread-block cluster per matrix:
// the panel rows are spread over the cluster's CTAs (cyclically) and kept in
// shared memory; per column the cluster exchanges two partial reductions
// (column norm, reflector projections) through distributed shared memory.
// Each panel also yields the compact-WY factor T (P_0 ... P_{b-1} =
// I - V T V^H).  Trailing updates and the explicit Q then apply each panel's
// block reflector (wy_apply).  All reductions are in a fixed order (deterministic).
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nne {

constexpr int QB = 32;   // panel width
constexpr int PS = QB + 1;   // padded row stride of the shared-memory panel (avoids bank conflicts)

template <typename R>
__global__ void __launch_bounds__(256) qr_panel_kernel(cx<R>* Ab, long long sA, int lda, int m, int pb, int bw,
                                                        cx<R>* Vb, long long sV, int ldv, cx<R>* Tb, long long sT,
                                                        int maxloc) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  cx<R>* A = Ab + z * sA;
  cx<R>* V = Vb + z * sV;
  cx<R>* T = Tb + z * sT;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* P = reinterpret_cast<cx<R>*>(smem_raw);       // [maxloc][PS]
  __shared__ double pn[2];
  __shared__ cx<R> x0s[2];
  __shared__ cx<R> pw[2][QB];
  __shared__ cx<R> red[8][QB];
  __shared__ cx<R> Gp[QB][QB];
  __shared__ cx<R> alphas[QB];
  __shared__ R taus[QB];
  __shared__ double dred[32];
  const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
  const int mp = m - pb;                                   // panel rows
  const int nloc = mp > rank ? (mp - rank + CS - 1) / CS : 0;
  // load own rows (global row pb + rank + li*CS)
  for (int e = tid; e < nloc * QB; e += blockDim.x) {
    const int li = e / QB, c = e % QB;
    const long long gi = pb + rank + (long long)li * CS;
    P[li * PS + c] = c < bw ? A[gi * lda + pb + c] : mk<R>(0, 0);
  }
  __syncthreads();
  for (int j = 0; j < bw; ++j) {
    const int buf = j & 1;
    const int owner = j % CS;                 // CTA owning panel row j
    const int ljo = j / CS;                   // its local index
    // first local row with panel index >= j
    const int lstart = (j - rank + CS - 1) / CS > 0 ? (j - rank + CS - 1) / CS : 0;
    double s = 0;
    for (int li = lstart + tid; li < nloc; li += blockDim.x) s += (double)norm2(P[li * PS + j]);
    s = warp_sum_r(s);
    if (lane == 0) dred[grp] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += dred[w];
      pn[buf] = t;
      if (rank == owner) x0s[buf] = P[ljo * PS + j];
    }
    cluster.sync();
    __shared__ double xn2s;
    __shared__ cx<R> x0l;
    if (tid == 0) {
      double t2 = 0;
      for (int c = 0; c < CS; ++c) t2 += *cluster.map_shared_rank(&pn[buf], c);
      xn2s = t2;
      x0l = *cluster.map_shared_rank(&x0s[buf], owner);
    }
    __syncthreads();
    const double xn2 = xn2s;
    const cx<R> x0 = x0l;
    const double ax0 = sqrt((double)norm2(x0)), xn = sqrt(xn2);
    cx<R> alpha = mk<R>(0, 0);
    double un = 0;
    if (xn > 0) {
      const double pr = ax0 > 0 ? (double)x0.re / ax0 : 1.0, pi = ax0 > 0 ? (double)x0.im / ax0 : 0.0;
      alpha = mk<R>((R)(-xn * pr), (R)(-xn * pi));
      un = sqrt(2.0 * xn2 + 2.0 * xn * ax0);
    }
    const R inv = un > 0 ? (R)(1.0 / un) : R(0);
    if (tid == 0) {
      alphas[j] = alpha;
      taus[j] = un > 0 ? R(2) : R(0);
    }
    // v = (x - alpha e_0) / un on own rows
    for (int li = lstart + tid; li < nloc; li += blockDim.x) {
      cx<R> u = P[li * PS + j];
      if (rank == owner && li == ljo) u = u - alpha;
      P[li * PS + j] = inv * u;
    }
    __syncthreads();
    // partial w_c = sum conj(v_i) P[i][c], c in (j, bw)
    {
      const int c = lane;
      cx<R> acc = mk<R>(0, 0);
      if (c > j && c < bw)
        for (int li = lstart + grp; li < nloc; li += 8) fmac_(acc, P[li * PS + j], P[li * PS + c]);
      red[grp][c] = acc;
    }
    __syncthreads();
    if (tid < QB) {
      cx<R> t = mk<R>(0, 0);
      for (int g = 0; g < 8; ++g) t = t + red[g][tid];
      pw[buf][tid] = t;
    }
    cluster.sync();
    if (j + 1 < bw) {
      // w_c over the cluster (fixed order), then P[i][c] -= 2 v_i w_c
      __shared__ cx<R> wfull[QB];
      if (tid < QB) {
        cx<R> t = mk<R>(0, 0);
        for (int cc = 0; cc < CS; ++cc) t = t + *cluster.map_shared_rank(&pw[buf][tid], cc);
        wfull[tid] = mk<R>(2 * t.re, 2 * t.im);
      }
      __syncthreads();
      for (int e = tid; e < (nloc - lstart) * QB; e += blockDim.x) {
        const int li = lstart + e / QB, c = e % QB;
        if (c > j && c < bw) {
          const cx<R> vi = P[li * PS + j];
          P[li * PS + c] = P[li * PS + c] - vi * wfull[c];
        }
      }
      __syncthreads();
    }
  }
  // Gram of the reflectors (v_c zero above panel row c) -> T
  for (int e = tid; e < QB * QB; e += blockDim.x) {
    const int a = e / QB, b = e % QB;
    cx<R> acc = mk<R>(0, 0);
    if (a < bw && b < bw && a <= b)
      for (int li = 0; li < nloc; ++li) {
        const int pi = rank + li * CS;       // panel row index
        if (pi >= b) fmac_(acc, P[li * PS + a], P[li * PS + b]);   // pi >= b >= a
      }
    Gp[a][b] = acc;
  }
  // write back V and the R part of A
  for (int e = tid; e < nloc * QB; e += blockDim.x) {
    const int li = e / QB, c = e % QB;
    if (c >= bw) continue;
    const int pi = rank + li * CS;
    const long long gi = pb + pi;
    const cx<R> val = P[li * PS + c];
    V[gi * ldv + pb + c] = pi >= c ? val : mk<R>(0, 0);
    A[gi * lda + pb + c] = pi < c ? val : (pi == c ? alphas[c] : mk<R>(0, 0));
  }
  cluster.sync();
  if (rank == 0) {
    __shared__ cx<R> G[QB][QB];
    for (int e = tid; e < QB * QB; e += blockDim.x) {
      const int a = e / QB, b = e % QB;
      cx<R> t = mk<R>(0, 0);
      for (int cc = 0; cc < CS; ++cc) t = t + *cluster.map_shared_rank(&Gp[a][b], cc);
      G[a][b] = t;
    }
    __syncthreads();
    if (tid < 32) {
      // T upper triangular: T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i]
      __shared__ cx<R> Ts[QB][QB];
      for (int i = 0; i < QB; ++i) Ts[tid][i] = mk<R>(0, 0);
      __syncwarp();
      for (int i = 0; i < bw; ++i) {
        const int rr = tid;
        cx<R> acc = mk<R>(0, 0);
        if (rr < i)
          for (int l = rr; l < i; ++l) fma_(acc, Ts[rr][l], G[l][i]);
        __syncwarp();
        if (rr < i) Ts[rr][i] = mk<R>(-taus[i] * acc.re, -taus[i] * acc.im);
        if (rr == i) Ts[i][i] = mk<R>(taus[i], 0);
        __syncwarp();
      }
      for (int i = 0; i < QB; ++i) T[tid * QB + i] = Ts[tid][i];
    }
  }
  cluster.sync();
}

template <typename R>
__global__ void qr_extract_r2_kernel(const cx<R>* Ab, long long sA, int lda, int k, int n, cx<R>* Rb, long long sR) {
  const int z = blockIdx.y;
  const cx<R>* A = Ab + z * sA;
  cx<R>* Rm = Rb + z * sR;
  const long long count = (long long)k * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(i / n), col = (int)(i % n);
    Rm[i] = col >= row ? A[(long long)row * lda + col] : mk<R>(0, 0);
  }
}

template <typename K, typename... Args>
static cudaError_t launch_cluster_qr(K kernel, int cs, int batch, size_t smem, cudaStream_t st, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cs > 8) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
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

QrWork qr_workspace(int m, int n) {
  QrWork w;
  const int k = std::min(m, n);
  const int np = (k + QB - 1) / QB;
  // V (m x n) + T (np x 32 x 32) + WY application workspace (n columns)
  w.cx_elems = (long long)m * n + (long long)np * QB * QB + wy_workspace(n) + 64;
  return w;
}

template <typename R>
cudaError_t qr(cudaStream_t st, cx<R>* A, long long sA, int m, int n, cx<R>* Q, long long sQ, cx<R>* Rout,
               long long sR, void* cx_ws, int batch) {
  const int k = std::min(m, n);
  if (k <= 0 || batch <= 0) return cudaSuccess;
  const int np = (k + QB - 1) / QB;
  cx<R>* V = reinterpret_cast<cx<R>*>(cx_ws);
  const long long sV = (long long)m * n;
  cx<R>* T = V + sV * batch;
  const long long sT = (long long)np * QB * QB;
  cx<R>* wyws = T + sT * batch;
  cudaError_t e;
  for (int p = 0; p < np; ++p) {
    const int pb = p * QB, bw = std::min(QB, k - pb);
    const int mp = m - pb;
    int cs = mp >= 512 ? 8 : (mp >= 128 ? 4 : (mp >= 32 ? 2 : 1));
    int maxloc = (mp + cs - 1) / cs;
    size_t smem = sizeof(cx<R>) * (size_t)maxloc * PS;
    if (smem > 160 * 1024) {
      cs = 16;
      maxloc = (mp + cs - 1) / cs;
      smem = sizeof(cx<R>) * (size_t)maxloc * PS;
    }
    {
      ProfScope ps(st, K_QR_FACTOR);
      e = launch_cluster_qr(qr_panel_kernel<R>, cs, batch, smem, st, A, sA, n, m, pb, bw, V, sV, n, T + p * QB * QB,
                            sT, maxloc);
    }
    if (e != cudaSuccess) return e;
    const int nt = n - pb - bw;
    if (nt > 0) {
      cx<R>* Vp = V + (long long)pb * n + pb;
      cx<R>* At = A + (long long)pb * n + pb + bw;
      // A_t <- (I - V T V^H)^H A_t
      if ((e = wy_apply<R>(st, false, Vp, sV, n, T + p * QB * QB, sT, QB, true, bw, mp, nt, At, sA, n, wyws,
                           batch)) != cudaSuccess)
        return e;
    }
  }
  if (Rout) {
    ProfScope ps(st, K_ELEMWISE);
    qr_extract_r2_kernel<R><<<dim3(64, batch), 256, 0, st>>>(A, sA, n, k, n, Rout, sR);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = identity<R>(st, Q, sQ, m, k, batch)) != cudaSuccess) return e;
  for (int p = np - 1; p >= 0; --p) {
    const int pb = p * QB, bw = std::min(QB, k - pb);
    const int mp = m - pb, kc = k - pb;
    cx<R>* Vp = V + (long long)pb * n + pb;
    cx<R>* Qp = Q + (long long)pb * k + pb;
    // Q_p <- (I - V T V^H) Q_p
    if ((e = wy_apply<R>(st, false, Vp, sV, n, T + p * QB * QB, sT, QB, false, bw, mp, kc, Qp, sQ, k, wyws, batch)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

template cudaError_t qr<float>(cudaStream_t, cx<float>*, long long, int, int, cx<float>*, long long, cx<float>*,
                               long long, void*, int);
template cudaError_t qr<double>(cudaStream_t, cx<double>*, long long, int, int, cx<double>*, long long, cx<double>*,
                                long long, void*, int);

}  // namespace nne
