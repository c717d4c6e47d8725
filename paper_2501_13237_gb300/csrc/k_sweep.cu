// a7 -- Pauli expectation values by transfer-matrix sweeps (Sec. 2.2.3:
// <O>_lambda from an exact contraction of the network).
//   T_P(k)[a][b] = sum_s v_P[s] M_k[a][s][b],  v_P[s] = P[j][i] for s = 2 i + j:
//   v_I = (1,0,0,1), v_X = (0,1,1,0), v_Y = (0,i,-i,0), v_Z = (1,0,0,-1).
//   L_0 = 1, L_{k+1} = L_k T_I(k);  R_n = 1, R_k = T_I(k) R_{k+1};
//   <P> = L_first T_P(first) ... T_P(last) R_{last+1} / L_n.
//
// Environment sweep (env_cluster_kernel): one thread-block cluster per
// (pass, instance); the left pass and the right pass of every instance run at
// the same time.  At each site the cluster's CTAs split the site tensor
// (left pass: output columns b; right pass: rows a), stream it from HBM with
// 16-byte coalesced loads, and exchange the new environment's slices and its
// max-abs through distributed shared memory, one cluster barrier per site.
// Besides the environments the sweep keeps, per site, the four partial
// contractions
//   ell_k[s][b] = sum_a L_k[a] M_k[a][s][b],   rho_k[t][a] = sum_b M_k[a][t][b] R_{k+1}[b],
// so every Pauli string on one site or two neighbouring sites is a dot product
// of stored vectors (obs_local_kernel) and the site tensors are read once per
// pass.  Strings with a longer support take obs_kernel, which carries a vector
// through the interior sites.
// Accumulation: float64 for complex128 states; for complex64 states the
// products are formed in float32, summed in float32 over at most 16 terms and
// then added into float64 accumulators.  Each environment is rescaled to
// max-abs 1 and its log-scale carried separately, so long chains neither
// overflow nor underflow.
#include <map>
#include <mutex>

#include "kernels.cuh"

namespace cg = cooperative_groups;

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

namespace sweep {

constexpr int THREADS = 256;
constexpr int NB = 8;            // loads per thread and batch; also the float32 run length before a float64 fold
constexpr int RING_STAGES = 4;   // batches in flight per thread (cp.async ring in shared memory)

// Elements of one 16-byte load: two complex64 or one complex128.
template <typename R> struct Vec;
template <> struct Vec<float> { static constexpr int V = 2; };
template <> struct Vec<double> { static constexpr int V = 1; };

// Streaming loads (site tensors are read once per pass).
template <typename R, int V>
__device__ __forceinline__ void ldv(const cx<R>* p, cx<R>* o);
template <>
__device__ __forceinline__ void ldv<float, 2>(const cx<float>* p, cx<float>* o) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  o[0] = mk<float>(v.x, v.y);
  o[1] = mk<float>(v.z, v.w);
}
template <>
__device__ __forceinline__ void ldv<float, 1>(const cx<float>* p, cx<float>* o) {
  const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  o[0] = mk<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ void ldv<double, 1>(const cx<double>* p, cx<double>* o) {
  const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  o[0] = mk<double>(v.x, v.y);
}

// Asynchronous global -> shared copy of one load unit (16 bytes, or 8 for a
// single complex64); bytes past `valid` are zero-filled.
template <int BYTES>
__device__ __forceinline__ void cp_unit(uint32_t dst, const void* src, bool valid) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ring() { asm volatile("cp.async.wait_group %0;" ::"n"(RING_STAGES - 1) : "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// This thread's slot i of ring stage st (16-byte slots, threads interleaved).
__device__ __forceinline__ uint32_t ring_slot(uint32_t ring, int st, int i) {
  return ring + (uint32_t)(((st * NB + i) * THREADS + (int)threadIdx.x) * 16);
}
template <typename R, int V>
__device__ __forceinline__ void ring_read(const unsigned char* ring_ptr, int st, int i, cx<R>* o) {
  const unsigned char* p = ring_ptr + ((st * NB + i) * THREADS + threadIdx.x) * 16;
#pragma unroll
  for (int v = 0; v < V; ++v) o[v] = reinterpret_cast<const cx<R>*>(p)[v];
}

__device__ __forceinline__ cx<double> up(cx<float> a) { return mk<double>(a.re, a.im); }
__device__ __forceinline__ cx<double> up(cx<double> a) { return a; }

// Shared-memory layout of env_cluster_kernel, in cx<double> units from the base.
struct Layout {
  int D, SL;
  __host__ __device__ int cur() const { return 0; }                 // D: current environment (float64)
  __host__ __device__ int slice() const { return D; }               // 2 x SL: this CTA's slice of the next one
  __host__ __device__ int fin() const { return D + 2 * SL; }        // 4 x SL: left-pass results of this CTA
  __host__ __device__ int part() const { return D + 6 * SL; }       // 2 x THREADS: row-group partial sums
  __host__ __device__ int scal() const { return D + 6 * SL + 2 * THREADS; }   // 8 doubles (maxes, reduction)
  __host__ __device__ int coef() const { return scal() + 8; }       // D x cx<R>: environment in the state's precision
  // per-thread rings of asynchronous copies (RING_STAGES x NB 16-byte slots per thread), 16-byte aligned
  __host__ __device__ size_t ring_off(size_t esz) const { return (16 * (size_t)coef() + esz * (size_t)D + 15) & ~size_t(15); }
  __host__ __device__ size_t bytes(size_t esz) const { return ring_off(esz) + (size_t)RING_STAGES * NB * THREADS * 16; }
};

__host__ __device__ inline int slice_cap(int D, int cs) { return (D + cs - 1) / cs + 2; }

__device__ __forceinline__ double block_max_sw(double v, double* red) {
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  for (int i = 0; i < THREADS / 32; ++i) t = fmax(t, red[i]);
  return t;
}

// Left pass at one site: fin[s][j] = sum_a coef[a] M[a][s][b0 + j] for this CTA's columns.
// Thread (unit u, row group g) streams the rows a = g, g + G, ... of its unit
// through its own ring of asynchronous copies, RING_STAGES batches of NB rows
// in flight.
template <typename R, int V>
__device__ void left_site(const cx<R>* __restrict__ M, int dl, int dr, int b0, int w, const cx<R>* coef,
                          cx<double>* fin, int SL, cx<double>* part, unsigned char* ring_ptr) {
  constexpr int BYTES = (int)sizeof(cx<R>) * V;
  const uint32_t ring = (uint32_t)__cvta_generic_to_shared(ring_ptr);
  const int t = threadIdx.x;
  const int wu = w / V, U = 4 * wu;
  if (U == 0) return;
  const int G = U >= THREADS ? 1 : THREADS / U;   // row groups
  for (int u0 = 0; u0 < U; u0 += THREADS) {
    const int u = u0 + (G > 1 ? t % U : t), g = G > 1 ? t / U : 0;
    const bool act = u < U && g < G;
    cx<double> acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = mk<double>(0, 0);
    if (act) {
      const int s = u / wu, j = (u % wu) * V;
      const cx<R>* col = M + (long long)s * dr + b0 + j;
      const long long rs = 4LL * dr * G;   // element step between this thread's rows
      const int nrows = (dl - g + G - 1) / G;
      const int nbatch = (nrows + NB - 1) / NB;
      auto issue = [&](int bi) {
        if (bi < nbatch) {
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int ri = bi * NB + i;
            const bool ok = ri < nrows;
            cp_unit<BYTES>(ring_slot(ring, bi % RING_STAGES, i), ok ? col + (long long)g * 4 * dr + ri * rs : col, ok);
          }
        }
        cp_commit();
      };
#pragma unroll
      for (int b = 0; b < RING_STAGES - 1; ++b) issue(b);
      for (int bi = 0; bi < nbatch; ++bi) {
        issue(bi + RING_STAGES - 1);
        cp_wait_ring();
        cx<R> s32[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s32[v] = mk<R>(0, 0);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const int ri = bi * NB + i;
          cx<R> m[V];
          ring_read<R, V>(ring_ptr, bi % RING_STAGES, i, m);
          const cx<R> c = ri < nrows ? coef[g + ri * G] : mk<R>(0, 0);
#pragma unroll
          for (int v = 0; v < V; ++v) fma_(s32[v], c, m[v]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = acc[v] + up(s32[v]);
      }
      cp_wait_all();
    }
    if (G == 1) {
      if (act) {
        const int s = u / wu, j = (u % wu) * V;
#pragma unroll
        for (int v = 0; v < V; ++v) fin[s * SL + j + v] = acc[v];
      }
    } else {
      // partial sums of the row groups, then added in group order
      if (act)
#pragma unroll
        for (int v = 0; v < V; ++v) part[(g * U + u) * V + v] = acc[v];
      __syncthreads();
      if (t < U) {
        const int s = t / wu, j = (t % wu) * V;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          cx<double> tot = mk<double>(0, 0);
          for (int gg = 0; gg < G; ++gg) tot = tot + part[(gg * U + t) * V + v];
          fin[s * SL + j + v] = tot;
        }
      }
    }
  }
}

// Right pass at one site: rho[tt][a] = sum_b M[a][tt][b] coef[b] for this CTA's rows, one warp per row.
// Writes rho to global memory and R[a] = rho[0][a] + rho[3][a] into the slice; returns the row max-abs.
// A warp's work is a flat list of jobs (row, segment tt, batch of 32 NB units),
// streamed through each lane's ring of asynchronous copies.
template <typename R, int V>
__device__ double right_site(const cx<R>* __restrict__ M, int dr, int a0, int a1, const cx<R>* coef, cx<double>* rho,
                             int D, cx<double>* slice, unsigned char* ring_ptr) {
  constexpr int BYTES = (int)sizeof(cx<R>) * V;
  const uint32_t ring = (uint32_t)__cvta_generic_to_shared(ring_ptr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = THREADS / 32;
  const int nu = dr / V;                                   // units per segment
  const int nbs = (nu + 32 * NB - 1) / (32 * NB);          // batches per segment
  const int rows_w = a1 - a0 > warp ? (a1 - a0 - warp + nw - 1) / nw : 0;
  const int jobs = rows_w * 4 * nbs;
  auto job_src = [&](int jb, int i, bool& ok) -> const cx<R>* {
    const int ri = jb / (4 * nbs), rem = jb % (4 * nbs), tt = rem / nbs, bb = rem % nbs;
    const int a = a0 + warp + ri * nw;
    const int uu = bb * 32 * NB + lane + 32 * i;
    ok = uu < nu;
    return M + ((long long)a * 4 + tt) * dr + (ok ? uu * V : 0);
  };
  auto issue = [&](int jb) {
    if (jb < jobs) {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        bool ok;
        const cx<R>* src = job_src(jb, i, ok);
        cp_unit<BYTES>(ring_slot(ring, jb % RING_STAGES, i), src, ok);
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int b = 0; b < RING_STAGES - 1; ++b) issue(b);
  double mx = 0;
  cx<double> acc = mk<double>(0, 0), seg0 = mk<double>(0, 0);
  for (int jb = 0; jb < jobs; ++jb) {
    issue(jb + RING_STAGES - 1);
    cp_wait_ring();
    const int ri = jb / (4 * nbs), rem = jb % (4 * nbs), tt = rem / nbs, bb = rem % nbs;
    cx<R> s32 = mk<R>(0, 0);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int uu = bb * 32 * NB + lane + 32 * i;
      cx<R> m[V];
      ring_read<R, V>(ring_ptr, jb % RING_STAGES, i, m);
      if (uu < nu)
#pragma unroll
        for (int v = 0; v < V; ++v) fma_(s32, m[v], coef[uu * V + v]);
    }
    acc = acc + up(s32);
    if (bb == nbs - 1) {   // segment tt of row a complete
      const cx<double> tot = warp_sum(acc);
      acc = mk<double>(0, 0);
      const int a = a0 + warp + ri * nw;
      if (lane == 0) rho[(long long)tt * D + a] = tot;
      if (tt == 0) seg0 = tot;
      if (tt == 3 && lane == 0) {
        const cx<double> Ra = seg0 + tot;
        slice[a - a0] = Ra;
        mx = fmax(mx, fmax(fabs(Ra.re), fabs(Ra.im)));
      }
    }
  }
  cp_wait_all();
  return mx;
}

}  // namespace sweep

// Both environment sweeps and the per-site partial contractions in one launch.
// grid (cs, 2, n_inst), cluster (cs, 1, 1): cluster (pass, z); pass 0 left, 1 right.
// env: [z][pass][k = 0..n][D] complex double, envscale: [z][pass][k], vecs: [z][pass][k = 0..n-1][4][D].
template <typename R>
__global__ void __launch_bounds__(sweep::THREADS) env_cluster_kernel(int n, const int* __restrict__ dims,
                                                                    const void* const* __restrict__ site,
                                                                    const long long* __restrict__ stride, int D,
                                                                    double* env, double* envscale, double* vecs) {
  using namespace sweep;
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int pass = blockIdx.y, z = blockIdx.z, t = threadIdx.x;
  constexpr int VV = Vec<R>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Layout L{D, slice_cap(D, cs)};
  cx<double>* base = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* cur = base + L.cur();
  cx<double>* slice = base + L.slice();
  cx<double>* fin = base + L.fin();
  cx<double>* part = base + L.part();
  double* scal = reinterpret_cast<double*>(base + L.scal());   // [0..1] maxes (double-buffered), [8..15] reduction
  cx<R>* coef = reinterpret_cast<cx<R>*>(base + L.coef());
  unsigned char* ring_ptr = smem_raw + L.ring_off(sizeof(cx<R>));
  cx<double>* E = reinterpret_cast<cx<double>*>(env) + ((long long)z * 2 + pass) * (n + 1) * D;
  double* ls = envscale + ((long long)z * 2 + pass) * (n + 1);
  cx<double>* VK = reinterpret_cast<cx<double>*>(vecs) + ((long long)z * 2 + pass) * n * 4 * D;
  const int first = pass == 0 ? 0 : n;
  if (t == 0) {
    cur[0] = mk<double>(1, 0);
    coef[0] = mk<R>(1, 0);
    if (rank == 0) {
      E[(long long)first * D] = mk<double>(1, 0);
      ls[first] = 0;
    }
  }
  __syncthreads();
  double lsc = 0;
  int pb = 0;
  for (int step = 0; step < n; ++step) {
    const int k = pass == 0 ? step : n - 1 - step;
    const int dl = dims[k], dr = dims[k + 1];
    const cx<R>* M = reinterpret_cast<const cx<R>*>(site[k]) + z * stride[k];
    const bool vec = VV > 1 && dr % VV == 0 && (reinterpret_cast<uintptr_t>(M) & 15) == 0;
    cx<double>* sl = slice + pb * L.SL;
    double mx = 0;
    int own0, own1;   // entries of the next environment this CTA owns
    if (pass == 0) {
      const int v = vec ? VV : 1;
      const int bs = ((dr + cs - 1) / cs + v - 1) / v * v;
      const int b0 = min(dr, rank * bs), b1 = min(dr, b0 + bs);
      own0 = b0;
      own1 = b1;
      if (vec) left_site<R, VV>(M, dl, dr, b0, b1 - b0, coef, fin, L.SL, part, ring_ptr);
      else left_site<R, 1>(M, dl, dr, b0, b1 - b0, coef, fin, L.SL, part, ring_ptr);
      __syncthreads();
      cx<double>* ell = VK + (long long)k * 4 * D;
      for (int q = t; q < 4 * (b1 - b0); q += THREADS) {
        const int s = q / (b1 - b0), j = q % (b1 - b0);
        ell[(long long)s * D + b0 + j] = fin[s * L.SL + j];
      }
      for (int j = t; j < b1 - b0; j += THREADS) {
        const cx<double> Lb = fin[j] + fin[3 * L.SL + j];
        sl[j] = Lb;
        mx = fmax(mx, fmax(fabs(Lb.re), fabs(Lb.im)));
      }
    } else {
      const int rs = (dl + cs - 1) / cs;
      const int a0 = min(dl, rank * rs), a1 = min(dl, a0 + rs);
      own0 = a0;
      own1 = a1;
      cx<double>* rho = VK + (long long)k * 4 * D;
      mx = vec ? right_site<R, VV>(M, dr, a0, a1, coef, rho, D, sl, ring_ptr)
               : right_site<R, 1>(M, dr, a0, a1, coef, rho, D, sl, ring_ptr);
    }
    mx = block_max_sw(mx, scal + 8);
    if (t == 0) scal[pb] = mx;
    (void)own0;
    (void)own1;
    cluster.sync();   // every slice and max of this site is published
    // the next environment, normalised to max-abs 1, gathered from the cluster's slices
    double m = 0;
    for (int r = 0; r < cs; ++r) m = fmax(m, *cluster.map_shared_rank(scal + pb, r));
    const double inv = m > 0 ? 1.0 / m : 1.0;
    const int nd = pass == 0 ? dr : dl;               // length of the next environment
    int width;
    if (pass == 0) {
      const int v = vec ? VV : 1;
      width = ((dr + cs - 1) / cs + v - 1) / v * v;
    } else {
      width = (dl + cs - 1) / cs;
    }
    const int knext = pass == 0 ? k + 1 : k;
    for (int i = t; i < nd; i += THREADS) {
      const int r = i / width;
      const cx<double> val = cluster.map_shared_rank(slice + pb * L.SL, r)[i - r * width];
      const cx<double> nv = inv * val;
      cur[i] = nv;
      coef[i] = mk<R>((R)nv.re, (R)nv.im);
      if (rank == 0) E[(long long)knext * D + i] = nv;
    }
    lsc += m > 0 ? log(m) : 0.0;
    if (rank == 0 && t == 0) ls[knext] = lsc;
    pb ^= 1;
    __syncthreads();
  }
  cluster.sync();   // no CTA leaves while a peer may still read its shared memory
}

// Strings whose support spans three or more sites: one CTA per (string,
// instance) carries S from R_{last+1} down to `first`; idx lists the strings.
template <typename R>
__global__ void __launch_bounds__(256) obs_kernel(int n, const int* dims, const void* const* site,
                                                   const long long* stride, int max_dim, const double* env,
                                                   const double* envscale, const uint8_t* paulis, const int* first,
                                                   const int* last, const int* idx, int n_obs, double* out) {
  extern __shared__ unsigned char smem_raw[];
  cx<double>* S = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* S2 = S + max_dim;
  __shared__ double red[32];
  __shared__ cx<double> cred[32];
  const int o = idx[blockIdx.x], z = blockIdx.y;
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

// Strings on at most two neighbouring sites (and the identity): one warp per
// (string, instance), dot products of the stored per-site vectors:
//   one site k:      sum_b (sum_s v_P[s] ell_k[s][b]) R_{k+1}[b]
//   sites k, k + 1:  sum_c (sum_s v_P[s] ell_k[s][c]) (sum_t v_Q[t] rho_{k+1}[t][c])
__global__ void __launch_bounds__(256) obs_local_kernel(int n, const int* __restrict__ dims, int D,
                                                        const double* env, const double* envscale,
                                                        const double* vecs, const uint8_t* __restrict__ paulis,
                                                        const int* __restrict__ first, const int* __restrict__ last,
                                                        int n_obs, double* out) {
  const int lane = threadIdx.x & 31;
  const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), z = blockIdx.y;
  if (o >= n_obs) return;
  const int f = first[o], l = last[o];
  double* res = out + ((long long)z * n_obs + o) * 2;
  if (f < 0) {
    if (lane == 0) { res[0] = 1.0; res[1] = 0.0; }
    return;
  }
  if (l - f > 1) return;
  const cx<double>* EL = reinterpret_cast<const cx<double>*>(env) + ((long long)z * 2 + 0) * (n + 1) * D;
  const cx<double>* ER = reinterpret_cast<const cx<double>*>(env) + ((long long)z * 2 + 1) * (n + 1) * D;
  const double* lsL = envscale + ((long long)z * 2 + 0) * (n + 1);
  const double* lsR = envscale + ((long long)z * 2 + 1) * (n + 1);
  const cx<double>* ell = reinterpret_cast<const cx<double>*>(vecs) + (((long long)z * 2 + 0) * n + f) * 4 * D;
  const int P = paulis[(long long)o * n + f];
  const cx<double> p0 = pvec(P, 0), p1 = pvec(P, 1), p2 = pvec(P, 2), p3 = pvec(P, 3);
  const int d = dims[f + 1];
  cx<double> acc = mk<double>(0, 0);
  double lscale;
  if (l == f) {
    const cx<double>* Rn = ER + (long long)(f + 1) * D;
    for (int b = lane; b < d; b += 32) {
      cx<double> u = mk<double>(0, 0);
      fma_(u, p0, ell[b]);
      fma_(u, p1, ell[D + b]);
      fma_(u, p2, ell[2 * D + b]);
      fma_(u, p3, ell[3 * D + b]);
      fma_(acc, u, Rn[b]);
    }
    lscale = lsL[f] + lsR[f + 1];
  } else {
    const cx<double>* rho = reinterpret_cast<const cx<double>*>(vecs) + (((long long)z * 2 + 1) * n + l) * 4 * D;
    const int Q = paulis[(long long)o * n + l];
    const cx<double> q0 = pvec(Q, 0), q1 = pvec(Q, 1), q2 = pvec(Q, 2), q3 = pvec(Q, 3);
    for (int c = lane; c < d; c += 32) {
      cx<double> u = mk<double>(0, 0), w = mk<double>(0, 0);
      fma_(u, p0, ell[c]);
      fma_(u, p1, ell[D + c]);
      fma_(u, p2, ell[2 * D + c]);
      fma_(u, p3, ell[3 * D + c]);
      fma_(w, q0, rho[c]);
      fma_(w, q1, rho[D + c]);
      fma_(w, q2, rho[2 * D + c]);
      fma_(w, q3, rho[3 * D + c]);
      fma_(acc, u, w);
    }
    lscale = lsL[f] + lsR[l + 1];
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const cx<double> tr = EL[(long long)n * D];
    const double scale = exp(lscale - lsL[n]);
    const double den = tr.re * tr.re + tr.im * tr.im;
    const double qr = (acc.re * tr.re + acc.im * tr.im) / den, qi = (acc.im * tr.re - acc.re * tr.im) / den;
    res[0] = qr * scale;
    res[1] = qi * scale;
  }
}

// Cluster size of the environment sweep: two clusters (left, right pass) per
// instance, one CTA per SM (the copy rings fill shared memory).  A cluster's
// time is its sites' bytes over its CTAs, so the size maximises CTAs per
// cluster / waves, the waves counted from the occupancy query of each size
// (2..16; GB300's GPCs hold 7 clusters of 16, 15 of 8, 16 of 9); small bonds
// take fewer.  NNE_OPT_SWEEP_CLUSTER forces a size.
int g_sweep_cluster = 0;
void set_sweep_cluster(int cs) { g_sweep_cluster = cs < 0 ? 0 : (cs > 16 ? 16 : cs); }

template <typename R>
static int sweep_cluster_size(int n_inst, int D) {
  if (g_sweep_cluster > 0) return g_sweep_cluster;
  if (D < 16) return 1;
  if (D < 64) return 4;
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> memo;
  const std::pair<int, int> key{n_inst, D};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  const int clusters = 2 * n_inst;
  int best = 8;
  double best_rate = 0;
  for (int cs = 16; cs >= 2; --cs) {
    const sweep::Layout L{D, sweep::slice_cap(D, cs)};
    const size_t smem = L.bytes(sizeof(cx<R>));
    if (smem > 227 * 1024) continue;
    if (ensure_kernel_smem((const void*)env_cluster_kernel<R>, smem, cs > 8) != cudaSuccess) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 2, n_inst);
    cfg.blockDim = dim3(sweep::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, (const void*)env_cluster_kernel<R>, &cfg) != cudaSuccess ||
        active < 1) {
      (void)cudaGetLastError();
      continue;
    }
    const int waves = (clusters + active - 1) / active;
    const double rate = (double)cs / waves;
    if (rate > best_rate) {
      best_rate = rate;
      best = cs;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  memo[key] = best;
  return best;
}

template <typename R>
cudaError_t expect_sweep(cudaStream_t st, int n, const int* d_dims, const void* const* d_site,
                         const long long* d_stride, int n_inst, int max_dim, int n_obs, const uint8_t* d_paulis,
                         const int* d_first, const int* d_last, const int* d_general, int n_general, double* d_env,
                         double* d_envscale, double* d_vecs, double* d_out) {
  cudaError_t e;
  {
    const int cs = sweep_cluster_size<R>(n_inst, max_dim);
    const sweep::Layout L{max_dim, sweep::slice_cap(max_dim, cs)};
    const size_t smem = L.bytes(sizeof(cx<R>));
    if (smem > 227 * 1024) return cudaErrorInvalidValue;   // bonds above ~3000 do not fit the copy rings
    if ((e = ensure_kernel_smem((const void*)env_cluster_kernel<R>, smem, cs > 8)) != cudaSuccess) return e;
    // algorithmic bytes: every site tensor read once by each pass
    ProfScope ps(st, K_SWEEP_ENV);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 2, n_inst);
    cfg.blockDim = dim3(sweep::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, env_cluster_kernel<R>, n, d_dims, d_site, d_stride, max_dim, d_env, d_envscale,
                           d_vecs);
  }
  if (e != cudaSuccess) return e;
  if (n_obs <= 0) return cudaSuccess;
  {
    ProfScope ps(st, K_SWEEP_OBS);
    obs_local_kernel<<<dim3((n_obs + 7) / 8, n_inst), 256, 0, st>>>(n, d_dims, max_dim, d_env, d_envscale, d_vecs,
                                                                   d_paulis, d_first, d_last, n_obs, d_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (n_general <= 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(cx<double>) * (size_t)max_dim;
  if ((e = ensure_kernel_smem((const void*)obs_kernel<R>, smem, false)) != cudaSuccess) return e;
  ProfScope ps(st, K_SWEEP_OBS);
  obs_kernel<R><<<dim3(n_general, n_inst), 256, smem, st>>>(n, d_dims, d_site, d_stride, max_dim, d_env, d_envscale,
                                                            d_paulis, d_first, d_last, d_general, n_obs, d_out);
  return cudaGetLastError();
}

#define NNE_INST_SWEEP(R)                                                                                          \
  template cudaError_t expect_sweep<R>(cudaStream_t, int, const int*, const void* const*, const long long*, int, int, \
                                       int, const uint8_t*, const int*, const int*, const int*, int, double*, double*, \
                                       double*, double*);
NNE_INST_SWEEP(float)
NNE_INST_SWEEP(double)

}  // namespace nne
