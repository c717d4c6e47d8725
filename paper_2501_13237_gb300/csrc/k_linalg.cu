// Dense linear algebra of the truncation step, written for GB300:
//   * Householder reduction of a Hermitian matrix to real tridiagonal form,
//     one thread-block cluster per matrix (hardware cluster barriers, matrix
//     resident in L2), two cluster barriers per column;
//   * eigenvalues of the tridiagonal by 32-way multisection with Sturm
//     counts (one warp per wanted eigenvalue);
//   * eigenvectors by inverse iteration with a partially pivoted tridiagonal
//     LU (one thread per eigenvector), back-transformed through the phase
//     scaling and the Householder reflectors (one CTA per 32 columns);
//   * Householder QR (one cluster per matrix, column blocks owned by CTAs,
//     one cluster barrier per column) and explicit Q formation; used to
//     orthonormalise the eigenvector block and for the centre moves.
// Precision follows the state: float for complex64 states, double for
// complex128.  The reductions are written in a fixed order, so results are
// bitwise reproducible run to run and independent of what else is batched.
#include <map>
#include <mutex>

#include "kernels.cuh"
#include <float.h>

namespace cg = cooperative_groups;

namespace nne {

template <typename R> struct Lim;
template <> struct Lim<float> {
  static __device__ __forceinline__ float eps() { return FLT_EPSILON; }
  static __device__ __forceinline__ float tiny() { return FLT_MIN; }
  static __device__ __forceinline__ float big() { return 1e30f; }
};
template <> struct Lim<double> {
  static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
  static __device__ __forceinline__ double tiny() { return DBL_MIN; }
  static __device__ __forceinline__ double big() { return 1e250; }
};

// Sum over the block in a fixed order; every thread gets the total.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum_r(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = 0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Householder vector of x (length m, in smem v, overwritten): P = I - 2 v v^H,
// P x = alpha e_1.  Returns alpha.  Whole block participates.
template <typename R>
__device__ cx<R> householder(cx<R>* v, int m, double* red) {
  double s = 0;
  for (int t = threadIdx.x; t < m; t += blockDim.x) s += norm2d(v[t]);
  const double xn2 = block_sum(s, red);
  const cx<R> x0 = v[0];
  double pr, pi, ax0;
  unit_phase_of(x0, &pr, &pi, &ax0);
  const double xn = sqrt(xn2);
  cx<R> alpha = mk<R>(0, 0);
  double un = 0;
  if (xn > 0) {
    alpha = mk<R>((R)(-xn * pr), (R)(-xn * pi));
    un = sqrt(2.0 * xn2 + 2.0 * xn * ax0);
  }
  __syncthreads();
  const R inv = un > 0 ? (R)(1.0 / un) : R(0);
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    cx<R> u = v[t];
    if (t == 0) u = u - alpha;
    v[t] = inv * u;
  }
  __syncthreads();
  return alpha;
}

// ---------------------------------------------------------------- tridiagonal
// H (n x n) -> real tridiagonal d, complex subdiagonal e (e[k] = T[k+1][k]);
// reflector j (length n-j-1) is stored conjugated in row j of Vh, columns j+1..n-1.
// LOWER: only the lower triangle of H is read and updated (the rank-2 update
// touches half the entries; the product A v reads each row's lower part and,
// strided, its upper part as the conjugated column), 2 m^2 instead of 3 m^2
// complex multiply-adds per column: the float64 instantiation, whose rate on
// GB300 is 1/64 of float32, takes it.
template <typename R, bool LOWER>
__global__ void __launch_bounds__(256) tridiag_kernel(cx<R>* Hb, long long sH, int n, R* db, cx<R>* eb, int ldde,
                                                       cx<R>* Pb, double* Kb, cx<R>* Vhb, long long sVh) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  cx<R>* H = Hb + z * sH;
  R* d = db + (long long)z * ldde;
  cx<R>* e = eb + (long long)z * ldde;
  cx<R>* P = Pb + (long long)z * ldde;
  double* Kp = Kb + z * 32;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* v = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* w = v + n;
  __shared__ double red[32];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int gw = rank * nw + warp, GW = CS * nw;

  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    if (LOWER) {
      const cx<R>* colj = H + (long long)(j + 1) * n + j;
      for (int t = tid; t < m; t += nth) v[t] = colj[(long long)t * n];   // column j below the diagonal
    } else {
      const cx<R>* rowj = H + (long long)j * n + (j + 1);
      for (int t = tid; t < m; t += nth) v[t] = conj(rowj[t]);   // column j below the diagonal
    }
    __syncthreads();
    const R djj = H[(long long)j * n + j].re;
    const cx<R> alpha = householder(v, m, red);
    if (rank == 0 && tid == 0) {
      d[j] = djj;
      e[j] = alpha;
    }
    // p = A v on own rows; partial of K = v^H p
    double kp = 0;
    for (int t = gw; t < m; t += GW) {
      const cx<R>* row = H + (long long)(j + 1 + t) * n + (j + 1);
      cx<R> acc = mk<R>(0, 0);
      if (LOWER) {
        for (int k = lane; k <= t; k += 32) fma_(acc, row[k], v[k]);
        // upper part of row t: conj(A[k][t]) for k > t, read down column t
        const cx<R>* colt = H + (long long)(j + 1) * n + (j + 1 + t);
        for (int k = t + 1 + lane; k < m; k += 32) fma_(acc, conj(colt[(long long)k * n]), v[k]);
      } else {
        for (int k = lane; k < m; k += 32) fma_(acc, row[k], v[k]);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        P[t] = acc;
        kp += (double)v[t].re * acc.re + (double)v[t].im * acc.im;
      }
    }
    kp = block_sum(kp, red);
    if (tid == 0) Kp[rank] = kp;
    __threadfence();
    cluster.sync();
    double K = 0;
    for (int c = 0; c < CS; ++c) K += Kp[c];
    const R twoK = (R)(2.0 * K);
    for (int t = tid; t < m; t += nth) {
      const cx<R> p = P[t];
      w[t] = mk<R>(2 * p.re - twoK * v[t].re, 2 * p.im - twoK * v[t].im);
    }
    if (rank == 0) {
      cx<R>* rj = Vhb + z * sVh + (long long)j * n + (j + 1);
      for (int t = tid; t < m; t += nth) rj[t] = conj(v[t]);   // reflector j, conjugated, for the back-transform
    }
    __syncthreads();
    for (int t = gw; t < m; t += GW) {
      cx<R>* row = H + (long long)(j + 1 + t) * n + (j + 1);
      const cx<R> vt = v[t], wt = w[t];
      const int kend = LOWER ? t + 1 : m;
      for (int k = lane; k < kend; k += 32) {
        cx<R> a = row[k];
        const cx<R> wk = w[k], vk = v[k];
        // a -= vt conj(wk) + wt conj(vk)
        a.re -= vt.re * wk.re + vt.im * wk.im + wt.re * vk.re + wt.im * vk.im;
        a.im -= vt.im * wk.re - vt.re * wk.im + wt.im * vk.re - wt.re * vk.im;
        row[k] = a;
      }
    }
    __threadfence();
    cluster.sync();
  }
  if (rank == 0 && tid == 0) {
    if (n >= 2) {
      d[n - 2] = H[(long long)(n - 2) * n + (n - 2)].re;
      d[n - 1] = H[(long long)(n - 1) * n + (n - 1)].re;
      e[n - 2] = H[(long long)(n - 1) * n + (n - 2)];
    } else {
      d[0] = H[0].re;
    }
  }
}

// |e_k| and the phases phi (phi_0 = 1, phi_{k+1} = phi_k e_k/|e_k|) that make
// the tridiagonal real: T = D T' D^H with T'_{k+1,k} = |e_k|.  One CTA per
// matrix: each thread multiplies the unit phases of a contiguous chunk, a
// block-wide scan (FP64, fixed order) gives every chunk its prefix.
__device__ __forceinline__ cx<double> shfl_up_cd(cx<double> v, int d) {
  return mk<double>(__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d));
}
__device__ __forceinline__ cx<double> unit_phase(double er, double ei, double* a) {
  const double a2 = er * er + ei * ei;
  *a = sqrt(a2);
  if (!(a2 > 0)) return mk<double>(1.0, 0.0);
  const double inv = 1.0 / *a;
  return mk<double>(er * inv, ei * inv);
}
template <typename R>
__global__ void __launch_bounds__(256) tridiag_phases_kernel(const cx<R>* eb, int n, int ldde, R* eabs,
                                                             cx<R>* phib) {
  __shared__ cx<double> wtot[8];
  const int z = blockIdx.x;
  const cx<R>* e = eb + (long long)z * ldde;
  R* ea = eabs + (long long)z * ldde;
  cx<R>* phi = phib + (long long)z * ldde;
  const int m = n - 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = m > 0 ? (m + 255) / 256 : 0;
  const int k0 = min(m, tid * chunk), k1 = min(m, k0 + chunk);
  cx<double> p = mk<double>(1.0, 0.0);
  for (int k = k0; k < k1; ++k) {
    double a;
    p = p * unit_phase((double)e[k].re, (double)e[k].im, &a);
    ea[k] = (R)a;
  }
  // inclusive scan within the warp, then over the warp totals
  for (int d = 1; d < 32; d <<= 1) {
    const cx<double> t = shfl_up_cd(p, d);
    if (lane >= d) p = t * p;
  }
  if (lane == 31) wtot[wid] = p;
  __syncthreads();
  cx<double> pre = mk<double>(1.0, 0.0);
  for (int w = 0; w < wid; ++w) pre = pre * wtot[w];
  cx<double> excl = shfl_up_cd(p, 1);
  if (lane == 0) excl = mk<double>(1.0, 0.0);
  cx<double> q = pre * excl;
  const double qa = sqrt(q.re * q.re + q.im * q.im);
  q = mk<double>(q.re / qa, q.im / qa);
  if (tid == 0) phi[0] = mk<R>(1, 0);
  for (int k = k0; k < k1; ++k) {
    double a;
    q = q * unit_phase((double)e[k].re, (double)e[k].im, &a);
    phi[k + 1] = mk<R>((R)q.re, (R)q.im);
  }
}

template <typename R>
__device__ __forceinline__ int sturm_count(const R* d, const R* e, int n, R x, R pivmin) {
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < R(0);
  for (int k = 1; k < n; ++k) {
    q = (d[k] - x) - (e[k - 1] * e[k - 1]) / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < R(0);
  }
  return c;
}

// Top r eigenvalues (descending) of the real tridiagonal (d, e): one warp each.
template <typename R>
__global__ void bisect_kernel(const R* db, const R* eb, int n, int r, int ldde, R* lamb, int ldl, int total) {
  const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= total) return;
  const int z = gw / r, t = gw % r;
  const R* d = db + (long long)z * ldde;
  const R* e = eb + (long long)z * ldde;
  R lo = Lim<R>::big(), hi = -Lim<R>::big(), emax = 0;
  for (int k = lane; k < n; k += 32) {
    const R rad = (k > 0 ? e[k - 1] : R(0)) + (k + 1 < n ? e[k] : R(0));
    lo = fmin(lo, d[k] - rad);
    hi = fmax(hi, d[k] + rad);
    if (k + 1 < n) emax = fmax(emax, e[k]);
  }
  for (int m = 16; m > 0; m >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, m));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, m));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, m));
  }
  const R tnorm = fmax(fabs(lo), fabs(hi));
  const R pivmin = Lim<R>::tiny() * fmax(R(1), emax * emax);
  const R eps = Lim<R>::eps();
  lo -= 4 * eps * tnorm + pivmin;
  hi += 4 * eps * tnorm + pivmin;
  const int idx = n - 1 - t;     // ascending index of the wanted eigenvalue
  const R tol = 2 * eps * tnorm + 2 * pivmin;
  for (int it = 0; it < 64 && (hi - lo) > tol; ++it) {
    const R x = lo + (hi - lo) * (R)(lane + 1) / R(33);
    const int cnt = sturm_count(d, e, n, x, pivmin);
    const unsigned mask = __ballot_sync(0xffffffffu, cnt <= idx);
    R nlo = lo, nhi = hi;
    if (mask) {
      const int l = 31 - __clz(mask);
      nlo = __shfl_sync(0xffffffffu, x, l);
      const R xn = __shfl_sync(0xffffffffu, x, (l + 1) & 31);
      if (l < 31) nhi = xn;
    } else {
      nhi = __shfl_sync(0xffffffffu, x, 0);
    }
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) lamb[(long long)z * ldl + t] = R(0.5) * (lo + hi);
}

__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

// Inverse iteration for eigenvalue lam[t] of the real tridiagonal (d, e):
// 3 solves with the partially pivoted LU of (T - lam I); tiny pivots are
// replaced by eps*||T||.  Output column t of Z (n x r, row-major).  The
// factorisation keeps the pivots' reciprocals, so the solves multiply (a
// divide costs several FMAs, dear in float64).  per_warp eigenvalues share a
// warp (the rest of its lanes idle), which spreads the sequential float64
// recurrences over more of the SMs' sub-partitions.
template <typename R>
__global__ void inviter_kernel(const R* db, const R* eb, int n, int r, int ldde, const R* lamb, int ldl, R* Zb,
                               long long sZ, R* Lb, R* U0b, R* U1b, R* U2b, uint8_t* pivb, long long sS, int total,
                               int per_warp) {
  const int wg = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), ln = threadIdx.x & 31;
  if (ln >= per_warp) return;
  const int gid = wg * per_warp + ln;
  if (gid >= total) return;
  const int z = gid / r, t = gid % r;
  const R* d = db + (long long)z * ldde;
  const R* e = eb + (long long)z * ldde;
  const R lam = lamb[(long long)z * ldl + t];
  R* y = Zb + z * sZ;
  R* L = Lb + z * sS;
  R* U0 = U0b + z * sS;
  R* U1 = U1b + z * sS;
  R* U2 = U2b + z * sS;
  uint8_t* piv = pivb + z * sS;
  R tnorm = 0;
  for (int k = 0; k < n; ++k) {
    const R rad = (k > 0 ? e[k - 1] : R(0)) + (k + 1 < n ? e[k] : R(0));
    tnorm = fmax(tnorm, fabs(d[k]) + rad);
  }
  if (tnorm == R(0)) tnorm = R(1);
  const R tiny = Lim<R>::eps() * tnorm;
  // factor
  R diag = d[0] - lam, sup1 = n > 1 ? e[0] : R(0);
  for (int k = 0; k + 1 < n; ++k) {
    const R sub = e[k], nd = d[k + 1] - lam, ns = (k + 2 < n) ? e[k + 1] : R(0);
    const long long o = (long long)k * r + t;
    if (fabs(diag) >= fabs(sub)) {
      const R l = diag != R(0) ? sub / diag : R(0);
      piv[o] = 0; L[o] = l; U0[o] = diag; U1[o] = sup1; U2[o] = 0;
      diag = nd - l * sup1;
      sup1 = ns;
    } else {
      const R l = diag / sub;
      piv[o] = 1; L[o] = l; U0[o] = sub; U1[o] = nd; U2[o] = ns;
      diag = sup1 - l * nd;
      sup1 = -l * ns;
    }
  }
  U0[(long long)(n - 1) * r + t] = diag;
  // pivots -> their reciprocals (tiny pivots replaced first)
  for (int k = 0; k < n; ++k) {
    const long long o = (long long)k * r + t;
    R u0 = U0[o];
    if (fabs(u0) < tiny) u0 = u0 < R(0) ? -tiny : tiny;
    U0[o] = R(1) / u0;
  }
  // start vector
  for (int k = 0; k < n; ++k) {
    // the same start vectors for every batch entry: identical inputs give bitwise identical outputs
    const unsigned long long h = splitmix(((unsigned long long)t << 20) ^ (unsigned long long)k);
    y[(long long)k * r + t] = (R)((double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
  const R big = Lim<R>::big();
  for (int it = 0; it < 3; ++it) {
    for (int k = 0; k + 1 < n; ++k) {
      const long long o = (long long)k * r + t, o1 = o + r;
      R yk = y[o], yk1 = y[o1];
      if (piv[o]) { const R tmp = yk; yk = yk1; yk1 = tmp; y[o] = yk; }
      y[o1] = yk1 - L[o] * yk;
    }
    for (int k = n - 1; k >= 0; --k) {
      const long long o = (long long)k * r + t;
      R acc = y[o];
      if (k + 1 < n) acc -= U1[o] * y[o + r];
      if (k + 2 < n) acc -= U2[o] * y[o + 2 * r];
      R yk = acc * U0[o];
      if (!(fabs(yk) < big)) {
        // rescale everything computed so far and the untouched right-hand side
        const R s = isfinite(yk) ? R(1) / fabs(yk) : R(0);
        for (int i = 0; i < n; ++i) y[(long long)i * r + t] *= s;
        yk = isfinite(yk) ? yk * s : R(1);
      }
      y[o] = yk;
    }
    R mx = 0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, fabs(y[(long long)k * r + t]));
    if (!(mx > R(0))) mx = R(1);
    const R imx = R(1) / mx;
    double s2 = 0;
    for (int k = 0; k < n; ++k) {
      const R v = y[(long long)k * r + t] * imx;
      s2 += (double)v * v;
    }
    const R inv = (R)(1.0 / (sqrt(s2) * (double)mx));
    for (int k = 0; k < n; ++k) y[(long long)k * r + t] *= inv;
  }
}

// S[z] = -sum_i p_i ln p_i, p_i = max(lam_i, 0) / sum_j max(lam_j, 0), over the
// n eigenvalues of a Gram matrix (the squared Schmidt values of a bond,
// App. A.1).  One block per matrix, FP64 sums in a fixed order; rounding can
// leave tiny negative eigenvalues, which count as zero.
template <typename R>
__global__ void __launch_bounds__(256) entropy_kernel(const R* lamb, int n, int ldl, double* S, long long sS) {
  __shared__ double red[8];
  const R* lam = lamb + (long long)blockIdx.x * ldl;
  double t = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += fmax((double)lam[i], 0.0);
  const double tot = block_sum(t, red);
  double h = 0;
  if (tot > 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double p = fmax((double)lam[i], 0.0) / tot;
      if (p > 0) h -= p * log(p);
    }
  h = block_sum(h, red);
  if (threadIdx.x == 0) S[(long long)blockIdx.x * sS] = h;
}

// ---------------------------------------------------------------- double-float reduction
// The complex64 path's float64-quality reduction with its O(n^3) arithmetic on
// the float32 pipes.  Every entry of the trailing matrix is an unevaluated sum
// hi + lo of two floats per component (a "double-float", Dekker 1971; about
// 2^-46 relative): float4 {re_hi, re_lo, im_hi, im_lo}, 16 bytes like a
// complex128.  Products take the exact rounding error of hi*hi from an FMA
// (TwoProduct) plus the hi*lo cross terms; sums carry their exact rounding
// error by Knuth's TwoSum into the lo part (the accumulation of Ogita, Rump
// and Oishi's Dot2), renormalised once per stored entry.  A float64 complex
// multiply-add (4 FMAs at GB300's 1/64 float64 rate) becomes 4 x 12 float32
// operations.  The Householder vector, the norms, K and w are formed in
// float64 (O(m) per column); d, e and the reflectors are written in float64.
// Lower triangle only, as in the float64 kernel.
__device__ __forceinline__ float4 df_from_cd(cx<double> a) {
  const float rh = (float)a.re, ih = (float)a.im;
  return make_float4(rh, (float)(a.re - (double)rh), ih, (float)(a.im - (double)ih));
}
__device__ __forceinline__ double df_to_d(float hi, float lo) { return (double)hi + (double)lo; }
// (hi, lo) += x * y, x = xh + xl, y = yh + yl
__device__ __forceinline__ void df_mac(float& hi, float& lo, float xh, float xl, float yh, float yl) {
  const float ph = __fmul_rn(xh, yh);
  const float pe = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -ph)));
  const float s = __fadd_rn(hi, ph);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
// (hi, lo) += (bh, bl)
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = __fadd_rn(hi, bh);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, bl));
}
__device__ __forceinline__ void df_norm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}
// acc (re, im) += a * v (conj_a: conj(a) * v)
template <bool CONJ_A>
__device__ __forceinline__ void df_cmac(float4& acc, float4 a, float4 v) {
  const float sa = CONJ_A ? -1.f : 1.f;
  df_mac(acc.x, acc.y, a.x, a.y, v.x, v.y);                       // re: a.re v.re
  df_mac(acc.x, acc.y, -sa * a.z, -sa * a.w, v.z, v.w);           //     -/+ a.im v.im
  df_mac(acc.z, acc.w, a.x, a.y, v.z, v.w);                       // im: a.re v.im
  df_mac(acc.z, acc.w, sa * a.z, sa * a.w, v.x, v.y);             //     +/- a.im v.re
  // renormalised every two terms: the lo parts stay small (10x less error over long sums)
  df_norm(acc.x, acc.y);
  df_norm(acc.z, acc.w);
}
__device__ __forceinline__ float4 df_warp_sum(float4 a) {
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, a.x, o), bl = __shfl_xor_sync(0xffffffffu, a.y, o);
    const float ch = __shfl_xor_sync(0xffffffffu, a.z, o), cl = __shfl_xor_sync(0xffffffffu, a.w, o);
    df_add(a.x, a.y, bh, bl);
    df_add(a.z, a.w, ch, cl);
  }
  return a;
}

__global__ void cx_f2df_kernel(const cx<float>* X, long long sX, int n, float4* Y, long long sY) {
  const long long count = (long long)n * n;
  const int z = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const cx<float> v = X[z * sX + i];
    Y[z * sY + i] = make_float4(v.re, 0.f, v.im, 0.f);
  }
}

// (ph, pl) = x * y for double-floats, renormalised
__device__ __forceinline__ float2 df_mul(float xh, float xl, float yh, float yl) {
  const float ph = __fmul_rn(xh, yh);
  const float pl = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -ph)));
  const float s = __fadd_rn(ph, pl);
  return make_float2(s, __fsub_rn(pl, __fsub_rn(s, ph)));
}
// block-wide double-float sum (every thread gets it); red holds 2 x 32 floats
__device__ __forceinline__ float2 df_block_sum(float hi, float lo, float* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o), bl = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, bh, bl);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = hi;
    red[2 * (threadIdx.x >> 5) + 1] = lo;
  }
  __syncthreads();
  float th = 0.f, tl = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(th, tl, red[2 * w], red[2 * w + 1]);
  return make_float2(th, tl);
}

// Every O(m) step of a column is double-float as well (norms, the reflector,
// K, w), so the float64 pipe only sees one thread's pivot per column; the
// reflectors go out rounded to float32 for the float32 back-transformation,
// d and e in float64.
template <int U>
__global__ void __launch_bounds__(512) tridiag_df_kernel(float4* Hb, long long sH, int n, double* db, cx<double>* eb,
                                                          int ldde, float4* Pb, float2* Kb, cx<float>* Vhb,
                                                          long long sVh) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  float4* H = Hb + z * sH;
  double* d = db + (long long)z * ldde;
  cx<double>* e = eb + (long long)z * ldde;
  float4* P = Pb + (long long)z * ldde;
  float2* Kp = Kb + z * 32;
  extern __shared__ __align__(16) unsigned char df_smem[];
  float4* vdf = reinterpret_cast<float4*>(df_smem);   // n: the Householder vector
  float4* wdf = vdf + n;                              // n: w = 2p - 2Kv
  __shared__ float red[64];
  __shared__ float4 alpha_s;
  __shared__ float2 inv_s;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int gw = rank * nw + warp, GW = CS * nw;

  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    // column j below the diagonal, and its squared norm
    float nh = 0.f, nl = 0.f;
    {
      const float4* colj = H + (long long)(j + 1) * n + j;
      for (int t = tid; t < m; t += nth) {
        const float4 a = colj[(long long)t * n];
        vdf[t] = a;
        df_mac(nh, nl, a.x, a.y, a.x, a.y);
        df_mac(nh, nl, a.z, a.w, a.z, a.w);
      }
    }
    const float2 xn2f = df_block_sum(nh, nl, red);
    if (tid == 0) {
      // pivot in float64 on one thread: alpha = -e^{i arg x0} ||x||, un = ||x - alpha e0||
      const float4 x0 = vdf[0];
      const cx<double> x0d = mk<double>(df_to_d(x0.x, x0.y), df_to_d(x0.z, x0.w));
      double pr, pi, ax0;
      unit_phase_of(x0d, &pr, &pi, &ax0);
      const double xn2 = df_to_d(xn2f.x, xn2f.y), xn = sqrt(xn2);
      cx<double> alpha = mk<double>(0, 0);
      double un = 0;
      if (xn > 0) {
        alpha = mk<double>(-xn * pr, -xn * pi);
        un = sqrt(2.0 * xn2 + 2.0 * xn * ax0);
      }
      const double inv = un > 0 ? 1.0 / un : 0.0;
      alpha_s = df_from_cd(alpha);
      const float ih = (float)inv;
      inv_s = make_float2(ih, (float)(inv - (double)ih));
      if (rank == 0) {
        const float4 hjj = H[(long long)j * n + j];
        d[j] = df_to_d(hjj.x, hjj.y);
        e[j] = alpha;
      }
    }
    __syncthreads();
    {
      const float4 al = alpha_s;
      const float2 iv = inv_s;
      cx<float>* rj = Vhb + z * sVh + (long long)j * n + (j + 1);
      for (int t = tid; t < m; t += nth) {
        float4 u = vdf[t];
        if (t == 0) {
          df_add(u.x, u.y, -al.x, -al.y);
          df_add(u.z, u.w, -al.z, -al.w);
        }
        const float2 vr = df_mul(u.x, u.y, iv.x, iv.y), vi = df_mul(u.z, u.w, iv.x, iv.y);
        vdf[t] = make_float4(vr.x, vr.y, vi.x, vi.y);
        if (rank == 0) rj[t] = mk<float>(vr.x, -vi.x);   // reflector j, conjugated, for the back-transform
      }
    }
    __syncthreads();
    // p = A v on own rows (lower part of row t, then its upper part read down column t); K = v^H p
    float kh = 0.f, kl = 0.f;
    for (int t = gw; t < m; t += GW) {
      const float4* row = H + (long long)(j + 1 + t) * n + (j + 1);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), acc2 = acc;
      int k = lane;
      for (; k + 32 * (U - 1) <= t; k += 32 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = row[k + 32 * u];
#pragma unroll
        for (int u = 0; u < U; ++u) df_cmac<false>((u & 1) ? acc2 : acc, a[u], vdf[k + 32 * u]);
      }
      for (; k <= t; k += 32) df_cmac<false>(acc, row[k], vdf[k]);
      const float4* colt = H + (long long)(j + 1) * n + (j + 1 + t);
      k = t + 1 + lane;
      for (; k + 32 * (U - 1) < m; k += 32 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = colt[(long long)(k + 32 * u) * n];
#pragma unroll
        for (int u = 0; u < U; ++u) df_cmac<true>((u & 1) ? acc2 : acc, a[u], vdf[k + 32 * u]);
      }
      for (; k < m; k += 32) df_cmac<true>(acc, colt[(long long)k * n], vdf[k]);
      df_add(acc.x, acc.y, acc2.x, acc2.y);
      df_add(acc.z, acc.w, acc2.z, acc2.w);
      acc = df_warp_sum(acc);
      if (lane == 0) {
        P[t] = acc;
        const float4 vt = vdf[t];
        df_mac(kh, kl, vt.x, vt.y, acc.x, acc.y);
        df_mac(kh, kl, vt.z, vt.w, acc.z, acc.w);
      }
    }
    {
      const float2 kp = df_block_sum(kh, kl, red);
      if (tid == 0) Kp[rank] = kp;
    }
    __threadfence();
    cluster.sync();
    float Kh = 0.f, Kl = 0.f;
    for (int c = 0; c < CS; ++c) df_add(Kh, Kl, Kp[c].x, Kp[c].y);
    // w = 2p - 2 K v  (2K exact in double-float)
    const float K2h = 2.f * Kh, K2l = 2.f * Kl;
    for (int t = tid; t < m; t += nth) {
      const float4 p = P[t], vt = vdf[t];
      float rh = 2.f * p.x, rl = 2.f * p.y, ih = 2.f * p.z, il = 2.f * p.w;
      df_mac(rh, rl, -K2h, -K2l, vt.x, vt.y);
      df_mac(ih, il, -K2h, -K2l, vt.z, vt.w);
      df_norm(rh, rl);
      df_norm(ih, il);
      wdf[t] = make_float4(rh, rl, ih, il);
    }
    __syncthreads();
    // A <- A - v w^H - w v^H on the lower triangle of own rows (U entries in flight per lane)
    for (int t = gw; t < m; t += GW) {
      float4* row = H + (long long)(j + 1 + t) * n + (j + 1);
      const float4 vt = vdf[t], wt = wdf[t];
      for (int k0 = lane; k0 <= t; k0 += 32 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + 32 * u <= t) a[u] = row[k0 + 32 * u];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + 32 * u;
          if (k > t) break;
          const float4 wk = wdf[k], vk = vdf[k];
          float4 b = a[u];
          // re: - (vt.re wk.re + vt.im wk.im + wt.re vk.re + wt.im vk.im)
          df_mac(b.x, b.y, -vt.x, -vt.y, wk.x, wk.y);
          df_mac(b.x, b.y, -vt.z, -vt.w, wk.z, wk.w);
          df_mac(b.x, b.y, -wt.x, -wt.y, vk.x, vk.y);
          df_mac(b.x, b.y, -wt.z, -wt.w, vk.z, vk.w);
          // im: - (vt.im wk.re - vt.re wk.im + wt.im vk.re - wt.re vk.im)
          df_mac(b.z, b.w, -vt.z, -vt.w, wk.x, wk.y);
          df_mac(b.z, b.w, vt.x, vt.y, wk.z, wk.w);
          df_mac(b.z, b.w, -wt.z, -wt.w, vk.x, vk.y);
          df_mac(b.z, b.w, wt.x, wt.y, vk.z, vk.w);
          df_norm(b.x, b.y);
          df_norm(b.z, b.w);
          row[k] = b;
        }
      }
    }
    __threadfence();
    cluster.sync();
  }
  if (rank == 0 && tid == 0) {
    if (n >= 2) {
      const float4 a = H[(long long)(n - 2) * n + (n - 2)], b = H[(long long)(n - 1) * n + (n - 1)];
      const float4 c = H[(long long)(n - 1) * n + (n - 2)];
      d[n - 2] = df_to_d(a.x, a.y);
      d[n - 1] = df_to_d(b.x, b.y);
      e[n - 2] = mk<double>(df_to_d(c.x, c.y), df_to_d(c.z, c.w));
    } else {
      d[0] = df_to_d(H[0].x, H[0].y);
    }
  }
}

// ---------------------------------------------------------------- launchers
template <typename K, typename... Args>
static cudaError_t launch_cluster_t(K kernel, int cs, int batch, int threads, size_t smem, cudaStream_t st,
                                    Args... args) {
  cudaError_t e = ensure_kernel_smem((const void*)kernel, smem, cs > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, batch, 1);
  cfg.blockDim = dim3(threads, 1, 1);
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

template <typename K, typename... Args>
static cudaError_t launch_cluster(K kernel, int cs, int batch, size_t smem, cudaStream_t st, Args... args) {
  return launch_cluster_t(kernel, cs, batch, 256, smem, st, args...);
}

static int cluster_size_for(int n) { return n >= 512 ? 8 : (n >= 128 ? 4 : (n >= 32 ? 2 : 1)); }

// Float64 reductions are bounded by their arithmetic (1/64 of the float32
// rate): each CTA gets an SM of its own (its shared-memory request is raised
// to TRIDIAG64_SMEM, so no two share a float64 pipe) and a matrix takes as
// many CTAs as let eight such clusters (a state's noise levels, over its
// sub-batch streams) run at once: the largest size whose occupancy query
// gives at least 8 active clusters (GB300's GPCs hold only 7 clusters of
// 13-16 single-SM CTAs).  The size depends on nothing but the kernel, so
// results do not depend on how instances are batched.
constexpr size_t TRIDIAG64_SMEM = 120 * 1024;
// double-float reduction launch: 256 threads, TRIDIAG_DF_UNROLL loads in flight per lane in the
// product A v and the rank-2 update (its loads wait on L2: ncu shows long-scoreboard stalls and
// 1.6 % L2 throughput with one load per lane)
constexpr int TRIDIAG_DF_THREADS = 256;
constexpr int TRIDIAG_DF_UNROLL = 4;
static int tridiag64_cluster_size(const void* kernel) {
  static std::mutex mu;
  static std::map<const void*, int> memo;
  std::lock_guard<std::mutex> lk(mu);
  auto it = memo.find(kernel);
  if (it != memo.end()) return it->second;
  int cs = 8;
  for (int c = 16; c > 8; --c) {
    if (ensure_kernel_smem(kernel, TRIDIAG64_SMEM, true) != cudaSuccess) break;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c, 8, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = TRIDIAG64_SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kernel, &cfg) == cudaSuccess && active >= 8) {
      cs = c;
      break;
    }
    (void)cudaGetLastError();
  }
  memo[kernel] = cs;
  return cs;
}

// The L2-resident reduction, one cluster per matrix; float64 reads and
// updates the lower triangle only.
template <typename R>
static cudaError_t tridiag_global(cudaStream_t st, cx<R>* H, long long sH, int n, R* d, cx<R>* e, int ldde, cx<R>* P,
                                  double* Kp, cx<R>* Vh, long long sVh, int batch) {
  constexpr bool lower = std::is_same<R, double>::value;
  const bool wide = lower && n >= 512;
  const int cs = wide ? tridiag64_cluster_size((const void*)tridiag_kernel<R, lower>) : cluster_size_for(n);
  size_t smem = 2 * sizeof(cx<R>) * (size_t)n;
  if (wide) smem = std::max(smem, TRIDIAG64_SMEM);
  ProfScope ps(st, K_TRIDIAG, 1, 16.0 / 3.0 * (double)n * n * n * batch);
  return launch_cluster(tridiag_kernel<R, lower>, cs, batch, smem, st, H, sH, n, d, e, ldde, P, Kp, Vh, sVh);
}

EighWork eigh_workspace(int n, int r) {
  EighWork w;
  const long long qn = std::max(n, r);
  // cx: e, phi, P (n each), Vh (n x n), WY factors (ceil(n/32) x 32 x 32), WY application workspace
  //     (for r columns), QR workspace of an n x r matrix
  w.cx_elems = 3LL * n + (long long)n * n + ((n + 31) / 32) * 1024LL + wy_workspace(r) + qr_workspace(n, r).cx_elems +
               32;
  // re: d, eabs (n each), lam (r), Z (n r), L/U0/U1/U2 (4 n r), Kpart (32 doubles = 64 floats)
  w.re_elems = 2LL * n + r + 5LL * n * r + 64 + qn;
  w.u8_elems = (long long)n * r;
  return w;
}

template <typename R>
cudaError_t eigh_top(cudaStream_t st, cx<R>* H, long long sH, int n, int r, cx<R>* U, long long sU, void* cx_ws,
                     void* re_ws, void* u8_ws, int batch, int* err) {
  (void)err;
  if (batch <= 0) return cudaSuccess;
  const EighWork w = eigh_workspace(n, r);
  cx<R>* cxb = reinterpret_cast<cx<R>*>(cx_ws);
  R* reb = reinterpret_cast<R*>(re_ws);
  uint8_t* u8b = reinterpret_cast<uint8_t*>(u8_ws);
  // per-batch-entry layouts are interleaved by "ld" strides below
  const int ldde = n;
  cx<R>* e = cxb;                                   // batch x n
  cx<R>* phi = e + (long long)batch * n;            // batch x n
  cx<R>* P = phi + (long long)batch * n;            // batch x n
  cx<R>* Vh = P + (long long)batch * n;             // batch x n x n
  cx<R>* Tw = Vh + (long long)batch * n * n;        // batch x nb x 1024
  const int nbw = (n + 31) / 32;
  cx<R>* wyws = Tw + (long long)batch * nbw * 1024;          // batch x wy_workspace(r)
  cx<R>* qrws = wyws + (long long)batch * wy_workspace(r);   // QR workspace for batch n x r matrices
  R* d = reb;                                       // batch x n
  R* eabs = d + (long long)batch * n;               // batch x n
  R* lam = eabs + (long long)batch * n;             // batch x r
  R* Z = lam + (long long)batch * r;                // batch x n r
  R* Ls = Z + (long long)batch * n * r;             // 4 arrays of batch x n r
  R* U0 = Ls + (long long)batch * n * r;
  R* U1 = U0 + (long long)batch * n * r;
  R* U2 = U1 + (long long)batch * n * r;
  double* Kp = reinterpret_cast<double*>(U2 + (long long)batch * n * r + 1);
  Kp = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(Kp) + 15) & ~uintptr_t(15));
  (void)w;
  cudaError_t ce = cudaMemsetAsync(Vh, 0, sizeof(cx<R>) * (size_t)batch * n * n, st);
  if (ce != cudaSuccess) return ce;
  if (smem_cluster_size<R>(n) > 0) {
    ce = tridiag_smem<R>(st, H, sH, n, d, e, ldde, Vh, (long long)n * n, batch);
  } else {
    ce = tridiag_global<R>(st, H, sH, n, d, e, ldde, P, Kp, Vh, (long long)n * n, batch);
  }
  if (ce != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_ELEMWISE);
    tridiag_phases_kernel<R><<<batch, 256, 0, st>>>(e, n, ldde, eabs, phi);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  const int total = batch * r;
  {
    ProfScope ps(st, K_BISECT);
    bisect_kernel<R><<<(total * 32 + 255) / 256, 256, 0, st>>>(d, eabs, n, r, ldde, lam, r, total);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  const long long sS = (long long)n * r;
  {
    ProfScope ps(st, K_INVITER);
    inviter_kernel<R><<<(total + 127) / 128, 128, 0, st>>>(d, eabs, n, r, ldde, lam, r, Z, sS, Ls, U0, U1, U2, u8b,
                                                           sS, total, 32);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  ce = backtransform_wy<R>(st, Vh, (long long)n * n, n, Z, sS, phi, ldde, r, U, sU, Tw, wyws, batch);
  if (ce != cudaSuccess) return ce;
  // orthonormalise the eigenvector block (QR; Q written over U)
  return qr<R>(st, U, sU, n, r, U, sU, nullptr, 0, qrws, batch);
}

// Eigenvalues per warp of the float64 inverse iteration (measured at n = 640,
// 2 x 512 eigenvalues: 32 per warp 2.87 ms, 8 per warp 2.52 ms, 2 per warp 2.78 ms).
constexpr int INVITER64_PER_WARP = 8;

// ---------------------------------------------------------------- mixed precision
// Top r eigenvalues (descending) of the real tridiagonal (d, e) in float64.
// Four lanes per eigenvalue, eight eigenvalues per warp: each round the four
// lanes count at four interior points of the bracket (it shrinks five-fold)
// until it is 4 eps_64 ||T|| wide.  The bracket starts at lamf[t] -/+
// 8 eps_32 ||T|| around the float32 eigenvalue of the rounded tridiagonal
// when Sturm counts confirm that it holds the wanted eigenvalue, else at the
// Gershgorin interval.  The counts use the three-term recurrence of the
// leading principal minors p_k of T - x I (eigenvalues below x = sign changes
// of 1, p_0, ..., p_{n-1}; Sturm): three float64 operations per step and no
// divide, where the quotient form q_k = p_k / p_{k-1} costs a float64 divide,
// several FMAs at GB300's 1/64 float64 rate.  T is scaled by a power of two
// (exactly) to norm <= 1, so |p_k| grows at most 3x per step and a pair
// (p_{k-1}, p_k) is rescaled by a power of two when its larger exponent
// leaves [-600, 600]; a minor that is zero (or underflows) is replaced by
// -2^-1000 p_{k-1}, the quotient form's -pivmin convention.
constexpr int BIS64_THREADS = 64;   // 16 eigenvalues per block: blocks spread over the SMs

__device__ __forceinline__ int sturm_minors(const double* ds, const double* b, int n, double x) {
  double p0 = 1.0, p1 = ds[0] - x;
  if (((__double2hiint(p1) & 0x7fffffff) | __double2loint(p1)) == 0) p1 = -0x1p-1000;
  int c = __double2hiint(p1) < 0;
  for (int k = 1; k < n; ++k) {
    double p = fma(-b[k - 1], p0, (ds[k] - x) * p1);
    if (((__double2hiint(p) & 0x7fffffff) | __double2loint(p)) == 0) p = -0x1p-1000 * p1;
    c += (__double2hiint(p) ^ __double2hiint(p1)) < 0;
    p0 = p1;
    p1 = p;
    const int em = max((__double2hiint(p1) >> 20) & 0x7ff, (__double2hiint(p0) >> 20) & 0x7ff);
    if (em > 1023 + 600 || em < 1023 - 600) {
      const double sc = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em)
      p0 *= sc;
      p1 *= sc;
    }
  }
  return c;
}

__global__ void __launch_bounds__(BIS64_THREADS) bisect64_kernel(const double* db, const double* eb, int n, int r,
                                                                 int ldde, const float* lamfb, double* lamb, int ldl) {
  extern __shared__ double bis_smem[];
  double* ds = bis_smem;        // n: d scaled
  double* bs = bis_smem + n;    // n: e^2 scaled
  __shared__ double red[2][BIS64_THREADS / 32];
  __shared__ int sexp;
  const int z = blockIdx.y, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double* d = db + (long long)z * ldde;
  const double* e = eb + (long long)z * ldde;
  // Gershgorin interval and the power-of-two scale
  double glo = 1e300, ghi = -1e300;
  for (int k = tid; k < n; k += BIS64_THREADS) {
    const double rad = (k > 0 ? e[k - 1] : 0.0) + (k + 1 < n ? e[k] : 0.0);
    glo = fmin(glo, d[k] - rad);
    ghi = fmax(ghi, d[k] + rad);
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  if (lane == 0) {
    red[0][wid] = glo;
    red[1][wid] = ghi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < BIS64_THREADS / 32; ++w) {
      red[0][0] = fmin(red[0][0], red[0][w]);
      red[1][0] = fmax(red[1][0], red[1][w]);
    }
    const double tn = fmax(fabs(red[0][0]), fabs(red[1][0]));
    sexp = tn > 0 ? ((__double2hiint(tn) >> 20) & 0x7ff) - 1023 + 1 : 0;   // tn < 2^sexp
  }
  __syncthreads();
  const double sc = __hiloint2double((1023 - sexp) << 20, 0);   // 2^-sexp
  for (int k = tid; k < n; k += BIS64_THREADS) {
    ds[k] = d[k] * sc;
    const double es = k + 1 < n ? e[k] * sc : 0.0;
    bs[k] = es * es;
  }
  glo = red[0][0] * sc;
  ghi = red[1][0] * sc;
  __syncthreads();
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double tol = 4 * DBL_EPSILON * tnorm + 0x1p-1000;
  glo -= 4 * DBL_EPSILON * tnorm;
  ghi += 4 * DBL_EPSILON * tnorm;
  const int g = lane >> 2, sub = lane & 3;
  const int t = blockIdx.x * (BIS64_THREADS / 4) + wid * 8 + g;
  const bool live = t < r;
  const int idx = n - 1 - (live ? t : 0);
  double lo = glo, hi = ghi;
  {
    // the float32 bracket, checked by two lanes of the group
    const double lf = live ? (double)lamfb[(long long)z * ldl + t] * sc : 0.0;
    const double w = 8.0 * (double)FLT_EPSILON * tnorm;
    const double x = sub == 0 ? lf - w : lf + w;
    const int cnt = sub < 2 ? sturm_minors(ds, bs, n, x) : 0;
    const int c0 = __shfl_sync(0xffffffffu, cnt, lane & ~3), c1 = __shfl_sync(0xffffffffu, cnt, (lane & ~3) + 1);
    if (c0 <= idx && c1 > idx) {
      lo = lf - w;
      hi = lf + w;
    }
  }
  for (int it = 0; it < 40; ++it) {
    const bool open = live && (hi - lo) > tol;
    if (!__any_sync(0xffffffffu, open)) break;
    const double x = lo + (hi - lo) * ((double)(sub + 1) / 5.0);
    const int cnt = open ? sturm_minors(ds, bs, n, x) : 0;
    const unsigned m = __ballot_sync(0xffffffffu, cnt <= idx);
    const int K = __popc((m >> (lane & ~3)) & 0xfu);   // points at or below the eigenvalue (a prefix)
    if (open) {
      const double nlo = K > 0 ? lo + (hi - lo) * ((double)K / 5.0) : lo;
      const double nhi = K < 4 ? lo + (hi - lo) * ((double)(K + 1) / 5.0) : hi;
      lo = nlo;
      hi = nhi;
    }
  }
  if (live && sub == 0) lamb[(long long)z * ldl + t] = 0.5 * (lo + hi) / sc;
}

__global__ void re_d2f_pair_kernel(const double* a, const double* b, float* fa, float* fb, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    fa[i] = (float)a[i];
    fb[i] = (float)b[i];
  }
}

__global__ void cx_f2d_kernel(const cx<float>* X, long long sX, int rows, int cols, int ldx, cx<double>* Y,
                              long long sY) {
  const long long count = (long long)rows * cols;
  const int z = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const cx<float> v = X[z * sX + (i / cols) * ldx + i % cols];
    Y[z * sY + i] = mk<double>(v.re, v.im);
  }
}

__global__ void cx_d2f_kernel(const cx<double>* X, cx<float>* Y, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    Y[i] = mk<float>((float)X[i].re, (float)X[i].im);
}

__global__ void re_d2f_kernel(const double* X, float* Y, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    Y[i] = (float)X[i];
}

static inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

MixedEighWork eigh_mixed_workspace(int n, int r) {
  // per matrix; every array is batch-major, so a batch of b matrices needs b times these bytes
  MixedEighWork w;
  const size_t nn = (size_t)n * n, nr = (size_t)n * r;
  const int nbw = (n + 31) / 32;
  w.cx_bytes = al256(16 * nn) * 2 + al256(16 * (size_t)n) * 3 + al256(8 * nn) + al256(8 * (size_t)n) +
               al256(8 * (size_t)nbw * 1024) + al256(8 * (size_t)wy_workspace(r)) +
               al256(8 * (size_t)qr_workspace(n, r).cx_elems) + 1024;
  w.re_bytes = al256(8 * (size_t)n) * 2 + al256(8 * (size_t)r) + al256(8 * nr) * 5 + al256(4 * nr) + 512 +
               al256(4 * (size_t)n) * 2 + al256(4 * (size_t)r) + 1024;
  w.u8_bytes = al256(nr) + 256;
  return w;
}

// Top-r eigenvectors of the complex64 Hermitian H[z] (n x n, ld n), written to
// U[z] (n x r, ld r, columns by decreasing eigenvalue, orthonormal).  The
// Householder reduction, the eigenvalues (bisection) and the eigenvectors of
// the tridiagonal (inverse iteration) run in float64; the back-transformation
// through the reflectors and the final orthonormalisation run in float32.  A
// float32 reduction has a backward error of eps_32 ||H||, which turns the
// eigenvectors next to the truncation cut by eps_32 ||H|| / gap there (about
// 0.1 on saturated chi = 512 states); in float64 that error is below the
// rounding of the input, and the float32 back-transformation only adds
// eps_32-sized, gap-independent errors.
cudaError_t eigh_top_mixed(cudaStream_t st, cx<float>* H, long long sH, int n, int r, cx<float>* U, long long sU,
                           void* cx_ws, void* re_ws, void* u8_ws, int batch, int* err) {
  (void)err;
  if (batch <= 0) return cudaSuccess;
  const size_t nn = (size_t)n * n, nr = (size_t)n * r;
  const int nbw = (n + 31) / 32;
  const size_t B = (size_t)batch;
  unsigned char* c = reinterpret_cast<unsigned char*>(cx_ws);
  auto take = [&](unsigned char*& base, size_t bytes) {
    unsigned char* p = base;
    base += al256(bytes);
    return p;
  };
  cx<double>* Hd = reinterpret_cast<cx<double>*>(take(c, 16 * nn * B));
  cx<double>* Vhd = reinterpret_cast<cx<double>*>(take(c, 16 * nn * B));
  cx<double>* ed = reinterpret_cast<cx<double>*>(take(c, 16 * (size_t)n * B));
  cx<double>* phid = reinterpret_cast<cx<double>*>(take(c, 16 * (size_t)n * B));
  cx<double>* Pd = reinterpret_cast<cx<double>*>(take(c, 16 * (size_t)n * B));
  cx<float>* Vhf = reinterpret_cast<cx<float>*>(take(c, 8 * nn * B));
  cx<float>* phif = reinterpret_cast<cx<float>*>(take(c, 8 * (size_t)n * B));
  cx<float>* Tw = reinterpret_cast<cx<float>*>(take(c, 8 * (size_t)nbw * 1024 * B));
  cx<float>* wyws = reinterpret_cast<cx<float>*>(take(c, 8 * (size_t)wy_workspace(r) * B));
  cx<float>* qrws = reinterpret_cast<cx<float>*>(take(c, 8 * (size_t)qr_workspace(n, r).cx_elems * B));
  unsigned char* q = reinterpret_cast<unsigned char*>(re_ws);
  double* dd = reinterpret_cast<double*>(take(q, 8 * (size_t)n * B));
  double* eabs = reinterpret_cast<double*>(take(q, 8 * (size_t)n * B));
  double* lam = reinterpret_cast<double*>(take(q, 8 * (size_t)r * B));
  double* Z = reinterpret_cast<double*>(take(q, 8 * nr * B));
  double* Ls = reinterpret_cast<double*>(take(q, 8 * nr * B));
  double* U0 = reinterpret_cast<double*>(take(q, 8 * nr * B));
  double* U1 = reinterpret_cast<double*>(take(q, 8 * nr * B));
  double* U2 = reinterpret_cast<double*>(take(q, 8 * nr * B));
  float* Zf = reinterpret_cast<float*>(take(q, 4 * nr * B));
  double* Kp = reinterpret_cast<double*>(take(q, 8 * 32 * B));
  float* df = reinterpret_cast<float*>(take(q, 4 * (size_t)n * B));
  float* ef = reinterpret_cast<float*>(take(q, 4 * (size_t)n * B));
  float* lamf = reinterpret_cast<float*>(take(q, 4 * (size_t)r * B));
  uint8_t* piv = reinterpret_cast<uint8_t*>(u8_ws);
  cudaError_t ce;
  const bool in_smem = smem_cluster_size<double>(n) > 0;
  {
    ProfScope ps(st, K_ELEMWISE);
    const dim3 grid((unsigned)std::min<size_t>((nn + 255) / 256, 1024), batch);
    if (in_smem)
      cx_f2d_kernel<<<grid, 256, 0, st>>>(H, sH, n, n, n, Hd, (long long)nn);
    else
      cx_f2df_kernel<<<grid, 256, 0, st>>>(H, sH, n, reinterpret_cast<float4*>(Hd), (long long)nn);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  if (in_smem) {
    if ((ce = cudaMemsetAsync(Vhd, 0, 16 * nn * B, st)) != cudaSuccess) return ce;
  } else {
    if ((ce = cudaMemsetAsync(Vhf, 0, 8 * nn * B, st)) != cudaSuccess) return ce;
  }
  if (in_smem) {
    ce = tridiag_smem<double>(st, Hd, (long long)nn, n, dd, ed, n, Vhd, (long long)nn, batch);
  } else {
    // double-float reduction: float64 quality on the float32 pipes; writes the
    // float32 reflectors directly
    const int cs = tridiag64_cluster_size((const void*)tridiag_df_kernel<TRIDIAG_DF_UNROLL>);
    const size_t smem = std::max<size_t>(32 * (size_t)n, TRIDIAG64_SMEM);
    ProfScope ps(st, K_TRIDIAG, 1, 16.0 / 3.0 * (double)n * n * n * batch);
    ce = launch_cluster_t(tridiag_df_kernel<TRIDIAG_DF_UNROLL>, cs, batch, TRIDIAG_DF_THREADS, smem, st,
                          reinterpret_cast<float4*>(Hd), (long long)nn, n, dd, ed, n, reinterpret_cast<float4*>(Pd),
                          reinterpret_cast<float2*>(Kp), Vhf, (long long)nn);
  }
  if (ce != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_ELEMWISE);
    tridiag_phases_kernel<double><<<batch, 256, 0, st>>>(ed, n, n, eabs, phid);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  const int total = batch * r;
  {
    // float32 multisection of the rounded tridiagonal brackets every eigenvalue
    // to about eps_32 ||T||; float64 bisection narrows the brackets
    ProfScope ps(st, K_BISECT);
    re_d2f_pair_kernel<<<64, 256, 0, st>>>(dd, eabs, df, ef, (long long)n * batch);
    bisect_kernel<float><<<(total * 32 + 255) / 256, 256, 0, st>>>(df, ef, n, r, n, lamf, r, total);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_BISECT64);
    const dim3 grid((r + BIS64_THREADS / 4 - 1) / (BIS64_THREADS / 4), batch);
    const size_t bsm = 2 * sizeof(double) * (size_t)n;
    if ((ce = ensure_kernel_smem((const void*)bisect64_kernel, bsm, false)) != cudaSuccess) return ce;
    bisect64_kernel<<<grid, BIS64_THREADS, bsm, st>>>(dd, eabs, n, r, n, lamf, lam, r);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_INVITER);
    const int pw = INVITER64_PER_WARP;
    const int warps = (total + pw - 1) / pw;
    inviter_kernel<double><<<(warps + 3) / 4, 128, 0, st>>>(dd, eabs, n, r, n, lam, r, Z, (long long)nr, Ls, U0, U1, U2,
                                                            piv, (long long)nr, total, pw);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_ELEMWISE);
    if (in_smem) cx_d2f_kernel<<<1024, 256, 0, st>>>(Vhd, Vhf, (long long)(nn * B));
    cx_d2f_kernel<<<64, 256, 0, st>>>(phid, phif, (long long)(n * B));
    re_d2f_kernel<<<1024, 256, 0, st>>>(Z, Zf, (long long)(nr * B));
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  ce = backtransform_wy<float>(st, Vhf, (long long)nn, n, Zf, (long long)nr, phif, n, r, U, sU, Tw, wyws, batch);
  if (ce != cudaSuccess) return ce;
  return qr<float>(st, U, sU, n, r, U, sU, nullptr, 0, qrws, batch);
}

template <typename R>
cudaError_t gram_entropy(cudaStream_t st, cx<R>* H, long long sH, int n, void* cx_ws, void* re_ws, int batch,
                         double* S, long long sS) {
  if (batch <= 0) return cudaSuccess;
  if (n <= 1) return cudaMemset2DAsync(S, sizeof(double) * sS, 0, sizeof(double), batch, st);
  cx<R>* e = reinterpret_cast<cx<R>*>(cx_ws);       // batch x n
  cx<R>* phi = e + (long long)batch * n;            // batch x n
  cx<R>* P = phi + (long long)batch * n;            // batch x n
  cx<R>* Vh = P + (long long)batch * n;             // batch x n x n
  R* d = reinterpret_cast<R*>(re_ws);               // batch x n
  R* eabs = d + (long long)batch * n;               // batch x n
  R* lam = eabs + (long long)batch * n;             // batch x n
  double* Kp = reinterpret_cast<double*>(lam + (long long)batch * n + 1);
  Kp = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(Kp) + 15) & ~uintptr_t(15));
  cudaError_t ce = cudaMemsetAsync(Vh, 0, sizeof(cx<R>) * (size_t)batch * n * n, st);
  if (ce != cudaSuccess) return ce;
  if (smem_cluster_size<R>(n) > 0) {
    ce = tridiag_smem<R>(st, H, sH, n, d, e, n, Vh, (long long)n * n, batch);
  } else {
    ce = tridiag_global<R>(st, H, sH, n, d, e, n, P, Kp, Vh, (long long)n * n, batch);
  }
  if (ce != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_ELEMWISE);
    tridiag_phases_kernel<R><<<batch, 256, 0, st>>>(e, n, n, eabs, phi);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  const int total = batch * n;
  {
    ProfScope ps(st, K_BISECT);
    bisect_kernel<R><<<(total * 32 + 255) / 256, 256, 0, st>>>(d, eabs, n, n, n, lam, n, total);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return ce;
  {
    ProfScope ps(st, K_ELEMWISE);
    entropy_kernel<R><<<batch, 256, 0, st>>>(lam, n, n, S, sS);
  }
  return cudaGetLastError();
}

#define NNE_INST_LINALG(R)                                                                                       \
  template cudaError_t eigh_top<R>(cudaStream_t, cx<R>*, long long, int, int, cx<R>*, long long, void*, void*, \
                                   void*, int, int*);                                                       \
  template cudaError_t gram_entropy<R>(cudaStream_t, cx<R>*, long long, int, void*, void*, int, double*, long long);
NNE_INST_LINALG(float)
NNE_INST_LINALG(double)

}  // namespace nne
