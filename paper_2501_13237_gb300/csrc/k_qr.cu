// Blocked Householder QR for tall complex matrices (m x n, row-major).
//
// Panels of 32 columns are factored by one thread-block cluster per matrix:
// the panel rows are spread over the cluster's CTAs (cyclically) and kept in
// shared memory; per column the cluster exchanges one round of partial sums
// through distributed shared memory.  Each panel also yields the compact-WY
// factor T (P_0 ... P_{b-1} = I - V T V^H).  Trailing updates and the explicit Q then apply each panel's
// block reflector (wy_apply).  All reductions are in a fixed order (deterministic).
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nne {

constexpr int QB = 32;   // panel width
constexpr int PS = QB + 1;   // padded row stride of the shared-memory panel (avoids bank conflicts)

constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_CS_MAX = 16;

// a - v * w, evaluated the same way wherever it is used (the owner of a row
// and every CTA predicting that row's next pivot must agree bit for bit)
template <typename R>
__device__ __forceinline__ cx<R> hh_upd(cx<R> a, cx<R> v, cx<R> w) {
  return mk<R>(fma(-v.re, w.re, fma(v.im, w.im, a.re)), fma(-v.re, w.im, fma(-v.im, w.re, a.im)));
}

// One round's contribution of a CTA to the cluster-wide sums.
template <typename R>
struct QrMsg {
  cx<R> w[QB];   // c < j: v_c^H v_j ; c > j: v_j^H a_c (partials over own rows)
  cx<R> ex[3];   // a_j[j+1] (owner of row j), v_{j+1} and a_{j+1}[j+1] (owner of row j+1); 0 elsewhere
  double nrm;    // partial squared norm of the next pivot column
};

// Factor the panel A[pb:m, pb:pb+bw] (bw <= 32) of matrix z = blockIdx.y.
// Column j takes one cluster barrier: every CTA pushes its partial sums into
// every CTA's shared memory, then all sum them in rank order.  The squared
// norm of column j+1 below row j is downdated from the same round (the
// reflector is unitary on rows >= j: ||a'_{j+1}||^2 over rows > j equals the
// pre-update norm over rows >= j minus |a'_j[j+1]|^2); when that cancels
// more than half of it, an extra round recomputes it.  The compact-WY factor
// T is built column by column from the v_c^H v_j of the same rounds.
template <typename R>
__global__ void __launch_bounds__(QR_THREADS) qr_panel_kernel(cx<R>* Ab, long long sA, int lda, int m, int pb, int bw,
                                                               cx<R>* Vb, long long sV, int ldv, cx<R>* Tb,
                                                               long long sT, int maxloc, int zr) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  cx<R>* A = Ab + z * sA;
  cx<R>* V = Vb + z * sV;
  cx<R>* T = Tb + z * sT;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* P = reinterpret_cast<cx<R>*>(smem_raw);       // [maxloc][PS]
  __shared__ QrMsg<R> msg[2][QR_CS_MAX];
  __shared__ cx<R> red[QR_WARPS][QB];
  __shared__ double redn[QR_WARPS];
  __shared__ cx<R> wfull[QB];
  __shared__ cx<R> gcol[QB];
  __shared__ cx<R> alphas[QB];
  __shared__ cx<R> Ts[QB][QB + 1];
  __shared__ cx<R> ex_s[3];
  __shared__ double nrm_s;
  __shared__ cx<R> x0_s;
  __shared__ double xn2_s;
  __shared__ int recompute_s;
  __shared__ cx<R> alpha_s;
  __shared__ R inv_s, tau_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int mp = m - pb;                                   // panel rows
  const int nloc = mp > rank ? (mp - rank + CS - 1) / CS : 0;
  for (int e = tid; e < nloc * QB; e += QR_THREADS) {
    const int li = e / QB, c = e % QB;
    const long long gi = pb + rank + (long long)li * CS;
    P[li * PS + c] = c < bw ? A[gi * lda + pb + c] : mk<R>(0, 0);
  }
  for (int e = tid; e < QB * QB; e += QR_THREADS) Ts[e / QB][e % QB] = mk<R>(0, 0);
  // every CTA of the cluster is running before anyone writes into its shared memory
  cluster.sync();
  int round = 0;
  // first local row whose panel row index is >= p
  auto first_local = [&](int p) { return p > rank ? (p - rank + CS - 1) / CS : 0; };
  // reflector of the next column from x0_s, xn2_s (one thread; FP64 is slow on this part)
  auto pivot = [&]() {
    const double xn2 = xn2_s;
    const cx<R> x0 = x0_s;
    double pr, pi, ax0;
    unit_phase_of(x0, &pr, &pi, &ax0);
    const double xn = sqrt(xn2);
    cx<R> alpha = mk<R>(0, 0);
    double un = 0;
    if (xn > 0) {
      alpha = mk<R>((R)(-xn * pr), (R)(-xn * pi));
      un = sqrt(2.0 * xn2 + 2.0 * xn * ax0);
    }
    alpha_s = alpha;
    inv_s = un > 0 ? (R)(1.0 / un) : R(0);
    tau_s = un > 0 ? R(2) : R(0);
  };
  // cluster-wide squared norm of column c over panel rows >= p (one round)
  auto norm_round = [&](int c, int p, bool with_x0) {
    const int l0 = first_local(p);
    R sacc = 0;
    for (int li = l0 + tid; li < nloc; li += QR_THREADS) sacc += norm2(P[li * PS + c]);
    sacc = warp_sum_r(sacc);
    if (lane == 0) redn[wid] = (double)sacc;
    __syncthreads();
    const int buf = round & 1;
    if (tid < CS) {
      double t = 0;
      for (int w = 0; w < QR_WARPS; ++w) t += redn[w];
      QrMsg<R>* dst = cluster.map_shared_rank(&msg[buf][rank], tid);
      dst->nrm = t;
      cx<R> x0 = mk<R>(0, 0);
      if (with_x0 && c < mp && rank == c % CS) x0 = P[(c / CS) * PS + c];
      dst->ex[2] = x0;
    }
    cluster.sync();
    if (tid == 0) {
      double t = 0;
      cx<R> x0 = mk<R>(0, 0);
      for (int src = 0; src < CS; ++src) {
        t += msg[buf][src].nrm;
        x0 = x0 + msg[buf][src].ex[2];
      }
      xn2_s = t;
      if (with_x0) x0_s = x0;
      pivot();
    }
    ++round;
    __syncthreads();
  };
  norm_round(0, 0, true);
  for (int j = 0; j < bw; ++j) {
    const int lstart = first_local(j);
    const cx<R> x0 = x0_s;
    const cx<R> alpha = alpha_s;
    const R inv = inv_s, tau = tau_s;
    if (tid == 0) alphas[j] = alpha;
    const int owner = j % CS, ljo = j / CS;
    // v = (x - alpha e_j) / un on own rows
    for (int li = lstart + tid; li < nloc; li += QR_THREADS) {
      cx<R> u = P[li * PS + j];
      if (rank == owner && li == ljo) u = u - alpha;
      P[li * PS + j] = inv * u;
    }
    __syncthreads();
    const bool has_next = j + 1 < bw;
    // partials: lane c holds v_c^H v_j (c < j) or v_j^H a_c (c > j); lane j+1 also |a_{j+1}|^2
    {
      const int c = lane;
      cx<R> acc = mk<R>(0, 0);
      R nacc = 0;
      if (c < j) {
        for (int li = lstart + wid; li < nloc; li += QR_WARPS) fmac_(acc, P[li * PS + c], P[li * PS + j]);
      } else if (c > j && c < bw) {
        for (int li = lstart + wid; li < nloc; li += QR_WARPS) {
          const cx<R> a = P[li * PS + c];
          fmac_(acc, P[li * PS + j], a);
          if (c == j + 1) nacc += norm2(a);
        }
      }
      red[wid][c] = acc;
      if (c == j + 1) redn[wid] = (double)nacc;
    }
    __syncthreads();
    const int buf = round & 1;
    if (tid < QB) {
      cx<R> t = mk<R>(0, 0);
      for (int w = 0; w < QR_WARPS; ++w) t = t + red[w][tid];
      for (int d = 0; d < CS; ++d) cluster.map_shared_rank(&msg[buf][rank], d)->w[tid] = t;
    } else if (tid == QB) {
      double nt = 0;
      if (has_next)
        for (int w = 0; w < QR_WARPS; ++w) nt += redn[w];
      cx<R> e0 = mk<R>(0, 0), e1 = mk<R>(0, 0), e2 = mk<R>(0, 0);
      if (has_next) {
        if (rank == owner) e0 = P[ljo * PS + j + 1];
        if (j + 1 < mp && rank == (j + 1) % CS) {
          const int l1 = (j + 1) / CS;
          e1 = P[l1 * PS + j];
          e2 = P[l1 * PS + j + 1];
        }
      }
      for (int d = 0; d < CS; ++d) {
        QrMsg<R>* dst = cluster.map_shared_rank(&msg[buf][rank], d);
        dst->ex[0] = e0;
        dst->ex[1] = e1;
        dst->ex[2] = e2;
        dst->nrm = nt;
      }
    }
    cluster.sync();
    ++round;
    if (tid < QB) {
      cx<R> t = mk<R>(0, 0);
      for (int src = 0; src < CS; ++src) t = t + msg[buf][src].w[tid];
      if (tid > j) wfull[tid] = mk<R>(2 * t.re, 2 * t.im);
      else wfull[tid] = mk<R>(0, 0);
      gcol[tid] = tid < j ? t : mk<R>(0, 0);
    } else if (tid == QB) {
      double nt = 0;
      cx<R> e0 = mk<R>(0, 0), e1 = mk<R>(0, 0), e2 = mk<R>(0, 0);
      for (int src = 0; src < CS; ++src) {
        nt += msg[buf][src].nrm;
        e0 = e0 + msg[buf][src].ex[0];
        e1 = e1 + msg[buf][src].ex[1];
        e2 = e2 + msg[buf][src].ex[2];
      }
      nrm_s = nt;
      ex_s[0] = e0;
      ex_s[1] = e1;
      ex_s[2] = e2;
    }
    __syncthreads();
    // T[0:j, j] = -tau_j T[0:j, 0:j] (V^H v_j), T[j][j] = tau_j (rank 0, last warp)
    if (rank == 0 && wid == QR_WARPS - 1) {
      cx<R> acc = mk<R>(0, 0);
      if (lane < j)
        for (int l = lane; l < j; ++l) fma_(acc, Ts[lane][l], gcol[l]);
      if (lane < j) Ts[lane][j] = mk<R>(-tau * acc.re, -tau * acc.im);
      if (lane == j) Ts[j][j] = mk<R>(tau, 0);
    }
    // a_c <- a_c - v (2 v^H a_c), c in (j, bw), own rows >= j
    if (has_next)
      for (int e = tid; e < (nloc - lstart) * QB; e += QR_THREADS) {
        const int li = lstart + e / QB, c = e % QB;
        if (c > j && c < bw) P[li * PS + c] = hh_upd(P[li * PS + c], P[li * PS + j], wfull[c]);
      }
    if (tid == 0 && has_next) {
      const cx<R> vj = inv * (x0 - alpha);                      // the owner's v_j, same operations
      const cx<R> ajn = hh_upd(ex_s[0], vj, wfull[j + 1]);      // a'_j[j+1]
      const cx<R> x0n = j + 1 < mp ? hh_upd(ex_s[2], ex_s[1], wfull[j + 1]) : mk<R>(0, 0);
      const double nA = nrm_s;
      const double xn2n = nA - (double)norm2(ajn);
      x0_s = x0n;
      xn2_s = xn2n > 0 ? xn2n : 0.0;
      recompute_s = !(xn2n > 0.5 * nA);
      if (!recompute_s) pivot();
    }
    __syncthreads();
    if (has_next && recompute_s) norm_round(j + 1, j + 1, false);
  }
  // write back V and the R part of A
  for (int e = tid; e < nloc * QB; e += QR_THREADS) {
    const int li = e / QB, c = e % QB;
    if (c >= bw) continue;
    const int pi = rank + li * CS;
    const long long gi = pb + pi;
    const cx<R> val = P[li * PS + c];
    V[gi * ldv + pb + c] = pi >= c ? val : mk<R>(0, 0);
    A[gi * lda + pb + c] = pi < c ? val : (pi == c ? alphas[c] : mk<R>(0, 0));
  }
  if (rank == 0) {
    for (int e = tid; e < QB * QB; e += QR_THREADS) T[e] = Ts[e / QB][e % QB];
    // rows of the outer block above this panel: zero in its reflector columns
    for (int e = tid; e < zr * QB; e += QR_THREADS)
      if (e % QB < bw) V[(long long)(pb - zr + e / QB) * ldv + pb + e % QB] = mk<R>(0, 0);
  }
}

// Shared-memory state of one register-resident panel factorisation.  Norm
// sums are kept in the state's precision R: the downdate below cancels at
// most half of a norm before an exact recompute, which bounds its relative
// error at a few units of R.
template <typename R>
struct PanelMsg {
  cx<R> w[QB];   // c < j: v_c^H v_j ; c > j: v_j^H a_c (partials over own rows)
  cx<R> ex[3];   // a_j[j+1] (owner of row j), v_{j+1} and a_{j+1}[j+1] (owner of row j+1); 0 elsewhere
  R nrm;         // partial squared norm of the next pivot column
};
template <typename R>
struct PanelShared {
  PanelMsg<R> msg[2][QR_CS_MAX];
  cx<R> red[QR_WARPS][QB];
  R redn[QR_WARPS];
  cx<R> wfull[QB];
  cx<R> gcol[QB];
  cx<R> alphas[QB];
  cx<R> Ts[QB][QB + 1];
  cx<R> ex_loc[3];
  cx<R> ex_s[3];
  R nrm_s;
  cx<R> x0_s;
  R xn2_s;
  int recompute_s;
  cx<R> alpha_s;
  R inv_s, tau_s;
};

// Reflector pivot from the squared norm xn2 of the column at and below the
// diagonal and its diagonal entry x0: alpha = -e^{i arg x0} ||x||,
// un = ||x - alpha e_0||, tau = 2 (0 for a zero column).  Evaluated in R,
// the phase of x0 by unit_phase_of.
template <typename R>
__device__ __forceinline__ void hh_pivot(R xn2, cx<R> x0, cx<R>* alpha, R* inv, R* tau) {
  R pr, pi, ax0;
  unit_phase_of(x0, &pr, &pi, &ax0);
  const R xn = sqrt(xn2);
  cx<R> a = mk<R>(0, 0);
  R un = 0;
  if (xn > R(0)) {
    a = mk<R>(-xn * pr, -xn * pi);
    un = sqrt(R(2) * xn2 + R(2) * xn * ax0);
  }
  *alpha = a;
  *inv = un > R(0) ? R(1) / un : R(0);
  *tau = un > R(0) ? R(2) : R(0);
}

// One cluster round: the squared norm of a column over the panel rows from
// a given row down (sacc: this thread's partial, meaningful on lane c), and
// with with_x0 the column's diagonal entry (x0_mine, held by the thread
// holds_x0); tid 0 then forms the reflector pivot.
template <typename R>
__device__ __forceinline__ void panel_norm_round(R sacc, cx<R> x0_mine, bool holds_x0, PanelShared<R>& sh,
                                                 cg::cluster_group& cluster, int CS, int rank, int c, bool with_x0,
                                                 bool x0_here, int& round) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (lane == c) sh.redn[wid] = sacc;
  if (with_x0 && holds_x0) sh.ex_loc[2] = x0_mine;
  __syncthreads();
  const int buf = round & 1;
  if (tid < CS) {
    R t0 = 0, t1 = 0;
    for (int w = 0; w < QR_WARPS; w += 2) {
      t0 += sh.redn[w];
      t1 += sh.redn[w + 1];
    }
    PanelMsg<R>* dst = cluster.map_shared_rank(&sh.msg[buf][rank], tid);
    dst->nrm = t0 + t1;
    dst->ex[2] = (with_x0 && x0_here) ? sh.ex_loc[2] : mk<R>(0, 0);
  }
  cluster.sync();
  if (tid == 0) {
    R t = 0;
    cx<R> x0 = mk<R>(0, 0);
    for (int src = 0; src < CS; ++src) {
      t += sh.msg[buf][src].nrm;
      x0 = x0 + sh.msg[buf][src].ex[2];
    }
    sh.xn2_s = t;
    if (with_x0) sh.x0_s = x0;
    cx<R> al;
    R iv, ta;
    hh_pivot<R>(sh.xn2_s, sh.x0_s, &al, &iv, &ta);
    sh.alpha_s = al;
    sh.inv_s = iv;
    sh.tau_s = ta;
  }
  ++round;
  __syncthreads();
}

// Register-resident panel factorisation (same arithmetic per column as a
// plain Householder QR): warp w of a CTA holds its local rows w, w + 16, ...
// (at most RPW of them), lane c holds column c, so the reflector entry of a
// row is a shuffle from lane j and no shared-memory traffic touches the
// panel.  Rows are dealt to the CTAs of the cluster cyclically.  Column j
// takes one cluster round: every CTA pushes its partial sums into every
// CTA's shared memory, then all sum them in rank order.  The squared norm of
// column j+1 below row j is downdated in the same round (the reflector is
// unitary on rows >= j); when that cancels more than half of it an extra
// round recomputes it.  T is built column by column from the v_c^H v_j of
// the same rounds.
template <typename R, int RPW>
__global__ void __launch_bounds__(QR_THREADS) qr_panel_reg_kernel(cx<R>* Ab, long long sA, int lda, int m, int pb,
                                                                   int bw, cx<R>* Vb, long long sV, int ldv,
                                                                   cx<R>* Tb, long long sT, int zr) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.y;
  cx<R>* A = Ab + z * sA;
  cx<R>* V = Vb + z * sV;
  cx<R>* T = Tb + z * sT;
  __shared__ PanelShared<R> sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int mp = m - pb;
  const int nloc = mp > rank ? (mp - rank + CS - 1) / CS : 0;
  // this warp's live registers: k < kmax (local row wid + 16 k < nloc)
  const int kmax = nloc > wid ? (nloc - wid + QR_WARPS - 1) / QR_WARPS : 0;
  cx<R> a[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int li = wid + QR_WARPS * k;
    a[k] = mk<R>(0, 0);
    if (li < nloc && lane < bw) a[k] = A[(long long)(pb + rank + li * CS) * lda + pb + lane];
  }
  for (int e = tid; e < QB * QB; e += QR_THREADS) sh.Ts[e / QB][e % QB] = mk<R>(0, 0);
  // every CTA of the cluster is running before anyone writes into its shared memory
  cluster.sync();
  int round = 0;
  {
    // column 0 over all rows, and its entry in row 0 (rank 0, warp 0, register 0, lane 0)
    R sacc = 0;
#pragma unroll
    for (int k = 0; k < RPW; ++k)
      if (k < kmax) sacc += norm2(a[k]);
    panel_norm_round<R>(sacc, a[0], rank == 0 && wid == 0 && lane == 0, sh, cluster, CS, rank, 0, true, rank == 0,
                        round);
  }
  for (int j = 0; j < bw; ++j) {
    const cx<R> x0 = sh.x0_s;
    const cx<R> alpha = sh.alpha_s;
    const R inv = sh.inv_s, tau = sh.tau_s;
    if (tid == 0) sh.alphas[j] = alpha;
    const int owner = j % CS;
    const bool has_next = j + 1 < bw;
    // registers k >= kmin of this warp hold rows >= j: local row li >= first local row >= j
    const int l0 = j > rank ? (j - rank + CS - 1) / CS : 0;
    const int kmin = l0 > wid ? (l0 - wid + QR_WARPS - 1) / QR_WARPS : 0;
    // row of register k: rank + (wid + 16 k) CS; rows j and j+1, if here, sit at these registers
    const int dj = j - rank - wid * CS, dj1 = j + 1 - rank - wid * CS;
    const int kj = (dj >= 0 && dj % (QR_WARPS * CS) == 0) ? dj / (QR_WARPS * CS) : -1;
    const int kj1 = (dj1 >= 0 && dj1 % (QR_WARPS * CS) == 0 && j + 1 < mp) ? dj1 / (QR_WARPS * CS) : -1;
    // v = (x - alpha e_j) / un (every lane forms it from lane j's entry; lane j keeps it);
    // partials: lane c < j: v_c^H v_j; lane c > j: v_j^H a_c; lane j+1 also |a_{j+1}|^2;
    // and the pre-update entries every CTA needs for the next pivot
    // branch-free: every lane accumulates conj(x) v; lanes c > j want v^H a_c = conj of that
    cx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
    R nacc = 0;
    cx<R> e_a = mk<R>(0, 0), e_b = mk<R>(0, 0);
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      if (k >= kmin && k < kmax) {
        cx<R> u = shfl_idx(a[k], j);
        if (k == kj) u = u - alpha;
        const cx<R> v = inv * u;
        if (lane == j) a[k] = v;
        const cx<R> x = a[k];
        if (k & 1) fmac_(acc1, x, v); else fmac_(acc0, x, v);
        nacc += norm2(x);
        if (k == kj) e_a = x;                       // row j: lane j+1 holds a_j[j+1]
        if (k == kj1) e_b = lane == j ? v : x;      // row j+1: lane j -> v_{j+1}, lane j+1 -> a_{j+1}[j+1]
      }
    }
    {
      const cx<R> acc = acc0 + acc1;
      sh.red[wid][lane] = lane > j ? conj(acc) : acc;
    }
    if (lane == j + 1) sh.redn[wid] = nacc;
    if (has_next) {
      if (kj >= 0 && lane == j + 1) sh.ex_loc[0] = e_a;
      if (kj1 >= 0 && lane == j) sh.ex_loc[1] = e_b;
      if (kj1 >= 0 && lane == j + 1) sh.ex_loc[2] = e_b;
    }
    __syncthreads();
    const int buf = round & 1;
    if (tid < QB) {
      cx<R> t0 = mk<R>(0, 0), t1 = t0, t2 = t0, t3 = t0;
      for (int w = 0; w < QR_WARPS; w += 4) {
        t0 = t0 + sh.red[w][tid];
        t1 = t1 + sh.red[w + 1][tid];
        t2 = t2 + sh.red[w + 2][tid];
        t3 = t3 + sh.red[w + 3][tid];
      }
      const cx<R> t = (t0 + t1) + (t2 + t3);
      for (int d = 0; d < CS; ++d) cluster.map_shared_rank(&sh.msg[buf][rank], d)->w[tid] = t;
    } else if (tid == QB) {
      R nt = 0;
      cx<R> e0 = mk<R>(0, 0), e1 = mk<R>(0, 0), e2 = mk<R>(0, 0);
      if (has_next) {
        R n0 = 0, n1 = 0;
        for (int w = 0; w < QR_WARPS; w += 2) {
          n0 += sh.redn[w];
          n1 += sh.redn[w + 1];
        }
        nt = n0 + n1;
        if (rank == owner) e0 = sh.ex_loc[0];
        if (j + 1 < mp && rank == (j + 1) % CS) {
          e1 = sh.ex_loc[1];
          e2 = sh.ex_loc[2];
        }
      }
      for (int d = 0; d < CS; ++d) {
        PanelMsg<R>* dst = cluster.map_shared_rank(&sh.msg[buf][rank], d);
        dst->ex[0] = e0;
        dst->ex[1] = e1;
        dst->ex[2] = e2;
        dst->nrm = nt;
      }
    }
    cluster.sync();
    ++round;
    if (tid < QB) {
      cx<R> t0 = mk<R>(0, 0), t1 = t0;
      int src = 0;
      for (; src + 1 < CS; src += 2) {
        t0 = t0 + sh.msg[buf][src].w[tid];
        t1 = t1 + sh.msg[buf][src + 1].w[tid];
      }
      if (src < CS) t0 = t0 + sh.msg[buf][src].w[tid];
      const cx<R> t = t0 + t1;
      sh.wfull[tid] = tid > j ? mk<R>(2 * t.re, 2 * t.im) : mk<R>(0, 0);
      sh.gcol[tid] = tid < j ? t : mk<R>(0, 0);
    } else if (tid == QB) {
      R nt = 0;
      cx<R> e0 = mk<R>(0, 0), e1 = mk<R>(0, 0), e2 = mk<R>(0, 0);
      for (int src = 0; src < CS; ++src) {
        nt += sh.msg[buf][src].nrm;
        e0 = e0 + sh.msg[buf][src].ex[0];
        e1 = e1 + sh.msg[buf][src].ex[1];
        e2 = e2 + sh.msg[buf][src].ex[2];
      }
      sh.nrm_s = nt;
      sh.ex_s[0] = e0;
      sh.ex_s[1] = e1;
      sh.ex_s[2] = e2;
    }
    __syncthreads();
    // T[0:j, j] = -tau_j T[0:j, 0:j] (V^H v_j), T[j][j] = tau_j (rank 0, last warp)
    if (rank == 0 && wid == QR_WARPS - 1) {
      cx<R> ta0 = mk<R>(0, 0), ta1 = ta0;
      if (lane < j) {
        int l = lane;
        for (; l + 1 < j; l += 2) {
          fma_(ta0, sh.Ts[lane][l], sh.gcol[l]);
          fma_(ta1, sh.Ts[lane][l + 1], sh.gcol[l + 1]);
        }
        if (l < j) fma_(ta0, sh.Ts[lane][l], sh.gcol[l]);
        const cx<R> ta = ta0 + ta1;
        sh.Ts[lane][j] = mk<R>(-tau * ta.re, -tau * ta.im);
      }
      if (lane == j) sh.Ts[j][j] = mk<R>(tau, 0);
    }
    // a_c <- a_c - v (2 v^H a_c), c in (j, bw), own rows >= j
    if (has_next) {
      const cx<R> wf = sh.wfull[lane];
      const bool upd = lane > j && lane < bw;
#pragma unroll
      for (int k = 0; k < RPW; ++k)
        if (k >= kmin && k < kmax) {
          const cx<R> v = shfl_idx(a[k], j);
          if (upd) a[k] = hh_upd(a[k], v, wf);
        }
    }
    if (tid == 0 && has_next) {
      const cx<R> vj = inv * (x0 - alpha);                      // the owner's v_j, same operations
      const cx<R> ajn = hh_upd(sh.ex_s[0], vj, sh.wfull[j + 1]);      // a'_j[j+1]
      const cx<R> x0n = j + 1 < mp ? hh_upd(sh.ex_s[2], sh.ex_s[1], sh.wfull[j + 1]) : mk<R>(0, 0);
      const R nA = sh.nrm_s;
      const R xn2n = nA - norm2(ajn);
      sh.x0_s = x0n;
      sh.xn2_s = xn2n > R(0) ? xn2n : R(0);
      sh.recompute_s = !(xn2n > R(0.5) * nA);
      if (!sh.recompute_s) {
        cx<R> al;
        R iv, ta;
        hh_pivot<R>(sh.xn2_s, x0n, &al, &iv, &ta);
        sh.alpha_s = al;
        sh.inv_s = iv;
        sh.tau_s = ta;
      }
    }
    __syncthreads();
    if (has_next && sh.recompute_s) {
      // column j+1 over rows >= j+1
      const int l1 = j + 1 > rank ? (j + 1 - rank + CS - 1) / CS : 0;
      const int kmin1 = l1 > wid ? (l1 - wid + QR_WARPS - 1) / QR_WARPS : 0;
      R sacc = 0;
#pragma unroll
      for (int k = 0; k < RPW; ++k)
        if (k >= kmin1 && k < kmax) sacc += norm2(a[k]);
      panel_norm_round<R>(sacc, mk<R>(0, 0), false, sh, cluster, CS, rank, j + 1, false, false, round);
    }
  }
  // write back V and the R part of A
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int li = wid + QR_WARPS * k;
    if (li < nloc && lane < bw) {
      const int pi = rank + li * CS;
      const long long gi = pb + pi;
      V[gi * ldv + pb + lane] = pi >= lane ? a[k] : mk<R>(0, 0);
      A[gi * lda + pb + lane] = pi < lane ? a[k] : (pi == lane ? sh.alphas[lane] : mk<R>(0, 0));
    }
  }
  if (rank == 0) {
    for (int e = tid; e < QB * QB; e += QR_THREADS) T[e] = sh.Ts[e / QB][e % QB];
    // rows of the outer block above this panel: zero in its reflector columns
    for (int e = tid; e < zr * QB; e += QR_THREADS)
      if (e % QB < bw) V[(long long)(pb - zr + e / QB) * ldv + pb + e % QB] = mk<R>(0, 0);
  }
}

constexpr int QNB = 128;   // outer block: 4 panels applied to the trailing matrix together

// Compact-WY factor of an outer block of np_in <= 4 panels from the panels'
// factors T_a (32 x 32, upper) and the Gram G = V^H V of the block's
// reflectors (nbw x nbw): the product of the panels' block reflectors is
// I - V T V^H with T upper triangular, T_aa = T_a and, block column by block
// column, T[0:a, a] = -T[0:a, 0:a] G[0:a, a] T_a.  One CTA per matrix;
// writes T (QNB x QNB, zero outside nbw x nbw).
template <typename R>
__global__ void __launch_bounds__(256) wy_merge_t_kernel(const cx<R>* Tpb, long long sTp, const cx<R>* Gb, long long sG,
                                                         int nbw, cx<R>* Tob, long long sTo) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* X = reinterpret_cast<cx<R>*>(smem_raw);   // [(QNB - QB)][QB + 1]
  const int z = blockIdx.x, tid = threadIdx.x;
  const cx<R>* Tp = Tpb + z * sTp;
  const cx<R>* G = Gb + z * sG;
  cx<R>* T = Tob + z * sTo;
  const int np_in = (nbw + QB - 1) / QB;
  for (int e = tid; e < QNB * QNB; e += 256) {
    const int r = e / QNB, c = e % QNB;
    const int a = r / QB, b = c / QB;
    T[e] = (a == b && a < np_in) ? Tp[(long long)a * QB * QB + (r % QB) * QB + (c % QB)] : mk<R>(0, 0);
  }
  __syncthreads();
  for (int b = 1; b < np_in; ++b) {
    const int rows = b * QB, c0 = b * QB;
    // X = T[0:rows, 0:rows] G[0:rows, c0:c0+32]   (T upper triangular)
    for (int e = tid; e < rows * QB; e += 256) {
      const int r = e / QB, c = e % QB;
      cx<R> acc = mk<R>(0, 0);
      if (c0 + c < nbw)
        for (int l = r; l < rows; ++l) fma_(acc, T[(long long)r * QNB + l], G[(long long)l * nbw + c0 + c]);
      X[r * (QB + 1) + c] = acc;
    }
    __syncthreads();
    // T[0:rows, c0:c0+32] = -X T_b   (T_b upper triangular)
    for (int e = tid; e < rows * QB; e += 256) {
      const int r = e / QB, c = e % QB;
      cx<R> acc = mk<R>(0, 0);
      for (int l = 0; l <= c; ++l) fma_(acc, X[r * (QB + 1) + l], T[(long long)(c0 + l) * QNB + c0 + c]);
      T[(long long)r * QNB + c0 + c] = mk<R>(-acc.re, -acc.im);
    }
    __syncthreads();
  }
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
  cudaError_t e = ensure_kernel_smem((const void*)kernel, smem, cs > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, batch, 1);
  cfg.blockDim = dim3(QR_THREADS, 1, 1);
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
  const int nblk = (k + QNB - 1) / QNB;
  // V (m x n) + panel T (np x 32 x 32) + WY application workspace (n columns)
  // + block T (nblk x 128 x 128) + Gram (128 x 128) + W1, W2 (128 x n each)
  w.cx_elems = (long long)m * n + (long long)np * QB * QB + wy_workspace(n) + (long long)nblk * QNB * QNB +
               (long long)QNB * QNB + 2LL * QNB * n + 64;
  return w;
}

// Factor the panel A[pb:m, pb:pb+bw] of every matrix (V, its T at Tp); zr rows
// above pb belong to the same outer block and get zeros in V's panel columns.
template <typename R>
static cudaError_t panel_factor(cudaStream_t st, cx<R>* A, long long sA, int m, int n, int pb, int bw, cx<R>* V,
                                long long sV, cx<R>* Tp, long long sT, int zr, int batch) {
  const int mp = m - pb;
  // panel flops: per column j, reflector products and update of the bw-1-j columns to its right
  // and the v_c^H v_j of the j columns to its left, over mp - j rows (8 real flops per complex MAC)
  double work = 0;
  for (int j = 0; j < bw; ++j) work += 8.0 * (double)(mp - j) * (2.0 * (bw - 1 - j) + j + 1);
  ProfScope ps(st, K_QR_FACTOR, 1, work * batch);
  // register-resident panel when every CTA's rows fit 16 warps x 16 registers
  int csr = mp >= 512 ? 8 : (mp >= 128 ? 4 : (mp >= 32 ? 2 : 1));
  if ((mp + csr - 1) / csr > 16 * QR_WARPS) csr = 16;
  const int nl = (mp + csr - 1) / csr;
  if (nl <= 1 * QR_WARPS)
    return launch_cluster_qr(qr_panel_reg_kernel<R, 1>, csr, batch, 0, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT, zr);
  if (nl <= 2 * QR_WARPS)
    return launch_cluster_qr(qr_panel_reg_kernel<R, 2>, csr, batch, 0, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT, zr);
  if (nl <= 4 * QR_WARPS)
    return launch_cluster_qr(qr_panel_reg_kernel<R, 4>, csr, batch, 0, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT, zr);
  if (nl <= 8 * QR_WARPS)
    return launch_cluster_qr(qr_panel_reg_kernel<R, 8>, csr, batch, 0, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT, zr);
  if (nl <= 16 * QR_WARPS)
    return launch_cluster_qr(qr_panel_reg_kernel<R, 16>, csr, batch, 0, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT,
                             zr);
  int cs = mp >= 512 ? 8 : (mp >= 128 ? 4 : (mp >= 32 ? 2 : 1));
  int maxloc = (mp + cs - 1) / cs;
  size_t smem = sizeof(cx<R>) * (size_t)maxloc * PS;
  if (smem > 160 * 1024) {
    cs = 16;
    maxloc = (mp + cs - 1) / cs;
    smem = sizeof(cx<R>) * (size_t)maxloc * PS;
  }
  return launch_cluster_qr(qr_panel_kernel<R>, cs, batch, smem, st, A, sA, n, m, pb, bw, V, sV, n, Tp, sT, maxloc, zr);
}

// Blocked Householder QR.  Outer blocks of 128 columns: their four 32-column
// panels are factored and applied to the rest of the block one at a time
// (wy_apply); the block's reflectors are then merged into one compact-WY
// factor (Gram V^H V and wy_merge_t) and applied to the trailing columns, and
// later to Q, with three GEMMs each (tensor cores for complex64).
template <typename R>
cudaError_t qr(cudaStream_t st, cx<R>* A, long long sA, int m, int n, cx<R>* Q, long long sQ, cx<R>* Rout,
               long long sR, void* cx_ws, int batch) {
  const int k = std::min(m, n);
  if (k <= 0 || batch <= 0) return cudaSuccess;
  const int np = (k + QB - 1) / QB, nblk = (k + QNB - 1) / QNB;
  cx<R>* V = reinterpret_cast<cx<R>*>(cx_ws);
  const long long sV = (long long)m * n;
  cx<R>* T = V + sV * batch;
  const long long sT = (long long)np * QB * QB;
  cx<R>* wyws = T + sT * batch;
  cx<R>* Tb = wyws + wy_workspace(n) * batch;
  const long long sTb = (long long)nblk * QNB * QNB;
  cx<R>* G = Tb + sTb * batch;
  const long long sG = (long long)QNB * QNB;
  cx<R>* W1 = G + sG * batch;
  const long long sW = (long long)QNB * n;
  cx<R>* W2 = W1 + sW * batch;
  const cx<R> one = mk<R>(1, 0), zero = mk<R>(0, 0), mone = mk<R>(-1, 0);
  const size_t merge_smem = sizeof(cx<R>) * (QNB - QB) * (QB + 1);
  cudaError_t e;
  if ((e = ensure_kernel_smem((const void*)wy_merge_t_kernel<R>, merge_smem, false)) != cudaSuccess) return e;
  for (int b = 0; b < nblk; ++b) {
    const int b0 = b * QNB, bend = std::min(k, b0 + QNB), nbw = bend - b0, mpb = m - b0;
    for (int pb = b0; pb < bend; pb += QB) {
      const int bw = std::min(QB, bend - pb), mp = m - pb, p = pb / QB;
      if ((e = panel_factor<R>(st, A, sA, m, n, pb, bw, V, sV, T + p * QB * QB, sT, pb - b0, batch)) != cudaSuccess)
        return e;
      const int nt_in = bend - pb - bw;
      if (nt_in > 0) {
        // rest of the block: A_t <- (I - V T V^H)^H A_t
        cx<R>* Vp = V + (long long)pb * n + pb;
        cx<R>* At = A + (long long)pb * n + pb + bw;
        if ((e = wy_apply<R>(st, false, Vp, sV, n, T + p * QB * QB, sT, QB, true, bw, mp, nt_in, At, sA, n, wyws,
                             batch)) != cudaSuccess)
          return e;
      }
    }
    // block factor: G = V_b^H V_b, then T_b
    cx<R>* Vb = V + (long long)b0 * n + b0;
    if ((e = cgemm<R>(st, OP_C, OP_N, nbw, nbw, mpb, one, Vb, sV, n, Vb, sV, n, zero, G, sG, nbw, batch)) !=
        cudaSuccess)
      return e;
    {
      ProfScope ps(st, K_WY);
      wy_merge_t_kernel<R><<<batch, 256, merge_smem, st>>>(T + (b0 / QB) * QB * QB, sT, G, sG, nbw,
                                                           Tb + (long long)b * QNB * QNB, sTb);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int ntr = n - bend;
    if (ntr > 0) {
      // trailing columns: C <- (I - V_b T_b V_b^H)^H C
      cx<R>* Ct = A + (long long)b0 * n + bend;
      cx<R>* Tbb = Tb + (long long)b * QNB * QNB;
      if ((e = cgemm<R>(st, OP_C, OP_N, nbw, ntr, mpb, one, Vb, sV, n, Ct, sA, n, zero, W1, sW, ntr, batch)) !=
          cudaSuccess)
        return e;
      if ((e = cgemm<R>(st, OP_C, OP_N, nbw, ntr, nbw, one, Tbb, sTb, QNB, W1, sW, ntr, zero, W2, sW, ntr, batch)) !=
          cudaSuccess)
        return e;
      if ((e = cgemm<R>(st, OP_N, OP_N, mpb, ntr, nbw, mone, Vb, sV, n, W2, sW, ntr, one, Ct, sA, n, batch)) !=
          cudaSuccess)
        return e;
    }
  }
  if (Rout) {
    ProfScope ps(st, K_ELEMWISE);
    qr_extract_r2_kernel<R><<<dim3(64, batch), 256, 0, st>>>(A, sA, n, k, n, Rout, sR);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = identity<R>(st, Q, sQ, m, k, batch)) != cudaSuccess) return e;
  for (int b = nblk - 1; b >= 0; --b) {
    const int b0 = b * QNB, nbw = std::min(k, b0 + QNB) - b0, mpb = m - b0, kc = k - b0;
    cx<R>* Vb = V + (long long)b0 * n + b0;
    cx<R>* Qb = Q + (long long)b0 * k + b0;
    cx<R>* Tbb = Tb + (long long)b * QNB * QNB;
    // Q_b <- (I - V_b T_b V_b^H) Q_b
    if ((e = cgemm<R>(st, OP_C, OP_N, nbw, kc, mpb, one, Vb, sV, n, Qb, sQ, k, zero, W1, sW, kc, batch)) !=
        cudaSuccess)
      return e;
    if ((e = cgemm<R>(st, OP_N, OP_N, nbw, kc, nbw, one, Tbb, sTb, QNB, W1, sW, kc, zero, W2, sW, kc, batch)) !=
        cudaSuccess)
      return e;
    if ((e = cgemm<R>(st, OP_N, OP_N, mpb, kc, nbw, mone, Vb, sV, n, W2, sW, kc, one, Qb, sQ, k, batch)) !=
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
