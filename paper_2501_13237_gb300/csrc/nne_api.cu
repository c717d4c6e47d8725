// C ABI of libnne: contexts, states, and the host-side orchestration of the
// gate step (theta formation, superoperator, truncation, normalisation,
// centre moves), the expectation sweep and the extrapolation fit.  Every
// arithmetic step runs in the kernels of k_*.cu; this file only sizes
// buffers, tracks bond dimensions and enqueues launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.cuh"

namespace nne {

static thread_local std::string g_last_error;

nne_status set_error(nne_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

nne_status set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  return set_error(e == cudaErrorMemoryAllocation ? NNE_ERR_OOM : NNE_ERR_CUDA, "%s failed: %s (%s:%d)", what,
                   cudaGetErrorString(e), file, line);
}

}  // namespace nne

using namespace nne;

struct ScratchF64 {
  double* p = nullptr;
  size_t n = 0;
};

struct nne_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t used = 0;
  ScratchF64 snoise;   // superoperator-build scratch, grown on demand
  ~nne_ctx() {
    if (snoise.p) {
      cudaFreeAsync(snoise.p, stream);
      cudaStreamSynchronize(stream);
    }
  }
};

namespace nne {
void ctx_device_stream(const nne_ctx* ctx, int* device, cudaStream_t* stream) {
  *device = ctx->device;
  *stream = ctx->stream;
}
}  // namespace nne

namespace {

struct DevAlloc {
  nne_ctx* ctx = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
  nne_status alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->budget && ctx->used + bytes > ctx->budget)
      return set_error(NNE_ERR_OOM, "HBM budget exceeded: %zu + %zu > %zu bytes", ctx->used, bytes, ctx->budget);
    // stream-ordered: no device-wide synchronisation, so states on other streams keep running
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    ctx->used += bytes;
    blocks.push_back({*p, bytes});
    return NNE_OK;
  }
  void release() {
    for (auto& b : blocks) {
      cudaFreeAsync(b.first, ctx->stream);
      ctx->used -= b.second;
    }
    blocks.clear();
  }
};

constexpr int PARTS = 64;   // partial sums per instance for Frobenius norms

ScratchF64& scratch_snoise(nne_ctx* ctx, int n_inst) {
  const size_t need = 512 * (size_t)n_inst;
  if (ctx->snoise.n < need) {
    if (ctx->snoise.p) cudaFreeAsync(ctx->snoise.p, ctx->stream);
    ctx->snoise.p = nullptr;
    ctx->snoise.n = 0;
    if (cudaMallocAsync(&ctx->snoise.p, need * sizeof(double), ctx->stream) == cudaSuccess) ctx->snoise.n = need;
    else ctx->snoise.p = nullptr;
  }
  return ctx->snoise;
}

}  // namespace

namespace nne {
// Bond capacities min(chi, 4^k, 4^(n-k)), k = 0..n.
std::vector<int> bond_caps(int n, int chi) {
  std::vector<int> cap(n + 1, 1);
  for (int k = 1; k < n; ++k) {
    long long c = chi;
    long long p = 1;
    for (int i = 0; i < k && p < c; ++i) p *= 4;
    c = std::min(c, p);
    p = 1;
    for (int i = 0; i < n - k && p < c; ++i) p *= 4;
    c = std::min(c, p);
    cap[k] = (int)c;
  }
  return cap;
}

static size_t round256(size_t b) { return ((b == 0 ? 16 : b) + 255) & ~size_t(255); }

// Eigensolver workspace per instance in elements of the state's precision
// (complex, real, bytes): the float path's needs, and for complex64 states
// also those of the mixed-precision path (float64 arrays carved from the same
// blocks), each rounded to 256 bytes so every instance's block stays aligned.
EighWork eigh_workspace_state(int n, int r, int dtype) {
  EighWork w = eigh_workspace(n, r);
  if (dtype == NNE_C64) {
    const MixedEighWork m = eigh_mixed_workspace(n, r);
    w.cx_elems = std::max<long long>(w.cx_elems, (long long)((m.cx_bytes + 4096 + 7) / 8));
    w.re_elems = std::max<long long>(w.re_elems, (long long)((m.re_bytes + 4096 + 3) / 4));
    w.u8_elems = std::max<long long>(w.u8_elems, (long long)(m.u8_bytes + 256));
  }
  const long long cq = 256 / (dtype == NNE_C64 ? 8 : 16), rq = 256 / (dtype == NNE_C64 ? 4 : 8);
  w.cx_elems = (w.cx_elems + cq - 1) / cq * cq;
  w.re_elems = (w.re_elems + rq - 1) / rq * rq;
  w.u8_elems = (w.u8_elems + 255) / 256 * 256;
  return w;
}

// Device bytes nne_create_state (and nne_set_sketch, when sketch_cols > 0)
// allocate for these arguments: the same blocks, rounded the same way.
size_t state_bytes(int n, int chi, int n_inst, int dtype, int sketch_rows, int sketch_cols) {
  const std::vector<int> cap = bond_caps(n, chi);
  int dmax = 1;
  for (int c : cap) dmax = std::max(dmax, c);
  const size_t esz = dtype == NNE_C64 ? 8 : 16;
  size_t total = 0;
  size_t arena = 0;
  for (int k = 0; k < n; ++k) {
    arena += (size_t)cap[k] * 4 * cap[k + 1] * n_inst * esz;
    arena = (arena + 255) & ~size_t(255);
  }
  total += round256(arena);
  total += round256(sizeof(double) * (3 * (size_t)n_inst + 3 * (size_t)n_inst * PARTS) + 64);
  const long long D = dmax, N4 = 4 * D;
  total += round256((size_t)(N4 * N4) * n_inst * esz) * 3;     // X, H, T
  total += round256((size_t)(N4 * D) * n_inst * esz);          // U
  total += round256((size_t)std::max(N4 * D, D * D) * n_inst * esz);
  const EighWork ew = eigh_workspace_state((int)N4, (int)D, dtype);
  total += round256((size_t)ew.cx_elems * n_inst * esz);
  total += round256((size_t)ew.re_elems * n_inst * (esz / 2) + 256);
  total += round256((size_t)ew.u8_elems * n_inst);
  total += round256((size_t)qr_workspace((int)N4, (int)N4).cx_elems * n_inst * esz);
  total += round256(n);
  total += round256(sizeof(int) * (n + 1)) + round256(sizeof(void*) * n) + round256(sizeof(long long) * n);
  total += round256(sizeof(double) * 2 * 2 * (size_t)(n + 1) * D * n_inst);
  total += round256(sizeof(double) * 2 * (size_t)(n + 1) * n_inst);
  if (sketch_cols > 0) {
    total += round256((size_t)sketch_rows * sketch_cols * esz);
    total += round256((size_t)(N4 * sketch_cols) * n_inst * esz) * 2;
    total += round256((size_t)sketch_cols * sketch_cols * n_inst * esz);
    total += round256((size_t)sketch_cols * D * n_inst * esz);
  }
  return total;
}
}  // namespace nne

struct nne_state {
  nne_ctx* ctx = nullptr;
  int n = 0, chi = 0, n_inst = 0;
  nne_dtype dtype = NNE_C64;
  nne_trunc trunc = NNE_TRUNC_EXACT;
  size_t esz = 8;
  std::vector<int> dims, cap;
  int centre = 0;
  int dmax = 1;
  std::vector<char*> site;           // instance 0 of site k
  std::vector<long long> sstride;    // elements between instances of site k
  DevAlloc mem;
  double* d_lognorm = nullptr;
  double* d_logfid = nullptr;
  double* d_scale = nullptr;
  double* d_parts = nullptr;   // 2 x n_inst x PARTS
  int* d_err = nullptr;
  // workspaces (per instance stride in elements)
  void* X = nullptr;  long long sX = 0;
  void* H = nullptr;  long long sH = 0;
  void* U = nullptr;  long long sU = 0;
  void* T = nullptr;  long long sT = 0;   // centre-move scratch
  void* Rm = nullptr; long long sR = 0;
  void* eig_cx = nullptr;
  void* eig_re = nullptr;
  void* eig_u8 = nullptr;
  void* qr_ws = nullptr;
  long long eig_cx_pi = 0, eig_re_pi = 0, eig_u8_pi = 0, qr_pi = 0;   // elements per instance
  // concurrent sub-batches of the gate steps: each on its own stream
  int nsub = 1;
  std::vector<cudaStream_t> sub_st;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  // sweep
  int* d_dims = nullptr;
  void** d_site = nullptr;
  long long* d_stride = nullptr;
  double* d_env = nullptr;
  double* d_envscale = nullptr;
  std::vector<uint8_t> bits;
  uint8_t* d_bits = nullptr;
  // randomized truncation
  void* d_omega = nullptr;
  int omega_rows = 0, omega_cols = 0, power_iters = 0;
  void* rs_Y = nullptr; void* rs_Z = nullptr; void* rs_C = nullptr; void* rs_W = nullptr;
  long long rs_sY = 0, rs_sZ = 0, rs_sC = 0, rs_sW = 0;
};

namespace {

// Sub-batches a new state splits its instances into (nne_set_option).
int g_substreams = 4;
// When set, nne_apply_layer runs every state's instances as one batch on the
// context stream (nne_set_option NNE_OPT_SERIAL_LAYERS).
int g_serial_layers = 0;
// complex64 eigenproblems with a float64 reduction and tridiagonal solve (NNE_OPT_EIG_FP64).
int g_eig_fp64 = 1;

void destroy_streams(nne_state* s) {
  for (cudaStream_t q : s->sub_st) cudaStreamDestroy(q);
  for (cudaEvent_t ev : s->ev_join) cudaEventDestroy(ev);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  s->sub_st.clear();
  s->ev_join.clear();
  s->ev_fork = nullptr;
  s->nsub = 1;
}

template <typename R>
cx<R>* sp(nne_state* s, int k) { return reinterpret_cast<cx<R>*>(s->site[k]); }

template <typename R>
nne_status check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return set_cuda_error(e, what, __FILE__, __LINE__);
  return NNE_OK;
}

#define TRY(x)                          \
  do {                                  \
    nne_status _s = (x);                \
    if (_s != NNE_OK) return _s;        \
  } while (0)
#define CTRY(x) TRY(check<R>((x), #x))

// A contiguous range of instances [i0, i0 + nb) whose arithmetic is enqueued
// on one stream; per-instance buffers are addressed from instance i0.
struct BatchView {
  cudaStream_t st;
  int i0, nb;
};
template <typename R>
cx<R>* spb(nne_state* s, const BatchView& b, int k) {
  return reinterpret_cast<cx<R>*>(s->site[k]) + (long long)b.i0 * s->sstride[k];
}
template <typename R>
cx<R>* wsb(void* base, long long stride, const BatchView& b) {
  return reinterpret_cast<cx<R>*>(base) + (long long)b.i0 * stride;
}
template <typename R>
cx<R>* qrws(nne_state* s, const BatchView& b) {
  return reinterpret_cast<cx<R>*>(s->qr_ws) + (long long)b.i0 * s->qr_pi;
}
template <typename R>
cx<R>* eigcx(nne_state* s, const BatchView& b) {
  return reinterpret_cast<cx<R>*>(s->eig_cx) + (long long)b.i0 * s->eig_cx_pi;
}
template <typename R>
R* eigre(nne_state* s, const BatchView& b) {
  return reinterpret_cast<R*>(s->eig_re) + (long long)b.i0 * s->eig_re_pi;
}
inline uint8_t* eigu8(nne_state* s, const BatchView& b) {
  return reinterpret_cast<uint8_t*>(s->eig_u8) + (long long)b.i0 * s->eig_u8_pi;
}

// The projection P X of a truncating split as a product of its two factors
// (rows x cols = op(F) op(G), K = r): X <- X - P X gives the discarded part.
template <typename R>
struct SplitProduct {
  int opF, opG, M, N, K;
  const cx<R>* F;
  long long sF;
  int ldf;
  const cx<R>* G;
  long long sG;
  int ldg;
};

// Norm bookkeeping after a split: kept = ||C||^2 normalises C, total =
// ||X||^2 (or kept), f = kept / total.  For complex64 truncations the kept
// weight of f is taken as total - ||X - P X||^2 instead: the tensor cores'
// float32 accumulation truncates, which biases ||C||^2 = ||W^H X||^2 low by
// about 1e-5 relative at K = 2048 -- as large as a tenth of a typical gate's
// discarded weight -- while the residual's own bias is relative to the small
// discarded part.  X is overwritten by the residual.
template <typename R>
nne_status finish_split(nne_state* s, const BatchView& b, cx<R>* C, long long sC, long long countC, cx<R>* Xt,
                        long long sXt, long long countX, const SplitProduct<R>* px = nullptr) {
  cudaStream_t st = b.st;
  double* kept = s->d_parts + (long long)b.i0 * PARTS;
  double* total = s->d_parts + (long long)s->n_inst * PARTS + (long long)b.i0 * PARTS;
  double* disc = s->d_parts + 2LL * s->n_inst * PARTS + (long long)b.i0 * PARTS;
  CTRY(sumsq_partial<R>(st, C, sC, countC, kept, PARTS, b.nb));
  if (Xt) CTRY(sumsq_partial<R>(st, Xt, sXt, countX, total, PARTS, b.nb));
  const bool resid = Xt && px && std::is_same<R, float>::value;
  if (resid) {
    CTRY(cgemm<R>(st, px->opF, px->opG, px->M, px->N, px->K, mk<R>(-1, 0), px->F, px->sF, px->ldf, px->G, px->sG,
                  px->ldg, mk<R>(1, 0), Xt, sXt, px->N, b.nb));
    CTRY(sumsq_partial<R>(st, Xt, sXt, countX, disc, PARTS, b.nb));
  }
  CTRY(finish_gate(st, kept, Xt ? total : nullptr, resid ? disc : nullptr, PARTS, b.nb, s->d_scale + b.i0,
                   s->d_lognorm + b.i0, s->d_logfid + b.i0, s->d_err));
  CTRY(scale_batched<R>(st, C, sC, countC, s->d_scale + b.i0, b.nb));
  return NNE_OK;
}

// Make site c left-isometric by QR and push R into site c+1.
template <typename R>
nne_status qr_right(nne_state* s, const BatchView& b, int c) {
  cudaStream_t st = b.st;
  const int dl = s->dims[c], dr = s->dims[c + 1], dn = s->dims[c + 2];
  const int m = 4 * dl, k = std::min(m, dr);
  cx<R>* M = spb<R>(s, b, c);
  cx<R>* Q = wsb<R>(s->T, s->sT, b);
  cx<R>* Rr = wsb<R>(s->Rm, s->sR, b);
  CTRY(qr<R>(st, M, s->sstride[c], m, dr, Q, s->sT, Rr, s->sR, qrws<R>(s, b), b.nb));
  CTRY(fix_qr<R>(st, Q, s->sT, m, k, Rr, s->sR, dr, b.nb));
  CTRY(copy_batched<R>(st, Q, s->sT, M, s->sstride[c], (long long)m * k, b.nb));
  // next <- R next
  cx<R>* N = spb<R>(s, b, c + 1);
  cx<R>* tmp = wsb<R>(s->H, s->sH, b);
  CTRY(cgemm<R>(st, OP_N, OP_N, k, 4 * dn, dr, mk<R>(1, 0), Rr, s->sR, dr, N, s->sstride[c + 1], 4 * dn,
                mk<R>(0, 0), tmp, s->sH, 4 * dn, b.nb));
  CTRY(copy_batched<R>(st, tmp, s->sH, N, s->sstride[c + 1], (long long)k * 4 * dn, b.nb));
  return NNE_OK;
}

// Make site c right-isometric by LQ (QR of M^H) and push L into site c-1.
template <typename R>
nne_status lq_left(nne_state* s, const BatchView& b, int c) {
  cudaStream_t st = b.st;
  const int dp = s->dims[c - 1], dl = s->dims[c], dr = s->dims[c + 1];
  const int m = 4 * dr, k = std::min(m, dl);
  cx<R>* M = spb<R>(s, b, c);
  cx<R>* Mh = wsb<R>(s->U, s->sU, b);
  CTRY(transpose<R>(st, true, M, s->sstride[c], dl, m, m, Mh, s->sU, dl, b.nb));   // (4dr x dl)
  cx<R>* Q = wsb<R>(s->T, s->sT, b);
  cx<R>* Rr = wsb<R>(s->Rm, s->sR, b);
  CTRY(qr<R>(st, Mh, s->sU, m, dl, Q, s->sT, Rr, s->sR, qrws<R>(s, b), b.nb));          // Q (m x k), R (k x dl)
  CTRY(fix_qr<R>(st, Q, s->sT, m, k, Rr, s->sR, dl, b.nb));
  CTRY(transpose<R>(st, true, Q, s->sT, m, k, k, M, s->sstride[c], m, b.nb));       // site c = Q^H (k x m)
  cx<R>* P = spb<R>(s, b, c - 1);
  cx<R>* tmp = wsb<R>(s->H, s->sH, b);
  CTRY(cgemm<R>(st, OP_N, OP_C, 4 * dp, k, dl, mk<R>(1, 0), P, s->sstride[c - 1], dl, Rr, s->sR, dl, mk<R>(0, 0),
                tmp, s->sH, k, b.nb));
  CTRY(copy_batched<R>(st, tmp, s->sH, P, s->sstride[c - 1], (long long)4 * dp * k, b.nb));
  return NNE_OK;
}

// Move the orthogonality centre to `target`, one site at a time; each step is
// enqueued for every batch view (each on its own stream) before the shared
// bond dimension is updated.
template <typename R>
nne_status move_centre(nne_state* s, const std::vector<BatchView>& views, int target) {
  while (s->centre < target) {
    const int c = s->centre;
    for (const BatchView& b : views) TRY(qr_right<R>(s, b, c));
    s->dims[c + 1] = std::min(4 * s->dims[c], s->dims[c + 1]);
    s->centre++;
  }
  while (s->centre > target) {
    const int c = s->centre;
    for (const BatchView& b : views) TRY(lq_left<R>(s, b, c));
    s->dims[c] = std::min(4 * s->dims[c + 1], s->dims[c]);
    s->centre--;
  }
  return NNE_OK;
}

// Top-r eigenvectors of the Hermitian H (n x n) into W (n x r): complex64
// states take the float64 reduction and tridiagonal solve unless disabled.
template <typename R>
nne_status eigh_state(nne_state* s, const BatchView& b, cx<R>* H, long long sH, int n, int r, cx<R>* W, long long sW) {
  if constexpr (std::is_same<R, float>::value) {
    if (g_eig_fp64)
      return check<R>(eigh_top_mixed(b.st, H, sH, n, r, W, sW, eigcx<R>(s, b), eigre<R>(s, b), eigu8(s, b), b.nb,
                                     s->d_err),
                      "eigh_top_mixed");
  }
  return check<R>(eigh_top<R>(b.st, H, sH, n, r, W, sW, eigcx<R>(s, b), eigre<R>(s, b), eigu8(s, b), b.nb, s->d_err),
                  "eigh_top");
}

// Top-r left (dir > 0) or right (dir < 0) singular subspace of X[z] as an
// isometry W (n_side x r, ld r) in s->U.
//  exact: eigenvectors of the Gram matrix X X^H (or X^H X);
//  subspace iteration (Halko-Martinsson-Tropp): Y = X Omega (k columns), q
//    power iterations Y <- X X^H Q each followed by re-orthonormalisation,
//    Rayleigh-Ritz on C = (Q^H X)(Q^H X)^H, W = Q * (top-r eigenvectors of C).
//    With enough columns and iterations it reaches the SVD truncation's
//    subspace (the kept weight converges from below); used when k < n_side,
//    otherwise the sketch spans the space and the exact path runs.
template <typename R>
nne_status subspace(nne_state* s, const BatchView& b, cx<R>* X, int rows, int cols, int r, int dir) {
  cudaStream_t st = b.st;
  cx<R>* Hm = wsb<R>(s->H, s->sH, b);
  cx<R>* W = wsb<R>(s->U, s->sU, b);
  const cx<R> one = mk<R>(1, 0), zero = mk<R>(0, 0);
  const int n = dir > 0 ? rows : cols;
  const int other = dir > 0 ? cols : rows;
  const int k = s->omega_cols;
  const bool rsvd = s->trunc == NNE_TRUNC_RSVD && s->d_omega && k < n && k >= r;
  if (rsvd) {
    cx<R>* Om = reinterpret_cast<cx<R>*>(s->d_omega);
    cx<R>* Y = wsb<R>(s->rs_Y, s->rs_sY, b);    // n x k
    cx<R>* Z = wsb<R>(s->rs_Z, s->rs_sZ, b);    // other x k
    cx<R>* Cm = wsb<R>(s->rs_C, s->rs_sC, b);   // k x k
    cx<R>* Wk = wsb<R>(s->rs_W, s->rs_sW, b);   // k x r
    const long long sY = s->rs_sY, sZ = s->rs_sZ, sC = s->rs_sC, sW = s->rs_sW;
    // A = X (dir > 0) or X^H (dir < 0): A is n x other
    const int opA = dir > 0 ? OP_N : OP_C, opAh = dir > 0 ? OP_C : OP_N;
    // X feeds 2 q + 2 products in both forms: split it into TF32 planes once each
    const bool hold = std::is_same<R, float>::value && tensor_cores_enabled() && gemm_tma_enabled() &&
                      cgemm_tma_available() && n >= 128 && other >= 128 && k >= 64;
    if constexpr (std::is_same<R, float>::value) {
      tma_release(st);   // nothing held from an earlier step that ended in an error
      if (hold) {
        CTRY(tma_hold_a(st, opA, n, other, X, s->sX, cols, b.nb));
        CTRY(tma_hold_a(st, opAh, other, n, X, s->sX, cols, b.nb));
      }
    }
    CTRY(cgemm<R>(st, opA, OP_N, n, k, other, one, X, s->sX, cols, Om, 0, k, zero, Y, sY, k, b.nb));
    CTRY(qr<R>(st, Y, sY, n, k, Y, sY, nullptr, 0, qrws<R>(s, b), b.nb));
    // power iterations Y <- A (A^H Q), re-orthonormalised after each application of A A^H
    for (int it = 0; it < s->power_iters; ++it) {
      CTRY(cgemm<R>(st, opAh, OP_N, other, k, n, one, X, s->sX, cols, Y, sY, k, zero, Z, sZ, k, b.nb));
      CTRY(cgemm<R>(st, opA, OP_N, n, k, other, one, X, s->sX, cols, Z, sZ, k, zero, Y, sY, k, b.nb));
      CTRY(qr<R>(st, Y, sY, n, k, Y, sY, nullptr, 0, qrws<R>(s, b), b.nb));
    }
    if (k == r) {   // the sketch space itself is the answer
      if (hold) tma_release(st);
      CTRY(copy_batched<R>(st, Y, sY, W, s->sU, (long long)n * k, b.nb));
      CTRY(fix_columns<R>(st, W, s->sU, n, r, b.nb));
      return NNE_OK;
    }
    // Bt = A^H Q (other x k); C = Bt^H Bt (k x k)
    CTRY(cgemm<R>(st, opAh, OP_N, other, k, n, one, X, s->sX, cols, Y, sY, k, zero, Z, sZ, k, b.nb));
    if (hold) tma_release(st);
    CTRY(cgemm<R>(st, OP_C, OP_N, k, k, other, one, Z, sZ, k, Z, sZ, k, zero, Cm, sC, k, b.nb));
    TRY(eigh_state<R>(s, b, Cm, sC, k, r, Wk, sW));
    CTRY(cgemm<R>(st, OP_N, OP_N, n, r, k, one, Y, sY, k, Wk, sW, r, zero, W, s->sU, r, b.nb));
  } else {
    if (dir > 0)
      CTRY(cgemm<R>(st, OP_N, OP_C, rows, rows, cols, one, X, s->sX, cols, X, s->sX, cols, zero, Hm, s->sH, rows,
                    b.nb));
    else
      CTRY(cgemm<R>(st, OP_C, OP_N, cols, cols, rows, one, X, s->sX, cols, X, s->sX, cols, zero, Hm, s->sH, cols,
                    b.nb));
    TRY(eigh_state<R>(s, b, Hm, s->sH, n, r, W, s->sU));
  }
  CTRY(fix_columns<R>(st, W, s->sU, n, r, b.nb));
  return NNE_OK;
}

template <typename R>
nne_status gate_compute(nne_state* s, const BatchView& b, int q, const double* G, long long sG, int dir) {
  cudaStream_t st = b.st;
  G += 2LL * b.i0 * sG;   // this view's instances
  const int dl = s->dims[q], dm = s->dims[q + 1], dr = s->dims[q + 2];
  const int rows = 4 * dl, cols = 4 * dr;
  const int r = std::min(s->chi, std::min(rows, cols));
  cx<R>* A = spb<R>(s, b, q);
  cx<R>* B = spb<R>(s, b, q + 1);
  cx<R>* X = wsb<R>(s->X, s->sX, b);
  // a2: theta = A B ; a3: theta' = G theta
  CTRY(cgemm<R>(st, OP_N, OP_N, rows, cols, dm, mk<R>(1, 0), A, s->sstride[q], dm, B, s->sstride[q + 1], cols,
                mk<R>(0, 0), X, s->sX, cols, b.nb));
  CTRY(apply_superop<R>(st, X, s->sX, dl, dr, G, sG, b.nb));
  const long long countX = (long long)rows * cols;
  if (dir > 0) {
    if (r == rows) {
      CTRY(identity<R>(st, A, s->sstride[q], rows, r, b.nb));
      CTRY(copy_batched<R>(st, X, s->sX, B, s->sstride[q + 1], countX, b.nb));
      TRY(finish_split<R>(s, b, B, s->sstride[q + 1], countX, nullptr, 0, 0));
    } else if (r == cols) {
      // nothing is cut: X = Q R exactly (Householder), left factor Q, centre R
      cx<R>* Q = wsb<R>(s->T, s->sT, b);
      CTRY(qr<R>(st, X, s->sX, rows, cols, Q, s->sT, B, s->sstride[q + 1], qrws<R>(s, b), b.nb));
      CTRY(fix_qr<R>(st, Q, s->sT, rows, r, B, s->sstride[q + 1], cols, b.nb));
      CTRY(copy_batched<R>(st, Q, s->sT, A, s->sstride[q], (long long)rows * r, b.nb));
      TRY(finish_split<R>(s, b, B, s->sstride[q + 1], (long long)r * cols, nullptr, 0, 0));
    } else {
      TRY(subspace<R>(s, b, X, rows, cols, r, +1));
      cx<R>* W = wsb<R>(s->U, s->sU, b);
      CTRY(copy_batched<R>(st, W, s->sU, A, s->sstride[q], (long long)rows * r, b.nb));
      CTRY(cgemm<R>(st, OP_C, OP_N, r, cols, rows, mk<R>(1, 0), W, s->sU, r, X, s->sX, cols, mk<R>(0, 0), B,
                    s->sstride[q + 1], cols, b.nb));
      const SplitProduct<R> px{OP_N, OP_N, rows, cols, r, W, s->sU, r, B, s->sstride[q + 1], cols};   // W B'
      TRY(finish_split<R>(s, b, B, s->sstride[q + 1], (long long)r * cols, X, s->sX, countX, &px));
    }
  } else {
    if (r == cols) {
      CTRY(identity<R>(st, B, s->sstride[q + 1], r, cols, b.nb));
      CTRY(copy_batched<R>(st, X, s->sX, A, s->sstride[q], countX, b.nb));
      TRY(finish_split<R>(s, b, A, s->sstride[q], countX, nullptr, 0, 0));
    } else if (r == rows) {
      // nothing is cut: X^H = Q R exactly, right factor Q^H, centre R^H
      cx<R>* Xh = wsb<R>(s->H, s->sH, b);
      cx<R>* Q = wsb<R>(s->T, s->sT, b);
      cx<R>* Rr = wsb<R>(s->Rm, s->sR, b);
      CTRY(transpose<R>(st, true, X, s->sX, rows, cols, cols, Xh, s->sH, rows, b.nb));
      CTRY(qr<R>(st, Xh, s->sH, cols, rows, Q, s->sT, Rr, s->sR, qrws<R>(s, b), b.nb));
      CTRY(fix_qr<R>(st, Q, s->sT, cols, r, Rr, s->sR, rows, b.nb));
      CTRY(transpose<R>(st, true, Q, s->sT, cols, r, r, B, s->sstride[q + 1], cols, b.nb));
      CTRY(transpose<R>(st, true, Rr, s->sR, r, rows, rows, A, s->sstride[q], r, b.nb));
      TRY(finish_split<R>(s, b, A, s->sstride[q], (long long)rows * r, nullptr, 0, 0));
    } else {
      TRY(subspace<R>(s, b, X, rows, cols, r, -1));
      cx<R>* W = wsb<R>(s->U, s->sU, b);
      CTRY(transpose<R>(st, true, W, s->sU, cols, r, r, B, s->sstride[q + 1], cols, b.nb));
      CTRY(cgemm<R>(st, OP_N, OP_N, rows, r, cols, mk<R>(1, 0), X, s->sX, cols, W, s->sU, r, mk<R>(0, 0), A,
                    s->sstride[q], r, b.nb));
      const SplitProduct<R> px{OP_N, OP_C, rows, cols, r, A, s->sstride[q], r, W, s->sU, r};   // A' W^H
      TRY(finish_split<R>(s, b, A, s->sstride[q], (long long)rows * r, X, s->sX, countX, &px));
    }
  }
  return NNE_OK;
}

// One gate on every view: centre to the gate, the per-view arithmetic, then
// the shared bond dimension and centre.
template <typename R>
nne_status gate_step(nne_state* s, const std::vector<BatchView>& views, int q, const double* G, long long sG,
                     int dir) {
  TRY(move_centre<R>(s, views, dir > 0 ? q : q + 1));
  const int r = std::min(s->chi, std::min(4 * s->dims[q], 4 * s->dims[q + 2]));
  for (const BatchView& b : views) TRY(gate_compute<R>(s, b, q, G, sG, dir));
  s->dims[q + 1] = r;
  s->centre = dir > 0 ? q + 1 : q;
  return NNE_OK;
}

template <typename R>
nne_status compress(nne_state* s, int chi_new) {
  const BatchView b{s->ctx->stream, 0, s->n_inst};
  const std::vector<BatchView> views{b};
  cudaStream_t st = b.st;
  TRY(move_centre<R>(s, views, 0));
  for (int k = 0; k + 1 < s->n; ++k) {
    const int dl = s->dims[k], dr = s->dims[k + 1], dn = s->dims[k + 2];
    const int rows = 4 * dl;
    const int r = std::min(chi_new, std::min(rows, dr));
    if (r >= dr) {
      TRY(qr_right<R>(s, b, k));
      s->dims[k + 1] = std::min(rows, dr);
    } else {
      cx<R>* M = spb<R>(s, b, k);
      cx<R>* Hm = wsb<R>(s->H, s->sH, b);
      cx<R>* W = wsb<R>(s->U, s->sU, b);
      cx<R>* Cm = wsb<R>(s->Rm, s->sR, b);
      cx<R>* Xs = wsb<R>(s->X, s->sX, b);
      CTRY(copy_batched<R>(st, M, s->sstride[k], Xs, s->sX, (long long)rows * dr, b.nb));
      CTRY(cgemm<R>(st, OP_N, OP_C, rows, rows, dr, mk<R>(1, 0), Xs, s->sX, dr, Xs, s->sX, dr, mk<R>(0, 0), Hm,
                    s->sH, rows, b.nb));
      TRY(eigh_state<R>(s, b, Hm, s->sH, rows, r, W, s->sU));
      CTRY(fix_columns<R>(st, W, s->sU, rows, r, b.nb));
      CTRY(copy_batched<R>(st, W, s->sU, M, s->sstride[k], (long long)rows * r, b.nb));
      CTRY(cgemm<R>(st, OP_C, OP_N, r, dr, rows, mk<R>(1, 0), W, s->sU, r, Xs, s->sX, dr, mk<R>(0, 0), Cm, s->sR, dr,
                    b.nb));
      const SplitProduct<R> px{OP_N, OP_N, rows, dr, r, W, s->sU, r, Cm, s->sR, dr};   // W C
      TRY(finish_split<R>(s, b, Cm, s->sR, (long long)r * dr, Xs, s->sX, (long long)rows * dr, &px));
      cx<R>* N = spb<R>(s, b, k + 1);
      cx<R>* tmp = wsb<R>(s->T, s->sT, b);
      CTRY(cgemm<R>(st, OP_N, OP_N, r, 4 * dn, dr, mk<R>(1, 0), Cm, s->sR, dr, N, s->sstride[k + 1], 4 * dn,
                    mk<R>(0, 0), tmp, s->sT, 4 * dn, b.nb));
      CTRY(copy_batched<R>(st, tmp, s->sT, N, s->sstride[k + 1], (long long)r * 4 * dn, b.nb));
      s->dims[k + 1] = r;
    }
    s->centre = k + 1;
  }
  s->chi = chi_new;
  return NNE_OK;
}

// MPO entanglement entropy of every bond (App. A.1): centre to site 0, then
// for k = 0 .. n-2 the Gram matrix M_k^H M_k of the centre tensor (its
// eigenvalues are the squared Schmidt values of bond k | k+1) and a QR step
// that moves the centre on.  S[z * (n - 1) + k] on the device.
template <typename R>
nne_status entropy_sweep(nne_state* s, double* S) {
  const BatchView b{s->ctx->stream, 0, s->n_inst};
  const std::vector<BatchView> views{b};
  cudaStream_t st = b.st;
  TRY(move_centre<R>(s, views, 0));
  for (int k = 0; k + 1 < s->n; ++k) {
    const int dl = s->dims[k], dr = s->dims[k + 1];
    cx<R>* M = spb<R>(s, b, k);
    cx<R>* Hm = wsb<R>(s->H, s->sH, b);
    CTRY(cgemm<R>(st, OP_C, OP_N, dr, dr, 4 * dl, mk<R>(1, 0), M, s->sstride[k], dr, M, s->sstride[k], dr,
                  mk<R>(0, 0), Hm, s->sH, dr, b.nb));
    CTRY(gram_entropy<R>(st, Hm, s->sH, dr, eigcx<R>(s, b), eigre<R>(s, b), b.nb, S + k, s->n - 1));
    TRY(move_centre<R>(s, views, k + 1));
  }
  return NNE_OK;
}

nne_status read_err(nne_state* s) {
  int h = 0, t = 0;
  cudaError_t e = cudaMemcpyAsync(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->ctx->stream);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaMemcpyAsync", __FILE__, __LINE__);
  int* te = tc_error_ptr();
  if (te) e = cudaMemcpyAsync(&t, te, sizeof(int), cudaMemcpyDeviceToHost, s->ctx->stream);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaMemcpyAsync", __FILE__, __LINE__);
  e = cudaStreamSynchronize(s->ctx->stream);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  if (t != 0 && te) {
    // reported once: the word is cleared so that the next call starts clean
    e = cudaMemsetAsync(te, 0, sizeof(int), s->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctx->stream);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMemsetAsync", __FILE__, __LINE__);
  }
  if (h != 0) return set_error(h, "device-side failure status %d (non-finite or zero norm in a gate step)", h);
  if (t != 0) return set_error(t, "tensor-core GEMM reported status %d (a bounded wait expired)", t);
  return NNE_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

const char* nne_last_error(void) { return g_last_error.c_str(); }

nne_status nne_ctx_create(int device, void* cuda_stream, size_t hbm_budget_bytes, nne_ctx** out) {
  if (!out) return set_error(NNE_ERR_ARG, "out is null");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDeviceCount", __FILE__, __LINE__);
  if (device < 0 || device >= ndev) return set_error(NNE_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
  nne_ctx* c = new nne_ctx();
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->budget = hbm_budget_bytes;
  *out = c;
  return NNE_OK;
}

void nne_ctx_destroy(nne_ctx* ctx) { delete ctx; }

size_t nne_ctx_bytes_in_use(const nne_ctx* ctx) { return ctx ? ctx->used : 0; }

nne_status nne_build_superops(nne_ctx* ctx, int n_gates, const double* U, int n_inst, const double* rates,
                              void* G_out) {
  if (!ctx || n_gates < 0 || n_inst < 1 || !rates || (n_gates > 0 && (!U || !G_out)))
    return set_error(NNE_ERR_ARG, "nne_build_superops: bad arguments");
  DeviceGuard g(ctx->device);
  const bool u_dev = is_device_ptr(U), r_dev = is_device_ptr(rates);
  if (!r_dev)
    for (int i = 0; i < n_inst; ++i)
      for (int c = 0; c < 4; ++c) {
        const double p = rates[4 * i + c];
        const double hi = c == 0 ? 16.0 / 15.0 : 1.0;
        if (!(p >= 0.0 && p <= hi)) return set_error(NNE_ERR_ARG, "rate %d of instance %d out of range: %g", c, i, p);
      }
  if (u_dev && r_dev) {
    // inputs already resident: no staging copies
    ScratchF64& sc = scratch_snoise(ctx, n_inst);
    if (!sc.p) return set_error(NNE_ERR_OOM, "superoperator scratch");
    NNE_CUDA_TRY(build_superops(ctx->stream, n_gates, U, n_inst, rates, (double*)G_out, sc.p));
    return NNE_OK;
  }
  double *dU = nullptr, *dR = nullptr, *dS = nullptr;
  const size_t bu = sizeof(double) * 32 * (size_t)std::max(n_gates, 1), br = sizeof(double) * 4 * n_inst,
               bs = sizeof(double) * 512 * n_inst;
  NNE_CUDA_TRY(cudaMallocAsync(&dU, bu, ctx->stream));
  NNE_CUDA_TRY(cudaMallocAsync(&dR, br, ctx->stream));
  NNE_CUDA_TRY(cudaMallocAsync(&dS, bs, ctx->stream));
  nne_status rc = NNE_OK;
  cudaError_t e = cudaSuccess;
  if (n_gates > 0) e = cudaMemcpyAsync(dU, U, sizeof(double) * 32 * n_gates, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dR, rates, br, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess) e = build_superops(ctx->stream, n_gates, dU, n_inst, dR, (double*)G_out, dS);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) rc = set_cuda_error(e, "build_superops", __FILE__, __LINE__);
  cudaFreeAsync(dU, ctx->stream);
  cudaFreeAsync(dR, ctx->stream);
  cudaFreeAsync(dS, ctx->stream);
  return rc;
}

nne_status nne_build_pauli_superops(nne_ctx* ctx, int n_gates, const double* U, const double* pauli_rates,
                                    int n_inst, const double* lambdas, void* G_out) {
  if (!ctx || n_gates < 0 || n_inst < 1 || !lambdas || (n_gates > 0 && (!U || !pauli_rates || !G_out)))
    return set_error(NNE_ERR_ARG, "nne_build_pauli_superops: bad arguments");
  if (n_gates == 0) return NNE_OK;
  DeviceGuard g(ctx->device);
  const bool u_dev = is_device_ptr(U), p_dev = is_device_ptr(pauli_rates), l_dev = is_device_ptr(lambdas);
  if (!p_dev && !l_dev)
    for (int i = 0; i < n_inst; ++i)
      for (int k = 0; k < n_gates; ++k) {
        double tot = 0;
        for (int ab = 0; ab < 16; ++ab) {
          const double p = pauli_rates[32LL * k + ab] + lambdas[i] * pauli_rates[32LL * k + 16 + ab];
          if (!(p >= -1e-12 && p <= 1.0 + 1e-12))
            return set_error(NNE_ERR_ARG, "Pauli probability %d of gate %d at level %d out of [0,1]: %g", ab, k, i, p);
          tot += p;
        }
        if (!(std::fabs(tot - 1.0) <= 1e-12))
          return set_error(NNE_ERR_ARG, "Pauli probabilities of gate %d at level %d sum to %.17g", k, i, tot);
      }
  if (u_dev && p_dev && l_dev) {
    NNE_CUDA_TRY(build_pauli_superops(ctx->stream, n_gates, U, pauli_rates, n_inst, lambdas, (double*)G_out));
    return NNE_OK;
  }
  double *dU = nullptr, *dP = nullptr, *dL = nullptr;
  const size_t bu = sizeof(double) * 32 * (size_t)n_gates, bp = sizeof(double) * 32 * (size_t)n_gates,
               bl = sizeof(double) * n_inst;
  NNE_CUDA_TRY(cudaMallocAsync(&dU, bu, ctx->stream));
  NNE_CUDA_TRY(cudaMallocAsync(&dP, bp, ctx->stream));
  NNE_CUDA_TRY(cudaMallocAsync(&dL, bl, ctx->stream));
  nne_status rc = NNE_OK;
  cudaError_t e = cudaMemcpyAsync(dU, U, bu, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dP, pauli_rates, bp, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dL, lambdas, bl, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess) e = build_pauli_superops(ctx->stream, n_gates, dU, dP, n_inst, dL, (double*)G_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) rc = set_cuda_error(e, "build_pauli_superops", __FILE__, __LINE__);
  cudaFreeAsync(dU, ctx->stream);
  cudaFreeAsync(dP, ctx->stream);
  cudaFreeAsync(dL, ctx->stream);
  return rc;
}

nne_status nne_create_state(nne_ctx* ctx, int n_qubits, int chi, int n_inst, nne_dtype dtype, nne_trunc trunc,
                            const uint8_t* init_bits, nne_state** out) {
  if (!ctx || !out || n_qubits < 2 || chi < 1 || n_inst < 1 || (dtype != NNE_C64 && dtype != NNE_C128) ||
      (trunc != NNE_TRUNC_EXACT && trunc != NNE_TRUNC_RSVD))
    return set_error(NNE_ERR_ARG, "nne_create_state: bad arguments");
  if (chi > 4096) return set_error(NNE_ERR_ARG, "chi %d above the supported maximum 4096", chi);
  *out = nullptr;
  DeviceGuard g(ctx->device);
  nne_state* s = new nne_state();
  s->ctx = ctx;
  s->mem.ctx = ctx;
  s->n = n_qubits;
  s->chi = chi;
  s->n_inst = n_inst;
  s->dtype = dtype;
  s->trunc = trunc;
  s->esz = dtype == NNE_C64 ? 8 : 16;
  const int n = n_qubits;
  s->dims.assign(n + 1, 1);
  s->cap = bond_caps(n, chi);
  for (int k = 0; k <= n; ++k) s->dmax = std::max(s->dmax, s->cap[k]);
  auto fail = [&](nne_status rc) {
    s->mem.release();
    delete s;
    return rc;
  };
  // site arena
  size_t total = 0;
  std::vector<size_t> off(n);
  s->sstride.resize(n);
  for (int k = 0; k < n; ++k) {
    s->sstride[k] = (long long)s->cap[k] * 4 * s->cap[k + 1];
    off[k] = total;
    total += (size_t)s->sstride[k] * n_inst * s->esz;
    total = (total + 255) & ~size_t(255);
  }
  void* arena = nullptr;
  nne_status rc = s->mem.alloc(&arena, total);
  if (rc != NNE_OK) return fail(rc);
  s->site.resize(n);
  for (int k = 0; k < n; ++k) s->site[k] = reinterpret_cast<char*>(arena) + off[k];
  // initial product state |b><b| : s = 3 b
  {
    std::vector<char> host(total, 0);
    for (int k = 0; k < n; ++k) {
      const int b = init_bits ? (init_bits[k] ? 1 : 0) : 0;
      for (int i = 0; i < n_inst; ++i) {
        char* p = host.data() + off[k] + (size_t)i * s->sstride[k] * s->esz + (size_t)(3 * b) * s->esz;
        if (dtype == NNE_C64) {
          const float one = 1.0f;
          memcpy(p, &one, sizeof(float));
        } else {
          const double one = 1.0;
          memcpy(p, &one, sizeof(double));
        }
      }
    }
    cudaError_t e = cudaMemcpyAsync(arena, host.data(), total, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(set_cuda_error(e, "cudaMemcpyAsync", __FILE__, __LINE__));
  }
  // scalars
  void* p = nullptr;
  if ((rc = s->mem.alloc(&p, sizeof(double) * (3 * n_inst + 3 * (size_t)n_inst * PARTS) + 64)) != NNE_OK)
    return fail(rc);
  cudaMemsetAsync(p, 0, sizeof(double) * (3 * n_inst + 3 * (size_t)n_inst * PARTS) + 64, ctx->stream);
  s->d_lognorm = reinterpret_cast<double*>(p);
  s->d_logfid = s->d_lognorm + n_inst;
  s->d_scale = s->d_logfid + n_inst;
  s->d_parts = s->d_scale + n_inst;
  s->d_err = reinterpret_cast<int*>(s->d_parts + 3 * (size_t)n_inst * PARTS);
  // workspaces
  const long long D = s->dmax, N4 = 4 * D;
  s->sX = N4 * N4;
  s->sH = N4 * N4;
  s->sU = N4 * D;
  s->sT = N4 * N4;
  s->sR = N4 * D > D * D ? N4 * D : D * D;
  if ((rc = s->mem.alloc(&s->X, (size_t)s->sX * n_inst * s->esz)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->H, (size_t)s->sH * n_inst * s->esz)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->U, (size_t)s->sU * n_inst * s->esz)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->T, (size_t)s->sT * n_inst * s->esz)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->Rm, (size_t)s->sR * n_inst * s->esz)) != NNE_OK) return fail(rc);
  const EighWork ew = eigh_workspace_state((int)N4, (int)D, dtype);
  const size_t rsz = s->esz / 2;
  s->eig_cx_pi = ew.cx_elems;
  s->eig_re_pi = ew.re_elems;
  s->eig_u8_pi = ew.u8_elems;
  if ((rc = s->mem.alloc(&s->eig_cx, (size_t)ew.cx_elems * n_inst * s->esz)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->eig_re, (size_t)ew.re_elems * n_inst * rsz + 256)) != NNE_OK) return fail(rc);
  if ((rc = s->mem.alloc(&s->eig_u8, (size_t)ew.u8_elems * n_inst)) != NNE_OK) return fail(rc);
  const QrWork qw = qr_workspace((int)N4, (int)N4);
  s->qr_pi = qw.cx_elems;
  if ((rc = s->mem.alloc(&s->qr_ws, (size_t)qw.cx_elems * n_inst * s->esz)) != NNE_OK) return fail(rc);
  s->bits.assign(n, 0);
  if (init_bits)
    for (int k = 0; k < n; ++k) s->bits[k] = init_bits[k] ? 1 : 0;
  if ((rc = s->mem.alloc(&p, n)) != NNE_OK) return fail(rc);
  s->d_bits = reinterpret_cast<uint8_t*>(p);
  if (cudaMemcpyAsync(s->d_bits, s->bits.data(), n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return fail(set_error(NNE_ERR_CUDA, "cudaMemcpyAsync bits"));
  // sweep buffers
  if ((rc = s->mem.alloc(&p, sizeof(int) * (n + 1))) != NNE_OK) return fail(rc);
  s->d_dims = reinterpret_cast<int*>(p);
  if ((rc = s->mem.alloc(&p, sizeof(void*) * n)) != NNE_OK) return fail(rc);
  s->d_site = reinterpret_cast<void**>(p);
  if ((rc = s->mem.alloc(&p, sizeof(long long) * n)) != NNE_OK) return fail(rc);
  s->d_stride = reinterpret_cast<long long*>(p);
  if ((rc = s->mem.alloc(&p, sizeof(double) * 2 * 2 * (size_t)(n + 1) * D * n_inst)) != NNE_OK) return fail(rc);
  s->d_env = reinterpret_cast<double*>(p);
  if ((rc = s->mem.alloc(&p, sizeof(double) * 2 * (size_t)(n + 1) * n_inst)) != NNE_OK) return fail(rc);
  s->d_envscale = reinterpret_cast<double*>(p);
  {
    std::vector<void*> hs(s->site.begin(), s->site.end());
    cudaError_t e = cudaMemcpyAsync(s->d_site, hs.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_stride, s->sstride.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(set_cuda_error(e, "cudaMemcpyAsync", __FILE__, __LINE__));
  }
  // concurrent sub-batches of the gate steps (streams and fork/join events); only where the
  // kernels are large (bonds of 256 and more): small states are launch-bound, and splitting
  // them multiplies their launches
  s->nsub = s->dmax >= 256 ? std::max(1, std::min(g_substreams, n_inst)) : 1;
  if (s->nsub > 1) {
    cudaError_t e2 = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    for (int v = 0; v < s->nsub && e2 == cudaSuccess; ++v) {
      cudaStream_t q = nullptr;
      cudaEvent_t ev = nullptr;
      e2 = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
      if (e2 == cudaSuccess) s->sub_st.push_back(q);
      if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e2 == cudaSuccess) s->ev_join.push_back(ev);
    }
    if (e2 != cudaSuccess) {
      destroy_streams(s);
      return fail(set_cuda_error(e2, "sub-batch streams", __FILE__, __LINE__));
    }
  }
  *out = s;
  return NNE_OK;
}

void nne_destroy_state(nne_state* st) {
  if (!st) return;
  DeviceGuard g(st->ctx->device);
  cudaStreamSynchronize(st->ctx->stream);
  for (cudaStream_t q : st->sub_st) cudaStreamSynchronize(q);
  destroy_streams(st);
  st->mem.release();
  delete st;
}

nne_status nne_set_sketch(nne_state* st, const void* omega, int rows, int cols, int power_iters) {
  if (!st || !omega || rows < 4 * st->dmax || cols < 1 || cols > 4 * st->dmax || power_iters < 0 || power_iters > 16)
    return set_error(NNE_ERR_ARG, "nne_set_sketch: need rows >= 4*chi_max (%d), 1 <= cols <= 4*chi_max, 0 <= q <= 16",
                     4 * st->dmax);
  if (st->d_omega) return set_error(NNE_ERR_ARG, "nne_set_sketch: sketch already set");
  DeviceGuard dg(st->ctx->device);
  void* p = nullptr;
  nne_status rc;
  const size_t es = st->esz;
  const long long N4 = 4LL * st->dmax;
  if ((rc = st->mem.alloc(&p, (size_t)rows * cols * es)) != NNE_OK) return rc;
  st->d_omega = p;
  NNE_CUDA_TRY(cudaMemcpyAsync(st->d_omega, omega, (size_t)rows * cols * es, cudaMemcpyDefault, st->ctx->stream));
  NNE_CUDA_TRY(cudaStreamSynchronize(st->ctx->stream));
  st->rs_sY = N4 * cols;
  st->rs_sZ = N4 * cols;
  st->rs_sC = (long long)cols * cols;
  st->rs_sW = (long long)cols * st->dmax;
  if ((rc = st->mem.alloc(&st->rs_Y, (size_t)st->rs_sY * st->n_inst * es)) != NNE_OK) return rc;
  if ((rc = st->mem.alloc(&st->rs_Z, (size_t)st->rs_sZ * st->n_inst * es)) != NNE_OK) return rc;
  if ((rc = st->mem.alloc(&st->rs_C, (size_t)st->rs_sC * st->n_inst * es)) != NNE_OK) return rc;
  if ((rc = st->mem.alloc(&st->rs_W, (size_t)st->rs_sW * st->n_inst * es)) != NNE_OK) return rc;
  st->omega_rows = rows;
  st->omega_cols = cols;
  st->power_iters = power_iters;
  return NNE_OK;
}

nne_status nne_apply_layer(nne_state* st, int n_gates, const int* left_qubit, const void* G, int direction) {
  if (!st || n_gates < 0 || (n_gates > 0 && (!left_qubit || !G)) || (direction != 1 && direction != -1))
    return set_error(NNE_ERR_ARG, "nne_apply_layer: bad arguments");
  for (int g = 0; g < n_gates; ++g)
    if (left_qubit[g] < 0 || left_qubit[g] > st->n - 2)
      return set_error(NNE_ERR_ARG, "gate %d: left qubit %d out of range", g, left_qubit[g]);
  DeviceGuard dg(st->ctx->device);
  const double* Gd = reinterpret_cast<const double*>(G);
  const long long sG = (long long)n_gates * 256;   // complex elements between instances
  // the instances split into nsub views, each on its own stream, forked from and joined back
  // to the context stream; gate by gate the host enqueues every view's work in turn
  const int nv = g_serial_layers ? 1 : st->nsub;
  std::vector<BatchView> views;
  for (int v = 0; v < nv; ++v) {
    const int i0 = (int)((long long)st->n_inst * v / nv), i1 = (int)((long long)st->n_inst * (v + 1) / nv);
    views.push_back(BatchView{nv > 1 ? st->sub_st[v] : st->ctx->stream, i0, i1 - i0});
  }
  if (nv > 1) {
    NNE_CUDA_TRY(cudaEventRecord(st->ev_fork, st->ctx->stream));
    for (int v = 0; v < nv; ++v) NNE_CUDA_TRY(cudaStreamWaitEvent(st->sub_st[v], st->ev_fork, 0));
  }
  nne_status rc = NNE_OK;
  for (int g = 0; g < n_gates && rc == NNE_OK; ++g)
    rc = st->dtype == NNE_C64 ? gate_step<float>(st, views, left_qubit[g], Gd + 2LL * 256 * g, sG, direction)
                              : gate_step<double>(st, views, left_qubit[g], Gd + 2LL * 256 * g, sG, direction);
  if (nv > 1)
    for (int v = 0; v < nv; ++v) {
      cudaEventRecord(st->ev_join[v], st->sub_st[v]);
      cudaStreamWaitEvent(st->ctx->stream, st->ev_join[v], 0);
    }
  return rc;
}

nne_status nne_truncate(nne_state* st, int chi_new, double* log_fid_out) {
  if (!st || chi_new < 1 || chi_new > st->chi) return set_error(NNE_ERR_ARG, "nne_truncate: bad arguments");
  DeviceGuard dg(st->ctx->device);
  std::vector<double> before(st->n_inst), after(st->n_inst);
  NNE_CUDA_TRY(cudaMemcpyAsync(before.data(), st->d_logfid, sizeof(double) * st->n_inst, cudaMemcpyDeviceToHost,
                               st->ctx->stream));
  nne_status rc = st->dtype == NNE_C64 ? compress<float>(st, chi_new) : compress<double>(st, chi_new);
  if (rc != NNE_OK) return rc;
  NNE_CUDA_TRY(cudaMemcpyAsync(after.data(), st->d_logfid, sizeof(double) * st->n_inst, cudaMemcpyDeviceToHost,
                               st->ctx->stream));
  if ((rc = read_err(st)) != NNE_OK) return rc;
  if (log_fid_out)
    for (int i = 0; i < st->n_inst; ++i) log_fid_out[i] = after[i] - before[i];
  return NNE_OK;
}

nne_status nne_entropy(nne_state* st, double* S_out) {
  if (!st || !S_out) return set_error(NNE_ERR_ARG, "nne_entropy: bad arguments");
  if (st->n < 2) return NNE_OK;
  DeviceGuard dg(st->ctx->device);
  const size_t bytes = sizeof(double) * (size_t)st->n_inst * (st->n - 1);
  double* dS = nullptr;
  NNE_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&dS), bytes, st->ctx->stream));
  nne_status rc = st->dtype == NNE_C64 ? entropy_sweep<float>(st, dS) : entropy_sweep<double>(st, dS);
  cudaError_t ce = cudaSuccess;
  if (rc == NNE_OK) ce = cudaMemcpyAsync(S_out, dS, bytes, cudaMemcpyDeviceToHost, st->ctx->stream);
  cudaFreeAsync(dS, st->ctx->stream);
  if (rc != NNE_OK) return rc;
  if (ce != cudaSuccess) return set_cuda_error(ce, "cudaMemcpyAsync", __FILE__, __LINE__);
  return read_err(st);
}

nne_status nne_expect(nne_state* st, int n_obs, const uint8_t* paulis, double* re_out, double* im_out,
                      double* log_fid_out) {
  if (!st || n_obs < 0 || (n_obs > 0 && (!paulis || !re_out || !im_out)))
    return set_error(NNE_ERR_ARG, "nne_expect: bad arguments");
  DeviceGuard dg(st->ctx->device);
  const int n = st->n;
  std::vector<int> first(std::max(n_obs, 1), -1), last(std::max(n_obs, 1), -1);
  for (int o = 0; o < n_obs; ++o)
    for (int k = 0; k < n; ++k) {
      const int p = paulis[(size_t)o * n + k];
      if (p > 3) return set_error(NNE_ERR_ARG, "pauli code %d at (%d, %d)", p, o, k);
      if (p) {
        if (first[o] < 0) first[o] = k;
        last[o] = k;
      }
    }
  // strings spanning three or more sites take the carried-vector kernel
  std::vector<int> general;
  for (int o = 0; o < n_obs; ++o)
    if (first[o] >= 0 && last[o] - first[o] > 1) general.push_back(o);
  const int n_general = (int)general.size();
  cudaStream_t s = st->ctx->stream;
  void *dp = nullptr, *df = nullptr, *dl = nullptr, *dout = nullptr, *dgen = nullptr, *dv = nullptr;
  const size_t bp = (size_t)std::max(n_obs, 1) * n, bf = sizeof(int) * std::max(n_obs, 1),
               bo = sizeof(double) * 2 * (size_t)std::max(n_obs, 1) * st->n_inst,
               bv = sizeof(double) * 2 * 2 * 4 * (size_t)n * st->dmax * st->n_inst;
  NNE_CUDA_TRY(cudaMallocAsync(&dp, bp, s));
  NNE_CUDA_TRY(cudaMallocAsync(&df, bf, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dl, bf, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dgen, bf, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dout, bo, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dv, bv, s));
  std::vector<double> hout(2 * (size_t)std::max(n_obs, 1) * st->n_inst);
  cudaError_t e = cudaMemcpyAsync(st->d_dims, st->dims.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_obs > 0) e = cudaMemcpyAsync(dp, paulis, (size_t)n_obs * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(df, first.data(), bf, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dl, last.data(), bf, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_general > 0)
    e = cudaMemcpyAsync(dgen, general.data(), sizeof(int) * n_general, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = st->dtype == NNE_C64
            ? expect_sweep<float>(s, n, st->d_dims, (const void* const*)st->d_site, st->d_stride, st->n_inst, st->dmax,
                                  n_obs, (const uint8_t*)dp, (const int*)df, (const int*)dl, (const int*)dgen,
                                  n_general, st->d_env, st->d_envscale, (double*)dv, (double*)dout)
            : expect_sweep<double>(s, n, st->d_dims, (const void* const*)st->d_site, st->d_stride, st->n_inst,
                                   st->dmax, n_obs, (const uint8_t*)dp, (const int*)df, (const int*)dl,
                                   (const int*)dgen, n_general, st->d_env, st->d_envscale, (double*)dv, (double*)dout);
  if (e == cudaSuccess && n_obs > 0)
    e = cudaMemcpyAsync(hout.data(), dout, sizeof(double) * 2 * (size_t)n_obs * st->n_inst, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && log_fid_out)
    e = cudaMemcpyAsync(log_fid_out, st->d_logfid, sizeof(double) * st->n_inst, cudaMemcpyDeviceToHost, s);
  nne_status rc = NNE_OK;
  if (e != cudaSuccess) rc = set_cuda_error(e, "nne_expect", __FILE__, __LINE__);
  if (rc == NNE_OK) rc = read_err(st);
  cudaFreeAsync(dp, s);
  cudaFreeAsync(df, s);
  cudaFreeAsync(dl, s);
  cudaFreeAsync(dgen, s);
  cudaFreeAsync(dout, s);
  cudaFreeAsync(dv, s);
  if (rc != NNE_OK) return rc;
  for (int i = 0; i < st->n_inst; ++i)
    for (int o = 0; o < n_obs; ++o) {
      re_out[(size_t)i * n_obs + o] = hout[2 * ((size_t)i * n_obs + o)];
      im_out[(size_t)i * n_obs + o] = hout[2 * ((size_t)i * n_obs + o) + 1];
    }
  return NNE_OK;
}

nne_status nne_extrapolate(nne_ctx* ctx, int n_lambda, const double* lambdas, const double* values,
                           const double* log_fid, int n_obs, int method, int degree, double lambda_star,
                           const double* y_zero, double* out, int32_t* per_obs_status) {
  if (!ctx || n_lambda < 1 || n_lambda > 64 || !lambdas || !values || n_obs < 0 || !out || !per_obs_status ||
      method < 0 || method > 2 || (method == NNE_FIT_POLY && (degree < 1 || degree > 15)))
    return set_error(NNE_ERR_ARG, "nne_extrapolate: bad arguments");
  if (n_obs == 0) return NNE_OK;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = ctx->stream;
  double *dl = nullptr, *dv = nullptr, *df = nullptr, *dy = nullptr, *dout = nullptr;
  int* dst = nullptr;
  NNE_CUDA_TRY(cudaMallocAsync(&dl, sizeof(double) * n_lambda, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dv, sizeof(double) * n_lambda * (size_t)n_obs, s));
  NNE_CUDA_TRY(cudaMallocAsync(&df, sizeof(double) * n_lambda, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dy, sizeof(double) * (size_t)n_obs, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dout, sizeof(double) * (size_t)n_obs, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dst, sizeof(int) * (size_t)n_obs, s));
  cudaError_t e = cudaMemcpyAsync(dl, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dv, values, sizeof(double) * n_lambda * (size_t)n_obs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && log_fid) e = cudaMemcpyAsync(df, log_fid, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && y_zero) e = cudaMemcpyAsync(dy, y_zero, sizeof(double) * n_obs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = extrapolate_fit(s, n_lambda, dl, dv, log_fid ? df : nullptr, n_obs, method, degree, lambda_star,
                        y_zero ? dy : nullptr, dout, dst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * n_obs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(per_obs_status, dst, sizeof(int) * n_obs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  nne_status rc = e == cudaSuccess ? NNE_OK : set_cuda_error(e, "nne_extrapolate", __FILE__, __LINE__);
  cudaFreeAsync(dl, s);
  cudaFreeAsync(dv, s);
  cudaFreeAsync(df, s);
  cudaFreeAsync(dy, s);
  cudaFreeAsync(dout, s);
  cudaFreeAsync(dst, s);
  return rc;
}

nne_status nne_extrapolate_ladder(nne_ctx* ctx, int k, int n_lambda, const double* lambdas, const double* values,
                                  const double* log_fid, int n_obs, int method, int degree, double lambda_star,
                                  const double* y_zero, double* out, int32_t* per_obs_status, double* obar_out,
                                  uint8_t* conv_out) {
  if (!ctx || k < 1 || k > 64 || n_lambda < 1 || n_lambda > 64 || !lambdas || !values || !log_fid || n_obs < 0 ||
      !out || !per_obs_status || method < 0 || method > 2 || (method == NNE_FIT_POLY && (degree < 1 || degree > 15)))
    return set_error(NNE_ERR_ARG, "nne_extrapolate_ladder: bad arguments");
  if (n_obs == 0) return NNE_OK;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = ctx->stream;
  const size_t cells = (size_t)n_lambda * n_obs;
  double *dl = nullptr, *dv = nullptr, *df = nullptr, *dy = nullptr, *dob = nullptr, *dout = nullptr;
  uint8_t* dc = nullptr;
  int* dst = nullptr;
  NNE_CUDA_TRY(cudaMallocAsync(&dl, sizeof(double) * n_lambda, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dv, sizeof(double) * k * cells, s));
  NNE_CUDA_TRY(cudaMallocAsync(&df, sizeof(double) * k * (size_t)n_lambda, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dy, sizeof(double) * (size_t)n_obs, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dob, sizeof(double) * cells, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dc, cells, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dout, sizeof(double) * (size_t)n_obs, s));
  NNE_CUDA_TRY(cudaMallocAsync(&dst, sizeof(int) * (size_t)n_obs, s));
  cudaError_t e = cudaMemcpyAsync(dl, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dv, values, sizeof(double) * k * cells, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(df, log_fid, sizeof(double) * k * (size_t)n_lambda, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && y_zero) e = cudaMemcpyAsync(dy, y_zero, sizeof(double) * n_obs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = extrapolate_ladder(s, k, n_lambda, dl, dv, df, n_obs, method, degree, lambda_star, y_zero ? dy : nullptr, dob,
                           dc, dout, dst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * n_obs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(per_obs_status, dst, sizeof(int) * n_obs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && obar_out) e = cudaMemcpyAsync(obar_out, dob, sizeof(double) * cells, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && conv_out) e = cudaMemcpyAsync(conv_out, dc, cells, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  nne_status rc = e == cudaSuccess ? NNE_OK : set_cuda_error(e, "nne_extrapolate_ladder", __FILE__, __LINE__);
  cudaFreeAsync(dl, s);
  cudaFreeAsync(dv, s);
  cudaFreeAsync(df, s);
  cudaFreeAsync(dy, s);
  cudaFreeAsync(dob, s);
  cudaFreeAsync(dc, s);
  cudaFreeAsync(dout, s);
  cudaFreeAsync(dst, s);
  return rc;
}

nne_status nne_reset_state(nne_state* st, const uint8_t* init_bits) {
  if (!st) return set_error(NNE_ERR_ARG, "null state");
  DeviceGuard dg(st->ctx->device);
  cudaStream_t s = st->ctx->stream;
  if (init_bits) {
    for (int k = 0; k < st->n; ++k) st->bits[k] = init_bits[k] ? 1 : 0;
    NNE_CUDA_TRY(cudaMemcpyAsync(st->d_bits, st->bits.data(), st->n, cudaMemcpyHostToDevice, s));
  }
  cudaError_t e = st->dtype == NNE_C64
                      ? product_state<float>(s, st->n, (void* const*)st->d_site, st->d_stride, st->n_inst, st->d_bits)
                      : product_state<double>(s, st->n, (void* const*)st->d_site, st->d_stride, st->n_inst, st->d_bits);
  if (e != cudaSuccess) return set_cuda_error(e, "product_state", __FILE__, __LINE__);
  NNE_CUDA_TRY(cudaMemsetAsync(st->d_lognorm, 0, sizeof(double) * 2 * st->n_inst, s));
  NNE_CUDA_TRY(cudaMemsetAsync(st->d_err, 0, sizeof(int), s));
  std::fill(st->dims.begin(), st->dims.end(), 1);
  st->centre = 0;
  return NNE_OK;
}

void nne_set_option(int option, int value) {
  if (option == NNE_OPT_TENSOR_CORES) set_tensor_cores(value);
  if (option == NNE_OPT_SUBBATCHES) g_substreams = value < 1 ? 1 : (value > 8 ? 8 : value);
  if (option == NNE_OPT_SERIAL_LAYERS) g_serial_layers = value ? 1 : 0;
  if (option == NNE_OPT_EIG_FP64) g_eig_fp64 = value ? 1 : 0;
  if (option == NNE_OPT_GEMM_TMA) {
    set_gemm_tma(value);
    if (value) set_tma_variant(value);
  }
  if (option == NNE_OPT_TEST_WAIT_LIMIT) set_tc_wait_limit(value);
  if (option == NNE_OPT_SWEEP_CLUSTER) set_sweep_cluster(value);
}

nne_status nne_cgemm_c64(nne_ctx* ctx, int op_a, int op_b, int M, int N, int K, const float* alpha, const void* A,
                         int lda, long long stride_a, const void* B, int ldb, long long stride_b, const float* beta,
                         void* C, int ldc, long long stride_c, int batch) {
  if (!ctx || !alpha || !beta || !A || !B || !C || M < 0 || N < 0 || K < 0 || batch < 0 || op_a < 0 || op_a > 1 ||
      op_b < 0 || op_b > 1)
    return set_error(NNE_ERR_ARG, "nne_cgemm_c64: bad arguments");
  DeviceGuard dg(ctx->device);
  cudaError_t e = cgemm<float>(ctx->stream, op_a, op_b, M, N, K, mk<float>(alpha[0], alpha[1]),
                               reinterpret_cast<const cx<float>*>(A), stride_a, lda,
                               reinterpret_cast<const cx<float>*>(B), stride_b, ldb, mk<float>(beta[0], beta[1]),
                               reinterpret_cast<cx<float>*>(C), stride_c, ldc, batch);
  if (e != cudaSuccess) return set_cuda_error(e, "nne_cgemm_c64", __FILE__, __LINE__);
  int t = 0;
  int* te = tc_error_ptr();
  if (te) NNE_CUDA_TRY(cudaMemcpyAsync(&t, te, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  NNE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (t != 0) {
    // reported once: the word is cleared so that the next call starts clean
    NNE_CUDA_TRY(cudaMemsetAsync(te, 0, sizeof(int), ctx->stream));
    NNE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return set_error(t, "tensor-core GEMM reported status %d (a bounded wait expired)", t);
  }
  return NNE_OK;
}

nne_status nne_sync(nne_state* st) {
  if (!st) return set_error(NNE_ERR_ARG, "null state");
  DeviceGuard dg(st->ctx->device);
  return read_err(st);
}

nne_status nne_state_info(nne_state* st, int* dims_out, int* centre_out, double* log_norm_out, double* log_fid_out) {
  if (!st) return set_error(NNE_ERR_ARG, "null state");
  DeviceGuard dg(st->ctx->device);
  if (log_norm_out)
    NNE_CUDA_TRY(cudaMemcpyAsync(log_norm_out, st->d_lognorm, sizeof(double) * st->n_inst, cudaMemcpyDeviceToHost,
                                 st->ctx->stream));
  if (log_fid_out)
    NNE_CUDA_TRY(cudaMemcpyAsync(log_fid_out, st->d_logfid, sizeof(double) * st->n_inst, cudaMemcpyDeviceToHost,
                                 st->ctx->stream));
  nne_status rc = read_err(st);
  if (rc != NNE_OK) return rc;
  if (dims_out)
    for (int k = 0; k <= st->n; ++k) dims_out[k] = st->dims[k];
  if (centre_out) *centre_out = st->centre;
  return NNE_OK;
}

nne_status nne_state_read_site(nne_state* st, int inst, int k, void* host_out, size_t cap_bytes) {
  if (!st || inst < 0 || inst >= st->n_inst || k < 0 || k >= st->n || !host_out)
    return set_error(NNE_ERR_ARG, "nne_state_read_site: bad arguments");
  DeviceGuard dg(st->ctx->device);
  const size_t bytes = (size_t)st->dims[k] * 4 * st->dims[k + 1] * st->esz;
  if (cap_bytes < bytes) return set_error(NNE_ERR_ARG, "buffer too small: %zu < %zu", cap_bytes, bytes);
  NNE_CUDA_TRY(cudaMemcpyAsync(host_out, st->site[k] + (size_t)inst * st->sstride[k] * st->esz, bytes,
                               cudaMemcpyDeviceToHost, st->ctx->stream));
  return read_err(st);
}

nne_status nne_state_write_site(nne_state* st, int inst, int k, int dl, int dr, const void* host_in) {
  if (!st || inst < 0 || inst >= st->n_inst || k < 0 || k >= st->n || !host_in || dl < 1 || dr < 1 ||
      dl > st->cap[k] || dr > st->cap[k + 1])
    return set_error(NNE_ERR_ARG, "nne_state_write_site: bad arguments (dims above capacity?)");
  DeviceGuard dg(st->ctx->device);
  const size_t bytes = (size_t)dl * 4 * dr * st->esz;
  NNE_CUDA_TRY(cudaMemcpyAsync(st->site[k] + (size_t)inst * st->sstride[k] * st->esz, host_in, bytes,
                               cudaMemcpyHostToDevice, st->ctx->stream));
  st->dims[k] = dl;
  st->dims[k + 1] = dr;
  return read_err(st);
}

nne_status nne_state_set_centre(nne_state* st, int centre) {
  if (!st || centre < 0 || centre >= st->n) return set_error(NNE_ERR_ARG, "bad centre");
  st->centre = centre;
  return NNE_OK;
}

nne_status nne_state_set_log(nne_state* st, const double* log_norm, const double* log_fid) {
  if (!st) return set_error(NNE_ERR_ARG, "nne_state_set_log: null state");
  DeviceGuard dg(st->ctx->device);
  const size_t b = sizeof(double) * st->n_inst;
  if (log_norm) NNE_CUDA_TRY(cudaMemcpyAsync(st->d_lognorm, log_norm, b, cudaMemcpyHostToDevice, st->ctx->stream));
  if (log_fid) NNE_CUDA_TRY(cudaMemcpyAsync(st->d_logfid, log_fid, b, cudaMemcpyHostToDevice, st->ctx->stream));
  NNE_CUDA_TRY(cudaStreamSynchronize(st->ctx->stream));
  return NNE_OK;
}

}  // extern "C"
