// Declarations of the device kernels' host launchers (all enqueue on `st`).
#pragma once
#include <algorithm>
#include <vector>
#include "common.cuh"

namespace nne {

// ---- k_blas.cu
template <typename R>
cudaError_t cgemm(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<R> alpha, const cx<R>* A, long long sA,
                  int lda, const cx<R>* B, long long sB, int ldb, cx<R> beta, cx<R>* C, long long sC, int ldc,
                  int batch);
template <typename R>
cudaError_t apply_superop(cudaStream_t st, cx<R>* X, long long sX, int dl, int dr, const double* G, long long sG,
                          int batch);
template <typename R>
cudaError_t sumsq_partial(cudaStream_t st, const cx<R>* X, long long sX, long long count, double* out, int parts,
                          int batch);
cudaError_t finish_gate(cudaStream_t st, const double* kept_parts, const double* total_parts, const double* disc_parts,
                        int parts, int batch, double* scale, double* log_norm, double* log_fid, int* err);
template <typename R>
cudaError_t scale_batched(cudaStream_t st, cx<R>* X, long long sX, long long count, const double* scale, int batch);
template <typename R>
cudaError_t transpose(cudaStream_t st, bool conj_, const cx<R>* X, long long sX, int rows, int cols, int ldx,
                      cx<R>* Y, long long sY, int ldy, int batch);
template <typename R>
cudaError_t conj_inplace(cudaStream_t st, cx<R>* X, long long sX, long long count, int batch);
template <typename R>
cudaError_t identity(cudaStream_t st, cx<R>* X, long long sX, int rows, int cols, int batch);
template <typename R>
cudaError_t copy_batched(cudaStream_t st, const cx<R>* X, long long sX, cx<R>* Y, long long sY, long long count,
                         int batch);

// Y[z] (rows x cols, ld ldy) = X[z] (rows x cols, ld ldx).
template <typename R>
cudaError_t copy_2d(cudaStream_t st, const cx<R>* X, long long sX, int ldx, cx<R>* Y, long long sY, int ldy, int rows,
                    int cols, int batch);

template <typename R>
cudaError_t product_state(cudaStream_t st, int n, void* const* d_site, const long long* d_stride, int n_inst,
                          const uint8_t* d_bits);

template <typename R>
cudaError_t fix_columns(cudaStream_t st, cx<R>* W, long long sW, int n, int r, int batch);
template <typename R>
cudaError_t fix_qr(cudaStream_t st, cx<R>* Q, long long sQ, int m, int k, cx<R>* Rm, long long sR, int n, int batch);

// ---- k_gemm_tc.cu (complex64 on tcgen05, split TF32)
cudaError_t cgemm_tc(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<float> alpha, const cx<float>* A,
                     long long sA, int lda, const cx<float>* B, long long sB, int ldb, cx<float> beta, cx<float>* C,
                     long long sC, int ldc, int batch);
void set_tensor_cores(int on);
int tensor_cores_enabled();
int* tc_error_ptr();
// C[z] = alpha sum_s P[z S + s] + beta C[z] over the S K-slices of a split GEMM (M x N each, ld N).
cudaError_t cgemm_split_reduce(cudaStream_t st, int M, int N, int S, const float2* P, float2 alpha, float2 beta,
                               float2* C, long long sC, int ldc, int batch);
// ---- k_gemm_tma.cu (complex64 on tcgen05, operands pre-split into TF32 planes and fed by TMA)
cudaError_t cgemm_tma(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<float> alpha, const cx<float>* A,
                      long long sA, int lda, const cx<float>* B, long long sB, int ldb, cx<float> beta, cx<float>* C,
                      long long sC, int ldc, int batch);
bool cgemm_tma_available();
// Split op(A) (M x K) into TF32 planes now and let this host thread's later
// cgemm_tma calls on `st` with exactly this A, op, shape and batch reuse them
// (A must not change until tma_release(st), which frees the planes).
cudaError_t tma_hold_a(cudaStream_t st, int opA, int M, int K, const cx<float>* A, long long sA, int lda, int batch);
void tma_release(cudaStream_t st);
// Pipeline variant of the TMA GEMM (1: 128-byte swizzle, 2 stages; 2: 64-byte swizzle, 4 stages).
void set_tma_variant(int v);
// Test hook: bound (polls) of the TMA GEMM's pipeline waits; 0 restores the default.
void set_tc_wait_limit(long long polls);
void set_gemm_tma(int on);
int gemm_tma_enabled();

// ---- k_linalg.cu
// Workspace sizes (elements) for eigh_top on n x n matrices with r wanted vectors.
struct EighWork {
  long long cx_elems;    // complex R elements
  long long re_elems;    // real R elements
  long long u8_elems;    // bytes
};
EighWork eigh_workspace(int n, int r);
// Top-r eigenvectors of the Hermitian H[z] (n x n, row-major, overwritten),
// written as U[z] (n x r, row-major, columns ordered by decreasing eigenvalue)
// with orthonormal columns.  Workspace per batch entry as eigh_workspace.
template <typename R>
cudaError_t eigh_top(cudaStream_t st, cx<R>* H, long long sH, int n, int r, cx<R>* U, long long sU, void* cx_ws,
                     void* re_ws, void* u8_ws, int batch, int* err);

// Bytes per matrix of eigh_top_mixed's three workspaces.
struct MixedEighWork {
  size_t cx_bytes, re_bytes, u8_bytes;
};
MixedEighWork eigh_mixed_workspace(int n, int r);
// Top-r eigenvectors of complex64 Hermitian matrices with the reduction and the
// tridiagonal eigenproblem in float64 (see k_linalg.cu); same layout as eigh_top.
cudaError_t eigh_top_mixed(cudaStream_t st, cx<float>* H, long long sH, int n, int r, cx<float>* U, long long sU,
                           void* cx_ws, void* re_ws, void* u8_ws, int batch, int* err);

// Entropy -sum p ln p of the normalised eigenvalues p of each Hermitian
// positive semi-definite H[z] (n x n, overwritten), written to S[z * sS]:
// with H the Gram matrix of a canonical-form centre tensor it is the MPO
// entanglement entropy of that bond.  Workspace as eigh_workspace(n, n).
template <typename R>
cudaError_t gram_entropy(cudaStream_t st, cx<R>* H, long long sH, int n, void* cx_ws, void* re_ws, int batch,
                         double* S, long long sS);

template <typename R>
int smem_cluster_size(int n);
template <typename R>
cudaError_t tridiag_smem(cudaStream_t st, const cx<R>* H, long long sH, int n, R* d, cx<R>* e, int ldde, cx<R>* Vh,
                         long long sVh, int batch);
template <typename R>
cudaError_t backtransform_wy(cudaStream_t st, const cx<R>* Vh, long long sVh, int n, const R* Z, long long sZ,
                             const cx<R>* phi, int ldde, int r, cx<R>* U, long long sU, cx<R>* Tw, cx<R>* wy_ws,
                             int batch);

// ---- k_wy.cu
// C[z] <- C[z] - V op(T) V^H C[z] for bw <= 32 Householder vectors in compact-WY
// form (op(T) = T^H if t_adj).  V is K x bw with rows at V + i * ldv, or, if
// v_rows, given as V^H (bw x K, rows at V + c * ldv).  T is bw x bw (ld ldt),
// C is K x N (ld ldc).  ws holds batch * wy_workspace(N) elements.
long long wy_workspace(int N);
template <typename R>
cudaError_t wy_apply(cudaStream_t st, bool v_rows, const cx<R>* V, long long sV, int ldv, const cx<R>* T,
                     long long sT, int ldt, bool t_adj, int bw, int K, int N, cx<R>* C, long long sC, int ldc,
                     cx<R>* ws, int batch);

struct QrWork {
  long long cx_elems;
};
QrWork qr_workspace(int m, int n);
// Householder QR of A[z] (m x n, row-major, ld = n, overwritten): writes
// Q[z] (m x k, ld = k, k = min(m, n)) with orthonormal columns and, if Rout
// is not null, Rout[z] (k x n, ld = n, zero below the diagonal), A = Q R.
template <typename R>
cudaError_t qr(cudaStream_t st, cx<R>* A, long long sA, int m, int n, cx<R>* Q, long long sQ, cx<R>* Rout,
               long long sR, void* cx_ws, int batch);

// ---- k_sweep.cu
// <P> for n_obs Pauli strings on every instance (see nne_expect).
struct SweepSites {
  const void* const* site;   // per site k: pointer to instance 0's tensor
  const long long* stride;   // per site k: elements between instances
};
// d_env: n_inst x 2 x (n + 1) x max_dim complex double; d_envscale: n_inst x 2 x (n + 1);
// d_vecs: n_inst x 2 x n x 4 x max_dim complex double; d_general lists the n_general
// strings whose support spans three or more sites.
template <typename R>
cudaError_t expect_sweep(cudaStream_t st, int n, const int* d_dims, const void* const* d_site,
                         const long long* d_stride, int n_inst, int max_dim, int n_obs, const uint8_t* d_paulis,
                         const int* d_first, const int* d_last, const int* d_general, int n_general, double* d_env,
                         double* d_envscale, double* d_vecs, double* d_out /* n_inst x n_obs x 2 */);
// Cluster size of the environment sweep: 0 picks it from occupancy, 1..16 forces it.
void set_sweep_cluster(int cs);

// ---- k_superop.cu
cudaError_t build_superops(cudaStream_t st, int n_gates, const double* d_U, int n_inst, const double* d_rates,
                           double* d_G, double* d_Snoise /* n_inst x 256 complex128 scratch */);
// Gate-dependent Pauli channels: d_pr n_gates x 2 x 16 (c0, c1), d_lam n_inst.
cudaError_t build_pauli_superops(cudaStream_t st, int n_gates, const double* d_U, const double* d_pr, int n_inst,
                                 const double* d_lam, double* d_G);

// ---- k_fit.cu
cudaError_t extrapolate_fit(cudaStream_t st, int n_lambda, const double* d_lam, const double* d_vals,
                            const double* d_logfid, int n_obs, int method, int degree, double lambda_star,
                            const double* d_yzero, double* d_out, int* d_status);

// Fidelity extrapolation over a bond-dimension ladder, then the fit (see nne_extrapolate_ladder).
cudaError_t extrapolate_ladder(cudaStream_t st, int k, int n_lambda, const double* d_lam, const double* d_vals,
                               const double* d_logfid, int n_obs, int method, int degree, double lambda_star,
                               const double* d_yzero, double* d_obar, uint8_t* d_conv, double* d_out, int* d_status);

// ---- nne_api.cu
// Bond capacities min(chi, 4^k, 4^(n-k)), k = 0..n.
std::vector<int> bond_caps(int n, int chi);
// Device bytes a state (plus its sketch buffers when sketch_cols > 0) allocates.
size_t state_bytes(int n, int chi, int n_inst, int dtype, int sketch_rows, int sketch_cols);

// Device ordinal and stream of a context (defined with the context in nne_api.cu).
void ctx_device_stream(const nne_ctx* ctx, int* device, cudaStream_t* stream);

}  // namespace nne
