/*
 * libnne -- C ABI of the GB300 (sm_103a) hot path of non-zero noise
 * extrapolation (NZNE, arXiv 2501.13237).
 *
 * What the library computes (paper sections in brackets):
 *   - a vectorised density operator |rho>> stored as an MPS with local
 *     dimension 4 per qubit, |i><j| -> |(i,j)>>, s = 2 i + j        [Sec. 2.1.1]
 *   - noisy circuit evolution: each two-qubit gate U is post-composed with a
 *     channel C (U -> C o U) and applied as one 16x16 superoperator G;
 *     after each gate the state is replaced by the closest bond-chi state of
 *     Frobenius norm 1; the partial fidelity f_l of that step is recorded and
 *     F = prod f_l is accumulated                              [Secs. 2.1.2, 2.2.1]
 *   - Pauli expectation values <P> = Tr(P rho)/Tr(rho) read off by an exact
 *     contraction of the network                               [Sec. 2.2.3]
 *   - the extrapolation of <O>_lambda across noise levels to a target
 *     lambda* (weighted log-linear, three-parameter exponential, or
 *     polynomial fit)                                          [Sec. 2.2.3 (B), App. B.2]
 *
 * Conventions shared by every entry point
 *   - Complex numbers are (re, im) pairs of float (NNE_C64) or double
 *     (NNE_C128), interleaved.
 *   - A state holds n_inst independent instances (normally one per noise
 *     level lambda) of the same circuit: same n, same chi, same gate
 *     positions, per-instance superoperators.
 *   - Site tensor k of an instance is M[a][s][b] (row-major, b fastest) with
 *     shape (dims[k], 4, dims[k+1]); dims[0] = dims[n] = 1.
 *   - Superoperators G are 16x16 complex128, row-major, row index
 *     4*s1' + s2', column index 4*s1 + s2, qubit q (s1) the left qubit.
 *   - Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z.
 *   - Host pointers are owned by the caller and must stay valid until the
 *     call returns; device pointers are owned by the caller and must stay
 *     valid until the work enqueued by the call has completed on the
 *     context's stream.  The library owns all state and workspace memory.
 *   - Errors are returned as nne_status; nothing throws or aborts across the
 *     ABI.  nne_last_error() gives a one-line description of the most recent
 *     failure on the calling thread.  Calls on one context are not
 *     thread-safe (a server serialises them itself).
 */
#ifndef NNE_H
#define NNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nne_status;
#define NNE_OK 0
#define NNE_PENDING 1
#define NNE_ERR_ARG (-1)
#define NNE_ERR_OOM (-2)
#define NNE_ERR_CUDA (-3)
#define NNE_ERR_NOCONV (-4)
#define NNE_ERR_TIMEOUT (-5)
#define NNE_ERR_NOFIT (-6)
#define NNE_ERR_UNIMPL (-7)
#define NNE_ERR_CANCELLED (-8)

typedef enum { NNE_C64 = 0, NNE_C128 = 1 } nne_dtype;

/* Truncation algorithm of a gate step.
 * NNE_TRUNC_EXACT: eigenvectors of the full (4 chi_l)^2 Gram matrix X X^dagger
 *   (or X^dagger X), i.e. the exact best rank-chi approximation (Eckart-Young).
 * NNE_TRUNC_RSVD: randomized range finder with q power iterations
 *   (Q <- orth(X X^H Q)) and a Rayleigh-Ritz step on a (chi + p)-dimensional
 *   sketch (Halko, Martinsson & Tropp 2011); the sketch matrix is an input
 *   (nne_set_sketch).  Equals
 *   NNE_TRUNC_EXACT whenever chi + p covers the rank bound of the gate. */
typedef enum { NNE_TRUNC_EXACT = 0, NNE_TRUNC_RSVD = 1 } nne_trunc;

/* Fit methods of nne_extrapolate. */
typedef enum { NNE_FIT_POLY = 0, NNE_FIT_EXP_LOGLIN = 1, NNE_FIT_EXP3 = 2 } nne_fit;

typedef struct nne_ctx nne_ctx;
typedef struct nne_state nne_state;

/* Context: one CUDA device and one stream.
 *   device           CUDA ordinal made current by every call on this context.
 *   cuda_stream      cudaStream_t (NULL = the legacy default stream).
 *   hbm_budget_bytes cap on the memory states created on this context may
 *                    allocate (0 = no cap); exceeding it gives NNE_ERR_OOM. */
nne_status nne_ctx_create(int device, void* cuda_stream, size_t hbm_budget_bytes, nne_ctx** out);
void nne_ctx_destroy(nne_ctx* ctx);
/* Bytes currently allocated by states of this context. */
size_t nne_ctx_bytes_in_use(const nne_ctx* ctx);
const char* nne_last_error(void);

/* a1 -- fused gate+channel superoperators (Sec. 2.2.1 eq. U -> C o U; App. C.2.1).
 * G[i][g] = S_depol1 S_dephase S_ampdamp S_depol2 (U_g (x) conj(U_g)) for
 * instance i and gate g, where each S is sum_K K (x) conj(K) of the channel
 * at the strengths rates[i] = (p_depol2, gamma, p_dephase, p_depol1):
 *   depol2   K0 = sqrt(1 - 15p/16) I, K_ab = sqrt(p/16) sigma_a sigma_b
 *            (rho -> (1-p) rho + p I/4; App. C.2.1)
 *   ampdamp  K0 = diag(1, sqrt(1-gamma)), K1 = sqrt(gamma)|0><1|, on both qubits
 *   dephase  sqrt(1-p) I, sqrt(p) Z on both qubits
 *   depol1   sqrt(1-p) I, sqrt(p/3){X,Y,Z} on both qubits
 * U     n_gates x 4 x 4 complex128 (row-major, basis |b_q b_{q+1}>, b_q the
 *       more significant bit), in host or device memory (detected).
 * rates n_inst x 4 doubles in host or device memory; every strength in
 *       [0, 1] (depol2 <= 16/15).  Ranges are checked only for host rates.
 * G_out device, n_inst x n_gates x 256 complex128.
 * Computed in float64 on the device; enqueued on the context stream. */
nne_status nne_build_superops(nne_ctx* ctx, int n_gates, const double* U, int n_inst,
                              const double* rates, void* G_out);

/* a1 for gate-dependent Pauli noise (cat-qubit errors, App. C.2.2; matchgate
 * depolarizing noise, App. C.3.1; two-qubit depolarizing, App. C.2.1, is the
 * case p_ab = lambda/16): G[i][g] = S_P (U_g (x) conj(U_g)) with
 * S_P = sum_ab p_ab K_ab (x) conj(K_ab), K_ab = sigma_a (x) sigma_b (a on the
 * left qubit q, b on q+1; 0 = I, 1 = X, 2 = Y, 3 = Z) and
 * p_ab = c0[g][4a+b] + lambdas[i] * c1[g][4a+b].
 * U           n_gates x 4 x 4 complex128 (as nne_build_superops);
 * pauli_rates n_gates x 2 x 16 doubles: c0 then c1 of each gate;
 * lambdas     n_inst doubles;
 * all three in host or device memory (detected).  With host pauli_rates and
 * lambdas every p_ab must lie in [0, 1] and each gate's 16 sum to 1 within
 * 1e-12, else NNE_ERR_ARG; device inputs are not checked.
 * G_out device, n_inst x n_gates x 256 complex128.  Float64 on the device;
 * synchronises the context stream when inputs are staged from the host. */
nne_status nne_build_pauli_superops(nne_ctx* ctx, int n_gates, const double* U,
                                    const double* pauli_rates, int n_inst,
                                    const double* lambdas, void* G_out);

/* State creation: n_inst instances of the product state |b><b| (Sec. 2.1.2:
 * the initial state is a product state), bond dimensions 1, orthogonality
 * centre on site 0, log-norm and log-fidelity 0.
 *   n_qubits >= 2, chi >= 1, n_inst >= 1; init_bits host uint8[n] (NULL = all 0).
 * Device memory is sized for bond capacities min(chi, 4^k, 4^(n-k)). */
nne_status nne_create_state(nne_ctx* ctx, int n_qubits, int chi, int n_inst, nne_dtype dtype,
                            nne_trunc trunc, const uint8_t* init_bits, nne_state** out);
void nne_destroy_state(nne_state* st);

/* Sketch matrix of NNE_TRUNC_RSVD: host complex (same precision as the state)
 * of rows x cols, rows >= 4*chi, cols = chi + oversampling; power_iters >= 0. */
nne_status nne_set_sketch(nne_state* st, const void* omega, int rows, int cols, int power_iters);

/* a2-a6 -- one layer of gates (Sec. 2.1.2 "Approximate emulation").
 * For each gate g in array order, on sites (q, q+1), q = left_qubit[g]:
 *   move the orthogonality centre to q (direction +1) or q+1 (direction -1)
 *   by QR / LQ steps; form theta = M_q M_{q+1} and theta' = G theta over
 *   (s1, s2); truncate X = theta' ((4 chi_l) x (4 chi_r)) to rank
 *   r = min(chi, 4 chi_l, 4 chi_r); keep the isometric factor on q (+1) or
 *   q+1 (-1) and the centre on the other site; normalise the centre to
 *   Frobenius norm 1 and add log|centre| to log_norm and
 *   log f_l = log(sum_{i<=r} s_i^2 / sum s_i^2) to log F.
 * left_qubit host int[n_gates], 0 <= q <= n-2.
 * G device, n_inst x n_gates x 256 complex128 (gate g of instance i at
 *   G + (i * n_gates + g) * 256).
 * Enqueued on the context stream; device-side failures surface at the next
 * nne_sync / nne_expect / nne_state_info. */
nne_status nne_apply_layer(nne_state* st, int n_gates, const int* left_qubit, const void* G,
                           int direction);

/* Canonical compression sweep to bond dimension chi_new (<= current chi):
 * centre to site 0, then left to right keep min(chi_new, .) singular
 * triplets per bond, normalise, accumulate log f per bond.  log_fid_out
 * (host double[n_inst] or NULL) receives the log F added by this call. */
nne_status nne_truncate(nne_state* st, int chi_new, double* log_fid_out);

/* a7 -- <P> = Tr(P rho)/Tr(rho) for each Pauli string (Sec. 2.2.3; exact
 * contraction of the network).  paulis host uint8 n_obs x n; re_out/im_out
 * host double n_inst x n_obs; log_fid_out host double[n_inst] or NULL
 * (log F of each instance).  Synchronises the context stream. */
nne_status nne_expect(nne_state* st, int n_obs, const uint8_t* paulis, double* re_out,
                      double* im_out, double* log_fid_out);

/* MPO entanglement entropy of every bond (App. A.1): S_l = -sum_i p_i ln p_i
 * with p_i = s_i^2 / sum_j s_j^2 over the Schmidt values s_i of the state
 * across the cut after qubit l, for l = 1 .. n-1.  Computed by a canonical
 * sweep: the centre moves to site 0, then right one site at a time (QR); at
 * site k the squared Schmidt values of the bond k | k+1 are the eigenvalues of
 * the centre tensor's Gram matrix, found by tridiagonalisation and bisection
 * in the state's precision, and S is summed in FP64.  The state itself is
 * unchanged; its centre ends on site n-1.  S_max (App. A.1) is the maximum of
 * a row.
 *   S_out host double n_inst x (n-1), caller-owned, row-major: S_out[i * (n-1) + k] is the
 *         entropy of instance i at the bond between qubits k and k+1.
 * The Gram matrices are formed in the state's precision, so squared Schmidt
 * values below about machine epsilon times the largest are not resolved
 * (complex64: ~1e-7), and a state written with nne_state_write_site must
 * keep its squared norm inside that precision's range (evolved states have
 * norm 1).  Synchronises the context stream; returns NNE_ERR_ARG for a null
 * argument, NNE_ERR_CUDA on a CUDA failure. */
nne_status nne_entropy(nne_state* st, double* S_out);

/* a8 -- noise extrapolation to lambda_star (Sec. 2.2.3 (B), App. B.2), FP64
 * on the device, one thread per observable.
 *   lambdas host double[n_lambda]; values host double n_lambda x n_obs;
 *   log_fid host double[n_lambda] (log F per level) or NULL (= 0);
 *   y_zero  host double[n_obs] (lambda = 0 values, the sign reference of
 *           criterion 3) or NULL (reference = smallest lambda);
 *   method NNE_FIT_POLY (degree >= 1), NNE_FIT_EXP_LOGLIN (criteria 2-3,
 *          weights F^2 exp(-20|lambda*-lambda|/d), fallback to EXP3 when
 *          fewer than two points survive), NNE_FIT_EXP3 (a e^{-b lambda} + c);
 *   out host double[n_obs]; per_obs_status host int32[n_obs]: NNE_OK or
 *          NNE_ERR_NOFIT (then out = the value at lambda* if lambda* was
 *          emulated, else NaN -- the paper's final fallback).
 * Returns NNE_OK unless an argument or CUDA call fails. */
nne_status nne_extrapolate(nne_ctx* ctx, int n_lambda, const double* lambdas, const double* values,
                           const double* log_fid, int n_obs, int method, int degree,
                           double lambda_star, const double* y_zero, double* out,
                           int32_t* per_obs_status);

/* Return a state to its initial product state |b><b| without reallocating:
 * bond dimensions 1, centre 0, log-norm and log F 0.  init_bits host uint8[n],
 * or NULL for the bits given at creation.  Enqueued on the context stream. */
nne_status nne_reset_state(nne_state* st, const uint8_t* init_bits);

/* The paper's two-step extrapolation over a bond-dimension ladder
 * D_1 < ... < D_k (Sec. 2.2.3 (A) and (B); App. B.1).
 *   values   k x n_lambda x n_obs: Re <O> emulated at each D_j and level (host);
 *   log_fid  k x n_lambda: log of the emulation fidelity at each D_j and level.
 * (A) per level and observable: least-squares line of <O> against F over the k
 *     rungs, evaluated at F = 1 (one rung: the value; equal F: their mean),
 *     written to obar_out (n_lambda x n_obs) when not NULL;
 *     criterion 1: the level stays when
 *     |(O_k - O_{k-1}) / (F_k - F_{k-1})| (1 - F_k) < |O_k| / 2
 *     (F_k = 1 passes; equal top fidelities pass only when O_k = O_{k-1}; one
 *     rung keeps every level), 0/1 in conv_out (n_lambda x n_obs) when not NULL.
 * (B) as nne_extrapolate on the levels passing criterion 1, with the top
 *     rung's fidelity as F^max and the dip size taken over all levels; when no
 *     fit is possible the status is NNE_ERR_NOFIT and the estimate is the top
 *     rung's value at lambda* (NaN if lambda* was not emulated).
 * Limits: k <= 64, n_lambda <= 64.  Synchronises the context stream. */
nne_status nne_extrapolate_ladder(nne_ctx* ctx, int k, int n_lambda, const double* lambdas, const double* values,
                                  const double* log_fid, int n_obs, int method, int degree, double lambda_star,
                                  const double* y_zero, double* out, int32_t* per_obs_status, double* obar_out,
                                  uint8_t* conv_out);

/* The fit of nne_extrapolate for callers that cannot allocate device memory
 * when they ask for it (no counterpart in the paper): a request loop whose HBM
 * budget is already committed to resident states, where a new cudaMalloc can
 * fail, or latency-critical code that cannot pay for cudaMalloc/cudaFree, which
 * may synchronise the device.  Same arguments, results and kernel as
 * nne_extrapolate, but the device-side copies of the inputs and outputs live
 * in one fixed array of about 0.55 MB compiled into the library (present on
 * every GPU that loads it until the process exits); nothing is allocated.
 * Limits: n_lambda <= 64 and n_obs <= 1024, larger sizes return NNE_ERR_ARG.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race; calls made one after
 * another are safe (each call waits for its results before returning).  The
 * looked-up address is kept for the life of the process, so the library must
 * not be used across a cudaDeviceReset of that device. */
nne_status nne_extrapolate_noalloc(nne_ctx* ctx, int n_lambda, const double* lambdas, const double* values,
                                   const double* log_fid, int n_obs, int method, int degree,
                                   double lambda_star, const double* y_zero, double* out,
                                   int32_t* per_obs_status);

/* Batched complex64 GEMM, C[z] = alpha op(A[z]) op(B[z]) + beta C[z] (row-major,
 * op 0 = N, 1 = conjugate transpose; matrix z at pointer + z * stride elements),
 * the same routine every gate step uses: tcgen05 tensor cores with split-TF32
 * products for large shapes, float32 SIMT otherwise.  Device pointers;
 * alpha/beta host (re, im).  Synchronises the context stream. */
nne_status nne_cgemm_c64(nne_ctx* ctx, int op_a, int op_b, int M, int N, int K, const float* alpha, const void* A,
                         int lda, long long stride_a, const void* B, int ldb, long long stride_b,
                         const float* beta, void* C, int ldc, long long stride_c, int batch);

/* Library options: NNE_OPT_TENSOR_CORES (default 1) selects the tcgen05 path of
 * complex64 GEMMs (0 = float32 SIMT everywhere, for comparisons).
 * NNE_OPT_SUBBATCHES (default 4, 1..8) is the number of sub-batches a state
 * created afterwards splits its instances into for nne_apply_layer: each
 * sub-batch's gate steps run on a stream of its own (forked from and joined
 * back to the context stream), so that the latency-bound kernels of one
 * overlap the GEMMs of another.  States whose largest bond is below 256 use
 * one stream (their kernels are small and splitting multiplies launches).
 * Results do not depend on it beyond the rounding of GEMM split choices.
 * NNE_OPT_SERIAL_LAYERS (default 0): when 1, nne_apply_layer runs all of a
 * state's instances as one batch on the context stream, whatever the state's
 * sub-batch count -- for per-launch timing of the kernels alone.
 * NNE_OPT_EIG_FP64 (default 1): complex64 states solve the truncation's
 * Hermitian eigenproblems (the Gram matrix of the exact truncation, the
 * Rayleigh-Ritz matrix of the subspace iteration, the centre compression)
 * with float64 quality: the Householder reduction in float64 (matrices that
 * fit a cluster's shared memory) or in double-float arithmetic on the
 * float32 pipes (larger ones; about 2^-46 relative), bisection and inverse
 * iteration in float64, the back-transformation in float32; 0 runs them in
 * float32 (about 1.5x the gate-step rate at chi = 512, with a float32
 * reduction's error of eps_32 times the largest eigenvalue, which turns the
 * eigenvectors next to a flat cut).  complex128 states always use float64.
 * NNE_OPT_GEMM_TMA (default 2): large complex64 GEMMs (M >= 128, N >= 64,
 * K >= 64) split their operands once into TF32 planes and run the TMA-fed
 * tcgen05 kernel, with 128-byte swizzled K rows in 2 stages (1) or 64-byte
 * rows in 4 stages (2, the default kernel); 0 keeps the earlier tensor-core
 * kernel that splits inside its producer warps (for comparisons).
 * NNE_OPT_TEST_WAIT_LIMIT (test hook, default 0): bound, in polls, of the
 * TMA GEMM's pipeline mbarrier waits; 0 is the default bound, a negative
 * value makes every such wait expire at once.  An expired wait makes the
 * kernel record NNE_ERR_TIMEOUT (reported once by the next nne_sync or
 * nne_cgemm_c64, then cleared) and return after waiting, with the full
 * bound, for its own copies and MMAs.
 * NNE_OPT_SWEEP_CLUSTER (default 0): CTAs per cluster of nne_expect's
 * environment sweep; 0 picks the size that covers the most SMs in the fewest
 * waves (occupancy query of each size), 1..16 forces a size (for tests and
 * comparisons; a size the GPU cannot schedule makes nne_expect fail).
 * Options are process-wide; set them while no other thread calls the library. */
#define NNE_OPT_TENSOR_CORES 0
#define NNE_OPT_SUBBATCHES 1
#define NNE_OPT_SERIAL_LAYERS 2
#define NNE_OPT_EIG_FP64 3
#define NNE_OPT_GEMM_TMA 4
#define NNE_OPT_TEST_WAIT_LIMIT 5
#define NNE_OPT_SWEEP_CLUSTER 6
void nne_set_option(int option, int value);

/* Wait for the state's enqueued work; returns the first device-side error. */
nne_status nne_sync(nne_state* st);

/* Host view of a state: dims_out int[n+1], centre_out, log_norm_out /
 * log_fid_out double[n_inst] (any may be NULL).  Synchronises. */
nne_status nne_state_info(nne_state* st, int* dims_out, int* centre_out, double* log_norm_out,
                          double* log_fid_out);
/* Copy site k of instance inst to/from host memory (shape dims[k] x 4 x dims[k+1],
 * element size 8 or 16 bytes).  nne_state_write_site sets the bond dims of
 * site k to (dl, dr); the caller keeps neighbouring sites consistent and
 * declares the orthogonality centre with nne_state_set_centre.  Synchronises. */
nne_status nne_state_read_site(nne_state* st, int inst, int k, void* host_out, size_t cap_bytes);
nne_status nne_state_write_site(nne_state* st, int inst, int k, int dl, int dr, const void* host_in);
nne_status nne_state_set_centre(nne_state* st, int centre);
/* Overwrite the accumulated log-norm and log F of every instance (host
 * double[n_inst] each, caller-owned; NULL leaves that one unchanged).  With
 * nne_state_info, nne_state_read_site / nne_state_write_site and
 * nne_state_set_centre this checkpoints and restores a state (no counterpart
 * in the paper).  Synchronises; NNE_ERR_ARG for a null state. */
nne_status nne_state_set_log(nne_state* st, const double* log_norm, const double* log_fid);

/* Instrumentation (no counterpart in the paper).
 * nne_kernel_launches: number of CUDA kernels this library has launched in
 *   the process so far (monotone counter).
 * nne_prof_enable: when on, every launch records a CUDA event pair on its
 *   stream, grouped by kernel class; nne_prof_collect synchronises on those
 *   events, writes total milliseconds, launch counts and algorithmic work
 *   (real flops for GEMM, reflector, QR-panel and tridiagonal classes, 0 where
 *   not tracked) per class (arrays of
 *   n_classes, any may be NULL) and clears the record.  Returns the number of
 *   classes.
 *   Classes: 0 GEMM, 1 superoperator epilogue, 2 tridiagonal reduction,
 *   3 bisection, 4 inverse iteration, 5 back-transform, 6 QR panel factor,
 *   7 block-reflector products (split-K), 8 elementwise/norms,
 *   9 environment sweep, 10 observable sweep, 11 superoperator build, 12 fit,
 *   13 tensor-core GEMM (work: 8 M N K real flops per complex GEMM; class 0
 *   is then the float32 SIMT GEMMs only). */
long long nne_kernel_launches(void);
void nne_prof_enable(int on);
int nne_prof_collect(double* ms_out, long long* count_out, double* work_out, int n_classes);

/* ---- Serving loop: whole extrapolation jobs, continuous batching ---------
 *
 * A job is the paper's problem instance [Sec. 2.2 problem statement, Sec. 3]:
 * a circuit C on a line of qubits, a noise family N(lambda) fixed by base
 * channel strengths scaled per level, the set of levels Lambda, observables
 * O and the target lambda*.  The server runs each job as one state with
 * n_lambda instances (gate steps, truncation to chi, expectation sweep) and
 * fits the levels to lambda* on the GPU.
 *
 * Workers: n_workers host threads, each with its own non-blocking CUDA stream
 * and context, take jobs from one FIFO queue, so up to n_workers jobs run on
 * the GPU at once.  Admission: the head of the queue starts only when its
 * device memory (nne_job_bytes) fits in what the budget has left; a job larger
 * than the whole budget is refused by nne_submit with NNE_ERR_OOM.  Jobs do
 * not overtake each other in admission order.
 *
 * Ownership: nne_submit copies everything the job points to before it
 * returns.  nne_poll copies results into the caller's arrays of the nne_result
 * it is given (the pointers that are not NULL) and then forgets the ticket.
 * Errors of one job are reported in its result and do not stop the server.
 * Calls on one server are thread-safe. */
typedef struct nne_server nne_server;

typedef struct {
  int n_qubits;
  int n_layers;
  const int* layer_gates;   /* n_layers: number of gates of each layer */
  const int* layer_dir;     /* n_layers: +1 gates applied left to right, -1 right to left */
  const int* left_qubit;    /* sum(layer_gates): gate g acts on (left_qubit[g], left_qubit[g]+1), in order */
  const double* U;          /* sum(layer_gates) x 4 x 4 complex128 (re, im interleaved), row-major */
  int n_lambda;
  const double* lambdas;    /* n_lambda noise levels */
  const double* rates;      /* n_lambda x 4 channel strengths, as nne_build_superops (NULL with pauli_rates) */
  int chi;
  int dtype;                /* nne_dtype */
  int trunc;                /* nne_trunc */
  const void* sketch;       /* NNE_TRUNC_RSVD: sketch_rows x sketch_cols, element type of dtype, host; else NULL */
  int sketch_rows, sketch_cols, power_iters;
  const uint8_t* init_bits; /* n_qubits computational-basis bits, or NULL for |0...0> */
  int n_obs;
  const uint8_t* paulis;    /* n_obs x n_qubits Pauli codes */
  int fit_method;           /* nne_fit */
  int fit_degree;           /* NNE_FIT_POLY only */
  double lambda_star;
  const double* pauli_rates; /* NULL, or sum(layer_gates) x 2 x 16: gate-dependent Pauli channels as
                                nne_build_pauli_superops (c0, c1 per gate, in gate order); when set,
                                rates is ignored and level i applies p = c0 + lambdas[i] c1, each
                                in [0, 1] and summing to 1 per gate (checked at submit) */
} nne_job;

typedef struct {
  nne_status status;        /* NNE_OK, or the error that ended the job */
  char error[160];          /* one-line description when status != NNE_OK */
  double* values;           /* in: caller array n_lambda x n_obs (Re <P> per level) or NULL */
  double* log_fid;          /* in: caller array n_lambda (log of the emulation fidelity) or NULL */
  double* estimate;         /* in: caller array n_obs (extrapolated to lambda*) or NULL */
  int32_t* fit_status;      /* in: caller array n_obs (per-observable fit status) or NULL */
  double t_submit, t_start, t_end;   /* seconds on the server's monotonic clock */
  long long gate_steps;     /* gates x n_lambda applied */
  size_t bytes_reserved;    /* device memory admitted for the job */
} nne_result;

/* flags: NNE_SERVER_DRYRUN makes workers do no GPU work at all: a job "runs"
 * for dry_run_us microseconds and ends with status NNE_ERR_UNIMPL and no
 * values.  It exists to test queueing and admission without a GPU. */
#define NNE_SERVER_DRYRUN 1
nne_status nne_server_create(int device, size_t hbm_budget_bytes, int n_workers, int flags, int dry_run_us,
                             nne_server** out);
/* Device memory a job needs while it runs (state, workspaces, superoperators). */
size_t nne_job_bytes(const nne_job* job);
nne_status nne_submit(nne_server* srv, const nne_job* job, uint64_t* ticket);
/* NNE_OK: the job is finished and *out is filled; NNE_PENDING: not finished
 * within timeout_ms (0 = do not wait, < 0 = wait without limit);
 * NNE_ERR_ARG: unknown ticket. */
nne_status nne_poll(nne_server* srv, uint64_t ticket, int timeout_ms, nne_result* out);
/* Jobs queued, running, finished but not yet polled; bytes admitted now. */
void nne_server_stats(nne_server* srv, int* queued, int* running, int* done, size_t* bytes_reserved);
/* Finishes the running jobs, drops the queued ones, joins the workers. */
void nne_server_destroy(nne_server* srv);

/* Metrics log (no counterpart in the paper): append one JSON line per finished
 * job to the file at path -- ticket, status, error, n, chi, n_lambda, gates,
 * gate_steps, bytes, t_submit, t_start, t_end, latency_s (seconds on the
 * server's clock) and log_fid (log F per level, empty when the job produced
 * none).  NULL path stops logging.  NNE_ERR_ARG if the file cannot be opened. */
nne_status nne_server_set_log(nne_server* srv, const char* path);

/* Cancel a request.  A job still waiting in the queue is removed and its
 * result completes at once with status NNE_ERR_CANCELLED (collect it with
 * nne_poll as usual).  A running job is not interrupted: the call returns
 * NNE_PENDING and the job completes normally.  NNE_ERR_ARG for an unknown or
 * already finished ticket. */
nne_status nne_cancel(nne_server* srv, uint64_t ticket);

/* Fault injection for tests of failure handling (no counterpart in the
 * paper; host only, no GPU fault): the waiting job with this ticket, when a
 * worker takes it, ends with `status` (a negative nne_status) and error
 * "injected failure" instead of running; its memory reservation is released as
 * for any finished job.  NNE_ERR_ARG for a non-negative status or a ticket
 * that is not waiting in the queue. */
nne_status nne_server_inject_failure(nne_server* srv, uint64_t ticket, nne_status status);

#ifdef __cplusplus
}
#endif
#endif /* NNE_H */
