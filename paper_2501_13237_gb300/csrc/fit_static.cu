// nne_extrapolate_noalloc: the extrapolation fit of nne_extrapolate, staged
// through a fixed device array instead of freshly allocated device memory.
//
// Who needs it: a caller that must not allocate device memory at the moment
// it asks for a fit -- typically a request loop that has already committed
// the whole HBM budget to resident states (a new cudaMalloc can then fail),
// or latency-critical code that cannot afford cudaMalloc/cudaFree, which may
// synchronise the device and stall work running on other streams.
//
// The array below lives for as long as the library is loaded on every GPU
// that loads it (about 0.55 MB).  Every call shares it, so calls that overlap
// on the GPU (concurrent calls from different threads or streams) race; calls
// issued one after another are safe, because each call waits for its own
// results before returning.  The array keeps the previous call's contents;
// every entry the fit kernel reads is written by the call first, and the
// optional inputs are passed as null pointers when absent, so nothing has to
// start at zero.
#include <mutex>

#include "kernels.cuh"

namespace nne {

constexpr int NOALLOC_MAX_LAMBDA = 64;
constexpr int NOALLOC_MAX_OBS = 1024;
// doubles: lambdas, log F, then values (lambda-major), y_zero, out, status (as ints)
constexpr size_t NOALLOC_DOUBLES = 2 * NOALLOC_MAX_LAMBDA + (size_t)NOALLOC_MAX_LAMBDA * NOALLOC_MAX_OBS +
                                   2 * NOALLOC_MAX_OBS + NOALLOC_MAX_OBS / 2;

static __device__ __align__(256) double g_fit_scratch[NOALLOC_DOUBLES];

// Device address of g_fit_scratch per device, looked up once per device with
// that device current (the symbol's host-side name is not a device address).
static std::mutex g_fit_mu;
static double* g_fit_ptr[64] = {nullptr};

static nne_status fit_scratch_for(int device, double** out) {
  if (device < 0 || device >= 64) return set_error(NNE_ERR_ARG, "device ordinal %d out of range", device);
  std::lock_guard<std::mutex> lk(g_fit_mu);
  if (!g_fit_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fit_scratch);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(g_fit_scratch)", __FILE__, __LINE__);
    g_fit_ptr[device] = reinterpret_cast<double*>(p);
  }
  *out = g_fit_ptr[device];
  return NNE_OK;
}

}  // namespace nne

using namespace nne;

extern "C" nne_status nne_extrapolate_noalloc(nne_ctx* ctx, int n_lambda, const double* lambdas,
                                              const double* values, const double* log_fid, int n_obs, int method,
                                              int degree, double lambda_star, const double* y_zero, double* out,
                                              int32_t* per_obs_status) {
  if (!ctx || n_lambda < 1 || !lambdas || !values || n_obs < 0 || !out || !per_obs_status || method < 0 ||
      method > 2 || (method == NNE_FIT_POLY && (degree < 1 || degree > 15)))
    return set_error(NNE_ERR_ARG, "nne_extrapolate_noalloc: bad arguments");
  if (n_lambda > NOALLOC_MAX_LAMBDA || n_obs > NOALLOC_MAX_OBS)
    return set_error(NNE_ERR_ARG,
                     "nne_extrapolate_noalloc: %d levels x %d observables exceed the fixed scratch of %d x %d",
                     n_lambda, n_obs, NOALLOC_MAX_LAMBDA, NOALLOC_MAX_OBS);
  if (n_obs == 0) return NNE_OK;
  int device = 0;
  cudaStream_t s = nullptr;
  ctx_device_stream(ctx, &device, &s);
  nne_status rc = NNE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) NNE_CUDA_TRY(cudaSetDevice(device));
  double* base = nullptr;
  rc = fit_scratch_for(device, &base);
  if (rc == NNE_OK) {
    double* d_lam = base;
    double* d_lf = d_lam + NOALLOC_MAX_LAMBDA;
    double* d_vals = d_lf + NOALLOC_MAX_LAMBDA;
    double* d_yz = d_vals + (size_t)NOALLOC_MAX_LAMBDA * NOALLOC_MAX_OBS;
    double* d_out = d_yz + NOALLOC_MAX_OBS;
    int* d_st = reinterpret_cast<int*>(d_out + NOALLOC_MAX_OBS);
    cudaError_t e = cudaMemcpyAsync(d_lam, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_vals, values, sizeof(double) * n_lambda * (size_t)n_obs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && log_fid)
      e = cudaMemcpyAsync(d_lf, log_fid, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && y_zero)
      e = cudaMemcpyAsync(d_yz, y_zero, sizeof(double) * n_obs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = extrapolate_fit(s, n_lambda, d_lam, d_vals, log_fid ? d_lf : nullptr, n_obs, method, degree, lambda_star,
                          y_zero ? d_yz : nullptr, d_out, d_st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double) * n_obs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(per_obs_status, d_st, sizeof(int) * n_obs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = set_cuda_error(e, "nne_extrapolate_noalloc", __FILE__, __LINE__);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
