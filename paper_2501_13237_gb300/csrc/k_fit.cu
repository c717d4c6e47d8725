// a8 -- noise-strength extrapolation to lambda* in float64, one thread per
// observable (Sec. 2.2.3 (B); App. B.2).
//   POLY(m):     least squares in t = (lambda - lambda*)/max|lambda - lambda*| by
//                Householder QR; estimate = constant coefficient.
//   EXP_LOGLIN:  criterion 2 (|y| >= 1e-10), criterion 3 (sign of the
//                lambda = 0 value, else of the smallest-lambda value); weights
//                w = F^2 exp(-20 |lambda* - lambda| / d), d = smallest lambda > 0
//                with F > 0.99 (else the lambda span); weighted line through
//                (lambda, log|y|) in the pairwise closed form (no underflow when
//                F^2 underflows); estimate = sign * exp(alpha - b lambda*).
//                Fewer than two surviving points -> EXP3 on all points.
//   EXP3:        a e^{-b lambda} + c by variable projection: (a, c) linear in b;
//                b on a 4001-point grid of [-B, B], B = 50/span, then golden
//                section on the best bracket to 1e-12 B.
// NOFIT: value at lambda* when lambda* was emulated, else NaN.
//
// Fidelity extrapolation (A) over a bond-dimension ladder D_1 < ... < D_k
// (Sec. 2.2.3 (A); App. B.1), ladder_kernel, one thread per (lambda, obs):
//   obar = least-squares line of <O>^{(D_j)} against F^{(D_j)}, at F = 1
//   (one rung: the value; equal fidelities: the mean);
//   criterion 1: |(O_k - O_{k-1}) / (F_k - F_{k-1})| (1 - F_k) < |O_k| / 2
//   (F_k = 1: left side 0; F_k = F_{k-1}: 0 if O_k = O_{k-1}, else infinite).
// The fit then sees only the levels passing criterion 1 (mask), keeps the dip
// size of all levels, and falls back to the D_k emulation at lambda*.
#include "kernels.cuh"

namespace nne {

constexpr int FIT_MAXL = 64;
constexpr double DELTA_F = 2.0, DELTA_D = 20.0, SMALL = 1e-10, DIP_FID = 0.99;

__device__ void nofit(int nl, const double* lam, const double* y, double ls, double* est, int* st) {
  double v = nan("");
  for (int j = 0; j < nl; ++j)
    if (lam[j] == ls) { v = y[j]; break; }
  *est = v;
  *st = NNE_ERR_NOFIT;
}

__device__ void poly_fit(int nl, const double* lam, const double* y, double ls, int deg, double* est, int* st) {
  const int nc = deg + 1;
  if (nl < nc || nc > 16) { nofit(nl, lam, y, ls, est, st); return; }
  double V[FIT_MAXL][16];
  double b[FIT_MAXL];
  double scale = 0;
  for (int j = 0; j < nl; ++j) scale = fmax(scale, fabs(lam[j] - ls));
  if (scale == 0) scale = 1;
  for (int j = 0; j < nl; ++j) {
    const double t = (lam[j] - ls) / scale;
    double p = 1;
    for (int k = 0; k < nc; ++k) { V[j][k] = p; p *= t; }
    b[j] = y[j];
  }
  for (int k = 0; k < nc; ++k) {
    double xn = 0;
    for (int j = k; j < nl; ++j) xn += V[j][k] * V[j][k];
    xn = sqrt(xn);
    if (xn == 0) continue;
    const double alpha = V[k][k] >= 0 ? -xn : xn;
    double v[FIT_MAXL];
    for (int j = k; j < nl; ++j) v[j] = V[j][k];
    v[k] -= alpha;
    double vn = 0;
    for (int j = k; j < nl; ++j) vn += v[j] * v[j];
    if (vn == 0) continue;
    for (int c = k; c < nc; ++c) {
      double s = 0;
      for (int j = k; j < nl; ++j) s += v[j] * V[j][c];
      s = 2 * s / vn;
      for (int j = k; j < nl; ++j) V[j][c] -= s * v[j];
    }
    double s = 0;
    for (int j = k; j < nl; ++j) s += v[j] * b[j];
    s = 2 * s / vn;
    for (int j = k; j < nl; ++j) b[j] -= s * v[j];
  }
  double c[16];
  for (int k = nc - 1; k >= 0; --k) {
    double s = b[k];
    for (int q = k + 1; q < nc; ++q) s -= V[k][q] * c[q];
    if (V[k][k] == 0) { nofit(nl, lam, y, ls, est, st); return; }
    c[k] = s / V[k][k];
  }
  *est = c[0];
  *st = NNE_OK;
}

__device__ double exp3_profile(double b, int nl, const double* lam, const double* y, double* a_out, double* c_out) {
  double e[FIT_MAXL];
  double em = 0, ym = 0;
  for (int j = 0; j < nl; ++j) { e[j] = exp(-b * lam[j]); em += e[j]; ym += y[j]; }
  em /= nl;
  ym /= nl;
  double see = 0, sey = 0;
  for (int j = 0; j < nl; ++j) { see += (e[j] - em) * (e[j] - em); sey += (e[j] - em) * (y[j] - ym); }
  double a = see > 0 ? sey / see : 0.0;
  double c = ym - a * em;
  double loss = 0;
  for (int j = 0; j < nl; ++j) { const double r = a * e[j] + c - y[j]; loss += r * r; }
  *a_out = a;
  *c_out = c;
  return loss;
}

__device__ void exp3_fit(int nl, const double* lam, const double* y, double ls, double* est, int* st) {
  double lmin = 1e300, lmax = -1e300;
  for (int j = 0; j < nl; ++j) { lmin = fmin(lmin, lam[j]); lmax = fmax(lmax, lam[j]); }
  const double span = nl > 0 ? lmax - lmin : 0;
  if (nl < 3 || !(span > 0)) { nofit(nl, lam, y, ls, est, st); return; }
  const double B = 50.0 / span;
  const int NG = 4001;
  const double step = (2 * B) / (NG - 1);
  double a, c, best = 1e300;
  int bi = 0;
  for (int i = 0; i < NG; ++i) {
    const double b = (i == NG - 1) ? B : i * step - B;
    const double l = (b == 0.0) ? 1e300 : exp3_profile(b, nl, lam, y, &a, &c);
    if (l < best) { best = l; bi = i; }
  }
  auto gridb = [&](int i) { return (i == NG - 1) ? B : i * step - B; };
  double lo = gridb(max(bi - 1, 0)), hi = gridb(min(bi + 1, NG - 1));
  const double g = (sqrt(5.0) - 1.0) / 2.0;
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  auto f = [&](double b) { return b == 0.0 ? 1e300 : exp3_profile(b, nl, lam, y, &a, &c); };
  double f1 = f(x1), f2 = f(x2);
  const double tol = 1e-12 * B;
  for (int it = 0; it < 200 && hi - lo > tol; ++it) {
    if (f1 <= f2) {
      hi = x2; x2 = x1; f2 = f1;
      x1 = hi - g * (hi - lo);
      f1 = f(x1);
    } else {
      lo = x1; x1 = x2; f1 = f2;
      x2 = lo + g * (hi - lo);
      f2 = f(x2);
    }
  }
  double b = 0.5 * (lo + hi);
  if (b == 0.0) b = lo;
  exp3_profile(b, nl, lam, y, &a, &c);
  *est = a * exp(-b * ls) + c;
  *st = NNE_OK;
}

__device__ void loglin_fit(int nl, const double* lam, const double* y, const double* logf, double ls,
                           const double* yzero, int o, double dgiven, double* est, int* st) {
  int jmin = 0;
  for (int j = 1; j < nl; ++j)
    if (lam[j] < lam[jmin]) jmin = j;
  const double ref = yzero ? (yzero[o] >= 0 ? 1.0 : -1.0) : (y[jmin] >= 0 ? 1.0 : -1.0);
  bool keep[FIT_MAXL];
  int nk = 0;
  for (int j = 0; j < nl; ++j) {
    const double sg = y[j] > 0 ? 1.0 : (y[j] < 0 ? -1.0 : 0.0);
    keep[j] = fabs(y[j]) >= SMALL && sg == ref;
    nk += keep[j];
  }
  if (nk < 2) { exp3_fit(nl, lam, y, ls, est, st); return; }
  // dip size over all supplied levels (given by the caller when the fit sees a subset)
  double d = dgiven > 0 ? dgiven : 1e300;
  bool found = dgiven > 0;
  for (int j = 0; j < nl && dgiven <= 0; ++j) {
    const double F = exp(logf ? logf[j] : 0.0);
    if (lam[j] > 0 && F > DIP_FID && lam[j] < d) { d = lam[j]; found = true; }
  }
  if (!found) {
    double lmin = 1e300, lmax = -1e300;
    for (int j = 0; j < nl; ++j) { lmin = fmin(lmin, lam[j]); lmax = fmax(lmax, lam[j]); }
    d = lmax - lmin > 0 ? lmax - lmin : 1.0;
  }
  double lw2[FIT_MAXL], x[FIT_MAXL], zz[FIT_MAXL];
  int m = 0;
  for (int j = 0; j < nl; ++j) {
    if (!keep[j]) continue;
    const double lf = logf ? logf[j] : 0.0;
    lw2[m] = 2.0 * (DELTA_F * lf - DELTA_D * fabs(ls - lam[j]) / d);
    x[m] = lam[j];
    zz[m] = log(fabs(y[j]));
    ++m;
  }
  double lpmax = -1e308;
  bool any = false;
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (x[i] != x[j]) { lpmax = fmax(lpmax, lw2[i] + lw2[j] + 2.0 * log(fabs(x[i] - x[j]))); any = true; }
  if (!any) { exp3_fit(nl, lam, y, ls, est, st); return; }
  double num = 0, den = 0;
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (x[i] != x[j]) {
        const double c = exp(lw2[i] + lw2[j] + 2.0 * log(fabs(x[i] - x[j])) - lpmax);
        num += c * (zz[i] - zz[j]) / (x[i] - x[j]);
        den += c;
      }
  const double slope = num / den;
  double lwmax = -1e308;
  for (int i = 0; i < m; ++i) lwmax = fmax(lwmax, lw2[i]);
  double sw = 0, swz = 0;
  for (int i = 0; i < m; ++i) {
    const double W = exp(lw2[i] - lwmax);
    sw += W;
    swz += W * (zz[i] - slope * x[i]);
  }
  const double alpha = swz / sw;
  *est = ref * exp(alpha + slope * ls);
  *st = NNE_OK;
}

__device__ double dip_all(int nl, const double* lam, const double* logf) {
  double d = 1e300;
  bool found = false;
  for (int j = 0; j < nl; ++j) {
    const double F = exp(logf ? logf[j] : 0.0);
    if (lam[j] > 0 && F > DIP_FID && lam[j] < d) { d = lam[j]; found = true; }
  }
  if (found) return d;
  double lmin = 1e300, lmax = -1e300;
  for (int j = 0; j < nl; ++j) { lmin = fmin(lmin, lam[j]); lmax = fmax(lmax, lam[j]); }
  return lmax - lmin > 0 ? lmax - lmin : 1.0;
}

// mask (nl x n_obs, lambda-major; null: every level): levels the fit may use;
// fb (nl x n_obs; null: the fitted values): where the NOFIT fallback reads the
// value at lambda*.
__global__ void fit_kernel(int nl, const double* lam, const double* vals, const double* logf, int n_obs, int method,
                           int degree, double ls, const double* yzero, const uint8_t* mask, const double* fb,
                           double* out, int* status) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_obs) return;
  double y[FIT_MAXL], lc[FIT_MAXL], fc[FIT_MAXL];
  int m = 0;
  for (int j = 0; j < nl; ++j) {
    if (mask && !mask[(long long)j * n_obs + o]) continue;
    y[m] = vals[(long long)j * n_obs + o];
    lc[m] = lam[j];
    fc[m] = logf ? logf[j] : 0.0;
    ++m;
  }
  const double dgiven = mask ? dip_all(nl, lam, logf) : -1.0;
  double est = nan("");
  int st = NNE_ERR_NOFIT;
  if (m == 0) {
    st = NNE_ERR_NOFIT;
  } else if (method == NNE_FIT_POLY) {
    poly_fit(m, lc, y, ls, degree, &est, &st);
  } else if (method == NNE_FIT_EXP_LOGLIN) {
    loglin_fit(m, lc, y, logf ? fc : nullptr, ls, yzero, o, dgiven, &est, &st);
  } else {
    exp3_fit(m, lc, y, ls, &est, &st);
  }
  if (st == NNE_ERR_NOFIT && (fb || mask)) {
    const double* src = fb ? fb : vals;
    est = nan("");
    for (int j = 0; j < nl; ++j)
      if (lam[j] == ls) { est = src[(long long)j * n_obs + o]; break; }
  }
  out[o] = est;
  status[o] = st;
}

// (A) over k rungs: vals (k x nl x n_obs), logf (k x nl) -> obar (nl x n_obs), conv (nl x n_obs).
__global__ void ladder_kernel(int k, int nl, int n_obs, const double* vals, const double* logf, double* obar,
                              uint8_t* conv) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nl * n_obs) return;
  const int i = (int)(idx / n_obs), o = (int)(idx % n_obs);
  auto O = [&](int j) { return vals[((long long)j * nl + i) * n_obs + o]; };
  auto F = [&](int j) { return exp(logf[(long long)j * nl + i]); };
  double ob;
  if (k == 1) {
    ob = O(0);
  } else {
    double fm = 0, om = 0;
    for (int j = 0; j < k; ++j) { fm += F(j); om += O(j); }
    fm /= k;
    om /= k;
    double sff = 0, sfo = 0;
    for (int j = 0; j < k; ++j) {
      const double df = F(j) - fm;
      sff += df * df;
      sfo += df * (O(j) - om);
    }
    ob = sff == 0.0 ? om : om + (sfo / sff) * (1.0 - fm);
  }
  bool c = true;
  if (k >= 2) {
    const double ok = O(k - 1), ok1 = O(k - 2), fk = F(k - 1), fk1 = F(k - 2);
    double lhs;
    if (fk == 1.0) lhs = 0.0;
    else if (fk == fk1) lhs = ok == ok1 ? 0.0 : INFINITY;
    else lhs = fabs((ok - ok1) / (fk - fk1)) * (1.0 - fk);
    c = lhs < fabs(ok) / 2.0;
  }
  obar[idx] = ob;
  conv[idx] = c ? 1 : 0;
}

cudaError_t extrapolate_fit(cudaStream_t st, int n_lambda, const double* d_lam, const double* d_vals,
                            const double* d_logfid, int n_obs, int method, int degree, double lambda_star,
                            const double* d_yzero, double* d_out, int* d_status) {
  if (n_obs <= 0) return cudaSuccess;
  ProfScope ps(st, K_FIT);
  fit_kernel<<<(n_obs + 63) / 64, 64, 0, st>>>(n_lambda, d_lam, d_vals, d_logfid, n_obs, method, degree, lambda_star,
                                              d_yzero, nullptr, nullptr, d_out, d_status);
  return cudaGetLastError();
}

cudaError_t extrapolate_ladder(cudaStream_t st, int k, int n_lambda, const double* d_lam, const double* d_vals,
                               const double* d_logfid, int n_obs, int method, int degree, double lambda_star,
                               const double* d_yzero, double* d_obar, uint8_t* d_conv, double* d_out, int* d_status) {
  if (n_obs <= 0) return cudaSuccess;
  ProfScope ps(st, K_FIT, 2);
  const long long cells = (long long)n_lambda * n_obs;
  ladder_kernel<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(k, n_lambda, n_obs, d_vals, d_logfid, d_obar, d_conv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // (B) on the fidelity-extrapolated values, F^max = the top rung, fallback to the top rung's values
  const double* top_logf = d_logfid + (long long)(k - 1) * n_lambda;
  const double* top_vals = d_vals + (long long)(k - 1) * cells;
  fit_kernel<<<(n_obs + 63) / 64, 64, 0, st>>>(n_lambda, d_lam, d_obar, top_logf, n_obs, method, degree, lambda_star,
                                              d_yzero, d_conv, top_vals, d_out, d_status);
  return cudaGetLastError();
}

}  // namespace nne
