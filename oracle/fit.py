"""Noise-strength extrapolation fits -- ORACLE (test infrastructure only).

Sec. 2.2.3 (B) and App. B.2.  Inputs per observable: levels lambda_j, values
y_j = <O>_lambda_j (after fidelity extrapolation when a chi ladder exists;
the emulated value otherwise), emulation fidelities given as log F_j (log
because F reaches 1e-100 and below), and the target lambda*.

EXP_LOGLIN (the paper's primary fit, Ansatz a e^{-b lambda} with c = 0):
  criterion 2: keep lambda with |y| >= 1e-10;
  criterion 3: keep lambda whose sign matches the reference sign -- the
    lambda = 0 value when one is supplied, else (reading) the point with the
    smallest lambda; a takes that sign (App. B.2 footnote);
  dip size d: distance from 0 to the smallest nonzero lambda with F > 0.99
    (App. B.2), over all supplied levels; when no level has F > 0.99 the
    reading d = max(lambda) - min(lambda) is used;
  weights w = F^{delta_f} exp(-delta_d |lambda* - lambda| / d), delta_f = 2,
    delta_d = 20 (App. B.2, eq. for w_lambda and the stated constants);
  minimise sum w^2 (alpha - b lambda - log|y|)^2 (eq. for the weighted loss)
    by weighted least squares; estimate = sign * exp(alpha - b lambda*).
  Weights are formed in the log domain; the two-parameter minimiser is
  written in its pairwise closed form (slope = weighted mean of pairwise
  slopes with weights W_i W_j (x_i - x_j)^2), which is exact and does not
  underflow when F^2 does.
  If fewer than two points survive, fall back (Sec. 2.2.3, last paragraph
  of (B)) to EXP3 over all points.
EXP3 (fallback): unweighted least squares of a e^{-b lambda} + c over all
  points, >= 3 points.  The paper does not name an optimiser; reading:
  variable projection -- for fixed b the pair (a, c) is a linear least-squares
  problem; b is scanned on 4001 points of [-B, B], B = 50 / (max lambda -
  min lambda), then refined by golden-section search on the best bracket.
POLY(m): unweighted least squares polynomial of degree m in
  t = (lambda - lambda*) / max|lambda - lambda*|, solved by Householder QR;
  the estimate is the constant coefficient.
If no fit is possible the status is NOFIT and the value at lambda* is returned
when lambda* was emulated (the paper's final fallback), else NaN.

Fidelity extrapolation (A) over a bond-dimension ladder D_1 < ... < D_k
(Sec. 2.2.3 (A); App. B.1):
  per (lambda, observable), a least-squares straight line of <O>^{(D_j)}
    against F^{(D_j)} over the k rungs, evaluated at F = 1 (one rung: the
    value itself; all F equal: their mean, reading);
  criterion 1 (App. B.1 eq.): lambda stays in Lambda when
    |(O_k - O_{k-1}) / (F_k - F_{k-1})| (1 - F_k) < |O_k| / 2, with the
    readings: F_k = 1 gives a left side of 0 (the top rung is exact); equal
    top fidelities give 0 when O_k = O_{k-1} and infinity otherwise; one rung
    keeps every lambda.
  (B) then runs on the surviving lambdas with F^max = F^{(D_k)}; the dip size
    d is taken over all levels (it describes F^max(lambda), not the fit set);
    the NOFIT fallback is the D_k emulation at lambda* (Sec. 2.2.3, last
    paragraph of (B)).

Pins (tests/test_oracle_fit.py): POLY vs numpy.polyfit; EXP_LOGLIN recovers
exact a e^{-b lambda} data and equals a closed-form weighted line fit written
independently; EXP3 recovers noiseless a e^{-b lambda} + c and reaches a loss
no larger than scipy.optimize.curve_fit on noisy data; the printed constants
(delta_f = 2, delta_d = 20, 1e-10, 0.99) appear in golden fixtures.
"""
from __future__ import annotations

import math

import numpy as np

DELTA_F = 2.0
DELTA_D = 20.0
SMALL = 1e-10
DIP_FID = 0.99

OK, NOFIT = 0, -6
M_POLY, M_EXP_LOGLIN, M_EXP3 = 0, 1, 2


def poly(lams, y, lam_star: float, degree: int):
    lams = np.asarray(lams, float)
    y = np.asarray(y, float)
    if lams.size < degree + 1:
        return _nofit(lams, y, lam_star)
    dist = np.abs(lams - lam_star)
    scale = dist.max() if dist.max() > 0 else 1.0
    t = (lams - lam_star) / scale
    V = np.stack([t ** k for k in range(degree + 1)], axis=1)
    Q, R = np.linalg.qr(V)
    coef = np.linalg.solve(R, Q.T @ y)
    return float(coef[0]), OK


def dip_size(lams, log_fid) -> float:
    lams = np.asarray(lams, float)
    fid = np.exp(np.asarray(log_fid, float))
    cand = sorted(l for l, f in zip(lams, fid) if l > 0 and f > DIP_FID)
    if cand:
        return float(cand[0])
    span = float(lams.max() - lams.min())
    return span if span > 0 else 1.0


def log_weights(lams, log_fid, lam_star: float, d: float) -> np.ndarray:
    """log w = delta_f log F - delta_d |lambda* - lambda| / d."""
    return DELTA_F * np.asarray(log_fid, float) - DELTA_D * np.abs(lam_star - np.asarray(lams, float)) / d


def exp_loglin(lams, y, log_fid, lam_star: float, y_zero=None, d=None):
    lams = np.asarray(lams, float)
    y = np.asarray(y, float)
    log_fid = np.zeros_like(lams) if log_fid is None else np.asarray(log_fid, float)
    if y_zero is not None:
        ref_sign = 1.0 if y_zero >= 0 else -1.0
    else:
        ref_sign = 1.0 if y[np.argmin(lams)] >= 0 else -1.0
    keep = (np.abs(y) >= SMALL) & (np.sign(y) == ref_sign)
    if keep.sum() < 2:
        return exp3(lams, y, lam_star)
    if d is None:
        d = dip_size(lams, log_fid)
    lw2 = 2.0 * log_weights(lams, log_fid, lam_star, d)[keep]       # log w^2
    x = lams[keep]
    z = np.log(np.abs(y[keep]))
    # Weighted least squares line z = alpha + slope * x (slope = -b), in the
    # underflow-free pairwise form: slope = sum_{i<j} W_i W_j (x_i-x_j)(z_i-z_j)
    # / sum_{i<j} W_i W_j (x_i-x_j)^2, alpha = sum W (z - slope x) / sum W,
    # with W = w^2 scaled by a common factor (the minimiser is scale-free).
    lp, num_ratio = [], []
    for i in range(x.size):
        for j in range(i + 1, x.size):
            if x[i] != x[j]:
                lp.append(lw2[i] + lw2[j] + 2.0 * math.log(abs(x[i] - x[j])))
                num_ratio.append((z[i] - z[j]) / (x[i] - x[j]))
    if not lp:
        return exp3(lams, y, lam_star)
    lp = np.array(lp)
    c = np.exp(lp - lp.max())
    slope = float(np.sum(c * np.array(num_ratio)) / np.sum(c))
    W = np.exp(lw2 - lw2.max())
    alpha = float(np.sum(W * (z - slope * x)) / np.sum(W))
    return float(ref_sign * math.exp(alpha + slope * lam_star)), OK


def _exp3_profile(b: float, lams, y):
    """Residual sum of squares and (a, c) of the best a e^{-b lam} + c at fixed b."""
    e = np.exp(-b * lams)
    A = np.stack([e, np.ones_like(lams)], axis=1)
    sol, *_ = np.linalg.lstsq(A, y, rcond=None)
    r = A @ sol - y
    return float(r @ r), sol


def exp3_params(lams, y):
    """(a, b, c) minimising sum (a e^{-b lam} + c - y)^2, or None with < 3 points."""
    lams = np.asarray(lams, float)
    y = np.asarray(y, float)
    span = float(lams.max() - lams.min()) if lams.size else 0.0
    if lams.size < 3 or span <= 0:
        return None
    B = 50.0 / span
    grid = np.linspace(-B, B, 4001)
    losses = np.array([_exp3_profile(b, lams, y)[0] if b != 0.0 else np.inf for b in grid])
    i = int(np.argmin(losses))
    lo = grid[max(i - 1, 0)]
    hi = grid[min(i + 1, grid.size - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    x1 = hi - g * (hi - lo)
    x2 = lo + g * (hi - lo)
    f = lambda b: _exp3_profile(b, lams, y)[0] if b != 0.0 else np.inf
    f1, f2 = f(x1), f(x2)
    tol = 1e-12 * B
    while hi - lo > tol:
        if f1 <= f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = f(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = f(x2)
    b = 0.5 * (lo + hi)
    if b == 0.0:
        b = lo
    _, (a, c) = _exp3_profile(b, lams, y)
    return float(a), float(b), float(c)


def exp3(lams, y, lam_star: float):
    p = exp3_params(lams, y)
    if p is None:
        return _nofit(lams, y, lam_star)
    a, b, c = p
    return float(a * math.exp(-b * lam_star) + c), OK


def _nofit(lams, y, lam_star):
    hit = np.nonzero(np.asarray(lams) == lam_star)[0]
    return (float(np.asarray(y)[hit[0]]) if hit.size else float("nan")), NOFIT


def extrapolate(method: int, lams, values, lam_star: float, log_fid=None, degree: int = 2, y_zero=None):
    """values: (n_lambda, n_obs).  Returns (estimates[n_obs], status[n_obs])."""
    values = np.asarray(values, float)
    if values.ndim == 1:
        values = values[:, None]
    est = np.zeros(values.shape[1])
    st = np.zeros(values.shape[1], int)
    for j in range(values.shape[1]):
        yz = None if y_zero is None else float(np.asarray(y_zero)[j])
        if method == M_POLY:
            est[j], st[j] = poly(lams, values[:, j], lam_star, degree)
        elif method == M_EXP_LOGLIN:
            est[j], st[j] = exp_loglin(lams, values[:, j], log_fid, lam_star, yz)
        elif method == M_EXP3:
            est[j], st[j] = exp3(lams, values[:, j], lam_star)
        else:
            raise ValueError(method)
    return est, st


def fidelity_line(o, fid) -> float:
    """(A): least-squares line of o against fid (k rungs), evaluated at fid = 1."""
    o = np.asarray(o, float)
    fid = np.asarray(fid, float)
    if o.size == 1:
        return float(o[0])
    fm, om = fid.mean(), o.mean()
    sff = float(np.sum((fid - fm) ** 2))
    if sff == 0.0:
        return float(om)
    slope = float(np.sum((fid - fm) * (o - om))) / sff
    return float(om + slope * (1.0 - fm))


def converged(o, fid) -> bool:
    """Criterion 1 (App. B.1) on the two largest rungs (last two entries)."""
    o = np.asarray(o, float)
    fid = np.asarray(fid, float)
    if o.size < 2:
        return True
    ok, ok1, fk, fk1 = o[-1], o[-2], fid[-1], fid[-2]
    if fk == 1.0:
        lhs = 0.0
    elif fk == fk1:
        lhs = 0.0 if ok == ok1 else math.inf
    else:
        lhs = abs((ok - ok1) / (fk - fk1)) * (1.0 - fk)
    return lhs < abs(ok) / 2.0


def ladder(values, log_fid):
    """values (k, n_lambda, n_obs) at D_1..D_k, log_fid (k, n_lambda) ->
    (obar (n_lambda, n_obs), conv (n_lambda, n_obs) bool)."""
    values = np.asarray(values, float)
    fid = np.exp(np.asarray(log_fid, float))
    k, nl, no = values.shape
    obar = np.zeros((nl, no))
    conv = np.zeros((nl, no), bool)
    for i in range(nl):
        for o in range(no):
            obar[i, o] = fidelity_line(values[:, i, o], fid[:, i])
            conv[i, o] = converged(values[:, i, o], fid[:, i])
    return obar, conv


def nzne(method: int, lams, values, log_fid, lam_star: float, degree: int = 2, y_zero=None):
    """(A) then (B): values (k, n_lambda, n_obs), log_fid (k, n_lambda).
    Returns (estimates[n_obs], status[n_obs], obar, conv)."""
    lams = np.asarray(lams, float)
    values = np.asarray(values, float)
    log_fid = np.asarray(log_fid, float)
    obar, conv = ladder(values, log_fid)
    lf_max = log_fid[-1]
    d_all = dip_size(lams, lf_max)
    n_obs = values.shape[2]
    est = np.zeros(n_obs)
    st = np.zeros(n_obs, int)
    for o in range(n_obs):
        m = conv[:, o]
        x, y, lf = lams[m], obar[m, o], lf_max[m]
        yz = None if y_zero is None else float(np.asarray(y_zero)[o])
        if x.size == 0:
            e, s = float("nan"), NOFIT
        elif method == M_POLY:
            e, s = poly(x, y, lam_star, degree)
        elif method == M_EXP_LOGLIN:
            e, s = exp_loglin(x, y, lf, lam_star, yz, d=d_all)
        elif method == M_EXP3:
            e, s = exp3(x, y, lam_star)
        else:
            raise ValueError(method)
        if s == NOFIT:
            e = _nofit(lams, values[-1, :, o], lam_star)[0]
        est[o], st[o] = e, s
    return est, st, obar, conv
