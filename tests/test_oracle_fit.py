"""Pins for oracle/fit.py (Sec. 2.2.3 (B), App. B.2)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fit

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_constants_match_paper():
    assert fit.DELTA_F == GOLD["delta_f"]["value"]
    assert fit.DELTA_D == GOLD["delta_d"]["value"]
    assert fit.SMALL == GOLD["small_threshold"]["value"]
    assert fit.DIP_FID == GOLD["dip_fidelity"]["value"]


def test_poly_matches_numpy_polyfit():
    rng = np.random.default_rng(0)
    lams = np.array([1.0, 2.0, 4.0, 8.0])
    for _ in range(5):
        y = rng.standard_normal(4)
        est, st = fit.poly(lams, y, 1.0, 2)
        t = (lams - 1.0) / 7.0
        ref = np.polyfit(t, y, 2)[-1]
        assert st == fit.OK and abs(est - ref) < 1e-12


def test_poly_exact_on_quadratic():
    lams = np.array([1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
    y = 0.3 - 0.2 * lams + 0.01 * lams ** 2
    est, _ = fit.poly(lams, y, 1.0, 2)
    assert abs(est - (0.3 - 0.2 + 0.01)) < 1e-13
    est0, _ = fit.poly(lams, y, 0.0, 2)
    assert abs(est0 - 0.3) < 1e-13


@pytest.mark.parametrize("a,b", [(0.7, 0.3), (-0.4, 0.05), (1e-3, -0.2)])
def test_loglin_recovers_exact_exponential(a, b):
    lams = np.arange(1.0, 9.0)
    y = a * np.exp(-b * lams)
    log_fid = np.log(np.linspace(0.2, 0.999, 8))
    est, st = fit.exp_loglin(lams, y, log_fid, 1.0)
    assert st == fit.OK
    assert abs(est - a * math.exp(-b)) < 1e-12 * abs(a)
    est0, _ = fit.exp_loglin(lams, y, log_fid, 0.0)
    assert abs(est0 - a) < 1e-11 * abs(a)


def weighted_line_textbook(x, z, w2):
    """Weighted least squares line z ~ alpha + beta x by the closed-form normal equations."""
    S, Sx, Sz = w2.sum(), (w2 * x).sum(), (w2 * z).sum()
    Sxx, Sxz = (w2 * x * x).sum(), (w2 * x * z).sum()
    beta = (S * Sxz - Sx * Sz) / (S * Sxx - Sx * Sx)
    alpha = (Sz - beta * Sx) / S
    return alpha, beta


def test_loglin_equals_textbook_weighted_fit():
    rng = np.random.default_rng(1)
    lams = np.array([1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
    y = -0.3 * np.exp(-0.2 * lams) * (1 + 0.05 * rng.standard_normal(6))
    fids = np.array([0.3, 0.6, 0.95, 0.995, 0.999, 0.9999])
    lam_star = 1.0
    # dip size (App. B.2): smallest nonzero lambda with F > 0.99 -> 3.0
    d = 3.0
    w = fids ** GOLD["delta_f"]["value"] * np.exp(-GOLD["delta_d"]["value"] * np.abs(lam_star - lams) / d)
    alpha, beta = weighted_line_textbook(lams, np.log(np.abs(y)), w ** 2)
    ref = -math.exp(alpha + beta * lam_star)
    est, st = fit.exp_loglin(lams, y, np.log(fids), lam_star)
    assert st == fit.OK and abs(est - ref) < 1e-12
    assert fit.dip_size(lams, np.log(fids)) == 3.0


def test_loglin_criteria_two_and_three():
    lams = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    y = 0.5 * np.exp(-0.1 * lams)
    y_bad = y.copy()
    y_bad[2] = -0.01          # opposite sign: dropped by criterion 3
    y_bad[4] = 1e-12          # below 1e-10: dropped by criterion 2
    est, st = fit.exp_loglin(lams, y_bad, None, 1.0)
    keep = [0, 1, 3]
    ref, _ = fit.exp_loglin(lams[keep], y[keep], None, 1.0)
    assert st == fit.OK and abs(est - ref) < 1e-13 and abs(est - 0.5 * math.exp(-0.1)) < 1e-12


def test_loglin_falls_back_to_exp3():
    lams = np.array([1.0, 2.0, 3.0, 4.0])
    y = np.array([0.2, -0.1, -0.05, -0.3])        # only one point with the reference sign
    est, st = fit.exp_loglin(lams, y, None, 1.0)
    ref, st3 = fit.exp3(lams, y, 1.0)
    assert st == st3 and est == ref


def test_exp3_recovers_noiseless():
    lams = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    for a, b, c in ((0.8, 0.4, 0.1), (-0.3, 0.9, 0.05), (0.2, -0.15, -0.4)):
        y = a * np.exp(-b * lams) + c
        est, st = fit.exp3(lams, y, 1.0)
        assert st == fit.OK and abs(est - (a * math.exp(-b) + c)) < 1e-8


def test_exp3_loss_not_worse_than_curve_fit():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(2)
    lams = np.arange(1.0, 9.0)
    y = 0.6 * np.exp(-0.3 * lams) + 0.1 + 0.01 * rng.standard_normal(8)
    est, _ = fit.exp3(lams, y, 1.0)
    f = lambda x, a, b, c: a * np.exp(-b * x) + c
    p, _ = scipy_opt.curve_fit(f, lams, y, p0=(0.5, 0.2, 0.0), maxfev=20000)
    loss_ref = float(np.sum((f(lams, *p) - y) ** 2))
    a, b, c = fit.exp3_params(lams, y)
    best = float(np.sum((f(lams, a, b, c) - y) ** 2))
    assert best <= loss_ref * (1 + 1e-9)
    assert abs(est - f(1.0, *p)) < 1e-4


def test_nofit_returns_value_at_target():
    est, st = fit.exp3(np.array([1.0, 2.0]), np.array([0.3, 0.2]), 1.0)
    assert st == fit.NOFIT and est == 0.3
    est, st = fit.poly(np.array([2.0]), np.array([0.3]), 1.0, 2)
    assert st == fit.NOFIT and math.isnan(est)


def test_weights_survive_tiny_fidelity():
    # F ~ 1e-300 would underflow F^2; the log-domain weights must still fit
    lams = np.arange(1.0, 6.0)
    y = 0.4 * np.exp(-0.2 * lams)
    log_fid = np.array([-700.0, -500.0, -300.0, -100.0, -10.0])
    est, st = fit.exp_loglin(lams, y, log_fid, 1.0)
    assert st == fit.OK and abs(est - 0.4 * math.exp(-0.2)) < 1e-12


def test_extrapolate_dispatch():
    lams = np.array([1.0, 2.0, 4.0, 8.0])
    vals = np.stack([0.5 * np.exp(-0.1 * lams), 0.2 + 0.01 * lams], axis=1)
    est, st = fit.extrapolate(fit.M_POLY, lams, vals, 1.0, degree=2)
    assert est.shape == (2,) and (st == 0).all()
    assert abs(est[1] - 0.21) < 1e-13


def test_relative_error_definition_matches_table():
    # the brackets of the XYM table are |x - ref| / |ref|
    for ob in ("YX_30_31", "Z_30"):
        row = GOLD["xym_table"][ob]
        for k in ("single", "nzne"):
            rel = abs(row[k] - row["trajectory"]) / abs(row["trajectory"])
            assert abs(rel - row[k + "_rel"]) < 6e-4


# ---------------------------------------------------------------- (A) over a bond-dimension ladder

def test_fidelity_line_matches_polyfit():
    """The straight line in fidelity is numpy.polyfit(F, O, 1) evaluated at F = 1."""
    rng = np.random.default_rng(3)
    for k in (2, 3, 5):
        F = np.sort(rng.uniform(0.2, 0.99, k))
        O = rng.standard_normal(k)
        assert abs(fit.fidelity_line(O, F) - np.polyval(np.polyfit(F, O, 1), 1.0)) < 1e-12
    # exact on a line: O = a + b F -> a + b
    F = np.array([0.3, 0.6, 0.8])
    assert abs(fit.fidelity_line(0.25 - 0.5 * F, F) - (0.25 - 0.5)) < 1e-14
    assert fit.fidelity_line([0.7], [0.4]) == 0.7


def test_criterion_one_is_the_two_point_secant_test():
    """App. B.1: the criterion holds exactly when the secant through the two
    largest rungs, extrapolated to F = 1, lands within |O_k| / 2 of O_k."""
    rng = np.random.default_rng(4)
    hits = 0
    for _ in range(200):
        F = np.sort(rng.uniform(0.1, 0.99, 3))
        O = rng.standard_normal(3)
        secant = np.polyval(np.polyfit(F[1:], O[1:], 1), 1.0)
        want = abs(secant - O[2]) < abs(O[2]) / 2
        assert fit.converged(O, F) == want
        hits += want
    assert 20 < hits < 180
    # worked cases: slope 0.4 over 1 - F = 0.05 -> 0.02 < 0.26; slope 2 over 0.4 -> 0.8 > 0.15
    assert fit.converged([0.50, 0.52], [0.90, 0.95])
    assert not fit.converged([0.1, 0.3], [0.5, 0.6])


def test_criterion_one_readings():
    assert fit.converged([0.2, 0.4], [0.5, 1.0])          # exact top rung
    assert not fit.converged([0.2, 0.0], [0.5, 1.0])      # ... but a zero value never passes "< |O_k|/2"
    assert fit.converged([0.3, 0.3], [0.7, 0.7])          # flat step at equal fidelity
    assert not fit.converged([0.3, 0.4], [0.7, 0.7])      # jump at equal fidelity
    assert fit.converged([0.3], [0.7])                    # one rung keeps every level


def _ladder_data(seed=5, k=3, nl=5, no=4):
    rng = np.random.default_rng(seed)
    lams = np.arange(1.0, nl + 1)
    logf = np.log(np.sort(rng.uniform(0.3, 0.999, (k, nl)), axis=0))
    base = 0.8 * np.exp(-0.3 * lams)[:, None] * np.ones((nl, no))
    vals = base[None] + 0.02 * rng.standard_normal((k, nl, no)) * (1 - np.exp(logf))[:, :, None]
    return lams, vals, logf


@pytest.mark.parametrize("method", [fit.M_POLY, fit.M_EXP_LOGLIN, fit.M_EXP3])
def test_nzne_single_rung_equals_extrapolate(method):
    lams, vals, logf = _ladder_data(k=1)
    est, st, obar, conv = fit.nzne(method, lams, vals, logf, 1.0, degree=2)
    ref, rst = fit.extrapolate(method, lams, vals[0], 1.0, log_fid=logf[0], degree=2)
    assert conv.all() and np.array_equal(obar, vals[0])
    assert np.array_equal(st, rst)
    assert np.allclose(est, ref, rtol=1e-12, atol=1e-14)


def test_nzne_drops_unconverged_levels():
    """Levels failing criterion 1 leave Lambda; the log-linear fit on the rest
    keeps the dip size of all levels (written out here without nzne)."""
    lams, vals, logf = _ladder_data(k=3)
    vals[:, 2, 0] = [0.05, 0.4, 0.1]             # level 3, observable 0: far from converged
    est, st, obar, conv = fit.nzne(fit.M_EXP_LOGLIN, lams, vals, logf, 1.0)
    assert not conv[2, 0] and conv[:, 1:].all()
    m = conv[:, 0]
    d = fit.dip_size(lams, logf[-1])
    ref, rst = fit.exp_loglin(lams[m], obar[m, 0], logf[-1][m], 1.0, d=d)
    assert st[0] == rst and abs(est[0] - ref) < 1e-14
    pest, pst, _, _ = fit.nzne(fit.M_POLY, lams, vals, logf, 1.0, degree=2)
    pref, _ = fit.poly(lams[m], obar[m, 0], 1.0, 2)
    assert abs(pest[0] - pref) < 1e-13


def test_nzne_nofit_falls_back_to_top_rung_at_target():
    lams, vals, logf = _ladder_data(k=2, no=1)
    logf[0], logf[1] = np.log(0.5), np.log(0.7)
    vals[0, :, 0] = 0.9
    vals[1, :, 0] = 0.01                          # every level jumps: nothing converged
    est, st, obar, conv = fit.nzne(fit.M_EXP_LOGLIN, lams, vals, logf, 1.0)
    assert not conv.any() and st[0] == fit.NOFIT
    assert est[0] == vals[1, 0, 0]                # D_max emulation at lambda* = 1
