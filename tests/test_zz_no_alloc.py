"""nne_extrapolate_noalloc against nne_extrapolate through the C ABI.

The no-allocation variant serves callers that cannot allocate device memory
when they request a fit (a request loop with its HBM budget already committed,
or latency-critical code that cannot afford cudaMalloc's device
synchronisation).  It must give the same results as the allocating entry
point, on two calls in a row (the fixed array keeps the previous call's
contents), and reject sizes beyond its fixed capacity.  This file is named to
be collected last."""
import numpy as np
import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


def data(seed, n_lambda, n_obs):
    rng = np.random.default_rng(seed)
    lams = np.sort(rng.uniform(0.5, 8.0, n_lambda))
    a = rng.uniform(-1, 1, n_obs)
    b = rng.uniform(0.0, 0.5, n_obs)
    vals = a[None, :] * np.exp(-b[None, :] * lams[:, None]) * (1 + 0.03 * rng.standard_normal((n_lambda, n_obs)))
    log_fid = np.log(np.linspace(0.3, 0.999, n_lambda))
    return lams, vals, log_fid


def _same(got, gst, ref, rst, call):
    assert (gst == rst).all(), f"call {call}"
    both_nan = np.isnan(ref) & np.isnan(got)
    assert np.all(both_nan | (np.abs(got - ref) <= 1e-10 * np.maximum(1.0, np.abs(ref)))), f"call {call}"


@pytest.mark.parametrize("method", [0, 1, 2])
def test_noalloc_matches_allocating_fit_twice(ctx, method):
    # small, then the full capacity, then small again: the last call runs over
    # what the large one left in the shared array
    for call, (seed, nl, no) in enumerate([(11, 6, 300), (12, 8, 1024), (13, 3, 17)]):
        lams, vals, lf = data(seed + method, nl, no)
        ref, rst = ctx.extrapolate(lams, vals, lf, method=method, degree=2, lambda_star=1.0)
        got, gst = ctx.extrapolate_noalloc(lams, vals, lf, method=method, degree=2, lambda_star=1.0)
        _same(got, gst, ref, rst, call)


def test_noalloc_with_zero_noise_reference(ctx):
    # criterion 3 against supplied lambda = 0 values: the y_zero staging path
    from paper_2501_13237_gb300 import nne
    for call, (seed, nl, no) in enumerate([(21, 8, 1024), (22, 5, 40)]):
        lams, vals, lf = data(seed, nl, no)
        yz = np.sign(vals[0]) * np.where(np.arange(no) % 5 == 0, -1.0, 1.0)
        ref, rst = ctx.extrapolate(lams, vals, lf, method=nne.FIT_EXP_LOGLIN, y_zero=yz)
        got, gst = ctx.extrapolate_noalloc(lams, vals, lf, method=nne.FIT_EXP_LOGLIN, y_zero=yz)
        _same(got, gst, ref, rst, call)


@pytest.mark.parametrize("nl,no", [(4, 1025), (65, 8)])
def test_noalloc_rejects_oversize(ctx, nl, no):
    from paper_2501_13237_gb300 import nne
    lams, vals, lf = data(5, nl, no)
    with pytest.raises(nne.NNEError) as ei:
        ctx.extrapolate_noalloc(lams, vals, lf)
    assert ei.value.status == -1
