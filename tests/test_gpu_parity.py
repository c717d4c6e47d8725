"""GPU parity: every step of the hot path through the C ABI against the oracle.

Tolerances: the complex128 path must agree with the oracle within 1e-10 on
untruncated runs and 1e-8 at the same chi truncation; the complex64 path
within 1e-4 (single-precision arithmetic with float64 norms)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import channels, dense, fit as ofit, mps
from tests.gpu_util import rand_c, require_gpu

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}     # dtype -> tolerance (C64, C128)


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


def test_superops_match_oracle(ctx):
    rng = np.random.default_rng(0)
    U = np.stack([wl.haar_u4(rng) for _ in range(7)])
    rates = np.array([[1e-3, 5e-4, 2e-4, 0.0], [0.3, 0.1, 0.05, 0.02], [0, 0, 0, 0.4]])
    G = ctx.build_superops(U, rates).cpu().numpy()
    for i, r in enumerate(rates):
        for g in range(U.shape[0]):
            assert np.abs(G[i, g] - channels.gate_superop(U[g], r)).max() < 1e-13


def haar_u2(rng):
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("dl,dm,dr,chi,direction,sk", [
    (24, 40, 20, 50, +1, 0), (24, 40, 20, 50, -1, 0),      # truncating, ragged shapes
    (3, 9, 5, 64, +1, 0), (3, 9, 5, 64, -1, 0),            # r = 4 dl or 4 dr: identity branch
    (16, 64, 16, 64, +1, 0), (7, 33, 30, 37, -1, 0),       # several tiles, odd tails
    (170, 100, 60, 200, +1, 0),                            # Gram above the shared-memory size
    (24, 24, 20, 24, +1, 28), (24, 24, 20, 24, -1, 28),    # subspace iteration, k = 28
    (60, 64, 50, 64, +1, 100), (60, 64, 50, 64, -1, 72),
])
def test_single_gate_step(ctx, dtype, dl, dm, dr, chi, direction, sk):
    """One gate step on sites (4, 5) of a 10-site chain (capacities
    min(chi, 4^k, 4^(10-k)) admit the shapes) vs the oracle's two-site update
    (the exact SVD truncation).  The subspace-iteration cases (sk = k columns,
    two power iterations) take a gapped spectrum: the middle bond equals the
    kept rank, the gate is a product of one-qubit unitaries (which keeps the
    operator Schmidt rank) and the noise is weak, so the discarded singular
    values are far below the kept ones and the iteration reaches the exact
    subspace to rounding."""
    from paper_2501_13237_gb300 import nne
    rng = np.random.default_rng(dl * 1000 + dr + (direction > 0) + sk)
    A = rand_c(rng, (dl, 4, dm))
    B = rand_c(rng, (dm, 4, dr))
    n, q = 10, 4
    st = nne.State(ctx, n, chi, 2, dtype, nne.TRUNC_RSVD if sk else nne.TRUNC_EXACT)
    if sk:
        rows = 4 * min(chi, 256)
        om = wl.gaussian_sketch(rows, sk, 5).astype(np.complex64 if dtype == 0 else np.complex128)
        st.set_sketch(om, 2)
    for inst in range(2):
        st.write_site(inst, q, A)
        st.write_site(inst, q + 1, B)
    # a single step touches only the pair once the centre is on it
    st.set_centre(q if direction > 0 else q + 1)
    if sk:
        U = np.stack([np.kron(haar_u2(rng), haar_u2(rng))])
        rates = np.array([[2e-3, 1e-3, 0.0, 0.0], [5e-3, 0.0, 2e-3, 0.0]])
    else:
        U = np.stack([wl.haar_u4(rng)])
        rates = np.array([[0.02, 0.01, 0.0, 0.0], [0.1, 0.0, 0.03, 0.0]])
    G = ctx.build_superops(U, rates)
    st.apply_layer([q], G, direction)
    dims, centre, ln, lf = st.info()
    Gh = G.cpu().numpy()
    tol = TOL[dtype]
    for inst in range(2):
        left, right, f, nrm, s = mps.two_site_update(A, B, Gh[inst, 0], chi, direction)
        if sk:
            r = min(chi, 4 * dl, 4 * dr)
            assert s[r] < 0.2 * s[r - 1]                   # gapped cut
        L = st.read_site(inst, q).astype(np.complex128)
        R = st.read_site(inst, q + 1).astype(np.complex128)
        got = np.einsum("asc,ctb->astb", L, R).reshape(4 * dl, 4 * dr)
        ref = np.einsum("asc,ctb->astb", left, right).reshape(4 * dl, 4 * dr)
        assert np.abs(got - ref).max() < tol * max(1.0, np.abs(ref).max())
        assert abs(lf[inst] - math.log(f)) < tol
        assert abs(ln[inst] - math.log(nrm)) < tol
        r = L.shape[2]
        if direction > 0:
            Lm = L.reshape(-1, r)
            assert np.abs(Lm.conj().T @ Lm - np.eye(r)).max() < 10 * tol
        else:
            Rm = R.reshape(r, -1)
            assert np.abs(Rm @ Rm.conj().T - np.eye(r)).max() < 10 * tol
    assert centre == (q + 1 if direction > 0 else q)
    assert dims[q + 1] == min(chi, 4 * dl, 4 * dr)
    st.close()


def run_gpu(ctx, w, rates, chi, dtype, paulis):
    from paper_2501_13237_gb300 import runner
    st, vals, lf = runner.emulate(ctx, w.circuit, rates, chi, paulis, dtype, bits=w.bits())
    st.close()
    return vals, lf


@pytest.mark.parametrize("dtype", [1, 0])
def test_exact8_untruncated_vs_dense(ctx, dtype):
    w = wl.exact8()
    rates = w.rate_table()
    paulis = wl.pauli_codes(w.observables, w.n)
    vals, lf = run_gpu(ctx, w, rates, w.chi, dtype, paulis)
    for i, lam in enumerate(w.lambdas):
        rho = dense.run(w.circuit, rates[i])
        ref = np.array([dense.expect(rho, ob, w.n) for ob in w.observables])
        assert np.abs(vals[i] - ref).max() < TOL[dtype]
        assert abs(lf[i]) < TOL[dtype]
    # quadratic fit to lambda* = 1 on the device vs the oracle fit on the same data
    from paper_2501_13237_gb300 import nne
    est, st = ctx.extrapolate(w.lambdas, vals.real, lf, method=nne.FIT_POLY, degree=2, lambda_star=1.0)
    ref, rst = ofit.extrapolate(ofit.M_POLY, w.lambdas, vals.real, 1.0, degree=2)
    assert (st == 0).all() and np.abs(est - ref).max() < 1e-10


@pytest.mark.parametrize("dtype,tol", [(1, 1e-8), (0, 1e-4)])
@pytest.mark.parametrize("n,depth,chi,seed", [(10, 10, 16, 3), (9, 8, 12, 4)])
def test_truncated_vs_oracle_mps(ctx, dtype, tol, n, depth, chi, seed):
    c = wl.brickwork_circuit(n, depth, seed)
    noise = wl.NoiseModel(depol2=0.02, amp_damp=0.01, dephase=0.01)
    lams = (1.0, 2.0, 3.0)
    rates = np.stack([noise.rates(l) for l in lams])
    obs = wl.obs_z(n) + wl.obs_xx(n) + [((0, "Y"), (1, "X"), (2, "Z"))]
    paulis = wl.pauli_codes(obs, n)

    class W:
        pass
    w = W()
    w.circuit = c
    w.bits = lambda: None
    vals, lf = run_gpu(ctx, w, rates, chi, dtype, paulis)
    for i in range(len(lams)):
        ref_st = mps.run(c, rates[i], chi)
        ref = ref_st.expect_codes(paulis)
        assert np.abs(vals[i] - ref).max() < tol, (i, np.abs(vals[i] - ref).max())
        assert abs(lf[i] - ref_st.log_fid) < tol * max(1.0, abs(ref_st.log_fid))
        assert ref_st.log_fid < -1e-6


@pytest.mark.parametrize("dtype,tol", [(1, 1e-5), (0, 1e-4)])
@pytest.mark.parametrize("n,depth,chi,seed", [(10, 10, 16, 3), (9, 8, 12, 4), (12, 10, 32, 3)])
def test_truncated_rsvd_vs_exact_svd(ctx, dtype, tol, n, depth, chi, seed):
    """The fast truncation (subspace iteration with k = 3 chi columns and six
    power iterations, Rayleigh-Ritz) over whole truncated runs against the
    oracle's exact SVD truncation (Sec. 2.1.2: the closest state of bond
    dimension chi), on circuits whose cuts are gapped (the exact-path tests
    use the first two).  complex128 shows the iteration's own convergence
    error (1e-5); complex64 adds single-precision rounding (1e-4)."""
    from paper_2501_13237_gb300 import nne, runner
    k, q = 3 * chi, 6
    c = wl.brickwork_circuit(n, depth, seed)
    noise = wl.NoiseModel(depol2=0.02, amp_damp=0.01, dephase=0.01)
    rates = np.stack([noise.rates(l) for l in (1.0, 3.0)])
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    om = wl.gaussian_sketch(4 * chi, k, 9).astype(np.complex64 if dtype == 0 else np.complex128)
    st = nne.State(ctx, n, chi, 2, dtype, nne.TRUNC_RSVD)
    st.set_sketch(om, q)
    runner.evolve(st, runner.build_layer_superops(ctx, c, rates))
    vals, lf = st.expect(paulis)
    for i in range(2):
        ref_st = mps.run(c, rates[i], chi)
        ref = ref_st.expect_codes(paulis)
        assert np.abs(vals[i] - ref).max() < tol, np.abs(vals[i] - ref).max()
        assert abs(lf[i] - ref_st.log_fid) < tol * max(1.0, abs(ref_st.log_fid))
        assert ref_st.log_fid < -1e-3                  # the runs do truncate
    st.close()


def test_full_size_gate_step_vs_exact_svd(ctx):
    """One complex64 gate step at the headline size: bonds of 512 on both
    sides of the pair (X is 2048 x 2048), eight instances at noise levels
    lambda = 1..8, the bench's subspace iteration (k = 640 columns, four power
    iterations, 2048-row QR panels, Rayleigh-Ritz eigensolve of size 640,
    TMA-fed tensor-core GEMMs) against the oracle's exact SVD.  Gapped spectrum: the middle bond
    equals the kept rank and the gate is a product of one-qubit unitaries, so
    only the weak two-qubit noise spreads weight past the cut."""
    from paper_2501_13237_gb300 import nne
    rng = np.random.default_rng(2048)
    d, chi, n, q, k, n_inst = 512, 512, 12, 5, 640, 8
    A = rand_c(rng, (d, 4, d)) / np.sqrt(4 * d)
    B = rand_c(rng, (d, 4, d)) / np.sqrt(4 * d)
    A = A.astype(np.complex64).astype(np.complex128)
    B = B.astype(np.complex64).astype(np.complex128)
    st = nne.State(ctx, n, chi, n_inst, nne.C64, nne.TRUNC_RSVD)
    st.set_sketch(wl.gaussian_sketch(4 * chi, k, 1234).astype(np.complex64), 4)
    for inst in range(n_inst):
        st.write_site(inst, q, A)
        st.write_site(inst, q + 1, B)
    st.set_centre(q)
    U = np.stack([np.kron(haar_u2(rng), haar_u2(rng))])
    noise = wl.n100().noise
    rates = np.stack([noise.rates(l) for l in range(1, n_inst + 1)])
    G = ctx.build_superops(U, rates)
    st.apply_layer([q], G, +1)
    dims, centre, ln, lf = st.info()
    Gh = G.cpu().numpy()
    assert dims[q + 1] == chi and centre == q + 1
    for inst in range(n_inst):
        left, right, f, nrm, s = mps.two_site_update(A, B, Gh[inst, 0], chi, +1)
        assert s[chi] < 0.1 * s[chi - 1]
        L = st.read_site(inst, q).astype(np.complex128)
        R = st.read_site(inst, q + 1).astype(np.complex128)
        got = np.einsum("asc,ctb->astb", L, R).reshape(4 * d, 4 * d)
        ref = np.einsum("asc,ctb->astb", left, right).reshape(4 * d, 4 * d)
        assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max(), (inst, np.abs(got - ref).max())
        # log f from the residual's weight (1e-6); the stored factor's norm carries the tensor
        # cores' truncating float32 accumulation over K = 2048 (a few 1e-6 in log)
        assert abs(lf[inst] - math.log(f)) < 1e-6, (inst, lf[inst] - math.log(f))
        assert abs(ln[inst] - math.log(nrm)) < 3e-5, (inst, ln[inst] - math.log(nrm))
        Lm = L.reshape(-1, chi)
        assert np.abs(Lm.conj().T @ Lm - np.eye(chi)).max() < 1e-4
    st.close()


@pytest.mark.parametrize("dtype,tol", [(1, 1e-8), (0, 1e-4)])
def test_compression_sweep_vs_oracle(ctx, dtype, tol):
    from paper_2501_13237_gb300 import nne, runner
    n = 8
    c = wl.brickwork_circuit(n, 6, 21)
    rates = np.array([[0.01, 0.005, 0.0, 0.0]])
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_zz(n), n)
    st, _, _ = runner.emulate(ctx, c, rates, 64, paulis, dtype)
    dl = st.truncate(6)
    vals, lf = st.expect(paulis)
    ref_st = mps.run(c, rates[0], 64)
    before = ref_st.log_fid
    ref_st.truncate(6)
    ref = ref_st.expect_codes(paulis)
    assert np.abs(vals[0] - ref).max() < tol
    assert abs(dl[0] - (ref_st.log_fid - before)) < tol * 10
    st.close()


@pytest.mark.parametrize("method", [0, 1, 2])
def test_fit_kernel_vs_oracle(ctx, method):
    rng = np.random.default_rng(7 + method)
    lams = np.array([1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
    n_obs = 40
    a = rng.uniform(-1, 1, n_obs)
    b = rng.uniform(0.0, 0.6, n_obs)
    cst = rng.uniform(-0.05, 0.05, n_obs) * (method == 2)
    vals = a[None, :] * np.exp(-b[None, :] * lams[:, None]) + cst[None, :]
    vals = vals * (1 + 0.02 * rng.standard_normal(vals.shape))
    vals[:, 3] = [0.1, -0.2, 0.05, -0.1, 0.3, -0.01]      # sign changes: criteria 2-3 / fallback
    vals[:, 4] = [1e-12, 2e-12, 0.2, 0.1, 0.05, 0.02]     # criterion 2
    log_fid = np.log(np.array([0.2, 0.5, 0.9, 0.995, 0.999, 0.9999]))
    est, st = ctx.extrapolate(lams, vals, log_fid, method=method, degree=2, lambda_star=1.0)
    ref, rst = ofit.extrapolate(method, lams, vals, 1.0, log_fid=log_fid, degree=2)
    assert (st == rst).all()
    tol = 1e-10 if method != 2 else 1e-7
    assert np.abs(est - ref).max() < tol * max(1.0, np.abs(ref).max()), np.abs(est - ref).max()


def test_serial_layers_option_matches_sub_batches(ctx):
    """NNE_OPT_SERIAL_LAYERS runs a sub-batched state's layers on one stream:
    same results up to the rounding of GEMM split choices."""
    from paper_2501_13237_gb300 import nne, runner
    n, chi = 10, 256
    c = wl.brickwork_circuit(n, 7, 31)
    rates = np.stack([wl.NoiseModel(depol2=0.01, dephase=0.005).rates(l) for l in (1, 2, 3, 4)])
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    layers = runner.build_layer_superops(ctx, c, rates)
    out = []
    for serial in (0, 1):
        nne.set_option(nne.OPT_SERIAL_LAYERS, serial)
        try:
            st, vals, lf = runner.emulate(ctx, c, rates, chi, paulis, nne.C64, layers=layers)
            st.close()
        finally:
            nne.set_option(nne.OPT_SERIAL_LAYERS, 0)
        out.append((vals, lf))
    # complex64 tolerance: split-K choices depend on the batch size (measured 1.7e-5)
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-4
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-4
    assert (out[0][1] < -1e-4).all()          # truncation happens (bond 256 < 4^5)


def test_non_finite_state_reports_noconv(ctx):
    """A non-finite centre norm ends in NNE_ERR_NOCONV at the next sync (the
    gate bookkeeping's own check; nothing traps): a NaN site written on the
    host, one gate on it (bond 1, so the untruncated identity branch runs)."""
    from paper_2501_13237_gb300 import nne
    st = nne.State(ctx, 6, 8, 2, 1)
    st.write_site(0, 2, np.full((1, 4, 1), np.nan, complex))
    G = ctx.build_superops(np.stack([np.eye(4, dtype=complex)]), np.zeros((2, 4)))
    st.apply_layer([2], G, +1)
    with pytest.raises(nne.NNEError) as e:
        st.sync()
    assert e.value.status == -4
    st.close()


def test_checkpoint_restore_continues_bit_for_bit(ctx):
    """A state saved after four layers (sites, bond dims, centre, log-norm,
    log F) and restored into a fresh state continues exactly like the
    uninterrupted one (same kernels on the same data)."""
    from paper_2501_13237_gb300 import nne, runner
    n, chi = 8, 16
    c = wl.brickwork_circuit(n, 8, 41)
    rates = np.stack([wl.NoiseModel(depol2=0.02, dephase=0.01).rates(l) for l in (1, 2)])
    layers = runner.build_layer_superops(ctx, c, rates)
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    for dtype in (0, 1):
        a = nne.State(ctx, n, chi, 2, dtype)
        runner.evolve(a, layers[:4])
        ck = a.checkpoint()
        runner.evolve(a, layers[4:])
        va, lfa = a.expect(paulis)
        a.close()
        b = nne.State(ctx, n, chi, 2, dtype)
        b.restore(ck)
        dims, centre, ln, lf = b.info()
        assert np.array_equal(dims, ck["dims"]) and centre == ck["centre"] and np.array_equal(lf, ck["log_fid"])
        runner.evolve(b, layers[4:])
        vb, lfb = b.expect(paulis)
        b.close()
        assert np.array_equal(va, vb) and np.array_equal(lfa, lfb)
        assert (lfa < -1e-6).all()


def _tiny_noise(rng, shape, lo=1e-24, hi=1e-7):
    mag = np.exp(rng.uniform(np.log(lo), np.log(hi), shape))
    return mag * np.exp(2j * np.pi * rng.uniform(size=shape))


@pytest.mark.parametrize("dtype,tol", [(1, 1e-12), (0, 1e-6)])
@pytest.mark.parametrize("direction", [+1, -1])
def test_gauge_moves_on_nearly_null_columns(ctx, dtype, tol, direction):
    """Clifford circuits leave site tensors that are scaled permutations plus
    rounding noise spread over many decades (1e-24 .. 1e-7): the QR and LQ of
    a gauge move then meet reflector pivots and column remainders whose
    float32 squares are denormal.  An identity gate after the move must
    return theta unchanged (up to the kept norm): the reflectors stay unitary
    only with the pivots and norms formed in float64."""
    import torch
    from paper_2501_13237_gb300 import nne
    rng = np.random.default_rng(11)
    # 3 sites, bonds 1, 4, 4, 1; the middle tensor as a 16 x 4 (direction -1, QR
    # of M1) or 4 x 16 (direction +1, LQ of M1) matrix with one large entry per column
    big = np.zeros((16, 4), complex)
    for j, s in enumerate((0.52, 0.48, 0.48, 0.52)):
        big[4 * j, j] = s * np.exp(1j * rng.uniform(0, 2 * np.pi))
    P = big + _tiny_noise(rng, (16, 4))
    M1 = (P.conj().T if direction > 0 else P).reshape(4, 4, 4)
    M0 = np.eye(4, dtype=complex).reshape(1, 4, 4)
    M2 = np.eye(4, dtype=complex).reshape(4, 4, 1)
    if dtype == 0:
        M0, M1, M2 = (m.astype(np.complex64) for m in (M0, M1, M2))
    st = nne.State(ctx, 3, 4, 1, dtype)
    for k, M in enumerate((M0, M1, M2)):
        st.write_site(0, k, M)
    st.set_centre(1 if direction > 0 else 0)
    G = torch.from_numpy(np.eye(16, dtype=complex)[None, None].copy()).cuda()
    q = 0 if direction > 0 else 1
    st.apply_layer([q], G, direction)
    st.sync()
    A = [st.read_site(0, k).astype(complex) for k in range(3)]
    st.close()
    if direction > 0:
        before = np.einsum("asc,ctb->astb", M0.astype(complex), M1.astype(complex)).reshape(-1)
        after = np.einsum("asc,ctb->astb", A[0], A[1]).reshape(-1)
    else:
        before = np.einsum("asc,ctb->astb", M1.astype(complex), M2.astype(complex)).reshape(-1)
        after = np.einsum("asc,ctb->astb", A[1], A[2]).reshape(-1)
    err = np.abs(after / np.linalg.norm(after) - before / np.linalg.norm(before)).max()
    assert err < tol, err
