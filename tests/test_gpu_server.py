"""The serving loop on the GPU: jobs run through nne_submit / nne_poll by
concurrent workers give the same numbers as the same circuits run directly
through the state API (same kernels, bit for bit) and agree with the oracle;
the admission estimate covers what a state really allocates."""
import numpy as np
import pytest

import workloads as wl
from gpu_util import require_gpu
from oracle import fit, mps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


def _workloads():
    a = wl.Workload("a", wl.brickwork_circuit(8, 6, 3), wl.NoiseModel(depol2=0.01, amp_damp=0.005),
                    (1.0, 2.0, 3.0), 16, wl.obs_z(8) + wl.obs_xx(8), 1.0, "exp")
    b = wl.Workload("b", wl.brickwork_circuit(10, 8, 4), wl.NoiseModel(depol2=0.02, dephase=0.01),
                    (1.0, 1.5, 2.0, 3.0), 24, wl.obs_z(10), 1.0, "poly2")
    c = wl.Workload("c", wl.brickwork_circuit(6, 5, 5), wl.NoiseModel(depol2=0.005, amp_damp=0.01, dephase=0.01),
                    (1.0, 2.0), 64, wl.obs_z(6) + wl.obs_zz(6), 1.0, "exp", init_bits=(1, 0, 1, 1, 0, 0))
    return [a, b, c]


@pytest.mark.parametrize("dtype,tol", [(1, 1e-8), (0, 1e-4)])
def test_server_matches_direct_and_oracle(ctx, dtype, tol):
    from paper_2501_13237_gb300 import nne, runner
    ws = _workloads()
    jobs = [runner.job_for(w, dtype=dtype) for w in ws]
    srv = nne.Server(0, workers=3)
    tickets = [srv.submit(j) for j in jobs]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    for w, j, r in zip(ws, jobs, res):
        assert r["status"] == 0, r["error"]
        assert r["gate_steps"] == j.gate_steps
        paulis = wl.pauli_codes(w.observables, w.n)
        st, vals, lf = runner.emulate(ctx, w.circuit, w.rate_table(), w.chi, paulis, dtype, bits=w.bits())
        st.close()
        # same kernels on another stream: identical numbers
        assert np.array_equal(r["values"], vals.real)
        assert np.array_equal(r["log_fid"], lf)
        for i in range(len(w.lambdas)):
            ref_st = mps.run(w.circuit, w.rate_table()[i], w.chi, bits=w.bits())
            assert np.abs(r["values"][i] - ref_st.expect_codes(paulis).real).max() < tol
            assert abs(r["log_fid"][i] - ref_st.log_fid) < tol * max(1.0, abs(ref_st.log_fid))
        method = runner.FIT_CODES[w.fit]
        est, fst = fit.extrapolate(method, np.asarray(w.lambdas), r["values"], w.lambda_star, log_fid=r["log_fid"],
                                   degree=j.struct.fit_degree)
        assert np.array_equal(r["fit_status"], fst)
        assert np.allclose(r["estimate"], est, rtol=1e-8, atol=1e-10)


def test_server_budget_serialises(ctx):
    from paper_2501_13237_gb300 import nne, runner
    ws = _workloads()
    jobs = [runner.job_for(w, dtype=0) for w in ws]
    big = max(j.bytes() for j in jobs)
    srv = nne.Server(0, hbm_budget_bytes=int(big * 1.5), workers=3)
    tickets = [srv.submit(j) for j in jobs]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert all(r["status"] == 0 for r in res), [(r["status"], r["error"]) for r in res]
    # at every start, the jobs then running fit in the budget together
    for r in res:
        t = r["t_start"]
        held = sum(q["bytes"] for q in res if q["t_start"] <= t < q["t_end"])
        assert held <= int(big * 1.5)
    assert max(r["bytes"] for r in res) == big


def test_server_rsvd_job(ctx):
    from paper_2501_13237_gb300 import nne, runner
    w = wl.Workload("r", wl.brickwork_circuit(10, 10, 3), wl.NoiseModel(depol2=0.02, amp_damp=0.01, dephase=0.01),
                    (1.0, 3.0), 16, wl.obs_z(10) + wl.obs_xx(10), 1.0, "exp")
    # subspace iteration (k = 3 chi, six power iterations) against the exact SVD truncation
    om = wl.gaussian_sketch(4 * 16, 48, 9).astype(np.complex64)
    job = runner.job_for(w, dtype=0, trunc=nne.TRUNC_RSVD, sketch=om, power_iters=6)
    srv = nne.Server(0, workers=1)
    r = srv.poll(srv.submit(job))
    srv.close()
    assert r["status"] == 0, r["error"]
    paulis = wl.pauli_codes(w.observables, w.n)
    for i in range(2):
        ref = mps.run(w.circuit, w.rate_table()[i], 16)
        assert np.abs(r["values"][i] - ref.expect_codes(paulis).real).max() < 1e-4


def test_job_bytes_cover_state(ctx):
    """The admission estimate is at least what the state and its sketch allocate."""
    from paper_2501_13237_gb300 import nne, runner
    for chi, trunc in [(16, nne.TRUNC_EXACT), (64, nne.TRUNC_EXACT), (32, nne.TRUNC_RSVD)]:
        w = wl.Workload("s", wl.brickwork_circuit(12, 2, 1), wl.NoiseModel(depol2=0.01), (1.0, 2.0, 3.0), chi,
                        wl.obs_z(12), 1.0, "exp")
        om = wl.gaussian_sketch(4 * chi, chi + 8, 1).astype(np.complex64) if trunc else None
        job = runner.job_for(w, dtype=0, trunc=trunc, sketch=om)
        c2 = nne.Context(0)
        st = nne.State(c2, w.n, chi, 3, nne.C64, trunc)
        if om is not None:
            st.set_sketch(om, 1)
        used = c2.bytes_in_use()
        st.close()
        c2.close()
        assert used <= job.bytes() <= used + (4 << 20), (chi, used, job.bytes())


def test_server_many_concurrent_jobs(ctx):
    """Twelve mixed jobs (both dtypes, several chi and sizes) on four workers:
    every one succeeds and equals its direct run bit for bit."""
    from paper_2501_13237_gb300 import nne, runner
    rng = np.random.default_rng(7)
    ws, dts = [], []
    for i in range(12):
        n = int(rng.integers(5, 12))
        w = wl.Workload(f"m{i}", wl.brickwork_circuit(n, int(rng.integers(3, 9)), 100 + i),
                        wl.NoiseModel(depol2=0.01, amp_damp=0.005 * (i % 2), dephase=0.004),
                        tuple(float(x) for x in range(1, 2 + i % 4)), int(rng.choice([8, 16, 32, 64])),
                        wl.obs_z(n), 1.0, "exp")
        ws.append(w)
        dts.append(i % 2)
    srv = nne.Server(0, workers=4)
    tickets = [srv.submit(runner.job_for(w, dtype=d)) for w, d in zip(ws, dts)]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert all(r["status"] == 0 for r in res), [(r["status"], r["error"]) for r in res]
    for w, d, r in zip(ws, dts, res):
        paulis = wl.pauli_codes(w.observables, w.n)
        st, vals, lf = runner.emulate(ctx, w.circuit, w.rate_table(), w.chi, paulis, d, bits=w.bits())
        st.close()
        assert np.array_equal(r["values"], vals.real)
        assert np.array_equal(r["log_fid"], lf)


def test_batch_subsample_vs_oracle(ctx):
    """The multi-circuit batch workload (64 circuits, n 16-64, chi 32-128, five
    levels of depolarizing + dephasing) runs as concurrent server jobs; an
    8-circuit subsample, cut to its first six layers so the oracle finishes in
    seconds, matches the oracle MPS at lambda = 1."""
    import dataclasses
    from paper_2501_13237_gb300 import nne, runner
    ws = []
    for w in wl.batch64(0)[:8]:
        c = dataclasses.replace(w.circuit, depth=6, layers=w.circuit.layers[:6], unitaries=w.circuit.unitaries[:6])
        ws.append(dataclasses.replace(w, circuit=c))
    srv = nne.Server(0, workers=4)
    tickets = [srv.submit(runner.job_for(w, dtype=0)) for w in ws]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert all(r["status"] == 0 for r in res), [(r["status"], r["error"]) for r in res]
    for w, r in zip(ws, res):
        paulis = wl.pauli_codes(w.observables, w.n)
        ref = mps.run(w.circuit, w.rate_table()[0], w.chi, bits=w.bits())
        assert np.abs(r["values"][0] - ref.expect_codes(paulis).real).max() < 1e-4
        # log F sums one complex64-rounded log f per gate (about 1e-5 each): the bound grows with the gates
        assert abs(r["log_fid"][0] - ref.log_fid) < 2e-5 * w.circuit.n_gates
        assert r["gate_steps"] == w.circuit.n_gates * len(w.lambdas)


def test_server_pauli_noise_jobs(ctx):
    """Cat-qubit and XY-model circuits through nne_submit: identical to the
    direct path (same kernels) and to the oracle VMPO within 1e-8 (complex128)."""
    from oracle import channels as ch
    from paper_2501_13237_gb300 import nne, runner
    cases = [(wl.cat_circuit(10, 24, 7), (0.005, 0.02), 4, None),
             (wl.xym_circuit(10, 5, dt=0.3), (0.01, 0.05), 6, wl.neel_bits(10))]
    paulis = wl.pauli_codes(wl.obs_z(10) + wl.obs_xx(10), 10)
    jobs = [runner.pauli_job(pc, lams, chi, paulis, dtype=nne.C128, bits=bits) for pc, lams, chi, bits in cases]
    srv = nne.Server(0, workers=2)
    res = [srv.poll(srv.submit(j)) for j in jobs]
    srv.close()
    for (pc, lams, chi, bits), j, r in zip(cases, jobs, res):
        assert r["status"] == 0, r["error"]
        assert r["gate_steps"] == j.gate_steps
        layers = runner.build_pauli_layers(ctx, pc, np.asarray(lams))
        st, vals, lf = runner.emulate(ctx, pc, None, chi, paulis, nne.C128, bits=bits, layers=layers)
        st.close()
        assert np.array_equal(r["values"], vals.real)
        assert np.array_equal(r["log_fid"], lf)
        for i, lam in enumerate(lams):
            ref = mps.run(pc, None, chi, bits=bits, Gs=ch.pauli_superops_for(pc, lam))
            assert np.abs(r["values"][i] - ref.expect_codes(paulis).real).max() < 1e-8
