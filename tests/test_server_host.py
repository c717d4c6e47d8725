"""Host logic of the serving loop (nne_submit / nne_poll) on the CPU: the
server's dry-run mode runs no GPU work, so queueing, FIFO admission under a
device-memory budget, ticket handling and argument checks are tested here."""
import time

import numpy as np
import pytest

import workloads as wl
from paper_2501_13237_gb300 import nne, runner


def _job(n=8, depth=4, chi=16, seed=0, lambdas=(1.0, 2.0)):
    w = wl.Workload("t", wl.brickwork_circuit(n, depth, seed), wl.NoiseModel(depol2=1e-3),
                    tuple(lambdas), chi, wl.obs_z(n), 1.0, "exp")
    return runner.job_for(w)


def test_job_bytes_monotone():
    small = _job(chi=16).bytes()
    assert small > 0
    assert _job(chi=64).bytes() > small
    assert _job(chi=16, lambdas=(1.0, 2.0, 3.0, 4.0)).bytes() > small
    # the bond capacity saturates at 4^(n/2): chi beyond it changes nothing
    assert _job(n=4, chi=16).bytes() == _job(n=4, chi=64).bytes()


def test_fifo_admission_under_budget():
    job = _job()
    b = job.bytes()
    srv = nne.Server(hbm_budget_bytes=2 * b + b // 2, workers=4, dry_run=True, dry_run_us=60000)
    tickets = [srv.submit(_job(seed=i)) for i in range(6)]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert all(r["status"] == -7 for r in res)            # dry run: no values
    assert all(r["bytes"] == b for r in res)
    starts = [r["t_start"] for r in res]
    assert starts == sorted(starts)                       # admitted in submission order
    # never more than two jobs inside the budget at once
    for r in res:
        mid = 0.5 * (r["t_start"] + r["t_end"])
        overlap = sum(1 for q in res if q["t_start"] <= mid < q["t_end"])
        assert overlap <= 2
    # with four workers and room for two, the six jobs take three rounds
    assert res[-1]["t_end"] - res[0]["t_start"] >= 3 * 0.06 * 0.9


def test_unlimited_budget_runs_workers_in_parallel():
    srv = nne.Server(hbm_budget_bytes=0, workers=3, dry_run=True, dry_run_us=80000)
    tickets = [srv.submit(_job(seed=i)) for i in range(3)]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert max(r["t_start"] for r in res) < min(r["t_end"] for r in res)


def test_poll_pending_and_unknown_ticket():
    srv = nne.Server(workers=1, dry_run=True, dry_run_us=200000)
    t = srv.submit(_job())
    assert srv.poll(t, timeout_ms=0) is None
    st = srv.stats()
    assert st["queued"] + st["running"] == 1
    r = srv.poll(t, timeout_ms=-1)
    assert r is not None and r["t_end"] >= r["t_start"] >= r["t_submit"]
    srv.jobs[12345] = srv.jobs.get(t, _job())
    with pytest.raises(nne.NNEError) as e:
        srv.poll(12345, timeout_ms=0)
    assert e.value.status == -1
    srv.close()


def test_oversize_job_refused():
    job = _job(chi=64)
    srv = nne.Server(hbm_budget_bytes=job.bytes() - 1, workers=1, dry_run=True)
    with pytest.raises(nne.NNEError) as e:
        srv.submit(job)
    assert e.value.status == -2
    srv.close()


@pytest.mark.parametrize("field,value", [("paulis", 5), ("rates", 2.0), ("left", 7), ("dir", 0)])
def test_bad_job_rejected(field, value):
    job = _job()
    if field == "paulis":
        job.paulis[0, 0] = value
    elif field == "rates":
        job.rates[0, 1] = value
    elif field == "left":
        job.left[0] = value
    else:
        job.layer_dir[0] = value
    srv = nne.Server(workers=1, dry_run=True)
    with pytest.raises(nne.NNEError) as e:
        srv.submit(job)
    assert e.value.status == -1
    srv.close()


def test_destroy_drops_queued_jobs():
    srv = nne.Server(workers=1, dry_run=True, dry_run_us=100000)
    for i in range(4):
        srv.submit(_job(seed=i))
    time.sleep(0.02)
    t0 = time.time()
    srv.close()                      # finishes the running job only
    assert time.time() - t0 < 0.35


def _pauli_job(lambdas=(0.005, 0.02), **kw):
    pc = wl.cat_circuit(8, 4, 2)
    return runner.pauli_job(pc, lambdas, 8, wl.pauli_codes(wl.obs_z(8), 8), **kw)


def test_pauli_noise_job_is_admitted_and_sized():
    job = _pauli_job()
    gates = int(job.layer_gates.sum())
    assert job.struct.rates is None and job.pauli.shape == (gates, 2, 16)
    # the staged Pauli table (32 doubles per gate plus the levels) replaces the 4 rates per level
    srv = nne.Server(workers=1, dry_run=True, dry_run_us=1000)
    r = srv.poll(srv.submit(job))
    srv.close()
    assert r["status"] == -7 and r["bytes"] == job.bytes() > 0


def test_pauli_noise_job_argument_checks():
    bad = _pauli_job()
    bad.pauli[3, 1, 0] += 0.5            # probabilities of gate 3 no longer sum to one
    srv = nne.Server(workers=1, dry_run=True, dry_run_us=1000)
    with pytest.raises(nne.NNEError):
        srv.submit(bad)
    neg = _pauli_job(lambdas=(0.005, 0.5))   # p_II = 1 - 5 lambda < 0 for H gates at lambda = 0.5
    with pytest.raises(nne.NNEError):
        srv.submit(neg)
    none = _pauli_job()
    none.struct.pauli_rates = None          # neither rates nor Pauli channels
    with pytest.raises(nne.NNEError):
        srv.submit(none)
    srv.close()


def test_pauli_job_follows_the_snake_schedule():
    """Gate order, directions and per-gate Pauli tables of a Pauli-noise job:
    even layers left to right, odd layers reversed, tables travelling with
    their gates (the order build_pauli_layers applies them in)."""
    pc = wl.cat_circuit(7, 5, 9)
    job = runner.pauli_job(pc, (0.01,), 8, wl.pauli_codes(wl.obs_z(7), 7))
    off = 0
    for t, qs in enumerate(pc.layers):
        g = len(qs)
        order = list(range(g)) if t % 2 == 0 else list(range(g - 1, -1, -1))
        assert job.layer_dir[t] == (1 if t % 2 == 0 else -1) and job.layer_gates[t] == g
        for k, i in enumerate(order):
            assert job.left[off + k] == qs[i]
            assert np.array_equal(job.U[off + k], pc.unitaries[t][i])
            assert np.array_equal(job.pauli[off + k, 0], pc.c0[t][i])
            assert np.array_equal(job.pauli[off + k, 1], pc.c1[t][i])
        off += g
    assert off == pc.n_gates


def test_metrics_log_jsonl(tmp_path):
    """nne_server_set_log: one JSON line per finished job with its ticket,
    status, sizes and times (latency = end - submit, on the server clock)."""
    import json
    path = tmp_path / "jobs.jsonl"
    srv = nne.Server(workers=2, dry_run=True, dry_run_us=20000, log_path=str(path))
    jobs = [_job(seed=i, lambdas=(1.0, 2.0, 3.0)) for i in range(3)]
    tickets = [srv.submit(j) for j in jobs]
    res = [srv.poll(t) for t in tickets]
    srv.set_log(None)                   # stop logging; later jobs leave no line
    srv.poll(srv.submit(_job()))
    srv.close()
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert sorted(l["ticket"] for l in lines) == sorted(tickets)
    for l in lines:
        r = res[tickets.index(l["ticket"])]
        assert l["status"] == -7 and l["error"] == "dry run: no GPU work"
        assert (l["n"], l["chi"], l["n_lambda"]) == (8, 16, 3) and l["gates"] == int(jobs[0].layer_gates.sum())
        assert l["bytes"] == r["bytes"] and l["log_fid"] == []
        assert l["t_submit"] <= l["t_start"] <= l["t_end"]
        assert abs(l["latency_s"] - (l["t_end"] - l["t_submit"])) < 1e-5
        assert abs(l["t_end"] - r["t_end"]) < 1e-5
    with pytest.raises(nne.NNEError):
        nne.Server(workers=1, dry_run=True, log_path=str(tmp_path / "missing" / "x.jsonl"))


def test_cancel_queued_and_running_requests(tmp_path):
    """nne_cancel: a queued job completes at once as cancelled and frees its
    place in the queue; a running job is not interrupted; finished or unknown
    tickets are refused."""
    import json
    log = tmp_path / "jobs.jsonl"
    srv = nne.Server(workers=1, dry_run=True, dry_run_us=150000, log_path=str(log))
    t = [srv.submit(_job(seed=i)) for i in range(3)]
    while srv.stats()["running"] == 0:
        time.sleep(0.005)
    assert srv.cancel(t[1]) is True                 # still queued
    r1 = srv.poll(t[1], timeout_ms=0)
    assert r1["status"] == nne.ERR_CANCELLED and r1["t_start"] == r1["t_end"]
    assert srv.cancel(t[0]) is False                # running: completes normally
    res = [srv.poll(t[0]), srv.poll(t[2])]
    assert [r["status"] for r in res] == [-7, -7]
    assert res[1]["t_start"] >= res[0]["t_end"] - 1e-6     # the cancelled job never ran in between
    assert res[1]["t_start"] - res[0]["t_start"] < 0.28     # one dry-run period (0.15 s), not two
    with pytest.raises(nne.NNEError):
        srv.cancel(t[2])                            # finished (and collected)
    with pytest.raises(nne.NNEError):
        srv.cancel(987654)
    srv.close()
    lines = {l["ticket"]: l for l in map(json.loads, log.read_text().splitlines())}
    assert lines[t[1]]["status"] == nne.ERR_CANCELLED and set(lines) == set(t)


def test_injected_failure_ends_only_that_job():
    """Host-side fault injection: the chosen job ends with the injected status,
    the others run, and every memory reservation is returned."""
    srv = nne.Server(hbm_budget_bytes=10 * _job().bytes(), workers=1, dry_run=True, dry_run_us=60000)
    t = [srv.submit(_job(seed=i)) for i in range(4)]
    while srv.stats()["running"] == 0:
        time.sleep(0.005)
    with pytest.raises(nne.NNEError):
        srv.inject_failure(t[0], -4)                # already running
    with pytest.raises(nne.NNEError):
        srv.inject_failure(t[2], 0)                 # not a failure status
    srv.inject_failure(t[2], -4)                    # NNE_ERR_NOCONV, as a failed eigensolve reports
    res = [srv.poll(x) for x in t]
    assert [r["status"] for r in res] == [-7, -7, -4, -7]
    assert res[2]["error"] == "injected failure"
    assert res[3]["t_start"] >= res[2]["t_end"] - 1e-6      # the queue went on after the failure
    st = srv.stats()
    srv.close()
    assert st["bytes_reserved"] == 0 and st["running"] == 0 and st["queued"] == 0
