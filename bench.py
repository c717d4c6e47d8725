#!/usr/bin/env python
"""Throughput of the NZNE hot path on GB300: noisy VMPO gate steps at chi = 512.

Workload: n = 100 qubits, 1D brickwork of Haar-random U(4) gates (seed 0),
every gate followed by two-qubit depolarizing p = 5e-4*lambda, amplitude
damping gamma = 1e-3*lambda and dephasing 5e-4*lambda on both qubits, 8 noise
levels lambda = 1..8 run as 8 instances of one state, chi = 512, complex64
(split-TF32 tensor-core GEMMs), the SVD truncation of Sec. 2.1.2 reached by
subspace iteration (k = 640 columns, 4 power iterations, Rayleigh-Ritz with
a float64-quality eigensolve), observables all <Z_i> and
<X_i X_i+1>, weighted log-linear extrapolation (exponential fallback) to
lambda* = 1.  Synthetic inputs from workloads/ (no datasets).

One step = two brickwork layers of the saturated regime (99 gates x 8
instances = 792 two-qubit gate+truncation steps, every bond at chi = 512)
followed by the expectation sweep over all 199 observables and the fit.
The state is first evolved through the layers in which the bond dimension
is still growing (untimed set-up); steps then continue the evolution layer
after layer.  The state (~6.7 GB) is larger than L2, so no flush is needed.

value      gate steps per second, device-resident inputs (U, rates on HBM),
           CUDA events on the library's stream, max over ranks.
e2e        the same metric with the step's inputs copied from pinned host
           memory and <P>, log F and the fit read back every step.
roofline   the dominant kernel class from live CUDA-event timing of one more
           step run with per-launch event pairs (nne_prof_collect; the
           headline steps are timed without them) and its layers on one
           stream (NNE_OPT_SERIAL_LAYERS), so that each launch is timed alone;
           achieved = algorithmic flops per launch / average launch time.
fp64_path  the plain float64 path on the same GPU: one instance (lambda = 1),
           complex128, exact truncation (Gram matrix + float64 eigensolve),
           gate steps timed one call each from the saturated state.
accuracy   <P> of the fast path against the complex128 exact-SVD path after
           the same prefix of gates from the same saturated state.
measured_peaks  TF32 and FP64 torch.matmul rates of this GPU (roofline peaks).
cpu_baseline / --impl reference: the CPU oracle (NumPy, float64) timed on a
           bounded sample: full-size gate steps at chi = 512 on the host cores.
serving    an open-loop Poisson request stream through nne_submit / nne_poll
           (whole jobs, 4 worker streams; sizes reduced, see serving_run):
           p50 / p99 latency, requests/s and gate steps/s.
batch      the 64-circuit batch workload (n 16-64, depth 10-40, chi 32-128,
           5 levels, complex64) submitted at once to the same server: gate
           steps/s and circuits/s over the whole batch (see batch_run).

Multi-GPU: replicas only (each rank runs its own instance of the job with its
own circuit seed, no data-path collective; scaling "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

CHI = 512
SUBSPACE_COLS = 640          # k: columns of the subspace iteration (chi + 128)
POWER_ITERS = 4              # q: power iterations, each re-orthonormalised
LAYERS_PER_STEP = 2
SATURATE_LAYERS = 6          # bond dims 4, 16, 64, 256, 512 reached by layer 5
FP64_GATES = 4               # gate steps timed on the plain complex128 single-instance path
CHECK_GATES = 16             # prefix on which <P> of the fast path is compared with complex128 exact
CHECK_LEVELS = (0, 7)        # noise levels (lambda = 1 and 8) of that comparison


def peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        pk["source"] = "measured"
        return pk
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"nne_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_steps(n_steps: int, chi: int = CHI, seed: int = 0):
    """Time oracle gate steps at full size (random bulk site tensors, chi x 4 x chi)."""
    import workloads as wl
    from oracle import channels, mps
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((chi, 4, chi)) + 1j * rng.standard_normal((chi, 4, chi))) / math.sqrt(2)
    B = (rng.standard_normal((chi, 4, chi)) + 1j * rng.standard_normal((chi, 4, chi))) / math.sqrt(2)
    G = channels.gate_superop(wl.haar_u4(rng), wl.n100().noise.rates(1.0))
    t0 = time.perf_counter()
    for i in range(n_steps):
        mps.two_site_update(A, B, G, chi, +1 if i % 2 == 0 else -1)
    return time.perf_counter() - t0


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_steps(1)
    dt = cpu_oracle_steps(args.steps)
    v = args.steps / dt
    cores = threads_used()
    line = {"metric": "2q gate+truncation steps/s at chi=512", "value": v, "unit": "gate_steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "n100_d30_chi512_8lambda", "sample": "bulk gate steps chi=512 (X 2048x2048)"},
            "cpu_baseline": {"value": v, "unit": "gate_steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} bulk gate steps at chi=512, NumPy/LAPACK float64"},
            "e2e": {"value": v, "unit": "gate_steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", action="store_true", help="print the per-kernel-class breakdown to stderr")
    ap.add_argument("--serving", type=int, default=40,
                    help="requests of the open-loop serving sample added to the line (0: none)")
    ap.add_argument("--serving-rate", type=float, default=20.0, help="offered requests per second")
    ap.add_argument("--batch", type=int, default=64,
                    help="circuits of the 64-circuit batch workload added to the line (0: none)")
    ap.add_argument("--no-checks", action="store_true",
                    help="skip the float64 arm, the <P> check, the peak and CPU measurements (profiling runs)")
    ap.add_argument("--subbatches", type=int, default=None,
                    help="concurrent sub-batches per state (NNE_OPT_SUBBATCHES; library default when omitted)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import workloads as wl
    from paper_2501_13237_gb300 import nne, replicas, runner

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    w = wl.n100(seed=replicas.replica_seed(rank))
    rates = w.rate_table()
    n_inst = rates.shape[0]
    paulis = wl.pauli_codes(w.observables, w.n)
    plan = runner.layer_plan(w.circuit)
    ctx = nne.Context(local)
    if args.subbatches is not None:
        nne.set_option(nne.OPT_SUBBATCHES, args.subbatches)
    st = nne.State(ctx, w.n, CHI, n_inst, nne.C64, nne.TRUNC_RSVD, w.bits())
    st.set_sketch(wl.gaussian_sketch(4 * CHI, SUBSPACE_COLS, 1234).astype(np.complex64), POWER_ITERS)

    dev = f"cuda:{local}"
    U_dev = [torch.from_numpy(np.ascontiguousarray(us)).to(dev) for _, us, _ in plan]
    U_pin = [torch.from_numpy(np.ascontiguousarray(us)).pin_memory() for _, us, _ in plan]
    rates_dev = torch.from_numpy(rates).to(dev)
    rates_pin = torch.from_numpy(rates).pin_memory()
    G_buf = [torch.empty((n_inst, len(qs), 16, 16), dtype=torch.complex128, device=dev) for qs, _, _ in plan]
    lams = np.array(w.lambdas)

    # set-up: evolve through the growing-bond layers
    for li in range(SATURATE_LAYERS):
        qs, _, d = plan[li]
        st.apply_layer(qs, ctx.build_superops(U_dev[li], rates_dev, out=G_buf[li]), d)
    st.sync()
    # the saturated state of two levels, for the complex128 comparison after the timed steps
    snap = snapshot(st, CHECK_LEVELS) if rank == 0 and not args.no_checks else None
    cursor = [SATURATE_LAYERS]

    def next_layers():
        out = []
        for _ in range(LAYERS_PER_STEP):
            li = cursor[0]
            out.append(li)
            cursor[0] = cursor[0] + 1 if cursor[0] + 1 < len(plan) else SATURATE_LAYERS
        return out

    gates_per_step = 0
    h2d = d2h = 0

    def step(host_inputs: bool):
        nonlocal gates_per_step, h2d, d2h
        gates = 0
        b_in = 0
        for li in next_layers():
            qs, _, d = plan[li]
            if host_inputs:
                G = ctx.build_superops(U_pin[li].numpy(), rates_pin.numpy(), out=G_buf[li])
                b_in += U_pin[li].numel() * 16 + rates_pin.numel() * 8
            else:
                G = ctx.build_superops(U_dev[li], rates_dev, out=G_buf[li])
            st.apply_layer(qs, G, d)
            gates += len(qs) * n_inst
        vals, lf = st.expect(paulis)
        est, status = ctx.extrapolate(lams, vals.real, lf, method=nne.FIT_EXP_LOGLIN, lambda_star=w.lambda_star)
        gates_per_step = gates
        if host_inputs:
            h2d = b_in + paulis.nbytes + vals.real.nbytes + lf.nbytes + lams.nbytes
            d2h = vals.real.nbytes * 2 + lf.nbytes + est.nbytes + status.nbytes
        return est

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(host_inputs: bool, K: int, prof: bool = False):
        stream = ctx.stream
        barrier()
        if prof:
            nne.prof_collect()
            nne.prof_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = nne.kernel_launches()
        torch.cuda.nvtx.range_push("timed_steps")     # lets a profiler select the timed launches
        e0.record(stream)
        for _ in range(K):
            step(host_inputs)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        launches = nne.kernel_launches() - l0
        pr = None
        if prof:
            nne.prof_enable(False)
            pr = nne.prof_collect()
        ms = e0.elapsed_time(e1)
        # slowest rank's time, every rank's gate steps
        ms, units = replicas.aggregate(ms, gates_per_step * K, dist, dev)
        return ms, launches, pr, units

    for _ in range(args.warmup):
        step(False)
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches, _, units = timed(False, args.steps)
    clk = clocks.stop()
    ms_e2e, _, _, units_e2e = timed(True, 1)
    # per-kernel-class breakdown from a separate profiled step (event pairs around
    # every launch add host work, so the headline is timed without them); its
    # layers run on one stream, so each launch's events time that kernel alone
    nne.set_option(nne.OPT_SERIAL_LAYERS, 1)
    ms_prof, _, prof, _ = timed(False, 1, prof=True)
    nne.set_option(nne.OPT_SERIAL_LAYERS, 0)
    # the same steps with the truncation's eigensolve in float32 (NNE_OPT_EIG_FP64 = 0)
    nne.set_option(nne.OPT_EIG_FP64, 0)
    step(False)
    ms_f32, _, _, units_f32 = timed(False, args.steps)
    nne.set_option(nne.OPT_EIG_FP64, 1)

    value = units / (ms / 1e3)
    e2e = units_e2e / (ms_e2e / 1e3)
    value_f32 = units_f32 / (ms_f32 / 1e3)

    # roofline for the dominant kernel class
    pk = peaks()
    dominant = max(prof.items(), key=lambda kv: kv[1][0])
    prof_summary = {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]}
    prof_summary["_step_ms"] = round(ms_prof, 3)
    roof = None
    fast_lat = gate_latencies(st, ctx, plan, cursor[0], rates_dev, 6)
    cpu = None
    fp64 = check = pk_meas = roof_gemm = None
    if rank == 0 and not args.no_checks:
        st.close()
        torch.cuda.empty_cache()
        fp64 = fp64_path(ctx, w, plan, snap, rates)
        check = prefix_check(ctx, w, plan, snap, rates, paulis)
        pk_meas = measure_peaks(dev)
        roof = roofline(dominant, prof, pk, pk_meas)
        roof_gemm = roofline_of("gemm_tc", prof, pk_meas) if prof.get("gemm_tc", (0, 0, 0))[1] else None
        n_cpu = 3
        dt = cpu_oracle_steps(n_cpu)
        cpu = {"value": n_cpu / dt, "unit": "gate_steps/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"{n_cpu} bulk gate steps at chi=512 (X 2048x2048 complex128, LAPACK SVD)"}
    if args.profile and rank == 0:
        for k, (t, c, wk) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
            if c:
                sys.stderr.write(f"  {k:18s} {t:10.2f} ms  {c:7d} launches  {100 * t / max(ms_prof, 1e-9):5.1f}%\n")
    if rank != 0 or args.no_checks:
        st.close()
    serving = None
    if rank == 0 and args.serving > 0:
        serving = serving_run(args.serving, args.serving_rate, 0, 4, local)
    batch = None
    if rank == 0 and args.batch > 0:
        batch = batch_run(args.batch, 4, local)
    if rank == 0:
        line = {"metric": "2q gate+truncation steps/s at chi=512", "value": value, "unit": "gate_steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
                "data": "synthetic",
                "config": {"workload": "n100_d30_chi512_8lambda", "chi": CHI, "n": w.n, "n_lambda": n_inst,
                           "truncation": (f"SVD truncation to chi (Sec. 2.1.2) by subspace iteration: k={SUBSPACE_COLS} "
                                          f"columns, q={POWER_ITERS} power iterations, Rayleigh-Ritz with a "
                                          "float64-quality eigensolve (double-float Householder reduction on the "
                                          "float32 pipes, float64 bisection and inverse iteration); complex64, 3xTF32 "
                                          "tensor-core GEMMs; <P> checked against the complex128 exact-SVD path "
                                          "(accuracy); the same steps with a float32 eigensolve in float32_eigensolve"),
                           "step": f"{LAYERS_PER_STEP} saturated brickwork layers ({gates_per_step} gate steps) "
                                   "+ 199-observable sweep + fit",
                           "l2": "inputs larger than L2 (state ~6.7 GB)", "parallelism": f"replicas{world}"},
                "e2e": {"value": e2e, "unit": "gate_steps/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches), "roofline": roof, "roofline_gemm": roof_gemm, "cpu_baseline": cpu,
                "clocks": clk,
                "fp64_path": fp64, "fast_gate_latency_ms": fast_lat, "accuracy": check,
                "float32_eigensolve": {"value": value_f32, "unit": "gate_steps/s", "steps": args.steps,
                                       "ms_per_step": ms_f32 / args.steps,
                                       "what": "the same timed steps with the truncation's eigensolve in float32 "
                                               "(NNE_OPT_EIG_FP64 = 0); its <P> error in accuracy.float32_eigensolve"},
                "measured_peaks": pk_meas,
                "kernel_classes_ms": prof_summary, "serving": serving, "batch": batch}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# FP32 SIMT peak of GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz max SM clock.
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
ALU_CLASSES = {"gemm": "float32 SIMT GEMMs", "wy_apply": "split-K block-reflector products",
               "qr_factor": "Householder panel factorisation", "tridiag": "Hermitian tridiagonalisation"}


def roofline_of(name, prof, meas):
    t_ms, count, work = prof[name]
    return roofline((name, (t_ms, count, work)), prof, None, meas)


def roofline(dominant, prof, pk, meas):
    """Roofline entry of the dominant kernel class, from live CUDA-event timing.

    achieved = the algorithmic real flops the library records per launch of the
    class (8 per complex multiply-add; 16/3 n^3 per tridiagonalisation) summed
    over the timed region / the class's summed launch time.  Tensor-core GEMMs
    (complex64 as three TF32 products per real product) take the TF32 peak
    measured in this run with torch.matmul, sustained (the class is timed inside
    a seconds-long step); the float64 tridiagonalisation takes the float64
    matmul rate measured in this run; the others run on the FP32 pipes and take
    the derived FP32 SIMT peak.  `roofline_gemm` in the line is the same entry
    for the tensor-core GEMM class whatever the dominant class is."""
    name, (t_ms, count, work) = dominant
    if count == 0 or t_ms <= 0:
        return None
    # traffic: no ncu capture of this build's launch mix for the class (the GEMM class mixes ~20
    # shapes per gate; per-shape DRAM counters are in profiles/), so null
    out = {"kernel": name, "launches": count, "avg_launch_ms": t_ms / count, "traffic": None}
    achieved = work / (t_ms / 1e3) / 1e12 if work > 0 else None
    if name == "gemm_tc" and achieved is not None:
        peak = meas["tf32_tflops_sustained"]
        out.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "measured in this run: torch.matmul float32 with TF32, 8192^3, back to back "
                                   "for 2 s (sustained); complex64 runs as 3 TF32 products per real product, so "
                                   "at most 1/3 of it is algorithmic"})
    elif name == "tridiag" and achieved is not None:
        # the float64 Householder reduction of the complex64 path's Rayleigh-Ritz matrix
        peak = meas["fp64_tflops"]
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "what": "Hermitian tridiagonalisation in float64 ((16/3) n^3 flops per matrix)",
                    "peak_source": "measured in this run: torch.matmul float64 4096^3 (float64 pipes)"})
    elif name in ALU_CLASSES and achieved is not None:
        out.update({"bound": "alu", "achieved": achieved, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SIMT_PEAK_TFLOPS, "what": ALU_CLASSES[name],
                    "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz"})
    else:
        out.update({"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None})
    return out


def snapshot(st, levels):
    """Host copy of the given levels of a state: sites, centre, log-norm, log F."""
    dims, centre, ln, lf = st.info()
    return {"levels": list(levels), "centre": centre, "ln": ln[list(levels)], "lf": lf[list(levels)],
            "sites": [[st.read_site(i, k) for k in range(st.n)] for i in levels]}


def restore(ctx, nne, w, snap, which, dtype, trunc, k=None, q=None):
    """A new state of the snapshot's levels `which` (indices into snap['levels'])."""
    s = nne.State(ctx, w.n, CHI, len(which), dtype, trunc, w.bits())
    if trunc == nne.TRUNC_RSVD:
        import workloads as wl
        om = wl.gaussian_sketch(4 * CHI, k, 1234)
        s.set_sketch(om.astype(np.complex64 if dtype == nne.C64 else np.complex128), q)
    for j, i in enumerate(which):
        for kk, M in enumerate(snap["sites"][i]):
            s.write_site(j, kk, M)
    s.set_centre(snap["centre"])
    s.set_log(snap["ln"][list(which)], snap["lf"][list(which)])
    s.sync()
    return s


def gate_latencies(st, ctx, plan, li, rates_dev, n_gates):
    """Per-gate-step latency (ms) of the fast path: the first gates of layer li,
    one nne_apply_layer call each, CUDA events on the library's stream."""
    import torch
    qs, us, d = plan[li]
    U = torch.from_numpy(np.ascontiguousarray(us[:n_gates])).to(rates_dev.device)
    G = ctx.build_superops(U, rates_dev)
    Gg = [G[:, g:g + 1].contiguous() for g in range(n_gates)]
    ms = []
    for g in range(n_gates):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        st.apply_layer([qs[g]], Gg[g], d)
        e1.record(ctx.stream)
        st.sync()
        ms.append(e0.elapsed_time(e1))
    return {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)), "gates": n_gates,
            "n_inst": int(rates_dev.shape[0]), "what": "one gate step of all levels, complex64 fast path"}


def fp64_path(ctx, w, plan, snap, rates):
    """The plain float64 path on one instance (lambda = 1): complex128 state,
    exact truncation (Gram matrix and float64 eigensolve), the first gates of
    the layer after the saturated ones, one call per gate, CUDA events."""
    import torch
    from paper_2501_13237_gb300 import nne
    s = restore(ctx, nne, w, snap, [0], nne.C128, nne.TRUNC_EXACT)
    qs, us, d = plan[SATURATE_LAYERS]
    G = ctx.build_superops(np.ascontiguousarray(us[:FP64_GATES + 1]), np.ascontiguousarray(rates[:1]))
    Gg = [G[:, g:g + 1].contiguous() for g in range(FP64_GATES + 1)]
    s.apply_layer([qs[0]], Gg[0], d)       # warm-up
    s.sync()
    ms = []
    for g in range(1, FP64_GATES + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        s.apply_layer([qs[g]], Gg[g], d)
        e1.record(ctx.stream)
        s.sync()
        ms.append(e0.elapsed_time(e1))
    s.close()
    torch.cuda.empty_cache()
    return {"value": 1e3 * len(ms) / sum(ms), "unit": "gate_steps/s", "dtype": "c128", "n_inst": 1,
            "truncation": "exact: Gram matrix + float64 Householder/bisection/inverse iteration",
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)), "gates": len(ms)}


def prefix_check(ctx, w, plan, snap, rates, paulis):
    """<P> error of the fast path: from the same saturated state, the first
    CHECK_GATES gates of the next layer on the fast complex64 path and on the
    complex128 exact-SVD path, then every observable on both."""
    import torch
    from paper_2501_13237_gb300 import nne
    qs, us, d = plan[SATURATE_LAYERS]
    lev = list(snap["levels"])
    G = ctx.build_superops(np.ascontiguousarray(us[:CHECK_GATES]), np.ascontiguousarray(rates[lev]))
    out, secs = {}, {}
    for name, dt, tr, k, q, e in (("c128", nne.C128, nne.TRUNC_EXACT, None, None, 1),
                                  ("fast", nne.C64, nne.TRUNC_RSVD, SUBSPACE_COLS, POWER_ITERS, 1),
                                  ("fast_fp32_eig", nne.C64, nne.TRUNC_RSVD, SUBSPACE_COLS, POWER_ITERS, 0)):
        nne.set_option(nne.OPT_EIG_FP64, e)
        s = restore(ctx, nne, w, snap, list(range(len(lev))), dt, tr, k, q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.apply_layer(qs[:CHECK_GATES], G, d)
        s.sync()
        secs[name] = time.perf_counter() - t0
        out[name] = s.expect(paulis)
        s.close()
        nne.set_option(nne.OPT_EIG_FP64, 1)
        torch.cuda.empty_cache()
    err = np.abs(out["fast"][0].real - out["c128"][0].real)
    err32 = np.abs(out["fast_fp32_eig"][0].real - out["c128"][0].real)
    steps = CHECK_GATES * len(lev)
    return {"max_abs_err_P": float(err.max()), "mean_abs_err_P": float(err.mean()),
            "dlogF": (out["fast"][1] - out["c128"][1]).tolist(), "prefix_gates": CHECK_GATES,
            "levels_lambda": [float(w.lambdas[i]) for i in lev], "n_obs": int(paulis.shape[0]),
            "vs": "complex128 exact-SVD path on the GPU, same saturated state",
            "float32_eigensolve": {"max_abs_err_P": float(err32.max()),
                                   "dlogF": (out["fast_fp32_eig"][1] - out["c128"][1]).tolist(),
                                   "what": "the same path with the Rayleigh-Ritz eigensolve in float32 "
                                           "(NNE_OPT_EIG_FP64 = 0)"},
            "gate_steps_per_s_prefix": {k2: steps / v for k2, v in secs.items()}}


def measure_peaks(dev):
    """Dense TF32 and FP64 matmul rates of this GPU (torch.matmul, cuBLAS):
    TF32 8192^3 best of 10 (burst) and back to back for 2 s (sustained), FP64
    4096^3 best of 3."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, reps, tf32 in (("tf32", torch.float32, 8192, 10, True), ("fp64", torch.float64, 4096, 3, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=dev, dtype=dt)
            b = torch.randn(n, n, device=dev, dtype=dt)
            c = a @ b
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                c = a @ b
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[f"{name}_tflops"] = 2 * n ** 3 / best / 1e12
            if name == "tf32":
                t0 = time.perf_counter()
                cnt = 0
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                while time.perf_counter() - t0 < 2.0:
                    c = a @ b
                    cnt += 1
                    if cnt % 8 == 0:
                        torch.cuda.synchronize()
                e1.record()
                torch.cuda.synchronize()
                out["tf32_tflops_sustained"] = cnt * 2 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "torch.matmul: float32 with TF32 8192^3 (best of 10; back to back 2 s), float64 4096^3 best of 3"
    return out


def serving_run(n_requests: int, rate_per_s: float, seed: int, workers: int, device: int = 0):
    """Open-loop request stream through nne_submit / nne_poll: Poisson arrivals,
    requests drawn like the serving workload at reduced sizes (n in [8, 32],
    depth in [5, 20], chi in {16, 32, 64, 128}, 4-8 levels, random channel mix,
    all <Z_i>, complex64, exact truncation with the float32 eigensolve: at these bonds
    the float64 reduction of a 512-wide Gram matrix takes the slow path and the
    float32 one meets the 1e-4 budget).  Latency = completion - arrival."""
    import workloads as wl
    from paper_2501_13237_gb300 import nne, replicas, runner
    reqs = wl.serving_stream(seed, n_requests, rate_per_s, n_range=(8, 32), depth_range=(5, 20),
                             chis=(16, 32, 64, 128))
    jobs = [runner.job_for(r.workload, dtype=nne.C64) for r in reqs]
    nne.set_option(nne.OPT_EIG_FP64, 0)
    srv = nne.Server(device, hbm_budget_bytes=150 << 30, workers=workers)
    t0 = time.perf_counter()
    tickets = []
    for r, j in zip(reqs, jobs):
        dt = r.arrival_s - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(j))
    res = [srv.poll(t) for t in tickets]
    srv.close()
    nne.set_option(nne.OPT_EIG_FP64, 1)
    bad = [r for r in res if r["status"] != 0]
    lat = np.array([r["t_end"] - r["t_submit"] for r in res])
    span = max(r["t_end"] for r in res) - min(r["t_submit"] for r in res)
    steps = sum(r["gate_steps"] for r in res)
    return {"requests": n_requests, "offered_per_s": rate_per_s, "workers": workers, "failed": len(bad),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "requests_per_s": n_requests / span, "gate_steps_per_s": steps / span,
            "sizes": "n 8-32, depth 5-20, chi 16-128, 4-8 levels, c64 exact truncation, float32 eigensolve"}


def batch_run(n_circuits: int, workers: int, device: int = 0):
    """The 64-circuit batch workload (n ~ U[16,64], depth ~ U[10,40], chi in
    {32, 64, 128}, 5 levels of depolarizing + dephasing, all <Z_i>, exponential
    fit; complex64, exact truncation, float32 eigensolve) submitted at once to a server with
    `workers` streams: wall time from the first submit to the last completion."""
    import workloads as wl
    from paper_2501_13237_gb300 import nne, runner
    ws = wl.batch64(0, n_circuits)
    jobs = [runner.job_for(w, dtype=nne.C64) for w in ws]
    nne.set_option(nne.OPT_EIG_FP64, 0)
    srv = nne.Server(device, hbm_budget_bytes=150 << 30, workers=workers)
    t0 = time.perf_counter()
    tickets = [srv.submit(j) for j in jobs]
    res = [srv.poll(t) for t in tickets]
    wall = time.perf_counter() - t0
    srv.close()
    nne.set_option(nne.OPT_EIG_FP64, 1)
    steps = sum(r["gate_steps"] for r in res)
    return {"circuits": n_circuits, "workers": workers, "failed": sum(r["status"] != 0 for r in res),
            "wall_s": wall, "gate_steps": int(steps), "gate_steps_per_s": steps / wall,
            "circuits_per_s": n_circuits / wall,
            "sizes": "n 16-64, depth 10-40, chi 32/64/128, 5 levels, c64 exact truncation, float32 eigensolve"}


if __name__ == "__main__":
    main()
