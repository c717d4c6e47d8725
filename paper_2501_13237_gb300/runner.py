"""Brickwork schedule on top of the C ABI: which gates go into which
nne_apply_layer call, in which direction.  No arithmetic happens here.

Schedule (a reading of the paper, which fixes none): layer t holds the gates
(q, q+1) with q = t mod 2 (mod 2); even layers are applied left to right,
odd layers right to left, so the orthogonality centre snakes along the
chain and each layer needs no extra centre sweep.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

from . import nne


def layer_plan(circuit) -> List[Tuple[List[int], np.ndarray, int]]:
    """Per layer: (left qubits in application order, unitaries in that order, direction)."""
    plan = []
    for t, (qs, us) in enumerate(zip(circuit.layers, circuit.unitaries)):
        if len(qs) == 0:
            continue
        if t % 2 == 0:
            plan.append((list(qs), np.asarray(us), +1))
        else:
            plan.append((list(qs)[::-1], np.asarray(us)[::-1], -1))
    return plan


def build_pauli_layers(ctx: nne.Context, pc, lambdas):
    """Device superoperators for every layer of a Pauli-noise circuit (gate-
    dependent channels, e.g. cat-qubit or matchgate noise), one instance per
    level in lambdas, in the snake schedule's application order."""
    out = []
    for t, (qs, us) in enumerate(zip(pc.layers, pc.unitaries)):
        if len(qs) == 0:
            continue
        order = slice(None) if t % 2 == 0 else slice(None, None, -1)
        G = ctx.build_pauli_superops(np.asarray(us)[order], np.asarray(pc.c0[t])[order],
                                     np.asarray(pc.c1[t])[order], lambdas)
        out.append((list(qs)[order], G, +1 if t % 2 == 0 else -1))
    return out


def build_layer_superops(ctx: nne.Context, circuit, rates: np.ndarray):
    """Device superoperators for every layer (a1), in application order."""
    return [(qs, ctx.build_superops(us, rates), d) for qs, us, d in layer_plan(circuit)]


def evolve(state: nne.State, layers) -> None:
    for qs, G, d in layers:
        state.apply_layer(qs, G, d)


def emulate(ctx: nne.Context, circuit, rates: np.ndarray, chi: int, paulis: np.ndarray, dtype: int = nne.C64,
            trunc: int = nne.TRUNC_EXACT, bits=None, layers=None):
    """Run one circuit at all noise levels (one instance per row of rates).
    Returns (state, <P> (n_inst, n_obs) complex, log F (n_inst))."""
    n_inst = rates.shape[0] if rates is not None else layers[0][1].shape[0]
    st = nne.State(ctx, circuit.n, chi, n_inst, dtype, trunc, bits)
    evolve(st, layers if layers is not None else build_layer_superops(ctx, circuit, rates))
    vals, lf = st.expect(paulis)
    return st, vals, lf


FIT_CODES = {"exp": nne.FIT_EXP_LOGLIN, "exp3": nne.FIT_EXP3, "poly2": nne.FIT_POLY, "poly1": nne.FIT_POLY}


def job_for(w, chi=None, dtype: int = nne.C64, trunc: int = nne.TRUNC_EXACT, sketch=None, power_iters: int = 1,
            paulis=None) -> nne.Job:
    """A server job (nne_job) for a workload: its circuit in the snake schedule,
    one level per lambda, its observables and fit."""
    from workloads import pauli_codes
    fit = FIT_CODES.get(w.fit, nne.FIT_EXP_LOGLIN)
    degree = int(w.fit[4:]) if w.fit.startswith("poly") else 2
    return nne.Job(w.n, layer_plan(w.circuit), np.asarray(w.lambdas), w.rate_table(),
                   w.chi if chi is None else chi,
                   pauli_codes(w.observables, w.n) if paulis is None else paulis,
                   dtype=dtype, trunc=trunc, sketch=sketch, power_iters=power_iters, bits=w.bits(),
                   fit_method=fit, fit_degree=degree, lambda_star=w.lambda_star)


def pauli_job(pc, lambdas, chi: int, paulis: np.ndarray, dtype: int = nne.C64, trunc: int = nne.TRUNC_EXACT,
              sketch=None, power_iters: int = 1, bits=None, fit_method: int = nne.FIT_EXP_LOGLIN,
              fit_degree: int = 2, lambda_star: float = 1.0) -> nne.Job:
    """A server job for a circuit with gate-dependent Pauli channels (c0 +
    lambda c1 per gate), in the snake schedule of build_pauli_layers."""
    layers, pr = [], []
    for t, (qs, us) in enumerate(zip(pc.layers, pc.unitaries)):
        if len(qs) == 0:
            continue
        order = slice(None) if t % 2 == 0 else slice(None, None, -1)
        layers.append((list(qs)[order], np.asarray(us)[order], +1 if t % 2 == 0 else -1))
        pr.append(np.stack([np.asarray(pc.c0[t])[order], np.asarray(pc.c1[t])[order]], axis=1))
    return nne.Job(pc.n, layers, np.asarray(lambdas, np.float64), None, chi, paulis, dtype=dtype, trunc=trunc,
                   sketch=sketch, power_iters=power_iters, bits=bits, fit_method=fit_method, fit_degree=fit_degree,
                   lambda_star=lambda_star, pauli=np.concatenate(pr) if pr else np.zeros((0, 2, 16)))


def emulate_ladder(ctx: nne.Context, circuit, rates: np.ndarray, chis, paulis: np.ndarray, dtype: int = nne.C64,
                   trunc: int = nne.TRUNC_EXACT, bits=None, layers=None):
    """The same circuit at every noise level for each bond dimension of a ladder
    D_1 < ... < D_k (one state per rung).  Returns values (k, n_inst, n_obs)
    (real parts) and log F (k, n_inst) for nne_extrapolate_ladder.  `layers`
    (prebuilt superoperators) replaces `rates` when given."""
    layers = build_layer_superops(ctx, circuit, rates) if layers is None else layers
    vals, lfs = [], []
    for chi in chis:
        st, v, lf = emulate(ctx, circuit, rates, int(chi), paulis, dtype, trunc, bits, layers)
        st.close()
        vals.append(v.real)
        lfs.append(lf)
    return np.stack(vals), np.stack(lfs)


def nzne(ctx: nne.Context, circuit, noise, lambdas, chis, paulis: np.ndarray, lambda_star: float = 1.0,
         method: int = nne.FIT_EXP_LOGLIN, degree: int = 2, dtype: int = nne.C64, with_zero: bool = True, bits=None):
    """The paper's pipeline for one circuit: emulations at every level of
    `lambdas` (and at lambda = 0, noise free, when with_zero) for each bond
    dimension of the ladder `chis`, fidelity extrapolation and criterion 1
    (A), then extrapolation in the noise strength to lambda* (B).  The
    lambda = 0 emulation at the largest chi is the sign reference of
    criterion 3 and does not enter the fit.  `noise` is a workloads.NoiseModel
    (strengths scaled by lambda), or None for a circuit that carries its own
    gate-dependent Pauli channels (c0 + lambda c1 per gate)."""
    lam = np.asarray(lambdas, np.float64)
    levels = ([0.0] if with_zero else []) + list(lam)
    if noise is None:
        layers = build_pauli_layers(ctx, circuit, np.asarray(levels, np.float64))
        vals, lfs = emulate_ladder(ctx, circuit, None, chis, paulis, dtype, bits=bits, layers=layers)
    else:
        rates = np.stack([noise.rates(l) for l in levels])
        vals, lfs = emulate_ladder(ctx, circuit, rates, chis, paulis, dtype, bits=bits)
    y_zero = None
    if with_zero:
        y_zero = vals[-1, 0].copy()
        vals, lfs = vals[:, 1:], lfs[:, 1:]
    est, status, obar, conv = ctx.extrapolate_ladder(lam, vals, lfs, method=method, degree=degree,
                                                     lambda_star=lambda_star, y_zero=y_zero)
    return {"estimate": est, "status": status, "obar": obar, "converged": conv, "values": vals, "log_fid": lfs,
            "y_zero": y_zero}
