"""Exact noisy expectation values of matchgate circuits -- ORACLE (test infrastructure only).

App. C.3 benchmarks the method on matchgate circuits (the XY model, App.
C.1.3) under matchgate depolarizing noise (App. C.3.1), estimating the true
values by trajectory sampling.  For Pauli observables that are quadratic in
Majorana operators (Z_j, X_jX_{j+1}, Y_jX_{j+1}, ...) the noisy expectation
values can be computed exactly instead, in polynomial time:

  * Jordan-Wigner Majoranas g_{2j} = (prod_{k<j} Z_k) X_j,
    g_{2j+1} = (prod_{k<j} Z_k) Y_j; the covariance matrix
    C_ab = (i/2) <[g_a, g_b]> (real, antisymmetric, 2n x 2n) gives
    <g_a g_b> = delta_ab - i C_ab.
  * A parity-preserving Gaussian (matchgate) unitary U on (q, q+1) rotates the
    pair's four Majoranas: U^dagger g_a U = sum_b O_ab g_b with O real
    orthogonal, so C <- O C O^T on those rows and columns.  Other Majoranas
    are untouched: their strings hold Z_q Z_{q+1}, which commutes with U.
  * A parity-preserving Pauli P on the pair commutes or anticommutes with each
    of the four local Majoranas (P g_a P = s_a g_a, s_a = +-1) and commutes
    with all others, so the Pauli channel rho -> sum_P p_P P rho P maps
    C_ab -> (sum_P p_P s_a(P) s_b(P)) C_ab.
  * Both steps are linear in C and hold for any state, Gaussian or not, so
    the mixture's quadratic expectation values follow exactly.

O and s are read off 4x4 matrices (the local Majoranas X(x)I, Y(x)I, Z(x)X,
Z(x)Y, whose common string to the left cancels in every bilinear); a gate or
Pauli outside the matchgate family raises ValueError.

Pins (tests/test_oracle_matchgate.py): equals the dense density-matrix
simulator on small XY-model circuits with noise and the statevector at
lambda = 0; closed form of the channel on <Z_q> for an identity circuit.
"""
from __future__ import annotations

import numpy as np

from . import channels

_X, _Y, _Z, _I = channels.PX, channels.PY, channels.PZ, channels.I2
LOCAL = (np.kron(_X, _I), np.kron(_Y, _I), np.kron(_Z, _X), np.kron(_Z, _Y))
_PARITY = np.kron(_Z, _Z)


def rotation(U: np.ndarray, tol: float = 1e-10) -> np.ndarray:
    """O with U^dagger g_a U = sum_b O_ab g_b for the pair's local Majoranas."""
    if np.abs(U @ _PARITY - _PARITY @ U).max() > tol:
        raise ValueError("gate does not preserve parity")
    O = np.zeros((4, 4))
    for a, ga in enumerate(LOCAL):
        h = U.conj().T @ ga @ U
        coef = np.array([np.trace(gb @ h) / 4.0 for gb in LOCAL])   # Tr(g_b g_c) = 4 delta_bc
        if np.abs(h - sum(c * gb for c, gb in zip(coef, LOCAL))).max() > tol or np.abs(coef.imag).max() > tol:
            raise ValueError("gate is not Gaussian (not a matchgate)")
        O[a] = coef.real
    return O


def pauli_signs(P: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """s_a with P g_a P = s_a g_a for a parity-preserving two-qubit Pauli P."""
    if np.abs(P @ _PARITY - _PARITY @ P).max() > tol:
        raise ValueError("Pauli does not preserve parity (not a matchgate Pauli)")
    s = np.zeros(4)
    for a, ga in enumerate(LOCAL):
        h = P @ ga @ P
        if np.abs(h - ga).max() < tol:
            s[a] = 1.0
        elif np.abs(h + ga).max() < tol:
            s[a] = -1.0
        else:
            raise ValueError("not a Pauli")
    return s


def initial_covariance(bits) -> np.ndarray:
    """C of the basis state |b>: <Z_j> = -C_{2j,2j+1} = (-1)^{b_j}."""
    n = len(bits)
    C = np.zeros((2 * n, 2 * n))
    for j, b in enumerate(bits):
        z = -1.0 if int(b) else 1.0
        C[2 * j, 2 * j + 1] = -z
        C[2 * j + 1, 2 * j] = z
    return C


def apply_block(C: np.ndarray, q: int, U: np.ndarray, probs) -> np.ndarray:
    """One block of a Pauli-noise circuit: the gate, then its Pauli channel."""
    idx = np.arange(2 * q, 2 * q + 4)
    O = np.eye(C.shape[0])
    O[np.ix_(idx, idx)] = rotation(U)
    C = O @ C @ O.T
    p = np.asarray(probs, float)
    w = np.zeros(C.shape[0])   # sum_P p_P s_a(P) for the local a ...
    W = np.zeros((4, 4))       # ... and sum_P p_P s_a(P) s_b(P)
    for a in range(4):
        for b in range(4):
            pk = p[4 * a + b]
            if pk == 0.0:
                continue
            s = pauli_signs(np.kron(channels.PAULI[a], channels.PAULI[b]))
            W += pk * np.outer(s, s)
            w[idx] += pk * s
    tot = p.sum()
    F = np.full(C.shape, tot)          # pairs with no local index: every P commutes
    F[np.ix_(idx, np.arange(C.shape[0]))] = w[idx][:, None]
    F[np.ix_(np.arange(C.shape[0]), idx)] = w[idx][None, :]
    F[np.ix_(idx, idx)] = W
    return C * F


def run(pc, lam: float, bits) -> np.ndarray:
    """Covariance matrix after a Pauli-noise matchgate circuit at level lam."""
    C = initial_covariance(bits)
    for t, (qs, us) in enumerate(zip(pc.layers, pc.unitaries)):
        for q, U, pr in zip(qs, us, pc.probs(t, lam)):
            C = apply_block(C, q, U, pr)
    return C


def expect_pair(C: np.ndarray, q: int, op4: np.ndarray, tol: float = 1e-12) -> float:
    """<op4 on (q, q+1)> for an operator quadratic in the pair's Majoranas
    (plus a multiple of the identity): op4 = c I + sum_{a<b} w_ab g_a g_b."""
    idx = 2 * q
    val = np.trace(op4) / 4.0
    rebuilt = val * np.eye(4, dtype=complex)
    for a in range(4):
        for b in range(a + 1, 4):
            m = LOCAL[a] @ LOCAL[b]
            w = np.trace(m.conj().T @ op4) / 4.0
            rebuilt = rebuilt + w * m
            val = val + w * (-1j * C[idx + a, idx + b])
    if np.abs(rebuilt - op4).max() > tol:
        raise ValueError("observable is not quadratic in the pair's Majoranas")
    return float(np.real(val))


_P = {"I": _I, "X": _X, "Y": _Y, "Z": _Z}


def expect(C: np.ndarray, ob, n: int) -> float:
    """<P> for a Pauli string on one qubit or two neighbouring qubits."""
    qs = sorted(q for q, _ in ob)
    if len(qs) == 1:
        q = qs[0]
        lq = q if q < n - 1 else q - 1
        ops = {q: dict(ob)[q]}
    elif len(qs) == 2 and qs[1] == qs[0] + 1:
        lq = qs[0]
        ops = dict(ob)
    else:
        raise ValueError("only single-qubit or neighbouring two-qubit strings")
    op4 = np.kron(_P[ops.get(lq, "I")], _P[ops.get(lq + 1, "I")])
    return expect_pair(C, lq, op4)
