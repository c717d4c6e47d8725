"""Exact density-matrix simulator for n <= 10 -- ORACLE (test infrastructure only).

Follows the setup of Sec. 2.1.2: rho_l = C_l ... C_1(rho_0) with each
subcircuit C_l = (channel) o U on a pair (q, q+1) (Sec. 2.2.1, eq. U -> C o U),
rho_0 = |b><b| a computational basis product state.  No approximation: this
is the exact target the VMPO emulation approximates, and the true fidelity
F of eq. (true_fidelity) is computed against it.

Pins (tests/test_oracle_dense.py, tests/test_oracle_entropy.py): trace preservation, Hermiticity, closed
forms for identity circuits under each channel, agreement with the
statevector simulator at zero noise.
"""
from __future__ import annotations

import numpy as np

from . import channels

_PAULI = {"I": channels.I2, "X": channels.PX, "Y": channels.PY, "Z": channels.PZ}


def basis_state(bits) -> np.ndarray:
    n = len(bits)
    idx = 0
    for b in bits:
        idx = 2 * idx + int(b)
    rho = np.zeros((2 ** n, 2 ** n), dtype=complex)
    rho[idx, idx] = 1.0
    return rho


def embed(op4: np.ndarray, q: int, n: int) -> np.ndarray:
    """4x4 operator on qubits (q, q+1) as a 2^n x 2^n matrix (qubit 0 most significant)."""
    return np.kron(np.kron(np.eye(2 ** q), op4), np.eye(2 ** (n - q - 2)))


def apply_gate(rho: np.ndarray, U: np.ndarray, rates, q: int, n: int) -> np.ndarray:
    """rho <- C(U rho U^dagger) with C the channel at strengths rates on (q, q+1)."""
    Ue = embed(U, q, n)
    rho = Ue @ rho @ Ue.conj().T
    p2, g, pz, p1 = (float(x) for x in rates)
    for on, kraus in ((p2, channels.kraus_depol2(p2) if p2 else None),
                      (g, channels.on_both(channels.kraus_amp_damp(g)) if g else None),
                      (pz, channels.on_both(channels.kraus_dephase(pz)) if pz else None),
                      (p1, channels.on_both(channels.kraus_depol1(p1)) if p1 else None)):
        if on:
            rho = channels.apply_kraus_dense(rho, [embed(K, q, n) for K in kraus])
    return rho


def run(circuit, rates, bits=None) -> np.ndarray:
    """Final density matrix of a brickwork circuit at one noise level."""
    n = circuit.n
    rho = basis_state(bits if bits is not None else [0] * n)
    for qs, us in zip(circuit.layers, circuit.unitaries):
        for q, U in zip(qs, us):
            rho = apply_gate(rho, U, rates, q, n)
    return rho


def run_pauli(pc, lam: float, bits=None) -> np.ndarray:
    """Final density matrix of a Pauli-noise circuit at level lam: each block
    rho <- sum_K K U rho U^dagger K^dagger with the block's Pauli Kraus set."""
    n = pc.n
    rho = basis_state(bits if bits is not None else [0] * n)
    for t, (qs, us) in enumerate(zip(pc.layers, pc.unitaries)):
        for q, U, pr in zip(qs, us, pc.probs(t, lam)):
            Ue = embed(U, q, n)
            rho = Ue @ rho @ Ue.conj().T
            rho = channels.apply_kraus_dense(rho, [embed(K, q, n) for K in channels.kraus_pauli(pr)])
    return rho


def pauli_matrix(ob, n: int) -> np.ndarray:
    """Pauli string given as ((qubit, 'X'|'Y'|'Z'), ...) as a 2^n x 2^n matrix."""
    ops = ["I"] * n
    for q, p in ob:
        ops[q] = p
    M = np.array([[1.0 + 0j]])
    for p in ops:
        M = np.kron(M, _PAULI[p])
    return M


def expect(rho: np.ndarray, ob, n: int) -> complex:
    """Tr(P rho) / Tr(rho)."""
    return np.trace(pauli_matrix(ob, n) @ rho) / np.trace(rho)


def true_fidelity(rho_approx: np.ndarray, rho_exact: np.ndarray) -> float:
    """F of eq. (true_fidelity): |<<a|b>>|^2 / (||a||^2 ||b||^2), Frobenius inner product."""
    ip = np.vdot(rho_approx.ravel(), rho_exact.ravel())
    return float(abs(ip) ** 2 / (np.vdot(rho_approx.ravel(), rho_approx.ravel()).real
                                 * np.vdot(rho_exact.ravel(), rho_exact.ravel()).real))


def mpo_entropy(rho: np.ndarray, l: int, n: int) -> float:
    """MPO entanglement entropy of vec(rho) across the cut after qubit l (App. A.1).

    The definition itself: write vec(rho) with site index s = 2 i + j for the
    ket / bra bits (i, j) of each qubit, reshape it into a matrix from the
    first l sites to the last n - l, and take the Shannon entropy of its
    normalised squared singular values."""
    T = np.asarray(rho).reshape([2] * (2 * n))                 # kets i_0..i_{n-1}, then bras j_0..j_{n-1}
    perm = [a for k in range(n) for a in (k, n + k)]           # (i_0, j_0, i_1, j_1, ...)
    V = T.transpose(perm).reshape(4 ** l, 4 ** (n - l))
    s = np.linalg.svd(V, compute_uv=False)
    w = s ** 2
    p = w[w > 0.0] / np.sum(w)
    return float(-np.sum(p * np.log(p)))
