"""Noise channels and gate+channel superoperators -- ORACLE (test infrastructure only).

Vectorisation (Sec. 2.1.1, eq. vectorized_dm): per qubit |i><j| -> |(i,j)>>,
local index s = 2*i + j (i = ket, j = bra).  A two-qubit superoperator is a
16x16 matrix G[(s1',s2'), (s1,s2)] with row index 4*s1' + s2', qubit 1 the
left (more significant) qubit.

For a map E(rho) = sum_K K rho K^dagger, the vectorised action is
  E(rho)_{i,j} = sum_K sum_{i',j'} K_{i i'} conj(K_{j j'}) rho_{i' j'},
so its superoperator entry is sum_K K_{i i'} conj(K_{j j'}) with the ket and
bra indices of each qubit interleaved into s.

Noise model (Sec. 2.2.1, eq. U -> C o U): every gate U is post-composed with a
channel C; here C is the composition, in this order, of
  1. two-qubit depolarizing with map strength p (App. C.2.1:
     K0 = sqrt(1-15p/16) I, K_ij = sqrt(p/16) sigma_i sigma_j; net map
     rho -> (1-p) rho + p I/4),
  2. amplitude damping gamma on each qubit (standard K0 = diag(1, sqrt(1-gamma)),
     K1 = sqrt(gamma)|0><1|; named but not defined in the paper),
  3. dephasing p_z on each qubit (K0 = sqrt(1-p_z) I, K1 = sqrt(p_z) Z),
  4. single-qubit depolarizing with error probability p1 on each qubit
     (K0 = sqrt(1-p1) I, sqrt(p1/3){X,Y,Z}; <Z> -> (1 - 4 p1/3) <Z>).
The order of 2-4 is a reading: the paper never composes channels.

Gate-dependent Pauli channels (cat-qubit noise, App. C.2.2; matchgate
depolarizing noise, App. C.3.1) are built by kraus_pauli from 16
probabilities per gate.

Pins (tests/test_oracle_channels.py): Kraus completeness; the closed-form maps
of App. C.2.1 and of the single-qubit channels applied to random density
matrices by explicit K rho K^dagger products; unitality; agreement of the
superoperator with K rho K^dagger on random inputs.
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = (I2, PX, PY, PZ)


def kraus_depol2(p: float):
    """Two-qubit depolarizing channel of App. C.2.1 (map strength p)."""
    ops = [np.sqrt(1.0 - 15.0 * p / 16.0) * np.eye(4, dtype=complex)]
    for i in range(4):
        for j in range(4):
            if i == 0 and j == 0:
                continue
            ops.append(np.sqrt(p / 16.0) * np.kron(PAULI[i], PAULI[j]))
    return ops


def kraus_depol1(p: float):
    """Single-qubit depolarizing with error probability p."""
    return [np.sqrt(1.0 - p) * I2] + [np.sqrt(p / 3.0) * P for P in (PX, PY, PZ)]


def kraus_amp_damp(g: float):
    return [np.array([[1, 0], [0, np.sqrt(1.0 - g)]], dtype=complex),
            np.array([[0, np.sqrt(g)], [0, 0]], dtype=complex)]


def kraus_dephase(p: float):
    return [np.sqrt(1.0 - p) * I2, np.sqrt(p) * PZ]


def on_both(kraus_1q):
    """Kraus set of the same single-qubit channel acting on both qubits."""
    return [np.kron(a, b) for a in kraus_1q for b in kraus_1q]


def superop(kraus_4x4) -> np.ndarray:
    """16x16 superoperator of a two-qubit map, interleaved (s1, s2) indexing."""
    S = np.zeros((16, 16), dtype=complex)
    for K in kraus_4x4:
        for i1 in range(2):
            for j1 in range(2):
                for i2 in range(2):
                    for j2 in range(2):
                        row = 4 * (2 * i1 + j1) + (2 * i2 + j2)
                        for k1 in range(2):
                            for l1 in range(2):
                                for k2 in range(2):
                                    for l2 in range(2):
                                        col = 4 * (2 * k1 + l1) + (2 * k2 + l2)
                                        S[row, col] += (K[2 * i1 + i2, 2 * k1 + k2]
                                                        * np.conj(K[2 * j1 + j2, 2 * l1 + l2]))
    return S


def noise_superop(rates) -> np.ndarray:
    """Superoperator of the channel C at strengths (p_depol2, gamma, p_z, p1)."""
    p2, g, pz, p1 = (float(x) for x in rates)
    S = np.eye(16, dtype=complex)
    if p2:
        S = superop(kraus_depol2(p2)) @ S
    if g:
        S = superop(on_both(kraus_amp_damp(g))) @ S
    if pz:
        S = superop(on_both(kraus_dephase(pz))) @ S
    if p1:
        S = superop(on_both(kraus_depol1(p1))) @ S
    return S


def gate_superop(U: np.ndarray, rates) -> np.ndarray:
    """G = S_C . S_U, the fused gate+channel superoperator (eq. U -> C o U)."""
    return noise_superop(rates) @ superop([U])


def kraus_pauli(probs) -> list:
    """Pauli channel on two qubits: K_ab = sqrt(p_ab) sigma_a (x) sigma_b, p_ab =
    probs[4a+b] (a on the left qubit).  The two-qubit depolarizing channel of
    App. C.2.1, the cat-qubit errors of App. C.2.2 and the matchgate
    depolarizing channel of App. C.3.1 are all of this form."""
    p = np.asarray(probs, dtype=float)
    if p.shape != (16,) or (p < -1e-15).any():
        raise ValueError("need 16 non-negative probabilities")
    return [np.sqrt(max(p[4 * a + b], 0.0)) * np.kron(PAULI[a], PAULI[b])
            for a in range(4) for b in range(4) if p[4 * a + b] > 0.0]


def pauli_gate_superop(U: np.ndarray, probs) -> np.ndarray:
    """G = S_P . S_U: the gate followed by its Pauli channel (eq. U -> C o U)."""
    return superop(kraus_pauli(probs)) @ superop([U])


def pauli_superops_for(pc, lam: float) -> list:
    """Per layer of a Pauli-noise circuit: (blocks, 16, 16) superoperators at level lam."""
    return [np.stack([pauli_gate_superop(U, pr) for U, pr in zip(us, pc.probs(t, lam))])
            if len(us) else np.zeros((0, 16, 16), complex)
            for t, us in enumerate(pc.unitaries)]


def apply_kraus_dense(rho: np.ndarray, kraus) -> np.ndarray:
    """sum_K K rho K^dagger on a (d x d) density matrix."""
    return sum(K @ rho @ K.conj().T for K in kraus)
