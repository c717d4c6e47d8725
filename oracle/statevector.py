"""Pure-state simulator (zero-noise reference) -- ORACLE (test infrastructure only).

At lambda = 0 the noisy circuit of Sec. 2.2.1 reduces to the unitary circuit;
its expectation values <psi|P|psi> are the limit the noise extrapolation of
Sec. 2.2.3 aims at and the sign reference of criterion 3.

Pin (tests/test_oracle_dense.py): equals the dense simulator at zero noise;
norm preservation.
"""
from __future__ import annotations

import numpy as np

from . import dense


def run(circuit, bits=None) -> np.ndarray:
    n = circuit.n
    bits = bits if bits is not None else [0] * n
    idx = 0
    for b in bits:
        idx = 2 * idx + int(b)
    psi = np.zeros(2 ** n, dtype=complex)
    psi[idx] = 1.0
    for qs, us in zip(circuit.layers, circuit.unitaries):
        for q, U in zip(qs, us):
            psi = dense.embed(U, q, n) @ psi
    return psi


def expect(psi: np.ndarray, ob, n: int) -> complex:
    return np.vdot(psi, dense.pauli_matrix(ob, n) @ psi)
