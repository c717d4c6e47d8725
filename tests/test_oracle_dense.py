"""Pins for oracle/dense.py and oracle/statevector.py."""
import numpy as np
import pytest

from oracle import dense, statevector
from oracle import channels as ch
import workloads as wl


def test_trace_and_hermiticity():
    c = wl.brickwork_circuit(5, 6, seed=11)
    rho = dense.run(c, (0.05, 0.03, 0.02, 0.01))
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.allclose(rho, rho.conj().T, atol=1e-14)
    ev = np.linalg.eigvalsh(rho)
    assert ev.min() > -1e-13


def gates_touching(circ, q):
    return sum(1 for qs in circ.layers for g in qs if g == q or g + 1 == q)


def test_depol2_identity_closed_form():
    n, depth, p = 5, 5, 0.07
    c = wl.identity_circuit(n, depth)
    rho = dense.run(c, (p, 0, 0, 0))
    for q in range(n):
        assert abs(dense.expect(rho, ((q, "Z"),), n).real - (1 - p) ** gates_touching(c, q)) < 1e-13
    for q in range(n - 1):
        k = sum(1 for qs in c.layers for g in qs if {g, g + 1} & {q, q + 1})
        assert abs(dense.expect(rho, ((q, "Z"), (q + 1, "Z")), n).real - (1 - p) ** k) < 1e-13


def test_depol1_identity_closed_form():
    # single-qubit depolarizing on |0>: <Z> = (1 - 4p/3)^k
    n, depth, p = 4, 6, 0.05
    c = wl.identity_circuit(n, depth)
    rho = dense.run(c, (0, 0, 0, p))
    for q in range(n):
        assert abs(dense.expect(rho, ((q, "Z"),), n).real - (1 - 4 * p / 3) ** gates_touching(c, q)) < 1e-13


def test_amp_damp_from_one_closed_form():
    n, depth, g = 4, 5, 0.08
    c = wl.identity_circuit(n, depth)
    rho = dense.run(c, (0, g, 0, 0), bits=[1] * n)
    for q in range(n):
        k = gates_touching(c, q)
        assert abs(dense.expect(rho, ((q, "Z"),), n).real - (1 - 2 * (1 - g) ** k)) < 1e-13


def hadamard_circuit(n, depth):
    c = wl.identity_circuit(n, depth)
    H = np.array([[1, 1], [1, -1]], complex) / np.sqrt(2)
    c.unitaries[0] = np.stack([np.kron(H, H) for _ in c.layers[0]])
    return c


def test_dephase_plus_closed_form():
    n, depth, pz = 4, 5, 0.06
    c = hadamard_circuit(n, depth)
    rho = dense.run(c, (0, 0, pz, 0))
    for q in range(n):
        assert abs(dense.expect(rho, ((q, "X"),), n).real - (1 - 2 * pz) ** gates_touching(c, q)) < 1e-13


def test_zero_noise_matches_statevector():
    n = 6
    c = wl.brickwork_circuit(n, 5, seed=5)
    rho = dense.run(c, (0, 0, 0, 0))
    psi = statevector.run(c)
    assert abs(np.vdot(psi, psi) - 1) < 1e-13
    assert np.allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)
    for ob in (((2, "Z"),), ((1, "X"), (2, "X")), ((3, "Y"),)):
        assert abs(dense.expect(rho, ob, n) - statevector.expect(psi, ob, n)) < 1e-13


def test_true_fidelity_bounds():
    c = wl.brickwork_circuit(4, 4, seed=2)
    a = dense.run(c, (0.01, 0, 0, 0))
    b = dense.run(c, (0.2, 0, 0, 0))
    assert abs(dense.true_fidelity(a, a) - 1) < 1e-13
    assert 0 < dense.true_fidelity(a, b) < 1
