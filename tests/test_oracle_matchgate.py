"""Pins for the Pauli-noise oracle: Pauli-channel superoperators (cat-qubit
noise, App. C.2.2; matchgate depolarizing noise, App. C.3.1) and the exact
free-fermion evaluation of noisy matchgate circuits (oracle/matchgate.py).

Closed forms used (identity or Clifford circuits, explicit Kraus algebra):
  * Pauli channel with p_ab = lambda/16 for ab != II is the two-qubit
    depolarizing channel of App. C.2.1;
  * matchgate channel on <Z_q>: ZI, IZ, ZZ commute with Z_q, the four XX..YX
    terms anticommute, so <Z_q> -> (1 - 8 lambda / 7) <Z_q> per block;
  * cat CX on |++>: <X_control> picks up (1 - 2 (3 lambda + lambda / 2)) and
    <X_target> (1 - 2 lambda) per gate; Z(theta) noise on |+> multiplies
    <X> by (1 - 2 lambda) after undoing the rotation;
  * every table gives probabilities summing to one (trace preservation) and
    the channel is unital.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import channels as ch
from oracle import dense, matchgate, mps, statevector
import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_cat_table_is_the_papers():
    for gate, rows in GOLD["cat_table"].items():
        if gate == "cite":
            continue
        assert {k: tuple(v) for k, v in rows.items()} == {k: tuple(v) for k, v in wl.CAT_TABLE[gate].items()}


@pytest.mark.parametrize("gate", ["Z_theta", "H", "CX"])
@pytest.mark.parametrize("left", [True, False])
def test_cat_noise_vectors(gate, left):
    c0, c1 = wl.cat_gate_noise(gate, left)
    assert c0.sum() == 1.0 and abs(c1.sum()) < 1e-15
    lam = 0.01
    ks = ch.kraus_pauli(c0 + lam * c1)
    assert np.allclose(sum(K.conj().T @ K for K in ks), np.eye(4), atol=1e-15)
    # the error acts on the qubit of the gate (control for CX), nothing else
    if gate != "CX":
        other = wl.pauli_index("I", "Z") if left else wl.pauli_index("Z", "I")
        assert c1[other] == 0.0


def test_depolarizing_as_pauli_channel():
    lam = 0.23
    p = np.full(16, lam / 16.0)
    p[0] = 1.0 - 15.0 * lam / 16.0
    assert np.allclose(ch.superop(ch.kraus_pauli(p)), ch.superop(ch.kraus_depol2(lam)), atol=1e-15)


def _identity_pc(n, depth, c0, c1, U=None):
    layers = wl.brickwork_pairs(n, depth)
    U = np.eye(4, dtype=complex) if U is None else U
    return wl.PauliCircuit(n, "id", layers, [np.stack([U] * len(qs)) for qs in layers],
                           [np.tile(c0, (len(qs), 1)) for qs in layers], [np.tile(c1, (len(qs), 1)) for qs in layers])


def test_matchgate_channel_closed_form_on_z():
    pc = wl.xym_circuit(4, 1)
    c0, c1 = pc.c0[0][0], pc.c1[0][0]
    assert abs((c0 + 0.3 * c1).sum() - 1.0) < 1e-15
    n, depth, lam = 4, 5, 0.07
    idc = _identity_pc(n, depth, c0, c1)
    rho = dense.run_pauli(idc, lam, bits=[0, 1, 1, 0])
    C = matchgate.run(idc, lam, [0, 1, 1, 0])
    for q, b in enumerate([0, 1, 1, 0]):
        k = sum(q in (p, p + 1) for qs in idc.layers for p in qs)      # blocks touching q
        want = (-1) ** b * (1 - 8 * lam / 7) ** k
        assert abs(dense.expect(rho, ((q, "Z"),), n).real - want) < 1e-13
        assert abs(matchgate.expect(C, ((q, "Z"),), n) - want) < 1e-13


def test_cat_cx_closed_form_on_plus_states():
    lam, k = 0.02, 3
    c0, c1 = wl.cat_gate_noise("CX", True)
    pc = _identity_pc(2, 1, c0, c1, U=wl._CX_L)
    pc = wl.PauliCircuit(2, "cx", [[0]] * k, [pc.unitaries[0]] * k, [pc.c0[0]] * k, [pc.c1[0]] * k)
    plus = np.full(4, 0.5, complex)
    rho = np.outer(plus, plus.conj())
    for t in range(k):
        Ue = pc.unitaries[t][0]
        rho = ch.apply_kraus_dense(Ue @ rho @ Ue.conj().T, ch.kraus_pauli(pc.probs(t, lam)[0]))
    assert abs(np.trace(dense.pauli_matrix(((0, "X"),), 2) @ rho) - (1 - 7 * lam) ** k) < 1e-14
    assert abs(np.trace(dense.pauli_matrix(((1, "X"),), 2) @ rho) - (1 - 2 * lam) ** k) < 1e-14


def test_cat_z_theta_noise_closed_form():
    lam, th = 0.03, 0.7
    c0, c1 = wl.cat_gate_noise("Z_theta", True)
    Rz = np.kron(np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)]), np.eye(2))
    plus0 = np.kron(np.array([1, 1]) / math.sqrt(2), np.array([1, 0])).astype(complex)
    rho = ch.apply_kraus_dense(Rz @ np.outer(plus0, plus0.conj()) @ Rz.conj().T, ch.kraus_pauli(c0 + lam * c1))
    # <X cos th + Y sin th> on qubit 0 after Rz(th): (1 - 2 lam)
    got = np.trace((math.cos(th) * dense.pauli_matrix(((0, "X"),), 2)
                    + math.sin(th) * dense.pauli_matrix(((0, "Y"),), 2)) @ rho).real
    assert abs(got - (1 - 2 * lam)) < 1e-14


@pytest.mark.parametrize("lam", [0.0, 0.05])
def test_matchgate_oracle_equals_dense(lam):
    n = 6
    pc = wl.xym_circuit(n, 4, J=0.5, h=0.23, dt=0.3)
    bits = wl.neel_bits(n)
    rho = dense.run_pauli(pc, lam, bits)
    C = matchgate.run(pc, lam, bits)
    obs = wl.obs_z(n) + wl.obs_xx(n) + [((q, "Y"), (q + 1, "X")) for q in range(n - 1)] \
        + [((q, "X"), (q + 1, "Y")) for q in range(n - 1)] + [((q, "Y"), (q + 1, "Y")) for q in range(n - 1)]
    vals = []
    for ob in obs:
        want = dense.expect(rho, ob, n).real
        vals.append(want)
        assert abs(matchgate.expect(C, ob, n) - want) < 1e-12
    assert np.std(vals) > 0.05                     # non-trivial values
    if lam == 0.0:
        psi = statevector.run(wl.Circuit(n, len(pc.layers), pc.layers, pc.unitaries), bits)
        for ob in obs:
            assert abs(matchgate.expect(C, ob, n) - statevector.expect(psi, ob, n).real) < 1e-12


def test_matchgate_oracle_rejects_non_matchgates():
    with pytest.raises(ValueError):
        matchgate.rotation(wl._CX_L)
    with pytest.raises(ValueError):
        matchgate.pauli_signs(np.kron(ch.PX, ch.I2))
    C = matchgate.initial_covariance([0, 0, 0])
    with pytest.raises(ValueError):
        matchgate.expect_pair(C, 0, np.kron(ch.PZ, ch.PZ))    # quartic


def test_pauli_circuit_vmpo_equals_dense():
    n = 6
    pc = wl.cat_circuit(n, 6, 3)
    for lam in (0.0, 0.02):
        rho = dense.run_pauli(pc, lam)
        st = mps.run(pc, None, 4 ** (n // 2), Gs=ch.pauli_superops_for(pc, lam))
        obs = wl.obs_z(n) + wl.obs_xx(n)
        got = st.expect_codes(wl.pauli_codes(obs, n))
        for ob, g in zip(obs, got):
            assert abs(g - dense.expect(rho, ob, n)) < 1e-12


def test_xym_circuit_matches_paper_parameters():
    c = GOLD["xym_table"]["circuit"]
    pc = wl.xym_circuit(c["n"], c["steps"], J=c["J"], h=c["h"], dt=c["dt"])
    assert pc.n_gates == c["two_qubit_gates"]
    assert list(wl.neel_bits(6)) == [1, 0, 1, 0, 1, 0]


def test_xym_60_exact_values_within_paper_trajectory_error():
    """The exact noisy values of the 60-qubit XY-model circuit at lambda* =
    0.002 against the paper's trajectory means (qubits counted from 0; the
    even-bond layer first in each step -- the other order gives <YX> = -0.225)."""
    t = GOLD["xym_table"]
    c = t["circuit"]
    pc = wl.xym_circuit(c["n"], c["steps"], J=c["J"], h=c["h"], dt=c["dt"])
    C = matchgate.run(pc, c["lambda_star"], wl.neel_bits(c["n"]))
    yx = matchgate.expect(C, ((30, "Y"), (31, "X")), c["n"])
    z = matchgate.expect(C, ((30, "Z"),), c["n"])
    assert abs(yx - t["YX_30_31"]["trajectory"]) < 3 * t["YX_30_31"]["trajectory_std"]
    assert abs(z - t["Z_30"]["trajectory"]) < 3 * t["Z_30"]["trajectory_std"]
