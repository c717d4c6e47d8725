"""Pins for oracle/channels.py: Kraus sets and superoperators (Sec. 2.2.1, App. C.2)."""
import json
import os

import numpy as np
import pytest

from oracle import channels as ch

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def rand_rho(d, rng):
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = a @ a.conj().T
    return r / np.trace(r)


@pytest.mark.parametrize("kraus", [
    ch.kraus_depol2(0.3), ch.kraus_depol1(0.2), ch.kraus_amp_damp(0.4), ch.kraus_dephase(0.15),
    ch.on_both(ch.kraus_amp_damp(0.1)), ch.on_both(ch.kraus_depol1(0.05))])
def test_kraus_completeness(kraus):
    d = kraus[0].shape[0]
    S = sum(K.conj().T @ K for K in kraus)
    assert np.allclose(S, np.eye(d), atol=1e-14)


def test_depol2_coefficients_match_paper():
    p = 0.37
    ks = ch.kraus_depol2(p)
    assert len(ks) == 16
    assert abs(abs(ks[0][0, 0]) ** 2 - (1 - GOLD["depol2_k0_coeff"]["value"] * p)) < 1e-15
    for K in ks[1:]:
        assert abs(np.max(np.abs(K)) ** 2 - GOLD["depol2_kij_coeff"]["value"] * p) < 1e-15


def test_depol2_net_map_closed_form():
    # App. C.2.1: rho -> (1 - p) rho + p I/4
    rng = np.random.default_rng(1)
    for p in (0.0, 1e-3, 0.2, 0.9):
        rho = rand_rho(4, rng)
        out = ch.apply_kraus_dense(rho, ch.kraus_depol2(p))
        assert np.allclose(out, (1 - p) * rho + p * np.eye(4) / 4, atol=1e-14)


def test_depol1_closed_form():
    # (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z) = (1 - 4p/3) rho + (2p/3) Tr(rho) I
    rng = np.random.default_rng(2)
    p = 0.21
    rho = rand_rho(2, rng)
    out = ch.apply_kraus_dense(rho, ch.kraus_depol1(p))
    assert np.allclose(out, (1 - 4 * p / 3) * rho + (2 * p / 3) * np.eye(2), atol=1e-14)
    z = np.trace(ch.PZ @ out).real
    assert abs(z - (1 - 4 * p / 3) * np.trace(ch.PZ @ rho).real) < 1e-14


def test_amp_damp_and_dephase_closed_forms():
    g, pz = 0.3, 0.12
    one = np.diag([0.0, 1.0]).astype(complex)
    out = ch.apply_kraus_dense(one, ch.kraus_amp_damp(g))
    assert np.allclose(out, np.diag([g, 1 - g]), atol=1e-15)
    plus = 0.5 * np.ones((2, 2), complex)
    out = ch.apply_kraus_dense(plus, ch.kraus_amp_damp(g))
    assert abs(out[0, 1] - 0.5 * np.sqrt(1 - g)) < 1e-15
    out = ch.apply_kraus_dense(plus, ch.kraus_dephase(pz))
    assert abs(out[0, 1] - 0.5 * (1 - 2 * pz)) < 1e-15 and abs(out[0, 0] - 0.5) < 1e-15


def test_unitality():
    for ks in (ch.kraus_depol2(0.4), ch.on_both(ch.kraus_dephase(0.2)), ch.on_both(ch.kraus_depol1(0.1))):
        assert np.allclose(ch.apply_kraus_dense(np.eye(4, dtype=complex), ks), np.eye(4), atol=1e-14)
    ad = ch.on_both(ch.kraus_amp_damp(0.3))
    assert not np.allclose(ch.apply_kraus_dense(np.eye(4, dtype=complex), ad), np.eye(4))


def vec2(rho):
    """Interleaved vectorisation of a two-qubit operator: index 4*(2 i1 + j1) + (2 i2 + j2)."""
    v = np.zeros(16, complex)
    for i1 in range(2):
        for i2 in range(2):
            for j1 in range(2):
                for j2 in range(2):
                    v[4 * (2 * i1 + j1) + (2 * i2 + j2)] = rho[2 * i1 + i2, 2 * j1 + j2]
    return v


def test_superop_matches_kraus_action():
    rng = np.random.default_rng(3)
    from workloads import haar_u4
    U = haar_u4(rng)
    rates = (0.02, 0.03, 0.01, 0.015)
    G = ch.gate_superop(U, rates)
    for _ in range(3):
        rho = rand_rho(4, rng)
        out = U @ rho @ U.conj().T
        out = ch.apply_kraus_dense(out, ch.kraus_depol2(rates[0]))
        out = ch.apply_kraus_dense(out, ch.on_both(ch.kraus_amp_damp(rates[1])))
        out = ch.apply_kraus_dense(out, ch.on_both(ch.kraus_dephase(rates[2])))
        out = ch.apply_kraus_dense(out, ch.on_both(ch.kraus_depol1(rates[3])))
        assert np.allclose(G @ vec2(rho), vec2(out), atol=1e-13)


def test_unitary_superop_is_unitary_and_trace_preserving():
    rng = np.random.default_rng(4)
    from workloads import haar_u4
    S = ch.superop([haar_u4(rng)])
    assert np.allclose(S.conj().T @ S, np.eye(16), atol=1e-13)
    vI = vec2(np.eye(4, dtype=complex))
    G = ch.gate_superop(haar_u4(rng), (0.1, 0.2, 0.05, 0.02))
    # trace preservation: <<I| G = <<I|
    assert np.allclose(vI.conj() @ G, vI.conj(), atol=1e-13)


def test_cat_table_rows_sum_to_one():
    for gate, rows in GOLD["cat_table"].items():
        if gate == "cite":
            continue
        c0 = sum(v[0] for v in rows.values())
        c1 = sum(v[1] for v in rows.values())
        assert c0 == 1 and abs(c1) < 1e-15
