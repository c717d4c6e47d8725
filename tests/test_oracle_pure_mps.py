"""Pins for oracle/pure_mps.py (pure-state MPS for the lambda = 0 level).

* untruncated it reproduces the statevector exactly (vector and <P>);
* one truncation in canonical form keeps the closest state: the true
  fidelity |<psi_exact|psi_kept>|^2 equals the kept weight f (Eckart-Young);
* its bond entropies equal the statevector's Schmidt entropies, and the
  VMPO of the same noise-free circuit has exactly twice that MPO entropy;
* truncation keeps the norm at 1 and the bond dimension at chi.
"""
import math

import numpy as np
import pytest

from oracle import mps, pure_mps, statevector
import workloads as wl


def vn_entropy(psi, l, n):
    s = np.linalg.svd(psi.reshape(2 ** l, 2 ** (n - l)), compute_uv=False)
    p = s ** 2 / np.sum(s ** 2)
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


@pytest.mark.parametrize("n,depth,seed,bits", [(8, 7, 1, None), (7, 6, 2, (1, 0, 1, 1, 0, 0, 1))])
def test_untruncated_equals_statevector(n, depth, seed, bits):
    c = wl.brickwork_circuit(n, depth, seed)
    st = pure_mps.run(c, 2 ** (n // 2), bits)
    psi = statevector.run(c, bits)
    assert abs(st.log_fid) < 1e-13
    assert np.abs(st.to_vector() - psi).max() < 1e-12
    obs = wl.obs_z(n) + wl.obs_xx(n) + [((i, "Y"), (i + 1, "X")) for i in range(n - 1)] + [((0, "X"), (n - 1, "Y"))]
    got = st.expect_codes(wl.pauli_codes(obs, n))
    for ob, g in zip(obs, got):
        assert abs(g - statevector.expect(psi, ob, n)) < 1e-12


def test_single_truncation_keeps_the_closest_state():
    n = 8
    c = wl.brickwork_circuit(n, 6, 5)
    st = pure_mps.run(c, 16)                      # exact so far
    psi = st.to_vector()
    st.chi = 3                                    # the next gate truncates the middle bond
    q, U = 3, wl.haar_u4(np.random.default_rng(9))
    st.gate(q, U, +1)
    from oracle import dense
    exact = dense.embed(U, q, n) @ psi
    kept = st.to_vector()
    f = st.fids[-1]
    assert f < 0.999 and st.bond_dims()[q] == 3
    assert abs(np.vdot(kept, kept) - 1.0) < 1e-12
    assert abs(abs(np.vdot(exact, kept)) ** 2 - f) < 1e-12


def test_bond_entropies_equal_statevector_and_half_the_vmpo():
    n = 7
    c = wl.brickwork_circuit(n, 6, 7)
    psi = statevector.run(c)
    st = pure_mps.run(c, 2 ** (n // 2 + 1))
    S = st.entropies()
    want = np.array([vn_entropy(psi, l, n) for l in range(1, n)])
    assert np.all(want > 1e-3)
    assert np.allclose(S, want, atol=1e-10, rtol=0)
    vm = mps.run(c, (0, 0, 0, 0), 4 ** (n // 2 + 1))
    assert np.allclose(vm.mpo_entropies(), 2 * S, atol=1e-10, rtol=0)


def test_truncated_run_bookkeeping():
    n, chi = 10, 6
    c = wl.brickwork_circuit(n, 10, 11)
    st = pure_mps.run(c, chi)
    assert max(st.bond_dims()) == chi
    assert abs(st.log_fid - sum(math.log(f) for f in st.fids)) < 1e-12
    assert st.log_fid < -1e-3
    v = st.to_vector()
    assert abs(np.vdot(v, v) - 1.0) < 1e-12
    # the emulation fidelity estimates the true fidelity (Sec. 2.1.2); here they agree to a few per cent
    psi = statevector.run(c)
    true_f = abs(np.vdot(psi, v)) ** 2
    assert abs(true_f - math.exp(st.log_fid)) < 0.05 * true_f
