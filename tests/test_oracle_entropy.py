"""Pins for the MPO entanglement entropy of the oracle (App. A.1).

The VMPO's canonical-form entropies are checked against the definition
itself (dense.mpo_entropy: vec(rho) reshaped at the cut and decomposed), and
both against facts fixed by the mathematics: a product or maximally mixed
state has S_l = 0; for a pure state vec(|psi><psi|) across a cut is the
tensor product of the pure state's Schmidt matrix with its conjugate, so its
squared Schmidt values are products p_a p_b and S_l(rho) = 2 S_vN,l(psi);
the rank across bond l is at most the bond dimension, so S_l <= ln D_l.
"""
import math

import numpy as np
import pytest

from oracle import dense, mps, statevector
import workloads as wl

RATES = (0.02, 0.01, 0.015, 0.005)


def vn_entropy(psi, l, n):
    """von Neumann entanglement entropy of a pure state across the cut after qubit l."""
    s = np.linalg.svd(psi.reshape(2 ** l, 2 ** (n - l)), compute_uv=False)
    p = s ** 2 / np.sum(s ** 2)
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def test_product_and_maximally_mixed_are_zero():
    n = 4
    rho = dense.basis_state([1, 0, 1, 1])
    mixed = np.eye(2 ** n) / 2 ** n
    for l in range(1, n):
        assert abs(dense.mpo_entropy(rho, l, n)) < 1e-14
        assert abs(dense.mpo_entropy(mixed, l, n)) < 1e-14
    st = mps.VMPO(n, 8, bits=[1, 0, 1, 1])
    assert np.all(np.abs(st.mpo_entropies()) < 1e-14)


@pytest.mark.parametrize("n,seed", [(5, 4), (6, 5)])
def test_pure_state_is_twice_von_neumann(n, seed):
    c = wl.brickwork_circuit(n, 5, seed)
    psi = statevector.run(c)
    rho = np.outer(psi, psi.conj())
    st = mps.run(c, (0, 0, 0, 0), 4 ** (n // 2 + 1))
    got = st.mpo_entropies()
    for l in range(1, n):
        want = 2.0 * vn_entropy(psi, l, n)
        assert want > 1e-3                        # a non-trivial cut
        assert abs(dense.mpo_entropy(rho, l, n) - want) < 1e-10
        assert abs(got[l - 1] - want) < 1e-10


@pytest.mark.parametrize("n,depth,seed", [(6, 6, 1), (5, 7, 2)])
def test_canonical_sweep_equals_definition(n, depth, seed):
    c = wl.brickwork_circuit(n, depth, seed)
    st = mps.run(c, RATES, 4 ** (n // 2))         # untruncated
    rho = dense.run(c, RATES)
    got = st.mpo_entropies()
    want = np.array([dense.mpo_entropy(rho, l, n) for l in range(1, n)])
    assert np.all(want > 1e-3)
    assert len(set(np.round(want, 6))) > 1        # bonds differ, so an index shift would show
    assert np.allclose(got, want, atol=1e-10, rtol=0)
    assert st.s_max() == pytest.approx(want.max(), abs=1e-10)


def test_sweep_leaves_state_unchanged_and_bound_by_bond_dimension():
    n = 8
    c = wl.brickwork_circuit(n, 8, 6)
    st = mps.run(c, RATES, 6)                     # truncated
    codes = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    before = st.expect_codes(codes)
    dims = st.bond_dims()
    S = st.mpo_entropies()
    assert np.allclose(st.expect_codes(codes), before, atol=1e-12)
    assert st.centre == n - 1
    for l in range(n - 1):
        assert 0.0 <= S[l] <= math.log(dims[l]) + 1e-12
    assert max(dims) == 6 and S.max() > 0.1
