"""Pins for oracle/mps.py (VMPO emulation, Sec. 2.1)."""
import math

import numpy as np
import pytest

from oracle import channels as ch
from oracle import dense, mps, statevector
import workloads as wl

RATES = (0.02, 0.01, 0.015, 0.005)


def obs_list(n):
    return wl.obs_z(n) + wl.obs_zz(n) + wl.obs_xx(n) + [((i, "Y"),) for i in range(n)] + [((0, "X"), (n - 1, "Y"))]


@pytest.mark.parametrize("n,depth,seed", [(6, 6, 1), (5, 7, 2)])
def test_untruncated_equals_dense(n, depth, seed):
    c = wl.brickwork_circuit(n, depth, seed)
    chi = 4 ** (n // 2)
    st = mps.run(c, RATES, chi)
    rho = dense.run(c, RATES)
    assert abs(st.log_fid) < 1e-12                 # F = 1: nothing cut
    obs = obs_list(n)
    got = st.expect_codes(wl.pauli_codes(obs, n))
    for ob, g in zip(obs, got):
        assert abs(g - dense.expect(rho, ob, n)) < 1e-12
    r = st.to_dense()
    r = r / np.trace(r)
    assert np.allclose(r, rho, atol=1e-12)


def test_exact8_workload_untruncated():
    w = wl.exact8()
    st = mps.run(w.circuit, w.noise.rates(8.0), w.chi)
    rho = dense.run(w.circuit, w.noise.rates(8.0))
    got = st.expect_codes(wl.pauli_codes(w.observables, w.n))
    for ob, g in zip(w.observables, got):
        assert abs(g - dense.expect(rho, ob, w.n)) < 1e-12
    assert max(st.bond_dims()) == 256 and abs(st.log_fid) < 1e-12


def test_zero_noise_equals_statevector():
    n = 8
    c = wl.brickwork_circuit(n, 6, seed=3)
    st = mps.run(c, (0, 0, 0, 0), 4 ** 4)
    psi = statevector.run(c)
    obs = obs_list(n)
    got = st.expect_codes(wl.pauli_codes(obs, n))
    for ob, g in zip(obs, got):
        assert abs(g - statevector.expect(psi, ob, n)) < 1e-12


# --------------------------------------------------------------- brute force
PV = {"I": np.array([1, 0, 0, 1], complex), "X": np.array([0, 1, 1, 0], complex),
      "Y": np.array([0, 1j, -1j, 0], complex), "Z": np.array([1, 0, 0, -1], complex)}


def brute_force(circ, rates, chi, bits=None):
    """Dense vectorised rho (4^n entries, per-site interleaved index); after every
    gate project onto the best rank-chi approximation across the gate's bond with
    an explicit SVD of the whole vector, then renormalise (independent of oracle.mps)."""
    n = circ.n
    bits = bits or [0] * n
    v = np.zeros([4] * n, complex)
    v[tuple(3 * b for b in bits)] = 1.0
    fids = []
    for t, (qs, us) in enumerate(zip(circ.layers, circ.unitaries)):
        order = list(range(len(qs))) if t % 2 == 0 else list(range(len(qs)))[::-1]
        for i in order:
            q, U = qs[i], us[i]
            G = ch.gate_superop(U, rates).reshape(4, 4, 4, 4)
            v = np.moveaxis(np.tensordot(G, v, axes=([2, 3], [q, q + 1])), [0, 1], [q, q + 1])
            mat = v.reshape(4 ** (q + 1), 4 ** (n - q - 1))
            U_, S, Vh = np.linalg.svd(mat, full_matrices=False)
            r = min(chi, S.size)
            fids.append(float(np.sum(S[:r] ** 2) / np.sum(S ** 2)))
            mat = (U_[:, :r] * S[:r]) @ Vh[:r]
            v = (mat / np.linalg.norm(mat)).reshape([4] * n)
    return v, fids


def bf_expect(v, ob, n):
    vecs = [PV["I"]] * n
    for q, p in ob:
        vecs = list(vecs)
        vecs[q] = PV[p]
    num, den = v, v
    for k in range(n):
        num = np.tensordot(vecs[k], num, axes=([0], [0]))
        den = np.tensordot(PV["I"], den, axes=([0], [0]))
    return complex(num / den)


@pytest.mark.parametrize("n,depth,chi,seed", [(6, 6, 4, 7), (6, 5, 8, 8), (5, 6, 3, 9)])
def test_truncated_equals_brute_force(n, depth, chi, seed):
    c = wl.brickwork_circuit(n, depth, seed)
    st = mps.run(c, RATES, chi)
    v, fids = brute_force(c, RATES, chi)
    assert len(fids) == len(st.fids)
    assert np.allclose(st.fids, fids, atol=1e-11)
    assert st.log_fid < -1e-6                       # something was cut
    obs = obs_list(n)
    got = st.expect_codes(wl.pauli_codes(obs, n))
    for ob, g in zip(obs, got):
        assert abs(g - bf_expect(v, ob, n)) < 1e-10


def test_eckart_young_discarded_weight():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((8, 4, 16)) + 1j * rng.standard_normal((8, 4, 16))
    B = rng.standard_normal((16, 4, 8)) + 1j * rng.standard_normal((16, 4, 8))
    G = ch.gate_superop(wl.haar_u4(rng), RATES)
    X = mps.theta_superop(A, B, G)
    for direction in (+1, -1):
        left, right, f, nrm, s = mps.two_site_update(A, B, G, 12, direction)
        Xr = np.einsum("asc,ctb->astb", left, right).reshape(X.shape) * nrm
        assert abs(np.linalg.norm(X - Xr) ** 2 - np.sum(s[12:] ** 2)) < 1e-9 * np.sum(s ** 2)
        assert abs(f - np.sum(s[:12] ** 2) / np.sum(s ** 2)) < 1e-14
        # isometry of the non-centre factor
        if direction > 0:
            L = left.reshape(-1, 12)
            assert np.allclose(L.conj().T @ L, np.eye(12), atol=1e-12)
        else:
            R = right.reshape(12, -1)
            assert np.allclose(R @ R.conj().T, np.eye(12), atol=1e-12)


def test_theta_superop_layout():
    # X[(a,s1'),(s2',b)] = sum G[(s1's2'),(s1s2)] A[a,s1,c] B[c,s2,b], by explicit loops
    rng = np.random.default_rng(5)
    A = rng.standard_normal((2, 4, 3)) + 1j * rng.standard_normal((2, 4, 3))
    B = rng.standard_normal((3, 4, 2)) + 1j * rng.standard_normal((3, 4, 2))
    G = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    X = mps.theta_superop(A, B, G)
    for a in range(2):
        for u1 in range(4):
            for u2 in range(4):
                for b in range(2):
                    ref = 0
                    for s1 in range(4):
                        for s2 in range(4):
                            for c in range(3):
                                ref += G[4 * u1 + u2, 4 * s1 + s2] * A[a, s1, c] * B[c, s2, b]
                    assert abs(X[a * 4 + u1, u2 * 2 + b] - ref) < 1e-12


def test_identity_closed_forms_via_mps():
    n, depth, p = 6, 6, 0.04
    c = wl.identity_circuit(n, depth)
    st = mps.run(c, (p, 0, 0, 0), 16)
    got = st.expect_codes(wl.pauli_codes(wl.obs_z(n), n)).real
    for q in range(n):
        k = sum(1 for qs in c.layers for g in qs if g == q or g + 1 == q)
        assert abs(got[q] - (1 - p) ** k) < 1e-13
    st = mps.run(c, (0, 0, 0, p), 16)
    got = st.expect_codes(wl.pauli_codes(wl.obs_z(n), n)).real
    for q in range(n):
        k = sum(1 for qs in c.layers for g in qs if g == q or g + 1 == q)
        assert abs(got[q] - (1 - 4 * p / 3) ** k) < 1e-13


def test_frobenius_normalised_and_trace_real():
    c = wl.brickwork_circuit(6, 6, 12)
    st = mps.run(c, RATES, 8)
    C = st.M[st.centre]
    assert abs(np.linalg.norm(C) - 1) < 1e-12          # Frobenius norm 1 (Sec. 2.1.2)
    tr = st.trace()
    assert abs(tr.imag) < 1e-12 * abs(tr.real)


def test_truncate_sweep_matches_sequential_projection():
    n = 6
    c = wl.brickwork_circuit(n, 6, 13)
    st = mps.run(c, RATES, 64)
    v = st.to_dense()
    # dense vectorised tensor in per-site interleaved order, as brute_force uses
    T = v.reshape([2] * (2 * n))
    perm = []
    for k in range(n):
        perm += [k, n + k]
    vec = T.transpose(perm).reshape([4] * n)
    vec = vec / np.linalg.norm(vec)
    fids = []
    for k in range(n - 1):
        mat = vec.reshape(4 ** (k + 1), -1)
        U_, S, Vh = np.linalg.svd(mat, full_matrices=False)
        r = min(5, S.size)
        fids.append(float(np.sum(S[:r] ** 2) / np.sum(S ** 2)))
        mat = (U_[:, :r] * S[:r]) @ Vh[:r]
        vec = (mat / np.linalg.norm(mat)).reshape([4] * n)
    before = st.log_fid
    st.truncate(5)
    assert abs((st.log_fid - before) - sum(math.log(f) for f in fids)) < 1e-10
    obs = obs_list(n)
    got = st.expect_codes(wl.pauli_codes(obs, n))
    for ob, g in zip(obs, got):
        assert abs(g - bf_expect(vec, ob, n)) < 1e-10


