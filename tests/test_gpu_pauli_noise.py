"""GPU parity for gate-dependent Pauli noise (cat-qubit errors, App. C.2.2;
matchgate depolarizing noise, App. C.3.1) through the C ABI.

* the superoperator builder against the oracle's Kraus sums (1e-13);
* cat-qubit H / CX / Z(theta) circuits and the XY-model circuit, truncated,
  against the oracle VMPO (complex128 1e-8, complex64 1e-4);
* the XY-model circuit untruncated against the exact free-fermion values.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import channels as ch
from oracle import matchgate, mps
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


def test_pauli_superops_match_oracle(ctx):
    pc = wl.cat_circuit(8, 3, 1)
    xy = wl.xym_circuit(6, 1)
    U = np.concatenate(pc.unitaries + xy.unitaries)
    c0 = np.concatenate(pc.c0 + xy.c0)
    c1 = np.concatenate(pc.c1 + xy.c1)
    rng = np.random.default_rng(3)
    U = np.concatenate([U, np.stack([wl.haar_u4(rng) for _ in range(3)])])
    dep0 = np.zeros((3, 16)); dep0[:, 0] = 1.0
    dep1 = np.full((3, 16), 1.0 / 16.0); dep1[:, 0] = -15.0 / 16.0
    c0 = np.concatenate([c0, dep0]); c1 = np.concatenate([c1, dep1])
    lams = np.array([0.0, 0.004, 0.03, 0.1])
    G = ctx.build_pauli_superops(U, c0, c1, lams).cpu().numpy()
    for i, lam in enumerate(lams):
        for g in range(U.shape[0]):
            ref = ch.pauli_gate_superop(U[g], c0[g] + lam * c1[g])
            assert np.abs(G[i, g] - ref).max() < 1e-13
    # the depolarizing rows agree with the fixed-composition builder at strength lambda
    Gd = ctx.build_superops(U[-3:], np.array([[l, 0, 0, 0] for l in lams])).cpu().numpy()
    assert np.abs(G[:, -3:] - Gd).max() < 1e-13


def test_pauli_superops_reject_bad_probabilities(ctx):
    from paper_2501_13237_gb300 import nne
    U = np.stack([np.eye(4, dtype=complex)])
    c0 = np.zeros((1, 16)); c0[0, 0] = 1.0
    c1 = np.zeros((1, 16)); c1[0, 0] = -1.0; c1[0, 3] = 0.5          # sums to 1 - lambda/2
    with pytest.raises(nne.NNEError):
        ctx.build_pauli_superops(U, c0, c1, np.array([0.1]))
    c1[0, 3] = 1.0
    with pytest.raises(nne.NNEError):
        ctx.build_pauli_superops(U, c0, c1, np.array([1.5]))            # p_II < 0


def _vmpo_parity(ctx, pc, lams, chi, dtype, tol, bits=None):
    from paper_2501_13237_gb300 import runner
    n = pc.n
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n) + [((q, "Y"), (q + 1, "X")) for q in range(n - 1)], n)
    layers = runner.build_pauli_layers(ctx, pc, np.asarray(lams, float))
    st, vals, lf = runner.emulate(ctx, pc, None, chi, paulis, dtype, bits=bits, layers=layers)
    st.close()
    cut = False
    for i, lam in enumerate(lams):
        ref = mps.run(pc, None, chi, bits=bits, Gs=ch.pauli_superops_for(pc, lam))
        assert np.abs(vals[i] - ref.expect_codes(paulis)).max() < tol, (lam, np.abs(vals[i] - ref.expect_codes(paulis)).max())
        assert abs(lf[i] - ref.log_fid) < tol * max(1.0, abs(ref.log_fid))
        cut |= ref.log_fid < -1e-6
    return cut


@pytest.mark.parametrize("dtype,tol", [(1, 1e-8), (0, 1e-4)])
def test_cat_circuit_vs_oracle(ctx, dtype, tol):
    # Clifford-heavy circuits have exactly degenerate Schmidt values at many
    # cuts; this seed and chi keep every cut gapped (s_5 / s_4 <= 0.68).
    # Their site tensors are scaled permutations plus rounding noise down to
    # 1e-24, whose float32 squares are denormal: this circuit is the case that
    # needs the gauge moves' reflector pivots formed without squaring tiny
    # entries (before that, complex64 missed by up to 0.13).
    pc = wl.cat_circuit(10, 24, 7)
    assert _vmpo_parity(ctx, pc, (0.0, 0.005, 0.02), 4, dtype, tol)


@pytest.mark.parametrize("dtype,tol", [(1, 1e-8), (0, 1e-4)])
def test_xym_circuit_vs_oracle(ctx, dtype, tol):
    pc = wl.xym_circuit(10, 5, dt=0.3)      # every cut at chi = 6 gapped: s_7 / s_6 <= 0.92
    assert _vmpo_parity(ctx, pc, (0.0, 0.01, 0.05), 6, dtype, tol, bits=wl.neel_bits(10))


def test_xym_untruncated_vs_exact_free_fermions(ctx):
    from paper_2501_13237_gb300 import runner
    n = 8
    pc = wl.xym_circuit(n, 6, dt=0.25)
    bits = wl.neel_bits(n)
    obs = wl.obs_z(n) + wl.obs_xx(n) + [((q, "Y"), (q + 1, "X")) for q in range(n - 1)]
    paulis = wl.pauli_codes(obs, n)
    lams = np.array([0.0, 0.01, 0.05])
    layers = runner.build_pauli_layers(ctx, pc, lams)
    st, vals, lf = runner.emulate(ctx, pc, None, 256, paulis, 1, bits=bits, layers=layers)
    st.close()
    assert np.abs(lf).max() < 1e-10
    for i, lam in enumerate(lams):
        C = matchgate.run(pc, lam, bits)
        ref = np.array([matchgate.expect(C, ob, n) for ob in obs])
        assert np.abs(vals[i].real - ref).max() < 1e-10
        assert np.abs(vals[i].imag).max() < 1e-10
