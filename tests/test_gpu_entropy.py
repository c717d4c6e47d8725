"""GPU parity of the MPO entanglement entropy sweep (App. A.1) through the C ABI.

Compared with the oracle's canonical-sweep entropies on the same states:
truncated noisy circuits (complex128 within 1e-8; complex64 within 2e-3,
the entropies of states that already differ by the single-precision
truncations, whose expectation values agree to 1e-4), and random chains
written site by site with a bond of 520, where the Gram eigenproblem is
larger than one cluster's shared memory in complex128.  Properties that hold
at any size: the sweep leaves every expectation value unchanged and
0 <= S_l <= ln D_l."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import mps
from tests.gpu_util import rand_c, require_gpu

pytestmark = pytest.mark.gpu

TOL = {1: 1e-8, 0: 1e-4}


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("n,depth,chi,seed", [(10, 10, 16, 3), (9, 8, 12, 4)])
def test_entropy_truncated_vs_oracle(ctx, dtype, n, depth, chi, seed):
    from paper_2501_13237_gb300 import runner
    c = wl.brickwork_circuit(n, depth, seed)
    noise = wl.NoiseModel(depol2=0.02, amp_damp=0.01, dephase=0.01)
    lams = (1.0, 2.0, 3.0)      # gapped cuts (a pure-state VMPO has pairwise-equal Schmidt values)
    rates = np.stack([noise.rates(l) for l in lams])
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    st, before, _ = runner.emulate(ctx, c, rates, chi, paulis, dtype)
    S = st.entropy()
    after, _ = st.expect(paulis)
    dims, centre, _, _ = st.info()
    st.close()
    assert S.shape == (len(lams), n - 1) and centre == n - 1
    assert np.abs(after - before).max() < 10 * TOL[dtype]
    for i in range(len(lams)):
        ref = mps.run(c, rates[i], chi).mpo_entropies()
        assert np.abs(S[i] - ref).max() < TOL[dtype], (i, np.abs(S[i] - ref).max())
        assert ref.max() > 0.05                   # 0.2 to 2.4 on these states
        for k in range(n - 1):
            assert -1e-12 <= S[i, k] <= math.log(dims[k + 1]) + TOL[dtype]


@pytest.mark.parametrize("dtype,tol", [(1, 1e-9), (0, 1e-4)])
def test_entropy_random_chain_wide_bond(ctx, dtype, tol):
    """Random site tensors with bond dimensions 1,4,16,64,256,520,256,...: the
    sweep first brings the chain into canonical form (centre n-1 -> 0), as the
    oracle does from the same tensors."""
    from paper_2501_13237_gb300 import nne
    n, chi = 10, 520
    bonds = [min(chi, 4 ** k, 4 ** (n - k)) for k in range(n + 1)]
    rng = np.random.default_rng(11 + dtype)
    Ms = [rand_c(rng, (bonds[k], 4, bonds[k + 1])) for k in range(n)]
    Ms = [m / np.linalg.norm(m) for m in Ms]        # the chain's norm stays O(1), as in evolved states
    if dtype == 0:
        Ms = [m.astype(np.complex64).astype(np.complex128) for m in Ms]
    st = nne.State(ctx, n, chi, 1, dtype)
    for k in range(n):
        st.write_site(0, k, Ms[k])
    st.set_centre(n - 1)
    S = st.entropy()[0]
    st.close()
    ref_st = mps.VMPO(n, chi)
    ref_st.M = [m.copy() for m in Ms]
    ref_st.centre = n - 1
    ref = ref_st.mpo_entropies()
    assert np.abs(S - ref).max() < tol * max(1.0, ref.max()), np.abs(S - ref).max()
    assert ref[4] > 4.0                              # the 520-wide bond is far from a product


def test_entropy_product_state(ctx):
    from paper_2501_13237_gb300 import nne
    for dtype in (0, 1):
        st = nne.State(ctx, 6, 8, 2, dtype, bits=[1, 0, 0, 1, 1, 0])
        S = st.entropy()
        st.close()
        assert S.shape == (2, 5) and np.abs(S).max() == 0.0
