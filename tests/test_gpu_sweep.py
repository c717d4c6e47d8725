"""GPU parity of the expectation sweep (Sec. 2.2.3, <O> = Tr(O rho)/Tr(rho) by
an exact contraction) through the C ABI, against the oracle's contraction of
the same site tensors.

Random chains written site by site cover what an evolved state may not: bond
dimensions that are odd (the sweep's scalar-load path for complex64) and even
(its 16-byte path), cluster sizes from 1 to 16 CTAs per pass and instance
(the launcher's own choice and forced sizes, powers of two or not), strings on
one site, on two neighbouring sites, on
three or more sites (the carried-vector kernel), strings at both chain ends
and the identity string."""
import numpy as np
import pytest

from oracle import mps
from tests.gpu_util import rand_c, require_gpu

pytestmark = pytest.mark.gpu

# complex128 sweeps run in float64; complex64 sweeps form products in float32
# with float64 sums: relative error ~1e-7 per site of the chain
TOL = {1: 1e-11, 0: 2e-5}


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_2501_13237_gb300 import nne
    return nne.Context(0)


def strings(n, rng):
    codes = []
    for i in range(n):                      # every one-site Pauli
        for p in (1, 2, 3):
            c = np.zeros(n, np.uint8)
            c[i] = p
            codes.append(c)
    for i in range(n - 1):                  # neighbouring pairs, random Paulis
        c = np.zeros(n, np.uint8)
        c[i], c[i + 1] = rng.integers(1, 4, 2)
        codes.append(c)
    for f, l in [(0, 2), (1, n - 1), (0, n - 1), (2, 5)]:   # longer supports
        if l >= n or l - f < 2:
            continue
        c = np.zeros(n, np.uint8)
        c[f], c[l] = rng.integers(1, 4, 2)
        c[f + 1:l] = rng.integers(0, 4, l - f - 1)
        codes.append(c)
    codes.append(np.zeros(n, np.uint8))     # identity
    return np.array(codes, np.uint8)


def run_chain(ctx, dtype, bonds, n_inst, seed):
    from paper_2501_13237_gb300 import nne
    n = len(bonds) - 1
    rng = np.random.default_rng(seed)
    chains = []
    for z in range(n_inst):
        Ms = [rand_c(rng, (bonds[k], 4, bonds[k + 1])) for k in range(n)]
        Ms = [m / np.linalg.norm(m) * np.sqrt(bonds[k]) for k, m in enumerate(Ms)]
        if dtype == 0:
            Ms = [m.astype(np.complex64).astype(np.complex128) for m in Ms]
        chains.append(Ms)
    st = nne.State(ctx, n, max(bonds), n_inst, dtype)
    for z in range(n_inst):
        for k in range(n):
            st.write_site(z, k, chains[z][k])
    codes = strings(n, rng)
    vals, _ = st.expect(codes)
    st.close()
    for z in range(n_inst):
        ref_st = mps.VMPO(n, max(bonds))
        ref_st.M = [m.copy() for m in chains[z]]
        ref = ref_st.expect_codes(codes)
        err = np.abs(vals[z] - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() < TOL[dtype], (z, err.max(), int(np.argmax(err)))
        assert vals[z][-1] == 1.0                                # identity string


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("n_inst", [1, 3, 6, 8])
def test_sweep_random_chain_wide(ctx, dtype, n_inst):
    """Bonds 1, 4, 16, 64, 256, 520, 256, ...: the cluster size the launcher
    picks from occupancy for 2, 6, 12 and 16 clusters."""
    n, chi = 10, 520
    bonds = [min(chi, 4 ** k, 4 ** (n - k)) for k in range(n + 1)]
    run_chain(ctx, dtype, bonds, n_inst, 100 + n_inst + 7 * dtype)


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("cs", [2, 3, 5, 9, 12, 16])
def test_sweep_forced_cluster_sizes(ctx, dtype, cs):
    """Slices of 520- and 517-wide bonds (16-byte and scalar loads) split over
    cluster sizes that divide neither."""
    from paper_2501_13237_gb300 import nne
    n, chi = 11, 520
    bonds = [min(chi, 4 ** k, 4 ** (n - k)) for k in range(n + 1)]
    assert bonds[5] == bonds[6] == 520
    bonds[6] = 517
    nne.set_option(nne.OPT_SWEEP_CLUSTER, cs)
    try:
        run_chain(ctx, dtype, bonds, 2, 300 + cs + dtype)
    finally:
        nne.set_option(nne.OPT_SWEEP_CLUSTER, 0)


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("bonds", [
    [1, 3, 7, 9, 5, 3, 1],                 # odd bonds, 4-CTA clusters below 64 ... 1-CTA below 16
    [1, 4, 13, 33, 66, 31, 62, 15, 4, 1],  # mixed odd / even bonds around 64
    [1, 2, 1, 2, 1],
])
def test_sweep_random_chain_ragged(ctx, dtype, bonds):
    run_chain(ctx, dtype, bonds, 2, sum(bonds) + dtype)
