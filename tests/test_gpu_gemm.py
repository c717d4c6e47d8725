"""The complex64 GEMM used by every gate step (tcgen05 split-TF32 for large
shapes, float32 SIMT otherwise) against a float64 product of the same inputs."""
import numpy as np
import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = require_gpu()
    from paper_2501_13237_gb300 import nne
    return torch, nne, nne.Context(0)


def crand(rng, shape):
    return ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)


def op(a, o):
    return a if o == 0 else np.conj(np.swapaxes(a, -1, -2))


# tc: 3 / 2 = TMA-fed tensor-core kernel (operands pre-split into TF32 planes)
# with 64-byte rows in 4 stages / 128-byte rows in 2 stages, 1 = the
# tensor-core kernel that splits in its producer warps, 0 = float32 SIMT
@pytest.mark.parametrize("tc", [3, 2, 1, 0])
@pytest.mark.parametrize("opa,opb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(200, 150, 77), (128, 128, 16), (256, 384, 512), (65, 300, 33), (512, 64, 1024),
                                   (128, 96, 2055),    # these two split K over CTAs (few tiles, long K)
                                   (300, 257, 130)])   # ragged tiles in M, N and K
def test_cgemm_vs_float64(env, tc, opa, opb, M, N, K):
    torch, nne, ctx = env
    nne.set_option(nne.OPT_TENSOR_CORES, 1 if tc else 0)
    nne.set_option(nne.OPT_GEMM_TMA, {3: 2, 2: 1}.get(tc, 0))
    rng = np.random.default_rng(M + 7 * N + 13 * K + opa + 2 * opb)
    batch = 2
    A = crand(rng, (batch, M, K) if opa == 0 else (batch, K, M))
    B = crand(rng, (batch, K, N) if opb == 0 else (batch, N, K))
    C0 = crand(rng, (batch, M, N))
    alpha, beta = 0.7 - 0.2j, (0.3 + 0.1j if K % 2 else 0.0)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    ctx.cgemm(opa, opb, dA, dB, dC, alpha, beta)
    got = dC.cpu().numpy().astype(np.complex128)
    ref = alpha * (op(A.astype(np.complex128), opa) @ op(B.astype(np.complex128), opb)) + beta * C0
    scale = np.sqrt(K) * np.abs(alpha)
    err = np.abs(got - ref).max() / scale
    nne.set_option(nne.OPT_TENSOR_CORES, 1)
    nne.set_option(nne.OPT_GEMM_TMA, 2)
    # Error per unit sqrt(K) grows linearly in K for both paths: float32 FMA
    # chains (~7e-6 at K = 1024) and, ~8x larger, the tensor cores' float32
    # accumulation in tensor memory, whose additions truncate (5.5e-5 at K = 1024
    # measured on GB300).  A layout or descriptor error would give O(1).
    tol = (1e-5 + 6.5e-8 * K) if tc else (3e-6 + 8e-9 * K)
    assert err < tol, err


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("opa", [0, 1])
def test_cgemm_theta_shape(env, opa, variant):
    """The two-site contraction's shape at chi = 512 (2048 x 2048 x 512, batch
    2) on the TMA-fed kernel against float64."""
    torch, nne, ctx = env
    nne.set_option(nne.OPT_GEMM_TMA, variant)
    rng = np.random.default_rng(512 + opa)
    M, N, K, batch = 2048, 2048, 512, 2
    A = crand(rng, (batch, M, K) if opa == 0 else (batch, K, M))
    B = crand(rng, (batch, K, N))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((batch, M, N), dtype=torch.complex64, device="cuda")
    ctx.cgemm(opa, 0, dA, dB, dC, 1.0, 0.0)
    got = dC.cpu().numpy().astype(np.complex128)
    nne.set_option(nne.OPT_GEMM_TMA, 2)
    ref = op(A.astype(np.complex128), opa) @ B.astype(np.complex128)
    err = np.abs(got - ref).max() / np.sqrt(K)
    assert err < 1e-5 + 6.5e-8 * K, err


def test_expired_wait_reports_timeout_then_recovers(env):
    """Failure detection without a GPU fault: the test hook makes every
    pipeline wait of the TMA-fed GEMM expire at once.  The kernel must record
    NNE_ERR_TIMEOUT, drain its own copies and MMAs and return; the status is
    reported once, and the next GEMM on the same context is correct."""
    torch, nne, ctx = env
    rng = np.random.default_rng(5)
    A, B = crand(rng, (1, 256, 1024)), crand(rng, (1, 1024, 512))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((1, 256, 512), dtype=torch.complex64, device="cuda")
    nne.set_option(nne.OPT_GEMM_TMA, 2)
    nne.set_option(nne.OPT_TEST_WAIT_LIMIT, -1)
    try:
        with pytest.raises(nne.NNEError) as ei:
            ctx.cgemm(0, 0, dA, dB, dC)
        assert ei.value.status == -5
    finally:
        nne.set_option(nne.OPT_TEST_WAIT_LIMIT, 0)
    ctx.cgemm(0, 0, dA, dB, dC)
    ref = A[0].astype(np.complex128) @ B[0].astype(np.complex128)
    assert np.abs(dC.cpu().numpy()[0] - ref).max() / np.sqrt(1024) < 1e-5 + 6.5e-8 * 1024
