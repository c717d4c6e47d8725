"""Small, self-contained GPU cases for profiling single kernels with ncu.

    python -m paper_2501_13237_gb300.profile_cases gemm M N K BATCH [VARIANT]
        random complex64 A (M x K), B (K x N), C on the device; nne_cgemm_c64
        (C = A B + 0.5 C) four times; VARIANT is NNE_OPT_GEMM_TMA (default 2).
    python -m paper_2501_13237_gb300.profile_cases gate [CHI] [N_INST] [SERIAL]
        one saturated two-qubit gate step with the bench's truncation
        (bonds CHI, subspace iteration with k = CHI + 128 columns and four
        power iterations, Rayleigh-Ritz) on N_INST instances; SERIAL = 1 runs
        all instances as one batch on one stream (NNE_OPT_SERIAL_LAYERS), the
        launch mix of the bench's profiled step.
    python -m paper_2501_13237_gb300.profile_cases sweep N CHI N_INST
        a chain of N sites with every bond at CHI (random complex64 site
        tensors, N_INST instances) and one expectation sweep over every
        <Z_i> and <X_i X_i+1> (nne_expect), twice.

Inputs are seeded and synthetic; nothing here is timed or checked.
"""
from __future__ import annotations

import sys

import numpy as np


def gemm(M: int, N: int, K: int, batch: int, variant: int = 2) -> None:
    import torch
    from . import nne
    nne.set_option(nne.OPT_GEMM_TMA, variant)
    ctx = nne.Context(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(batch, M, K, dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn(batch, K, N, dtype=torch.complex64, device="cuda", generator=g)
    C = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    for _ in range(4):
        ctx.cgemm(0, 0, A, B, C, 1.0, 0.5)
    torch.cuda.synchronize()


def gate(chi: int = 512, n_inst: int = 8, serial: int = 0) -> None:
    import workloads as wl
    from . import nne
    n, q = 14, 5
    nne.set_option(nne.OPT_SERIAL_LAYERS, serial)
    ctx = nne.Context(0)
    st = nne.State(ctx, n, chi, n_inst, nne.C64, nne.TRUNC_RSVD)
    st.set_sketch(wl.gaussian_sketch(4 * chi, chi + 128, 1).astype(np.complex64), 4)
    rng = np.random.default_rng(0)

    def rc(shape):
        return ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)
    A, B = rc((chi, 4, chi)), rc((chi, 4, chi))
    G = ctx.build_superops(np.stack([wl.haar_u4(rng)]), wl.n100().rate_table()[:n_inst])
    for i in range(n_inst):
        st.write_site(i, q, A)
        st.write_site(i, q + 1, B)
    st.set_centre(q)
    st.apply_layer([q], G, +1)
    st.sync()
    st.close()


def sweep(n: int, chi: int, n_inst: int) -> None:
    import workloads as wl
    from . import nne
    ctx = nne.Context(0)
    rng = np.random.default_rng(0)
    st = nne.State(ctx, n, chi, n_inst, nne.C64)
    caps = [1] + [min(chi, 4 ** k, 4 ** (n - k)) for k in range(1, n)] + [1]
    for k in range(n):
        M = ((rng.standard_normal((caps[k], 4, caps[k + 1])) + 1j * rng.standard_normal((caps[k], 4, caps[k + 1])))
             / np.sqrt(8.0 * caps[k])).astype(np.complex64)
        for i in range(n_inst):
            st.write_site(i, k, M)
    paulis = wl.pauli_codes(wl.obs_z(n) + wl.obs_xx(n), n)
    for _ in range(2):
        st.expect(paulis)
    st.close()


if __name__ == "__main__":
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    what = sys.argv[1]
    args = [int(x) for x in sys.argv[2:]]
    if what == "gemm":
        gemm(*args)
    elif what == "gate":
        gate(*args)
    elif what == "sweep":
        sweep(*args)
    else:
        raise SystemExit(f"unknown case {what}")
    print("ok")
