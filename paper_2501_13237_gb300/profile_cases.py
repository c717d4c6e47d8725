"""Small, self-contained GPU cases for profiling single kernels with ncu.

    python -m paper_2501_13237_gb300.profile_cases gemm M N K BATCH
        random complex64 A (M x K), B (K x N), C on the device; nne_cgemm_c64
        (C = A B + 0.5 C) four times.
    python -m paper_2501_13237_gb300.profile_cases gate [CHI] [N_INST]
        one saturated two-qubit gate step with randomized truncation
        (bonds CHI, k = CHI + 64, one power iteration) on N_INST instances:
        theta GEMM, range finder, QR panels, the (CHI+64)-dimensional
        tridiagonalisation and the centre split, as in the bench's steps.

Inputs are seeded and synthetic; nothing here is timed or checked.
"""
from __future__ import annotations

import sys

import numpy as np


def gemm(M: int, N: int, K: int, batch: int) -> None:
    import torch
    from . import nne
    ctx = nne.Context(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(batch, M, K, dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn(batch, K, N, dtype=torch.complex64, device="cuda", generator=g)
    C = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    for _ in range(4):
        ctx.cgemm(0, 0, A, B, C, 1.0, 0.5)
    torch.cuda.synchronize()


def gate(chi: int = 512, n_inst: int = 8) -> None:
    import workloads as wl
    from . import nne
    n, q = 14, 5
    ctx = nne.Context(0)
    st = nne.State(ctx, n, chi, n_inst, nne.C64, nne.TRUNC_RSVD)
    st.set_sketch(wl.gaussian_sketch(4 * chi, chi + 64, 1).astype(np.complex64), 1)
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


if __name__ == "__main__":
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    what = sys.argv[1]
    args = [int(x) for x in sys.argv[2:]]
    if what == "gemm":
        gemm(*args)
    elif what == "gate":
        gate(*args)
    else:
        raise SystemExit(f"unknown case {what}")
    print("ok")
