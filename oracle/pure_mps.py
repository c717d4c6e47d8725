"""Pure-state MPS emulator for the noise-free level lambda = 0 -- ORACLE
(test infrastructure only).

At lambda = 0 the paper emulates the circuit as a pure state (an MPS with
local dimension 2) at a higher bond dimension than the noisy VMPO runs
(Sec. 2.2.3: the lambda = 0 point is the sign reference of criterion 3 and,
run at the higher bond dimension, is taken as converged; Sec. 3.2.1 uses
D = 100 pure against D = 300 mixed).  The algorithm is the VMPO one
(oracle/mps.py) with the local space of one qubit instead of its vectorised
density matrix:

  * site tensors A[k] of shape (chi_k, 2, chi_{k+1}); initial basis state;
  * a gate U on (q, q+1): centre onto the pair, theta[a,s1,s2,b] =
    sum_c A[q][a,s1,c] A[q+1][c,s2,b], theta'[a,s1',s2',b] = sum U[(s1' s2'),
    (s1 s2)] theta[a,s1,s2,b], SVD of theta' as (2 chi_l) x (2 chi_r), keep
    r = min(chi, 2 chi_l, 2 chi_r) triplets, normalise to norm 1, f_l = kept
    weight / total (Sec. 2.1.2, the same closest-state truncation);
  * the snake schedule and the gauge conventions of oracle/mps.py, so that
    an accelerated implementation can be compared tensor by tensor;
  * <P> = <psi|P|psi> / <psi|psi> by a two-layer transfer-matrix sweep;
  * bond entropies -sum p ln p of the squared Schmidt values (the ordinary
    entanglement entropy of a pure state, which the paper plots at
    lambda = 0, Sec. 2.2).

Pins (tests/test_oracle_pure_mps.py): untruncated runs equal the statevector;
after a single truncation the true fidelity |<psi_exact|psi>|^2 equals the
kept weight (Eckart-Young); bond entropies equal the statevector's Schmidt
entropies; untruncated, the VMPO's MPO entropy is twice this entropy.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from .mps import entropy_of_schmidt, fix_columns, qr_fixed

_P2 = {0: np.eye(2, dtype=complex), 1: np.array([[0, 1], [1, 0]], complex),
       2: np.array([[0, -1j], [1j, 0]]), 3: np.array([[1, 0], [0, -1]], complex)}


class PureMPS:
    def __init__(self, n: int, chi: int, bits=None):
        self.n, self.chi = n, chi
        bits = [0] * n if bits is None else [int(b) for b in bits]
        self.A: List[np.ndarray] = []
        for b in bits:
            t = np.zeros((1, 2, 1), dtype=complex)
            t[0, b, 0] = 1.0
            self.A.append(t)
        self.centre = 0
        self.log_norm = 0.0
        self.log_fid = 0.0
        self.fids: List[float] = []

    # ------------------------------------------------------------- gauge
    def _qr_right(self, k: int):
        A = self.A[k]
        cl, _, cr = A.shape
        Q, R = qr_fixed(A.reshape(cl * 2, cr))
        self.A[k] = Q.reshape(cl, 2, Q.shape[1])
        self.A[k + 1] = np.einsum("ij,jsb->isb", R, self.A[k + 1])

    def _lq_left(self, k: int):
        B = self.A[k]
        cl, _, cr = B.shape
        Q, R = qr_fixed(B.reshape(cl, 2 * cr).conj().T)
        self.A[k] = Q.conj().T.reshape(Q.shape[1], 2, cr)
        self.A[k - 1] = np.einsum("asj,ji->asi", self.A[k - 1], R.conj().T)

    def move_centre(self, target: int):
        while self.centre < target:
            self._qr_right(self.centre)
            self.centre += 1
        while self.centre > target:
            self._lq_left(self.centre)
            self.centre -= 1

    # ------------------------------------------------------------- gate step
    def gate(self, q: int, U: np.ndarray, direction: int):
        self.move_centre(q if direction > 0 else q + 1)
        A, B = self.A[q], self.A[q + 1]
        cl, cr = A.shape[0], B.shape[2]
        theta = np.einsum("asc,ctb->astb", A, B).reshape(cl, 4, cr)
        X = np.einsum("uv,avb->aub", U, theta).reshape(cl * 2, 2 * cr)
        r = min(self.chi, 2 * cl, 2 * cr)
        U_, S, Vh = np.linalg.svd(X, full_matrices=False)
        total = float(np.sum(S ** 2))
        kept = float(np.sum(S[:r] ** 2))
        if direction > 0:
            Ur = fix_columns(U_[:, :r])
            C = Ur.conj().T @ X
            nrm = float(np.linalg.norm(C))
            self.A[q] = Ur.reshape(cl, 2, r)
            self.A[q + 1] = (C / nrm).reshape(r, 2, cr)
            self.centre = q + 1
        else:
            Vr = fix_columns(Vh[:r].conj().T)
            C = X @ Vr
            nrm = float(np.linalg.norm(C))
            self.A[q] = (C / nrm).reshape(cl, 2, r)
            self.A[q + 1] = Vr.conj().T.reshape(r, 2, cr)
            self.centre = q
        f = kept / total
        self.log_norm += math.log(nrm)
        self.log_fid += math.log(f)
        self.fids.append(f)

    def apply_layer(self, qs: Sequence[int], Us: Sequence[np.ndarray], direction: int):
        for q, U in zip(qs, Us):
            self.gate(q, U, direction)

    # ------------------------------------------------------------- observables
    def _sandwich(self, ops) -> complex:
        """<psi| prod_k ops[k] |psi> by a two-layer left-to-right sweep."""
        E = np.ones((1, 1), dtype=complex)
        for k in range(self.n):
            A = self.A[k]
            OA = np.einsum("st,atb->asb", ops[k], A)
            E = np.einsum("ac,asb,csd->bd", E, A.conj(), OA)
        return complex(E[0, 0])

    def expect_codes(self, codes: np.ndarray) -> np.ndarray:
        """<psi|P|psi>/<psi|psi> for each row of an (n_obs, n) table of Pauli codes."""
        nrm = self._sandwich([_P2[0]] * self.n)
        return np.array([self._sandwich([_P2[int(c)] for c in row]) / nrm for row in codes])

    def to_vector(self) -> np.ndarray:
        T = self.A[0]
        for k in range(1, self.n):
            T = np.tensordot(T, self.A[k], axes=([T.ndim - 1], [0]))
        return T.reshape(2 ** self.n)

    def entropies(self) -> np.ndarray:
        """Entanglement entropy of every bond from a canonical sweep (centre ends on n-1)."""
        self.move_centre(0)
        out = np.zeros(self.n - 1)
        for k in range(self.n - 1):
            A = self.A[k]
            out[k] = entropy_of_schmidt(np.linalg.svd(A.reshape(A.shape[0] * 2, A.shape[2]), compute_uv=False))
            self.move_centre(k + 1)
        return out

    def bond_dims(self) -> List[int]:
        return [a.shape[2] for a in self.A[:-1]]


def run(circuit, chi: int, bits=None) -> PureMPS:
    """Emulate the unitary circuit (lambda = 0) with the snake schedule of oracle/mps.run."""
    st = PureMPS(circuit.n, chi, bits)
    for t, (qs, us) in enumerate(zip(circuit.layers, circuit.unitaries)):
        if len(qs) == 0:
            continue
        if t % 2 == 0:
            st.apply_layer(qs, us, +1)
        else:
            st.apply_layer(qs[::-1], us[::-1], -1)
    return st
