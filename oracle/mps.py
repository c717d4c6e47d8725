"""VMPO emulator (vectorised density matrix as an MPS, local dim 4) -- ORACLE.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State (Sec. 2.1.1, eqs. vectorized_dm and the MPS form): site tensors
M[k] of shape (chi_k, 4, chi_{k+1}), local index s = 2 i + j for |i><j|.
Initial state: the product |b><b| (Sec. 2.1.2: the initial state is always a
product state, so rho~_0 = rho_0), all bond dimensions 1.

One subcircuit = one gate and its channel on (q, q+1) (the granularity of
the paper's partial fidelities is left open, so this is a reading of
Sec. 2.1.2).  Each subcircuit (Sec. 2.1.2 "Approximate emulation"):
  1. move the orthogonality centre onto the pair (QR / LQ steps; canonical
     form of App. A.1, footnote on bond-local Schmidt values);
  2. theta[a,s1,s2,b] = sum_c M[q][a,s1,c] M[q+1][c,s2,b];
  3. theta'[a,s1',s2',b] = sum G[(s1',s2'),(s1,s2)] theta[a,s1,s2,b]
     (eq. U -> C o U in superoperator form);
  4. X = theta' as a (4 chi_l) x (4 chi_r) matrix, SVD X = U S V^dagger, keep
     r = min(chi, 4 chi_l, 4 chi_r) singular triplets (no relative cutoff):
     by Eckart-Young this is the closest bond-chi state to C_l rho~_{l-1}
     when the rest of the chain is in canonical form.  When nothing is cut
     (r = min(4 chi_l, 4 chi_r)) the split is exact and any basis will do:
     the identity when the isometry's side has dimension r, else the Q of a
     QR factorisation;
  5. normalise the kept part to Frobenius norm 1 (the "closest ... state with
     Frobenius norm 1"), accumulating the dropped scale in log_norm;
  6. partial fidelity f_l = sum_{i<=r} s_i^2 / sum_i s_i^2, which is the
     eq. for f_l evaluated for an orthogonal projection; log F += log f_l
     (eq. emulation_fidelity).
Direction +1 (left to right): the left factor U_r stays on q, the centre
S_r V_r^dagger moves to q+1.  Direction -1: V_r^dagger stays on q+1, the
centre U_r S_r moves to q.  Brickwork schedule (a reading: the paper fixes none): even
layers left to right, odd layers right to left.

Expectation values (Sec. 2.2.3, <O>_lambda; exact contraction of the tensor
network): <P> = Tr(P rho~) / Tr(rho~) with per-site vectors v_P[s] = P[j, i].

Gauge convention (shared with the GPU path so that site tensors are unique):
QR factors have a real non-negative R diagonal; every truncation isometry
(columns ordered by decreasing weight) has each column scaled so its column
sum is real and non-negative.  Observables do not depend on it.

The truncation here is always the exact SVD truncation of the paper; how a
fast implementation reaches the same kept subspace is not modelled.

Pins (tests/test_oracle_mps.py): untruncated runs equal the dense simulator
to 1e-12 (n <= 8); lambda = 0 equals the statevector; truncated runs equal an
independent brute-force emulation that applies each gate to the full dense
rho and projects it with an explicit SVD (n = 6, chi = 4); discarded weight
equals sum_{i>r} s_i^2 (Eckart-Young); F = 1 exactly when nothing is cut
(Sec. 2.1.2 footnote on F = 1); closed forms for identity circuits.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

# v_P[s] = P[j, i] with s = 2 i + j
PAULI_VEC = {
    0: np.array([1, 0, 0, 1], dtype=complex),        # I
    1: np.array([0, 1, 1, 0], dtype=complex),        # X
    2: np.array([0, 1j, -1j, 0], dtype=complex),     # Y
    3: np.array([1, 0, 0, -1], dtype=complex),       # Z
}


def svd(X: np.ndarray, compute_uv: bool = True):
    """Thin SVD by LAPACK: the divide-and-conquer driver (gesdd), or, when it
    reports non-convergence (it does on rare inputs), the QR-iteration driver
    (gesvd).  Both compute the same decomposition."""
    try:
        return np.linalg.svd(X, full_matrices=False, compute_uv=compute_uv)
    except np.linalg.LinAlgError:
        import scipy.linalg
        return scipy.linalg.svd(X, full_matrices=False, compute_uv=compute_uv, lapack_driver="gesvd")


def fix_columns(W: np.ndarray) -> np.ndarray:
    """Gauge convention for an isometry: each column times conj(sum)/|sum| so that
    its column sum is real and non-negative (unchanged when the sum is zero)."""
    s = W.sum(axis=0)
    a = np.abs(s)
    ph = np.where(a > 0, np.conj(s) / np.where(a > 0, a, 1.0), 1.0)
    return W * ph[None, :]


def qr_fixed(M: np.ndarray):
    """Reduced QR with the gauge convention R_jj real and non-negative."""
    Q, R = np.linalg.qr(M)
    d = np.diagonal(R)
    a = np.abs(d)
    ph = np.where(a > 0, d / np.where(a > 0, a, 1.0), 1.0)
    return Q * ph[None, :], np.conj(ph)[:, None] * R


class VMPO:
    def __init__(self, n: int, chi: int, bits=None):
        self.n = n
        self.chi = chi
        bits = [0] * n if bits is None else [int(b) for b in bits]
        self.M: List[np.ndarray] = []
        for b in bits:
            t = np.zeros((1, 4, 1), dtype=complex)
            t[0, 3 * b, 0] = 1.0          # |b><b| -> s = 2b + b
            self.M.append(t)
        self.centre = 0
        self.log_norm = 0.0
        self.log_fid = 0.0
        self.fids: List[float] = []
        self.spectra: List[np.ndarray] = []

    # ------------------------------------------------------------- gauge
    def _qr_right(self, k: int):
        """Make site k left-isometric and push R into site k+1."""
        A = self.M[k]
        cl, _, cr = A.shape
        Q, R = qr_fixed(A.reshape(cl * 4, cr))
        self.M[k] = Q.reshape(cl, 4, Q.shape[1])
        self.M[k + 1] = np.einsum("ij,jsb->isb", R, self.M[k + 1])

    def _lq_left(self, k: int):
        """Make site k right-isometric and push L into site k-1."""
        B = self.M[k]
        cl, _, cr = B.shape
        Q, R = qr_fixed(B.reshape(cl, 4 * cr).conj().T)        # B^dagger = Q R  ->  B = R^dagger Q^dagger
        self.M[k] = Q.conj().T.reshape(Q.shape[1], 4, cr)
        self.M[k - 1] = np.einsum("asj,ji->asi", self.M[k - 1], R.conj().T)

    def move_centre(self, target: int):
        while self.centre < target:
            self._qr_right(self.centre)
            self.centre += 1
        while self.centre > target:
            self._lq_left(self.centre)
            self.centre -= 1

    # ------------------------------------------------------------- gate step
    def gate(self, q: int, G: np.ndarray, direction: int):
        self.move_centre(q if direction > 0 else q + 1)
        left, right, f, nrm, s = two_site_update(self.M[q], self.M[q + 1], G, self.chi, direction)
        self.M[q], self.M[q + 1] = left, right
        self.centre = q + 1 if direction > 0 else q
        self.log_norm += math.log(nrm)
        self.log_fid += math.log(f)
        self.fids.append(f)
        self.spectra.append(s)

    def apply_layer(self, qs: Sequence[int], Gs: Sequence[np.ndarray], direction: int):
        for q, G in zip(qs, Gs):
            self.gate(q, G, direction)

    # ------------------------------------------------------------- compression
    def truncate(self, chi_new: int):
        """Canonical compression sweep to bond dimension chi_new.

        Centre to site 0, then left to right: SVD of each site as a
        (4 chi_l) x chi_r matrix, keep min(chi_new, ...) triplets, push
        S V^dagger right, normalise; f per bond into log F."""
        self.move_centre(0)
        for k in range(self.n - 1):
            A = self.M[k]
            cl, _, cr = A.shape
            Am = A.reshape(cl * 4, cr)
            U, S, Vh = svd(Am)
            r = min(chi_new, S.size)
            total = float(np.sum(S ** 2))
            kept = float(np.sum(S[:r] ** 2))
            Ur = fix_columns(U[:, :r])
            C = Ur.conj().T @ Am
            nrm = float(np.linalg.norm(C))
            self.M[k] = Ur.reshape(cl, 4, r)
            self.M[k + 1] = np.einsum("ij,jsb->isb", C / nrm, self.M[k + 1])
            self.log_norm += math.log(nrm)
            self.log_fid += math.log(kept / total)
            self.centre = k + 1
        self.chi = chi_new

    # ------------------------------------------------------------- observables
    def contract(self, vecs: Sequence[np.ndarray]) -> complex:
        """sum over all s of prod_k v_k[s_k] M[k][:, s_k, :] (full contraction)."""
        E = np.ones((1,), dtype=complex)
        for k in range(self.n):
            T = np.einsum("s,asb->ab", vecs[k], self.M[k])
            E = E @ T
        return complex(E[0])

    def expect_codes(self, codes: np.ndarray) -> np.ndarray:
        """<P> = Tr(P rho)/Tr(rho) for each row of an (n_obs, n) table of Pauli codes."""
        tr = self.contract([PAULI_VEC[0]] * self.n)
        out = np.zeros(codes.shape[0], dtype=complex)
        for i, row in enumerate(codes):
            out[i] = self.contract([PAULI_VEC[int(c)] for c in row]) / tr
        return out

    def trace(self) -> complex:
        return self.contract([PAULI_VEC[0]] * self.n)

    def to_dense(self) -> np.ndarray:
        """Dense rho (2^n x 2^n) times the norm scale exp(log_norm) omitted."""
        T = self.M[0]
        for k in range(1, self.n):
            T = np.tensordot(T, self.M[k], axes=([T.ndim - 1], [0]))
        T = T.reshape([4] * self.n)
        # s = 2 i + j -> split into (i, j) per site, then ket indices first
        T = T.reshape([2, 2] * self.n)
        perm = [2 * k for k in range(self.n)] + [2 * k + 1 for k in range(self.n)]
        return T.transpose(perm).reshape(2 ** self.n, 2 ** self.n)

    def bond_dims(self) -> List[int]:
        return [m.shape[2] for m in self.M[:-1]]

    # ------------------------------------------------------------- entanglement
    def mpo_entropies(self) -> np.ndarray:
        """MPO entanglement entropy S_l for every bond l = 1..n-1 (App. A.1).

        S_l = -sum_i p_i ln p_i with p_i = s_i^2 / sum_j s_j^2, s_i the Schmidt
        coefficients of |rho>> across the cut after qubit l.  In canonical form
        with the centre on site k (App. A.1 footnote) they are the singular
        values of M[k] as a (4 chi_l) x chi_r matrix, for the bond right of k:
        move the centre to site 0, then take the SVD of each site and move on
        by QR.  Leaves the centre at site n-1; the state is unchanged."""
        self.move_centre(0)
        out = np.zeros(self.n - 1)
        for k in range(self.n - 1):
            A = self.M[k]
            s = svd(A.reshape(A.shape[0] * 4, A.shape[2]), compute_uv=False)
            out[k] = entropy_of_schmidt(s)
            self.move_centre(k + 1)
        return out

    def s_max(self) -> float:
        """S_max = max over bonds of S_l (App. A.1); 0 for a single site."""
        return float(np.max(self.mpo_entropies())) if self.n > 1 else 0.0


def entropy_of_schmidt(s: np.ndarray) -> float:
    """-sum p ln p over p_i = s_i^2 / sum s^2 (App. A.1), with 0 ln 0 = 0."""
    w = np.asarray(s, dtype=float) ** 2
    t = float(np.sum(w))
    if t <= 0.0:
        return 0.0
    p = w[w > 0.0] / t
    return float(-np.sum(p * np.log(p)))


def theta_superop(A: np.ndarray, B: np.ndarray, G: np.ndarray) -> np.ndarray:
    """X = (G . theta) as a (4 chi_l) x (4 chi_r) matrix, rows (a, s1'), cols (s2', b)."""
    cl, cr = A.shape[0], B.shape[2]
    theta = np.einsum("asc,ctb->astb", A, B).reshape(cl, 16, cr)
    thetap = np.einsum("uv,avb->aub", G, theta)
    return thetap.reshape(cl * 4, 4 * cr)


def two_site_update(A: np.ndarray, B: np.ndarray, G: np.ndarray, chi: int, direction: int):
    """One subcircuit on a pair in canonical form (steps 2-6 of the module header).
    Returns (new_left, new_right, f, norm_of_kept_part, singular_values)."""
    cl, cr = A.shape[0], B.shape[2]
    X = theta_superop(A, B, G)
    r = min(chi, 4 * cl, 4 * cr)
    if (direction > 0 and r == 4 * cl) or (direction < 0 and r == 4 * cr):
        # nothing can be cut on the isometry's side: keep the identity basis
        S = svd(X, compute_uv=False)
        nrm = float(np.linalg.norm(X))
        if direction > 0:
            return np.eye(4 * cl, dtype=X.dtype).reshape(cl, 4, r), (X / nrm).reshape(r, 4, cr), 1.0, nrm, S
        return (X / nrm).reshape(cl, 4, r), np.eye(4 * cr, dtype=X.dtype).reshape(r, 4, cr), 1.0, nrm, S
    if r == min(4 * cl, 4 * cr):
        # nothing is cut, but the isometry's side is the larger one: exact QR split
        S = svd(X, compute_uv=False)
        if direction > 0:
            Q, Rm = qr_fixed(X)
            nrm = float(np.linalg.norm(Rm))
            return Q.reshape(cl, 4, r), (Rm / nrm).reshape(r, 4, cr), 1.0, nrm, S
        Q, Rm = qr_fixed(X.conj().T)
        nrm = float(np.linalg.norm(Rm))
        return (Rm.conj().T / nrm).reshape(cl, 4, r), Q.conj().T.reshape(r, 4, cr), 1.0, nrm, S
    U, S, Vh = svd(X)
    total = float(np.sum(S ** 2))
    kept = float(np.sum(S[:r] ** 2))
    if direction > 0:
        Ur = fix_columns(U[:, :r])
        C = Ur.conj().T @ X
        nrm = float(np.linalg.norm(C))
        left = Ur.reshape(cl, 4, r)
        right = (C / nrm).reshape(r, 4, cr)
    else:
        Vr = fix_columns(Vh[:r].conj().T)
        C = X @ Vr
        nrm = float(np.linalg.norm(C))
        left = (C / nrm).reshape(cl, 4, r)
        right = Vr.conj().T.reshape(r, 4, cr)
    return left, right, kept / total, nrm, S


def superops_for(circuit, rates) -> List[np.ndarray]:
    """Per layer: (gates, 16, 16) superoperators G at one noise level."""
    from . import channels
    return [np.stack([channels.gate_superop(U, rates) for U in us]) if len(us) else np.zeros((0, 16, 16), complex)
            for us in circuit.unitaries]


def run(circuit, rates, chi: int, bits=None, Gs=None) -> VMPO:
    """Emulate a brickwork circuit at one noise level with the snake schedule."""
    st = VMPO(circuit.n, chi, bits)
    Gs = superops_for(circuit, rates) if Gs is None else Gs
    for t, (qs, G) in enumerate(zip(circuit.layers, Gs)):
        if len(qs) == 0:
            continue
        if t % 2 == 0:
            st.apply_layer(qs, G, +1)
        else:
            st.apply_layer(qs[::-1], G[::-1], -1)
    return st
