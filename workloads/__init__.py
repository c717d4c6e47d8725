"""Seeded synthetic inputs for the NZNE hot path.

This module is the only code that both the CPU oracle and the CUDA path use.
It draws random numbers and describes workloads; it holds none of the
method's arithmetic (no channel, superoperator, contraction, truncation or
fit).  Everything the method consumes that is random -- the Haar-random
two-qubit gates, the mix of circuit sizes, the request arrival times -- is
generated here once and handed to both sides as plain arrays.

Circuit recipe (1D brickwork, open boundary):
  * qubits 0..n-1 on a line; layer t holds the gates on pairs (q, q+1) with
    q = t mod 2, 2 + t mod 2, ...;
  * every gate is a Haar-random U(4): Z = (randn + i randn)/sqrt(2) as a 4x4
    matrix, Q, R = qr(Z), U = Q diag(R_ii / |R_ii|) (the phase fix makes the
    distribution exactly Haar);
  * gates are drawn layer-major, left to right, from
    numpy.random.default_rng(seed);
  * U acts on |b_q b_{q+1}> with b_q the more significant bit.

Noise recipe: each workload names base rates for the channels the paper
builds its noise models from (two-qubit depolarizing, App. C.2.1; plus
amplitude damping, dephasing and single-qubit depolarizing named in
Sec. 2.2.1) and a set of amplification multipliers lambda; the channel
strength at level lambda is base_rate * lambda.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import numpy as np

# Channel kinds, in the order they are composed after every gate.
CHANNELS = ("depol2", "amp_damp", "dephase", "depol1")


def haar_u4(rng: np.random.Generator) -> np.ndarray:
    """One Haar-random 4x4 unitary (QR of a complex Gaussian with phase fix)."""
    z = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def brickwork_pairs(n: int, depth: int) -> List[List[int]]:
    """Left qubit q of every gate (q, q+1), per layer, left to right."""
    return [list(range(t % 2, n - 1, 2)) for t in range(depth)]


@dataclasses.dataclass
class Circuit:
    n: int
    depth: int
    layers: List[List[int]]          # left qubit per gate, per layer (left to right)
    unitaries: List[np.ndarray]      # per layer: (gates_in_layer, 4, 4) complex128

    @property
    def n_gates(self) -> int:
        return sum(len(l) for l in self.layers)


def brickwork_circuit(n: int, depth: int, seed: int) -> Circuit:
    rng = np.random.default_rng(seed)
    layers = brickwork_pairs(n, depth)
    us = []
    for qs in layers:
        us.append(np.stack([haar_u4(rng) for _ in qs]) if qs else np.zeros((0, 4, 4), complex))
    return Circuit(n=n, depth=depth, layers=layers, unitaries=us)


def identity_circuit(n: int, depth: int) -> Circuit:
    """Brickwork of identity gates: the noise channels act alone."""
    layers = brickwork_pairs(n, depth)
    us = [np.stack([np.eye(4, dtype=complex) for _ in qs]) if qs else np.zeros((0, 4, 4), complex)
          for qs in layers]
    return Circuit(n=n, depth=depth, layers=layers, unitaries=us)


@dataclasses.dataclass
class NoiseModel:
    """Base rates (strength at lambda = 1) of each channel applied after every gate."""
    depol2: float = 0.0
    amp_damp: float = 0.0
    dephase: float = 0.0
    depol1: float = 0.0

    def rates(self, lam: float) -> np.ndarray:
        """Channel strengths at multiplier lam, in CHANNELS order (float64[4])."""
        return np.array([self.depol2, self.amp_damp, self.dephase, self.depol1], float) * lam


@dataclasses.dataclass
class Workload:
    name: str
    circuit: Circuit
    noise: NoiseModel
    lambdas: Tuple[float, ...]
    chi: int
    observables: List[Tuple[Tuple[int, str], ...]]   # each a tuple of (qubit, 'X'|'Y'|'Z')
    lambda_star: float = 1.0
    fit: str = "poly2"
    init_bits: Tuple[int, ...] = ()

    @property
    def n(self) -> int:
        return self.circuit.n

    def bits(self) -> np.ndarray:
        b = np.zeros(self.n, np.uint8)
        if self.init_bits:
            b[:] = np.asarray(self.init_bits, np.uint8)
        return b

    def rate_table(self) -> np.ndarray:
        """(n_lambda, 4) channel strengths per level."""
        return np.stack([self.noise.rates(l) for l in self.lambdas])


def obs_z(n: int) -> List[Tuple[Tuple[int, str], ...]]:
    return [((i, "Z"),) for i in range(n)]


def obs_zz(n: int) -> List[Tuple[Tuple[int, str], ...]]:
    return [((i, "Z"), (i + 1, "Z")) for i in range(n - 1)]


def obs_xx(n: int) -> List[Tuple[Tuple[int, str], ...]]:
    return [((i, "X"), (i + 1, "X")) for i in range(n - 1)]


def pauli_codes(observables, n: int) -> np.ndarray:
    """(n_obs, n) uint8 table: 0=I 1=X 2=Y 3=Z."""
    code = {"I": 0, "X": 1, "Y": 2, "Z": 3}
    out = np.zeros((len(observables), n), np.uint8)
    for i, ob in enumerate(observables):
        for q, p in ob:
            out[i, q] = code[p]
    return out


# ---------------------------------------------------------------- workloads
def exact8(seed: int = 0) -> Workload:
    """n=8, 8 brickwork layers, 2q depolarizing p=1e-3*lambda, lambda in {1,2,4,8};
    chi=256 (=4^(n/2): no truncation); <Z_i> and <Z_i Z_i+1>; quadratic fit to lambda*=1."""
    return Workload("exact8_n8_d8_chi256", brickwork_circuit(8, 8, seed), NoiseModel(depol2=1e-3),
                    (1.0, 2.0, 4.0, 8.0), 256, obs_z(8) + obs_zz(8), 1.0, "poly2")


def n32(seed: int = 0) -> Workload:
    """n=32, depth 20, depolarizing 1e-3*lambda + amplitude damping 5e-4*lambda,
    lambda in {1,1.5,2,3,4,6}, chi=128, all <Z_i>."""
    return Workload("n32_d20_chi128", brickwork_circuit(32, 20, seed),
                    NoiseModel(depol2=1e-3, amp_damp=5e-4), (1.0, 1.5, 2.0, 3.0, 4.0, 6.0), 128,
                    obs_z(32), 1.0, "exp")


def n100(seed: int = 0, depth: int = 30, chi: int = 512) -> Workload:
    """n=100, depth 30, depolarizing 5e-4*lambda, amplitude damping 1e-3*lambda,
    dephasing 5e-4*lambda, lambda in {1..8}, chi=512; <Z_i> and <X_i X_i+1>;
    exponential fit to lambda*=1."""
    return Workload(f"n100_d{depth}_chi{chi}", brickwork_circuit(100, depth, seed),
                    NoiseModel(depol2=5e-4, amp_damp=1e-3, dephase=5e-4),
                    tuple(float(l) for l in range(1, 9)), chi, obs_z(100) + obs_xx(100), 1.0, "exp")


def batch64(seed: int = 0, n_circuits: int = 64) -> List[Workload]:
    """64 circuits, n ~ U[16,64], depth ~ U[10,40], chi ~ U{32,64,128};
    5 levels lambda in {1..5} of depolarizing 1e-3*lambda + dephasing 5e-4*lambda."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_circuits):
        n = int(rng.integers(16, 65))
        depth = int(rng.integers(10, 41))
        chi = int(rng.choice([32, 64, 128]))
        cseed = int(rng.integers(0, 2**31 - 1))
        out.append(Workload(f"batch{c}_n{n}_d{depth}_chi{chi}", brickwork_circuit(n, depth, cseed),
                            NoiseModel(depol2=1e-3, dephase=5e-4), (1.0, 2.0, 3.0, 4.0, 5.0), chi,
                            obs_z(n), 1.0, "exp"))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    workload: Workload


def serving_stream(seed: int = 0, n_requests: int = 2000, rate_per_s: float = 200.0,
                   n_range=(8, 128), depth_range=(5, 50), chis=(64, 128, 256, 512, 1024),
                   rate_range=(1e-4, 2e-3), levels=(4, 8)) -> List[Request]:
    """Poisson arrivals; per request n, depth, chi, a random mix of channel kinds
    (each of depolarizing / amplitude damping / dephasing on with probability 1/2,
    at least one on) at log-uniform rates, and K levels lambda_j = 1..K."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        chi = int(rng.choice(chis))
        on = rng.random(3) < 0.5
        if not on.any():
            on[int(rng.integers(0, 3))] = True
        r = np.exp(rng.uniform(np.log(rate_range[0]), np.log(rate_range[1]), 3)) * on
        k = int(rng.integers(levels[0], levels[1] + 1))
        cseed = int(rng.integers(0, 2**31 - 1))
        wl = Workload(f"req{i}_n{n}_d{depth}_chi{chi}", brickwork_circuit(n, depth, cseed),
                      NoiseModel(depol2=float(r[0]), amp_damp=float(r[1]), dephase=float(r[2])),
                      tuple(float(j) for j in range(1, k + 1)), chi, obs_z(n), 1.0, "exp")
        out.append(Request(t, wl))
    return out


# ---------------------------------------------------------------- Pauli-noise circuits
# Gate-dependent Pauli noise: after each gate on (q, q+1) the Pauli sigma_a (x)
# sigma_b (a on q, b on q+1; 0=I 1=X 2=Y 3=Z) is applied with probability
# c0[4a+b] + lambda * c1[4a+b].  The tables below are the paper's noise models,
# written as data.

# Cat-qubit noise (App. C.2.2, Table): errors per gate at strength lambda, as
# (probability at lambda = 0, coefficient of lambda) per error.
CAT_TABLE = {
    "Z_theta": {"I": (1.0, -1.0), "Z": (0.0, 1.0)},
    "H": {"I": (1.0, -5.0), "Z": (0.0, 3.0), "X": (0.0, 2.0)},
    "CX": {"I": (1.0, -4.0), "Z1": (0.0, 3.0), "Z2": (0.0, 0.5), "Z1Z2": (0.0, 0.5)},
}

# Matchgate depolarizing channel (App. C.3.1): I with 1 - lambda, each of
# ZI, IZ, XX, XY, YY, YX, ZZ with lambda / 7 (first letter on qubit q).
MATCHGATE_PAULIS = ("ZI", "IZ", "XX", "XY", "YY", "YX", "ZZ")

_PIDX = {"I": 0, "X": 1, "Y": 2, "Z": 3}


def pauli_index(left: str, right: str) -> int:
    return 4 * _PIDX[left] + _PIDX[right]


@dataclasses.dataclass
class PauliCircuit:
    """Two-qubit blocks on (q, q+1), each a unitary followed by a Pauli channel
    whose probabilities are linear in lambda (c0 + lambda c1, 16 per block)."""
    n: int
    name: str
    layers: List[List[int]]          # left qubit per block, per layer
    unitaries: List[np.ndarray]      # per layer: (blocks, 4, 4) complex128
    c0: List[np.ndarray]             # per layer: (blocks, 16) float64
    c1: List[np.ndarray]             # per layer: (blocks, 16) float64

    @property
    def n_gates(self) -> int:
        return sum(len(l) for l in self.layers)

    def probs(self, layer: int, lam: float) -> np.ndarray:
        return self.c0[layer] + lam * self.c1[layer]


def _embed_1q(u2: np.ndarray, on_left: bool) -> np.ndarray:
    return np.kron(u2, np.eye(2)) if on_left else np.kron(np.eye(2), u2)


_H2 = np.array([[1, 1], [1, -1]], complex) / np.sqrt(2.0)
# CX with the control on the more significant (left) qubit, and on the right one
_CX_L = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
_CX_R = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], complex)


def cat_gate_noise(gate: str, on_left: bool) -> Tuple[np.ndarray, np.ndarray]:
    """(c0, c1) over the 16 two-qubit Paulis for one gate of the cat-qubit
    model; on_left: the single-qubit gate, or the CX control, is on qubit q."""
    c0, c1 = np.zeros(16), np.zeros(16)
    for err, (a0, a1) in CAT_TABLE[gate].items():
        if err == "I":
            k = 0
        elif gate == "CX":
            ctrl, targ = ("Z", "I") if err == "Z1" else (("I", "Z") if err == "Z2" else ("Z", "Z"))
            k = pauli_index(ctrl, targ) if on_left else pauli_index(targ, ctrl)
        else:
            k = pauli_index(err, "I") if on_left else pauli_index("I", err)
        c0[k] += a0
        c1[k] += a1
    return c0, c1


def cat_circuit(n: int, depth: int, seed: int) -> PauliCircuit:
    """Random H / CX / Z(theta) circuit under cat-qubit noise: brickwork pairs,
    each block one gate drawn uniformly from {CX, H, Z(theta)}; the CX control,
    and the qubit of a single-qubit gate, is left or right with probability
    1/2; theta ~ U[0, 2 pi).  Single-qubit gates and their noise are embedded
    in the pair's 4x4 space."""
    rng = np.random.default_rng(seed)
    layers = brickwork_pairs(n, depth)
    us, c0s, c1s = [], [], []
    for qs in layers:
        u, a, b = [], [], []
        for _ in qs:
            kind = int(rng.integers(0, 3))
            left = bool(rng.integers(0, 2))
            if kind == 0:
                U, g = (_CX_L if left else _CX_R), "CX"
            elif kind == 1:
                U, g = _embed_1q(_H2, left), "H"
            else:
                th = float(rng.uniform(0.0, 2.0 * np.pi))
                U, g = _embed_1q(np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)]), left), "Z_theta"
            x0, x1 = cat_gate_noise(g, left)
            u.append(U)
            a.append(x0)
            b.append(x1)
        us.append(np.stack(u) if u else np.zeros((0, 4, 4), complex))
        c0s.append(np.stack(a) if a else np.zeros((0, 16)))
        c1s.append(np.stack(b) if b else np.zeros((0, 16)))
    return PauliCircuit(n, f"cat_n{n}_d{depth}_s{seed}", layers, us, c0s, c1s)


def xym_circuit(n: int = 60, steps: int = 30, J: float = 0.5, h: float = 0.23, dt: float = 0.1) -> PauliCircuit:
    """Trotterised XY-model evolution (App. C.1.3) under matchgate depolarizing
    noise: each step is a layer of gates on the even bonds (0,1), (2,3), ...
    followed by a layer on the odd bonds, 59 two-qubit gates per step for
    n = 60 (1770 over 30 steps).  Bond gate exp(-i dt J (XX + YY)); the field
    exp(-i dt h Z) of every qubit is carried by its even-bond gate (n even),
    which is exact because XX + YY commutes with Z (x) I + I (x) Z."""
    XX = np.kron([[0, 1], [1, 0]], [[0, 1], [1, 0]]).astype(complex)
    YY = np.kron([[0, -1j], [1j, 0]], [[0, -1j], [1j, 0]])
    ZI = np.kron(np.diag([1.0, -1.0]), np.eye(2)).astype(complex)
    IZ = np.kron(np.eye(2), np.diag([1.0, -1.0])).astype(complex)

    def expi(Hm):   # exp(-i dt Hm) of a Hermitian 4x4
        w, V = np.linalg.eigh(Hm)
        return (V * np.exp(-1j * dt * w)[None, :]) @ V.conj().T

    U_even = expi(J * (XX + YY) + h * (ZI + IZ))
    U_odd = expi(J * (XX + YY))
    c0, c1 = np.zeros(16), np.zeros(16)
    c0[0], c1[0] = 1.0, -1.0
    for p in MATCHGATE_PAULIS:
        c1[pauli_index(p[0], p[1])] += 1.0 / 7.0
    layers, us, c0s, c1s = [], [], [], []
    for _ in range(steps):
        for par, U in ((0, U_even), (1, U_odd)):
            qs = list(range(par, n - 1, 2))
            layers.append(qs)
            us.append(np.stack([U] * len(qs)))
            c0s.append(np.tile(c0, (len(qs), 1)))
            c1s.append(np.tile(c1, (len(qs), 1)))
    return PauliCircuit(n, f"xym_n{n}_steps{steps}", layers, us, c0s, c1s)


def neel_bits(n: int) -> np.ndarray:
    """|1010...>: qubit 0 in |1>, alternating (App. C.1.3 initial state)."""
    return np.array([(k + 1) % 2 for k in range(n)], np.uint8)


def gaussian_sketch(rows: int, cols: int, seed: int) -> np.ndarray:
    """Complex Gaussian test matrix (rows x cols), unit variance per entry."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))) / np.sqrt(2.0)


def random_site_tensors(n: int, chi: int, seed: int, dtype=np.complex128) -> List[np.ndarray]:
    """Random (unnormalised, non-canonical) site tensors with bond dims
    min(chi, 4^k, 4^(n-k)); used for single-step kernel tests."""
    rng = np.random.default_rng(seed)
    dims = [1] + [min(chi, 4 ** k, 4 ** (n - k)) for k in range(1, n)] + [1]
    out = []
    for k in range(n):
        shp = (dims[k], 4, dims[k + 1])
        out.append(((rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2)).astype(dtype))
    return out
