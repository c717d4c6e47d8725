"""Thin ctypes binding of libnne (include/nne.h): argument marshalling only.

Every arithmetic step runs in the CUDA kernels of libnne.so.  Loading fails
loudly when the library is missing: there is no CPU or PyTorch fallback.
Device buffers are torch CUDA tensors (plumbing only); host buffers are
numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnne.so")

OK, PENDING = 0, 1
ERR = {-1: "ARG", -2: "OOM", -3: "CUDA", -4: "NOCONV", -5: "TIMEOUT", -6: "NOFIT", -7: "UNIMPL", -8: "CANCELLED"}
ERR_CANCELLED = -8
C64, C128 = 0, 1
TRUNC_EXACT, TRUNC_RSVD = 0, 1
FIT_POLY, FIT_EXP_LOGLIN, FIT_EXP3 = 0, 1, 2
ERR_NOFIT = -6

# Every symbol include/nne.h declares.
SYMBOLS = (
    "nne_ctx_create", "nne_ctx_destroy", "nne_ctx_bytes_in_use", "nne_last_error", "nne_build_superops",
    "nne_create_state", "nne_destroy_state", "nne_set_sketch", "nne_apply_layer", "nne_truncate", "nne_expect",
    "nne_extrapolate", "nne_sync", "nne_state_info", "nne_state_read_site", "nne_state_write_site",
    "nne_state_set_centre", "nne_reset_state", "nne_kernel_launches", "nne_prof_enable", "nne_prof_collect",
    "nne_extrapolate_noalloc", "nne_cgemm_c64", "nne_set_option",
    "nne_server_create", "nne_job_bytes", "nne_submit", "nne_poll", "nne_server_stats", "nne_server_destroy",
    "nne_extrapolate_ladder", "nne_entropy", "nne_build_pauli_superops", "nne_state_set_log",
    "nne_server_set_log", "nne_cancel", "nne_server_inject_failure",
)
SERVER_DRYRUN = 1


class JobStruct(C.Structure):
    """nne_job (include/nne.h)."""
    _fields_ = [("n_qubits", C.c_int), ("n_layers", C.c_int), ("layer_gates", C.c_void_p),
                ("layer_dir", C.c_void_p), ("left_qubit", C.c_void_p), ("U", C.c_void_p), ("n_lambda", C.c_int),
                ("lambdas", C.c_void_p), ("rates", C.c_void_p), ("chi", C.c_int), ("dtype", C.c_int),
                ("trunc", C.c_int), ("sketch", C.c_void_p), ("sketch_rows", C.c_int), ("sketch_cols", C.c_int),
                ("power_iters", C.c_int), ("init_bits", C.c_void_p), ("n_obs", C.c_int), ("paulis", C.c_void_p),
                ("fit_method", C.c_int), ("fit_degree", C.c_int), ("lambda_star", C.c_double),
                ("pauli_rates", C.c_void_p)]


class ResultStruct(C.Structure):
    """nne_result (include/nne.h)."""
    _fields_ = [("status", C.c_int), ("error", C.c_char * 160), ("values", C.c_void_p), ("log_fid", C.c_void_p),
                ("estimate", C.c_void_p), ("fit_status", C.c_void_p), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double), ("gate_steps", C.c_longlong),
                ("bytes_reserved", C.c_size_t)]


class NNEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libnne status {status} ({ERR.get(status, '?')}): {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libnne.so and declare signatures (raises if the library is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_2501_13237_gb300.build "
                           "(no CPU fallback exists)")
    L = C.CDLL(path)
    vp, i32, dbl, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "nne_ctx_create": (i32, [i32, vp, sz, P(vp)]),
        "nne_ctx_destroy": (None, [vp]),
        "nne_ctx_bytes_in_use": (sz, [vp]),
        "nne_last_error": (C.c_char_p, []),
        "nne_build_superops": (i32, [vp, i32, vp, i32, vp, vp]),
        "nne_create_state": (i32, [vp, i32, i32, i32, i32, i32, vp, P(vp)]),
        "nne_destroy_state": (None, [vp]),
        "nne_set_sketch": (i32, [vp, vp, i32, i32, i32]),
        "nne_apply_layer": (i32, [vp, i32, vp, vp, i32]),
        "nne_truncate": (i32, [vp, i32, vp]),
        "nne_expect": (i32, [vp, i32, vp, vp, vp, vp]),
        "nne_entropy": (i32, [vp, vp]),
        "nne_build_pauli_superops": (i32, [vp, i32, vp, vp, i32, vp, vp]),
        "nne_extrapolate": (i32, [vp, i32, vp, vp, vp, i32, i32, i32, dbl, vp, vp, vp]),
        "nne_sync": (i32, [vp]),
        "nne_state_info": (i32, [vp, vp, vp, vp, vp]),
        "nne_state_read_site": (i32, [vp, i32, i32, vp, sz]),
        "nne_state_write_site": (i32, [vp, i32, i32, i32, i32, vp]),
        "nne_state_set_centre": (i32, [vp, i32]),
        "nne_state_set_log": (i32, [vp, vp, vp]),
        "nne_reset_state": (i32, [vp, vp]),
        "nne_kernel_launches": (C.c_longlong, []),
        "nne_prof_enable": (None, [i32]),
        "nne_prof_collect": (i32, [vp, vp, vp, i32]),
        "nne_extrapolate_noalloc": (i32, [vp, i32, vp, vp, vp, i32, i32, i32, dbl, vp, vp, vp]),
        "nne_cgemm_c64": (i32, [vp, i32, i32, i32, i32, i32, vp, vp, i32, C.c_longlong, vp, i32, C.c_longlong,
                                vp, vp, i32, C.c_longlong, i32]),
        "nne_set_option": (None, [i32, i32]),
        "nne_server_create": (i32, [i32, sz, i32, i32, i32, P(vp)]),
        "nne_job_bytes": (sz, [P(JobStruct)]),
        "nne_submit": (i32, [vp, P(JobStruct), P(C.c_uint64)]),
        "nne_poll": (i32, [vp, C.c_uint64, i32, P(ResultStruct)]),
        "nne_server_stats": (None, [vp, P(i32), P(i32), P(i32), P(sz)]),
        "nne_server_destroy": (None, [vp]),
        "nne_server_set_log": (i32, [vp, C.c_char_p]),
        "nne_cancel": (i32, [vp, C.c_uint64]),
        "nne_server_inject_failure": (i32, [vp, C.c_uint64, i32]),
        "nne_extrapolate_ladder": (i32, [vp, i32, i32, vp, vp, vp, i32, i32, i32, dbl, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        raise NNEError(status, load().nne_last_error().decode(errors="replace"))


def _hptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dptr(t) -> int:
    return int(t.data_ptr())


class Context:
    def __init__(self, device: int = 0, stream=None, hbm_budget_bytes: int = 0):
        L = load()
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        _check(L.nne_ctx_create(device, C.c_void_p(int(stream.cuda_stream)), hbm_budget_bytes, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            load().nne_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self) -> int:
        return int(load().nne_ctx_bytes_in_use(self.h))

    def build_superops(self, U, rates, out=None):
        """a1: U (g,4,4) complex128, rates (n_inst,4) float64 -- numpy (host) or torch CUDA
        tensors (device) -> device tensor (n_inst, g, 16, 16) complex128."""
        import torch

        def ptr(a, dt):
            if isinstance(a, torch.Tensor):
                assert a.is_cuda and a.is_contiguous() and a.dtype == dt
                return C.c_void_p(_dptr(a)), a.shape
            a = np.ascontiguousarray(a, dtype=np.complex128 if dt == torch.complex128 else np.float64)
            return _hptr(a), a.shape, a
        pu = ptr(U, torch.complex128)
        pr = ptr(rates, torch.float64)
        g = pu[1][0]
        ni = (pr[1][0] * pr[1][1]) // 4 if len(pr[1]) == 2 else pr[1][0] // 4
        G = out if out is not None else torch.empty((ni, g, 16, 16), dtype=torch.complex128,
                                                    device=f"cuda:{self.device}")
        _check(load().nne_build_superops(self.h, g, pu[0], ni, pr[0], C.c_void_p(_dptr(G))))
        return G

    def build_pauli_superops(self, U, c0, c1, lambdas, out=None):
        """a1 for gate-dependent Pauli noise: U (g,4,4) complex128, c0 / c1 (g,16)
        probabilities at lambda = 0 and their slopes, lambdas (n_inst,) -> device
        tensor (n_inst, g, 16, 16) complex128."""
        import torch
        U = np.ascontiguousarray(U, dtype=np.complex128)
        pr = np.ascontiguousarray(np.stack([np.asarray(c0, float), np.asarray(c1, float)], axis=1))
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        g, ni = U.shape[0], lam.size
        G = out if out is not None else torch.empty((ni, g, 16, 16), dtype=torch.complex128,
                                                    device=f"cuda:{self.device}")
        _check(load().nne_build_pauli_superops(self.h, g, _hptr(U), _hptr(pr), ni, _hptr(lam),
                                               C.c_void_p(_dptr(G))))
        return G

    def extrapolate(self, lambdas, values, log_fid=None, method=FIT_EXP_LOGLIN, degree=2, lambda_star=1.0,
                    y_zero=None):
        """a8: values (n_lambda, n_obs) -> (estimates[n_obs], status[n_obs])."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        vals = np.ascontiguousarray(values, dtype=np.float64)
        if vals.ndim == 1:
            vals = vals[:, None]
        nl, no = vals.shape
        lf = None if log_fid is None else np.ascontiguousarray(log_fid, dtype=np.float64)
        yz = None if y_zero is None else np.ascontiguousarray(y_zero, dtype=np.float64)
        _check_fit_shapes(lam, lf, yz, nl, no)
        out = np.zeros(no)
        st = np.zeros(no, np.int32)
        _check(load().nne_extrapolate(self.h, nl, _hptr(lam), _hptr(vals), _hptr(lf), no, method, degree,
                                      float(lambda_star), _hptr(yz), _hptr(out), _hptr(st)))
        return out, st


    def extrapolate_ladder(self, lambdas, values, log_fid, method=FIT_EXP_LOGLIN, degree=2, lambda_star=1.0,
                           y_zero=None):
        """(A) + (B) over a bond-dimension ladder: values (k, n_lambda, n_obs), log_fid (k, n_lambda).
        Returns (estimates[n_obs], status[n_obs], obar (n_lambda, n_obs), converged (n_lambda, n_obs))."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        v = np.ascontiguousarray(values, dtype=np.float64)
        lf = np.ascontiguousarray(log_fid, dtype=np.float64)
        k, nl, no = v.shape
        assert lf.shape == (k, nl) and lam.shape == (nl,)
        yz = None if y_zero is None else np.ascontiguousarray(y_zero, dtype=np.float64)
        out = np.zeros(no)
        st = np.zeros(no, dtype=np.int32)
        ob = np.zeros((nl, no))
        cv = np.zeros((nl, no), dtype=np.uint8)
        _check(load().nne_extrapolate_ladder(self.h, k, nl, _hptr(lam), _hptr(v), _hptr(lf), no, method, degree,
                                             float(lambda_star), _hptr(yz), _hptr(out), _hptr(st), _hptr(ob),
                                             _hptr(cv)))
        return out, st, ob, cv.astype(bool)

    def extrapolate_noalloc(self, lambdas, values, log_fid=None, method=FIT_EXP_LOGLIN, degree=2,
                            lambda_star=1.0, y_zero=None):
        """nne_extrapolate_noalloc: the same fit staged through the library's fixed device array
        (for callers that cannot allocate device memory at call time)."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        vals = np.ascontiguousarray(values, dtype=np.float64)
        if vals.ndim == 1:
            vals = vals[:, None]
        nl, no = vals.shape
        lf = None if log_fid is None else np.ascontiguousarray(log_fid, dtype=np.float64)
        yz = None if y_zero is None else np.ascontiguousarray(y_zero, dtype=np.float64)
        _check_fit_shapes(lam, lf, yz, nl, no)
        out = np.zeros(no)
        st = np.zeros(no, np.int32)
        _check(load().nne_extrapolate_noalloc(self.h, nl, _hptr(lam), _hptr(vals), _hptr(lf), no, method, degree,
                                              float(lambda_star), _hptr(yz), _hptr(out), _hptr(st)))
        return out, st


    def cgemm(self, op_a: int, op_b: int, A, B, Cout, alpha=1.0, beta=0.0):
        """Cout[z] = alpha op(A[z]) op(B[z]) + beta Cout[z] on torch complex64 CUDA tensors (batch, rows, cols)."""
        al = np.array([complex(alpha).real, complex(alpha).imag], np.float32)
        be = np.array([complex(beta).real, complex(beta).imag], np.float32)
        M, N = Cout.shape[1], Cout.shape[2]
        K = A.shape[2] if op_a == 0 else A.shape[1]
        _check(load().nne_cgemm_c64(self.h, op_a, op_b, M, N, K, _hptr(al), _vp(A), A.shape[2],
                                    A.shape[1] * A.shape[2], _vp(B), B.shape[2], B.shape[1] * B.shape[2],
                                    _hptr(be), _vp(Cout), Cout.shape[2], Cout.shape[1] * Cout.shape[2],
                                    A.shape[0]))


def _check_fit_shapes(lam, lf, yz, nl: int, no: int):
    """The C side reads n_lambda levels and log-fidelities and n_obs lambda = 0
    values from these host arrays: shorter arrays would be read past their end."""
    if lam.shape != (nl,):
        raise ValueError(f"lambdas has shape {lam.shape}, expected ({nl},)")
    if lf is not None and lf.shape != (nl,):
        raise ValueError(f"log_fid has shape {lf.shape}, expected ({nl},)")
    if yz is not None and yz.shape != (no,):
        raise ValueError(f"y_zero has shape {yz.shape}, expected ({no},)")


def _vp(t):
    return C.c_void_p(_dptr(t))


def set_option(option: int, value: int):
    load().nne_set_option(option, value)


OPT_TENSOR_CORES = 0
OPT_SUBBATCHES = 1
OPT_SERIAL_LAYERS = 2
OPT_EIG_FP64 = 3
OPT_GEMM_TMA = 4
OPT_TEST_WAIT_LIMIT = 5
OPT_SWEEP_CLUSTER = 6


class State:
    def __init__(self, ctx: Context, n: int, chi: int, n_inst: int, dtype: int = C64, trunc: int = TRUNC_EXACT,
                 bits: Optional[Sequence[int]] = None):
        self.ctx, self.n, self.chi, self.n_inst, self.dtype = ctx, n, chi, n_inst, dtype
        b = None if bits is None else np.ascontiguousarray(bits, dtype=np.uint8)
        h = C.c_void_p()
        _check(load().nne_create_state(ctx.h, n, chi, n_inst, dtype, trunc, _hptr(b), C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            load().nne_destroy_state(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sketch(self, omega: np.ndarray, power_iters: int):
        om = np.ascontiguousarray(omega, dtype=np.complex64 if self.dtype == C64 else np.complex128)
        _check(load().nne_set_sketch(self.h, _hptr(om), om.shape[0], om.shape[1], power_iters))

    def apply_layer(self, left_qubits: Sequence[int], G, direction: int):
        """G: device complex128 tensor (n_inst, n_gates, 16, 16) for exactly these gates, in order."""
        qs = np.ascontiguousarray(left_qubits, dtype=np.int32)
        _check(load().nne_apply_layer(self.h, int(qs.size), _hptr(qs), C.c_void_p(_dptr(G)), int(direction)))

    def truncate(self, chi_new: int) -> np.ndarray:
        out = np.zeros(self.n_inst)
        _check(load().nne_truncate(self.h, chi_new, _hptr(out)))
        self.chi = chi_new
        return out

    def expect(self, paulis: np.ndarray):
        """paulis (n_obs, n) uint8 -> (values complex (n_inst, n_obs), log_fid (n_inst))."""
        p = np.ascontiguousarray(paulis, dtype=np.uint8)
        no = p.shape[0]
        re = np.zeros((self.n_inst, no))
        im = np.zeros((self.n_inst, no))
        lf = np.zeros(self.n_inst)
        _check(load().nne_expect(self.h, no, _hptr(p), _hptr(re), _hptr(im), _hptr(lf)))
        return re + 1j * im, lf

    def entropy(self) -> np.ndarray:
        """MPO entanglement entropy per bond, (n_inst, n - 1); S_max is the row maximum."""
        out = np.zeros((self.n_inst, max(self.n - 1, 0)))
        _check(load().nne_entropy(self.h, _hptr(out)))
        return out

    def sync(self):
        _check(load().nne_sync(self.h))

    def info(self):
        dims = np.zeros(self.n + 1, np.int32)
        centre = C.c_int()
        ln = np.zeros(self.n_inst)
        lf = np.zeros(self.n_inst)
        _check(load().nne_state_info(self.h, _hptr(dims), C.byref(centre), _hptr(ln), _hptr(lf)))
        return dims, centre.value, ln, lf

    def read_site(self, inst: int, k: int) -> np.ndarray:
        dims, _, _, _ = self.info()
        dt = np.complex64 if self.dtype == C64 else np.complex128
        out = np.zeros((dims[k], 4, dims[k + 1]), dt)
        _check(load().nne_state_read_site(self.h, inst, k, _hptr(out), out.nbytes))
        return out

    def write_site(self, inst: int, k: int, M: np.ndarray):
        dt = np.complex64 if self.dtype == C64 else np.complex128
        M = np.ascontiguousarray(M, dtype=dt)
        _check(load().nne_state_write_site(self.h, inst, k, M.shape[0], M.shape[2], _hptr(M)))

    def set_centre(self, c: int):
        _check(load().nne_state_set_centre(self.h, c))

    def set_log(self, log_norm=None, log_fid=None):
        ln = None if log_norm is None else np.ascontiguousarray(log_norm, dtype=np.float64)
        lf = None if log_fid is None else np.ascontiguousarray(log_fid, dtype=np.float64)
        _check(load().nne_state_set_log(self.h, _hptr(ln), _hptr(lf)))

    def checkpoint(self) -> dict:
        """Host copy of the whole state: bond dims, centre, log-norm, log F and
        every site tensor of every instance."""
        dims, centre, ln, lf = self.info()
        sites = [[self.read_site(i, k) for k in range(self.n)] for i in range(self.n_inst)]
        return {"dims": dims, "centre": centre, "log_norm": ln, "log_fid": lf, "sites": sites}

    def restore(self, ck: dict):
        """Load a checkpoint of a state with the same n, chi, n_inst and dtype."""
        for i, row in enumerate(ck["sites"]):
            for k, M in enumerate(row):
                self.write_site(i, k, M)
        self.set_centre(int(ck["centre"]))
        self.set_log(ck["log_norm"], ck["log_fid"])

    def reset(self, bits=None):
        b = None if bits is None else np.ascontiguousarray(bits, dtype=np.uint8)
        _check(load().nne_reset_state(self.h, _hptr(b)))


PROF_CLASSES = ("gemm", "superop_epilogue", "tridiag", "bisect", "inviter", "backtransform", "qr_factor",
                "wy_apply", "elementwise", "sweep_env", "sweep_obs", "superop_build", "fit", "gemm_tc", "bisect64")


def kernel_launches() -> int:
    return int(load().nne_kernel_launches())


def prof_enable(on: bool):
    load().nne_prof_enable(1 if on else 0)


def prof_collect():
    """{class: (total_ms, launches, work)} since the last collect (synchronises)."""
    ms = np.zeros(16)
    cnt = np.zeros(16, np.int64)
    wk = np.zeros(16)
    load().nne_prof_collect(_hptr(ms), _hptr(cnt), _hptr(wk), 16)
    return {name: (float(ms[i]), int(cnt[i]), float(wk[i])) for i, name in enumerate(PROF_CLASSES)}


class Job:
    """Host arrays of one nne_job, kept alive while the struct points at them.

    layers: sequence of (left_qubits, U (g,4,4) complex128, direction) in
    application order; rates (n_lambda, 4) channel strengths per level, or
    pauli (gates, 2, 16): gate-dependent Pauli channels (c0, c1 per gate, in
    the same order), with rates None."""

    def __init__(self, n: int, layers, lambdas, rates, chi: int, paulis, dtype: int = C64,
                 trunc: int = TRUNC_EXACT, sketch: Optional[np.ndarray] = None, power_iters: int = 1,
                 bits=None, fit_method: int = FIT_EXP_LOGLIN, fit_degree: int = 2, lambda_star: float = 1.0,
                 pauli: Optional[np.ndarray] = None):
        self.n, self.chi = n, chi
        self.layer_gates = np.array([len(qs) for qs, _, _ in layers], dtype=np.int32)
        self.layer_dir = np.array([d for _, _, d in layers], dtype=np.int32)
        self.left = np.ascontiguousarray(np.concatenate([np.asarray(qs, np.int32) for qs, _, _ in layers])
                                         if layers else np.zeros(0, np.int32))
        self.U = np.ascontiguousarray(np.concatenate([np.asarray(us, np.complex128).reshape(-1, 4, 4)
                                                      for _, us, _ in layers]) if layers
                                      else np.zeros((0, 4, 4), np.complex128))
        self.lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
        self.rates = None if rates is None else np.ascontiguousarray(rates, dtype=np.float64).reshape(-1, 4)
        self.pauli = None if pauli is None else np.ascontiguousarray(pauli, dtype=np.float64).reshape(-1, 2, 16)
        self.paulis = np.ascontiguousarray(paulis, dtype=np.uint8).reshape(-1, n)
        self.bits = None if bits is None else np.ascontiguousarray(bits, dtype=np.uint8)
        self.sketch = None if sketch is None else np.ascontiguousarray(sketch)
        self.n_lambda, self.n_obs = len(self.lambdas), self.paulis.shape[0]
        s = JobStruct()
        s.n_qubits, s.n_layers = n, len(self.layer_gates)
        s.layer_gates, s.layer_dir = _hptr(self.layer_gates), _hptr(self.layer_dir)
        s.left_qubit, s.U = _hptr(self.left), _hptr(self.U)
        s.n_lambda, s.lambdas, s.rates = self.n_lambda, _hptr(self.lambdas), _hptr(self.rates)
        s.chi, s.dtype, s.trunc = chi, dtype, trunc
        if self.sketch is not None:
            s.sketch, s.sketch_rows, s.sketch_cols = _hptr(self.sketch), self.sketch.shape[0], self.sketch.shape[1]
            s.power_iters = power_iters
        s.init_bits = _hptr(self.bits)
        s.n_obs, s.paulis = self.n_obs, _hptr(self.paulis)
        s.fit_method, s.fit_degree, s.lambda_star = fit_method, fit_degree, lambda_star
        s.pauli_rates = _hptr(self.pauli)
        self.struct = s
        self.gate_steps = int(self.layer_gates.sum()) * self.n_lambda

    def bytes(self) -> int:
        return int(load().nne_job_bytes(C.byref(self.struct)))


class Server:
    """nne_server: worker threads running whole jobs on the GPU (FIFO admission
    under a device-memory budget).  dry_run: queueing only, no GPU work."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, workers: int = 2, dry_run: bool = False,
                 dry_run_us: int = 0, log_path: Optional[str] = None):
        L = load()
        h = C.c_void_p()
        _check(L.nne_server_create(device, hbm_budget_bytes, workers, SERVER_DRYRUN if dry_run else 0,
                                   dry_run_us, C.byref(h)))
        self.h = h
        self.jobs = {}
        if log_path is not None:
            self.set_log(log_path)

    def cancel(self, ticket: int) -> bool:
        """Cancel a queued request (True); False if it is already running and
        will complete normally.  Raises for an unknown or finished ticket."""
        rc = load().nne_cancel(self.h, C.c_uint64(ticket))
        if rc == PENDING:
            return False
        _check(rc)
        return True

    def inject_failure(self, ticket: int, status: int):
        """Test hook: the waiting job ends with `status` when a worker takes it."""
        _check(load().nne_server_inject_failure(self.h, C.c_uint64(ticket), status))

    def set_log(self, path: Optional[str]):
        """Append one JSON line per finished job to path (None: stop)."""
        _check(load().nne_server_set_log(self.h, None if path is None else path.encode()))

    def close(self):
        if self.h:
            load().nne_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, job: Job) -> int:
        t = C.c_uint64()
        _check(load().nne_submit(self.h, C.byref(job.struct), C.byref(t)))
        self.jobs[t.value] = job
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """None while pending, else a dict with the job's status and results."""
        job = self.jobs[ticket]
        vals = np.zeros((job.n_lambda, job.n_obs))
        lf = np.zeros(job.n_lambda)
        est = np.zeros(job.n_obs)
        fst = np.zeros(job.n_obs, dtype=np.int32)
        r = ResultStruct()
        r.values, r.log_fid, r.estimate, r.fit_status = _hptr(vals), _hptr(lf), _hptr(est), _hptr(fst)
        rc = load().nne_poll(self.h, ticket, timeout_ms, C.byref(r))
        if rc == PENDING:
            return None
        _check(rc)
        del self.jobs[ticket]
        return {"status": r.status, "error": r.error.decode(errors="replace"), "values": vals, "log_fid": lf,
                "estimate": est, "fit_status": fst, "t_submit": r.t_submit, "t_start": r.t_start,
                "t_end": r.t_end, "gate_steps": r.gate_steps, "bytes": r.bytes_reserved}

    def stats(self):
        q, ru, d, b = C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
        load().nne_server_stats(self.h, C.byref(q), C.byref(ru), C.byref(d), C.byref(b))
        return {"queued": q.value, "running": ru.value, "done": d.value, "bytes_reserved": b.value}
