"""Python face of the complex128 CPU oracle (oracle/rcs_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use this module; the product library never does.
It imports nothing from the CUDA package. Gate lists arrive as numpy structured
arrays with fields kind, flags, q0, q1, theta, phi (the shared input format);
caller-supplied U1/U2 matrices come in a separate {gate index: matrix} dict.

What each function computes is the plain definition of the paper's pipeline
(Section 3.2: state construction, measurement sampling, linear XEB); the
readings the paper leaves open are stated in rcs_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcs_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_uint64_p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2 -fopenmp); returns the library path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_threads.restype = ctypes.c_int
            L.orc_gate_matrix.restype = ctypes.c_int
            L.orc_gate_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          c_double_p, c_double_p]
            L.orc_apply_matrix.restype = None
            L.orc_apply_matrix.argtypes = [c_double_p, ctypes.c_int, ctypes.c_int, c_int32_p, c_double_p]
            L.orc_init_zero.restype = None
            L.orc_init_zero.argtypes = [c_double_p, ctypes.c_int]
            L.orc_run.restype = ctypes.c_int64
            L.orc_run.argtypes = [c_double_p, ctypes.c_int, ctypes.c_int64, c_int32_p, c_int32_p, c_int32_p,
                                  c_int32_p, c_double_p, c_double_p, ctypes.POINTER(c_double_p)]
            L.orc_norm2.restype = ctypes.c_double
            L.orc_norm2.argtypes = [c_double_p, ctypes.c_int]
            L.orc_philox4x64_10.restype = None
            L.orc_philox4x64_10.argtypes = [c_uint64_p, c_uint64_p, c_uint64_p]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_sample.restype = ctypes.c_int
            L.orc_sample.argtypes = [c_double_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     c_uint64_p]
            L.orc_xeb.restype = ctypes.c_double
            L.orc_xeb.argtypes = [c_double_p, ctypes.c_int, c_uint64_p, ctypes.c_int64]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(c_double_p)


def _n_of(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.dtype != np.complex128 or psi.size != 1 << n or not psi.flags.c_contiguous:
        raise ValueError("psi must be a contiguous complex128 array of length 2^n")
    return n


def threads() -> int:
    return lib().orc_threads()


def gate_matrix(kind: int, flags: int = 0, theta: float = 0.0, phi: float = 0.0, u=None) -> np.ndarray:
    """Matrix of one gate as the oracle defines it (2x2 or 4x4 complex128)."""
    m = np.zeros(16, dtype=np.complex128)
    up = None
    if u is not None:
        uu = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(-1))
        up = uu.view(np.float64).ctypes.data_as(c_double_p)
    nq = lib().orc_gate_matrix(int(kind), int(flags), float(theta), float(phi), up, _dp(m.view(np.float64)))
    if nq < 0:
        raise ValueError(f"unknown gate kind {kind}")
    d = 1 << nq
    return m[: d * d].reshape(d, d).copy()


def zero_state(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().orc_init_zero(_dp(psi.view(np.float64)), n)
    return psi


def apply_matrix(psi: np.ndarray, targets, m: np.ndarray) -> np.ndarray:
    """In place: applies the 2^k x 2^k matrix m to qubits `targets` (local index
    j = sum_i bit(targets[i]) 2^i)."""
    n = _n_of(psi)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    k = len(t)
    if len(set(t.tolist())) != k or (k and (t.min() < 0 or t.max() >= n)) or k > 10:
        raise ValueError("bad targets")
    mm = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(1 << k, 1 << k))
    lib().orc_apply_matrix(_dp(psi.view(np.float64)), n, k, t.ctypes.data_as(c_int32_p), _dp(mm.view(np.float64)))
    return psi


def run(psi: np.ndarray, gates: np.ndarray, umats: dict | None = None) -> np.ndarray:
    """In place: applies the gate records to psi one at a time, in order."""
    n = _n_of(psi)
    G = len(gates)
    kind = np.ascontiguousarray(gates["kind"], dtype=np.int32)
    flags = np.ascontiguousarray(gates["flags"], dtype=np.int32)
    q0 = np.ascontiguousarray(gates["q0"], dtype=np.int32)
    q1 = np.ascontiguousarray(gates["q1"], dtype=np.int32)
    th = np.ascontiguousarray(gates["theta"], dtype=np.float64)
    ph = np.ascontiguousarray(gates["phi"], dtype=np.float64)
    keep = []
    uptr = None
    if umats:
        arr = (c_double_p * max(G, 1))()
        for i, m in umats.items():
            mm = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(-1))
            keep.append(mm)
            arr[i] = mm.view(np.float64).ctypes.data_as(c_double_p)
        uptr = arr
    rc = lib().orc_run(_dp(psi.view(np.float64)), n, G, kind.ctypes.data_as(c_int32_p),
                       flags.ctypes.data_as(c_int32_p), q0.ctypes.data_as(c_int32_p), q1.ctypes.data_as(c_int32_p),
                       _dp(th), _dp(ph), uptr)
    if rc != 0:
        raise ValueError(f"oracle rejected gate {-rc - 1}")
    return psi


def simulate(n: int, gates: np.ndarray, umats: dict | None = None) -> np.ndarray:
    return run(zero_state(n), gates, umats)


def norm2(psi: np.ndarray) -> float:
    return lib().orc_norm2(_dp(psi.view(np.float64)), _n_of(psi))


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(c.ctypes.data_as(c_uint64_p), k.ctypes.data_as(c_uint64_p),
                            out.ctypes.data_as(c_uint64_p))
    return out


def uniform(seed: int, s: int) -> float:
    return lib().orc_uniform(seed, s)


def sample(psi: np.ndarray, shots: int, seed: int, first: int = 0) -> np.ndarray:
    """Inverse-CDF samples for shots first .. first+shots-1 (uint64 indices)."""
    out = np.zeros(shots, dtype=np.uint64)
    rc = lib().orc_sample(_dp(psi.view(np.float64)), _n_of(psi), seed, first, shots,
                          out.ctypes.data_as(c_uint64_p))
    if rc != 0:
        raise MemoryError("oracle CDF does not fit in host memory")
    return out


def xeb(psi: np.ndarray, samples: np.ndarray) -> float:
    x = np.ascontiguousarray(samples, dtype=np.uint64)
    return lib().orc_xeb(_dp(psi.view(np.float64)), _n_of(psi), x.ctypes.data_as(c_uint64_p), len(x))
