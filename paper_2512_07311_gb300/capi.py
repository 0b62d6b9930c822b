"""ctypes binding of the C ABI in include/rcs.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing
but convert Python/numpy arguments to C ones and raise RcsError on a non-zero
status. All computation happens in librcs.so's CUDA kernels; if the library is
not built (or cannot load) every call raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .circuits import GATE_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librcs.so")

RCS_OK = 0
RCS_ERR_ARG, RCS_ERR_QUBIT, RCS_ERR_OOM, RCS_ERR_CUDA, RCS_ERR_TIMEOUT, RCS_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
RCS_PREC_FP32_PLAIN, RCS_PREC_FP32_FUSED, RCS_PREC_BF16X3, RCS_PREC_TF32X3 = 0, 1, 2, 3
RCS_OPT_PAIR_PASSES = 1  # opt-in: consecutive BF16x3 passes share one round trip (the pair kernel)
PRECISIONS = {"fp32_plain": RCS_PREC_FP32_PLAIN, "fp32_fused": RCS_PREC_FP32_FUSED, "bf16x3": RCS_PREC_BF16X3,
              "tf32x3": RCS_PREC_TF32X3}


class RcsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rcs error {code}: {msg}")
        self.code = code


class rcs_grid(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("n_removed", ctypes.c_int32),
                ("removed", ctypes.POINTER(ctypes.c_int32))]


class rcs_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("k_max", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_uint64)]


class rcs_plan_stats(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_gates", ctypes.c_int64),
                ("n_passes", ctypes.c_int64), ("k_max", ctypes.c_int32), ("pair_passes", ctypes.c_int32),
                ("hbm_bytes", ctypes.c_double), ("flops", ctypes.c_double), ("prefix_passes", ctypes.c_int64),
                ("prefix_qubits", ctypes.c_int32), ("prefix_stages", ctypes.c_int32),
                ("zero_hbm_bytes", ctypes.c_double)]


class rcs_batch_item(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("n_gates", ctypes.c_size_t), ("shots", ctypes.c_uint64), ("seed", ctypes.c_uint64)]


_P = ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("rcs_create", ctypes.c_int, [ctypes.POINTER(rcs_grid), ctypes.POINTER(rcs_opts), ctypes.POINTER(_P)]),
    ("rcs_destroy", None, [_P]),
    ("rcs_last_error", ctypes.c_char_p, [_P]),
    ("rcs_num_qubits", ctypes.c_int, [_P]),
    ("rcs_set_stream", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("rcs_reset", ctypes.c_int, [_P]),
    ("rcs_apply_circuit", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("rcs_apply_unitary", ctypes.c_int, [_P, ctypes.c_int, _i32p, _f64p]),
    ("rcs_apply_unitaries", ctypes.c_int, [_P, ctypes.c_size_t, _i32p, _i32p, ctypes.POINTER(_f64p)]),
    ("rcs_tc_test_fault", ctypes.c_int, [ctypes.c_int64, ctypes.c_double]),
    ("rcs_plan_build", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_size_t, ctypes.POINTER(rcs_opts), ctypes.POINTER(_P)]),
    ("rcs_plan_info", ctypes.c_int, [_P, ctypes.POINTER(rcs_plan_stats)]),
    ("rcs_plan_layout", ctypes.c_int, [_P, _i32p]),
    ("rcs_qubit_layout", ctypes.c_int, [_P, _i32p]),
    ("rcs_plan_pass", ctypes.c_int, [_P, ctypes.c_size_t, _i32p, _i32p, _f64p]),
    ("rcs_plan_upload", ctypes.c_int, [_P, _P]),
    ("rcs_last_pass_timing", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64)]),
    ("rcs_plan_run", ctypes.c_int, [_P, _P]),
    ("rcs_plan_destroy", None, [_P]),
    ("rcs_amplitudes", ctypes.c_int, [_P, _u64p, ctypes.c_size_t, _f64p]),
    ("rcs_state_read", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, _f32p]),
    ("rcs_state_write", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, _f32p]),
    ("rcs_state_device", ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    ("rcs_sync", ctypes.c_int, [_P]),
    ("rcs_norm", ctypes.c_int, [_P, _f64p]),
    ("rcs_sample", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, _u64p]),
    ("rcs_sample_device", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]),
    ("rcs_sample_range", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _u64p]),
    ("rcs_state_save", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("rcs_state_load", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("rcs_xeb", ctypes.c_int, [_P, _u64p, ctypes.c_size_t, _f64p]),
    ("rcs_xeb_device", ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("rcs_batch_create", ctypes.c_int, [ctypes.POINTER(rcs_batch_item), ctypes.c_size_t, ctypes.POINTER(rcs_opts),
                                        ctypes.POINTER(_P)]),
    ("rcs_batch_launch", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("rcs_batch_wait", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("rcs_batch_size", ctypes.c_int, [_P]),
    ("rcs_batch_info", ctypes.c_int, [_P, ctypes.c_size_t, _i32p, _i32p, ctypes.POINTER(ctypes.c_int64)]),
    ("rcs_batch_result", ctypes.c_int, [_P, ctypes.c_size_t, _u64p, _f64p]),
    ("rcs_batch_state_read", ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_uint64, _f32p]),
    ("rcs_batch_set_fault", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    ("rcs_batch_last_error", ctypes.c_char_p, [_P]),
    ("rcs_batch_tuning", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double)]),
    ("rcs_batch_destroy", None, [_P]),
    ("rcs_batch_run", ctypes.c_int, [ctypes.POINTER(rcs_grid), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.c_size_t, _u64p, _u64p, ctypes.POINTER(_u64p), _f64p,
                                     ctypes.POINTER(rcs_opts)]),
    ("rcs_xeb_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p, ctypes.c_uint64]),
]

_lib = None


def load(path: str | None = None):
    """Loads librcs.so (built by paper_2512_07311_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run paper_2512_07311_gb300.build.build())")
        L = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, ctx=None):
    if code != RCS_OK:
        msg = load().rcs_last_error(ctx)
        raise RcsError(code, msg.decode() if msg else "")


def _gates_ptr(gates: np.ndarray, umats: dict | None):
    """Returns (pointer, keep-alive list) for a GATE_DTYPE array, filling the u
    field of U1/U2 gates from `umats` ({index: complex matrix})."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    keep = [g]
    if umats:
        g = g.copy()
        keep = [g]
        for i, m in umats.items():
            mm = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(-1))
            keep.append(mm)
            g["u"][i] = mm.ctypes.data
    return (g.ctypes.data if len(g) else None), keep


def _opts(precision: int, k_max: int, stream: int, autotune: int = 0, flags: int = 0):
    o = rcs_opts()
    o.precision = precision
    o.k_max = k_max
    o.autotune = autotune
    o.flags = flags
    o.stream = stream
    return o


def rcs_create(n_or_grid, precision: int = RCS_PREC_FP32_FUSED, k_max: int = 0, stream: int = 0,
               autotune: int = 0, flags: int = 0):
    """n_or_grid: a qubit count (1 x n grid) or a circuits.Grid."""
    L = load()
    g = rcs_grid()
    if isinstance(n_or_grid, int):
        g.rows, g.cols, g.n_removed, rem = 1, n_or_grid, 0, None
    else:
        g.rows, g.cols = n_or_grid.rows, n_or_grid.cols
        rem = np.ascontiguousarray(n_or_grid.removed, dtype=np.int32)
        g.n_removed = len(rem)
        g.removed = rem.ctypes.data_as(_i32p) if len(rem) else None
    o = _opts(precision, k_max, stream, autotune, flags)
    out = _P()
    _check(L.rcs_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(out)))
    return out


def rcs_destroy(ctx):
    load().rcs_destroy(ctx)


def rcs_num_qubits(ctx) -> int:
    return load().rcs_num_qubits(ctx)


def rcs_set_stream(ctx, stream: int):
    _check(load().rcs_set_stream(ctx, stream), ctx)


def rcs_reset(ctx):
    _check(load().rcs_reset(ctx), ctx)


def rcs_apply_circuit(ctx, gates: np.ndarray, umats: dict | None = None):
    ptr, keep = _gates_ptr(gates, umats)
    _check(load().rcs_apply_circuit(ctx, ptr, len(keep[0])), ctx)


def rcs_apply_unitary(ctx, targets, u: np.ndarray):
    t = np.ascontiguousarray(targets, dtype=np.int32)
    m = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(-1)).view(np.float64)
    _check(load().rcs_apply_unitary(ctx, len(t), t.ctypes.data_as(_i32p), m.ctypes.data_as(_f64p)), ctx)


def rcs_apply_unitaries(ctx, items):
    """items: sequence of (targets, u) applied in order (consecutive 6-qubit ones share a
    round trip of the state under BF16X3 when the context has RCS_OPT_PAIR_PASSES)."""
    items = list(items)
    ks = np.array([len(t) for t, _ in items], dtype=np.int32)
    tg = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.int32) for t, _ in items]) if items
                              else np.zeros(0, dtype=np.int32))
    mats = [np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(-1)).view(np.float64) for _, u in items]
    ptrs = (_f64p * max(1, len(mats)))(*[m.ctypes.data_as(_f64p) for m in mats])
    _check(load().rcs_apply_unitaries(ctx, len(items), ks.ctypes.data_as(_i32p), tg.ctypes.data_as(_i32p), ptrs),
           ctx)


def rcs_tc_test_fault(skip_tile: int, wait_limit_s: float = 0.0):
    """Test hook of the tensor-core kernels' bounded waits (see include/rcs.h)."""
    _check(load().rcs_tc_test_fault(skip_tile, wait_limit_s))


def rcs_plan_build(n: int, gates: np.ndarray, precision: int = RCS_PREC_FP32_FUSED, k_max: int = 0,
                   umats: dict | None = None, flags: int = 0):
    ptr, keep = _gates_ptr(gates, umats)
    o = _opts(precision, k_max, 0, 0, flags)
    out = _P()
    _check(load().rcs_plan_build(n, ptr, len(keep[0]), ctypes.byref(o), ctypes.byref(out)))
    return out


def rcs_plan_info(plan) -> dict:
    s = rcs_plan_stats()
    _check(load().rcs_plan_info(plan, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in rcs_plan_stats._fields_ if not f.startswith("reserved")}


def rcs_plan_layout(plan, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    _check(load().rcs_plan_layout(plan, out.ctypes.data_as(_i32p)))
    return out


def rcs_qubit_layout(ctx) -> np.ndarray:
    out = np.zeros(rcs_num_qubits(ctx), dtype=np.int32)
    _check(load().rcs_qubit_layout(ctx, out.ctypes.data_as(_i32p)), ctx)
    return out


def rcs_plan_pass(plan, i: int, with_matrix: bool = True):
    k = ctypes.c_int32()
    t = np.zeros(8, dtype=np.int32)
    u = np.zeros(2 * 4**7, dtype=np.float64) if with_matrix else None
    _check(load().rcs_plan_pass(plan, i, ctypes.byref(k), t.ctypes.data_as(_i32p),
                                u.ctypes.data_as(_f64p) if u is not None else None))
    kk = k.value
    mat = None
    if u is not None:
        d = 1 << kk
        mat = u[: 2 * d * d].view(np.complex128).reshape(d, d).copy()
    return t[:kk].copy(), mat


def rcs_last_pass_timing(ctx):
    """(ms, passes) of the full-state passes of the last run on ctx."""
    ms, n = ctypes.c_float(), ctypes.c_int64()
    _check(load().rcs_last_pass_timing(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def rcs_plan_upload(ctx, plan):
    _check(load().rcs_plan_upload(ctx, plan), ctx)


def rcs_plan_run(ctx, plan):
    _check(load().rcs_plan_run(ctx, plan), ctx)


def rcs_plan_destroy(plan):
    load().rcs_plan_destroy(plan)


def rcs_amplitudes(ctx, bits) -> np.ndarray:
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros(2 * len(b), dtype=np.float64)
    _check(load().rcs_amplitudes(ctx, b.ctypes.data_as(_u64p), len(b), out.ctypes.data_as(_f64p)), ctx)
    return out.view(np.complex128)


def rcs_state_read(ctx, first: int = 0, count: int | None = None) -> np.ndarray:
    n = rcs_num_qubits(ctx)
    if count is None:
        count = (1 << n) - first
    out = np.zeros(2 * count, dtype=np.float32)
    _check(load().rcs_state_read(ctx, first, count, out.ctypes.data_as(_f32p)), ctx)
    return out.view(np.complex64)


def rcs_state_write(ctx, values: np.ndarray, first: int = 0):
    v = np.ascontiguousarray(values, dtype=np.complex64).view(np.float32)
    _check(load().rcs_state_write(ctx, first, len(v) // 2, v.ctypes.data_as(_f32p)), ctx)


def rcs_state_device(ctx) -> int:
    p = _P()
    _check(load().rcs_state_device(ctx, ctypes.byref(p)), ctx)
    return p.value or 0


def rcs_sync(ctx):
    _check(load().rcs_sync(ctx), ctx)


def rcs_norm(ctx) -> float:
    out = ctypes.c_double()
    _check(load().rcs_norm(ctx, ctypes.byref(out)), ctx)
    return out.value


def rcs_sample(ctx, shots: int, seed: int) -> np.ndarray:
    out = np.zeros(shots, dtype=np.uint64)
    _check(load().rcs_sample(ctx, shots, seed, out.ctypes.data_as(_u64p)), ctx)
    return out


def rcs_sample_range(ctx, first_shot: int, shots: int, seed: int) -> np.ndarray:
    out = np.zeros(shots, dtype=np.uint64)
    _check(load().rcs_sample_range(ctx, first_shot, shots, seed, out.ctypes.data_as(_u64p)), ctx)
    return out


def rcs_state_save(ctx, path: str):
    _check(load().rcs_state_save(ctx, os.fsencode(path)), ctx)


def rcs_state_load(ctx, path: str):
    _check(load().rcs_state_load(ctx, os.fsencode(path)), ctx)


def rcs_sample_device(ctx, shots: int, seed: int, d_out: int):
    _check(load().rcs_sample_device(ctx, shots, seed, d_out), ctx)


def rcs_xeb(ctx, samples) -> float:
    s = np.ascontiguousarray(samples, dtype=np.uint64)
    out = ctypes.c_double()
    _check(load().rcs_xeb(ctx, s.ctypes.data_as(_u64p), len(s), ctypes.byref(out)), ctx)
    return out.value


def rcs_xeb_device(ctx, d_samples: int, n: int, d_out: int):
    _check(load().rcs_xeb_device(ctx, d_samples, n, d_out), ctx)


def rcs_xeb_static(d_state: int, n_qubits: int, d_samples: int, count: int, d_out: int, stream: int = 0):
    """Allocation-free XEB on caller-owned device buffers (see include/rcs.h)."""
    _check(load().rcs_xeb_static(d_state, n_qubits, d_samples, count, d_out, stream))


# ------------------------------------------------------------------ batched circuits

def rcs_batch_create(items, k_max: int = 0, autotune: int = 1, precision: int = RCS_PREC_FP32_FUSED):
    """items: iterable of (n_qubits, gates GATE_DTYPE array, shots, seed). precision
    RCS_PREC_BF16X3 / RCS_PREC_TF32X3 selects the tensor-core engine (k_max 0 or 6)."""
    items = list(items)
    arr = (rcs_batch_item * len(items))()
    keep = []
    for slot, (n, gates, shots, seed) in zip(arr, items):
        ptr, k = _gates_ptr(gates, None)
        keep.append(k)
        slot.n_qubits = n
        slot.gates = ptr
        slot.n_gates = len(k[0])
        slot.shots = shots
        slot.seed = seed
    o = _opts(precision, k_max, 0, autotune)
    out = _P()
    _check(load().rcs_batch_create(arr, len(items), ctypes.byref(o), ctypes.byref(out)))
    return out


def rcs_batch_launch(batch, stream: int = 0):
    _check(load().rcs_batch_launch(batch, stream))


def rcs_batch_wait(batch, stream: int = 0):
    _check(load().rcs_batch_wait(batch, stream))


def rcs_batch_size(batch) -> int:
    return load().rcs_batch_size(batch)


def rcs_batch_info(batch, i: int) -> dict:
    n, k, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().rcs_batch_info(batch, i, ctypes.byref(n), ctypes.byref(k), ctypes.byref(p)))
    return {"n_qubits": n.value, "k": k.value, "n_passes": p.value}


def rcs_batch_tuning(batch) -> dict:
    """The persistent tensor-core kernel's chosen tiles per work item and the trial time of
    each candidate (ms per launch)."""
    g = ctypes.c_uint32()
    ms = (ctypes.c_double * 5)()
    _check(load().rcs_batch_tuning(batch, ctypes.byref(g), ms))
    return {"tiles_per_item": g.value, "trial_ms": dict(zip((2, 4, 8, 16, 32), list(ms)))}


def rcs_batch_result(batch, i: int, shots: int):
    bits = np.zeros(shots, dtype=np.uint64)
    xeb = ctypes.c_double()
    _check(load().rcs_batch_result(batch, i, bits.ctypes.data_as(_u64p) if shots else None, ctypes.byref(xeb)))
    return bits, xeb.value


def rcs_batch_state_read(batch, i: int) -> np.ndarray:
    n = rcs_batch_info(batch, i)["n_qubits"]
    out = np.zeros(2 << n, dtype=np.float32)
    _check(load().rcs_batch_state_read(batch, i, 0, 1 << n, out.ctypes.data_as(_f32p)))
    return out.view(np.complex64)


def rcs_batch_set_fault(batch, skip_item: int, wait_limit_s: float = 2.0):
    _check(load().rcs_batch_set_fault(batch, skip_item, wait_limit_s))


def rcs_batch_destroy(batch):
    load().rcs_batch_destroy(batch)


def rcs_batch_run(items, precision: int = RCS_PREC_FP32_FUSED, k_max: int = 0, autotune: int = 1, stream: int = 0):
    """items: iterable of (circuits.Grid, gates GATE_DTYPE array, shots, seed). One synchronous call
    for the whole batch; returns [(samples uint64 array, xeb float)] per circuit."""
    items = list(items)
    m = len(items)
    grids = (rcs_grid * m)()
    gptrs = (_P * m)()
    ngates = (ctypes.c_size_t * m)()
    shots = np.array([it[2] for it in items], dtype=np.uint64)
    seeds = np.array([it[3] for it in items], dtype=np.uint64)
    outs = [np.zeros(int(s), dtype=np.uint64) for s in shots]
    optr = (_u64p * m)(*[o.ctypes.data_as(_u64p) for o in outs])
    xeb = np.zeros(m, dtype=np.float64)
    keep = []
    for i, (grid, gates, _, _) in enumerate(items):
        rem = np.ascontiguousarray(grid.removed, dtype=np.int32)
        keep.append(rem)
        grids[i].rows, grids[i].cols, grids[i].n_removed = grid.rows, grid.cols, len(rem)
        grids[i].removed = rem.ctypes.data_as(_i32p) if len(rem) else None
        ptr, k = _gates_ptr(gates, None)
        keep.append(k)
        gptrs[i] = ptr
        ngates[i] = len(k[0])
    o = _opts(precision, k_max, stream, autotune)
    _check(load().rcs_batch_run(grids, gptrs, ngates, m, shots.ctypes.data_as(_u64p), seeds.ctypes.data_as(_u64p),
                                optr, xeb.ctypes.data_as(_f64p), ctypes.byref(o)))
    return [(outs[i], float(xeb[i])) for i in range(m)]
