"""Thin ctypes binding of the C ABI in include/lelbm.h (argument marshalling only).

Every computation runs in liblelbm.so on the GPU.  There is no fallback: when the
library is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblelbm.so")

LELBM_OK, LELBM_E_INVAL, LELBM_E_NOMEM, LELBM_E_CUDA, LELBM_E_EPR, LELBM_E_TIMEOUT, LELBM_E_STATE = range(7)
LELBM_BC_OUTFLOW, LELBM_BC_INFLOW, LELBM_BC_PERIODIC = 0, 1, 2
LELBM_FP64 = 0
LELBM_MIXED = 1
LELBM_FP32 = 2
STATUS = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_EPR", 5: "E_TIMEOUT", 6: "E_STATE"}


class lelbm_params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("n_batch", ctypes.c_int),
        ("lengths", ctypes.POINTER(ctypes.c_int)),
        ("pads", ctypes.POINTER(ctypes.c_int)),
        ("bc", ctypes.c_int * 4),
        ("inlet", ctypes.c_double * 4),
        ("pad", ctypes.c_int),
        ("K", ctypes.c_double),
        ("nu_shear", ctypes.c_double),
        ("nu_bulk", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("n_conform", ctypes.c_double),
        ("r_min", ctypes.c_double),
        ("refine_div", ctypes.c_double),
        ("refine_rad", ctypes.c_double),
        ("max_refine", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_newton", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("solid", ctypes.POINTER(ctypes.c_ubyte)),
        ("stream", ctypes.c_void_p),
        ("nz", ctypes.c_int),
        ("bc_z", ctypes.c_int * 2),
        ("inlet_uz", ctypes.c_double),
        ("deterministic", ctypes.c_int),
        ("wall_u", ctypes.c_double * 2),
    ]


class lelbm_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("order", ctypes.c_int),
                ("ms", ctypes.c_double)]


class lelbm_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_longlong),
        ("cells", ctypes.c_longlong),
        ("newton_hist", ctypes.c_longlong * 64),
        ("fallback_eq", ctypes.c_longlong),
        ("fallback_mx", ctypes.c_longlong),
        ("q_max", ctypes.c_longlong),
        ("disp_max", ctypes.c_double),
        ("first_fail_cell", ctypes.c_longlong),
        ("cell_kernel_ms", ctypes.c_double),
        ("cell_kernel_launches", ctypes.c_longlong),
        ("points_f", ctypes.c_longlong),
        ("points_g", ctypes.c_longlong),
        ("points_ms", ctypes.c_longlong),
        ("points_32", ctypes.c_longlong),
        ("judge_redo", ctypes.c_longlong),
        ("mlp_retry", ctypes.c_longlong),
        ("wall_hits", ctypes.c_longlong),
        ("mlp_cells", ctypes.c_longlong),
        ("points_df", ctypes.c_longlong),
        ("points_df_corr", ctypes.c_longlong),
    ]


EXPORTS = [
    "lelbm_abi_sizes", "lelbm_default_params", "lelbm_create", "lelbm_destroy", "lelbm_layout", "lelbm_instance",
    "lelbm_set_state", "lelbm_set_moments", "lelbm_set_moments_device", "lelbm_step",
    "lelbm_synchronize", "lelbm_get_moments", "lelbm_get_moments_device", "lelbm_get_macros",
    "lelbm_get_stats", "lelbm_reset_stats", "lelbm_set_timing", "lelbm_last_error",
    "lelbm_step_noalloc", "lelbm_set_steps", "lelbm_run_batch", "lelbm_autotune", "lelbm_set_tuning",
    "lelbm_mlp_size", "lelbm_mlp_init", "lelbm_mlp_loss_grad", "lelbm_mlp_train", "lelbm_step_record",
    "lelbm_set_mlp", "lelbm_set_warmstart", "lelbm_fma_peak", "lelbm_mlp_infer", "lelbm_df_exp2", "lelbm_df_dot",
    "lelbm_set_mlp_gate",
]
LELBM_NOALLOC_MAX_INSTANCES = 16384

_lib = None
_lock = threading.Lock()
_DP = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p


class LelbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblelbm.so (built by ``paper_2508_06911_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2508_06911_gb300.build.build()")
        L = ctypes.CDLL(path)
        L.lelbm_abi_sizes.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        L.lelbm_abi_sizes.restype = None
        L.lelbm_default_params.argtypes = [ctypes.POINTER(lelbm_params)]
        L.lelbm_default_params.restype = None
        L.lelbm_create.argtypes = [ctypes.POINTER(_H), ctypes.POINTER(lelbm_params)]
        L.lelbm_destroy.argtypes = [_H]
        L.lelbm_destroy.restype = None
        L.lelbm_layout.argtypes = [_H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.lelbm_instance.argtypes = [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_int)]
        L.lelbm_set_state.argtypes = [_H, _DP, _DP, _DP]
        L.lelbm_set_moments.argtypes = [_H, _DP]
        L.lelbm_set_moments_device.argtypes = [_H, ctypes.c_void_p]
        L.lelbm_step.argtypes = [_H, ctypes.c_int]
        L.lelbm_synchronize.argtypes = [_H]
        L.lelbm_get_moments.argtypes = [_H, _DP]
        L.lelbm_get_moments_device.argtypes = [_H, ctypes.c_void_p]
        L.lelbm_get_macros.argtypes = [_H, _DP, _DP, _DP]
        L.lelbm_get_stats.argtypes = [_H, ctypes.POINTER(lelbm_stats)]
        L.lelbm_reset_stats.argtypes = [_H]
        L.lelbm_set_timing.argtypes = [_H, ctypes.c_int]
        L.lelbm_fma_peak.argtypes = [ctypes.c_int, _DP]
        L.lelbm_set_mlp_gate.argtypes = [_H, ctypes.c_double]
        L.lelbm_df_exp2.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong, _DP]
        L.lelbm_df_dot.argtypes = [ctypes.POINTER(ctypes.c_float), _DP, ctypes.c_longlong, ctypes.c_longlong, _DP]
        L.lelbm_mlp_infer.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p,
                                      ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
        L.lelbm_last_error.argtypes = [_H]
        L.lelbm_last_error.restype = ctypes.c_char_p
        L.lelbm_set_steps.argtypes = [_H, ctypes.POINTER(ctypes.c_int)]
        L.lelbm_run_batch.argtypes = [_H, ctypes.c_int]
        L.lelbm_autotune.argtypes = [_H, ctypes.c_int, ctypes.POINTER(lelbm_tuning)]
        L.lelbm_set_tuning.argtypes = [_H, ctypes.POINTER(lelbm_tuning)]
        L.lelbm_mlp_size.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        L.lelbm_mlp_init.argtypes = [ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)]
        L.lelbm_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_longlong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]
        L.lelbm_mlp_train.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.lelbm_step_record.argtypes = [_H, ctypes.c_void_p, ctypes.c_void_p]
        L.lelbm_set_mlp.argtypes = [_H, ctypes.POINTER(ctypes.c_float)]
        L.lelbm_set_warmstart.argtypes = [_H, ctypes.c_int]
        L.lelbm_step_noalloc.argtypes = [ctypes.POINTER(lelbm_params), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(lelbm_stats)]
        _lib = L
    return _lib


def _check(rc: int, h=None) -> int:
    if rc != LELBM_OK:
        msg = load().lelbm_last_error(h)
        raise LelbmError(rc, msg.decode() if msg else "")
    return rc


def _dp(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous float64 array")
    return a.ctypes.data_as(_DP)


def lelbm_default_params() -> lelbm_params:
    p = lelbm_params()
    load().lelbm_default_params(ctypes.byref(p))
    return p


def lelbm_abi_sizes():
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    load().lelbm_abi_sizes(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def lelbm_create(p: lelbm_params, lengths=None, solid=None, pads=None) -> int:
    """Create a handle; ``lengths``/``pads`` (1D batch) and ``solid`` (padded uint8 mask) are host arrays.

    They go into a copy of ``p`` (the library copies what it needs during the call), so the
    caller's parameters never point at them afterwards.
    """
    q = lelbm_params.from_buffer_copy(p)
    keep = []
    if lengths is not None:
        arr = np.ascontiguousarray(lengths, dtype=np.int32)
        keep.append(arr)
        q.lengths = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        q.n_batch = len(arr)
    if pads is not None:
        pa = np.ascontiguousarray(pads, dtype=np.int32)
        keep.append(pa)
        q.pads = pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    if solid is not None:
        s = np.ascontiguousarray(solid, dtype=np.uint8)
        keep.append(s)
        q.solid = s.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    h = _H()
    rc = load().lelbm_create(ctypes.byref(h), ctypes.byref(q))
    _check(rc, None)
    return h.value


def lelbm_destroy(h) -> None:
    load().lelbm_destroy(h)


def lelbm_layout(h):
    n, nm, NX, NY = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().lelbm_layout(h, ctypes.byref(n), ctypes.byref(nm), ctypes.byref(NX), ctypes.byref(NY)), h)
    return n.value, nm.value, NX.value, NY.value


def lelbm_instance(h, b: int):
    first, length = ctypes.c_longlong(), ctypes.c_int()
    _check(load().lelbm_instance(h, b, ctypes.byref(first), ctypes.byref(length)), h)
    return first.value, length.value


def lelbm_set_state(h, rho: np.ndarray, u: np.ndarray, RT: np.ndarray) -> None:
    _check(load().lelbm_set_state(h, _dp(rho), _dp(u), _dp(RT)), h)


def lelbm_set_moments(h, m: np.ndarray) -> None:
    _check(load().lelbm_set_moments(h, _dp(m)), h)


def lelbm_set_moments_device(h, ptr: int) -> None:
    _check(load().lelbm_set_moments_device(h, ctypes.c_void_p(ptr)), h)


def lelbm_step(h, n: int = 1) -> None:
    _check(load().lelbm_step(h, n), h)


def lelbm_synchronize(h) -> int:
    """Returns the status (LELBM_E_EPR is returned, not raised)."""
    rc = load().lelbm_synchronize(h)
    if rc not in (LELBM_OK, LELBM_E_EPR):
        _check(rc, h)
    return rc


def lelbm_get_moments(h, out: np.ndarray) -> np.ndarray:
    _check(load().lelbm_get_moments(h, _dp(out)), h)
    return out


def lelbm_get_moments_device(h, ptr: int) -> None:
    _check(load().lelbm_get_moments_device(h, ctypes.c_void_p(ptr)), h)


def lelbm_get_macros(h, rho: np.ndarray, u: np.ndarray, RT: np.ndarray) -> None:
    _check(load().lelbm_get_macros(h, _dp(rho), _dp(u), _dp(RT)), h)


def lelbm_get_stats(h) -> lelbm_stats:
    s = lelbm_stats()
    _check(load().lelbm_get_stats(h, ctypes.byref(s)), h)
    return s


def lelbm_reset_stats(h) -> None:
    _check(load().lelbm_reset_stats(h), h)


def lelbm_set_timing(h, on: bool) -> None:
    _check(load().lelbm_set_timing(h, int(on)), h)


def lelbm_fma_peak(fp64: bool) -> float:
    """Measured FMA throughput (FLOP/s) of the current device's FP32 or FP64 pipe."""
    v = ctypes.c_double(0.0)
    _check(load().lelbm_fma_peak(int(fp64), ctypes.byref(v)), None)
    return v.value


def lelbm_set_mlp_gate(h, departure: float) -> None:
    """Learned start only for cells whose constraints depart from equilibrium by >= departure."""
    _check(load().lelbm_set_mlp_gate(h, float(departure)), h)


def lelbm_df_exp2(w: np.ndarray) -> np.ndarray:
    """The mixed path's double-float 2^(w 2^-54) of int64 fixed-point exponents, as FP64."""
    w = np.ascontiguousarray(w, dtype=np.int64)
    out = np.empty(w.shape[0])
    _check(load().lelbm_df_exp2(w.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), w.shape[0],
                                out.ctypes.data_as(_DP)), None)
    return out


def lelbm_df_dot(k: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Row sums of k * v (k FP32, v FP64 split into double-floats) in the mixed path's
    double-float accumulator; k and v are [rows, terms]."""
    k = np.ascontiguousarray(k, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert k.shape == v.shape and k.ndim == 2
    out = np.empty(k.shape[0])
    _check(load().lelbm_df_dot(k.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.ctypes.data_as(_DP),
                               k.shape[1], k.shape[0], out.ctypes.data_as(_DP)), None)
    return out


def lelbm_mlp_infer(dims: int, params: np.ndarray, X_dev: int, n: int, Y_dev: int, stream: int = 0) -> None:
    """The network's in-kernel inference on n device feature rows (pointers), into Y_dev."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().lelbm_mlp_infer(dims, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), X_dev, n, Y_dev,
                                  stream), None)


def lelbm_set_steps(h, steps) -> None:
    """Per-instance step budgets of a 1D batch (None removes them)."""
    if steps is None:
        _check(load().lelbm_set_steps(h, ctypes.POINTER(ctypes.c_int)()), h)
        return
    arr = np.ascontiguousarray(steps, dtype=np.int32)
    _check(load().lelbm_set_steps(h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), h)


def lelbm_run_batch(h, n: int) -> None:
    _check(load().lelbm_run_batch(h, n), h)


def lelbm_autotune(h, trial_steps: int = 1) -> lelbm_tuning:
    t = lelbm_tuning()
    _check(load().lelbm_autotune(h, trial_steps, ctypes.byref(t)), h)
    return t


def lelbm_set_tuning(h, threads: int = 128, blocks_per_sm: int = 0, order: int = 0) -> None:
    t = lelbm_tuning(threads, blocks_per_sm, order, 0.0)
    _check(load().lelbm_set_tuning(h, ctypes.byref(t)), h)


def lelbm_mlp_size(dims: int):
    """(n_in, n_out, n_params, n_weights) of the warm-start network."""
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().lelbm_mlp_size(dims, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def lelbm_mlp_init(dims: int, seed: int, X_ptr: int, Y_ptr: int, n: int) -> np.ndarray:
    _, _, ntot, _ = lelbm_mlp_size(dims)
    out = np.zeros(ntot, dtype=np.float32)
    _check(load().lelbm_mlp_init(dims, seed, ctypes.c_void_p(X_ptr), ctypes.c_void_p(Y_ptr), n,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def lelbm_mlp_loss_grad(dims: int, params_ptr: int, X_ptr: int, Y_ptr: int, n: int, grad_ptr: int,
                        stream: int | None = None) -> float:
    loss = ctypes.c_double()
    _check(load().lelbm_mlp_loss_grad(dims, ctypes.c_void_p(params_ptr), ctypes.c_void_p(X_ptr),
                                      ctypes.c_void_p(Y_ptr), n, ctypes.c_void_p(grad_ptr), ctypes.byref(loss),
                                      ctypes.c_void_p(stream)))
    return loss.value


def lelbm_mlp_train(dims: int, params_ptr: int, X_ptr: int, Y_ptr: int, n: int, epochs: int, batch: int,
                    lr: float, seed: int = 0, stream: int | None = None) -> np.ndarray:
    losses = np.zeros(epochs)
    _check(load().lelbm_mlp_train(dims, ctypes.c_void_p(params_ptr), ctypes.c_void_p(X_ptr), ctypes.c_void_p(Y_ptr),
                                  n, epochs, batch, lr, seed, losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(stream)))
    return losses


def lelbm_step_record(h, x_ptr: int, y_ptr: int) -> None:
    _check(load().lelbm_step_record(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)), h)


def lelbm_set_mlp(h, params) -> None:
    if params is None:
        _check(load().lelbm_set_mlp(h, ctypes.POINTER(ctypes.c_float)()), h)
        return
    arr = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().lelbm_set_mlp(h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), h)


def lelbm_set_warmstart(h, stored: bool) -> None:
    _check(load().lelbm_set_warmstart(h, int(bool(stored))), h)


def lelbm_last_error(h) -> str:
    m = load().lelbm_last_error(h)
    return m.decode() if m else ""


def lelbm_step_noalloc(p: lelbm_params, m_in_ptr: int, m_out_ptr: int, stats: lelbm_stats | None = None,
                       lengths=None, pads=None) -> int:
    """One allocation-free step on caller-owned device buffers (returns the status code).

    ``lengths``/``pads`` (1D batch) are host arrays kept alive for the call; they go into a
    copy of ``p``, so the caller's parameters never point at them afterwards.
    """
    q = lelbm_params.from_buffer_copy(p)
    keep = []
    if lengths is not None:
        arr = np.ascontiguousarray(lengths, dtype=np.int32)
        keep.append(arr)
        q.lengths = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        q.n_batch = len(arr)
    if pads is not None:
        pa = np.ascontiguousarray(pads, dtype=np.int32)
        keep.append(pa)
        q.pads = pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    sp = ctypes.byref(stats) if stats is not None else ctypes.POINTER(lelbm_stats)()
    return load().lelbm_step_noalloc(ctypes.byref(q), ctypes.c_void_p(m_in_ptr), ctypes.c_void_p(m_out_ptr), sp)
