"""Thin ctypes binding to libpcomp.so (the C ABI in include/pcomp.h).

Functions keep the C names; this module only marshals numpy arrays and
raw device pointers (e.g. ``torch.Tensor.data_ptr()``).  Every step of the
Monte Carlo runs in the CUDA library: if libpcomp.so cannot be loaded the
import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libpcomp.so")

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_ESTATE, PC_EDEVICE = 0, -1, -2, -3, -4, -5

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_u32p = ctypes.POINTER(ctypes.c_uint32)
c_i8p = ctypes.POINTER(ctypes.c_int8)
c_f64p = ctypes.POINTER(ctypes.c_double)
c_f32p = ctypes.POINTER(ctypes.c_float)
c_vp = ctypes.c_void_p
c_int, c_u32, c_u64, c_i64, c_dbl, c_flt = (ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_int64, ctypes.c_double, ctypes.c_float)
c_f32pp = ctypes.POINTER(c_f32p)

# name -> (restype, argtypes); mirrors include/pcomp.h
SIGNATURES = {
    "pc_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_u64]),
    "pc_destroy": (None, [c_vp]),
    "pc_last_error": (ctypes.c_char_p, []),
    "pc_set_stream": (c_int, [c_vp, c_vp]),
    "pc_synchronize": (c_int, [c_vp]),
    "pc_device_sm_count": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "pc_philox": (c_int, [c_vp, c_i64, c_u32p, c_u32p]),
    "pc_pbit_threshold": (c_u32, [c_dbl, c_int]),
    "pc_swap_threshold": (c_u32, [c_dbl, c_i64]),
    "pc_jperp_q": (ctypes.c_int32, [c_dbl, c_int, c_dbl]),
    "pc_apt_load": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_i32p, c_f64p, c_int, c_u32]),
    "pc_apt_run": (c_int, [c_vp, c_i64, c_int, c_int]),
    "pc_apt_progress": (c_int, [c_vp, c_i64p, c_i64p]),
    "pc_apt_set_target": (c_int, [c_vp, c_int, c_i64]),
    "pc_apt_get_state": (c_int, [c_vp, c_int, c_i8p, c_i64p, c_i32p]),
    "pc_apt_get_best": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i32p, c_i64p, c_i8p]),
    "pc_apt_get_best_all": (c_int, [c_vp, c_i64p, c_i64p]),
    "pc_apt_get_stats": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i64p]),
    "pc_apt_get_pbit_table": (c_int, [c_vp, c_int, c_u32p]),
    "pc_apt_get_swap_table": (c_int, [c_vp, c_int, c_int, c_u32p, c_int, ctypes.POINTER(c_int)]),
    "pc_sqa_setup": (c_int, [c_vp, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p]),
    "pc_sqa_get_table": (c_int, [c_vp, c_int, c_u32p, ctypes.POINTER(ctypes.c_int32)]),
    "pc_sqa_run": (c_int, [c_vp, c_int, c_u32, c_i64p, c_i8p]),
    "pc_sqa_run_dev": (c_int, [c_vp, c_int, c_u32, c_vp, c_vp]),
    "pc_sqa_anneal": (c_int, [c_vp, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p, c_int, c_u32, c_i64p]),
    "pc_sqa_anneal_noalloc": (c_int, [c_int, c_vp, c_u64, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p,
                                      c_int, c_u32, c_vp, c_vp]),
    "pc_adaptive_ladder": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_dbl, c_dbl, c_int, c_int,
                                   c_int, c_dbl, c_int, c_f64p, c_f64p, c_i32p, c_i32p]),
    "pc_resample_ladder": (c_int, [c_f64p, c_int, c_int, c_f64p]),
    "pc_pilot_hist": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_int, c_f64p, c_int, c_int, c_int,
                              c_int, c_i64p]),
    "pc_instance_features": (c_int, [c_i32p, c_i8p, c_f64p]),
    "pc_mlp_create": (c_int, [c_vp, ctypes.POINTER(c_vp), c_f32pp, c_f32pp, c_flt]),
    "pc_mlp_destroy": (None, [c_vp]),
    "pc_mlp_forward": (c_int, [c_vp, c_int, c_f32p, c_f32p]),
    "pc_mlp_grads": (c_int, [c_vp, c_int, c_f32p, c_f32p, c_f32p, c_f32pp, c_f32pp]),
    "pc_mlp_train_step": (c_int, [c_vp, c_int, c_f32p, c_f32p, c_flt, c_f32p]),
    "pc_mlp_train_step_dev": (c_int, [c_vp, c_int, c_vp, c_vp, c_flt, c_vp]),
    "pc_mlp_get_params": (c_int, [c_vp, c_f32pp, c_f32pp]),
}

_lib = None


class PcompError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what} failed ({code}): {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libpcomp.so (built by paper_2503_10302_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise ImportError(f"{SO_PATH} is missing: build it with "
                              "`python -m paper_2503_10302_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(SO_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue   # tests/test_abi.py checks that every declared symbol exists
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    m = lib().pc_last_error()
    return m.decode() if m else ""


def check(rc: int, what: str) -> int:
    if rc < 0:
        raise PcompError(rc, what, last_error())
    return rc


def ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _call(name: str, *args) -> int:
    return check(getattr(lib(), name)(*args), name)


# ------------------------------------------------------------------ wrappers
def pc_create(device: int = 0, seed: int = 0) -> ctypes.c_void_p:
    h = c_vp()
    _call("pc_create", ctypes.byref(h), device, c_u64(seed))
    return h


def pc_destroy(ctx) -> None:
    lib().pc_destroy(ctx)


def pc_set_stream(ctx, stream_handle: int) -> None:
    _call("pc_set_stream", ctx, c_vp(stream_handle))


def pc_synchronize(ctx) -> None:
    _call("pc_synchronize", ctx)


def pc_device_sm_count(ctx) -> int:
    n = c_int()
    _call("pc_device_sm_count", ctx, ctypes.byref(n))
    return n.value


def pc_philox(ctx, ctr: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(-1, 4))
    out = np.zeros_like(ctr)
    _call("pc_philox", ctx, ctr.shape[0], ptr(ctr, ctypes.c_uint32), ptr(out, ctypes.c_uint32))
    return out


def pc_pbit_threshold(beta: float, I: int) -> int:
    return int(lib().pc_pbit_threshold(beta, I))


def pc_swap_threshold(dbeta: float, dE: int) -> int:
    return int(lib().pc_swap_threshold(dbeta, dE))


def pc_jperp_q(gamma: float, P: int, T: float) -> int:
    return int(lib().pc_jperp_q(gamma, P, T))


def _dims(d) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(d, np.int32).reshape(-1))


def _J(J) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(J, np.int8))


def pc_sqa_setup(ctx, dims, J, P: int, T: float, gamma) -> None:
    d, j = _dims(dims), _J(J)
    g = np.ascontiguousarray(np.asarray(gamma, np.float64))
    _call("pc_sqa_setup", ctx, ptr(d, ctypes.c_int32), ptr(j, ctypes.c_int8), P, T, len(g),
          ptr(g, ctypes.c_double))


def pc_sqa_get_table(ctx, sweep: int):
    out = np.zeros((3, 7), np.uint32)
    jq = ctypes.c_int32()
    _call("pc_sqa_get_table", ctx, sweep, ptr(out, ctypes.c_uint32), ctypes.byref(jq))
    return out, jq.value


def pc_sqa_run(ctx, R: int, run0: int, P: int, N: int, want_spins: bool = False):
    E = np.zeros((R, P), np.int64)
    S = np.zeros((R, P, N), np.int8) if want_spins else None
    _call("pc_sqa_run", ctx, R, c_u32(run0), ptr(E, ctypes.c_int64), ptr(S, ctypes.c_int8))
    return (E, S) if want_spins else E


def pc_sqa_run_dev(ctx, R: int, run0: int, E_dev_ptr: int, best_dev_ptr: int = 0) -> None:
    _call("pc_sqa_run_dev", ctx, R, c_u32(run0), c_vp(E_dev_ptr), c_vp(best_dev_ptr or None))


def pc_sqa_anneal(ctx, dims, J, P: int, T: float, gamma, R: int, run0: int = 0) -> np.ndarray:
    d, j = _dims(dims), _J(J)
    g = np.ascontiguousarray(np.asarray(gamma, np.float64))
    E = np.zeros((R, P), np.int64)
    _call("pc_sqa_anneal", ctx, ptr(d, ctypes.c_int32), ptr(j, ctypes.c_int8), P, T, len(g),
          ptr(g, ctypes.c_double), R, c_u32(run0), ptr(E, ctypes.c_int64))
    return E


def pc_sqa_anneal_noalloc(device: int, stream_handle: int, seed: int, dims, J, P: int, T: float,
                          gamma, R: int, run0: int, E_dev_ptr: int, best_dev_ptr: int = 0) -> None:
    """Allocation-free DT-SQA anneal into caller-owned device buffers."""
    d, j = _dims(dims), _J(J)
    g = np.ascontiguousarray(np.asarray(gamma, np.float64))
    _call("pc_sqa_anneal_noalloc", device, c_vp(stream_handle or None), c_u64(seed),
          ptr(d, ctypes.c_int32), ptr(j, ctypes.c_int8), P, T, len(g), ptr(g, ctypes.c_double), R,
          c_u32(run0), c_vp(E_dev_ptr), c_vp(best_dev_ptr or None))


class Context:
    """Owns a pc_ctx on one device."""

    def __init__(self, device: int = 0, seed: int = 0):
        self.h = pc_create(device, seed)
        self.seed = seed

    def close(self):
        if getattr(self, "h", None) is not None:
            pc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
