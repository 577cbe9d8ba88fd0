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
    "pc_apt_load_bc": (c_int, [c_vp, c_int, c_i32p, c_vp, c_vp, c_i8p, c_i32p, c_f64p, c_int, c_u32]),
    "pc_apt_run": (c_int, [c_vp, c_i64, c_int, c_int]),
    "pc_apt_set_joint_swap": (c_int, [c_vp, c_int]),
    "pc_apt_set_icm_rules": (c_int, [c_vp, c_int, c_int]),
    "pc_apt_set_split": (c_int, [c_vp, c_int]),
    "pc_apt_is_split": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "pc_apt_autotune": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "pc_apt_set_launch": (c_int, [c_vp, c_int, c_int, c_int, c_int]),
    "pc_apt_set_block_threads": (c_int, [c_vp, c_int]),
    "pc_apt_save": (c_int, [c_vp, ctypes.c_char_p]),
    "pc_apt_restore": (c_int, [c_vp, ctypes.c_char_p]),
    "pc_apt_progress": (c_int, [c_vp, c_i64p, c_i64p]),
    "pc_apt_set_target": (c_int, [c_vp, c_int, c_i64]),
    "pc_apt_get_state": (c_int, [c_vp, c_int, c_i8p, c_i64p, c_i32p]),
    "pc_apt_get_best": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i32p, c_i64p, c_i8p]),
    "pc_apt_get_best_all": (c_int, [c_vp, c_i64p, c_i64p]),
    "pc_apt_get_stats": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i64p]),
    "pc_apt_get_pbit_table": (c_int, [c_vp, c_int, c_u32p]),
    "pc_apt_get_swap_table": (c_int, [c_vp, c_int, c_int, c_u32p, c_int, ctypes.POINTER(c_int)]),
    "pc_sqa_setup": (c_int, [c_vp, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p]),
    "pc_sqa_setup_bc": (c_int, [c_vp, c_i32p, c_vp, c_vp, c_i8p, c_int, c_dbl, c_int, c_f64p]),
    "pc_sqa_upload_bytes": (c_i64, [c_int, c_int]),
    "pc_sqa_get_table": (c_int, [c_vp, c_int, c_u32p, ctypes.POINTER(ctypes.c_int32)]),
    "pc_sqa_run": (c_int, [c_vp, c_int, c_u32, c_i64p, c_i8p]),
    "pc_sqa_run_dev": (c_int, [c_vp, c_int, c_u32, c_vp, c_vp]),
    "pc_sqa_run_corr_dev": (c_int, [c_vp, c_int, c_u32, c_vp, c_vp, c_vp]),
    "pc_sqa_selftest_wait": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "pc_sqa_anneal": (c_int, [c_vp, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p, c_int, c_u32, c_i64p]),
    "pc_sqa_anneal_noalloc": (c_int, [c_int, c_vp, c_u64, c_i32p, c_i8p, c_int, c_dbl, c_int, c_f64p,
                                      c_int, c_u32, c_vp, c_vp]),
    "pc_adaptive_ladder": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_dbl, c_dbl, c_int, c_int,
                                   c_int, c_dbl, c_int, c_f64p, c_f64p, c_i32p, c_i32p]),
    "pc_resample_ladder": (c_int, [c_f64p, c_int, c_int, c_f64p]),
    "pc_pilot_hist": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_int, c_f64p, c_int, c_int, c_int,
                              c_int, c_i64p]),
    "pc_instance_features": (c_int, [c_i32p, c_i8p, c_f64p]),
    "pc_graph_dsatur": (c_int, [c_int, c_i32p, c_i32p, c_i32p, ctypes.POINTER(c_int)]),
    "pc_gapt_load": (c_int, [c_vp, c_int, c_i32p, c_i32p, c_i32p, c_i8p, c_vp, c_vp, c_i32p, c_f64p,
                             c_int, c_u32]),
    "pc_gapt_run": (c_int, [c_vp, c_i64, c_int, c_int]),
    "pc_gapt_set_joint_swap": (c_int, [c_vp, c_int]),
    "pc_gapt_set_target": (c_int, [c_vp, c_int, c_i64]),
    "pc_gapt_get_energies": (c_int, [c_vp, c_int, c_i64p]),
    "pc_gapt_get_spins": (c_int, [c_vp, c_int, c_i8p]),
    "pc_gapt_get_colours": (c_int, [c_vp, c_int, c_i32p]),
    "pc_gapt_get_best": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i32p, c_i64p, c_i8p]),
    "pc_gapt_get_stats": (c_int, [c_vp, c_int, c_i64p, c_i64p, c_i64p]),
    "pc_graph_adaptive_ladder": (c_int, [c_vp, c_int, c_i32p, c_i32p, c_i32p, c_i8p, c_vp, c_vp, c_u32, c_dbl,
                                         c_dbl, c_int, c_int, c_int, c_dbl, c_int, c_f64p, c_f64p, c_i32p,
                                         c_i32p]),
    "pc_gsqa_anneal": (c_int, [c_vp, c_int, c_i32p, c_i32p, c_i8p, c_vp, c_vp, c_int, c_dbl, c_int, c_f64p,
                               c_int, c_u32, c_i64p, c_vp]),
    "pc_mlp_create": (c_int, [c_vp, ctypes.POINTER(c_vp), c_f32pp, c_f32pp, c_flt]),
    "pc_mlp_destroy": (None, [c_vp]),
    "pc_mlp_forward": (c_int, [c_vp, c_int, c_f32p, c_f32p]),
    "pc_mlp_grads": (c_int, [c_vp, c_int, c_f32p, c_f32p, c_f32p, c_f32pp, c_f32pp]),
    "pc_mlp_train_step": (c_int, [c_vp, c_int, c_f32p, c_f32p, c_flt, c_f32p]),
    "pc_mlp_train_step_dev": (c_int, [c_vp, c_int, c_vp, c_vp, c_flt, c_vp]),
    "pc_mlp_get_params": (c_int, [c_vp, c_f32pp, c_f32pp]),
    "pc_mlp_set_gap_weight": (c_int, [c_vp, c_flt]),
    "pc_mlp_save": (c_int, [c_vp, ctypes.c_char_p]),
    "pc_mlp_load": (c_int, [c_vp, ctypes.c_char_p, ctypes.POINTER(c_vp)]),
    "pc_ladder_judge": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_int, c_f64p, c_int, c_int, c_dbl, c_f64p,
                                c_i32p]),
    "pc_learned_features": (c_int, [c_vp, c_int, c_i32p, c_i8p, c_u32, c_vp, c_f32p]),
    "pc_learned_ladder": (c_int, [c_vp, c_vp, c_int, c_i32p, c_i8p, c_u32, c_vp, c_f64p, c_f64p, c_i32p,
                                  c_f64p]),
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


def pc_sqa_setup_bc(ctx, dims, periodic, J, P: int, T: float, gamma, present=None) -> None:
    """pc_sqa_setup with per-axis boundary conditions (periodic [3], nonzero = periodic)
    and an optional vacancy mask (present [N], 0 = vacancy)."""
    d, j = _dims(dims), _J(J)
    per = None if periodic is None else np.ascontiguousarray(np.asarray(periodic, np.uint8).reshape(3))
    pres = None if present is None else np.ascontiguousarray(np.asarray(present, np.uint8).ravel())
    g = np.ascontiguousarray(np.asarray(gamma, np.float64))
    _call("pc_sqa_setup_bc", ctx, ptr(d, ctypes.c_int32), None if per is None else per.ctypes.data,
          None if pres is None else pres.ctypes.data, ptr(j, ctypes.c_int8), P, T, len(g),
          ptr(g, ctypes.c_double))


def pc_sqa_upload_bytes(N: int, n_sweeps: int) -> int:
    return int(lib().pc_sqa_upload_bytes(N, n_sweeps))


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


def pc_sqa_run_corr_dev(ctx, R: int, run0: int, E_dev_ptr: int, corr_dev_ptr: int,
                        best_dev_ptr: int = 0) -> None:
    """pc_sqa_run_dev plus corr [R][P] int32 = sum_s s(s,0) s(s,k) (Fig. S17's N C_k)."""
    _call("pc_sqa_run_corr_dev", ctx, R, c_u32(run0), c_vp(E_dev_ptr), c_vp(best_dev_ptr or None),
          c_vp(corr_dev_ptr))


def pc_sqa_selftest_wait(ctx) -> int:
    st = c_int()
    _call("pc_sqa_selftest_wait", ctx, ctypes.byref(st))
    return st.value


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


def _concat_J(J_list):
    return np.ascontiguousarray(np.concatenate([np.asarray(j, np.int8).reshape(-1, 3) for j in J_list]))


def pc_apt_load(ctx, dims, J_list, betas_list, n_labels: int = 2, entry0: int = 0) -> None:
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(-1, 3))
    J = _concat_J(J_list)
    nt = np.ascontiguousarray([len(b) for b in betas_list], dtype=np.int32)
    be = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64) for b in betas_list]))
    _call("pc_apt_load", ctx, len(J_list), ptr(d, ctypes.c_int32), ptr(J, ctypes.c_int8),
          ptr(nt, ctypes.c_int32), ptr(be, ctypes.c_double), n_labels, c_u32(entry0))


def pc_apt_load_bc(ctx, dims, periodic, J_list, betas_list, n_labels: int = 2, entry0: int = 0,
                   present_list=None) -> None:
    """pc_apt_load with per-axis boundary conditions (periodic [n][3], nonzero =
    periodic) and optional vacancy masks (present_list: per instance [N], 0 = vacancy)."""
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(-1, 3))
    per = None if periodic is None else np.ascontiguousarray(np.asarray(periodic, np.uint8).reshape(-1, 3))
    pres = None if present_list is None else np.ascontiguousarray(
        np.concatenate([np.asarray(p, np.uint8).ravel() for p in present_list]))
    J = _concat_J(J_list)
    nt = np.ascontiguousarray([len(b) for b in betas_list], dtype=np.int32)
    be = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64) for b in betas_list]))
    _call("pc_apt_load_bc", ctx, len(J_list), ptr(d, ctypes.c_int32), None if per is None else per.ctypes.data,
          None if pres is None else pres.ctypes.data, ptr(J, ctypes.c_int8), ptr(nt, ctypes.c_int32),
          ptr(be, ctypes.c_double), n_labels, c_u32(entry0))


def pc_apt_set_joint_swap(ctx, joint: bool) -> None:
    _call("pc_apt_set_joint_swap", ctx, int(bool(joint)))


def pc_apt_set_icm_rules(ctx, big_cluster_rule: bool = True, cluster_seed: bool = False) -> None:
    _call("pc_apt_set_icm_rules", ctx, int(bool(big_cluster_rule)), int(bool(cluster_seed)))


def pc_apt_set_split(ctx, pref: int) -> None:
    """0: split when needed or when the batch is small; 1: only when needed; 2: whenever possible;
    3: problem by problem, those that need it or whose work exceeds the mean per SM."""
    _call("pc_apt_set_split", ctx, int(pref))


def pc_apt_is_split(ctx) -> int:
    """0: one CTA per problem, 1: every problem a two-CTA cluster, 2: some."""
    v = c_int()
    _call("pc_apt_is_split", ctx, ctypes.byref(v))
    return v.value


def pc_apt_run(ctx, n_swaps: int, sweeps_per_swap: int = 1, icm: bool = True) -> None:
    _call("pc_apt_run", ctx, c_i64(n_swaps), sweeps_per_swap, int(bool(icm)))


def pc_apt_autotune(ctx, trial_swaps: int = 16, icm: bool = True):
    """Returns the chosen (threads per CTA, thread chunks, placement (0: one
    CTA per problem, 1: two-CTA clusters, 2: clusters for some problems),
    split groups)."""
    tpb, nch, split, grp = c_int(), c_int(), c_int(), c_int()
    _call("pc_apt_autotune", ctx, trial_swaps, int(icm), ctypes.byref(tpb), ctypes.byref(nch), ctypes.byref(split),
          ctypes.byref(grp))
    return tpb.value, nch.value, split.value, grp.value


def pc_apt_set_launch(ctx, tpb: int, nch: int = 0, split_pref: int = 0, split_groups: int = 0) -> None:
    _call("pc_apt_set_launch", ctx, tpb, nch, split_pref, split_groups)


def pc_apt_set_block_threads(ctx, tpb: int) -> None:
    _call("pc_apt_set_block_threads", ctx, tpb)


def pc_apt_save(ctx, path: str) -> None:
    _call("pc_apt_save", ctx, os.fsencode(path))


def pc_apt_restore(ctx, path: str) -> None:
    _call("pc_apt_restore", ctx, os.fsencode(path))


def pc_apt_progress(ctx):
    a, b = c_i64(), c_i64()
    _call("pc_apt_progress", ctx, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def pc_apt_set_target(ctx, inst: int, e_target: int) -> None:
    _call("pc_apt_set_target", ctx, inst, c_i64(e_target))


def pc_apt_get_state(ctx, inst: int, N: int, B: int):
    s = np.zeros((B, N), np.int8)
    E = np.zeros(B, np.int64)
    t = np.zeros(B, np.int32)
    _call("pc_apt_get_state", ctx, inst, ptr(s, ctypes.c_int8), ptr(E, ctypes.c_int64),
          ptr(t, ctypes.c_int32))
    return s, E, t


def pc_apt_get_best(ctx, inst: int, N: int):
    E, sw, hit = c_i64(), c_i64(), c_i64()
    b = ctypes.c_int32()
    s = np.zeros(N, np.int8)
    _call("pc_apt_get_best", ctx, inst, ctypes.byref(E), ctypes.byref(sw), ctypes.byref(b),
          ctypes.byref(hit), ptr(s, ctypes.c_int8))
    return dict(E=E.value, sweep=sw.value, buf=b.value, hit_sweep=hit.value, spins=s)


def pc_apt_get_best_all(ctx, n: int):
    E = np.zeros(n, np.int64)
    hit = np.zeros(n, np.int64)
    _call("pc_apt_get_best_all", ctx, ptr(E, ctypes.c_int64), ptr(hit, ctypes.c_int64))
    return E, hit


def pc_apt_get_stats(ctx, inst: int, T: int, A: int):
    att = np.zeros((max(T - 1, 0), A), np.int64)
    acc = np.zeros_like(att)
    icm = np.zeros(3, np.int64)
    _call("pc_apt_get_stats", ctx, inst, ptr(att, ctypes.c_int64), ptr(acc, ctypes.c_int64),
          ptr(icm, ctypes.c_int64))
    return att, acc, icm


def pc_apt_get_pbit_table(ctx, inst: int, T: int) -> np.ndarray:
    out = np.zeros((T, 7), np.uint32)
    _call("pc_apt_get_pbit_table", ctx, inst, ptr(out, ctypes.c_uint32))
    return out


def pc_apt_get_swap_table(ctx, inst: int, pair: int, max_len: int = 1 << 16) -> np.ndarray:
    out = np.zeros(max_len, np.uint32)
    n = c_int()
    _call("pc_apt_get_swap_table", ctx, inst, pair, ptr(out, ctypes.c_uint32), max_len, ctypes.byref(n))
    return out[: min(n.value, max_len)].copy()


def pc_adaptive_ladder(ctx, dims, J_list, entry0=0, beta0=0.5, alpha=1.25, n_chains=100, sweeps=10000,
                       tail=1000, tol=1.0, max_len=64):
    n = len(J_list)
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(n, 3))
    J = _concat_J(J_list)
    beta = np.zeros((n, max_len), np.float64)
    sig = np.zeros((n, max_len), np.float64)
    ln = np.zeros(n, np.int32)
    conv = np.zeros(n, np.int32)
    _call("pc_adaptive_ladder", ctx, n, ptr(d, ctypes.c_int32), ptr(J, ctypes.c_int8), c_u32(entry0),
          beta0, alpha, n_chains, sweeps, tail, tol, max_len, ptr(beta, ctypes.c_double),
          ptr(sig, ctypes.c_double), ptr(ln, ctypes.c_int32), ptr(conv, ctypes.c_int32))
    return [(beta[i, : ln[i]].copy(), sig[i, : ln[i]].copy(), bool(conv[i])) for i in range(n)]


def pc_resample_ladder(beta, n: int = 32) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(beta, np.float64))
    out = np.zeros(n, np.float64)
    _call("pc_resample_ladder", ptr(b, ctypes.c_double), len(b), n, ptr(out, ctypes.c_double))
    return out


def pc_pilot_hist(ctx, dims, J_list, betas, entry0=0, chains_per_beta=8, sweeps=256, burn=128,
                  n_bins=64) -> np.ndarray:
    n = len(J_list)
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(n, 3))
    J = _concat_J(J_list)
    be = np.ascontiguousarray(np.asarray(betas, np.float64))
    out = np.zeros((n, len(be), n_bins), np.int64)
    _call("pc_pilot_hist", ctx, n, ptr(d, ctypes.c_int32), ptr(J, ctypes.c_int8), c_u32(entry0), len(be),
          ptr(be, ctypes.c_double), chains_per_beta, sweeps, burn, n_bins, ptr(out, ctypes.c_int64))
    return out


def pc_instance_features(dims, J) -> np.ndarray:
    d = _dims(dims)
    j = _J(J)
    out = np.zeros(3, np.float64)
    _call("pc_instance_features", ptr(d, ctypes.c_int32), ptr(j, ctypes.c_int8), ptr(out, ctypes.c_double))
    return out


def pc_ladder_judge(ctx, dims, J_list, betas, entry0=0, n_labels=2, probe_attempts=500, acc_floor=0.0271):
    """Swap-acceptance judge of ladders [n][T]: (acceptance [n][T-1], pass [n])."""
    n = len(J_list)
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(n, 3))
    J = _concat_J(J_list)
    b = np.ascontiguousarray(np.asarray(betas, np.float64).reshape(n, -1))
    T = b.shape[1]
    acc = np.zeros((n, T - 1), np.float64)
    ok = np.zeros(n, np.int32)
    _call("pc_ladder_judge", ctx, n, ptr(d, ctypes.c_int32), ptr(J, ctypes.c_int8), c_u32(entry0), T,
          ptr(b, ctypes.c_double), n_labels, probe_attempts, acc_floor, ptr(acc, ctypes.c_double),
          ptr(ok, ctypes.c_int32))
    return acc, ok.astype(bool)


class LearnedOpts(ctypes.Structure):
    """pc_learned_opts."""
    _fields_ = [("pilot_betas", c_f64p), ("pilot_chains", c_int), ("pilot_sweeps", c_int),
                ("pilot_burn", c_int), ("probe_attempts", c_int), ("probe_labels", c_int),
                ("acc_floor", c_dbl), ("beta0", c_dbl), ("alpha", c_dbl), ("n_chains", c_int),
                ("sweeps", c_int), ("tail", c_int), ("tol", c_dbl), ("max_len", c_int)]


def _learned_opts(pb, pilot_chains, pilot_sweeps, pilot_burn, probe_attempts=0, probe_labels=2, acc_floor=0.0,
                  beta0=0.5, alpha=1.25, n_chains=32, sweeps=2000, tail=500, tol=1.0, max_len=64):
    return LearnedOpts(ptr(pb, ctypes.c_double), pilot_chains, pilot_sweeps, pilot_burn, probe_attempts,
                       probe_labels, acc_floor, beta0, alpha, n_chains, sweeps, tail, tol, max_len)


def _pilot_betas(pilot_betas) -> np.ndarray:
    pb = np.ascontiguousarray(np.asarray(pilot_betas, np.float64))
    if pb.shape != (4,):
        raise ValueError("pilot_betas must hold 4 temperatures")
    return pb


def pc_learned_features(ctx, dims, J_list, pilot_betas, entry0=0, pilot_chains=8, pilot_sweeps=256,
                        pilot_burn=128) -> np.ndarray:
    """The network's inputs [n][259] (pc_learned_features)."""
    n = len(J_list)
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(n, 3))
    J = _concat_J(J_list)
    pb = _pilot_betas(pilot_betas)
    o = _learned_opts(pb, pilot_chains, pilot_sweeps, pilot_burn)
    X = np.zeros((n, MLP_SIZES[0]), np.float32)
    _call("pc_learned_features", ctx, n, ptr(d, ctypes.c_int32), ptr(J, ctypes.c_int8), c_u32(entry0),
          ctypes.byref(o), ptr(X, ctypes.c_float))
    return X


def pc_learned_ladder(ctx, mlp, dims, J_list, pilot_betas, entry0=0, pilot_chains=8, pilot_sweeps=256,
                      pilot_burn=128, probe_attempts=500, probe_labels=2, acc_floor=0.0271, beta0=0.5,
                      alpha=1.25, n_chains=32, sweeps=2000, tail=500, tol=1.0, max_len=64, with_ready=False):
    """Learned ladders [n][32] with the judge's acceptances [n][31] and the
    fallback flags [n] (pc_learned_ladder); with_ready adds each instance's
    ready time [n] in seconds."""
    n = len(J_list)
    d = np.ascontiguousarray(np.asarray(dims, np.int32).reshape(n, 3))
    J = _concat_J(J_list)
    pb = _pilot_betas(pilot_betas)
    o = _learned_opts(pb, pilot_chains, pilot_sweeps, pilot_burn, probe_attempts, probe_labels, acc_floor,
                      beta0, alpha, n_chains, sweeps, tail, tol, max_len)
    beta = np.zeros((n, 32), np.float64)
    acc = np.zeros((n, 31), np.float64)
    fb = np.zeros(n, np.int32)
    ready = np.zeros(n, np.float64)
    _call("pc_learned_ladder", ctx, mlp.h if isinstance(mlp, Mlp) else mlp, n, ptr(d, ctypes.c_int32),
          ptr(J, ctypes.c_int8), c_u32(entry0), ctypes.byref(o), ptr(beta, ctypes.c_double),
          ptr(acc, ctypes.c_double), ptr(fb, ctypes.c_int32), ptr(ready, ctypes.c_double))
    if with_ready:
        return beta, acc, fb.astype(bool), ready
    return beta, acc, fb.astype(bool)


MLP_SIZES = (259, 256, 256, 256, 32)


def _fpp(arrs):
    arr_t = c_f32p * len(arrs)
    return arr_t(*[a.ctypes.data_as(c_f32p) for a in arrs])


class Mlp:
    """The ladder predictor on the GPU (pc_mlp_*): params [(W [out,in], b [out])] x 4."""

    def __init__(self, ctx, params=None, beta_min: float = 0.0, path: Optional[str] = None):
        # ctx: a Context (kept alive as long as the network) or a raw handle
        self._owner = ctx if isinstance(ctx, Context) else None
        ctx = ctx.h if isinstance(ctx, Context) else ctx
        self.ctx = ctx
        h = c_vp()
        if path is not None:
            _call("pc_mlp_load", ctx, os.fsencode(path), ctypes.byref(h))
        else:
            Ws = [np.ascontiguousarray(W, np.float32) for W, _ in params]
            bs = [np.ascontiguousarray(b, np.float32) for _, b in params]
            _call("pc_mlp_create", ctx, ctypes.byref(h), _fpp(Ws), _fpp(bs), c_flt(beta_min))
        self.h = h

    def save(self, path: str) -> None:
        _call("pc_mlp_save", self.h, os.fsencode(path))

    def set_gap_weight(self, w: float) -> None:
        _call("pc_mlp_set_gap_weight", self.h, c_flt(w))

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().pc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros((X.shape[0], MLP_SIZES[-1]), np.float32)
        _call("pc_mlp_forward", self.h, X.shape[0], ptr(X, ctypes.c_float), ptr(out, ctypes.c_float))
        return out

    def _bufs(self):
        Ws = [np.zeros((o, i), np.float32) for i, o in zip(MLP_SIZES[:-1], MLP_SIZES[1:])]
        bs = [np.zeros(o, np.float32) for o in MLP_SIZES[1:]]
        return Ws, bs

    def grads(self, X, Y):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        Ws, bs = self._bufs()
        loss = c_flt()
        _call("pc_mlp_grads", self.h, X.shape[0], ptr(X, ctypes.c_float), ptr(Y, ctypes.c_float),
              ctypes.byref(loss), _fpp(Ws), _fpp(bs))
        return loss.value, list(zip(Ws, bs))

    def train_step(self, X, Y, lr: float = 1e-3) -> float:
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        loss = c_flt()
        _call("pc_mlp_train_step", self.h, X.shape[0], ptr(X, ctypes.c_float), ptr(Y, ctypes.c_float),
              c_flt(lr), ctypes.byref(loss))
        return loss.value

    def train_step_dev(self, batch: int, X_ptr: int, Y_ptr: int, lr: float, loss_ptr: int = 0) -> None:
        _call("pc_mlp_train_step_dev", self.h, batch, c_vp(X_ptr), c_vp(Y_ptr), c_flt(lr),
              c_vp(loss_ptr or None))

    def params(self):
        Ws, bs = self._bufs()
        _call("pc_mlp_get_params", self.h, _fpp(Ws), _fpp(bs))
        return list(zip(Ws, bs))


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


# ---------------------------------------------------------------- general graphs
def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).ravel())


def _i8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int8).ravel())


def pc_graph_dsatur(row_ptr, col):
    """DSATUR colouring of a CSR graph: (colour [n], number of colours)."""
    rp, cl = _i32(row_ptr), _i32(col)
    n = len(rp) - 1
    out = np.zeros(n, np.int32)
    C = c_int(0)
    _call("pc_graph_dsatur", n, ptr(rp, ctypes.c_int32), ptr(cl, ctypes.c_int32), ptr(out, ctypes.c_int32),
          ctypes.byref(C))
    return out, C.value


def pc_gapt_load(ctx, graphs, betas_list, n_labels: int = 2, entry0: int = 0, h_list=None,
                 colours=None) -> None:
    """graphs: list of (row_ptr, col, w) CSR triples; h_list / colours: per
    problem arrays or None (no biases / DSATUR colouring)."""
    nv = np.ascontiguousarray([len(g[0]) - 1 for g in graphs], dtype=np.int32)
    rp = np.ascontiguousarray(np.concatenate([_i32(g[0]) for g in graphs]))
    cl = np.ascontiguousarray(np.concatenate([_i32(g[1]) for g in graphs]))
    w = np.ascontiguousarray(np.concatenate([_i8(g[2]) for g in graphs]))
    h = None if h_list is None else np.ascontiguousarray(np.concatenate([_i8(x) for x in h_list]))
    co = None if colours is None else np.ascontiguousarray(np.concatenate([_i32(x) for x in colours]))
    nt = np.ascontiguousarray([len(b) for b in betas_list], dtype=np.int32)
    be = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64) for b in betas_list]))
    _call("pc_gapt_load", ctx, len(graphs), ptr(nv, ctypes.c_int32), ptr(rp, ctypes.c_int32),
          ptr(cl, ctypes.c_int32), ptr(w, ctypes.c_int8), None if h is None else h.ctypes.data,
          None if co is None else co.ctypes.data, ptr(nt, ctypes.c_int32), ptr(be, ctypes.c_double),
          n_labels, c_u32(entry0))


def pc_gapt_run(ctx, n_swaps: int, sweeps_per_swap: int = 1, icm: bool = True) -> None:
    _call("pc_gapt_run", ctx, c_i64(n_swaps), sweeps_per_swap, int(bool(icm)))


def pc_gapt_set_joint_swap(ctx, joint: bool) -> None:
    _call("pc_gapt_set_joint_swap", ctx, int(bool(joint)))


def pc_gapt_set_target(ctx, prob: int, e_target: int) -> None:
    _call("pc_gapt_set_target", ctx, prob, c_i64(e_target))


def pc_gapt_get_energies(ctx, prob: int, T: int, A: int) -> np.ndarray:
    E = np.zeros(T * A, np.int64)
    _call("pc_gapt_get_energies", ctx, prob, ptr(E, ctypes.c_int64))
    return E


def pc_gapt_get_spins(ctx, prob: int, T: int, A: int, n: int) -> np.ndarray:
    s = np.zeros((T * A, n), np.int8)
    _call("pc_gapt_get_spins", ctx, prob, ptr(s, ctypes.c_int8))
    return s


def pc_gapt_get_colours(ctx, prob: int, n: int) -> np.ndarray:
    c = np.zeros(n, np.int32)
    _call("pc_gapt_get_colours", ctx, prob, ptr(c, ctypes.c_int32))
    return c


def pc_gapt_get_best(ctx, prob: int, n: int):
    E, sw, hit = c_i64(), c_i64(), c_i64()
    b = ctypes.c_int32()
    s = np.zeros(n, np.int8)
    _call("pc_gapt_get_best", ctx, prob, ctypes.byref(E), ctypes.byref(sw), ctypes.byref(b),
          ctypes.byref(hit), ptr(s, ctypes.c_int8))
    return dict(E=E.value, sweep=sw.value, buf=b.value, hit_sweep=hit.value, spins=s)


def pc_gapt_get_stats(ctx, prob: int, T: int, A: int):
    att = np.zeros((max(T - 1, 0), A), np.int64)
    acc = np.zeros_like(att)
    icm = np.zeros(3, np.int64)
    _call("pc_gapt_get_stats", ctx, prob, ptr(att, ctypes.c_int64), ptr(acc, ctypes.c_int64),
          ptr(icm, ctypes.c_int64))
    return att, acc, icm


def pc_gsqa_anneal(ctx, row_ptr, col, w, P: int, T: float, gamma, R: int, run0: int = 0, h=None,
                   colour=None, want_spins: bool = False):
    """DT-SQA on a graph: slice energies [R][P] (and spins [R][P][n])."""
    rp, cl, ww = _i32(row_ptr), _i32(col), _i8(w)
    hh = None if h is None else _i8(h)
    co = None if colour is None else _i32(colour)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    n = len(rp) - 1
    E = np.zeros((R, P), np.int64)
    s = np.zeros((R, P, n), np.int8) if want_spins else None
    _call("pc_gsqa_anneal", ctx, n, ptr(rp, ctypes.c_int32), ptr(cl, ctypes.c_int32), ptr(ww, ctypes.c_int8),
          None if hh is None else hh.ctypes.data, None if co is None else co.ctypes.data, P, T, len(g),
          ptr(g, ctypes.c_double), R, c_u32(run0), ptr(E, ctypes.c_int64),
          None if s is None else s.ctypes.data)
    return (E, s) if want_spins else E


def pc_graph_adaptive_ladder(ctx, graphs, entry0: int = 0, beta0: float = 0.5, alpha: float = 1.25,
                             n_chains: int = 100, sweeps: int = 10000, tail: int = 1000, tol: float = 1.0,
                             max_len: int = 64, h_list=None, colours=None):
    """Adaptive ladders of graphs [(row_ptr, col, w)]: list of (betas, sigmas, converged)."""
    nv = np.ascontiguousarray([len(g[0]) - 1 for g in graphs], dtype=np.int32)
    rp = np.ascontiguousarray(np.concatenate([_i32(g[0]) for g in graphs]))
    cl = np.ascontiguousarray(np.concatenate([_i32(g[1]) for g in graphs]))
    w = np.ascontiguousarray(np.concatenate([_i8(g[2]) for g in graphs]))
    h = None if h_list is None else np.ascontiguousarray(np.concatenate([_i8(x) for x in h_list]))
    co = None if colours is None else np.ascontiguousarray(np.concatenate([_i32(x) for x in colours]))
    n = len(graphs)
    beta = np.zeros((n, max_len), np.float64)
    sig = np.zeros((n, max_len), np.float64)
    ln = np.zeros(n, np.int32)
    conv = np.zeros(n, np.int32)
    _call("pc_graph_adaptive_ladder", ctx, n, ptr(nv, ctypes.c_int32), ptr(rp, ctypes.c_int32),
          ptr(cl, ctypes.c_int32), ptr(w, ctypes.c_int8), None if h is None else h.ctypes.data,
          None if co is None else co.ctypes.data, c_u32(entry0), beta0, alpha, n_chains, sweeps, tail, tol,
          max_len, ptr(beta, ctypes.c_double), ptr(sig, ctypes.c_double), ptr(ln, ctypes.c_int32),
          ptr(conv, ctypes.c_int32))
    return [(beta[i, :ln[i]].copy(), sig[i, :ln[i]].copy(), bool(conv[i])) for i in range(n)]
