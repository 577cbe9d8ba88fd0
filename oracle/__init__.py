"""CPU oracle for the p-bit Monte Carlo of arXiv 2503.10302 (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The C sources next to this file are a
plain restatement of the paper's method; they share no code with the CUDA
library.  ``build()`` compiles them with gcc into ``liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = ["core.c", "apt.c", "sqa.c", "graph.c"]

TAG_APT_INIT, TAG_APT_SWEEP, TAG_APT_REFINE, TAG_SWAP, TAG_ICM = 1, 2, 3, 4, 5
TAG_LAD_INIT, TAG_LAD_SWEEP, TAG_LAD_REFINE = 6, 7, 8
TAG_PIL_INIT, TAG_PIL_SWEEP, TAG_PIL_REFINE = 9, 10, 11
TAG_SQA_INIT, TAG_SQA_SWEEP, TAG_SQA_REFINE = 12, 13, 14


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, "oracle.h"), os.path.join(_HERE, "oracle_internal.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        u32p, u64, i64p = P(ctypes.c_uint32), ctypes.c_uint64, P(ctypes.c_int64)
        i32p, i8p, u8p, f64p = P(ctypes.c_int32), P(ctypes.c_int8), P(ctypes.c_uint8), P(ctypes.c_double)
        L.or_philox_many.argtypes = [ctypes.c_int64, u32p, u64, u32p]
        L.or_pbit_threshold.argtypes = [ctypes.c_double, ctypes.c_int64]
        L.or_pbit_threshold.restype = ctypes.c_uint32
        L.or_swap_threshold.argtypes = [ctypes.c_double, ctypes.c_int64]
        L.or_swap_threshold.restype = ctypes.c_uint32
        L.or_jperp_q.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double]
        L.or_jperp_q.restype = ctypes.c_int32
        L.or_sqa_threshold.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int]
        L.or_sqa_threshold.restype = ctypes.c_uint32
        L.or_energy.argtypes = [i32p, u8p, u8p, i8p, i8p, i8p, i64p]
        L.or_apt_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, i32p, u8p, u8p, i8p, i8p, i32p,
                                    f64p, ctypes.c_int, u64, ctypes.c_uint32]
        L.or_apt_destroy.argtypes = [ctypes.c_void_p]
        L.or_apt_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_apt_set_target.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
        L.or_apt_set_joint_swap.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_apt_set_icm_rules.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.or_icm_apply_rules.argtypes = [i32p, u8p, i8p, i8p, u64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, i64p]
        L.or_icm_choice.argtypes = [i32p, u8p, i8p, i8p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, i64p, i64p]
        L.or_apt_state.argtypes = [ctypes.c_void_p, ctypes.c_int, i8p, i64p, i32p]
        L.or_apt_best.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i64p, i32p, i64p, i8p]
        L.or_apt_stats.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i64p, i64p]
        L.or_apt_sweeps.argtypes = [ctypes.c_void_p]
        L.or_apt_sweeps.restype = ctypes.c_int64
        L.or_icm_apply.argtypes = [i32p, u8p, i8p, i8p, u64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint32, i64p]
        L.or_icm_pairing.argtypes = [u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                     i32p]
        L.or_adaptive_ladder.argtypes = [i32p, u8p, i8p, i8p, ctypes.c_uint32, u64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, f64p, f64p, P(ctypes.c_int)]
        L.or_pilot_hist.argtypes = [i32p, u8p, i8p, i8p, ctypes.c_uint32, u64, ctypes.c_int, f64p,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p]
        L.or_sqa_anneal.argtypes = [i32p, u8p, u8p, i8p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    f64p, ctypes.c_int, ctypes.c_uint32, u64, i64p, i8p, ctypes.c_int]
        L.or_graph_check.argtypes = [ctypes.c_int, i32p, i32p, i8p]
        L.or_dsatur.argtypes = [ctypes.c_int, i32p, i32p, i32p, P(ctypes.c_int)]
        L.or_graph_sqa_colouring.argtypes = [ctypes.c_int, i32p, ctypes.c_int, i32p, P(ctypes.c_int)]
        L.or_graph_energy.argtypes = [ctypes.c_int, i32p, i32p, i8p, i8p, i8p, i64p]
        L.or_gapt_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, i32p, i32p, i32p, i8p, i8p, i32p,
                                     i32p, f64p, ctypes.c_int, u64, ctypes.c_uint32]
        L.or_gapt_destroy.argtypes = [ctypes.c_void_p]
        L.or_gapt_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_gapt_set_joint_swap.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_gapt_set_target.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
        L.or_gapt_state.argtypes = [ctypes.c_void_p, ctypes.c_int, i8p, i64p, i32p]
        L.or_gapt_best.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i64p, i32p, i64p, i8p]
        L.or_gapt_stats.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i64p, i64p]
        L.or_graph_adaptive_ladder.argtypes = [ctypes.c_int, i32p, i32p, i8p, i8p, i32p, ctypes.c_uint32, u64,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_int, f64p, f64p,
                                               P(ctypes.c_int)]
        L.or_gicm_apply.argtypes = [ctypes.c_int, i32p, i32p, i32p, i8p, i8p, u64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, i64p]
        L.or_gsqa_anneal.argtypes = [ctypes.c_int, i32p, i32p, i8p, i8p, i32p, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, f64p, ctypes.c_int, ctypes.c_uint32, u64, i64p, i8p,
                                     ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise ValueError(f"oracle {what} failed with status {rc}")
    return rc


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(3))


def _per(periodic) -> np.ndarray:
    if periodic is None:
        periodic = (1, 1, 1)
    return np.ascontiguousarray(np.asarray(periodic, dtype=np.uint8).reshape(3))


def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    out = np.zeros_like(ctr)
    lib().or_philox_many(ctr.shape[0], _ptr(ctr, ctypes.c_uint32), ctypes.c_uint64(seed),
                         _ptr(out, ctypes.c_uint32))
    return out


def pbit_threshold(beta: float, I: int) -> int:
    return int(lib().or_pbit_threshold(beta, I))


def swap_threshold(dbeta: float, dE: int) -> int:
    return int(lib().or_swap_threshold(dbeta, dE))


def jperp_q(gamma: float, P: int, T: float) -> int:
    return int(lib().or_jperp_q(gamma, P, T))


def sqa_threshold(beta_eff: float, I: int, jq: int, n: int) -> int:
    return int(lib().or_sqa_threshold(beta_eff, I, jq, n))


def _present(present) -> Optional[np.ndarray]:
    return None if present is None else np.ascontiguousarray(np.asarray(present, dtype=np.uint8).ravel())


def energy(dims, J, spins, h=None, periodic=None, present=None) -> int:
    d, p = _dims(dims), _per(periodic)
    pr = _present(present)
    J = np.ascontiguousarray(J, dtype=np.int8)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int8)
    out = np.zeros(1, dtype=np.int64)
    _check(lib().or_energy(_ptr(d, ctypes.c_int32), _ptr(p, ctypes.c_uint8), _ptr(pr, ctypes.c_uint8),
                           _ptr(J, ctypes.c_int8),
                           _ptr(hh, ctypes.c_int8), _ptr(s, ctypes.c_int8), _ptr(out, ctypes.c_int64)),
           "energy")
    return int(out[0])


class Apt:
    """Batch of APT problems advanced in lockstep (Algorithm S2)."""

    def __init__(self, dims, J_list, betas_list, n_labels=2, seed=0, entry0=0,
                 h_list=None, periodic=None, present_list=None):
        n = len(J_list)
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(n, 3))
        self.N = [int(np.prod(d)) for d in self.dims]
        self.n_temps = np.ascontiguousarray([len(b) for b in betas_list], dtype=np.int32)
        self.n_labels = n_labels
        J = np.ascontiguousarray(np.concatenate([np.asarray(j, np.int8).reshape(-1, 3) for j in J_list]))
        betas = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64) for b in betas_list]))
        per = None if periodic is None else np.ascontiguousarray(
            np.asarray(periodic, dtype=np.uint8).reshape(n, 3))
        h = None if h_list is None else np.ascontiguousarray(
            np.concatenate([np.asarray(x, np.int8) for x in h_list]))
        pres = None if present_list is None else np.ascontiguousarray(
            np.concatenate([np.asarray(x, np.uint8).ravel() for x in present_list]))
        self._keep = (J, betas, per, h, pres)
        handle = ctypes.c_void_p()
        _check(lib().or_apt_create(ctypes.byref(handle), n, _ptr(self.dims, ctypes.c_int32),
                                   _ptr(per, ctypes.c_uint8), _ptr(pres, ctypes.c_uint8), _ptr(J, ctypes.c_int8),
                                   _ptr(h, ctypes.c_int8), _ptr(self.n_temps, ctypes.c_int32),
                                   _ptr(betas, ctypes.c_double), n_labels, ctypes.c_uint64(seed),
                                   ctypes.c_uint32(entry0)), "apt_create")
        self.h = handle
        self.n = n

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.or_apt_destroy(self.h)
            self.h = None

    def run(self, n_swaps: int, sweeps_per_swap: int = 1, icm: bool = True, threads: int = 0):
        _check(lib().or_apt_run(self.h, n_swaps, sweeps_per_swap, int(icm), threads), "apt_run")

    def set_joint_swap(self, joint: bool):
        _check(lib().or_apt_set_joint_swap(self.h, int(bool(joint))), "set_joint_swap")

    def set_icm_rules(self, big_cluster_rule: bool = True, cluster_seed: bool = False):
        _check(lib().or_apt_set_icm_rules(self.h, int(bool(big_cluster_rule)), int(bool(cluster_seed))),
               "set_icm_rules")

    def set_target(self, inst: int, e_target: int):
        _check(lib().or_apt_set_target(self.h, inst, e_target), "set_target")

    def state(self, inst: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        B = int(self.n_temps[inst]) * self.n_labels
        s = np.zeros((B, self.N[inst]), np.int8)
        E = np.zeros(B, np.int64)
        t = np.zeros(B, np.int32)
        _check(lib().or_apt_state(self.h, inst, _ptr(s, ctypes.c_int8), _ptr(E, ctypes.c_int64),
                                  _ptr(t, ctypes.c_int32)), "state")
        return s, E, t

    def best(self, inst: int):
        E = np.zeros(1, np.int64); sw = np.zeros(1, np.int64); hit = np.zeros(1, np.int64)
        b = np.zeros(1, np.int32); s = np.zeros(self.N[inst], np.int8)
        _check(lib().or_apt_best(self.h, inst, _ptr(E, ctypes.c_int64), _ptr(sw, ctypes.c_int64),
                                 _ptr(b, ctypes.c_int32), _ptr(hit, ctypes.c_int64),
                                 _ptr(s, ctypes.c_int8)), "best")
        return dict(E=int(E[0]), sweep=int(sw[0]), buf=int(b[0]), hit_sweep=int(hit[0]), spins=s)

    def stats(self, inst: int):
        T, A = int(self.n_temps[inst]), self.n_labels
        att = np.zeros((max(T - 1, 0), A), np.int64); acc = np.zeros_like(att)
        icm = np.zeros(3, np.int64)
        _check(lib().or_apt_stats(self.h, inst, _ptr(att, ctypes.c_int64), _ptr(acc, ctypes.c_int64),
                                  _ptr(icm, ctypes.c_int64)), "stats")
        return att, acc, icm

    @property
    def sweeps(self) -> int:
        return int(lib().or_apt_sweeps(self.h))


def icm_apply(dims, sa, sb, seed=0, entry=0, r=0, t=0, p=0, periodic=None):
    """One ICMop on copies of (sa, sb); returns (branch, cluster_size, sa', sb')."""
    d, per = _dims(dims), _per(periodic)
    a = np.ascontiguousarray(sa, dtype=np.int8).copy()
    b = np.ascontiguousarray(sb, dtype=np.int8).copy()
    size = np.zeros(1, np.int64)
    br = _check(lib().or_icm_apply(_ptr(d, ctypes.c_int32), _ptr(per, ctypes.c_uint8),
                                   _ptr(a, ctypes.c_int8), _ptr(b, ctypes.c_int8), ctypes.c_uint64(seed),
                                   ctypes.c_uint32(entry), ctypes.c_uint32(r), ctypes.c_uint32(t),
                                   ctypes.c_uint32(p), _ptr(size, ctypes.c_int64)), "icm_apply")
    return br, int(size[0]), a, b


def icm_apply_rules(dims, sa, sb, seed=0, entry=0, r=0, t=0, p=0, big_cluster_rule=True, cluster_seed=False,
                    periodic=None):
    """One ICMop under the given rules on copies of (sa, sb); returns
    (branch, cluster_size, sa', sb')."""
    d, per = _dims(dims), _per(periodic)
    a = np.ascontiguousarray(sa, dtype=np.int8).copy()
    b = np.ascontiguousarray(sb, dtype=np.int8).copy()
    size = np.zeros(1, np.int64)
    br = _check(lib().or_icm_apply_rules(_ptr(d, ctypes.c_int32), _ptr(per, ctypes.c_uint8),
                                         _ptr(a, ctypes.c_int8), _ptr(b, ctypes.c_int8), ctypes.c_uint64(seed),
                                         ctypes.c_uint32(entry), ctypes.c_uint32(r), ctypes.c_uint32(t),
                                         ctypes.c_uint32(p), int(bool(big_cluster_rule)), int(bool(cluster_seed)),
                                         _ptr(size, ctypes.c_int64)), "icm_apply_rules")
    return br, int(size[0]), a, b


def icm_choice(dims, sa, sb, k, flip_b=False, big_cluster_rule=True, cluster_seed=False, periodic=None):
    """ICMop with its choices given: (branch, n_choices, cluster_size, sa', sb')."""
    d, per = _dims(dims), _per(periodic)
    a = np.ascontiguousarray(sa, dtype=np.int8).copy()
    b = np.ascontiguousarray(sb, dtype=np.int8).copy()
    n = np.zeros(1, np.int64)
    size = np.zeros(1, np.int64)
    br = lib().or_icm_choice(_ptr(d, ctypes.c_int32), _ptr(per, ctypes.c_uint8), _ptr(a, ctypes.c_int8),
                             _ptr(b, ctypes.c_int8), k, int(bool(flip_b)), int(bool(big_cluster_rule)),
                             int(bool(cluster_seed)), _ptr(n, ctypes.c_int64), _ptr(size, ctypes.c_int64))
    if br < 0 and n[0] > 0 and not (0 <= k < n[0]):
        raise ValueError("choice out of range")
    return br, int(n[0]), int(size[0]), a, b


def icm_pairing(seed, entry, r, t, n_labels=4):
    """Matching index and label pairs of the ICM at temperature r, attempt t."""
    q = np.zeros(4, np.int32)
    m = _check(lib().or_icm_pairing(ctypes.c_uint64(seed), ctypes.c_uint32(entry), ctypes.c_uint32(r),
                                    ctypes.c_uint32(t), n_labels, _ptr(q, ctypes.c_int32)), "icm_pairing")
    return m, [int(v) for v in q[: (4 if n_labels == 4 else 2)]]


def adaptive_ladder(dims, J, entry=0, seed=0, beta0=0.5, alpha=1.25, n_chains=100, sweeps=10000,
                    tail=1000, tol=1.0, max_len=64, h=None, periodic=None):
    d, p = _dims(dims), _per(periodic)
    J = np.ascontiguousarray(J, dtype=np.int8)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int8)
    beta = np.zeros(max_len, np.float64); sig = np.zeros(max_len, np.float64)
    n = ctypes.c_int(0)
    rc = _check(lib().or_adaptive_ladder(_ptr(d, ctypes.c_int32), _ptr(p, ctypes.c_uint8),
                                         _ptr(J, ctypes.c_int8), _ptr(hh, ctypes.c_int8),
                                         ctypes.c_uint32(entry), ctypes.c_uint64(seed), beta0, alpha,
                                         n_chains, sweeps, tail, tol, max_len,
                                         _ptr(beta, ctypes.c_double), _ptr(sig, ctypes.c_double),
                                         ctypes.byref(n)), "adaptive_ladder")
    return beta[: n.value].copy(), sig[: n.value].copy(), rc == 0


def pilot_hist(dims, J, betas, entry=0, seed=0, chains_per_beta=8, sweeps=256, burn=128, n_bins=64,
               h=None, periodic=None) -> np.ndarray:
    d, p = _dims(dims), _per(periodic)
    J = np.ascontiguousarray(J, dtype=np.int8)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int8)
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    counts = np.zeros((len(betas), n_bins), np.int64)
    _check(lib().or_pilot_hist(_ptr(d, ctypes.c_int32), _ptr(p, ctypes.c_uint8), _ptr(J, ctypes.c_int8),
                               _ptr(hh, ctypes.c_int8), ctypes.c_uint32(entry), ctypes.c_uint64(seed),
                               len(betas), _ptr(betas, ctypes.c_double), chains_per_beta, sweeps, burn,
                               n_bins, _ptr(counts, ctypes.c_int64)), "pilot_hist")
    return counts


def sqa_anneal(dims, J, P, T, gamma, R, run0=0, seed=0, want_spins=False, threads=0, periodic=None,
               present=None):
    d, p = _dims(dims), _per(periodic)
    pr = _present(present)
    J = np.ascontiguousarray(J, dtype=np.int8)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    N = int(np.prod(d))
    E = np.zeros((R, P), np.int64)
    s = np.zeros((R, P, N), np.int8) if want_spins else None
    _check(lib().or_sqa_anneal(_ptr(d, ctypes.c_int32), _ptr(p, ctypes.c_uint8), _ptr(pr, ctypes.c_uint8),
                               _ptr(J, ctypes.c_int8),
                               P, T, len(gamma), _ptr(gamma, ctypes.c_double), R, ctypes.c_uint32(run0),
                               ctypes.c_uint64(seed), _ptr(E, ctypes.c_int64), _ptr(s, ctypes.c_int8),
                               threads), "sqa_anneal")
    return (E, s) if want_spins else E


# ---------------------------------------------------------------- general graphs
TAG_G_INIT, TAG_G_SWEEP, TAG_G_REFINE, TAG_G_SWAP, TAG_G_ICM = 15, 16, 17, 18, 19
TAG_GS_INIT, TAG_GS_SWEEP, TAG_GS_REFINE = 20, 21, 22
TAG_GL_INIT, TAG_GL_SWEEP, TAG_GL_REFINE = 23, 24, 25


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).ravel())


def _i8(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.int8).ravel())


def graph_check(rp, col, w=None) -> bool:
    rp, col, w = _i32(rp), _i32(col), _i8(w)
    return lib().or_graph_check(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                _ptr(w, ctypes.c_int8)) == 0


def dsatur(rp, col) -> Tuple[np.ndarray, int]:
    """DSATUR colouring of a CSR graph: (colour [n], number of colours)."""
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    out = np.zeros(n, np.int32)
    C = ctypes.c_int(0)
    _check(lib().or_dsatur(n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                           _ptr(out, ctypes.c_int32), ctypes.byref(C)), "dsatur")
    return out, C.value


def graph_sqa_colouring(colour, P: int) -> Tuple[np.ndarray, int]:
    """Colours [P][n] of the replicated DT-SQA network and their count."""
    colour = _i32(colour)
    n = len(colour)
    out = np.zeros((P, n), np.int32)
    C = ctypes.c_int(0)
    _check(lib().or_graph_sqa_colouring(n, _ptr(colour, ctypes.c_int32), P, _ptr(out, ctypes.c_int32),
                                        ctypes.byref(C)), "graph_sqa_colouring")
    return out, C.value


def graph_energy(rp, col, w, spins, h=None) -> int:
    rp, col, w, hh = _i32(rp), _i32(col), _i8(w), _i8(h)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    out = np.zeros(1, np.int64)
    _check(lib().or_graph_energy(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                 _ptr(w, ctypes.c_int8), _ptr(hh, ctypes.c_int8), _ptr(s, ctypes.c_int8),
                                 _ptr(out, ctypes.c_int64)), "graph_energy")
    return int(out[0])


class GApt:
    """Batch of APT problems on general graphs (Algorithm S2 with a colormap).

    graphs: list of (rp, col, w) CSR triples; colours: list of colour arrays or
    None (DSATUR); slot order r * A + a as in :class:`Apt`.
    """

    def __init__(self, graphs, betas_list, n_labels=2, seed=0, entry0=0, h_list=None, colours=None):
        n = len(graphs)
        self.nv = [len(g[0]) - 1 for g in graphs]
        nv = np.ascontiguousarray(self.nv, dtype=np.int32)
        rp = np.ascontiguousarray(np.concatenate([_i32(g[0]) for g in graphs]))
        col = np.ascontiguousarray(np.concatenate([_i32(g[1]) for g in graphs]))
        w = np.ascontiguousarray(np.concatenate([_i8(g[2]) for g in graphs]))
        h = None if h_list is None else np.ascontiguousarray(np.concatenate([_i8(x) for x in h_list]))
        cl = None if colours is None else np.ascontiguousarray(np.concatenate([_i32(c) for c in colours]))
        self.n_temps = np.ascontiguousarray([len(b) for b in betas_list], dtype=np.int32)
        betas = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64) for b in betas_list]))
        self.n_labels = n_labels
        self._keep = (nv, rp, col, w, h, cl, betas)
        handle = ctypes.c_void_p()
        _check(lib().or_gapt_create(ctypes.byref(handle), n, _ptr(nv, ctypes.c_int32), _ptr(rp, ctypes.c_int32),
                                    _ptr(col, ctypes.c_int32), _ptr(w, ctypes.c_int8), _ptr(h, ctypes.c_int8),
                                    _ptr(cl, ctypes.c_int32), _ptr(self.n_temps, ctypes.c_int32),
                                    _ptr(betas, ctypes.c_double), n_labels, ctypes.c_uint64(seed),
                                    ctypes.c_uint32(entry0)), "gapt_create")
        self.h = handle
        self.n = n

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.or_gapt_destroy(self.h)
            self.h = None

    def run(self, n_swaps: int, sweeps_per_swap: int = 1, icm: bool = True, threads: int = 0):
        _check(lib().or_gapt_run(self.h, n_swaps, sweeps_per_swap, int(icm), threads), "gapt_run")

    def set_joint_swap(self, joint: bool):
        _check(lib().or_gapt_set_joint_swap(self.h, int(bool(joint))), "gapt_set_joint_swap")

    def set_target(self, prob: int, e_target: int):
        _check(lib().or_gapt_set_target(self.h, prob, e_target), "gapt_set_target")

    def state(self, prob: int):
        B = int(self.n_temps[prob]) * self.n_labels
        s = np.zeros((B, self.nv[prob]), np.int8)
        E = np.zeros(B, np.int64)
        c = np.zeros(self.nv[prob], np.int32)
        _check(lib().or_gapt_state(self.h, prob, _ptr(s, ctypes.c_int8), _ptr(E, ctypes.c_int64),
                                   _ptr(c, ctypes.c_int32)), "gapt_state")
        return s, E, c

    def best(self, prob: int):
        E = np.zeros(1, np.int64); sw = np.zeros(1, np.int64); hit = np.zeros(1, np.int64)
        b = np.zeros(1, np.int32); s = np.zeros(self.nv[prob], np.int8)
        _check(lib().or_gapt_best(self.h, prob, _ptr(E, ctypes.c_int64), _ptr(sw, ctypes.c_int64),
                                  _ptr(b, ctypes.c_int32), _ptr(hit, ctypes.c_int64),
                                  _ptr(s, ctypes.c_int8)), "gapt_best")
        return dict(E=int(E[0]), sweep=int(sw[0]), buf=int(b[0]), hit_sweep=int(hit[0]), spins=s)

    def stats(self, prob: int):
        T, A = int(self.n_temps[prob]), self.n_labels
        att = np.zeros((max(T - 1, 0), A), np.int64); acc = np.zeros_like(att)
        icm = np.zeros(3, np.int64)
        _check(lib().or_gapt_stats(self.h, prob, _ptr(att, ctypes.c_int64), _ptr(acc, ctypes.c_int64),
                                   _ptr(icm, ctypes.c_int64)), "gapt_stats")
        return att, acc, icm


def gicm_apply(rp, col, colour, sa, sb, seed=0, entry=0, r=0, t=0, p=0):
    """One ICMop on copies of (sa, sb) on a graph; returns (branch, size, sa', sb')."""
    rp, col, colour = _i32(rp), _i32(col), _i32(colour)
    a = np.ascontiguousarray(sa, dtype=np.int8).copy()
    b = np.ascontiguousarray(sb, dtype=np.int8).copy()
    size = np.zeros(1, np.int64)
    br = _check(lib().or_gicm_apply(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                    _ptr(colour, ctypes.c_int32), _ptr(a, ctypes.c_int8), _ptr(b, ctypes.c_int8),
                                    ctypes.c_uint64(seed), ctypes.c_uint32(entry), ctypes.c_uint32(r),
                                    ctypes.c_uint32(t), ctypes.c_uint32(p), _ptr(size, ctypes.c_int64)),
                "gicm_apply")
    return br, int(size[0]), a, b


def gsqa_anneal(rp, col, w, P, T, gamma, R, run0=0, seed=0, h=None, colour=None, want_spins=False,
                threads=0):
    """DT-SQA on a graph: final slice energies [R][P] (and spins [R][P][n])."""
    rp, col, w, hh = _i32(rp), _i32(col), _i8(w), _i8(h)
    cl = None if colour is None else _i32(colour)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    n = len(rp) - 1
    E = np.zeros((R, P), np.int64)
    s = np.zeros((R, P, n), np.int8) if want_spins else None
    _check(lib().or_gsqa_anneal(n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32), _ptr(w, ctypes.c_int8),
                                _ptr(hh, ctypes.c_int8), _ptr(cl, ctypes.c_int32), P, T, len(gamma),
                                _ptr(gamma, ctypes.c_double), R, ctypes.c_uint32(run0), ctypes.c_uint64(seed),
                                _ptr(E, ctypes.c_int64), _ptr(s, ctypes.c_int8), threads), "gsqa_anneal")
    return (E, s) if want_spins else E


def graph_adaptive_ladder(rp, col, w, h=None, colour=None, entry=0, seed=0, beta0=0.5, alpha=1.25,
                          n_chains=100, sweeps=10000, tail=1000, tol=1.0, max_len=64):
    """Adaptive beta ladder on a graph: (betas, sigmas, converged)."""
    rp, col, w, hh = _i32(rp), _i32(col), _i8(w), _i8(h)
    cl = None if colour is None else _i32(colour)
    beta = np.zeros(max_len, np.float64); sig = np.zeros(max_len, np.float64)
    n = ctypes.c_int(0)
    rc = _check(lib().or_graph_adaptive_ladder(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                               _ptr(w, ctypes.c_int8), _ptr(hh, ctypes.c_int8),
                                               _ptr(cl, ctypes.c_int32), ctypes.c_uint32(entry),
                                               ctypes.c_uint64(seed), beta0, alpha, n_chains, sweeps, tail, tol,
                                               max_len, _ptr(beta, ctypes.c_double), _ptr(sig, ctypes.c_double),
                                               ctypes.byref(n)), "graph_adaptive_ladder")
    return beta[: n.value].copy(), sig[: n.value].copy(), rc == 0
