"""ORACLE -- test infrastructure only.

A plain CPU restatement of what the local-max matching path computes, used by
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline and
reference legs, and by nothing else.  It shares no code with the CUDA library and never
imports it.  The arithmetic lives in ``oracle.c`` (plain C, compiled on first
use into ``oracle/_build/``); this module only marshals numpy arrays.

Passages followed (see the header of ``oracle.c`` for each function):
  * the edge order -- Sec. 1 (local max, random-perturbation tie breaking),
    read as (float32 weight, seeded bijective permutation of the edge index);
  * ``greedy``        -- Sec. 3, the greedy algorithm (the oracle for mate[]);
  * ``seq_local_max`` -- Sec. 2, sequential model, three passes per iteration;
  * ``brute_mwm``     -- exact maximum weight matching for small n, used for
    the 1/2-approximation property (Sec. 1);
  * ``contract``      -- contraction of a matching into the coarser graph, the
    multilevel step that motivates the matching (Sec. 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NIL = 0xFFFFFFFF
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build() -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (rebuilt when the source is newer)."""
    src = os.path.join(_HERE, "oracle.c")
    out = os.path.join(_BUILD, "liboracle.so")
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-o", tmp, src])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            f32p = ctypes.POINTER(ctypes.c_float)
            lib.lmo_ord.restype = ctypes.c_uint32
            lib.lmo_ord.argtypes = [ctypes.c_float]
            lib.lmo_fmix32.restype = ctypes.c_uint32
            lib.lmo_fmix32.argtypes = [ctypes.c_uint32]
            lib.lmo_splitmix64.restype = ctypes.c_uint64
            lib.lmo_splitmix64.argtypes = [ctypes.c_uint64]
            lib.lmo_perm.restype = ctypes.c_uint32
            lib.lmo_perm.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            lib.lmo_perm_inv.restype = ctypes.c_uint32
            lib.lmo_perm_inv.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            lib.lmo_key.restype = ctypes.c_uint64
            lib.lmo_key.argtypes = [ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32]
            lib.lmo_keys.restype = None
            lib.lmo_keys.argtypes = [ctypes.c_uint64, f32p, ctypes.c_uint64, u64p]
            lib.lmo_greedy.restype = ctypes.c_int64
            lib.lmo_greedy.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, f32p,
                                       ctypes.c_uint64, u32p]
            lib.lmo_seq_local_max.restype = ctypes.c_int64
            lib.lmo_seq_local_max.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, f32p,
                                              ctypes.c_uint64, u32p, u64p, u64p, ctypes.c_uint64]
            lib.lmo_seq_local_max_renew.restype = ctypes.c_int64
            lib.lmo_seq_local_max_renew.argtypes = lib.lmo_seq_local_max.argtypes
            lib.lmo_brute_mwm.restype = ctypes.c_double
            lib.lmo_brute_mwm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, f32p]
            lib.lmo_contract.restype = ctypes.c_int
            lib.lmo_contract.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, f32p, u32p, u32p,
                                         u32p, u32p, u32p, u32p, f32p, u32p, u64p]
            _LIB = lib
    return _LIB


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _seed(s: int) -> int:
    return int(s) & (2**64 - 1)


def ord32(w: float) -> int:
    return int(_lib().lmo_ord(float(np.float32(w))))


def splitmix64(state: int) -> int:
    return int(_lib().lmo_splitmix64(_seed(state)))


def fmix32(h: int) -> int:
    return int(_lib().lmo_fmix32(h & 0xFFFFFFFF))


def perm(seed: int, e: int) -> int:
    return int(_lib().lmo_perm(_seed(seed), e & 0xFFFFFFFF))


def perm_inv(seed: int, x: int) -> int:
    return int(_lib().lmo_perm_inv(_seed(seed), x & 0xFFFFFFFF))


def key(w: float, seed: int, e: int) -> int:
    return int(_lib().lmo_key(float(np.float32(w)), _seed(seed), e & 0xFFFFFFFF))


def keys(w, seed: int) -> np.ndarray:
    w, wp = _f32(w)
    out = np.empty(w.shape[0], dtype=np.uint64)
    if w.shape[0]:
        _lib().lmo_keys(w.shape[0], wp, _seed(seed), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def greedy(n: int, eu, ev, w, seed: int) -> np.ndarray:
    """mate[] of the greedy matching under the order K(e) (Sec. 3)."""
    eu, up = _u32(eu)
    ev, vp = _u32(ev)
    w, wp = _f32(w)
    mate = np.empty(max(n, 1), dtype=np.uint32)
    r = _lib().lmo_greedy(n, eu.shape[0], up, vp, wp, _seed(seed),
                          mate.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if r < 0:
        raise MemoryError("oracle greedy: allocation failed")
    return mate[:n]


def seq_local_max(n: int, eu, ev, w, seed: int, max_rounds: int = 1 << 16, renew: bool = False):
    """(mate[], rounds, round_m[], round_n[]) of the sequential local max (Sec. 2); with
    renew=True the perturbation is renewed in every iteration (the footnote to Lemma 1)."""
    eu, up = _u32(eu)
    ev, vp = _u32(ev)
    w, wp = _f32(w)
    mate = np.empty(max(n, 1), dtype=np.uint32)
    rm = np.zeros(max_rounds, dtype=np.uint64)
    rn = np.zeros(max_rounds, dtype=np.uint64)
    fn = _lib().lmo_seq_local_max_renew if renew else _lib().lmo_seq_local_max
    r = fn(n, eu.shape[0], up, vp, wp, _seed(seed),
                                 mate.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 rm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 rn.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), max_rounds)
    if r < 0:
        raise MemoryError("oracle seq_local_max: allocation failed")
    k = min(int(r), max_rounds)
    return mate[:n], int(r), rm[:k].copy(), rn[:k].copy()


def brute_mwm(n: int, eu, ev, w) -> float:
    """Exact maximum matching weight (n <= 22)."""
    eu, up = _u32(eu)
    ev, vp = _u32(ev)
    w, wp = _f32(w)
    r = _lib().lmo_brute_mwm(n, eu.shape[0], up, vp, wp)
    if r < 0:
        raise ValueError("brute_mwm: n too large or allocation failed")
    return float(r)


def contract(n: int, eu, ev, w, mate, vw=None):
    """Contraction of the matching `mate` (Sec. 1, the multilevel use of
    maximal matchings): (cmap[n], cvw[n'], ceu[m'], cev[m'], cw[m'])."""
    eu, up = _u32(eu)
    ev, vp = _u32(ev)
    w, wp = _f32(w)
    mate, mp = _u32(mate)
    vwp = None
    if vw is not None:
        vw, vwp = _u32(vw)
    m = eu.shape[0]
    cmap = np.empty(max(n, 1), dtype=np.uint32)
    cvw = np.empty(max(n, 1), dtype=np.uint32)
    ceu = np.empty(max(m, 1), dtype=np.uint32)
    cev = np.empty(max(m, 1), dtype=np.uint32)
    cw = np.empty(max(m, 1), dtype=np.float32)
    no = ctypes.c_uint32()
    mo = ctypes.c_uint64()
    p = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    r = _lib().lmo_contract(n, m, up, vp, wp, vwp, mp, p(cmap, ctypes.c_uint32), p(cvw, ctypes.c_uint32),
                            p(ceu, ctypes.c_uint32), p(cev, ctypes.c_uint32), p(cw, ctypes.c_float),
                            ctypes.byref(no), ctypes.byref(mo))
    if r == -1:
        raise MemoryError("oracle contract: allocation failed")
    if r == -2:
        raise ValueError("oracle contract: mate is not a matching of the vertex set, or an endpoint is out of range")
    k, g = int(no.value), int(mo.value)
    return cmap[:n].copy(), cvw[:k].copy(), ceu[:g].copy(), cev[:g].copy(), cw[:g].copy()
