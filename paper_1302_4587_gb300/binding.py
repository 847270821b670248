"""Thin Python binding of liblm.so (include/lm.h), argument marshalling only.

The functions carry the C names.  Arrays are torch tensors (CUDA or CPU) or
numpy arrays; device memory and streams come from PyTorch.  Every step of the
matching runs in the library's CUDA kernels: there is no Python or CPU
fallback, and loading fails loudly when the library cannot be built or
loaded.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _build

LM_OK, LM_EINVAL, LM_ENOMEM, LM_EAGAIN, LM_ETIMEOUT, LM_ECUDA, LM_ENOTFOUND = range(7)
LM_NIL = 0xFFFFFFFF
LM_HOST, LM_DEVICE = 0, 1
LM_F_PROFILE = 1
LM_F_EDGE_CENTRIC = 2
LM_F_RENEW = 4
LM_F_ASYNC = 8
LM_STATS_ROUNDS = 64
LM_K_INIT, LM_K_SWEEP, LM_K_VERTEX, LM_K_CAND, LM_K_OTHER, LM_K_TAIL, LM_K_COUNT = range(7)

# names exported by include/lm.h (the loader checks that every one is present)
EXPORTS = ("lm_create", "lm_destroy", "lm_graph_create", "lm_graph_destroy", "lm_graph_info", "lm_match",
           "lm_batch_match", "lm_submit", "lm_poll", "lm_wait", "lm_strerror", "lm_last_error",
           "lm_match_small_noalloc", "lm_get_tuning", "lm_set_tuning", "lm_autotune", "lm_sync", "lm_contract",
           "lm_set_limits")
LM_NOALLOC_MAX_N, LM_NOALLOC_MAX_M = 65536, 262144


class LmConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class LmStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("launches", ctypes.c_uint32), ("matched", ctypes.c_uint64),
                ("round_m", ctypes.c_uint64 * LM_STATS_ROUNDS), ("round_n", ctypes.c_uint64 * LM_STATS_ROUNDS),
                ("kernel_ms", ctypes.c_double * LM_K_COUNT), ("kernel_launches", ctypes.c_uint32 * LM_K_COUNT),
                ("total_ms", ctypes.c_double)]

    def to_dict(self) -> dict:
        r = int(self.rounds)
        k = min(r, LM_STATS_ROUNDS)
        return {"rounds": r, "launches": int(self.launches), "matched": int(self.matched),
                "round_m": [int(x) for x in self.round_m[:k]], "round_n": [int(x) for x in self.round_n[:k]],
                "kernel_ms": [float(x) for x in self.kernel_ms],
                "kernel_launches": [int(x) for x in self.kernel_launches], "total_ms": float(self.total_ms)}


class LmTuning(ctypes.Structure):
    _fields_ = [("rmax", ctypes.c_uint32), ("chunk", ctypes.c_uint32), ("sweep_ctas_per_sm", ctypes.c_uint32),
                ("vertex_ctas_per_sm", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("contract_bits", ctypes.c_uint32),
                ("ms", ctypes.c_double)]

    def to_dict(self) -> dict:
        return {"rmax": int(self.rmax), "chunk": int(self.chunk), "sweep_ctas_per_sm": int(self.sweep_ctas_per_sm),
                "vertex_ctas_per_sm": int(self.vertex_ctas_per_sm), "batch": int(self.batch),
                "contract_bits": int(self.contract_bits), "ms": float(self.ms)}


class LmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_LIB = None
_LOCK = threading.Lock()


def load(build: bool = True) -> ctypes.CDLL:
    """Load liblm.so (building it in-tree first if needed).  Raises if impossible."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        missing = [n for n in EXPORTS if not hasattr(lib, n)]
        if missing:
            raise RuntimeError(f"liblm.so lacks exports {missing}")
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.lm_create.argtypes = [ctypes.POINTER(LmConfig), ctypes.POINTER(vp)]
        lib.lm_destroy.argtypes = [vp]
        lib.lm_destroy.restype = None
        lib.lm_graph_create.argtypes = [vp, u32, u32, vp, vp, vp, ctypes.c_int, ctypes.POINTER(vp)]
        lib.lm_graph_destroy.argtypes = [vp]
        lib.lm_graph_destroy.restype = None
        lib.lm_graph_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u64)]
        lib.lm_match.argtypes = [vp, vp, u64, vp, ctypes.POINTER(LmStats)]
        lib.lm_batch_match.argtypes = [vp, ctypes.POINTER(vp), u32, ctypes.POINTER(u64), ctypes.POINTER(vp),
                                       ctypes.POINTER(LmStats)]
        lib.lm_submit.argtypes = [vp, vp, u64, vp, ctypes.POINTER(u64)]
        lib.lm_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(LmStats)]
        lib.lm_wait.argtypes = [vp, u64, u32]
        lib.lm_sync.argtypes = [vp]
        lib.lm_contract.argtypes = [vp, u32, u32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(u32), ctypes.POINTER(u32)]
        lib.lm_strerror.argtypes = [ctypes.c_int]
        lib.lm_strerror.restype = ctypes.c_char_p
        lib.lm_last_error.argtypes = [vp]
        lib.lm_last_error.restype = ctypes.c_char_p
        lib.lm_match_small_noalloc.argtypes = [u32, u32, vp, vp, vp, u64, vp, vp, vp]
        lib.lm_set_limits.argtypes = [vp, u32, u32]
        lib.lm_get_tuning.argtypes = [vp, ctypes.POINTER(LmTuning)]
        lib.lm_set_tuning.argtypes = [vp, ctypes.POINTER(LmTuning)]
        lib.lm_autotune.argtypes = [vp, ctypes.POINTER(vp), u32, ctypes.POINTER(u64), ctypes.POINTER(vp),
                                    ctypes.POINTER(LmTuning)]
        _LIB = lib
        return lib


def _check(rc: int, ctx=None):
    if rc != LM_OK:
        lib = load()
        msg = lib.lm_strerror(rc).decode()
        if ctx is not None:
            detail = lib.lm_last_error(ctx).decode()
            if detail:
                msg = f"{msg}: {detail}"
        raise LmError(rc, msg)


def _ptr(a):
    """(pointer, keepalive, is_device) of a torch tensor or numpy array."""
    if a is None:
        return None, None, False
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, a, False
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a, a.is_cuda
    raise TypeError(f"unsupported array type {type(a)}")


def _out(a, count: int, what: str):
    """(pointer, the buffer itself) of a caller-provided output of at least
    `count` 4-byte elements, written in place: a contiguous, writable numpy
    array or torch tensor (host or CUDA).  Anything else is refused here, since
    the library writes `count` elements through the pointer."""
    if isinstance(a, np.ndarray):
        if a.dtype.itemsize != 4 or not a.flags.c_contiguous or not a.flags.writeable or a.size < count:
            raise ValueError(f"{what}: needs a contiguous writable array of at least {count} 4-byte elements")
        return a.ctypes.data, a
    import torch
    if isinstance(a, torch.Tensor):
        if a.element_size() != 4 or not a.is_contiguous() or a.numel() < count:
            raise ValueError(f"{what}: needs a contiguous tensor of at least {count} 4-byte elements")
        return a.data_ptr(), a
    raise TypeError(f"{what}: unsupported array type {type(a)}")


# vertex count of each graph handle this binding created (output sizes are checked against it)
_GRAPH_N: dict = {}


def _handle(g) -> int:
    return g.value if isinstance(g, ctypes.c_void_p) else int(g)


def _graph_n(g) -> int:
    n = _GRAPH_N.get(_handle(g))
    return lm_graph_info(g)[0] if n is None else n


def _as(a, np_dtype, torch_dtype):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np_dtype)
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch_dtype:
            a = a.to(torch_dtype)
        return a.contiguous()
    return np.ascontiguousarray(np.asarray(a), dtype=np_dtype)


# ------------------------------------------------------------------ C-named functions

def lm_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0, max_slots: int = 0, flags: int = 0):
    """Create a context; `stream` is a torch.cuda.Stream, a raw cudaStream_t int, or None
    for torch's current stream on `device`."""
    lib = load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    cfg = LmConfig(device, ctypes.c_void_p(stream), hbm_budget_bytes, max_slots, flags)
    out = ctypes.c_void_p()
    _check(lib.lm_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def lm_destroy(ctx) -> None:
    load().lm_destroy(ctx)


def lm_graph_create(ctx, n: int, eu, ev, w):
    """Build a device graph from edge arrays (uint32 endpoints, float32 weights),
    all on the host (numpy / CPU tensors) or all on the device (CUDA tensors)."""
    lib = load()
    import torch
    u32 = torch.int32
    eu = _as(eu, np.uint32, u32)
    ev = _as(ev, np.uint32, u32)
    w = _as(w, np.float32, torch.float32)
    pu, ku, du = _ptr(eu)
    pv, kv, dv = _ptr(ev)
    pw, kw, dw = _ptr(w)
    m = int(eu.shape[0])
    if not (int(ev.shape[0]) == m == int(w.shape[0])):
        raise ValueError("eu, ev, w must have the same length")
    if len({du, dv, dw}) != 1:
        raise ValueError("eu, ev, w must all be host arrays or all device tensors")
    mem = LM_DEVICE if du else LM_HOST
    out = ctypes.c_void_p()
    _check(lib.lm_graph_create(ctx, n, m, pu, pv, pw, mem, ctypes.byref(out)), ctx)
    _GRAPH_N[out.value] = int(n)
    return out


def lm_graph_destroy(g) -> None:
    if g is not None:
        _GRAPH_N.pop(_handle(g), None)
    load().lm_graph_destroy(g)


def lm_graph_info(g):
    n, m, b = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
    _check(load().lm_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(b)))
    return int(n.value), int(m.value), int(b.value)


def lm_match(ctx, g, seed: int, mate=None, stats: bool = False):
    """Run local max on g; `mate` is an int32 tensor of n entries (CUDA or CPU) or a
    uint32 numpy array, allocated on the graph's device when None.  Returns mate
    (and the stats dict when stats=True)."""
    lib = load()
    if mate is None:
        import torch
        n = lm_graph_info(g)[0]
        dev = torch.cuda.current_device()
        mate = torch.empty(max(n, 1), dtype=torch.int32, device=f"cuda:{dev}")[:n]
    p, keep = _out(mate, _graph_n(g), "mate")
    st = LmStats()
    _check(lib.lm_match(ctx, g, seed & (2**64 - 1), p, ctypes.byref(st) if stats else None), ctx)
    return (keep, st.to_dict()) if stats else keep


class BatchArgs:
    """The marshalled arguments of lm_batch_match (graph handles, seeds, result
    pointers).  Build it once and pass it instead of the three lists to match
    the same graphs into the same buffers again without re-marshalling them."""

    def __init__(self, graphs, seeds, mates):
        cnt = len(graphs)
        if len(seeds) != cnt or len(mates) != cnt:
            raise ValueError("graphs, seeds and mates differ in length")
        self.count = cnt
        self.graphs = (ctypes.c_void_p * cnt)(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in graphs])
        self.seeds = (ctypes.c_uint64 * cnt)(*[int(x) & (2**64 - 1) for x in seeds])
        ptrs, self.keep = [], []
        for i, (g, mt) in enumerate(zip(graphs, mates)):
            p, k = _out(mt, _graph_n(g), f"mates[{i}]")
            ptrs.append(p)
            self.keep.append(k)
        self.mates = (ctypes.c_void_p * cnt)(*ptrs)


def lm_batch_match(ctx, graphs, seeds=None, mates=None, stats: bool = False):
    """Match many graphs in shared launches.  `graphs` is a list of graph
    handles (with `seeds` and `mates` lists) or a BatchArgs.  Returns the mate
    buffers (and per-graph stats dicts when stats=True)."""
    lib = load()
    b = graphs if isinstance(graphs, BatchArgs) else BatchArgs(graphs, seeds, mates)
    st = (LmStats * b.count)() if stats else None
    _check(lib.lm_batch_match(ctx, b.graphs, b.count, b.seeds, b.mates, st), ctx)
    return (b.keep, [s.to_dict() for s in st]) if stats else b.keep


def lm_submit(ctx, g, seed: int, mate) -> int:
    p, _ = _out(mate, _graph_n(g), "mate")
    t = ctypes.c_uint64()
    _check(load().lm_submit(ctx, g, seed & (2**64 - 1), p, ctypes.byref(t)), ctx)
    return int(t.value)


def lm_poll(ctx, ticket: int):
    """(done, stats dict or None); raises the request's error if it failed."""
    d = ctypes.c_int()
    st = LmStats()
    _check(load().lm_poll(ctx, ticket, ctypes.byref(d), ctypes.byref(st)), ctx)
    return bool(d.value), (st.to_dict() if d.value else None)


def lm_wait(ctx, ticket: int, timeout_ms: int) -> bool:
    rc = load().lm_wait(ctx, ticket, timeout_ms)
    if rc == LM_ETIMEOUT:
        return False
    _check(rc, ctx)
    return True


def lm_sync(ctx) -> None:
    """Wait for the matches queued on an LM_F_ASYNC context; raises LmError for a
    device-side error any of them met."""
    _check(load().lm_sync(ctx), ctx)


def lm_contract(ctx, n: int, eu, ev, w, mate, vw=None):
    """Contract the matching `mate` of the graph (n, eu, ev, w) on the device
    (torch CUDA tensors; int32 / float32).  Returns (cmap[n], cvw[n'], ceu[m'],
    cev[m'], cw[m']) as CUDA tensors (views of buffers of n and m entries)."""
    import torch
    m = int(eu.shape[0])
    # eu / ev / w hold exactly m edges; mate and vw cover at least the n vertices
    for t, cnt, exact, what in ((eu, m, True, "eu"), (ev, m, True, "ev"), (w, m, True, "w"),
                                (mate, n, False, "mate"), (vw, n, False, "vw")):
        if t is None:
            continue
        if (not isinstance(t, torch.Tensor) or t.element_size() != 4 or not t.is_contiguous()
                or (t.numel() != cnt if exact else t.numel() < cnt)):
            raise ValueError(f"{what}: needs a contiguous tensor of {'' if exact else 'at least '}{cnt} 4-byte elements")
    dev = eu.device if m else mate.device
    cmap = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cvw = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ceu = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    cev = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    cw = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    no, mo = ctypes.c_uint32(), ctypes.c_uint32()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().lm_contract(ctx, n, m, ptr(eu), ptr(ev), ptr(w), ptr(vw), ptr(mate), ptr(cmap), ptr(cvw),
                              ptr(ceu), ptr(cev), ptr(cw), ctypes.byref(no), ctypes.byref(mo)), ctx)
    k, g = int(no.value), int(mo.value)
    return cmap[:n], cvw[:k], ceu[:g], cev[:g], cw[:g]


def lm_strerror(code: int) -> str:
    return load().lm_strerror(code).decode()


def lm_match_small_noalloc(n: int, eu, ev, w, seed: int, mate, status, stream=None) -> None:
    """Queue local max of one small device-resident graph (n <= LM_NOALLOC_MAX_N,
    m <= LM_NOALLOC_MAX_M) on `stream` without any allocation by the library.
    eu / ev (int32 or uint32), w (float32), mate (int32[n]) and status (int32[1])
    are CUDA tensors; mate and status are written when the kernel ends.  Raises
    LmError on rejected arguments (sizes beyond the limits, null pointers)."""
    lib = load()
    m = int(eu.numel())
    if int(ev.numel()) != m or int(w.numel()) != m:
        raise ValueError("eu, ev and w differ in length")
    import torch
    dev = torch.cuda.current_device()
    for t in (eu, ev, w, mate, status):
        if not (t.is_cuda and t.is_contiguous() and t.element_size() == 4):
            raise ValueError("lm_match_small_noalloc takes contiguous CUDA tensors of 4-byte elements")
        if t.device.index != dev:
            raise ValueError(f"lm_match_small_noalloc runs on the current device (cuda:{dev}); "
                             f"a tensor lives on {t.device}")
    if int(mate.numel()) < n or int(status.numel()) < 1:
        raise ValueError("mate needs n entries and status one")
    if stream is None:
        s = None
    elif isinstance(stream, int):
        s = stream
    else:
        s = stream.cuda_stream
    _check(lib.lm_match_small_noalloc(n, m, eu.data_ptr(), ev.data_ptr(), w.data_ptr(), seed & (2**64 - 1),
                                      mate.data_ptr(), status.data_ptr(), s))


def lm_set_limits(ctx, max_rounds: int = 0, time_limit_ms: int = 0) -> None:
    """Round cap and time limit of the context's later matches (0 = the defaults:
    no cap beyond m + 2 rounds, 120 s); a match beyond either raises LmError
    with code LM_ETIMEOUT."""
    _check(load().lm_set_limits(ctx, max_rounds, time_limit_ms), ctx)


def lm_get_tuning(ctx) -> dict:
    t = LmTuning()
    _check(load().lm_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t.to_dict()


def lm_set_tuning(ctx, rmax: int, chunk: int, sweep_ctas_per_sm: int = 0, vertex_ctas_per_sm: int = 4,
                  batch: int = 512, contract_bits: int = 0) -> None:
    t = LmTuning(rmax, chunk, sweep_ctas_per_sm, vertex_ctas_per_sm, batch, contract_bits, 0.0)
    _check(load().lm_set_tuning(ctx, ctypes.byref(t)), ctx)


def lm_autotune(ctx, graphs, seeds=None, mates=None) -> dict:
    """Time the candidate launch parameters on these graphs (a list of handles with
    seeds and mates, or a BatchArgs), keep the fastest in the context, return it."""
    b = graphs if isinstance(graphs, BatchArgs) else BatchArgs(graphs, seeds, mates)
    t = LmTuning()
    _check(load().lm_autotune(ctx, b.graphs, b.count, b.seeds, b.mates, ctypes.byref(t)), ctx)
    return t.to_dict()
