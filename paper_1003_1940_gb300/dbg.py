"""Thin ctypes binding of libdbg (include/dbg.h), with the same names.

Only argument marshalling lives here: every step of graph construction and
compaction runs in the library's CUDA kernels.  PyTorch supplies device
memory (its caching allocator, through the library's allocator hooks) and
streams.  There is no CPU fallback: if libdbg.so is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_lib

DBG_OK, DBG_EINVAL, DBG_ENOMEM, DBG_ECUDA, DBG_ETIMEOUT, DBG_ECANCELLED, DBG_EOVERFLOW, DBG_EAGAIN, \
    DBG_EINTERNAL = range(9)
_STATUS = {0: "DBG_OK", 1: "DBG_EINVAL", 2: "DBG_ENOMEM", 3: "DBG_ECUDA", 4: "DBG_ETIMEOUT",
           5: "DBG_ECANCELLED", 6: "DBG_EOVERFLOW", 7: "DBG_EAGAIN", 8: "DBG_EINTERNAL"}

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class dbg_options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("device", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("alloc", _ALLOC_FN),
        ("free", _FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("mem_budget", ctypes.c_uint64),
        ("spin_limit", ctypes.c_uint32),
        ("reserved0", ctypes.c_uint32),
        ("reserved1", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 8),
    ]


class dbg_graph_view(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint32), ("key_words", ctypes.c_uint32),
        ("num_nodes", ctypes.c_uint64), ("num_edges", ctypes.c_uint64), ("num_instances", ctypes.c_uint64),
        ("node_keys", ctypes.c_void_p), ("edge_keys", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
        ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("mult", ctypes.c_void_p),
        ("adj_nbr", ctypes.c_void_p), ("adj_edge", ctypes.c_void_p),
        ("orient", ctypes.c_void_p), ("adj_role", ctypes.c_void_p),
    ]


class dbg_stage_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


# (name, restype, argtypes) of every C entry point
_P = ctypes.c_void_p
_SIGNATURES = [
    ("dbg_options_init", None, [_P]),
    ("dbg_create", ctypes.c_int, [_P, _P]),
    ("dbg_destroy", None, [_P]),
    ("dbg_last_error", ctypes.c_char_p, []),
    ("dbg_build", ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, ctypes.c_uint32, _P]),
    ("dbg_graph_k", ctypes.c_uint32, [_P]),
    ("dbg_graph_key_words", ctypes.c_uint32, [_P]),
    ("dbg_graph_num_nodes", ctypes.c_uint64, [_P]),
    ("dbg_graph_num_edges", ctypes.c_uint64, [_P]),
    ("dbg_graph_num_instances", ctypes.c_uint64, [_P]),
    ("dbg_graph_nodes", ctypes.c_int, [_P, _P]),
    ("dbg_graph_edges", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dbg_graph_edges_async", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dbg_graph_nodes_async", ctypes.c_int, [_P, _P]),
    ("dbg_graph_csr_async", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("dbg_node_mult_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_graph_node_mult", ctypes.c_int, [_P, _P]),
    ("dbg_node_reads_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_graph_node_reads", ctypes.c_int, [_P, _P]),
    ("dbg_roadmap_nodes", ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P]),
    ("dbg_graph_wait", ctypes.c_int, [_P]),
    ("dbg_graph_csr", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("dbg_graph_device_view", ctypes.c_int, [_P, _P]),
    ("dbg_graph_free", None, [_P]),
    ("dbg_compact", ctypes.c_int, [_P, _P, _P]),
    ("dbg_compact_bucketed", ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P]),
    ("dbg_unitigs_count", ctypes.c_uint64, [_P]),
    ("dbg_unitigs_total_bases", ctypes.c_uint64, [_P]),
    ("dbg_unitigs_get", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dbg_unitigs_free", None, [_P]),
    ("dbg_simplify", ctypes.c_int, [_P, _P, ctypes.c_uint32, _P]),
    ("dbg_simple_num_units", ctypes.c_uint64, [_P]),
    ("dbg_simple_num_edges", ctypes.c_uint64, [_P]),
    ("dbg_simple_removed_edges", ctypes.c_uint64, [_P]),
    ("dbg_simple_total_bases", ctypes.c_uint64, [_P]),
    ("dbg_simple_units", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dbg_simple_edges", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dbg_simple_free", None, [_P]),
    ("dbg_profile_enable", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_profile_read", ctypes.c_uint32, [_P, _P, ctypes.c_uint32]),
    ("dbg_launch_count", ctypes.c_uint64, [_P]),
    ("dbg_rle_u64_noalloc", ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, _P]),
    ("dbg_sort_variant_count", ctypes.c_uint32, [ctypes.c_uint32]),
    ("dbg_sort_variant_name", ctypes.c_char_p, [ctypes.c_uint32, ctypes.c_uint32]),
    ("dbg_sort_variant_set", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32]),
    ("dbg_sort_variant_get", ctypes.c_int32, [_P, ctypes.c_uint32]),
    ("dbg_sort_hybrid_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_sort_count_first_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_sort_count_overflows", ctypes.c_uint64, [_P]),
    ("dbg_sort_partition_first_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_sort_local_rank_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_sort_rank_fallbacks", ctypes.c_uint64, [_P]),
    ("dbg_compact_mode_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_copy_streams_set", ctypes.c_int, [_P, ctypes.c_int]),
    ("dbg_sort_fallbacks", ctypes.c_uint64, [_P]),
    ("dbg_autotune", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_char_p, _P]),
]

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return build_lib.LIB_PATH


def load(build: bool = False):
    """Loads libdbg.so (building it first when `build`); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib.build() if build else build_lib.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"libdbg.so not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, res, args in _SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DbgError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")
        self.status = status


def _check(status: int, where: str):
    if status != DBG_OK:
        msg = _lib.dbg_last_error()
        raise DbgError(status, where, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# device memory from PyTorch's caching allocator
# ---------------------------------------------------------------------------
class _TorchAllocator:
    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(user, nbytes, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:  # out of memory: report NULL, the library returns DBG_ENOMEM
                return None

        def _free(user, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = _ALLOC_FN(_alloc)
        self.free = _FREE_FN(_free)


class Context:
    """dbg_ctx: device, stream, allocator."""

    def __init__(self, device: int | None = None, stream=None, torch_allocator: bool = True,
                 mem_budget: int = 0, spin_limit: int = 0):
        import torch
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        opt = dbg_options()
        lib.dbg_options_init(ctypes.byref(opt))
        opt.device = device
        opt.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        opt.mem_budget = mem_budget
        opt.spin_limit = spin_limit
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator(device)
            opt.alloc = self._alloc.alloc
            opt.free = self._alloc.free
        self._opt = opt
        h = ctypes.c_void_p()
        _check(lib.dbg_create(ctypes.byref(h), ctypes.byref(opt)), "dbg_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dbg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def _ptr(x) -> tuple[int, object]:
    """Data pointer of a numpy array, bytes or torch tensor (host or device)."""
    if isinstance(x, (bytes, bytearray)):
        x = np.frombuffer(bytes(x), dtype=np.uint8)
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x)
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x
    raise TypeError(f"unsupported buffer type {type(x)}")


class Graph:
    """dbg_graph handle; holds its context so the context outlives it."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def free(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dbg_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


class Unitigs:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def free(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dbg_unitigs_free(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


def dbg_create(**kw) -> Context:
    return Context(**kw)


def dbg_destroy(ctx: Context):
    ctx.close()


def dbg_build(ctx: Context, reads, lengths, k: int) -> Graph:
    """reads: uint8 ASCII (numpy / bytes / torch, host or cuda); lengths: uint32."""
    rp, rkeep = _ptr(reads)
    if isinstance(lengths, np.ndarray) and lengths.dtype != np.uint32:
        lengths = lengths.astype(np.uint32)
    lp, lkeep = _ptr(lengths)
    n = len(lengths) if not hasattr(lengths, "numel") else int(lengths.numel())
    out = ctypes.c_void_p()
    _check(_lib.dbg_build(ctx.handle, ctypes.c_void_p(rp), ctypes.c_void_p(lp), n, k, ctypes.byref(out)),
           "dbg_build")
    del rkeep, lkeep
    return Graph(ctx, out)


def dbg_graph_k(g: Graph) -> int:
    return int(_lib.dbg_graph_k(g.handle))


def dbg_graph_key_words(g: Graph) -> int:
    return int(_lib.dbg_graph_key_words(g.handle))


def dbg_graph_num_nodes(g: Graph) -> int:
    return int(_lib.dbg_graph_num_nodes(g.handle))


def dbg_graph_num_edges(g: Graph) -> int:
    return int(_lib.dbg_graph_num_edges(g.handle))


def dbg_graph_num_instances(g: Graph) -> int:
    return int(_lib.dbg_graph_num_instances(g.handle))


def _np_out(n, dtype):
    return np.zeros(max(0, n), dtype=dtype)


def dbg_graph_nodes(g: Graph) -> np.ndarray:
    W = dbg_graph_key_words(g)
    out = _np_out(dbg_graph_num_nodes(g) * W, np.uint64)
    _check(_lib.dbg_graph_nodes(g.handle, ctypes.c_void_p(out.ctypes.data)), "dbg_graph_nodes")
    return out.reshape(-1, W)


def dbg_graph_edges(g: Graph) -> dict:
    W, E = dbg_graph_key_words(g), dbg_graph_num_edges(g)
    keys, src, dst = _np_out(E * W, np.uint64), _np_out(E, np.uint32), _np_out(E, np.uint32)
    orient, mult = _np_out(E, np.uint8), _np_out(E, np.uint32)
    _check(_lib.dbg_graph_edges(g.handle, *(ctypes.c_void_p(a.ctypes.data) for a in (keys, src, dst, orient, mult))),
           "dbg_graph_edges")
    return {"keys": keys.reshape(-1, W), "src": src, "dst": dst, "orient": orient, "mult": mult}


def dbg_node_mult_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_node_mult_set(ctx.handle, 1 if on else 0), "dbg_node_mult_set")


def dbg_graph_node_mult(g: Graph) -> np.ndarray:
    """k-mer occurrences per node (the build must have counted them)."""
    out = _np_out(dbg_graph_num_nodes(g), np.uint32)
    _check(_lib.dbg_graph_node_mult(g.handle, ctypes.c_void_p(out.ctypes.data)), "dbg_graph_node_mult")
    return out


def dbg_node_reads_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_node_reads_set(ctx.handle, 1 if on else 0), "dbg_node_reads_set")


def dbg_graph_node_reads(g: Graph) -> np.ndarray:
    """Distinct reads holding each node's k-mer (either strand), node order."""
    out = _np_out(dbg_graph_num_nodes(g), np.uint32)
    _check(_lib.dbg_graph_node_reads(g.handle, ctypes.c_void_p(out.ctypes.data)), "dbg_graph_node_reads")
    return out


def dbg_roadmap_nodes(ctx: Context, g: Graph, min_reads: int = 2) -> np.ndarray:
    """IDs (ascending) of the nodes held by at least min_reads distinct reads."""
    count = ctypes.c_uint64(0)
    _check(_lib.dbg_roadmap_nodes(ctx.handle, g.handle, min_reads, None, ctypes.byref(count)), "dbg_roadmap_nodes")
    ids = _np_out(count.value, np.uint32)
    if count.value:
        _check(_lib.dbg_roadmap_nodes(ctx.handle, g.handle, min_reads, ctypes.c_void_p(ids.ctypes.data),
                                      ctypes.byref(count)), "dbg_roadmap_nodes")
    return ids


def dbg_graph_edges_async(g: Graph, keys: int | None = None, src: int | None = None, dst: int | None = None,
                          orient: int | None = None, mult: int | None = None) -> None:
    """Starts the edge-array copies into caller-owned buffers (raw addresses,
    e.g. pinned tensors' data_ptr(); None skips an array); dbg_graph_wait
    finishes them."""
    ptrs = (ctypes.c_void_p(a) if a else None for a in (keys, src, dst, orient, mult))
    _check(_lib.dbg_graph_edges_async(g.handle, *ptrs), "dbg_graph_edges_async")


def dbg_graph_nodes_async(g: Graph, keys: int | None = None) -> None:
    """Starts the node-key copy into a caller-owned buffer (raw address)."""
    _check(_lib.dbg_graph_nodes_async(g.handle, ctypes.c_void_p(keys) if keys else None), "dbg_graph_nodes_async")


def dbg_graph_csr_async(g: Graph, row_ptr: int | None = None, nbr: int | None = None, edge: int | None = None,
                        role: int | None = None) -> None:
    """Starts the adjacency copies into caller-owned buffers (raw addresses)."""
    ptrs = (ctypes.c_void_p(a) if a else None for a in (row_ptr, nbr, edge, role))
    _check(_lib.dbg_graph_csr_async(g.handle, *ptrs), "dbg_graph_csr_async")


def dbg_graph_wait(g: Graph) -> None:
    _check(_lib.dbg_graph_wait(g.handle), "dbg_graph_wait")


def dbg_graph_csr(g: Graph) -> dict:
    V, E = dbg_graph_num_nodes(g), dbg_graph_num_edges(g)
    row_ptr, nbr = _np_out(V + 1, np.uint64), _np_out(2 * E, np.uint32)
    edge, role = _np_out(2 * E, np.uint32), _np_out(2 * E, np.uint8)
    _check(_lib.dbg_graph_csr(g.handle, *(ctypes.c_void_p(a.ctypes.data) for a in (row_ptr, nbr, edge, role))),
           "dbg_graph_csr")
    return {"row_ptr": row_ptr, "nbr": nbr, "edge": edge, "role": role}


def dbg_graph_device_view(g: Graph) -> dbg_graph_view:
    v = dbg_graph_view()
    _check(_lib.dbg_graph_device_view(g.handle, ctypes.byref(v)), "dbg_graph_device_view")
    return v


def dbg_graph_free(g: Graph):
    g.free()


def dbg_compact(ctx: Context, g: Graph) -> Unitigs:
    out = ctypes.c_void_p()
    _check(_lib.dbg_compact(ctx.handle, g.handle, ctypes.byref(out)), "dbg_compact")
    return Unitigs(ctx, out)


def dbg_compact_bucketed(ctx: Context, g: Graph, mem_budget: int = 0) -> tuple:
    """Unitigs by the out-of-core list ranking (sort-join rounds over key
    ranges of host-resident ranking words); returns (Unitigs, join launches)."""
    out = ctypes.c_void_p()
    launches = ctypes.c_uint32(0)
    _check(_lib.dbg_compact_bucketed(ctx.handle, g.handle, mem_budget, ctypes.byref(out), ctypes.byref(launches)),
           "dbg_compact_bucketed")
    return Unitigs(ctx, out), int(launches.value)


def dbg_unitigs_count(u: Unitigs) -> int:
    return int(_lib.dbg_unitigs_count(u.handle))


def dbg_unitigs_total_bases(u: Unitigs) -> int:
    return int(_lib.dbg_unitigs_total_bases(u.handle))


def dbg_unitigs_get(u: Unitigs) -> dict:
    U = dbg_unitigs_count(u)
    node_off, seq_off = _np_out(U + 1, np.uint64), _np_out(U + 1, np.uint64)
    n_nodes = 0
    _check(_lib.dbg_unitigs_get(u.handle, ctypes.c_void_p(node_off.ctypes.data), None,
                                None, None, None), "dbg_unitigs_get")
    n_nodes = int(node_off[-1]) if U else 0
    nodes = _np_out(n_nodes, np.uint64)
    seq = _np_out(dbg_unitigs_total_bases(u), np.uint8)
    circ = _np_out(U, np.uint8)
    _check(_lib.dbg_unitigs_get(u.handle, None, ctypes.c_void_p(nodes.ctypes.data),
                                ctypes.c_void_p(seq_off.ctypes.data), ctypes.c_void_p(seq.ctypes.data),
                                ctypes.c_void_p(circ.ctypes.data)), "dbg_unitigs_get")
    return {"node_off": node_off, "nodes": nodes, "seq_off": seq_off, "seq": seq.tobytes(), "circular": circ}


def dbg_unitigs_get_into(u: Unitigs, node_off: int | None = None, nodes: int | None = None,
                         seq_off: int | None = None, seq: int | None = None, circular: int | None = None) -> None:
    """dbg_unitigs_get into caller-owned buffers (raw host or device
    addresses, e.g. pinned tensors' data_ptr(); None skips an array)."""
    ptrs = (ctypes.c_void_p(a) if a else None for a in (node_off, nodes, seq_off, seq, circular))
    _check(_lib.dbg_unitigs_get(u.handle, *ptrs), "dbg_unitigs_get")


class Simple:
    """dbg_simple: the simplified graph (units and relabelled edges)."""

    def __init__(self, ctx: Context, handle):
        self.ctx, self.handle = ctx, handle

    def free(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dbg_simple_free(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


def dbg_simplify(ctx: Context, g: Graph, min_nodes: int = 3) -> Simple:
    out = ctypes.c_void_p()
    _check(_lib.dbg_simplify(ctx.handle, g.handle, min_nodes, ctypes.byref(out)), "dbg_simplify")
    return Simple(ctx, out)


def dbg_simple_get(s: Simple) -> dict:
    """Units (node_off, nodes, seq_off, seq, circular) and edges (unit_a,
    side_a, unit_b, side_b, edge) as host arrays, plus removed."""
    U, M = int(_lib.dbg_simple_num_units(s.handle)), int(_lib.dbg_simple_num_edges(s.handle))
    node_off, seq_off = _np_out(U + 1, np.uint64), _np_out(U + 1, np.uint64)
    _check(_lib.dbg_simple_units(s.handle, ctypes.c_void_p(node_off.ctypes.data), None, None, None, None),
           "dbg_simple_units")
    nodes = _np_out(int(node_off[-1]) if U else 0, np.uint64)
    seq = _np_out(int(_lib.dbg_simple_total_bases(s.handle)), np.uint8)
    circ = _np_out(U, np.uint8)
    _check(_lib.dbg_simple_units(s.handle, None, ctypes.c_void_p(nodes.ctypes.data),
                                 ctypes.c_void_p(seq_off.ctypes.data), ctypes.c_void_p(seq.ctypes.data),
                                 ctypes.c_void_p(circ.ctypes.data)), "dbg_simple_units")
    ua, ub, ed = _np_out(M, np.uint32), _np_out(M, np.uint32), _np_out(M, np.uint32)
    sa, sb = _np_out(M, np.uint8), _np_out(M, np.uint8)
    _check(_lib.dbg_simple_edges(s.handle, *(ctypes.c_void_p(a.ctypes.data) for a in (ua, sa, ub, sb, ed))),
           "dbg_simple_edges")
    return {"node_off": node_off, "nodes": nodes, "seq_off": seq_off, "seq": seq.tobytes(), "circular": circ,
            "unit_a": ua, "side_a": sa, "unit_b": ub, "side_b": sb, "edge": ed,
            "removed": int(_lib.dbg_simple_removed_edges(s.handle))}


def dbg_unitigs_free(u: Unitigs):
    u.free()


def dbg_profile_enable(ctx: Context, on: bool = True):
    _check(_lib.dbg_profile_enable(ctx.handle, 1 if on else 0), "dbg_profile_enable")


def dbg_profile_read(ctx: Context) -> dict:
    """{stage: {"launches", "ms", "bytes"}} for the stages with launches."""
    arr = (dbg_stage_stat * 32)()
    n = _lib.dbg_profile_read(ctx.handle, arr, 32)
    out = {}
    for i in range(min(n, 32)):
        st = arr[i]
        if st.launches:
            out[st.name.decode()] = {"launches": int(st.launches), "ms": float(st.ms), "bytes": float(st.bytes)}
    return out


def dbg_launch_count(ctx: Context) -> int:
    return int(_lib.dbg_launch_count(ctx.handle))


def dbg_rle_u64_noalloc(keys, n: int, uniq, run_start, stream=None) -> int:
    """Run-length reduce of n sorted u64 keys with no allocation (device
    tensors in, device tensors out); returns the number of distinct keys.
    keys and uniq hold at least n 8-byte elements, run_start at least n + 1
    4-byte elements; all three contiguous, on the current CUDA device."""
    import torch
    if n < 0:
        raise ValueError("n must be >= 0")
    for name, t, need, size in (("keys", keys, n, 8), ("uniq", uniq, n, 8), ("run_start", run_start, n + 1, 4)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.element_size() != size or t.is_floating_point():
            raise ValueError(f"{name} must hold {size}-byte integers")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {need}")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, not the current device")
    count = ctypes.c_uint64(0)
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(_lib.dbg_rle_u64_noalloc(ctypes.c_void_p(_ptr(keys)[0]), n, ctypes.c_void_p(_ptr(uniq)[0]),
                                    ctypes.c_void_p(_ptr(run_start)[0]), ctypes.byref(count), ctypes.c_void_p(s)),
           "dbg_rle_u64_noalloc")
    return int(count.value)


def dbg_sort_variant_count(kind: int) -> int:
    return int(_lib.dbg_sort_variant_count(kind))


def dbg_sort_variant_name(kind: int, variant: int) -> str:
    r = _lib.dbg_sort_variant_name(kind, variant)
    return r.decode() if r else ""


def dbg_sort_variant_set(ctx: Context, kind: int, variant: int):
    _check(_lib.dbg_sort_variant_set(ctx.handle, kind, variant), "dbg_sort_variant_set")


def dbg_sort_variant_get(ctx: Context, kind: int) -> int:
    return int(_lib.dbg_sort_variant_get(ctx.handle, kind))


def dbg_sort_hybrid_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_sort_hybrid_set(ctx.handle, 1 if on else 0), "dbg_sort_hybrid_set")


def dbg_sort_count_first_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_sort_count_first_set(ctx.handle, 1 if on else 0), "dbg_sort_count_first_set")


def dbg_sort_count_overflows(ctx: Context) -> int:
    return int(_lib.dbg_sort_count_overflows(ctx.handle))


def dbg_sort_partition_first_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_sort_partition_first_set(ctx.handle, 1 if on else 0), "dbg_sort_partition_first_set")


def dbg_sort_local_rank_set(ctx: Context, on: bool) -> None:
    _check(_lib.dbg_sort_local_rank_set(ctx.handle, 1 if on else 0), "dbg_sort_local_rank_set")


def dbg_sort_rank_fallbacks(ctx: Context) -> int:
    return int(_lib.dbg_sort_rank_fallbacks(ctx.handle))


def dbg_compact_mode_set(ctx: Context, mode: int) -> None:
    _check(_lib.dbg_compact_mode_set(ctx.handle, int(mode)), "dbg_compact_mode_set")


def dbg_copy_streams_set(ctx: Context, n: int) -> None:
    _check(_lib.dbg_copy_streams_set(ctx.handle, int(n)), "dbg_copy_streams_set")


def dbg_sort_fallbacks(ctx: Context) -> int:
    return int(_lib.dbg_sort_fallbacks(ctx.handle))


MAX_SORT_VARIANTS = 64  # DBG_MAX_SORT_VARIANTS of dbg.h: stride of the autotune report


def dbg_autotune(ctx: Context, n: int = 0, cache_path: str | None = None) -> dict:
    """Times every radix-sort variant; returns {kind: [ms per variant]}."""
    ms = (ctypes.c_double * (4 * MAX_SORT_VARIANTS))()
    _check(_lib.dbg_autotune(ctx.handle, n, cache_path.encode() if cache_path else None, ms), "dbg_autotune")
    return {kd: [ms[kd * MAX_SORT_VARIANTS + v] for v in range(dbg_sort_variant_count(kd))] for kd in range(4)}


# ---------------------------------------------------------------------------
# many constructions at once: batch, server, bucket path
# ---------------------------------------------------------------------------
class dbg_readset(ctypes.Structure):
    _fields_ = [("reads", ctypes.c_void_p), ("lengths", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("k", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class dbg_server_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("device", ctypes.c_int32), ("workers", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("sort_variant", ctypes.c_uint32 * 4), ("reserved", ctypes.c_uint32 * 8)]


class dbg_request_stats(ctypes.Structure):
    _fields_ = [("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("footprint", ctypes.c_uint64), ("bucketed", ctypes.c_uint32), ("retries", ctypes.c_uint32),
                ("charged", ctypes.c_uint64)]


class dbg_server_counters(ctypes.Structure):
    _fields_ = [("charged", ctypes.c_uint64), ("peak_charged", ctypes.c_uint64), ("finished", ctypes.c_uint64),
                ("running", ctypes.c_uint32), ("peak_running", ctypes.c_uint32), ("queued", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


DBG_REQ_BUCKETED = 1
_SIGNATURES += [
    ("dbg_server_options_init", None, [_P]),
    ("dbg_server_create", ctypes.c_int, [_P, _P]),
    ("dbg_server_destroy", None, [_P]),
    ("dbg_server_budget", ctypes.c_uint64, [_P]),
    ("dbg_server_charged", ctypes.c_uint64, [_P]),
    ("dbg_server_stats", ctypes.c_int, [_P, _P]),
    ("dbg_submit", ctypes.c_int, [_P, _P, _P]),
    ("dbg_poll", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, _P, _P]),
    ("dbg_build_batch", ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_uint32, _P]),
    ("dbg_build_bucketed", ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _P]),
    ("dbg_graph_buckets", None, [_P, _P, _P]),
    ("dbg_selftest_wait", ctypes.c_int, [_P, ctypes.c_uint32]),
]


def _bind_late():
    lib = load()
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _readset(reads, lengths, k, flags=0):
    rp, rkeep = _ptr(reads)
    lp, lkeep = _ptr(lengths)
    n = len(lengths) if not hasattr(lengths, "numel") else int(lengths.numel())
    rs = dbg_readset(ctypes.c_void_p(rp), ctypes.c_void_p(lp), n, k, flags)
    return rs, (rkeep, lkeep)


class Server:
    """dbg_server: worker threads with one context and stream each."""

    def __init__(self, device=None, workers=4, mem_budget=0, spin_limit=0, sort_variant=(0, 0, 0, 0)):
        import torch
        lib = _bind_late()
        o = dbg_server_options()
        lib.dbg_server_options_init(ctypes.byref(o))
        o.device = torch.cuda.current_device() if device is None else device
        o.workers = workers
        o.mem_budget = mem_budget
        o.spin_limit = spin_limit
        for i, v in enumerate(sort_variant):
            o.sort_variant[i] = v
        h = ctypes.c_void_p()
        _check(lib.dbg_server_create(ctypes.byref(h), ctypes.byref(o)), "dbg_server_create")
        self.handle = h
        self._inputs = {}

    def budget(self) -> int:
        return int(_lib.dbg_server_budget(self.handle))

    def charged(self) -> int:
        """Bytes charged to the budget: running requests and unfreed results."""
        return int(_lib.dbg_server_charged(self.handle))

    def stats(self) -> dict:
        c = dbg_server_counters()
        _check(_lib.dbg_server_stats(self.handle, ctypes.byref(c)), "dbg_server_stats")
        return {f: int(getattr(c, f)) for f, _ in dbg_server_counters._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dbg_server_destroy(self.handle)
            self.handle = None
            self._inputs.clear()

    def __del__(self):
        self.close()


def dbg_server_create(**kw) -> Server:
    return Server(**kw)


def dbg_server_destroy(srv: Server):
    srv.close()


def dbg_submit(srv: Server, reads, lengths, k: int, flags: int = 0) -> int:
    rs, keep = _readset(reads, lengths, k, flags)
    t = ctypes.c_uint64(0)
    _check(_lib.dbg_submit(srv.handle, ctypes.byref(rs), ctypes.byref(t)), "dbg_submit")
    srv._inputs[int(t.value)] = keep  # borrowed by the library until polled
    return int(t.value)


def dbg_poll(srv: Server, ticket: int, wait: bool = True):
    """(Graph, stats dict), or None while the request runs (wait=False)."""
    out = ctypes.c_void_p()
    st = dbg_request_stats()
    rc = _lib.dbg_poll(srv.handle, ticket, 1 if wait else 0, ctypes.byref(out), ctypes.byref(st))
    if rc == DBG_EAGAIN:
        return None
    srv._inputs.pop(ticket, None)
    _check(rc, "dbg_poll")
    stats = {"queue_s": st.queue_s, "run_s": st.run_s, "latency_s": st.latency_s,
             "footprint": int(st.footprint), "bucketed": bool(st.bucketed), "retries": int(st.retries),
             "charged": int(st.charged)}
    return Graph(srv, out), stats


def dbg_build_batch(ctx: Context, sets, workers: int = 0) -> list:
    """sets: list of (reads, lengths, k); one Graph per set."""
    _bind_late()
    arr = (dbg_readset * max(1, len(sets)))()
    keep = []
    for i, (r, l, k) in enumerate(sets):
        rs, kp = _readset(r, l, k)
        arr[i] = rs
        keep.append(kp)
    outs = (ctypes.c_void_p * max(1, len(sets)))()
    _check(_lib.dbg_build_batch(ctx.handle, arr, len(sets), workers, outs), "dbg_build_batch")
    return [Graph(ctx, ctypes.c_void_p(outs[i])) for i in range(len(sets))]


def dbg_build_bucketed(ctx: Context, reads, lengths, k: int, mem_budget: int = 0) -> Graph:
    _bind_late()
    rp, rkeep = _ptr(reads)
    lp, lkeep = _ptr(lengths)
    n = len(lengths) if not hasattr(lengths, "numel") else int(lengths.numel())
    out = ctypes.c_void_p()
    _check(_lib.dbg_build_bucketed(ctx.handle, ctypes.c_void_p(rp), ctypes.c_void_p(lp), n, k, mem_budget,
                                   ctypes.byref(out)), "dbg_build_bucketed")
    del rkeep, lkeep
    return Graph(ctx, out)


def dbg_graph_buckets(g: Graph) -> tuple[int, int]:
    a, b = ctypes.c_uint32(0), ctypes.c_uint32(0)
    _lib.dbg_graph_buckets(g.handle, ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


class _DeviceArray:
    """Zero-copy view of one of a graph's device arrays (for torch.as_tensor)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def device_tensor(g: Graph, field: str, n: int, typestr: str):
    """torch view of the graph array `field` of dbg_graph_view (no copy;
    valid while the graph lives).  typestr: numpy-style, e.g. '<u8', '<u4', '|u1'."""
    import torch
    v = dbg_graph_device_view(g)
    return torch.as_tensor(_DeviceArray(int(getattr(v, field)), n, typestr), device="cuda")


def dbg_selftest_wait(ctx: Context, spin_limit: int) -> int:
    """Runs one bounded device wait that cannot succeed; returns the status."""
    _bind_late()
    return int(_lib.dbg_selftest_wait(ctx.handle, spin_limit))
