"""Test infrastructure: ctypes wrapper around the plain C oracle (oracle.c).

The oracle restates the definitions of the bi-directed de Bruijn graph
(Section 2 of Kundeti et al., arXiv 1003.1940), the adjacency of STEP-4
(Section 3), chain compaction (Section 6) and node multiplicities (the
k-mer occurrence counts of Section 7's roadmap discussion) on the CPU.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it;
the GPU library never imports it and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EINTERNAL = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compiles oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Graph(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint32),
        ("n_nodes", ctypes.c_uint64),
        ("n_edges", ctypes.c_uint64),
        ("node_keys", ctypes.POINTER(ctypes.c_uint64)),
        ("edge_keys", ctypes.POINTER(ctypes.c_uint64)),
        ("src", ctypes.POINTER(ctypes.c_uint32)),
        ("dst", ctypes.POINTER(ctypes.c_uint32)),
        ("orient", ctypes.POINTER(ctypes.c_uint8)),
        ("mult", ctypes.POINTER(ctypes.c_uint32)),
        ("row_ptr", ctypes.POINTER(ctypes.c_uint64)),
        ("adj_nbr", ctypes.POINTER(ctypes.c_uint32)),
        ("adj_edge", ctypes.POINTER(ctypes.c_uint32)),
        ("adj_role", ctypes.POINTER(ctypes.c_uint8)),
        ("flags", ctypes.c_uint32),
    ]


class _Unitigs(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_uint64),
        ("node_off", ctypes.POINTER(ctypes.c_uint64)),
        ("nodes", ctypes.POINTER(ctypes.c_uint64)),
        ("seq_off", ctypes.POINTER(ctypes.c_uint64)),
        ("seq", ctypes.POINTER(ctypes.c_char)),
        ("circular", ctypes.POINTER(ctypes.c_uint8)),
    ]


class _Range(ctypes.Structure):
    _fields_ = [
        ("n_edges", ctypes.c_uint64),
        ("n_nodes", ctypes.c_uint64),
        ("edge_keys", ctypes.POINTER(ctypes.c_uint64)),
        ("src_keys", ctypes.POINTER(ctypes.c_uint64)),
        ("dst_keys", ctypes.POINTER(ctypes.c_uint64)),
        ("orient", ctypes.POINTER(ctypes.c_uint8)),
        ("mult", ctypes.POINTER(ctypes.c_uint64)),
        ("node_keys", ctypes.POINTER(ctypes.c_uint64)),
    ]


class _Simple(ctypes.Structure):
    _fields_ = [
        ("n_units", ctypes.c_uint64),
        ("n_edges", ctypes.c_uint64),
        ("removed", ctypes.c_uint64),
        ("node_off", ctypes.POINTER(ctypes.c_uint64)),
        ("nodes", ctypes.POINTER(ctypes.c_uint64)),
        ("seq_off", ctypes.POINTER(ctypes.c_uint64)),
        ("seq", ctypes.POINTER(ctypes.c_char)),
        ("circular", ctypes.POINTER(ctypes.c_uint8)),
        ("unit_a", ctypes.POINTER(ctypes.c_uint32)),
        ("unit_b", ctypes.POINTER(ctypes.c_uint32)),
        ("side_a", ctypes.POINTER(ctypes.c_uint8)),
        ("side_b", ctypes.POINTER(ctypes.c_uint8)),
        ("edge", ctypes.POINTER(ctypes.c_uint32)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_build.restype = ctypes.c_int
            lib.orc_build.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.POINTER(ctypes.POINTER(_Graph))]
            lib.orc_graph_free.restype = None
            lib.orc_graph_free.argtypes = [ctypes.POINTER(_Graph)]
            lib.orc_compact.restype = ctypes.c_int
            lib.orc_compact.argtypes = [ctypes.POINTER(_Graph),
                                        ctypes.POINTER(ctypes.POINTER(_Unitigs))]
            lib.orc_unitigs_free.restype = None
            lib.orc_unitigs_free.argtypes = [ctypes.POINTER(_Unitigs)]
            lib.orc_count_kplus1.restype = ctypes.c_int
            lib.orc_count_kplus1.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                             ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                             ctypes.c_void_p]
            lib.orc_node_mult.restype = ctypes.c_int
            lib.orc_node_mult.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64)),
                                          ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))]
            lib.orc_node_reads.restype = ctypes.c_int
            lib.orc_node_reads.argtypes = lib.orc_node_mult.argtypes
            lib.orc_free.restype = None
            lib.orc_free.argtypes = [ctypes.c_void_p]
            lib.orc_edges_in_partition.restype = ctypes.c_int
            lib.orc_edges_in_partition.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                   ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_graph_range.restype = ctypes.c_int
            lib.orc_graph_range.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.POINTER(_Range))]
            lib.orc_simplify.restype = ctypes.c_int
            lib.orc_simplify.argtypes = [ctypes.POINTER(_Graph), ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.POINTER(_Simple))]
            lib.orc_simple_free.restype = None
            lib.orc_simple_free.argtypes = [ctypes.POINTER(_Simple)]
            lib.orc_range_free.restype = None
            lib.orc_range_free.argtypes = [ctypes.POINTER(_Range)]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with oracle status {code}")
        self.code = code


def _as_reads(reads, lengths):
    if isinstance(reads, (bytes, bytearray)):
        reads = np.frombuffer(bytes(reads), dtype=np.uint8)
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    return reads, lengths


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def _key_words(words: np.ndarray) -> list[int]:
    """(high, low) word pairs -> Python ints."""
    w = words.reshape(-1, 2)
    return [(int(h) << 64) | int(l) for h, l in w]


class OracleGraph:
    """Bi-directed de Bruijn graph computed by the oracle.

    Arrays: ``node_keys`` (n_nodes, 2) u64 high/low words of the canonical
    k-mer; ``edge_keys`` (n_edges, 2) canonical (k+1)-mer; ``src``/``dst``
    node IDs; ``orient`` = (o1 << 1) | o2; ``mult``; CSR ``row_ptr``,
    ``adj_nbr``, ``adj_edge``, ``adj_role``.
    """

    def __init__(self, ptr):
        self._ptr = ptr
        g = ptr.contents
        self.k = int(g.k)
        self.n_nodes = int(g.n_nodes)
        self.n_edges = int(g.n_edges)
        nv, ne = self.n_nodes, self.n_edges
        self.node_keys = _copy(g.node_keys, 2 * nv, np.uint64).reshape(nv, 2)
        self.edge_keys = _copy(g.edge_keys, 2 * ne, np.uint64).reshape(ne, 2)
        self.src = _copy(g.src, ne, np.uint32)
        self.dst = _copy(g.dst, ne, np.uint32)
        self.orient = _copy(g.orient, ne, np.uint8)
        self.mult = _copy(g.mult, ne, np.uint32)
        self.row_ptr = _copy(g.row_ptr, nv + 1, np.uint64)
        self.adj_nbr = _copy(g.adj_nbr, 2 * ne, np.uint32)
        self.adj_edge = _copy(g.adj_edge, 2 * ne, np.uint32)
        self.adj_role = _copy(g.adj_role, 2 * ne, np.uint8)
        self.flags = int(g.flags)

    def node_ints(self) -> list[int]:
        return _key_words(self.node_keys)

    def edge_ints(self) -> list[int]:
        return _key_words(self.edge_keys)

    def __del__(self):
        ptr, self._ptr = getattr(self, "_ptr", None), None
        if ptr is not None and _lib is not None:
            _lib.orc_graph_free(ptr)


class OracleUnitigs:
    def __init__(self, ptr, k):
        u = ptr.contents
        self.count = int(u.count)
        self.node_off = _copy(u.node_off, self.count + 1, np.uint64)
        n_nodes = int(self.node_off[-1]) if self.count else 0
        self.nodes = _copy(u.nodes, n_nodes, np.uint64)
        self.seq_off = _copy(u.seq_off, self.count + 1, np.uint64)
        n_seq = int(self.seq_off[-1]) if self.count else 0
        self.seq = ctypes.string_at(u.seq, n_seq) if n_seq else b""
        self.circular = _copy(u.circular, self.count, np.uint8)
        self.k = k
        _lib.orc_unitigs_free(ptr)

    def strings(self) -> list[str]:
        return [self.seq[self.seq_off[i]:self.seq_off[i + 1]].decode()
                for i in range(self.count)]

    def node_lists(self) -> list[list[tuple[int, int]]]:
        out = []
        for i in range(self.count):
            seg = self.nodes[self.node_off[i]:self.node_off[i + 1]]
            out.append([(int(x) >> 1, int(x) & 1) for x in seg])
        return out


def build_graph(reads, lengths, k: int) -> OracleGraph:
    """Graph of the reads by the definitions of Section 2 (forward reads only)."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    out = ctypes.POINTER(_Graph)()
    rc = lib.orc_build(reads.ctypes.data, lengths.ctypes.data, len(lengths), k, ctypes.byref(out))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_build")
    return OracleGraph(out)


def compact(graph: OracleGraph) -> OracleUnitigs:
    """Unitigs of the graph by walking its mergeable chains (Section 6)."""
    lib = _load()
    out = ctypes.POINTER(_Unitigs)()
    rc = lib.orc_compact(graph._ptr, ctypes.byref(out))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_compact")
    return OracleUnitigs(out, graph.k)


def count_kplus1(reads, lengths, k: int, queries: list[str]) -> np.ndarray:
    """Multiplicity of the edge spelled by each query (k+1)-mer."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    q = "".join(queries).encode()
    if any(len(s) != k + 1 for s in queries):
        raise ValueError("queries must be (k+1)-mers")
    qbuf = np.frombuffer(q, dtype=np.uint8) if q else np.zeros(1, np.uint8)
    counts = np.zeros(max(1, len(queries)), dtype=np.uint64)
    rc = lib.orc_count_kplus1(reads.ctypes.data, lengths.ctypes.data, len(lengths), k,
                              qbuf.ctypes.data, len(queries), counts.ctypes.data)
    if rc != ORC_OK:
        raise OracleError(rc, "orc_count_kplus1")
    return counts[:len(queries)]


def edges_in_partition(reads, lengths, k: int, part: int, parts: int) -> tuple[int, int]:
    """(distinct edges, edge instances) of partition `part` of `parts` of the
    edges (partitioned by a hash of the canonical (k+1)-mer), counted over all
    reads: the unit of work of the multi-core CPU baseline."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    d = ctypes.c_uint64(0)
    i = ctypes.c_uint64(0)
    rc = lib.orc_edges_in_partition(reads.ctypes.data, lengths.ctypes.data, len(lengths), k, part, parts,
                                    ctypes.byref(d), ctypes.byref(i))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_edges_in_partition")
    return int(d.value), int(i.value)


def node_multiplicities(reads, lengths, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Canonical k-mers of the forward reads (the nodes of Section 2) in
    ascending order as (n, 2) high/low u64 words, and how many positions of
    the forward reads hold each of them or its reverse complement."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    m = ctypes.c_uint64(0)
    kp, cp = ctypes.POINTER(ctypes.c_uint64)(), ctypes.POINTER(ctypes.c_uint64)()
    rc = lib.orc_node_mult(reads.ctypes.data, lengths.ctypes.data, len(lengths), k, ctypes.byref(m),
                           ctypes.byref(kp), ctypes.byref(cp))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_node_mult")
    try:
        keys = _copy(kp, 2 * m.value, np.uint64).reshape(-1, 2)
        counts = _copy(cp, m.value, np.uint64)
    finally:
        lib.orc_free(ctypes.cast(kp, ctypes.c_void_p))
        lib.orc_free(ctypes.cast(cp, ctypes.c_void_p))
    return keys, counts


def _bound_words(v: int) -> np.ndarray:
    if not 0 <= v < (1 << 128):
        raise ValueError("key bound out of range")
    return np.array([v >> 64, v & ((1 << 64) - 1)], dtype=np.uint64)


def graph_range(reads, lengths, k: int, edge_range: tuple[int, int],
                node_range: tuple[int, int]) -> dict:
    """The slice of the oracle graph whose keys lie in the given inclusive
    ranges: edges with lo <= canonical (k+1)-mer <= hi, ascending, each with
    the keys of its src and dst nodes, its orientation and multiplicity; and
    the nodes (canonical k-mers) with lo <= key <= hi, ascending.  Keys are
    (n, 2) high/low u64 words.  Concatenating the slices of consecutive
    ranges gives the node and edge lists of ``build_graph``."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    b = [_bound_words(x) for x in (*edge_range, *node_range)]
    out = ctypes.POINTER(_Range)()
    rc = lib.orc_graph_range(reads.ctypes.data, lengths.ctypes.data, len(lengths), k,
                             b[0].ctypes.data, b[1].ctypes.data, b[2].ctypes.data, b[3].ctypes.data,
                             ctypes.byref(out))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_graph_range")
    try:
        r = out.contents
        ne, nv = int(r.n_edges), int(r.n_nodes)
        res = {
            "edge_keys": _copy(r.edge_keys, 2 * ne, np.uint64).reshape(ne, 2),
            "src_keys": _copy(r.src_keys, 2 * ne, np.uint64).reshape(ne, 2),
            "dst_keys": _copy(r.dst_keys, 2 * ne, np.uint64).reshape(ne, 2),
            "orient": _copy(r.orient, ne, np.uint8),
            "mult": _copy(r.mult, ne, np.uint64),
            "node_keys": _copy(r.node_keys, 2 * nv, np.uint64).reshape(nv, 2),
        }
    finally:
        lib.orc_range_free(out)
    return res


def node_reads(reads, lengths, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Canonical k-mers of the forward reads (the nodes) in ascending order
    as (n, 2) high/low u64 words, and how many distinct reads contain each
    of them on either strand (VELVET's roadmap keeps those in >= 2 reads)."""
    lib = _load()
    reads, lengths = _as_reads(reads, lengths)
    m = ctypes.c_uint64(0)
    kp, cp = ctypes.POINTER(ctypes.c_uint64)(), ctypes.POINTER(ctypes.c_uint64)()
    rc = lib.orc_node_reads(reads.ctypes.data, lengths.ctypes.data, len(lengths), k, ctypes.byref(m),
                            ctypes.byref(kp), ctypes.byref(cp))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_node_reads")
    try:
        keys = _copy(kp, 2 * m.value, np.uint64).reshape(-1, 2)
        counts = _copy(cp, m.value, np.uint64)
    finally:
        lib.orc_free(ctypes.cast(kp, ctypes.c_void_p))
        lib.orc_free(ctypes.cast(cp, ctypes.c_void_p))
    return keys, counts


class OracleSimple:
    """The simplified graph (Section 6 / 6.1): units (reported chains and
    single nodes) as node lists and strings, and the edges between units."""

    def __init__(self, ptr, k):
        r = ptr.contents
        self.k = k
        self.n_units, self.n_edges, self.removed = int(r.n_units), int(r.n_edges), int(r.removed)
        U, M = self.n_units, self.n_edges
        self.node_off = _copy(r.node_off, U + 1, np.uint64)
        self.nodes = _copy(r.nodes, int(self.node_off[-1]) if U else 0, np.uint64)
        self.seq_off = _copy(r.seq_off, U + 1, np.uint64)
        n_seq = int(self.seq_off[-1]) if U else 0
        self.seq = ctypes.string_at(r.seq, n_seq) if n_seq else b""
        self.circular = _copy(r.circular, U, np.uint8)
        self.unit_a = _copy(r.unit_a, M, np.uint32)
        self.unit_b = _copy(r.unit_b, M, np.uint32)
        self.side_a = _copy(r.side_a, M, np.uint8)
        self.side_b = _copy(r.side_b, M, np.uint8)
        self.edge = _copy(r.edge, M, np.uint32)
        _lib.orc_simple_free(ptr)

    def strings(self) -> list[str]:
        return [self.seq[self.seq_off[i]:self.seq_off[i + 1]].decode() for i in range(self.n_units)]


def simplify(graph: OracleGraph, min_nodes: int = 3) -> OracleSimple:
    """The simplified graph with chains of at least min_nodes nodes merged."""
    lib = _load()
    out = ctypes.POINTER(_Simple)()
    rc = lib.orc_simplify(graph._ptr, min_nodes, ctypes.byref(out))
    if rc != ORC_OK:
        raise OracleError(rc, "orc_simplify")
    return OracleSimple(out, graph.k)
