"""Element-by-element parity of a built graph against the oracle at sizes the
oracle cannot build in one piece.

The canonical key spaces (edges: 2(k+1) bits, nodes: 2k bits) are cut into
ranges.  One process per range scans every read and keeps only the edges and
nodes whose keys fall in its range (``oracle.graph_range``); the ranges cover
both key spaces, so together the processes compare every node and every edge
of the graph: edge keys, the keys of both end nodes (through the library's
src / dst IDs), orientation and multiplicity, and the node keys.  Since node
IDs are ranks of the node keys, equal node lists make the IDs equal too.

The processes are started with ``spawn`` (safe after CUDA use) and read the
reads and the library's result arrays from memory-mapped .npy files.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

import oracle


def first_base_cuts(bits: int, parts: int) -> list[int]:
    """parts + 1 cut points of a `bits`-bit canonical key space, spaced so
    that the ranges hold roughly equally many keys.  For uniform random
    sequence the canonical form min(z, rc z) starts with A, C, G, T with
    probability 7, 5, 3, 1 in 16 (its first base is the smaller of z's first
    base and the complement of z's last), so the four first-base quarters of
    the key space get parts in those proportions, each cut evenly.  Only the
    balance between processes depends on this; the cuts always cover the
    whole space."""
    if bits < 8 or parts < 4:
        return [0, 1 << bits]
    weights = np.array([7, 5, 3, 1], dtype=np.float64)
    share = [int(x) for x in np.maximum(1, np.round(weights / weights.sum() * parts))]
    quarter = 1 << (bits - 2)
    cuts = [0]
    for b in range(4):
        for i in range(1, share[b] + 1):
            cuts.append(b * quarter + (quarter * i) // share[b])
    assert cuts[-1] == 1 << bits
    return cuts


def key_slice(words: np.ndarray, lo: int, hi: int) -> tuple[int, int]:
    """[a, b): the rows of ascending (n, W) key words with lo <= key <= hi."""
    if words.shape[1] == 1:
        col = words[:, 0]
        return int(np.searchsorted(col, np.uint64(lo), "left")), int(np.searchsorted(col, np.uint64(hi), "right"))

    def bound(v: int, side: str) -> int:
        h, l = np.uint64(v >> 64), np.uint64(v & ((1 << 64) - 1))
        a = int(np.searchsorted(words[:, 0], h, "left"))
        b = int(np.searchsorted(words[:, 0], h, "right"))
        return a + int(np.searchsorted(words[a:b, 1], l, side))

    return bound(lo, "left"), bound(hi, "right")


def _oracle_words(pairs: np.ndarray, W: int) -> np.ndarray:
    if W == 1:
        return pairs[:, 1:2]
    return pairs


def _first_diff(name: str, got: np.ndarray, want: np.ndarray, at: int):
    if got.shape != want.shape:
        return f"{name}: {got.shape[0]} rows from the library, {want.shape[0]} from the oracle (range start {at})"
    bad = np.nonzero((got != want).reshape(got.shape[0], -1).any(axis=1))[0]
    if bad.size:
        i = int(bad[0])
        return f"{name}: {bad.size} rows differ, first at {at + i}: library {got[i]} oracle {want[i]}"
    return None


def _worker(job):
    d, k, W, erange, nrange = job
    ld = lambda name: np.load(os.path.join(d, name + ".npy"), mmap_mode="r")
    s = oracle.graph_range(ld("reads"), ld("lengths"), k, erange, nrange)
    ek, nk = ld("edge_keys"), ld("node_keys")
    errors = []
    a, b = key_slice(ek, *erange)
    src, dst = np.asarray(ld("src")[a:b]), np.asarray(ld("dst")[a:b])
    checks = [("edge keys", np.asarray(ek[a:b]), _oracle_words(s["edge_keys"], W))]
    if b > a and max(int(src.max()), int(dst.max())) >= nk.shape[0]:
        errors.append(f"edges {a}..{b}: node IDs beyond the {nk.shape[0]} nodes")
    elif b - a == len(s["mult"]):
        checks += [
            ("src node keys", np.asarray(nk[src]), _oracle_words(s["src_keys"], W)),
            ("dst node keys", np.asarray(nk[dst]), _oracle_words(s["dst_keys"], W)),
            ("orient", np.asarray(ld("orient")[a:b]), s["orient"]),
            ("mult", np.asarray(ld("mult")[a:b]).astype(np.uint64), s["mult"]),
        ]
    na, nb = key_slice(nk, *nrange)
    checks.append(("node keys", np.asarray(nk[na:nb]), _oracle_words(s["node_keys"], W)))
    for name, got, want in checks:
        msg = _first_diff(name, got, want, na if name == "node keys" else a)
        if msg:
            errors.append(msg)
    return b - a, nb - na, errors


def _save_case(d: str, arrays: dict, reads, lengths) -> int:
    os.makedirs(d, exist_ok=True)
    W = arrays["edge_keys"].shape[1] if arrays["edge_keys"].ndim == 2 else 1
    np.save(os.path.join(d, "reads.npy"), np.ascontiguousarray(reads, dtype=np.uint8))
    np.save(os.path.join(d, "lengths.npy"), np.ascontiguousarray(lengths, dtype=np.uint32))
    for name in ("edge_keys", "node_keys"):
        np.save(os.path.join(d, name + ".npy"), np.ascontiguousarray(arrays[name]).reshape(-1, W))
    for name in ("src", "dst", "orient", "mult"):
        np.save(os.path.join(d, name + ".npy"), np.ascontiguousarray(arrays[name]))
    return W


def _jobs(d: str, k: int, W: int, parts: int) -> list:
    ecuts = first_base_cuts(2 * (k + 1), parts)
    ncuts = first_base_cuts(2 * k, parts)
    m = max(len(ecuts), len(ncuts)) - 1
    ranges_e = [(ecuts[i], ecuts[i + 1] - 1) if i + 1 < len(ecuts) else (1, 0) for i in range(m)]
    ranges_n = [(ncuts[i], ncuts[i + 1] - 1) if i + 1 < len(ncuts) else (1, 0) for i in range(m)]
    return [(d, k, W, re, rn) for re, rn in zip(ranges_e, ranges_n)]


def compare_cases(cases: list, procs: int | None = None, tmp_dir: str | None = None) -> list:
    """Compares several graphs with the oracle, range by range, in one pool.

    cases: (arrays, reads, lengths, k, parts) tuples; arrays are host copies
    of a graph -- ``edge_keys`` and ``node_keys`` as (n, W) uint64 words,
    ``src``, ``dst``, ``orient``, ``mult``.  Raises AssertionError listing
    the first differences.  Returns the totals per case."""
    procs = procs or len(os.sched_getaffinity(0)) or 1
    with tempfile.TemporaryDirectory(dir=tmp_dir) as root:
        jobs, owner = [], []
        for c, (arrays, reads, lengths, k, parts) in enumerate(cases):
            d = os.path.join(root, f"case{c}")
            W = _save_case(d, arrays, reads, lengths)
            js = _jobs(d, k, W, parts)
            jobs += js
            owner += [c] * len(js)
        # the largest cases first, so that no process is left with one at the end
        order = sorted(range(len(jobs)), key=lambda j: -len(cases[owner[j]][2]))
        if procs == 1 or len(jobs) == 1:
            res = [_worker(jobs[j]) for j in order]
        else:
            with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
                res = pool.map(_worker, [jobs[j] for j in order], chunksize=1)
    out = []
    for c, (arrays, reads, lengths, k, parts) in enumerate(cases):
        mine = [r for j, r in zip(order, res) if owner[j] == c]
        errors = [e for r in mine for e in r[2]]
        assert not errors, f"case {c} (k = {k}):\n" + "\n".join(errors[:20])
        E, V = arrays["edge_keys"].shape[0], arrays["node_keys"].shape[0]
        ne, nv = sum(r[0] for r in mine), sum(r[1] for r in mine)
        assert ne == E, f"case {c}: the key ranges hold {ne} of the library's {E} edges"
        assert nv == V, f"case {c}: the key ranges hold {nv} of the library's {V} nodes"
        out.append({"edges": ne, "nodes": nv, "ranges": len(mine), "processes": procs})
    return out


def compare_by_ranges(arrays: dict, reads: np.ndarray, lengths: np.ndarray, k: int, parts: int = 64,
                      procs: int | None = None, tmp_dir: str | None = None) -> dict:
    """compare_cases for one graph."""
    return compare_cases([(arrays, reads, lengths, k, parts)], procs, tmp_dir)[0]
