"""The hybrid sort (global passes over the high digits, then a local sort of
group-aligned tiles in shared memory, fused with the run-length reduce for the
edge keys) gives bit-for-bit the graph of the all-global sort and the oracle's,
including when a group is too long for a tile and is sorted globally."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_graph_equal, check_parity, gpu_graph
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_1940_gb300 import dbg as d
    d.load()
    return d


def same(a: dict, b: dict):
    assert a.keys() == b.keys()
    for key in a:
        if isinstance(a[key], np.ndarray):
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)
        else:
            assert a[key] == b[key], key


@pytest.mark.parametrize("k,n_reads,L", [(15, 20_000, 60), (21, 30_000, 100), (31, 40_000, 100),
                                         (33, 15_000, 120), (55, 12_000, 150), (63, 8_000, 150)])
def test_hybrid_equals_global_sort(dbg, k, n_reads, L):
    """Hundreds of local tiles with a ragged last one, for every key width."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(200_000, n_reads, L, 0.01, k, 500 + k))
    lengths = lengths.copy()
    lengths[-1] = L - 7  # a ragged tail
    reads = reads[:int(lengths.sum())]
    ctx = dbg.Context()
    _, hyb = gpu_graph(dbg, ctx, reads, lengths, k)
    assert dbg.dbg_sort_fallbacks(ctx) == 0
    dbg.dbg_sort_hybrid_set(ctx, False)
    _, glob = gpu_graph(dbg, ctx, reads, lengths, k)
    same(hyb, glob)
    assert_graph_equal(hyb, oracle.build_graph(reads, lengths, k))


def test_group_longer_than_window_falls_back(dbg):
    """10,000 copies of one (k+1)-mer form a group longer than a tile can
    hold (6,144 keys): that tile is gathered and sorted over every digit."""
    k = 21
    rng = np.random.default_rng(7)
    rep = "".join("ACGT"[c] for c in rng.integers(0, 4, size=k + 1))
    reads, lengths = readgen.generate(readgen.ReadSetSpec(50_000, 2_000, 60, 0.01, k, 71))
    reads = np.concatenate([reads, np.frombuffer((rep * 10_000).encode(), dtype=np.uint8)])
    lengths = np.concatenate([lengths, np.full(10_000, k + 1, dtype=np.uint32)])
    ctx = dbg.Context()
    got = check_parity(dbg, ctx, reads, lengths, k)
    assert dbg.dbg_sort_fallbacks(ctx) >= 1
    assert got["e_mult"].max() >= 10_000


def test_node_records_fall_back(dbg):
    """8,000 reads of exactly k bases that share their first seven: 8,000
    node records with equal high bits, a group longer than a tile of the
    node-record sort can hold, which is gathered and sorted globally; plus
    ordinary reads."""
    k = 15
    rng = np.random.default_rng(8)
    tails = rng.integers(0, 4, size=(8_000, k - 7))
    reads = ["AAAAAAA" + "".join("ACGT"[c] for c in t) for t in tails]
    r2, l2 = readgen.generate(readgen.ReadSetSpec(20_000, 300, 50, 0.01, k, 81))
    data = np.concatenate([np.frombuffer("".join(reads).encode(), dtype=np.uint8), r2])
    lengths = np.concatenate([np.full(8_000, k, dtype=np.uint32), l2])
    ctx = dbg.Context()
    check_parity(dbg, ctx, data, lengths, k)
    assert dbg.dbg_sort_fallbacks(ctx) >= 1


def test_long_runs_in_first_and_last_tiles(dbg):
    """Runs of 10,000 equal keys at the very start (AAA...A, the smallest
    key) and near the end of the key order (GCC...C), with ordinary reads in
    between: oversize tiles at both ends and normal tiles in the middle."""
    k = 31
    first = "A" * (k + 1)
    last = "G" + "C" * k
    reads, lengths = readgen.generate(readgen.ReadSetSpec(100_000, 3_000, 100, 0.01, k, 91))
    extra = (first * 10_000 + last * 10_000).encode()
    reads = np.concatenate([reads, np.frombuffer(extra, dtype=np.uint8)])
    lengths = np.concatenate([lengths, np.full(20_000, k + 1, dtype=np.uint32)])
    ctx = dbg.Context()
    got = check_parity(dbg, ctx, reads, lengths, k)
    assert dbg.dbg_sort_fallbacks(ctx) >= 1
    assert got["e_mult"][0] >= 10_000 and got["e_mult"].max() >= 10_000


@pytest.mark.parametrize("k,genome,n_reads,L", [(31, 40_000_000, 6_000, 100), (27, 300_000, 40_000, 90),
                                                (15, 20_000, 20_000, 40), (55, 40_000_000, 4_000, 150),
                                                (47, 300_000, 20_000, 120), (63, 100_000, 6_000, 150)])
def test_count_first_equals_sorted_runs(dbg, k, genome, n_reads, L):
    """Counting each tile's copies in a hash table and sorting the distinct
    keys gives the edge list of sorting every copy: at coverage ~0.015 (almost
    every key distinct: every tile overflows its table and is sorted copy by
    copy), ~12 (some tiles near the table's limit) and ~40 (none)."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(genome, n_reads, L, 0.01, k, 600 + k))
    ctx = dbg.Context()
    _, counted = gpu_graph(dbg, ctx, reads, lengths, k)
    over = dbg.dbg_sort_count_overflows(ctx)
    if n_reads * L * 10 < genome:  # coverage below 0.1
        assert over > 0
    if k == 15:
        assert over == 0
    dbg.dbg_sort_count_first_set(ctx, False)
    _, runs = gpu_graph(dbg, ctx, reads, lengths, k)
    same(counted, runs)
    assert_graph_equal(counted, oracle.build_graph(reads, lengths, k))


def test_count_first_one_key_many_copies(dbg):
    """3,000 copies of one (k+1)-mer (fewer than a tile holds) among
    ordinary reads: one hash slot takes every copy."""
    k = 31
    rng = np.random.default_rng(9)
    rep = "".join("ACGT"[c] for c in rng.integers(0, 4, size=k + 1))
    reads, lengths = readgen.generate(readgen.ReadSetSpec(100_000, 4_000, 100, 0.01, k, 92))
    reads = np.concatenate([reads, np.frombuffer((rep * 3_000).encode(), dtype=np.uint8)])
    lengths = np.concatenate([lengths, np.full(3_000, k + 1, dtype=np.uint32)])
    ctx = dbg.Context()
    got = check_parity(dbg, ctx, reads, lengths, k)
    assert got["e_mult"].max() >= 3_000


@pytest.mark.parametrize("k,hybrid", [(21, True), (31, True), (31, False), (55, True), (63, False)])
def test_partition_first_equals_stable_first_pass(dbg, k, hybrid):
    """The first global pass of the edge keys as an unordered partition gives
    the graph of a stable first pass, with the hybrid sort and with every
    digit sorted globally, for 64- and 128-bit keys."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(150_000, 12_000, 120, 0.01, k, 700 + k))
    ctx = dbg.Context()
    dbg.dbg_sort_hybrid_set(ctx, hybrid)
    _, part = gpu_graph(dbg, ctx, reads, lengths, k)
    dbg.dbg_sort_partition_first_set(ctx, False)
    _, stable = gpu_graph(dbg, ctx, reads, lengths, k)
    same(part, stable)
    assert_graph_equal(part, oracle.build_graph(reads, lengths, k))


@pytest.mark.parametrize("k,n_reads,L", [(21, 30_000, 100), (31, 40_000, 100), (55, 12_000, 150)])
def test_local_sort_variants_identical(dbg, k, n_reads, L):
    """Every local ranking method, in the 256-thread and the wide (384-
    thread) form of the node records' local sort (the digit passes: ranking
    within groups switched off), gives the same graph, and the oracle's; a
    group longer than a tile is in the input too."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(200_000, n_reads, L, 0.01, k, 600 + k))
    rep = "ACGTTGCA" * 40
    reads = np.concatenate([reads, np.frombuffer((rep[:k + 3] * 7_000).encode(), dtype=np.uint8)])
    lengths = np.concatenate([lengths, np.full(7_000, k + 3, dtype=np.uint32)])
    kind = 5 if k > 31 else 4
    ref = None
    for v in range(dbg.dbg_sort_variant_count(kind)):
        ctx = dbg.Context()
        dbg.dbg_sort_local_rank_set(ctx, False)
        dbg.dbg_sort_variant_set(ctx, kind, v)
        _, got = gpu_graph(dbg, ctx, reads, lengths, k)
        if ref is None:
            ref = got
            assert_graph_equal(got, oracle.build_graph(reads, lengths, k))
        else:
            same(got, ref)
