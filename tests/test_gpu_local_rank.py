"""The local passes by ranking within groups (each key placed at its group's
start plus the number of the group's keys before it) give bit for bit the
graph of the shared-memory digit passes and the oracle's: for node keys of
both widths modulo 8 bits (the record sort aligns its digits with the top of
the 2k-bit key), with groups long enough to send their tile to the digit
passes, and with a group longer than a tile."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_graph_equal, gpu_graph
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


def both_ways(dbg, reads, lengths, k, with_oracle=True):
    ctx = dbg.Context()
    _, ranked = gpu_graph(dbg, ctx, reads, lengths, k)
    # tiles sent to the digit passes, and tiles too long for any local pass
    # (gathered and sorted globally)
    fallbacks = dbg.dbg_sort_rank_fallbacks(ctx) + dbg.dbg_sort_fallbacks(ctx)
    ctx2 = dbg.Context()
    dbg.dbg_sort_local_rank_set(ctx2, False)
    _, digits = gpu_graph(dbg, ctx2, reads, lengths, k)
    assert dbg.dbg_sort_rank_fallbacks(ctx2) == 0
    same(ranked, digits)
    if with_oracle:
        assert_graph_equal(ranked, oracle.build_graph(reads, lengths, k))
    return ranked, fallbacks


@pytest.mark.parametrize("k", [9, 13, 21, 23, 25, 27, 29, 31, 33, 35, 45, 55, 63])
def test_ranked_equals_digit_passes(dbg, k):
    """2k mod 8 = 2 and 6 (digit alignment 6 and 2; k is odd), for 64- and
    128-bit keys."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(300_000, 30_000, 100, 0.01, k, 900 + k))
    lengths = lengths.copy()
    lengths[-1] = 100 - 9  # a ragged tail
    reads = reads[:int(lengths.sum())]
    _, fb = both_ways(dbg, reads, lengths, k)
    if k >= 21:
        assert fb == 0


def group_reads(prefix: str, n: int, k: int, seed: int):
    """n reads of length k + 1 whose first k-mer starts with `prefix` (and is
    canonical: the prefix is all A and no read ends in as many T): n distinct
    k-mers and n distinct edge keys sharing their high bits."""
    rng = np.random.default_rng(seed)
    tail = rng.integers(0, 3, size=(n, k + 1 - len(prefix)))  # A, C, G only
    body = np.array([ord(c) for c in "ACG"], dtype=np.uint8)[tail]
    head = np.frombuffer(prefix.encode(), dtype=np.uint8)
    reads = np.concatenate([np.broadcast_to(head, (n, len(prefix))), body], axis=1).reshape(-1)
    return np.ascontiguousarray(reads), np.full(n, k + 1, dtype=np.uint32)


@pytest.mark.parametrize("k", [31, 55])
@pytest.mark.parametrize("n_group,expect_fallback", [(200, False), (400, True), (2_000, True)])
def test_long_groups(dbg, k, n_group, expect_fallback):
    """Background reads plus n_group distinct k-mers with one 12-base
    prefix: a group of that many edge keys (the count pass ranks up to 256
    distinct keys in a group) and node records (the record pass ranks
    groups of up to 512), for 64- and 128-bit keys; longer groups send their
    tile to the digit passes, or, longer than a tile holds (3072 128-bit
    records), to the global sort."""
    bg, bl = readgen.generate(readgen.ReadSetSpec(200_000, 20_000, 100 if k < 33 else 150, 0.01, k, 77))
    gr, gl = group_reads("A" * 12, n_group, k, 78)
    reads = np.concatenate([bg, gr])
    lengths = np.concatenate([bl, gl])
    _, fb = both_ways(dbg, reads, lengths, k)
    if expect_fallback:
        assert fb >= 1
    else:
        assert fb == 0


def test_group_longer_than_tile_and_isolated_reads(dbg):
    """A group of 8,000 records (longer than a tile: gathered and sorted
    globally) next to ranked tiles, and reads of length exactly k (records
    without an edge) in many copies."""
    k = 27
    bg, bl = readgen.generate(readgen.ReadSetSpec(100_000, 10_000, 100, 0.01, k, 79))
    gr, gl = group_reads("A" * 12, 8_000, k, 80)
    iso = np.frombuffer(("ACGT" * 8)[:k].encode() * 500, dtype=np.uint8)
    reads = np.concatenate([bg, gr, iso])
    lengths = np.concatenate([bl, gl, np.full(500, k, dtype=np.uint32)])
    both_ways(dbg, reads, lengths, k)


def test_large_workload_slice_ranked(dbg):
    """A 1/20 slice of the large workload's recipe (0.75 M reads x 100 bp,
    k = 31): tens of thousands of ranked tiles, the same graph both ways."""
    reads, lengths = readgen.generate(readgen.large_spec(0.05))
    _, fb = both_ways(dbg, reads, lengths, 31, with_oracle=False)
    assert fb < 50
