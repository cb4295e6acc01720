"""Node multiplicities (dbg_node_mult_set): every node's k-mer occurrences
over the forward reads, counted on the GPU by an extra k-mer sort, equal
the oracle's count element by element, in node order."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import gpu_graph, oracle_words
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_1940_gb300 import dbg as d
    d.load()
    return d


def with_short_reads(reads, lengths, k, rng):
    """Adds reads shorter than k and of exactly k bases."""
    extra = [int(x) for x in rng.integers(0, k, size=50)] + [k] * 50
    bases = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=sum(extra))]
    return np.concatenate([reads, bases]), np.concatenate([lengths, np.array(extra, dtype=np.uint32)])


def check(dbg, ctx, reads, lengths, k):
    g, got = gpu_graph(dbg, ctx, reads, lengths, k)
    mult = dbg.dbg_graph_node_mult(g)
    keys, counts = oracle.node_multiplicities(reads, lengths, k)
    np.testing.assert_array_equal(got["nodes"], oracle_words(keys, got["W"]))
    np.testing.assert_array_equal(mult.astype(np.uint64), counts)
    assert int(mult.sum()) == int(np.maximum(lengths.astype(np.int64) - k + 1, 0).sum())
    return mult


@pytest.mark.parametrize("k,n_reads,L", [(15, 20_000, 60), (21, 30_000, 100), (31, 40_000, 100),
                                         (33, 15_000, 120), (55, 12_000, 150), (63, 8_000, 150)])
def test_node_multiplicities_match_oracle(dbg, k, n_reads, L):
    rng = np.random.default_rng(900 + k)
    reads, lengths = readgen.generate(readgen.ReadSetSpec(200_000, n_reads, L, 0.01, k, 900 + k))
    reads, lengths = with_short_reads(reads, lengths, k, rng)
    ctx = dbg.Context()
    dbg.dbg_node_mult_set(ctx, True)
    check(dbg, ctx, reads, lengths, k)


def test_node_multiplicities_global_sort_and_off(dbg):
    """Every digit sorted globally gives the same counts; a graph built with
    the switch off has none, and its edges are unchanged."""
    k = 21
    rng = np.random.default_rng(77)
    reads, lengths = readgen.generate(readgen.ReadSetSpec(100_000, 10_000, 90, 0.01, k, 77))
    reads, lengths = with_short_reads(reads, lengths, k, rng)
    ctx = dbg.Context()
    dbg.dbg_node_mult_set(ctx, True)
    dbg.dbg_sort_hybrid_set(ctx, False)
    a = check(dbg, ctx, reads, lengths, k)
    dbg.dbg_sort_hybrid_set(ctx, True)
    b = check(dbg, ctx, reads, lengths, k)
    np.testing.assert_array_equal(a, b)
    _, with_counts = gpu_graph(dbg, ctx, reads, lengths, k)
    dbg.dbg_node_mult_set(ctx, False)
    g, without = gpu_graph(dbg, ctx, reads, lengths, k)
    with pytest.raises(RuntimeError):
        dbg.dbg_graph_node_mult(g)
    for key in with_counts:
        if isinstance(with_counts[key], np.ndarray):
            np.testing.assert_array_equal(with_counts[key], without[key], err_msg=key)


@pytest.mark.parametrize("k", [1, 3, 5])
@pytest.mark.parametrize("hybrid", [True, False])
def test_node_multiplicities_smallest_k(dbg, k, hybrid):
    """The smallest k: the k-mer windows are emitted by the edge-key kernel
    run with k - 1 (0, 2 or 4 bases of overlap), on short random reads of
    lengths 0 .. 12, with the hybrid and the all-global sort."""
    rng = np.random.default_rng(950 + k)
    reads, lengths = readgen.random_reads(rng, 3_000, 0, 12)
    ctx = dbg.Context()
    dbg.dbg_node_mult_set(ctx, True)
    dbg.dbg_sort_hybrid_set(ctx, hybrid)
    check(dbg, ctx, reads, lengths, k)
