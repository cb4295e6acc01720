"""Roadmap counts (dbg_node_reads_set): for every node, the number of
distinct reads holding its k-mer on either strand, counted on the GPU by a
sort of (k-mer, read) records, equal the oracle's element by element in node
order; dbg_roadmap_nodes lists the nodes held by at least t reads (VELVET's
roadmap keeps those in at least 2 reads, Section 7)."""
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
    cnt = dbg.dbg_graph_node_reads(g)
    keys, want = oracle.node_reads(reads, lengths, k)
    np.testing.assert_array_equal(got["nodes"], oracle_words(keys, got["W"]))
    np.testing.assert_array_equal(cnt.astype(np.uint64), want)
    for t in (1, 2, 3):
        np.testing.assert_array_equal(dbg.dbg_roadmap_nodes(ctx, g, t), np.nonzero(want >= t)[0].astype(np.uint32))
    return cnt


@pytest.mark.parametrize("k,n_reads,L", [(15, 20_000, 60), (21, 30_000, 100), (31, 40_000, 100),
                                         (33, 15_000, 120), (55, 12_000, 150), (63, 8_000, 150)])
def test_node_reads_match_oracle(dbg, k, n_reads, L):
    rng = np.random.default_rng(960 + k)
    reads, lengths = readgen.generate(readgen.ReadSetSpec(200_000, n_reads, L, 0.01, k, 960 + k))
    reads, lengths = with_short_reads(reads, lengths, k, rng)
    ctx = dbg.Context()
    dbg.dbg_node_reads_set(ctx, True)
    cnt = check(dbg, ctx, reads, lengths, k)
    assert int((cnt >= 2).sum()) > 0 and int((cnt == 1).sum()) > 0


@pytest.mark.parametrize("k", [1, 3, 5, 7])
@pytest.mark.parametrize("hybrid", [True, False])
def test_node_reads_small_k_and_repeats(dbg, k, hybrid):
    """Short random reads over a two-letter alphabet: k-mers repeat inside
    a read (counted once per read) and across reads; hybrid and all-global
    record sorts."""
    rng = np.random.default_rng(970 + k)
    reads, lengths = readgen.random_reads(rng, 4_000, 0, 3 * k + 10, b"AC")
    ctx = dbg.Context()
    dbg.dbg_node_reads_set(ctx, True)
    dbg.dbg_sort_hybrid_set(ctx, hybrid)
    check(dbg, ctx, reads, lengths, k)


def test_node_reads_with_multiplicities_and_off(dbg):
    """Both counts in one build; the read counts never exceed the
    occurrences; with the switch off there are none and the graph is the
    same."""
    k = 21
    reads, lengths = readgen.generate(readgen.ReadSetSpec(50_000, 20_000, 80, 0.01, k, 975))
    ctx = dbg.Context()
    dbg.dbg_node_reads_set(ctx, True)
    dbg.dbg_node_mult_set(ctx, True)
    g, with_counts = gpu_graph(dbg, ctx, reads, lengths, k)
    r, m = dbg.dbg_graph_node_reads(g), dbg.dbg_graph_node_mult(g)
    assert bool((r <= m).all()) and bool((r >= 1).all())
    dbg.dbg_node_reads_set(ctx, False)
    dbg.dbg_node_mult_set(ctx, False)
    g2, without = gpu_graph(dbg, ctx, reads, lengths, k)
    with pytest.raises(RuntimeError):
        dbg.dbg_graph_node_reads(g2)
    for key in with_counts:
        if isinstance(with_counts[key], np.ndarray):
            np.testing.assert_array_equal(with_counts[key], without[key], err_msg=key)
