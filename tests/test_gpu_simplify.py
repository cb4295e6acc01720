"""The simplified graph (dbg_simplify: Section 6.1's literal chain
compaction with the >= min_nodes filter, and Section 6's relabelled edges)
equals the oracle's element by element: units (node lists, strings,
circular flags) and edges (units and sides of both ends, edge IDs)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_1940_gb300 import dbg as d
    d.load()
    return d


def check(dbg, ctx, reads, lengths, k, min_nodes):
    g = dbg.dbg_build(ctx, reads, lengths, k)
    got = dbg.dbg_simple_get(dbg.dbg_simplify(ctx, g, min_nodes))
    want = oracle.simplify(oracle.build_graph(reads, lengths, k), min_nodes)
    for f in ("node_off", "nodes", "seq_off", "circular", "unit_a", "side_a", "unit_b", "side_b", "edge"):
        np.testing.assert_array_equal(got[f], getattr(want, f), err_msg=f)
    assert got["seq"] == want.seq
    assert got["removed"] == want.removed == 0
    return got


@pytest.mark.parametrize("k,min_nodes", [(21, 3), (31, 3), (31, 1), (31, 2), (33, 3), (55, 5)])
def test_simplify_matches_oracle(dbg, k, min_nodes):
    L = 100 if k < 33 else 150
    reads, lengths = readgen.generate(readgen.ReadSetSpec(60_000, 12_000, L, 0.005, k, 40 + k,
                                                          repeat_fraction=0.02))
    got = check(dbg, dbg.Context(), reads, lengths, k, min_nodes)
    assert len(got["circular"]) > 0 and len(got["edge"]) > 0


def test_simplify_long_chains_cycles_and_tiny(dbg):
    """A long unitig (the list-ranking path beyond the walk cap), a circular
    genome (one circular unit), reads too short for any edge, empty input."""
    ctx = dbg.Context()
    rng = np.random.default_rng(7)
    k = 31
    genome = readgen.ALPHABET[rng.integers(0, 4, size=9000)].tobytes().decode()
    reads = [genome[i:i + 100] for i in range(0, len(genome) - 100, 30)]
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    check(dbg, ctx, "".join(reads).encode(), lengths, k, 3)
    circ = genome[:3000] + genome[:k + 100]
    reads = [circ[i:i + 120] for i in range(0, 3000, 40)]
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    got = check(dbg, ctx, "".join(reads).encode(), lengths, k, 3)
    assert got["circular"].tolist() == [1]
    check(dbg, ctx, b"ACGTACGTAC", np.array([10], dtype=np.uint32), 11, 3)
    for mn in (1, 3):
        check(dbg, ctx, b"ACGTTGCATGGACCTTAGGA", np.array([20], dtype=np.uint32), 5, mn)
