"""dbg_compact_bucketed (the out-of-core list ranking of Section 6.2: sort-
join rounds over key ranges of host-resident ranking words) gives the same
unitigs as dbg_compact, array for array, and the oracle's: with budgets that
cut the strand-nodes into many key ranges, on lists, long lists and
cycles."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_unitigs_equal
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_1940_gb300 import dbg as d
    d.load()
    return d


def as_input(reads):
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    return "".join(reads).encode(), lengths


def check(dbg, ctx, reads, lengths, k, budgets, with_oracle=True):
    g = dbg.dbg_build(ctx, reads, lengths, k)
    want = dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, g))
    if with_oracle:
        assert_unitigs_equal(want, oracle.compact(oracle.build_graph(reads, lengths, k)))
    launches = []
    for b in budgets:
        u, n_join = dbg.dbg_compact_bucketed(ctx, g, b)
        got = dbg.dbg_unitigs_get(u)
        for f in ("node_off", "nodes", "seq_off", "circular"):
            np.testing.assert_array_equal(got[f], want[f], err_msg=f"{f} at budget {b}")
        assert got["seq"] == want["seq"]
        launches.append(n_join)
    return want, launches


@pytest.mark.parametrize("k", [21, 31, 33])
def test_bucketed_ranking_equals_in_core(dbg, k):
    L = 100 if k < 33 else 150
    reads, lengths = readgen.generate(readgen.ReadSetSpec(80_000, 20_000, L, 0.005, k, 70 + k,
                                                          repeat_fraction=0.02))
    _, launches = check(dbg, dbg.Context(), reads, lengths, k, [0, 1 << 20, 200_000])
    # smaller budgets cut the strand-nodes into more key ranges
    assert 0 < launches[0] < launches[1] <= launches[2]


def test_bucketed_ranking_long_lists_and_cycles(dbg):
    ctx = dbg.Context()
    rng = np.random.default_rng(99)
    gnm = rng.integers(0, 4, size=6_000 + 40).astype(np.uint8)
    reads = ["".join("ACGT"[c] for c in gnm[s:s + 100]) for s in range(0, 6_000, 40)]
    reads += ["ACACACACACACACACACACAC" * 2]  # a circular unitig
    circ = "".join("ACGT"[c] for c in rng.integers(0, 4, size=3000))
    circ2 = circ + circ[:60]
    reads += [circ2[i:i + 80] for i in range(0, 3000, 30)]  # a long cycle
    r, l = as_input(reads)
    want, launches = check(dbg, ctx, r, l, 21, [0, 300_000, 100_000])
    assert min(launches) > 0
    assert int(want["circular"].sum()) >= 2


def test_bucketed_ranking_low_complexity_and_tiny(dbg):
    ctx = dbg.Context()
    reads = ["A" * 50, "T" * 40, "ACACACACACACACACAC", "ACGT" * 10, "GATC" * 12,
             "AAAAACCCCCGGGGGTTTTT" * 3, "TGCA" * 9]
    for k in (1, 3, 5, 7, 11):
        r, l = as_input(reads)
        check(dbg, ctx, r, l, k, [0, 4096])
    r, l = as_input([])
    check(dbg, ctx, r, l, 21, [0])
    r, l = as_input(["ACGTACGTAACCGGTT"])
    check(dbg, ctx, r, l, 5, [0, 4096])


def test_bucketed_ranking_mid_size(dbg):
    """750 K reads of the large workload's recipe (52 M edge instances): the
    out-of-core ranking in 1 GB of device memory gives dbg_compact's unitigs."""
    import torch
    spec = readgen.large_spec(0.05)
    reads, lengths = readgen.generate(spec)
    ctx = dbg.Context()
    g = dbg.dbg_build(ctx, torch.from_numpy(reads).cuda(), torch.from_numpy(lengths.view(np.int32)).cuda(), 31)
    want = dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, g))
    u, launches = dbg.dbg_compact_bucketed(ctx, g, 1 << 30)
    got = dbg.dbg_unitigs_get(u)
    for f in ("node_off", "nodes", "seq_off", "circular"):
        np.testing.assert_array_equal(got[f], want[f], err_msg=f)
    assert got["seq"] == want["seq"] and launches > 0
