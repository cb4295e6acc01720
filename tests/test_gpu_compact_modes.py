"""dbg_compact's three ways of ranking the lists give the same unitigs, and
the oracle's: the meeting walks with 32-bit walk words (the default at these
sizes), the walks with 64-bit words (the form used above 2^29 - 1
strand-nodes, forced here), and pointer jumping with cycle breaking (Section
6.2).  Inputs: ordinary read sets for 64- and 128-bit keys, lists long
enough and cycles that send the walks to pointer jumping, the literal rule
of the simplified graph, tiny and empty graphs, and a 1/20 slice of the
large workload."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_unitigs_equal
from unitig_checks import check_unitigs_maximal
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu

FIELDS = ("node_off", "nodes", "seq_off", "circular")


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


def all_modes(dbg, reads, lengths, k, with_oracle=True):
    ctx = dbg.Context()
    g = dbg.dbg_build(ctx, reads, lengths, k)
    got = []
    for mode in (0, 1, 2):
        dbg.dbg_compact_mode_set(ctx, mode)
        got.append(dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, g)))
    for mode in (1, 2):
        for f in FIELDS:
            np.testing.assert_array_equal(got[mode][f], got[0][f], err_msg=f"{f} in mode {mode}")
        assert got[mode]["seq"] == got[0]["seq"], f"seq in mode {mode}"
    if with_oracle:
        assert_unitigs_equal(got[0], oracle.compact(oracle.build_graph(reads, lengths, k)))
    return dbg, ctx, g, got[0]


@pytest.mark.parametrize("k", [9, 21, 31, 33, 55])
def test_modes_agree(dbg, k):
    L = 100 if k < 33 else 150
    reads, lengths = readgen.generate(readgen.ReadSetSpec(60_000, 12_000, L, 0.005, k, 300 + k,
                                                          repeat_fraction=0.02))
    all_modes(dbg, reads, lengths, k)


def test_modes_long_lists_and_cycles(dbg):
    rng = np.random.default_rng(7)
    gnm = rng.integers(0, 4, size=12_000 + 40).astype(np.uint8)
    reads = ["".join("ACGT"[c] for c in gnm[s:s + 100]) for s in range(0, 12_000, 40)]  # one 12 kb list
    reads += ["ACACACACACACACACACACAC" * 2]  # a circular unitig
    circ = "".join("ACGT"[c] for c in rng.integers(0, 4, size=3000))
    circ2 = circ + circ[:60]
    reads += [circ2[i:i + 80] for i in range(0, 3000, 30)]  # a long cycle
    r, l = as_input(reads)
    _, _, _, u = all_modes(dbg, r, l, 21)
    assert int(u["circular"].sum()) >= 2


def test_modes_tiny_and_empty(dbg):
    reads = ["A" * 50, "T" * 40, "ACACACACACACACACAC", "ACGT" * 10, "GATC" * 12,
             "AAAAACCCCCGGGGGTTTTT" * 3, "TGCA" * 9]
    for k in (1, 3, 5, 7, 11):
        r, l = as_input(reads)
        all_modes(dbg, r, l, k)
    r, l = as_input(["ACGTACGTAACCGGTT"])
    all_modes(dbg, r, l, 5)
    r, l = as_input([])
    all_modes(dbg, r, l, 21)


def test_modes_literal_rule(dbg):
    """The simplified graph's chains (the literal rule) in every mode."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(50_000, 10_000, 100, 0.005, 21, 91,
                                                          repeat_fraction=0.02))
    ctx = dbg.Context()
    g = dbg.dbg_build(ctx, reads, lengths, 21)
    got = []
    for mode in (0, 1, 2):
        dbg.dbg_compact_mode_set(ctx, mode)
        got.append(dbg.dbg_simple_get(dbg.dbg_simplify(ctx, g, 3)))
    for mode in (1, 2):
        for f in got[0]:
            if isinstance(got[0][f], np.ndarray):
                np.testing.assert_array_equal(got[mode][f], got[0][f], err_msg=f"{f} in mode {mode}")
            else:
                assert got[mode][f] == got[0][f], f"{f} in mode {mode}"


def test_modes_large_slice(dbg):
    """0.75 M reads of the large workload's recipe (52 M edge instances):
    the same unitigs in every mode, maximal."""
    import torch
    reads, lengths = readgen.generate(readgen.large_spec(0.05))
    ctx = dbg.Context()
    g = dbg.dbg_build(ctx, torch.from_numpy(reads).cuda(), torch.from_numpy(lengths.view(np.int32)).cuda(), 31)
    got = []
    for mode in (0, 1, 2):
        dbg.dbg_compact_mode_set(ctx, mode)
        got.append(dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, g)))
    for mode in (1, 2):
        for f in FIELDS:
            np.testing.assert_array_equal(got[mode][f], got[0][f], err_msg=f"{f} in mode {mode}")
        assert got[mode]["seq"] == got[0]["seq"]
    res = check_unitigs_maximal(dbg, g, got[0])
    assert res["unitigs"] == len(got[0]["node_off"]) - 1 and res["mergeable"] > 0


@pytest.mark.parametrize("k", [21, 33])
def test_side_bytes_and_orient_gather_agree(dbg, k):
    """dbg_build stores each adjacency slot's side bits, which the side pass
    of the compaction reads in order; the same graph from dbg_build_bucketed
    has none, and the side pass gathers each edge's orient instead.  Both
    give the same unitigs and the same simplified graph (the literal rule),
    and the unitigs are the oracle's."""
    L = 100 if k < 33 else 150
    reads, lengths = readgen.generate(readgen.ReadSetSpec(60_000, 12_000, L, 0.005, k, 500 + k,
                                                          repeat_fraction=0.02))
    ctx = dbg.Context()
    g = dbg.dbg_build(ctx, reads, lengths, k)
    gb = dbg.dbg_build_bucketed(ctx, reads, lengths, k, 4 << 20)
    a = dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, g))
    b = dbg.dbg_unitigs_get(dbg.dbg_compact(ctx, gb))
    for f in FIELDS:
        np.testing.assert_array_equal(b[f], a[f], err_msg=f)
    assert b["seq"] == a["seq"]
    assert_unitigs_equal(a, oracle.compact(oracle.build_graph(reads, lengths, k)))
    sa = dbg.dbg_simple_get(dbg.dbg_simplify(ctx, g, 3))
    sb = dbg.dbg_simple_get(dbg.dbg_simplify(ctx, gb, 3))
    for f in sa:
        if isinstance(sa[f], np.ndarray):
            np.testing.assert_array_equal(sb[f], sa[f], err_msg=f)
        else:
            assert sb[f] == sa[f], f
