"""The range-by-range comparison used by the full-size parity tests: on a
small input, the oracle's own graph passes it, and a planted mistake in the
arrays under test (a multiplicity, an orientation, an end node, a missing
node or edge) is caught.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1003_1940_gb300 import readgen
from range_parity import compare_by_ranges, first_base_cuts, key_slice


def arrays_of(og, W):
    words = lambda a: a[:, 1:2].copy() if W == 1 else a.copy()
    return {"edge_keys": words(og.edge_keys), "node_keys": words(og.node_keys), "src": og.src.copy(),
            "dst": og.dst.copy(), "orient": og.orient.copy(), "mult": og.mult.copy()}


@pytest.fixture(scope="module", params=[(21, 60), (33, 80)])
def case(request):
    k, L = request.param
    reads, lengths = readgen.generate(readgen.ReadSetSpec(4_000, 600, L, 0.01, k, 9 + k))
    og = oracle.build_graph(reads, lengths, k)
    return k, reads, lengths, og, 1 if k <= 31 else 2


def test_cuts_cover_the_key_space():
    for bits in (6, 44, 62, 64, 110, 128):
        for parts in (1, 4, 16, 64):
            c = first_base_cuts(bits, parts)
            assert c[0] == 0 and c[-1] == 1 << bits and all(a < b for a, b in zip(c[:-1], c[1:]))


def test_key_slice_two_words():
    w = np.array([[0, 5], [1, 0], [1, 7], [1, 9], [3, 0]], dtype=np.uint64)
    assert key_slice(w, (1 << 64) + 1, (1 << 64) + 9) == (2, 4)
    assert key_slice(w, 0, (2 << 64)) == (0, 4)


def test_oracle_graph_passes(case):
    k, reads, lengths, og, W = case
    res = compare_by_ranges(arrays_of(og, W), reads, lengths, k, parts=8, procs=2)
    assert res["edges"] == og.n_edges and res["nodes"] == og.n_nodes


@pytest.mark.parametrize("plant", ["mult", "orient", "dst", "drop_node", "drop_edge"])
def test_planted_mistake_is_caught(case, plant):
    k, reads, lengths, og, W = case
    a = arrays_of(og, W)
    i = len(a["mult"]) // 3
    if plant == "mult":
        a["mult"][i] += 1
    elif plant == "orient":
        a["orient"][i] ^= 1
    elif plant == "dst":
        a["dst"][i] = (a["dst"][i] + 1) % len(a["node_keys"])
    elif plant == "drop_node":
        a["node_keys"] = np.delete(a["node_keys"], len(a["node_keys"]) // 2, axis=0)
    else:
        for f in ("edge_keys", "src", "dst", "orient", "mult"):
            a[f] = np.delete(a[f], i, axis=0)
    with pytest.raises(AssertionError):
        compare_by_ranges(a, reads, lengths, k, parts=8, procs=1)


# ---------------------------------------------------------------------------
# the full-size maximality check of the unitigs, on the oracle's own result
# ---------------------------------------------------------------------------

def maximal_args(og, ou):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.int64))
    return (og.n_nodes, t(og.src), t(og.dst), t(og.orient), t(ou.nodes), t(ou.node_off),
            torch.from_numpy(ou.circular.astype(np.bool_)))


def test_maximality_check_passes_the_oracle_and_catches_splits():
    from unitig_checks import check_maximal
    reads, lengths = readgen.generate(readgen.ReadSetSpec(3_000, 700, 40, 0.005, 15, 12))
    og = oracle.build_graph(reads, lengths, 15)
    ou = oracle.compact(og)
    args = list(maximal_args(og, ou))
    res = check_maximal(*args)
    assert res["mergeable"] > 100 and res["unitigs"] == ou.count
    # split the longest open unitig in two: its halves are not maximal
    lens = np.diff(ou.node_off.astype(np.int64))
    u = int(np.argmax(np.where(ou.circular == 0, lens, 0)))
    assert lens[u] >= 2
    cut = int(ou.node_off[u]) + 1
    import torch
    bad = list(args)
    bad[5] = torch.from_numpy(np.insert(ou.node_off.astype(np.int64), u + 1, cut))
    bad[6] = torch.from_numpy(np.insert(ou.circular.astype(np.bool_), u + 1, False))
    with pytest.raises(AssertionError):
        check_maximal(*bad)
    # join two unitigs that no mergeable edge joins
    bad = list(args)
    bad[5] = torch.from_numpy(np.delete(ou.node_off.astype(np.int64), 1))
    bad[6] = torch.from_numpy(np.delete(ou.circular.astype(np.bool_), 0))
    with pytest.raises(AssertionError):
        check_maximal(*bad)


def test_several_cases_in_one_pool(case):
    k, reads, lengths, og, W = case
    from range_parity import compare_cases
    good = arrays_of(og, W)
    res = compare_cases([(good, reads, lengths, k, 4), (good, reads, lengths, k, 1)], procs=2)
    assert [r["edges"] for r in res] == [og.n_edges] * 2
    bad = arrays_of(og, W)
    bad["mult"][-1] += 1
    with pytest.raises(AssertionError, match="case 1"):
        compare_cases([(good, reads, lengths, k, 4), (bad, reads, lengths, k, 8)], procs=2)
