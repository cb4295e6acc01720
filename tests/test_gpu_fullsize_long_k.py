"""Parity at the second benchmark size: the 20 Mbp repeat + tandem-array
workload (4 M reads x 150 bp, k = 55, 128-bit keys, 380 M edge instances),
built with the autotuned launch configuration.  The tandem arrays give runs of
equal keys far longer than a local sort tile, so the gathered global sort of
oversize tiles runs here at full size.

Checked: properties that hold at any size (ordering, sums, adjacency), the
multiplicities of sampled edges and non-edges against the oracle's scan of all
reads, the STEP-1 decoding of sampled edges against string arithmetic, and the
unitigs of a sample against the node keys."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import strings_model as sm
from range_parity import compare_by_ranges
from unitig_checks import check_unitigs_maximal
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu

K = 55


def kmer_int(s: str) -> int:
    v = 0
    for c in s:
        v = (v << 2) | "ACGT".index(c)
    return v


def kmer_str(v: int, m: int) -> str:
    return "".join("ACGT"[(v >> (2 * (m - 1 - i))) & 3] for i in range(m))


def word_int(words: np.ndarray, i: int) -> int:
    """Row i of (n, 2) high/low words as a Python integer."""
    return (int(words[i, 0]) << 64) | int(words[i, 1])


def find(words: np.ndarray, c: int) -> int:
    """Index of key c in sorted (n, 2) high/low words, or -1."""
    hi, lo = np.uint64(c >> 64), np.uint64(c & ((1 << 64) - 1))
    a = int(np.searchsorted(words[:, 0], hi, "left"))
    b = int(np.searchsorted(words[:, 0], hi, "right"))
    i = a + int(np.searchsorted(words[a:b, 1], lo, "left"))
    return i if i < b and words[i, 1] == lo else -1


@pytest.fixture(scope="module")
def built():
    import torch
    from paper_1003_1940_gb300 import dbg
    dbg.load()
    spec = readgen.long_k_spec()
    reads, lengths = readgen.generate(spec)
    ctx = dbg.Context()
    dbg.dbg_autotune(ctx)
    g = dbg.dbg_build(ctx, torch.from_numpy(reads).cuda(), torch.from_numpy(lengths.view(np.int32)).cuda(), K)
    return dbg, ctx, g, reads, lengths


def test_long_k_invariants(built):
    import torch
    dbg, ctx, g, reads, lengths = built
    V, E, N = dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g), dbg.dbg_graph_num_instances(g)
    assert dbg.dbg_graph_key_words(g) == 2
    assert N == 4_000_000 * (150 - K)
    t = lambda f, n, ty: dbg.device_tensor(g, f, n, ty)
    keys = t("edge_keys", 2 * E, "<u8").view(torch.int64).view(E, 2)
    nodes = t("node_keys", 2 * V, "<u8").view(torch.int64).view(V, 2)
    mult = t("mult", E, "<u4").to(torch.int64)
    src = t("src", E, "<u4").to(torch.int64)
    dst = t("dst", E, "<u4").to(torch.int64)
    row = t("row_ptr", V + 1, "<u8").view(torch.int64)
    nbr = t("adj_nbr", 2 * E, "<u4").to(torch.int64)
    aed = t("adj_edge", 2 * E, "<u4").to(torch.int64)
    aro = t("adj_role", 2 * E, "|u1").to(torch.int64)
    assert int(mult.sum()) == N and int(mult.min()) >= 1
    # 112-bit edge keys and 110-bit node keys: the high words are below 2^63,
    # so (high, low) order is signed order on high, then unsigned on low
    flip = lambda x: x ^ torch.iinfo(torch.int64).min

    def strictly_increasing(w):
        hi, lo = w[:, 0], flip(w[:, 1])
        return bool(((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))).all())

    assert strictly_increasing(keys) and strictly_increasing(nodes)
    assert bool((src <= dst).all()) and int(dst.max()) < V
    assert int(row[0]) == 0 and int(row[-1]) == 2 * E
    deg = row[1:] - row[:-1]
    owner = torch.repeat_interleave(torch.arange(V, device="cuda"), deg)
    assert bool((torch.where(aro == 0, src[aed], dst[aed]) == owner).all())
    assert bool((torch.where(aro == 0, dst[aed], src[aed]) == nbr).all())
    order = aed * 2 + aro
    same_row = owner[1:] == owner[:-1]
    assert bool((order[1:][same_row] > order[:-1][same_row]).all())
    assert bool((deg > 0).all())


def test_long_k_step1_decoding_sampled(built):
    """Sampled edges: STEP-1's table, by string arithmetic, gives the node
    keys at src and dst and the orientation."""
    dbg, ctx, g, reads, lengths = built
    E = dbg.dbg_graph_num_edges(g)
    ed = dbg.dbg_graph_edges(g)
    nw = dbg.dbg_graph_nodes(g)
    rng = np.random.default_rng(55)
    for e in rng.integers(0, E, size=2000):
        z = kmer_str(word_int(ed["keys"], int(e)), K + 1)
        x, y = z[:K], z[1:]
        xh, yh = sm.canonical(x), sm.canonical(y)
        o1, o2 = int(x != xh), int(y != yh)
        s, d, a, b = (xh, yh, o1, o2) if xh <= yh else (yh, xh, 1 - o2, 1 - o1)
        assert word_int(nw, int(ed["src"][e])) == kmer_int(s)
        assert word_int(nw, int(ed["dst"][e])) == kmer_int(d)
        assert int(ed["orient"][e]) == (a << 1) | b


def test_long_k_sampled_multiplicities(built):
    dbg, ctx, g, reads, lengths = built
    rng = np.random.default_rng(56)
    ed = dbg.dbg_graph_edges(g)
    picks = rng.integers(0, len(lengths), size=800)
    offs = rng.integers(0, 150 - K, size=800)
    queries = [reads[r * 150 + j:r * 150 + j + K + 1].tobytes().decode() for r, j in zip(picks, offs)]
    letters = np.frombuffer(b"ACGT", dtype=np.uint8)
    queries += [letters[rng.integers(0, 4, size=K + 1)].tobytes().decode() for _ in range(200)]
    want = oracle.count_kplus1(reads, lengths, K, queries)
    got = []
    for q in queries:
        i = find(ed["keys"], kmer_int(sm.canonical(q)))
        got.append(int(ed["mult"][i]) if i >= 0 else 0)
    np.testing.assert_array_equal(np.array(got, dtype=np.uint64), want)
    assert int((want[:800] > 0).sum()) == 800


def test_long_k_compaction_invariants(built):
    import torch
    dbg, ctx, g, reads, lengths = built
    V = dbg.dbg_graph_num_nodes(g)
    u = dbg.dbg_compact(ctx, g)
    U = dbg.dbg_unitigs_count(u)
    res = dbg.dbg_unitigs_get(u)
    node_off, nodes = res["node_off"], res["nodes"]
    assert int(node_off[-1]) == V
    ids = torch.from_numpy(nodes.view(np.int64) >> 1).cuda()
    assert bool((torch.bincount(ids, minlength=V) == 1).all())
    assert len(res["seq"]) == V + U * (K - 1)
    heads = ids[torch.from_numpy(node_off[:-1].view(np.int64)).cuda()]
    assert bool((heads[1:] > heads[:-1]).all())
    nw = dbg.dbg_graph_nodes(g)
    rng = np.random.default_rng(57)
    for ui in rng.integers(0, U, size=200):
        s = res["seq"][res["seq_off"][ui]:res["seq_off"][ui + 1]].decode()
        lst = nodes[node_off[ui]:node_off[ui + 1]]
        assert len(s) == len(lst) + K - 1
        for i, x in enumerate(lst):
            km = s[i:i + K]
            assert kmer_int(sm.canonical(km)) == word_int(nw, int(x) >> 1)
            assert (km == sm.canonical(km)) == ((int(x) & 1) == 0)


def test_long_k_against_oracle_by_key_ranges(built):
    """Every node and every edge against the oracle, element by element: the
    key spaces are cut into 64 ranges and each range's slice of the oracle
    graph (one process per host core, every read scanned) is compared with
    the same keys of the library's graph -- edge keys, both end nodes through
    src / dst, orientation, multiplicity, node keys -- and the ranges together
    hold all of the library's edges and nodes."""
    dbg, ctx, g, reads, lengths = built
    e = dbg.dbg_graph_edges(g)
    arrays = {"edge_keys": e["keys"], "node_keys": dbg.dbg_graph_nodes(g), "src": e["src"], "dst": e["dst"],
              "orient": e["orient"], "mult": e["mult"]}
    res = compare_by_ranges(arrays, reads, lengths, K, parts=64)
    assert res["edges"] == dbg.dbg_graph_num_edges(g) and res["nodes"] == dbg.dbg_graph_num_nodes(g)


def test_long_k_compaction_is_maximal(built):
    """Every pair of consecutive unitig nodes is joined by a mergeable edge
    (distinct nodes, both end sides of degree 1) and every mergeable edge
    joins such a pair: no unitig is split or could be extended."""
    dbg, ctx, g, reads, lengths = built
    u = dbg.dbg_compact(ctx, g)
    res = check_unitigs_maximal(dbg, g, dbg.dbg_unitigs_get(u))
    assert res["unitigs"] == dbg.dbg_unitigs_count(u) and res["mergeable"] > 0
