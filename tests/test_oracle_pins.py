"""Pins for the CPU oracle: worked examples printed in the paper, an
independent string-only model on exhaustive and random tiny inputs, closed
forms and invariants.  No GPU involved."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle
import strings_model as sm
from golden_io import all_fixtures, load
from paper_1003_1940_gb300 import readgen


def kmer_str(v: int, m: int) -> str:
    return "".join("ACGT"[(v >> (2 * (m - 1 - i))) & 3] for i in range(m))


def build(reads: list[str], k: int):
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    return oracle.build_graph("".join(reads).encode(), lengths, k)


def graph_strings(g):
    k = g.k
    nodes = [kmer_str(v, k) for v in g.node_ints()]
    edges = []
    for i in range(g.n_edges):
        o = int(g.orient[i])
        edges.append((nodes[g.src[i]], nodes[g.dst[i]], o >> 1, o & 1, int(g.mult[i])))
    return nodes, edges


# --------------------------------------------------------------------------
# worked examples (tests/golden, each citing its section)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", all_fixtures())
def test_golden_example(name):
    fx = load(name)
    k = fx["k"]
    g = build(fx["reads"], k)
    nodes, edges = graph_strings(g)
    if fx["nodes"]:
        assert nodes == sorted(fx["nodes"])
    if fx["edges"]:
        assert sorted(edges) == sorted(fx["edges"])
    u = oracle.compact(g)
    assert sorted(u.strings()) == sorted(fx["unitigs"])
    kp1 = {kmer_str(z, k + 1) for z in g.edge_ints()}
    for what, args in fx["paper"]:
        if what == "kmers":
            # every printed k-mer is on one strand of a node
            for s in args:
                assert sm.canonical(s) in nodes
        elif what == "absent_pair":
            a, b = (sm.canonical(s) for s in args)
            assert not any({e[0], e[1]} == {a, b} for e in edges)
        elif what == "molecule":
            pos, neg = args
            assert pos in nodes and sm.rc(pos) == neg
        elif what == "edge":
            a, b, o1, o2 = args[0], args[1], int(args[2]), int(args[3])
            # the named edge may be stored from its other end
            alt = (b, a, 1 - o2, 1 - o1)
            assert any(e[:4] in ((a, b, o1, o2), alt) for e in edges)
        elif what == "walk":
            w = args[0]
            for j in range(len(w) - k):
                assert sm.canonical(w[j:j + k + 1]) in kp1
        elif what == "label":
            assert len(args[0]) == 4 + k - 1
        elif what == "label_reverse":
            assert sm.rc(args[0]) in [a for t, (a, *_) in fx["paper"] if t == "label"]


# --------------------------------------------------------------------------
# the oracle against the string-only model
# --------------------------------------------------------------------------

def check_against_strings(reads: list[str], k: int):
    g = build(reads, k)
    nodes, edges = graph_strings(g)
    assert nodes == sm.nodes_of(reads, k)
    want = sm.edge_multiset(reads, k)
    got = {}
    for (a, b, o1, o2, m) in edges:
        x, y = sm.oriented_kmer(a, o1), sm.oriented_kmer(b, o2)
        assert x[1:] == y[:-1]
        assert a <= b
        cls = sm.edge_class(x, y)
        assert cls not in got
        got[cls] = m
    assert got == dict(want)
    # edges are listed by the canonical (k+1)-mer they spell
    keys = [kmer_str(z, k + 1) for z in g.edge_ints()]
    for (a, b, o1, o2, _), key in zip(edges, keys):
        x, y = sm.oriented_kmer(a, o1), sm.oriented_kmer(b, o2)
        assert key == sm.canonical(x + y[-1])
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # adjacency rows list each node's edge ends in edge order
    for v in range(g.n_nodes):
        row = range(int(g.row_ptr[v]), int(g.row_ptr[v + 1]))
        ends = [(int(g.adj_edge[p]), int(g.adj_role[p])) for p in row]
        assert ends == sorted(ends)
        for p in row:
            e, role = int(g.adj_edge[p]), int(g.adj_role[p])
            assert (g.src[e], g.dst[e])[role] == v
            assert (g.dst[e], g.src[e])[role] == g.adj_nbr[p]
    assert int(g.row_ptr[-1]) == 2 * g.n_edges
    return g


@pytest.mark.parametrize("k,L", [(1, 1), (1, 4), (3, 3), (3, 4), (3, 5), (3, 6), (5, 6), (5, 7)])
def test_exhaustive_single_reads(k, L):
    """Every read over {A,C,G,T}^L (sampled at L = 7) as a one-read input."""
    rng = np.random.default_rng(L * 10 + k)
    reads = ["".join(t) for t in itertools.product("ACGT", repeat=L)]
    if len(reads) > 1500:
        reads = [reads[i] for i in rng.choice(len(reads), 1500, replace=False)]
    for r in reads:
        check_against_strings([r], k)


@pytest.mark.parametrize("k", [1, 3, 5, 7, 9])
def test_random_read_sets(k):
    rng = np.random.default_rng(100 + k)
    for trial in range(60):
        alphabet = "ACGT" if trial % 3 else "AC"  # small alphabets force repeats
        n = int(rng.integers(1, 8))
        reads = ["".join(rng.choice(list(alphabet), size=int(rng.integers(1, 3 * k + 6))))
                 for _ in range(n)]
        check_against_strings(reads, k)


def test_reads_shorter_than_k_and_exactly_k():
    # a read of length k adds its node but no edge; a shorter read adds nothing
    g = check_against_strings(["ACGTA", "GGA", "TTTTTT", "AC"], 5)
    nodes, _ = graph_strings(g)
    assert "ACGTA" in nodes or sm.rc("ACGTA") in nodes


def test_empty_input():
    g = build([], 21)
    assert g.n_nodes == 0 and g.n_edges == 0
    assert oracle.compact(g).count == 0


@pytest.mark.parametrize("k", [0, 2, 64, 65])
def test_bad_k_rejected(k):
    with pytest.raises(oracle.OracleError):
        build(["ACGTACGT"], k)


@pytest.mark.parametrize("bad", ["ACGN", "acgt", "ACG-"])
def test_bad_bases_rejected(bad):
    with pytest.raises(oracle.OracleError):
        build([bad + "ACGT"], 3)


def test_long_k_63():
    rng = np.random.default_rng(5)
    reads = ["".join(rng.choice(list("ACGT"), size=80)) for _ in range(4)]
    reads.append(reads[0][10:75])  # overlapping read: multiplicities above 1
    check_against_strings(reads, 63)


# --------------------------------------------------------------------------
# invariants on a workload-shaped input
# --------------------------------------------------------------------------

def test_invariants_tiny_workload():
    spec = readgen.tiny_spec()
    spec = readgen.ReadSetSpec(20_000, 2_000, 36, 0.01, 21, 0)
    reads, lengths = readgen.generate(spec)
    g = oracle.build_graph(reads, lengths, 21)
    # summed multiplicity = sum over reads of (L - k)
    assert int(g.mult.sum()) == int(np.maximum(lengths.astype(np.int64) - 21, 0).sum())
    # node count = number of distinct canonical k-mers
    strs = sm.split_reads(reads.tobytes(), lengths)
    assert g.n_nodes == len(sm.nodes_of(strs, 21))
    assert np.all(g.src <= g.dst)
    # every read spells a valid walk: at each inner k-mer the read enters the
    # node through one side and leaves through the other (Section 2)
    nodes = [kmer_str(v, 21) for v in g.node_ints()]
    by_key = {kmer_str(z, 22): i for i, z in enumerate(g.edge_ints())}

    def side_at(e, v):
        o = int(g.orient[e])
        if g.src[e] == v:
            return "R" if (o >> 1) == 0 else "L"
        return "L" if (o & 1) == 0 else "R"

    index = {s: i for i, s in enumerate(nodes)}
    checked = 0
    for r in strs[:400]:
        for j in range(len(r) - 22):
            e1 = by_key[sm.canonical(r[j:j + 22])]
            e2 = by_key[sm.canonical(r[j + 1:j + 23])]
            v = index[sm.canonical(r[j + 1:j + 22])]
            if g.src[e1] == g.dst[e1] or g.src[e2] == g.dst[e2]:
                continue
            assert side_at(e1, v) != side_at(e2, v)
            checked += 1
    assert checked > 1000


# --------------------------------------------------------------------------
# compaction: closed forms, the string model, invariants
# --------------------------------------------------------------------------

def distinct_kmer_read(rng, length, k):
    """A random read whose k-mers and their reverse complements are all distinct."""
    while True:
        r = "".join(rng.choice(list("ACGT"), size=length))
        kms = [r[j:j + k] for j in range(length - k + 1)]
        can = [sm.canonical(x) for x in kms]
        if len(set(can)) == len(can):
            return r


def test_single_read_is_one_unitig():
    rng = np.random.default_rng(7)
    for k in (3, 5, 21, 31):
        r = distinct_kmer_read(rng, 4 * k + 10, k)
        u = oracle.compact(build([r], k))
        assert u.count == 1
        assert u.strings() == [min(r, sm.rc(r))]
        assert int(u.circular[0]) == 0
        assert len(u.strings()[0]) == (len(r) - k + 1) + k - 1


def test_circular_genome_is_one_cycle():
    rng = np.random.default_rng(8)
    k = 11
    while True:
        gnm = "".join(rng.choice(list("ACGT"), size=200))
        ext = gnm + gnm[:k]
        can = [sm.canonical(ext[j:j + k]) for j in range(len(gnm))]
        if len(set(can)) == len(can):
            break
    # reads tile the circle, each shifted by 7 bases
    reads = [(gnm + gnm)[s:s + 40] for s in range(0, len(gnm), 7)]
    u = oracle.compact(build(reads, k))
    assert u.count == 1 and int(u.circular[0]) == 1
    s = u.strings()[0]
    assert len(s) == len(gnm) + k - 1
    # it starts at the smallest k-mer molecule, on its positive strand
    assert s[:k] == min(can)
    assert s in (gnm + gnm) or sm.rc(s) in (gnm + gnm)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_compaction_against_string_model(k):
    rng = np.random.default_rng(200 + k)
    for trial in range(40):
        glen = int(rng.integers(k + 2, 40))
        gnm = "".join(rng.choice(list("ACGT" if trial % 4 else "ACG"), size=glen))
        reads = []
        for _ in range(int(rng.integers(1, 10))):
            s = int(rng.integers(0, glen - k))
            e = int(rng.integers(s + k, glen + 1))
            rd = gnm[s:e]
            reads.append(rd if rng.random() < 0.5 else sm.rc(rd))
        g = build(reads, k)
        u = oracle.compact(g)
        got = sorted(("C" if c else "P", s) for c, s in zip(u.circular, u.strings()))
        assert got == sm.unitigs_of(reads, k)
        check_unitig_invariants(g, u)


def check_unitig_invariants(g, u):
    k = g.k
    nodes = [kmer_str(v, k) for v in g.node_ints()]
    lists = u.node_lists()
    allnodes = [v for lst in lists for v, _ in lst]
    # every node in exactly one unitig
    assert sorted(allnodes) == list(range(g.n_nodes))
    # total sequence is preserved: sum of m = |V|, each string m + k - 1 long
    for lst, s in zip(lists, u.strings()):
        assert len(s) == len(lst) + k - 1
        for i, (v, strand) in enumerate(lst):
            assert s[i:i + k] == sm.oriented_kmer(nodes[v], strand)
    heads = [lst[0][0] for lst in lists]
    assert heads == sorted(heads)


def test_compaction_invariants_tiny_workload():
    spec = readgen.ReadSetSpec(5_000, 1_500, 36, 0.01, 21, 0)
    reads, lengths = readgen.generate(spec)
    g = oracle.build_graph(reads, lengths, 21)
    check_unitig_invariants(g, oracle.compact(g))


def test_sampled_counts_match_full_build():
    spec = readgen.ReadSetSpec(3_000, 800, 50, 0.01, 15, 4)
    reads, lengths = readgen.generate(spec)
    g = oracle.build_graph(reads, lengths, 15)
    keys = [kmer_str(z, 16) for z in g.edge_ints()]
    pick = list(range(0, len(keys), 37))
    got = oracle.count_kplus1(reads, lengths, 15, [keys[i] for i in pick])
    assert list(got) == [int(g.mult[i]) for i in pick]
    # a (k+1)-mer given as its reverse complement counts the same edge
    got_rc = oracle.count_kplus1(reads, lengths, 15, [sm.rc(keys[i]) for i in pick])
    assert list(got_rc) == list(got)


def test_edge_partitions_add_up_to_the_graph():
    """The multi-core baseline's unit of work: the hash partitions of the
    edges, counted separately, add up to the oracle graph's distinct edges
    and to sum(L - k) instances, for several partition counts."""
    from paper_1003_1940_gb300 import readgen
    reads, lengths = readgen.generate(readgen.ReadSetSpec(20_000, 800, 50, 0.01, 15, 5))
    g = oracle.build_graph(reads, lengths, 15)
    inst = int(np.maximum(lengths.astype(np.int64) - 15, 0).sum())
    for parts in (1, 3, 8):
        res = [oracle.edges_in_partition(reads, lengths, 15, p, parts) for p in range(parts)]
        assert sum(d for d, _ in res) == g.n_edges
        assert sum(i for _, i in res) == inst


# ---------------------------------------------------------------------------
# node multiplicities (the k-mer counting of STEP-2 applied to nodes; the
# k-mer occurrence table behind VELVET's roadmap, Section 7)
# ---------------------------------------------------------------------------

def node_counts_by_strings(reads: list[str], k: int) -> dict[str, int]:
    """Occurrences of each canonical k-mer over the forward reads, by strings."""
    c: dict[str, int] = {}
    for r in reads:
        for j in range(len(r) - k + 1):
            s = sm.canonical(r[j:j + k])
            c[s] = c.get(s, 0) + 1
    return c


def oracle_node_counts(reads: list[str], k: int) -> dict[str, int]:
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    keys, counts = oracle.node_multiplicities("".join(reads).encode(), lengths, k)
    vals = [(int(h) << 64) | int(l) for h, l in keys]
    assert vals == sorted(vals) and len(set(vals)) == len(vals)
    return {kmer_str(v, k): int(c) for v, c in zip(vals, counts)}


def test_node_multiplicities_worked_example():
    """By hand: ACGT at k = 3 reads ACG and CGT = rc(ACG), so ACG twice;
    AAGTA reads AAG, AGT (canonical ACT, its reverse complement) and GTA."""
    assert oracle_node_counts(["ACGT", "AAGTA"], 3) == {"ACG": 2, "AAG": 1, "ACT": 1, "GTA": 1}


@pytest.mark.parametrize("k,L", [(1, 6), (3, 6), (5, 6)])
def test_node_multiplicities_exhaustive_single_reads(k, L):
    for t in itertools.product("ACGT", repeat=L):
        r = "".join(t)
        assert oracle_node_counts([r], k) == node_counts_by_strings([r], k), r


@pytest.mark.parametrize("k", [3, 5, 7, 11])
def test_node_multiplicities_random_read_sets(k):
    """Random read sets with reads shorter than k, of exactly k and longer;
    also the closed form (each read of length L >= k holds L - k + 1 k-mers)
    and the node set of the graph."""
    rng = np.random.default_rng(k)
    for _ in range(30):
        reads = ["".join("ACGT"[c] for c in rng.integers(0, 4, size=int(rng.integers(0, 25))))
                 for _ in range(int(rng.integers(1, 12)))]
        got = oracle_node_counts(reads, k)
        assert got == node_counts_by_strings(reads, k)
        assert sum(got.values()) == sum(max(0, len(r) - k + 1) for r in reads)
        assert sorted(got) == graph_strings(build(reads, k))[0]


# ---------------------------------------------------------------------------
# roadmap counts: distinct reads per node (VELVET keeps the k-mers present in
# at least 2 reads, Section 7)
# ---------------------------------------------------------------------------

def node_reads_by_strings(reads: list[str], k: int) -> dict[str, int]:
    """Distinct reads holding each canonical k-mer (either strand), by strings."""
    c: dict[str, int] = {}
    for r in reads:
        for s in {sm.canonical(r[j:j + k]) for j in range(len(r) - k + 1)}:
            c[s] = c.get(s, 0) + 1
    return c


def oracle_node_reads(reads: list[str], k: int) -> dict[str, int]:
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    keys, counts = oracle.node_reads("".join(reads).encode(), lengths, k)
    vals = [(int(h) << 64) | int(l) for h, l in keys]
    assert vals == sorted(vals) and len(set(vals)) == len(vals)
    return {kmer_str(v, k): int(c) for v, c in zip(vals, counts)}


def test_node_reads_worked_example():
    """By hand, k = 3: ACGT holds ACG twice (ACG, and CGT = rc ACG) but is
    one read; CGTT holds CGT (ACG) and GTT (AAC); AAC also in AACA."""
    got = oracle_node_reads(["ACGT", "CGTT", "AACA"], 3)
    assert got == {"ACG": 2, "AAC": 2, "ACA": 1}


@pytest.mark.parametrize("k", [1, 3, 5, 9])
def test_node_reads_random_read_sets(k):
    """Against the string model; never above the occurrence count, equal to
    it where no read holds a k-mer twice; same node set as the graph."""
    rng = np.random.default_rng(40 + k)
    for trial in range(40):
        alphabet = "ACGT" if trial % 2 else "AC"
        reads = ["".join(rng.choice(list(alphabet), size=int(rng.integers(0, 3 * k + 8))))
                 for _ in range(int(rng.integers(1, 10)))]
        got = oracle_node_reads(reads, k)
        assert got == node_reads_by_strings(reads, k)
        occ = oracle_node_counts(reads, k)
        assert got.keys() == occ.keys() and all(got[x] <= occ[x] for x in got)
        once = all(len({sm.canonical(r[j:j + k]) for j in range(len(r) - k + 1)}) == max(0, len(r) - k + 1)
                   for r in reads)
        if once:
            assert got == occ
        assert sorted(got) == graph_strings(build(reads, k))[0]


# ---------------------------------------------------------------------------
# key-range slices of the graph (the unit of work of the full-size parity
# tests: one process per key range, every read scanned)
# ---------------------------------------------------------------------------

def range_slices(reads, lengths, k, cuts_e, cuts_n):
    """Concatenated slices over the ranges [c_i, c_{i+1} - 1] (edge and node
    ranges cut independently; (1, 0) is an empty range)."""
    ep = [oracle.graph_range(reads, lengths, k, (a, b - 1), (1, 0)) for a, b in zip(cuts_e[:-1], cuts_e[1:])]
    np_ = [oracle.graph_range(reads, lengths, k, (1, 0), (a, b - 1)) for a, b in zip(cuts_n[:-1], cuts_n[1:])]
    out = {f: np.concatenate([p[f] for p in ep]) for f in ep[0] if f != "node_keys"}
    out["node_keys"] = np.concatenate([p["node_keys"] for p in np_])
    return out


def random_cuts(rng, bits, count):
    inner = sorted({int(rng.integers(0, 1 << 62)) << max(0, bits - 62) >> max(0, 62 - bits)
                    for _ in range(count)})
    return [0] + [c for c in inner if 0 < c < (1 << bits)] + [1 << bits]


@pytest.mark.parametrize("k,lo,hi", [(1, 2, 6), (5, 4, 30), (15, 10, 60), (31, 30, 90), (33, 30, 90),
                                     (55, 50, 160), (63, 60, 160)])
def test_graph_range_slices_make_up_the_graph(k, lo, hi):
    """Slices over consecutive key ranges, concatenated in range order, give
    orc_build's node list and its edge list: keys, the keys of both end
    nodes (through orc_build's IDs), orientation and multiplicity."""
    rng = np.random.default_rng(700 + k)
    reads, lengths = readgen.random_reads(rng, 300, lo, hi, b"ACGT" if k > 3 else b"ACG")
    g = oracle.build_graph(reads, lengths, k)
    for count in (1, 5, 17):
        s = range_slices(reads, lengths, k, random_cuts(rng, 2 * k + 2, count - 1),
                         random_cuts(rng, 2 * k, count - 1))
        np.testing.assert_array_equal(s["node_keys"], g.node_keys)
        np.testing.assert_array_equal(s["edge_keys"], g.edge_keys)
        np.testing.assert_array_equal(s["src_keys"], g.node_keys[g.src])
        np.testing.assert_array_equal(s["dst_keys"], g.node_keys[g.dst])
        np.testing.assert_array_equal(s["orient"], g.orient)
        np.testing.assert_array_equal(s["mult"], g.mult.astype(np.uint64))
    assert int(s["mult"].sum()) == int(np.maximum(lengths.astype(np.int64) - k, 0).sum())


def test_graph_range_against_strings():
    """A narrow slice equals the string model's edges and nodes whose
    canonical strings fall in the range (lexicographic = integer order)."""
    rng = np.random.default_rng(71)
    k = 5
    reads = ["".join(rng.choice(list("ACGT"), size=int(rng.integers(4, 30)))) for _ in range(40)]
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    raw = "".join(reads).encode()
    to_int = lambda s: int("".join("0123"["ACGT".index(c)] for c in s), 4)
    want_edges = sm.edge_multiset(reads, k)
    for lo_s, hi_s in (("AAAAAA", "CTTTTT"), ("CAGAAA", "GGGGGG"), ("TAAAAA", "TTTTTT")):
        nlo, nhi = to_int(lo_s[:k]), to_int(hi_s[:k])
        s = oracle.graph_range(raw, lengths, k, (to_int(lo_s), to_int(hi_s)), (nlo, nhi))
        got_nodes = [kmer_str(int(h) << 64 | int(l), k) for h, l in s["node_keys"]]
        assert got_nodes == [v for v in sm.nodes_of(reads, k) if lo_s[:k] <= v <= hi_s[:k]]
        got = {}
        for i in range(len(s["mult"])):
            a = kmer_str(int(s["src_keys"][i, 1]), k)
            b = kmer_str(int(s["dst_keys"][i, 1]), k)
            o = int(s["orient"][i])
            x, y = sm.oriented_kmer(a, o >> 1), sm.oriented_kmer(b, o & 1)
            assert kmer_str(int(s["edge_keys"][i, 1]), k + 1) == sm.canonical(x + y[-1])
            got[sm.edge_class(x, y)] = int(s["mult"][i])
        want = {c: m for c, m in want_edges.items()
                if lo_s <= sm.canonical(next(iter(c))[0] + next(iter(c))[1][-1]) <= hi_s}
        assert got == want


def test_graph_range_empty_and_bad_arguments():
    reads, lengths = b"ACGTACGTTG", np.array([10], dtype=np.uint32)
    s = oracle.graph_range(reads, lengths, 3, (5, 4), (9, 2))  # lo > hi: nothing
    assert len(s["mult"]) == 0 and len(s["node_keys"]) == 0
    with pytest.raises(oracle.OracleError):
        oracle.graph_range(reads, lengths, 4, (0, 255), (0, 63))
    with pytest.raises(oracle.OracleError):
        oracle.graph_range(b"ACGTNCGTTG", lengths, 3, (0, 255), (0, 63))


# ---------------------------------------------------------------------------
# the simplified graph: Section 6.1's literal compaction (candidate edges on
# nodes with one edge end on each side, chains of at least min_nodes nodes
# reported) and the relabelled edges between units (Section 6)
# ---------------------------------------------------------------------------

def side_degrees(g):
    deg = np.zeros((g.n_nodes, 2), dtype=np.int64)  # [:, 0] left, [:, 1] right
    for i in range(g.n_edges):
        o1, o2 = int(g.orient[i]) >> 1, int(g.orient[i]) & 1
        deg[g.src[i], 0 if o1 else 1] += 1
        deg[g.dst[i], 1 if o2 else 0] += 1
    return deg


def literal_components(g):
    """Node sets of the chains by definition: union-find over the candidate
    edges (distinct end nodes, both with exactly one edge end per side)."""
    deg = side_degrees(g)
    simple = (deg[:, 0] == 1) & (deg[:, 1] == 1)
    parent = list(range(g.n_nodes))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    cand = 0
    for i in range(g.n_edges):
        a, b = int(g.src[i]), int(g.dst[i])
        if a != b and simple[a] and simple[b]:
            parent[find(a)] = find(b)
            cand += 1
    comps = {}
    for v in range(g.n_nodes):
        comps.setdefault(find(v), set()).add(v)
    return sorted(sorted(c) for c in comps.values()), cand


def check_simple(g, s, min_nodes):
    k = g.k
    nodes = [kmer_str(v, k) for v in g.node_ints()]
    # units hold every node once and spell their nodes, like unitigs
    ids = [int(x) >> 1 for x in s.nodes]
    assert sorted(ids) == list(range(g.n_nodes))
    firsts = [int(s.nodes[s.node_off[u]]) >> 1 for u in range(s.n_units)]
    assert firsts == sorted(firsts)
    strs = s.strings()
    for u in range(s.n_units):
        lst = s.nodes[s.node_off[u]:s.node_off[u + 1]]
        assert len(strs[u]) == len(lst) + k - 1
        for i, x in enumerate(lst):
            km = strs[u][i:i + k]
            assert sm.canonical(km) == nodes[int(x) >> 1] and (km == nodes[int(x) >> 1]) == ((int(x) & 1) == 0)
    # the reported chains are exactly the definition's components of size >= min_nodes
    comps, cand = literal_components(g)
    multi = [sorted(int(x) >> 1 for x in s.nodes[s.node_off[u]:s.node_off[u + 1]])
             for u in range(s.n_units) if s.node_off[u + 1] - s.node_off[u] > 1]
    assert sorted(multi) == [c for c in comps if len(c) >= max(2, min_nodes)]
    # every edge is inside a reported chain or relabelled, none is removed
    inside = sum(len(c) - 1 for c in comps if len(c) >= max(2, min_nodes))
    inside += sum(1 for u in range(s.n_units) if s.circular[u])
    assert s.removed == 0 and s.n_edges + inside == g.n_edges
    assert list(s.edge) == sorted(s.edge)
    # a relabelled edge joins the unit strings consistently: read unit a so
    # that the edge leaves by side_a and unit b so that it enters by side_b;
    # they overlap in k - 1 bases and spell the edge's (k+1)-mer
    keys = [kmer_str(z, k + 1) for z in g.edge_ints()]
    for j in range(s.n_edges):
        x = strs[s.unit_a[j]] if s.side_a[j] == 1 else sm.rc(strs[s.unit_a[j]])
        y = strs[s.unit_b[j]] if s.side_b[j] == 0 else sm.rc(strs[s.unit_b[j]])
        assert x[len(x) - k + 1:] == y[:k - 1]
        assert sm.canonical(x[len(x) - k:] + y[k - 1]) == keys[s.edge[j]]


def test_simplify_single_read_closed_form():
    """One read whose k-mers are distinct is a path of m nodes: its two end
    nodes have a side with no edge, so the candidates join the m - 2 inner
    nodes; with m - 2 >= 3 the units are first node, inner chain, last node
    joined by two edges, otherwise m single nodes and m - 1 edges."""
    rng = np.random.default_rng(31)
    for k, L in ((5, 12), (7, 13), (7, 16), (9, 30), (5, 9)):
        r = distinct_kmer_read(rng, L, k)
        g = build([r], k)
        s = oracle.simplify(g, 3)
        m = L - k + 1
        check_simple(g, s, 3)
        if m - 2 >= 3:
            assert s.n_units == 3 and s.n_edges == 2
            assert sorted(len(x) for x in s.strings()) == [k, k, m - 2 + k - 1]
        else:
            assert s.n_units == m and s.n_edges == m - 1


@pytest.mark.parametrize("k,min_nodes", [(3, 1), (3, 3), (5, 2), (5, 3), (7, 3), (9, 4)])
def test_simplify_random_read_sets(k, min_nodes):
    rng = np.random.default_rng(500 + 10 * k + min_nodes)
    for trial in range(25):
        genome = "".join(rng.choice(list("ACGT"), size=int(rng.integers(20, 120))))
        reads = []
        for _ in range(int(rng.integers(3, 30))):
            a = int(rng.integers(0, len(genome) - k))
            r = genome[a:a + int(rng.integers(k, 3 * k + 10))]
            reads.append(sm.rc(r) if rng.random() < 0.5 else r)
        g = build(reads, k)
        s = oracle.simplify(g, min_nodes)
        check_simple(g, s, min_nodes)


def test_simplify_circular_and_min_nodes_one():
    """A circular genome tiled by reads whose nodes all have one edge end per
    side is one circular unit; with min_nodes = 1 the units are exactly the
    components of the candidate edges (the literal chains)."""
    rng = np.random.default_rng(33)
    k = 7
    genome = distinct_kmer_read(rng, 60, k)
    circ = genome + genome[:k]
    reads = [circ[i:i + 20] for i in range(0, len(genome), 5)] + [circ[len(genome) - 10:] + circ[k:k + 15]]
    g = build(reads, k)
    s = oracle.simplify(g, 3)
    check_simple(g, s, 3)
    assert s.n_units == 1 and s.circular[0] == 1 and s.n_edges == 0
    g2 = build([genome[:40], genome[30:]], k)
    s1 = oracle.simplify(g2, 1)
    check_simple(g2, s1, 1)
    comps, _ = literal_components(g2)
    assert s1.n_units == len(comps)
