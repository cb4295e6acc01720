"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Integer work: every comparison is bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from golden_io import all_fixtures, load
from parity import check_parity, gpu_graph
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_1940_gb300 import dbg as d
    d.load()
    return d


@pytest.fixture(scope="module")
def ctx(dbg):
    return dbg.Context()


def as_input(reads: list[str]):
    lengths = np.array([len(r) for r in reads], dtype=np.uint32)
    return np.frombuffer("".join(reads).encode(), dtype=np.uint8).copy(), lengths


@pytest.mark.parametrize("name", all_fixtures())
def test_worked_examples(dbg, ctx, name):
    fx = load(name)
    reads, lengths = as_input(fx["reads"])
    check_parity(dbg, ctx, reads, lengths, fx["k"])


def test_tiny_workload(dbg, ctx):
    """The 10,000-read, 100 kbp, k = 21 workload in full."""
    reads, lengths = readgen.generate(readgen.tiny_spec())
    got = check_parity(dbg, ctx, reads, lengths, 21)
    assert got["N"] == 10_000 * (36 - 21)


@pytest.mark.parametrize("k", [1, 3, 5, 15, 21, 31, 33, 45, 55, 63])
def test_ragged_reads_all_widths(dbg, ctx, k):
    """Ragged lengths around k (shorter, equal, one longer, much longer)."""
    rng = np.random.default_rng(1000 + k)
    spec = readgen.ReadSetSpec(4_000, 1, 10, 0.0, k, 7 + k)
    reads_g, _ = readgen.generate(readgen.ReadSetSpec(3_000, 400, 2 * k + 40, 0.01, k, 9 + k))
    lens = rng.integers(max(1, k - 3), 2 * k + 40, size=400).astype(np.uint32)
    lens[:5] = [k, k, k + 1, max(1, k - 1), 2 * k + 39]
    reads = reads_g[:int(lens.sum())]
    check_parity(dbg, ctx, reads, lens, k)
    del spec


@pytest.mark.parametrize("k", [21, 55])
def test_many_tiles_ragged_tail(dbg, ctx, k):
    """Enough edge instances for several hundred sort tiles plus a partial one."""
    L = 100 if k < 33 else 150
    n = 7_777
    reads, lengths = readgen.generate(readgen.ReadSetSpec(60_000, n, L, 0.01, k, 11))
    check_parity(dbg, ctx, reads, lengths, k, compact=True)


def test_repeats_workload_scaled(dbg, ctx):
    """The 50 Mbp repeat workload's recipe at 1/500 scale (k = 31)."""
    spec = readgen.large_spec(scale=1 / 500)
    reads, lengths = readgen.generate(spec)
    check_parity(dbg, ctx, reads, lengths, 31)


def test_long_k_workload_scaled(dbg, ctx):
    """The long-k workload (tandem arrays, k = 55, 128-bit keys) at 1/400 scale."""
    spec = readgen.long_k_spec(scale=1 / 400)
    reads, lengths = readgen.generate(spec)
    check_parity(dbg, ctx, reads, lengths, 55)


def test_low_complexity(dbg, ctx):
    """Homopolymers, dinucleotide repeats and palindromes: self-loops,
    parallel edges with different orientations, cycles."""
    reads = ["A" * 50, "T" * 40, "ACACACACACACACACAC", "ACGT" * 10, "GATC" * 12,
             "AAAAACCCCCGGGGGTTTTT" * 3, "TGCA" * 9]
    for k in (1, 3, 5, 7, 11):
        r, l = as_input(reads)
        check_parity(dbg, ctx, r, l, k)


def test_empty_and_short(dbg, ctx):
    r, l = as_input([])
    got = check_parity(dbg, ctx, r, l, 21)
    assert got["V"] == 0 and got["E"] == 0
    r, l = as_input(["ACGT", "GG", "A" * 20])
    got = check_parity(dbg, ctx, r, l, 21)
    assert got["V"] == 0
    # a read of exactly k bases: one node, no edge
    r, l = as_input(["ACGTACGTACGTACGTACGTA"])
    got = check_parity(dbg, ctx, r, l, 21)
    assert got["V"] == 1 and got["E"] == 0


def test_reads_with_few_keys_mixed(dbg, ctx):
    """Runs of reads with no (k+1)-mer (empty, shorter than k + 1) between
    reads with 1, 2, 32, 33 and 170 of them, in blocks longer than a warp:
    the emit kernel's lanes step over many reads and their ends."""
    k = 21
    rng = np.random.default_rng(31)
    choices = np.array([0, 5, k, k + 1, k + 2, k + 32, k + 33, 191])
    lengths = []
    for _ in range(400):
        run = int(rng.integers(1, 80))
        lengths += [int(choices[rng.integers(0, len(choices))])] * run
    lengths = np.array(lengths, dtype=np.uint32)
    reads = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=int(lengths.sum()))]
    check_parity(dbg, ctx, reads, lengths, k)


def test_device_resident_input(dbg, ctx):
    import torch
    reads, lengths = readgen.generate(readgen.tiny_spec())
    og = oracle.build_graph(reads, lengths, 21)
    d_reads = torch.from_numpy(reads).cuda()
    d_len = torch.from_numpy(lengths.view(np.int32)).cuda()
    _, got = gpu_graph(dbg, ctx, d_reads, d_len, 21)
    from parity import assert_graph_equal
    assert_graph_equal(got, og)


def test_unaligned_host_input(dbg, ctx):
    reads, lengths = readgen.generate(readgen.ReadSetSpec(5_000, 500, 50, 0.01, 15, 3))
    buf = np.zeros(reads.size + 3, dtype=np.uint8)
    buf[3:] = reads
    check_parity(dbg, ctx, buf[3:], lengths, 15)


@pytest.mark.parametrize("k", [0, 2, 64])
def test_bad_k(dbg, ctx, k):
    r, l = as_input(["ACGTACGT"])
    with pytest.raises(dbg.DbgError) as e:
        dbg.dbg_build(ctx, r, l, k)
    assert e.value.status == dbg.DBG_EINVAL


def test_bad_base_is_reported(dbg, ctx):
    r, l = as_input(["ACGTACGTNACGT", "ACGT"])
    with pytest.raises(dbg.DbgError) as e:
        dbg.dbg_build(ctx, r, l, 3)
    assert e.value.status == dbg.DBG_EINVAL
    # the context stays usable
    r, l = as_input(["ACGTACGTTACGT"])
    check_parity(dbg, ctx, r, l, 3)


def test_repeat_calls_identical(dbg, ctx):
    reads, lengths = readgen.generate(readgen.tiny_spec())
    _, a = gpu_graph(dbg, ctx, reads, lengths, 21)
    _, b = gpu_graph(dbg, ctx, reads, lengths, 21)
    for key in a:
        if isinstance(a[key], np.ndarray):
            np.testing.assert_array_equal(a[key], b[key])


def test_every_sort_variant_sorts_identically(dbg, ctx):
    """Each compiled radix-sort configuration (onesweep passes and the local
    sort's ranking methods) gives the oracle's graph."""
    small64 = readgen.generate(readgen.ReadSetSpec(40_000, 3_000, 100, 0.01, 31, 41))
    small128 = readgen.generate(readgen.ReadSetSpec(30_000, 1_500, 120, 0.01, 55, 42))
    og64 = oracle.build_graph(*small64, 31)
    og128 = oracle.build_graph(*small128, 55)
    counts = [dbg.dbg_sort_variant_count(kd) for kd in range(6)]
    from parity import assert_graph_equal
    try:
        for v in range(max(counts)):
            for kd in range(6):
                dbg.dbg_sort_variant_set(ctx, kd, min(v, counts[kd] - 1))
            _, got = gpu_graph(dbg, ctx, *small64, 31)
            assert_graph_equal(got, og64)
            _, got = gpu_graph(dbg, ctx, *small128, 55)
            assert_graph_equal(got, og128)
    finally:
        for kd in range(6):
            dbg.dbg_sort_variant_set(ctx, kd, 0)


@pytest.mark.parametrize("k,kinds", [(31, (0, 1)), (55, (2, 3))])
def test_persistent_sort_variants_many_tiles(dbg, k, kinds):
    """The persistent onesweep variants (each CTA loops over tiles, the next
    tile's bulk copy in flight) on enough keys for several tiles per CTA:
    every digit sorted globally, 5.7-7.1 M edge keys and 4-5 M node records,
    64- and 128-bit keys, graphs identical to variant 0's, which matches the
    oracle's."""
    reads, lengths = readgen.generate(readgen.ReadSetSpec(2_000_000, 60_000, 150, 0.01, k, 43))
    ctx = dbg.Context()
    dbg.dbg_sort_hybrid_set(ctx, False)
    _, ref = gpu_graph(dbg, ctx, reads, lengths, k)
    from parity import assert_graph_equal
    assert_graph_equal(ref, oracle.build_graph(reads, lengths, k))
    tried = 0
    for kd in kinds:
        for v in range(dbg.dbg_sort_variant_count(kd)):
            if "persistent" not in dbg.dbg_sort_variant_name(kd, v):
                continue
            dbg.dbg_sort_variant_set(ctx, kd, v)
            _, got = gpu_graph(dbg, ctx, reads, lengths, k)
            for key in ref:
                if isinstance(ref[key], np.ndarray):
                    np.testing.assert_array_equal(got[key], ref[key], err_msg=f"{kd}/{v} {key}")
                else:
                    assert got[key] == ref[key], (kd, v, key)
            dbg.dbg_sort_variant_set(ctx, kd, 0)
            tried += 1
    assert tried >= 2


@pytest.mark.parametrize("n_reads,L", [(2_400_000, 150), (2_200_000, 128)])
def test_host_reads_over_several_chunks(dbg, ctx, n_reads, L):
    """Host reads of more than one 256 M-base chunk: each chunk is copied
    while the previous one is packed and its complete reads emitted.  Reads
    straddle the chunk boundary (L = 150) or end exactly on it (L = 128:
    2^21 reads per chunk).  The graph equals the one built from device
    reads, from pageable and from pinned host memory."""
    import torch
    reads, lengths = readgen.generate(readgen.ReadSetSpec(3_000_000, n_reads, L, 0.01, 31, 45))
    assert int(lengths.sum()) > 256 << 20
    _, dev = gpu_graph(dbg, ctx, torch.from_numpy(reads).cuda(),
                       torch.from_numpy(lengths.view(np.int32)).cuda(), 31)
    for host in (reads, torch.from_numpy(reads).pin_memory()):
        _, got = gpu_graph(dbg, ctx, host, lengths, 31)
        for key in dev:
            if isinstance(dev[key], np.ndarray):
                np.testing.assert_array_equal(got[key], dev[key], err_msg=key)
            else:
                assert got[key] == dev[key], key


def test_async_edge_readback_during_compaction(dbg, ctx):
    """dbg_graph_edges_async into pinned host buffers, overlapped with the
    compaction of the same graph, gives what dbg_graph_edges gives; waiting
    with nothing started returns at once; freeing a graph with copies in
    flight waits for them."""
    import torch
    reads, lengths = readgen.generate(readgen.ReadSetSpec(300_000, 40_000, 100, 0.01, 31, 44))
    g = dbg.dbg_build(ctx, reads, lengths, 31)
    dbg.dbg_graph_wait(g)
    E, W = dbg.dbg_graph_num_edges(g), dbg.dbg_graph_key_words(g)
    keys = torch.empty(E * W, dtype=torch.int64).pin_memory()
    src, dst, mult = (torch.empty(E, dtype=torch.int32).pin_memory() for _ in range(3))
    orient = torch.empty(E, dtype=torch.uint8).pin_memory()
    dbg.dbg_graph_edges_async(g, keys.data_ptr(), src.data_ptr(), dst.data_ptr(), orient.data_ptr(),
                              mult.data_ptr())
    u = dbg.dbg_compact(ctx, g)
    dbg.dbg_graph_wait(g)
    want = dbg.dbg_graph_edges(g)
    np.testing.assert_array_equal(keys.numpy().view(np.uint64).reshape(-1, W), want["keys"])
    np.testing.assert_array_equal(src.numpy().view(np.uint32), want["src"])
    np.testing.assert_array_equal(dst.numpy().view(np.uint32), want["dst"])
    np.testing.assert_array_equal(orient.numpy(), want["orient"])
    np.testing.assert_array_equal(mult.numpy().view(np.uint32), want["mult"])
    assert dbg.dbg_unitigs_count(u) > 0
    u.free()
    mult2 = torch.zeros(E, dtype=torch.int32).pin_memory()
    dbg.dbg_graph_edges_async(g, mult=mult2.data_ptr())
    g.free()  # waits for the copy
    np.testing.assert_array_equal(mult2.numpy().view(np.uint32), want["mult"])


def test_autotune_and_cache(dbg, tmp_path):
    c = dbg.Context()
    cache = str(tmp_path / "tune.txt")
    ms = dbg.dbg_autotune(c, 1 << 20, cache)
    chosen = [dbg.dbg_sort_variant_get(c, kd) for kd in range(4)]
    for kd in range(4):
        assert 0 <= chosen[kd] < dbg.dbg_sort_variant_count(kd)
        assert all(t > 0 for t in ms[kd])
        assert ms[kd][chosen[kd]] == min(ms[kd])
    c2 = dbg.Context()
    dbg.dbg_autotune(c2, 1 << 20, cache)  # answered from the cache file
    assert [dbg.dbg_sort_variant_get(c2, kd) for kd in range(4)] == chosen
    reads, lengths = readgen.generate(readgen.tiny_spec())
    check_parity(dbg, c2, reads, lengths, 21)


def test_bounded_wait_reports_timeout_and_context_survives(dbg, ctx):
    """A device wait on a flag that nothing sets gives up after its spin
    limit with DBG_ETIMEOUT; the same context then builds normally."""
    import time
    t = time.perf_counter()
    assert dbg.dbg_selftest_wait(ctx, 2000) == dbg.DBG_ETIMEOUT
    assert time.perf_counter() - t < 5.0
    reads, lengths = readgen.generate(readgen.tiny_spec())
    check_parity(dbg, ctx, reads, lengths, 21)


def test_unitig_longer_than_walk_cap(dbg, ctx):
    """One 6,000-node unitig (longer than the walkers' cap) plus a cycle:
    the general ranking path, against the oracle."""
    rng = np.random.default_rng(99)
    gnm = rng.integers(0, 4, size=6_000 + 40).astype(np.uint8)
    reads = ["".join("ACGT"[c] for c in gnm[s:s + 100]) for s in range(0, 6_000, 40)]
    reads += ["ACACACACACACACACACACAC" * 2]  # a circular unitig as well
    r, l = as_input(reads)
    check_parity(dbg, ctx, r, l, 21)
