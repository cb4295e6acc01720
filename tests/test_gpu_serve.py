"""Batched builds, the request server and the key-range bucket path give the
same graphs as one-at-a-time dbg_build (bit for bit), and the oracle's."""
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


@pytest.fixture(scope="module")
def ctx(dbg):
    return dbg.Context()


def graph_arrays(dbg, g):
    return {
        "W": dbg.dbg_graph_key_words(g), "k": dbg.dbg_graph_k(g), "V": dbg.dbg_graph_num_nodes(g),
        "E": dbg.dbg_graph_num_edges(g), "N": dbg.dbg_graph_num_instances(g), "nodes": dbg.dbg_graph_nodes(g),
        **{f"e_{a}": b for a, b in dbg.dbg_graph_edges(g).items()},
        **{f"c_{a}": b for a, b in dbg.dbg_graph_csr(g).items()},
    }


def assert_same(a: dict, b: dict):
    assert a.keys() == b.keys()
    for key in a:
        if isinstance(a[key], np.ndarray):
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)
        else:
            assert a[key] == b[key], key


def small_sets(n_sets=12, seed=5):
    specs = readgen.batched_specs(n_sets, seed=seed, max_genome=60_000, min_genome=2_000)
    return [(*readgen.generate(s), s.k) for s in specs]


@pytest.mark.parametrize("k,budget", [(31, 6 << 20), (21, 3 << 20), (55, 12 << 20)])
def test_bucketed_equals_in_memory(dbg, ctx, k, budget):
    L = 100 if k < 33 else 150
    reads, lengths = readgen.generate(readgen.ReadSetSpec(80_000, 25_000, L, 0.01, k, 31 + k))
    ref = graph_arrays(dbg, dbg.dbg_build(ctx, reads, lengths, k))
    g = dbg.dbg_build_bucketed(ctx, reads, lengths, k, budget)
    eb, nb = dbg.dbg_graph_buckets(g)
    assert eb > 2 and nb > 1, (eb, nb)
    assert_same(graph_arrays(dbg, g), ref)


def test_bucketed_device_input_and_isolated_reads(dbg, ctx):
    import torch
    reads, lengths = readgen.generate(readgen.ReadSetSpec(30_000, 8_000, 60, 0.01, 21, 77))
    lengths = lengths.copy()
    lengths[::50] = 21  # reads of exactly k bases: nodes without edges
    reads = reads[:int(lengths.sum())]
    og = oracle.build_graph(reads, lengths, 21)
    g = dbg.dbg_build_bucketed(ctx, torch.from_numpy(reads).cuda(), torch.from_numpy(lengths.view(np.int32)).cuda(),
                               21, 1 << 20)
    assert dbg.dbg_graph_buckets(g)[0] > 2
    got = graph_arrays(dbg, g)
    assert_graph_equal(got, og)


def test_batch_equals_one_at_a_time(dbg, ctx):
    sets = small_sets()
    graphs = dbg.dbg_build_batch(ctx, sets, workers=4)
    for (r, l, k), g in zip(sets, graphs):
        assert_same(graph_arrays(dbg, g), graph_arrays(dbg, dbg.dbg_build(ctx, r, l, k)))
    # and the oracle's, on three of them
    for (r, l, k), g in list(zip(sets, graphs))[:3]:
        assert_graph_equal(graph_arrays(dbg, g), oracle.build_graph(r, l, k))


def test_server_mixed_stream(dbg, ctx):
    """Requests submitted while others run (continuous admission), one forced
    onto the bucket path, polled out of order: each result equals its
    one-at-a-time build."""
    sets = small_sets(10, seed=9)
    srv = dbg.Server(workers=3)
    tickets = []
    for i, (r, l, k) in enumerate(sets):
        tickets.append(dbg.dbg_submit(srv, r, l, k, flags=dbg.DBG_REQ_BUCKETED if i == 4 else 0))
    seen_pending = False
    results = {}
    for t in reversed(tickets):
        res = dbg.dbg_poll(srv, t, wait=False)
        if res is None:
            seen_pending = True
            res = dbg.dbg_poll(srv, t, wait=True)
        results[t] = res
    for i, ((r, l, k), t) in enumerate(zip(sets, tickets)):
        g, stats = results[t]
        assert stats["latency_s"] >= stats["run_s"] >= 0
        assert stats["bucketed"] == (i == 4)
        assert_same(graph_arrays(dbg, g), graph_arrays(dbg, dbg.dbg_build(ctx, r, l, k)))
        g.free()
    srv.close()
    del seen_pending


def test_server_over_budget_request_takes_bucket_path(dbg, ctx):
    reads, lengths = readgen.generate(readgen.ReadSetSpec(50_000, 20_000, 100, 0.01, 31, 123))
    srv = dbg.Server(workers=2, mem_budget=24 << 20)
    t = dbg.dbg_submit(srv, reads, lengths, 31)
    g, stats = dbg.dbg_poll(srv, t)
    assert stats["bucketed"]
    assert_same(graph_arrays(dbg, g), graph_arrays(dbg, dbg.dbg_build(ctx, reads, lengths, 31)))
    g.free()
    srv.close()


def test_server_queues_requests_over_budget(dbg, ctx):
    """Requests whose combined worst-case footprint exceeds the budget queue
    instead of failing: at most two run at once under a budget of 2.5
    footprints, results stay charged until they are freed, and each result
    equals its one-at-a-time build."""
    specs = [readgen.ReadSetSpec(100_000, 25_000, 100, 0.01, 31, 300 + i) for i in range(8)]
    sets = [readgen.generate(sp) for sp in specs]
    probe = dbg.Server(workers=1, mem_budget=1 << 40)
    g, st = dbg.dbg_poll(probe, dbg.dbg_submit(probe, *sets[0], 31))
    footprint = st["footprint"]
    g.free()
    assert probe.charged() == 0
    probe.close()
    budget = int(2.5 * footprint)
    srv = dbg.Server(workers=6, mem_budget=budget)
    tickets = [dbg.dbg_submit(srv, r, l, 31) for r, l in sets]
    results = [dbg.dbg_poll(srv, t) for t in tickets]
    assert all(not s["bucketed"] and s["charged"] == s["footprint"] for _, s in results)
    c = srv.stats()
    assert c["finished"] == 8 and c["running"] == 0 and c["queued"] == 0
    assert 1 <= c["peak_running"] <= 2, c  # a third never fit next to two
    assert c["charged"] == srv.charged() > 0  # the results, not yet freed
    for (r, l), (g, _) in zip(sets, results):
        assert_same(graph_arrays(dbg, g), graph_arrays(dbg, dbg.dbg_build(ctx, r, l, 31)))
        g.free()
    assert srv.charged() == 0
    srv.close()


def test_server_device_lengths_footprint(dbg):
    """The footprint of a request with device-resident lengths is that of the
    same request with host lengths (it is computed from the lengths, copied
    to the host at submission), less the device copy of the lengths that a
    build from host lengths makes."""
    import torch
    reads, lengths = readgen.generate(readgen.ReadSetSpec(50_000, 10_000, 75, 0.01, 21, 71))
    srv = dbg.Server(workers=2, mem_budget=1 << 40)
    g1, s1 = dbg.dbg_poll(srv, dbg.dbg_submit(srv, torch.from_numpy(reads).cuda(), lengths, 21))
    g2, s2 = dbg.dbg_poll(srv, dbg.dbg_submit(srv, torch.from_numpy(reads).cuda(),
                                              torch.from_numpy(lengths.view(np.int32)).cuda(), 21))
    assert s1["footprint"] == s2["footprint"] + 4 * len(lengths) and s2["footprint"] > 0
    assert_same(graph_arrays(dbg, g1), graph_arrays(dbg, g2))
    g1.free()
    g2.free()
    srv.close()
