"""Parity of the batched workload at its stated size: 256 read sets (genomes
log-uniform on [10 kbp, 5 Mbp], coverage U[10, 60], reads of 36-150 bp,
k = 21 or 31; 4.53 G edge instances in all) built by one dbg_build_batch call.

  - every one of the 256 graphs equals, array by array and bit for bit, the
    graph dbg_build returns for the same set on its own;
  - 32 sets spread over the size range (every eighth set by edge instances,
    the smallest and the largest included) equal the oracle's graph in full,
    element by element (nodes, edge keys, both end nodes, orientation,
    multiplicity), the larger ones compared key range by key range."""
from __future__ import annotations

import numpy as np
import pytest

from range_parity import compare_cases
from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu

FIELDS = (("node_keys", "<u8", "V", True), ("edge_keys", "<u8", "E", True), ("src", "<u4", "E", False),
          ("dst", "<u4", "E", False), ("orient", "|u1", "E", False), ("mult", "<u4", "E", False),
          ("row_ptr", "<u8", "V+1", False), ("adj_nbr", "<u4", "2E", False), ("adj_edge", "<u4", "2E", False),
          ("adj_role", "|u1", "2E", False))


@pytest.fixture(scope="module")
def batch():
    import torch
    from paper_1003_1940_gb300 import dbg
    dbg.load()
    specs = readgen.batched_specs()
    host = [readgen.generate(sp) for sp in specs]
    sets = [(torch.from_numpy(r).cuda(), torch.from_numpy(l.view(np.int32)).cuda(), sp.k)
            for (r, l), sp in zip(host, specs)]
    ctx = dbg.Context()
    dbg.dbg_autotune(ctx)
    graphs = dbg.dbg_build_batch(ctx, sets, workers=8)
    return dbg, ctx, specs, host, sets, graphs


def device_arrays(dbg, g) -> dict:
    V, E, W = dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g), dbg.dbg_graph_key_words(g)
    n = {"V": V, "E": E, "V+1": V + 1, "2E": 2 * E}
    return {f: dbg.device_tensor(g, f, n[c] * (W if keyed else 1), ty) for f, ty, c, keyed in FIELDS}


def test_all_256_sets_equal_one_at_a_time(batch):
    import torch
    dbg, ctx, specs, host, sets, graphs = batch
    assert len(graphs) == 256
    total = 0
    for i, ((r, l, k), g) in enumerate(zip(sets, graphs)):
        one = dbg.dbg_build(ctx, r, l, k)
        assert dbg.dbg_graph_num_instances(g) == dbg.dbg_graph_num_instances(one) == specs[i].raw_edges
        assert (dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g)) == \
            (dbg.dbg_graph_num_nodes(one), dbg.dbg_graph_num_edges(one)), i
        a, b = device_arrays(dbg, g), device_arrays(dbg, one)
        for f in a:
            assert torch.equal(a[f], b[f]), (i, f)
        total += specs[i].raw_edges
        one.free()
    assert total == sum(sp.raw_edges for sp in specs)


def test_32_sets_against_oracle(batch):
    dbg, ctx, specs, host, sets, graphs = batch
    by_size = np.argsort([sp.raw_edges for sp in specs], kind="stable")
    picks = [int(by_size[i]) for i in np.linspace(0, 255, 32).round().astype(int)]
    assert specs[picks[-1]].raw_edges == max(sp.raw_edges for sp in specs)
    cases = []
    for i in picks:
        g = graphs[i]
        e = dbg.dbg_graph_edges(g)
        arrays = {"edge_keys": e["keys"], "node_keys": dbg.dbg_graph_nodes(g), "src": e["src"],
                  "dst": e["dst"], "orient": e["orient"], "mult": e["mult"]}
        # about 8 M edge instances per key range
        parts = int(min(64, max(1, 2 ** round(np.log2(max(1, specs[i].raw_edges / 8e6))))))
        cases.append((arrays, *host[i], specs[i].k, parts))
    res = compare_cases(cases)
    for i, r in zip(picks, res):
        assert r["edges"] == dbg.dbg_graph_num_edges(graphs[i])
