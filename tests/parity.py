"""Helpers that compare the CUDA path (through the C ABI) with the oracle."""
from __future__ import annotations

import numpy as np

import oracle


def oracle_words(keys2: np.ndarray, W: int) -> np.ndarray:
    """Oracle (high, low) word pairs -> the library's W-word layout."""
    if W == 1:
        assert np.all(keys2[:, 0] == 0)
        return keys2[:, 1:2].copy()
    return keys2.copy()


def gpu_graph(dbg, ctx, reads, lengths, k):
    g = dbg.dbg_build(ctx, reads, lengths, k)
    out = {
        "k": dbg.dbg_graph_k(g),
        "W": dbg.dbg_graph_key_words(g),
        "V": dbg.dbg_graph_num_nodes(g),
        "E": dbg.dbg_graph_num_edges(g),
        "N": dbg.dbg_graph_num_instances(g),
        "nodes": dbg.dbg_graph_nodes(g),
        **{f"e_{a}": b for a, b in dbg.dbg_graph_edges(g).items()},
        **{f"c_{a}": b for a, b in dbg.dbg_graph_csr(g).items()},
    }
    return g, out


def assert_graph_equal(got: dict, og) -> None:
    """Element-by-element, bit-exact comparison with the oracle graph."""
    W = got["W"]
    assert got["k"] == og.k
    assert got["V"] == og.n_nodes, (got["V"], og.n_nodes)
    assert got["E"] == og.n_edges, (got["E"], og.n_edges)
    np.testing.assert_array_equal(got["nodes"], oracle_words(og.node_keys, W))
    np.testing.assert_array_equal(got["e_keys"], oracle_words(og.edge_keys, W))
    np.testing.assert_array_equal(got["e_src"], og.src)
    np.testing.assert_array_equal(got["e_dst"], og.dst)
    np.testing.assert_array_equal(got["e_orient"], og.orient)
    np.testing.assert_array_equal(got["e_mult"], og.mult)
    np.testing.assert_array_equal(got["c_row_ptr"], og.row_ptr)
    np.testing.assert_array_equal(got["c_nbr"], og.adj_nbr)
    np.testing.assert_array_equal(got["c_edge"], og.adj_edge)
    np.testing.assert_array_equal(got["c_role"], og.adj_role)


def assert_unitigs_equal(got: dict, ou) -> None:
    np.testing.assert_array_equal(got["node_off"], ou.node_off)
    np.testing.assert_array_equal(got["nodes"], ou.nodes)
    np.testing.assert_array_equal(got["seq_off"], ou.seq_off)
    assert got["seq"] == ou.seq
    np.testing.assert_array_equal(got["circular"], ou.circular)


def check_parity(dbg, ctx, reads, lengths, k, compact=True):
    g, got = gpu_graph(dbg, ctx, reads, lengths, k)
    og = oracle.build_graph(reads, lengths, k)
    assert_graph_equal(got, og)
    if compact:
        u = dbg.dbg_compact(ctx, g)
        assert_unitigs_equal(dbg.dbg_unitigs_get(u), oracle.compact(og))
    return got
