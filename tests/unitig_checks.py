"""Maximality of the unitigs at full size, checked on the GPU with plain
torch operations on the graph's src / dst / orient arrays (independent of the
library's compaction kernels).

Sides (Section 6, as the oracle reads them): the src end of an edge
(u, v, o1, o2) sits on u's right side when o1 = 0 and on its left side when
o1 = 1; the dst end on v's left side when o2 = 0 and its right side when
o2 = 1.  An edge is mergeable when u != v and both of its sides carry exactly
one edge end.  A unitig lists (node, strand) pairs; strand 0 enters a node by
its left side and leaves by its right side, strand 1 the other way round.

The unitigs are maximal chains exactly when every pair of consecutive nodes
(and the closing pair of a circular unitig) is joined by the mergeable edge
at the first node's exit side, which ends at the second node's entry side,
and there are as many such pairs as mergeable edges: distinct pairs leave by
distinct sides, so then every mergeable edge joins one pair and none leaves a
unitig's end.
"""
from __future__ import annotations

import numpy as np


def check_maximal(V: int, src, dst, orient, nodes, node_off, circular) -> dict:
    """src, dst, orient: the graph's edge arrays; nodes, node_off, circular:
    the unitigs (node ID << 1 | strand).  torch int64 / bool tensors on one
    device."""
    import torch
    dev = src.device
    s_src = 2 * src + (1 - (orient >> 1))  # side index 2v + (0 left, 1 right)
    s_dst = 2 * dst + (orient & 1)
    deg = torch.bincount(torch.cat([s_src, s_dst]), minlength=2 * V)
    merge = (src != dst) & (deg[s_src] == 1) & (deg[s_dst] == 1)
    M = int(merge.sum())
    other = torch.full((2 * V,), -1, dtype=torch.int64, device=dev)
    other[s_src[merge]] = s_dst[merge]
    other[s_dst[merge]] = s_src[merge]
    del s_src, s_dst, deg, merge

    ids, st = nodes >> 1, nodes & 1
    assert int(node_off[-1]) == V and bool((torch.bincount(ids, minlength=V) == 1).all()), \
        "the unitigs do not hold every node exactly once"
    exit_side = 2 * ids + (1 - st)
    entry_side = 2 * ids + st
    first, last = node_off[:-1], node_off[1:] - 1
    is_last = torch.zeros(V, dtype=torch.bool, device=dev)
    is_last[last] = True
    p = torch.nonzero(~is_last).squeeze(1)
    frm = torch.cat([exit_side[p], exit_side[last[circular]]])
    to = torch.cat([entry_side[p + 1], entry_side[first[circular]]])
    assert bool((other[frm] == to).all()), "consecutive unitig nodes not joined by a mergeable edge"
    assert frm.numel() == M, f"{M} mergeable edges, {frm.numel()} consecutive pairs"
    # the ends of open unitigs carry no mergeable edge (implied by the count;
    # checked directly for a clearer message)
    open_ = ~circular
    assert bool((other[entry_side[first[open_]]] == -1).all()), "a mergeable edge enters an open unitig's head"
    assert bool((other[exit_side[last[open_]]] == -1).all()), "a mergeable edge leaves an open unitig's tail"
    return {"mergeable": M, "unitigs": int(node_off.numel() - 1), "circular": int(circular.sum())}


def check_unitigs_maximal(dbg, g, res) -> dict:
    """The library's graph g (device arrays) and its unitigs res
    (dbg_unitigs_get), checked on the GPU."""
    import torch
    V, E = dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g)
    t = lambda f, n, ty: dbg.device_tensor(g, f, n, ty).to(torch.int64)
    cu = lambda a: torch.from_numpy(a).cuda()
    return check_maximal(V, t("src", E, "<u4"), t("dst", E, "<u4"), t("orient", E, "|u1"),
                         cu(res["nodes"].view(np.int64)), cu(res["node_off"].view(np.int64)),
                         cu(res["circular"].astype(np.bool_)))
