"""dbg_rle_u64_noalloc, the run-length reduce that allocates nothing, gives
the same distinct edge keys and multiplicities as dbg_build.

It is meant for callers that cannot allocate device memory at call time; its
scratch is a fixed device array inside the library.  This file is collected
last on purpose, and it works alone in a fresh process too."""
import numpy as np
import pytest

from paper_1003_1940_gb300 import readgen

pytestmark = pytest.mark.gpu


def test_noalloc_rle_matches_dbg_build():
    import torch
    from paper_1003_1940_gb300 import dbg
    dbg.load()
    ctx = dbg.Context()
    reads, lengths = readgen.generate(readgen.ReadSetSpec(200_000, 60_000, 100, 0.01, 31, 21))
    g = dbg.dbg_build(ctx, reads, lengths, 31)
    edges = dbg.dbg_graph_edges(g)
    keys, mult = edges["keys"][:, 0], edges["mult"]
    # the sorted (k+1)-mer keys that the build reduced: each key mult times
    sorted_keys = np.repeat(keys, mult.astype(np.int64))
    n = sorted_keys.size
    assert n == dbg.dbg_graph_num_instances(g) and n > 4 * 4096
    d_keys = torch.from_numpy(sorted_keys.view(np.int64)).cuda()
    for call in range(2):  # two calls in a row share the scratch array
        d_uniq = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        d_run = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
        count = dbg.dbg_rle_u64_noalloc(d_keys, n, d_uniq, d_run)
        assert count == len(keys), call
        uniq = d_uniq[:count].cpu().numpy().view(np.uint64)
        run = d_run[:count + 1].cpu().numpy().view(np.uint32).astype(np.int64)
        np.testing.assert_array_equal(uniq, keys)
        np.testing.assert_array_equal(np.diff(run), mult.astype(np.int64))
        assert run[0] == 0 and run[-1] == n


def test_noalloc_rle_rejects_oversize_and_handles_empty():
    import torch
    from paper_1003_1940_gb300 import dbg
    dbg.load()
    d = torch.zeros(1, dtype=torch.int64, device="cuda")
    r = torch.zeros(2, dtype=torch.int32, device="cuda")
    # the library's own check, through the raw C ABI (the Python wrapper
    # refuses the undersized buffers before calling it)
    import ctypes
    cnt = ctypes.c_uint64(0)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = dbg._lib.dbg_rle_u64_noalloc(p(d), (1 << 26) + 1, p(d), p(r), ctypes.byref(cnt), None)
    assert st == dbg.DBG_EINVAL
    assert dbg._lib.dbg_rle_u64_noalloc(p(d), 0, p(d), None, ctypes.byref(cnt), None) == dbg.DBG_EINVAL
    r.fill_(7)
    assert dbg.dbg_rle_u64_noalloc(d, 0, d, r) == 0
    assert int(r[0]) == 0  # run_start[n] = n, written before the call returns
    # buffers too small, of the wrong element size or on the host are refused
    # before anything reaches the GPU
    with pytest.raises(ValueError):
        dbg.dbg_rle_u64_noalloc(d, 2, d, r)
    with pytest.raises(ValueError):
        dbg.dbg_rle_u64_noalloc(d.view(torch.int32), 1, d, r)
    with pytest.raises(ValueError):
        dbg.dbg_rle_u64_noalloc(d.cpu(), 1, d, r)
