"""The multi-GPU bench path runs independent replicas: each rank builds its
own graph and the job's value is all ranks' edge instances over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r built 1000 * (r + 1) units in 100 * (r + 1) ms
    rate, ms = bench.job_rate(1000.0 * (rank + 1), 100.0 * (rank + 1), ws)
    out[rank] = (rate, ms, bench.max_over_ranks(float(rank), ws))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        for r in range(ws):
            rate, ms, mx = out[r]
            assert ms == 200.0 and mx == 1.0
            assert abs(rate - 3000.0 / 0.2) < 1e-6


def test_host_binding_helpers():
    """The bench's host placement: CPU lists as Linux writes them, and a
    machine without a usable GPU leaves the process where it is."""
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("") == set()
    before = os.sched_getaffinity(0)
    info = bench.bind_near_gpu(0)
    if info["bound"]:  # a GPU machine whose process may use cores away from the GPU
        assert os.sched_getaffinity(0) < before
        os.sched_setaffinity(0, info["_restore"])
    else:
        assert os.sched_getaffinity(0) == before and "_restore" not in info


def test_measured_traffic_scales_with_the_launch():
    """The roofline's DRAM traffic comes from the committed capture of the
    onesweep pass, scaled to the measured launch by its algorithmic bytes;
    another workload, scale or variant gives none."""
    import re
    import bench
    v = "1024x11 atomic persistent occ1 lb8 h16"
    text = open(os.path.join(os.path.dirname(bench.__file__), "profiles", "onesweep_large_k31.md")).read()
    captured = float(re.search(r"bytes_per_launch " + re.escape(v) + r": (\d+)", text).group(1))
    full = bench.measured_traffic("large", 1.0, v, 16.56e9)
    assert full is not None and abs(full - captured) < 1e6
    half = bench.measured_traffic("large", 1.0, v, 8.28e9)
    assert abs(half - full / 2) < 1e6
    assert bench.measured_traffic("long_k", 1.0, v, 16.56e9) is None
    assert bench.measured_traffic("large", 0.1, v, 16.56e9) is None
    assert bench.measured_traffic("large", 1.0, "512x8 atomic persistent occ2 lb4", 16.56e9) is None
