"""Benchmark: bi-directed de Bruijn graph construction + chain compaction.

One step = dbg_build (2-bit pack, canonical (k+1)-mer emission, onesweep
radix sort, run-length reduce, node sort, node IDs, CSR adjacency) followed
by dbg_compact (list-ranking chain compaction), on the 50 Mbp repeat-genome
workload: 15 M reads x 100 bp (30x), 0.5 % errors, k = 31, 1.035 G edge
instances.  Inputs are synthetic (seeded) and resident in HBM for `value`;
`e2e` repeats the step through the same C ABI from pinned host buffers.

Metric: edge instances (sum over reads of L - k) built per second, whole job.
With --gpus N > 1 (torchrun) every rank builds its own replica on its GPU
(weak scaling, no data-path collective); time = max over ranks.

--impl reference times the CPU oracle (plain C, one core) on a bounded
sample of the same workload, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1003_1940_gb300 import readgen  # noqa: E402

METRIC = "bi-directed edges built/s"
UNIT = "edges/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large", "long_k", "tiny"], default="large")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served measurements added to the default line (N = 1 only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target oracle sample time")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (profiling captures only)")
    ap.add_argument("--mode", choices=["build", "batched", "served"], default="build",
                    help="build: the large workload (default); batched: 256 read sets, batch vs one at a "
                         "time; served: Poisson request stream through the server")
    ap.add_argument("--sets", type=int, default=256, help="read sets of the batched/served workloads")
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--local-variant", type=int, default=-1,
                    help="ranking method of the hybrid sort's local pass (sort kinds 4 and 5)")
    ap.add_argument("--count-first", type=int, default=1, choices=(0, 1),
                    help="1: the edge keys' local pass counts copies in a hash table before sorting")
    ap.add_argument("--partition-first", type=int, default=1, choices=(0, 1),
                    help="1: the edge keys' first global pass is an unordered partition")
    ap.add_argument("--copy-streams", type=int, default=0,
                    help="streams the end-to-end read-back is spread over (0: the library's default)")
    ap.add_argument("--local-rank", type=int, default=1, choices=(0, 1),
                    help="1: the local passes rank keys within their groups instead of digit passes")
    ap.add_argument("--node-mult", action="store_true",
                    help="the build also counts node multiplicities (an extra k-mer sort)")
    ap.add_argument("--sort-variant", default="", help="a,b,c,d: fixed radix variants per key kind instead "
                                                        "of the autotuner (profiling captures)")
    return ap.parse_args()


def workload(name, scale=1.0):
    tag = "" if scale == 1.0 else f" scaled x{scale:g}"
    if name == "large":
        return (readgen.large_spec(scale), "50Mbp-repeats 15Mx100bp 30x 0.5%err k=31 (build+compact)" + tag)
    if name == "long_k":
        return (readgen.long_k_spec(scale),
                "20Mbp-repeats+tandem 4Mx150bp 30x 0.3%err k=55 (build+compact)" + tag)
    return readgen.tiny_spec(), "100kbp 10000x36bp 1%err k=21 (build+compact)"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._drain, daemon=True).start()
        except Exception:
            self.proc = None

    def _drain(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(workload_name, scale, variant, pass_bytes):
    """DRAM bytes per onesweep launch from the committed ncu summary, scaled
    from the captured launch to this one by algorithmic bytes (DRAM traffic
    grows with the keys a launch moves), or None when the kernel source or
    the chosen variant differs from the capture's."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "onesweep_large_k31.md")
    src = os.path.join(ROOT, "paper_1003_1940_gb300", "csrc", "k_build.cuh")
    if scale != 1.0 or not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if line.startswith("    ") and ": " in line and not line.strip().startswith(("ncu", "python")):
            key, _, val = line.strip().partition(": ")
            fields[key.strip()] = val.strip()
    text = open(src).read()
    section = text[text.index("// K3 onesweep radix pass"):text.index("// K4 run-length reduce")]
    digest = hashlib.sha256(section.encode()).hexdigest()[:16]
    if fields.get("source_sha256_16") != digest or fields.get("workload") != workload_name:
        return None
    # one captured figure per variant: "bytes_per_launch <variant name>: <bytes>"
    got = fields.get(f"bytes_per_launch {variant}")
    if not got:
        return None
    alg = float(fields.get("algorithmic_bytes_per_launch", "0"))
    return float(got) * (pass_bytes / alg) if alg > 0 and pass_bytes > 0 else float(got)


def parse_cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_near_gpu(device):
    """Runs this process on the host cores local to the GPU (those of them it
    may use), so that the pinned host buffers of the end-to-end step are
    allocated on the GPU's NUMA node; reports what it found and did."""
    import torch
    info = {"bound": False}
    try:
        p = torch.cuda.get_device_properties(device)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        info["gpu_pci"] = bus
        info["gpu_numa_node"] = int(open(f"{base}/numa_node").read())
        local = parse_cpulist(open(f"{base}/local_cpulist").read())
        allowed = set(os.sched_getaffinity(0))
        both = local & allowed
        info["allowed_cpus"] = len(allowed)
        info["gpu_local_allowed_cpus"] = len(both)
        if both and both != allowed:
            os.sched_setaffinity(0, both)
            info["bound"] = True
            info["_restore"] = sorted(allowed)
    except Exception as e:  # no GPU, no sysfs entry, an older torch: leave placement alone
        info["error"] = type(e).__name__
    return info


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return x if ws == 1 else _reduce(x, ws, dist.ReduceOp.MAX)


def job_rate(units_per_rank, ms_per_rank, ws):
    """Whole-job throughput of replicas: all units of all ranks over the
    slowest rank's time (weak scaling; no data-path collective)."""
    import torch.distributed as dist
    units = units_per_rank if ws == 1 else _reduce(units_per_rank, ws, dist.ReduceOp.SUM)
    ms = max_over_ranks(ms_per_rank, ws)
    return units / (ms / 1000.0), ms


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded prefix of the same reads
# ---------------------------------------------------------------------------
def oracle_sample_rate(reads, lengths, k, target_s):
    import oracle
    oracle.build()
    lengths64 = lengths.astype(np.int64)
    edges_per_read = np.maximum(lengths64 - k, 0)
    # calibrate on a small prefix, then size the sample for ~target_s
    m0 = min(len(lengths), 2000)
    t = time.perf_counter()
    g = oracle.build_graph(reads[:int(lengths64[:m0].sum())], lengths[:m0], k)
    oracle.compact(g)
    t0 = max(time.perf_counter() - t, 1e-3)
    m = int(min(len(lengths), max(m0, m0 * target_s / t0)))
    nb = int(lengths64[:m].sum())
    t = time.perf_counter()
    g = oracle.build_graph(reads[:nb], lengths[:m], k)
    oracle.compact(g)
    dt = time.perf_counter() - t
    edges = int(edges_per_read[:m].sum())
    return edges / dt, dt, m, edges


def _partition_worker(job):
    """One process of the multi-core CPU baseline: every read, one key partition."""
    reads_path, lengths_path, k, part, parts = job
    import oracle
    reads, lengths = np.load(reads_path), np.load(lengths_path)
    t = time.perf_counter()
    distinct, inst = oracle.edges_in_partition(reads, lengths, k, part, parts)
    return time.perf_counter() - t, distinct, inst


def oracle_parallel_rate(reads, lengths, k, m):
    """Edge counting of the first m reads by one process per host core, each
    scanning every read and keeping one hash partition of the canonical
    (k+1)-mers.  Returns (edges/s, seconds, processes)."""
    import multiprocessing as mp
    import tempfile
    import oracle
    oracle.build()
    parts = len(os.sched_getaffinity(0)) or 1
    nb = int(lengths[:m].astype(np.int64).sum())
    with tempfile.TemporaryDirectory() as d:
        rp, lp = os.path.join(d, "reads.npy"), os.path.join(d, "lengths.npy")
        np.save(rp, reads[:nb])
        np.save(lp, lengths[:m])
        with mp.get_context("spawn").Pool(parts) as pool:
            res = pool.map(_partition_worker, [(rp, lp, k, p, parts) for p in range(parts)])
    dt = max(r[0] for r in res)
    inst = sum(r[2] for r in res)
    return inst / dt, dt, parts


def cpu_model():
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    spec, wl = workload(args.workload, args.scale)
    reads, lengths = readgen.generate(spec)
    import oracle
    oracle.build()
    # size one step so that warmup + steps finish within a few minutes
    rate0, dt0, m0, _ = oracle_sample_rate(reads, lengths, spec.k, 2.0)
    m = max(1, int(m0 * min(15.0, 150.0 / max(1, args.steps + args.warmup)) / 2.0))
    m = min(m, len(lengths))
    nb = int(lengths[:m].astype(np.int64).sum())
    edges = int(np.maximum(lengths[:m].astype(np.int64) - spec.k, 0).sum())

    def step():
        g = oracle.build_graph(reads[:nb], lengths[:m], spec.k)
        oracle.compact(g)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t
    value = edges * args.steps / el
    sample = f"first {m} of {len(lengths)} reads ({edges} edge instances) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": wl, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    host = bind_near_gpu(local)
    from paper_1003_1940_gb300 import build_lib, dbg
    build_lib.build()
    dbg.load()
    spec, wl = workload(args.workload, args.scale)
    reads, lengths = readgen.generate(spec)
    k = spec.k
    N = int(np.maximum(lengths.astype(np.int64) - k, 0).sum())

    stream = torch.cuda.Stream()
    ctx = dbg.Context(device=local, stream=stream)
    with torch.cuda.stream(stream):
        d_reads = torch.from_numpy(reads).to("cuda", non_blocking=False)
        d_len = torch.from_numpy(lengths.view(np.int32)).to("cuda")
    torch.cuda.synchronize()

    info = {}

    def step():
        g = dbg.dbg_build(ctx, d_reads, d_len, k)
        u = dbg.dbg_compact(ctx, g)
        info["nodes"], info["edges"] = dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g)
        info["unitigs"] = dbg.dbg_unitigs_count(u)
        u.free()
        g.free()

    if args.sort_variant:
        tune_ms = {}
        for kd, v in enumerate(int(x) for x in args.sort_variant.split(",")):
            dbg.dbg_sort_variant_set(ctx, kd, v)
    else:
        tune_ms = dbg.dbg_autotune(ctx)
    if args.local_variant >= 0:
        for kd in (4, 5):
            dbg.dbg_sort_variant_set(ctx, kd, args.local_variant)
    dbg.dbg_sort_count_first_set(ctx, bool(args.count_first))
    dbg.dbg_sort_partition_first_set(ctx, bool(args.partition_first))
    dbg.dbg_sort_local_rank_set(ctx, bool(args.local_rank))
    if args.copy_streams:
        dbg.dbg_copy_streams_set(ctx, args.copy_streams)
    dbg.dbg_node_mult_set(ctx, bool(args.node_mult))
    variants = {kd: dbg.dbg_sort_variant_name(kd, dbg.dbg_sort_variant_get(ctx, kd)) for kd in range(6)}
    variant_ids = ",".join(str(dbg.dbg_sort_variant_get(ctx, kd)) for kd in range(6))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dbg.dbg_profile_enable(ctx, True)
    launches0 = dbg.dbg_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = dbg.dbg_launch_count(ctx) - launches0
    prof = dbg.dbg_profile_read(ctx)
    dbg.dbg_profile_enable(ctx, False)
    value, ms_max = job_rate(N * args.steps, ms, ws)

    peak, peak_kind = load_peaks()
    srt = prof.get("sort_edges", {"launches": 0, "ms": 0.0, "bytes": 0.0})
    # the dominant kernel: one onesweep pass over the edge keys (the first
    # launch of each sort is the digit-prefix kernel, which moves ~no bytes)
    n_pass = srt["launches"] - args.steps
    pass_ms = srt["ms"] / max(1, srt["launches"] - args.steps) if n_pass > 0 else 0.0
    pass_bytes = srt["bytes"] / max(1, n_pass)
    achieved = pass_bytes / (pass_ms / 1000.0) / 1e9 if pass_ms > 0 else 0.0
    ekind = 0 if k <= 31 else 2  # sort kind of the edge keys: 64- or 128-bit
    traffic = measured_traffic(args.workload, args.scale, variants.get(ekind), pass_bytes)

    stages = {name: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                     "GBps": (v["bytes"] / (v["ms"] / 1000.0) / 1e9) if v["ms"] > 0 else None}
              for name, v in prof.items()}

    # end to end through the same C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        h_reads = torch.from_numpy(reads).pin_memory()
        h_len = torch.from_numpy(lengths.view(np.int32)).pin_memory()
        # the step's whole result comes back into pinned host memory: node
        # keys, edges, adjacency and unitigs.  Buffers are sized by the first
        # (untimed) call; the same input gives the same sizes every step.
        bufs = {}
        out_bytes = {}

        def buf(name, n, dtype, alloc):
            if alloc:
                bufs[name] = torch.empty(max(1, n), dtype=dtype).pin_memory()
            t = bufs[name]
            assert t.numel() >= n, name
            out_bytes[name] = n * t.element_size()
            return t.data_ptr() if n else None

        def step_host(alloc=False):
            g = dbg.dbg_build(ctx, h_reads, h_len, k)
            V, E, W = dbg.dbg_graph_num_nodes(g), dbg.dbg_graph_num_edges(g), dbg.dbg_graph_key_words(g)
            # the graph comes back while it is compacted
            dbg.dbg_graph_nodes_async(g, buf("nodes", V * W, torch.int64, alloc))
            dbg.dbg_graph_edges_async(g, buf("keys", E * W, torch.int64, alloc), buf("src", E, torch.int32, alloc),
                                      buf("dst", E, torch.int32, alloc), buf("orient", E, torch.uint8, alloc),
                                      buf("mult", E, torch.int32, alloc))
            dbg.dbg_graph_csr_async(g, buf("row_ptr", V + 1, torch.int64, alloc), buf("nbr", 2 * E, torch.int32, alloc),
                                    buf("edge", 2 * E, torch.int32, alloc), buf("role", 2 * E, torch.uint8, alloc))
            u = dbg.dbg_compact(ctx, g)
            U, T = dbg.dbg_unitigs_count(u), dbg.dbg_unitigs_total_bases(u)
            dbg.dbg_unitigs_get_into(u, buf("u_node_off", U + 1, torch.int64, alloc),
                                     buf("u_nodes", V, torch.int64, alloc),
                                     buf("u_seq_off", U + 1, torch.int64, alloc),
                                     buf("u_seq", T, torch.uint8, alloc), buf("u_circular", U, torch.uint8, alloc))
            dbg.dbg_graph_wait(g)
            u.free()
            g.free()

        step_host(alloc=True)
        barrier(ws)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t, ws)
        e2e = {"value": N * args.steps * ws / el, "unit": UNIT,
               "h2d_bytes_per_step": int(reads.nbytes + lengths.nbytes),
               "d2h_bytes_per_step": int(sum(out_bytes.values())),
               "d2h": "the whole result: node keys, edges (keys, src, dst, orient, mult), adjacency "
                      "(row_ptr, neighbour, edge, role) and unitigs (offsets, nodes, sequence, circular flags)"}
        bufs.clear()

    # the batched and served workloads, beside the main line (one GPU only)
    extras = {}
    if rank == 0 and ws == 1 and not args.no_extras and args.workload == "large" and args.scale == 1.0 \
            and not args.node_mult:
        specs_b, sets_b = batched_inputs(args)
        ctx_b = dbg.Context(device=local)
        for kd in range(6):
            dbg.dbg_sort_variant_set(ctx_b, kd, dbg.dbg_sort_variant_get(ctx, kd))
        extras["batched"] = measure_batched(args, sets_b, ctx_b)
        extras["served"] = measure_served(args, sets_b, ctx_b, d_reads, d_len, spec)
        del sets_b
        ctx_b.close()
        torch.cuda.empty_cache()

    cpu = None
    if host.get("bound"):  # the host baselines use every core the process may use
        os.sched_setaffinity(0, host.pop("_restore"))
    host.pop("_restore", None)
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt, m, edges = oracle_sample_rate(reads, lengths, k, args.cpu_seconds)
        # the parallel run scans more reads, about as long as the 1-core run
        m_par = int(min(len(lengths), m * max(1, len(os.sched_getaffinity(0)) // 2)))
        prate, pdt, parts = oracle_parallel_rate(reads, lengths, k, m_par)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {m} reads ({edges} edge instances) of the same workload, build+compact, "
                         f"{dt:.1f} s",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "parallel": {"value": prate, "unit": UNIT, "cores": parts, "kind": "oracle",
                            "sample": f"the first {m_par} reads, edge counting only: {parts} processes, each "
                                      f"scanning every read and keeping one hash partition of the edges, "
                                      f"{pdt:.1f} s (slowest process)"}}

    # end to end through HBM: the bytes the library's kernels account per step
    step_bytes = sum(v["bytes"] for v in prof.values()) / args.steps
    build_ms = sum(v["ms"] for kname, v in prof.items() if not kname.startswith("compact")) / args.steps
    compact_ms = sum(v["ms"] for kname, v in prof.items() if kname.startswith("compact")) / args.steps

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64" if k <= 31 else "u128",
            "data": "synthetic",
            "config": {"workload": wl, "edge_instances": N, "reads": int(len(lengths)), "k": k,
                       "nodes": info.get("nodes"), "edges": info.get("edges"), "unitigs": info.get("unitigs"),
                       "l2": "inputs and sort buffers far larger than L2 (1.5 GB reads, 8.3 GB keys)",
                       "parallelism": f"replicas x{ws}",
                       "sort_variants": variants, "sort_variant_ids": variant_ids,
                       "count_first": bool(args.count_first),
                       "partition_first": bool(args.partition_first), "local_rank": bool(args.local_rank),
                       "copy_streams": args.copy_streams or 1,
                       "node_mult": bool(args.node_mult),
                       "autotune_pass_ms": {kd: [round(x, 4) for x in v] for kd, v in tune_ms.items()}},
            "roofline": {"bound": "hbm",
                         "kernel": f"{'k_onesweep_p' if 'persistent' in (variants.get(ekind) or '') else 'k_onesweep'}"
                                   f" ({variants.get(ekind)}; {'64' if ekind == 0 else '128'}-bit edge keys,"
                                   f" one stable 8-bit digit pass)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "peak_kind": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": pass_bytes,
                         "launch_ms": pass_ms},
            "stages": stages,
            "unique_edges_per_s": (info.get("edges") or 0) * args.steps * ws / (ms_max / 1000.0),
            "build_ms_per_step": build_ms, "compact_ms_per_step": compact_ms,
            "hbm_end_to_end": {"bytes_per_step": step_bytes,
                               "GBps": step_bytes / (ms_max / args.steps / 1000.0) / 1e9,
                               "frac": step_bytes / (ms_max / args.steps / 1000.0) / 1e9 / peak if peak else None,
                               "bytes": "algorithmic bytes of every kernel of the step, as the library accounts them"},
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            **extras,
            "host": host,
            "cpu_baseline": cpu,
        }))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched and served modes (reported beside the main line)
# ---------------------------------------------------------------------------
def batched_inputs(args):
    import torch
    specs = readgen.batched_specs(args.sets)
    sets = []
    for sp in specs:
        r, l = readgen.generate(sp)
        sets.append((torch.from_numpy(r).cuda(), torch.from_numpy(l.view(np.int32)).cuda(), sp.k,
                     int(np.maximum(l.astype(np.int64) - sp.k, 0).sum())))
    torch.cuda.synchronize()
    return specs, sets


def measure_batched(args, sets, ctx):
    """256 one-at-a-time dbg_build calls against one dbg_build_batch call
    over the same read sets (device-resident inputs)."""
    import torch
    from paper_1003_1940_gb300 import dbg
    N = sum(s[3] for s in sets)
    trip = [(r, l, k) for r, l, k, _ in sets]
    # warm-up: a few sets both ways
    for g in dbg.dbg_build_batch(ctx, trip[:8], workers=args.workers):
        g.free()
    for r, l, k in trip[:8]:
        dbg.dbg_build(ctx, r, l, k).free()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for r, l, k in trip:
        dbg.dbg_build(ctx, r, l, k).free()
    torch.cuda.synchronize()
    one = time.perf_counter() - t
    t = time.perf_counter()
    graphs = dbg.dbg_build_batch(ctx, trip, workers=args.workers)
    torch.cuda.synchronize()
    bat = time.perf_counter() - t
    for g in graphs:
        g.free()
    return {"value": N / bat, "unit": UNIT, "one_at_a_time": N / one, "speedup": one / bat, "batched_s": bat,
            "one_at_a_time_s": one, "edge_instances": N, "sets": len(sets), "workers": args.workers,
            "largest_set_instances": max(s[3] for s in sets),
            "workload": f"{len(sets)} read sets: genome log-uniform 10 kbp-5 Mbp, coverage U[10,60], "
                        f"L in {{36,75,100,150}}, errors U[0,1%], k in {{21,31}}"}


def run_batched(args):
    from paper_1003_1940_gb300 import build_lib, dbg
    build_lib.build()
    dbg.load()
    specs, sets = batched_inputs(args)
    ctx = dbg.Context()
    dbg.dbg_autotune(ctx)
    res = measure_batched(args, sets, ctx)
    print(json.dumps({
        "metric": METRIC + " (batched vs one-at-a-time)", "value": res["value"], "unit": UNIT,
        "one_at_a_time": res["one_at_a_time"], "speedup": res["speedup"], "batched_s": res["batched_s"],
        "one_at_a_time_s": res["one_at_a_time_s"], "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": res["workload"], "edge_instances": res["edge_instances"], "workers": args.workers,
                   "largest_set_instances": res["largest_set_instances"]}}))


def measure_served(args, sets, ctx, big_r=None, big_l=None, big_spec=None):
    """Request-server capacity (closed loop over the read sets), then
    Poisson arrivals at 0.5, 0.8 and 1.0 of it: latency p50 / p99 and
    throughput; at 0.8 one larger request (the large workload, on the key-
    range bucket path) joins the stream."""
    import threading as th
    import torch
    from paper_1003_1940_gb300 import dbg
    variants = [dbg.dbg_sort_variant_get(ctx, kd) for kd in range(4)]
    # capacity: a closed loop over the whole set list
    srv = dbg.Server(workers=args.workers, sort_variant=variants)
    t = time.perf_counter()
    ts = [dbg.dbg_submit(srv, r, l, k) for r, l, k, _ in sets]
    for x in ts:
        dbg.dbg_poll(srv, x)[0].free()
    cap = len(sets) / (time.perf_counter() - t)
    if big_spec is None:
        # one larger request: the 15 M-read workload, through the bucket path
        big_spec = readgen.large_spec(args.scale)
        big_r, big_l = readgen.generate(big_spec)
        big_r, big_l = torch.from_numpy(big_r).cuda(), torch.from_numpy(big_l.view(np.int32)).cuda()
    out = {}
    for load in (0.5, 0.8, 1.0):
        rate = load * cap
        arrivals = readgen.poisson_arrivals(rate, 2 * len(sets), seed=4)
        order = np.random.default_rng(4).integers(0, len(sets), size=len(arrivals))
        lat, tickets = [], []
        done_n = [0]
        t0 = time.perf_counter()
        lock = th.Lock()

        def poller():
            while True:
                with lock:
                    if not tickets:
                        if done_n[0] < 0:
                            return
                        item = None
                    else:
                        item = tickets.pop(0)
                if item is None:
                    time.sleep(0.0005)
                    continue
                g, st = dbg.dbg_poll(srv, item)
                lat.append(st["latency_s"])
                g.free()

        pt = th.Thread(target=poller)
        pt.start()
        N = 0
        big_t = None
        for i, (a, j) in enumerate(zip(arrivals, order)):
            while time.perf_counter() - t0 < a:
                time.sleep(0.0002)
            r, l, k, ni = sets[j]
            tk = dbg.dbg_submit(srv, r, l, k)
            N += ni
            with lock:
                tickets.append(tk)
            if load == 0.8 and i == len(arrivals) // 2:
                big_t = dbg.dbg_submit(srv, big_r, big_l, big_spec.k, flags=dbg.DBG_REQ_BUCKETED)
        with lock:
            done_n[0] = -1
        pt.join()
        big = None
        if big_t is not None:
            g, st = dbg.dbg_poll(srv, big_t)
            big = {"latency_s": st["latency_s"], "bucketed": st["bucketed"],
                   "edge_instances": big_spec.raw_edges, "edge_ranges": dbg.dbg_graph_buckets(g)[0]}
            g.free()
            N += big_spec.raw_edges
        span = time.perf_counter() - t0
        lat = np.array(lat)
        out[str(load)] = {"rate_per_s": rate, "requests": len(arrivals), "throughput": N / span,
                          "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                          "big_request": big}
    srv.close()
    return {"unit": UNIT, "capacity_sets_per_s": cap, "loads": out, "workers": args.workers,
            "requests_per_load": 2 * len(sets)}


def run_served(args):
    from paper_1003_1940_gb300 import build_lib, dbg
    build_lib.build()
    dbg.load()
    specs, sets = batched_inputs(args)
    ctx = dbg.Context()
    dbg.dbg_autotune(ctx)
    res = measure_served(args, sets, ctx)
    print(json.dumps({"metric": METRIC + " (served, Poisson arrivals)", "data": "synthetic", "n_gpus": 1, **res}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
