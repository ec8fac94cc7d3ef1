"""Benchmark of the tile-based query operators on GB300.

Default workload (``--workload served``): the served star-schema stream — a fact table of
600M rows x 8 int32 columns resident in HBM and four dimensions (2556 / 200K / 3M / 1.4M
rows) held as direct tables of packed attribute codes; a step is one batch of 32 seeded
select-join-group-by queries compiled against those tables and run in ONE tagged shared
scan of the fact table (the batch's dimension rows tagged with query bitmaps, then one
scan).  ``value`` is queries/s over the K timed steps (CUDA events, inputs resident, fact
table 19.2 GB >> L2).  The JSON line also carries the one-query-at-a-time baseline on the
same GPU, the serving loop (continuous batching over row segments through the public
API, every launch a CUDA-graph replay: queries in from the host, results back to pinned
host memory) with p50/p99 latency at several offered loads, the dominant kernel's
roofline, the CPU oracle timed on a sample of the same workload, SM clocks sampled
during the timed region, and the number of library kernels launched.

Other workloads (``--workload select|project|join|sort|q1``) time one operator of the
hot path each and report GB/s of algorithmic traffic against measured HBM bandwidth.

``--impl reference`` times the oracle (plain CPU code) on the same workload, on the
host cores, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "scanned GB/s vs GB300 HBM peak per query; served queries/s, p50/p99 latency"
BATCH = 32
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------------------- helpers

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        # NCCL between the GPUs of our arm; gloo for the host-only reference arm (and
        # wherever no GPU is visible)
        gpu = args.impl != "reference" and torch.cuda.is_available()
        if gpu:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if gpu else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class KernelTimer:
    """CUDA events around launches on one stream; returns per-launch milliseconds."""

    def __init__(self, stream):
        self.stream = stream
        self.pairs = []

    def __enter__(self):
        import torch
        self.a = torch.cuda.Event(enable_timing=True)
        self.a.record(self.stream)
        return self

    def __exit__(self, *exc):
        import torch
        b = torch.cuda.Event(enable_timing=True)
        b.record(self.stream)
        self.pairs.append((self.a, b))

    def ms(self):
        return [a.elapsed_time(b) for a, b in self.pairs]


def l2_flush(buf):
    buf.zero_()


def graph_differential_ms(fn, flush, k=20, rounds=7):
    """Device time of one launch of `fn` after an L2 flush, free of per-launch host and
    event overhead: two CUDA graphs, k x {flush, fn} and k x {flush}, each replayed
    `rounds` times and timed with events; (median1 - median0) / k."""
    import torch
    g1, g0 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    fn()                                   # first call outside capture (attributes, caches)
    with torch.cuda.graph(g1):
        for _ in range(k):
            flush()
            fn()
    with torch.cuda.graph(g0):
        for _ in range(k):
            flush()
    stream = torch.cuda.current_stream()
    t1, t0 = [], []
    for _ in range(rounds):
        for g, out in ((g1, t1), (g0, t0)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
    return max(0.0, (statistics.median(t1) - statistics.median(t0)) / k)


# ----------------------------------------------------------------------------- served

def served_store(seed, n_rows, dim_scale, device):
    import datagen
    import datagen.device as dgd
    from paper_2003_01178_gb300.starschema import ResidentStarSchema, Schema
    t = dgd.ss_tables(seed, n_rows, device, dim_scale)
    return ResidentStarSchema(Schema.from_spec(datagen.SS_FACT_COLS, datagen.SS_DIMS), t["fact"], t["dims"])


def batch_queries(seed, step, rank=0):
    import datagen
    base = (rank * 100_000) + step * BATCH
    return [datagen.ss_query(seed, base + i) for i in range(BATCH)]


def served_config(args, world):
    """The served workload's config, identical in both arms of the bench."""
    return {"workload": f"served star-schema stream: fact {args.rows // 1_000_000}M rows x 8 int32 cols "
                        f"({args.rows * 32 / 1e9:.1f} GB), dims 2556/200K/3M/1.4M rows, batches of {BATCH} "
                        "seeded select-join-group-by queries (1-4 joins, selectivity 1e-4..0.5, <=1e4 groups, "
                        "int64 sums)",
            "fact_rows": args.rows, "batch_queries": BATCH, "seed": args.seed,
            "l2": "inputs larger than L2 (the fact table is read whole by every step)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_served(args, rank, world, local):
    import torch
    import datagen
    import paper_2003_01178_gb300 as crys

    dev = torch.device("cuda", local)
    seed = args.seed
    store = served_store(seed, args.rows, args.dim_scale, dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    peak, peak_kind = measured_hbm_peak()

    def one_step(step, timers=None, qs=None):
        qs = batch_queries(seed, step, rank) if qs is None else qs
        # outputs are cleared by the shared scan itself (it does not accumulate here)
        cqs = [store.compile(q, mode="resident", zero=False) for q in qs]
        if timers is not None:
            with timers:
                store.run_shared(cqs)
        else:
            store.run_shared(cqs)
        return qs, cqs

    tune_cqs = [store.compile(q, mode="resident") for q in batch_queries(seed, 20_000, rank)]
    tile = autotune(crys.OP_TAGGED_SCAN, lambda: store.run_shared(tune_cqs), args)
    del tune_cqs
    for w in range(args.warmup):
        one_step(10_000 + w)
    torch.cuda.synchronize(dev)
    scan_timer = KernelTimer(stream)
    # the workload's query dicts are inputs, generated before the timed region; planning
    # them against the store is part of every step
    step_queries = [batch_queries(seed, s, rank) for s in range(args.steps)]
    launches0 = crys.crys_launch_count()
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for s in range(args.steps):
            one_step(s, scan_timer, step_queries[s])
        end.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    launches = crys.crys_launch_count() - launches0
    elapsed_ms = max_over_ranks(start.elapsed_time(end), world)
    total_queries = BATCH * args.steps * world
    qps = total_queries / (elapsed_ms / 1e3)
    scan_ms = scan_timer.ms()
    avg_scan_ms = sum(scan_ms) / len(scan_ms)
    union_cols = len(store.schema.fact_cols)
    scan_bytes = union_cols * store.n_rows * 4
    per_query_bytes = [store.bytes_scanned(q) for qs in step_queries for q in qs]
    scanned_gbs = sum(per_query_bytes) / (elapsed_ms / 1e3) / 1e9 * world

    out = {
        "metric": METRIC, "value": round(qps, 2), "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded counter-based generator, generated in HBM)",
        "config": served_config(args, world), "tile": tile,
        "step_detail": f"compile {BATCH} queries against the resident direct dimension tables + one tagged "
                       "shared scan of the fact table: annotate_kernel tags every dimension row with "
                       "the bitmap of the batch's queries it satisfies, tagged_scan_kernel reads one "
                       "tag per dimension and fact row and finishes only the qualifying (row, query) "
                       "pairs; the query dicts (workload input) are generated before the timed region",
        "scanned_gbs": {"aggregate": round(scanned_gbs, 1),
                        "per_query_mean_gb": round(sum(per_query_bytes) / len(per_query_bytes) / 1e9, 3),
                        "note": "sum over queries of each query's own column bytes / wall time"},
        "gpu_launches": int(launches),
    }
    achieved = scan_bytes / (avg_scan_ms / 1e3) / 1e9
    out["roofline"] = {"kernel": "tagged_scan_kernel", "bound": "hbm", "achieved": round(achieved, 1),
                       "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                       "peak_source": peak_kind, "traffic": traffic_for("tagged_scan_kernel", "served"),
                       "algorithmic_bytes_per_launch": scan_bytes, "avg_launch_ms": round(avg_scan_ms, 4),
                       "timed": "one shared-scan call per batch on its stream: annotate_kernel + "
                                "tagged_scan_kernel"}
    # one query at a time on the same GPU, same batches: the paper's plan (per-query
    # filtered builds + one fused probe kernel) and the same kernel on the resident tables
    if not args.quick:
        out["one_at_a_time"] = {}
        # the single-query kernel gets its own tuned tile shape, as the shared scan did
        plan_cqs = [store.compile(q, mode="resident") for q in batch_queries(seed, 20_001, rank)[:8]]
        out["one_at_a_time"]["tile"] = autotune(crys.OP_PLAN, lambda: [store.run(c) for c in plan_cqs], args)
        del plan_cqs
        for mode in ("filtered", "resident"):
            alone_ms = []
            for s in range(min(args.steps, 3)):
                qs = batch_queries(seed, s, rank)
                torch.cuda.synchronize(dev)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for q in qs:
                    cq = store.compile(q, mode=mode)
                    store.run(cq)
                b.record(stream)
                torch.cuda.synchronize(dev)
                alone_ms.append(a.elapsed_time(b))
            out["one_at_a_time"][mode] = round(BATCH / (sum(alone_ms) / len(alone_ms) / 1e3), 2)
        out["one_at_a_time"]["unit"] = "queries/s"
        out["one_at_a_time"]["note"] = ("same batches, one fused probe kernel per query, same GPU; "
                                        "filtered = per-query filtered dimension builds (the paper's plan), "
                                        "resident = shared packed dimension tables")
        out["served"] = served_loop(store, args, rank)
        out["e2e"] = {"value": out["served"]["closed_loop_qps"], "unit": "queries/s",
                      "h2d_bytes_per_step": out["served"]["h2d_bytes_per_batch"],
                      "d2h_bytes_per_step": out["served"]["d2h_bytes_per_batch"],
                      "bytes_counted": "from the tensors copied in the closed loop, per batch of "
                                       f"{BATCH} queries",
                      "what": "public serving API, closed loop: query dicts in from the host, plans "
                              "compiled, each launch's argument block copied from pinned host memory "
                              "(h2d), circular tagged shared scans replayed from CUDA graphs, int64 "
                              "results copied to pinned host memory (d2h); fact table resident (the "
                              "workload's premise)"}
    out["clocks"] = clocks.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_served(store, args)
    if not args.no_operators and not args.quick:
        # configs 1-4 at their stated sizes on the same GPU (the served store stays resident)
        out["operators"] = run_operators_block(args, dev, stream)
        out["paper_context"] = {
            "note": "the paper's figures, for context only (other hardware, other baselines)",
            "bandwidth_ratio": "16.2x: V100 (880 GB/s) over i7-6900 (about 54 GB/s), Section 4",
            "ssb_end_to_end": "25x average: SSB at scale factor 20, V100 over i7-6900, Section 5.2",
            "this_run_gpu_over_oracle": round(out["value"] / out["cpu_baseline"]["value"], 1)
            if out["cpu_baseline"]["value"] else None}
    return out


def served_loop(store, args, rank):
    import datagen
    from paper_2003_01178_gb300.server import QueryServer
    n = args.served_queries
    queries = [datagen.ss_query(args.seed, 500_000 + rank * 100_000 + i) for i in range(n)]
    server = QueryServer(store, segments=args.segments, max_slots=BATCH, memory_budget=16 << 30)
    # closed loop: every request queued at t=0 (throughput)
    _, st_closed = server.serve(queries, np.zeros(n), realtime=False)
    # open loop: Poisson arrivals at 70% of the closed-loop rate (latency), and the
    # latency at a few other offered loads
    rate = max(1.0, 0.7 * st_closed.qps)
    arrivals = datagen.ss_arrivals(args.seed, n, rate)
    _, st_open = server.serve(queries, arrivals, realtime=True)
    curve = []
    for load in (0.3, 0.5, 0.9):
        r = max(1.0, load * st_closed.qps)
        _, st = server.serve(queries, datagen.ss_arrivals(args.seed + 1, n, r), realtime=True)
        curve.append({"offered_qps": round(r, 1), "served_qps": round(st.qps, 1),
                      "p50_ms": round(st.percentile_ms(50), 2), "p99_ms": round(st.percentile_ms(99), 2)})
    batches = max(1.0, st_closed.completed / BATCH)
    return {"closed_loop_qps": round(st_closed.qps, 2), "open_loop_offered_qps": round(rate, 2),
            "open_loop_qps": round(st_open.qps, 2),
            "p50_ms": round(st_open.percentile_ms(50), 3), "p99_ms": round(st_open.percentile_ms(99), 3),
            "latency_by_load": curve,
            "closed_loop_p50_ms": round(st_closed.percentile_ms(50), 3),
            "closed_loop_p99_ms": round(st_closed.percentile_ms(99), 3),
            "queries": n, "segments": args.segments, "max_active": st_open.max_active,
            "launches": st_open.launches,
            "graph_replays": st_open.replays + st_closed.replays,
            "launch": "each launch replays a captured CUDA graph {pinned argument block -> device, "
                      "prepare_kernel, tagged_scan_kernel_dev}",
            # bytes the closed loop copied (argument blocks in, int64 results out), per batch
            "h2d_bytes_per_batch": int(st_closed.h2d_bytes / batches),
            "d2h_bytes_per_batch": int(st_closed.d2h_bytes / batches),
            "peak_held_bytes": st_closed.peak_held_bytes}


def oracle_threads():
    import oracle
    return oracle.hardware_threads()


def time_oracle_query(host, query, threads, fact_rows=None):
    """Wall seconds of the oracle (as it stands) for one served query."""
    import oracle
    t0 = time.perf_counter()
    oracle.ss_run(host, query, threads=threads, fact_rows=fact_rows)
    return time.perf_counter() - t0


def cpu_baseline_served(store, args):
    """The oracle (plain row-at-a-time C, rows split over all host threads) timed over ALL
    fact rows for the first `cpu_queries` queries of the first batch; a linear
    extrapolation from the first 2M rows is kept beside it as a cross-check."""
    host = {"fact": {c: store.fact[c].cpu().numpy() for c in store.schema.fact_cols},
            "dims": {d: {k: v.cpu().numpy() for k, v in t.items()} for d, t in store.dims.items()}}
    threads = oracle_threads()
    qs = batch_queries(args.seed, 0)[: args.cpu_queries]
    full = [time_oracle_query(host, q, threads) for q in qs]
    sample = min(2_000_000, store.n_rows)
    extrap = []
    for q in qs:
        fixed = time_oracle_query(host, q, threads, fact_rows=0)
        part = time_oracle_query(host, q, threads, fact_rows=sample)
        extrap.append(fixed + max(0.0, part - fixed) / sample * store.n_rows)
    del host
    return {"value": round(len(qs) / sum(full), 4), "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(qs)} queries of the first batch, each timed over all {store.n_rows} fact rows "
                      f"({sum(full):.1f} s of oracle time)",
            "seconds_per_query": [round(t, 3) for t in full],
            "cross_check_extrapolated_from_2M_rows": round(len(qs) / sum(extrap), 4)}


def host_star_schema(seed, rows, dim_scale, threads):
    """Host copy of the served star schema, generated in row chunks on `threads` threads
    (the generator is a pure function of (seed, stream, row), so chunks are independent)."""
    from concurrent.futures import ThreadPoolExecutor
    import datagen
    chunk = 1 << 24
    fact = {c: np.empty(rows, dtype=np.int32) for c in datagen.SS_FACT_COLS}

    def fill(job):
        c, b = job
        e = min(rows, b + chunk)
        fact[c][b:e] = datagen.ss_fact_col(seed, c, e - b, start=b, dim_scale=dim_scale)
    with ThreadPoolExecutor(max(1, threads)) as ex:
        list(ex.map(fill, [(c, b) for c in datagen.SS_FACT_COLS for b in range(0, rows, chunk)]))
    dims = {d: datagen.ss_dimension(seed, d, dim_scale) for d in datagen.SS_DIMS}
    return {"fact": fact, "dims": dims}


# ----------------------------------------------------------------------------- operators
#
# Configs 1-4 (Section 4 microbenchmarks and the fused query of Section 5.3), each timed
# by one function that returns a plain dict: milliseconds, algorithmic GB/s against the
# measured HBM peak, and the tile shape the tuner chose.  The default run puts them all in
# an "operators" block of the served line; ``--workload <name>`` prints one as its own line.

KERNEL_FILES = {"select_kernel": "select.cu", "project_kernel": "project.cu", "probe_kernel": "hash.cu",
                "sort_pass_kernel": "sort.cu", "plan_kernel": "plan.cu", "plan_fixed_kernel": "plan.cu",
                "tagged_scan_kernel": "plan.cu",
                "shared_scan_kernel": "plan.cu"}


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current source of the kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        src_hash = kernel_source_hash(kernel)
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[2] == src_hash:
                    return int(parts[3])
    except Exception:
        pass
    return None


def kernel_source_hash(kernel):
    """Hash of the source file that defines `kernel` and of every header of the library."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_01178_gb300", "csrc")
    files = [KERNEL_FILES[kernel]] + sorted(f for f in os.listdir(csrc) if f.endswith((".cuh", ".h")))
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def gbs(alg_bytes, ms):
    return alg_bytes / (ms / 1e3) / 1e9


def frac(alg_bytes, ms):
    return round(gbs(alg_bytes, ms) / measured_hbm_peak()[0], 4)


def autotune(op, launch, args):
    """Pick the tile shape of `op` on this workload (crys_tile_variants x timing) unless
    --no-tune; returns the chosen (threads, items) and the median ms of every variant."""
    import paper_2003_01178_gb300 as crys
    from paper_2003_01178_gb300 import tuner
    times = {}
    if not args.no_tune:
        res = tuner.tune(op, launch, reps=3, warmup=1)
        times = {f"{v['threads']}x{v['items']}": round(v["ms"], 4) for v in res["variants"].values()}
    v = crys.crys_get_tile(op)
    return {"shape": list(crys.crys_tile_variants(op)[v]), "variants_ms": times}


def time_launches(fn, steps, warmup, stream, flush=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def op_select(args, dev, stream, n=1 << 29, strawman=True):
    """Config 2(1): selection of 2^29 int32 uniform in [0, 2^31), x < v, sigma 0..1."""
    import torch
    import datagen
    import datagen.device as dgd
    import paper_2003_01178_gb300 as crys
    x = dgd.uniform_i32(args.seed, datagen.STREAMS["sel.x"], n, 0, (1 << 31) - 1, dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    his = [datagen.select_threshold(i / 10) for i in range(11)]

    def whole_sweep():  # the metric is the mean over the sweep, so tune on all of it
        for hi in his:
            crys.crys_select(x, n, -(1 << 31), hi, out, cnt, 0)
    tile = autotune(crys.OP_SELECT, whole_sweep, args)
    sweep = {}
    for sigma in [i / 10 for i in range(11)]:
        hi = datagen.select_threshold(sigma)
        ms = time_launches(lambda: crys.crys_select(x, n, -(1 << 31), hi, out, cnt, 0), args.steps, args.warmup, stream)
        sweep[f"{sigma:.1f}"] = statistics.median(ms)
    avg = statistics.mean(sweep.values())
    alg = statistics.mean([4 * n * (1 + float(s)) for s in sweep])
    res = {"kernel": "select_kernel", "rows": n, "ms_mean": round(avg, 4), "alg_bytes_mean": int(alg),
           "GB/s": round(gbs(alg, avg), 1), "frac": frac(alg, avg),
           "ms_at_0.5": round(sweep["0.5"], 4), "frac_at_0.5": frac(4 * n * 1.5, sweep["0.5"]),
           "sweep_ms": {k: round(v, 4) for k, v in sweep.items()}, "tile": tile,
           "bytes": "4N read + 4 sigma N written (Section 4.2 model)"}
    if strawman:
        # the independent-threads selection the paper compares against (ablation)
        stb = crys.crys_select_strawman(None, n, -(1 << 31), 0, None, None, None, -1)
        stemp = crys.scratch(stb, dev)
        straw = {}
        for sigma in (0.0, 0.5, 1.0):
            hi = datagen.select_threshold(sigma)
            ms = time_launches(lambda: crys.crys_select_strawman(x, n, -(1 << 31), hi, out, cnt, stemp, stb),
                               args.steps, args.warmup, stream)
            straw[f"{sigma:.1f}"] = round(statistics.median(ms), 4)
        res["independent_threads"] = {
            "ms": straw, "slowdown_at_0.5": round(straw["0.5"] / sweep["0.5"], 2),
            "paper": "19 ms independent threads vs 2.1 ms tile-based, V100, 2^29 rows, sigma 0.5 (Section 3.2)"}
    del x, out
    return res


def op_project(args, dev, stream, n=1 << 29):
    """Config 2(2): y = 2 x1 + 3 x2 and its sigmoid over 2^29 float32 rows."""
    import torch
    import datagen
    import datagen.device as dgd
    import paper_2003_01178_gb300 as crys
    x1 = dgd.uniform_f32(args.seed, datagen.STREAMS["proj.x1"], n, dev)
    x2 = dgd.uniform_f32(args.seed, datagen.STREAMS["proj.x2"], n, dev)
    y = torch.empty_like(x1)
    tile = autotune(crys.OP_PROJECT, lambda: crys.crys_project(x1, x2, n, 2.0, 3.0, crys.PROJ_LINEAR, y), args)
    ms = {}
    for op, nm in ((crys.PROJ_LINEAR, "linear"), (crys.PROJ_SIGMOID, "sigmoid")):
        ms[nm] = statistics.median(time_launches(lambda: crys.crys_project(x1, x2, n, 2.0, 3.0, op, y),
                                                 args.steps, args.warmup, stream))
    avg = statistics.mean(ms.values())
    del x1, x2, y
    return {"kernel": "project_kernel", "rows": n, "ms_mean": round(avg, 4), "alg_bytes": 12 * n,
            "GB/s": round(gbs(12 * n, avg), 1), "frac": frac(12 * n, avg),
            "ms": {k: round(v, 4) for k, v in ms.items()},
            "frac_by_op": {k: frac(12 * n, v) for k, v in ms.items()}, "tile": tile,
            "bytes": "8N read + 4N written (Section 4.1 model)"}


def op_q1(args, dev, stream, sizes):
    """Config 1: the fused filter-probe-aggregate query (yr == 3 AND a < 25 AND 1 <= b <= 3,
    SUM(c * b)) at each fact size, L2 flushed before every timed launch."""
    import torch
    import datagen.device as dgd
    import paper_2003_01178_gb300 as crys
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for n in sizes:
        t = dgd.q1_tables(args.seed, n, dev)
        f, d = t["fact"], t["dim"]
        # the dense date keys get a direct table (perfect hashing: slot k holds key k)
        ht = crys.HashTable.build(d["key"], d["yr"], filters=[(d["yr"], 3, 3)], capacity=d["key"].numel(),
                                  kind=crys.HASH_DIRECT)
        sums = torch.zeros(1, dtype=torch.int64, device=dev)
        cnts = torch.zeros(1, dtype=torch.int64, device=dev)
        table = crys.make_table([f["fk"], f["a"], f["b"], f["c"]])
        plan = crys.make_plan([(1, -(1 << 31), args.q1_a_max), (2, 1, 3)], [(0, ht, 0)], ("mul", 3, 2), sums, cnts)
        tile = autotune(crys.OP_PLAN, lambda: (l2_flush(flush_buf), crys.crys_run_plan(table, plan)), args)
        if tile.get("variants_ms"):
            tile["variants_note"] = "each variant timed with the 512 MB L2 flush before its launch"
        ms = statistics.median(time_launches(lambda: crys.crys_run_plan(table, plan), args.steps, args.warmup,
                                             stream, flush=lambda: l2_flush(flush_buf)))
        graphed = graph_differential_ms(lambda: crys.crys_run_plan(table, plan), lambda: l2_flush(flush_buf))
        out[str(n)] = {"ms": round(ms, 4), "GB/s": round(gbs(16 * n, ms), 1), "frac": frac(16 * n, ms),
                       "graph_ms": round(graphed, 4),
                       "graph_frac": frac(16 * n, graphed) if graphed > 0 else None, "tile": tile}
        # the same query with a selective first predicate (a == 1, 2% of rows): the
        # aggregate column c is then read only for the few 16-byte groups with a live row
        sel = crys.make_plan([(1, 1, 1), (2, 1, 3)], [(0, ht, 0)], ("mul", 3, 2), sums, cnts)
        sms = statistics.median(time_launches(lambda: crys.crys_run_plan(table, sel), args.steps, args.warmup,
                                              stream, flush=lambda: l2_flush(flush_buf)))
        out[str(n)]["selective_a_eq_1"] = {"ms": round(sms, 4), "GB/s_of_16B_rows": round(gbs(16 * n, sms), 1),
                                           "speedup_over_dense_query": round(ms / sms, 3)}
        del t, f, d, ht, table, plan, sel
    del flush_buf
    return {"kernel": "plan_kernel", "by_rows": out, "bytes": "16 B per fact row: 4 columns (Section 3.1 bound)",
            "plan": "the 2556-row date dimension in a direct table (perfect hashing of the dense keys) filtered "
                    "on yr == 3, probed by one fused kernel",
            "l2": "flushed before each timed launch (512 MB write)",
            "graph_ms_note": "per-launch device time from CUDA-graph replays of k x {L2 flush, kernel} minus "
                             "k x {L2 flush}: no launch or event overhead"}


def op_sort(args, dev, stream, n=1 << 28):
    """Config 4: radix sort of 2^28 (key, row id) pairs."""
    import torch
    import datagen
    import datagen.device as dgd
    import paper_2003_01178_gb300 as crys
    keys = dgd.bits_i32(args.seed, datagen.STREAMS["sort.key"], n, dev)
    vals = torch.arange(n, dtype=torch.int32, device=dev)
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    tb = crys.crys_sort(None, None, None, None, n, None, -1)
    temp = crys.scratch(tb, dev)
    tile = autotune(crys.OP_SORT, lambda: crys.crys_sort(keys, vals, ko, vo, n, temp, tb), args)
    ms = statistics.median(time_launches(lambda: crys.crys_sort(keys, vals, ko, vo, n, temp, tb),
                                         args.steps, args.warmup, stream))
    res = {"kernel": "sort_pass_kernel", "rows": n, "lsd_stable": {
        "ms": round(ms, 4), "Mkeys/s": round(n / (ms / 1e3) / 1e6, 1), "GB/s": round(gbs(68 * n, ms), 1),
        "frac": frac(68 * n, ms), "tile": tile,
        "bytes": "one 4N key read for all digit histograms + 4 passes x (8N read + 8N written) = 68N"},
        "paper": "V100: 27.08 ms for 2^28 key+value pairs, unstable MSB sort (Section 4.4)"}
    del temp
    # the paper's own GPU sort: most-significant-digit first, unstable
    tb = crys.crys_sort_msb(None, None, None, None, n, None, -1)
    temp = crys.scratch(tb, dev)
    ms = statistics.median(time_launches(lambda: crys.crys_sort_msb(keys, vals, ko, vo, n, temp, tb),
                                         args.steps, args.warmup, stream))
    res["msb_unstable"] = {
        "ms": round(ms, 4), "Mkeys/s": round(n / (ms / 1e3) / 1e6, 1), "GB/s": round(gbs(56 * n, ms), 1),
        "frac": frac(56 * n, ms), "over_lsd": round(res["lsd_stable"]["ms"] / ms, 3),
        "bytes": "2 partition passes x (4N histogram read + 8N read + 8N written) + local sort of every "
                 "16-bit bucket (8N read + 8N written) = 56N"}
    del keys, vals, ko, vo, temp
    return res


def op_join(args, dev, stream, sizes, n_probe=1 << 28, partial=True):
    """Config 3: build N unique keys at 50% fill, probe 2^28 foreign keys, SUM(payload * value)."""
    import torch
    import datagen
    import datagen.device as dgd
    import paper_2003_01178_gb300 as crys
    res = {}
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 126 << 20))
    pay = dgd.uniform_i32(args.seed, datagen.STREAMS["join.pay"], n_probe, 1, 100, dev)
    for lg in sizes:
        nb = 1 << lg
        bk = dgd.perm_i32(args.seed, datagen.STREAMS["join.bkey"], nb, dev)
        bv = dgd.uniform_i32(args.seed, datagen.STREAMS["join.bval"], nb, 1, 100, dev)
        ht = crys.HashTable.build(bk, bv)
        fk = dgd.uniform_i32(args.seed, datagen.STREAMS["join.fk"], n_probe, 0, nb - 1, dev)
        s = torch.zeros(2, dtype=torch.int64, device=dev)
        tile = autotune(crys.OP_PROBE, lambda: crys.crys_probe_aggregate(fk, pay, n_probe, ht.struct, s[0:1], s[1:2]),
                        args)
        pm = statistics.median(time_launches(
            lambda: crys.crys_probe_aggregate(fk, pay, n_probe, ht.struct, s[0:1], s[1:2]), args.steps, args.warmup,
            stream))
        bms = statistics.median(time_launches(
            lambda: (crys.crys_hash_init(ht.struct), crys.crys_hash_build(bk, bv, nb, [], ht.struct)),
            max(1, args.steps // 2), 1, stream))
        # Section 4.3 model: the probe scan plus, for each probe that misses L2 (hit share
        # pi = L2 size / table size, at most 1), the line a miss fills: 32 B in the paper's
        # sector reading, 128 B as measured on this GPU (every random miss fills a whole
        # 128-byte line; see the probe_kernel locality summary)
        pi = min(1.0, l2_bytes / ht.nbytes)
        model32 = 8 * n_probe + (1.0 - pi) * n_probe * 32
        model128 = 8 * n_probe + (1.0 - pi) * n_probe * 128
        res[f"2^{lg}"] = {"probe_ms": round(pm, 4), "build_ms": round(bms, 4),
                          "table_mb": round(ht.nbytes / 2 ** 20, 3), "tile": tile,
                          "model_bytes": int(model32), "model_frac": frac(model32, pm),
                          "model_bytes_128B_lines": int(model128), "model_frac_128B_lines": frac(model128, pm)}
        del ht
        if lg >= args.partition_from:
            # the radix-partitioned join on the same inputs (build and probe included)
            jtb = crys.crys_join_partitioned(None, None, nb, None, None, n_probe, None, None, None, -1)
            jtemp = crys.scratch(jtb, dev)
            jm = statistics.median(time_launches(
                lambda: crys.crys_join_partitioned(bk, bv, nb, fk, pay, n_probe, s[0:1], s[1:2], jtemp, jtb),
                args.steps, args.warmup, stream))
            bits = 0
            while bits < 16 and (nb >> bits) > 2048:
                bits += 1
            passes = 0 if bits == 0 else (1 if bits == 1 else 2)
            jbytes = passes * 20 * (nb + n_probe) + 8 * (nb + n_probe)
            res[f"2^{lg}"]["partitioned"] = {
                "ms": round(jm, 4), "over_build_plus_probe": round((pm + bms) / jm, 3),
                "over_probe_alone": round(pm / jm, 3), "hash_bits": bits, "passes": passes,
                "GB/s": round(gbs(jbytes, jm), 1), "frac": frac(jbytes, jm),
                "bytes": "per partition pass 20 B per row of each side (4 B histogram read, 8 B read, 8 B "
                         "written), then 8 B per row of each side read by the per-partition build and probe"}
            del jtemp
        del bk, bv, fk
    out = {"kernel": "probe_kernel", "probe_rows": n_probe, "fill": "50%", "sweep": res, "l2_bytes": l2_bytes,
           "note": "model bytes = probe scan 8|P| + (1 - pi)|P| x line, pi = min(1, L2 / table) (Section 4.3 "
                   "model); line = 32 B (sector) or 128 B (the line a random miss fills on this GPU)"}
    if partial:
        # partial matches on the largest table: probe keys spread over [0, N / pi), so a
        # share pi of them finds its key (the others read a slot and miss)
        lg = sizes[-1]
        nb = 1 << lg
        bk = dgd.perm_i32(args.seed, datagen.STREAMS["join.bkey"], nb, dev)
        bv = dgd.uniform_i32(args.seed, datagen.STREAMS["join.bval"], nb, 1, 100, dev)
        ht = crys.HashTable.build(bk, bv)
        part = {}
        for pi in (0.5, 0.1):
            fk = dgd.uniform_i32(args.seed, datagen.STREAMS["join.fk"], n_probe, 0, int(nb / pi) - 1, dev)
            s = torch.zeros(2, dtype=torch.int64, device=dev)
            ms = time_launches(lambda: crys.crys_probe_aggregate(fk, pay, n_probe, ht.struct, s[0:1], s[1:2]),
                               args.steps, args.warmup, stream)
            part[f"{pi}"] = {"probe_ms": round(statistics.median(ms), 4),
                             "matched": round(int(s[1].item()) / n_probe, 4)}
            del fk
        out["partial_match_largest_table"] = part
        del ht, bk, bv
    del pay
    return out


def run_operators_block(args, dev, stream):
    """Every operator config at its stated size, with its own clock record."""
    import torch
    ops = {}
    with ClockSampler(dev.index if dev.index is not None else 0) as clocks:
        ops["q1"] = op_q1(args, dev, stream, [1 << 22, 1 << 28])
        ops["select"] = op_select(args, dev, stream)
        ops["project"] = op_project(args, dev, stream)
        ops["sort"] = op_sort(args, dev, stream)
        ops["join"] = op_join(args, dev, stream, [10, 22, 27], partial=False)
        torch.cuda.synchronize(dev)
    ops["clocks"] = clocks.summary()
    ops["peak_gbs"], ops["peak_source"] = measured_hbm_peak()
    return ops


def op_line(args, world, name, value, unit, kernel, alg_bytes, avg_ms, config, extra=None):
    peak, kind = measured_hbm_peak()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    out = {"metric": METRIC, "value": round(value, 2), "unit": unit, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(avg_ms, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": config.pop("dtype", "int32"), "data": "synthetic (seeded counter-based generator)",
           "config": dict(workload=name, **config),
           "roofline": {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": kind,
                        "traffic": traffic_for(kernel, name), "algorithmic_bytes_per_launch": int(alg_bytes),
                        "avg_launch_ms": round(avg_ms, 4)}}
    if extra:
        out.update(extra)
    return out


def run_operator(args, rank, world, local):
    import torch
    import paper_2003_01178_gb300 as crys

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    launches0 = crys.crys_launch_count()
    with ClockSampler(local) as clocks:
        if args.workload == "select":
            r = op_select(args, dev, stream, args.rows or (1 << 29))
            line = op_line(args, world, "select", r["GB/s"], "GB/s", "select_kernel", r["alg_bytes_mean"],
                           r["ms_mean"], {"rows": r["rows"], "selectivity": "0.0..1.0 step 0.1 (mean over the sweep)",
                                          "l2": "inputs larger than L2"}, {"select": r})
        elif args.workload == "project":
            r = op_project(args, dev, stream, args.rows or (1 << 29))
            line = op_line(args, world, "project", r["GB/s"], "GB/s", "project_kernel", r["alg_bytes"], r["ms_mean"],
                           {"rows": r["rows"], "dtype": "f32", "l2": "inputs larger than L2"}, {"project": r})
        elif args.workload == "join":
            r = op_join(args, dev, stream, args.join_sizes, args.rows or (1 << 28))
            last = r["sweep"][f"2^{args.join_sizes[-1]}"]
            line = op_line(args, world, "join", gbs(last["model_bytes"], last["probe_ms"]), "GB/s", "probe_kernel",
                           last["model_bytes"], last["probe_ms"],
                           {"probe_rows": r["probe_rows"], "build_rows": f"2^{args.join_sizes[0]}..2^{args.join_sizes[-1]}",
                            "fill": "50%", "l2": "probe side larger than L2"}, {"join": r})
        elif args.workload == "sort":
            r = op_sort(args, dev, stream, args.rows or (1 << 28))
            s = r["lsd_stable"]
            line = op_line(args, world, "sort", s["Mkeys/s"], "Mkeys/s", "sort_pass_kernel", 68 * r["rows"], s["ms"],
                           {"rows": r["rows"], "l2": "inputs larger than L2", "passes": "4 x 8-bit, stable"},
                           {"sort": r})
        elif args.workload == "q1":
            sizes = [args.rows] if args.rows else [1 << 22, 1 << 28]
            r = op_q1(args, dev, stream, sizes)
            n = sizes[0]
            q = r["by_rows"][str(n)]
            # the library runs the kernel compiled for this plan's shape when each block takes
            # at most 8 tiles (every tile shape at 2^22 rows), the generic one otherwise
            kernel = "plan_fixed_kernel" if n <= (1 << 22) else "plan_kernel"
            per_call = q["graph_ms"] if q.get("graph_ms") else q["ms"]
            line = op_line(args, world, "q1", q["GB/s"], "GB/s", kernel, 16 * n, per_call,
                           {"rows": n, "dtype": "int64", "l2": "flushed between timed launches (512 MB write)",
                            "query": f"yr == 3 AND a <= {args.q1_a_max} AND 1 <= b <= 3, SUM(c * b), 2556-row "
                                     "date-like dimension"},
                           {"q1": r})
            line["ms_per_step"] = q["ms"]
            line["roofline"]["timed"] = ("per call from CUDA-graph replays of k x {L2 flush, call} minus k x {L2 flush} "
                                         "on the launching stream (events around the replays): the output clearing "
                                         "and the query kernel, without the host's launch preparation; the event-timed "
                                         "single call is `ms_per_step` and q1.by_rows.ms")
        else:
            raise SystemExit(f"unknown workload {args.workload}")
    line["gpu_launches"] = int(crys.crys_launch_count() - launches0)
    line["clocks"] = clocks.summary()
    return line


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, as the reference arm: every step runs
    `ref_queries` queries of the step's batch over ALL fact rows (wall time per step is
    the measured duration), reported in our arm's unit and config."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    threads = oracle.hardware_threads()
    if args.workload != "served":
        raise SystemExit("--impl reference is implemented for the served workload")
    t0 = time.perf_counter()
    host = host_star_schema(args.seed, args.rows, args.dim_scale, threads)
    gen_s = time.perf_counter() - t0
    step_s = []
    for s in range(args.warmup + args.steps):
        qs = batch_queries(args.seed, s)[: args.ref_queries]
        t0 = time.perf_counter()
        for q in qs:
            oracle.ss_run(host, q, threads=threads)
        if s >= args.warmup:
            step_s.append(time.perf_counter() - t0)
    total = sum(step_s)
    nq = args.ref_queries * args.steps
    qps = nq / total
    return {"metric": METRIC, "value": round(qps, 4), "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded counter-based generator)", "impl": "reference",
            "config": served_config(args, world),
            "cpu_baseline": {"value": round(qps, 4), "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: {args.ref_queries} of the step's {BATCH} queries, timed over "
                                       f"all {args.rows} fact rows (a step is a fraction of a batch: the oracle "
                                       f"takes seconds per query); inputs generated on the host in {gen_s:.1f} s "
                                       "before the timed steps"},
            "e2e": {"value": round(qps, 4), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- main

def main():
    global BATCH
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="served", choices=["served", "select", "project", "join", "sort", "q1"])
    p.add_argument("--rows", type=int, default=None)
    p.add_argument("--dim-scale", type=float, default=1.0)
    p.add_argument("--seed", type=int, default=0xC0FFEE + 4)
    p.add_argument("--segments", type=int, default=8)
    p.add_argument("--batch", type=int, default=BATCH, help="queries per shared scan (1..32)")
    p.add_argument("--served-queries", type=int, default=512)
    p.add_argument("--cpu-queries", type=int, default=2, help="queries timed on the CPU for cpu_baseline")
    p.add_argument("--ref-queries", type=int, default=1, help="queries per step of the reference arm")
    p.add_argument("--join-sizes", type=int, nargs="+", default=[10, 14, 18, 20, 22, 24, 26, 27])
    p.add_argument("--partition-from", type=int, default=20,
                   help="time the radix-partitioned join for build sides of at least 2^k rows")
    p.add_argument("--q1-a-max", type=int, default=24, help="Q1's fact predicate a <= this (24: a < 25)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true", help="skip the one-at-a-time, served-loop and operator legs")
    p.add_argument("--no-operators", action="store_true", help="skip the operators block (configs 1-4)")
    p.add_argument("--no-tune", action="store_true", help="keep the default tile shapes")
    args = p.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if not 1 <= args.batch <= 32:
        raise SystemExit("--batch must be in 1..32")
    BATCH = args.batch
    if args.workload == "served" and args.rows is None:
        args.rows = 600_000_000
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    import paper_2003_01178_gb300 as crys
    crys.lib()
    if args.workload == "served":
        line = run_served(args, rank, world, local)
    else:
        line = run_operator(args, rank, world, local)
    crys.check_device_errors()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
