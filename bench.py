"""Benchmark: forward + backward predicate transfer on one B300.

Workload (default): the 6-table snowflake at 10x (fact 60M rows, mid 15M,
dim2 2M, dim1 1.5M, dim3 100k, a 25-row table), int64 keys, a two-column
composite key on the fact->mid edge, Zipf(1.1)-skewed fact foreign keys,
predicates keeping 10% / 1% / 30% of dim1 / dim2 / dim3, Bloom filters of
16 bits per key (k = 4, 256-bit blocks).  Synthetic data (seeded), a
stand-in for TPC-H at scale factor 10.

One step = pt_run_forward + pt_run_backward over every table (both passes
of the paper's Section 3.2 schedule).  Metric: transfer rows/s = rows of
every visited table summed over both passes / step time.  Inputs are
resident in HBM when the timed region starts; the working set (~2.3 GB)
is far larger than L2 (126 MB), so no flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (the paper's engine is a single-core CPU program; the oracle is
its stand-in here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FALLBACK_HBM_GBS = 6400.0
NOMINAL_HBM_GBS = 8000.0


def make_workload(name: str, bpk: int, scale: float = 10.0):
    if name == "snowflake_x10":
        return W.snowflake(scale=scale, int64=True, composite=True, zipf=1.1, bits_per_key=bpk)
    if name == "snowflake":
        return W.snowflake(scale=1, bits_per_key=bpk)
    if name == "cyclic5":
        return W.cyclic5(bits_per_key=bpk)
    if name == "chain3":
        return W.chain3(bits_per_key=bpk)
    raise SystemExit(f"unknown workload {name}")


def workload_desc(w) -> dict:
    return {
        "workload": w.name,
        "tables": {t.name: t.n_rows for t in w.tables},
        "key_dtypes": sorted({str(c.dtype) for t in w.tables for c in t.cols}),
        "edges": len(w.edges),
        "bits_per_key": w.bits_per_key, "k": w.k, "block_bits": w.block_bits,
        "passes": "forward+backward",
        "l2": (f"inputs larger than L2 (working set {w.nbytes() / 1e9:.2f} GB vs 126 MB), no flush"
               if w.nbytes() > 126e6 else
               f"working set {w.nbytes() / 1e9:.3f} GB fits the 126 MB L2 (no flush: a small-scale run)"),
    }


def visit_rows(w) -> int:
    return 2 * sum(t.n_rows for t in w.tables)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as f:
                return json.load(f)
        except Exception:
            return {}
    return {}


def hbm_peak() -> tuple:
    pk = measured_peaks()
    for key in ("hbm_gbs", "hbm_copy_gbs", "hbm"):
        if key in pk and isinstance(pk[key], (int, float)):
            return float(pk[key]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_timing(w, budget_s: float, threads: int) -> dict:
    """The C oracle as it stands, on `threads` host threads (1: the plain
    build; more: the OpenMP build of the same source, identical results),
    repeated full transfers of the workload for about budget_s seconds."""
    import oracle
    oracle.build()
    used = 1
    if threads > 1:
        used = oracle.lib_threads(threads)[1]
    rows = visit_rows(w)
    oracle.transfer(w, threads=used)  # warm: page in the columns
    t0 = time.perf_counter()
    runs = 0
    while True:
        oracle.transfer(w, threads=used)
        runs += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    build = "single-threaded C oracle" if used == 1 else f"C oracle, OpenMP build on {used} threads"
    return {"value": rows * runs / dt, "unit": "rows/s", "cores": used, "kind": "oracle",
            "sample": f"{runs} full forward+backward transfer(s) of {w.name} ({rows} visit rows each), "
                      f"{build}, {dt:.1f} s"}


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload, args.bpk, args.scale)
    rows = visit_rows(w)
    import oracle
    oracle.build()
    # every host core: the OpenMP build of the oracle (identical results)
    cores = oracle.lib_threads(host_cores())[1]
    for _ in range(args.warmup):
        oracle.transfer(w, threads=cores)
    # each step: one oracle transfer of the full workload
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.transfer(w, threads=cores)
    dt = time.perf_counter() - t0
    value = rows * args.steps / dt
    line = {"impl": "reference", "metric": "transfer rows/s", "value": value, "unit": "rows/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": workload_desc(w),
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full transfers of {w.name}, OpenMP build of the C oracle "
                                       f"on {cores} host threads"},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: resident star, Poisson arrivals, batched server vs one at a time
# ---------------------------------------------------------------------------
def serving_bench(args) -> dict:
    import threading

    import torch

    from paper_2307_15255_b300 import pt as P
    from paper_2307_15255_b300.session import TransferSession

    t0 = time.perf_counter()
    w = W.star(scale=args.serving_scale, bits_per_key=args.bpk)
    pool = W.selection_pool(w, size=32)
    n_q = args.serving_queries
    qs = W.serving_queries(w, n_q, rate_qps=0, pool=pool)
    gen_s = time.perf_counter() - t0
    cols_dev = [[torch.from_numpy(c).cuda() for c in t.cols] for t in w.tables]
    # the selection pool lives on the device; queries borrow its bitmaps
    pool_dev = {}
    for d in range(1, len(pool)):
        for b in pool[d]:
            pool_dev[id(b)] = torch.from_numpy(np.ascontiguousarray(b).view(np.int32)).cuda()
    sel_ptrs = [[None if x is None else pool_dev[id(x)].data_ptr() for x in q.sel] for q in qs]
    edges = [[(e.t0, e.c0, e.t1, e.c1) for e in q.edges] for q in qs]

    def make(max_batch, inflight):
        srv = P.pt_server_create(w.bits_per_key, w.k, w.block_bits, w.seed, args.serving_arena_gb << 30, max_batch,
                                 inflight)
        for t, cols in zip(w.tables, cols_dev):
            P.pt_server_register_table(srv, t.n_rows, [(c.data_ptr(), P.PT_I64, P.PT_MEM_DEVICE) for c in cols])
        P.pt_server_start(srv)
        return srv

    def submit(srv, i):
        return P.pt_server_submit(srv, qs[i].inst_table, sel_ptrs[i], edges[i], P.PT_MEM_DEVICE)

    def wait_release(srv, t, deadline):
        while not P.pt_server_poll(srv, t)[0]:
            if time.perf_counter() > deadline:
                raise RuntimeError("serving run did not finish in time")
            time.sleep(2e-5)
        P.pt_server_release(srv, t)

    def run_open(srv, idx, arrivals):
        """Submit queries idx at the given arrival offsets (s) from a client
        thread; release results as they complete (in submission order)."""
        P.pt_server_reset_stats(srv)
        tickets = [None] * len(idx)
        start = time.perf_counter()

        def submitter():
            for j, i in enumerate(idx):
                delay = arrivals[j] - (time.perf_counter() - start)
                if delay > 0:
                    time.sleep(delay)
                tickets[j] = submit(srv, i)
        th = threading.Thread(target=submitter)
        th.start()
        deadline = time.perf_counter() + args.serving_timeout
        for j in range(len(idx)):
            while tickets[j] is None:
                if time.perf_counter() > deadline:
                    raise RuntimeError("serving run did not finish in time")
                time.sleep(1e-4)
            wait_release(srv, tickets[j], deadline)
        th.join()
        wall = time.perf_counter() - start
        st = P.pt_server_stats(srv)
        return {"queries": len(idx), "achieved_qps": len(idx) / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"]}

    # one at a time through the server (batch of one, one in flight): each
    # query is submitted when the previous one is done
    srv1 = make(1, 1)
    deadline = time.perf_counter() + args.serving_timeout
    for i in range(min(20, n_q)):
        wait_release(srv1, submit(srv1, i), deadline)
    P.pt_server_reset_stats(srv1)
    n1 = min(args.serving_single, n_q)
    start = time.perf_counter()
    for i in range(n1):
        wait_release(srv1, submit(srv1, i), deadline)
    wall1 = time.perf_counter() - start
    st1 = P.pt_server_stats(srv1)
    P.pt_server_destroy(srv1)
    single = {"queries": n1, "achieved_qps": n1 / wall1, "p50_ms": st1["p50_ms"], "p99_ms": st1["p99_ms"]}
    cap1 = single["achieved_qps"]

    # the plain path, one query at a time: a context per query (plan, run,
    # read the survivors, free), keys hashed by the scan as in a single transfer
    n_plain = min(args.serving_plain, n_q)
    lat = []
    for i in range(n_plain + 3):
        q = qs[i]
        t1 = time.perf_counter()
        tabs = [(w.tables[t].n_rows, cols_dev[t], None if q.sel[j] is None else pool_dev[id(q.sel[j])])
                for j, t in enumerate(q.inst_table)]
        with TransferSession(tabs, edges[i], w.bits_per_key, w.k, w.block_bits, w.seed) as ts:
            ts.run()
            for j in range(len(tabs)):
                ts.survivors(j)
        if i >= 3:
            lat.append(time.perf_counter() - t1)
    lat.sort()
    plain = {"queries": n_plain, "achieved_qps": n_plain / sum(lat), "p50_ms": lat[len(lat) // 2] * 1e3,
             "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3}

    # batched server: the same queries at Poisson arrival rates relative to the
    # one-at-a-time capacity, then all at once
    rng = np.random.default_rng(20230728 + 44)
    srv = make(args.serving_batch, 2)
    run_open(srv, list(range(min(64, n_q))), [0.0] * min(64, n_q))  # warm-up: graphs captured
    sweep = []
    for mult in (0.5, 1.0, 2.0, 4.0, 8.0):
        rate = mult * cap1
        nq = min(n_q, max(200, int(rate * 1.0)))
        arr = np.cumsum(rng.exponential(1.0 / rate, nq))
        r = run_open(srv, list(range(nq)), list(arr))
        r.update({"offered_qps": rate, "offered_x_single": mult})
        sweep.append(r)
    sat = run_open(srv, list(range(n_q)), [0.0] * n_q)
    sat.update({"offered": "all at once"})
    P.pt_server_destroy(srv)
    del cols_dev, pool_dev
    torch.cuda.empty_cache()
    return {
        "workload": f"star: fact {w.tables[0].n_rows} rows x 4 int64 FKs, dims "
                    f"{[t.n_rows for t in w.tables[1:]]}; {n_q} queries of 3-6 instances, selectivity 0.1-50% "
                    f"(seeded pool of 32 selections per dimension, device-resident)",
        "one_at_a_time": single,
        "plain_context_one_at_a_time": plain,
        "batched_sweep": sweep,
        "batched_saturated": sat,
        "throughput_x_one_at_a_time": sat["achieved_qps"] / cap1,
        "throughput_x_plain_context": sat["achieved_qps"] / plain["achieved_qps"],
        "max_batch": args.serving_batch, "inflight": 2, "generation_s": gen_s,
    }


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pt_kernels.cu", "pt_internal.h"):
        with open(os.path.join(ROOT, "paper_2307_15255_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str, bpk: int):
    """Per-launch DRAM bytes of `kernel` from a committed ncu summary, or
    None when none exists for the current kernel source."""
    p = os.path.join(ROOT, "profiles", "probe_kernels_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    key = f"{workload}_b{bpk}"
    ent = d.get("kernels", {}).get(kernel, {}).get(key)
    return None if ent is None else ent.get("dram_bytes_per_launch")


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's step time (every rank runs its own replica)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rows_per_s(rows_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank's rows over the slowest rank's time."""
    return rows_per_rank * world / (ms * 1e-3)


def accounting(s, w):
    """Algorithmic bytes of the session's last run, from every visit's stats:
    (breakdown, bytes of the scan/list launches, bytes of the first-probe
    launches).  A first-probe pass reads its key sectors and writes the rows
    that pass as a bitmap, which the scan kernel reads back as its input."""
    acc = {"bitmap": 0, "probe_keys": 0, "build_keys": 0, "ids": 0, "filters": 0}
    scan_bytes = first_bytes = 0
    for p in range(2):
        for v, t in enumerate(w.tables):
            st = s.stats(p, v)
            nw = (t.n_rows + 31) // 32
            bm = 4 * nw * (2 if st["has_input_bitmap"] else 1)
            acc["bitmap"] += bm
            acc["probe_keys"] += 32 * st["probe_sectors"]
            acc["build_keys"] += 32 * st["build_sectors"]
            ids = 8 * st["survivors"] if st["n_out"] > 0 else 0
            acc["ids"] += ids
            acc["filters"] += st["filter_bytes"]
            if st["first_probe"]:
                first_bytes += 32 * st["first_probe_sectors"] + 4 * nw
                scan_bytes += bm + 4 * nw + 32 * (st["probe_sectors"] - st["first_probe_sectors"]) + ids // 2
            else:
                scan_bytes += bm + 32 * st["probe_sectors"] + ids // 2
    return acc, scan_bytes, first_bytes


def graph_ms(s, stream, steps: int, warmup: int) -> float:
    """Mean time of one transfer replayed from the session's CUDA graph."""
    import torch
    from paper_2307_15255_b300 import pt as P
    P.pt_set_graph_mode(s.ctx, True)
    for _ in range(max(warmup, 1)):
        s.run()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        s.run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def ours(args) -> None:
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("gloo")

    from paper_2307_15255_b300 import pt as P
    from paper_2307_15255_b300.session import TransferSession

    w = make_workload(args.workload, args.bpk, args.scale)
    rows = visit_rows(w)
    tables_dev = []
    for t in w.tables:
        cols = [torch.from_numpy(c).cuda() for c in t.cols]
        sel = None if t.sel is None else torch.from_numpy(t.sel.view(np.int32)).cuda()
        tables_dev.append((t.n_rows, cols, sel))
    edges = [(e.t0, e.c0, e.t1, e.c1) for e in w.edges]
    stream = torch.cuda.Stream()
    launch = tuple(args.launch) if args.launch else None
    first = False if args.no_first_probe else None
    s = TransferSession(tables_dev, edges, w.bits_per_key, w.k, w.block_bits, w.seed, stream=stream,
                        launch=launch, first_probe=first)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    if args.only_run:
        # profiling mode: warm-up and a few plain transfers (direct launches), nothing timed
        for _ in range(max(args.warmup, 0) + args.only_run):
            s.run()
        torch.cuda.synchronize()
        s.close()
        return

    # launch shape from the autotuner (outside the timed region)
    tuned = None
    if not args.no_autotune and launch is None:
        from paper_2307_15255_b300 import autotune
        tuned = autotune.tune(s, use_cache=False)
        tuned = {"launch": list(tuned["launch"]), "ms": tuned["ms"],
                 "trials": [[list(l), m] for l, m in tuned["trials"]]}

    # accounting of one run (identical every step: same inputs)
    s.run()
    torch.cuda.synchronize()
    acc, scan_bytes, first_bytes = accounting(s, w)
    alg_bytes = sum(acc.values())
    pt_survivors = [s.survivors(v)[1] for v in range(w.n_tables)]

    # direct launches (no graph), untimed by kernel events: reported beside the headline
    for _ in range(max(args.warmup, 0)):
        s.run()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(args.steps):
        s.run()
    d1.record(stream)
    torch.cuda.synchronize()
    direct_ms = d0.elapsed_time(d1) / args.steps

    # timed region: the transfer replayed from one CUDA graph
    P.pt_set_graph_mode(s.ctx, True)
    for _ in range(max(args.warmup, 0)):
        s.run()
    torch.cuda.synchronize()
    launches0 = P.pt_get_launch_count(s.ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            s.run()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    launches = P.pt_get_launch_count(s.ctx) - launches0

    # per-kernel times: the same graph recaptured with CUDA events around every
    # launch (event-record nodes on the launching stream) and every launch on one
    # stream, so that each kernel is timed alone; the events hold the last
    # replay's durations
    P.pt_set_streams(s.ctx, 1)
    P.pt_set_kernel_timing(s.ctx, True)
    for _ in range(max(args.warmup, 0) + args.steps):
        s.run()
    kt = P.pt_get_kernel_times(s.ctx)
    # the concurrent step's last replay, launch by launch: [pass, table, kind, start ms, ms]
    P.pt_set_streams(s.ctx, 3)
    for _ in range(max(args.warmup, 0) + 1):
        s.run()
    timeline = [[x["pass"], w.tables[x["table"]].name, x["kind"], round(x["start_ms"], 4), round(x["ms"], 4)]
                for x in P.pt_get_launch_times(s.ctx)]
    P.pt_set_kernel_timing(s.ctx, False)
    P.pt_set_graph_mode(s.ctx, False)

    # probe orders (Section 3.2: LIP-style ordering of the incoming filters is
    # optional): the same survivors; the key sectors read and the step differ.
    # The LIP order's bytes are the method's own count, the default order's are
    # what this schedule reads.
    orders = {}
    for name, order in (("level_then_lip", 0), ("lip", 1), ("edge_id", 2)):
        P.pt_set_probe_order(s.ctx, order)
        s.run()
        torch.cuda.synchronize()
        a_o, _, _ = accounting(s, w)
        ms_o = graph_ms(s, stream, max(5, args.steps // 2), args.warmup)
        P.pt_set_graph_mode(s.ctx, False)
        orders[name] = {"order": order, "alg_bytes_per_step": sum(a_o.values()), "ms_per_step": ms_o,
                        "rows_per_s": rows / (ms_o * 1e-3)}
    P.pt_set_probe_order(s.ctx, 0)

    # the Bloom join (Section 2.1; the BloomJoin baseline of Section 4) on the
    # same tables: every filter built from its table's selection, probed once.
    # What the join phase would get from each schedule, and each one's step.
    one_hop = None
    if not args.no_one_hop:
        so = TransferSession(tables_dev, edges, w.bits_per_key, w.k, w.block_bits, w.seed, stream=stream,
                             launch=tuple(tuned["launch"]) if tuned else launch, first_probe=first,
                             schedule=P.PT_SCHEDULE_ONE_HOP)
        so.run()
        torch.cuda.synchronize()
        oh_survivors = [so.survivors(v)[1] for v in range(w.n_tables)]
        ms_oh = graph_ms(so, stream, args.steps, args.warmup)
        so.close()
        one_hop = {
            "ms_per_step": ms_oh, "rows_per_s": rows / (ms_oh * 1e-3),
            "survivors": {t.name: c for t, c in zip(w.tables, oh_survivors)},
            "transfer_survivors": {t.name: c for t, c in zip(w.tables, pt_survivors)},
            "join_input_rows": sum(oh_survivors), "transfer_join_input_rows": sum(pt_survivors),
            "join_input_ratio": sum(oh_survivors) / max(1, sum(pt_survivors)),
        }

    # end to end through the C ABI from pinned host buffers: H2D of every
    # column and selection, both passes, D2H of every final survivor bitmap
    e2e = None
    if not args.no_e2e:
        host = []
        h2d = 0
        for t in w.tables:
            cols = [torch.from_numpy(c).pin_memory() for c in t.cols]
            sel = None if t.sel is None else torch.from_numpy(t.sel.view(np.int32)).pin_memory()
            h2d += sum(c.numel() * c.element_size() for c in cols) + (0 if sel is None else sel.numel() * 4)
            host.append((cols, sel))
        outs = [torch.empty(max((t.n_rows + 31) // 32, 1), dtype=torch.int32).pin_memory() for t in w.tables]
        d2h = sum(((t.n_rows + 31) // 32) * 4 + 8 for t in w.tables)
        se = TransferSession([(t.n_rows, c, sl) for t, (c, sl) in zip(w.tables, host)], edges, w.bits_per_key,
                             w.k, w.block_bits, w.seed, stream=stream, launch=launch, first_probe=first)
        n_e2e = max(1, min(args.steps, 5))
        se.run()
        for v in range(w.n_tables):
            P.pt_get_survivors(se.ctx, v, outs[v].data_ptr())
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            for v, (cols, sel) in enumerate(host):
                se.update(v, cols, sel)
            se.run()
            for v in range(w.n_tables):
                P.pt_get_survivors(se.ctx, v, outs[v].data_ptr())
        dt = (time.perf_counter() - t0) / n_e2e
        barrier()
        se.close()
        e2e = {"value": rows * world / dt, "unit": "rows/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "steps": n_e2e}

    s.close()
    # the same snowflake at 8 bits per key (the configuration's other swept size)
    bpk_sweep = {}
    if not args.no_bpk_sweep:
        for bpk in (8, 16):
            if bpk == w.bits_per_key:
                continue
            sb = TransferSession(tables_dev, edges, bpk, w.k, w.block_bits, w.seed, stream=stream,
                                 launch=tuple(tuned["launch"]) if tuned else launch, first_probe=first)
            sb.run()
            torch.cuda.synchronize()
            a_b, _, _ = accounting(sb, w)
            ms_b = graph_ms(sb, stream, args.steps, args.warmup)
            sb.close()
            bpk_sweep[f"bits_per_key_{bpk}"] = {
                "ms_per_step": ms_b, "value": rows / (ms_b * 1e-3), "unit": "rows/s",
                "alg_bytes_per_step": sum(a_b.values()),
                "alg_gbs": sum(a_b.values()) / (ms_b * 1e-3) / 1e9}
    del tables_dev
    torch.cuda.empty_cache()
    serving = None
    if not args.no_serving and rank == 0:
        serving = serving_bench(args)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = hbm_peak()
    for v in bpk_sweep.values():
        v["frac_of_peak"] = v["alg_gbs"] / peak
    # one replay: one scan per visit, one first-probe pass per visit that has one
    kernels = []
    for name, nbytes, kms, nl in (("pt_probe_first_kernel", first_bytes, kt["first_ms"], kt["first_launches"]),
                                  ("pt_scan_kernel", scan_bytes, kt["scan_ms"], kt["scan_launches"])):
        if nl <= 0:
            continue
        per_ms = kms / nl
        ach = (nbytes / nl) / (per_ms * 1e-3) / 1e9
        kernels.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                        "launches_of": ("pt_scan_kernel, pt_scan_sparse_kernel (forward visits with an input bitmap) "
                                        "and pt_probe_list_kernel (backward visits)"
                                        if name == "pt_scan_kernel" else name),
                        "frac": ach / peak, "peak_kind": peak_kind,
                        "traffic": committed_traffic(name, args.workload, args.bpk),
                        "alg_bytes_per_launch": nbytes / nl, "ms_per_launch": per_ms, "launches_timed": nl,
                        "ms_per_step": kms})
    roof = max(kernels, key=lambda r: r["ms_per_step"])  # the kernel with the most time per step
    cpu = None
    if not args.no_cpu:
        # every host core (the headline baseline), and one core as in the paper's setup
        cpu = oracle_timing(w, args.cpu_seconds, host_cores())
        cpu["one_core"] = oracle_timing(w, args.cpu_seconds, 1)
    line = {
        "metric": "transfer rows/s",
        "value": job_rows_per_s(rows, world, ms),
        "unit": "rows/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic (seeded star/snowflake generator; stands in for TPC-H SF10)",
        "config": workload_desc(w),
        "hbm": {"alg_bytes_per_step": alg_bytes, "alg_breakdown": acc,
                "alg_gbs": alg_bytes / (ms * 1e-3) / 1e9,
                "frac_of_peak": alg_bytes / (ms * 1e-3) / 1e9 / peak, "peak_gbs": peak, "peak_kind": peak_kind,
                "frac_of_nominal_8tbs": alg_bytes / (ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                # the method's own byte count (LIP probe order) over the same step
                "alg_bytes_lip_order": orders["lip"]["alg_bytes_per_step"],
                "frac_of_peak_lip_order_bytes": orders["lip"]["alg_bytes_per_step"] / (ms * 1e-3) / 1e9 / peak},
        "roofline": roof,
        "roofline_kernels": kernels,
        "probe_orders": orders,
        "one_hop": one_hop,
        "bpk_sweep": bpk_sweep,
        "build_ms_per_step": kt["build_ms"],
        "launch_timeline": timeline,
        "mode": "CUDA graph replay (direct launches: see direct_ms_per_step)",
        "direct_ms_per_step": direct_ms,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "autotune": tuned,
        "scale_mode": "replicas" if world > 1 else "single",
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="snowflake_x10")
    ap.add_argument("--bpk", type=int, default=16)
    ap.add_argument("--scale", type=float, default=10.0, help="size of the snowflake (10 = fact 60M rows)")
    ap.add_argument("--only-run", type=int, default=0, help="profiling: run this many transfers and exit")
    ap.add_argument("--launch", type=int, nargs=3, metavar=("THREADS", "SMEM", "CTAS_PER_SM"))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-one-hop", action="store_true", help="skip the one-hop (Bloom join) comparison")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-first-probe", action="store_true", help="keep every probe in the scan kernel")
    ap.add_argument("--no-bpk-sweep", action="store_true", help="skip the other bits-per-key size")
    ap.add_argument("--serving-scale", type=float, default=1.0, help="star size (1 = fact 100M rows)")
    ap.add_argument("--serving-queries", type=int, default=2000)
    ap.add_argument("--serving-single", type=int, default=200, help="queries timed one at a time")
    ap.add_argument("--serving-plain", type=int, default=30, help="queries timed through plain contexts")
    ap.add_argument("--serving-batch", type=int, default=32)
    ap.add_argument("--serving-arena-gb", type=int, default=96)
    ap.add_argument("--serving-timeout", type=float, default=120.0, help="seconds per serving run")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
