#!/usr/bin/env python3
"""Benchmark: protein database search GCUPS on GB300 (Eq. 5: GCUPS = |Q| x |D| / (t x 1e9)).

Workload (default): 20 synthetic queries of 144..5478 residues (log-uniform)
against a 200,000-sequence synthetic database (~67.5M residues; log-normal
lengths, median 300, clamped 20..1000; Robinson background residues),
BLOSUM62, gaps 10 + 2k.  The synthetic inputs stand in for the paper's
Swiss-Prot queries and Env. NR database (Sec. 4.1).

One step = one full search of all queries against the resident database:
profile build, packed s16x2 DP kernel, overflow rescue, scatter.  `value` is
kernel-side GCUPS with inputs resident in HBM (device-side CUDA events,
L2 flushed between steps); `e2e` is the same search through the one-call
C-ABI entry point sw_search with host query and score buffers (copies
inside the timed region).  The plain int32 kernel is timed on the same
workload and reported beside it.

--impl reference times the CPU oracle (scalar int32 Gotoh, threaded across
pairs) on a bounded sample of the same workload on the host cores.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS per GB300, packed-int16/8 batched vs plain int32; p50/p99 query latency"
WORKLOAD = "protein DB search: 20 queries (144-5478 aa) x 200,000 synthetic proteins (~67.5M aa), BLOSUM62, gaps 10+2k"
SM_COUNT_FALLBACK = 152
# The integer ALU pipe of an sm_103 SMSP accepts one warp instruction every
# second cycle (ncu: a stream of IMNMX / VIMNMX / IADD / PRMT runs the ALU pipe
# at ~99% with issue at ~51%), i.e. 64 lanes per clock per SM.  Every max of
# the recurrences runs there; the DP kernels are bound by it.  The FMA pipe is
# a second integer pipe of the same width (it takes the per-half 16x2 adds).
ALU_LANES_PER_SM_CLK = 64
INT_PIPES = 2  # ALU + FMA: the lanes the paper's instruction model (Eqs. 4-6) can use for adds and maxima
# Algorithmic integer operations per cell, the roofline's count:
#  - packed s16x2: about 6 operations per 32-bit word of two cells (H - Go
#    shared by E and F, the E and F max-adds, H_diag + SM, the three-way max
#    with the zero floor, the running best), i.e. 3 per cell -- every one of
#    them issues on the ALU pipe (adds fuse into the maxima that consume them);
#  - int32: the 12 statements of Algorithm 1 (the paper's model, Eq. 6),
#    against both integer pipes.
# The maxima alone (the ALU pipe's irreducible work): 5 per word (2.5 per
# cell) packed, 6 per cell int32.
ALG_OPS_PER_CELL = {"packed": 3.0, "int32": 12.0}
ALG_PIPES = {"packed": 1, "int32": INT_PIPES}
ALU_MAX_OPS_PER_CELL = {"packed": 2.5, "int32": 6.0}


def roofline_of(gcups, mode, n_sm, sm_mhz):
    """ALU-pipe roofline fields of a DP kernel that ran at `gcups` (kernel time)."""
    lanes = n_sm * ALU_LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e9  # Gop/s of one integer pipe
    peak = lanes * ALG_PIPES[mode]
    achieved = gcups * ALG_OPS_PER_CELL[mode]
    maxima = gcups * ALU_MAX_OPS_PER_CELL[mode]
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Gop/s",
            "frac": round(achieved / peak, 4), "ops_per_cell": ALG_OPS_PER_CELL[mode],
            "pipes": ALG_PIPES[mode],
            "frac_maxima_only": round(maxima / lanes, 4), "maxima_per_cell": ALU_MAX_OPS_PER_CELL[mode],
            "peak_basis": f"{n_sm} SMs x {ALU_LANES_PER_SM_CLK} lanes/clk per integer pipe x "
                          f"{ALG_PIPES[mode]} pipe(s) x {sm_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
            "kernel_gcups": round(gcups, 1)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed steps (the paper reports 20 runs per point)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="twenty_queries_vs_200k",
                    help="named synthetic workload (workload.gen.WORKLOADS, or a DNA pair of workload.gen.DNA_PAIRS)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the int32 and small-workload side measurements")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving run (Poisson 50/s, 500,000-protein database); 0 skips it")
    ap.add_argument("--serve-half-requests", type=int, default=2500,
                    help="requests of the second serving run at half the rate (25/s); 0 skips it")
    ap.add_argument("--mode", default="packed", choices=["packed", "int32"], help="form of the timed search")
    ap.add_argument("--no-query-pairs", action="store_true",
                    help="packed mode: keep every query in the two-sequences-per-chain form")
    ap.add_argument("--shard", action="store_true",
                    help="with N ranks: each GPU holds 1/N of the database (residue-balanced, length-stratified "
                         "shards) and searches every query against it (strong scaling); default: every GPU "
                         "searches its own full copy (weak scaling)")
    ap.add_argument("--band-stream", default="auto", choices=["auto", "never", "always"],
                    help="small-batch plan of the timed search (sw_options.band_stream)")
    ap.add_argument("--queries", type=int, default=0, help="use only the first K queries (profiling runs)")
    ap.add_argument("--db-limit", type=int, default=0, help="use only the first N database sequences (profiling runs)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed helpers (one process per GPU; weak scaling, no data-path collective)
# ----------------------------------------------------------------------------

def workload_label(name):
    """The config label of a workload: the benchmark's own description, or
    the workload's name and shape for the side workloads."""
    if name == "twenty_queries_vs_200k":
        return WORKLOAD
    from workload import WORKLOADS

    return f"{name}: {WORKLOADS[name]}, BLOSUM62, gaps 10+2k"


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device])
        else:
            pg.barrier()


def sharded_e2e_step(search_local, parts, pg, device="cpu"):
    """One end-to-end step of the sharded search (--shard): this rank's scores
    against its shard (search_local() returns int32 [n_queries,
    len(parts[rank])] on the host), then the all-gather of every rank's slice
    into the caller's order (the design's one exchange).  Returns the full
    [n_queries, n_db] matrix, on every rank."""
    from paper_2412_08308_gb300.shard import gather_scores

    return gather_scores(search_local(), parts, pg, device)


def max_over_ranks(pg, x, device=None):
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=f"cuda:{device}" if device is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        under = [x for x in sm if smax and x > 0.5 * max(smax)] or sm
        return {"sm_mhz": float(np.median(under)) if under else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dp_kernel_traffic(workload, mode="packed"):
    """DRAM bytes per launch of the DP kernel on `workload` from the committed
    ncu summary, or None if none was captured for that workload and form or
    the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "dp_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("workload_name") != workload or rec.get("mode", "packed") != mode:
        return None
    if rec.get("source_sha1") != dp_kernel_source_sha1():
        return None
    return rec.get("dram_bytes_per_launch")


def strip_c_comments(text):
    """C/C++ source without comments and blank lines (string and character
    literals kept), so that documentation edits leave the hash unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = ("".join(out)).splitlines()
    return "\n".join(line.rstrip() for line in lines if line.strip())


def dp_kernel_source_sha1():
    """SHA-1 over the code (comments removed) of the sources that define the
    inter-task DP kernel."""
    h = hashlib.sha1()
    for f in ("k_inter.cu", "dp_common.cuh", "internal.h", "devutil.cuh"):
        text = open(os.path.join(ROOT, "paper_2412_08308_gb300", "csrc", f), encoding="utf-8").read()
        h.update(strip_c_comments(text).encode())
    return h.hexdigest()


# ----------------------------------------------------------------------------
# the CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------

def oracle_sample_gcups(w, n_subjects, seed=4000, threads=None):
    import oracle
    from workload import sample_indices
    from workload.matrices import BLOSUM62

    oracle.build()
    idx = sample_indices(len(w["db"]), n_subjects, seed=seed)
    cells = float(w["queries"].total) * float(w["db"].lengths[idx].sum())
    threads = threads or oracle.default_threads()
    t0 = time.perf_counter()
    oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2, subset=idx, threads=threads)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, threads, cells, dt


def run_reference(args, w):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    n_sub = 400
    for _ in range(args.warmup):
        oracle_sample_gcups(w, 50, seed=4100)
    times, cells_total = [], 0.0
    threads = 1
    for s in range(args.steps):
        g, threads, cells, dt = oracle_sample_gcups(w, n_sub, seed=4200 + s)
        times.append(dt)
        cells_total += cells
    T = sum(times)
    value = cells_total / T / 1e9
    sample = f"all {len(w['queries'])} queries x {n_sub} seeded database sequences per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * T / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": workload_label(getattr(args, "workload", "twenty_queries_vs_200k")), "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": "GCUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def time_prepared(pq, out, steps, flush, timing=False):
    import torch

    t_steps, k_steps = [], []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        pq.search(out)
        e.record()
        torch.cuda.synchronize()
        t_steps.append(s.elapsed_time(e) / 1e3)
        if timing:
            k_steps.append(pq.kernel_ms() / 1e3)
    return t_steps, k_steps


def run_serving(n_requests, n_half, mode, gpu=0):
    """Continuous-batching serving runs on the serving_500k workload: 500,000 synthetic
    proteins (~180M residues) resident in HBM, queries (median 400, 30-3000)
    arriving as a Poisson process at 50/s (the first n_requests arrivals), and
    the same arrival sequence at half the rate (25/s, the first n_half
    arrivals: about half the sustained capacity).  Reports latency
    percentiles, offered vs sustained GCUPS and the clocks of each run."""
    from paper_2412_08308_gb300 import api
    from workload import make_workload

    w = make_workload("serving_500k", n_queries=max(n_requests, n_half))
    db = api.Database.from_sequences(w["db"])
    clk = Clocks(gpu)
    clk.start()
    st = serve_once(db, w, n_requests, 1.0, mode)
    st["clocks"] = clk.stop()
    if n_half > 0:
        clk = Clocks(gpu)
        clk.start()
        st["half_rate"] = serve_once(db, w, n_half, 2.0, mode)
        st["half_rate"]["clocks"] = clk.stop()
    db.close()
    return st


def graph_search_ms(pq, out, stream, flush, reps):
    """Per-search times (ms) of sw_search_graph launches on `stream`, CUDA
    events on that stream around each launch, L2 flushed before each."""
    import torch

    ts = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pq.search_graph(out, stream=stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def small_config_block(api, name, flush, gpu, n_sm, sm_mhz, reps=50, batch=0, rescue_path=False):
    """One of the small configurations (the 144-residue query against 2,000
    proteins; the homolog workload) in both forms: whole searches replayed
    through sw_search_graph (median of `reps`), the DP kernel's own time
    (events around it in a plain enqueue), its ALU roofline, the pairs rescued
    and the clocks sampled during the block.  batch > 0: also `batch` seeded
    requests of the same shape searched together, in both forms.
    rescue_path: also the packed search through the flag-and-rescue path."""
    import torch

    from workload import WORKLOADS, make_workload
    from workload.matrices import BLOSUM62

    w = make_workload(name)
    q, dbs = w["queries"], w["db"]
    cells = float(q.total) * float(dbs.total)
    db = api.Database.from_sequences(dbs)
    stream = torch.cuda.Stream()
    out = torch.empty((len(q), len(dbs)), dtype=torch.int32, device="cuda")
    clk = Clocks(gpu)
    clk.start()
    res = {"workload": f"{name}: {WORKLOADS[name]}", "cells": cells, "timed": "sw_search_graph, median of "
           f"{reps} searches, L2 flushed before each"}
    for mode in ("packed", "int32"):
        pq = api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, mode, stream=stream)
        for _ in range(3):
            pq.search_graph(out, stream=stream)
        rescued = pq.status(stream=stream)
        ts = graph_search_ms(pq, out, stream, flush, reps)
        pq.set_timing(True)
        ks = []
        for _ in range(min(reps, 20)):
            with torch.cuda.stream(stream):
                flush.zero_()
            pq.search(out, stream=stream)
            ks.append(pq.kernel_ms(stream=stream))
        ms, kms = float(np.median(ts)), float(np.median(ks))
        info = pq.info()
        pq.close()
        # the one-call API (sw_search: plan, uploads, search, scores to host
        # memory, free), as a caller without a prepared batch sees it
        host = np.empty((len(q), len(dbs)), dtype=np.int32)
        te = []
        for _ in range(min(reps, 20)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.search(db, q.residues, q.offsets, BLOSUM62, 10, 2, mode, out=host)
            te.append(1e3 * (time.perf_counter() - t0))
        res[mode] = {"ms": round(ms, 4), "gcups": round(cells / ms / 1e6, 1), "dp_kernel_ms": round(kms, 4),
                     "e2e_ms": round(float(np.median(te)), 4), "rescued_pairs": int(rescued),
                     "launches_per_search": int(info[3]), "roofline": roofline_of(cells / kms / 1e6, mode, n_sm, sm_mhz)}
    res["packed_over_int32"] = round(res["packed"]["gcups"] / res["int32"]["gcups"], 3)
    if rescue_path:
        # the flag-and-rescue path on the same batch: every unit on the
        # inter-task kernel (no band-stream jobs, no intra-task cutover), so
        # the pairs that pass the 16-bit range saturate, are flagged and
        # recomputed exactly in int32
        pq = api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, "packed", stream=stream,
                                 opts=api.options(cutover=1 << 20, band_stream="never"))
        pq.search_graph(out, stream=stream)
        rescued = pq.status(stream=stream)
        ts = graph_search_ms(pq, out, stream, flush, 5)
        ms = float(np.median(ts))
        res["rescue_path"] = {"plan": "inter-task kernel for every unit, 16-bit with flags and int32 rescue",
                              "ms": round(ms, 3), "gcups": round(cells / ms / 1e6, 1), "rescued_pairs": int(rescued)}
        pq.close()
    if batch:
        # the same shape of request, `batch` of them in one search (the
        # batched form): both forms, and the packed batch against the single
        # int32 search above
        from workload import query_batch_144

        qb = query_batch_144(batch)
        bcells = float(qb.total) * float(dbs.total)
        outb = torch.empty((len(qb), len(dbs)), dtype=torch.int32, device="cuda")
        bres = {"requests": batch, "queries": f"{batch} seeded queries of 144 residues", "cells": bcells}
        for mode in ("packed", "int32"):
            pq = api.PreparedQueries(db, qb.residues, qb.offsets, BLOSUM62, 10, 2, mode, stream=stream)
            for _ in range(3):
                pq.search_graph(outb, stream=stream)
            ts = graph_search_ms(pq, outb, stream, flush, 10)
            ms = float(np.median(ts))
            bres[mode] = {"ms": round(ms, 4), "gcups": round(bcells / ms / 1e6, 1),
                          "roofline": roofline_of(bcells / ms / 1e6, mode, n_sm, sm_mhz)}
            pq.close()
        bres["packed_over_int32"] = round(bres["packed"]["gcups"] / bres["int32"]["gcups"], 3)
        bres["packed_batched_over_int32_single"] = round(bres["packed"]["gcups"] / res["int32"]["gcups"], 3)
        res["batched"] = bres
    res["clocks"] = clk.stop()
    db.close()
    return res


def batch_config_block(api, flush, n_sm, sm_mhz):
    """The 1,000-query batch against 50,000 proteins: the autotuner's sweep
    (residues per thread x cutover) on the real batch, then both forms with
    the tuned options, one graph-captured search each (median of 3)."""
    import torch

    from paper_2412_08308_gb300 import tune
    from workload import WORKLOADS, make_workload
    from workload.matrices import BLOSUM62

    w = make_workload("thousand_queries_vs_50k")
    q, dbs = w["queries"], w["db"]
    cells = float(q.total) * float(dbs.total)
    db = api.Database.from_sequences(dbs)
    t0 = time.perf_counter()
    opts, table = tune.tune(db, dbs.lengths, q.residues, q.offsets, BLOSUM62, rows=(8, 16, 24),
                            cutovers=(512, 2048), reps=1)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    out = torch.empty((len(q), len(dbs)), dtype=torch.int32, device="cuda")
    res = {"workload": f"thousand_queries_vs_50k: {WORKLOADS['thousand_queries_vs_50k']}", "cells": cells,
           "tuner": {"rows_per_lane": opts.rows_per_lane, "cutover": opts.cutover, "seconds": round(tune_s, 1),
                     "table": [{"rows_per_lane": r, "cutover": c, "gcups": g} for r, c, g in table],
                     "note": "database sequences are at most 1,000 residues, so every cutover above 1,000 gives "
                             "the plan of 2,048; 4 rows per lane is left out (3,555 GCUPS at best when swept)"}}
    for mode in ("packed", "int32"):
        pq = api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, mode,
                                 opts=opts if mode == "packed" else None, stream=stream)
        pq.search_graph(out, stream=stream)
        rescued = pq.status(stream=stream)
        ts = graph_search_ms(pq, out, stream, flush, 3)
        ms = float(np.median(ts))
        res[mode] = {"ms": round(ms, 2), "gcups": round(cells / ms / 1e6, 1), "rescued_pairs": int(rescued),
                     "roofline": roofline_of(cells / ms / 1e6, mode, n_sm, sm_mhz)}
        pq.close()
    res["packed_over_int32"] = round(res["packed"]["gcups"] / res["int32"]["gcups"], 3)
    db.close()
    return res


def serve_once(db, w, n_requests, stretch, mode, prestage=True):
    import threading

    from paper_2412_08308_gb300.serve import Server
    from workload.matrices import BLOSUM62

    q = w["queries"].subset(range(n_requests))
    arrivals = w["arrivals"][:n_requests] * stretch
    # two queries per batch (a query pair) and two batches in flight gave the
    # lowest mean and p99 latency of the (batch, streams) settings measured;
    # shortest queries first (requests older than 1 s first of all)
    srv = Server(db, BLOSUM62, 10, 2, mode, max_batch=2, n_streams=2, policy="sjf", age_s=1.0, prestage=prestage)
    t0 = time.perf_counter()
    futs = []

    def client():
        for i in range(len(q)):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(q[i], arrival=t0 + arrivals[i]))

    th = threading.Thread(target=client)
    th.start()
    th.join()
    for f in futs:
        f.result()
    t_end = time.perf_counter()
    srv.close()
    st = srv.latency_stats()
    cells = float(q.total) * float(w["db"].total)
    span = t_end - t0
    st.update({"workload": f"{len(q)} Poisson({50 / stretch:g}/s) queries (median 400 aa) x {len(w['db'])} "
                           f"proteins ({w['db'].total} aa)",
               "offered_gcups": round(cells / float(arrivals[-1]) / 1e9, 1),
               "sustained_gcups": round(cells / span / 1e9, 1), "wall_s": round(span, 2),
               "batching": "continuous: up to 2 queries per batch, 2 batches in flight on separate streams, "
                           "shortest queries first (any request older than 1 s ahead), "
                           + ("the next batch planned while both slots are busy" if prestage else
                              "each batch planned when a slot frees up")})
    return st


def run_ours(args, w):
    import torch

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2412_08308_gb300 import api, build
    from workload.matrices import BLOSUM62

    build()
    q = w["queries"]
    db_s = w["db"]
    # whole-job cells per step: every rank's full copy (weak scaling), or the
    # one database split over the ranks (--shard, strong scaling)
    job_cells = float(q.total) * float(db_s.total) * (1 if args.shard else world)
    shard_note = None
    parts = None
    if args.shard and world > 1:
        from paper_2412_08308_gb300.shard import partition

        parts = partition(db_s.lengths, world)
        mine = parts[rank]
        shard_note = f"database sharded over {world} GPUs: this rank {len(mine)} of {len(db_s)} sequences"
        db_s = db_s.subset(mine)
    cells = float(q.total) * float(db_s.total)
    # one-time setup, outside the timed steps: database packing and upload
    # (sw_db_prepare), query planning, profiles' layout and upload
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    db = api.Database.from_sequences(db_s)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    opts = api.options(query_pairs=not args.no_query_pairs, band_stream=args.band_stream)
    pq = api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, args.mode, opts=opts)
    torch.cuda.synchronize()
    setup_ms = {"db_prepare": round(1e3 * (t1 - t0), 2), "queries_prepare": round(1e3 * (time.perf_counter() - t1), 2)}
    pq.set_timing(True)
    out = torch.empty((len(q), len(db_s)), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > 129 MB L2

    for _ in range(max(3, args.warmup)):
        pq.search(out)
    torch.cuda.synchronize()
    rescued = pq.status()

    clocks = Clocks(local)
    barrier(pg, local)
    torch.cuda.synchronize()
    clocks.start()
    t_steps, k_steps = time_prepared(pq, out, args.steps, flush, timing=True)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(pg, local)
    T = max_over_ranks(pg, sum(t_steps), local)
    value = job_cells * args.steps / T / 1e9
    k_mean = float(np.mean(k_steps))
    launches_per_step = pq.info()[3]

    # roofline of the DP kernel: the integer ALU pipe (alu)
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count or SM_COUNT_FALLBACK
    roofline = roofline_of(cells / k_mean / 1e9, args.mode, n_sm, sm_mhz)
    roofline["traffic"] = dp_kernel_traffic(args.workload, args.mode) if not (args.queries or args.db_limit) else None
    if pq.info()[2] == 0:  # a small batch: band-stream and transposed jobs only
        roofline["kernel"] = "band_stream_kernel / band_track_kernel (small-batch plan), " + (
            "16-bit forms where no pair can pass the 16-bit range, int32 elsewhere" if args.mode == "packed"
            else "int32 form")
    else:
        roofline["kernel"] = ("inter_kernel, 16-bit forms (query pairs; two sequences per chain for unpaired "
                              "queries)" if args.mode == "packed" else "inter_kernel, int32 form")

    extras = {}
    # the side measurements (other configurations, serving, the CPU oracle)
    # are single-GPU figures: taken at N = 1 only, so that a multi-GPU run
    # holds its GPUs for the timed steps alone
    if not args.no_extras and world == 1:
        xclk = Clocks(local)
        xclk.start()
        # alignments of each query's best hits (sw_traceback)
        extras["traceback_top10"] = traceback_rate(api, db, q, out)
        # the plain int32 kernel (Algorithm 1 body) on the same workload
        pq32 = api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, "int32")
        pq32.set_timing(True)
        pq32.search(out)
        torch.cuda.synchronize()
        t32, k32 = time_prepared(pq32, out, max(1, min(3, args.steps)), flush, timing=True)
        extras["int32_gcups"] = round(cells * len(t32) / sum(t32) / 1e9, 1)
        extras["packed_over_int32"] = round(cells * args.steps / T / 1e9 / extras["int32_gcups"], 3)
        extras["int32_roofline"] = roofline_of(cells / float(np.mean(k32)) / 1e9, "int32", n_sm, sm_mhz)
        pq32.close()
        # the other configurations of the method, each in both forms
        extras["one_query_vs_2k"] = small_config_block(api, "one_query_vs_2k", flush, local, n_sm, sm_mhz,
                                                       batch=256)
        extras["homologs_8k"] = small_config_block(api, "homologs_8k", flush, local, n_sm, sm_mhz, reps=10,
                                                   rescue_path=True)
        extras["thousand_queries_vs_50k"] = batch_config_block(api, flush, n_sm, sm_mhz)
        # the paper's DNA pairwise workload at its 1M x 1M size (sw_align_pair, int32)
        extras["dna_pair_1m_x_1m"] = dna_pair_gcups("dna_1m_x_1m")
        extras["extras_clocks"] = xclk.stop()

    # end to end through sw_search with host buffers; sharded: each rank's
    # slice, then the all-gather into the caller's order, inside the timed region
    e2e = None
    if not args.no_e2e:
        h2d = pq.info()[0]
        host_out = np.empty((len(q), len(db_s)), dtype=np.int32)

        def one():
            return api.search(db, q.residues, q.offsets, BLOSUM62, 10, 2, args.mode, out=host_out)

        dev = f"cuda:{local}"
        step = (lambda: sharded_e2e_step(one, parts, pg, dev)) if parts is not None else one
        full = step()
        barrier(pg, local)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            full = step()
        torch.cuda.synchronize()
        te = max_over_ranks(pg, time.perf_counter() - t0, local)
        e2e = {"value": round(job_cells * args.steps / te / 1e9, 1), "unit": "GCUPS",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(full.nbytes)}
        if parts is not None:
            e2e["gather"] = "all-gather of the score slices (NCCL) inside the timed region"

    serving = None
    if world == 1 and args.serve_requests > 0 and not (args.queries or args.db_limit):
        serving = run_serving(args.serve_requests, args.serve_half_requests, args.mode, local)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        g, threads, c, dt = oracle_sample_gcups(w, 8000)
        g1, _, c1, dt1 = oracle_sample_gcups(w, 200, seed=4300, threads=1)
        cpu = {"value": round(g, 3), "unit": "GCUPS", "cores": threads, "kind": "oracle",
               "sample": f"all {len(q)} queries x 8,000 seeded database sequences ({c:.3g} cells, {dt:.1f} s)",
               "one_core": {"value": round(g1, 3), "unit": "GCUPS",
                            "sample": f"all {len(q)} queries x 200 seeded sequences ({c1:.3g} cells, {dt1:.1f} s)"}}

    if rank == 0:
        wl = workload_label(args.workload)
        if args.queries or args.db_limit:
            wl = f"reduced profiling case: {len(q)} queries x {len(db_s)} synthetic proteins"
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(1e3 * T / args.steps, 3), "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": "s16x2+int32" if args.mode == "packed" else "int32", "data": "synthetic",
            "config": {"workload": wl, "queries": len(q), "db_sequences": len(db_s), "db_residues": db_s.total,
                       "cells_per_step": cells, "l2": "flushed between steps (256 MB write)",
                       "parallelism": shard_note or (f"{world} GPU(s), one database sharded" if args.shard else
                                                     f"{world} GPU(s), independent full workload per GPU"),
                       "form": "packed s16x2 + exact int32 rescue" if args.mode == "packed" else "plain int32 (Algorithm 1)",
                       "rescued_pairs": rescued},
            "step_ms": {"median": round(1e3 * float(np.median(t_steps)), 3),
                        "mean": round(1e3 * float(np.mean(t_steps)), 3),
                        "min": round(1e3 * min(t_steps), 3), "max": round(1e3 * max(t_steps), 3)},
            "setup_ms": setup_ms,
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk, "roofline": roofline,
            "cpu_baseline": cpu, "serving": serving,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    pq.close()
    db.close()
    if pg is not None:
        pg.destroy_process_group()


def traceback_rate(api, db, q, out, k=10):
    """sw_traceback on each query's k best-scoring database sequences (the hits
    a caller keeps), timed on the host around the call (uploads, kernels,
    downloads); its rate counts the cells of the recomputed matrices.  Each
    alignment's score must equal the search score of its pair."""
    from workload.matrices import BLOSUM62

    scores = out.cpu().numpy()
    hits = []
    for i in range(scores.shape[0]):
        hits += [(i, int(t)) for t in np.argsort(-scores[i], kind="stable")[:k]]
    qlen = np.diff(q.offsets)
    cells = float(sum(int(qlen[a]) * int(db.lengths[b]) for a, b in hits))
    api.traceback(db, q.residues, q.offsets, hits, BLOSUM62, 10, 2)  # warm-up
    t0 = time.perf_counter()
    res = api.traceback(db, q.residues, q.offsets, hits, BLOSUM62, 10, 2)
    dt = time.perf_counter() - t0
    same = all(int(r[0]) == int(scores[a, b]) for r, (a, b) in zip(res, hits))
    return {"hits": len(hits), "cells": cells, "ms": round(1e3 * dt, 2), "gcups": round(cells / dt / 1e9, 1),
            "scores_match_search": same}


def dna_pair_gcups(name, reps=2):
    """GCUPS of sw_align_pair on a seeded DNA pair (+1/-3, gaps 5 + 2k),
    timed by CUDA events around the pair kernel; the best of `reps` calls."""
    from paper_2412_08308_gb300 import api
    from workload import make_dna_pair
    from workload.matrices import DNA_GAP_EXTEND, DNA_GAP_OPEN, DNA_SUBMAT

    q, t = make_dna_pair(name)
    cells = float(q.size) * float(t.size)
    best, score = None, None
    for _ in range(reps):
        score, ms = api.align_pair(q, t, DNA_SUBMAT, DNA_GAP_OPEN, DNA_GAP_EXTEND, timed=True)
        best = ms if best is None else min(best, ms)
    return {"gcups": round(cells / (best * 1e-3) / 1e9, 1), "kernel_ms": round(best, 2), "cells": cells,
            "score": int(score), "workload": f"{name}: {q.size} x {t.size} bases, +1/-3, gaps 5+2k"}


def run_dna(args):
    """--workload dna_*: one long pair per step on the pair-band kernel."""
    import torch

    from paper_2412_08308_gb300 import build

    build()
    torch.cuda.set_device(0)
    res = dna_pair_gcups(args.workload, reps=max(1, args.steps))
    print(json.dumps({"metric": "GCUPS per GB300, DNA pairwise alignment (score only)", "value": res["gcups"],
                      "unit": "GCUPS", "n_gpus": 1, "steps": max(1, args.steps), "higher_is_better": True,
                      "dtype": "int32", "data": "synthetic", "config": {"workload": res["workload"]},
                      "kernel_ms": res["kernel_ms"], "score": res["score"]}), flush=True)


def main():
    args = parse()
    from workload import DNA_PAIRS, make_workload

    if args.workload in DNA_PAIRS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle would take hours on one long DNA "
                                                                   "pair (it threads across pairs only)"}))
            return
        run_dna(args)
        return
    w = make_workload(args.workload)
    if args.queries:
        w["queries"] = w["queries"].subset(range(min(args.queries, len(w["queries"]))))
    if args.db_limit:
        w["db"] = w["db"].subset(range(min(args.db_limit, len(w["db"]))))
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
