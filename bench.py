#!/usr/bin/env python3
"""Benchmark: NLO real-minus-counterterm events/s on GB300.

Workload (one step = one pass of the whole hot path over one batch): g g -> t tbar g
at sqrt(s) = 1 TeV, m_t = 173 GeV, 2^20 flat massive-RAMBO phase-space points
(Philox seed 4), evaluated by me_eval_real_subtracted: FKS initial-state sector maps,
real matrix element, soft counterterm with colour-correlated Borns, collinear
counterterm with spin-correlated Borns, branch-free masking, stability test with
float64 re-evaluation of flagged points, weight accumulation.  Mixed precision
(float32 amplitudes, float64 maps/combination/rescue) is timed; the plain float64
GPU path is timed on the same batch for comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank runs an independent
replica on its own points (the method has no cross-point exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PROCESS = "gg_ttg"
SEED = 4
N_POINTS = 1 << 20
METRIC = "NLO real-minus-counterterm events/s (gg->ttg, FKS, 1 GB300)"
UNIT = "events/s"
CUT_PT_MIN, CUT_ABS_Y_MAX = 100.0, 1.0  # heavy-quark cuts of the per-term queue comparison
WORKLOAD = ("gg->ttg real-emission minus FKS soft/collinear counterterms, sqrt(s)=1 TeV, m_t=173, "
            "2^20 flat massive-RAMBO points, mixed precision (fp32 amplitudes; fp64 re-evaluation of the "
            "flagged points' real-emission blocks and counterterm Borns that their tolerance needs)")
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
NB_REAL = {"gg_ttg": 4, "uu_ttg": 2, "ee_uug": 2}  # live helicity blocks of the real emission
FP64_PER_SM_CLK = 2  # DFMA thread-ops per SM per clock (ncu: ..._op_dfma_pred_on.avg.peak_sustained)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu --set full
# capture of each kernel (summaries in profiles/), with the hash of the kernel sources they
# were taken on; reported only while the sources still hash the same.
KERNEL_SOURCES_SHA = "160a62aeb5ea1b7f"
TRAFFIC = {
    # DRAM bytes per launch from one ncu capture of each kernel (the profile named), and the
    # points of that launch; traffic_per_launch scales them to the launch measured
    ("c2", "term_items"): {"bytes": 0.401756e9 + 0.498245e9, "points": 172941,
                           "profile": "profiles/k_term_items_double_gg_ttg_2p20.md"},
    ("c1", "main"): {"bytes": 4489728 + 0, "points": 32768,
                     "profile": "profiles/k_tree_gg_tt_float_2p20.md"},
    ("c3", "main"): {"bytes": 6718208 + 2575872, "points": 32768,
                     "profile": "profiles/k_tree_gg_ttgg_float_tc_2p18.md"},
}


def kernel_sources_sha() -> str:
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2503_07439_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(csrc, "*.cuh")) + glob.glob(os.path.join(csrc, "me_inst_*.cu"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload: str, stage: str, points: int):
    t = TRAFFIC.get((workload, stage))
    if t is None or kernel_sources_sha() != KERNEL_SOURCES_SHA:
        return None
    return t["bytes"] * points / t["points"]  # scales with the points of the launch
WORKLOADS = {
    "c2": {"calls": [("gg_ttg", "real_subtracted", SEED)], "n": N_POINTS, "metric": METRIC, "workload": WORKLOAD,
           "kernels": {"gg_ttg": "k_real_sub<gg_ttg, float>"},
           "l2": "inputs 168 MB per batch > 129 MB L2 (no flush)"},
    "c0": {"calls": [("ee_uu", "nbody_nlo", 1), ("ee_uug", "real_subtracted", 2)], "n": 65536,
           "metric": "e+e- -> u ubar NLO events/s (n-body + real-minus-counterterm, 1 GB300)",
           "workload": "e+e- -> u ubar (g) at sqrt(s)=100 GeV: 65536 Born points (n-body NLO weight) + 65536 "
                       "real points (FKS final-state sectors), mixed precision",
           "kernels": {"ee_uu": "k_tree<ee_uu, float>", "ee_uug": "k_real_sub<ee_uug, float>"},
           "l2": "inputs 15 MB (< L2; compute-bound kernels)"},
    "c1": {"calls": [("gg_tt", "born", 3)], "n": N_POINTS,
           "metric": "gg -> t tbar LO events/s (1 GB300)",
           "workload": "gg -> t tbar LO, sqrt(s_hat) ~ U[400,2000] GeV, 2^20 points, float32 amplitudes",
           "kernels": {"gg_tt": "k_tree<gg_tt, float>"}, "l2": "inputs 134 MB per batch > 129 MB L2 (no flush)"},
    "c3": {"calls": [("gg_ttgg", "born", 6)], "n": 1 << 18,
           "metric": "gg -> t tbar g g tree events/s (tensor-core colour sum, 1 GB300)",
           "workload": "gg -> t tbar g g tree at sqrt(s)=2 TeV, 2^18 flat massive-RAMBO points, float32 "
                       "amplitudes, 24-flow colour sum on tensor cores (bf16 x3 split, f32 accumulate)",
           "kernels": {"gg_ttgg": "k_tree_tc4 (gg_ttgg, float; four lanes per event, mma.sync bf16 colour sum)"},
           "l2": "inputs 50 MB (< L2; compute-bound kernel)"},
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling (every 50 ms, time-stamped) of SM clock and throttle reasons.

    The sampler starts before the warm-up so that it is running when the timed region
    begins; `mark(t0, t1)` records the wall-clock bounds of the timed region and the
    summary keeps the samples taken inside it (if the region is shorter than the
    sampling interval and none falls inside, the first sample after its start)."""

    def __init__(self, index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def mark(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)  # let a sample after the region land
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as fh:
                lines = fh.readlines()
            os.unlink(self.path)
        except OSError:
            lines = []
        try:
            for line in lines:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
                rows.append((ts, float(f[1]), float(f[2]), [n for n, v in zip(names, f[5:9]) if v.lower() == "active"]))
        except Exception:
            pass
        inside = [r for r in rows if r[0] is not None and self.t0 is not None and self.t0 <= r[0] <= self.t1]
        where = "timed region"
        if not inside:
            after = [r for r in rows if r[0] is not None and self.t0 is not None and r[0] >= self.t0]
            inside, where = after[:1], "first sample after the start of the timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted({n for r in inside for n in r[3]}), "samples": len(inside), "window": where,
                "interval_ms": 50}


def _oracle_chunk(args):
    """CPU-baseline worker: the FP64 oracle on one chunk of the workload (spawned)."""
    first, n = args
    sys.path.insert(0, ROOT)
    import synth
    from oracle import fks
    from oracle.matrix_element import to_points
    b = synth.flat_points(PROCESS, n, SEED, first_point=first)
    t0 = time.perf_counter()
    fks.real_subtracted(PROCESS, to_points(b.p))
    return n, time.perf_counter() - t0


def _one_thread_per_worker():
    """numpy in every spawned worker runs single-threaded (one core each): the
    environment is set before the pool starts, since a spawned child imports numpy
    before any initializer runs."""
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    return old


def _restore_env(old):
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def cpu_baseline(points_per_worker: int = 8192):
    """The float64 oracle on every host core (one spawned process per core)."""
    workers = max(1, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    old = _one_thread_per_worker()
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_chunk, [(i * points_per_worker, points_per_worker) for i in range(workers)])
    wall = time.perf_counter() - t0
    _restore_env(old)
    n = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": n / busy, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{n} points of the same workload (first {n} of seed {SEED}), {workers} spawned "
                      f"processes x {points_per_worker} points, FP64 numpy oracle, {wall:.1f} s wall"}


def reduce_replicas(ms: float, events: float, dist=None, device: str = "cpu"):
    """Replicas (one process per GPU, independent points): the job's time is the slowest
    rank's, its work the sum over ranks.  No collective touches the data path."""
    if dist is None:
        return ms, events
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    e = torch.tensor([events], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


SERVE_KIND = {"ee_uu": "born", "ee_uug": "real_subtracted", "gg_tt": "born", "gg_ttg": "real_subtracted",
              "gg_ttgg": "born", "uu_ttg": "real_subtracted"}


def _warm_server(me, srv, n_slots):
    """The handles of every slot, and the lane layouts of every process and batch-size class
    the stream holds (256 .. 65536 points), tuned one request at a time."""
    import synth
    for proc in SERVE_KIND:
        for size in (256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536):
            srv.poll(srv.submit(proc, SERVE_KIND[proc], synth.flat_points(proc, size, 99).p))
        b = synth.flat_points(proc, 4096, 99)
        ts = [srv.submit(proc, SERVE_KIND[proc], b.p) for _ in range(2 * n_slots)]
        for t in ts:
            srv.poll(t)


def _run_load(srv, reqs, data, total, capacity, load):
    """Live arrivals at `load` x capacity (events/s); latency submit -> completion."""
    n_requests = len(reqs)
    rate = load * capacity / (total / n_requests)  # requests per second
    arrivals = [r["arrival"] / rate for r in reqs]
    lat = [0.0] * n_requests
    tickets = [None] * n_requests
    done = threading.Event()

    def poller():
        for i in range(n_requests):
            while tickets[i] is None:
                time.sleep(1e-4)
            lat[i] = srv.poll(tickets[i])["t_total_us"] * 1e-3
        done.set()

    th = threading.Thread(target=poller)
    th.start()
    start = time.perf_counter()
    for i, (r, d) in enumerate(zip(reqs, data)):
        while time.perf_counter() - start < arrivals[i]:
            time.sleep(5e-5)
        tickets[i] = srv.submit(r["process"], SERVE_KIND[r["process"]], d.p, d.wgt)
    done.wait()
    th.join()
    return arrivals, {"offered_load": load, "events_per_s": total / (time.perf_counter() - start),
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}


def serving_metrics(me, n_requests: int = 400, loads=(0.5, 0.9, 1.2), seed: int = 7, device: int = 0,
                    n_slots: int = 8):
    """Served mixed stream: Poisson arrivals scaled to each offered load x the measured
    capacity, sizes log-uniform in [256, 65536], processes uniform; latency submit ->
    completion.  The slots with replayed CUDA graphs (default server) and the persistent
    family kernels run the same arrivals; the plain FP64 path runs them live, one batch at
    a time."""
    import synth
    reqs = synth.mixed_stream(n_requests, seed)
    data = [synth.flat_points(r["process"], r["n"], r["seed"]) for r in reqs]
    total = sum(r["n"] for r in reqs)
    srv = me.Server(device=device, n_slots=n_slots, precision=me.ME_PREC_MIXED)
    _warm_server(me, srv, n_slots)

    def burst(server):
        # every request submitted at once; the fastest of three bursts (host threads of
        # other processes only ever slow one down)
        best = 0.0
        for _ in range(3):
            t0 = time.perf_counter()
            ts = [server.submit(r["process"], SERVE_KIND[r["process"]], d.p, d.wgt) for r, d in zip(reqs, data)]
            for t in ts:
                server.poll(t)
            best = max(best, total / (time.perf_counter() - t0))
        return best

    capacity = burst(srv)

    def run_load(load):
        return _run_load(srv, reqs, data, total, capacity, load)

    runs = [run_load(x) for x in loads]
    gstats = srv.stats()
    srv.close()
    # persistent family kernels (gg_ttgg on the slots), same arrivals at the same rates
    psrv = me.Server(device=device, n_slots=n_slots, precision=me.ME_PREC_MIXED, persistent=True)
    _warm_server(me, psrv, n_slots)
    pcap = burst(psrv)
    pruns = [_run_load(psrv, reqs, data, total, capacity, x)[1] for x in loads]
    pstats = psrv.stats()
    psrv.close()
    # the plain FP64 path, one batch at a time (no slots, no graphs), on the same arrivals,
    # live: each request starts when it has arrived and the previous one has finished;
    # latency = finish - arrival
    hs = {p: me.Handle(p, precision=me.ME_PREC_FP64, device=device) for p in SERVE_KIND}
    for p, h in hs.items():  # lane layouts of every batch-size class of the stream
        f = h.born if SERVE_KIND[p] == "born" else h.real_subtracted
        for size in (256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536):
            f(synth.flat_points(p, size, 98).p)
    out = []
    busy = 0.0
    for arrivals, m in runs:
        lat64 = []
        start = time.perf_counter()
        for a, r, d in zip(arrivals, reqs, data):
            while time.perf_counter() - start < a:
                time.sleep(5e-5)
            h = hs[r["process"]]
            f = h.born if SERVE_KIND[r["process"]] == "born" else h.real_subtracted
            t1 = time.perf_counter()
            f(d.p, d.wgt)
            t2 = time.perf_counter()
            busy += t2 - t1
            lat64.append(1e3 * (t2 - start - a))
        m["fp64_per_batch"] = {"events_per_s": total / (time.perf_counter() - start),
                               "p50_ms": float(np.percentile(lat64, 50)), "p99_ms": float(np.percentile(lat64, 99)),
                               "measured": "live, same arrival times, one batch at a time"}
        out.append(m)
    for h in hs.values():
        h.close()
    return {"requests": n_requests, "points": total, "slots": n_slots, "capacity_events_per_s": capacity,
            "fp64_per_batch_events_per_s_busy": total * len(runs) / busy, "loads": out,
            "graph_replays": gstats["graph_runs"], "ordinary_runs": gstats["plain_runs"],
            "persistent": {"capacity_events_per_s": pcap, "loads": pruns,
                           "kernel_launches": pstats["persistent_launches"],
                           "idle_timeouts": pstats["persistent_idle_timeouts"],
                           "requests_on_persistent_kernels": pstats["persistent_requests"],
                           "note": "ee/gg/uu families on one persistent kernel each (half the SMs each), "
                                   "gg_ttgg on the slots; arrival rates as for the graph-replay server"}}


def _reference_chunk(args):
    """Reference-arm worker: the FP64 oracle on one block of points of one call (spawned)."""
    proc, entry, seed, first, n = args
    sys.path.insert(0, ROOT)
    import synth
    from oracle import fks
    from oracle import matrix_element as ome
    from oracle import nlo_ee
    if proc == "gg_tt":
        b = synth.gg_tt_scan(n, seed, first_point=first)
    else:
        b = synth.flat_points(proc, n, seed, first_point=first)
    k = ome.to_points(b.p)
    t0 = time.perf_counter()
    if entry == "real_subtracted":
        fks.real_subtracted(proc, k)
    elif entry == "nbody_nlo":
        nlo_ee.nbody_nlo(k)
    else:
        ome.me2(proc, k)
    return n, time.perf_counter() - t0


def run_reference(args):
    """The oracle as the reference arm: bounded samples of the selected workload, spread
    over the host cores (spawned processes), one sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    workers = max(1, os.cpu_count() or 1)
    per_worker = {"c2": 1024, "c0": 4096, "c1": 4096, "c3": 16}[args.workload]
    ctx = mp.get_context("spawn")
    t_total, points = 0.0, 0
    old_env = _one_thread_per_worker()
    with ctx.Pool(workers) as pool:
        for s in range(args.warmup + args.steps):
            jobs = [(proc, entry, seed, (s * workers + i) * per_worker, per_worker)
                    for proc, entry, seed in wl["calls"] for i in range(workers)]
            t0 = time.perf_counter()
            pool.map(_reference_chunk, jobs)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                t_total += dt
                points += workers * per_worker  # events per step (one per call, as in the GPU arm)
    _restore_env(old_env)
    value = points / t_total
    sample = (f"{workers} spawned processes x {per_worker} points per call per step of the same workload "
              f"({len(wl['calls'])} call(s)), FP64 numpy oracle, wall clock")
    line = {"impl": "reference", "metric": wl["metric"], "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox + RAMBO)",
            "config": {"workload": wl["workload"], "points_per_step": workers * per_worker},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _stage_roofline(ops, calls, stages, n, workload, queued=False):
    """Roofline of the dominant kernel of a step: the stage (main kernel or float64
    rescue, over all calls of the step) with the largest CUDA-event time.  The queued
    one-launch kernel (float32 pass plus queued float64 re-evaluation) is limited by its
    float64 work: its fraction counts the re-evaluated points' flops against the float64
    peak (a lower bound: the float64 maps of the float32 pass are not counted)."""
    peak32 = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    peak64 = SM_COUNT * FP64_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    note32 = ("fp32 FMA peak 152 SMs x 128 lanes x 2 flops x 2070 MHz (nominal units at max clock; "
              "MEASURED_PEAKS.json has no fp32 figure)")
    note64 = ("fp64 peak 152 SMs x 2 DFMA/clk x 2 flops x 2070 MHz (nominal units at max clock; "
              "MEASURED_PEAKS.json has no fp64 figure)")
    cands = []
    for (proc, entry, _), (t_main, t_resc, _t_red, ncalls, resc_pts, work, cfg) in zip(calls, stages):
        per = max(1, ncalls)
        flops = ops["real_subtracted_per_event" if entry == "real_subtracted" else "born_per_event"][proc]
        kname = WORKLOADS[workload]["kernels"][proc]
        if entry == "real_subtracted" and (cfg[0] or cfg[1]) and t_resc > 0:
            # per-term queues (the default for large mixed-precision batches): the float64
            # rescue queues hold real blocks and Born configurations of two kinds
            real = ops["born_per_event"][proc]
            per_block = real / NB_REAL[proc]
            c_soft, c_coll = ops["term_config_per_event"][proc]
            item_flops = work[1] * per_block + cfg[0] * c_soft + cfg[1] * c_coll
            cands.append({"bound": "alu", "achieved": item_flops / (t_resc / per * 1e-3) / 1e12, "peak": peak64,
                          "unit": "TFLOP/s", "traffic": traffic_per_launch(workload, "term_items", resc_pts),
                          "kernel": f"k_term_items<{proc}, double> + k_terms_final (float64 rescue queues of "
                                    "the per-term path: real-emission helicity blocks and counterterm Born "
                                    "configurations of the flagged points)",
                          "peak_note": note64, "flops_per_block": per_block,
                          "flops_per_config": [c_soft, c_coll], "points": resc_pts, "real_blocks": work[1],
                          "born_configs": list(cfg), "ms_per_launch": t_resc / per})
            cands.append({"bound": "alu", "achieved": flops * n / (t_main / per * 1e-3) / 1e12 if t_main else 0.0,
                          "peak": peak32, "unit": "TFLOP/s", "traffic": None,
                          "kernel": f"k_terms<{proc}> + k_term_items<{proc}, float> + k_terms_combine (float64 "
                                    "maps and queues, bulk amplitudes, recombination)",
                          "peak_note": note32, "flops_per_event": flops, "points_per_launch": n,
                          "ms_per_launch": t_main / per,
                          "note": "flops counted as for the masked evaluation (every Born set); the queues "
                                  "evaluate only the active ones"})
            continue
        if entry == "real_subtracted" and (work[1] or work[2]) and t_resc > 0:
            # item rescue: the float64 work is the real's helicity blocks and the counterterm
            # Born sets actually re-evaluated (op counts: real = born_per_event[proc] over
            # its live blocks; Born set = the rest of the subtracted real)
            real = ops["born_per_event"][proc]
            per_block = real / NB_REAL[proc]
            born_set = flops - real
            item_flops = work[1] * per_block + work[2] * born_set
            cands.append({"bound": "alu", "achieved": item_flops / (t_resc / per * 1e-3) / 1e12, "peak": peak64,
                          "unit": "TFLOP/s", "traffic": traffic_per_launch(workload, "items", resc_pts),
                          "kernel": f"k_rescue_items<{proc}> + k_rescue_combine (float64 items of the flagged "
                                    "points: real-emission helicity blocks and counterterm Born sets)",
                          "peak_note": note64, "flops_per_block": per_block, "flops_per_born_set": born_set,
                          "points": resc_pts, "real_blocks": work[1], "born_sets": work[2],
                          "ms_per_launch": t_resc / per})
            resc_pts = 0  # accounted for above
        if queued and entry == "real_subtracted" and resc_pts > 0:
            cands.append({"bound": "alu", "achieved": flops * resc_pts / (t_main / per * 1e-3) / 1e12,
                          "peak": peak64, "unit": "TFLOP/s", "traffic": traffic_per_launch(workload, "queued", n),
                          "kernel": kname.replace("k_real_sub<", "k_real_sub_queued<").replace(", float>", ">")
                          + " (float32 pass over all points + queued float64 re-evaluation of the flagged points)",
                          "peak_note": note64, "flops_per_event": flops, "points_per_launch": n,
                          "fp64_points_per_launch": resc_pts, "ms_per_launch": t_main / per})
            continue
        cands.append({"bound": "alu", "achieved": flops * n / (t_main / per * 1e-3) / 1e12 if t_main else 0.0,
                      "peak": peak32, "unit": "TFLOP/s", "traffic": traffic_per_launch(workload, "main", n),
                      "kernel": kname, "peak_note": note32, "flops_per_event": flops, "points_per_launch": n,
                      "ms_per_launch": t_main / per})
        if resc_pts > 0 and t_resc > 0:
            cands.append({"bound": "alu", "achieved": flops * resc_pts / (t_resc / per * 1e-3) / 1e12, "peak": peak64,
                          "unit": "TFLOP/s", "traffic": traffic_per_launch(workload, "rescue", resc_pts),
                          "kernel": kname.replace("float", "double") + " (float64 re-evaluation of the flagged points)",
                          "peak_note": note64, "flops_per_event": flops, "points_per_launch": resc_pts,
                          "ms_per_launch": t_resc / per})
    for c in cands:
        c["frac"] = c["achieved"] / c["peak"]
    cands.sort(key=lambda c: -c["ms_per_launch"])
    return cands[0], (cands[1] if len(cands) > 1 else None)


def _link_rate(host, torch):
    """GB/s of a plain pinned-host -> device copy of `host` (the copy engine's rate over
    the CPU-GPU link): the ceiling of an end-to-end step whose inputs start on the host."""
    dev = torch.empty_like(host, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            dev.copy_(host, non_blocking=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(5):
            dev.copy_(host, non_blocking=True)
        b.record(s)
    torch.cuda.synchronize()
    return host.numel() * host.element_size() * 5 / (a.elapsed_time(b) * 1e-3) / 1e9


def measure(me, mebuild, workload, args, n, rank, world, local, dist, full):
    """One workload: warm-up, K timed steps (CUDA events on the launching stream, clocks
    sampled meanwhile), the plain float64 GPU path on the same batches, the end-to-end
    C-ABI call on pinned host buffers, and the roofline of the dominant kernel.  `full`
    adds the comparisons of the headline workload (the other rescue organisation, the
    step with device-generated points, unweighting)."""
    import torch
    import synth
    wl = WORKLOADS[workload]
    calls = []  # (process, entry point, batch)
    for proc, entry, seed in wl["calls"]:
        if proc == "gg_tt":
            bb = synth.gg_tt_scan(n, seed, first_point=rank * n)
        else:
            bb = synth.flat_points(proc, n, seed, first_point=rank * n)
        calls.append((proc, entry, bb))
    stream = torch.cuda.Stream()

    def make(prec, queued=args.queued_rescue, **extra):
        hs = []
        for proc, entry, bb in calls:
            hh = me.Handle(proc, precision=prec, device=local, lanes_per_event=args.lanes_per_event,
                           queued_rescue=int(queued), **extra)
            hh.set_stream(stream.cuda_stream)
            hs.append((hh, getattr(hh, entry), torch.from_numpy(bb.p).cuda(), torch.from_numpy(bb.wgt).cuda(),
                       torch.empty(n, dtype=torch.float64, device="cuda")))
        return hs

    handles = make(me.ME_PREC_MIXED)

    def step(hs):
        for hh, f, pd, wd, od in hs:
            f(pd, wd, od)

    def barrier():
        if dist is not None:
            dist.barrier()

    warmup = max(3, args.warmup)
    clk = Clocks(local).__enter__()  # sampling runs from before the warm-up
    for _ in range(warmup):
        step(handles)
    torch.cuda.synchronize()
    for hh, *_ in handles:
        hh.stage_times()
        hh.enable_stage_timers(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step(handles)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_direct = e0.elapsed_time(e1)
    stages = []
    for hh, *_ in handles:
        t_main, t_resc, t_red, ncalls = hh.stage_times()
        hh.enable_stage_timers(False)
        stages.append((t_main, t_resc, t_red, ncalls, hh.last_rescued(), hh.last_rescue_work(),
                       hh.last_rescue_configs()))
    rescued = sum(st[4] for st in stages)
    # The same step captured once in a CUDA graph and replayed: the launch mode of the
    # library's request loop for fixed-shape batches (the C-ABI calls of a step are
    # stream-ordered launches with no host synchronisation once their first call has run).
    # This is the headline: the step's kernels without per-launch host cost.
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        step(handles)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            graph.replay()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        g1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    barrier()
    clk.mark(w0, w1)
    clk.__exit__()
    ms = g0.elapsed_time(g1)
    ms_direct, _ = reduce_replicas(ms_direct, float(n * args.steps), dist, device="cuda")
    ms, events = reduce_replicas(ms, float(n * args.steps), dist, device="cuda")
    value = events / (ms * 1e-3)
    direct = {"value": events / (ms_direct * 1e-3), "unit": UNIT, "ms_per_step": ms_direct / args.steps,
              "launch": "one C-ABI call per entry point per step (stream-ordered, no graph)"}

    def time_steps(hs, k):
        step(hs)  # first call: lane-layout tuning, scratch sizing
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k):
            step(hs)
        f1.record(stream)
        torch.cuda.synchronize()
        return f0.elapsed_time(f1) / k

    fp64_ms = time_steps(make(me.ME_PREC_FP64), args.fp64_steps)
    fp64_value = n / (fp64_ms * 1e-3)
    has_real = any(entry == "real_subtracted" for _, entry, _ in calls)
    alt = devgen = unw = None
    if full and has_real:
        alt_ms = time_steps(make(me.ME_PREC_MIXED, queued=not args.queued_rescue), max(3, args.fp64_steps))
        alt = {"value": n / (alt_ms * 1e-3), "unit": UNIT, "ms_per_step": alt_ms,
               "rescue": "float32 launch, then float64 launch over the compacted list" if args.queued_rescue else
                         "queued one-launch kernel"}
    terms = None
    if full and has_real:
        # cuts of every term (Algorithm 2, masked) against the per-term queues, without
        # and with the cuts of a t tbar analysis (both heavy quarks: p_T >= 100 GeV,
        # |y| <= 1); mixed precision, the same batches
        cut = dict(cut_pt_min=CUT_PT_MIN, cut_abs_y_max=CUT_ABS_Y_MAX)
        terms = {"cuts": {"heavy_quark_pt_min_gev": CUT_PT_MIN, "heavy_quark_abs_y_max": CUT_ABS_Y_MAX}}
        for label, extra in (("masked", {"term_queues": 0}), ("queued", {"term_queues": 1}),
                             ("masked_cuts", dict(cut, term_queues=0)), ("queued_cuts", dict(cut, term_queues=1))):
            hs = make(me.ME_PREC_MIXED, **extra)
            t_ms = time_steps(hs, max(3, args.fp64_steps))
            kept = float(sum(torch.count_nonzero(od).item() for *_, od in hs)) / (n * len(hs))
            terms[label] = {"value": n / (t_ms * 1e-3), "unit": UNIT, "ms_per_step": t_ms,
                            "points_with_weight": kept}
    if full and all(proc != "gg_tt" for proc, _, _ in calls):
        # the same step with the points generated on the device every step (Philox4x32-10
        # + RAMBO, me_generate_flat)
        def gen_step(step_no):
            for (_, _, seed), (_, _, bb), (hh, f, pd, wd, od) in zip(wl["calls"], calls, handles):
                hh.generate_flat(n, seed, bb.sqrt_s, first_point=(rank + world * step_no) * n, out=(pd, wd))
                f(pd, wd, od)
        gen_step(0)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k_ in range(args.steps):
            gen_step(k_ + 1)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.steps
        devgen = {"value": n / (gms * 1e-3), "unit": UNIT, "ms_per_step": gms,
                  "note": "momenta and weights generated on the device each step, then evaluated"}
    if full and calls[0][1] == "real_subtracted":
        # unweighted events from the step's subtracted-real weights (me_unweight: accept/
        # reject against the batch maximum of |w|, on the device; synchronous, host-timed)
        hh0, _, _, _, od0 = handles[0]
        hh0.unweight(od0, seed=SEED, stream=9)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            kept, _, wm, _ = hh0.unweight(od0, seed=SEED, stream=9)
        uw_s = (time.perf_counter() - t0) / reps
        unw = {"points_per_s": n / uw_s, "ms_per_call": uw_s * 1e3, "events_kept": int(kept.shape[0]),
               "w_max": wm, "note": "accept/reject of the c2 weights against max |w| (me_unweight, host-timed)"}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    hosts = []
    for (proc, entry, bb), (hh, f, *_rest) in zip(calls, handles):
        hh.set_stream(None)
        hosts.append((f, torch.from_numpy(bb.p).pin_memory(), torch.from_numpy(bb.wgt).pin_memory(),
                      torch.empty(n, dtype=torch.float64).pin_memory()))

    def host_step():
        for f, ph, wh, oh in hosts:
            f(ph.numpy(), wh.numpy(), oh.numpy())

    host_step()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 2)
    for _ in range(e2e_steps):
        host_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    barrier()
    h2d = sum(bb.p.nbytes + bb.wgt.nbytes for _, _, bb in calls)
    d2h = len(calls) * n * 8
    link = _link_rate(hosts[0][1], torch)
    ops = mebuild.op_counts()
    roofline, other = _stage_roofline(ops, calls, stages, n, workload, queued=args.queued_rescue)
    # per call: the main kernel, the float64 work of the two-launch subtracted real (item
    # rescue: items + recombination; whole points: one launch) and the two reduction kernels
    # per-term queues (mixed precision): k_terms, the reals' and the Born configurations'
    # float32 items, k_terms_combine, the float64 items, k_terms_final
    def call_launches(entry, st):
        if entry == "real_subtracted" and (st[6][0] or st[6][1]):
            return 6 + 2
        return 1 + ((2 if st[5][1] or st[5][2] else 1) if entry == "real_subtracted" and
                    not args.queued_rescue else 0) + 2
    launches_per_step = sum(call_launches(entry, st) for (_, entry, _), st in zip(calls, stages))
    return {
        "metric": wl["metric"], "value": value, "unit": UNIT, "ms_per_step": ms / args.steps, "steps": args.steps,
        "direct_calls": direct,
        "warmup": warmup, "n_points": n, "processes": [c[0] for c in calls], "workload": wl["workload"],
        "l2": wl["l2"],
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": fp64_ms,
                      "mixed_over_fp64": value / world / fp64_value},
        "other_rescue_path": alt, "per_term_queues": terms, "rescued_per_step": rescued,
        "rescue_work_per_step": [{"process": c[0], "points": st[5][0], "real_blocks": st[5][1],
                                  "born_sets": st[5][2], "born_configs_soft_coll": list(st[6]),
                                  "path": "per-term queues" if st[6][0] or st[6][1] else "masked"}
                                 for c, st in zip(calls, stages)],
        "stage_ms_per_step": [{"process": c[0], "main_kernel": st[0] / max(1, st[3]),
                               "rescue_kernel": st[1] / max(1, st[3]), "reduction": st[2] / max(1, st[3])}
                              for c, st in zip(calls, stages)],
        "roofline": roofline, "roofline_other_kernel": other,
        "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "link_gbs": link, "h2d_gbs": h2d / e2e_s / 1e9,
                "h2d_frac_of_link": h2d / e2e_s / 1e9 / link,
                "path": "C-ABI call on pinned host buffers: the kernels read the inputs and write the results in "
                        "place over the CPU-GPU link (no staging copy); the call returns with results on the host"},
        "device_generated": devgen, "unweighting": unw,
        "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the c0, c1 and c3 sub-lines of the default (c2) run")
    ap.add_argument("--lanes-per-event", type=int, default=0,
                    help="pin the lane layout of every handle (0: autotune; profiling runs pin it, "
                         "since launch timing under a profiler misleads the tuner)")
    ap.add_argument("--queued-rescue", action="store_true",
                    help="time the queued one-launch rescue kernel instead of the two launches (float32, then "
                         "float64 over the compacted list)")
    ap.add_argument("--workload", default="c2", choices=["c0", "c1", "c2", "c3"],
                    help="c2 (default): gg->ttg real-minus-CT; c0: e+e- NLO (n-body + real-minus-CT); "
                         "c1: gg->tt LO; c3: gg->ttgg tree with the tensor-core colour sum")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # CPU baseline first (spawned pool, before any CUDA work in this process)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "c2":
        cpu = cpu_baseline()

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as me
    from paper_2503_07439_gb300 import build as mebuild

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n if args.workload == "c2" else WORKLOADS[args.workload]["n"]
    head = measure(me, mebuild, args.workload, args, n, rank, world, local, dist, full=True)
    # the other configurations of the method, measured in the same run (sub-lines), before
    # the serving run, so that every lane layout is tuned on an otherwise idle GPU
    configs = None
    if args.workload == "c2" and not args.no_configs:
        configs = {}
        for wk in ("c0", "c1", "c3"):
            m = measure(me, mebuild, wk, args, WORKLOADS[wk]["n"], rank, world, local, dist, full=False)
            configs[wk] = {k: m[k] for k in ("metric", "value", "unit", "ms_per_step", "direct_calls", "n_points",
                                             "processes",
                                             "workload", "l2", "fp64_path", "rescued_per_step",
                                             "rescue_work_per_step", "stage_ms_per_step",
                                             "roofline", "roofline_other_kernel", "e2e", "gpu_launches", "clocks")}
    serve = None
    if rank == 0 and not args.no_serving and args.workload == "c2":
        serve = serving_metrics(me, device=local)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": head["metric"], "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": head["warmup"], "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded Philox + RAMBO phase space)",
        "config": {"workload": head["workload"], "processes": head["processes"], "n_points": n,
                   "precision": "mixed", "l2": head["l2"],
                   "launch": "each step's C-ABI calls captured once in a CUDA graph, replayed per step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "direct_calls": head["direct_calls"],
        "fp64_path": head["fp64_path"],
        "other_rescue_path": head["other_rescue_path"],
        "per_term_queues": head["per_term_queues"],
        "rescued_per_step": head["rescued_per_step"],
        "rescue_work_per_step": head["rescue_work_per_step"],
        "stage_ms_per_step": head["stage_ms_per_step"],
        "roofline": head["roofline"],
        "roofline_other_kernel": head["roofline_other_kernel"],
        "e2e": head["e2e"],
        "device_generated": head["device_generated"],
        "unweighting": head["unweighting"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
        "serving": serve,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
