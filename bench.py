#!/usr/bin/env python
"""Benchmark: pins/s of the deterministic multilevel path (coarsen every
level, initial partition, project + label propagation on every level) on
the n = m = 1e6 Zipf workload (n = m = 1e6, Zipf(2.2) net sizes in [2, 1024],
preferential pins, node and net weights in [1, 10], k = 8, eps = 0.03).

One step = hg_create from the device-resident input CSR (incidence build)
+ hg_partition (the whole hot path) + hg_destroy.  value = sum over levels
of the level's pins / step time.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

# The executor's slots each run on their own stream; the CUDA runtime maps
# streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by default), and
# streams sharing a queue serialise each other's dependent launches.  32
# queues (the maximum) let 16-32 slots overlap; read when the process creates
# its CUDA context, so it is set before anything touches CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "pins/s per coarsen+LP level on 1 GB300, batched vs plain; serve p50/p99 ms"
K_BLOCKS, EPS_PPM, PASSES, SEED = 8, 30000, 5, 1
WORKLOAD = ("hypergraph n=m=1,000,000: Zipf(2.2) net sizes in [2,1024], preferential pins, "
            "node/net weights uniform in [1,10], k=8, eps=0.03, S=16, T=1000, f=160, "
            "5 LP passes per level, full V-cycle")
L2_FLUSH_BYTES = 512 << 20

# DRAM traffic per launch of a kernel family (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture, averaged per launch), reported
# only while the source the counters were taken from is unchanged; the
# captures are summarised under profiles/.
TRAFFIC = {
    "rating": {"source": "paper_2303_17679_gb300/csrc/coarsen.cu",
               "source_sha256": "e791612ac7ac4700d2b822fa47e78481781f9cf5a71578e9c4b1bce5f331d485",
               "bytes_per_launch": 21268333},
    "lp_gain": {"source": "paper_2303_17679_gb300/csrc/refine.cu",
                "source_sha256": "c51f75595d69410e0552f2464010ee93326afdafa9c1137fd140d2ace5ac64d2",
                "bytes_per_launch": 7014247},
}


def _source_sha256(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------ CPU oracle

# Bounded samples of the workload for the CPU oracle: the baseline leg of the
# GPU line (one run, about 10-30 s of single-threaded work on the GPU machine's
# host) and every step of the reference arm (a few seconds, so that its
# warm-up and timed steps end within a few minutes).
ORACLE_SAMPLE_N = int(os.environ.get("BENCH_ORACLE_N", "60000"))
REFERENCE_STEP_N = int(os.environ.get("BENCH_REFERENCE_N", "20000"))


def oracle_sample(n=None):
    """Times the CPU oracle (as it stands, one core) on a bounded sample of
    the same workload shape: the Zipf(2.2) hypergraph scaled to n = m nodes
    and nets (full V-cycle, k = 8)."""
    import oracle
    import synth
    n = ORACLE_SAMPLE_N if n is None else n
    hgr = synth.zipf_1m(SEED, n=n)
    t0 = time.perf_counter()
    vc = oracle.multilevel(hgr, K_BLOCKS, EPS_PPM, S=16, T=1000, factor=160, seed=SEED,
                           max_passes=PASSES)
    dt = time.perf_counter() - t0
    pins = sum(int(l.p) for l in vc.levels)
    return dict(value=pins / dt, seconds=dt, pins=pins, levels=len(vc.levels),
                sample=f"Zipf(2.2) hypergraph scaled to n=m={n:,} ({hgr.p} pins, "
                       f"{len(vc.levels)} levels, {pins} level-pins), full V-cycle, one process, "
                       "single-threaded oracle")


def run_reference(args, world, rank):
    if rank != 0:
        return
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        r = oracle_sample(REFERENCE_STEP_N)
        if i >= args.warmup:
            vals.append(r["value"])
            info = r
    v = statistics.mean(vals) if vals else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pins/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": info["seconds"] * 1e3 if info else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (CPU oracle on a bounded sample)"},
        "cpu_baseline": {"value": v, "unit": "pins/s", "cores": 1, "kind": "oracle",
                         "sample": info["sample"] if info else ""},
        "e2e": {"value": v, "unit": "pins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ batching and serving

def level_pins_of(h, hg):
    return sum(hg.hg_level_info(h, lv)[2] for lv in range(hg.hg_num_levels(h)))


def run_plain_job(hg, torch, stream, hgr, k):
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     None, stream)
    try:
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        obj = hg.hg_partition(h, k, EPS_PPM, PASSES, part)
        part.cpu()
        return obj, level_pins_of(h, hg)
    finally:
        hg.hg_destroy(h)


def run_batch(hg, torch, slots):
    """Batch of 512 seeded instances (n log-uniform in [1e3, 2e5]); the plain
    form runs them one call after another (host CSR in, partition out), the
    batched form through the executor's slots, largest first."""
    import synth
    jobs = synth.batch_instances(SEED)
    stream = torch.cuda.current_stream()
    for hgr, k in jobs[:8]:
        run_plain_job(hg, torch, stream, hgr, k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [run_plain_job(hg, torch, stream, hgr, k) for hgr, k in jobs]
    t_plain = time.perf_counter() - t0
    pins = sum(p for _, p in plain)
    ex = hg.Executor(slots)
    try:
        for i, (hgr, k) in enumerate(jobs[:slots]):
            ex.submit(hgr, k, EPS_PPM, PASSES, tag=i)
        seen = 0
        while seen < min(slots, len(jobs)):
            seen += len(ex.wait())
        t0 = time.perf_counter()
        for i in sorted(range(len(jobs)), key=lambda i: -jobs[i][0].p):
            ex.submit(jobs[i][0], jobs[i][1], EPS_PPM, PASSES, tag=i)
        got = {}
        while len(got) < len(jobs):
            for r in ex.wait():
                got[r["tag"]] = r
        t_batch = time.perf_counter() - t0
    finally:
        ex.close()
    same = all(got[i]["status"] == 0 and got[i]["objective"] == plain[i][0] for i in range(len(jobs)))
    return {"workload": "batch of 512 instances: n log-uniform in [1e3, 2e5], m/n in [0.5, 3], "
                        "net sizes 2 + Geom(0.3) <= 64, weights in [1, 10], k in {2,4,8,16,32}, host CSR in, "
                        "partition out",
            "instances": len(jobs), "level_pins": pins, "slots": slots,
            "plain_s": t_plain, "batched_s": t_batch,
            "plain_pins_per_s": pins / t_plain, "batched_pins_per_s": pins / t_batch,
            "speedup": t_plain / t_batch, "identical_objectives": same}


def serve_stream(hg, arrivals, slots, gen_workers=8):
    """Submits each request at its arrival time (generated just ahead of it by
    a thread pool) and collects results; latency = completion - arrival."""
    import concurrent.futures as cf

    import synth
    ex = hg.Executor(slots)
    pool = cf.ThreadPoolExecutor(gen_workers)
    futs = {}
    lookahead = 64
    lat, pins, objs = [], 0, {}
    t_first = t_last = None
    try:
        for i in range(min(lookahead, len(arrivals))):
            _, s, p, _ = arrivals[i]
            futs[i] = pool.submit(synth.poisson_request, s, p)
        t0_ns = hg.hg_exec_now_ns()
        done = 0

        def collect(timeout_ms):
            nonlocal done, pins, t_last
            for r in ex.wait(timeout_ms=timeout_ms):
                arr_ns = t0_ns + int(arrivals[r["tag"]][0] * 1e9)
                lat.append((r["t_end_ns"] - arr_ns) / 1e6)
                pins += r["level_pins"]
                objs[r["tag"]] = r["objective"]
                t_last = r["t_end_ns"]
                done += 1

        for i, (t_arr, _, _, k) in enumerate(arrivals):
            while True:
                wait_ns = t0_ns + int(t_arr * 1e9) - hg.hg_exec_now_ns()
                if wait_ns <= 0:
                    break
                collect(min(50, max(0, wait_ns // 1_000_000)))
            hgr = futs.pop(i).result()
            j = i + lookahead
            if j < len(arrivals):
                futs[j] = pool.submit(synth.poisson_request, arrivals[j][1], arrivals[j][2])
            ex.submit(hgr, k, EPS_PPM, PASSES, tag=i)
            if t_first is None:
                t_first = t0_ns + int(t_arr * 1e9)
            collect(0)
        while done < len(arrivals):
            collect(-1)
    finally:
        ex.close()
        pool.shutdown()
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    wall = (t_last - t_first) / 1e9
    return {"slots": slots, "requests": len(arrivals), "p50_ms": q(0.50), "p99_ms": q(0.99),
            "max_ms": lat[-1], "level_pins": pins, "pins_per_s": pins / wall, "wall_s": wall}, objs


def run_serve(hg, seconds, slots):
    """Serving stream: Poisson(200/s) requests of 1e4..2e6 pins (log-uniform), Zipf
    net sizes, k in {2, 8, 32}; continuous batching over the executor's slots
    against the plain form (one request at a time, same arrivals)."""
    import synth
    arrivals = synth.poisson_arrivals(SEED, rate=200.0, duration=seconds)
    served, objs_s = serve_stream(hg, arrivals, slots)
    # the plain form cannot keep up with the offered load, so it runs the first
    # second of arrivals only (its queue, and latency, grow without bound)
    head = [a for a in arrivals if a[0] < 1.0]
    plain, objs_p = serve_stream(hg, head, 1)
    return {"workload": f"serving stream: Poisson 200 req/s for {seconds:g} s, 1e4..2e6 pins "
                        "log-uniform, Zipf(2.2) net sizes, k in {2, 8, 32}",
            "served": served, "plain_first_second": plain,
            "identical_objectives": all(objs_s[i] == objs_p[i] for i in objs_p)}


def run_gain_recalc(hg, torch, hgr, d_off, d_pins, d_w, d_c, opt, stream, part, peak):
    """Exact gains of a move sequence (Sec. 6.3) on the n = m = 1e6 Zipf hypergraph, level 0: a seeded
    sequence moving 10 % of the nodes (from the V-cycle's partition) to
    random other blocks.  Algorithmic bytes: 16 per move (node, target, index
    write and read), 8 per incidence of a moved node (net id, mark), 20 per
    pin of a touched net (pin, index, block; the second loop re-reads pin and
    index), 8 per touched net (offsets, weight)."""
    import numpy as np
    rng = np.random.default_rng(SEED + 7)
    p0 = part.cpu().numpy()
    nodes = rng.permutation(hgr.n)[: hgr.n // 10].astype(np.int32)
    targets = ((p0[nodes] + 1 + rng.integers(0, K_BLOCKS - 1, size=len(nodes))) % K_BLOCKS)
    dn = torch.from_numpy(nodes).cuda()
    dt = torch.from_numpy(targets.astype(np.int32)).cuda()
    gains = torch.zeros(len(nodes), dtype=torch.int64, device="cuda")
    h = hg.hg_create(hgr.n, hgr.m, d_off, d_pins, d_w, d_c, hg.HG_MEM_DEVICE, opt, stream)
    try:
        for _ in range(3):
            hg.hg_recalculate_gains(h, 0, K_BLOCKS, part, dn, dt, gains)
        ms = []
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hg.hg_recalculate_gains(h, 0, K_BLOCKS, part, dn, dt, gains)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    finally:
        hg.hg_destroy(h)
    off = np.asarray(hgr.offsets, np.int64)
    sizes = np.diff(off)
    pins = np.asarray(hgr.pins)
    moved = np.zeros(hgr.n, bool)
    moved[nodes] = True
    net_of = np.repeat(np.arange(hgr.m), sizes)
    touched = np.zeros(hgr.m, bool)
    touched[net_of[moved[pins]]] = True
    incid = int(moved[pins].sum())
    tpins = int(sizes[touched].sum())
    nbytes = 16 * len(nodes) + 8 * incid + 20 * tpins + 8 * int(touched.sum())
    t = statistics.median(ms) / 1e3
    out = {"workload": "Zipf(2.2) n=m=1e6 hypergraph, level 0, 100,000 seeded moves to random other blocks",
           "moves": len(nodes), "touched_nets": int(touched.sum()), "touched_pins": tpins,
           "ms": t * 1e3, "moves_per_s": len(nodes) / t,
           "achieved_gbs": nbytes / t / 1e9, "frac_of_hbm": nbytes / t / 1e9 / peak}
    # gain table (Sec. 6.2): build for the partition, then the same moves
    # applied with the update rules (each call restores the partition first)
    b = torch.zeros(hgr.n, dtype=torch.int64, device="cuda")
    pen = torch.zeros((hgr.n, K_BLOCKS), dtype=torch.int64, device="cuda")
    work = part.clone()
    h = hg.hg_create(hgr.n, hgr.m, d_off, d_pins, d_w, d_c, hg.HG_MEM_DEVICE, opt, stream)
    try:
        tb, tm = [], []
        for rep in range(6):
            work.copy_(part)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            hg.hg_gain_table(h, 0, K_BLOCKS, work, b, pen)
            e1.record(stream)
            hg.hg_gain_table_move(h, 0, K_BLOCKS, work, dn, dt, b, pen)
            e2.record(stream)
            e2.synchronize()
            if rep >= 2:
                tb.append(e0.elapsed_time(e1))
                tm.append(e1.elapsed_time(e2))
    finally:
        hg.hg_destroy(h)
    out["gain_table"] = {"build_ms": statistics.median(tb), "move_ms": statistics.median(tm),
                         "nodes": hgr.n, "k": K_BLOCKS, "moves": len(nodes)}
    return out


# ------------------------------------------------------------ byte model

# Algorithmic bytes per level (4-byte ints, 8-byte Lambda, compulsory
# traffic), phase by phase:
#   rating      4(n+1) + 4p + 12 sum_e min(|e|, S) + 8 sum_{2<=|e|<=T} |e| min(|e|, S) + 24n
#   approval    24 per accepted join (n - n')
#   contraction 32p + 40m + 16n
#   pin counts  8p + 8m
#   LP pass     20p + 30n (best moves), plus 24 per incidence of a moved node
#               (application)
#   objective   12m
# Rating, approval and contraction count on the levels that were coarsened;
# the rest on every level.

def level_accounting(hg, torch, hgr, k, opt, stream, S=16, T=1000):
    """One untimed V-cycle, level by level, with the statistics reset per
    level: sizes, the net-size sums of the rating term, LP passes and moved
    incidences.  Results are deterministic, so these are the timed steps'."""
    import numpy as np
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    h = hg.hg_create(hgr.n, hgr.m, t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w),
                     hg.HG_MEM_DEVICE, opt, stream)
    try:
        while hg.hg_coarsen_level(h, k)[0] == hg.HG_OK:
            pass
        nl = hg.hg_num_levels(h)
        lv = []
        for l in range(nl):
            n, m, p = hg.hg_level_info(h, l)
            off = hg.hg_get_level(h, l)["offsets"].astype(np.int64)
            sz = np.diff(off)
            mn = np.minimum(sz, S)
            rated = (sz >= 2) & (sz <= T)
            lv.append({"n": n, "m": m, "p": p, "sum_min": int(mn.sum()),
                       "sum_visit": int((sz[rated] * mn[rated]).sum())})
        parts = [torch.empty(max(x["n"], 1), dtype=torch.int32, device="cuda") for x in lv]
        hg.hg_initial_partition(h, nl - 1, k, parts[-1])
        for l in range(nl - 1, -1, -1):
            if l < nl - 1:
                hg.hg_project(h, l + 1, parts[l + 1], parts[l])
            hg.hg_reset_stats(h)
            _, moves = hg.hg_lp_refine(h, l, k, EPS_PPM, PASSES, parts[l])
            st = hg.hg_get_stats(h)
            lv[l].update(passes=st["lp_passes"], moves=moves,
                         moved_incidences=st["lp_moved_incidences"])
    finally:
        hg.hg_destroy(h)
    return lv


def byte_model(lv):
    """Per-phase algorithmic bytes of one V-cycle step from level_accounting."""
    b = dict(rating=0, approval=0, contraction=0, pin_counts=0, lp_gain=0, lp_apply=0, objective=0)
    for l, x in enumerate(lv):
        n, m, p = x["n"], x["m"], x["p"]
        if l + 1 < len(lv):
            b["rating"] += 4 * (n + 1) + 4 * p + 12 * x["sum_min"] + 8 * x["sum_visit"] + 24 * n
            b["approval"] += 24 * (n - lv[l + 1]["n"])
            b["contraction"] += 32 * p + 40 * m + 16 * n
        b["pin_counts"] += 8 * p + 8 * m
        b["lp_gain"] += x["passes"] * (20 * p + 30 * n)
        b["lp_apply"] += 24 * x["moved_incidences"]
        b["objective"] += 12 * m
    b["total"] = sum(b.values())
    return b


# ------------------------------------------------------------ GPU path

def load_mapping(hg, opt):
    """Launch mapping chosen by paper_2303_17679_gb300.autotune for the Zipf
    workload (results are identical under every mapping; only speed differs)."""
    tuned_path = os.path.join(ROOT, "paper_2303_17679_gb300", "tuned_zipf1m_k8.json")
    if not os.path.exists(tuned_path):
        return "built-in defaults"
    from paper_2303_17679_gb300 import autotune
    with open(tuned_path) as f:
        autotune.apply(opt, json.load(f))
    return "autotuned (paper_2303_17679_gb300/tuned_zipf1m_k8.json)"


def add_stats(agg, st):
    for key, val in st.items():
        if isinstance(val, list):
            agg[key] = [a + b for a, b in zip(agg.get(key, [0] * len(val)), val)]
        else:
            agg[key] = agg.get(key, 0) + val


def family_rooflines(agg, steps, bm, peak):
    """Per-kernel-family achieved GB/s from the byte model and the families'
    event-timed durations inside the timed steps."""
    fam = {}
    spec = [("rating", "k_rate_* (heavy-edge rating, a3)", "ms_rating_kernels", bm["rating"],
             agg["rating_launches"]),
            ("lp_gain", "k_lp_gain_* (LP best moves, a11; both branches of a sub-round, "
                        "so a 'launch' here is one sub-round of two kernels)",
             "ms_lp_gain_kernels", bm["lp_gain"], agg["lp_gain_launches"] // 2),
            ("lp_select", "k_lp_select / k_lp_bucket (a12)", "ms_lp_select_kernels", None, None),
            ("lp_apply", "k_lp_apply (a13)", "ms_lp_apply_kernels", bm["lp_apply"],
             agg["lp_gain_launches"] // 2)]
    for key, name, ms_key, nbytes, launches in spec:
        ms = agg.get(ms_key, 0.0) / steps
        rec = {"kernel": name, "ms_per_step": ms}
        if nbytes is not None and ms > 0:
            gbs = nbytes / (ms / 1e3) / 1e9
            rec.update(alg_bytes_per_step=nbytes, achieved_gbs=gbs, frac=gbs / peak,
                       launches_per_step=int(launches // steps),
                       ms_per_launch=ms / max(1, launches // steps))
        fam[key] = rec
    return fam


def timed_vcycle(hg, torch, hgr, k, opt, stream, steps, warmup, flush, instrumented=3):
    """create (device CSR) + hg_partition + destroy, per-step CUDA events on
    the library's stream, L2 flushed between steps.  The timed steps run
    without per-kernel events; `instrumented` further steps with the kernel-
    family events on (event pairs around every rating launch, event nodes
    around every phase of the captured LP pass) give the family durations:
    those events lengthen a step by about a tenth, so they stay out of the
    headline steps."""
    import numpy as np
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    d = (t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w))
    part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")

    def step(kernel_events):
        h = hg.hg_create(hgr.n, hgr.m, *d, hg.HG_MEM_DEVICE, opt, stream)
        try:
            if kernel_events:
                hg.hg_enable_timing(h, 2)
            obj = hg.hg_partition(h, k, EPS_PPM, PASSES, part)
            levels = [hg.hg_level_info(h, i) for i in range(hg.hg_num_levels(h))]
            return obj, levels, hg.hg_get_stats(h)
        finally:
            hg.hg_destroy(h)

    def run(count, kernel_events):
        ms, agg = [], {}
        for _ in range(count):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            obj, levels, st = step(kernel_events)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            add_stats(agg, st)
            results.append((obj, levels))
        return ms, agg

    results = []
    for _ in range(warmup):
        step(False)
    step(True)
    torch.cuda.synchronize()
    step_ms, agg = run(steps, False)
    instr_ms, iagg = run(instrumented, True)
    assert all(r == results[0] for r in results), "non-deterministic result"
    iagg["instrumented_steps"] = instrumented
    iagg["instrumented_ms_per_step"] = statistics.mean(instr_ms) if instr_ms else None
    return step_ms, agg, iagg, results[0][0], results[0][1], part


def config1_line(hg, torch, stream, flush, peak, steps=20, warmup=5):
    """n = m = 10,000 uniform hypergraph, k = 2: one clustering + contraction
    step, seeded initial partition of the fine level, 5 LP passes on it."""
    import numpy as np
    import synth
    hgr = synth.uniform_10k(SEED)
    opt = hg.hg_default_options()
    opt.seed = SEED
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    d = (t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w))
    part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
    ms, obj0 = [], None
    for i in range(warmup + steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = hg.hg_create(hgr.n, hgr.m, *d, hg.HG_MEM_DEVICE, opt, stream)
        try:
            hg.hg_coarsen_level(h, 2)
            hg.hg_initial_partition(h, 0, 2, part)
            obj, moves = hg.hg_lp_refine(h, 0, 2, EPS_PPM, PASSES, part)
        finally:
            hg.hg_destroy(h)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
        obj0 = obj if obj0 is None else obj0
        assert obj == obj0, "non-deterministic result"
    t_ms = statistics.mean(ms)
    return {"workload": "n=m=10,000 uniform hypergraph, 2 + Geom(0.3) <= 64 sizes, unit weights, k=2: "
                        "create + one clustering/contraction step + initial partition + 5 LP passes "
                        "on the fine level", "pins": hgr.p, "ms_per_step": t_ms,
            "pins_per_s": hgr.p / (t_ms / 1e3), "objective": obj0,
            "note": "launch-latency bound by design (about 2 MB of algorithmic bytes)"}


def config3_line(hg, torch, stream, flush, peak, steps=2, warmup=1):
    """n = 4e6, m = 2e6 large-net hypergraph, k = 64, full V-cycle."""
    import synth
    hgr = synth.large_net_4m(SEED)
    opt = hg.hg_default_options()
    opt.seed = SEED
    step_ms, _, iagg, obj, levels, _ = timed_vcycle(hg, torch, hgr, 64, opt, stream, steps,
                                                    warmup, flush, instrumented=1)
    lv = level_accounting(hg, torch, hgr, 64, opt, stream)
    bm = byte_model(lv)
    t_ms = statistics.mean(step_ms)
    pins = sum(p for (_, _, p) in levels)
    fam = family_rooflines(iagg, 1, bm, peak)
    return {"workload": "n=4e6, m=2e6: 99% nets 2 + Geom(0.3) <= 16, 1% of 1k-100k pins (x^-4), "
                        "net 0 = 100k pins; unit node weights, net weights in [1, 100]; k=64, "
                        "eps=0.03, T=1000, full V-cycle", "levels": len(levels),
            "pins_per_step": pins, "ms_per_step": t_ms, "pins_per_s": pins / (t_ms / 1e3),
            "objective": obj, "level_frac": bm["total"] / (t_ms / 1e3) / 1e9 / peak,
            "alg_bytes_per_step": bm, "families": fam,
            "instrumented_ms_per_step": iagg["instrumented_ms_per_step"], "level_sizes": [list(x) for x in levels]}


def graph_line(hg, torch, stream, flush, steps=3, warmup=1):
    """Graph path (Sec. 10) against the hypergraph path on the same graph:
    n = 1e6 nodes, m = 4e6 edges with preferential endpoints, weights in
    [1, 10], k = 8, full V-cycle; identical results are asserted."""
    import synth
    hgr = synth.graph_preferential(SEED, 1_000_000, 4_000_000)
    out = {"workload": "graph n=1e6, m=4e6 edges (nets of two pins), preferential endpoints, "
                       "node/edge weights in [1,10], k=8, eps=0.03, full V-cycle"}
    objs = {}
    for name, gp in (("graph_path", 0), ("hypergraph_path", 1)):
        opt = hg.hg_default_options()
        opt.seed = SEED
        opt.graph_path = gp
        step_ms, _, iagg, obj, levels, _ = timed_vcycle(hg, torch, hgr, K_BLOCKS, opt, stream,
                                                        steps, warmup, flush, instrumented=1)
        t_ms = statistics.mean(step_ms)
        pins = sum(p for (_, _, p) in levels)
        objs[name] = (obj, levels)
        out[name] = {"ms_per_step": t_ms, "pins_per_s": pins / (t_ms / 1e3), "levels": len(levels),
                     "pins_per_step": pins, "objective": obj,
                     "rating_kernels_ms": iagg["ms_rating_kernels"],
                     "lp_kernels_ms": iagg["ms_lp_gain_kernels"] + iagg["ms_lp_select_kernels"]
                     + iagg["ms_lp_apply_kernels"]}
    out["identical_results"] = objs["graph_path"] == objs["hypergraph_path"]
    out["speedup"] = out["hypergraph_path"]["ms_per_step"] / out["graph_path"]["ms_per_step"]
    return out


def communities_line(hg, torch, stream, flush, plain_obj, steps=3, warmup=1):
    """Community-aware V-cycle (Sec. 4, Sec. 11) on the n = m = 1e6 Zipf
    workload: deterministic Louvain on the bipartite graph before coarsening,
    contractions kept inside communities; against the plain V-cycle's cut."""
    import numpy as np
    import synth
    hgr = synth.zipf_1m(SEED)
    opt = hg.hg_default_options()
    opt.seed = SEED
    opt.community_detection = 1
    step_ms, _, _, obj, levels, _ = timed_vcycle(hg, torch, hgr, K_BLOCKS, opt, stream, steps,
                                                 warmup, flush, instrumented=0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    h = hg.hg_create(hgr.n, hgr.m, t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w),
                     hg.HG_MEM_DEVICE, opt, stream)
    try:
        hg.hg_enable_timing(h, 1)
        count = hg.hg_detect_communities(h)
        st = hg.hg_get_stats(h)
    finally:
        hg.hg_destroy(h)
    t_ms = statistics.mean(step_ms)
    pins = sum(p for (_, _, p) in levels)
    return {"workload": WORKLOAD + ", communities detected first (Louvain on the bipartite graph)",
            "ms_per_step": t_ms, "pins_per_s": pins / (t_ms / 1e3), "levels": len(levels),
            "objective": obj, "objective_without_communities": plain_obj,
            "communities": count, "detection_ms": st["ms_communities"],
            "louvain_levels": st["louvain_levels"], "louvain_rounds": st["louvain_rounds"],
            "louvain_moves": st["louvain_moves"]}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import synth
    from paper_2303_17679_gb300 import build as libbuild
    from paper_2303_17679_gb300 import hg

    torch.cuda.set_device(local)
    libbuild.build()
    hg.load()
    stream = torch.cuda.current_stream()
    hgr = synth.zipf_1m(SEED)
    opt = hg.hg_default_options()
    opt.seed = SEED
    mapping = load_mapping(hg, opt)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()
    h_off, h_pins, h_w, h_c = pin(hgr.offsets), pin(hgr.pins), pin(hgr.net_w), pin(hgr.node_w)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    peak, peak_kind = peaks()

    # ---- device-resident timed region
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, agg, iagg, obj, levels, part = timed_vcycle(hg, torch, hgr, K_BLOCKS, opt, stream,
                                                         args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    barrier(world)
    pins_per_step = sum(p for (_, _, p) in levels)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    t_total = max_over_ranks(world, sum(step_ms) / 1e3)
    total_pins = sum_over_ranks(world, pins_per_step * args.steps)
    value = total_pins / t_total
    launches = agg["launches"]

    # ---- end to end through the public API with host buffers
    e2e_ms = []
    for _ in range(0 if args.no_e2e else args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = hg.hg_create(hgr.n, hgr.m, h_off.numpy(), h_pins.numpy(), h_w.numpy(), h_c.numpy(),
                         hg.HG_MEM_HOST, opt, stream)
        try:
            hg.hg_partition(h, K_BLOCKS, EPS_PPM, PASSES, part)
            out = part.cpu()
            assert out.shape[0] == hgr.n
        finally:
            hg.hg_destroy(h)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = max_over_ranks(world, sum(e2e_ms) / 1e3) if e2e_ms else 0.0
    e2e_value = total_pins / e2e_t if e2e_ms else None
    h2d = 4 * (hgr.m + 1 + hgr.p + hgr.m + hgr.n)
    d2h = 4 * hgr.n

    # ---- byte model (untimed accounting pass) and rooflines
    lv = level_accounting(hg, torch, hgr, K_BLOCKS, opt, stream)
    bm = byte_model(lv)
    ms_step = statistics.mean(step_ms)
    ni = iagg["instrumented_steps"]
    fam = family_rooflines(iagg, ni, bm, peak)
    for key, tref in TRAFFIC.items():
        fresh = tref["source_sha256"] == _source_sha256(tref["source"])
        fam[key]["dram_bytes_per_launch_ncu"] = tref["bytes_per_launch"] if fresh else None
    dom = max(("rating", "lp_gain"), key=lambda f: fam[f]["ms_per_step"])
    d = fam[dom]
    traffic = None
    tref = TRAFFIC.get(dom)
    if tref and tref["source_sha256"] == _source_sha256(tref["source"]):
        traffic = tref["bytes_per_launch"]
    u32_rate, u64_rate = hg.hg_calibrate_smem_atomics(stream)
    rating_ms = iagg["ms_rating_kernels"] / ni
    visits = iagg["rating_pin_visits"] / ni
    visit_bytes = (24 * iagg["rating_nodes"] + 16 * iagg["rating_incidences"]
                   + 8 * iagg["rating_pin_visits"]) / ni

    line = {
        "metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded generator: Zipf(2.2) net sizes, preferential pins, n=m=1e6)",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between steps (512 MiB write outside the timed events)",
                   "launch_mapping": mapping,
                   "levels": len(levels), "pins_per_step": pins_per_step, "objective": obj},
        "e2e": {"value": e2e_value, "unit": "pins/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms) if e2e_ms else None},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": d["kernel"], "achieved": d.get("achieved_gbs", 0.0),
                     "peak": peak, "unit": "GB/s", "frac": d.get("frac", 0.0), "traffic": traffic,
                     "peak_kind": peak_kind + " (hbm_gbs, copy burst)",
                     "bytes_model": "per-phase algorithmic byte formulas (rating, approval, contraction, pin counts, LP gain and apply, objective) from per-level statistics",
                     "durations": f"CUDA events on the library's stream over {ni} instrumented "
                                  "steps run right after the timed steps (the per-kernel events "
                                  "stay out of the headline steps)",
                     "instrumented_ms_per_step": iagg["instrumented_ms_per_step"],
                     "launches_per_step": d.get("launches_per_step"),
                     "algorithmic_bytes_per_launch":
                         d.get("alg_bytes_per_step", 0) / max(1, d.get("launches_per_step") or 1),
                     "ms_per_launch": d.get("ms_per_launch"),
                     "share_of_step": d["ms_per_step"] / ms_step,
                     "level_frac": bm["total"] / (ms_step / 1e3) / 1e9 / peak,
                     "alg_bytes_per_step": bm, "families": fam,
                     "rating_visit_model": {
                         "note": "24 B per rated node + 16 B per incidence + 8 B per pin visit "
                                 "(visits are served from L2 and shared memory)",
                         "bytes_per_step": visit_bytes,
                         "achieved_gbs": visit_bytes / (rating_ms / 1e3) / 1e9 if rating_ms else None},
                     "smem_atomics": {
                         "bound": "rating table updates (one shared-memory atomic add per pin visit)",
                         "visits_per_step": visits,
                         "achieved_per_s": visits / (rating_ms / 1e3) if rating_ms else None,
                         "peak_u32_per_s": u32_rate, "peak_u64_per_s": u64_rate,
                         "peak_kind": "measured (hg_calibrate_smem_atomics, conflict-free adds)",
                         "frac": (visits / (rating_ms / 1e3)) / u32_rate if rating_ms else None}},
        "clocks": clocks,
        "wall_s": wall,
        "phase_ms": {"rating_kernels": rating_ms,
                     "lp_gain_kernels": iagg["ms_lp_gain_kernels"] / ni,
                     "lp_select_kernels": iagg["ms_lp_select_kernels"] / ni,
                     "lp_apply_kernels": iagg["ms_lp_apply_kernels"] / ni,
                     "timing_failures": int(iagg["timing_failures"]),
                     "from": f"{ni} instrumented steps"},
        "work_per_step": {key: int(agg[key] // args.steps) for key in (
            "rating_nodes", "rating_incidences", "rating_pin_visits", "lp_nodes", "lp_incidences",
            "lp_moved_incidences", "lp_passes")},
        "rating_classes": [
            {"class": c, "ms": round(iagg["ms_rating_class"][c] / ni, 3),
             "visits": int(iagg["rating_visits_class"][c] // ni),
             "Gvisits_per_s": round(iagg["rating_visits_class"][c] / iagg["ms_rating_class"][c] / 1e6, 2)
             if iagg["ms_rating_class"][c] > 0 else None}
            for c in range(5)],
        "level_sizes": [list(x) for x in levels],
        "unshrunk_levels": {
            "note": "levels identical in size to the level they were contracted from (the 1 % "
                    "rule keeps such a level and runs LP on it)",
            "count": sum(1 for i in range(1, len(levels)) if levels[i] == levels[i - 1]),
            "pins_per_step": sum(levels[i][2] for i in range(1, len(levels))
                                 if levels[i] == levels[i - 1])},
    }
    if world == 1 and not args.no_configs:
        line["config1"] = config1_line(hg, torch, stream, flush, peak)
        line["config3"] = config3_line(hg, torch, stream, flush, peak)
        line["graph"] = graph_line(hg, torch, stream, flush)
        line["communities"] = communities_line(hg, torch, stream, flush, obj)
    if world == 1:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
        line["gain_recalc"] = run_gain_recalc(hg, torch, hgr, t(hgr.offsets), t(hgr.pins),
                                              t(hgr.net_w), t(hgr.node_w), opt, stream, part, peak)
    if world == 1 and not args.no_batch:
        line["batch"] = run_batch(hg, torch, args.slots)
    if world == 1 and args.serve_seconds > 0:
        line["serve"] = run_serve(hg, args.serve_seconds, args.slots)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample()
        line["cpu_baseline"] = {"value": cb["value"], "unit": "pins/s", "cores": 1, "kind": "oracle",
                                "sample": cb["sample"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_profile(args):
    """For profilers: `warmup` untimed V-cycle steps then one more step of the
    named workload (the same calls as a timed step), no output."""
    import numpy as np
    import torch

    import synth
    from paper_2303_17679_gb300 import build as libbuild
    from paper_2303_17679_gb300 import hg

    libbuild.build()
    hg.load()
    stream = torch.cuda.current_stream()
    opt = hg.hg_default_options()
    opt.seed = SEED
    if args.profile == "zipf1m":
        hgr, k = synth.zipf_1m(SEED), K_BLOCKS
        load_mapping(hg, opt)
    elif args.profile == "largenet4m":
        hgr, k = synth.large_net_4m(SEED), 64
    else:
        hgr, k = synth.graph_preferential(SEED, 1_000_000, 4_000_000), K_BLOCKS
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    d = (t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w))
    part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup + 1):
        h = hg.hg_create(hgr.n, hgr.m, *d, hg.HG_MEM_DEVICE, opt, stream)
        try:
            hg.hg_partition(h, k, EPS_PPM, PASSES, part)
        finally:
            hg.hg_destroy(h)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end steps")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batch comparison")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson serving run (0: skip)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the n=m=1e4 and 4e6-node large-net sub-objects")
    ap.add_argument("--slots", type=int, default=16, help="executor slots for batch and serve")
    ap.add_argument("--profile", choices=["zipf1m", "largenet4m", "graph1m"], default=None,
                    help="run warm-up steps and one step of a workload for a profiler, no output")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
