#!/usr/bin/env python
"""Writes the stored expected values of the full-size parity tests.

Calls only the CPU oracle (``oracle/``) on the seeded inputs of ``synth/``;
nothing here touches the CUDA library.  Run once on a CPU host:

    python tests/golden/make_fullsize.py zipf1m      # n = m = 1e6 Zipf(2.2), k = 8
    python tests/golden/make_fullsize.py largenet4m  # n = 4e6, m = 2e6 large nets, k = 64
    python tests/golden/make_fullsize.py batch       # a subset of the 512-instance batch
    python tests/golden/make_fullsize.py serve       # a sample of the Poisson serving stream

Each run writes one JSON file next to this script.  For a V-cycle it holds,
per level, the sizes and SHA-256 digests of the level's canonical CSR
(offsets, pins, net weights, node weights) and of its map to the next level,
and, per level, the objective, the moves and the digest of the partition
after label propagation (Algorithm 1 with the deterministic rules of Sec. 11).
Digests are over the little-endian int32 bytes of each array.  The
configuration is the one bench.py times: S = 16, T = 1000, f = 160, seed 1,
eps = 0.03, at most 5 passes per level.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

S, T, FACTOR, SEED, EPS, PASSES = 16, 1000, 160, 1, 30000, 5


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def vcycle_record(hgr, k: int, name: str) -> dict:
    import oracle
    t0 = time.time()
    vc = oracle.multilevel(hgr, k, EPS, S=S, T=T, factor=FACTOR, seed=SEED, max_passes=PASSES)
    levels = []
    for lv, L in enumerate(vc.levels):
        rec = {"n": int(L.n), "m": int(L.m), "p": int(L.p),
               "offsets": digest(L.offsets), "pins": digest(L.pins),
               "net_w": digest(L.net_w), "node_w": digest(L.node_w),
               "part": digest(vc.parts[lv]), "objective": int(vc.objectives[lv]),
               "moves": int(vc.moves[lv])}
        if lv < len(vc.maps):
            rec["map"] = digest(vc.maps[lv])
        levels.append(rec)
    return {"workload": name, "k": k, "eps_ppm": EPS, "S": S, "T": T, "factor": FACTOR,
            "seed": SEED, "max_passes": PASSES, "initial_objective": int(vc.initial_objective),
            "levels": levels, "oracle_seconds": round(time.time() - t0, 1)}


def run_zipf1m():
    import synth
    hgr = synth.zipf_1m(SEED)
    return vcycle_record(hgr, 8, "synth.zipf_1m(1): n = m = 1e6, Zipf(2.2) sizes in [2, 1024], "
                                 "preferential pins, weights in [1, 10]")


def run_largenet4m():
    import synth
    hgr = synth.large_net_4m(SEED)
    return vcycle_record(hgr, 64, "synth.large_net_4m(1): n = 4e6, m = 2e6, 1 % nets of "
                                  "1k-100k pins, net 0 = 100k pins, net weights in [1, 100]")


# batch: the 16 largest instances by pins, plus per k in {2, 4, 8, 16, 32} the
# four largest of the rest (36 instances in all)
def batch_subset(jobs):
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][0].p)
    pick = order[:16]
    for k in (2, 4, 8, 16, 32):
        rest = [i for i in order if i not in pick and jobs[i][1] == k]
        pick += rest[:4]
    return sorted(pick)


def _batch_one(i):
    import oracle
    import synth
    hgr, k = synth.batch_instances(SEED)[i]
    vc = oracle.multilevel(hgr, k, EPS, max_passes=PASSES)
    return {"index": i, "n": int(hgr.n), "p": int(hgr.p), "k": k, "levels": len(vc.levels),
            "objective": int(vc.objectives[0]), "part": digest(vc.parts[0])}


def run_batch():
    import synth
    jobs = synth.batch_instances(SEED)
    pick = batch_subset(jobs)
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(pick), os.cpu_count() or 1))) as pool:
        recs = pool.map(_batch_one, pick)
    return {"workload": "synth.batch_instances(1): 512 instances, n log-uniform in [1e3, 2e5], "
                        "m/n in [0.5, 3], sizes 2 + Geom(0.3) <= 64, weights in [1, 10], "
                        "k in {2, 4, 8, 16, 32}; the 16 largest plus the 4 largest of the rest "
                        "for every k", "eps_ppm": EPS, "max_passes": PASSES, "seed": SEED,
            "instances": recs}


# serve: the first 48 requests of the 200 req/s stream with at most 400,000
# pins (the oracle then needs seconds, not minutes, per request)
def serve_sample():
    import synth
    arr = synth.poisson_arrivals(SEED, rate=200.0, duration=60.0)
    return [i for i, a in enumerate(arr) if a[2] <= 400_000][:48]


def _serve_one(i):
    import oracle
    import synth
    t_arr, req_seed, pins, k = synth.poisson_arrivals(SEED, rate=200.0, duration=60.0)[i]
    hgr = synth.poisson_request(req_seed, pins)
    vc = oracle.multilevel(hgr, k, EPS, max_passes=PASSES)
    return {"index": i, "arrival_s": t_arr, "n": int(hgr.n), "p": int(hgr.p), "k": k,
            "levels": len(vc.levels), "objective": int(vc.objectives[0]),
            "part": digest(vc.parts[0])}


def run_serve():
    pick = serve_sample()
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(pick), os.cpu_count() or 1))) as pool:
        recs = pool.map(_serve_one, pick)
    return {"workload": "synth.poisson_arrivals(1, 200/s, 60 s): requests of 1e4..2e6 pins "
                        "(log-uniform), Zipf(2.2) sizes, k in {2, 8, 32}; the first 48 with at "
                        "most 400,000 pins", "eps_ppm": EPS, "max_passes": PASSES, "seed": SEED,
            "requests": recs}


TARGETS = {"zipf1m": ("fullsize_zipf1m_k8.json", run_zipf1m),
           "largenet4m": ("fullsize_largenet4m_k64.json", run_largenet4m),
           "batch": ("batch_subset.json", run_batch),
           "serve": ("serve_sample.json", run_serve)}


def main():
    names = sys.argv[1:] or list(TARGETS)
    for nm in names:
        fname, fn = TARGETS[nm]
        rec = fn()
        with open(os.path.join(HERE, fname), "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(f"{nm}: wrote {fname}", flush=True)


if __name__ == "__main__":
    main()
