"""The executor (many jobs on one GPU, overlapping on the device): every job's
partition and objective equal those of the plain single call, and the oracle's
for instances small enough to run it; admission keeps the device-memory
estimates of the running jobs within the budget; a serving-style stream with
jobs arriving while others run returns the same results as each job alone."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_17679_gb300 import hg  # noqa: E402

EPS, PASSES = 30000, 5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def plain(hgr, k):
    stream = torch.cuda.current_stream()
    h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w, hg.HG_MEM_HOST,
                     None, stream)
    try:
        part = torch.empty(hgr.n, dtype=torch.int32, device="cuda")
        obj = hg.hg_partition(h, k, EPS, PASSES, part)
        return obj, part.cpu().numpy()
    finally:
        hg.hg_destroy(h)


def run_all(ex, jobs):
    for i, (hgr, k) in enumerate(jobs):
        ex.submit(hgr, k, EPS, PASSES, tag=i)
    got = {}
    while len(got) < len(jobs):
        for r in ex.wait():
            got[r["tag"]] = r
    return got


def test_batch_equals_plain_and_oracle(oracle_mod):
    jobs = synth.batch_instances(7, count=24, n_lo=1000, n_hi=20_000)
    ex = hg.Executor(slots=6)
    try:
        got = run_all(ex, jobs)
    finally:
        ex.close()
    for i, (hgr, k) in enumerate(jobs):
        r = got[i]
        assert r["status"] == hg.HG_OK
        obj, part = plain(hgr, k)
        assert r["objective"] == obj
        assert np.array_equal(r["part"], part)
    small = sorted(range(len(jobs)), key=lambda i: jobs[i][0].p)[:3]
    for i in small:
        hgr, k = jobs[i]
        vc = oracle_mod.multilevel(hgr, k, EPS, max_passes=PASSES)
        assert np.array_equal(got[i]["part"], vc.parts[0])
        assert got[i]["objective"] == vc.objectives[0]


def test_admission_respects_the_memory_budget():
    jobs = synth.batch_instances(9, count=12, n_lo=2000, n_hi=30_000)
    ex = hg.Executor(slots=8, mem_budget_bytes=600 << 20)
    try:
        got = run_all(ex, jobs)
    finally:
        ex.close()
    res = list(got.values())
    assert all(r["status"] == hg.HG_OK for r in res)
    budget = 600 << 20
    for r in res:
        t = r["t_start_ns"]
        running = [x for x in res if x["t_start_ns"] <= t < x["t_end_ns"]]
        if len(running) > 1:
            assert sum(x["est_bytes"] for x in running) <= budget
    for i, (hgr, k) in enumerate(jobs):
        obj, part = plain(hgr, k)
        assert got[i]["objective"] == obj and np.array_equal(got[i]["part"], part)


def test_serving_stream_results_match_alone():
    arrivals = synth.poisson_arrivals(3, rate=400.0, duration=0.1, pins_lo=2e4, pins_hi=3e5)
    reqs = [(synth.poisson_request(s, pins), k) for (_, s, pins, k) in arrivals]
    assert len(reqs) >= 10
    ex = hg.Executor(slots=4)
    got = {}
    try:
        t0 = time.perf_counter()
        for i, ((t_arr, _, _, _), (hgr, k)) in enumerate(zip(arrivals, reqs)):
            delay = t_arr - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ex.submit(hgr, k, EPS, PASSES, tag=i)
            for r in ex.wait(timeout_ms=0):
                got[r["tag"]] = r
        while len(got) < len(reqs):
            for r in ex.wait():
                got[r["tag"]] = r
    finally:
        ex.close()
    overlapped = 0
    res = list(got.values())
    for r in res:
        overlapped += sum(1 for x in res if x is not r and x["t_start_ns"] < r["t_end_ns"]
                          and r["t_start_ns"] < x["t_end_ns"])
        assert r["t_submit_ns"] <= r["t_start_ns"] <= r["t_end_ns"]
    assert overlapped > 0  # jobs ran concurrently
    for i, (hgr, k) in enumerate(reqs):
        obj, part = plain(hgr, k)
        assert got[i]["status"] == hg.HG_OK
        assert got[i]["objective"] == obj and np.array_equal(got[i]["part"], part)


def test_submit_rejects_bad_jobs():
    ex = hg.Executor(slots=1)
    try:
        hgr = synth.uniform_10k(1)
        with pytest.raises(hg.HgError):
            ex.submit(hgr, 1)
        with pytest.raises(hg.HgError):
            ex.submit(hgr, 65)
        assert ex.wait(timeout_ms=0) == []
    finally:
        ex.close()
