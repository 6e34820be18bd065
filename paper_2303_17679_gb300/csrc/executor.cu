// Job executor for many partition jobs on one GPU: a pool of slots, each a
// host thread with its own non-blocking CUDA stream, that runs whole jobs
// (hg_create from host CSR, hg_partition, the partition copied to the host,
// hg_destroy) through the same entry points as a plain call, so a job's
// result does not depend on what else runs.  Jobs start in submission order
// when a slot is free and the device-memory estimate of the running jobs
// plus the next one fits the budget (a job larger than the whole budget runs
// alone).  The kernels of concurrently running jobs overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Device bytes a job may hold at its peak: the level hierarchy (about eight
// times the input's pins, net and node arrays on a Zipf(2.2) n = m = 1e6 input), the
// clustering temporaries of the finest level (pin-cluster map: 12 bytes per
// slot, 4 slots per pin), Phi (m x k int32) and Lambda, plus a fixed margin.
int64_t estimate_bytes(const hg_job& j, int64_t p) {
  const int64_t n = j.n, m = j.m, k = j.k;
  return 8 * (12 * p + 16 * m + 24 * n) + 64 * p + 4 * m * k + 8 * m + (32ll << 20);
}

struct Pending {
  int64_t ticket;
  hg_job job;
  int64_t est;
  int64_t t_submit;
};

}  // namespace

struct hg_exec_t {
  int device = 0;
  int slots = 0;
  int64_t budget = 0;
  int64_t reserved = 0;
  int running = 0;
  hg_options opt{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::deque<hg_job_result> done;
  std::vector<std::thread> threads;
  bool stop = false;
  int64_t next_ticket = 1;
};

namespace {

void run_job(hg_exec_t* ex, cudaStream_t st, cudaEvent_t waiter, const Pending& pj,
             hg_job_result& r) {
  const hg_job& j = pj.job;
  hg_t* h = nullptr;
  int rc = hg_create(j.n, j.m, j.net_offsets, j.pins, j.net_weights, j.node_weights, HG_MEM_HOST,
                     &ex->opt, st, &h);
  int32_t* dpart = nullptr;
  if (rc == HG_OK) {
    try {
      if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&dpart),
                                  sizeof(int32_t) * (size_t)std::max(j.n, 1),
                                  hgk::library_pool(ex->device), st) != cudaSuccess) {
        cudaGetLastError();
        dpart = nullptr;
        rc = HG_ERR_OOM;
      }
    } catch (const hgk::HgError& e) {
      rc = e.code;
    }
  }
  int64_t obj = 0;
  if (rc == HG_OK) rc = hg_partition(h, j.k, j.eps_ppm, j.max_passes, dpart, &obj);
  if (rc == HG_OK && cudaMemcpyAsync(j.part_out, dpart, sizeof(int32_t) * (size_t)j.n,
                                     cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = HG_ERR_CUDA;
  if (dpart) cudaFreeAsync(dpart, st);
  if (waiter && cudaEventRecord(waiter, st) == cudaSuccess) cudaEventSynchronize(waiter);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == HG_OK) rc = HG_ERR_CUDA;
  int32_t levels = 0;
  int64_t pins = 0;
  if (rc == HG_OK && hg_num_levels(h, &levels) == HG_OK) {
    for (int32_t l = 0; l < levels; ++l) {
      int64_t p = 0;
      if (hg_level_info(h, l, nullptr, nullptr, &p) == HG_OK) pins += p;
    }
  }
  hg_destroy(h);
  r.status = rc;
  r.objective = obj;
  r.levels = levels;
  r.level_pins = pins;
}

void slot_main(hg_exec_t* ex) {
  cudaSetDevice(ex->device);
  cudaStream_t st = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  cudaEvent_t waiter = nullptr;
  if (cudaEventCreateWithFlags(&waiter, cudaEventBlockingSync | cudaEventDisableTiming) !=
      cudaSuccess)
    waiter = nullptr;
  while (true) {
    Pending pj;
    {
      std::unique_lock<std::mutex> lk(ex->mu);
      ex->cv_work.wait(lk, [&] {
        if (ex->stop && ex->queue.empty()) return true;
        if (ex->queue.empty()) return false;
        return ex->running == 0 || ex->reserved + ex->queue.front().est <= ex->budget;
      });
      if (ex->queue.empty()) break;  // stopping
      pj = ex->queue.front();
      ex->queue.pop_front();
      ex->reserved += pj.est;
      ex->running += 1;
    }
    hg_job_result r{};
    r.ticket = pj.ticket;
    r.tag = pj.job.tag;
    r.est_bytes = pj.est;
    r.t_submit_ns = pj.t_submit;
    r.t_start_ns = now_ns();
    if (have_stream) run_job(ex, st, waiter, pj, r);
    else r.status = HG_ERR_CUDA;
    r.t_end_ns = now_ns();
    {
      std::lock_guard<std::mutex> lk(ex->mu);
      ex->reserved -= pj.est;
      ex->running -= 1;
      ex->done.push_back(r);
    }
    ex->cv_done.notify_all();
    ex->cv_work.notify_all();
  }
  if (waiter) cudaEventDestroy(waiter);
  if (have_stream) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int hg_exec_create(int32_t slots, int64_t mem_budget_bytes, const hg_options* opt,
                   hg_exec_t** out) {
  if (!out) return HG_ERR_INVALID;
  *out = nullptr;
  if (slots < 1 || slots > 256 || mem_budget_bytes < 0) return HG_ERR_INVALID;
  auto* ex = new (std::nothrow) hg_exec_t();
  if (!ex) return HG_ERR_OOM;
  if (opt) ex->opt = *opt;
  else hg_default_options(&ex->opt);
  ex->opt.blocking_sync = 1;  // slot threads sleep while their jobs run
  if (cudaGetDevice(&ex->device) != cudaSuccess) {
    delete ex;
    return HG_ERR_CUDA;
  }
  if (mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete ex;
      return HG_ERR_CUDA;
    }
    mem_budget_bytes = (int64_t)(fr / 10 * 8);
  }
  ex->budget = mem_budget_bytes;
  ex->slots = slots;
  try {
    for (int i = 0; i < slots; ++i) ex->threads.emplace_back(slot_main, ex);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(ex->mu);
      ex->stop = true;
    }
    ex->cv_work.notify_all();
    for (auto& t : ex->threads) t.join();
    delete ex;
    return HG_ERR_OOM;
  }
  *out = ex;
  return HG_OK;
}

int hg_exec_submit(hg_exec_t* ex, const hg_job* job, int64_t* out_ticket) {
  if (!ex || !job) return HG_ERR_INVALID;
  const hg_job& j = *job;
  if (j.n < 1 || j.m < 0 || !j.net_offsets || !j.part_out || j.k < 2 || j.k > HG_MAX_K ||
      j.eps_ppm < 0 || j.max_passes < 0)
    return HG_ERR_INVALID;
  const int64_t p = j.net_offsets[j.m];  // host CSR: the pin count
  if (p < 0 || (p > 0 && !j.pins)) return HG_ERR_INVALID;
  Pending pj;
  pj.job = j;
  pj.est = estimate_bytes(j, p);
  pj.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(ex->mu);
    if (ex->stop) return HG_ERR_STATE;
    pj.ticket = ex->next_ticket++;
    ex->queue.push_back(pj);
  }
  ex->cv_work.notify_all();
  if (out_ticket) *out_ticket = pj.ticket;
  return HG_OK;
}

int hg_exec_wait(hg_exec_t* ex, int32_t max_results, int32_t timeout_ms, hg_job_result* out,
                 int32_t* out_count) {
  if (!ex || !out || !out_count || max_results < 1) return HG_ERR_INVALID;
  std::unique_lock<std::mutex> lk(ex->mu);
  // a result, or nothing left that could produce one
  auto ready = [&] { return !ex->done.empty() || (ex->queue.empty() && ex->running == 0); };
  if (timeout_ms < 0) ex->cv_done.wait(lk, ready);
  else ex->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  int32_t c = 0;
  while (c < max_results && !ex->done.empty()) {
    out[c++] = ex->done.front();
    ex->done.pop_front();
  }
  *out_count = c;
  return HG_OK;
}

int hg_exec_pending(hg_exec_t* ex, int32_t* out_queued, int32_t* out_running) {
  if (!ex) return HG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ex->mu);
  if (out_queued) *out_queued = (int32_t)ex->queue.size();
  if (out_running) *out_running = ex->running;
  return HG_OK;
}

int64_t hg_exec_now_ns(void) { return now_ns(); }

int hg_exec_destroy(hg_exec_t* ex) {
  if (!ex) return HG_OK;
  {
    std::lock_guard<std::mutex> lk(ex->mu);
    ex->stop = true;
  }
  ex->cv_work.notify_all();
  for (auto& t : ex->threads) t.join();
  delete ex;
  return HG_OK;
}

}  // extern "C"
