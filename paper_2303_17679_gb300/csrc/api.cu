// C ABI of the library (declared in include/hg.h): the handle holding the
// level hierarchy, argument checking, the multilevel loop of Algorithm 1 and
// the seeded host-side initial partition.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <thread>
#include <vector>

#include "common.cuh"

using hgk::DBuf;
using hgk::HgError;
using hgk::Level;

struct hg_t {
  hgk::Ctx cx;
  hg_options opt;
  int device = 0;
  int64_t W0 = 0;            // total node weight c(V), invariant under contraction
  bool finished = false;     // the last coarsening step shrank by < 1 %
  int sticky = 0;            // HG_ERR_CUDA once a CUDA error was seen
  int64_t launches = 0;
  hg_stats stats{};
  std::vector<std::unique_ptr<Level>> levels;
};

namespace {

template <typename F>
int guarded(hg_t* h, F&& body) {
  if (h && h->sticky) return h->sticky;
  try {
    if (h) cudaSetDevice(h->device);
    return body();
  } catch (const HgError& e) {
    if (h && (e.code == HG_ERR_CUDA)) h->sticky = HG_ERR_CUDA;
    if (std::getenv("HG_VERBOSE")) std::fprintf(stderr, "hg: %s\n", e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    return HG_ERR_OOM;
  } catch (...) {
    if (h) h->sticky = HG_ERR_CUDA;
    return HG_ERR_CUDA;
  }
}

// Host inputs with at most this many pins have their pins checked on the
// host, larger ones on the device.
constexpr int64_t HOST_PIN_CHECK_MAX = 1 << 16;
constexpr int64_t HOST_CSR_CHECK_MAX = 1 << 22;

bool valid_level(const hg_t* h, int32_t level) {
  return level >= 0 && level < (int32_t)h->levels.size();
}

// Pins of nets [e0, e1) in [0, n) and no node twice in a net: nets of up to
// 16 pins compare their pins pairwise, larger nets stamp their nodes in
// `stamp` (n entries, allocated on first use).
bool check_pins_range(int32_t n, const int32_t* off, const int32_t* pins, int32_t e0, int32_t e1,
                      std::vector<int32_t>& stamp) {
  for (int32_t e = e0; e < e1; ++e) {
    const int32_t b = off[e], sz = off[e + 1] - b;
    for (int32_t q = b; q < b + sz; ++q)
      if (pins[q] < 0 || pins[q] >= n) return false;
    if (sz <= 16) {
      for (int32_t i = 1; i < sz; ++i)
        for (int32_t j = 0; j < i; ++j)
          if (pins[b + i] == pins[b + j]) return false;
    } else {
      if (stamp.empty()) stamp.assign((size_t)n, -1);
      for (int32_t q = b; q < b + sz; ++q) {
        if (stamp[pins[q]] == e) return false;
        stamp[pins[q]] = e;
      }
    }
  }
  return true;
}

// Host-side checks of a host CSR (hg_create contract): offsets and weights,
// and the pins when `pins` is given (on up to 8 host threads over ranges of
// nets; hg_create passes NULL and checks the pins on the device instead).
int check_host_csr(int32_t n, int32_t m, const int32_t* off, const int32_t* pins, const int32_t* w,
                   const int32_t* c, int64_t* W) {
  if (off[0] != 0) return HG_ERR_INVALID;
  for (int32_t e = 0; e < m; ++e)
    if (off[e + 1] <= off[e]) return HG_ERR_INVALID;  // decreasing or empty net
  const int64_t p = pins ? off[m] : 0;
  const int threads = (int)std::max<int64_t>(
      1, std::min<int64_t>({8, (int64_t)std::thread::hardware_concurrency(), p / (1 << 20) + 1}));
  std::vector<char> ok((size_t)threads, 1);
  if (!pins) {
    // pins checked elsewhere
  } else if (threads == 1) {
    std::vector<int32_t> stamp;
    ok[0] = check_pins_range(n, off, pins, 0, m, stamp);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
      pool.emplace_back([&, t] {
        std::vector<int32_t> stamp;
        const int32_t e0 = (int32_t)((int64_t)m * t / threads);
        const int32_t e1 = (int32_t)((int64_t)m * (t + 1) / threads);
        ok[t] = check_pins_range(n, off, pins, e0, e1, stamp);
      });
    for (auto& th : pool) th.join();
  }
  for (char x : ok)
    if (!x) return HG_ERR_INVALID;
  int64_t sw = 0, sc = 0;
  if (w)
    for (int32_t e = 0; e < m; ++e) {
      if (w[e] <= 0) return HG_ERR_INVALID;
      sw += w[e];
    }
  else sw = m;
  if (c)
    for (int32_t u = 0; u < n; ++u) {
      if (c[u] <= 0) return HG_ERR_INVALID;
      sc += c[u];
    }
  else sc = n;
  if (sw >= (1ll << 31) || sc >= (1ll << 31)) return HG_ERR_INVALID;
  (void)p;
  *W = sc;
  return HG_OK;
}

void upload(const hgk::Ctx& cx, DBuf<int32_t>& dst, const int32_t* src, size_t count, int mem,
            int32_t fill_if_null) {
  dst.alloc(&cx.alloc, std::max<size_t>(count, 1));
  if (count == 0) return;
  if (src) {
    HG_CUDA(cudaMemcpyAsync(dst.p, src, count * sizeof(int32_t),
                            mem == HG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            cx.stream));
  } else {
    hgk::fill_i32(cx, dst.p, fill_if_null, (int64_t)count);
  }
}

void sync_stats(hg_t* h) { h->stats.launches = h->launches; }

}  // namespace

extern "C" {

void hg_default_options(hg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->seed = 1;
  opt->subrounds = 16;
  opt->rating_max_net_size = 1000;
  opt->contraction_limit_factor = 160;
  opt->fingerprint_bits = 0;
}

const char* hg_strerror(int status) {
  switch (status) {
    case HG_OK: return "ok";
    case HG_STOP: return "stop: no further coarsening";
    case HG_ERR_INVALID: return "invalid argument";
    case HG_ERR_UNSUPPORTED: return "unsupported size or parameter";
    case HG_ERR_OOM: return "out of device memory";
    case HG_ERR_CUDA: return "CUDA error (handle unusable)";
    case HG_ERR_TIMEOUT: return "bounded device wait timed out";
    case HG_ERR_STATE: return "call out of order for this handle";
    default: return "unknown status";
  }
}

const char* hg_version(void) { return "hgpart-gb300 0.1 (sm_103a)"; }

int hg_create(int32_t n, int32_t m, const int32_t* net_offsets, const int32_t* pins,
              const int32_t* net_weights, const int32_t* node_weights, int32_t mem,
              const hg_options* opt, void* cuda_stream, hg_t** out) {
  if (!out) return HG_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || m < 0 || !net_offsets || (mem != HG_MEM_HOST && mem != HG_MEM_DEVICE))
    return HG_ERR_INVALID;
  hg_options o;
  hg_default_options(&o);
  if (opt) o = *opt;
  if (o.subrounds < 1 || o.subrounds > 256 || o.rating_max_net_size < 2 ||
      o.rating_max_net_size > (1 << 20) || o.contraction_limit_factor < 1 ||
      o.fingerprint_bits < 0 || o.fingerprint_bits > 64 || (!o.dev_alloc != !o.dev_free))
    return HG_ERR_INVALID;
  if (o.rate_warp_max_d < 0 || o.rate_warp_max_d > 256 || o.rate_pair_max_d < 0 ||
      o.rate_pair_max_d > 1024 || o.rate_quad_max_d < 0 || o.rate_quad_max_d > 2048 ||
      o.rate_block_max_d < 0 || o.rate_block_max_d > 4096 || o.lp_block_min_deg < 0 ||
      o.lp_block_min_deg > (1 << 20) || o.blocking_sync < 0 || o.blocking_sync > 1 ||
      o.graph_path < 0 || o.graph_path > 1 || o.community_detection < 0 ||
      o.community_detection > 1)
    return HG_ERR_INVALID;
  int64_t W = 0;
  int64_t p = 0;
  if (mem == HG_MEM_HOST) {
    p = net_offsets[m];
    if (p > 0 && !pins) return HG_ERR_INVALID;
    if (p < 0 || p >= (1ll << 31) || net_offsets[0] != 0) return HG_ERR_INVALID;
    // small inputs are checked here in full; mid-sized ones here for their
    // offsets and weights and on the device for their pins (ranges and
    // repeats inside a net); large ones entirely on the device right after
    // the upload, where the checks of millions of entries cost less than on
    // the caller's thread (many concurrent callers of mid-sized inputs keep
    // their O(m + n) host checks, which run in parallel on their threads)
    if (p <= HOST_CSR_CHECK_MAX) {
      const int rc = check_host_csr(n, m, net_offsets, p <= HOST_PIN_CHECK_MAX ? pins : nullptr,
                                    net_weights, node_weights, &W);
      if (rc != HG_OK) return rc;
    }
  }
  auto h = std::make_unique<hg_t>();
  h->opt = o;
  const int rc = guarded(nullptr, [&]() -> int {
    HG_CUDA(cudaGetDevice(&h->device));
    int sms = 0;
    HG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->cx.num_sms = sms;
    h->cx.stream = static_cast<cudaStream_t>(cuda_stream);
    if (o.blocking_sync)
      HG_CUDA(cudaEventCreateWithFlags(&h->cx.sync_event,
                                       cudaEventBlockingSync | cudaEventDisableTiming));
    h->cx.alloc.fn_alloc = o.dev_alloc;
    h->cx.alloc.fn_free = o.dev_free;
    h->cx.alloc.ctx = o.alloc_ctx;
    h->cx.alloc.stream = h->cx.stream;
    h->cx.launches = &h->launches;
    if (!o.dev_alloc) h->cx.alloc.pool = hgk::library_pool(h->device);
    h->cx.d_status = static_cast<int32_t*>(h->cx.alloc.get(sizeof(int32_t) * 4));
    HG_CUDA(cudaMemsetAsync(h->cx.d_status, 0, sizeof(int32_t) * 4, h->cx.stream));
    if (mem == HG_MEM_DEVICE) {
      int32_t ends[2] = {0, 0};
      HG_CUDA(cudaMemcpyAsync(&ends[0], net_offsets, sizeof(int32_t), cudaMemcpyDeviceToHost,
                              h->cx.stream));
      HG_CUDA(cudaMemcpyAsync(&ends[1], net_offsets + m, sizeof(int32_t), cudaMemcpyDeviceToHost,
                              h->cx.stream));
      HG_CUDA(cudaStreamSynchronize(h->cx.stream));
      if (ends[0] != 0 || ends[1] < 0) throw HgError(HG_ERR_INVALID, "bad offsets");
      p = ends[1];
      if (p > 0 && !pins) throw HgError(HG_ERR_INVALID, "pins missing");
    }
    auto L = std::make_unique<Level>();
    L->n = n;
    L->m = m;
    L->p = p;
    upload(h->cx, L->eoff, net_offsets, (size_t)m + 1, mem, 0);
    upload(h->cx, L->pins, pins, (size_t)p, mem, 0);
    upload(h->cx, L->w, net_weights, (size_t)m, mem, 1);
    upload(h->cx, L->c, node_weights, (size_t)n, mem, 1);
    if (mem == HG_MEM_HOST && p <= HOST_PIN_CHECK_MAX) {
      // checked on the host above
    } else if (mem == HG_MEM_HOST && p <= HOST_CSR_CHECK_MAX) {
      if (!hgk::validate_pins_device(h->cx, *L))
        throw HgError(HG_ERR_INVALID, "pins failed validation");
    } else {
      int64_t wn = 0, ww = 0;
      if (!hgk::validate_level_device(h->cx, *L, &wn, &ww))
        throw HgError(HG_ERR_INVALID, "device input failed validation");
      if (wn >= (1ll << 31) || ww >= (1ll << 31))
        throw HgError(HG_ERR_INVALID, "total weight too large");
      W = wn;
    }
    h->W0 = W;
    {
      hgk::EventTimer tm(h->cx, &h->stats.ms_transpose);
      hgk::build_incidence(h->cx, *L);
      if (o.graph_path == 0 && hgk::level_is_graph(h->cx, *L)) hgk::build_graph_adjacency(h->cx, *L);
    }
    hgk::check_status(h->cx);
    h->levels.push_back(std::move(L));
    return HG_OK;
  });
  if (rc != HG_OK) {
    hg_destroy(h.release());
    return rc;
  }
  *out = h.release();
  return HG_OK;
}

int hg_num_levels(const hg_t* h, int32_t* out_levels) {
  if (!h || !out_levels) return HG_ERR_INVALID;
  *out_levels = (int32_t)h->levels.size();
  return HG_OK;
}

int hg_level_is_graph(const hg_t* h, int32_t level, int32_t* out_graph) {
  if (!h || !out_graph) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  *out_graph = h->levels[level]->graph ? 1 : 0;
  return HG_OK;
}

int hg_level_info(const hg_t* h, int32_t level, int32_t* out_n, int32_t* out_m, int64_t* out_p) {
  if (!h) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  const Level& L = *h->levels[level];
  if (out_n) *out_n = L.n;
  if (out_m) *out_m = L.m;
  if (out_p) *out_p = L.p;
  return HG_OK;
}

int hg_coarsen_level(hg_t* h, int32_t k, int32_t* out_level, int32_t* out_n, int32_t* out_m,
                     int64_t* out_p) {
  if (!h) return HG_ERR_INVALID;
  if (k < 1 || k > HG_MAX_K) return HG_ERR_INVALID;
  return guarded(h, [&]() -> int {
    Level& L = *h->levels.back();
    const int64_t limit = (int64_t)h->opt.contraction_limit_factor * k;
    if (h->finished || (int64_t)L.n <= limit) return HG_STOP;
    const int level = (int)h->levels.size() - 1;
    hgk::CoarsenParams P;
    P.seed = h->opt.seed;
    P.level = level;
    P.S = h->opt.subrounds;
    P.T = h->opt.rating_max_net_size;
    P.c_max = (int32_t)((h->W0 + limit - 1) / limit);
    P.cuts.warp = h->opt.rate_warp_max_d ? h->opt.rate_warp_max_d : 256;
    P.cuts.pair = h->opt.rate_pair_max_d ? h->opt.rate_pair_max_d : 1024;
    P.cuts.quad = h->opt.rate_quad_max_d ? h->opt.rate_quad_max_d : 2048;
    P.cuts.block = h->opt.rate_block_max_d ? h->opt.rate_block_max_d : 4096;
    hgk::CoarsenCounters cc;
    DBuf<int32_t> cw;
    hgk::cluster_level(h->cx, L, P, cc, cw);
    auto out = std::make_unique<Level>();
    hgk::ContractCounters kc;
    hgk::contract_level(h->cx, L, cw.p, *out, h->opt.fingerprint_bits, kc);
    hgk::check_status(h->cx);
    h->stats.ms_rating += cc.ms_rating;
    h->stats.ms_approve += cc.ms_approve;
    h->stats.ms_rating_refresh += cc.ms_refresh;
    for (int c = 0; c < 8; ++c) {
      h->stats.ms_rating_class[c] += cc.class_ms[c];
      h->stats.rating_visits_class[c] += cc.class_visits[c];
    }
    h->stats.ms_rating_kernels += cc.ms_rating_kernels;
    h->stats.rating_launches += cc.rating_launches;
    h->stats.rating_pin_visits += cc.rating_pin_visits;
    h->stats.rating_nodes += cc.rating_nodes;
    h->stats.rating_incidences += cc.rating_incidences;
    h->stats.ms_contract += kc.ms;
    if (100 * (int64_t)out->n > 99 * (int64_t)L.n) h->finished = true;
    if (out_level) *out_level = level + 1;
    if (out_n) *out_n = out->n;
    if (out_m) *out_m = out->m;
    if (out_p) *out_p = out->p;
    h->levels.push_back(std::move(out));
    sync_stats(h);
    return HG_OK;
  });
}

int hg_initial_partition(hg_t* h, int32_t level, int32_t k, int32_t* part) {
  if (!h || !part) return HG_ERR_INVALID;
  if (k < 1 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::EventTimer tm(h->cx, &h->stats.ms_initial);
    const Level& L = *h->levels[level];
    std::vector<int32_t> c((size_t)L.n), out((size_t)L.n);
    HG_CUDA(cudaMemcpyAsync(c.data(), L.c.p, sizeof(int32_t) * (size_t)L.n,
                            cudaMemcpyDeviceToHost, h->cx.stream));
    HG_CUDA(cudaStreamSynchronize(h->cx.stream));
    // order of (mix64(seed ^ 2^63 ^ u), u); each node to the lightest block
    std::vector<std::pair<uint64_t, int32_t>> order((size_t)L.n);
    for (int32_t u = 0; u < L.n; ++u)
      order[u] = {hgk::mix64(h->opt.seed ^ (1ull << 63) ^ (uint64_t)(uint32_t)u), u};
    std::sort(order.begin(), order.end());
    std::vector<int64_t> bw((size_t)k, 0);
    for (const auto& kv : order) {
      int best = 0;
      for (int b = 1; b < k; ++b)
        if (bw[b] < bw[best]) best = b;
      out[kv.second] = best;
      bw[best] += c[kv.second];
    }
    HG_CUDA(cudaMemcpyAsync(part, out.data(), sizeof(int32_t) * (size_t)L.n,
                            cudaMemcpyHostToDevice, h->cx.stream));
    HG_CUDA(cudaStreamSynchronize(h->cx.stream));
    return HG_OK;
  });
}

int hg_project(hg_t* h, int32_t coarse_level, const int32_t* coarse_part, int32_t* fine_part) {
  if (!h || !coarse_part || !fine_part) return HG_ERR_INVALID;
  if (coarse_level < 1 || !valid_level(h, coarse_level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::EventTimer tm(h->cx, &h->stats.ms_project);
    const Level& F = *h->levels[coarse_level - 1];
    if (!F.coarsened) return HG_ERR_STATE;
    hgk::project_partition(h->cx, F, coarse_part, fine_part);
    sync_stats(h);
    return HG_OK;
  });
}

int hg_lp_refine(hg_t* h, int32_t level, int32_t k, int32_t eps_ppm, int32_t max_passes,
                 int32_t* part, int64_t* out_objective, int64_t* out_moves) {
  if (!h || !part) return HG_ERR_INVALID;
  if (k < 2 || k > HG_MAX_K || eps_ppm < 0 || max_passes < 0) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::RefineCounters rc;
    const Level& L = *h->levels[level];
    hgk::validate_partition(h->cx, part, L.n, k);
    hgk::LPResult r = hgk::lp_refine_level(h->cx, L, level, k, eps_ppm, max_passes,
                                           h->opt.subrounds, h->opt.seed, h->W0,
                                           h->opt.lp_block_min_deg ? h->opt.lp_block_min_deg : 64,
                                           part, rc);
    h->stats.ms_phi += rc.ms_phi;
    h->stats.ms_lp_gain += rc.ms_gain;
    h->stats.ms_lp_select += rc.ms_select;
    h->stats.ms_lp_apply += rc.ms_apply;
    h->stats.ms_objective += rc.ms_objective;
    h->stats.ms_lp_gain_kernels += rc.ms_gain_kernels;
    h->stats.ms_lp_select_kernels += rc.ms_select_kernels;
    h->stats.ms_lp_apply_kernels += rc.ms_apply_kernels;
    h->stats.lp_moved_incidences += rc.lp_moved_incidences;
    h->stats.lp_passes += rc.lp_passes;
    h->stats.timing_failures += rc.timing_failures;
    h->stats.lp_incidences += rc.lp_incidences;
    h->stats.lp_nodes += rc.lp_nodes;
    h->stats.lp_gain_launches += rc.lp_gain_launches;
    if (out_objective) *out_objective = r.objective;
    if (out_moves) *out_moves = r.moves;
    sync_stats(h);
    return HG_OK;
  });
}

int hg_objective(hg_t* h, int32_t level, int32_t k, const int32_t* part, int64_t* out) {
  if (!h || !part || !out) return HG_ERR_INVALID;
  if (k < 1 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::validate_partition(h->cx, part, h->levels[level]->n, k);
    hgk::EventTimer tm(h->cx, &h->stats.ms_objective);
    *out = hgk::objective_of(h->cx, *h->levels[level], k, part);
    sync_stats(h);
    return HG_OK;
  });
}

int hg_recalculate_gains(hg_t* h, int32_t level, int32_t k, const int32_t* part,
                         int32_t num_moves, const int32_t* move_nodes,
                         const int32_t* move_targets, int64_t* gains) {
  if (!h || !part || num_moves < 0) return HG_ERR_INVALID;
  if (k < 2 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (num_moves > 0 && (!move_nodes || !move_targets || !gains)) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  if (num_moves > h->levels[level]->n) return HG_ERR_INVALID;  // a node would move twice
  return guarded(h, [&]() -> int {
    hgk::recalculate_gains(h->cx, *h->levels[level], k, part, num_moves, move_nodes, move_targets,
                           gains);
    sync_stats(h);
    return HG_OK;
  });
}

int hg_gain_table(hg_t* h, int32_t level, int32_t k, const int32_t* part, int64_t* benefit,
                  int64_t* penalty) {
  if (!h || !part || !benefit || !penalty) return HG_ERR_INVALID;
  if (k < 2 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::gain_table_build(h->cx, *h->levels[level], k, part, benefit, penalty);
    sync_stats(h);
    return HG_OK;
  });
}

int hg_gain_table_move(hg_t* h, int32_t level, int32_t k, int32_t* part, int32_t num_moves,
                       const int32_t* move_nodes, const int32_t* move_targets, int64_t* benefit,
                       int64_t* penalty) {
  if (!h || !part || !benefit || !penalty || num_moves < 0) return HG_ERR_INVALID;
  if (k < 2 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (num_moves > 0 && (!move_nodes || !move_targets)) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  if (num_moves > h->levels[level]->n) return HG_ERR_INVALID;
  return guarded(h, [&]() -> int {
    hgk::gain_table_move(h->cx, *h->levels[level], k, part, num_moves, move_nodes, move_targets,
                         benefit, penalty);
    sync_stats(h);
    return HG_OK;
  });
}

int hg_pin_counts(hg_t* h, int32_t level, int32_t k, const int32_t* part, int32_t* phi,
                  uint64_t* lambda, int64_t* block_weights) {
  if (!h || !part) return HG_ERR_INVALID;
  if (k < 1 || k > HG_MAX_K) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    hgk::validate_partition(h->cx, part, h->levels[level]->n, k);
    hgk::pin_counts_of(h->cx, *h->levels[level], k, part, phi, lambda, block_weights);
    return HG_OK;
  });
}

int hg_detect_communities(hg_t* h, int32_t* out_communities) {
  if (!h) return HG_ERR_INVALID;
  if (h->levels.size() != 1) return HG_ERR_STATE;  // before any coarsening
  return guarded(h, [&]() -> int {
    hgk::EventTimer tm(h->cx, &h->stats.ms_communities);
    Level& L = *h->levels[0];
    hgk::LouvainCounters lc;
    DBuf<int32_t> comm;
    const int32_t count =
        hgk::detect_communities(h->cx, L, h->opt.subrounds, h->opt.seed, comm, lc);
    L.comm = std::move(comm);
    h->stats.louvain_levels += lc.levels;
    h->stats.louvain_rounds += lc.rounds;
    h->stats.louvain_moves += lc.moves;
    h->launches += lc.launches;
    if (out_communities) *out_communities = count;
    sync_stats(h);
    return HG_OK;
  });
}

int hg_get_communities(const hg_t* hc, int32_t level, int32_t* comm) {
  hg_t* h = const_cast<hg_t*>(hc);
  if (!h || !comm) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  const Level& L = *h->levels[level];
  if (!L.comm.p) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    HG_CUDA(cudaMemcpyAsync(comm, L.comm.p, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost,
                            h->cx.stream));
    HG_CUDA(cudaStreamSynchronize(h->cx.stream));
    return HG_OK;
  });
}

int hg_partition(hg_t* h, int32_t k, int32_t eps_ppm, int32_t max_passes, int32_t* part,
                 int64_t* out_objective) {
  if (!h || !part) return HG_ERR_INVALID;
  if (k < 2 || k > HG_MAX_K || eps_ppm < 0 || max_passes < 0) return HG_ERR_INVALID;
  if (h->sticky) return h->sticky;
  int rc;
  if (h->opt.community_detection && h->levels.size() == 1 && !h->levels[0]->comm.p) {
    rc = hg_detect_communities(h, nullptr);
    if (rc != HG_OK) return rc;
  }
  while ((rc = hg_coarsen_level(h, k, nullptr, nullptr, nullptr, nullptr)) == HG_OK) {
  }
  if (rc != HG_STOP) return rc;
  return guarded(h, [&]() -> int {
    const int top = (int)h->levels.size() - 1;
    std::vector<DBuf<int32_t>> parts(h->levels.size());
    for (int l = 1; l <= top; ++l) parts[l].alloc(&h->cx.alloc, (size_t)h->levels[l]->n);
    int32_t* cur = top == 0 ? part : parts[top].p;
    int r = hg_initial_partition(h, top, k, cur);
    if (r != HG_OK) return r;
    int64_t obj = 0;
    for (int l = top; l >= 0; --l) {
      int32_t* dst = l == 0 ? part : parts[l].p;
      if (l < top) {
        r = hg_project(h, l + 1, parts[l + 1].p, dst);
        if (r != HG_OK) return r;
      }
      r = hg_lp_refine(h, l, k, eps_ppm, max_passes, dst, &obj, nullptr);
      if (r != HG_OK) return r;
    }
    if (out_objective) *out_objective = obj;
    return HG_OK;
  });
}

int hg_get_level(const hg_t* hc, int32_t level, int32_t* offsets, int32_t* pins,
                 int32_t* net_weights, int32_t* node_weights, int32_t* map, int32_t* rep) {
  hg_t* h = const_cast<hg_t*>(hc);
  if (!h) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  const Level& L = *h->levels[level];
  if ((map || rep) && !L.coarsened) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    auto cp = [&](int32_t* dst, const int32_t* src, size_t cnt) {
      if (dst && cnt)
        HG_CUDA(cudaMemcpyAsync(dst, src, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                h->cx.stream));
    };
    cp(offsets, L.eoff.p, (size_t)L.m + 1);
    cp(pins, L.pins.p, (size_t)L.p);
    cp(net_weights, L.w.p, (size_t)L.m);
    cp(node_weights, L.c.p, (size_t)L.n);
    cp(map, L.map.p, (size_t)L.n);
    cp(rep, L.rep.p, (size_t)L.n);
    HG_CUDA(cudaStreamSynchronize(h->cx.stream));
    return HG_OK;
  });
}

int hg_get_incidence(const hg_t* hc, int32_t level, int32_t* offsets, int32_t* nets) {
  hg_t* h = const_cast<hg_t*>(hc);
  if (!h) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  const Level& L = *h->levels[level];
  return guarded(h, [&]() -> int {
    if (offsets)
      HG_CUDA(cudaMemcpyAsync(offsets, L.ioff.p, sizeof(int32_t) * ((size_t)L.n + 1),
                              cudaMemcpyDeviceToHost, h->cx.stream));
    if (nets && L.p)
      HG_CUDA(cudaMemcpyAsync(nets, L.inets.p, sizeof(int32_t) * (size_t)L.p,
                              cudaMemcpyDeviceToHost, h->cx.stream));
    HG_CUDA(cudaStreamSynchronize(h->cx.stream));
    return HG_OK;
  });
}

int hg_truncate(hg_t* h, int32_t level) {
  if (!h) return HG_ERR_INVALID;
  if (!valid_level(h, level)) return HG_ERR_STATE;
  return guarded(h, [&]() -> int {
    while ((int32_t)h->levels.size() > level + 1) h->levels.pop_back();
    Level& L = *h->levels.back();
    L.map.release();
    L.rep.release();
    L.coarsened = false;
    h->finished = false;
    return HG_OK;
  });
}

int hg_enable_timing(hg_t* h, int32_t on) {
  if (!h) return HG_ERR_INVALID;
  h->cx.timing = (on & 1) != 0;
  h->cx.kernel_timing = (on & 2) != 0;
  return HG_OK;
}

int hg_get_stats(hg_t* h, hg_stats* out) {
  if (!h || !out) return HG_ERR_INVALID;
  sync_stats(h);
  *out = h->stats;
  return HG_OK;
}

int hg_reset_stats(hg_t* h) {
  if (!h) return HG_ERR_INVALID;
  h->stats = hg_stats{};
  h->launches = 0;
  return HG_OK;
}

int hg_trim_memory(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HG_ERR_CUDA;
  }
  try {
    if (cudaMemPoolTrimTo(hgk::library_pool(dev), 0) != cudaSuccess) {
      cudaGetLastError();
      return HG_ERR_CUDA;
    }
  } catch (const HgError& e) {
    return e.code;
  }
  return HG_OK;
}

int hg_destroy(hg_t* h) {
  if (!h) return HG_OK;
  cudaSetDevice(h->device);
  h->levels.clear();
  if (h->cx.d_status) h->cx.alloc.put(h->cx.d_status);
  h->cx.d_status = nullptr;
  cudaStreamSynchronize(h->cx.stream);
  if (h->cx.sync_event) cudaEventDestroy(h->cx.sync_event);
  delete h;
  return HG_OK;
}

}  // extern "C"
