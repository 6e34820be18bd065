// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/hg.h"

namespace hgk {

// ------------------------------------------------------------------ errors

// Thrown inside the library and turned into a status code at the ABI.
struct HgError : std::runtime_error {
  int code;
  HgError(int c, const std::string& what) : std::runtime_error(what), code(c) {}
};

#define HG_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) {                                                            \
      if (_e == cudaErrorMemoryAllocation)                                              \
        throw ::hgk::HgError(HG_ERR_OOM, std::string(#call) + ": " + cudaGetErrorString(_e)); \
      throw ::hgk::HgError(HG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));  \
    }                                                                                   \
  } while (0)

// Device-side error codes, written into Ctx::d_status[0] by kernels that hit
// a bounded wait or a capacity limit; read back at the next host sync.
enum DevStatus : int32_t {
  DEV_OK = 0,
  DEV_HASH_FULL = 1,      // a hash table ran out of slots
  DEV_TIMEOUT = 2,        // a bounded spin gave up
  DEV_BAD_INPUT = 3,      // device-side input validation failed
  DEV_CAPACITY = 4,       // a work list exceeded its capacity
};

// Forces a device lambda to be inlined at its call sites (hot loops pass
// lambdas through several template layers).
#define HG_INLINE __attribute__((always_inline))

__device__ __forceinline__ void dev_fail(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

// Signed 64-bit atomic add (two's complement wrap-around of the unsigned op).
__device__ __forceinline__ void atomic_add_i64(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// ---------------------------------------------------------------- hashing

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): the first
// output of a SplitMix64 generator whose state is x.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Sub-round of node u in clustering round `level` (Sec. 11: nodes are split
// into sub-rounds by a hash of the seed, the level and the node id).
__host__ __device__ __forceinline__ int subround_of_node_cluster(uint64_t seed, int level, int u,
                                                                 int S) {
  const uint64_t x = seed ^ ((uint64_t)(uint32_t)level << 32) ^ (uint64_t)(uint32_t)u;
  return (int)(mix64(x) % (uint64_t)S);
}

// Sub-round of node u in label-propagation pass `pass` of level `level`.
__host__ __device__ __forceinline__ int subround_of_node_lp(uint64_t seed, int level, int pass,
                                                            int u, int S) {
  const uint64_t x = seed ^ ((uint64_t)(uint32_t)level << 32) ^
                     ((uint64_t)(uint32_t)(pass + 1) << 48) ^ (uint64_t)(uint32_t)u;
  return (int)(mix64(x) % (uint64_t)S);
}

// ------------------------------------------------------------- warp utils

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_in_block() { return threadIdx.x >> 5; }

// Claims one slot from counter[key] for every lane of `active` (a ballot
// taken in converged code) with key >= 0: lanes with equal keys share one
// atomicAdd and take consecutive slots in lane order.  Returns the lane's
// slot, or -1 for a lane outside `active` or with key < 0.
__device__ __forceinline__ int32_t warp_claim_slot(int32_t* counter, int key, unsigned active) {
  const int lane = threadIdx.x & 31;
  const bool mine = ((active >> lane) & 1u) && key >= 0;
  const unsigned want = __ballot_sync(0xffffffffu, mine);
  const unsigned peers = __match_any_sync(0xffffffffu, mine ? key : -1 - lane) & want;
  int32_t slot = -1;
  if (mine) {
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(&counter[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    slot = base + rank;
  }
  return slot;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(FULL, x, d);
    if (lane_id() >= d) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
  return x;
}

// Adds every thread's v[i] to the global counter dst[i] with one atomic per
// block and counter (a counter hit by an atomic from every warp of a large
// grid serialises those atomics in one L2 slice).  All threads of the block
// must call it; it synchronises the block.
template <int N>
__device__ __forceinline__ void block_add_counters(unsigned long long* dst,
                                                   const unsigned long long (&v)[N]) {
  __shared__ unsigned long long s_sum[N];
  if (threadIdx.x < N) s_sum[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const unsigned long long w = warp_sum(v[i]);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_sum[i], w);
  }
  __syncthreads();
  if (threadIdx.x < N && s_sum[threadIdx.x]) atomicAdd(&dst[threadIdx.x], s_sum[threadIdx.x]);
}

template <typename T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T y = __shfl_xor_sync(FULL, x, d);
    x = y > x ? y : x;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_min(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T y = __shfl_xor_sync(FULL, x, d);
    x = y < x ? y : x;
  }
  return x;
}

// Block-wide sum for blockDim.x <= 1024 (all threads must call).
template <typename T>
__device__ __forceinline__ T block_sum(T x, T* smem32) {
  x = warp_sum(x);
  __syncthreads();
  if (lane_id() == 0) smem32[warp_in_block()] = x;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? smem32[threadIdx.x] : T(0);
  if (warp_in_block() == 0) r = warp_sum(r);
  if (threadIdx.x == 0) smem32[0] = r;
  __syncthreads();
  r = smem32[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------- memory

// A device allocation tied to the handle's allocator.
struct Alloc {
  void* (*fn_alloc)(size_t, void*) = nullptr;
  void (*fn_free)(void*, void*) = nullptr;
  void* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;  // library_pool(device) when no hook is given
  void* get(size_t bytes) const;
  void put(void* p) const;
};

// The library's private stream-ordered memory pool of a device (prim.cu).
cudaMemPool_t library_pool(int device);

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  const Alloc* a = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; a = o.a;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(const Alloc* al, size_t count) {
    release();
    a = al;
    n = count;
    p = count ? static_cast<T*>(al->get(count * sizeof(T))) : nullptr;
  }
  void release() {
    if (p && a) a->put(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------- context

struct Ctx {
  Alloc alloc;
  cudaStream_t stream = nullptr;
  int32_t* d_status = nullptr;   // device status word (DevStatus)
  int num_sms = 0;
  int64_t* launches = nullptr;   // host counter
  bool timing = false;           // per-phase event timing (synchronizes at phase ends)
  bool kernel_timing = false;    // event pair around every rating / gain launch (no sync)
  cudaEvent_t sync_event = nullptr;  // blocking-sync event: waits sleep instead of spinning
};

// Grid size helper: enough blocks for `work` items of `per_block` each,
// capped at `cap_per_sm` resident blocks per SM.
inline int grid_for(int64_t work, int per_block, int num_sms, int cap_per_sm = 32) {
  int64_t b = (work + per_block - 1) / per_block;
  int64_t cap = (int64_t)num_sms * cap_per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw HgError(HG_ERR_CUDA, std::string("launch ") + what + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------- levels

// One hypergraph level resident in device memory.
struct Level {
  int32_t n = 0, m = 0;
  int64_t p = 0;
  DBuf<int32_t> eoff;   // m+1  net -> first pin
  DBuf<int32_t> pins;   // p    pin lists, ascending inside a net for coarse levels
  DBuf<int32_t> w;      // m    net weights
  DBuf<int32_t> c;      // n    node weights
  DBuf<int32_t> ioff;   // n+1  node -> first incident net
  DBuf<int32_t> inets;  // p    incident nets (order unspecified)
  DBuf<int32_t> ipin;   // p    for every incidence, the index of its pin in `pins`
  DBuf<int32_t> map;    // n    node -> node of the next level (after coarsening)
  DBuf<int32_t> rep;    // n    representative in the clustering that made the next level
  bool coarsened = false;
  // Graph levels (every net has exactly two pins, Sec. 10): the one
  // adjacency array adj[j] = {other endpoint, w(e)} of incidence j = (u, e),
  // aligned with inets.  The coarse level of a graph level is a graph level.
  bool graph = false;
  DBuf<int2> adj;       // p (graph levels only)
  // community of every node (Sec. 4, community-aware coarsening), when
  // detected: contractions stay inside a community
  DBuf<int32_t> comm;   // n (or empty)
};

// --------------------------------------------------------- primitives (prim.cu)

// Exclusive prefix sum of n int32 values into out (n entries); writes the
// total into *d_total (device) if non-null.  in and out may alias.
void scan_exclusive_i32(const Ctx& cx, const int32_t* in, int32_t* out, int64_t n,
                        int32_t* d_total);
// Same with int64 output.
void scan_exclusive_i32_to_i64(const Ctx& cx, const int32_t* in, int64_t* out, int64_t n,
                               int64_t* d_total);

// Copies a device scalar to the host (synchronizes the stream) and checks
// the device status word.
int32_t read_i32(const Ctx& cx, const int32_t* d);
int64_t read_i64(const Ctx& cx, const int64_t* d);
void check_status(const Ctx& cx);

void fill_i32(const Ctx& cx, int32_t* p, int32_t value, int64_t n);
// Waits until the stream's work is done: spinning, or sleeping on the
// handle's blocking-sync event when it has one.  A following copy to pageable
// host memory then finds the stream idle.
void wait_stream(const Ctx& cx);
void iota_i32(const Ctx& cx, int32_t* p, int64_t n);

// ---------------------------------------------------- structure (structure.cu)

// Builds ioff/inets of a level from eoff/pins (a1).
void build_incidence(const Ctx& cx, Level& L);
// True when the level has nets and every net has exactly two pins.
bool level_is_graph(const Ctx& cx, const Level& L);
// Sets L.graph and builds L.adj (after build_incidence).
void build_graph_adjacency(const Ctx& cx, Level& L);
// The pins alone (in range, no node twice in a net) of a level whose offsets
// are valid: mid-sized host inputs, whose offsets and weights the host checks.
bool validate_pins_device(const Ctx& cx, const Level& L);

// Device-side validation of a level given by device pointers: offsets
// monotone, pins in range, no net empty, no repeated pin in a net, weights
// positive.  Returns false if invalid.
bool validate_level_device(const Ctx& cx, const Level& L, int64_t* total_node_w,
                           int64_t* total_net_w);

// ------------------------------------------------------ coarsening (coarsen.cu)

// Upper bounds on D = min(W(u), n) of the rating team classes (launch
// mapping only; the tables hold 2 D slots).
struct RateCuts {
  int32_t warp, pair, quad, block;
};

struct CoarsenParams {
  uint64_t seed;
  int level;      // index of the level being clustered
  int S;          // sub-rounds
  int T;          // rating net-size threshold
  int32_t c_max;  // cluster weight cap
  RateCuts cuts;
};

struct CoarsenCounters {
  int64_t rating_launches = 0, rating_pin_visits = 0, rating_nodes = 0, rating_incidences = 0;
  double ms_rating = 0, ms_approve = 0, ms_refresh = 0, ms_rating_kernels = 0;
  double class_ms[8] = {0};        // rating kernel time per node class (kernel timing on)
  int64_t class_visits[8] = {0};   // pin visits per node class
};

// Deterministic clustering of level L: fills L.rep (representatives) and
// cw (cluster weight, valid at representatives).
void cluster_level(const Ctx& cx, Level& L, const CoarsenParams& P, CoarsenCounters& cc,
                   DBuf<int32_t>& cw);

struct ContractCounters {
  double ms = 0;
  int ident_rounds = 0;
};

// Contraction of L's clustering into a new level (a5-a8); fills L.map.
void contract_level(const Ctx& cx, Level& L, const int32_t* cw, Level& out, int fingerprint_bits,
                    ContractCounters& kc);

// ----------------------------------------------- communities (community.cu)

struct LouvainCounters {
  int64_t levels = 0, rounds = 0, moves = 0, launches = 0;
};

// Deterministic Louvain community detection on the bipartite graph of L
// (Sec. 4, Sec. 11): comm receives the community of every node; returns the
// number of distinct communities.
int32_t detect_communities(const Ctx& cx, const Level& L, int S, uint64_t seed,
                           DBuf<int32_t>& comm, LouvainCounters& lc);

// ------------------------------------------------------- refinement (refine.cu)

struct RefineCounters {
  int64_t lp_incidences = 0, lp_nodes = 0, lp_gain_launches = 0, lp_moved_incidences = 0,
          lp_passes = 0, timing_failures = 0;
  double ms_phi = 0, ms_gain = 0, ms_select = 0, ms_apply = 0, ms_objective = 0,
         ms_gain_kernels = 0, ms_select_kernels = 0, ms_apply_kernels = 0;
};

void project_partition(const Ctx& cx, const Level& fine, const int32_t* coarse_part,
                       int32_t* fine_part);

int64_t objective_of(const Ctx& cx, const Level& L, int k, const int32_t* part);

void pin_counts_of(const Ctx& cx, const Level& L, int k, const int32_t* part, int32_t* phi,
                   uint64_t* lambda, int64_t* bw);
// Throws HG_ERR_INVALID unless every block id of a caller's partition is in
// [0, k) (a block id indexes Phi).
void validate_partition(const Ctx& cx, const int32_t* part, int32_t n, int k);
// Phi (m x k) and Lambda of a partition, left on the device.
void device_pin_counts(const Ctx& cx, const Level& L, int k, const int32_t* part,
                       DBuf<int32_t>& phi, DBuf<unsigned long long>& lam);
void gain_table_build(const Ctx& cx, const Level& L, int k, const int32_t* part, int64_t* b,
                      int64_t* p);
void gain_table_move(const Ctx& cx, const Level& L, int k, int32_t* part, int32_t l,
                     const int32_t* nodes, const int32_t* targets, int64_t* b, int64_t* p);

struct LPResult {
  int64_t objective = 0;
  int64_t moves = 0;
  int passes = 0;
};

void recalculate_gains(const Ctx& cx, const Level& L, int k, const int32_t* part, int32_t l,
                       const int32_t* nodes, const int32_t* targets, int64_t* gains);

LPResult lp_refine_level(const Ctx& cx, const Level& L, int level_index, int k, int eps_ppm,
                         int max_passes, int S, uint64_t seed, int64_t total_node_weight,
                         int lp_block_deg, int32_t* part, RefineCounters& rc);

// ---------------------------------------------------------------- timing

// Records an event pair around a region on the stream when timing is on.
struct EventTimer {
  const Ctx* cx;
  cudaEvent_t a = nullptr, b = nullptr;
  double* acc;
  explicit EventTimer(const Ctx& c, double* accumulate) : cx(&c), acc(accumulate) {
    if (cx->timing && acc) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, cx->stream);
    }
  }
  void stop() {
    if (a) {
      cudaEventRecord(b, cx->stream);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      *acc += ms;
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      a = b = nullptr;
    }
  }
  ~EventTimer() { stop(); }
};

// Accumulates the summed duration of a set of kernel launches (each launch
// bracketed by its own event pair) when timing is on; resolved by flush().
struct KernelTimer {
  const Ctx* cx;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  explicit KernelTimer(const Ctx& c) : cx(&c) {}
  void begin() {
    if (!cx->kernel_timing) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, cx->stream);
    ev.push_back({a, b});
  }
  void end() {
    if (!cx->kernel_timing || ev.empty()) return;
    cudaEventRecord(ev.back().second, cx->stream);
  }
  double flush() {
    double total = 0;
    for (auto& p : ev) {
      cudaEventSynchronize(p.second);
      float ms = 0;
      cudaEventElapsedTime(&ms, p.first, p.second);
      total += ms;
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    ev.clear();
    return total;
  }
  ~KernelTimer() { flush(); }
};

}  // namespace hgk
