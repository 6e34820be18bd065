// Hypergraph structure on the device: the pin-tile index, the incident-net
// lists I(u) (the second adjacency array of Sec. 4.2, "The Contraction
// Algorithm"), the single adjacency array of graph levels (Sec. 10, "Graph
// Data Structure"), and validation of caller-provided device arrays.
#include "common.cuh"
#include "pintile.cuh"

namespace hgk {

namespace {

// tile_net[t] = net containing pin position t * PIN_TILE.
__global__ void k_tile_index(const int32_t* __restrict__ eoff, int32_t m, int64_t ntiles,
                             int32_t* __restrict__ tile_net) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = eoff[e], b = eoff[e + 1];
    if (b <= a) continue;
    for (int64_t t = (a + PIN_TILE - 1) / PIN_TILE; t * PIN_TILE < b && t < ntiles; ++t)
      tile_net[t] = (int32_t)e;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_net[ntiles] = m > 0 ? m - 1 : 0;
}

__global__ void k_degrees(const int32_t* __restrict__ pins, int64_t p, int32_t* __restrict__ deg) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p;
       q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[pins[q]], 1);
}

// Scatter every pin (e, v) into I(v) at a slot taken from v's cursor; the
// slot also records the pin's index q in `pins`.
__global__ void __launch_bounds__(PIN_TILE_THREADS)
k_scatter_incidence(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                    const int32_t* __restrict__ tile_net, int32_t m, int64_t p,
                    int32_t* __restrict__ cursor, int32_t* __restrict__ inets,
                    int32_t* __restrict__ ipin) {
  __shared__ int32_t s_off[PIN_TILE + 3];
  const int64_t ntiles = num_pin_tiles(p);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    PinTileView v = stage_pin_tile(eoff, tile_net, m, p, t, s_off);
    for (int64_t q = v.q0 + threadIdx.x; q < v.q1; q += blockDim.x) {
      const int32_t e = v.e_lo + net_in_tile(s_off, v.count, q);
      const int32_t u = pins[q];
      const int32_t slot = atomicAdd(&cursor[u], 1);
      inets[slot] = e;
      ipin[slot] = (int32_t)q;
    }
    __syncthreads();
  }
}

__global__ void k_validate_nets(const int32_t* __restrict__ eoff, int32_t m,
                                const int32_t* __restrict__ w, int32_t* status,
                                unsigned long long* total_w) {
  int64_t local = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (eoff[e + 1] <= eoff[e]) dev_fail(status, DEV_BAD_INPUT);
    const int32_t x = w ? w[e] : 1;
    if (x <= 0) dev_fail(status, DEV_BAD_INPUT);
    local += x;
  }
  local = warp_sum(local);
  if (lane_id() == 0 && local) atomicAdd(total_w, (unsigned long long)local);
}

__global__ void k_validate_pins(const int32_t* __restrict__ pins, int64_t p, int32_t n,
                                int32_t* status) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = pins[q];
    if (v < 0 || v >= n) dev_fail(status, DEV_BAD_INPUT);
  }
}

__global__ void k_validate_nodes(const int32_t* __restrict__ c, int32_t n, int32_t* status,
                                 unsigned long long* total_c) {
  int64_t local = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = c ? c[u] : 1;
    if (x <= 0) dev_fail(status, DEV_BAD_INPUT);
    local += x;
  }
  local = warp_sum(local);
  if (lane_id() == 0 && local) atomicAdd(total_c, (unsigned long long)local);
}

// No node twice in a net.  One warp per net of at most DISTINCT_SMALL pins:
// nets of at most 32 pins compare lanes with a match; larger ones insert
// their pins into a per-warp hash set in shared memory (a pin found already
// present is a repeat).  Larger nets are left to k_distinct_big.  Runs only
// on offsets and pins already checked, so every read stays in bounds.
constexpr int DISTINCT_WARPS = 4;
constexpr int DISTINCT_SMALL = 1024;
// largest total of the per-block node bitmaps of k_distinct_big_bitmap
constexpr int64_t DISTINCT_BITMAP_BYTES = 256ll << 20;
constexpr int DISTINCT_SET = 2 * DISTINCT_SMALL;

__device__ __forceinline__ bool set_insert_new(int32_t* set, uint32_t mask, int32_t v) {
  uint32_t h = ((uint32_t)v * 0x9E3779B1u) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t old = atomicCAS(&set[h], -1, v);
    if (old == -1) return true;
    if (old == v) return false;
    h = (h + 1) & mask;
  }
  return false;  // full: cannot happen at load <= 1/2
}

// Removes v (probing past empty slots: other pins of the net are erased at
// the same time and leave holes in the probe chains).
__device__ __forceinline__ void set_erase(int32_t* set, uint32_t mask, int32_t v) {
  uint32_t h = ((uint32_t)v * 0x9E3779B1u) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (set[h] == v) {
      set[h] = -1;
      return;
    }
    h = (h + 1) & mask;
  }
}

__global__ void __launch_bounds__(DISTINCT_WARPS * 32)
k_distinct_small(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins, int32_t m,
                 int32_t* status) {
  __shared__ int32_t s_set[DISTINCT_WARPS][DISTINCT_SET];
  const int wv = warp_in_block(), lane = lane_id();
  int32_t* set = s_set[wv];
  for (int i = lane; i < DISTINCT_SET; i += 32) set[i] = -1;
  __syncwarp();
  for (int64_t e = (int64_t)blockIdx.x * DISTINCT_WARPS + wv; e < m;
       e += (int64_t)gridDim.x * DISTINCT_WARPS) {
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    if (sz > DISTINCT_SMALL) continue;
    bool dup = false;
    if (sz <= 32) {
      const int32_t v = lane < sz ? pins[b + lane] : -1 - lane;
      dup = __popc(__match_any_sync(FULL, v)) > 1;
    } else {
      for (int32_t q = lane; q < sz; q += 32) dup |= !set_insert_new(set, DISTINCT_SET - 1, pins[b + q]);
      __syncwarp();
      for (int32_t q = lane; q < sz; q += 32) set_erase(set, DISTINCT_SET - 1, pins[b + q]);
      __syncwarp();
    }
    if (__any_sync(FULL, dup) && lane == 0) dev_fail(status, DEV_BAD_INPUT);
  }
}

// Nets above DISTINCT_SMALL pins: one block per net with a hash set of `cap`
// slots (a power of two >= twice the largest net) in this block's region of
// `scratch` (all slots -1 on entry, restored before the block moves on).
__global__ void k_distinct_big(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                               int32_t m, int32_t* __restrict__ scratch, uint32_t cap,
                               int32_t* status) {
  int32_t* set = scratch + (size_t)blockIdx.x * cap;
  __shared__ int s_dup;
  for (int64_t e = blockIdx.x; e < m; e += gridDim.x) {
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    if (sz <= DISTINCT_SMALL) continue;
    if (threadIdx.x == 0) s_dup = 0;
    __syncthreads();
    bool dup = false;
    for (int32_t q = threadIdx.x; q < sz; q += blockDim.x) dup |= !set_insert_new(set, cap - 1, pins[b + q]);
    if (dup) s_dup = 1;
    __syncthreads();
    for (int32_t q = threadIdx.x; q < sz; q += blockDim.x) set_erase(set, cap - 1, pins[b + q]);
    if (threadIdx.x == 0 && s_dup) dev_fail(status, DEV_BAD_INPUT);
    __syncthreads();
  }
}

// The same check with a bitmap of the n nodes per block (n bits), when the
// bitmaps of all blocks are small: one atomicOr per pin finds a repeat and one
// atomicAnd per pin clears the net's bits again, with no probing.
__global__ void k_distinct_big_bitmap(const int32_t* __restrict__ eoff,
                                      const int32_t* __restrict__ pins, int32_t m,
                                      uint32_t* __restrict__ scratch, int64_t words,
                                      int32_t* status) {
  uint32_t* set = scratch + (size_t)blockIdx.x * (size_t)words;
  __shared__ int s_dup;
  for (int64_t e = blockIdx.x; e < m; e += gridDim.x) {
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    if (sz <= DISTINCT_SMALL) continue;
    if (threadIdx.x == 0) s_dup = 0;
    __syncthreads();
    bool dup = false;
    for (int32_t q = threadIdx.x; q < sz; q += blockDim.x) {
      const int32_t v = pins[b + q];
      const uint32_t bit = 1u << (v & 31);
      dup |= (atomicOr(&set[v >> 5], bit) & bit) != 0;
    }
    if (dup) s_dup = 1;
    __syncthreads();
    for (int32_t q = threadIdx.x; q < sz; q += blockDim.x) {
      const int32_t v = pins[b + q];
      atomicAnd(&set[v >> 5], ~(1u << (v & 31)));
    }
    if (threadIdx.x == 0 && s_dup) dev_fail(status, DEV_BAD_INPUT);
    __syncthreads();
  }
}

__global__ void k_max_net_size(const int32_t* __restrict__ eoff, int32_t m, int32_t* out) {
  int32_t mx = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, eoff[e + 1] - eoff[e]);
  mx = warp_max(mx);
  if (lane_id() == 0 && mx) atomicMax(out, mx);
}

__global__ void k_net_size_range(const int32_t* __restrict__ eoff, int32_t m,
                                 int32_t* __restrict__ out) {
  int32_t lo = 0x7fffffff, hi = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sz = eoff[e + 1] - eoff[e];
    lo = min(lo, sz);
    hi = max(hi, sz);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (lane_id() == 0) {
    atomicMin(&out[0], lo);
    atomicMax(&out[1], hi);
  }
}

// adj[j] = {the other pin of net inets[j], w(inets[j])} for every incidence
// of a graph level (ipin[j] is the incidence's own pin position).
__global__ void k_adjacency(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                            const int32_t* __restrict__ w, const int32_t* __restrict__ inets,
                            const int32_t* __restrict__ ipin, int64_t p, int2* __restrict__ adj) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = inets[j];
    const int32_t b = eoff[e];
    const int32_t other = ipin[j] == b ? b + 1 : b;
    adj[j] = make_int2(pins[other], w[e]);
  }
}

}  // namespace

bool level_is_graph(const Ctx& cx, const Level& L) {
  if (L.m <= 0) return false;
  DBuf<int32_t> range;
  range.alloc(&cx.alloc, 2);
  const int32_t init[2] = {0x7fffffff, 0};
  HG_CUDA(cudaMemcpyAsync(range.p, init, sizeof(init), cudaMemcpyHostToDevice, cx.stream));
  k_net_size_range<<<grid_for(L.m, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.eoff.p, L.m,
                                                                            range.p);
  check_launch("net_size_range");
  if (cx.launches) *cx.launches += 1;
  int32_t h[2];
  HG_CUDA(cudaMemcpyAsync(h, range.p, sizeof(h), cudaMemcpyDeviceToHost, cx.stream));
  HG_CUDA(cudaStreamSynchronize(cx.stream));
  return h[0] == 2 && h[1] == 2;
}

void build_graph_adjacency(const Ctx& cx, Level& L) {
  L.graph = true;
  L.adj.alloc(&cx.alloc, (size_t)(L.p > 0 ? L.p : 1));
  if (L.p > 0) {
    k_adjacency<<<grid_for(L.p, 256, cx.num_sms, 16), 256, 0, cx.stream>>>(
        L.eoff.p, L.pins.p, L.w.p, L.inets.p, L.ipin.p, L.p, L.adj.p);
    check_launch("adjacency");
    if (cx.launches) *cx.launches += 1;
  }
}

void build_tile_index(const Ctx& cx, const int32_t* eoff, int32_t m, int64_t p, int32_t* tile_net) {
  const int64_t ntiles = num_pin_tiles(p);
  k_tile_index<<<grid_for(m > 0 ? m : 1, 256, cx.num_sms, 16), 256, 0, cx.stream>>>(eoff, m, ntiles,
                                                                                  tile_net);
  check_launch("tile_index");
  if (cx.launches) *cx.launches += 1;
}

void build_incidence(const Ctx& cx, Level& L) {
  L.ioff.alloc(&cx.alloc, (size_t)L.n + 1);
  L.inets.alloc(&cx.alloc, (size_t)(L.p > 0 ? L.p : 1));
  L.ipin.alloc(&cx.alloc, (size_t)(L.p > 0 ? L.p : 1));
  HG_CUDA(cudaMemsetAsync(L.ioff.p, 0, sizeof(int32_t) * ((size_t)L.n + 1), cx.stream));
  if (L.p > 0) {
    k_degrees<<<grid_for(L.p, 256, cx.num_sms, 16), 256, 0, cx.stream>>>(L.pins.p, L.p, L.ioff.p);
    check_launch("degrees");
  }
  scan_exclusive_i32(cx, L.ioff.p, L.ioff.p, L.n, L.ioff.p + L.n);
  if (L.p > 0) {
    DBuf<int32_t> cursor, tiles;
    cursor.alloc(&cx.alloc, (size_t)L.n);
    HG_CUDA(cudaMemcpyAsync(cursor.p, L.ioff.p, sizeof(int32_t) * (size_t)L.n,
                            cudaMemcpyDeviceToDevice, cx.stream));
    tiles.alloc(&cx.alloc, (size_t)num_pin_tiles(L.p) + 1);
    build_tile_index(cx, L.eoff.p, L.m, L.p, tiles.p);
    k_scatter_incidence<<<grid_for(num_pin_tiles(L.p), 1, cx.num_sms, 8), PIN_TILE_THREADS, 0,
                          cx.stream>>>(L.eoff.p, L.pins.p, tiles.p, L.m, L.p, cursor.p,
                                       L.inets.p, L.ipin.p);
    check_launch("scatter_incidence");
    if (cx.launches) *cx.launches += 2;
  }
  if (cx.launches) *cx.launches += 1;
}

namespace {

// No node twice in a net (offsets and pin ranges already valid).
bool distinct_pins(const Ctx& cx, const Level& L) {
  if (L.m <= 0) return true;
  DBuf<int32_t> mx;
  mx.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int32_t), cx.stream));
  k_max_net_size<<<grid_for(L.m, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.eoff.p, L.m, mx.p);
  check_launch("max_net_size");
  k_distinct_small<<<grid_for(L.m, DISTINCT_WARPS, cx.num_sms, 16), DISTINCT_WARPS * 32, 0,
                     cx.stream>>>(L.eoff.p, L.pins.p, L.m, cx.d_status);
  check_launch("distinct_small");
  const int32_t biggest = read_i32(cx, mx.p);
  const int64_t words = ((int64_t)L.n + 31) / 32;
  if (biggest > DISTINCT_SMALL && (int64_t)cx.num_sms * words * 4 <= DISTINCT_BITMAP_BYTES) {
    const int blocks = cx.num_sms;
    DBuf<uint32_t> scratch;
    scratch.alloc(&cx.alloc, (size_t)blocks * (size_t)words);
    HG_CUDA(cudaMemsetAsync(scratch.p, 0, scratch.bytes(), cx.stream));
    k_distinct_big_bitmap<<<blocks, 256, 0, cx.stream>>>(L.eoff.p, L.pins.p, L.m, scratch.p,
                                                         words, cx.d_status);
    check_launch("distinct_big_bitmap");
  } else if (biggest > DISTINCT_SMALL) {
    uint32_t cap = 1;
    while (cap < 2u * (uint32_t)biggest) cap <<= 1;
    const int blocks = cx.num_sms;
    DBuf<int32_t> scratch;
    scratch.alloc(&cx.alloc, (size_t)blocks * cap);
    HG_CUDA(cudaMemsetAsync(scratch.p, 0xff, scratch.bytes(), cx.stream));
    k_distinct_big<<<blocks, 256, 0, cx.stream>>>(L.eoff.p, L.pins.p, L.m, scratch.p, cap,
                                                  cx.d_status);
    check_launch("distinct_big");
  }
  int32_t st = 0;
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(&st, cx.d_status, sizeof(st), cudaMemcpyDeviceToHost, cx.stream));
  HG_CUDA(cudaStreamSynchronize(cx.stream));
  if (st != DEV_OK) {
    int32_t zero = 0;
    HG_CUDA(cudaMemcpy(cx.d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return false;
  }
  return true;
}

}  // namespace

bool validate_pins_device(const Ctx& cx, const Level& L) {
  if (L.p > 0) {
    k_validate_pins<<<grid_for(L.p, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.pins.p, L.p, L.n,
                                                                             cx.d_status);
    check_launch("validate_pins");
    int32_t st = 0;
    HG_CUDA(cudaMemcpyAsync(&st, cx.d_status, sizeof(st), cudaMemcpyDeviceToHost, cx.stream));
    HG_CUDA(cudaStreamSynchronize(cx.stream));
    if (st != DEV_OK) {
      int32_t zero = 0;
      HG_CUDA(cudaMemcpy(cx.d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
      return false;
    }
  }
  return distinct_pins(cx, L);
}

bool validate_level_device(const Ctx& cx, const Level& L, int64_t* total_node_w,
                           int64_t* total_net_w) {
  DBuf<unsigned long long> sums;
  sums.alloc(&cx.alloc, 2);
  HG_CUDA(cudaMemsetAsync(sums.p, 0, 2 * sizeof(unsigned long long), cx.stream));
  if (L.m > 0) {
    k_validate_nets<<<grid_for(L.m, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
        L.eoff.p, L.m, L.w.p, cx.d_status, sums.p + 1);
    check_launch("validate_nets");
  }
  if (L.p > 0) {
    k_validate_pins<<<grid_for(L.p, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.pins.p, L.p, L.n,
                                                                             cx.d_status);
    check_launch("validate_pins");
  }
  k_validate_nodes<<<grid_for(L.n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.c.p, L.n,
                                                                           cx.d_status, sums.p);
  check_launch("validate_nodes");
  unsigned long long h[2] = {0, 0};
  HG_CUDA(cudaMemcpyAsync(h, sums.p, sizeof(h), cudaMemcpyDeviceToHost, cx.stream));
  int32_t st = 0;
  HG_CUDA(cudaMemcpyAsync(&st, cx.d_status, sizeof(st), cudaMemcpyDeviceToHost, cx.stream));
  HG_CUDA(cudaStreamSynchronize(cx.stream));
  if (st != DEV_OK) {
    int32_t zero = 0;
    HG_CUDA(cudaMemcpy(cx.d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return false;
  }
  // offsets and pins are sound: no node twice in a net
  if (!distinct_pins(cx, L)) return false;
  *total_node_w = (int64_t)h[0];
  *total_net_w = (int64_t)h[1];
  return true;
}

}  // namespace hgk
