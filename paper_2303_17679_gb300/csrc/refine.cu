// Uncoarsening on the device: projection (Algorithm 1), pin counts and
// connectivity sets (Sec. 2, Sec. 6.1 data layout), the connectivity
// objective (Sec. 2), and deterministic label propagation (Sec. 11
// "Deterministic Label Propagation Refinement" with the gain of Sec. 6).
//
// Layout: Phi is a dense m x k int32 table (row = net), Lambda one 64-bit
// mask per net (k <= 64), block weights int64[k].  One label-propagation
// sub-round is four launches for k <= 16 and five above: best moves of the
// warp and block node classes (a11, parallel branches of the captured
// pass), bucketing by block pair (k > 16 only), per-pair prefix selection
// (a12), application (a13).  Every move carries its source block, and the
// selection reads the block weights of the sub-round's start as the pass's
// starting weights plus the changes of its earlier sub-rounds, so nothing a
// kernel of the sub-round reads is changed by another one before the
// application.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "pintile.cuh"

namespace hgk {

namespace {

constexpr int WARPS = 8;  // warps per block for warp-per-item kernels

// ------------------------------------------------------------ projection

__global__ void k_project(const int32_t* __restrict__ map, const int32_t* __restrict__ coarse_part,
                          int32_t n, int32_t* __restrict__ fine_part) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    fine_part[u] = coarse_part[map[u]];
}

// ------------------------------------------------------ pin counts (a10)

// Phi(e, V_i) += 1 and Lambda(e) |= bit(i) for every pin; lanes that hold the
// same (net, block) combine their increments first.
__global__ void __launch_bounds__(PIN_TILE_THREADS)
k_pin_counts(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
             const int32_t* __restrict__ tile_net, int32_t m, int64_t p,
             const int32_t* __restrict__ part, int k, int32_t* __restrict__ phi,
             unsigned long long* __restrict__ lam) {
  __shared__ int32_t s_off[PIN_TILE + 3];
  const int64_t ntiles = num_pin_tiles(p);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    PinTileView v = stage_pin_tile(eoff, tile_net, m, p, t, s_off);
    for (int64_t base = v.q0; base < v.q1; base += blockDim.x) {
      const int64_t q = base + threadIdx.x;
      const bool valid = q < v.q1;
      int64_t key = -1 - (int64_t)threadIdx.x;  // unique for idle lanes
      int32_t e = 0, b = 0;
      if (valid) {
        e = v.e_lo + net_in_tile(s_off, v.count, q);
        b = part[pins[q]];
        key = (int64_t)e * k + b;
      }
      const unsigned peers = __match_any_sync(FULL, (unsigned long long)key);
      const int leader = __ffs(peers) - 1;
      if (valid && lane_id() == leader) {
        atomicAdd(&phi[(int64_t)e * k + b], __popc(peers));
        atomicOr(&lam[e], 1ull << b);
      }
    }
    __syncthreads();
  }
}

__global__ void k_block_weights(const int32_t* __restrict__ part, const int32_t* __restrict__ c,
                                int32_t n, int k, long long* __restrict__ bw) {
  __shared__ long long s_bw[HG_MAX_K];
  for (int i = threadIdx.x; i < k; i += blockDim.x) s_bw[i] = 0;
  __syncthreads();
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    atomic_add_i64(&s_bw[part[u]], (long long)c[u]);
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (s_bw[i]) atomic_add_i64(&bw[i], s_bw[i]);
}

// ------------------------------------------------------- objective (a14)

__global__ void k_objective(const unsigned long long* __restrict__ lam,
                            const int32_t* __restrict__ w, int32_t m,
                            unsigned long long* __restrict__ out) {
  __shared__ int64_t red[32];
  int64_t f = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int l = __popcll(lam[e]);
    if (l > 1) f += (int64_t)(l - 1) * w[e];
  }
  f = block_sum(f, red);
  if (threadIdx.x == 0 && f) atomicAdd(out, (unsigned long long)f);
}

// Objective of a graph level: the weight of the cut edges (lambda(e) - 1 is
// 1 for a cut edge and 0 otherwise).
__global__ void k_objective_graph(const int32_t* __restrict__ eoff,
                                  const int32_t* __restrict__ pins, const int32_t* __restrict__ w,
                                  const int32_t* __restrict__ part, int32_t m,
                                  unsigned long long* __restrict__ out) {
  __shared__ int64_t red[32];
  int64_t f = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = eoff[e];
    if (part[pins[b]] != part[pins[b + 1]]) f += w[e];
  }
  f = block_sum(f, red);
  if (threadIdx.x == 0 && f) atomicAdd(out, (unsigned long long)f);
}

// ------------------------------------------------ packed net records (a11)

// Label propagation reads, for every incidence (u, e), w(e), Lambda(e) and
// whether Phi(e, Pi[u]) = 1.  They live in one record per net, so the gain
// gathers one 32-byte sector per incidence instead of three:
//   k <= 32: 16 bytes {w(e), ones(e), Lambda(e), 0} (one int4);
//   k >  32: 32 bytes {w(e), 0, ones(e) as 64 bits}, {Lambda(e) as 64 bits, 0, 0},
// with ones(e) = {i : Phi(e, i) = 1}.  Phi stays the authority: the
// application changes a pin count with an atomic that returns the old
// count, and flips the record's bits for the transitions it caused
// (0 <-> 1 toggles Lambda and ones, 1 <-> 2 toggles ones); the flips commute,
// so the records equal their definition whatever the order of the moves.
struct NetRec {
  int32_t w;
  unsigned long long ones, lam;
};

__device__ __forceinline__ NetRec load_rec(const int4* __restrict__ rec, int64_t e, bool wide) {
  if (!wide) {
    const int4 r = rec[e];
    return NetRec{r.x, (unsigned long long)(uint32_t)r.y, (unsigned long long)(uint32_t)r.z};
  }
  const int4 a = rec[2 * e], b = rec[2 * e + 1];
  return NetRec{a.x, (unsigned long long)(uint32_t)a.z | ((unsigned long long)(uint32_t)a.w << 32),
                (unsigned long long)(uint32_t)b.x | ((unsigned long long)(uint32_t)b.y << 32)};
}

// Applies the bit flips of one pin-count change to net e's record.
__device__ __forceinline__ void flip_rec(int4* rec, int64_t e, bool wide, unsigned long long ones_x,
                                         unsigned long long lam_x) {
  if (!wide) {
    if (ones_x) atomicXor(reinterpret_cast<unsigned*>(&rec[e].y), (unsigned)ones_x);
    if (lam_x) atomicXor(reinterpret_cast<unsigned*>(&rec[e].z), (unsigned)lam_x);
  } else {
    if (ones_x) atomicXor(reinterpret_cast<unsigned long long*>(&rec[2 * e].z), ones_x);
    if (lam_x) atomicXor(reinterpret_cast<unsigned long long*>(&rec[2 * e + 1].x), lam_x);
  }
}

// Records from Phi, Lambda and w (one thread per net).
__global__ void k_net_records(const int32_t* __restrict__ phi, const unsigned long long* __restrict__ lam,
                              const int32_t* __restrict__ w, int32_t m, int k, bool wide,
                              int4* __restrict__ rec) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long ones = 0;
    for (int i = 0; i < k; ++i)
      if (phi[e * k + i] == 1) ones |= 1ull << i;
    const unsigned long long l = lam[e];
    if (!wide) {
      rec[e] = make_int4(w[e], (int32_t)(uint32_t)ones, (int32_t)(uint32_t)l, 0);
    } else {
      rec[2 * e] = make_int4(w[e], 0, (int32_t)(uint32_t)ones, (int32_t)(uint32_t)(ones >> 32));
      rec[2 * e + 1] = make_int4((int32_t)(uint32_t)l, (int32_t)(uint32_t)(l >> 32), 0, 0);
    }
  }
}

// Objective from the records' Lambda.
__global__ void k_objective_rec(const int4* __restrict__ rec, int32_t m, bool wide,
                                unsigned long long* __restrict__ out) {
  __shared__ int64_t red[32];
  int64_t f = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const NetRec r = load_rec(rec, e, wide);
    const int l = __popcll(r.lam);
    if (l > 1) f += (int64_t)(l - 1) * r.w;
  }
  f = block_sum(f, red);
  if (threadIdx.x == 0 && f) atomicAdd(out, (unsigned long long)f);
}

// -------------------------------------------- sub-round node lists (a11)

// Nodes of a pass are listed by key = sub-round * 2 + class, class 1 for
// nodes with more than block_deg incident nets (a block per node).
__device__ __forceinline__ int lp_key(const int32_t* ioff, uint64_t seed, int level, int pass,
                                      int64_t u, int S, int block_deg) {
  const int32_t deg = ioff[u + 1] - ioff[u];
  if (deg == 0) return -1;  // isolated nodes never move
  return subround_of_node_lp(seed, level, pass, (int)u, S) * 2 + (deg > block_deg ? 1 : 0);
}

__global__ void k_lp_count(const int32_t* __restrict__ ioff, int32_t n, uint64_t seed, int level,
                           const int32_t* __restrict__ d_pass, int S, int block_deg,
                           int32_t* __restrict__ cnt) {
  extern __shared__ int32_t s_cnt[];
  const int pass = *d_pass;
  for (int i = threadIdx.x; i < 2 * S; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int key = lp_key(ioff, seed, level, pass, u, S, block_deg);
    if (key >= 0) atomicAdd(&s_cnt[key], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * S; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

// Every block recomputes the (tiny) exclusive scan of the 2S counts.
__global__ void k_lp_scatter(const int32_t* __restrict__ ioff, int32_t n, uint64_t seed, int level,
                             const int32_t* __restrict__ d_pass, int S, int block_deg,
                             const int32_t* __restrict__ cnt, int32_t* __restrict__ fill,
                             int32_t* __restrict__ off, int32_t* __restrict__ list) {
  extern __shared__ int32_t s_off[];
  const int pass = *d_pass;
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int i = 0; i < 2 * S; ++i) {
      s_off[i] = run;
      run += cnt[i];
    }
    s_off[2 * S] = run;
    if (blockIdx.x == 0)
      for (int i = 0; i <= 2 * S; ++i) off[i] = s_off[i];
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const int64_t u = b + lane_id();
    const bool valid = u < n;
    const int key = valid ? lp_key(ioff, seed, level, pass, u, S, block_deg) : -1;
    const int32_t slot = warp_claim_slot(fill, key, __ballot_sync(FULL, valid));
    if (slot >= 0) list[s_off[key] + slot] = (int32_t)u;
  }
}

// Per sub-round bookkeeping words.
enum SubroundWord { SW_MOVES = 0, SW_APPROVED = 1, SW_WORDS = 4 };

// ------------------------------------------------- best moves (a11)

// With b(u) = w(nets where u is the only pin of its block) and W_I = w(I(u)),
// the gain of Sec. 6 is
//   g(u, t) = b(u) - W_I + w({e in I(u) : t in Lambda(e)}),
// evaluated for all t at once.  For k > 16 every lane takes one incident net
// and adds w(e) to the warp's shared counter of each block of Lambda(e); a
// net with lambda(e) > k/2 instead adds w(e) to a per-lane scalar `full` (a
// term of every block's sum) and takes it back from the counters of the
// blocks outside Lambda(e), so a net costs at most k/2 shared atomics (the
// 1k-100k-pin nets of large-net inputs touch nearly every block).  Counters
// are int32: every true sum is below 2^31 (the total net weight), and the
// wrap-around of intermediate values cancels.  For k <= 16 the warp reduces
// each block's sum directly.  A warp handles the chunks
// c0 = beg + 32 * (first + i * stride) of I(u); acc0 / acc1 are filled from
// the sums of blocks lane and lane + 32 by gain_collect.
struct GainPart {
  long long acc0, acc1, ben, wsum, full;
};

constexpr int GAIN_REDUCE_K = 16;

__device__ __forceinline__ GainPart gain_partial(const int32_t* __restrict__ inets,
                                                 const int4* __restrict__ rec, bool wide, int k,
                                                 int from, int32_t beg, int32_t end, int first,
                                                 int stride, int32_t* s_cnt) {
  const int lane = lane_id();
  const unsigned long long kmask = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  GainPart g{0, 0, 0, 0, 0};
  for (int32_t c0 = beg + 32 * first; c0 < end; c0 += 32 * stride) {
    const int32_t j = c0 + lane;
    int32_t we = 0;
    unsigned long long le = 0;
    if (j < end) {
      const NetRec r = load_rec(rec, inets[j], wide);
      we = r.w;
      le = r.lam;
      if ((r.ones >> from) & 1ull) g.ben += we;  // u is the only pin of its block in e
      g.wsum += we;
    }
    if (k <= GAIN_REDUCE_K) {
      // small k: one warp reduction per block instead of atomics, which on
      // coarse levels (many blocks per net) would all hit the same k counters
      for (int t = 0; t < k; ++t) {
        const unsigned x = __reduce_add_sync(FULL, ((le >> t) & 1ull) ? (unsigned)we : 0u);
        if (lane == t) g.acc0 += x;
      }
    } else {
      int32_t delta = we;
      if (2 * __popcll(le) > k) {
        g.full += we;
        le = ~le & kmask;
        delta = -we;
      }
      while (le) {
        atomicAdd(&s_cnt[__ffsll((long long)le) - 1], delta);
        le &= le - 1;
      }
    }
  }
  return g;
}

// gain_partial for nodes of many incident nets (the block class) and k <= 16:
// every lane takes four consecutive incidences of a 128-incidence chunk with
// one 16-byte load of their net ids, so four record gathers are in flight per
// lane, and the warp reduces each block's sum once per 128 incidences.  (For
// k > 16 the per-lane shared-counter loops of four nets serialise; there the
// one-incidence form is faster.)
// Chunks start at beg rounded down to a multiple of 4 (the 16-byte loads stay
// aligned); positions outside [beg, end) count nothing.
constexpr int GAIN_VEC = 4;

__device__ __forceinline__ GainPart gain_partial_vec(const int32_t* __restrict__ inets,
                                                     const int4* __restrict__ rec, bool wide,
                                                     int k, int from, int32_t beg, int32_t end,
                                                     int first, int stride, int32_t* s_cnt) {
  const int lane = lane_id();
  const unsigned long long kmask = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  GainPart g{0, 0, 0, 0, 0};
  constexpr int32_t CH = 32 * GAIN_VEC;
  const int32_t a0 = beg & ~(GAIN_VEC - 1);
  for (int32_t c0 = a0 + CH * first; c0 < end; c0 += CH * stride) {
    const int32_t j0 = c0 + GAIN_VEC * lane;
    int32_t e[GAIN_VEC];
    if (j0 >= beg && j0 + GAIN_VEC <= end) {
      const int4 v = *reinterpret_cast<const int4*>(inets + j0);
      e[0] = v.x;
      e[1] = v.y;
      e[2] = v.z;
      e[3] = v.w;
    } else {
#pragma unroll
      for (int x = 0; x < GAIN_VEC; ++x) {
        const int32_t j = j0 + x;
        e[x] = j >= beg && j < end ? inets[j] : -1;
      }
    }
    int32_t we[GAIN_VEC];
    unsigned long long le[GAIN_VEC];
#pragma unroll
    for (int x = 0; x < GAIN_VEC; ++x) {
      we[x] = 0;
      le[x] = 0;
      if (e[x] >= 0) {
        const NetRec r = load_rec(rec, e[x], wide);
        we[x] = r.w;
        le[x] = r.lam;
        if ((r.ones >> from) & 1ull) g.ben += r.w;
        g.wsum += r.w;
      }
    }
    if (k <= GAIN_REDUCE_K) {
      for (int t = 0; t < k; ++t) {
        unsigned mine = 0;
#pragma unroll
        for (int x = 0; x < GAIN_VEC; ++x) mine += ((le[x] >> t) & 1ull) ? (unsigned)we[x] : 0u;
        const unsigned sum = __reduce_add_sync(FULL, mine);
        if (lane == t) g.acc0 += sum;
      }
    } else {
#pragma unroll
      for (int x = 0; x < GAIN_VEC; ++x) {
        unsigned long long l = le[x];
        int32_t delta = we[x];
        if (2 * __popcll(l) > k) {
          g.full += we[x];
          l = ~l & kmask;
          delta = -we[x];
        }
        while (l) {
          atomicAdd(&s_cnt[__ffsll((long long)l) - 1], delta);
          l &= l - 1;
        }
      }
    }
  }
  return g;
}

// Graph levels (Sec. 10, "The Gain Table"): the gain of moving u to V_t is
// w(u, V_t) - w(u, V_Pi(u)), the weight of u's edges into V_t minus that of
// its edges into its own block, which equals the gain of Sec. 6 for nets of
// two pins.  The lanes sum the edge weights per neighbour block: a warp
// reduction per block for k <= 16, shared counters above.
__device__ __forceinline__ GainPart gain_partial_graph(const int2* __restrict__ adj,
                                                       const int32_t* __restrict__ part, int k,
                                                       int32_t beg, int32_t end, int first,
                                                       int stride, int32_t* s_cnt) {
  const int lane = lane_id();
  GainPart g{0, 0, 0, 0, 0};
  for (int32_t c0 = beg + 32 * first; c0 < end; c0 += 32 * stride) {
    const int32_t j = c0 + lane;
    int32_t we = 0, tb = -1;
    if (j < end) {
      const int2 a = adj[j];
      we = a.y;
      tb = part[a.x];
    }
    if (k <= GAIN_REDUCE_K) {
      for (int t = 0; t < k; ++t) {
        const unsigned x = __reduce_add_sync(FULL, tb == t ? (unsigned)we : 0u);
        if (lane == t) g.acc0 += x;
      }
    } else if (tb >= 0) {
      atomicAdd(&s_cnt[tb], we);
    }
  }
  return g;
}

// After gain_collect on a graph level: ben - wsum = -w(u, V_from), so that
// gain_best computes w(u, V_t) - w(u, V_from).
__device__ __forceinline__ void graph_gain_terms(GainPart& g, int from) {
  const int lane = lane_id();
  g.ben = 0;
  g.wsum = lane == from ? g.acc0 : (lane + 32 == from ? g.acc1 : 0);
}

// Moves the warp's block counters plus its `full` sum into acc0 / acc1 and
// clears the counters (k above GAIN_REDUCE_K; for smaller k the sums are in
// acc0 already).
__device__ __forceinline__ void gain_collect(GainPart& g, int32_t* s_cnt, int k) {
  if (k <= GAIN_REDUCE_K) return;
  const int lane = lane_id();
  const long long full = warp_sum(g.full);
  g.full = 0;
  __syncwarp();
  g.acc0 = (long long)s_cnt[lane] + full;
  g.acc1 = (long long)s_cnt[lane + 32] + full;
  s_cnt[lane] = 0;
  s_cnt[lane + 32] = 0;
  __syncwarp();
}

// Best target of the warp's complete accumulators: (gain desc, t asc), t != from.
__device__ __forceinline__ void gain_best(const GainPart& g, int k, int from, long long& best_g,
                                          int& best_t) {
  const int lane = lane_id();
  const long long ben = warp_sum(g.ben), wsum = warp_sum(g.wsum);
  best_g = LLONG_MIN;
  best_t = -1;
  if (lane < k && lane != from) {
    best_g = ben - wsum + g.acc0;
    best_t = lane;
  }
  if (lane + 32 < k && lane + 32 != from) {
    const long long g1 = ben - wsum + g.acc1;
    if (g1 > best_g) {
      best_g = g1;
      best_t = lane + 32;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const long long og = __shfl_xor_sync(FULL, best_g, d);
    const int ot = __shfl_xor_sync(FULL, best_t, d);
    if (og > best_g || (og == best_g && ot >= 0 && (best_t < 0 || ot < best_t))) {
      best_g = og;
      best_t = ot;
    }
  }
}

// Sort key: gain descending, node id ascending (gains are < 2^31).
__device__ __forceinline__ unsigned long long sel_key(long long g, int32_t u) {
  return ((unsigned long long)(0x7fffffffLL - g) << 32) | (unsigned)u;
}

struct GainArgs {
  const int32_t* ioff;
  const int32_t* inets;
  const int4* rec;  // packed net records (hypergraph levels)
  bool wide;        // k > 32: 32-byte records
  const int32_t* part;
  int k;
  const int32_t* list;
  const int32_t* sr_off;
  int s;
  int32_t* mv_u;
  int32_t* mv_to;  // target | source << 8
  long long* mv_g;
  int32_t* dcount;
  // k <= 16: the sort keys of each direction's first dcap moves, dcap slots
  // per direction (dcap = 0: not kept)
  unsigned long long* dkeys;
  int32_t dcap;
  int32_t* words;
  unsigned long long* work;
  bool graph;       // graph level: gains from adj and part, no Phi / Lambda
  const int2* adj;
};

__device__ __forceinline__ void gain_emit(const GainArgs& A, int32_t u, int from, long long g,
                                          int t) {
  if (g > 0) {
    const int32_t slot = atomicAdd(&A.words[SW_MOVES], 1);
    A.mv_u[slot] = u;
    A.mv_to[slot] = t | (from << 8);  // target block, source block above bit 8
    A.mv_g[slot] = g;
    const int d = from * A.k + t;
    const int32_t pos = atomicAdd(&A.dcount[d], 1);
    if (pos < A.dcap) A.dkeys[(size_t)d * A.dcap + pos] = sel_key(g, u);
  }
}

// class 0 (at most block_deg incident nets): one warp per node
__global__ void __launch_bounds__(WARPS * 32) k_lp_gain_warp(GainArgs A) {
  __shared__ int32_t s_cnt[WARPS][64];
  const int lane = lane_id();
  int32_t* cnt = s_cnt[warp_in_block()];
  cnt[lane] = 0;
  cnt[lane + 32] = 0;
  __syncwarp();
  const int32_t lo = A.sr_off[2 * A.s], hi = A.sr_off[2 * A.s + 1];
  int64_t incid = 0;
  for (int32_t i = lo + blockIdx.x * WARPS + warp_in_block(); i < hi; i += gridDim.x * WARPS) {
    const int32_t u = A.list[i];
    const int from = A.part[u];
    const int32_t beg = A.ioff[u], end = A.ioff[u + 1];
    GainPart g = A.graph ? gain_partial_graph(A.adj, A.part, A.k, beg, end, 0, 1, cnt)
                         : gain_partial(A.inets, A.rec, A.wide, A.k, from, beg, end, 0, 1, cnt);
    gain_collect(g, cnt, A.k);
    if (A.graph) graph_gain_terms(g, from);
    long long bg;
    int bt;
    gain_best(g, A.k, from, bg, bt);
    if (lane == 0) gain_emit(A, u, from, bg, bt);
    incid += end - beg;
  }
  const unsigned long long cv[1] = {lane == 0 ? (unsigned long long)incid : 0ull};
  block_add_counters(A.work, cv);
}

// class 0 on hypergraph levels with k <= 16 and few incident nets per node
// (mean degree <= SUB_MEAN_DEG): one group of SUB_G lanes per node instead of
// a warp, so a warp has NG nodes' load chains in flight.  Every lane sums
// w(e) per block of Lambda(e) over its incidences in registers, the group
// combines the sums with xor shuffles among its own lanes, and every lane of
// the group picks the same best target.  Groups run independently (their
// shuffles name only the group's lanes).
constexpr int SUB_G = 8;
constexpr int SUB_MEAN_DEG = 16;

__global__ void __launch_bounds__(WARPS * 32) k_lp_gain_sub(GainArgs A) {
  constexpr int NG = 32 / SUB_G;
  const int lane = lane_id(), sub = lane % SUB_G, grp = lane / SUB_G;
  const unsigned gmask = ((1u << SUB_G) - 1u) << (grp * SUB_G);
  const int32_t lo = A.sr_off[2 * A.s], hi = A.sr_off[2 * A.s + 1];
  const int k = A.k;
  unsigned long long incid = 0;
  for (int32_t i = lo + (blockIdx.x * WARPS + warp_in_block()) * NG + grp; i < hi;
       i += gridDim.x * WARPS * NG) {
    const int32_t u = A.list[i];
    const int from = A.part[u];
    const int32_t beg = A.ioff[u], end = A.ioff[u + 1];
    int32_t acc[GAIN_REDUCE_K];
#pragma unroll
    for (int t = 0; t < GAIN_REDUCE_K; ++t) acc[t] = 0;
    long long ben = 0, wsum = 0;
    for (int32_t j = beg + sub; j < end; j += SUB_G) {
      const NetRec r = load_rec(A.rec, A.inets[j], A.wide);
      if ((r.ones >> from) & 1ull) ben += r.w;  // u is the only pin of its block in e
      wsum += r.w;
#pragma unroll
      for (int t = 0; t < GAIN_REDUCE_K; ++t)
        if ((r.lam >> t) & 1ull) acc[t] += r.w;
    }
#pragma unroll
    for (int d = SUB_G / 2; d > 0; d >>= 1) {
      ben += __shfl_xor_sync(gmask, ben, d);
      wsum += __shfl_xor_sync(gmask, wsum, d);
#pragma unroll
      for (int t = 0; t < GAIN_REDUCE_K; ++t) acc[t] += __shfl_xor_sync(gmask, acc[t], d);
    }
    // (gain desc, t asc), t != from
    long long best_g = LLONG_MIN;
    int best_t = -1;
#pragma unroll
    for (int t = 0; t < GAIN_REDUCE_K; ++t) {
      if (t >= k || t == from) continue;
      const long long g = ben - wsum + acc[t];
      if (g > best_g) {
        best_g = g;
        best_t = t;
      }
    }
    if (sub == 0) {
      gain_emit(A, u, from, best_g, best_t);
      incid += (unsigned long long)(end - beg);
    }
  }
  const unsigned long long cv[1] = {incid};
  block_add_counters(A.work, cv);
}

// class 1: one block (GAIN_BLOCK_WARPS warps) per node; the warps split I(u)
// and their partial accumulators are summed in shared memory before the argmax
constexpr int GAIN_BLOCK_WARPS = 16;

__global__ void __launch_bounds__(GAIN_BLOCK_WARPS * 32) k_lp_gain_block(GainArgs A) {
  constexpr int WARPS = GAIN_BLOCK_WARPS;
  __shared__ long long s_acc[WARPS][64];
  __shared__ long long s_bw[WARPS][2];
  __shared__ int32_t s_cnt[WARPS][64];
  const int lane = lane_id(), wv = warp_in_block();
  int32_t* cnt = s_cnt[wv];
  cnt[lane] = 0;
  cnt[lane + 32] = 0;
  __syncwarp();
  const int32_t lo = A.sr_off[2 * A.s + 1], hi = A.sr_off[2 * A.s + 2];
  int64_t incid = 0;
  for (int32_t i = lo + blockIdx.x; i < hi; i += gridDim.x) {
    const int32_t u = A.list[i];
    const int from = A.part[u];
    const int32_t beg = A.ioff[u], end = A.ioff[u + 1];
    GainPart g =
        A.graph ? gain_partial_graph(A.adj, A.part, A.k, beg, end, wv, WARPS, cnt)
        : A.k <= GAIN_REDUCE_K
            ? gain_partial_vec(A.inets, A.rec, A.wide, A.k, from, beg, end, wv, WARPS, cnt)
            : gain_partial(A.inets, A.rec, A.wide, A.k, from, beg, end, wv, WARPS, cnt);
    gain_collect(g, cnt, A.k);
    if (A.graph) graph_gain_terms(g, from);
    s_acc[wv][lane] = g.acc0;
    s_acc[wv][lane + 32] = g.acc1;
    const long long b = warp_sum(g.ben), ws = warp_sum(g.wsum);
    if (lane == 0) {
      s_bw[wv][0] = b;
      s_bw[wv][1] = ws;
    }
    __syncthreads();
    if (wv == 0) {
      GainPart t{0, 0, 0, 0, 0};
      for (int x = 0; x < WARPS; ++x) {
        t.acc0 += s_acc[x][lane];
        t.acc1 += s_acc[x][lane + 32];
      }
      // ben and wsum enter gain_best through warp sums: put them on lane 0
      if (lane == 0)
        for (int x = 0; x < WARPS; ++x) {
          t.ben += s_bw[x][0];
          t.wsum += s_bw[x][1];
        }
      long long bg;
      int bt;
      gain_best(t, A.k, from, bg, bt);
      if (lane == 0) gain_emit(A, u, from, bg, bt);
    }
    __syncthreads();
    incid += end - beg;
  }
  if (threadIdx.x == 0 && incid) atomicAdd(A.work, (unsigned long long)incid);
}

// ------------------------------------- pair bucketing + selection (a12)

// Exclusive scan of the k*k direction counts into s_doff[0..kk] by the whole
// block (kk <= 4096: each thread scans a contiguous run, then the run totals
// are scanned by warps).
__device__ void direction_offsets(const int32_t* dcount, int kk, int32_t* s_doff) {
  __shared__ int32_t s_tot[32];
  const int nt = blockDim.x;
  const int per = (kk + nt - 1) / nt;
  const int d0 = threadIdx.x * per;
  int32_t run = 0;
  for (int d = d0; d < d0 + per && d < kk; ++d) run += dcount[d];
  const int32_t incl = warp_inclusive_scan(run);
  if (lane_id() == 31) s_tot[warp_in_block()] = incl;
  __syncthreads();
  if (warp_in_block() == 0) {
    const int nw = nt >> 5;
    int32_t x = lane_id() < nw ? s_tot[lane_id()] : 0;
    x = warp_inclusive_scan(x);
    if (lane_id() < nw) s_tot[lane_id()] = x;
  }
  __syncthreads();
  int32_t base = (warp_in_block() ? s_tot[warp_in_block() - 1] : 0) + incl - run;
  for (int d = d0; d < d0 + per && d < kk; ++d) {
    s_doff[d] = base;
    base += dcount[d];
  }
  if (threadIdx.x == nt - 1) s_doff[kk] = s_tot[(nt >> 5) - 1];
  __syncthreads();
}

__global__ void k_lp_bucket(const int32_t* __restrict__ mv_to, int k,
                            const int32_t* __restrict__ dcount, int32_t* __restrict__ dfill,
                            int32_t* __restrict__ doff, const int32_t* __restrict__ words,
                            int32_t* __restrict__ bucket) {
  extern __shared__ int32_t s_doff[];
  const int kk = k * k;
  direction_offsets(dcount, kk, s_doff);
  if (blockIdx.x == 0)
    for (int d = threadIdx.x; d <= kk; d += blockDim.x) doff[d] = s_doff[d];
  const int32_t nm = words[SW_MOVES];
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < nm; b += stride) {
    const int32_t i = b + lane_id();
    const bool valid = i < nm;
    const int d = valid ? (mv_to[i] >> 8) * k + (mv_to[i] & 0xff) : -1;
    const int32_t slot = warp_claim_slot(dfill, d, __ballot_sync(FULL, valid));
    if (slot >= 0) bucket[s_doff[d] + slot] = i;
  }
}

constexpr int SEL_THREADS = 256;
constexpr int SEL_GATHER_K = 16;
// Moves per direction kept in the best-move kernels' key lists (k <= 16);
// a direction with more moves is gathered from the move list.
constexpr int32_t SEL_DIR_KEYS = 1024;
// Moves per direction sorted in shared memory (more go through global
// memory): 4096 for k <= 8, 2048 for k <= 16, else 1024 (pairs hold fewer
// moves as k grows, and a smaller buffer lets more pair blocks share an SM).
__host__ __device__ inline int sel_cap_for(int k) { return k <= 8 ? 4096 : (k <= 16 ? 2048 : 1024); }
inline size_t sel_smem_bytes(int cap) { return (size_t)(4 * cap + 2) * sizeof(unsigned long long); }


// The weight prefixes of both directions of a pair from one block-wide scan
// over the concatenation of their sorted moves: A[x] = weight of the first x
// moves a->b (x = 0..na), B[x] likewise for b->a.
__device__ void block_weight_prefix2(const unsigned long long* ka, int na,
                                     const unsigned long long* kb, int nb,
                                     const int32_t* __restrict__ c, long long* A, long long* B,
                                     long long* s_red) {
  __shared__ long long s_tot_a;
  if (threadIdx.x == 0) {
    s_red[32] = 0;
    s_tot_a = 0;
    A[0] = 0;
    B[0] = 0;
  }
  __syncthreads();
  const int cnt = na + nb;
  for (int base = 0; base < cnt; base += blockDim.x) {
    const int x = base + threadIdx.x;
    long long v = 0;
    if (x < na) v = (long long)c[(int32_t)(ka[x] & 0xffffffffu)];
    else if (x < cnt) v = (long long)c[(int32_t)(kb[x - na] & 0xffffffffu)];
    long long y = warp_inclusive_scan(v);
    if (lane_id() == 31) s_red[warp_in_block()] = y;
    __syncthreads();
    if (warp_in_block() == 0) {
      long long z = lane_id() < (int)(blockDim.x >> 5) ? s_red[lane_id()] : 0;
      z = warp_inclusive_scan(z);
      if (lane_id() < (int)(blockDim.x >> 5)) s_red[lane_id()] = z;
    }
    __syncthreads();
    const long long carry = s_red[32];
    const long long incl = carry + (warp_in_block() ? s_red[warp_in_block() - 1] : 0) + y;
    if (x < na) A[x + 1] = incl;
    if (x == na - 1) s_tot_a = incl;
    __syncthreads();
    if (x >= na && x < cnt) B[x - na + 1] = incl - s_tot_a;
    if (threadIdx.x == blockDim.x - 1) s_red[32] = incl;
    __syncthreads();
  }
}

// Bitonic sorts of the two directions of a pair (Pa and Pb powers of two) by
// the block, stage by stage together: one barrier per stage for both.
__device__ void block_bitonic_sort2(unsigned long long* a, int Pa, unsigned long long* b, int Pb) {
  const int P = Pa > Pb ? Pa : Pb;
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int x = threadIdx.x; x < Pa + Pb; x += blockDim.x) {
        unsigned long long* buf = x < Pa ? a : b;
        const int i = x < Pa ? x : x - Pa;
        const int n = x < Pa ? Pa : Pb;
        if (kk > n) continue;
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long u = buf[i], v = buf[ixj];
          const bool up = (i & kk) == 0;
          if ((u > v) == up) {
            buf[i] = v;
            buf[ixj] = u;
          }
        }
      }
      __syncthreads();
    }
  }
}

// One block per unordered block pair (a, b), a < b.  Sorts the moves a->b
// and b->a by (gain desc, id asc), builds their weight prefixes A and B, and
// finds the last state (i, j) on the merge path of A[0..na-1] and
// B[0..nb-1] (ties to A) with -slack_a <= A[i] - B[j] <= slack_b.  Moves in
// the chosen prefixes are approved.
// GATHER (small k): no bucket pass; a pair block reads its two directions'
// sort keys from the lists the best-move kernels filled (dkeys, dcap slots
// per direction), or, when a direction has more moves than that, reads the
// whole move list of the sub-round and keeps the moves of its two directions
// (their order is irrelevant, the keys are sorted); the global offsets of a
// direction too long for shared memory are summed from dcount.
template <bool GATHER>
__global__ void __launch_bounds__(SEL_THREADS)
k_lp_select(const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets,
            const int32_t* __restrict__ bucket, const int32_t* __restrict__ doff,
            const int32_t* __restrict__ dcount, const int32_t* __restrict__ mv_u,
            const int32_t* __restrict__ mv_to, const long long* __restrict__ mv_g,
            const int32_t* __restrict__ c, const long long* __restrict__ bw_base,
            long long* __restrict__ dbw, int s, long long lmax, int k,
            unsigned long long* __restrict__ gkeys, long long* __restrict__ gpre,
            const int32_t* __restrict__ words, int32_t* __restrict__ part,
            unsigned long long* __restrict__ moved, int32_t* __restrict__ ap_u,
            int32_t* __restrict__ ap_from, int32_t* __restrict__ ap_to,
            int32_t* __restrict__ ap_count, bool graph,
            const unsigned long long* __restrict__ dkeys, int32_t dcap) {
  extern __shared__ __align__(16) unsigned long long sel_smem[];
  const int cap = sel_cap_for(k);
  unsigned long long* s_keys0 = sel_smem;
  unsigned long long* s_keys1 = sel_smem + cap;
  long long* s_pre0 = reinterpret_cast<long long*>(sel_smem + 2 * cap);
  long long* s_pre1 = s_pre0 + cap + 1;
  __shared__ long long s_red[33];
  __shared__ int s_best;
  // decode the pair index into (a, b), a < b
  int pair = blockIdx.x, a = 0;
  while (pair >= k - 1 - a) {
    pair -= k - 1 - a;
    ++a;
  }
  const int b = a + 1 + pair;
  const int dab = a * k + b, dba = b * k + a;
  const int na = dcount[dab], nb = dcount[dba];
  if (na + nb == 0) return;
  auto pow2 = [](int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
  };
  const int Pa = pow2(na), Pb = pow2(nb);
  int oa = 0, ob = 0;
  __shared__ int s_gat[4];  // GATHER: offsets of the two directions, fill counters
  if constexpr (GATHER) {
    if (threadIdx.x < 4) s_gat[threadIdx.x] = 0;
    __syncthreads();
    if (Pa > cap || Pb > cap) {
      int sa = 0, sb = 0;
      for (int d = threadIdx.x; d < k * k; d += blockDim.x) {
        const int cd = dcount[d];
        if (d < dab) sa += cd;
        if (d < dba) sb += cd;
      }
      sa = warp_sum(sa);
      sb = warp_sum(sb);
      if (lane_id() == 0) {
        atomicAdd(&s_gat[0], sa);
        atomicAdd(&s_gat[1], sb);
      }
      __syncthreads();
      oa = s_gat[0];
      ob = s_gat[1];
    }
  } else {
    oa = doff[dab];
    ob = doff[dba];
  }
  // buffers: shared memory when the padded sequence fits, else a global
  // region of 2 * count slots at twice the direction's bucket offset
  unsigned long long* ka = Pa <= cap ? s_keys0 : gkeys + 2 * (int64_t)oa;
  unsigned long long* kb = Pb <= cap ? s_keys1 : gkeys + 2 * (int64_t)ob;
  long long* A = na <= cap ? s_pre0 : gpre + (int64_t)oa + dab;
  long long* B = nb <= cap ? s_pre1 : gpre + (int64_t)ob + dba;

  if (GATHER && na <= dcap && nb <= dcap) {
    // both directions fit the key lists the best-move kernels filled
    const unsigned long long* da = dkeys + (size_t)dab * dcap;
    const unsigned long long* db = dkeys + (size_t)dba * dcap;
    for (int i = threadIdx.x; i < Pa; i += blockDim.x) ka[i] = i < na ? da[i] : ~0ull;
    for (int i = threadIdx.x; i < Pb; i += blockDim.x) kb[i] = i < nb ? db[i] : ~0ull;
  } else if constexpr (GATHER) {
    const int32_t nm = words[SW_MOVES];
    const unsigned below = (1u << lane_id()) - 1u;
    // GATHER_ILP moves per thread and round: their directions are loaded
    // before any is classified (only the pair's own moves load the rest)
    constexpr int GATHER_ILP = 4;
    for (int32_t b0 = 0; b0 < nm; b0 += GATHER_ILP * blockDim.x) {
      int32_t dir[GATHER_ILP];
#pragma unroll
      for (int x = 0; x < GATHER_ILP; ++x) {
        const int32_t i = b0 + x * blockDim.x + threadIdx.x;
        dir[x] = i < nm ? mv_to[i] : -1;
      }
#pragma unroll
      for (int x = 0; x < GATHER_ILP; ++x) {
        const int32_t i = b0 + x * blockDim.x + threadIdx.x;
        const int t = dir[x] & 0xff, src = dir[x] >> 8;
        const bool in_a = dir[x] >= 0 && src == a && t == b;
        const bool in_b = dir[x] >= 0 && src == b && t == a;
        unsigned long long key = 0;
        if (in_a || in_b) key = sel_key(mv_g[i], mv_u[i]);
        const unsigned ma = __ballot_sync(FULL, in_a), mb = __ballot_sync(FULL, in_b);
        if ((ma | mb) == 0) continue;
        int base_a = 0, base_b = 0;
        if (lane_id() == 0) {
          if (ma) base_a = atomicAdd(&s_gat[2], __popc(ma));
          if (mb) base_b = atomicAdd(&s_gat[3], __popc(mb));
        }
        base_a = __shfl_sync(FULL, base_a, 0);
        base_b = __shfl_sync(FULL, base_b, 0);
        if (in_a) ka[base_a + __popc(ma & below)] = key;
        if (in_b) kb[base_b + __popc(mb & below)] = key;
      }
    }
    for (int i = na + threadIdx.x; i < Pa; i += blockDim.x) ka[i] = ~0ull;
    for (int i = nb + threadIdx.x; i < Pb; i += blockDim.x) kb[i] = ~0ull;
  } else {
    for (int i = threadIdx.x; i < Pa; i += blockDim.x) {
      if (i < na) {
        const int32_t mi = bucket[oa + i];
        ka[i] = sel_key(mv_g[mi], mv_u[mi]);
      } else {
        ka[i] = ~0ull;
      }
    }
    for (int i = threadIdx.x; i < Pb; i += blockDim.x) {
      if (i < nb) {
        const int32_t mi = bucket[ob + i];
        kb[i] = sel_key(mv_g[mi], mv_u[mi]);
      } else {
        kb[i] = ~0ull;
      }
    }
  }
  __syncthreads();
  block_bitonic_sort2(ka, Pa, kb, Pb);
  block_weight_prefix2(ka, na, kb, nb, c, A, B, s_red);

  // block weights at the start of sub-round s: the pass's starting weights
  // plus the changes applied in its earlier sub-rounds (pair blocks of this
  // sub-round add theirs to dbw[s] only, so every block reads the same)
  __shared__ long long s_w[2];
  if (threadIdx.x < 2) {
    const int blk = threadIdx.x == 0 ? a : b;
    long long wv = bw_base[blk];
    for (int x = 0; x < s; ++x) wv += dbw[(size_t)x * k + blk];
    s_w[threadIdx.x] = wv;
  }
  __syncthreads();
  const long long slack_a = (lmax - s_w[0] > 0 ? lmax - s_w[0] : 0) / (k - 1);
  const long long slack_b = (lmax - s_w[1] > 0 ? lmax - s_w[1] : 0) / (k - 1);
  if (threadIdx.x == 0) s_best = 0;
  __syncthreads();
  // diagonal r: i(r) = number of A-steps among the first r steps
  int best = 0;
  for (int r = threadIdx.x; r <= na + nb; r += blockDim.x) {
    int lo = r - nb > 0 ? r - nb : 0, hi = r < na ? r : na;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (A[mid] <= B[r - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    const long long x = A[lo] - B[r - lo];
    if (-slack_a <= x && x <= slack_b) best = r > best ? r : best;
  }
  best = warp_max(best);
  if (lane_id() == 0) atomicMax(&s_best, best);
  __syncthreads();
  const int r = s_best;
  int lo = r - nb > 0 ? r - nb : 0, hi = r < na ? r : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A[mid] <= B[r - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  const int ia = lo, jb = r - lo;
  if (graph) {
    // graph level: a move only rewrites Pi[u] (no pin counts to update).
    // No kernel of the sub-round reads Pi after the best moves, and the
    // moves carry their source block, so the pair block writes it here.
    unsigned long long incid = 0;
    for (int i = threadIdx.x; i < ia + jb; i += blockDim.x) {
      const bool fromA = i < ia;
      const unsigned long long key = fromA ? ka[i] : kb[i - ia];
      const int32_t u = (int32_t)(key & 0xffffffffu);
      part[u] = fromA ? b : a;
      incid += (unsigned long long)(ioff[u + 1] - ioff[u]);
    }
    incid = warp_sum(incid);
    if (lane_id() == 0 && incid) atomicAdd(moved + 2, incid);
  } else {
    // every selected move becomes ceil(deg/32) work items of at most 32
    // incident nets for k_lp_apply, which spreads them over the whole grid
    // (a block applying its own pair's moves serialises the nodes with
    // thousands of nets on coarse levels); the item's chunk index is packed
    // above the 6 bits of the source block
    for (int i = threadIdx.x; i < ia + jb; i += blockDim.x) {
      const bool fromA = i < ia;
      const unsigned long long key = fromA ? ka[i] : kb[i - ia];
      const int32_t u = (int32_t)(key & 0xffffffffu);
      const int32_t deg = ioff[u + 1] - ioff[u];
      const int32_t nch = deg > 0 ? (deg + 31) / 32 : 1;
      const int32_t slot = atomicAdd(ap_count, nch);
      for (int32_t ch = 0; ch < nch; ++ch) {
        ap_u[slot + ch] = u;
        ap_from[slot + ch] = (fromA ? a : b) | (ch << 6);
        ap_to[slot + ch] = fromA ? b : a;
      }
    }
  }
  if (threadIdx.x == 0 && ia + jb > 0) {
    // weight moved a -> b is A[ia], b -> a is B[jb]
    const long long delta = A[ia] - B[jb];
    atomic_add_i64(&dbw[(size_t)s * k + a], -delta);
    atomic_add_i64(&dbw[(size_t)s * k + b], delta);
    atomicAdd(moved, (unsigned long long)(ia + jb));
  }
}

// ------------------------------------------------------- apply (a13)

// One warp per work item (u, s, t, chunk): for the <= 32 nets e of the
// chunk: Phi(e, s) -= 1, Phi(e, t) += 1, clearing bit s of Lambda(e) when
// Phi(e, s) reaches 0 and setting bit t when Phi(e, t) leaves 0 (Algorithm
// 3's updates), and toggling the ones(e) bits of counts that reach or leave
// 1, all in net e's record; the atomic xor flips commute, so the final masks
// equal {i : Phi(e, i) > 0} and {i : Phi(e, i) = 1} whatever the order of the
// moves.  The chunk-0 item also sets Pi[u] = t.  The block weights were
// moved by the selection.
__global__ void __launch_bounds__(WARPS * 32)
k_lp_apply(const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets, int k,
           const int32_t* __restrict__ ap_u, const int32_t* __restrict__ ap_from,
           const int32_t* __restrict__ ap_to, const int32_t* __restrict__ ap_count,
           int32_t* __restrict__ part, int32_t* __restrict__ phi, int4* __restrict__ rec,
           bool wide, unsigned long long* __restrict__ moved) {
  const int32_t na = *ap_count;
  const int lane = lane_id();
  unsigned long long incid = 0;
  for (int32_t i = blockIdx.x * WARPS + warp_in_block(); i < na; i += gridDim.x * WARPS) {
    const int32_t u = ap_u[i];
    const int32_t fw = ap_from[i];
    const int s = fw & 63, ch = fw >> 6, t = ap_to[i];
    const int32_t j0 = ioff[u] + 32 * ch, j1 = min(ioff[u + 1], j0 + 32);
    const int32_t j = j0 + lane;
    if (lane == 0 && j1 > j0) incid += (unsigned long long)(j1 - j0);
    if (j < j1) {
      const int32_t e = inets[j];
      const int32_t os = atomicSub(&phi[(int64_t)e * k + s], 1);  // s: os -> os - 1
      const int32_t ot = atomicAdd(&phi[(int64_t)e * k + t], 1);  // t: ot -> ot + 1
      const unsigned long long bs = 1ull << s, bt = 1ull << t;
      unsigned long long ones_x = 0, lam_x = 0;
      if (os == 1) {
        ones_x ^= bs;
        lam_x ^= bs;
      } else if (os == 2) {
        ones_x ^= bs;
      }
      if (ot == 0) {
        ones_x ^= bt;
        lam_x ^= bt;
      } else if (ot == 1) {
        ones_x ^= bt;
      }
      flip_rec(rec, e, wide, ones_x, lam_x);
    }
    if (ch == 0 && lane == 0) part[u] = t;
  }
  const unsigned long long cv[1] = {lane == 0 ? incid : 0ull};
  block_add_counters(moved + 2, cv);
}

// Folds the pass's block-weight changes into the starting weights of the
// next pass and advances the pass index read by k_lp_count / k_lp_scatter
// (the last launch of a pass, so one captured pass can be replayed).
__global__ void k_lp_next_pass(int32_t* d_pass, long long* __restrict__ bw,
                               const long long* __restrict__ dbw, int S, int k) {
  const int i = threadIdx.x;
  if (i < k) {
    long long wv = bw[i];
    for (int x = 0; x < S; ++x) wv += dbw[(size_t)x * k + i];
    bw[i] = wv;
  }
  if (i == 0) *d_pass += 1;
}

}  // namespace

// ===================================================================== host

void project_partition(const Ctx& cx, const Level& fine, const int32_t* coarse_part,
                       int32_t* fine_part) {
  if (fine.n == 0) return;
  k_project<<<grid_for(fine.n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(fine.map.p, coarse_part,
                                                                        fine.n, fine_part);
  check_launch("project");
  if (cx.launches) *cx.launches += 1;
}

namespace {

struct PinState {
  DBuf<int32_t> phi;
  DBuf<unsigned long long> lam;
  DBuf<long long> bw;
  DBuf<int32_t> tiles;
};

// Phi, Lambda (unless counts == false: graph levels in label propagation)
// and the block weights of a partition.
void build_pin_state(const Ctx& cx, const Level& L, int k, const int32_t* part, PinState& st,
                     bool counts = true) {
  st.bw.alloc(&cx.alloc, (size_t)k);
  HG_CUDA(cudaMemsetAsync(st.bw.p, 0, st.bw.bytes(), cx.stream));
  if (counts) {
    st.phi.alloc(&cx.alloc, (size_t)L.m * k + 1);
    st.lam.alloc(&cx.alloc, (size_t)L.m + 1);
    HG_CUDA(cudaMemsetAsync(st.phi.p, 0, st.phi.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(st.lam.p, 0, st.lam.bytes(), cx.stream));
  }
  if (counts && L.p > 0) {
    st.tiles.alloc(&cx.alloc, (size_t)num_pin_tiles(L.p) + 1);
    build_tile_index(cx, L.eoff.p, L.m, L.p, st.tiles.p);
    k_pin_counts<<<grid_for(num_pin_tiles(L.p), 1, cx.num_sms, 8), PIN_TILE_THREADS, 0,
                   cx.stream>>>(L.eoff.p, L.pins.p, st.tiles.p, L.m, L.p, part, k, st.phi.p,
                                st.lam.p);
    check_launch("pin_counts");
  }
  k_block_weights<<<grid_for(L.n, 256, cx.num_sms, 4), 256, 0, cx.stream>>>(part, L.c.p, L.n, k,
                                                                          st.bw.p);
  check_launch("block_weights");
  if (cx.launches) *cx.launches += 3;
}

int64_t objective_of_graph(const Ctx& cx, const Level& L, const int32_t* part) {
  DBuf<unsigned long long> acc;
  acc.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), cx.stream));
  if (L.m > 0) {
    k_objective_graph<<<grid_for(L.m, 256, cx.num_sms, 4), 256, 0, cx.stream>>>(
        L.eoff.p, L.pins.p, L.w.p, part, L.m, acc.p);
    check_launch("objective_graph");
    if (cx.launches) *cx.launches += 1;
  }
  return read_i64(cx, reinterpret_cast<const int64_t*>(acc.p));
}

int64_t objective_from_records(const Ctx& cx, const Level& L, const int4* rec, bool wide) {
  DBuf<unsigned long long> acc;
  acc.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), cx.stream));
  if (L.m > 0) {
    k_objective_rec<<<grid_for(L.m, 256, cx.num_sms, 4), 256, 0, cx.stream>>>(rec, L.m, wide,
                                                                              acc.p);
    check_launch("objective_rec");
    if (cx.launches) *cx.launches += 1;
  }
  return read_i64(cx, reinterpret_cast<const int64_t*>(acc.p));
}

int64_t objective_from_lambda(const Ctx& cx, const Level& L, const unsigned long long* lam) {
  DBuf<unsigned long long> acc;
  acc.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), cx.stream));
  if (L.m > 0) {
    k_objective<<<grid_for(L.m, 256, cx.num_sms, 4), 256, 0, cx.stream>>>(lam, L.w.p, L.m, acc.p);
    check_launch("objective");
    if (cx.launches) *cx.launches += 1;
  }
  return read_i64(cx, reinterpret_cast<const int64_t*>(acc.p));
}

}  // namespace

int64_t objective_of(const Ctx& cx, const Level& L, int k, const int32_t* part) {
  PinState st;
  build_pin_state(cx, L, k, part, st);
  return objective_from_lambda(cx, L, st.lam.p);
}

namespace {

__global__ void k_check_part(const int32_t* __restrict__ part, int32_t n, int k, int32_t* status) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    if (part[u] < 0 || part[u] >= k) dev_fail(status, DEV_BAD_INPUT);
}

}  // namespace

void validate_partition(const Ctx& cx, const int32_t* part, int32_t n, int k) {
  if (n <= 0) return;
  k_check_part<<<grid_for(n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(part, n, k, cx.d_status);
  check_launch("check_part");
  if (cx.launches) *cx.launches += 1;
  check_status(cx);
}

void device_pin_counts(const Ctx& cx, const Level& L, int k, const int32_t* part,
                       DBuf<int32_t>& phi, DBuf<unsigned long long>& lam) {
  PinState st;
  build_pin_state(cx, L, k, part, st);
  phi = std::move(st.phi);
  lam = std::move(st.lam);
}

void pin_counts_of(const Ctx& cx, const Level& L, int k, const int32_t* part, int32_t* phi,
                   uint64_t* lambda, int64_t* bw) {
  PinState st;
  build_pin_state(cx, L, k, part, st);
  if (phi && L.m)
    HG_CUDA(cudaMemcpyAsync(phi, st.phi.p, sizeof(int32_t) * (size_t)L.m * k,
                            cudaMemcpyDeviceToHost, cx.stream));
  if (lambda && L.m)
    HG_CUDA(cudaMemcpyAsync(lambda, st.lam.p, sizeof(uint64_t) * (size_t)L.m,
                            cudaMemcpyDeviceToHost, cx.stream));
  if (bw)
    HG_CUDA(cudaMemcpyAsync(bw, st.bw.p, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost,
                            cx.stream));
  check_status(cx);
}

namespace {

// The instantiated graph of one LP pass is kept per host thread and updated
// in place (cudaGraphExecUpdate) for every new level and handle: its
// topology depends on S only, and instantiating anew for every level is
// costly, the more so when several host threads (executor slots) do it at
// once.  Captures run on a private stream of the thread, since the caller's
// stream may be the legacy default stream, which cannot be captured.  Every
// use of the graph ends with a host wait before the next update.
struct PassGraphCache {
  int device = -1;
  int S = -1;
  cudaStream_t capture = nullptr;
  cudaStream_t side = nullptr;  // second branch of the captured pass
  cudaEvent_t fork = nullptr, join = nullptr;
  // kernel timing: 4 events per sub-round recorded by event nodes of the
  // captured pass (before the best-move kernels, after them, after the
  // selection, after the application)
  std::vector<cudaEvent_t> tev;
  cudaGraphExec_t exec = nullptr;
  void reset() {
    for (cudaEvent_t e : tev) cudaEventDestroy(e);
    tev.clear();
    if (exec) cudaGraphExecDestroy(exec);
    if (capture) cudaStreamDestroy(capture);
    if (side) cudaStreamDestroy(side);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    exec = nullptr;
    capture = side = nullptr;
    fork = join = nullptr;
    device = S = -1;
  }
  // Makes exec run `graph` (which it consumes) and returns it.
  cudaGraphExec_t bind(cudaGraph_t graph, int subrounds) {
    if (exec && S == subrounds) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess) {
        cudaGraphDestroy(graph);
        return exec;
      }
      cudaGetLastError();  // topology changed: instantiate anew
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      exec = nullptr;
      HG_CUDA(ie);
    }
    S = subrounds;
    return exec;
  }
  // At least `count` timing events (created with timing enabled).
  void timing_events(size_t count) {
    while (tev.size() < count) {
      cudaEvent_t e = nullptr;
      HG_CUDA(cudaEventCreate(&e));
      tev.push_back(e);
    }
  }
  ~PassGraphCache() { reset(); }
};

PassGraphCache& pass_graph_cache(const Ctx& cx) {
  thread_local PassGraphCache cache;
  int dev = 0;
  HG_CUDA(cudaGetDevice(&dev));
  if (cache.device != dev) {
    cache.reset();
    HG_CUDA(cudaStreamCreateWithFlags(&cache.capture, cudaStreamNonBlocking));
    HG_CUDA(cudaStreamCreateWithFlags(&cache.side, cudaStreamNonBlocking));
    HG_CUDA(cudaEventCreateWithFlags(&cache.fork, cudaEventDisableTiming));
    HG_CUDA(cudaEventCreateWithFlags(&cache.join, cudaEventDisableTiming));
    cache.device = dev;
  }
  (void)cx;
  return cache;
}

}  // namespace

LPResult lp_refine_level(const Ctx& cx, const Level& L, int level_index, int k, int eps_ppm,
                         int max_passes, int S, uint64_t seed, int64_t total_node_weight,
                         int lp_block_deg, int32_t* part, RefineCounters& rc) {
  LPResult res;
  PinState st;
  {
    EventTimer tm(cx, &rc.ms_phi);
    build_pin_state(cx, L, k, part, st, !L.graph);
  }
  // packed net records (hypergraph levels); Lambda is then kept in them only
  const bool wide = k > 32;
  DBuf<int4> rec;
  if (!L.graph) {
    EventTimer tm(cx, &rc.ms_phi);
    rec.alloc(&cx.alloc, (size_t)std::max<int32_t>(L.m, 1) * (wide ? 2 : 1));
    if (L.m > 0) {
      k_net_records<<<grid_for(L.m, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
          st.phi.p, st.lam.p, L.w.p, L.m, k, wide, rec.p);
      check_launch("net_records");
      if (cx.launches) *cx.launches += 1;
    }
    st.lam.release();
  }
  const int64_t per_block = (total_node_weight + k - 1) / k;
  const long long lmax = (long long)(per_block * (1000000 + (int64_t)eps_ppm) / 1000000);
  const int kk = k * k;
  const int32_t n = L.n;

  DBuf<int32_t> list, sr_cnt, sr_fill, sr_off, mv_u, mv_to, bucket, dcnt, dfill, doff, words,
      ap_u, ap_from, ap_to;
  DBuf<long long> mv_g, gpre, dbw;
  DBuf<unsigned long long> gkeys, counters;
  const size_t ncap = (size_t)n + 1;
  list.alloc(&cx.alloc, ncap);
  sr_cnt.alloc(&cx.alloc, (size_t)2 * S);
  sr_fill.alloc(&cx.alloc, (size_t)2 * S);
  sr_off.alloc(&cx.alloc, (size_t)2 * S + 1);
  mv_u.alloc(&cx.alloc, ncap);
  mv_to.alloc(&cx.alloc, ncap);
  mv_g.alloc(&cx.alloc, ncap);
  bucket.alloc(&cx.alloc, ncap);
  // block-weight change of every sub-round of a pass (k per sub-round)
  dbw.alloc(&cx.alloc, (size_t)S * k);
  // work items of the application: one per 32 incident nets of a moved node
  // (graph levels: the selection rewrites Pi itself, no application launch)
  const size_t acap = L.graph ? 1 : ncap + (size_t)(L.p / 32) + 1;
  ap_u.alloc(&cx.alloc, acap);
  ap_from.alloc(&cx.alloc, acap);
  ap_to.alloc(&cx.alloc, acap);
  gkeys.alloc(&cx.alloc, 2 * ncap + 2);
  // k <= 16: per-direction key lists filled by the best-move kernels, read by
  // the pair blocks instead of gathering the sub-round's whole move list
  const int32_t dcap = k <= SEL_GATHER_K ? SEL_DIR_KEYS : 0;
  DBuf<unsigned long long> dkeys;
  if (dcap > 0) dkeys.alloc(&cx.alloc, (size_t)kk * dcap);
  gpre.alloc(&cx.alloc, ncap + (size_t)kk + 2);
  dcnt.alloc(&cx.alloc, (size_t)S * kk);
  dfill.alloc(&cx.alloc, (size_t)S * kk);
  doff.alloc(&cx.alloc, (size_t)kk + 1);
  words.alloc(&cx.alloc, (size_t)S * SW_WORDS);
  // [0] nodes moved in the pass, [1] incidences read by the gain kernels,
  // [2] incidences of the moved nodes
  counters.alloc(&cx.alloc, 4);
  HG_CUDA(cudaMemsetAsync(counters.p, 0, counters.bytes(), cx.stream));

  const int nodes_per_sr = (int)((n + S - 1) / S);
  const int g_gain = grid_for(nodes_per_sr, WARPS, cx.num_sms, 16);
  // warp-class nodes of hypergraph levels with k <= 16 and a small mean
  // degree go to lane groups
  const bool sub_class =
      !L.graph && k <= GAIN_REDUCE_K && L.p <= (int64_t)SUB_MEAN_DEG * std::max<int32_t>(n, 1);
  const int g_gain_sub = grid_for(nodes_per_sr, WARPS * (32 / SUB_G), cx.num_sms, 16);
  const int g_gain_block = grid_for(nodes_per_sr, 1, cx.num_sms, 8);
  const int g_bucket = grid_for(nodes_per_sr, 256, cx.num_sms, 4);
  const int g_apply = grid_for((int64_t)acap / S + 1, WARPS, cx.num_sms, 16);
  const int g_sel = k * (k - 1) / 2;
  const int g_nodes = grid_for(n, 256, cx.num_sms, 4);
  KernelTimer gain_timer(cx);
  // nodes above the warp class exist at this level?
  GainArgs G;
  auto launch_gain_warp = [&](cudaStream_t st) {
    if (sub_class) k_lp_gain_sub<<<g_gain_sub, WARPS * 32, 0, st>>>(G);
    else k_lp_gain_warp<<<g_gain, WARPS * 32, 0, st>>>(G);
  };
  G.ioff = L.ioff.p;
  G.inets = L.inets.p;
  G.rec = rec.p;
  G.wide = wide;
  G.part = part;
  G.k = k;
  G.list = list.p;
  G.sr_off = sr_off.p;
  G.mv_u = mv_u.p;
  G.mv_to = mv_to.p;
  G.mv_g = mv_g.p;
  G.dkeys = dkeys.p;
  G.dcap = dcap;
  G.work = counters.p + 1;
  G.graph = L.graph;
  G.adj = L.adj.p;

  // One pass = the sub-round lists, then per sub-round best moves, pair
  // bucketing and selection, application.  Every launch has a fixed geometry
  // and reads its sizes on the device, so a pass is captured once per level
  // as a CUDA graph and replayed; with phase timing on (which synchronizes
  // around phases) the launches are issued directly.
  DBuf<int32_t> d_pass;
  d_pass.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(d_pass.p, 0, sizeof(int32_t), cx.stream));
  const bool use_graph = !cx.timing;
  const size_t sel_bytes = sel_smem_bytes(sel_cap_for(k));
  {
    static std::once_flag once;
    std::call_once(once, [] {
      const int bytes = (int)sel_smem_bytes(sel_cap_for(2));
      HG_CUDA(cudaFuncSetAttribute(k_lp_select<false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      HG_CUDA(cudaFuncSetAttribute(k_lp_select<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    });
  }
  // k <= SEL_GATHER_K: the pair blocks gather their own moves (k (k - 1) / 2
  // blocks each reading the move list), no bucket pass
  const bool gather = k <= SEL_GATHER_K;
  const int per_pass_launches = 3 + (3 + (gather ? 0 : 1) + (L.graph ? 0 : 1)) * S;
  // side != nullptr: the two best-move kernels of a sub-round are captured
  // as parallel branches (they only meet in atomics on the move list), so
  // the few high-degree nodes of the block class overlap with the warp class
  // kernel timing inside the captured pass: event nodes around each phase
  // of every sub-round, read after each pass (the pass ends with a host wait)
  const bool graph_events = use_graph && cx.kernel_timing;
  auto mark = [&](const PassGraphCache* fj, cudaStream_t sm, int s, int which) {
    if (graph_events && fj)
      HG_CUDA(cudaEventRecordWithFlags(fj->tev[(size_t)4 * s + which], sm,
                                       cudaEventRecordExternal));
  };
  auto enqueue_pass = [&](bool timed, cudaStream_t sm, const PassGraphCache* fj) {
    HG_CUDA(cudaMemsetAsync(sr_cnt.p, 0, sr_cnt.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(sr_fill.p, 0, sr_fill.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(dcnt.p, 0, dcnt.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(dfill.p, 0, dfill.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(words.p, 0, words.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(counters.p, 0, counters.bytes(), sm));
    HG_CUDA(cudaMemsetAsync(dbw.p, 0, dbw.bytes(), sm));
    {
      EventTimer tm(cx, timed ? &rc.ms_gain : nullptr);
      k_lp_count<<<g_nodes, 256, 2 * S * sizeof(int32_t), sm>>>(L.ioff.p, n, seed,
                                                                      level_index, d_pass.p, S,
                                                                      lp_block_deg, sr_cnt.p);
      check_launch("lp_count");
      k_lp_scatter<<<g_nodes, 256, (2 * S + 1) * sizeof(int32_t), sm>>>(
          L.ioff.p, n, seed, level_index, d_pass.p, S, lp_block_deg, sr_cnt.p, sr_fill.p,
          sr_off.p, list.p);
      check_launch("lp_scatter");
    }
    for (int s = 0; s < S; ++s) {
      int32_t* w_s = words.p + (size_t)s * SW_WORDS;
      int32_t* dc_s = dcnt.p + (size_t)s * kk;
      int32_t* df_s = dfill.p + (size_t)s * kk;
      G.s = s;
      G.dcount = dc_s;
      G.words = w_s;
      {
        EventTimer tm(cx, timed ? &rc.ms_gain : nullptr);
        if (fj) {
          mark(fj, sm, s, 0);
          HG_CUDA(cudaEventRecord(fj->fork, sm));
          HG_CUDA(cudaStreamWaitEvent(fj->side, fj->fork, 0));
          k_lp_gain_block<<<g_gain_block, GAIN_BLOCK_WARPS * 32, 0, fj->side>>>(G);
          check_launch("lp_gain_block");
          launch_gain_warp(sm);
          check_launch("lp_gain_warp");
          HG_CUDA(cudaEventRecord(fj->join, fj->side));
          HG_CUDA(cudaStreamWaitEvent(sm, fj->join, 0));
          mark(fj, sm, s, 1);
        } else {
          if (timed) gain_timer.begin();
          launch_gain_warp(sm);
          if (timed) gain_timer.end();
          check_launch("lp_gain_warp");
          if (timed) gain_timer.begin();
          k_lp_gain_block<<<g_gain_block, GAIN_BLOCK_WARPS * 32, 0, sm>>>(G);
          if (timed) gain_timer.end();
          check_launch("lp_gain_block");
        }
        if (!fj) rc.lp_gain_launches += 2;
      }
      {
        EventTimer tm(cx, timed ? &rc.ms_select : nullptr);
        if (!gather) {
          k_lp_bucket<<<g_bucket, 256, (kk + 1) * sizeof(int32_t), sm>>>(
              mv_to.p, k, dc_s, df_s, doff.p, w_s, bucket.p);
          check_launch("lp_bucket");
        }
        auto sel = gather ? k_lp_select<true> : k_lp_select<false>;
        sel<<<g_sel, SEL_THREADS, sel_bytes, sm>>>(
            L.ioff.p, L.inets.p, bucket.p, doff.p, dc_s, mv_u.p, mv_to.p, mv_g.p, L.c.p, st.bw.p,
            dbw.p, s, lmax, k, gkeys.p, gpre.p, w_s, part, counters.p, ap_u.p,
            ap_from.p, ap_to.p, w_s + SW_APPROVED, L.graph, dkeys.p, dcap);
        check_launch("lp_select");
        mark(fj, sm, s, 2);
      }
      {
        EventTimer tm(cx, timed ? &rc.ms_apply : nullptr);
        if (!L.graph) {
          k_lp_apply<<<g_apply, WARPS * 32, 0, sm>>>(L.ioff.p, L.inets.p, k, ap_u.p, ap_from.p,
                                                      ap_to.p, w_s + SW_APPROVED, part, st.phi.p,
                                                      rec.p, wide, counters.p);
          check_launch("lp_apply");
        }
        mark(fj, sm, s, 3);
      }
    }
    k_lp_next_pass<<<1, 64, 0, sm>>>(d_pass.p, st.bw.p, dbw.p, S, k);
    check_launch("lp_next_pass");
  };
  cudaGraphExec_t exec = nullptr;
  PassGraphCache* gcp = nullptr;
  if (use_graph && max_passes > 0) {
    PassGraphCache& gc = pass_graph_cache(cx);
    gcp = &gc;
    if (graph_events) gc.timing_events((size_t)4 * S);
    cudaGraph_t graph = nullptr;
    HG_CUDA(cudaStreamBeginCapture(gc.capture, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_pass(false, gc.capture, &gc);
    } catch (...) {
      cudaStreamEndCapture(gc.capture, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    HG_CUDA(cudaStreamEndCapture(gc.capture, &graph));
    exec = gc.bind(graph, S);
  }
  for (int pass = 0; pass < max_passes; ++pass) {
    if (exec) {
      HG_CUDA(cudaGraphLaunch(exec, cx.stream));
      rc.lp_gain_launches += 2 * S;
    } else {
      enqueue_pass(true, cx.stream, nullptr);
    }
    if (cx.launches) *cx.launches += per_pass_launches;
    unsigned long long hc[3];
    wait_stream(cx);  // the pass is done, so the graph is idle before its next update
    HG_CUDA(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, cx.stream));
    check_status(cx);
    if (graph_events) {
      double* acc[3] = {&rc.ms_gain_kernels, &rc.ms_select_kernels, &rc.ms_apply_kernels};
      for (int s = 0; s < S; ++s)
        for (int ph = 0; ph < 3; ++ph) {
          float ms = 0;
          if (cudaEventElapsedTime(&ms, gcp->tev[(size_t)4 * s + ph],
                                   gcp->tev[(size_t)4 * s + ph + 1]) == cudaSuccess) {
            *acc[ph] += ms;
          } else {
            cudaGetLastError();
            rc.timing_failures += 1;
          }
        }
    }
    res.passes = pass + 1;
    res.moves += (int64_t)hc[0];
    rc.lp_incidences += (int64_t)hc[1];
    rc.lp_moved_incidences += (int64_t)hc[2];
    if (hc[0] == 0) break;
  }
  rc.ms_gain_kernels += gain_timer.flush();
  rc.lp_nodes += (int64_t)res.passes * n;
  rc.lp_passes += res.passes;
  {
    EventTimer tm(cx, &rc.ms_objective);
    res.objective = L.graph ? objective_of_graph(cx, L, part) : objective_from_records(cx, L, rec.p, wide);
  }
  return res;
}

}  // namespace hgk
