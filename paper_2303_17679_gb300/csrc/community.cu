// Community detection before coarsening (Sec. 4 "Community-Aware Coarsening",
// Sec. 11 "Deterministic Louvain Method") on the device.
//
// The hypergraph becomes its bipartite graph: a vertex per node (0..n-1) and
// per net (n + e), an edge {v, n + e} for every pin with weight
// floor(w(e) * 2^20 / |e|), an integer reading of the fractional w(e) / |e|
// model.  Every sum below is an integer sum, so the cluster volumes that the
// paper aggregates in a fixed order are exact here whatever the order of the
// atomics, and every decision is bit-identical from run to run.
//
// The Louvain method, per level: clusters start as singletons; up to
// LV_ROUNDS rounds of S synchronous sub-rounds (vertex i is in sub-round
// mix64(seed ^ 2^62 ^ level<<32 ^ (round+1)<<48 ^ i) mod S); in a sub-round
// every listed vertex picks, from the state at the sub-round's start, the
// neighbouring cluster C maximising s(C) = 2W k_{i,C} - k_i vol(C) (128-bit
// integers, ties to the smaller id) and moves when s(C) exceeds its own
// cluster's s(A) = 2W k_{i,A} - k_i (vol(A) - k_i); all moves are applied
// (no weight limit), volumes updated with integer atomics.  A round moving
// fewer than 1 % of the vertices ends the level; a level without any move
// ends the detection.  Otherwise the clusters are aggregated (coarse vertex
// = rank of the cluster id; edges between clusters summed, edges inside a
// cluster added to its self-loop weight) and the next level starts.
//
// Layout per level: CSR with int64 offsets, int32 neighbours, int64 weights,
// int64 self-loop weights, degrees k and volumes.  Per round the vertices
// are listed by (sub-round, class): class 0 (degree <= LV_SMALL) is decided
// by one warp per vertex with a shared-memory table of its neighbouring
// clusters; class 1 inserts its edges into per-vertex tables in global
// memory with one thread per edge over the whole grid, then one block per
// vertex takes the best entry.  Aggregation uses the same global tables, one
// per coarse vertex.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace hgk {

namespace {

constexpr int LV_ROUNDS = 5;
constexpr int LV_LEVELS = 32;
constexpr int LV_SMALL = 256;          // class 0: degree <= LV_SMALL
constexpr int LV_SLOTS = 2 * LV_SMALL;  // shared slots per warp (load <= 1/2)
constexpr int LV_WARPS = 8;
constexpr int LV_ARGMAX_THREADS = 256;
constexpr int32_t LV_EMPTY = -1;

using i128 = __int128;

__device__ __forceinline__ int subround_louvain(uint64_t seed, int level, int round, int64_t i,
                                                int S) {
  const uint64_t x = seed ^ (1ull << 62) ^ ((uint64_t)(uint32_t)level << 32) ^
                     ((uint64_t)(uint32_t)(round + 1) << 48) ^ (uint64_t)(uint32_t)i;
  return (int)(mix64(x) % (uint64_t)S);
}

// ------------------------------------------------------------ level 0

// Bipartite CSR from the hypergraph: node v's edges are its incidences
// (positions ioff[v]..), net e's edges its pins (positions p + eoff[e]..).
// One thread per incidence j = (v, e), q = ipin[j] the pin position.
__global__ void k_lv_bipartite(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                               const int32_t* __restrict__ w, const int32_t* __restrict__ inets,
                               const int32_t* __restrict__ ipin, int32_t n, int64_t p,
                               int32_t* __restrict__ adj, long long* __restrict__ aw) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = inets[j];
    const int32_t q = ipin[j];
    const int32_t size = eoff[e + 1] - eoff[e];
    const long long we = (long long)(((unsigned long long)w[e] << 20) / (unsigned long long)size);
    adj[j] = n + e;
    aw[j] = we;
    adj[p + q] = pins[q];
    aw[p + q] = we;
  }
}

__global__ void k_lv_offsets(const int32_t* __restrict__ ioff, const int32_t* __restrict__ eoff,
                             int32_t n, int32_t m, int64_t p, long long* __restrict__ off) {
  const int64_t V = (int64_t)n + m;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= V;
       i += (int64_t)gridDim.x * blockDim.x)
    off[i] = i <= n ? (long long)ioff[i] : (long long)(p + eoff[i - n]);
}

// k_i = 2 self_i + sum of i's edge weights (a warp per vertex); W2 = sum k_i.
__global__ void k_lv_degrees(const long long* __restrict__ off, const long long* __restrict__ aw,
                             const long long* __restrict__ self, int64_t V,
                             long long* __restrict__ k, unsigned long long* __restrict__ total) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  long long acc = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < V; i += nw) {
    long long s = 0;
    for (long long q = off[i] + lane_id(); q < off[i + 1]; q += 32) s += aw[q];
    s = warp_sum(s);
    s += 2 * self[i];
    if (lane_id() == 0) k[i] = s;
    acc += s;
  }
  if (lane_id() == 0 && acc) atomicAdd(total, (unsigned long long)acc);
}

__global__ void k_lv_init(int64_t V, const long long* __restrict__ k, int32_t* __restrict__ cl,
                          long long* __restrict__ vol) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    cl[i] = (int32_t)i;
    vol[i] = k[i];
  }
}

// ------------------------------------------------------------ lists

// key = sub-round * 2 + class of every vertex with at least one edge.
__device__ __forceinline__ int lv_key(const long long* off, uint64_t seed, int level, int round,
                                      int64_t i, int S) {
  const long long deg = off[i + 1] - off[i];
  if (deg == 0) return -1;  // no neighbouring cluster: never moves
  return subround_louvain(seed, level, round, i, S) * 2 + (deg > LV_SMALL ? 1 : 0);
}

__global__ void k_lv_count(const long long* __restrict__ off, int64_t V, uint64_t seed, int level,
                           int round, int S, int32_t* __restrict__ cnt) {
  extern __shared__ int32_t s_cnt[];
  for (int i = threadIdx.x; i < 2 * S; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int key = lv_key(off, seed, level, round, i, S);
    if (key >= 0) atomicAdd(&s_cnt[key], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * S; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

// Scatters vertices by key; the list order inside a key is unspecified
// (every later step is a set operation or an integer sum).
__global__ void k_lv_scatter(const long long* __restrict__ off, int64_t V, uint64_t seed,
                             int level, int round, int S, const int32_t* __restrict__ koff,
                             int32_t* __restrict__ fill, int32_t* __restrict__ list) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < V; b += stride) {
    const int64_t i = b + lane_id();
    const bool valid = i < V;
    const int key = valid ? lv_key(off, seed, level, round, i, S) : -1;
    const int32_t slot = warp_claim_slot(fill, key, __ballot_sync(FULL, valid));
    if (slot >= 0) list[koff[key] + slot] = (int32_t)i;
  }
}

// Degrees and global table sizes (power of two >= 2 deg + 2) along a list.
__global__ void k_lv_list_sizes(const int32_t* __restrict__ list, int32_t cnt,
                                const long long* __restrict__ off, int32_t* __restrict__ deg,
                                int32_t* __restrict__ tsize) {
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < cnt; x += gridDim.x * blockDim.x) {
    const int32_t i = list[x];
    const int32_t d = (int32_t)(off[i + 1] - off[i]);
    deg[x] = d;
    if (tsize) {
      // at most 2^30 slots: a larger vertex fills its table, which the
      // insertion reports as a full table
      int64_t c = 4;
      while (c < 2 * (int64_t)d + 2 && c < (1ll << 30)) c <<= 1;
      tsize[x] = (int32_t)c;
    }
  }
}

// ------------------------------------------------------------ tables

// Adds `val` to `key`'s entry of a global table (keys LV_EMPTY when free).
__device__ __forceinline__ bool table_add(int32_t* keys, long long* vals, uint32_t mask,
                                          int32_t key, long long val) {
  uint32_t h = ((uint32_t)key * 0x9E3779B1u) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t k = keys[h];
    if (k == LV_EMPTY) {
      const int32_t old = atomicCAS(&keys[h], LV_EMPTY, key);
      k = old == LV_EMPTY ? key : old;
    }
    if (k == key) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&vals[h]), (unsigned long long)val);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

// Candidate (score, cluster) comparison: larger score, ties to smaller id.
struct Cand {
  i128 s;
  int32_t c;
};

__device__ __forceinline__ void cand_better(Cand& a, const Cand& b) {
  if (b.c >= 0 && (a.c < 0 || b.s > a.s || (b.s == a.s && b.c < a.c))) a = b;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& x, int d) {
  Cand y;
  const unsigned long long lo = (unsigned long long)x.s;
  const long long hi = (long long)(x.s >> 64);
  const unsigned long long ylo = __shfl_xor_sync(FULL, lo, d);
  const long long yhi = __shfl_xor_sync(FULL, hi, d);
  y.s = ((i128)yhi << 64) | (i128)ylo;
  y.c = __shfl_xor_sync(FULL, x.c, d);
  return y;
}

__device__ __forceinline__ void warp_best(Cand& x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) cand_better(x, shfl_cand(x, d));
}

struct LvArgs {
  const long long* off;
  const int32_t* adj;
  const long long* aw;
  const long long* k;
  const int32_t* cl;
  const long long* vol;
  long long W2;
  const int32_t* list;
  int32_t* mv_v;
  int32_t* mv_to;
  int32_t* words;  // [0] moves of the sub-round
  int32_t* status;
};

// The move of vertex i from its own cluster's entry kia and the best other
// candidate: moves iff s(best) > s(own).
__device__ __forceinline__ void lv_emit(const LvArgs& A, int32_t i, long long kia, const Cand& best) {
  const int32_t own = A.cl[i];
  const long long ki = A.k[i];
  const i128 s_own = (i128)A.W2 * kia - (i128)ki * (A.vol[own] - ki);
  if (best.c >= 0 && best.s > s_own) {
    const int32_t slot = atomicAdd(&A.words[0], 1);
    A.mv_v[slot] = i;
    A.mv_to[slot] = best.c;
  }
}

// Class 0: one warp per vertex, shared table of LV_SLOTS entries.
__global__ void __launch_bounds__(LV_WARPS * 32) k_lv_small(LvArgs A, int32_t lo, int32_t hi) {
  __shared__ int32_t s_key[LV_WARPS][LV_SLOTS];
  __shared__ long long s_val[LV_WARPS][LV_SLOTS];
  const int wv = warp_in_block(), lane = lane_id();
  int32_t* keys = s_key[wv];
  long long* vals = s_val[wv];
  for (int x = lane; x < LV_SLOTS; x += 32) {
    keys[x] = LV_EMPTY;
    vals[x] = 0;
  }
  __syncwarp();
  for (int32_t x = lo + blockIdx.x * LV_WARPS + wv; x < hi; x += gridDim.x * LV_WARPS) {
    const int32_t i = A.list[x];
    const long long b = A.off[i], e = A.off[i + 1];
    for (long long q = b + lane; q < e; q += 32) {
      const int32_t C = A.cl[A.adj[q]];
      if (!table_add(keys, vals, LV_SLOTS - 1, C, A.aw[q])) dev_fail(A.status, DEV_HASH_FULL);
    }
    __syncwarp();
    const int32_t own = A.cl[i];
    const long long ki = A.k[i];
    Cand best{0, -1};
    long long kia = 0;
    for (int s = lane; s < LV_SLOTS; s += 32) {
      const int32_t C = keys[s];
      if (C == LV_EMPTY) continue;
      const long long kic = vals[s];
      keys[s] = LV_EMPTY;
      vals[s] = 0;
      if (C == own) {
        kia = kic;
        continue;
      }
      cand_better(best, Cand{(i128)A.W2 * kic - (i128)ki * A.vol[C], C});
    }
    warp_best(best);
    kia = warp_sum(kia);
    if (lane == 0) lv_emit(A, i, kia, best);
    __syncwarp();
  }
}

// Class 1, step 1: one thread per edge of the listed vertices [lo, hi):
// lpre = exclusive prefix of their degrees along the list, toff = offsets of
// their global tables (relative to tbase).
__global__ void k_lv_big_insert(LvArgs A, int32_t lo, int32_t hi, const long long* __restrict__ lpre,
                                const long long* __restrict__ toff, long long tbase,
                                const int32_t* __restrict__ tsize, int32_t* __restrict__ tkey,
                                long long* __restrict__ tval) {
  const long long base = lpre[lo], cnt = lpre[hi] - base;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    const long long y = base + t;
    int32_t a = lo, b = hi - 1;  // largest x in [lo, hi) with lpre[x] <= y
    while (a < b) {
      const int32_t mid = (a + b + 1) >> 1;
      if (lpre[mid] <= y) a = mid;
      else b = mid - 1;
    }
    const int32_t i = A.list[a];
    const long long q = A.off[i] + (y - lpre[a]);
    const long long tb = toff[a] - tbase;
    if (!table_add(tkey + tb, tval + tb, (uint32_t)tsize[a] - 1, A.cl[A.adj[q]], A.aw[q]))
      dev_fail(A.status, DEV_HASH_FULL);
  }
}

// Class 1, step 2: one block per listed vertex, best entry of its table
// (cleared on the way for the next sub-round).
__global__ void __launch_bounds__(LV_ARGMAX_THREADS)
k_lv_big_argmax(LvArgs A, int32_t lo, int32_t hi, const long long* __restrict__ toff,
                long long tbase, const int32_t* __restrict__ tsize, int32_t* __restrict__ tkey,
                long long* __restrict__ tval) {
  __shared__ long long s_lo[32], s_hi[32], s_kia[32];
  __shared__ int32_t s_c[32];
  for (int32_t x = lo + blockIdx.x; x < hi; x += gridDim.x) {
    const int32_t i = A.list[x];
    const int32_t own = A.cl[i];
    const long long ki = A.k[i];
    const long long tb = toff[x] - tbase;
    Cand best{0, -1};
    long long kia = 0;
    for (int32_t s = threadIdx.x; s < tsize[x]; s += blockDim.x) {
      const int32_t C = tkey[tb + s];
      if (C == LV_EMPTY) continue;
      const long long kic = tval[tb + s];
      tkey[tb + s] = LV_EMPTY;
      tval[tb + s] = 0;
      if (C == own) {
        kia = kic;
        continue;
      }
      cand_better(best, Cand{(i128)A.W2 * kic - (i128)ki * A.vol[C], C});
    }
    warp_best(best);
    kia = warp_sum(kia);
    if (lane_id() == 0) {
      s_lo[warp_in_block()] = (long long)(unsigned long long)best.s;
      s_hi[warp_in_block()] = (long long)(best.s >> 64);
      s_c[warp_in_block()] = best.c;
      s_kia[warp_in_block()] = kia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b{0, -1};
      long long ka = 0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) {
        cand_better(b, Cand{((i128)s_hi[wv] << 64) | (i128)(unsigned long long)s_lo[wv], s_c[wv]});
        ka += s_kia[wv];
      }
      lv_emit(A, i, ka, b);
    }
    __syncthreads();
  }
}

// Applies the sub-round's moves: cluster and integer volume updates.
__global__ void k_lv_apply(const int32_t* __restrict__ mv_v, const int32_t* __restrict__ mv_to,
                           const int32_t* __restrict__ words, const long long* __restrict__ k,
                           int32_t* __restrict__ cl, long long* __restrict__ vol,
                           unsigned long long* __restrict__ moved) {
  const int32_t nm = words[0];
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nm; x += gridDim.x * blockDim.x) {
    const int32_t i = mv_v[x], to = mv_to[x];
    const long long ki = k[i];
    atomic_add_i64(&vol[cl[i]], -ki);
    atomic_add_i64(&vol[to], ki);
    cl[i] = to;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && nm) atomicAdd(moved, (unsigned long long)nm);
}

// ------------------------------------------------------------ aggregation

__global__ void k_lv_used(const int32_t* __restrict__ cl, int64_t V, int32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[cl[i]] = 1;
}

// cv[i] = coarse vertex of i; member counts per coarse vertex.
__global__ void k_lv_coarse_of(const int32_t* __restrict__ cl, const int32_t* __restrict__ cid,
                               int64_t V, int32_t* __restrict__ cv, int32_t* __restrict__ mcnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cid[cl[i]];
    cv[i] = c;
    atomicAdd(&mcnt[c], 1);
  }
}

__global__ void k_lv_members(const int32_t* __restrict__ cv, int64_t V,
                             const int32_t* __restrict__ moff, int32_t* __restrict__ mfill,
                             int32_t* __restrict__ members) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cv[i];
    members[moff[c] + atomicAdd(&mfill[c], 1)] = (int32_t)i;
  }
}

// Per coarse vertex: the sum of its members' degrees in the edge lists (a
// bound on its coarse degree) and of their self-loop weights.
__global__ void k_lv_coarse_bounds(const int32_t* __restrict__ members, const int32_t* __restrict__ moff,
                                   int32_t V2, const long long* __restrict__ off,
                                   const long long* __restrict__ self,
                                   long long* __restrict__ bound, long long* __restrict__ self2) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < V2; c += nw) {
    long long d = 0, sl = 0;
    for (int32_t x = moff[c] + lane_id(); x < moff[c + 1]; x += 32) {
      const int32_t i = members[x];
      d += off[i + 1] - off[i];
      sl += self[i];
    }
    d = warp_sum(d);
    sl = warp_sum(sl);
    if (lane_id() == 0) {
      bound[c] = d;
      self2[c] = sl;
    }
  }
}

__global__ void k_lv_table_sizes(const long long* __restrict__ bound, int32_t V2,
                                 long long* __restrict__ tsz) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < V2; c += gridDim.x * blockDim.x) {
    long long s = 4;
    while (s < 2 * bound[c] + 2) s <<= 1;
    tsz[c] = s;
  }
}

// One thread per member edge (in member order; mpre = exclusive prefix of
// the members' degrees): an edge to another coarse vertex is added to the
// coarse vertex's table, an edge inside it to its internal weight.
__global__ void k_lv_agg_insert(const int32_t* __restrict__ members, const long long* __restrict__ mpre,
                                int64_t V, const int32_t* __restrict__ cv,
                                const long long* __restrict__ off, const int32_t* __restrict__ adj,
                                const long long* __restrict__ aw, const long long* __restrict__ toff,
                                int32_t* __restrict__ tkey, long long* __restrict__ tval,
                                long long* __restrict__ internal, int32_t* status) {
  const long long total = mpre[V];
  for (long long y = (long long)blockIdx.x * blockDim.x + threadIdx.x; y < total;
       y += (long long)gridDim.x * blockDim.x) {
    int64_t a = 0, b = V - 1;  // largest x with mpre[x] <= y
    while (a < b) {
      const int64_t mid = (a + b + 1) >> 1;
      if (mpre[mid] <= y) a = mid;
      else b = mid - 1;
    }
    const int32_t i = members[a];
    const long long q = off[i] + (y - mpre[a]);
    const int32_t ci = cv[i], cj = cv[adj[q]];
    if (ci == cj) {
      atomic_add_i64(&internal[ci], aw[q]);
    } else {
      const long long tb = toff[ci];
      const uint32_t mask = (uint32_t)(toff[ci + 1] - tb) - 1;
      if (!table_add(tkey + tb, tval + tb, mask, cj, aw[q])) dev_fail(status, DEV_HASH_FULL);
    }
  }
}

// The coarse vertex owning table slot s: the largest c with toff[c] <= s.
__device__ __forceinline__ int32_t table_owner(const long long* toff, int32_t V2, long long s) {
  int32_t a = 0, b = V2 - 1;
  while (a < b) {
    const int32_t mid = (a + b + 1) >> 1;
    if (toff[mid] <= s) a = mid;
    else b = mid - 1;
  }
  return a;
}

// Distinct neighbours of every coarse vertex: one thread per table slot over
// all tables (a hub's table is spread over the grid), lanes of a warp that
// count for the same coarse vertex share one atomic.
__global__ void k_lv_agg_count(const long long* __restrict__ toff, int32_t V2,
                               const int32_t* __restrict__ tkey, int32_t* __restrict__ deg2) {
  const long long total = toff[V2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < total;
       b += stride) {
    const long long s = b + lane_id();
    const bool used = s < total && tkey[s] != LV_EMPTY;
    const int32_t c = used ? table_owner(toff, V2, s) : -1;
    warp_claim_slot(deg2, c, __ballot_sync(FULL, used));
  }
}

// Writes the coarse edge lists (order inside a list unspecified), again one
// thread per table slot; positions come from a per-vertex cursor claimed
// once per warp and coarse vertex.
__global__ void k_lv_agg_write(const long long* __restrict__ toff, int32_t V2,
                               const int32_t* __restrict__ tkey, const long long* __restrict__ tval,
                               const long long* __restrict__ off2, int32_t* __restrict__ adj2,
                               long long* __restrict__ aw2, int32_t* __restrict__ fill) {
  const long long total = toff[V2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < total;
       b += stride) {
    const long long s = b + lane_id();
    const int32_t key = s < total ? tkey[s] : LV_EMPTY;
    const bool used = key != LV_EMPTY;
    const int32_t c = used ? table_owner(toff, V2, s) : -1;
    const int32_t slot = warp_claim_slot(fill, c, __ballot_sync(FULL, used));
    if (used) {
      const long long pos = off2[c] + slot;
      adj2[pos] = key;
      aw2[pos] = tval[s];
    }
  }
}

// Coarse self-loop weights: own self loops plus half the internal weight
// (every internal edge was seen from both of its ends).
__global__ void k_lv_self2(int32_t V2, const long long* __restrict__ internal,
                           long long* __restrict__ self2) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < V2; c += gridDim.x * blockDim.x)
    self2[c] += internal[c] / 2;
}

__global__ void k_lv_vmap(int32_t* __restrict__ vmap, int32_t n, const int32_t* __restrict__ cv) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    vmap[v] = cv[vmap[v]];
}

// Distinct community ids among the nodes.
__global__ void k_lv_mark(const int32_t* __restrict__ comm, int32_t n, int32_t* __restrict__ flag) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    flag[comm[v]] = 1;
}

// ------------------------------------------------------------ host

struct LvGraph {
  int64_t V = 0, E = 0;
  DBuf<long long> off, aw, self, k;
  DBuf<int32_t> adj;
};

void lv_degrees(const Ctx& cx, LvGraph& g, long long* W2) {
  g.k.alloc(&cx.alloc, (size_t)std::max<int64_t>(g.V, 1));
  DBuf<unsigned long long> tot;
  tot.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(tot.p, 0, sizeof(unsigned long long), cx.stream));
  k_lv_degrees<<<grid_for(g.V, 8, cx.num_sms, 16), 256, 0, cx.stream>>>(g.off.p, g.aw.p, g.self.p,
                                                                      g.V, g.k.p, tot.p);
  check_launch("lv_degrees");
  *W2 = read_i64(cx, reinterpret_cast<const int64_t*>(tot.p));
}

// Aggregates the clustering cl of g into the next level's graph; cv[i] =
// coarse vertex of i.
void lv_aggregate(const Ctx& cx, const LvGraph& g, const int32_t* cl, LvGraph& out,
                  DBuf<int32_t>& cv) {
  const int64_t V = g.V;
  const int gV = grid_for(V, 256, cx.num_sms, 8);
  DBuf<int32_t> flag, cid, mcnt, moff, mfill, members;
  flag.alloc(&cx.alloc, (size_t)V + 1);
  cid.alloc(&cx.alloc, (size_t)V + 1);
  HG_CUDA(cudaMemsetAsync(flag.p, 0, flag.bytes(), cx.stream));
  k_lv_used<<<gV, 256, 0, cx.stream>>>(cl, V, flag.p);
  check_launch("lv_used");
  scan_exclusive_i32(cx, flag.p, cid.p, V, cid.p + V);
  const int32_t V2 = read_i32(cx, cid.p + V);
  cv.alloc(&cx.alloc, (size_t)V);
  mcnt.alloc(&cx.alloc, (size_t)V2 + 1);
  moff.alloc(&cx.alloc, (size_t)V2 + 1);
  mfill.alloc(&cx.alloc, (size_t)V2 + 1);
  members.alloc(&cx.alloc, (size_t)V);
  HG_CUDA(cudaMemsetAsync(mcnt.p, 0, mcnt.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(mfill.p, 0, mfill.bytes(), cx.stream));
  k_lv_coarse_of<<<gV, 256, 0, cx.stream>>>(cl, cid.p, V, cv.p, mcnt.p);
  check_launch("lv_coarse_of");
  scan_exclusive_i32(cx, mcnt.p, moff.p, V2, moff.p + V2);
  k_lv_members<<<gV, 256, 0, cx.stream>>>(cv.p, V, moff.p, mfill.p, members.p);
  check_launch("lv_members");
  // member degrees along the member list, table offsets per coarse vertex
  DBuf<int32_t> mdeg;
  DBuf<long long> mpre, bound, tsz, toff, internal;
  mdeg.alloc(&cx.alloc, (size_t)V + 1);
  mpre.alloc(&cx.alloc, (size_t)V + 1);
  k_lv_list_sizes<<<gV, 256, 0, cx.stream>>>(members.p, (int32_t)V, g.off.p, mdeg.p, nullptr);
  check_launch("lv_member_degrees");
  scan_exclusive_i32_to_i64(cx, mdeg.p, reinterpret_cast<int64_t*>(mpre.p), V,
                            reinterpret_cast<int64_t*>(mpre.p) + V);
  bound.alloc(&cx.alloc, (size_t)V2 + 1);
  tsz.alloc(&cx.alloc, (size_t)V2 + 1);
  toff.alloc(&cx.alloc, (size_t)V2 + 1);
  internal.alloc(&cx.alloc, (size_t)V2 + 1);
  out.self.alloc(&cx.alloc, (size_t)V2 + 1);
  HG_CUDA(cudaMemsetAsync(internal.p, 0, internal.bytes(), cx.stream));
  const int gC = grid_for(V2, 8, cx.num_sms, 16);
  k_lv_coarse_bounds<<<gC, 256, 0, cx.stream>>>(members.p, moff.p, V2, g.off.p, g.self.p, bound.p,
                                              out.self.p);
  check_launch("lv_coarse_bounds");
  k_lv_table_sizes<<<grid_for(V2, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(bound.p, V2, tsz.p);
  check_launch("lv_table_sizes");
  std::vector<long long> htsz((size_t)V2);
  HG_CUDA(cudaMemcpyAsync(htsz.data(), tsz.p, sizeof(long long) * (size_t)V2,
                          cudaMemcpyDeviceToHost, cx.stream));
  wait_stream(cx);
  check_status(cx);
  std::vector<long long> htoff((size_t)V2 + 1, 0);
  for (int32_t c = 0; c < V2; ++c) {
    if (htsz[c] > (1ll << 31)) throw HgError(HG_ERR_UNSUPPORTED, "coarse vertex degree too large");
    htoff[c + 1] = htoff[c] + htsz[c];
  }
  HG_CUDA(cudaMemcpyAsync(toff.p, htoff.data(), sizeof(long long) * ((size_t)V2 + 1),
                          cudaMemcpyHostToDevice, cx.stream));
  const long long tslots = htoff[V2];
  DBuf<int32_t> tkey;
  DBuf<long long> tval;
  tkey.alloc(&cx.alloc, (size_t)std::max<long long>(tslots, 1));
  tval.alloc(&cx.alloc, (size_t)std::max<long long>(tslots, 1));
  HG_CUDA(cudaMemsetAsync(tkey.p, 0xff, tkey.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(tval.p, 0, tval.bytes(), cx.stream));
  k_lv_agg_insert<<<grid_for(g.E, 256, cx.num_sms, 16), 256, 0, cx.stream>>>(
      members.p, mpre.p, V, cv.p, g.off.p, g.adj.p, g.aw.p, toff.p, tkey.p, tval.p, internal.p,
      cx.d_status);
  check_launch("lv_agg_insert");
  DBuf<int32_t> deg2, fill2;
  deg2.alloc(&cx.alloc, (size_t)V2 + 1);
  fill2.alloc(&cx.alloc, (size_t)V2 + 1);
  HG_CUDA(cudaMemsetAsync(fill2.p, 0, fill2.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(deg2.p, 0, deg2.bytes(), cx.stream));
  const int gT = grid_for(tslots, 256, cx.num_sms, 8);
  k_lv_agg_count<<<gT, 256, 0, cx.stream>>>(toff.p, V2, tkey.p, deg2.p);
  check_launch("lv_agg_count");
  out.V = V2;
  out.off.alloc(&cx.alloc, (size_t)V2 + 1);
  scan_exclusive_i32_to_i64(cx, deg2.p, reinterpret_cast<int64_t*>(out.off.p), V2,
                            reinterpret_cast<int64_t*>(out.off.p) + V2);
  out.E = read_i64(cx, reinterpret_cast<const int64_t*>(out.off.p) + V2);
  out.adj.alloc(&cx.alloc, (size_t)std::max<int64_t>(out.E, 1));
  out.aw.alloc(&cx.alloc, (size_t)std::max<int64_t>(out.E, 1));
  k_lv_agg_write<<<gT, 256, 0, cx.stream>>>(toff.p, V2, tkey.p, tval.p, out.off.p, out.adj.p,
                                          out.aw.p, fill2.p);
  check_launch("lv_agg_write");
  k_lv_self2<<<grid_for(V2, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(V2, internal.p, out.self.p);
  check_launch("lv_self2");
  if (cx.launches) *cx.launches += 14;
}

// One Louvain level on g (clusters start as singletons).  Returns the moves.
int64_t lv_local_moving(const Ctx& cx, const LvGraph& g, long long W2, int S, uint64_t seed,
                        int level, DBuf<int32_t>& cl, LouvainCounters& lc) {
  const int64_t V = g.V;
  DBuf<long long> vol;
  cl.alloc(&cx.alloc, (size_t)std::max<int64_t>(V, 1));
  vol.alloc(&cx.alloc, (size_t)std::max<int64_t>(V, 1));
  const int gV = grid_for(V, 256, cx.num_sms, 8);
  k_lv_init<<<gV, 256, 0, cx.stream>>>(V, g.k.p, cl.p, vol.p);
  check_launch("lv_init");
  DBuf<int32_t> cnt, fill, koff, list, mv_v, mv_to, words, ldeg, tsize;
  DBuf<long long> lpre, toff;
  DBuf<unsigned long long> moved;
  const int nkeys = 2 * S;
  cnt.alloc(&cx.alloc, (size_t)nkeys);
  fill.alloc(&cx.alloc, (size_t)nkeys);
  koff.alloc(&cx.alloc, (size_t)nkeys + 1);
  list.alloc(&cx.alloc, (size_t)V + 1);
  mv_v.alloc(&cx.alloc, (size_t)V + 1);
  mv_to.alloc(&cx.alloc, (size_t)V + 1);
  words.alloc(&cx.alloc, (size_t)S * 4);
  ldeg.alloc(&cx.alloc, (size_t)V + 1);
  tsize.alloc(&cx.alloc, (size_t)V + 1);
  lpre.alloc(&cx.alloc, (size_t)V + 1);
  toff.alloc(&cx.alloc, (size_t)V + 1);
  moved.alloc(&cx.alloc, 1);
  DBuf<int32_t> tkey;
  DBuf<long long> tval;
  size_t tcap = 0;
  LvArgs A;
  A.off = g.off.p;
  A.adj = g.adj.p;
  A.aw = g.aw.p;
  A.k = g.k.p;
  A.cl = cl.p;
  A.vol = vol.p;
  A.W2 = W2;
  A.list = list.p;
  A.mv_v = mv_v.p;
  A.mv_to = mv_to.p;
  A.status = cx.d_status;
  int64_t level_moves = 0;
  for (int round = 0; round < LV_ROUNDS; ++round) {
    HG_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(fill.p, 0, fill.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(words.p, 0, words.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(moved.p, 0, moved.bytes(), cx.stream));
    k_lv_count<<<gV, 256, nkeys * sizeof(int32_t), cx.stream>>>(g.off.p, V, seed, level, round, S,
                                                                 cnt.p);
    check_launch("lv_count");
    scan_exclusive_i32(cx, cnt.p, koff.p, nkeys, koff.p + nkeys);
    k_lv_scatter<<<gV, 256, 0, cx.stream>>>(g.off.p, V, seed, level, round, S, koff.p, fill.p,
                                            list.p);
    check_launch("lv_scatter");
    std::vector<int32_t> hkoff((size_t)nkeys + 1);
    HG_CUDA(cudaMemcpyAsync(hkoff.data(), koff.p, sizeof(int32_t) * hkoff.size(),
                            cudaMemcpyDeviceToHost, cx.stream));
    wait_stream(cx);
    check_status(cx);
    const int32_t listed = hkoff[nkeys];
    // degrees and table sizes along the list; class-1 tables per sub-round
    if (listed > 0) {
      k_lv_list_sizes<<<grid_for(listed, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
          list.p, listed, g.off.p, ldeg.p, tsize.p);
      check_launch("lv_list_sizes");
    }
    scan_exclusive_i32_to_i64(cx, ldeg.p, reinterpret_cast<int64_t*>(lpre.p), listed,
                              reinterpret_cast<int64_t*>(lpre.p) + listed);
    scan_exclusive_i32_to_i64(cx, tsize.p, reinterpret_cast<int64_t*>(toff.p), listed,
                              reinterpret_cast<int64_t*>(toff.p) + listed);
    std::vector<long long> htoff((size_t)listed + 1);
    HG_CUDA(cudaMemcpyAsync(htoff.data(), toff.p, sizeof(long long) * htoff.size(),
                            cudaMemcpyDeviceToHost, cx.stream));
    wait_stream(cx);
    size_t need = 1;
    for (int s = 0; s < S; ++s)
      need = std::max<size_t>(need, (size_t)(htoff[hkoff[2 * s + 2]] - htoff[hkoff[2 * s + 1]]));
    if (need > tcap) {
      tkey.alloc(&cx.alloc, need);
      tval.alloc(&cx.alloc, need);
      HG_CUDA(cudaMemsetAsync(tkey.p, 0xff, tkey.bytes(), cx.stream));
      HG_CUDA(cudaMemsetAsync(tval.p, 0, tval.bytes(), cx.stream));
      tcap = need;
    }
    for (int s = 0; s < S; ++s) {
      A.words = words.p + 4 * s;
      const int32_t lo0 = hkoff[2 * s], hi0 = hkoff[2 * s + 1], hi1 = hkoff[2 * s + 2];
      if (hi0 > lo0) {
        k_lv_small<<<grid_for(hi0 - lo0, LV_WARPS, cx.num_sms, 8), LV_WARPS * 32, 0, cx.stream>>>(
            A, lo0, hi0);
        check_launch("lv_small");
        lc.launches += 1;
      }
      if (hi1 > hi0) {
        k_lv_big_insert<<<cx.num_sms * 8, 256, 0, cx.stream>>>(A, hi0, hi1, lpre.p, toff.p,
                                                               htoff[hi0], tsize.p, tkey.p, tval.p);
        check_launch("lv_big_insert");
        k_lv_big_argmax<<<grid_for(hi1 - hi0, 1, cx.num_sms, 8), LV_ARGMAX_THREADS, 0,
                          cx.stream>>>(A, hi0, hi1, toff.p, htoff[hi0], tsize.p, tkey.p, tval.p);
        check_launch("lv_big_argmax");
        lc.launches += 2;
      }
      k_lv_apply<<<grid_for((V + S - 1) / S, 256, cx.num_sms, 4), 256, 0, cx.stream>>>(
          mv_v.p, mv_to.p, A.words, g.k.p, cl.p, vol.p, moved.p);
      check_launch("lv_apply");
      lc.launches += 1;
    }
    const int64_t m = read_i64(cx, reinterpret_cast<const int64_t*>(moved.p));
    level_moves += m;
    lc.rounds += 1;
    if (100 * m < V) break;
  }
  return level_moves;
}

}  // namespace

int32_t detect_communities(const Ctx& cx, const Level& L, int S, uint64_t seed,
                           DBuf<int32_t>& comm, LouvainCounters& lc) {
  const int32_t n = L.n, m = L.m;
  const int64_t p = L.p;
  comm.alloc(&cx.alloc, (size_t)n);
  iota_i32(cx, comm.p, n);  // vmap: node -> vertex of the current level
  if (p == 0) return n;
  LvGraph g;
  g.V = (int64_t)n + m;
  g.E = 2 * p;
  g.off.alloc(&cx.alloc, (size_t)g.V + 1);
  g.adj.alloc(&cx.alloc, (size_t)g.E);
  g.aw.alloc(&cx.alloc, (size_t)g.E);
  g.self.alloc(&cx.alloc, (size_t)g.V);
  HG_CUDA(cudaMemsetAsync(g.self.p, 0, g.self.bytes(), cx.stream));
  k_lv_offsets<<<grid_for(g.V + 1, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
      L.ioff.p, L.eoff.p, n, m, p, g.off.p);
  check_launch("lv_offsets");
  k_lv_bipartite<<<grid_for(p, 256, cx.num_sms, 16), 256, 0, cx.stream>>>(
      L.eoff.p, L.pins.p, L.w.p, L.inets.p, L.ipin.p, n, p, g.adj.p, g.aw.p);
  check_launch("lv_bipartite");
  long long W2 = 0;
  lv_degrees(cx, g, &W2);
  for (int level = 0; level < LV_LEVELS; ++level) {
    DBuf<int32_t> cl;
    const int64_t moves = lv_local_moving(cx, g, W2, S, seed, level, cl, lc);
    lc.moves += moves;
    if (moves == 0) break;
    lc.levels = level + 1;
    LvGraph next;
    DBuf<int32_t> cv;
    lv_aggregate(cx, g, cl.p, next, cv);
    k_lv_vmap<<<grid_for(n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(comm.p, n, cv.p);
    check_launch("lv_vmap");
    const bool shrank = next.V < g.V;
    long long W2n = 0;
    lv_degrees(cx, next, &W2n);
    g = std::move(next);
    if (!shrank) break;
  }
  check_status(cx);
  // number of distinct communities among the nodes
  DBuf<int32_t> flag;
  flag.alloc(&cx.alloc, (size_t)g.V + 1);
  HG_CUDA(cudaMemsetAsync(flag.p, 0, flag.bytes(), cx.stream));
  k_lv_mark<<<grid_for(n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(comm.p, n, flag.p);
  check_launch("lv_mark");
  scan_exclusive_i32(cx, flag.p, flag.p, g.V, flag.p + g.V);
  return read_i32(cx, flag.p + g.V);
}

}  // namespace hgk
