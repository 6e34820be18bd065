// Deterministic clustering for coarsening (Sec. 4.1 rating function, cluster
// weight limit and contraction limit; Sec. 11 "Deterministic Clustering for
// Coarsening").
//
// Per sub-round s (nodes hashed into S sub-rounds):
//   rating   every unclustered node u of s picks the admissible cluster C
//            maximising r(u, C) = sum over e in I(u), e meeting C, of
//            w(e) / (|e| - 1), in Q20 fixed point with each net term floored,
//            nets of more than T pins skipped, a net counted once per cluster,
//            ties to the smaller id.  Admissible: C != u, C not an unclustered
//            node of the same sub-round, cw[C] + c(u) <= c_max (state at the
//            start of the sub-round).  While rating, the weights of the moves
//            into every target are summed (the paper's fast path).
//   approval a target whose moves all fit under c_max accepts them all;
//            otherwise its movers are sorted by (c(u), u) and the longest
//            prefix that fits is accepted.
// Nodes are bucketed per level by sub-round and by a bound on their rating
// work, W(u) = sum of |e| over rated nets, which decides the team and the
// hash-table storage: a warp with a 256-slot shared-memory table (W <= 128),
// a block with a 4096-slot shared-memory table (W <= 2048), or a block with a
// global-memory table sized for the largest such node.
#include <algorithm>

#include "common.cuh"

namespace hgk {

namespace {

constexpr int NCLASS = 3;
constexpr int WARP_TABLE = 256;   // slots per warp table
constexpr int WARP_MAXW = 128;
constexpr int CTA_TABLE = 4096;   // slots per block table
constexpr int CTA_MAXW = 2048;
constexpr int RATE_WARPS = 8;
constexpr int CTA_THREADS = 256;
constexpr int BIG_THREADS = 512;
constexpr int32_t EMPTY_KEY = -1;

// per sub-round bookkeeping words
enum { CW_MOVES = 0, CW_TOUCHED = 1, CW_SLOTS = 2, CW_CURSOR = 3, CW_WORDS = 4 };
// work counters
enum { ST_PINS = 0, ST_INCID = 1, ST_NODES = 2, ST_WORDS = 4 };

struct RateArgs {
  const int32_t* ioff;
  const int32_t* inets;
  const int32_t* eoff;
  const int32_t* pins;
  const int32_t* w;
  const int32_t* c;
  const int32_t* rep;
  const int32_t* cw;
  const uint8_t* joined;
  uint64_t seed;
  int level, S, s, T;
  int32_t c_max, n;
  const int32_t* list;  // nodes of this (sub-round, class)
  int32_t count;
  const int32_t* clusters;
  int32_t* target;
  int32_t* gw;
  int32_t* gcnt;
  int32_t* mv;
  int32_t* touched;
  int32_t* words;
  unsigned long long* stats;
  int32_t* status;
};

struct Table {
  int32_t* key;
  unsigned long long* claim;
  long long* val;
  uint32_t mask;   // capacity - 1 (power of two)
  int32_t* used;   // slots in use (global tables only)
  int32_t* nused;
};

__device__ __forceinline__ void team_sync(bool cta) {
  if (cta) __syncthreads();
  else __syncwarp();
}

__device__ __forceinline__ uint32_t slot_hash(int32_t C) { return (uint32_t)C * 0x9E3779B1u; }

// Finds or inserts C; returns the slot or -1 when the table is full.
__device__ __forceinline__ int32_t table_insert(const Table& T, int32_t C, bool track_used) {
  uint32_t h = slot_hash(C) & T.mask;
  for (uint32_t probe = 0; probe <= T.mask; ++probe) {
    const int32_t k = T.key[h];
    if (k == C) return (int32_t)h;
    if (k == EMPTY_KEY) {
      const int32_t old = atomicCAS(&T.key[h], EMPTY_KEY, C);
      if (old == EMPTY_KEY) {
        if (track_used) T.used[atomicAdd(T.nused, 1)] = (int32_t)h;
        return (int32_t)h;
      }
      if (old == C) return (int32_t)h;
    }
    h = (h + 1) & T.mask;
  }
  return -1;
}

// Sets bit j of the claim word of a slot for net group g; true if this call
// set it (the net has not yet contributed to this cluster).
__device__ __forceinline__ bool claim_net(unsigned long long* word, uint32_t g, int j) {
  const unsigned long long tag = (unsigned long long)(g + 1) << 32;
  const unsigned long long bit = 1ull << j;
  unsigned long long old = *(volatile unsigned long long*)word;
  while (true) {
    unsigned long long nw;
    if ((old & 0xffffffff00000000ull) == tag) {
      if (old & bit) return false;
      nw = old | bit;
    } else {
      nw = tag | bit;
    }
    const unsigned long long prev = atomicCAS(word, old, nw);
    if (prev == old) return true;
    old = prev;
  }
}

// Rates node u with a team of `nthreads` threads (a warp, or a whole block
// when cta is true).  tid = thread index inside the team.
template <bool CTA>
__device__ void rate_node(const RateArgs& A, int32_t u, const Table& T, int tid, int nthreads,
                          long long* s_red_val, int32_t* s_red_c, bool global_table) {
  const int lane = tid & 31;
  const int32_t cu = A.c[u];
  const int32_t beg = A.ioff[u], end = A.ioff[u + 1];
  int64_t visits = 0;
  for (int32_t g0 = beg; g0 < end; g0 += 32) {
    const uint32_t g = (uint32_t)((g0 - beg) >> 5);
    // every warp of the team describes the same group of (up to) 32 nets
    int32_t e = -1, size = 0, start = 0, eff = 0;
    long long r = 0;
    if (g0 + lane < end) {
      e = A.inets[g0 + lane];
      start = A.eoff[e];
      size = A.eoff[e + 1] - start;
      if (size >= 2 && size <= A.T) {
        eff = size;
        r = ((long long)A.w[e] << 20) / (size - 1);
      }
    }
    const int32_t incl = warp_inclusive_scan(eff);
    const int32_t Z = __shfl_sync(FULL, incl, 31);
    visits += Z;
    for (int32_t f0 = 0; f0 < Z; f0 += nthreads) {
      const int32_t f = f0 + tid;
      // net index j: number of lanes whose inclusive count is <= f
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int32_t probe = __shfl_sync(FULL, incl, j + step - 1);
        if (probe <= f) j += step;
      }
      j = j > 31 ? 31 : j;
      const int32_t incl_j = __shfl_sync(FULL, incl, j);
      const int32_t eff_j = __shfl_sync(FULL, eff, j);
      const int32_t start_j = __shfl_sync(FULL, start, j);
      const long long r_j = __shfl_sync(FULL, r, j);
      if (f < Z) {
        const int32_t pos = f - (incl_j - eff_j);
        const int32_t v = A.pins[start_j + pos];
        const int32_t C = A.rep[v];
        bool ok = C != u;
        if (ok && !A.joined[C]) ok = subround_of_node_cluster(A.seed, A.level, C, A.S) != A.s;
        if (ok) ok = (long long)A.cw[C] + cu <= (long long)A.c_max;
        if (ok) {
          const int32_t slot = table_insert(T, C, global_table);
          if (slot < 0) {
            dev_fail(A.status, DEV_HASH_FULL);
          } else if (claim_net(&T.claim[slot], g, j)) {
            atomicAdd((unsigned long long*)&T.val[slot], (unsigned long long)r_j);
          }
        }
      }
    }
    team_sync(CTA);
  }
  // argmax over the table: rating desc, cluster id asc
  long long best_v = -1;
  int32_t best_c = -1;
  if (global_table) {
    const int32_t nu = *T.nused;
    for (int32_t i = tid; i < nu; i += nthreads) {
      const int32_t sl = T.used[i];
      const long long v = T.val[sl];
      const int32_t C = T.key[sl];
      if (v > best_v || (v == best_v && C < best_c)) {
        best_v = v;
        best_c = C;
      }
    }
  } else {
    for (uint32_t sl = tid; sl <= T.mask; sl += nthreads) {
      const int32_t C = T.key[sl];
      if (C == EMPTY_KEY) continue;
      const long long v = T.val[sl];
      if (v > best_v || (v == best_v && C < best_c)) {
        best_v = v;
        best_c = C;
      }
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const long long ov = __shfl_xor_sync(FULL, best_v, d);
    const int32_t oc = __shfl_xor_sync(FULL, best_c, d);
    if (ov > best_v || (ov == best_v && oc >= 0 && (best_c < 0 || oc < best_c))) {
      best_v = ov;
      best_c = oc;
    }
  }
  if (CTA) {
    if (lane == 0) {
      s_red_val[tid >> 5] = best_v;
      s_red_c[tid >> 5] = best_c;
    }
    __syncthreads();
    if (tid == 0) {
      for (int wv = 1; wv < nthreads / 32; ++wv) {
        const long long ov = s_red_val[wv];
        const int32_t oc = s_red_c[wv];
        if (ov > best_v || (ov == best_v && oc >= 0 && (best_c < 0 || oc < best_c))) {
          best_v = ov;
          best_c = oc;
        }
      }
    }
  }
  team_sync(CTA);
  // reset the table for the next node
  if (global_table) {
    const int32_t nu = *T.nused;
    for (int32_t i = tid; i < nu; i += nthreads) {
      const int32_t sl = T.used[i];
      T.key[sl] = EMPTY_KEY;
      T.claim[sl] = 0;
      T.val[sl] = 0;
    }
    team_sync(CTA);
    if (tid == 0) *T.nused = 0;
  } else {
    for (uint32_t sl = tid; sl <= T.mask; sl += nthreads) {
      T.key[sl] = EMPTY_KEY;
      T.claim[sl] = 0;
      T.val[sl] = 0;
    }
  }
  team_sync(CTA);
  if (tid == 0) {
    A.target[u] = best_c;
    atomicAdd(&A.stats[ST_PINS], (unsigned long long)visits);
    atomicAdd(&A.stats[ST_INCID], (unsigned long long)(end - beg));
    atomicAdd(&A.stats[ST_NODES], 1ull);
    if (best_c >= 0) {
      A.mv[atomicAdd(&A.words[CW_MOVES], 1)] = u;
      atomicAdd(&A.gw[best_c], cu);
      if (atomicAdd(&A.gcnt[best_c], 1) == 0) A.touched[atomicAdd(&A.words[CW_TOUCHED], 1)] = best_c;
    }
  }
}

__device__ __forceinline__ bool subround_stopped(const RateArgs& A) {
  return 5ll * (long long)(*A.clusters) <= 2ll * (long long)A.n;
}

// warp per node, 256-slot shared table per warp
__global__ void __launch_bounds__(RATE_WARPS * 32) k_rate_warp(RateArgs A) {
  __shared__ int32_t s_key[RATE_WARPS][WARP_TABLE];
  __shared__ unsigned long long s_claim[RATE_WARPS][WARP_TABLE];
  __shared__ long long s_val[RATE_WARPS][WARP_TABLE];
  if (subround_stopped(A)) return;
  const int wv = warp_in_block(), lane = lane_id();
  Table T{s_key[wv], s_claim[wv], s_val[wv], WARP_TABLE - 1, nullptr, nullptr};
  for (int i = lane; i < WARP_TABLE; i += 32) {
    s_key[wv][i] = EMPTY_KEY;
    s_claim[wv][i] = 0;
    s_val[wv][i] = 0;
  }
  __syncwarp();
  for (int32_t i = blockIdx.x * RATE_WARPS + wv; i < A.count; i += gridDim.x * RATE_WARPS) {
    const int32_t u = A.list[i];
    if (A.joined[u]) continue;
    rate_node<false>(A, u, T, lane, 32, nullptr, nullptr, false);
  }
}

// block per node, 4096-slot shared table (dynamic shared memory)
__global__ void __launch_bounds__(CTA_THREADS) k_rate_cta(RateArgs A) {
  extern __shared__ unsigned char smem[];
  __shared__ long long s_rv[32];
  __shared__ int32_t s_rc[32];
  if (subround_stopped(A)) return;
  unsigned long long* claim = reinterpret_cast<unsigned long long*>(smem);
  long long* val = reinterpret_cast<long long*>(claim + CTA_TABLE);
  int32_t* key = reinterpret_cast<int32_t*>(val + CTA_TABLE);
  Table T{key, claim, val, CTA_TABLE - 1, nullptr, nullptr};
  for (int i = threadIdx.x; i < CTA_TABLE; i += blockDim.x) {
    key[i] = EMPTY_KEY;
    claim[i] = 0;
    val[i] = 0;
  }
  __syncthreads();
  for (int32_t i = blockIdx.x; i < A.count; i += gridDim.x) {
    const int32_t u = A.list[i];
    if (A.joined[u]) continue;
    rate_node<true>(A, u, T, threadIdx.x, blockDim.x, s_rv, s_rc, false);
  }
}

// block per node, global table of 2^k slots per block
__global__ void __launch_bounds__(BIG_THREADS)
k_rate_big(RateArgs A, int32_t* gkey, unsigned long long* gclaim, long long* gval, int32_t* gused,
           int32_t* gnused, uint32_t cap) {
  __shared__ long long s_rv[32];
  __shared__ int32_t s_rc[32];
  if (subround_stopped(A)) return;
  const size_t off = (size_t)blockIdx.x * cap;
  Table T{gkey + off, gclaim + off, gval + off, cap - 1, gused + off, gnused + blockIdx.x};
  for (int32_t i = blockIdx.x; i < A.count; i += gridDim.x) {
    const int32_t u = A.list[i];
    if (A.joined[u]) continue;
    rate_node<true>(A, u, T, threadIdx.x, blockDim.x, s_rv, s_rc, true);
  }
}

// ------------------------------------------------------- node bucketing

__device__ __forceinline__ int work_class(int32_t W) {
  return W <= WARP_MAXW ? 0 : (W <= CTA_MAXW ? 1 : 2);
}

// W(u) and the (sub-round, class) key of every node with W(u) > 0.
__global__ void k_node_work(const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets,
                            const int32_t* __restrict__ eoff, int32_t n, int T, uint64_t seed,
                            int level, int S, int32_t* __restrict__ key_of,
                            int32_t* __restrict__ kcount, int32_t* __restrict__ max_big) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t W = 0;
    for (int32_t j = ioff[u]; j < ioff[u + 1]; ++j) {
      const int32_t e = inets[j];
      const int32_t sz = eoff[e + 1] - eoff[e];
      if (sz >= 2 && sz <= T) W += sz;
    }
    int32_t key = -1;
    if (W > 0) {
      const int32_t Wc = W > 0x7fffffff ? 0x7fffffff : (int32_t)W;
      const int cls = work_class(Wc);
      key = subround_of_node_cluster(seed, level, (int)u, S) * NCLASS + cls;
      atomicAdd(&kcount[key], 1);
      if (cls == 2) atomicMax(max_big, Wc);
    }
    key_of[u] = key;
  }
}

__global__ void k_node_scatter(const int32_t* __restrict__ key_of, int32_t n, int nkeys,
                               const int32_t* __restrict__ kcount, int32_t* __restrict__ kfill,
                               int32_t* __restrict__ list) {
  extern __shared__ int32_t s_off[];
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int i = 0; i < nkeys; ++i) {
      s_off[i] = run;
      run += kcount[i];
    }
  }
  __syncthreads();
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t key = key_of[u];
    if (key >= 0) list[s_off[key] + atomicAdd(&kfill[key], 1)] = (int32_t)u;
  }
}

// ------------------------------------------------------------- approval

__global__ void k_approve(const int32_t* __restrict__ mv, const int32_t* __restrict__ words,
                          const int32_t* __restrict__ target, const int32_t* __restrict__ cw,
                          const int32_t* __restrict__ gw, const int32_t* __restrict__ gcnt,
                          int32_t c_max, int32_t* __restrict__ rep, uint8_t* __restrict__ joined,
                          int32_t* __restrict__ slot_of, int32_t* __restrict__ slot_c,
                          int32_t* __restrict__ slot_off, int32_t* __restrict__ wslots,
                          int32_t* __restrict__ wcursor) {
  const int32_t nm = words[CW_MOVES];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const int32_t u = mv[i];
    const int32_t C = target[u];
    if ((long long)cw[C] + gw[C] <= (long long)c_max) {
      rep[u] = C;   // fast path: every move into C fits
      joined[u] = 1;
    } else if (atomicCAS(&slot_of[C], -1, -2) == -1) {
      const int32_t sl = atomicAdd(wslots, 1);
      slot_c[sl] = C;
      slot_off[sl] = atomicAdd(wcursor, gcnt[C]);
      slot_of[C] = sl;
    }
  }
}

__global__ void k_contest_scatter(const int32_t* __restrict__ mv, const int32_t* __restrict__ words,
                                  const int32_t* __restrict__ target, const int32_t* __restrict__ cw,
                                  const int32_t* __restrict__ gw, int32_t c_max,
                                  const int32_t* __restrict__ slot_of,
                                  const int32_t* __restrict__ slot_off,
                                  int32_t* __restrict__ slot_fill, int32_t* __restrict__ glist) {
  const int32_t nm = words[CW_MOVES];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const int32_t u = mv[i];
    const int32_t C = target[u];
    if ((long long)cw[C] + gw[C] > (long long)c_max) {
      const int32_t sl = slot_of[C];
      glist[slot_off[sl] + atomicAdd(&slot_fill[sl], 1)] = u;
    }
  }
}

constexpr int GROUP_THREADS = 512;
constexpr int GROUP_SMEM_CAP = 4096;

__device__ void group_bitonic(unsigned long long* buf, int P) {
  for (int kk = 2; kk <= P; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = buf[i], b = buf[ixj];
          if ((a > b) == ((i & kk) == 0)) {
            buf[i] = b;
            buf[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
}

// One block per contested target C: order the movers by (c(u), u), accept
// the longest prefix with cw[C] + weight <= c_max.
__global__ void __launch_bounds__(GROUP_THREADS)
k_contest_group(const int32_t* __restrict__ words, const int32_t* __restrict__ slot_c,
                const int32_t* __restrict__ slot_off, int32_t* __restrict__ slot_fill,
                int32_t* __restrict__ slot_of, const int32_t* __restrict__ glist,
                const int32_t* __restrict__ gcnt, const int32_t* __restrict__ c, int32_t c_max,
                int32_t* __restrict__ cw, int32_t* __restrict__ rep, uint8_t* __restrict__ joined,
                int32_t* __restrict__ clusters) {
  __shared__ unsigned long long s_keys[GROUP_SMEM_CAP];
  __shared__ long long s_red[32];
  __shared__ unsigned long long s_tau;
  const int32_t nslots = words[CW_SLOTS];
  for (int32_t sl = blockIdx.x; sl < nslots; sl += gridDim.x) {
    const int32_t C = slot_c[sl];
    const int32_t cnt = gcnt[C];
    const int32_t off = slot_off[sl];
    const long long cap = (long long)c_max - cw[C];
    // accepted = members whose key (c(u) << 32 | u) is <= tau, the largest key
    // with (sum of c over keys <= tau) <= cap
    if (cnt <= GROUP_SMEM_CAP) {
      int P = 1;
      while (P < cnt) P <<= 1;
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < cnt) {
          const int32_t u = glist[off + i];
          s_keys[i] = ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)u;
        } else {
          s_keys[i] = ~0ull;
        }
      }
      __syncthreads();
      group_bitonic(s_keys, P);
      // prefix sums in chunks; the accepted count is the number of positions
      // whose inclusive prefix is <= cap (weights are positive)
      long long carry = 0;
      if (threadIdx.x == 0) s_tau = 0;
      __syncthreads();
      for (int base = 0; base < cnt; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < cnt ? (long long)(s_keys[i] >> 32) : 0;
        long long x = warp_inclusive_scan(v);
        if (lane_id() == 31) s_red[warp_in_block()] = x;
        __syncthreads();
        if (warp_in_block() == 0) {
          long long y = lane_id() < (int)(blockDim.x >> 5) ? s_red[lane_id()] : 0;
          y = warp_inclusive_scan(y);
          if (lane_id() < (int)(blockDim.x >> 5)) s_red[lane_id()] = y;
        }
        __syncthreads();
        const long long incl = carry + (warp_in_block() ? s_red[warp_in_block() - 1] : 0) + x;
        const long long chunk_total = s_red[(blockDim.x >> 5) - 1];
        if (i < cnt && incl <= cap) atomicAdd(&s_tau, 1ull);
        carry += chunk_total;
        __syncthreads();
      }
      const int32_t acc = (int32_t)s_tau;
      long long added = 0;
      for (int i = threadIdx.x; i < acc; i += blockDim.x) {
        const int32_t u = (int32_t)(s_keys[i] & 0xffffffffu);
        rep[u] = C;
        joined[u] = 1;
        added += (long long)(s_keys[i] >> 32);
      }
      added = block_sum(added, s_red);
      if (threadIdx.x == 0) {
        cw[C] += (int32_t)added;
        if (acc > 0) {
          joined[C] = 1;
          atomicSub(clusters, acc);
        }
        slot_of[C] = -1;
        slot_fill[sl] = 0;
      }
      __syncthreads();
    } else {
      // large group: binary search for tau over the 63-bit key space
      unsigned long long lo = 0, hi = (1ull << 63);  // answer in [lo, hi); lo - 1 = "none"
      // find the largest tau with F(tau) <= cap, F(tau) = sum of c over keys <= tau
      // invariant: F(lo - 1) <= cap (F(-1) = 0), F(hi) > cap or hi = 2^63
      while (hi - lo > 1) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        long long f = 0;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
          const int32_t u = glist[off + i];
          const unsigned long long kk = ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)u;
          if (kk <= mid - 1) f += c[u];
        }
        f = block_sum(f, s_red);
        if (f <= cap) lo = mid; else hi = mid;
      }
      // accepted: keys <= lo - 1 ... written as keys < lo
      long long added = 0;
      int32_t acc = 0;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int32_t u = glist[off + i];
        const unsigned long long kk = ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)u;
        if (kk < lo) {
          rep[u] = C;
          joined[u] = 1;
          added += c[u];
          ++acc;
        }
      }
      added = block_sum(added, s_red);
      const long long acc_all = block_sum((long long)acc, s_red);
      if (threadIdx.x == 0) {
        cw[C] += (int32_t)added;
        if (acc_all > 0) {
          joined[C] = 1;
          atomicSub(clusters, (int32_t)acc_all);
        }
        slot_of[C] = -1;
        slot_fill[sl] = 0;
      }
      __syncthreads();
    }
  }
}

// Uncontested targets: add the summed weight of their movers; reset the sums.
__global__ void k_finish(const int32_t* __restrict__ touched, const int32_t* __restrict__ words,
                         int32_t c_max, int32_t* __restrict__ cw, int32_t* __restrict__ gw,
                         int32_t* __restrict__ gcnt, uint8_t* __restrict__ joined,
                         int32_t* __restrict__ clusters) {
  const int32_t nt = words[CW_TOUCHED];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
    const int32_t C = touched[i];
    if ((long long)cw[C] + gw[C] <= (long long)c_max) {
      cw[C] += gw[C];
      joined[C] = 1;
      atomicSub(clusters, gcnt[C]);
    }
    gw[C] = 0;
    gcnt[C] = 0;
  }
}

__global__ void k_init_cluster(const int32_t* __restrict__ c, int32_t n, int32_t* __restrict__ rep,
                               int32_t* __restrict__ cw, uint8_t* __restrict__ joined,
                               int32_t* __restrict__ slot_of) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    rep[u] = (int32_t)u;
    cw[u] = c[u];
    joined[u] = 0;
    slot_of[u] = -1;
  }
}

__global__ void k_init_table(int32_t* key, unsigned long long* claim, long long* val, size_t cnt) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (size_t)gridDim.x * blockDim.x) {
    key[i] = EMPTY_KEY;
    claim[i] = 0;
    val[i] = 0;
  }
}

}  // namespace

void cluster_level(const Ctx& cx, Level& L, const CoarsenParams& P, CoarsenCounters& cc,
                   DBuf<int32_t>& cw_out) {
  const int32_t n = L.n;
  const int S = P.S;
  const int nkeys = S * NCLASS;
  L.rep.alloc(&cx.alloc, (size_t)n);
  cw_out.alloc(&cx.alloc, (size_t)n);
  DBuf<uint8_t> joined;
  DBuf<int32_t> target, gw, gcnt, slot_of, slot_c, slot_off, slot_fill, mv, touched, glist, key_of,
      kcount, kfill, list, words, clusters, max_big;
  DBuf<unsigned long long> stats;
  const size_t ncap = (size_t)n + 1;
  joined.alloc(&cx.alloc, ncap);
  target.alloc(&cx.alloc, ncap);
  gw.alloc(&cx.alloc, ncap);
  gcnt.alloc(&cx.alloc, ncap);
  slot_of.alloc(&cx.alloc, ncap);
  slot_c.alloc(&cx.alloc, ncap);
  slot_off.alloc(&cx.alloc, ncap);
  slot_fill.alloc(&cx.alloc, ncap);
  mv.alloc(&cx.alloc, ncap);
  touched.alloc(&cx.alloc, ncap);
  glist.alloc(&cx.alloc, ncap);
  key_of.alloc(&cx.alloc, ncap);
  list.alloc(&cx.alloc, ncap);
  kcount.alloc(&cx.alloc, (size_t)nkeys);
  kfill.alloc(&cx.alloc, (size_t)nkeys);
  words.alloc(&cx.alloc, (size_t)S * CW_WORDS);
  clusters.alloc(&cx.alloc, 1);
  max_big.alloc(&cx.alloc, 1);
  stats.alloc(&cx.alloc, ST_WORDS);
  HG_CUDA(cudaMemsetAsync(gw.p, 0, gw.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(gcnt.p, 0, gcnt.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(slot_fill.p, 0, slot_fill.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(kcount.p, 0, kcount.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(kfill.p, 0, kfill.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(words.p, 0, words.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(max_big.p, 0, max_big.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(stats.p, 0, stats.bytes(), cx.stream));
  HG_CUDA(cudaMemcpyAsync(clusters.p, &n, sizeof(int32_t), cudaMemcpyHostToDevice, cx.stream));

  const int g_nodes = grid_for(n, 256, cx.num_sms, 4);
  k_init_cluster<<<g_nodes, 256, 0, cx.stream>>>(L.c.p, n, L.rep.p, cw_out.p, joined.p, slot_of.p);
  check_launch("init_cluster");
  k_node_work<<<g_nodes, 256, 0, cx.stream>>>(L.ioff.p, L.inets.p, L.eoff.p, n, P.T, P.seed,
                                               P.level, S, key_of.p, kcount.p, max_big.p);
  check_launch("node_work");
  k_node_scatter<<<g_nodes, 256, nkeys * sizeof(int32_t), cx.stream>>>(key_of.p, n, nkeys,
                                                                        kcount.p, kfill.p, list.p);
  check_launch("node_scatter");
  if (cx.launches) *cx.launches += 3;

  std::vector<int32_t> hcount(nkeys);
  HG_CUDA(cudaMemcpyAsync(hcount.data(), kcount.p, sizeof(int32_t) * nkeys, cudaMemcpyDeviceToHost,
                          cx.stream));
  const int32_t maxW = read_i32(cx, max_big.p);
  std::vector<int32_t> hoff(nkeys + 1, 0);
  for (int i = 0; i < nkeys; ++i) hoff[i + 1] = hoff[i] + hcount[i];
  int32_t big_max_count = 0;
  for (int s = 0; s < S; ++s) big_max_count = std::max(big_max_count, hcount[s * NCLASS + 2]);

  // global tables for the largest nodes: one per block, sized for maxW
  DBuf<int32_t> gkey, gused, gnused;
  DBuf<unsigned long long> gclaim;
  DBuf<long long> gval;
  uint32_t gcap = 0;
  int g_big = 0;
  if (big_max_count > 0) {
    const int64_t want = 2 * (int64_t)std::min<int64_t>(maxW, n) + 2;
    gcap = 1;
    while ((int64_t)gcap < want) gcap <<= 1;
    // at most ~1 GiB of tables; at least one block
    const int64_t per = (int64_t)gcap * 24;
    int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)cx.num_sms, (1ll << 30) / per));
    blocks = std::min<int64_t>(blocks, big_max_count);
    g_big = (int)blocks;
    gkey.alloc(&cx.alloc, (size_t)g_big * gcap);
    gclaim.alloc(&cx.alloc, (size_t)g_big * gcap);
    gval.alloc(&cx.alloc, (size_t)g_big * gcap);
    gused.alloc(&cx.alloc, (size_t)g_big * gcap);
    gnused.alloc(&cx.alloc, (size_t)g_big);
    HG_CUDA(cudaMemsetAsync(gnused.p, 0, gnused.bytes(), cx.stream));
    k_init_table<<<grid_for((int64_t)g_big * gcap, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
        gkey.p, gclaim.p, gval.p, (size_t)g_big * gcap);
    check_launch("init_table");
  }
  static bool attr_done = false;
  const size_t cta_smem = (size_t)CTA_TABLE * (8 + 8 + 4);
  if (!attr_done) {
    HG_CUDA(cudaFuncSetAttribute(k_rate_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cta_smem));
    attr_done = true;
  }

  RateArgs A;
  A.ioff = L.ioff.p;
  A.inets = L.inets.p;
  A.eoff = L.eoff.p;
  A.pins = L.pins.p;
  A.w = L.w.p;
  A.c = L.c.p;
  A.rep = L.rep.p;
  A.cw = cw_out.p;
  A.joined = joined.p;
  A.seed = P.seed;
  A.level = P.level;
  A.S = S;
  A.T = P.T;
  A.c_max = P.c_max;
  A.n = n;
  A.clusters = clusters.p;
  A.target = target.p;
  A.gw = gw.p;
  A.gcnt = gcnt.p;
  A.mv = mv.p;
  A.touched = touched.p;
  A.stats = stats.p;
  A.status = cx.d_status;

  KernelTimer rate_timer(cx);
  for (int s = 0; s < S; ++s) {
    A.s = s;
    A.words = words.p + (size_t)s * CW_WORDS;
    int32_t* w_s = words.p + (size_t)s * CW_WORDS;
    {
      EventTimer tm(cx, &cc.ms_rating);
      for (int cls = 0; cls < NCLASS; ++cls) {
        const int key = s * NCLASS + cls;
        A.count = hcount[key];
        if (A.count == 0) continue;
        A.list = list.p + hoff[key];
        rate_timer.begin();
        if (cls == 0) {
          k_rate_warp<<<grid_for(A.count, RATE_WARPS, cx.num_sms, 8), RATE_WARPS * 32, 0,
                        cx.stream>>>(A);
        } else if (cls == 1) {
          k_rate_cta<<<grid_for(A.count, 1, cx.num_sms, 2), CTA_THREADS, cta_smem, cx.stream>>>(A);
        } else {
          k_rate_big<<<std::min<int>(g_big, A.count), BIG_THREADS, 0, cx.stream>>>(
              A, gkey.p, gclaim.p, gval.p, gused.p, gnused.p, gcap);
        }
        rate_timer.end();
        check_launch("rate");
        cc.rating_launches += 1;
        if (cx.launches) *cx.launches += 1;
      }
    }
    {
      EventTimer tm(cx, &cc.ms_approve);
      const int g = grid_for((n + S - 1) / S, 256, cx.num_sms, 4);
      k_approve<<<g, 256, 0, cx.stream>>>(mv.p, w_s, target.p, cw_out.p, gw.p, gcnt.p, P.c_max,
                                          L.rep.p, joined.p, slot_of.p, slot_c.p, slot_off.p,
                                          w_s + CW_SLOTS, w_s + CW_CURSOR);
      check_launch("approve");
      k_contest_scatter<<<g, 256, 0, cx.stream>>>(mv.p, w_s, target.p, cw_out.p, gw.p, P.c_max,
                                                  slot_of.p, slot_off.p, slot_fill.p, glist.p);
      check_launch("contest_scatter");
      k_contest_group<<<cx.num_sms, GROUP_THREADS, 0, cx.stream>>>(
          w_s, slot_c.p, slot_off.p, slot_fill.p, slot_of.p, glist.p, gcnt.p, L.c.p, P.c_max,
          cw_out.p, L.rep.p, joined.p, clusters.p);
      check_launch("contest_group");
      k_finish<<<g, 256, 0, cx.stream>>>(touched.p, w_s, P.c_max, cw_out.p, gw.p, gcnt.p,
                                         joined.p, clusters.p);
      check_launch("finish");
      if (cx.launches) *cx.launches += 4;
    }
  }
  cc.ms_rating_kernels += rate_timer.flush();
  unsigned long long hs[ST_WORDS];
  HG_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  cc.rating_pin_visits += (int64_t)hs[ST_PINS];
  cc.rating_incidences += (int64_t)hs[ST_INCID];
  cc.rating_nodes += (int64_t)hs[ST_NODES];
}

}  // namespace hgk
