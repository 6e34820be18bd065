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
//
// Device state per level:
//   rinfo[q] = {cluster, weight word} for every pin position q:
//              the cluster word is rep[pins[q]] for the pins of rated nets
//              (2 <= |e| <= T), with every repeat of a cluster inside its net
//              replaced by -1, so a net contributes once per cluster without
//              any per-visit check (-1 for the pins of unrated nets too).  At
//              the start of a level every cluster is a singleton and the word
//              is the pin; after each sub-round the incidences of the nodes
//              that joined a cluster update it through a map from (net,
//              cluster) to the cluster's first pin index in the net.
//              The weight word is refreshed before every sub-round by one
//              streaming pass: the cluster's weight, or INT32_MAX when the
//              cluster is an unclustered node of this sub-round (never a
//              candidate).  A pin visit of the rating is then one coalesced
//              8-byte load, with no dependent gather.
//   cst[C]   = {cw[C], status[C]}: cluster weight and status (the node's
//              sub-round while it is unclustered, -1 once clustered).
//   imeta[j] = {first pin, rated size or 0, Q20 term} of the net of
//              incidence j, and lnode[x] = {u, ioff[u], ioff[u+1], c(u)} for
//              every listed node: a node's walk reads its own record, then one
//              record per incident net.
// Nodes are bucketed per level by class and sub-round.  With W(u) = sum of
// |e| over u's rated nets (the pins its rating visits) and D = min(W(u), n)
// (a bound on its distinct candidates), a team accumulates u's ratings in a
// shared-memory hash table of 2 D slots (rate_class; the D bounds are the
// autotuner's cutoffs, defaults shown):
//   class 0  D <= 256: one warp, 512 slots (eight teams per block);
//   class 1  D <= 1024: four warps, 2048 slots (two teams per block);
//   class 2  on levels whose n fits a shared table direct-indexed by cluster
//            id, W <= 32768: one block with that table; on other levels
//            D <= 2048, W <= 65536: eight warps, 4096 slots;
//   class 3  D <= 4096, W <= 65536 (other levels): one block of sixteen
//            warps (eight with 64-bit ratings), 8192 slots;
//   class 4  the rest, split over the grid: a table in global memory direct-
//            indexed by cluster id when n <= min(2 W, 65536), filled by items
//            of 32 incident nets spread over the grid (the table padded to a
//            multiple of 4 entries); else P = ceil(D / 13516) part blocks
//            (64-bit ratings: ceil(D / 9830); P <= 8) of 1024 threads, each
//            owning the candidates of one hash part in a 22528-slot (16384)
//            shared table with a list of its inserted slots; else a global
//            hash table filled by items.  A second kernel takes the argmax per
//            node (or the best of the parts' bests).
// Class 4 keeps the heaviest nodes (coarse levels: hundreds of thousands of
// pin visits per node) from serialising a sub-round on one block.  Ratings
// are accumulated in 32-bit words when the level's largest possible rating
// fits, else in 64-bit words; a hash table keeps its cluster ids and its
// ratings in separate arrays (a 32-bit CAS claims a key, an atomic add sums
// into the value).
#include <algorithm>
#include <type_traits>
#include <mutex>

#include "common.cuh"
#include "pintile.cuh"

namespace hgk {

namespace {

constexpr int NCLASS = 5;
constexpr int SPLIT_CLASS = NCLASS - 1;
constexpr int32_t D_WARP = 256;
constexpr int32_t D_PAIR = 1024;
constexpr int32_t D_QUAD = 2048;
constexpr int32_t D_BLOCK = 4096;
constexpr int32_t TEAM_W = 65536;        // largest W of a node rated by one eight-warp team
constexpr int32_t DENSE_W = 32768;       // largest W of a direct-indexed block node
constexpr int32_t SPLIT_DENSE_MAX = 65536;
constexpr int SPLIT_WARPS = 8;
constexpr int PART_THREADS = 1024;
constexpr int PART_TEAMS = 1;
// part blocks: see PartCfg (table slots and distinct candidates per part)
constexpr int32_t PART_MAX = 8;          // more parts: the node uses a global hash table
constexpr int ARGMAX_THREADS = 256;
constexpr int32_t EMPTY_KEY = -1;
constexpr size_t SMEM_BUDGET = 200 * 1024;

// per sub-round bookkeeping words
enum { CW_MOVES = 0, CW_TOUCHED = 1, CW_SLOTS = 2, CW_CURSOR = 3, CW_WORDS = 8 };
// work counters
enum { ST_PINS = 0, ST_INCID = 1, ST_NODES = 2, ST_WORDS = 4 };

// Per incidence (aligned with inets): the first pin position of its net,
// the net's size when it is rated (2 <= |e| <= T), else 0, and its Q20 term
// (0 when not rated).
struct __align__(16) IncMeta {
  int32_t start, eff;
  unsigned long long r;
};

struct RateArgs {
  const int32_t* ioff;
  const int32_t* inets;
  const int32_t* eoff;
  const int2* rinfo;  // {deduplicated cluster, weight or INT32_MAX} per pin position
  // graph levels: visits come from the adjacency array, the cluster of a
  // neighbour from rep and its weight and status from cst
  bool graph;
  const int2* adj;
  const int32_t* rep;
  // community-aware coarsening (Sec. 4): comm[v] per node, pcomm[q] =
  // comm[pins[q]] per pin position (hypergraph levels); both NULL when off.
  // A cluster's members share its community, so the pin's community is the
  // community of the pin's cluster.
  const int32_t* comm;
  const int32_t* pcomm;
  const unsigned long long* rterm;  // Q20 net term of every rated net, 0 otherwise
  // hypergraph levels: the metadata of the net of every incidence (aligned
  // with inets), so a walk reads one record per incident net
  const IncMeta* imeta;
  // {u, ioff[u], ioff[u + 1], c(u)} of every listed node: lnode is aligned
  // with list (this class and sub-round), lsplit with the split nodes
  const int4* lnode;
  const int4* lsplit;
  const int32_t* c;
  const int2* cst;  // {cw, status}
  int s, T;
  int32_t c_max, n;
  const int32_t* list;  // nodes of this (class, sub-round)
  int32_t count;
  const int32_t* clusters;
  int32_t* target;
  int32_t* gw;
  int32_t* gcnt;
  int32_t* mv;
  int32_t* touched_targets;
  int32_t* words;
  unsigned long long* stats;
  int32_t* status_word;
};

__device__ __forceinline__ uint32_t slot_hash(int32_t C) { return (uint32_t)C * 0x9E3779B1u; }

// ---------------------------------------------------- shared hash tables

// add() results besides the slot index of a new insertion
constexpr int32_t ADD_EXISTING = -1;
constexpr int32_t ADD_FULL = -2;

// 32-bit ratings: a key array and a value array (32-bit each).  An insertion
// claims the key with a 32-bit CAS and every visit adds its term with a
// 32-bit atomic add; both commute, so the sums do not depend on the order.
struct PackedHash {
  uint32_t* val;
  int32_t* key;
  uint32_t mask;
  static constexpr size_t BYTES_PER_SLOT = 8;
  __device__ __forceinline__ void init(uint32_t i) {
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
  // the slot index when C was inserted by this call, else ADD_EXISTING / ADD_FULL
  __device__ __forceinline__ int32_t add(int32_t C, uint32_t r, uint32_t max_probe = 0xFFFFFFFFu) {
    uint32_t h = slot_hash(C) & mask;
    for (uint32_t probe = 0; probe <= mask && probe < max_probe; ++probe) {
      int32_t k = key[h];
      bool fresh = false;
      if (k == EMPTY_KEY) {
        const int32_t old = atomicCAS(&key[h], EMPTY_KEY, C);
        fresh = old == EMPTY_KEY;
        k = fresh ? C : old;
      }
      if (k == C) {
        atomicAdd(&val[h], r);
        return fresh ? (int32_t)h : ADD_EXISTING;
      }
      h = (h + 1) & mask;
    }
    return ADD_FULL;
  }
  // cluster and rating of slot i (C = -1 when empty); the slot is cleared
  __device__ __forceinline__ void take(uint32_t i, int32_t& C, uint32_t& v) {
    C = key[i];
    v = val[i];
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
};

// 64-bit ratings: separate key and value arrays.
struct WideHash {
  int32_t* key;
  unsigned long long* val;
  uint32_t mask;
  static constexpr size_t BYTES_PER_SLOT = 12;
  __device__ __forceinline__ void init(uint32_t i) {
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
  __device__ __forceinline__ int32_t add(int32_t C, unsigned long long r,
                                         uint32_t max_probe = 0xFFFFFFFFu) {
    uint32_t h = slot_hash(C) & mask;
    for (uint32_t probe = 0; probe <= mask && probe < max_probe; ++probe) {
      int32_t k = key[h];
      bool fresh = false;
      if (k == EMPTY_KEY) {
        const int32_t old = atomicCAS(&key[h], EMPTY_KEY, C);
        fresh = old == EMPTY_KEY;
        k = fresh ? C : old;
      }
      if (k == C) {
        atomicAdd(&val[h], r);
        return fresh ? (int32_t)h : ADD_EXISTING;
      }
      h = (h + 1) & mask;
    }
    return ADD_FULL;
  }
  __device__ __forceinline__ void take(uint32_t i, int32_t& C, unsigned long long& v) {
    C = key[i];
    v = val[i];
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
};

// 32-bit ratings in a table of any size (not a power of two): the first slot
// is the high half of hash * slots, probing wraps at the end.  Used by the
// part blocks, whose table takes the whole shared-memory budget.
struct ModHash {
  uint32_t* val;
  int32_t* key;
  uint32_t slots;
  static constexpr size_t BYTES_PER_SLOT = 8;
  __device__ __forceinline__ void init(uint32_t i) {
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
  __device__ __forceinline__ int32_t add(int32_t C, uint32_t r) {
    uint32_t h = (uint32_t)(((uint64_t)slot_hash(C) * slots) >> 32);
    for (uint32_t probe = 0; probe < slots; ++probe) {
      int32_t k = key[h];
      bool fresh = false;
      if (k == EMPTY_KEY) {
        const int32_t old = atomicCAS(&key[h], EMPTY_KEY, C);
        fresh = old == EMPTY_KEY;
        k = fresh ? C : old;
      }
      if (k == C) {
        atomicAdd(&val[h], r);
        return fresh ? (int32_t)h : ADD_EXISTING;
      }
      h = h + 1 == slots ? 0 : h + 1;
    }
    return ADD_FULL;
  }
  __device__ __forceinline__ void take(uint32_t i, int32_t& C, uint32_t& v) {
    C = key[i];
    v = val[i];
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
};

template <typename VT> struct HashOf;
template <> struct HashOf<uint32_t> { using type = PackedHash; };
template <> struct HashOf<unsigned long long> { using type = WideHash; };

template <typename H>
__device__ __forceinline__ H make_hash(unsigned char* base, uint32_t slots);
template <>
__device__ __forceinline__ PackedHash make_hash<PackedHash>(unsigned char* base, uint32_t slots) {
  uint32_t* val = reinterpret_cast<uint32_t*>(base);
  return PackedHash{val, reinterpret_cast<int32_t*>(val + slots), slots - 1};
}
template <>
__device__ __forceinline__ ModHash make_hash<ModHash>(unsigned char* base, uint32_t slots) {
  uint32_t* val = reinterpret_cast<uint32_t*>(base);
  return ModHash{val, reinterpret_cast<int32_t*>(val + slots), slots};
}
template <>
__device__ __forceinline__ WideHash make_hash<WideHash>(unsigned char* base, uint32_t slots) {
  unsigned long long* val = reinterpret_cast<unsigned long long*>(base);
  return WideHash{reinterpret_cast<int32_t*>(val + slots), val, slots - 1};
}

// ------------------------------------------------------- the rating walk

// Visits per lane kept in flight (ILP, a template parameter of the walks):
// the record loads of ILP visits are issued before any of them is used.  The
// team kernels, whose time goes to the per-node steps, walk two at a time;
// the direct-indexed blocks, part blocks and split items, which walk the
// long visit lists of heavy nodes, four.
constexpr int TEAM_ILP = 2;
constexpr int DENSE_ILP = 4;
constexpr int PART_ILP = 4;
constexpr int SPLIT_ILP = 4;

// Adapts a per-visit adder f(C, r) to the batch interface of rate_group.
template <typename VT, int ILP, typename F>
struct EachVisit {
  F f;
  __device__ __forceinline__ void operator()(const int32_t (&C)[ILP], const VT (&rr)[ILP],
                                             const bool (&ok)[ILP]) const {
#pragma unroll
    for (int k = 0; k < ILP; ++k)
      if (ok[k]) f(C[k], rr[k]);
  }
};
template <typename VT, int ILP, typename F>
__device__ __forceinline__ EachVisit<VT, ILP, F> each_visit(F f) {
  return EachVisit<VT, ILP, F>{f};
}

// {cluster, weight word} of a batch of visits (-1 = no visit): on
// hypergraph levels q is a pin position and the record is rinfo[q]; on graph
// levels q is the neighbour node, whose cluster is rep[q] (a net of two pins
// needs no deduplication: u is a singleton, so rep[q] != u) and whose weight
// word is the cluster's weight, or INT32_MAX for an unclustered node of this
// sub-round.
// cmu >= 0: u's community; a visit in another community is dropped.
template <int ILP>
__device__ __forceinline__ void resolve_batch(const RateArgs& A, const int32_t (&q)[ILP],
                                              int2 (&ri)[ILP], int32_t cmu) {
  if (!A.graph) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) ri[k] = q[k] >= 0 ? A.rinfo[q[k]] : make_int2(-1, 0);
    if (cmu >= 0) {
#pragma unroll
      for (int k = 0; k < ILP; ++k)
        if (ri[k].x >= 0 && A.pcomm[q[k]] != cmu) ri[k].x = -1;
    }
    return;
  }
  int32_t C[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k)
    C[k] = q[k] >= 0 && (cmu < 0 || A.comm[q[k]] == cmu) ? A.rep[q[k]] : -1;
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const int2 cs = C[k] >= 0 ? A.cst[C[k]] : make_int2(0, 0);
    ri[k] = make_int2(C[k], cs.y == A.s ? 0x7fffffff : cs.x);
  }
}

// Filters a batch of visits (-1 = no visit) and hands it to `add`:
// admissible C is not u, not an unclustered node of this sub-round (weight
// word INT32_MAX), and fits c_max.
template <typename VT, int ILP, typename Add>
__device__ __forceinline__ void visit_filtered(const RateArgs& A, int32_t u, int32_t cu,
                                               const int32_t (&q)[ILP],
                                               const VT (&rr)[ILP], Add& add) {
  int2 ri[ILP];
  resolve_batch(A, q, ri, A.comm ? A.comm[u] : -1);
  int32_t C[ILP];
  bool ok[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    C[k] = ri[k].x;
    ok[k] = C[k] >= 0 && C[k] != u && (long long)ri[k].y + cu <= (long long)A.c_max;
  }
  add(C, rr, ok);
}

// Graph levels: the visits of incidences [lo, hi) of u are the other
// endpoints of its edges, each with the edge's term w(e) * 2^20 (the Q20 term
// of a two-pin net); chunk c of 32 * ILP incidences goes to warp c mod
// TW of the team.  Returns the visits in warp 0 (0 in the other warps).
template <typename VT, int ILP, typename Visit>
__device__ __forceinline__ int32_t graph_walk(const RateArgs& A, int32_t lo, int32_t hi, int wt,
                                              int TW, Visit& visit_batch) {
  constexpr int32_t CH = 32 * ILP;
  const int lane = lane_id();
  for (int32_t c0 = lo + CH * wt; c0 < hi; c0 += CH * TW) {
    int32_t q[ILP];
    VT rr[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
      const int32_t j = c0 + 32 * k + lane;
      if (j < hi) {
        const int2 a = A.adj[j];
        q[k] = a.x;
        rr[k] = (VT)((unsigned long long)(uint32_t)a.y << 20);
      } else {
        q[k] = -1;
        rr[k] = (VT)0;
      }
    }
    visit_batch(q, rr);
  }
  return wt == 0 ? hi - lo : 0;
}

// Adds one group of (up to) 32 consecutive incident nets of u, starting at
// position g0 of I(u), through `add`.  Nets of at least 32 rated pins are
// walked one at a time with the lanes over their pins; the smaller nets of
// the group are walked together over their flattened pins.  A team of TW
// warps shares the group: the chunks of 32 * ILP visits are numbered on
// from `run` (the chunks the team has walked before, for this node) and warp
// wt takes those whose number is wt modulo TW, so the team stays balanced
// across groups; `run` is advanced past the group's chunks.  Returns the
// group's pin visits in warp 0 (0 in the other warps, so the team counts each
// visit once).
// Per lane: first pin, rated size (0 if the net is not rated) and Q20 term of
// one incident net.
template <typename VT>
struct NetMeta {
  int32_t start, eff;
  VT r;
};

// The metadata of incidence j (-1: none): the first pin position of its net,
// the net's size if it is rated (else 0) and its Q20 term.
template <typename VT>
__device__ __forceinline__ NetMeta<VT> inc_meta(const RateArgs& A, int32_t j) {
  NetMeta<VT> m{0, 0, (VT)0};
  if (j >= 0) {
    const IncMeta x = A.imeta[j];
    m.start = x.start;
    m.eff = x.eff;
    m.r = (VT)x.r;
  }
  return m;
}

template <typename VT, int ILP, typename Visit>
__device__ __forceinline__ int32_t walk_group(const NetMeta<VT>& m, int wt, int TW, int32_t& run,
                                              Visit& visit_batch) {
  constexpr int32_t CH = 32 * ILP;
  const int lane = lane_id();
  const int32_t start = m.start, eff = m.eff;
  const VT r = m.r;
  // big nets, one at a time
  unsigned big = __ballot_sync(FULL, eff >= 32);
  int32_t visits = 0;
  while (big) {
    const int j = __ffs(big) - 1;
    big &= big - 1;
    const int32_t st = __shfl_sync(FULL, start, j);
    const int32_t sz = __shfl_sync(FULL, eff, j);
    const VT rj = __shfl_sync(FULL, r, j);
    const int32_t first = ((wt - run) % TW + TW) % TW;  // this warp's first chunk of the net
    run += (sz + CH - 1) / CH;
    for (int32_t q0 = CH * first; q0 < sz; q0 += CH * TW) {
      int32_t q[ILP];
      VT rr[ILP];
#pragma unroll
      for (int k = 0; k < ILP; ++k) {
        const int32_t qq = q0 + 32 * k + lane;
        q[k] = qq < sz ? st + qq : -1;
        rr[k] = rj;
      }
      visit_batch(q, rr);
    }
    visits += sz;
  }
  // small nets together
  const int32_t small = eff < 32 ? eff : 0;
  const int32_t incl = warp_inclusive_scan(small);
  const int32_t Z = __shfl_sync(FULL, incl, 31);
  const int32_t first = ((wt - run) % TW + TW) % TW;
  run += (Z + CH - 1) / CH;
  for (int32_t f0 = CH * first; f0 < Z; f0 += CH * TW) {
    int32_t q[ILP];
    VT rr[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
      const int32_t f = f0 + 32 * k + lane;
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int32_t probe = __shfl_sync(FULL, incl, j + step - 1);
        if (probe <= f) j += step;
      }
      j = j > 31 ? 31 : j;
      const int32_t incl_j = __shfl_sync(FULL, incl, j);
      const int32_t eff_j = __shfl_sync(FULL, small, j);
      const int32_t start_j = __shfl_sync(FULL, start, j);
      rr[k] = __shfl_sync(FULL, r, j);
      q[k] = f < Z ? start_j + f - (incl_j - eff_j) : -1;
    }
    visit_batch(q, rr);
  }
  return wt == 0 ? visits + Z : 0;
}

template <typename VT, int ILP, typename Visit>
__device__ __forceinline__ int32_t rate_group_raw(const RateArgs& A, int32_t g0, int32_t end,
                                                  int wt, int TW, int32_t& run, Visit& visit_batch) {
  if (A.graph) return graph_walk<VT, ILP>(A, g0, min(g0 + 32, end), wt, TW, visit_batch);
  const int32_t j = g0 + lane_id();
  return walk_group<VT, ILP>(inc_meta<VT>(A, j < end ? j : -1), wt, TW, run, visit_batch);
}

// The groups g0 = first, first + step, ... (< end) of I(u), walked as by
// rate_group_raw with the load of the next group's net metadata issued
// before the current group is walked.
template <typename VT, int ILP, typename Visit>
__device__ __forceinline__ int64_t rate_groups_raw(const RateArgs& A, int32_t first, int32_t end,
                                                   int32_t step, int wt, int TW, int32_t& run,
                                                   Visit& visit_batch) {
  const int lane = lane_id();
  int64_t visits = 0;
  if (first >= end) return 0;
  if (A.graph) {
    if (step == 32) return graph_walk<VT, ILP>(A, first, end, wt, TW, visit_batch);
    for (int32_t g = first; g < end; g += step)
      visits += graph_walk<VT, ILP>(A, g, min(g + 32, end), wt, TW, visit_batch);
    return visits;
  }
  int32_t g = first;
  NetMeta<VT> m = inc_meta<VT>(A, g + lane < end ? g + lane : -1);
  while (g < end) {
    const int32_t gn = g + step;
    const NetMeta<VT> mn = inc_meta<VT>(A, gn + lane < end ? gn + lane : -1);
    visits += walk_group<VT, ILP>(m, wt, TW, run, visit_batch);
    m = mn;
    g = gn;
  }
  return visits;
}

// rate_group_raw / rate_groups_raw with the admissibility filter of
// visit_filtered in front of `add`.
template <typename VT, int ILP, typename Add>
__device__ __forceinline__ int32_t rate_group(const RateArgs& A, int32_t u, int32_t cu, int32_t g0,
                                              int32_t end, int wt, int TW, int32_t& run, Add add) {
  auto visit = [&](const int32_t(&q)[ILP], const VT(&rr)[ILP]) HG_INLINE {
    visit_filtered<VT, ILP>(A, u, cu, q, rr, add);
  };
  return rate_group_raw<VT, ILP>(A, g0, end, wt, TW, run, visit);
}

template <typename VT, int ILP, typename Add>
__device__ __forceinline__ int64_t rate_groups(const RateArgs& A, int32_t u, int32_t cu,
                                               int32_t first, int32_t end, int32_t step, int wt,
                                               int TW, int32_t& run, Add add) {
  auto visit = [&](const int32_t(&q)[ILP], const VT(&rr)[ILP]) HG_INLINE {
    visit_filtered<VT, ILP>(A, u, cu, q, rr, add);
  };
  return rate_groups_raw<VT, ILP>(A, first, end, step, wt, TW, run, visit);
}

template <typename VT>
__device__ __forceinline__ void better(VT& bv, int32_t& bc, VT v, int32_t C) {
  if (C >= 0 && (bc < 0 || v > bv || (v == bv && C < bc))) {
    bv = v;
    bc = C;
  }
}

template <typename VT>
__device__ __forceinline__ void warp_argmax(VT& best_v, int32_t& best_c) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const VT ov = __shfl_xor_sync(FULL, best_v, d);
    const int32_t oc = __shfl_xor_sync(FULL, best_c, d);
    better(best_v, best_c, ov, oc);
  }
}

__device__ __forceinline__ void publish(const RateArgs& A, int32_t u, int32_t best_c) {
  A.target[u] = best_c;
  if (best_c >= 0) {
    A.mv[atomicAdd(&A.words[CW_MOVES], 1)] = u;
    atomicAdd(&A.gw[best_c], A.c[u]);
    if (atomicAdd(&A.gcnt[best_c], 1) == 0)
      A.touched_targets[atomicAdd(&A.words[CW_TOUCHED], 1)] = best_c;
  }
}

__device__ __forceinline__ bool subround_stopped(const RateArgs& A) {
  return 5ll * (long long)(*A.clusters) <= 2ll * (long long)A.n;
}

// Synchronises the TW warps of team `team` (TW = 1: the warp; TW = warps per
// block: the block; else a named barrier per team).
template <int TW>
__device__ __forceinline__ void team_sync(int team) {
  if (TW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TW * 32) : "memory");
  }
}

// classes 0-2 with hash tables: TEAMS teams of TW warps per block, each team
// rating one node at a time with a SLOTS-slot shared hash table
// Shared memory of one team: the hash slots, then a list of the slots the
// current node inserted (capacity slots / 2: a class's distinct bound).
template <typename H>
constexpr size_t team_bytes(uint32_t slots) {
  return (size_t)slots * H::BYTES_PER_SLOT + (size_t)(slots / 2) * sizeof(int32_t);
}

template <typename VT, int TW, int TEAMS>
__global__ void __launch_bounds__(TW * 32 * TEAMS, 1024 / (TW * 32 * TEAMS)) k_rate_team(RateArgs A, uint32_t slots) {
  using H = typename HashOf<VT>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VT s_rv[TEAMS][TW];
  __shared__ int32_t s_rc[TEAMS][TW];
  __shared__ int32_t s_nused[TEAMS][2];
  if (subround_stopped(A)) return;
  const int team = warp_in_block() / TW, wt = warp_in_block() % TW;
  const int tid = threadIdx.x % (TW * 32), nthr = TW * 32;
  unsigned char* base = smem + (size_t)team * team_bytes<H>(slots);
  H tab = make_hash<H>(base, slots);
  int32_t* used = reinterpret_cast<int32_t*>(base + (size_t)slots * H::BYTES_PER_SLOT);
  for (uint32_t i = tid; i < slots; i += nthr) tab.init(i);
  if (tid == 0) s_nused[team][0] = s_nused[team][1] = 0;
  team_sync<TW>(team);
  int64_t visits = 0, incid = 0, nodes = 0;
  int it = 0;
  for (int32_t i = blockIdx.x * TEAMS + team; i < A.count; i += gridDim.x * TEAMS) {
    const int4 nd = A.lnode[i];
    const int32_t u = nd.x, beg = nd.y, end = nd.z, cu = nd.w;
    if (A.cst[u].y < 0) continue;  // joined a cluster in an earlier sub-round
    // the used-slot counter of this node; the other one is cleared for the
    // next node once every thread has read this one
    int32_t* nused = &s_nused[team][it & 1];
    int32_t run = 0;
    visits += rate_groups<VT, TEAM_ILP>(A, u, cu, beg, end, 32, wt, TW, run,
                                        each_visit<VT, TEAM_ILP>([&](int32_t C, VT r) HG_INLINE {
                                const int32_t sl = tab.add(C, r);
                                if (sl >= 0) used[atomicAdd(nused, 1)] = sl;
                                else if (sl == ADD_FULL) dev_fail(A.status_word, DEV_HASH_FULL);
                              }));
    team_sync<TW>(team);
    VT bv = 0;
    int32_t bc = -1;
    const int32_t nu = *nused;
    if (tid == 0) s_nused[team][(it + 1) & 1] = 0;
    for (int32_t x = tid; x < nu; x += nthr) {
      int32_t C;
      VT v;
      tab.take((uint32_t)used[x], C, v);
      better(bv, bc, v, C);
    }
    warp_argmax(bv, bc);
    if (TW > 1) {
      if (lane_id() == 0) {
        s_rv[team][wt] = bv;
        s_rc[team][wt] = bc;
      }
      team_sync<TW>(team);
      // the team's first warp combines and publishes while the others go on
      // to the next node (the slots and results it reads are not written
      // again before the next node's first barrier)
      if (wt == 0) {
        bv = lane_id() < TW ? s_rv[team][lane_id()] : (VT)0;
        bc = lane_id() < TW ? s_rc[team][lane_id()] : -1;
        warp_argmax(bv, bc);
      }
    } else {
      __syncwarp();
    }
    if (tid == 0) publish(A, u, bc);
    incid += end - beg;
    ++nodes;
    ++it;
  }
  if (lane_id() == 0 && visits) atomicAdd(&A.stats[ST_PINS], (unsigned long long)visits);
  if (tid == 0 && nodes) {
    atomicAdd(&A.stats[ST_INCID], (unsigned long long)incid);
    atomicAdd(&A.stats[ST_NODES], (unsigned long long)nodes);
  }
}

// class 2 on small levels: one block per node with a table direct-indexed by
// cluster id (n values, then the list of touched ids)
template <typename VT>
__global__ void __launch_bounds__(256, 4) k_rate_dense(RateArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t s_nused[2];
  __shared__ VT s_rv[8];
  __shared__ int32_t s_rc[8];
  if (subround_stopped(A)) return;
  const uint32_t cap = (uint32_t)A.n;
  VT* val = reinterpret_cast<VT*>(smem);
  int32_t* used = reinterpret_cast<int32_t*>(val + cap);
  for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) val[i] = 0;
  if (threadIdx.x == 0) s_nused[0] = s_nused[1] = 0;
  __syncthreads();
  const int nw = blockDim.x >> 5, wv = warp_in_block();
  int64_t visits = 0, incid = 0, nodes = 0;
  int it = 0;
  for (int32_t i = blockIdx.x; i < A.count; i += gridDim.x) {
    const int4 nd = A.lnode[i];
    const int32_t u = nd.x, beg = nd.y, end = nd.z, cu = nd.w;
    if (A.cst[u].y < 0) continue;
    // touched-id counter of this node; the other one is cleared for the next
    // node once every thread has read this one
    int32_t* nused = &s_nused[it & 1];
    int32_t run = 0;
    visits += rate_groups<VT, DENSE_ILP>(A, u, cu, beg, end, 32, wv, nw, run,
                                         each_visit<VT, DENSE_ILP>([&](int32_t C, VT r) HG_INLINE {
                                // every term is >= 1, so a zero before the add
                                // marks the first touch
                                if (atomicAdd(&val[C], r) == (VT)0)
                                  used[atomicAdd(nused, 1)] = C;
                              }));
    __syncthreads();
    VT bv = 0;
    int32_t bc = -1;
    const int32_t nu = *nused;
    if (threadIdx.x == 0) s_nused[(it + 1) & 1] = 0;
    for (int32_t x = threadIdx.x; x < nu; x += blockDim.x) {
      const int32_t C = used[x];
      better(bv, bc, val[C], C);
      val[C] = 0;
    }
    warp_argmax(bv, bc);
    if (lane_id() == 0) {
      s_rv[wv] = bv;
      s_rc[wv] = bc;
    }
    __syncthreads();
    // warp 0 combines and publishes while the other warps start the next node
    if (wv == 0) {
      bv = lane_id() < nw ? s_rv[lane_id()] : (VT)0;
      bc = lane_id() < nw ? s_rc[lane_id()] : -1;
      warp_argmax(bv, bc);
      if (lane_id() == 0) {
        publish(A, u, bc);
        incid += end - beg;
        ++nodes;
      }
    }
    ++it;
  }
  if (lane_id() == 0 && visits) atomicAdd(&A.stats[ST_PINS], (unsigned long long)visits);
  if (threadIdx.x == 0 && nodes) {
    atomicAdd(&A.stats[ST_INCID], (unsigned long long)incid);
    atomicAdd(&A.stats[ST_NODES], (unsigned long long)nodes);
  }
}

// class 3, phase 1: one warp per item (a class-3 node of the sub-round and
// one group of 32 of its incident nets); accumulates into the node's global
// table at tab_off[i] - tab_base (values; keys in hash mode; the list of
// used slots with its counter tnused[i])
template <typename VT>
__global__ void __launch_bounds__(SPLIT_WARPS * 32, 1024 / (SPLIT_WARPS * 32))
k_rate_split_acc(RateArgs A, const int32_t* __restrict__ split, const int32_t* __restrict__ item_node,
                 const int32_t* __restrict__ item_off, const int64_t* __restrict__ tab_off,
                 const int64_t* __restrict__ tab_cap, const int8_t* __restrict__ tab_dense,
                 int32_t item_lo, int32_t item_hi, int64_t tab_base, int32_t* __restrict__ tkey,
                 VT* __restrict__ tval, int32_t* __restrict__ tused, int32_t* __restrict__ tnused) {
  if (subround_stopped(A)) return;
  int64_t visits = 0, incid = 0;
  for (int32_t t = item_lo + blockIdx.x * SPLIT_WARPS + warp_in_block(); t < item_hi;
       t += gridDim.x * SPLIT_WARPS) {
    const int32_t i = item_node[t];
    const int4 nd = A.lsplit[i];
    const int32_t u = nd.x, beg = nd.y, end = nd.z, cu = nd.w;
    if (A.cst[u].y < 0) continue;
    const int32_t g0 = beg + 32 * (t - item_off[i]);
    const int64_t base = tab_off[i] - tab_base;
    VT* val = tval + base;
    int32_t* used = tused + base;
    int32_t* nused = tnused + i;
    int32_t run = 0;
    if (tab_dense[i]) {
      // direct-indexed: a reduction without a returned value; the argmax
      // scans the whole table, which is no larger than twice the visits
      visits += rate_group<VT, SPLIT_ILP>(A, u, cu, g0, end, 0, 1, run,
                                          each_visit<VT, SPLIT_ILP>([&](int32_t C, VT r) HG_INLINE {
        atomicAdd(&val[C], r);
      }));
    } else {
      int32_t* key = tkey + base;
      const uint32_t mask = (uint32_t)tab_cap[i] - 1;
      visits += rate_group<VT, SPLIT_ILP>(
          A, u, cu, g0, end, 0, 1, run,
          [&](const int32_t(&C)[SPLIT_ILP], const VT(&rr)[SPLIT_ILP], const bool(&ok)[SPLIT_ILP]) HG_INLINE {
            // the first slot of every visit of the batch is loaded at once
            uint32_t h[SPLIT_ILP];
            int32_t k0[SPLIT_ILP];
#pragma unroll
            for (int k = 0; k < SPLIT_ILP; ++k) {
              h[k] = slot_hash(C[k]) & mask;
              k0[k] = ok[k] ? key[h[k]] : C[k];
            }
#pragma unroll
            for (int k = 0; k < SPLIT_ILP; ++k) {
              if (!ok[k]) continue;
              uint32_t hh = h[k];
              int32_t kk = k0[k];
              bool found = false;
              for (uint32_t probe = 0; probe <= mask; ++probe) {
                if (kk == C[k]) {
                  found = true;
                  break;
                }
                if (kk == EMPTY_KEY) {
                  const int32_t old = atomicCAS(&key[hh], EMPTY_KEY, C[k]);
                  if (old == EMPTY_KEY) used[atomicAdd(nused, 1)] = (int32_t)hh;
                  if (old == EMPTY_KEY || old == C[k]) {
                    found = true;
                    break;
                  }
                }
                hh = (hh + 1) & mask;
                kk = key[hh];
              }
              if (found) atomicAdd(&val[hh], rr[k]);
              else dev_fail(A.status_word, DEV_HASH_FULL);
            }
          });
    }
    incid += min(32, end - g0);
  }
  if (lane_id() == 0 && visits) {
    atomicAdd(&A.stats[ST_PINS], (unsigned long long)visits);
    atomicAdd(&A.stats[ST_INCID], (unsigned long long)incid);
  }
}

// Hashed split nodes whose distinct candidates need more than one shared
// table: the candidates are partitioned over P blocks by a hash of the
// cluster id (part_of).  Every block walks all of the node's visits (the pin
// clusters are read P times, from L2 at the levels where this happens) and
// accumulates the candidates of its part in a shared table (PartCfg);
// P = ceil(min(W, n) / PartCfg::D) keeps every table at most 60 % full, so no
// insertion can fail.  A node of one part publishes its argmax directly;
// otherwise each part leaves its best (rating, cluster) for the per-node
// combine in k_rate_split_argmax.  All warps of the block walk the node's
// groups of 32 nets, sharing the chunks in turn.
// Table of a part block: SLOTS shared slots holding at most D distinct
// candidates per part (60 % load), and a list of the inserted slots of
// capacity CAP (more insertions: the whole table is scanned).  32-bit
// ratings take the whole shared-memory budget (22,528 slots, so fewer nodes
// need more than one part and every part re-reads the node's visits);
// 64-bit ratings 16,384 slots.
template <typename VT> struct PartCfg {
  using Hash = WideHash;
  static constexpr uint32_t SLOTS = 16384, CAP = 2048;
  static constexpr int32_t D = 9830;
};
template <> struct PartCfg<uint32_t> {
  using Hash = ModHash;
  static constexpr uint32_t SLOTS = 22528, CAP = 10240;
  static constexpr int32_t D = 13516;
};
template <typename VT>
constexpr size_t part_bytes() {
  return (size_t)PartCfg<VT>::SLOTS * PartCfg<VT>::Hash::BYTES_PER_SLOT +
         (size_t)PartCfg<VT>::CAP * 4;
}

__device__ __forceinline__ int32_t part_of(int32_t C, int32_t P) {
  return (int32_t)(((uint64_t)((uint32_t)C * 0x85EBCA77u) * (uint32_t)P) >> 32);
}

template <typename VT>
__global__ void __launch_bounds__(PART_THREADS)
k_rate_part(RateArgs A, const int32_t* __restrict__ split, const int32_t* __restrict__ part_node,
            const int32_t* __restrict__ part_off, int32_t part_lo, int32_t part_hi,
            VT* __restrict__ res_v, int32_t* __restrict__ res_c) {
  using H = typename PartCfg<VT>::Hash;
  constexpr uint32_t PART_SLOTS = PartCfg<VT>::SLOTS;
  constexpr int NW = PART_THREADS / 32, TW = NW / PART_TEAMS;
  constexpr uint32_t CAP = PartCfg<VT>::CAP;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ VT s_rv[NW];
  __shared__ int32_t s_rc[NW];
  __shared__ int32_t s_nused[2];
  if (subround_stopped(A)) return;
  H tab = make_hash<H>(smem, PART_SLOTS);
  int32_t* used = reinterpret_cast<int32_t*>(smem + (size_t)PART_SLOTS * H::BYTES_PER_SLOT);
  for (uint32_t x = threadIdx.x; x < PART_SLOTS; x += blockDim.x) tab.init(x);
  if (threadIdx.x == 0) s_nused[0] = s_nused[1] = 0;
  __syncthreads();
  const int wv = warp_in_block(), team = wv / TW, wt = wv % TW;
  int64_t visits = 0, incid = 0, nodes = 0;
  int it = 0;
  for (int32_t t = part_lo + blockIdx.x; t < part_hi; t += gridDim.x) {
    const int32_t i = part_node[t];
    const int4 nd = A.lsplit[i];
    const int32_t u = nd.x, beg = nd.y, end = nd.z, cu = nd.w;
    if (A.cst[u].y < 0) continue;  // joined a cluster in an earlier sub-round
    const int32_t P = part_off[i + 1] - part_off[i], k = t - part_off[i];
    // slots inserted for this part (listed while they fit the list); the
    // other counter is cleared for the next part once every thread has read
    // this one
    int32_t* nused = &s_nused[it & 1];
    const int32_t cmu = A.comm ? A.comm[u] : -1;
    auto visit = [&](const int32_t(&q)[PART_ILP], const VT(&rr)[PART_ILP]) HG_INLINE {
      int2 ri[PART_ILP];
      resolve_batch(A, q, ri, cmu);
#pragma unroll
      for (int j = 0; j < PART_ILP; ++j) {
        const int32_t Cj = ri[j].x;
        if (Cj < 0 || Cj == u || (P != 1 && part_of(Cj, P) != k) ||
            (long long)ri[j].y + cu > (long long)A.c_max)
          continue;
        const int32_t sl = tab.add(Cj, rr[j]);
        if (sl >= 0) {
          const int32_t x = atomicAdd(nused, 1);
          if (x < (int32_t)CAP) used[x] = sl;
        } else if (sl == ADD_FULL) {
          dev_fail(A.status_word, DEV_HASH_FULL);
        }
      }
    };
    int32_t run = 0;
    const int64_t v = rate_groups_raw<VT, PART_ILP>(A, beg + 32 * team, end, 32 * PART_TEAMS, wt, TW, run,
                                          visit);
    if (k == 0) visits += v;
    __syncthreads();
    const int32_t nu = *nused;
    if (threadIdx.x == 0) s_nused[(it + 1) & 1] = 0;
    VT bv = 0;
    int32_t bc = -1;
    if (nu <= (int32_t)CAP) {
      for (int32_t x = threadIdx.x; x < nu; x += blockDim.x) {
        int32_t C;
        VT val;
        tab.take((uint32_t)used[x], C, val);
        better(bv, bc, val, C);
      }
    } else {  // more insertions than the list holds: every slot
      for (uint32_t x = threadIdx.x; x < PART_SLOTS; x += blockDim.x) {
        int32_t C;
        VT val;
        tab.take(x, C, val);
        better(bv, bc, val, C);
      }
    }
    warp_argmax(bv, bc);
    if (lane_id() == 0) {
      s_rv[wv] = bv;
      s_rc[wv] = bc;
    }
    __syncthreads();
    // warp 0 combines and publishes while the other warps start the next
    // part (the table is clear, and s_rv / s_rc are written again only after
    // the next part's first barrier)
    if (wv == 0) {
      bv = lane_id() < NW ? s_rv[lane_id()] : (VT)0;
      bc = lane_id() < NW ? s_rc[lane_id()] : -1;
      warp_argmax(bv, bc);
      if (lane_id() == 0) {
        if (P == 1) {
          publish(A, u, bc);
          ++nodes;
        } else {
          res_v[t] = bv;
          res_c[t] = bc;
        }
        if (k == 0) incid += end - beg;
      }
    }
    ++it;
  }
  if (lane_id() == 0 && visits) atomicAdd(&A.stats[ST_PINS], (unsigned long long)visits);
  if (threadIdx.x == 0 && (incid || nodes)) {
    atomicAdd(&A.stats[ST_INCID], (unsigned long long)incid);
    atomicAdd(&A.stats[ST_NODES], (unsigned long long)nodes);
  }
}

// class 3, phase 2: one block per class-3 node of the sub-round: argmax over
// its used slots, which are cleared on the way for the next sub-round
template <typename VT>
__global__ void __launch_bounds__(ARGMAX_THREADS)
k_rate_split_argmax(RateArgs A, const int32_t* __restrict__ split, int32_t lo, int32_t hi,
                    const int64_t* __restrict__ tab_off, const int64_t* __restrict__ tab_cap,
                    const int8_t* __restrict__ tab_dense,
                    int64_t tab_base, int32_t* __restrict__ tkey, VT* __restrict__ tval,
                    const int32_t* __restrict__ tused, int32_t* __restrict__ tnused,
                    const int32_t* __restrict__ part_off, const VT* __restrict__ res_v,
                    const int32_t* __restrict__ res_c) {
  __shared__ VT s_rv[32];
  __shared__ int32_t s_rc[32];
  if (subround_stopped(A)) return;
  for (int32_t i = lo + blockIdx.x; i < hi; i += gridDim.x) {
    const int32_t u = split[i];
    if (A.cst[u].y < 0) continue;
    const bool dense = tab_dense[i] != 0;
    const int32_t P = part_off[i + 1] - part_off[i];
    if (P == 1) continue;  // published by its only part
    const int64_t base = tab_off[i] - tab_base;
    VT bv = 0;
    int32_t bc = -1;
    if (P > 1) {
      // the parts hold disjoint candidates: the best of their bests
      for (int32_t t = part_off[i] + threadIdx.x; t < part_off[i + 1]; t += blockDim.x)
        better(bv, bc, res_v[t], res_c[t]);
    } else if (dense) {
      // 16-byte loads over the whole table (every table offset and capacity
      // is a multiple of 4 entries); only vectors holding a rating are
      // cleared
      constexpr int PER = 16 / (int)sizeof(VT);
      using V = typename std::conditional<sizeof(VT) == 4, uint4, ulonglong2>::type;
      const int32_t nvec = (int32_t)tab_cap[i] / PER;
      V* tv = reinterpret_cast<V*>(tval + base);
      for (int32_t x = threadIdx.x; x < nvec; x += blockDim.x) {
        const V vv = tv[x];
        const VT* e = reinterpret_cast<const VT*>(&vv);
        bool any = false;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          if (e[q] == (VT)0) continue;
          any = true;
          better(bv, bc, e[q], x * PER + q);
        }
        if (any) tv[x] = V{};
      }
    } else {
      const int32_t nu = tnused[i];
      for (int32_t x = threadIdx.x; x < nu; x += blockDim.x) {
        const int32_t sl = tused[base + x];
        better(bv, bc, tval[base + sl], tkey[base + sl]);
        tval[base + sl] = 0;
        tkey[base + sl] = EMPTY_KEY;
      }
    }
    warp_argmax(bv, bc);
    const int nw = blockDim.x >> 5;
    if (lane_id() == 0) {
      s_rv[warp_in_block()] = bv;
      s_rc[warp_in_block()] = bc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int x = 1; x < nw; ++x) better(bv, bc, s_rv[x], s_rc[x]);
      tnused[i] = 0;
      publish(A, u, bc);
      atomicAdd(&A.stats[ST_NODES], 1ull);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- node bucketing

// Team class of a node from W(u) and D = min(W(u), n):
//   0 warp (512 slots)                     D <= 256
//   1 four warps (2048 slots)              D <= 1024 (unless the level is dense)
//   2 block, direct-indexed                the level fits a dense shared table,
//                                          W <= 32768
//     eight warps, 4096-slot hash          D <= 2048, W <= 65536 (other levels)
//   3 sixteen warps, 8192-slot hash        D <= 4096, W <= 65536 (other levels)
//   4 split over the grid                  the rest
__device__ __forceinline__ int rate_class(int64_t W, int32_t n, bool dense_block, RateCuts cut) {
  const int64_t D = W < n ? W : n;  // bound on the distinct candidate clusters
  if (D <= cut.warp) return 0;
  if (dense_block && W <= DENSE_W) return 2;
  if (D <= cut.pair) return 1;
  if (!dense_block && W <= TEAM_W) {
    if (D <= cut.quad) return 2;
    if (D <= cut.block) return 3;
  }
  return 4;
}

// W(u) (pins of rated nets, or rated incident edges on graph levels) of every
// node, and the largest bound on a node's rating (sum of its net terms),
// which decides the value width.
// floor(w(e) * 2^20 / (|e| - 1)) for the rated nets (2 <= |e| <= T), else 0;
// at least 1 for a rated net since |e| - 1 < 2^20.
__global__ void k_net_terms(const int32_t* __restrict__ eoff, const int32_t* __restrict__ w,
                            int32_t m, int T, unsigned long long* __restrict__ rterm) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sz = eoff[e + 1] - eoff[e];
    rterm[e] = (sz >= 2 && sz <= T)
                   ? (((unsigned long long)w[e]) << 20) / (unsigned long long)(sz - 1)
                   : 0ull;
  }
}

// IncMeta of every incidence of a hypergraph level.
__global__ void k_inc_meta(const int32_t* __restrict__ inets, const int32_t* __restrict__ eoff,
                           const unsigned long long* __restrict__ rterm, int64_t p,
                           IncMeta* __restrict__ imeta) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = inets[j];
    const unsigned long long r = rterm[e];
    IncMeta x;
    x.start = eoff[e];
    x.eff = r != 0 ? eoff[e + 1] - x.start : 0;
    x.r = r;
    imeta[j] = x;
  }
}

// {u, ioff[u], ioff[u + 1], c(u)} of every listed node.
__global__ void k_list_nodes(const int32_t* __restrict__ list, int32_t cnt,
                             const int32_t* __restrict__ ioff, const int32_t* __restrict__ c,
                             int4* __restrict__ lnode) {
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < cnt; x += gridDim.x * blockDim.x) {
    const int32_t u = list[x];
    lnode[x] = make_int4(u, ioff[u], ioff[u + 1], c[u]);
  }
}

// One warp per node, lanes over its incident nets.
__global__ void k_node_work(const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets,
                            const int32_t* __restrict__ eoff,
                            const unsigned long long* __restrict__ rterm, int32_t n, bool graph,
                            int32_t* __restrict__ wof, unsigned long long* __restrict__ max_r) {
  unsigned long long lr = 0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    long long W = 0;
    unsigned long long R = 0;
    for (int32_t j = ioff[u] + lane_id(); j < ioff[u + 1]; j += 32) {
      const int32_t e = inets[j];
      const unsigned long long r = rterm[e];
      if (r != 0) {
        W += graph ? 1 : eoff[e + 1] - eoff[e];  // a graph visits the other endpoint only
        R += r;
      }
    }
    W = warp_sum(W);
    R = warp_sum(R);
    lr = R > lr ? R : lr;
    if (lane_id() == 0) wof[u] = W > 0x7fffffff ? 0x7fffffff : (int32_t)W;
  }
  if (lane_id() == 0 && lr) atomicMax(max_r, lr);
}

// key = class * S + sub-round of every node with W(u) > 0, and the counts.
__global__ void k_node_classify(const int32_t* __restrict__ wof, int32_t n, uint64_t seed,
                                int level, int S, bool dense_block, RateCuts cut,
                                int32_t* __restrict__ key_of, int32_t* __restrict__ kcount) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t W = wof[u];
    int32_t key = -1;
    if (W > 0) {
      key = rate_class(W, n, dense_block, cut) * S +
            subround_of_node_cluster(seed, level, (int)u, S);
      atomicAdd(&kcount[key], 1);
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
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const int64_t u = b + lane_id();
    const bool valid = u < n;
    const int32_t key = valid ? key_of[u] : -1;
    const int32_t slot = warp_claim_slot(kfill, key, __ballot_sync(FULL, valid));
    if (slot >= 0) list[s_off[key] + slot] = (int32_t)u;
  }
}

// Work items and global table of every split node (D = min(W(u), n)):
//   direct-indexed global table (n entries) when n <= min(2 W(u), 65536), so
//   the table costs no more than the accumulation: groups of 32 nets over
//   the grid (items);
//   else P = ceil(D / part_d) shared-memory parts when P <= PART_MAX (no
//   global table);
//   else a global hash table of a power of two >= 2 D + 2 slots, with items.
__global__ void k_split_sizes(const int32_t* __restrict__ split, int32_t nsplit,
                              const int32_t* __restrict__ ioff, const int32_t* __restrict__ wof,
                              int32_t n, int32_t part_d, int32_t* __restrict__ items,
                              int32_t* __restrict__ parts, int32_t* __restrict__ cap,
                              int8_t* __restrict__ dense) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nsplit; i += gridDim.x * blockDim.x) {
    const int32_t u = split[i];
    const int32_t deg = ioff[u + 1] - ioff[u];
    const bool d = n <= SPLIT_DENSE_MAX && (int64_t)n <= 2 * (int64_t)wof[u];
    const int32_t D = min(wof[u], n);
    const int32_t P = d ? 0 : (D + part_d - 1) / part_d;
    const bool part = !d && P <= PART_MAX;
    items[i] = part ? 0 : (deg + 31) / 32;
    parts[i] = part ? P : 0;
    dense[i] = d ? 1 : 0;
    if (d) {
      cap[i] = (n + 3) & ~3;  // a multiple of 4: every table starts 16-byte aligned
    } else if (part) {
      cap[i] = 0;
    } else {
      const int64_t want = 2 * (int64_t)D + 2;
      int64_t c = 1;
      while (c < want) c <<= 1;
      cap[i] = (int32_t)c;
    }
  }
}

__global__ void k_split_items(const int32_t* __restrict__ item_off, int32_t nsplit,
                              int32_t* __restrict__ item_node) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nsplit; i += gridDim.x * blockDim.x)
    for (int32_t t = item_off[i]; t < item_off[i + 1]; ++t) item_node[t] = i;
}

__global__ void k_widen(const int32_t* __restrict__ in, int64_t* __restrict__ out, int32_t cnt) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    out[i] = in[i];
}

template <typename VT>
__global__ void k_init_table(int32_t* key, VT* val, size_t cnt) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (size_t)gridDim.x * blockDim.x) {
    key[i] = EMPTY_KEY;
    val[i] = 0;
  }
}

// ------------------------------------------------------------- approval

__global__ void k_approve(const int32_t* __restrict__ mv, const int32_t* __restrict__ words,
                          const int32_t* __restrict__ target, int2* __restrict__ cst,
                          const int32_t* __restrict__ gw, const int32_t* __restrict__ gcnt,
                          int32_t c_max, int32_t* __restrict__ rep, int32_t* __restrict__ slot_of,
                          int32_t* __restrict__ slot_c, int32_t* __restrict__ slot_off,
                          int32_t* __restrict__ wslots, int32_t* __restrict__ wcursor) {
  const int32_t nm = words[CW_MOVES];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const int32_t u = mv[i];
    const int32_t C = target[u];
    if ((long long)cst[C].x + gw[C] <= (long long)c_max) {
      rep[u] = C;   // fast path: every move into C fits
      cst[u].y = -1;
    } else if (atomicCAS(&slot_of[C], -1, -2) == -1) {
      const int32_t sl = atomicAdd(wslots, 1);
      slot_c[sl] = C;
      slot_off[sl] = atomicAdd(wcursor, gcnt[C]);
      slot_of[C] = sl;
    }
  }
}

__global__ void k_contest_scatter(const int32_t* __restrict__ mv, const int32_t* __restrict__ words,
                                  const int32_t* __restrict__ target, const int2* __restrict__ cst,
                                  const int32_t* __restrict__ gw, int32_t c_max,
                                  const int32_t* __restrict__ slot_of,
                                  const int32_t* __restrict__ slot_off,
                                  int32_t* __restrict__ slot_fill, int32_t* __restrict__ glist) {
  const int32_t nm = words[CW_MOVES];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const int32_t u = mv[i];
    const int32_t C = target[u];
    if ((long long)cst[C].x + gw[C] > (long long)c_max) {
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
__global__ void __launch_bounds__(GROUP_THREADS, 1024 / GROUP_THREADS)
k_contest_group(const int32_t* __restrict__ words, const int32_t* __restrict__ slot_c,
                const int32_t* __restrict__ slot_off, int32_t* __restrict__ slot_fill,
                int32_t* __restrict__ slot_of, const int32_t* __restrict__ glist,
                const int32_t* __restrict__ gcnt, const int32_t* __restrict__ c, int32_t c_max,
                int2* __restrict__ cst, int32_t* __restrict__ rep, int32_t* __restrict__ clusters) {
  __shared__ unsigned long long s_keys[GROUP_SMEM_CAP];
  __shared__ long long s_red[32];
  __shared__ unsigned long long s_acc;
  const int32_t nslots = words[CW_SLOTS];
  for (int32_t sl = blockIdx.x; sl < nslots; sl += gridDim.x) {
    const int32_t C = slot_c[sl];
    const int32_t cnt = gcnt[C];
    const int32_t off = slot_off[sl];
    const long long cap = (long long)c_max - cst[C].x;
    long long added = 0;
    int32_t acc = 0;
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
      if (threadIdx.x == 0) s_acc = 0;
      __syncthreads();
      group_bitonic(s_keys, P);
      // the accepted count is the number of positions whose inclusive weight
      // prefix is <= cap (weights are positive, so these form a prefix)
      long long carry = 0;
      for (int base = 0; base < cnt; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < cnt ? (long long)(s_keys[i] >> 32) : 0;
        const long long x = warp_inclusive_scan(v);
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
        if (i < cnt && incl <= cap) atomicAdd(&s_acc, 1ull);
        carry += chunk_total;
        __syncthreads();
      }
      acc = (int32_t)s_acc;
      for (int i = threadIdx.x; i < acc; i += blockDim.x) {
        const int32_t u = (int32_t)(s_keys[i] & 0xffffffffu);
        rep[u] = C;
        cst[u].y = -1;
        added += (long long)(s_keys[i] >> 32);
      }
    } else {
      // large group: binary search for the first excluded key x, the largest
      // x with (sum of c over keys < x) <= cap; all keys < x are accepted
      unsigned long long lo = 0, hi = (1ull << 63);
      while (hi - lo > 1) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        long long f = 0;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
          const int32_t u = glist[off + i];
          const unsigned long long kk = ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)u;
          if (kk < mid) f += c[u];
        }
        f = block_sum(f, s_red);
        if (f <= cap) lo = mid; else hi = mid;
      }
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int32_t u = glist[off + i];
        const unsigned long long kk = ((unsigned long long)(uint32_t)c[u] << 32) | (uint32_t)u;
        if (kk < lo) {
          rep[u] = C;
          cst[u].y = -1;
          added += c[u];
          ++acc;
        }
      }
      acc = (int32_t)block_sum((long long)acc, s_red);
    }
    added = block_sum(added, s_red);
    if (threadIdx.x == 0) {
      cst[C].x += (int32_t)added;
      if (acc > 0) {
        cst[C].y = -1;
        atomicSub(clusters, acc);
      }
      slot_of[C] = -1;
      slot_fill[sl] = 0;
    }
    __syncthreads();
  }
}

// Uncontested targets: add the summed weight of their movers; reset the sums.
__global__ void k_finish(const int32_t* __restrict__ touched, const int32_t* __restrict__ words,
                         int32_t c_max, int2* __restrict__ cst, int32_t* __restrict__ gw,
                         int32_t* __restrict__ gcnt, int32_t* __restrict__ clusters) {
  const int32_t nt = words[CW_TOUCHED];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
    const int32_t C = touched[i];
    const int32_t cw = cst[C].x;
    if ((long long)cw + gw[C] <= (long long)c_max) {
      cst[C] = make_int2(cw + gw[C], -1);
      atomicSub(clusters, gcnt[C]);
    }
    gw[C] = 0;
    gcnt[C] = 0;
  }
}

// ------------------------------------------ cluster word maintenance

// The first position of every cluster in every rated net is kept in a global
// hash map keyed by (net, cluster): at the start of a level every pin is its
// own cluster, so the map holds (e, pins[q]) -> q for all rated pins.  When a
// node v joins cluster C, for each rated net e of v at pin index q: an
// atomicMin of q into (e, C) finds whether q becomes C's first position in e
// (then the position it displaces, if any, gets cluster word -1 in rinfo)
// and, in a second pass, the cluster word of q becomes C if q is the first
// position of C in e, else -1.
// The work per sub-round is the degree of the nodes that joined.
struct PosMap {
  unsigned long long* key;  // net << 32 | cluster, all ones when empty
  int32_t* pos;             // smallest pin index, INT32_MAX when none yet
  uint64_t mask;
};

__device__ __forceinline__ int64_t posmap_slot(const PosMap& M, int32_t e, int32_t C) {
  const unsigned long long mine = ((unsigned long long)(uint32_t)e << 32) | (uint32_t)C;
  uint64_t h = mix64(mine) & M.mask;
  for (uint64_t probe = 0; probe <= M.mask; ++probe) {
    unsigned long long k = M.key[h];
    if (k == ~0ull) {
      const unsigned long long old = atomicCAS(&M.key[h], ~0ull, mine);
      k = old == ~0ull ? mine : old;
    }
    if (k == mine) return (int64_t)h;
    h = (h + 1) & M.mask;
  }
  return -1;
}

// (e, pins[q]) -> q for every pin of every rated net (pin tiles).
__global__ void __launch_bounds__(PIN_TILE_THREADS)
k_posmap_init(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
              const int32_t* __restrict__ tile_net, int32_t m, int64_t p, int T, PosMap M,
              int32_t* status) {
  __shared__ int32_t s_off[PIN_TILE + 3];
  const int64_t ntiles = num_pin_tiles(p);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    PinTileView v = stage_pin_tile(eoff, tile_net, m, p, t, s_off);
    for (int64_t q = v.q0 + threadIdx.x; q < v.q1; q += blockDim.x) {
      const int32_t i = net_in_tile(s_off, v.count, q);
      const int32_t sz = s_off[i + 1] - s_off[i];
      if (sz < 2 || sz > T) continue;
      const int64_t sl = posmap_slot(M, v.e_lo + i, pins[q]);
      if (sl < 0) dev_fail(status, DEV_HASH_FULL);
      else M.pos[sl] = (int32_t)q;
    }
    __syncthreads();
  }
}

// The incidences of the listed nodes of one sub-round, one thread each: the
// nodes of sub-round s sit in one range of the class-ordered node list per
// class, and lpre is the exclusive prefix sum of the degrees along that list,
// so the incidence ranks of each range are contiguous.  The ranks are cut
// into tiles of POS_TILE; tile_node[T] is the listed node holding rank
// T * POS_TILE, and since every listed node has an incident net, the tile's
// ranks belong to that node and the POS_TILE after it at most: a block stages
// their prefix sums in shared memory and each thread finds its node there.
// Nodes that did not join a cluster in the sub-round (rep[u] == u) are
// skipped.
constexpr int POS_TILE = 256;

struct SubRanges {
  int32_t lo[NCLASS], hi[NCLASS];
};

// tile_node[T] for every tile T of the ranks of the whole list.
__global__ void k_tile_node(const int32_t* __restrict__ lpre, int32_t nlisted,
                            int32_t* __restrict__ tile_node) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nlisted;
       i += gridDim.x * blockDim.x) {
    const int32_t t0 = (lpre[i] + POS_TILE - 1) / POS_TILE;
    const int32_t t1 = (lpre[i + 1] + POS_TILE - 1) / POS_TILE;
    for (int32_t t = t0; t < t1; ++t) tile_node[t] = i;
  }
}

// Pass 1 (JOIN): for a rated incidence (u, e) of a node that joined C, insert
// (e, C), lower its first position to q and clear the position it displaced;
// the map slot is kept for pass 2 (all ones for an unrated net).
// Pass 2: cluster word of q = C where q is now C's first position in the
// net, else -1.  `rx` is the cluster word of the rinfo records (stride 2).
template <bool JOIN>
__global__ void __launch_bounds__(POS_TILE)
k_posmap_pass(const int4* __restrict__ lnode, const int32_t* __restrict__ lpre,
              const int32_t* __restrict__ tile_node, int32_t nlisted, SubRanges R,
              const int32_t* __restrict__ rep, const int32_t* __restrict__ inets,
              const int32_t* __restrict__ ipin, const int32_t* __restrict__ eoff, int T, PosMap M,
              uint32_t* __restrict__ jslot, int32_t* __restrict__ rx, int32_t* status) {
  __shared__ int32_t s_pre[POS_TILE + 1];
#pragma unroll 1
  for (int c = 0; c < NCLASS; ++c) {
    const int32_t lo = R.lo[c], hi = R.hi[c];
    if (lo >= hi) continue;
    const int32_t r0 = lpre[lo], r1 = lpre[hi];
    const int32_t t_end = (r1 + POS_TILE - 1) / POS_TILE;
    for (int32_t tile = r0 / POS_TILE + blockIdx.x; tile < t_end; tile += gridDim.x) {
      const int32_t a0 = tile_node[tile];
      const int32_t nn = min(POS_TILE + 1, nlisted - a0 + 1);
      for (int i = threadIdx.x; i < nn; i += blockDim.x) s_pre[i] = lpre[a0 + i];
      __syncthreads();
      const int32_t x = tile * POS_TILE + (int32_t)threadIdx.x;
      if (x >= r0 && x < r1) {
        int32_t a = 0, b = nn - 2;  // largest i with s_pre[i] <= x
        while (a < b) {
          const int32_t mid = (a + b + 1) >> 1;
          if (s_pre[mid] <= x) a = mid;
          else b = mid - 1;
        }
        const int4 nd = lnode[a0 + a];
        const int32_t u = nd.x;
        const int32_t C = rep[u];
        const int32_t j = nd.y + (x - s_pre[a]);
        if (j >= nd.z) {
          dev_fail(status, DEV_CAPACITY);  // the tile outran its staged nodes
        } else if (C == u) {
          // not joined
        } else if (JOIN) {
          const int32_t e = inets[j];
          const int32_t sz = eoff[e + 1] - eoff[e];
          uint32_t slot = ~0u;
          if (sz >= 2 && sz <= T) {
            const int32_t q = ipin[j];
            const int64_t sl = posmap_slot(M, e, C);
            if (sl < 0) {
              dev_fail(status, DEV_HASH_FULL);
            } else {
              slot = (uint32_t)sl;
              const int32_t old = atomicMin(&M.pos[sl], q);
              if (old != 0x7fffffff && q < old) rx[2 * (int64_t)old] = -1;  // the displaced first position
            }
          }
          jslot[j] = slot;
        } else {
          const uint32_t sl = jslot[j];
          if (sl != ~0u) {
            const int32_t q = ipin[j];
            rx[2 * (int64_t)q] = M.pos[sl] == q ? C : -1;
          }
        }
      }
      __syncthreads();
    }
  }
}

// rinfo at the start of a level: cluster word = the pin for the pins of
// rated nets, -1 for the others (pin tiles).
__global__ void __launch_bounds__(PIN_TILE_THREADS)
k_rinfo_init(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
             const int32_t* __restrict__ tile_net, int32_t m, int64_t p, int T,
             int2* __restrict__ rinfo) {
  __shared__ int32_t s_off[PIN_TILE + 3];
  const int64_t ntiles = num_pin_tiles(p);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    PinTileView v = stage_pin_tile(eoff, tile_net, m, p, t, s_off);
    for (int64_t q = v.q0 + threadIdx.x; q < v.q1; q += blockDim.x) {
      const int32_t i = net_in_tile(s_off, v.count, q);
      const int32_t sz = s_off[i + 1] - s_off[i];
      rinfo[q] = make_int2(sz >= 2 && sz <= T ? pins[q] : -1, 0);
    }
    __syncthreads();
  }
}

// pcomm[q] = comm[pins[q]] for every pin position.
__global__ void k_pin_comm(const int32_t* __restrict__ pins, int64_t p,
                           const int32_t* __restrict__ comm, int32_t* __restrict__ pcomm) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p;
       q += (int64_t)gridDim.x * blockDim.x)
    pcomm[q] = comm[pins[q]];
}

// Weight words of every record before sub-round s: the cluster's weight, or
// INT32_MAX for an unclustered node of sub-round s.  A thread takes
// REFRESH_ILP pairs of records per iteration (16-byte loads, all issued before
// the cluster gathers) and stores only the weight words that change.
constexpr int REFRESH_ILP = 4;

__device__ __forceinline__ int32_t refresh_word(const int2* __restrict__ cst, int32_t C, int s,
                                                int32_t old) {
  if (C < 0) return old;
  const int2 cs = cst[C];
  return cs.y == s ? 0x7fffffff : cs.x;
}

__global__ void k_rinfo_refresh(int2* __restrict__ rinfo, int64_t p, const int2* __restrict__ cst,
                                int s) {
  const int64_t pairs = p >> 1;
  const int4* r4 = reinterpret_cast<const int4*>(rinfo);
  int32_t* words = reinterpret_cast<int32_t*>(rinfo);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < pairs;
       i0 += REFRESH_ILP * stride) {
    int4 r[REFRESH_ILP];
#pragma unroll
    for (int k = 0; k < REFRESH_ILP; ++k) {
      const int64_t i = i0 + k * stride;
      r[k] = i < pairs ? r4[i] : make_int4(-1, 0, -1, 0);
    }
    int32_t y[REFRESH_ILP], w[REFRESH_ILP];
#pragma unroll
    for (int k = 0; k < REFRESH_ILP; ++k) {
      y[k] = refresh_word(cst, r[k].x, s, r[k].y);
      w[k] = refresh_word(cst, r[k].z, s, r[k].w);
    }
#pragma unroll
    for (int k = 0; k < REFRESH_ILP; ++k) {
      const int64_t i = i0 + k * stride;
      if (y[k] != r[k].y) words[4 * i + 1] = y[k];
      if (w[k] != r[k].w) words[4 * i + 3] = w[k];
    }
  }
  if ((p & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int2 r = rinfo[p - 1];
    const int32_t y = refresh_word(cst, r.x, s, r.y);
    if (y != r.y) rinfo[p - 1].y = y;
  }
}

__global__ void k_list_degree(const int32_t* __restrict__ list, int32_t cnt,
                              const int32_t* __restrict__ ioff, int32_t* __restrict__ deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = list[i];
    deg[i] = ioff[u + 1] - ioff[u];
  }
}

__global__ void k_init_cluster(const int32_t* __restrict__ c, int32_t n, uint64_t seed, int level,
                               int S, int32_t* __restrict__ rep, int2* __restrict__ cst,
                               int32_t* __restrict__ slot_of) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    rep[u] = (int32_t)u;
    cst[u] = make_int2(c[u], subround_of_node_cluster(seed, level, (int)u, S));
    slot_of[u] = -1;
  }
}


// ---------------------------------------------------------- host side

template <typename F>
void allow_smem(F* kernel) {
  HG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BUDGET));
}

template <typename VT>
void set_rate_attrs_once() {
  allow_smem(k_rate_team<VT, 1, 8>);
  allow_smem(k_rate_team<VT, 4, 2>);
  allow_smem(k_rate_team<VT, 16, 1>);
  allow_smem(k_rate_team<VT, 8, 1>);
  allow_smem(k_rate_team<VT, 8, 2>);
  allow_smem(k_rate_team<VT, 8, 4>);
  allow_smem(k_rate_dense<VT>);
  HG_CUDA(cudaFuncSetAttribute(k_rate_part<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)part_bytes<VT>()));
}

// Attributes belong to the functions: set once per process, also when
// several handles rate concurrently from different host threads.
template <typename VT>
void set_rate_attrs() {
  static std::once_flag once;
  std::call_once(once, set_rate_attrs_once<VT>);
}

struct SplitPlan {
  std::vector<int32_t> lo, hi;          // class-3 node range of every sub-round (in split order)
  std::vector<int32_t> item_lo, item_hi;
  std::vector<int32_t> part_lo, part_hi;
  std::vector<int64_t> tab_lo;          // first table entry of every sub-round
  int64_t tab_span = 0;                 // largest table footprint of one sub-round
  const int32_t* split = nullptr;
  DBuf<int32_t> item_node, item_off, part_node, part_off, tnused, res_c;
  DBuf<int64_t> tab_off, tab_cap;
  DBuf<int8_t> tab_dense;
  DBuf<unsigned char> res_v;
  DBuf<int32_t> tkey, tused;
  DBuf<unsigned char> tval;
};

template <typename VT, int TW, int TEAMS>
void launch_team(const Ctx& cx, const RateArgs& A, uint32_t slots) {
  using H = typename HashOf<VT>::type;
  const size_t bytes = (size_t)TEAMS * team_bytes<H>(slots);
  const int per_sm = std::max<int>(1, (int)(SMEM_BUDGET / bytes));
  k_rate_team<VT, TW, TEAMS><<<grid_for(A.count, TEAMS, cx.num_sms, per_sm), TW * 32 * TEAMS,
                               bytes, cx.stream>>>(A, slots);
}

template <typename VT>
void rate_subround(const Ctx& cx, RateArgs A, const std::vector<int32_t>& hoff, const int32_t* list,
                   const int4* lnode, int S, int s, bool dense_block, SplitPlan& sp,
                   KernelTimer* timers,
                   unsigned long long* stats_base, CoarsenCounters& cc) {
  set_rate_attrs<VT>();
  for (int cls = 0; cls < SPLIT_CLASS; ++cls) {
    A.count = hoff[cls * S + s + 1] - hoff[cls * S + s];
    A.list = list + hoff[cls * S + s];
    A.lnode = lnode + hoff[cls * S + s];
    if (A.count == 0) continue;
    A.stats = stats_base + (size_t)cls * ST_WORDS;
    KernelTimer& timer = timers[cls];
    timer.begin();
    if (cls == 0) {
      launch_team<VT, 1, 8>(cx, A, 2 * D_WARP);
    } else if (cls == 1) {
      launch_team<VT, 4, 2>(cx, A, 2 * D_PAIR);
    } else if (cls == 2 && dense_block) {
      const size_t bytes = (size_t)std::max<int32_t>(A.n, 1) * (sizeof(VT) + 4);
      const int per_sm = std::max<int>(1, (int)(SMEM_BUDGET / bytes));
      k_rate_dense<VT><<<grid_for(A.count, 1, cx.num_sms, per_sm), 256, bytes, cx.stream>>>(A);
    } else if (cls == 2) {
      if (sizeof(VT) == 4) launch_team<VT, 8, 4>(cx, A, 2 * D_QUAD);
      else launch_team<VT, 8, 2>(cx, A, 2 * D_QUAD);
    } else {
      if (sizeof(VT) == 4) launch_team<VT, 16, 1>(cx, A, 2 * D_BLOCK);
      else launch_team<VT, 8, 1>(cx, A, 2 * D_BLOCK);
    }
    timer.end();
    check_launch("rate_team");
    cc.rating_launches += 1;
  }
  // class 4 (split)
  if (sp.hi[s] > sp.lo[s]) {
    const int32_t items = sp.item_hi[s] - sp.item_lo[s];
    VT* tval = reinterpret_cast<VT*>(sp.tval.p);
    A.stats = stats_base + (size_t)SPLIT_CLASS * ST_WORDS;
    KernelTimer& timer = timers[SPLIT_CLASS];
    timer.begin();
    if (items > 0) {
      const int g = grid_for(items, SPLIT_WARPS, cx.num_sms, 16);
      k_rate_split_acc<VT><<<g, SPLIT_WARPS * 32, 0, cx.stream>>>(
          A, sp.split, sp.item_node.p, sp.item_off.p, sp.tab_off.p, sp.tab_cap.p, sp.tab_dense.p,
          sp.item_lo[s], sp.item_hi[s], sp.tab_lo[s], sp.tkey.p, tval, sp.tused.p, sp.tnused.p);
      check_launch("rate_split_acc");
      cc.rating_launches += 1;
    }
    const int32_t parts = sp.part_hi[s] - sp.part_lo[s];
    if (parts > 0) {
      const size_t bytes = part_bytes<VT>();
      k_rate_part<VT><<<grid_for(parts, 1, cx.num_sms, 1), PART_THREADS, bytes, cx.stream>>>(
          A, sp.split, sp.part_node.p, sp.part_off.p, sp.part_lo[s], sp.part_hi[s],
          reinterpret_cast<VT*>(sp.res_v.p), sp.res_c.p);
      check_launch("rate_part");
      cc.rating_launches += 1;
    }
    const int g2 = grid_for(sp.hi[s] - sp.lo[s], 1, cx.num_sms, 8);
    k_rate_split_argmax<VT><<<g2, ARGMAX_THREADS, 0, cx.stream>>>(
        A, sp.split, sp.lo[s], sp.hi[s], sp.tab_off.p, sp.tab_cap.p, sp.tab_dense.p, sp.tab_lo[s],
        sp.tkey.p, tval, sp.tused.p, sp.tnused.p, sp.part_off.p,
        reinterpret_cast<const VT*>(sp.res_v.p), sp.res_c.p);
    timer.end();
    check_launch("rate_split_argmax");
    cc.rating_launches += 1;
  }
}

// A private stream of the calling host thread on its current device, for
// capturing a level's sub-round loop (the caller's stream may be the legacy
// default stream, which cannot be captured).
cudaStream_t level_capture_stream() {
  struct Cache {
    int device = -1;
    cudaStream_t s = nullptr;
    ~Cache() {
      if (s) cudaStreamDestroy(s);
    }
  };
  thread_local Cache cache;
  int dev = 0;
  HG_CUDA(cudaGetDevice(&dev));
  if (cache.device != dev) {
    if (cache.s) cudaStreamDestroy(cache.s);
    cache.s = nullptr;
    HG_CUDA(cudaStreamCreateWithFlags(&cache.s, cudaStreamNonBlocking));
    cache.device = dev;
  }
  return cache.s;
}

}  // namespace

void cluster_level(const Ctx& cx, Level& L, const CoarsenParams& P, CoarsenCounters& cc,
                   DBuf<int32_t>& cw_out) {
  const int32_t n = L.n;
  const int S = P.S;
  const int nkeys = S * NCLASS;
  L.rep.alloc(&cx.alloc, (size_t)n);
  cw_out.alloc(&cx.alloc, (size_t)n);
  DBuf<int2> cst;
  DBuf<int32_t> target, gw, gcnt, slot_of, slot_c, slot_off, slot_fill, mv, touched, glist, key_of,
      wof, kcount, kfill, list, words, clusters;
  DBuf<int2> rinfo;
  DBuf<unsigned long long> stats, max_r;
  const size_t ncap = (size_t)n + 1;
  cst.alloc(&cx.alloc, ncap);
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
  wof.alloc(&cx.alloc, ncap);
  list.alloc(&cx.alloc, ncap);
  kcount.alloc(&cx.alloc, (size_t)nkeys);
  kfill.alloc(&cx.alloc, (size_t)nkeys);
  words.alloc(&cx.alloc, (size_t)S * CW_WORDS);
  clusters.alloc(&cx.alloc, 1);
  max_r.alloc(&cx.alloc, 1);
  stats.alloc(&cx.alloc, (size_t)ST_WORDS * NCLASS);
  rinfo.alloc(&cx.alloc, L.graph ? 1 : (size_t)std::max<int64_t>(L.p, 1));
  HG_CUDA(cudaMemsetAsync(gw.p, 0, gw.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(gcnt.p, 0, gcnt.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(slot_fill.p, 0, slot_fill.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(kcount.p, 0, kcount.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(kfill.p, 0, kfill.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(words.p, 0, words.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(max_r.p, 0, max_r.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(stats.p, 0, stats.bytes(), cx.stream));
  HG_CUDA(cudaMemcpyAsync(clusters.p, &n, sizeof(int32_t), cudaMemcpyHostToDevice, cx.stream));
  // graph levels rate from the adjacency array: no pin records, no
  // (net, cluster) map
  const bool records = L.p > 0 && !L.graph;
  DBuf<int32_t> tiles;
  if (records) {
    tiles.alloc(&cx.alloc, (size_t)num_pin_tiles(L.p) + 1);
    build_tile_index(cx, L.eoff.p, L.m, L.p, tiles.p);
    k_rinfo_init<<<grid_for(num_pin_tiles(L.p), 1, cx.num_sms, 8), PIN_TILE_THREADS, 0,
                   cx.stream>>>(L.eoff.p, L.pins.p, tiles.p, L.m, L.p, P.T, rinfo.p);
    check_launch("rinfo_init");
    if (cx.launches) *cx.launches += 1;
  }

  const int g_nodes = grid_for(n, 256, cx.num_sms, 4);
  k_init_cluster<<<g_nodes, 256, 0, cx.stream>>>(L.c.p, n, P.seed, P.level, S, L.rep.p, cst.p,
                                                 slot_of.p);
  check_launch("init_cluster");
  DBuf<unsigned long long> rterm;
  rterm.alloc(&cx.alloc, (size_t)std::max<int32_t>(L.m, 1));
  if (L.m > 0) {
    k_net_terms<<<grid_for(L.m, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.eoff.p, L.w.p, L.m,
                                                                          P.T, rterm.p);
    check_launch("net_terms");
  }
  k_node_work<<<grid_for(n, 8, cx.num_sms, 16), 256, 0, cx.stream>>>(
      L.ioff.p, L.inets.p, L.eoff.p, rterm.p, n, L.graph, wof.p, max_r.p);
  check_launch("node_work");
  const unsigned long long hmax_r = (unsigned long long)read_i64(cx, (const int64_t*)max_r.p);
  // 32-bit rating words when no node's total rating can reach 2^31; block
  // tables are direct-indexed when one value and one used-list entry per
  // node of the level fit the shared-memory budget
  const bool narrow = hmax_r < (1ull << 31);
  const size_t vbytes = narrow ? 4 : 8;
  const bool dense_block = (size_t)n * (vbytes + 4) <= SMEM_BUDGET;
  k_node_classify<<<g_nodes, 256, 0, cx.stream>>>(wof.p, n, P.seed, P.level, S, dense_block,
                                                   P.cuts, key_of.p, kcount.p);
  check_launch("node_classify");
  k_node_scatter<<<g_nodes, 256, nkeys * sizeof(int32_t), cx.stream>>>(key_of.p, n, nkeys,
                                                                        kcount.p, kfill.p, list.p);
  check_launch("node_scatter");
  if (cx.launches) *cx.launches += 5;

  std::vector<int32_t> hcount(nkeys);
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(hcount.data(), kcount.p, sizeof(int32_t) * nkeys, cudaMemcpyDeviceToHost,
                          cx.stream));
  check_status(cx);
  std::vector<int32_t> hoff(nkeys + 1, 0);
  for (int i = 0; i < nkeys; ++i) hoff[i + 1] = hoff[i] + hcount[i];
  // per listed node {u, ioff[u], ioff[u + 1], c(u)}, and on hypergraph
  // levels the net metadata of every incidence, for the rating walks
  DBuf<int4> lnode;
  lnode.alloc(&cx.alloc, (size_t)std::max<int32_t>(hoff[nkeys], 1));
  if (hoff[nkeys] > 0) {
    k_list_nodes<<<grid_for(hoff[nkeys], 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
        list.p, hoff[nkeys], L.ioff.p, L.c.p, lnode.p);
    check_launch("list_nodes");
    if (cx.launches) *cx.launches += 1;
  }
  DBuf<IncMeta> imeta;
  if (!L.graph && L.p > 0) {
    imeta.alloc(&cx.alloc, (size_t)L.p);
    k_inc_meta<<<grid_for(L.p, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.inets.p, L.eoff.p,
                                                                         rterm.p, L.p, imeta.p);
    check_launch("inc_meta");
    if (cx.launches) *cx.launches += 1;
  }

  // ---- split plan: items, table offsets and footprint per sub-round
  SplitPlan sp;
  sp.lo.resize(S);
  sp.hi.resize(S);
  sp.item_lo.assign(S, 0);
  sp.item_hi.assign(S, 0);
  sp.part_lo.assign(S, 0);
  sp.part_hi.assign(S, 0);
  sp.tab_lo.assign(S, 0);
  const int32_t split_base = hoff[SPLIT_CLASS * S];
  const int32_t nsplit = hoff[NCLASS * S] - split_base;
  for (int s = 0; s < S; ++s) {
    sp.lo[s] = hoff[SPLIT_CLASS * S + s] - split_base;
    sp.hi[s] = hoff[SPLIT_CLASS * S + s + 1] - split_base;
  }
  sp.split = list.p + split_base;
  if (nsplit > 0) {
    DBuf<int32_t> items, parts, cap32;
    items.alloc(&cx.alloc, (size_t)nsplit + 1);
    parts.alloc(&cx.alloc, (size_t)nsplit + 1);
    cap32.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.item_off.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.part_off.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.tab_off.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.tab_cap.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.tab_dense.alloc(&cx.alloc, (size_t)nsplit + 1);
    sp.tnused.alloc(&cx.alloc, (size_t)nsplit + 1);
    HG_CUDA(cudaMemsetAsync(sp.tnused.p, 0, sp.tnused.bytes(), cx.stream));
    const int gs = grid_for(nsplit, 256, cx.num_sms, 4);
    k_split_sizes<<<gs, 256, 0, cx.stream>>>(
        sp.split, nsplit, L.ioff.p, wof.p, n, narrow ? PartCfg<uint32_t>::D : PartCfg<unsigned long long>::D,
        items.p, parts.p, cap32.p, sp.tab_dense.p);
    check_launch("split_sizes");
    scan_exclusive_i32(cx, items.p, sp.item_off.p, nsplit, sp.item_off.p + nsplit);
    scan_exclusive_i32(cx, parts.p, sp.part_off.p, nsplit, sp.part_off.p + nsplit);
    scan_exclusive_i32_to_i64(cx, cap32.p, sp.tab_off.p, nsplit, sp.tab_off.p + nsplit);
    k_widen<<<gs, 256, 0, cx.stream>>>(cap32.p, sp.tab_cap.p, nsplit);
    check_launch("widen");
    std::vector<int32_t> hio((size_t)nsplit + 1), hso((size_t)nsplit + 1);
    std::vector<int64_t> hto((size_t)nsplit + 1);
    wait_stream(cx);
    HG_CUDA(cudaMemcpyAsync(hio.data(), sp.item_off.p, sizeof(int32_t) * hio.size(),
                            cudaMemcpyDeviceToHost, cx.stream));
    HG_CUDA(cudaMemcpyAsync(hso.data(), sp.part_off.p, sizeof(int32_t) * hso.size(),
                            cudaMemcpyDeviceToHost, cx.stream));
    HG_CUDA(cudaMemcpyAsync(hto.data(), sp.tab_off.p, sizeof(int64_t) * hto.size(),
                            cudaMemcpyDeviceToHost, cx.stream));
    check_status(cx);
    for (int s = 0; s < S; ++s) {
      sp.item_lo[s] = hio[sp.lo[s]];
      sp.item_hi[s] = hio[sp.hi[s]];
      sp.part_lo[s] = hso[sp.lo[s]];
      sp.part_hi[s] = hso[sp.hi[s]];
      sp.tab_lo[s] = hto[sp.lo[s]];
      sp.tab_span = std::max<int64_t>(sp.tab_span, hto[sp.hi[s]] - hto[sp.lo[s]]);
    }
    sp.item_node.alloc(&cx.alloc, (size_t)std::max<int32_t>(hio[nsplit], 1));
    k_split_items<<<gs, 256, 0, cx.stream>>>(sp.item_off.p, nsplit, sp.item_node.p);
    check_launch("split_items");
    const size_t nparts = (size_t)std::max<int32_t>(hso[nsplit], 1);
    sp.part_node.alloc(&cx.alloc, nparts);
    sp.res_v.alloc(&cx.alloc, nparts * vbytes);
    sp.res_c.alloc(&cx.alloc, nparts);
    k_split_items<<<gs, 256, 0, cx.stream>>>(sp.part_off.p, nsplit, sp.part_node.p);
    check_launch("split_parts");
    const size_t span = (size_t)std::max<int64_t>(sp.tab_span, 1);
    sp.tval.alloc(&cx.alloc, span * vbytes);
    sp.tkey.alloc(&cx.alloc, span);
    sp.tused.alloc(&cx.alloc, span);
    const int gi = grid_for((int64_t)span, 256, cx.num_sms, 8);
    if (narrow)
      k_init_table<uint32_t><<<gi, 256, 0, cx.stream>>>(
          sp.tkey.p, reinterpret_cast<uint32_t*>(sp.tval.p), span);
    else
      k_init_table<unsigned long long><<<gi, 256, 0, cx.stream>>>(
          sp.tkey.p, reinterpret_cast<unsigned long long*>(sp.tval.p), span);
    check_launch("init_table");
    if (cx.launches) *cx.launches += 11;
  }

  // (net, cluster) -> first position map: at most one key per rated pin at
  // the start plus one per joining incidence, so 2p keys; capacity >= 4p
  // (at most 2^32, which still exceeds 2p since p < 2^31).
  DBuf<unsigned long long> pm_key;
  DBuf<int32_t> pm_pos, lpre, tile_node;
  DBuf<uint32_t> jslot;
  PosMap pm;
  pm.key = nullptr;
  pm.pos = nullptr;
  pm.mask = 0;
  if (records && S > 1) {
    uint64_t cap = 1024;
    while (cap < 4 * (uint64_t)L.p && cap < (1ull << 32)) cap <<= 1;
    pm_key.alloc(&cx.alloc, cap);
    pm_pos.alloc(&cx.alloc, cap);
    jslot.alloc(&cx.alloc, (size_t)L.p);
    HG_CUDA(cudaMemsetAsync(pm_key.p, 0xff, pm_key.bytes(), cx.stream));
    fill_i32(cx, pm_pos.p, 0x7fffffff, (int64_t)cap);
    pm.key = pm_key.p;
    pm.pos = pm_pos.p;
    pm.mask = cap - 1;
    const int32_t nlisted = hoff[nkeys];
    lpre.alloc(&cx.alloc, (size_t)nlisted + 1);
    EventTimer tm(cx, &cc.ms_refresh);
    if (nlisted > 0) {
      k_list_degree<<<grid_for(nlisted, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(
          list.p, nlisted, L.ioff.p, lpre.p);
      check_launch("list_degree");
    }
    scan_exclusive_i32(cx, lpre.p, lpre.p, nlisted, lpre.p + nlisted);
    tile_node.alloc(&cx.alloc, (size_t)(L.p / POS_TILE + 2));
    if (nlisted > 0) {
      k_tile_node<<<grid_for(nlisted, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(lpre.p, nlisted,
                                                                               tile_node.p);
      check_launch("tile_node");
    }
    k_posmap_init<<<grid_for(num_pin_tiles(L.p), 1, cx.num_sms, 8), PIN_TILE_THREADS, 0,
                    cx.stream>>>(L.eoff.p, L.pins.p, tiles.p, L.m, L.p, P.T, pm, cx.d_status);
    check_launch("posmap_init");
    if (cx.launches) *cx.launches += 1 + 2 * (nlisted > 0);
  }

  RateArgs A;
  A.ioff = L.ioff.p;
  A.inets = L.inets.p;
  A.eoff = L.eoff.p;
  A.rinfo = rinfo.p;
  A.graph = L.graph;
  A.adj = L.adj.p;
  A.rep = L.rep.p;
  A.comm = L.comm.p;
  A.pcomm = nullptr;
  DBuf<int32_t> pcomm;
  if (L.comm.p && !L.graph && L.p > 0) {
    pcomm.alloc(&cx.alloc, (size_t)L.p);
    k_pin_comm<<<grid_for(L.p, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.pins.p, L.p, L.comm.p,
                                                                         pcomm.p);
    check_launch("pin_comm");
    if (cx.launches) *cx.launches += 1;
    A.pcomm = pcomm.p;
  }
  A.rterm = rterm.p;
  A.imeta = imeta.p;
  A.lsplit = lnode.p + split_base;
  A.c = L.c.p;
  A.cst = cst.p;
  A.T = P.T;
  A.c_max = P.c_max;
  A.n = n;
  A.clusters = clusters.p;
  A.target = target.p;
  A.gw = gw.p;
  A.gcnt = gcnt.p;
  A.mv = mv.p;
  A.touched_targets = touched.p;
  A.stats = stats.p;
  A.status_word = cx.d_status;

  std::vector<KernelTimer> rate_timers;
  for (int c = 0; c < NCLASS; ++c) rate_timers.emplace_back(cx);
  // The S sub-rounds have no host interaction after the readbacks above, so
  // without phase or kernel timing they are captured as one CUDA graph per
  // level and launched once (lx = the context whose stream the launches go
  // to; nothing is allocated inside the loop).
  auto subrounds = [&](const Ctx& lx) {
  for (int s = 0; s < S; ++s) {
    A.s = s;
    A.words = words.p + (size_t)s * CW_WORDS;
    int32_t* w_s = words.p + (size_t)s * CW_WORDS;
    if (records) {
      EventTimer tm(cx, &cc.ms_refresh);
      k_rinfo_refresh<<<grid_for(L.p / 2 + 1, 256, cx.num_sms, 8), 256, 0, lx.stream>>>(
          rinfo.p, L.p, cst.p, s);
      check_launch("rinfo_refresh");
      if (cx.launches) *cx.launches += 1;
    }
    {
      EventTimer tm(cx, &cc.ms_rating);
      const int64_t before = cc.rating_launches;
      if (narrow)
        rate_subround<uint32_t>(lx, A, hoff, list.p, lnode.p, S, s, dense_block, sp,
                                rate_timers.data(), stats.p, cc);
      else
        rate_subround<unsigned long long>(lx, A, hoff, list.p, lnode.p, S, s, dense_block, sp,
                                          rate_timers.data(), stats.p, cc);
      if (cx.launches) *cx.launches += cc.rating_launches - before;
    }
    {
      EventTimer tm(cx, &cc.ms_approve);
      const int g = grid_for((n + S - 1) / S, 256, cx.num_sms, 4);
      k_approve<<<g, 256, 0, lx.stream>>>(mv.p, w_s, target.p, cst.p, gw.p, gcnt.p, P.c_max,
                                          L.rep.p, slot_of.p, slot_c.p, slot_off.p,
                                          w_s + CW_SLOTS, w_s + CW_CURSOR);
      check_launch("approve");
      k_contest_scatter<<<g, 256, 0, lx.stream>>>(mv.p, w_s, target.p, cst.p, gw.p, P.c_max,
                                                  slot_of.p, slot_off.p, slot_fill.p, glist.p);
      check_launch("contest_scatter");
      k_contest_group<<<cx.num_sms, GROUP_THREADS, 0, lx.stream>>>(
          w_s, slot_c.p, slot_off.p, slot_fill.p, slot_of.p, glist.p, gcnt.p, L.c.p, P.c_max,
          cst.p, L.rep.p, clusters.p);
      check_launch("contest_group");
      k_finish<<<g, 256, 0, lx.stream>>>(touched.p, w_s, P.c_max, cst.p, gw.p, gcnt.p, clusters.p);
      check_launch("finish");
      if (cx.launches) *cx.launches += 4;
    }
    if (s + 1 < S && records) {
      EventTimer tm(cx, &cc.ms_refresh);
      SubRanges R;
      for (int c = 0; c < NCLASS; ++c) {
        R.lo[c] = hoff[c * S + s];
        R.hi[c] = hoff[c * S + s + 1];
      }
      const int g = cx.num_sms * 8;
      k_posmap_pass<true><<<g, POS_TILE, 0, lx.stream>>>(
          lnode.p, lpre.p, tile_node.p, hoff[nkeys], R, L.rep.p, L.inets.p, L.ipin.p, L.eoff.p,
          P.T, pm, jslot.p, reinterpret_cast<int32_t*>(rinfo.p), cx.d_status);
      check_launch("posmap_join");
      k_posmap_pass<false><<<g, POS_TILE, 0, lx.stream>>>(
          lnode.p, lpre.p, tile_node.p, hoff[nkeys], R, L.rep.p, L.inets.p, L.ipin.p, L.eoff.p,
          P.T, pm, jslot.p, reinterpret_cast<int32_t*>(rinfo.p), cx.d_status);
      check_launch("posmap_fix");
      if (cx.launches) *cx.launches += 2;
    }
  }
  };
  if (!cx.timing && !cx.kernel_timing) {
    set_rate_attrs<uint32_t>();
    set_rate_attrs<unsigned long long>();
    Ctx lx = cx;
    lx.stream = level_capture_stream();
    cudaGraph_t graph = nullptr;
    HG_CUDA(cudaStreamBeginCapture(lx.stream, cudaStreamCaptureModeThreadLocal));
    try {
      subrounds(lx);
    } catch (...) {
      cudaStreamEndCapture(lx.stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    HG_CUDA(cudaStreamEndCapture(lx.stream, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    HG_CUDA(ie);
    const cudaError_t le = cudaGraphLaunch(exec, cx.stream);
    cudaGraphExecDestroy(exec);  // freed once the launch completes
    HG_CUDA(le);
  } else {
    subrounds(cx);
  }
  for (int c = 0; c < NCLASS; ++c) {
    const double ms = rate_timers[c].flush();
    cc.ms_rating_kernels += ms;
    cc.class_ms[c] += ms;
  }
  // cluster weights for the contraction (valid at representatives)
  HG_CUDA(cudaMemcpy2DAsync(cw_out.p, sizeof(int32_t), cst.p, sizeof(int2), sizeof(int32_t),
                            (size_t)n, cudaMemcpyDeviceToDevice, cx.stream));
  unsigned long long hs[ST_WORDS * NCLASS];
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  for (int c = 0; c < NCLASS; ++c) {
    cc.rating_pin_visits += (int64_t)hs[c * ST_WORDS + ST_PINS];
    cc.rating_incidences += (int64_t)hs[c * ST_WORDS + ST_INCID];
    cc.rating_nodes += (int64_t)hs[c * ST_WORDS + ST_NODES];
    cc.class_visits[c] += (int64_t)hs[c * ST_WORDS + ST_PINS];
  }
}

}  // namespace hgk
