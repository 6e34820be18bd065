// Contraction of a clustering (Sec. 4.2 "The Contraction Algorithm"):
//   a5  representatives -> consecutive coarse ids by a prefix sum over
//       representative flags (rank of the representative's id); coarse node
//       weight = cluster weight;
//   a6  every pin replaced by its coarse node, each net's pins sorted and
//       deduplicated, single-pin nets dropped;
//   a7  identical nets found by fingerprint (a 64-bit sum of hashed pins plus
//       the size) in a hash table keyed by the fingerprint, the smallest net
//       id of each fingerprint group as candidate representative, and an
//       exact pin-by-pin comparison; nets that differ from their group's
//       candidate go through further rounds among themselves; weights of
//       identical nets are summed at the representative (smallest id);
//   a8  kept nets compacted in order of their representative's id by prefix
//       sums over a keep flag and the kept sizes, then the incidence lists.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace hgk {

namespace {

constexpr int SMALL_NET = 32;
constexpr int MID_NET = 4096;
constexpr int MID_THREADS = 256;
constexpr int BIG_THREADS = 512;
constexpr unsigned long long EMPTY_FP = ~0ull;

__global__ void k_rep_flags(const int32_t* __restrict__ rep, int32_t n, int32_t* __restrict__ flag) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    flag[u] = rep[u] == (int32_t)u ? 1 : 0;
}

__global__ void k_map(const int32_t* __restrict__ rep, const int32_t* __restrict__ cid,
                      const int32_t* __restrict__ cw, int32_t n, int32_t* __restrict__ map,
                      int32_t* __restrict__ c2) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rep[u];
    map[u] = cid[r];
    if (r == (int32_t)u) c2[cid[u]] = cw[u];
  }
}

__global__ void k_classify_nets(const int32_t* __restrict__ eoff, int32_t m,
                                int32_t* __restrict__ lists, int32_t* __restrict__ counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < m; b += stride) {
    const int64_t e = b + lane_id();
    const bool valid = e < m;
    int cls = -1;
    if (valid) {
      const int32_t sz = eoff[e + 1] - eoff[e];
      cls = sz <= SMALL_NET ? 0 : (sz <= MID_NET ? 1 : 2);
    }
    const int32_t slot = warp_claim_slot(counts, cls, __ballot_sync(FULL, valid));
    if (valid) lists[(int64_t)cls * m + slot] = (int32_t)e;
  }
}

__device__ __forceinline__ unsigned long long fingerprint_finish(unsigned long long sum, int32_t size,
                                                                 int bits) {
  unsigned long long f = sum + mix64((unsigned long long)(uint32_t)size ^ 0x5bd1e995ull);
  if (bits > 0 && bits < 64) f &= (1ull << bits) - 1;
  if (f == EMPTY_FP) f = EMPTY_FP - 1;
  return f;
}

// Nets of <= 32 pins: one thread per net, insertion sort in registers.
__global__ void k_remap_small(const int32_t* __restrict__ list, int32_t count,
                              const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                              const int32_t* __restrict__ map, int fp_bits,
                              int32_t* __restrict__ tpins, int32_t* __restrict__ tsize,
                              unsigned long long* __restrict__ fp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = list[i];
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    int32_t v[SMALL_NET];
    for (int q = 0; q < sz; ++q) {
      const int32_t x = map[pins[b + q]];
      int r = q;
      while (r > 0 && v[r - 1] > x) {
        v[r] = v[r - 1];
        --r;
      }
      v[r] = x;
    }
    int32_t out = 0;
    unsigned long long sum = 0;
    for (int q = 0; q < sz; ++q) {
      if (q == 0 || v[q] != v[q - 1]) {
        tpins[b + out] = v[q];
        sum += mix64((unsigned long long)(uint32_t)v[q]);
        ++out;
      }
    }
    tsize[e] = out;
    fp[e] = fingerprint_finish(sum, out, fp_bits);
  }
}

// Nets of 33..4096 pins: one block per net, bitonic sort with the keys in
// registers (shared memory only for the exchanges between warps).
__global__ void __launch_bounds__(MID_THREADS, 1024 / MID_THREADS)
k_remap_mid(const int32_t* __restrict__ list, int32_t count, const int32_t* __restrict__ eoff,
            const int32_t* __restrict__ pins, const int32_t* __restrict__ map, int fp_bits,
            int32_t* __restrict__ tpins, int32_t* __restrict__ tsize,
            unsigned long long* __restrict__ fp) {
  __shared__ int32_t s[MID_NET];
  __shared__ int32_t s_wsum[MID_THREADS / 32];
  __shared__ unsigned long long s_red[32];
  constexpr int PER = MID_NET / MID_THREADS;  // 16 consecutive items per thread
  for (int32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t e = list[i];
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    int P = 64;
    while (P < sz) P <<= 1;
    // bitonic sort with the keys in registers: thread t holds items
    // [t*PER, t*PER+PER); distances below PER are swaps inside a thread,
    // below 32*PER lane shuffles, the rest exchanges through s (warps that
    // hold only padding sit the network out)
    const int t = threadIdx.x;
    const bool warp_live = warp_in_block() * 32 * PER < P;
    int32_t v[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int q = t * PER + r;
      v[r] = q < sz ? map[pins[b + q]] : INT_MAX;
    }
    for (int kk = 2; kk <= P; kk <<= 1) {
      for (int j = kk >> 1; j >= PER; j >>= 1) {
        if (j >= 32 * PER) {
          __syncthreads();
#pragma unroll
          for (int r = 0; r < PER; ++r) s[t * PER + r] = v[r];
          __syncthreads();
#pragma unroll
          for (int r = 0; r < PER; ++r) {
            const int q = t * PER + r;
            if (q >= P) continue;
            const int32_t y = s[q ^ j];
            const bool up = (q & kk) == 0, lower = (q & j) == 0;
            const int32_t lo = min(v[r], y), hi = max(v[r], y);
            v[r] = lower == up ? lo : hi;
          }
        } else if (warp_live) {
          const int lj = j / PER;  // partner lane distance
#pragma unroll
          for (int r = 0; r < PER; ++r) {
            const int q = t * PER + r;
            const int32_t y = __shfl_xor_sync(FULL, v[r], lj);
            const bool up = (q & kk) == 0, lower = (q & j) == 0;
            const int32_t lo = min(v[r], y), hi = max(v[r], y);
            v[r] = lower == up ? lo : hi;
          }
        }
      }
      if (warp_live) {
#pragma unroll
        for (int jj = PER / 2; jj > 0; jj >>= 1) {
          if (jj >= kk) continue;
#pragma unroll
          for (int r = 0; r < PER; ++r) {
            const int l = r ^ jj;
            if (l > r) {
              const bool up = ((t * PER + r) & kk) == 0;
              const int32_t lo = min(v[r], v[l]), hi = max(v[r], v[l]);
              v[r] = up ? lo : hi;
              v[l] = up ? hi : lo;
            }
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) s[t * PER + r] = v[r];
    __syncthreads();
    // keep the first of every run: thread t owns items [t*PER, t*PER+PER)
    int32_t local = 0;
    bool keep[PER];
    int32_t vals[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int q = threadIdx.x * PER + r;
      vals[r] = q < P ? s[q] : INT_MAX;
      keep[r] = q < sz && (q == 0 || s[q] != s[q - 1]);
      local += keep[r];
    }
    int32_t x = warp_inclusive_scan(local);
    if (lane_id() == 31) s_wsum[warp_in_block()] = x;
    __syncthreads();
    int32_t before = 0;
    for (int wv = 0; wv < warp_in_block(); ++wv) before += s_wsum[wv];
    int32_t total = 0;
    for (int wv = 0; wv < MID_THREADS / 32; ++wv) total += s_wsum[wv];
    int32_t pos = before + x - local;
    unsigned long long sum = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r)
      if (keep[r]) {
        tpins[b + pos++] = vals[r];
        sum += mix64((unsigned long long)(uint32_t)vals[r]);
      }
    sum = block_sum(sum, s_red);
    if (threadIdx.x == 0) {
      tsize[e] = total;
      fp[e] = fingerprint_finish(sum, total, fp_bits);
    }
    __syncthreads();
  }
}

// Nets of more than 4096 pins: one block per net marks its coarse nodes in a
// bitmap (one bitmap per block, words = ceil(n2 / 32)) and writes the set
// bits in ascending order.
__global__ void __launch_bounds__(BIG_THREADS)
k_remap_big(const int32_t* __restrict__ list, int32_t count, const int32_t* __restrict__ eoff,
            const int32_t* __restrict__ pins, const int32_t* __restrict__ map, int32_t words,
            unsigned* __restrict__ bitmaps, int fp_bits, int32_t* __restrict__ tpins,
            int32_t* __restrict__ tsize, unsigned long long* __restrict__ fp) {
  __shared__ int32_t s_wsum[32];
  __shared__ unsigned long long s_red[32];
  __shared__ int32_t s_carry;
  unsigned* bm = bitmaps + (size_t)blockIdx.x * words;
  for (int32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t e = list[i];
    const int32_t b = eoff[e], sz = eoff[e + 1] - b;
    for (int32_t q = threadIdx.x; q < words; q += blockDim.x) bm[q] = 0u;
    __syncthreads();
    for (int32_t q = threadIdx.x; q < sz; q += blockDim.x) {
      const int32_t v = map[pins[b + q]];
      atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    unsigned long long sum = 0;
    for (int32_t base = 0; base < words; base += blockDim.x) {
      const int32_t q = base + threadIdx.x;
      const unsigned word = q < words ? bm[q] : 0u;
      const int32_t c = __popc(word);
      int32_t x = warp_inclusive_scan(c);
      if (lane_id() == 31) s_wsum[warp_in_block()] = x;
      __syncthreads();
      int32_t before = s_carry;
      for (int wv = 0; wv < warp_in_block(); ++wv) before += s_wsum[wv];
      int32_t pos = before + x - c;
      unsigned rest = word;
      while (rest) {
        const int bit = __ffs(rest) - 1;
        rest &= rest - 1;
        const int32_t v = (q << 5) + bit;
        tpins[b + pos++] = v;
        sum += mix64((unsigned long long)(uint32_t)v);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) t += s_wsum[wv];
        s_carry += t;
      }
      __syncthreads();
    }
    sum = block_sum(sum, s_red);
    if (threadIdx.x == 0) {
      tsize[e] = s_carry;
      fp[e] = fingerprint_finish(sum, s_carry, fp_bits);
    }
    __syncthreads();
  }
}

// --------------------------------------------------- identical nets (a7)

__global__ void k_candidates(const int32_t* __restrict__ tsize, int32_t m,
                             int32_t* __restrict__ list, int32_t* __restrict__ count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    if (tsize[e] >= 2) list[atomicAdd(count, 1)] = (int32_t)e;
}

__global__ void k_ident_insert(const int32_t* __restrict__ list, const int32_t* __restrict__ count,
                               const unsigned long long* __restrict__ fp, unsigned long long* tkey,
                               int32_t* tmin, uint64_t mask, int32_t* __restrict__ slot_of_net,
                               int32_t* status) {
  const int32_t cnt = *count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = list[i];
    const unsigned long long f = fp[e];
    uint64_t h = mix64(f) & mask;
    int32_t slot = -1;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long k = tkey[h];
      if (k == f) { slot = (int32_t)h; break; }
      if (k == EMPTY_FP) {
        const unsigned long long old = atomicCAS(&tkey[h], EMPTY_FP, f);
        if (old == EMPTY_FP || old == f) { slot = (int32_t)h; break; }
      }
      h = (h + 1) & mask;
    }
    if (slot < 0) {
      dev_fail(status, DEV_HASH_FULL);
      continue;
    }
    atomicMin(&tmin[slot], e);
    slot_of_net[e] = slot;
  }
}

// One warp per candidate net: compare with its group's smallest id.
__global__ void k_ident_compare(const int32_t* __restrict__ list, const int32_t* __restrict__ count,
                                const int32_t* __restrict__ eoff, const int32_t* __restrict__ tpins,
                                const int32_t* __restrict__ tsize,
                                const int32_t* __restrict__ slot_of_net,
                                const int32_t* __restrict__ tmin, int32_t* __restrict__ repnet,
                                int32_t* __restrict__ failed, int32_t* __restrict__ nfailed) {
  const int32_t cnt = *count;
  const int wv = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = wv; i < cnt; i += nwarps) {
    const int32_t e = list[i];
    const int32_t r = tmin[slot_of_net[e]];
    bool same = true;
    if (r != e) {
      const int32_t sz = tsize[e];
      if (tsize[r] != sz) {
        same = false;
      } else {
        const int32_t* a = tpins + eoff[e];
        const int32_t* bb = tpins + eoff[r];
        for (int32_t q = lane_id(); q < sz; q += 32)
          if (a[q] != bb[q]) same = false;
        same = __all_sync(FULL, same);
      }
    }
    if (lane_id() == 0) {
      if (same) repnet[e] = r;
      else failed[atomicAdd(nfailed, 1)] = e;
    }
  }
}

__global__ void k_net_weights(const int32_t* __restrict__ tsize, const int32_t* __restrict__ repnet,
                              const int32_t* __restrict__ w, int32_t m, int32_t* __restrict__ wsum,
                              int32_t* __restrict__ keep, int32_t* __restrict__ ksize) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool valid = tsize[e] >= 2;
    const bool k = valid && repnet[e] == (int32_t)e;
    if (valid) atomicAdd(&wsum[repnet[e]], w[e]);
    keep[e] = k ? 1 : 0;
    ksize[e] = k ? tsize[e] : 0;
  }
}

// One warp per kept net: write its coarse offset, weight and pins.
__global__ void k_compact(const int32_t* __restrict__ keep, const int32_t* __restrict__ newid,
                          const int32_t* __restrict__ poff, const int32_t* __restrict__ eoff,
                          const int32_t* __restrict__ tpins, const int32_t* __restrict__ tsize,
                          const int32_t* __restrict__ wsum, int32_t m, int32_t* __restrict__ eoff2,
                          int32_t* __restrict__ pins2, int32_t* __restrict__ w2) {
  const int wv = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t e = wv; e < m; e += nwarps) {
    if (!keep[e]) continue;
    const int32_t id = newid[e], dst = poff[e], src = eoff[e], sz = tsize[e];
    for (int32_t q = lane_id(); q < sz; q += 32) pins2[dst + q] = tpins[src + q];
    if (lane_id() == 0) {
      eoff2[id] = dst;
      w2[id] = wsum[e];
    }
  }
}

// Community of every coarse node: the community of its members (a cluster
// never spans two communities).
__global__ void k_coarse_comm(const int32_t* __restrict__ map, const int32_t* __restrict__ comm,
                              int32_t n, int32_t* __restrict__ ccomm) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    ccomm[map[u]] = comm[u];
}

void coarse_communities(const Ctx& cx, const Level& L, Level& out) {
  if (!L.comm.p) return;
  out.comm.alloc(&cx.alloc, (size_t)std::max<int32_t>(out.n, 1));
  k_coarse_comm<<<grid_for(L.n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(L.map.p, L.comm.p, L.n,
                                                                        out.comm.p);
  check_launch("coarse_comm");
  if (cx.launches) *cx.launches += 1;
}

}  // namespace

void contract_level(const Ctx& cx, Level& L, const int32_t* cw, Level& out, int fingerprint_bits,
                    ContractCounters& kc) {
  EventTimer tm(cx, &kc.ms);
  const int32_t n = L.n, m = L.m;
  const int gn = grid_for(n, 256, cx.num_sms, 4);
  // a5: coarse ids and node weights
  DBuf<int32_t> cid, d_n2;
  cid.alloc(&cx.alloc, (size_t)n + 1);
  d_n2.alloc(&cx.alloc, 1);
  k_rep_flags<<<gn, 256, 0, cx.stream>>>(L.rep.p, n, cid.p);
  check_launch("rep_flags");
  scan_exclusive_i32(cx, cid.p, cid.p, n, d_n2.p);
  const int32_t n2 = read_i32(cx, d_n2.p);
  out.n = n2;
  out.c.alloc(&cx.alloc, (size_t)n2);
  L.map.alloc(&cx.alloc, (size_t)n);
  k_map<<<gn, 256, 0, cx.stream>>>(L.rep.p, cid.p, cw, n, L.map.p, out.c.p);
  check_launch("map");
  if (cx.launches) *cx.launches += 2;
  cid.release();

  if (m == 0) {
    out.m = 0;
    out.p = 0;
    out.eoff.alloc(&cx.alloc, 1);
    HG_CUDA(cudaMemsetAsync(out.eoff.p, 0, sizeof(int32_t), cx.stream));
    build_incidence(cx, out);
    coarse_communities(cx, L, out);
    L.coarsened = true;
    return;
  }

  // a6: remap, sort, deduplicate
  const int gm = grid_for(m, 256, cx.num_sms, 4);
  DBuf<int32_t> lists, counts, tpins, tsize;
  DBuf<unsigned long long> fp;
  lists.alloc(&cx.alloc, (size_t)m * 3);
  counts.alloc(&cx.alloc, 4);
  tpins.alloc(&cx.alloc, (size_t)std::max<int64_t>(L.p, 1));
  tsize.alloc(&cx.alloc, (size_t)m);
  fp.alloc(&cx.alloc, (size_t)m);
  HG_CUDA(cudaMemsetAsync(counts.p, 0, counts.bytes(), cx.stream));
  k_classify_nets<<<gm, 256, 0, cx.stream>>>(L.eoff.p, m, lists.p, counts.p);
  check_launch("classify_nets");
  int32_t hc[4];
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(hc, counts.p, sizeof(hc), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  if (hc[0])
    k_remap_small<<<grid_for(hc[0], 128, cx.num_sms, 16), 128, 0, cx.stream>>>(
        lists.p, hc[0], L.eoff.p, L.pins.p, L.map.p, fingerprint_bits, tpins.p, tsize.p, fp.p);
  if (hc[1])
    k_remap_mid<<<grid_for(hc[1], 1, cx.num_sms, 8), MID_THREADS, 0, cx.stream>>>(
        lists.p + m, hc[1], L.eoff.p, L.pins.p, L.map.p, fingerprint_bits, tpins.p, tsize.p, fp.p);
  DBuf<unsigned> bitmaps;
  if (hc[2]) {
    const int32_t words = (n2 + 31) / 32;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)hc[2], (int64_t)cx.num_sms * 2,
                              (int64_t)((256ll << 20) / ((int64_t)words * 4 + 1))}));
    bitmaps.alloc(&cx.alloc, (size_t)blocks * words);
    k_remap_big<<<blocks, BIG_THREADS, 0, cx.stream>>>(lists.p + 2 * (size_t)m, hc[2], L.eoff.p,
                                                       L.pins.p, L.map.p, words, bitmaps.p,
                                                       fingerprint_bits, tpins.p, tsize.p, fp.p);
  }
  check_launch("remap");
  if (cx.launches) *cx.launches += 1 + (hc[0] > 0) + (hc[1] > 0) + (hc[2] > 0);
  bitmaps.release();

  // a7: identical nets
  uint64_t cap = 2;
  while (cap < 2 * (uint64_t)m) cap <<= 1;
  DBuf<unsigned long long> tkey;
  DBuf<int32_t> tmin, slot_of_net, repnet, cand, ncand, failed, nfailed;
  tkey.alloc(&cx.alloc, (size_t)cap);
  tmin.alloc(&cx.alloc, (size_t)cap);
  slot_of_net.alloc(&cx.alloc, (size_t)m);
  repnet.alloc(&cx.alloc, (size_t)m);
  cand.alloc(&cx.alloc, (size_t)m);
  failed.alloc(&cx.alloc, (size_t)m);
  ncand.alloc(&cx.alloc, 1);
  nfailed.alloc(&cx.alloc, 1);
  HG_CUDA(cudaMemsetAsync(ncand.p, 0, sizeof(int32_t), cx.stream));
  k_candidates<<<gm, 256, 0, cx.stream>>>(tsize.p, m, cand.p, ncand.p);
  check_launch("candidates");
  const int g_ins = grid_for(m, 256, cx.num_sms, 8);
  const int g_cmp = grid_for(m, 8, cx.num_sms, 16);
  for (int round = 0;; ++round) {
    HG_CUDA(cudaMemsetAsync(tkey.p, 0xff, tkey.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(tmin.p, 0x7f, tmin.bytes(), cx.stream));
    HG_CUDA(cudaMemsetAsync(nfailed.p, 0, sizeof(int32_t), cx.stream));
    k_ident_insert<<<g_ins, 256, 0, cx.stream>>>(cand.p, ncand.p, fp.p, tkey.p, tmin.p, cap - 1,
                                                 slot_of_net.p, cx.d_status);
    check_launch("ident_insert");
    k_ident_compare<<<g_cmp, 256, 0, cx.stream>>>(cand.p, ncand.p, L.eoff.p, tpins.p, tsize.p,
                                                  slot_of_net.p, tmin.p, repnet.p, failed.p,
                                                  nfailed.p);
    check_launch("ident_compare");
    if (cx.launches) *cx.launches += 2;
    kc.ident_rounds = round + 1;
    const int32_t nf = read_i32(cx, nfailed.p);
    if (nf == 0) break;
    // the failed nets become the candidates of the next round
    std::swap(cand, failed);
    HG_CUDA(cudaMemcpyAsync(ncand.p, nfailed.p, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            cx.stream));
  }
  tkey.release();
  tmin.release();
  slot_of_net.release();

  // a8: weights, compaction
  DBuf<int32_t> wsum, kflag, newid, ksize, d_tot;
  wsum.alloc(&cx.alloc, (size_t)m);
  kflag.alloc(&cx.alloc, (size_t)m);
  newid.alloc(&cx.alloc, (size_t)m);
  ksize.alloc(&cx.alloc, (size_t)m);
  d_tot.alloc(&cx.alloc, 2);
  HG_CUDA(cudaMemsetAsync(wsum.p, 0, wsum.bytes(), cx.stream));
  k_net_weights<<<gm, 256, 0, cx.stream>>>(tsize.p, repnet.p, L.w.p, m, wsum.p, kflag.p, ksize.p);
  check_launch("net_weights");
  scan_exclusive_i32(cx, kflag.p, newid.p, m, d_tot.p);      // keep flag -> new id
  scan_exclusive_i32(cx, ksize.p, ksize.p, m, d_tot.p + 1);  // kept size -> coarse offset
  int32_t tot[2];
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(tot, d_tot.p, sizeof(tot), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  out.m = tot[0];
  out.p = tot[1];
  out.eoff.alloc(&cx.alloc, (size_t)out.m + 1);
  out.pins.alloc(&cx.alloc, (size_t)std::max<int64_t>(out.p, 1));
  out.w.alloc(&cx.alloc, (size_t)std::max<int32_t>(out.m, 1));
  k_compact<<<grid_for(m, 8, cx.num_sms, 16), 256, 0, cx.stream>>>(
      kflag.p, newid.p, ksize.p, L.eoff.p, tpins.p, tsize.p, wsum.p, m, out.eoff.p, out.pins.p,
      out.w.p);
  check_launch("compact");
  HG_CUDA(cudaMemcpyAsync(out.eoff.p + out.m, d_tot.p + 1, sizeof(int32_t),
                          cudaMemcpyDeviceToDevice, cx.stream));
  if (cx.launches) *cx.launches += 2;
  build_incidence(cx, out);
  // a graph's coarse nets have two pins again (one-pin nets are dropped)
  if (L.graph && out.m > 0) build_graph_adjacency(cx, out);
  coarse_communities(cx, L, out);
  L.coarsened = true;
}

}  // namespace hgk
