// Gain table of Sec. 6.2: benefit b(u) = w({e in I(u) : Phi(e, Pi[u]) = 1})
// and penalty p(u, V_i) = w({e in I(u) : Phi(e, V_i) = 0}), so that the gain
// of Sec. 6 is g_u(V_t) = b(u) - p(u, V_t).
//
// Build: one warp per node over its incident nets; every lane adds w(e) to
// the warp's shared counter of each block of Lambda(e), and
// p(u, V_i) = w(I(u)) - counter[i].
// Moves (the update rules of Sec. 6.2, applied to a set of moves at once):
// one warp per move walks the nets of the moved node; one lane applies
// Phi(e, V_s) -= 1 and Phi(e, V_t) += 1 atomically, and the warp applies,
// with the counts after its own updates,
//   (1) Phi(e, V_s) = 0: p(v, V_s) += w(e) for every pin v of e,
//   (2) Phi(e, V_s) = 1: b(v) += w(e) for the pins v of e in V_s,
//   (3) Phi(e, V_t) = 1: p(v, V_t) -= w(e) for every pin v of e,
//   (4) Phi(e, V_t) = 2: b(v) -= w(e) for the pins v of e in V_t.
// The atomics give some sequential order of the pin-count updates, and by the
// lemma of Sec. 6.2 the final penalties of all nodes and the final benefits
// of the unmoved nodes do not depend on it; the benefits of the moved nodes
// are recomputed from the final pin counts afterwards.
//
// Graph levels (Sec. 10, "The Gain Table"): the table of a graph is
// w(u, V_i), the weight of u's edges into V_i, one warp per node over its
// adjacency list; the benefit and penalties follow from it:
//   b(u) = w(I(u)) - w(u, V_Pi(u)),  p(u, V_Pi(u)) = 0,
//   p(u, V_i) = w(I(u)) - w(u, V_i) for i != Pi(u)
// (an edge has no pin in V_i exactly when neither endpoint is in V_i).
#include "common.cuh"

namespace hgk {

namespace {

constexpr int GT_WARPS = 8;

__global__ void __launch_bounds__(GT_WARPS * 32)
k_gt_build(const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets,
           const int32_t* __restrict__ w, const int32_t* __restrict__ phi,
           const unsigned long long* __restrict__ lam, const int32_t* __restrict__ part, int32_t n,
           int k, long long* __restrict__ b, long long* __restrict__ p, int32_t* status) {
  __shared__ long long s_cnt[GT_WARPS][HG_MAX_K];
  const int wv = warp_in_block(), lane = lane_id();
  long long* cnt = s_cnt[wv];
  const unsigned long long kmask = k == 64 ? ~0ull : ((1ull << k) - 1ull);
  for (int i = lane; i < HG_MAX_K; i += 32) cnt[i] = 0;
  __syncwarp();
  for (int64_t u = (int64_t)blockIdx.x * GT_WARPS + wv; u < n; u += (int64_t)gridDim.x * GT_WARPS) {
    const int32_t pu = part[u];
    if (pu < 0 || pu >= k) {  // bad input: reported, never indexed
      if (lane == 0) dev_fail(status, DEV_BAD_INPUT);
      continue;
    }
    // a net in more than k/2 blocks adds w(e) to `full` (every block) and
    // takes it back from the blocks outside Lambda(e): at most k/2 atomics
    long long bu = 0, wsum = 0, full = 0;
    for (int32_t j = ioff[u] + lane; j < ioff[u + 1]; j += 32) {
      const int32_t e = inets[j];
      const long long we = w[e];
      wsum += we;
      if (phi[(int64_t)e * k + pu] == 1) bu += we;
      unsigned long long le = lam[e];
      unsigned long long delta = (unsigned long long)we;
      if (2 * __popcll(le) > k) {
        full += we;
        le = ~le & kmask;
        delta = (unsigned long long)(-we);
      }
      while (le) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[__ffsll((long long)le) - 1]), delta);
        le &= le - 1;
      }
    }
    bu = warp_sum(bu);
    wsum = warp_sum(wsum);
    full = warp_sum(full);
    __syncwarp();
    if (lane == 0) b[u] = bu;
    for (int i = lane; i < k; i += 32) {
      p[u * k + i] = wsum - (cnt[i] + full);
      cnt[i] = 0;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(GT_WARPS * 32)
k_gt_build_graph(const int32_t* __restrict__ ioff, const int2* __restrict__ adj,
                 const int32_t* __restrict__ part, int32_t n, int k, long long* __restrict__ b,
                 long long* __restrict__ p, int32_t* status) {
  __shared__ long long s_cnt[GT_WARPS][HG_MAX_K];
  const int wv = warp_in_block(), lane = lane_id();
  long long* cnt = s_cnt[wv];
  for (int i = lane; i < HG_MAX_K; i += 32) cnt[i] = 0;
  __syncwarp();
  for (int64_t u = (int64_t)blockIdx.x * GT_WARPS + wv; u < n; u += (int64_t)gridDim.x * GT_WARPS) {
    const int32_t pu = part[u];
    if (pu < 0 || pu >= k) {  // bad input: reported, never indexed
      if (lane == 0) dev_fail(status, DEV_BAD_INPUT);
      continue;
    }
    long long wsum = 0;
    for (int32_t j = ioff[u] + lane; j < ioff[u + 1]; j += 32) {
      const int2 a = adj[j];
      const int32_t pv = part[a.x];
      wsum += a.y;
      if (pv >= 0 && pv < k)
        atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[pv]), (unsigned long long)a.y);
      else
        dev_fail(status, DEV_BAD_INPUT);
    }
    wsum = warp_sum(wsum);
    __syncwarp();
    if (lane == 0) b[u] = wsum - cnt[pu];
    for (int i = lane; i < k; i += 32) {
      p[u * k + i] = i == pu ? 0 : wsum - cnt[i];
      cnt[i] = 0;
    }
    __syncwarp();
  }
}

__global__ void k_gt_check(const int32_t* __restrict__ nodes, const int32_t* __restrict__ targets,
                           int32_t l, int32_t n, int k, const int32_t* __restrict__ part,
                           int32_t* __restrict__ seen, int32_t* status) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < l; i += gridDim.x * blockDim.x) {
    const int32_t u = nodes[i], t = targets[i];
    if (u < 0 || u >= n || t < 0 || t >= k || part[u] < 0 || part[u] >= k || t == part[u] ||
        atomicExch(&seen[u], 1) != 0)
      dev_fail(status, DEV_BAD_INPUT);
  }
}

// One warp per move; the moved node's nets one after another, lanes over the
// net's pins.  Runs only after k_gt_check found the moves valid.
__global__ void k_gt_move(const int32_t* __restrict__ nodes, const int32_t* __restrict__ targets,
                          int32_t l, const int32_t* __restrict__ ioff,
                          const int32_t* __restrict__ inets, const int32_t* __restrict__ eoff,
                          const int32_t* __restrict__ pins, const int32_t* __restrict__ w,
                          const int32_t* __restrict__ part, int k, int32_t* __restrict__ phi,
                          unsigned long long* __restrict__ b, unsigned long long* __restrict__ p) {
  const int wv = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int lane = lane_id();
  for (int32_t i = wv; i < l; i += nw) {
    const int32_t u = nodes[i], t = targets[i];
    const int s = part[u];
    for (int32_t j = ioff[u]; j < ioff[u + 1]; ++j) {
      const int32_t e = inets[j];
      int32_t ns = 0, nt = 0;
      if (lane == 0) {
        ns = atomicSub(&phi[(int64_t)e * k + s], 1) - 1;
        nt = atomicAdd(&phi[(int64_t)e * k + t], 1) + 1;
      }
      ns = __shfl_sync(FULL, ns, 0);
      nt = __shfl_sync(FULL, nt, 0);
      if (ns > 1 && nt > 2) continue;  // no rule applies
      const unsigned long long we = (unsigned long long)(long long)w[e];
      const unsigned long long neg = (unsigned long long)(-(long long)w[e]);
      for (int32_t q = eoff[e] + lane; q < eoff[e + 1]; q += 32) {
        const int32_t v = pins[q];
        if (ns == 0) atomicAdd(&p[(int64_t)v * k + s], we);
        if (ns == 1 && part[v] == s) atomicAdd(&b[v], we);
        if (nt == 1) atomicAdd(&p[(int64_t)v * k + t], neg);
        if (nt == 2 && part[v] == t) atomicAdd(&b[v], neg);
      }
    }
  }
}

__global__ void k_gt_set_part(const int32_t* __restrict__ nodes,
                              const int32_t* __restrict__ targets, int32_t l,
                              int32_t* __restrict__ part) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < l; i += gridDim.x * blockDim.x)
    part[nodes[i]] = targets[i];
}

// b(u) of the moved nodes from the final pin counts.
__global__ void k_gt_moved_benefit(const int32_t* __restrict__ nodes, int32_t l,
                                   const int32_t* __restrict__ ioff,
                                   const int32_t* __restrict__ inets,
                                   const int32_t* __restrict__ w, const int32_t* __restrict__ phi,
                                   const int32_t* __restrict__ part, int k,
                                   long long* __restrict__ b) {
  const int wv = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = wv; i < l; i += nw) {
    const int32_t u = nodes[i];
    const int pu = part[u];
    long long bu = 0;
    for (int32_t j = ioff[u] + lane_id(); j < ioff[u + 1]; j += 32) {
      const int32_t e = inets[j];
      if (phi[(int64_t)e * k + pu] == 1) bu += w[e];
    }
    bu = warp_sum(bu);
    if (lane_id() == 0) b[u] = bu;
  }
}

}  // namespace

void gain_table_build(const Ctx& cx, const Level& L, int k, const int32_t* part, int64_t* b,
                      int64_t* p) {
  validate_partition(cx, part, L.n, k);
  if (L.graph) {
    k_gt_build_graph<<<grid_for(L.n, GT_WARPS, cx.num_sms, 16), GT_WARPS * 32, 0, cx.stream>>>(
        L.ioff.p, L.adj.p, part, L.n, k, reinterpret_cast<long long*>(b),
        reinterpret_cast<long long*>(p), cx.d_status);
    check_launch("gt_build_graph");
    if (cx.launches) *cx.launches += 1;
    check_status(cx);
    return;
  }
  DBuf<int32_t> phi;
  DBuf<unsigned long long> lam;
  device_pin_counts(cx, L, k, part, phi, lam);
  k_gt_build<<<grid_for(L.n, GT_WARPS, cx.num_sms, 16), GT_WARPS * 32, 0, cx.stream>>>(
      L.ioff.p, L.inets.p, L.w.p, phi.p, lam.p, part, L.n, k, reinterpret_cast<long long*>(b),
      reinterpret_cast<long long*>(p), cx.d_status);
  check_launch("gt_build");
  if (cx.launches) *cx.launches += 1;
  check_status(cx);
}

void gain_table_move(const Ctx& cx, const Level& L, int k, int32_t* part, int32_t l,
                     const int32_t* nodes, const int32_t* targets, int64_t* b, int64_t* p) {
  validate_partition(cx, part, L.n, k);
  if (l == 0) return;
  DBuf<int32_t> seen;
  seen.alloc(&cx.alloc, (size_t)L.n);
  HG_CUDA(cudaMemsetAsync(seen.p, 0, seen.bytes(), cx.stream));
  k_gt_check<<<grid_for(l, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(nodes, targets, l, L.n, k,
                                                                     part, seen.p, cx.d_status);
  check_launch("gt_check");
  check_status(cx);  // nothing below runs on bad moves
  DBuf<int32_t> phi;
  DBuf<unsigned long long> lam;
  device_pin_counts(cx, L, k, part, phi, lam);
  const int g = grid_for(l, 8, cx.num_sms, 16);
  k_gt_move<<<g, 256, 0, cx.stream>>>(nodes, targets, l, L.ioff.p, L.inets.p, L.eoff.p, L.pins.p,
                                      L.w.p, part, k, phi.p,
                                      reinterpret_cast<unsigned long long*>(b),
                                      reinterpret_cast<unsigned long long*>(p));
  check_launch("gt_move");
  k_gt_set_part<<<grid_for(l, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(nodes, targets, l, part);
  check_launch("gt_set_part");
  k_gt_moved_benefit<<<g, 256, 0, cx.stream>>>(nodes, l, L.ioff.p, L.inets.p, L.w.p, phi.p, part,
                                               k, reinterpret_cast<long long*>(b));
  check_launch("gt_moved_benefit");
  if (cx.launches) *cx.launches += 4;
  check_status(cx);
}

}  // namespace hgk
