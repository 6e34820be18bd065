// Exact gains of a move sequence M = <m_1, ..., m_l>, m_i = (u_i, Pi[u_i], t_i)
// with every node moved at most once (Sec. 6.3, "The Parallel Gain
// Recalculation Algorithm", Algorithm 4): g_i is the objective decrease that
// m_i causes when the moves are performed in sequence order.  Per net e that
// contains a moved pin, with first_in[b] = smallest index of a move into
// block b among the pins of e, last_out[b] = largest index of a move out of
// b, and non_moved[b] = pins of e in b that do not move:
//   m_i = (u, s, t) gains w(e) when last_out[s] = i, i < first_in[s] and
//   non_moved[s] = 0 (u is the last pin to leave s and nothing entered s
//   before), and loses w(e) when first_in[t] = i, i > last_out[t] and
//   non_moved[t] = 0 (u is the first pin to enter t after t was emptied).
// Only the nets of moved nodes are visited, each once.
#include "common.cuh"

namespace hgk {

namespace {

constexpr int GR_WARPS = 8;

// idx[u] = i for the move of u; a node moved twice, a node out of range, or
// a target outside [0, k) or equal to the node's block is bad input.
__global__ void k_gr_index(const int32_t* __restrict__ nodes, const int32_t* __restrict__ targets,
                           int32_t l, int32_t n, int k, const int32_t* __restrict__ part,
                           int32_t* __restrict__ idx, int32_t* status) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < l; i += gridDim.x * blockDim.x) {
    const int32_t u = nodes[i], t = targets[i];
    if (u < 0 || u >= n || t < 0 || t >= k || part[u] < 0 || part[u] >= k || t == part[u]) {
      dev_fail(status, DEV_BAD_INPUT);
      continue;
    }
    if (atomicCAS(&idx[u], -1, i) != -1) dev_fail(status, DEV_BAD_INPUT);
  }
}

// The nets of the moved nodes, each listed once (one warp per move, lanes
// over its incident nets).
__global__ void k_gr_nets(const int32_t* __restrict__ nodes, int32_t l, int32_t n,
                          const int32_t* __restrict__ ioff, const int32_t* __restrict__ inets,
                          int32_t* __restrict__ mark, int32_t* __restrict__ list,
                          int32_t* __restrict__ count) {
  const int wv = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int32_t i = wv; i < l; i += nw) {
    const int32_t u = nodes[i];
    if (u < 0 || u >= n) continue;  // reported by k_gr_index
    for (int32_t j = ioff[u] + lane_id(); j < ioff[u + 1]; j += 32) {
      const int32_t e = inets[j];
      if (atomicExch(&mark[e], 1) == 0) list[atomicAdd(count, 1)] = e;
    }
  }
}

// One warp per listed net: the two loops of Algorithm 4 over the net's pins,
// with the per-block first_in / last_out / non_moved arrays of the warp in
// shared memory (k <= 64).
__global__ void __launch_bounds__(GR_WARPS * 32)
k_gr_net(const int32_t* __restrict__ list, const int32_t* __restrict__ count,
         const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
         const int32_t* __restrict__ w, const int32_t* __restrict__ part,
         const int32_t* __restrict__ idx, const int32_t* __restrict__ targets, int k,
         unsigned long long* __restrict__ gains, int32_t* status) {
  __shared__ int32_t s_first_in[GR_WARPS][HG_MAX_K];
  __shared__ int32_t s_last_out[GR_WARPS][HG_MAX_K];
  __shared__ int32_t s_non_moved[GR_WARPS][HG_MAX_K];
  const int wv = warp_in_block(), lane = lane_id();
  int32_t* first_in = s_first_in[wv];
  int32_t* last_out = s_last_out[wv];
  int32_t* non_moved = s_non_moved[wv];
  for (int b = lane; b < HG_MAX_K; b += 32) {
    first_in[b] = INT32_MAX;
    last_out[b] = -1;
    non_moved[b] = 0;
  }
  __syncwarp();
  const int32_t cnt = *count;
  for (int32_t x = blockIdx.x * GR_WARPS + wv; x < cnt; x += gridDim.x * GR_WARPS) {
    const int32_t e = list[x];
    const int32_t b = eoff[e], end = eoff[e + 1];
    for (int32_t q = b + lane; q < end; q += 32) {
      const int32_t v = pins[q];
      const int32_t i = idx[v];
      const int32_t s = part[v];
      if (s < 0 || s >= k) {  // a block id out of range: bad input, never indexed
        dev_fail(status, DEV_BAD_INPUT);
        continue;
      }
      if (i >= 0) {
        atomicMax(&last_out[s], i);
        atomicMin(&first_in[targets[i]], i);
      } else {
        atomicAdd(&non_moved[s], 1);
      }
    }
    __syncwarp();
    const long long we = w[e];
    for (int32_t q = b + lane; q < end; q += 32) {
      const int32_t v = pins[q];
      const int32_t i = idx[v];
      if (i < 0) continue;
      const int s = part[v], t = targets[i];  // both checked by k_gr_index
      long long d = 0;
      if (last_out[s] == i && i < first_in[s] && non_moved[s] == 0) d += we;
      if (first_in[t] == i && i > last_out[t] && non_moved[t] == 0) d -= we;
      if (d) atomicAdd(&gains[i], (unsigned long long)d);
    }
    __syncwarp();
    for (int bb = lane; bb < k; bb += 32) {
      first_in[bb] = INT32_MAX;
      last_out[bb] = -1;
      non_moved[bb] = 0;
    }
    __syncwarp();
  }
}

}  // namespace

void recalculate_gains(const Ctx& cx, const Level& L, int k, const int32_t* part, int32_t l,
                       const int32_t* nodes, const int32_t* targets, int64_t* gains) {
  if (l == 0) return;
  HG_CUDA(cudaMemsetAsync(gains, 0, sizeof(int64_t) * (size_t)l, cx.stream));
  DBuf<int32_t> idx, mark, list, count;
  idx.alloc(&cx.alloc, (size_t)L.n);
  mark.alloc(&cx.alloc, (size_t)std::max<int32_t>(L.m, 1));
  list.alloc(&cx.alloc, (size_t)std::max<int32_t>(L.m, 1));
  count.alloc(&cx.alloc, 1);
  fill_i32(cx, idx.p, -1, L.n);
  HG_CUDA(cudaMemsetAsync(mark.p, 0, mark.bytes(), cx.stream));
  HG_CUDA(cudaMemsetAsync(count.p, 0, sizeof(int32_t), cx.stream));
  k_gr_index<<<grid_for(l, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(nodes, targets, l, L.n, k,
                                                                     part, idx.p, cx.d_status);
  check_launch("gr_index");
  k_gr_nets<<<grid_for(l, 8, cx.num_sms, 16), 256, 0, cx.stream>>>(nodes, l, L.n, L.ioff.p,
                                                                   L.inets.p, mark.p, list.p,
                                                                   count.p);
  check_launch("gr_nets");
  k_gr_net<<<cx.num_sms * 8, GR_WARPS * 32, 0, cx.stream>>>(
      list.p, count.p, L.eoff.p, L.pins.p, L.w.p, part, idx.p, targets, k,
      reinterpret_cast<unsigned long long*>(gains), cx.d_status);
  check_launch("gr_net");
  if (cx.launches) *cx.launches += 4;
  check_status(cx);
}

}  // namespace hgk
