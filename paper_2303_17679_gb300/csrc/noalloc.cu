// hg_objective_noalloc: the connectivity objective (for every net, its
// weight times the number of blocks it touches minus one, summed) and the
// block weights of a partition of a caller-held device CSR, with no handle
// and no device allocation.  The paper has no counterpart; this is a library
// convenience for callers that must not allocate.
//
// All scratch lives in one file-scope device array.  Host code looks its
// address up with cudaGetSymbolAddress on every call (cheap, allocates
// nothing, and stays right if the module is loaded again, for example after
// cudaDeviceReset or under another context):
//   [0, NA_BLOCKS)            objective partial of every block (written by
//                             its block before it is read; no initial value)
//   [NA_BW, NA_BW + 64)       block-weight accumulators      - must be zero
//   NA_TICKET                 count of finished blocks       - must be zero
//   NA_STATUS                 bad-input flag                 - must be zero
//   [NA_RES, NA_RES + 66)     result record: objective, status, 64 weights
// Before every launch the host clears the zero words and marks the result
// record's status as unwritten (both with cudaMemsetAsync, which allocates
// nothing), so a launch that did not finish is reported instead of leaving
// an earlier call's result to be read; the last block of a launch also sets
// the zero words back to zero after it has read them.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int NA_BLOCKS = 1024;  // grid cap = objective partial slots
constexpr int NA_THREADS = 256;
constexpr int NA_BW = NA_BLOCKS;
constexpr int NA_TICKET = NA_BW + HG_MAX_K;
constexpr int NA_STATUS = NA_TICKET + 1;
constexpr int NA_RES = NA_STATUS + 1;  // objective, status, weights[64]
constexpr int NA_WORDS = NA_RES + 2 + HG_MAX_K;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_WORDS];

// One warp per net: lambda(e) = popcount of the OR of the blocks of its pins;
// one thread per node for the block weights.  Offsets outside [0, p], pins
// outside [0, n) and block ids outside [0, k) set the status word and are
// skipped, so no access leaves the caller's arrays.  The last block to finish
// sums the partials in block order and publishes the result record.
__global__ void __launch_bounds__(NA_THREADS)
k_objective_noalloc(const int32_t* __restrict__ eoff, const int32_t* __restrict__ pins,
                    const int32_t* __restrict__ w, const int32_t* __restrict__ c, int32_t n,
                    int32_t m, int64_t p, int32_t k, const int32_t* __restrict__ part,
                    unsigned long long* __restrict__ S) {
  __shared__ unsigned long long s_bw[HG_MAX_K];
  __shared__ unsigned long long s_warp[NA_THREADS / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < HG_MAX_K; i += blockDim.x) s_bw[i] = 0;
  __syncthreads();

  bool bad = false;
  unsigned long long obj = 0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = gw; e < m; e += nw) {
    const int64_t b = eoff[e], t = eoff[e + 1];
    if (b < 0 || t < b || t > p) {
      bad = true;
      continue;
    }
    unsigned long long mask = 0;
    for (int64_t q = b + lane; q < t; q += 32) {
      const int32_t v = pins[q];
      if (v < 0 || v >= n) { bad = true; continue; }
      const int32_t blk = part[v];
      if (blk < 0 || blk >= k) { bad = true; continue; }
      mask |= 1ull << blk;
    }
    for (int o = 16; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    const int lam = __popcll(mask);
    if (lane == 0 && lam > 1) obj += (unsigned long long)(lam - 1) * (unsigned long long)(w ? w[e] : 1);
  }
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t blk = part[u];
    if (blk < 0 || blk >= k) { bad = true; continue; }
    atomicAdd(&s_bw[blk], (unsigned long long)(c ? c[u] : 1));
  }

  for (int o = 16; o > 0; o >>= 1) obj += __shfl_xor_sync(0xffffffffu, obj, o);
  if (lane == 0) s_warp[wv] = obj;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&S[NA_STATUS], 1ull);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int i = 0; i < NA_THREADS / 32; ++i) sum += s_warp[i];
    S[blockIdx.x] = sum;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (s_bw[i]) atomicAdd(&S[NA_BW + i], s_bw[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = atomicAdd(&S[NA_TICKET], 1ull) == (unsigned long long)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;

  // last block: every other block's writes are visible after the fence
  __threadfence();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (unsigned i = 0; i < gridDim.x; ++i) sum += __ldcg(&S[i]);
    S[NA_RES] = sum;
    S[NA_RES + 1] = atomicExch(&S[NA_STATUS], 0ull);
  }
  for (int i = threadIdx.x; i < HG_MAX_K; i += blockDim.x)
    S[NA_RES + 2 + i] = atomicExch(&S[NA_BW + i], 0ull);
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(&S[NA_TICKET], 0ull);
}

constexpr unsigned long long NA_UNWRITTEN = ~0ull;  // result status before the last block

int cuda_fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? HG_ERR_OOM : HG_ERR_CUDA;
}

}  // namespace

extern "C" int hg_objective_noalloc(int32_t n, int32_t m, int64_t p, const int32_t* net_offsets,
                                    const int32_t* pins, const int32_t* net_weights,
                                    const int32_t* node_weights, int32_t k, const int32_t* part,
                                    void* cuda_stream, int64_t* out_objective,
                                    int64_t* out_block_weights) {
  if (n < 1 || m < 0 || p < 0 || p > INT32_MAX || out_objective == nullptr) return HG_ERR_INVALID;
  if (k < 1) return HG_ERR_INVALID;
  if (k > HG_MAX_K) return HG_ERR_UNSUPPORTED;  // 64 block-weight slots in the scratch
  if (net_offsets == nullptr || part == nullptr || (p > 0 && pins == nullptr))
    return HG_ERR_INVALID;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  // the scratch address in the current context (the first call on a device
  // loads the module, so it should come before any stream capture)
  void* addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned long long* S = static_cast<unsigned long long*>(addr);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t work = std::max<int64_t>((int64_t)m * 32, n);
  int64_t blocks = (work + NA_THREADS - 1) / NA_THREADS;
  blocks = std::min<int64_t>(blocks, std::min<int64_t>(NA_BLOCKS, (int64_t)sms * 8));
  blocks = std::max<int64_t>(blocks, 1);
  // zero words cleared, result status marked unwritten
  e = cudaMemsetAsync(S + NA_BW, 0, sizeof(unsigned long long) * (HG_MAX_K + 2), st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemsetAsync(S + NA_RES + 1, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e);
  k_objective_noalloc<<<(unsigned)blocks, NA_THREADS, 0, st>>>(net_offsets, pins, net_weights,
                                                               node_weights, n, m, p, k, part, S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned long long res[2 + HG_MAX_K];
  e = cudaMemcpyAsync(res, S + NA_RES, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (res[1] == NA_UNWRITTEN) return HG_ERR_CUDA;
  if (res[1] != 0) return HG_ERR_INVALID;
  *out_objective = (int64_t)res[0];
  if (out_block_weights)
    for (int i = 0; i < k; ++i) out_block_weights[i] = (int64_t)res[2 + i];
  return HG_OK;
}
