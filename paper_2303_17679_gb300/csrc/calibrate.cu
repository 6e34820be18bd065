// hg_calibrate_smem_atomics: a measured ceiling for the rating's secondary
// bound.  The rating (Sec. 4.1) adds every pin visit's term to a cluster's
// entry of a shared-memory hash table, so at most one shared-memory atomic
// add per visit can retire per lane and cycle.  This times conflict-free
// 32-bit and 64-bit shared-memory atomic adds over every SM with CUDA events
// and returns the rate in operations per second, against which the rating's
// visits per second are reported.  The paper has no counterpart.
#include "common.cuh"

namespace {

constexpr int CAL_THREADS = 1024;
constexpr int CAL_ITERS = 4096;

static __device__ unsigned long long g_cal_sink;

// Every lane adds to its own word (lane i of a warp in bank i), so no two
// lanes of a warp conflict; the words are summed into a sink at the end so
// the adds cannot be dropped.
template <typename T>
__global__ void __launch_bounds__(CAL_THREADS) k_smem_atomics(T step) {
  __shared__ T s[CAL_THREADS];
  s[threadIdx.x] = 0;
  __syncthreads();
  T* mine = &s[threadIdx.x];
  for (int i = 0; i < CAL_ITERS; ++i) atomicAdd(mine, step);
  __syncthreads();
  if (*mine == (T)0x7fffffff) atomicAdd(&g_cal_sink, 1ull);
}

template <typename T>
double time_kernel(cudaStream_t st, int blocks) {
  cudaEvent_t a = nullptr, b = nullptr;
  HG_CUDA(cudaEventCreate(&a));
  HG_CUDA(cudaEventCreate(&b));
  float best = 0;
  for (int rep = 0; rep < 5; ++rep) {
    HG_CUDA(cudaEventRecord(a, st));
    k_smem_atomics<T><<<blocks, CAL_THREADS, 0, st>>>((T)1);
    hgk::check_launch("smem_atomics");
    HG_CUDA(cudaEventRecord(b, st));
    HG_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    HG_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0 && (best == 0 || ms < best)) best = ms;  // first run warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)blocks * CAL_THREADS * CAL_ITERS / (best * 1e-3);
}

}  // namespace

extern "C" int hg_calibrate_smem_atomics(void* cuda_stream, double* out_u32_per_s,
                                         double* out_u64_per_s) {
  if (!out_u32_per_s || !out_u64_per_s) return HG_ERR_INVALID;
  try {
    int dev = 0, sms = 0, per_sm = 0;
    HG_CUDA(cudaGetDevice(&dev));
    HG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smem_atomics<uint32_t>,
                                                          CAL_THREADS, 0));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    *out_u32_per_s = time_kernel<uint32_t>(st, blocks);
    *out_u64_per_s = time_kernel<unsigned long long>(st, blocks);
  } catch (const hgk::HgError& e) {
    return e.code;
  }
  return HG_OK;
}
