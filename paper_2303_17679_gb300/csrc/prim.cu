// Data-parallel primitives: exclusive prefix sums, fills, scalar readback.
// The prefix sums are the "parallel prefix sum operations" the contraction
// algorithm relies on (Sec. 4.2), written here without CUB.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace hgk {

// The library's own stream-ordered pool per device, created on first use and
// kept for the life of the process.  Its release threshold is unlimited, so
// blocks freed by one handle stay in the pool for the next instead of going
// back to the driver (and hg_trim_memory returns them); the device's default
// pool, which other code in the process may use, is left as it is.
cudaMemPool_t library_pool(int device) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> g(mu);
  if (device < 0) throw HgError(HG_ERR_CUDA, "bad device ordinal");
  if ((size_t)device >= pools.size()) pools.resize((size_t)device + 1, nullptr);
  if (!pools[device]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    HG_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = ~0ull;
    HG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    pools[device] = pool;
  }
  return pools[device];
}

void* Alloc::get(size_t bytes) const {
  void* p = nullptr;
  if (bytes == 0) return nullptr;
  if (fn_alloc) {
    p = fn_alloc(bytes, ctx);
    if (!p) throw HgError(HG_ERR_OOM, "device allocation hook returned NULL");
    return p;
  }
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw HgError(e == cudaErrorMemoryAllocation ? HG_ERR_OOM : HG_ERR_CUDA,
                  std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
  }
  return p;
}

void Alloc::put(void* p) const {
  if (!p) return;
  if (fn_free) fn_free(p, ctx);
  else cudaFreeAsync(p, stream);
}

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename TIn>
__global__ void k_tile_sums(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ partial) {
  __shared__ int64_t red[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t q = base + i * SCAN_THREADS + threadIdx.x;
    if (q < n) s += (int64_t)in[q];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Exclusive scan of the tile sums by one block; also writes the grand total.
template <typename TOut>
__global__ void k_scan_partials(int64_t* __restrict__ partial, int64_t nb, TOut* __restrict__ total) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? partial[i] : 0;
    int64_t x = warp_inclusive_scan(v);
    if (lane_id() == 31) wsum[warp_in_block()] = x;
    __syncthreads();
    if (warp_in_block() == 0) {
      int64_t w = lane_id() < (int)(blockDim.x >> 5) ? wsum[lane_id()] : 0;
      wsum[lane_id()] = warp_inclusive_scan(w);
    }
    __syncthreads();
    const int64_t before = warp_in_block() ? wsum[warp_in_block() - 1] : 0;
    const int64_t c0 = carry;
    if (i < nb) partial[i] = c0 + before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = (TOut)carry;
}

template <typename TIn, typename TOut>
__global__ void k_tile_scan(const TIn* in, TOut* out, int64_t n, const int64_t* __restrict__ partial) {
  __shared__ int64_t tile[SCAN_TILE];
  __shared__ int64_t wsum[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t q = base + i * SCAN_THREADS + threadIdx.x;
    tile[i * SCAN_THREADS + threadIdx.x] = q < n ? (int64_t)in[q] : 0;
  }
  __syncthreads();
  int64_t vals[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    vals[i] = tile[threadIdx.x * SCAN_ITEMS + i];
    s += vals[i];
  }
  int64_t x = warp_inclusive_scan(s);
  if (lane_id() == 31) wsum[warp_in_block()] = x;
  __syncthreads();
  if (warp_in_block() == 0) {
    int64_t w = lane_id() < SCAN_THREADS / 32 ? wsum[lane_id()] : 0;
    w = warp_inclusive_scan(w);
    if (lane_id() < SCAN_THREADS / 32) wsum[lane_id()] = w;
  }
  __syncthreads();
  int64_t run = partial[blockIdx.x] + (warp_in_block() ? wsum[warp_in_block() - 1] : 0) + x - s;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    tile[threadIdx.x * SCAN_ITEMS + i] = run;
    run += vals[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t q = base + i * SCAN_THREADS + threadIdx.x;
    if (q < n) out[q] = (TOut)tile[i * SCAN_THREADS + threadIdx.x];
  }
}

template <typename TIn, typename TOut>
void scan_impl(const Ctx& cx, const TIn* in, TOut* out, int64_t n, TOut* d_total) {
  if (n <= 0) {
    if (d_total) HG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(TOut), cx.stream));
    return;
  }
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBuf<int64_t> partial;
  partial.alloc(&cx.alloc, (size_t)nb);
  k_tile_sums<TIn><<<(unsigned)nb, SCAN_THREADS, 0, cx.stream>>>(in, n, partial.p);
  check_launch("tile_sums");
  k_scan_partials<TOut><<<1, 1024, 0, cx.stream>>>(partial.p, nb, d_total);
  check_launch("scan_partials");
  k_tile_scan<TIn, TOut><<<(unsigned)nb, SCAN_THREADS, 0, cx.stream>>>(in, out, n, partial.p);
  check_launch("tile_scan");
  if (cx.launches) *cx.launches += 3;
}

__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_iota_i32(int32_t* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

}  // namespace

void scan_exclusive_i32(const Ctx& cx, const int32_t* in, int32_t* out, int64_t n, int32_t* d_total) {
  scan_impl<int32_t, int32_t>(cx, in, out, n, d_total);
}

void scan_exclusive_i32_to_i64(const Ctx& cx, const int32_t* in, int64_t* out, int64_t n,
                               int64_t* d_total) {
  scan_impl<int32_t, int64_t>(cx, in, out, n, d_total);
}

void fill_i32(const Ctx& cx, int32_t* p, int32_t value, int64_t n) {
  if (n <= 0) return;
  k_fill_i32<<<grid_for(n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(p, value, n);
  check_launch("fill");
  if (cx.launches) *cx.launches += 1;
}

void iota_i32(const Ctx& cx, int32_t* p, int64_t n) {
  if (n <= 0) return;
  k_iota_i32<<<grid_for(n, 256, cx.num_sms, 8), 256, 0, cx.stream>>>(p, n);
  check_launch("iota");
  if (cx.launches) *cx.launches += 1;
}

void wait_stream(const Ctx& cx) {
  if (cx.sync_event) {
    HG_CUDA(cudaEventRecord(cx.sync_event, cx.stream));
    HG_CUDA(cudaEventSynchronize(cx.sync_event));
  } else {
    HG_CUDA(cudaStreamSynchronize(cx.stream));
  }
}

void check_status(const Ctx& cx) {
  wait_stream(cx);
  int32_t st = 0;
  HG_CUDA(cudaMemcpyAsync(&st, cx.d_status, sizeof(st), cudaMemcpyDeviceToHost, cx.stream));
  HG_CUDA(cudaStreamSynchronize(cx.stream));
  if (st != DEV_OK) {
    int32_t zero = 0;
    cudaMemcpy(cx.d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    switch (st) {
      case DEV_TIMEOUT: throw HgError(HG_ERR_TIMEOUT, "a bounded device wait gave up");
      case DEV_BAD_INPUT: throw HgError(HG_ERR_INVALID, "device-side input validation failed");
      case DEV_HASH_FULL: throw HgError(HG_ERR_CUDA, "internal: hash table full");
      default: throw HgError(HG_ERR_CUDA, "internal: device capacity exceeded");
    }
  }
}

int32_t read_i32(const Ctx& cx, const int32_t* d) {
  int32_t v = 0;
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  return v;
}

int64_t read_i64(const Ctx& cx, const int64_t* d) {
  int64_t v = 0;
  wait_stream(cx);
  HG_CUDA(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, cx.stream));
  check_status(cx);
  return v;
}

}  // namespace hgk
