// Load-balanced iteration over the pins of a net-major CSR.
//
// A pin tile is PIN_TILE consecutive pin positions.  tile_net[t] holds the
// net that contains pin position t * PIN_TILE (built once per level), so a
// block handling tile t finds every net overlapping its tile between
// tile_net[t] and tile_net[t+1], stages their offsets in shared memory and
// maps each of its pins to its net with a short binary search there.  Every
// block gets the same number of pins whatever the net-size distribution
// (100,000-pin nets and 2-pin nets alike).
#pragma once

#include "common.cuh"

namespace hgk {

constexpr int PIN_TILE = 2048;
constexpr int PIN_TILE_THREADS = 256;

__host__ __device__ inline int64_t num_pin_tiles(int64_t p) { return (p + PIN_TILE - 1) / PIN_TILE; }

// Builds tile_net (num_pin_tiles(p) + 1 entries) for a CSR without empty nets.
void build_tile_index(const Ctx& cx, const int32_t* eoff, int32_t m, int64_t p, int32_t* tile_net);

struct PinTileView {
  int64_t q0;      // first pin position of the tile
  int64_t q1;      // one past the last
  int32_t e_lo;    // first net overlapping the tile
  int32_t count;   // nets e_lo .. e_lo + count - 1 overlap the tile
};

// Stages eoff[e_lo .. e_lo + count] in s_off (capacity PIN_TILE + 3).  All
// threads of the block must call it.
__device__ __forceinline__ PinTileView stage_pin_tile(const int32_t* __restrict__ eoff,
                                                      const int32_t* __restrict__ tile_net,
                                                      int32_t m, int64_t p, int64_t tile,
                                                      int32_t* s_off) {
  PinTileView v;
  v.q0 = tile * PIN_TILE;
  v.q1 = v.q0 + PIN_TILE < p ? v.q0 + PIN_TILE : p;
  v.e_lo = tile_net[tile];
  const int32_t e_hi = tile_net[tile + 1];  // net of the next tile's first pin (or m - 1)
  v.count = e_hi - v.e_lo + 1;
  for (int i = threadIdx.x; i <= v.count; i += blockDim.x) {
    const int32_t e = v.e_lo + i;
    s_off[i] = e <= m ? eoff[e] : eoff[m];
  }
  __syncthreads();
  return v;
}

// Index (relative to e_lo) of the net holding pin position q of the tile.
__device__ __forceinline__ int32_t net_in_tile(const int32_t* s_off, int32_t count, int64_t q) {
  int32_t lo = 0, hi = count - 1;  // largest i with s_off[i] <= q
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)s_off[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace hgk
