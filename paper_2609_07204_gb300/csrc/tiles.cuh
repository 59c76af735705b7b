// tiles.cuh -- entry tiles shared by the entry-parallel kernels.
//
// An entry tile is kEntryTile consecutive CSR entries handled by one block of
// kETThreads threads (kETItems entries each).  tile_rows() records the row of
// each tile's first entry; a block loads the row offsets its tile spans into
// shared memory and finds the row of an entry by binary search there.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mc {

constexpr int kET = kEntryTile;
constexpr int kETThreads = 256;
constexpr int kETItems = kET / kETThreads;  // 8

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

inline int grid_blocks(long long work, int per_block, int cap_per_sm = 32) {
  long long b = (work + per_block - 1) / per_block;
  const long long cap = (long long)num_sms() * cap_per_sm;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Largest index i in [lo, hi) with a[i] <= x (a non-decreasing, a[lo] <= x).
template <typename P>
__device__ __forceinline__ int row_in(const P* a, int lo, int hi, long long x) {
  while (hi - lo > 1) {
    int mid = lo + ((hi - lo) >> 1);
    if ((long long)a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Shared-memory description of the rows covering one entry tile.
struct TileRowsSmem {
  long long rp[kET + 2];
  int r0, r1, use;
};

__device__ __forceinline__ void tile_rows_load(TileRowsSmem& s, const int64_t* rp, int n,
                                               const int* tile_row, int ntiles, int t) {
  if (threadIdx.x == 0) {
    s.r0 = tile_row[t];
    s.r1 = (t + 1 < ntiles) ? tile_row[t + 1] : n - 1;
    s.use = (s.r1 - s.r0 + 2) <= (kET + 2);
  }
  __syncthreads();
  if (s.use)
    for (int i = threadIdx.x; i < s.r1 - s.r0 + 2; i += blockDim.x) s.rp[i] = rp[s.r0 + i];
  __syncthreads();
}

__device__ __forceinline__ int tile_row_of(const TileRowsSmem& s, const int64_t* rp, long long e) {
  return s.use ? s.r0 + row_in(s.rp, 0, s.r1 - s.r0 + 1, e) : row_in(rp, s.r0, s.r1 + 1, e);
}

// Warp-level segmented sum over 32 consecutive entries whose segment keys
// (row ids) are non-decreasing across lanes; the last lane of each segment
// adds the segment's total to out[target].  Lanes with valid == false must
// come after all valid lanes (tile tails).
template <typename T, typename O>
__device__ __forceinline__ void warp_segment_add(int seg, int target, T val, bool valid, O* out) {
  const int lane = threadIdx.x & 31;
  T x = valid ? val : T(0);
  const int r = valid ? seg : -1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(FULL, x, o);
    const int ry = __shfl_up_sync(FULL, r, o);
    if (lane >= o && ry == r) x += y;
  }
  const int rn = __shfl_down_sync(FULL, r, 1);
  const bool last = lane == 31 || rn != r;
  if (valid && last && x != T(0)) atomic_add_w(&out[target], (O)x);
}

}  // namespace mc
