// tiles.cuh -- entry tiles shared by the entry-parallel kernels.
//
// An entry tile is kEntryTile consecutive CSR entries handled by one block of
// kETThreads threads (kETItems entries each).  tile_rows() records the row of
// each tile's first entry; a block loads the row offsets its tile spans into
// shared memory and finds the row of an entry by binary search there.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

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

// Run layout of an entry tile: thread t owns the kETItems consecutive
// entries e0 + kETItems * t ... (clipped to M), so that it finds its first
// entry's row once and walks the rows forward instead of searching the row
// of every entry.  tile_rp(s, rp, r) = rp[r] for rows r0 .. r1 + 1.
__device__ __forceinline__ long long tile_rp(const TileRowsSmem& s, const int64_t* rp, int r) {
  return s.use ? s.rp[r - s.r0] : (long long)rp[r];
}

// Loads a thread's run of cnt <= kETItems entries starting at eb: 16-byte
// vector loads when the run is whole and the arrays are 16-byte aligned.
template <typename WT>
__device__ __forceinline__ void load_run(const int* __restrict__ col, const WT* __restrict__ w,
                                         long long eb, int cnt, int (&c)[kETItems],
                                         WT (&x)[kETItems]) {
  static_assert(kETItems == 8, "run loads assume 8 entries per thread");
  const bool vec = cnt == kETItems && ((reinterpret_cast<uintptr_t>(col) |
                                         reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  if (vec) {
    const int4* cp = reinterpret_cast<const int4*>(col + eb);
    const int4 a = cp[0], b = cp[1];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    if (sizeof(WT) == 4) {
      const int4* wp = reinterpret_cast<const int4*>(w + eb);
      const int4 p = wp[0], q = wp[1];
      x[0] = (WT)p.x; x[1] = (WT)p.y; x[2] = (WT)p.z; x[3] = (WT)p.w;
      x[4] = (WT)q.x; x[5] = (WT)q.y; x[6] = (WT)q.z; x[7] = (WT)q.w;
    } else {
      const longlong2* wp = reinterpret_cast<const longlong2*>(w + eb);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const longlong2 p = wp[k];
        x[2 * k] = (WT)p.x;
        x[2 * k + 1] = (WT)p.y;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < kETItems; ++k) {
      c[k] = k < cnt ? col[eb + k] : 0;
      x[k] = k < cnt ? w[eb + k] : WT(0);
    }
  }
}

}  // namespace mc
