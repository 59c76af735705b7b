// ingest.cu -- one pass over an input CSR's entries that copies them to the
// device and takes everything graph creation needs to know about them.
//
// The entries may be read straight from host memory that is mapped into the
// device's address space (pinned host buffers): the pass then runs at the
// host link's rate and the checks cost nothing extra.  Per entry (u, v, w):
//   * the weight statistics: sum of the non-negative weights, any negative
//     weight (the weights must be non-negative, Sec. 2: c : E -> N);
//   * the canonical-form test: every row strictly increasing, v in [0, n),
//     no self-loop, w > 0 (the form every contraction writes; an input in
//     that form needs no canonicalisation sort);
//   * a symmetry fingerprint of the undirected graph: the entries with
//     u < v and the mirrored entries with u > v must be the same set of
//     triples (min, max, w).  Each triple is mapped by two 64-bit mixing
//     functions and the images are added (u < v) or subtracted (u > v)
//     modulo 2^64, together with a +1/-1 count.  A symmetric canonical
//     graph gives (0, 0, 0); an asymmetric one does so only if its two
//     triple sets differ yet collide in both 64-bit sums.
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "tiles.cuh"

namespace mc {

namespace {

// MurmurHash3's 64-bit finalizer (A. Appleby, public domain).
__device__ __forceinline__ unsigned long long mix_murmur(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// The SplitMix64 output function (G. Steele, D. Lea, C. Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014).
__device__ __forceinline__ unsigned long long mix_splitmix(unsigned long long x) {
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

constexpr unsigned long long kGolden = 0x9e3779b97f4a7c15ull;

// stats: [0] weight sum, [1] negative weight, [2] non-canonical entry,
// [3], [4] signed fingerprints, [5] signed (u < v) - (u > v) count.
template <bool kCopy>
__global__ void __launch_bounds__(kETThreads)
    ingest_kernel(int n, long long M, const int64_t* __restrict__ rp,
                  const int* __restrict__ col_src, const int* __restrict__ w_src,
                  int* __restrict__ col_dst, int* __restrict__ w_dst,
                  const int* __restrict__ tile_row, int ntiles,
                  unsigned long long* __restrict__ stats) {
  __shared__ TileRowsSmem tr;
  __shared__ int s_col[kETThreads];
  __shared__ unsigned long long s_red[4][kETThreads / 32];
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long e0 = (long long)blockIdx.x * kET;
  // the entry before the tile (tile starts are < M)
  int carry = (t == 0 && e0 > 0) ? col_src[e0 - 1] : 0;
  unsigned long long sum = 0, h1 = 0, h2 = 0;
  int bal = 0;
  bool neg = false, bad = false;
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + (long long)i * kETThreads + t;
    const bool valid = e < M;
    const int v = valid ? col_src[e] : 0;
    const int c = valid ? w_src[e] : 0;
    if (kCopy && valid) {
      col_dst[e] = v;
      w_dst[e] = c;
    }
    s_col[t] = v;
    __syncthreads();
    const int prev = t > 0 ? s_col[t - 1] : carry;
    if (t == 0) carry = s_col[kETThreads - 1];
    __syncthreads();
    if (valid) {
      const int u = tile_row_of(tr, rp, e);
      const long long row_start =
          tr.use ? tr.rp[u - tr.r0] : (long long)rp[u];
      if (c < 0) neg = true; else sum += (unsigned long long)c;
      bad |= v < 0 || v >= n || v == u || c <= 0 || (e > row_start && prev >= v);
      if (v != u) {
        const unsigned a = (unsigned)min(u, v), b = (unsigned)max(u, v);
        const unsigned long long key = ((unsigned long long)a << 32) | b;
        const unsigned long long wc = (unsigned long long)(unsigned)c;
        const unsigned long long x1 = mix_murmur(key ^ (wc * kGolden));
        const unsigned long long x2 = mix_splitmix(key + kGolden * (wc + 1));
        if (u < v) {
          h1 += x1;
          h2 += x2;
          ++bal;
        } else {
          h1 -= x1;
          h2 -= x2;
          --bal;
        }
      }
    }
  }
  // block reduction, then one atomic per word
  sum = warp_sum(sum);
  h1 = warp_sum(h1);
  h2 = warp_sum(h2);
  bal = (int)__reduce_add_sync(FULL, (unsigned)bal);
  if (lane == 0) {
    s_red[0][warp] = sum;
    s_red[1][warp] = h1;
    s_red[2][warp] = h2;
    s_red[3][warp] = (unsigned long long)(long long)bal;
  }
  const bool any_neg = __syncthreads_or(neg);
  const bool any_bad = __syncthreads_or(bad);
  if (t < 4) {
    unsigned long long r = 0;
    for (int k = 0; k < kETThreads / 32; ++k) r += s_red[t][k];
    const int slot = t == 0 ? 0 : t + 2;  // sum -> 0, h1 -> 3, h2 -> 4, balance -> 5
    if (r) atomicAdd(&stats[slot], r);
  }
  if (t == 0) {
    if (any_neg) atomicOr(&stats[1], 1ull);
    if (any_bad) atomicOr(&stats[2], 1ull);
  }
}

}  // namespace

cudaError_t ingest_csr(int n, long long M, const int64_t* rp, const int* col_src,
                       const int* w_src, int* col_dst, int* w_dst, const int* tile_row,
                       unsigned long long* stats, cudaStream_t s, int* launches) {
  if (M <= 0) return cudaGetLastError();
  const int ntiles = (int)((M + kET - 1) / kET);
  if (col_dst != col_src)
    ingest_kernel<true><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col_src, w_src, col_dst, w_dst,
                                                      tile_row, ntiles, stats);
  else
    ingest_kernel<false><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col_src, w_src, col_dst,
                                                       w_dst, tile_row, ntiles, stats);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace mc
