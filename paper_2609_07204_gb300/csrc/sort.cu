// sort.cu -- onesweep LSD radix sort of (u64 key, weight) pairs and a
// device-wide exclusive scan.
//
// The contraction sorts the relabelled entries on the key (u' << b) | v'
// (Sec. 2 "Basic Concepts": contracted vertices inherit their members' edges;
// parallel edges are then adjacent and summed).  The sort is a single-pass
// ("onesweep") LSD radix sort, 8 bits per pass:
//   1. one histogram kernel counts every digit of every pass in one read;
//   2. each pass is one kernel: a tile of 3072 keys is ranked inside the block
//      (warp-striped layout + match.any keeps it stable), its digit counts
//      are published to a decoupled look-back array, the tile reads its
//      predecessors' counts, and the keys are scattered through shared memory
//      so that runs of equal digits are written contiguously.
// Tile ids come from an atomic counter, so a tile only waits on tiles that
// already started; every wait is also bounded (spin_limit) and a timeout
// sets ERR_TIMEOUT instead of hanging.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mc {

namespace {
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = kSortTile / kRsThreads;  // 12
constexpr int kRsTile = kSortTile;
static_assert(kRsItems * kRsThreads == kRsTile, "tile");
constexpr u64 kFlagAgg = 1ull << 62;
constexpr u64 kFlagInc = 2ull << 62;
constexpr u64 kCountMask = (1ull << 62) - 1;

__global__ void rs_hist_kernel(const u64* __restrict__ keys, int N, int passes,
                               unsigned* __restrict__ ghist) {
  __shared__ unsigned sh[8 * 256];
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    u64 k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * 256 + ((k >> (8 * p)) & 255)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&ghist[i], sh[i]);
}

// One block of 256 threads per pass: goff[p][d] = sum_{d' < d} hist[p][d'].
__global__ void rs_scan_hist_kernel(const unsigned* __restrict__ ghist,
                                    unsigned* __restrict__ goff) {
  __shared__ unsigned s[256];
  const int p = blockIdx.x, d = threadIdx.x;
  unsigned v = ghist[p * 256 + d];
  s[d] = v;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    unsigned t = d >= o ? s[d - o] : 0;
    __syncthreads();
    s[d] += t;
    __syncthreads();
  }
  goff[p * 256 + d] = s[d] - v;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ unsigned block_exclusive_256(unsigned v, unsigned* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  unsigned add = 0;
  for (int w2 = 0; w2 < warp; ++w2) add += warp_tot[w2];
  return x - v + add;
}

template <typename WT>
__global__ void __launch_bounds__(kRsThreads, 3)
    rs_pass_kernel(const u64* __restrict__ kin, const WT* __restrict__ vin,
                   u64* __restrict__ kout, WT* __restrict__ vout, int N, int shift, const unsigned* __restrict__ goff, u64* lookback,
                   unsigned long long* tile_counter, unsigned* err, long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64* skeys = reinterpret_cast<u64*>(smem);
  WT* svals = reinterpret_cast<WT*>(skeys + kRsTile);
  unsigned* whist = reinterpret_cast<unsigned*>(svals + kRsTile);  // [8][256]
  __shared__ unsigned s_tile_start[256];
  __shared__ unsigned long long s_gbase[256];
  __shared__ unsigned s_warp_tot[kRsWarps];
  __shared__ int s_tile;
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = (int)atomicAdd(tile_counter, 1ull);
    s_fail = 0;
  }
  for (int i = tid; i < kRsWarps * 256; i += kRsThreads) whist[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  const long long tile_base = (long long)tile * kRsTile;
  if (tile_base >= N) return;  // surplus block (grid sized for the upper bound)

  // ---- load (warp-striped: warp w owns keys [w*384, w*384+384) of the tile)
  u64 k[kRsItems];
  WT v[kRsItems];
  unsigned short rank[kRsItems];
  const long long wbase = tile_base + warp * (kRsItems * 32);
#pragma unroll
  for (int i = 0; i < kRsItems; ++i) {
    long long idx = wbase + i * 32 + lane;
    if (idx < N) {
      k[i] = kin[idx];
      v[i] = vin[idx];
    } else {
      k[i] = ~0ull;
      v[i] = 0;
    }
  }
  // ---- stable rank within the warp: (item, lane) order == input order
  unsigned* wh = whist + warp * 256;
#pragma unroll
  for (int i = 0; i < kRsItems; ++i) {
    const long long idx = wbase + i * 32 + lane;
    const int d = idx < N ? (int)((k[i] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(FULL, d);
    const int leader = __ffs(peers) - 1;
    const unsigned before = __popc(peers & lanemask_lt());
    unsigned old = 0;
    if (lane == leader && d < 256) {
      old = wh[d];
      wh[d] = old + __popc(peers);
    }
    old = __shfl_sync(FULL, old, leader);
    rank[i] = (unsigned short)(old + before);
    __syncwarp();
  }
  __syncthreads();

  // ---- per digit (thread d): exclusive prefix over warps, tile total
  const int d = tid;
  unsigned tcount = 0;
#pragma unroll
  for (int w2 = 0; w2 < kRsWarps; ++w2) {
    unsigned c = whist[w2 * 256 + d];
    whist[w2 * 256 + d] = tcount;
    tcount += c;
  }
  // ---- decoupled look-back across tiles for digit d
  volatile u64* lb = reinterpret_cast<volatile u64*>(lookback);
  u64 excl = 0;
  if (tile == 0) {
    lb[d] = kFlagInc | (u64)tcount;
  } else {
    lb[(long long)tile * 256 + d] = kFlagAgg | (u64)tcount;
    long long t = tile - 1;
    long long spins = 0;
    while (t >= 0) {
      u64 x = lb[t * 256 + d];
      u64 fl = x & ~kCountMask;
      if (fl == 0) {
        if (++spins > spin_limit) {
          s_fail = 1;
          atomicOr(err, ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
        continue;
      }
      excl += x & kCountMask;
      if (fl == kFlagInc) break;
      --t;
    }
    lb[(long long)tile * 256 + d] = kFlagInc | ((excl + tcount) & kCountMask);
  }
  s_gbase[d] = (unsigned long long)goff[d] + excl;
  const unsigned tstart = block_exclusive_256(tcount, s_warp_tot);
  s_tile_start[d] = tstart;
  __syncthreads();

  // ---- scatter into shared memory in digit order
#pragma unroll
  for (int i = 0; i < kRsItems; ++i) {
    const long long idx = wbase + i * 32 + lane;
    if (idx < N) {
      const int dd = (int)((k[i] >> shift) & 255);
      const unsigned pos = s_tile_start[dd] + wh[dd] + rank[i];
      skeys[pos] = k[i];
      svals[pos] = v[i];
    }
  }
  __syncthreads();
  // ---- coalesced write-out
  const int valid = (int)min((long long)kRsTile, (long long)N - tile_base);
  const bool fail = s_fail != 0;
  for (int j = tid; j < valid; j += kRsThreads) {
    const u64 kk = skeys[j];
    const int dd = (int)((kk >> shift) & 255);
    const unsigned long long o = s_gbase[dd] + (unsigned long long)(j - (int)s_tile_start[dd]);
    if (!fail && o < (unsigned long long)N) {
      kout[o] = kk;
      vout[o] = svals[j];
    }
  }
}

// ------------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kScanFold = 2048;  // blocks that sum the partials before them themselves

__device__ __forceinline__ int block_exclusive_int(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  int add = 0, tot = 0;
  for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
    if (w2 < warp) add += warp_tot[w2];
    tot += warp_tot[w2];
  }
  *total = tot;
  return x - v + add;
}

// Thread t of block b owns the kScanItems consecutive values from
// b * kScanTile + t * kScanItems (whole 16-byte vectors when they can be).
__device__ __forceinline__ void scan_load_run(const int* __restrict__ in, long long i0, int N,
                                              int (&v)[kScanItems]) {
  if (i0 + kScanItems <= N && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
    const int4* p = reinterpret_cast<const int4*>(in + i0);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
      const int4 a = p[q];
      v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = i0 + k < N ? in[i0 + k] : 0;
  }
}

__device__ __forceinline__ int block_sum_int(int v, int* warp_tot) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = 0;
  for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += warp_tot[w2];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_kernel(const int* __restrict__ in, int N, int* __restrict__ part) {
  __shared__ int s_w[kScanThreads / 32];
  int v[kScanItems];
  scan_load_run(in, (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems, N, v);
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += v[k];
  s = block_sum_int(s, s_w);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Single block: exclusive scan of part[0..nb) in place; *total = sum.
__global__ void scan_partials_kernel(int* part, int nb, int* total) {
  __shared__ int s_w[32];
  __shared__ int s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? part[i] : 0;
    int tot;
    int ex = block_exclusive_int(v, s_w, &tot);
    int carry = s_carry;
    if (i < nb) part[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = s_carry;
}

// Down-sweep.  fold = 0: part[b] is block b's exclusive prefix.  fold = 1:
// part[b] is block b's sum, and each block adds up those of the blocks
// before it (a few thousand at most), the last block writing *total.
__global__ void __launch_bounds__(kScanThreads)
    scan_down_kernel(const int* __restrict__ in, int* __restrict__ out, int N,
                     const int* __restrict__ part, int fold, int* __restrict__ total) {
  __shared__ int s_w[kScanThreads / 32];
  const long long i0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  scan_load_run(in, i0, N, v);
  int pre;
  if (fold) {
    int p = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) p += part[i];
    pre = block_sum_int(p, s_w);
  } else {
    pre = part[blockIdx.x];
  }
  int run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) run += v[k];
  int tot;
  int ex = pre + block_exclusive_int(run, s_w, &tot);
  if (i0 + kScanItems <= N && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    int4* q = reinterpret_cast<int4*>(out + i0);
#pragma unroll
    for (int r = 0; r < kScanItems / 4; ++r) {
      int4 a;
      a.x = ex; ex += v[4 * r];
      a.y = ex; ex += v[4 * r + 1];
      a.z = ex; ex += v[4 * r + 2];
      a.w = ex; ex += v[4 * r + 3];
      q[r] = a;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (i0 + k < N) out[i0 + k] = ex;
      ex += v[k];
    }
  }
  if (fold && total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = pre + tot;
}

}  // namespace

long long sort_lookback_words(long long maxN) {
  return ((maxN + kRsTile - 1) / kRsTile + 1) * 256;
}

template <typename WT>
cudaError_t radix_sort_pairs(u64* k0, WT* v0, u64* k1, WT* v1, int N, int bits, SortScratch sc, DevState* st, long long spin_limit,
                             cudaStream_t s, bool* in_alt, int* launches) {
  *in_alt = false;
  if (N <= 1 || bits <= 0) return cudaSuccess;
  const long long maxN = N;
  if (sort_lookback_words(maxN) > sc.lookback_words) return cudaErrorInvalidValue;
  const int passes = (bits + 7) / 8;
  if (passes > 8) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kRsTile * (sizeof(u64) + sizeof(WT)) + kRsWarps * 256 * sizeof(unsigned);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(rs_pass_kernel<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  cudaMemsetAsync(sc.hist, 0, 8 * 256 * sizeof(unsigned), s);
  cudaMemsetAsync(st->tile_counter, 0, sizeof(st->tile_counter), s);
  int dev = 0, sms = kDefaultSms;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int hgrid = (int)std::min<long long>((maxN + 4095) / 4096, (long long)sms * 4);
  {
    ProfScope ps(P_SORT_HIST, N, s);
    rs_hist_kernel<<<std::max(hgrid, 1), 512, 0, s>>>(k0, N, passes, sc.hist);
    rs_scan_hist_kernel<<<passes, 256, 0, s>>>(sc.hist, sc.goff);
  }
  *launches += 2;
  const int tiles = (int)((maxN + kRsTile - 1) / kRsTile);
  u64 *ki = k0, *ko = k1;
  WT *vi = v0, *vo = v1;
  for (int p = 0; p < passes; ++p) {
    cudaMemsetAsync(sc.lookback, 0, (size_t)tiles * 256 * sizeof(u64), s);
    ProfScope ps(P_SORT_PASS, N, s);
    rs_pass_kernel<WT><<<tiles, kRsThreads, smem, s>>>(
        ki, vi, ko, vo, N, 8 * p, sc.goff + p * 256, sc.lookback,
        reinterpret_cast<unsigned long long*>(&st->tile_counter[p]), &st->error, spin_limit);
    ++*launches;
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  *in_alt = (passes & 1) != 0;
  return cudaGetLastError();
}

template cudaError_t radix_sort_pairs<int32_t>(u64*, int32_t*, u64*, int32_t*, int, int,
                                               SortScratch, DevState*, long long, cudaStream_t,
                                               bool*, int*);
template cudaError_t radix_sort_pairs<int64_t>(u64*, int64_t*, u64*, int64_t*, int, int,
                                               SortScratch, DevState*, long long, cudaStream_t,
                                               bool*, int*);

cudaError_t scan_exclusive_i32(const int* in, int* out, int N, int* part, int* total,
                               cudaStream_t s, int* launches) {
  if (N <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(int), s);
    return cudaGetLastError();
  }
  const int nb = (N + kScanTile - 1) / kScanTile;
  if (nb == 1) {  // one block: no partials
    scan_down_kernel<<<1, kScanThreads, 0, s>>>(in, out, N, part, 1, total);
    ++*launches;
    return cudaGetLastError();
  }
  scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(in, N, part);
  // up to kScanFold blocks add up the sums before them themselves
  const bool fold = nb <= kScanFold;
  if (!fold) scan_partials_kernel<<<1, 1024, 0, s>>>(part, nb, total);
  scan_down_kernel<<<nb, kScanThreads, 0, s>>>(in, out, N, part, fold ? 1 : 0, total);
  *launches += fold ? 2 : 3;
  return cudaGetLastError();
}

}  // namespace mc
