// noalloc.cu -- contraction of a small device CSR that allocates no memory.
//
// Some callers cannot allocate device memory: a plug-in running inside a
// host application that owns the whole device pool and forbids other
// allocations, or a latency-critical loop where cudaMalloc's implicit
// synchronisation and latency are not acceptable.  For them this file offers
// mincut_contract_csr_noalloc(): the caller passes the input CSR, the labels
// and the output buffers; every intermediate buffer (sort keys and values,
// radix histograms and look-back words, scan partials, the device status
// block) lives in one file-scope __device__ array of fixed size, which every
// GPU that loads the library keeps until the process exits.
//
// The host cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it.  Every call shares the one array:
// calls whose work overlaps on the GPU (two streams, two threads) race and
// must be serialised by the caller.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/mincut.h"
#include "common.cuh"
#include "kernels.h"

using namespace mc;

namespace {

constexpr long long kNaMaxEntries = 1ll << 18;   // directed CSR entries
constexpr long long kNaMaxVertices = 1ll << 18;  // vertices

constexpr size_t a256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = kOffKeys0 + a256(kNaMaxEntries * 8);
constexpr size_t kOffVals0 = kOffKeys1 + a256(kNaMaxEntries * 8);
constexpr size_t kOffVals1 = kOffVals0 + a256(kNaMaxEntries * 4);
constexpr size_t kOffUid = kOffVals1 + a256(kNaMaxEntries * 4);
constexpr size_t kTiles = kNaMaxEntries / kEntryTile + 2;
constexpr size_t kOffTiles = kOffUid + a256(kNaMaxEntries * 4);
constexpr size_t kParts = (kNaMaxEntries > kNaMaxVertices ? kNaMaxEntries : kNaMaxVertices) / 4096 + 2;
constexpr size_t kOffPart = kOffTiles + a256(kTiles * 4);
constexpr size_t kLookWords = (kNaMaxEntries / kSortTile + 2) * 256;
constexpr size_t kOffLook = kOffPart + a256(kParts * 4);
constexpr size_t kOffHist = kOffLook + a256(kLookWords * 8);
constexpr size_t kOffGoff = kOffHist + a256(8 * 256 * 4);
constexpr size_t kOffState = kOffGoff + a256(8 * 256 * 4);
constexpr size_t kOffM2 = kOffState + a256(sizeof(DevState));
constexpr size_t kScratchBytes = kOffM2 + 256;  // about 7.2 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_ptr[128] = {};

int na_fail(int status, const char* msg) {
  set_last_error(msg);
  return status;
}

// One pass over the caller's arrays before anything else reads them: row
// offsets non-decreasing, labels in [0, n2), columns in [0, n), weights >= 0
// (ERR_INPUT otherwise), and the sum of the weights into st->wsum.
__global__ void input_check_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ w, const int32_t* __restrict__ lab,
                                   int n, long long M, int n2, DevState* st) {
  unsigned long long sum = 0;
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long v = first; v < n; v += stride) {
    const int l = lab[v];
    if (l < 0 || l >= n2 || rp[v] > rp[v + 1]) bad = true;
  }
  for (long long e = first; e < M; e += stride) {
    const int c = col[e];
    const int x = w[e];
    if (c < 0 || c >= n || x < 0) bad = true;
    else sum += (unsigned long long)x;
  }
  sum = warp_sum(sum);
  if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&st->wsum, sum);
  if (bad) set_error(st, ERR_INPUT);
}

int bits_for_na(long long x) {
  int b = 1;
  while (b < 62 && (1ll << b) < x) ++b;
  return b;
}

}  // namespace

extern "C" {

int mincut_contract_csr_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                const int32_t* w, int64_t m_directed, const int32_t* labels,
                                int64_t n2, int64_t* row_ptr_out, int32_t* col_out,
                                int32_t* w_out, int64_t* m_out, void* cuda_stream) {
  set_last_error("");
  if (!row_ptr || !labels || !row_ptr_out || !m_out || (m_directed > 0 && (!col || !w)) ||
      (m_directed > 0 && (!col_out || !w_out)))
    return na_fail(MINCUT_ERR_INVALID, "NULL pointer argument");
  if (n < 1 || n2 < 1 || n2 > n || m_directed < 0)
    return na_fail(MINCUT_ERR_INVALID, "need 1 <= n2 <= n and m_directed >= 0");
  if (n > kNaMaxVertices || m_directed > kNaMaxEntries)
    return na_fail(MINCUT_ERR_OVERFLOW,
                   "graph exceeds the fixed scratch: at most 262144 vertices and 262144 "
                   "directed entries");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
    return na_fail(MINCUT_ERR_CUDA, "cudaGetDevice failed");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return na_fail(MINCUT_ERR_CUDA, "cudaGetSymbolAddress failed");
      g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch_ptr[dev];
  }
  u64* keys0 = reinterpret_cast<u64*>(base + kOffKeys0);
  u64* keys1 = reinterpret_cast<u64*>(base + kOffKeys1);
  int32_t* vals0 = reinterpret_cast<int32_t*>(base + kOffVals0);
  int32_t* vals1 = reinterpret_cast<int32_t*>(base + kOffVals1);
  int* uid = reinterpret_cast<int*>(base + kOffUid);
  int* tiles = reinterpret_cast<int*>(base + kOffTiles);
  int* part = reinterpret_cast<int*>(base + kOffPart);
  SortScratch sc;
  sc.lookback = reinterpret_cast<u64*>(base + kOffLook);
  sc.hist = reinterpret_cast<unsigned*>(base + kOffHist);
  sc.goff = reinterpret_cast<unsigned*>(base + kOffGoff);
  sc.lookback_words = (long long)kLookWords;
  DevState* st = reinterpret_cast<DevState*>(base + kOffState);
  int* m2_dev = reinterpret_cast<int*>(base + kOffM2);
  int launches = 0;
  const int ni = (int)n, n2i = (int)n2;
  const int vbits = bits_for_na(n2);

  // the row offsets' ends first (host reads): rp[0] = 0 and rp[n] = M
  int64_t ends[2] = {-1, -1};
  if (cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "reading row_ptr failed");
  if (ends[0] != 0 || ends[1] != m_directed)
    return na_fail(MINCUT_ERR_INVALID, "need row_ptr[0] = 0 and row_ptr[n] = m_directed");
  // the status block keeps the previous call's contents: clear it, then
  // check the whole input before any kernel relies on it
  if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "cudaMemsetAsync failed");
  {
    const long long work = std::max<long long>(n, m_directed);
    const int blocks = (int)std::min<long long>((work + 255) / 256, 1024);
    input_check_kernel<<<blocks, 256, 0, s>>>(row_ptr, col, w, labels, ni, m_directed, n2i, st);
  }
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "input check failed");
  if (h.error & ERR_INPUT)
    return na_fail(MINCUT_ERR_INVALID,
                   "row_ptr decreasing, or column index, weight or label out of range");
  if (h.wsum > 0x7fffffffull)
    return na_fail(MINCUT_ERR_OVERFLOW,
                   "total weight of the directed entries exceeds 2^31 - 1 (32-bit sums)");
  if (tile_rows(row_ptr, ni, m_directed, tiles, s, &launches) != cudaSuccess ||
      emit_pairs<int32_t>(ni, m_directed, row_ptr, col, w, labels, vbits, tiles, keys0, vals0,
                          st, 1, s, &launches) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "launch failed (relabel)");
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "relabel failed");
  if (h.error & ERR_INPUT)
    return na_fail(MINCUT_ERR_INVALID, "column index, weight or label out of range");
  const long long N = h.emit_count;
  bool alt = false;
  if (radix_sort_pairs<int32_t>(keys0, vals0, keys1, vals1, (int)N, 2 * vbits, sc, st,
                                1ll << 22, s, &alt, &launches) != cudaSuccess ||
      build_csr<int32_t>(alt ? keys1 : keys0, alt ? vals1 : vals0, (int)N, vbits, n2i, uid, part,
                         row_ptr_out, col_out, w_out, st, m2_dev,
                         reinterpret_cast<int*>(alt ? keys0 : keys1), s, &launches) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "launch failed (sort/build)");
  int m2 = 0;
  if (cudaMemcpyAsync(&m2, m2_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(MINCUT_ERR_CUDA, "sort/build failed");
  if (h.error & ERR_TIMEOUT) return na_fail(MINCUT_ERR_DEVICE_TIMEOUT, "a bounded wait ran out");
  if (h.error) return na_fail(MINCUT_ERR_INTERNAL, "device check failed");
  *m_out = m2;
  return MINCUT_OK;
}

}  // extern "C"
