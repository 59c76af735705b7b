// common.cuh -- shared device definitions of the GB300 minimum-cut library.
//
// Weight/sum type WT: every kernel that touches edge weights is instantiated
// for int32_t and int64_t.  A graph whose total edge weight W is < 2^31 runs
// with WT = int32_t: every degree, r-value, cut value and contracted weight is
// at most W, so 32-bit arithmetic is exact.  Larger graphs run with int64_t.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWarp = 32;
// SM count assumed when the device cannot be asked (GB300: two dies of 76)
constexpr int kDefaultSms = 152;
constexpr long long kInf = 0x7fffffffffffffffll;

// Error bits written by kernels into DevState::error.
enum : unsigned {
  ERR_INPUT = 1u,      // index out of range or negative weight
  ERR_ASYM = 2u,       // input CSR is not symmetric
  ERR_TIMEOUT = 4u,    // a bounded wait ran out
  ERR_INTERNAL = 8u,   // a consistency check failed
  ERR_OVERFLOW = 16u,  // a size exceeded a kernel's capacity
};

// Small device-resident state shared by the kernels of a round.  The host
// reads it with one copy per synchronisation point.
struct DevState {
  unsigned long long lambda;   // current upper bound (kInf: none)
  unsigned long long marks_pr; // edges hooked by the PR tests this round
  unsigned long long marks_cf; // edges hooked by CAPFOREST this round
  unsigned int error;          // ERR_* bits
  int n_next;                  // vertices after union-find relabel
  long long emit_count;        // entries emitted by the contraction
  long long m_next;            // entries of the contracted graph
  // bound candidates of this round with the data that names their cut
  unsigned long long deg_val;  // minimum degree and its vertex
  int deg_arg;
  int lp_label;                // label of the LP cluster attaining lp_val
  unsigned long long lp_val;
  unsigned long long cf_val;   // best CAPFOREST alpha, pass id and prefix length
  int cf_pass;
  int cf_len;
  long long cf_nscanned;       // vertices scanned by the sequential pass
  long long cf_nmarks;         // marks of the sequential pass
  long long claimed;           // vertices claimed by concurrent passes this wave
  long long tile_counter[8];   // per-pass tile counters of the radix sort
  int lambda_src;              // 1 degree, 2 LP, 3 CAPFOREST (set by the witness step)
  int batch_done;              // graphs of a batch that finished
  long long sym_balance;       // symmetry check: entries u < v minus entries u > v
  unsigned long long single_entries;  // contraction: entries of single-vertex groups' rows
  unsigned long long dense_entries;   // contraction: entries of dense groups' rows
  int ndense;                         // contraction: dense groups asked for this round
  int m_rows;                         // contraction: entries of the row-wise contracted graph
  int internal_code;                  // which internal check failed (0: none), for the message
  unsigned long long wsum;            // input check: sum of the directed entries' weights
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(FULL, v, o);
    v = x > v ? x : v;
  }
  return v;
}

// 32-bit unsigned maximum in one warp reduction instruction.
template <>
__device__ __forceinline__ unsigned warp_max<unsigned>(unsigned v) {
  return __reduce_max_sync(FULL, v);
}

template <>
__device__ __forceinline__ int warp_max<int>(int v) {
  return __reduce_max_sync(FULL, v);
}

__device__ __forceinline__ void set_error(DevState* st, unsigned bits) {
  atomicOr(&st->error, bits);
}

// Largest i in [lo, hi) with a[i] <= x (a non-decreasing, a[lo] <= x).
__device__ __forceinline__ int row_of(const int64_t* __restrict__ a, int lo, int hi,
                                      long long x) {
  while (hi - lo > 1) {
    int mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- union-find
// parent[v] <= v always, so a root is its component's smallest vertex.  All
// accesses go through volatile pointers (L2-coherent across SMs).  find()
// halves paths; concurrent halving writes are benign because every write
// stores an ancestor of the written vertex, and only roots are ever CAS'ed.
__device__ __forceinline__ int uf_find(volatile int* parent, int x) {
  while (true) {
    int p = parent[x];
    if (p == x) return x;
    int gp = parent[p];
    if (gp == p) return p;
    parent[x] = gp;
    x = gp;
  }
}

// Hook the components of a and b: the larger root goes under the smaller one
// by a CAS on the larger root's entry.  Returns false only if the retry
// bound ran out (never observed; callers report it as an internal error).
__device__ __forceinline__ bool uf_union(int* parent, int a, int b) {
  volatile int* vp = parent;
  for (int it = 0; it < (1 << 24); ++it) {
    a = uf_find(vp, a);
    b = uf_find(vp, b);
    if (a == b) return true;
    if (a > b) { int t = a; a = b; b = t; }
    if (atomicCAS(&parent[b], b, a) == b) return true;
  }
  return false;
}

// 64-bit atomic min / max on non-negative values stored as unsigned.
__device__ __forceinline__ unsigned long long atomic_min_u64(unsigned long long* p,
                                                             unsigned long long v) {
  return atomicMin(p, v);
}

template <typename WT> struct WTraits;
template <> struct WTraits<int32_t> {
  using U = unsigned int;
  static constexpr long long kMax = 0x7fffffffll;
};
template <> struct WTraits<int64_t> {
  using U = unsigned long long;
  static constexpr long long kMax = kInf;
};

__device__ __forceinline__ int atomic_add_w(int* p, int v) { return atomicAdd(p, v); }
__device__ __forceinline__ long long atomic_add_w(long long* p, long long v) {
  return (long long)atomicAdd((unsigned long long*)p, (unsigned long long)v);
}
__device__ __forceinline__ int64_t atomic_add_w(int64_t* p, int64_t v) {
  return (int64_t)atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace mc
