// round.cu -- the bandwidth-bound kernels of one contraction round.
//
//   degrees_min   trivial-cut / collapsed-vertex bound (Sec. 2, Sec. 2.1)
//   lp_sweep      label propagation sweeps (Sec. 2.1, "Lowering the upper bound")
//   lp_bound      cluster cut values of the LP labelling
//   pr_marks      Padberg-Rinaldi tests PR1-PR4 (Sec. 2.1, App. A)
//   uf_*          union-find over marked edges and canonical relabel (Alg. 1 "U")
//   emit_pairs    relabel endpoints and drop self-loops (contraction, Sec. 2)
//   build_csr     sum parallel edges after the sort and rebuild the CSR
//   side_*        materialise the side of the best cut over the input vertices
//
// Entry-parallel kernels work on tiles of kEntryTile consecutive CSR entries;
// tile_rows() records the row of each tile's first entry so a block finds the
// rows of its entries with a binary search in shared memory.  Strided tiles
// (thread t takes entries t, t + 256, ...) keep a warp's atomics on
// neighbouring addresses; the per-row reductions (degrees, the first LP
// sweep, the cluster cut) take runs of 8 consecutive entries per thread
// instead, searching a run's first row once and walking forward.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "tiles.cuh"

namespace mc {

namespace {

// Warp-level segmented maximum of packed 64-bit values (same layout rules).
__device__ __forceinline__ void warp_segment_max(int seg, unsigned long long val, bool valid,
                                                 unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long x = valid ? val : 0ull;
  const int r = valid ? seg : -1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, x, o);
    const int ry = __shfl_up_sync(FULL, r, o);
    if (lane >= o && ry == r && y > x) x = y;
  }
  const int rn = __shfl_down_sync(FULL, r, 1);
  const bool last = lane == 31 || rn != r;
  if (valid && last && x) atomicMax(&out[seg], x);
}

__global__ void tile_rows_kernel(const int64_t* __restrict__ rp, int n, int* __restrict__ tile_row) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    long long b = rp[u], e = rp[u + 1];
    if (e <= b) continue;
    long long t0 = (b + kET - 1) / kET, t1 = (e + kET - 1) / kET;
    for (long long t = t0; t < t1; ++t) tile_row[t] = u;
  }
}

// ------------------------------------------------------------ degrees / bound
struct ValArg {
  unsigned long long v;
  int a;
};
__device__ __forceinline__ ValArg va_min(ValArg x, ValArg y) {
  return (y.v < x.v || (y.v == x.v && y.a < x.a)) ? y : x;
}
__device__ __forceinline__ ValArg warp_va_min(ValArg x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ValArg y;
    y.v = __shfl_xor_sync(FULL, x.v, o);
    y.a = __shfl_xor_sync(FULL, x.a, o);
    x = va_min(x, y);
  }
  return x;
}
// Block-wide (value, arg) minimum; result valid in thread 0.
__device__ __forceinline__ ValArg block_va_min(ValArg x) {
  __shared__ unsigned long long sv[32];
  __shared__ int sa[32];
  x = warp_va_min(x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sv[warp] = x.v; sa[warp] = x.a; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    ValArg y{~0ull, 0x7fffffff};
    if (lane < nw) { y.v = sv[lane]; y.a = sa[lane]; }
    x = warp_va_min(y);
  }
  __syncthreads();
  return x;
}

// Per-block (min, argmin) of the degrees deg[0..n) (computed with the CSR).
template <typename WT>
__global__ void degmin_kernel(const WT* __restrict__ deg, int n, unsigned long long* __restrict__ blk) {
  ValArg best{~0ull, 0x7fffffff};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    best = va_min(best, ValArg{(unsigned long long)(long long)deg[v], v});
  ValArg r = block_va_min(best);
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = r.v;
    blk[2 * blockIdx.x + 1] = (unsigned long long)(unsigned)r.a;
  }
}

__global__ void degmin_final_kernel(const unsigned long long* __restrict__ blk, int nb,
                                    DevState* st) {
  ValArg best{~0ull, 0x7fffffff};
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    best = va_min(best, ValArg{blk[2 * i], (int)blk[2 * i + 1]});
  ValArg r = block_va_min(best);
  if (threadIdx.x == 0) {
    st->deg_val = r.v;
    st->deg_arg = r.a;
    atomicMin(&st->lambda, r.v);
  }
}

// ---------------------------------------------------------------- emit
// Relabel every entry (u, v, w) to the key (L[u] << vbits) | L[v]; drop
// self-loops (L[u] == L[v]) and zero weights.  With `validate`, also flag
// out-of-range indices and negative weights (input canonicalisation).
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    emit_kernel(int n, long long M, const int64_t* __restrict__ rp, const int* __restrict__ col,
                const WT* __restrict__ w, const int* __restrict__ L, int vbits,
                const int* __restrict__ tile_row, int ntiles, u64* __restrict__ keys,
                WT* __restrict__ vals, DevState* st, int validate,
                const int* __restrict__ keep_row) {
  __shared__ TileRowsSmem tr;
  __shared__ int s_cnt[kETItems][kETThreads / 32];
  __shared__ long long s_base;
  const int t = blockIdx.x;
  tile_rows_load(tr, rp, n, tile_row, ntiles, t);
  if (keep_row) {
    // a tile whose rows are all filtered out reads none of its entries
    bool any = false;
    for (int r = tr.r0 + threadIdx.x; r <= tr.r1 && !any; r += blockDim.x)
      any = keep_row[L ? L[r] : r] == 1;
    if (!__syncthreads_or(any)) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long e0 = (long long)t * kET;
  u64 key[kETItems];
  WT val[kETItems];
  unsigned ball[kETItems];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    bool keep = false;
    if (e < M) {
      const int u = tile_row_of(tr, rp, e);
      const int lu = L ? L[u] : u;
      if (keep_row && keep_row[lu] != 1) {
        // row not emitted: its entries are not read
      } else {
        const int v = col[e];
        const WT c = w[e];
        if (validate && (v < 0 || v >= n || c < 0)) {
          bad = true;
        } else {
          const int lv = L ? L[v] : v;
          keep = (lu != lv) && (c != 0);
          key[i] = ((u64)(unsigned)lu << vbits) | (u64)(unsigned)lv;
          val[i] = c;
        }
      }
    }
    ball[i] = __ballot_sync(FULL, keep);
    if (lane == 0) s_cnt[i][warp] = __popc(ball[i]);
  }
  if (bad) set_error(st, ERR_INPUT);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < kETItems; ++i)
      for (int w2 = 0; w2 < kETThreads / 32; ++w2) {
        int c = s_cnt[i][w2];
        s_cnt[i][w2] = s;
        s += c;
      }
    s_base = s ? (long long)atomicAdd((unsigned long long*)&st->emit_count, (unsigned long long)s) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    if ((ball[i] >> lane) & 1u) {
      const long long o = s_base + s_cnt[i][warp] + __popc(ball[i] & lanemask_lt());
      keys[o] = key[i];
      vals[o] = val[i];
    }
  }
}

// ----------------------------------------------------------- build CSR
__global__ void head_flags_kernel(const u64* __restrict__ keys, int N, int* __restrict__ flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Each thread owns 8 consecutive sorted entries.  Runs of equal keys are
// summed locally; a run that crosses a chunk boundary is finished with
// atomics (w2 starts at zero), a run inside the chunk with a plain store.
// Heads also write col2 and the row pointers of their row and of any empty
// rows before it.
template <typename WT>
__global__ void segsum_kernel(const u64* __restrict__ keys, const WT* __restrict__ vals, int N,
                              const int* __restrict__ uid, int vbits, int* __restrict__ urow,
                              int* __restrict__ col2, WT* __restrict__ w2) {
  const u64 vmask = (vbits >= 64) ? ~0ull : ((1ull << vbits) - 1);
  const long long nchunks = ((long long)N + 7) / 8;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (long long)gridDim.x * blockDim.x) {
    const long long i0 = c * 8, i1 = min(i0 + 8, (long long)N);
    u64 prev = i0 > 0 ? keys[i0 - 1] : ~0ull;
    long long acc = 0;
    bool run_started_here = false;
    int cur_uid = -1;
    for (long long i = i0; i < i1; ++i) {
      const u64 k = keys[i];
      const bool head = (i == 0) || (k != prev);
      if (head) {
        if (cur_uid >= 0) {
          if (run_started_here) w2[cur_uid] = (WT)acc;
          else atomic_add_w(&w2[cur_uid], (WT)acc);
        }
        cur_uid = uid[i];
        acc = 0;
        run_started_here = true;
        col2[cur_uid] = (int)(k & vmask);
        urow[cur_uid] = (int)(k >> vbits);
      } else if (cur_uid < 0) {
        // run continues from the previous chunk; uid is an exclusive scan of
        // head flags, so a non-head entry of run k holds k + 1
        cur_uid = uid[i] - 1;
        run_started_here = false;
      }
      acc += (long long)vals[i];
      prev = k;
    }
    if (cur_uid >= 0) {
      const bool run_ends_here = (i1 == N) || (keys[i1] != prev);
      if (run_started_here && run_ends_here) w2[cur_uid] = (WT)acc;
      else atomic_add_w(&w2[cur_uid], (WT)acc);
    }
  }
}

// rp2[r] = first unique entry whose row is >= r (rows of the unique entries
// ascend); rp2[n2] = m2.
__global__ void rp_search_kernel(const int* __restrict__ urow, const int* __restrict__ m2p, int n2,
                                 int64_t* __restrict__ rp2) {
  const int m2 = *m2p;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= n2; r += gridDim.x * blockDim.x) {
    int lo = 0, hi = m2;
    while (lo < hi) {
      const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
      if (urow[mid] < r) lo = mid + 1; else hi = mid;
    }
    rp2[r] = lo;
  }
}

// deg[u] = sum of w over row u.  Run layout: each thread sums its 8
// consecutive entries per row; rows wholly inside a run are written by it,
// the first and last rows of the runs are combined across the warp.
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    degree_kernel(int n, long long M, const int64_t* __restrict__ rp, const WT* __restrict__ w,
                  const int* __restrict__ tile_row, int ntiles, WT* __restrict__ deg) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  const long long eb = (long long)blockIdx.x * kET + (long long)threadIdx.x * kETItems;
  const int cnt = (int)max(0ll, min((long long)kETItems, M - eb));
  WT x[kETItems];
  if (cnt == kETItems && (reinterpret_cast<uintptr_t>(w) & 15) == 0) {
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
    for (int k = 0; k < kETItems; ++k) x[k] = k < cnt ? w[eb + k] : WT(0);
  }
  int first = 0, cur = 0;
  long long first_acc = 0, acc = 0;
  if (cnt > 0) {
    first = cur = tile_row_of(tr, rp, eb);
    long long rend = tile_rp(tr, rp, cur + 1);
#pragma unroll
    for (int k = 0; k < kETItems; ++k) {
      if (k < cnt) {
        while (eb + k >= rend) {  // leave row cur (empty rows keep deg 0)
          if (cur == first) first_acc = acc;
          else deg[cur] = (WT)acc;  // the whole row lies in this run
          acc = 0;
          ++cur;
          rend = tile_rp(tr, rp, cur + 1);
        }
        acc += (long long)x[k];
      }
    }
    if (cur == first) {
      first_acc = acc;
      acc = 0;
    }
  }
  warp_segment_add<long long, WT>(first, first, first_acc, cnt > 0, deg);
  // (the last rows of the lanes whose run spans several rows are distinct)
  warp_segment_add<long long, WT>(cur, cur, acc, cnt > 0 && cur != first, deg);
}

__global__ void rp_fill_kernel(int64_t* rp2, int n2) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= n2; r += gridDim.x * blockDim.x)
    rp2[r] = 0;
}

// Symmetry of a canonical graph (rows strictly increasing): every entry
// (u, v, W) with u < v has its mirror (v, u, W) (binary search in the sorted
// row v), and there are as many entries with u < v as with u > v.  The
// mirrors found are distinct, so together the two facts give a one-to-one
// pairing of all entries.  Each block adds its (u < v) - (u > v) count to
// st->sym_balance; sym_final_kernel flags a non-zero balance.
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    symmetric_kernel(int n, long long M, const int64_t* __restrict__ rp,
                     const int* __restrict__ col, const WT* __restrict__ w,
                     const int* __restrict__ tile_row, int ntiles, DevState* st) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  const long long e0 = (long long)blockIdx.x * kET;
  bool bad = false;
  int balance = 0;
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    if (e >= M) break;
    const int u = tile_row_of(tr, rp, e);
    const int v = col[e];
    if (u > v) {
      --balance;
      continue;
    }
    ++balance;
    long long lo = rp[v], hi = rp[v + 1];
    while (lo < hi) {
      long long mid = (lo + hi) >> 1;
      if (col[mid] < u) lo = mid + 1; else hi = mid;
    }
    if (lo >= rp[v + 1] || col[lo] != u || w[lo] != w[e]) bad = true;
  }
  if (bad) set_error(st, ERR_ASYM);
  balance = __reduce_add_sync(FULL, balance);
  if ((threadIdx.x & 31) == 0 && balance)
    atomicAdd((unsigned long long*)&st->sym_balance, (unsigned long long)(long long)balance);
}

__global__ void sym_final_kernel(DevState* st) {
  if (st->sym_balance != 0) set_error(st, ERR_ASYM);
}

// ------------------------------------------------------------------ PR tests
// PR1-PR4 on every canonical edge {u, v} (u < v), with the bound lambda read
// at kernel start and c(.) the weighted degrees:
//   PR1 c(u,v) >= lambda; PR2 c(u) < 2c(u,v) or c(v) < 2c(u,v);
//   PR3 a common neighbour x with c(u) < 2(c(u,v)+c(u,x)) and
//       c(v) < 2(c(u,v)+c(v,x)); PR4 c(u,v) + sum_x min(c(u,x), c(v,x)) >= lambda.
// PR3/PR4 only when min(|N(u)|, |N(v)|) <= budget (budget < 0: always); the
// shorter row is walked and each neighbour binary-searched in the longer one.
// A passing edge is hooked in the union-find.  With flags_out every directed
// entry gets its flag byte (both directions evaluated).
//
// Two phases per tile.  Phase 1 (one thread per entry) applies PR1/PR2 and
// the budget and queues the entries that need the PR3/PR4 intersection in
// shared memory; phase 2 spreads the queued intersections over all threads
// of the block, g lanes per entry with g the largest power of two that still
// gives every entry its own lane group, so that a few long intersections in a
// tile do not leave the other lanes idle; each lane searches kPrIlp of the
// shorter row's entries at once, in lockstep over the longer row.
constexpr int kPrQueue = kET;
// a's entries a lane of a PR3/PR4 intersection searches at once
constexpr int kPrIlp = 4;

// bits[v / 32] bit v % 32: row v has at most `budget` entries (a 1-bit copy
// of the budget test that stays in L1 where the row offsets do not).
__global__ void short_rows_kernel(int n, const int64_t* __restrict__ rp, long long budget,
                                  unsigned* __restrict__ bits) {
  const int nw = (n + 31) >> 5;
  for (int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nw;
       wi += (gridDim.x * blockDim.x) >> 5) {
    const int v = (wi << 5) + (threadIdx.x & 31);
    const unsigned b = __ballot_sync(FULL, v < n && rp[v + 1] - rp[v] <= budget);
    if ((threadIdx.x & 31) == 0) bits[wi] = b;
  }
}

template <typename WT>
__global__ void __launch_bounds__(kETThreads, 4)
    pr_kernel(int n, long long M, const int64_t* __restrict__ rp, const int* __restrict__ col,
              const WT* __restrict__ w, const WT* __restrict__ deg,
              const int* __restrict__ tile_row, int ntiles, uint32_t mask, long long budget,
              int* parent, uint8_t* __restrict__ flags_out,
              const unsigned* __restrict__ short_bits, DevState* st, BatchView bv, int batch) {
  __shared__ TileRowsSmem tr;
  __shared__ int q_u[kPrQueue];
  __shared__ unsigned q_ef[kPrQueue];  // entry offset in the tile | PR1/PR2 flags << 16
  __shared__ int q_n;
  if (threadIdx.x == 0) q_n = 0;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  // entry offsets fit 32 bits: graphs hold fewer than 2^31 entries
  const bool exact = flags_out != nullptr;
  const long long lam_global = (long long)*(volatile unsigned long long*)&st->lambda;
  // every weighted degree is at least the round's minimum degree: PR2 needs
  // 2c(u,v) > it, so lighter edges skip the degree gathers
  const long long dmin = batch ? 0 : (long long)*(volatile unsigned long long*)&st->deg_val;
  const long long e0 = (long long)blockIdx.x * kET;
  unsigned long long nmarks = 0;
  bool uf_fail = false;
  // ---- phase 1: PR1/PR2, budget, queue
  int pv[kETItems];
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    pv[i] = e < M ? col[e] : 0;
  }
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    if (e >= M) break;
    const int u = tile_row_of(tr, rp, e);
    const int v = pv[i];
    if (u > v && !exact) continue;
    int gu = 0;
    if (batch) {
      gu = bv.gid[u];
      if (bv.done_g[gu]) continue;
    }
    const long long lam = batch ? (long long)*(volatile unsigned long long*)&bv.lam_g[gu] : lam_global;
    const long long c = (long long)w[e];
    uint8_t f = 0;
    if ((mask & 1u) && c >= lam) f |= 1;
    if ((mask & 2u) && 2 * c > dmin) {
      const long long du = (long long)deg[u], dv = (long long)deg[v];
      if (du < 2 * c || dv < 2 * c) f |= 2;
    }
    if ((mask & 12u) && (exact || f == 0)) {
      // u's row length from the tile's row offsets; v's budget test from
      // the bit map
      const long long lu = tile_rp(tr, rp, u + 1) - tile_rp(tr, rp, u);
      bool within = budget < 0 || lu <= budget;
      if (!within)
        within = short_bits ? ((__ldg(&short_bits[v >> 5]) >> (v & 31)) & 1u)
                            : rp[v + 1] - rp[v] <= budget;
      if (within) {
        const int slot = atomicAdd(&q_n, 1);
        q_u[slot] = u;
        q_ef[slot] = (unsigned)(e - e0) | ((unsigned)f << 16);
        continue;
      }
    }
    if (exact) flags_out[e] = f;
    if (f && u < v) {
      if (!uf_union(parent, u, v)) uf_fail = true;
      ++nmarks;
      if (batch) atomicAdd(&bv.marks_g[gu], 1);
    }
  }
  __syncthreads();
  // ---- phase 2: PR3/PR4 intersections, g lanes per queued entry
  const int nq = q_n;
  int g = 1;
  while (g < 32 && nq * (2 * g) <= kETThreads) g *= 2;
  const int lane = threadIdx.x & 31;
  const int r = lane & (g - 1);
  const unsigned gmask = g == 32 ? FULL : (((1u << g) - 1u) << (lane & ~(g - 1)));
  for (int q = threadIdx.x / g; q < nq; q += kETThreads / g) {
    const int u = q_u[q];
    const long long e = e0 + (q_ef[q] & 0xffffu);
    uint8_t f = (uint8_t)(q_ef[q] >> 16);
    const int v = col[e];
    int gu = 0;
    if (batch) gu = bv.gid[u];
    const long long lam = batch ? (long long)*(volatile unsigned long long*)&bv.lam_g[gu] : lam_global;
    const long long c = (long long)w[e];
    const long long du = (long long)deg[u], dv = (long long)deg[v];
    // Without a flags output an edge whose endpoints are already joined in
    // the union-find (by marks hooked so far) cannot change the contraction:
    // skip its intersection.
    bool joined = false;
    if (!exact && r == 0) joined = uf_find(parent, u) == uf_find(parent, v);
    joined = __shfl_sync(gmask, joined, 0, g);
    if (!joined) {
      const int bu = (int)rp[u], eu = (int)rp[u + 1], bv_ = (int)rp[v], ev = (int)rp[v + 1];
      const bool a_is_u = eu - bu <= ev - bv_;
      const int ab = a_is_u ? bu : bv_, ae = a_is_u ? eu : ev;
      const int bb = a_is_u ? bv_ : bu, be = a_is_u ? ev : eu;
      const long long da = a_is_u ? du : dv;
      long long sum = c;
      bool pr3 = false;
      // Without a flags output only "some test passes" matters, so the scan
      // stops once the answer is known: PR4 reached, PR3 found, or neither
      // still possible (rem = weight of a's unscanned edges bounds the PR4
      // sum still to come; PR3 needs a single edge heavier than da/2 - c).
      long long rem = da - c;
      // b's entries are ascending and a lane's neighbours too: once one is
      // past b's last entry the lane has nothing left to find
      const int bmax = be > bb ? col[be - 1] : INT_MIN;
      bool lane_done = false;
      // lane r of the group takes a's entries ab + r, ab + r + g, ..., kPrIlp
      // of them per step; their lower bounds in b's row are searched in
      // lockstep (over the same row every search takes the same number of
      // halvings), so a lane keeps kPrIlp loads in flight per halving
      // instead of walking its entries one dependent chain after another
      for (int base = ab; base < ae; base += g * kPrIlp) {
        int xs[kPrIlp], pos[kPrIlp];
        WT ca[kPrIlp];
        bool act[kPrIlp];
#pragma unroll
        for (int j = 0; j < kPrIlp; ++j) {
          const int ea = base + r + j * g;
          act[j] = ea < ae && !lane_done;
          xs[j] = act[j] ? col[ea] : INT_MAX;
          ca[j] = act[j] ? w[ea] : (WT)0;
        }
        long long add = 0, used = 0;
        bool p3 = false;
#pragma unroll
        for (int j = 0; j < kPrIlp; ++j) {
          if (xs[j] == u || xs[j] == v) act[j] = false;
          if (act[j]) used += (long long)ca[j];
          if (act[j] && xs[j] > bmax) {
            act[j] = false;
            lane_done = true;
          }
          pos[j] = bb;
        }
        // answer (first entry >= x) in [pos, pos + nn]; lanes whose x are
        // all inactive skip the loads but not the loop
        int nn = be - bb;
        while (nn > 1) {
          const int half = nn >> 1;
#pragma unroll
          for (int j = 0; j < kPrIlp; ++j)
            if (act[j] && col[pos[j] + half - 1] < xs[j]) pos[j] += half;
          nn -= half;
        }
        int hit[kPrIlp];
#pragma unroll
        for (int j = 0; j < kPrIlp; ++j) {
          hit[j] = -1;
          if (act[j]) {
            const int c0 = col[pos[j]];
            const int c1 = pos[j] + 1 < be ? col[pos[j] + 1] : INT_MAX;
            hit[j] = c0 == xs[j] ? pos[j] : c1 == xs[j] ? pos[j] + 1 : -1;
          }
        }
#pragma unroll
        for (int j = 0; j < kPrIlp; ++j) {
          if (hit[j] >= 0) {
            const long long cax = (long long)ca[j], cbx = (long long)w[hit[j]];
            const long long cux = a_is_u ? cax : cbx, cvx = a_is_u ? cbx : cax;
            add += cux < cvx ? cux : cvx;
            p3 = p3 || (du < 2 * (c + cux) && dv < 2 * (c + cvx));
          }
        }
        for (int o = g >> 1; o > 0; o >>= 1) {
          add += __shfl_xor_sync(gmask, add, o, g);
          used += __shfl_xor_sync(gmask, used, o, g);
          p3 |= __shfl_xor_sync(gmask, (int)p3, o, g) != 0;
        }
        sum += add;
        rem -= used;
        pr3 = pr3 || p3;
        if (!exact) {
          if (((mask & 8u) && sum >= lam) || ((mask & 4u) && pr3)) break;
          if (sum + rem < lam && !((mask & 4u) && 2 * (c + rem) > da)) break;
        }
        if (__all_sync(gmask, lane_done)) break;
      }
      if ((mask & 4u) && pr3) f |= 4;
      if ((mask & 8u) && sum >= lam) f |= 8;
    }
    if (r == 0) {
      if (exact) flags_out[e] = f;
      if (f && u < v) {
        if (!uf_union(parent, u, v)) uf_fail = true;
        ++nmarks;
        if (batch) atomicAdd(&bv.marks_g[gu], 1);
      }
    }
  }
  if (uf_fail) set_error(st, ERR_INTERNAL);
  nmarks = warp_sum(nmarks);
  if ((threadIdx.x & 31) == 0 && nmarks) atomicAdd(&st->marks_pr, nmarks);
}

// -------------------------------------------------------- label propagation
constexpr int kLpShort = 128;       // rows up to this length use a warp table
constexpr int kLpSlots = 256;       // slots of a warp table (power of two)
constexpr int kLpWarps = 8;
constexpr int kLpMidSmall = 1024;   // medium rows up to this length: small block tables
constexpr int kLpMedium = 4096;     // rows up to this length use a block table
constexpr int kLpMidSlots = 8192;

__device__ __forceinline__ unsigned lp_hash(int l) { return (unsigned)l * 0x9E3779B1u; }

struct LabScore {
  long long s;
  int l;
};
__device__ __forceinline__ LabScore ls_best(LabScore a, LabScore b) {
  return (b.s > a.s || (b.s == a.s && (unsigned)b.l < (unsigned)a.l)) ? b : a;
}
__device__ __forceinline__ LabScore warp_ls_best(LabScore x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    LabScore y;
    y.s = __shfl_xor_sync(FULL, x.s, o);
    y.l = __shfl_xor_sync(FULL, x.l, o);
    x = ls_best(x, y);
  }
  return x;
}

// One LP sweep for the vertices v with ((v ^ sweep) & 1) == 0: v adopts the
// neighbour label of largest total weight (ties: smaller label) if it beats
// the weight of v's own label; labels are read from lab_in only.  Rows longer
// than kLpShort are queued for lp_long_kernel.
template <typename WT>
__global__ void __launch_bounds__(kLpWarps * 32)
    lp_short_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                    const WT* __restrict__ w, const int* __restrict__ lab_in,
                    int* __restrict__ lab_out, int sweep, int* __restrict__ long_rows,
                    int* long_count, int* __restrict__ mid_rows, int* mid_count,
                    int* big_count) {
  __shared__ int s_key[kLpWarps][kLpSlots];
  __shared__ long long s_sc[kLpWarps][kLpSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* key = s_key[warp];
  long long* sc = s_sc[warp];
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
    const int own = lab_in[v];
    if (((v ^ sweep) & 1) != 0) {
      if (lane == 0) lab_out[v] = own;
      continue;
    }
    const long long b = rp[v], e = rp[v + 1];
    const long long d = e - b;
    if (d == 0) {
      if (lane == 0) lab_out[v] = own;
      continue;
    }
    if (d > kLpShort) {
      if (lane == 0) {
        if (d <= kLpMidSmall) mid_rows[atomicAdd(mid_count, 1)] = v;
        else if (d <= kLpMedium) mid_rows[n - 1 - atomicAdd(big_count, 1)] = v;
        else long_rows[atomicAdd(long_count, 1)] = v;
      }
      continue;
    }
    for (int i = lane; i < kLpSlots; i += 32) { key[i] = -1; sc[i] = 0; }
    __syncwarp();
    for (long long i = b + lane; i < e; i += 32) {
      const int l = lab_in[col[i]];
      const long long c = (long long)w[i];
      unsigned h = lp_hash(l) & (kLpSlots - 1);
      for (int p = 0; p < kLpSlots; ++p) {
        int prev = atomicCAS(&key[h], -1, l);
        if (prev == -1 || prev == l) {
          atomicAdd((unsigned long long*)&sc[h], (unsigned long long)c);
          break;
        }
        h = (h + 1) & (kLpSlots - 1);
      }
    }
    __syncwarp();
    LabScore best{-1, 0x7fffffff};
    long long own_s = 0;
    for (int i = lane; i < kLpSlots; i += 32) {
      const int l = key[i];
      if (l < 0) continue;
      best = ls_best(best, LabScore{sc[i], l});
      if (l == own) own_s = sc[i];
    }
    best = warp_ls_best(best);
    own_s = warp_sum(own_s);
    if (lane == 0) lab_out[v] = (best.s > own_s) ? best.l : own;
    __syncwarp();
  }
}

// Medium rows: one block per row with a shared-memory table of up to SLOTS
// slots (the smallest power of two >= 2d).  Scores are kept in the weight
// type: a row's weighted degree fits it.  Rows are read as rows[dir * r].
template <typename WT, int SLOTS>
__global__ void __launch_bounds__(256)
    lp_mid_kernel(const int64_t* __restrict__ rp, const int* __restrict__ col,
                  const WT* __restrict__ w, const int* __restrict__ lab_in,
                  int* __restrict__ lab_out, const int* __restrict__ rows, int dir,
                  const int* count) {
  extern __shared__ __align__(16) unsigned char lp_smem[];
  WT* sc = reinterpret_cast<WT*>(lp_smem);
  int* key = reinterpret_cast<int*>(sc + SLOTS);
  __shared__ long long s_bs[8];
  __shared__ int s_bl[8];
  __shared__ long long s_own[8];
  const int cnt = *count;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = blockIdx.x; r < cnt; r += gridDim.x) {
    const int v = rows[(long long)dir * r];
    const int own = lab_in[v];
    const long long b = rp[v], e = rp[v + 1];
    int slots = 256;  // smallest power of two >= 2d
    while (slots < 2 * (e - b) && slots < SLOTS) slots <<= 1;
    for (int i = threadIdx.x; i < slots; i += blockDim.x) { key[i] = -1; sc[i] = 0; }
    __syncthreads();
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
      const int l = lab_in[col[i]];
      const WT c = w[i];
      unsigned h = lp_hash(l) & (slots - 1);
      for (int p = 0; p < slots; ++p) {
        const int prev = atomicCAS(&key[h], -1, l);
        if (prev == -1 || prev == l) {
          atomic_add_w(&sc[h], c);
          break;
        }
        h = (h + 1) & (slots - 1);
      }
    }
    __syncthreads();
    LabScore best{-1, 0x7fffffff};
    long long own_s = 0;
    for (int i = threadIdx.x; i < slots; i += blockDim.x) {
      const int l = key[i];
      if (l < 0) continue;
      best = ls_best(best, LabScore{(long long)sc[i], l});
      if (l == own) own_s = (long long)sc[i];
    }
    best = warp_ls_best(best);
    own_s = warp_sum(own_s);
    if (lane == 0) { s_bs[warp] = best.s; s_bl[warp] = best.l; s_own[warp] = own_s; }
    __syncthreads();
    if (threadIdx.x == 0) {
      LabScore bb{-1, 0x7fffffff};
      long long os = 0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
        bb = ls_best(bb, LabScore{s_bs[w2], s_bl[w2]});
        os += s_own[w2];
      }
      lab_out[v] = (bb.s > os) ? bb.l : own;
    }
    __syncthreads();
  }
}

// First sweep from identity labels: all labels differ, so the weight of a
// neighbour label at v is the single edge weight; v (with ((v ^ sweep) & 1)
// == 0) adopts the neighbour of largest edge weight, ties to the smaller id
// (its own label has weight 0: there are no self-loops).  Entry tiles with a
// segmented maximum of (w << 32 | ~col) per row; requires w < 2^32.
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    lp_first_kernel(int n, long long M, const int64_t* __restrict__ rp,
                    const int* __restrict__ col, const WT* __restrict__ w,
                    const int* __restrict__ tile_row, int ntiles, int sweep,
                    unsigned long long* __restrict__ best) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  // run layout: this thread's kETItems consecutive entries; rows wholly
  // inside the run publish their maximum directly, the first and the last
  // row's are combined across the warp
  const long long eb = (long long)blockIdx.x * kET + (long long)threadIdx.x * kETItems;
  const int cnt = (int)max(0ll, min((long long)kETItems, M - eb));
  int c[kETItems];
  WT x[kETItems];
  load_run<WT>(col, w, eb, cnt, c, x);
  int first = 0, cur = 0;
  unsigned long long first_max = 0, m = 0;
  if (cnt > 0) {
    first = cur = tile_row_of(tr, rp, eb);
    long long rend = tile_rp(tr, rp, cur + 1);
#pragma unroll
    for (int k = 0; k < kETItems; ++k) {
      if (k < cnt) {
        const long long e = eb + k;
        while (e >= rend) {  // leave row cur (skipping empty rows)
          if (cur == first) first_max = m;
          else if (m && ((cur ^ sweep) & 1) == 0) atomicMax(&best[cur], m);
          m = 0;
          ++cur;
          rend = tile_rp(tr, rp, cur + 1);
        }
        const unsigned long long key =
            ((unsigned long long)(unsigned)x[k] << 32) | (0xffffffffu - (unsigned)c[k]);
        if (key > m) m = key;
      }
    }
    if (cur == first) {
      first_max = m;
      m = 0;
    }
  }
  warp_segment_max(first, first_max, cnt > 0 && ((first ^ sweep) & 1) == 0, best);
  // (the last rows of the lanes whose run spans several rows are distinct)
  warp_segment_max(cur, m, cnt > 0 && cur != first && ((cur ^ sweep) & 1) == 0, best);
}

__global__ void lp_first_finish_kernel(int n, const unsigned long long* __restrict__ best,
                                       int* __restrict__ lab_out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const unsigned long long b = best[v];
    lab_out[v] = b ? (int)(0xffffffffu - (unsigned)(b & 0xffffffffull)) : v;
  }
}

// Long rows: one block per row with an open-addressing table of 2d slots
// taken from a global pool.
template <typename WT>
__global__ void lp_long_kernel(const int64_t* __restrict__ rp, const int* __restrict__ col,
                               const WT* __restrict__ w, const int* __restrict__ lab_in,
                               int* __restrict__ lab_out, const int* __restrict__ long_rows,
                               const int* long_count, int* pool_lab, long long* pool_sc,
                               long long pool_slots, unsigned long long* pool_cursor,
                               DevState* st) {
  __shared__ long long s_base;
  __shared__ long long s_bs[32];
  __shared__ int s_bl[32];
  __shared__ long long s_own[32];
  const int cnt = *long_count;
  for (int r = blockIdx.x; r < cnt; r += gridDim.x) {
    const int v = long_rows[r];
    const int own = lab_in[v];
    const long long b = rp[v], e = rp[v + 1];
    const long long slots = 2 * (e - b);
    if (threadIdx.x == 0) {
      unsigned long long base = atomicAdd(pool_cursor, (unsigned long long)slots);
      s_base = (base + slots <= (unsigned long long)pool_slots) ? (long long)base : -1;
    }
    __syncthreads();
    const long long base = s_base;
    if (base < 0) {
      if (threadIdx.x == 0) {
        lab_out[v] = own;
        set_error(st, ERR_OVERFLOW);
      }
      __syncthreads();
      continue;
    }
    volatile int* key = pool_lab + base;
    long long* sc = pool_sc + base;
    for (long long i = threadIdx.x; i < slots; i += blockDim.x) { key[i] = -1; sc[i] = 0; }
    __threadfence_block();
    __syncthreads();
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
      const int l = lab_in[col[i]];
      const long long c = (long long)w[i];
      long long h = (long long)(lp_hash(l) % (unsigned long long)slots);
      for (long long p = 0; p < slots; ++p) {
        int prev = atomicCAS((int*)&key[h], -1, l);
        if (prev == -1 || prev == l) {
          atomicAdd((unsigned long long*)&sc[h], (unsigned long long)c);
          break;
        }
        h = (h + 1 == slots) ? 0 : h + 1;
      }
    }
    __threadfence_block();
    __syncthreads();
    LabScore best{-1, 0x7fffffff};
    long long own_s = 0;
    volatile long long* vsc = sc;
    for (long long i = threadIdx.x; i < slots; i += blockDim.x) {
      const int l = key[i];
      if (l < 0) continue;
      const long long s = vsc[i];
      best = ls_best(best, LabScore{s, l});
      if (l == own) own_s = s;
    }
    best = warp_ls_best(best);
    own_s = warp_sum(own_s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_bs[warp] = best.s; s_bl[warp] = best.l; s_own[warp] = own_s; }
    __syncthreads();
    if (threadIdx.x == 0) {
      LabScore bb{-1, 0x7fffffff};
      long long os = 0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
        bb = ls_best(bb, LabScore{s_bs[w2], s_bl[w2]});
        os += s_own[w2];
      }
      lab_out[v] = (bb.s > os) ? bb.l : own;
    }
    __syncthreads();
  }
}

// ---- long rows split across blocks (rows longer than kLpMedium entries) ----
// Each long row r owns a table of 2 d_r slots in the pool and ceil(d_r / kLpChunk)
// chunks of work; chunk0[r] / tbase[r] are exclusive prefix sums over the
// long rows.  Blocks walk the chunks; a block finds its row by binary search.
constexpr int kLpChunk = 4096;

__global__ void lp_long_prep_kernel(const int64_t* __restrict__ rp, const int* __restrict__ rows,
                                    const int* count, int* __restrict__ chunk0,
                                    long long* __restrict__ tbase, int* tot_chunks) {
  __shared__ int s_w[32];
  __shared__ long long s_wl[32];
  __shared__ int s_c;
  __shared__ long long s_t;
  const int K = *count;
  if (threadIdx.x == 0) { s_c = 0; s_t = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < K; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int c = 0;
    long long t = 0;
    if (i < K) {
      const long long d = rp[rows[i] + 1] - rp[rows[i]];
      c = (int)((d + kLpChunk - 1) / kLpChunk);
      t = 2 * d;
    }
    int xc = c;
    long long xt = t;
    for (int o = 1; o < 32; o <<= 1) {
      const int yc = __shfl_up_sync(FULL, xc, o);
      const long long yt = __shfl_up_sync(FULL, xt, o);
      if (lane >= o) { xc += yc; xt += yt; }
    }
    if (lane == 31) { s_w[warp] = xc; s_wl[warp] = xt; }
    __syncthreads();
    int ac = 0;
    long long at = 0, tc = 0, tt = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
      if (w2 < warp) { ac += s_w[w2]; at += s_wl[w2]; }
      tc += s_w[w2];
      tt += s_wl[w2];
    }
    const int cb = s_c;
    const long long tb = s_t;
    if (i < K) {
      chunk0[i] = cb + ac + xc - c;
      tbase[i] = tb + at + xt - t;
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_c = cb + (int)tc; s_t = tb + tt; }
    __syncthreads();
  }
  if (threadIdx.x == 0) *tot_chunks = s_c;
}

__device__ __forceinline__ int chunk_row(const int* chunk0, int K, int b) {
  int lo = 0, hi = K;  // largest r with chunk0[r] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (chunk0[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void lp_long_clear_kernel(const int64_t* __restrict__ rp, const int* __restrict__ rows,
                                     const int* count, const int* __restrict__ chunk0,
                                     const long long* __restrict__ tbase, const int* tot_chunks,
                                     int* pool_lab, long long* pool_sc) {
  const int K = *count, T = *tot_chunks;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int r = chunk_row(chunk0, K, b);
    const long long slots = 2 * (rp[rows[r] + 1] - rp[rows[r]]);
    const long long s0 = (long long)(b - chunk0[r]) * 2 * kLpChunk;
    const long long s1 = min(s0 + 2 * kLpChunk, slots);
    for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      pool_lab[tbase[r] + i] = -1;
      pool_sc[tbase[r] + i] = 0;
    }
  }
}

template <typename WT>
__global__ void lp_long_insert_kernel(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                      const WT* __restrict__ w, const int* __restrict__ lab_in,
                                      const int* __restrict__ rows, const int* count,
                                      const int* __restrict__ chunk0,
                                      const long long* __restrict__ tbase, const int* tot_chunks,
                                      int* pool_lab, long long* pool_sc) {
  const int K = *count, T = *tot_chunks;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int r = chunk_row(chunk0, K, b);
    const int v = rows[r];
    const long long rb = rp[v], d = rp[v + 1] - rb;
    const long long slots = 2 * d;
    int* key = pool_lab + tbase[r];
    long long* sc = pool_sc + tbase[r];
    const long long e0 = rb + (long long)(b - chunk0[r]) * kLpChunk;
    const long long e1 = min(e0 + kLpChunk, rb + d);
    for (long long i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
      const int l = lab_in[col[i]];
      const long long c = (long long)w[i];
      long long h = (long long)(lp_hash(l) % (unsigned long long)slots);
      for (long long p = 0; p < slots; ++p) {
        const int prev = atomicCAS(&key[h], -1, l);
        if (prev == -1 || prev == l) {
          atomicAdd((unsigned long long*)&sc[h], (unsigned long long)c);
          break;
        }
        h = (h + 1 == slots) ? 0 : h + 1;
      }
    }
  }
}

// Best (score, smaller label) of each long row's table as score << 32 | ~label.
__global__ void lp_long_scan_kernel(const int64_t* __restrict__ rp, const int* __restrict__ rows,
                                    const int* count, const int* __restrict__ chunk0,
                                    const long long* __restrict__ tbase, const int* tot_chunks,
                                    const int* pool_lab, const long long* pool_sc,
                                    unsigned long long* __restrict__ best) {
  __shared__ unsigned long long s_b[32];
  const int K = *count, T = *tot_chunks;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int r = chunk_row(chunk0, K, b);
    const long long slots = 2 * (rp[rows[r] + 1] - rp[rows[r]]);
    const long long s0 = (long long)(b - chunk0[r]) * 2 * kLpChunk;
    const long long s1 = min(s0 + 2 * kLpChunk, slots);
    const volatile int* key = pool_lab + tbase[r];
    const volatile long long* sc = pool_sc + tbase[r];
    unsigned long long m = 0;
    for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      const int l = key[i];
      if (l < 0) continue;
      const unsigned long long pk =
          ((unsigned long long)sc[i] << 32) | (0xffffffffu - (unsigned)l);
      m = pk > m ? pk : m;
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) s_b[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2) m = s_b[w2] > m ? s_b[w2] : m;
      if (m) atomicMax(&best[r], m);
    }
    __syncthreads();
  }
}

__global__ void lp_long_finish_kernel(const int64_t* __restrict__ rp, const int* __restrict__ rows,
                                      const int* count, const long long* __restrict__ tbase,
                                      const int* pool_lab, const long long* pool_sc,
                                      const unsigned long long* __restrict__ best,
                                      const int* __restrict__ lab_in, int* __restrict__ lab_out) {
  const int K = *count;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < K; r += gridDim.x * blockDim.x) {
    const int v = rows[r];
    const int own = lab_in[v];
    const long long slots = 2 * (rp[v + 1] - rp[v]);
    const volatile int* key = pool_lab + tbase[r];
    const volatile long long* sc = pool_sc + tbase[r];
    long long own_s = 0;
    long long h = (long long)(lp_hash(own) % (unsigned long long)slots);
    for (long long p = 0; p < slots; ++p) {
      const int l = key[h];
      if (l == own) { own_s = sc[h]; break; }
      if (l < 0) break;
      h = (h + 1 == slots) ? 0 : h + 1;
    }
    const unsigned long long b = best[r];
    const long long bs = (long long)(b >> 32);
    const int bl = (int)(0xffffffffu - (unsigned)(b & 0xffffffffull));
    lab_out[v] = (b && bs > own_s) ? bl : own;
  }
}

// Cluster cut values: cut[l] += w for every entry (u, v) with lab[u] = l != lab[v]
// (entry tiles; one atomic per row segment of a warp).
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    lp_cut_kernel(int n, long long M, const int64_t* __restrict__ rp, const int* __restrict__ col,
                  const WT* __restrict__ w, const int* __restrict__ lab,
                  const int* __restrict__ tile_row, int ntiles, long long* __restrict__ cut) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  // run layout: this thread's kETItems consecutive entries
  const long long eb = (long long)blockIdx.x * kET + (long long)threadIdx.x * kETItems;
  const int cnt = (int)max(0ll, min((long long)kETItems, M - eb));
  int c[kETItems];
  WT x[kETItems];
  load_run<WT>(col, w, eb, cnt, c, x);
  int lv[kETItems];
#pragma unroll
  for (int k = 0; k < kETItems; ++k) lv[k] = k < cnt ? lab[c[k]] : 0;  // independent gathers
  // walk the rows: rows wholly inside the run add their cut share directly;
  // the first and the last row's shares are combined across the warp
  int first = 0, cur = 0, lfirst = 0, lcur = 0;
  long long first_acc = 0, acc = 0;
  if (cnt > 0) {
    first = cur = tile_row_of(tr, rp, eb);
    lfirst = lcur = lab[cur];
    long long rend = tile_rp(tr, rp, cur + 1);
#pragma unroll
    for (int k = 0; k < kETItems; ++k) {
      if (k < cnt) {
        const long long e = eb + k;
        while (e >= rend) {  // leave row cur (skipping empty rows)
          if (cur == first) first_acc = acc;
          else if (acc) atomicAdd((unsigned long long*)&cut[lcur], (unsigned long long)acc);
          acc = 0;
          ++cur;
          rend = tile_rp(tr, rp, cur + 1);
          lcur = lab[cur];
        }
        if (lv[k] != lcur) acc += (long long)x[k];
      }
    }
    if (cur == first) {
      first_acc = acc;
      acc = 0;
    }
  }
  warp_segment_add<long long, long long>(first, lfirst, first_acc, cnt > 0, cut);
  // (the last rows of the lanes whose run spans several rows are distinct)
  warp_segment_add<long long, long long>(cur, lcur, acc, cnt > 0 && cur != first, cut);
}

// Cluster sizes; lanes of a warp with the same label add once (large
// clusters would otherwise serialise on one counter).
__global__ void lp_size_kernel(const int* __restrict__ lab, int n, int* __restrict__ size) {
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int v = base + threadIdx.x;
    const int l = v < n ? lab[v] : -1;
    const unsigned peers = __match_any_sync(FULL, l);
    if (l >= 0 && lane == __ffs(peers) - 1) atomicAdd(&size[l], __popc(peers));
  }
}

__global__ void lp_min_kernel(const long long* __restrict__ cut, const int* __restrict__ size,
                              int n, unsigned long long* __restrict__ blk) {
  ValArg best{~0ull, 0x7fffffff};
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    const int s = size[l];
    if (s > 0 && s < n) best = va_min(best, ValArg{(unsigned long long)cut[l], l});
  }
  ValArg r = block_va_min(best);
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = r.v;
    blk[2 * blockIdx.x + 1] = (unsigned long long)(unsigned)r.a;
  }
}

__global__ void lp_final_kernel(const unsigned long long* __restrict__ blk, int nb, DevState* st) {
  ValArg best{~0ull, 0x7fffffff};
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    best = va_min(best, ValArg{blk[2 * i], (int)blk[2 * i + 1]});
  ValArg r = block_va_min(best);
  if (threadIdx.x == 0) {
    st->lp_val = r.v;
    st->lp_label = r.a;
    if (r.v != ~0ull) atomicMin(&st->lambda, r.v);
  }
}

// ---------------------------------------------------------------- union-find
__global__ void uf_init_kernel(int* parent, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    parent[v] = v;
}

__global__ void uf_pairs_kernel(int* parent, const int* __restrict__ pu, const int* __restrict__ pv,
                                long long np, int n, DevState* st) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const int a = pu[i], b = pv[i];
    if (a < 0 || a >= n || b < 0 || b >= n) { set_error(st, ERR_INPUT); continue; }
    if (!uf_union(parent, a, b)) set_error(st, ERR_INTERNAL);
  }
}

__global__ void group_min_kernel(const int* __restrict__ group, int n, int* gmin, DevState* st) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int g = group[v];
    if (g < 0 || g >= n) { set_error(st, ERR_INPUT); continue; }
    atomicMin(&gmin[g], v);
  }
}

__global__ void group_parent_kernel(const int* __restrict__ group, const int* __restrict__ gmin,
                                    int n, int* parent) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int g = group[v];
    parent[v] = (g >= 0 && g < n) ? gmin[g] : v;
  }
}

__global__ void fill_i32_kernel(int* a, int n, int val) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) a[v] = val;
}

__global__ void uf_roots_kernel(int* parent, int n, int* __restrict__ flags) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int r = uf_find(parent, v);
    flags[v] = (r == v) ? 1 : 0;
  }
}

// After uf_roots every path has been compressed at least once; finish with
// a full find (no writes) and map to the dense rank of the root.
__global__ void uf_label_kernel(int* parent, int n, const int* __restrict__ rank,
                                int* __restrict__ L) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int r = v;
    volatile int* vp = parent;
    while (vp[r] != r) r = vp[r];
    L[v] = rank[r];
  }
}

__global__ void compose_map_kernel(int* map0, const int* __restrict__ L, int n0) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x)
    map0[i] = L[map0[i]];
}

// ----------------------------------------------------------------- witness
__global__ void side_vertex_kernel(uint8_t* side0, const int* __restrict__ map0, int n0, int x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x)
    side0[i] = map0[i] == x ? 1 : 0;
}
__global__ void side_label_kernel(uint8_t* side0, const int* __restrict__ map0, int n0,
                                  const int* __restrict__ lab, int l) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x)
    side0[i] = lab[map0[i]] == l ? 1 : 0;
}
__global__ void mark_list_kernel(uint8_t* cur, const int* __restrict__ list, int len) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    cur[list[i]] = 1;
}
__global__ void side_cur_kernel(uint8_t* side0, const int* __restrict__ map0, int n0,
                                const uint8_t* __restrict__ cur) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x)
    side0[i] = cur[map0[i]];
}
// bit v = side0[v] xor side0[0]: 1 on the side that does not hold vertex 0.
__global__ void bitmap_kernel(const uint8_t* __restrict__ side0, int n0, u64* __restrict__ bitmap) {
  const int words = (n0 + 63) / 64;
  const uint8_t flip = side0[0];
  for (int wd = blockIdx.x * blockDim.x + threadIdx.x; wd < words; wd += gridDim.x * blockDim.x) {
    u64 x = 0;
    for (int b = 0; b < 64; ++b) {
      const int v = wd * 64 + b;
      if (v < n0 && (side0[v] ^ flip)) x |= 1ull << b;
    }
    bitmap[wd] = x;
  }
}

int grid_for(long long work, int block) {
  long long g = (work + block - 1) / block;
  long long cap = (long long)num_sms() * 32;
  return (int)std::max<long long>(1, std::min(g, cap));
}

}  // namespace

// ================================================================= launchers
cudaError_t tile_rows(const int64_t* rp, int n, long long M, int* tile_row, cudaStream_t s,
                      int* launches) {
  if (M <= 0 || n <= 0) return cudaSuccess;
  tile_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(rp, n, tile_row);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t degrees_min(const WT* deg, int n, unsigned long long* blk, DevState* st,
                        cudaStream_t s, int* launches) {
  const int nb = std::min(grid_for(n, 256), 1024);
  degmin_kernel<WT><<<nb, 256, 0, s>>>(deg, n, blk);
  degmin_final_kernel<<<1, 1024, 0, s>>>(blk, nb, st);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t emit_pairs(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                       const int* L, int vbits, const int* tile_row, u64* keys, WT* vals,
                       DevState* st, int validate, cudaStream_t s, int* launches,
                       const int* keep_row) {
  if (M <= 0) return cudaSuccess;
  const int ntiles = (int)((M + kET - 1) / kET);
  emit_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, w, L, vbits, tile_row, ntiles,
                                                 keys, vals, st, validate, keep_row);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t build_csr(const u64* keys, const WT* vals, int N, int vbits, int n2, int* uid,
                      int* part, int64_t* rp2, int* col2, WT* w2, DevState* st,
                      int* m2_dev, int* urow, cudaStream_t s, int* launches) {
  if (N <= 0) {
    rp_fill_kernel<<<grid_for(n2 + 1, 256), 256, 0, s>>>(rp2, n2);
    cudaMemsetAsync(m2_dev, 0, sizeof(int), s);
    ++*launches;
    return cudaGetLastError();
  }
  head_flags_kernel<<<grid_for(N, 256), 256, 0, s>>>(keys, N, uid);
  ++*launches;
  cudaError_t err = scan_exclusive_i32(uid, uid, N, part, m2_dev, s, launches);
  if (err != cudaSuccess) return err;
  cudaMemsetAsync(w2, 0, (size_t)N * sizeof(WT), s);
  segsum_kernel<WT><<<grid_for((N + 7) / 8, 256), 256, 0, s>>>(keys, vals, N, uid, vbits, urow,
                                                               col2, w2);
  rp_search_kernel<<<grid_for(n2 + 1, 256), 256, 0, s>>>(urow, m2_dev, n2, rp2);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t row_degrees(int n, long long M, const int64_t* rp, const WT* w, int* tile_row,
                        WT* deg, cudaStream_t s, int* launches) {
  cudaMemsetAsync(deg, 0, (size_t)std::max(n, 1) * sizeof(WT), s);
  if (M <= 0) return cudaGetLastError();
  tile_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(rp, n, tile_row);
  const int ntiles = (int)((M + kET - 1) / kET);
  degree_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, w, tile_row, ntiles, deg);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t check_symmetric(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                            const int* tile_row, DevState* st, cudaStream_t s, int* launches) {
  if (M <= 0) return cudaSuccess;
  const int ntiles = (int)((M + kET - 1) / kET);
  cudaMemsetAsync(&st->sym_balance, 0, sizeof(st->sym_balance), s);
  symmetric_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, w, tile_row, ntiles, st);
  sym_final_kernel<<<1, 1, 0, s>>>(st);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t pr_marks(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                     const WT* deg, const int* tile_row, uint32_t mask, long long budget,
                     int* parent, uint8_t* flags_out, unsigned* short_bits, DevState* st,
                     cudaStream_t s, int* launches, const BatchView* bv) {
  if (M <= 0 || mask == 0) return cudaSuccess;
  const int ntiles = (int)((M + kET - 1) / kET);
  BatchView v{};
  if (bv) v = *bv;
  const bool bits = (mask & 12u) && budget >= 0;
  if (bits) {
    short_rows_kernel<<<grid_for((n + 31) / 32 * 32, 256), 256, 0, s>>>(n, rp, budget,
                                                                         short_bits);
    ++*launches;
  }
  pr_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, w, deg, tile_row, ntiles, mask,
                                               budget, parent, flags_out,
                                               bits ? short_bits : nullptr, st, v, bv ? 1 : 0);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t lp_first_sweep(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                           const int* tile_row, int sweep, unsigned long long* best, int* lab_out,
                           cudaStream_t s, int* launches) {
  cudaMemsetAsync(best, 0, (size_t)n * sizeof(unsigned long long), s);
  if (M > 0) {
    const int ntiles = (int)((M + kET - 1) / kET);
    lp_first_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, w, tile_row, ntiles, sweep,
                                                      best);
    ++*launches;
  }
  lp_first_finish_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, best, lab_out);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t lp_sweep(int n, const int64_t* rp, const int* col, const WT* w, const int* lab_in,
                     int* lab_out, int sweep, const LpScratch& sc, DevState* st, cudaStream_t s,
                     int* launches) {
  // counts[0] long rows, counts[1] medium rows, counts[2] chunks of long rows;
  // medium rows are listed after the n-entry long list
  int* mid_rows = sc.long_rows + n;
  cudaMemsetAsync(sc.counts, 0, 4 * sizeof(int), s);
  cudaMemsetAsync(sc.pool_cursor, 0, sizeof(unsigned long long), s);
  lp_short_kernel<WT><<<grid_for((long long)n * 32, kLpWarps * 32), kLpWarps * 32, 0, s>>>(
      n, rp, col, w, lab_in, lab_out, sweep, sc.long_rows, sc.counts, mid_rows, sc.counts + 1,
      sc.counts + 3);
  // medium rows in two table sizes: up to kLpMidSmall entries (many blocks
  // per SM) from the front of the list, longer ones from its back
  constexpr int kSmallSlots = 2 * kLpMidSmall;
  const size_t small_smem = (size_t)kSmallSlots * (sizeof(WT) + sizeof(int));
  const size_t big_smem = (size_t)kLpMidSlots * (sizeof(WT) + sizeof(int));
  static bool mid_attr[2] = {false, false};
  if (!mid_attr[sizeof(WT) == 8]) {
    cudaFuncSetAttribute(lp_mid_kernel<WT, kSmallSlots>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem);
    cudaFuncSetAttribute(lp_mid_kernel<WT, kLpMidSlots>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
    mid_attr[sizeof(WT) == 8] = true;
  }
  lp_mid_kernel<WT, kSmallSlots><<<num_sms() * 8, 256, small_smem, s>>>(
      rp, col, w, lab_in, lab_out, mid_rows, 1, sc.counts + 1);
  lp_mid_kernel<WT, kLpMidSlots><<<num_sms() * (sizeof(WT) == 8 ? 2 : 3), 256, big_smem, s>>>(
      rp, col, w, lab_in, lab_out, mid_rows + (n - 1), -1, sc.counts + 3);
  *launches += 3;
  if (sizeof(WT) == 8) {  // scores may exceed 32 bits: one block per long row
    lp_long_kernel<WT><<<num_sms() * 2, 512, 0, s>>>(rp, col, w, lab_in, lab_out, sc.long_rows,
                                                     sc.counts, sc.pool_lab, sc.pool_sc,
                                                     sc.pool_slots, sc.pool_cursor, st);
    ++*launches;
    return cudaGetLastError();
  }
  cudaMemsetAsync(sc.best, 0, (size_t)std::max(n, 1) * sizeof(unsigned long long), s);
  lp_long_prep_kernel<<<1, 1024, 0, s>>>(rp, sc.long_rows, sc.counts, sc.chunk0, sc.tbase,
                                         sc.counts + 2);
  const int g = num_sms() * 8;
  lp_long_clear_kernel<<<g, 256, 0, s>>>(rp, sc.long_rows, sc.counts, sc.chunk0, sc.tbase,
                                         sc.counts + 2, sc.pool_lab, sc.pool_sc);
  lp_long_insert_kernel<WT><<<g, 256, 0, s>>>(rp, col, w, lab_in, sc.long_rows, sc.counts,
                                              sc.chunk0, sc.tbase, sc.counts + 2, sc.pool_lab,
                                              sc.pool_sc);
  lp_long_scan_kernel<<<g, 256, 0, s>>>(rp, sc.long_rows, sc.counts, sc.chunk0, sc.tbase,
                                        sc.counts + 2, sc.pool_lab, sc.pool_sc, sc.best);
  lp_long_finish_kernel<<<num_sms(), 256, 0, s>>>(rp, sc.long_rows, sc.counts, sc.tbase,
                                                  sc.pool_lab, sc.pool_sc, sc.best, lab_in,
                                                  lab_out);
  *launches += 5;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t lp_bound(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                     const int* lab, const int* tile_row, long long* cut, int* size,
                     unsigned long long* blk, DevState* st, cudaStream_t s, int* launches) {
  cudaMemsetAsync(cut, 0, (size_t)n * sizeof(long long), s);
  cudaMemsetAsync(size, 0, (size_t)n * sizeof(int), s);
  if (M > 0) {
    const int ntiles = (int)((M + kET - 1) / kET);
    lp_cut_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, w, lab, tile_row, ntiles, cut);
    ++*launches;
  }
  lp_size_kernel<<<grid_for(n, 256), 256, 0, s>>>(lab, n, size);
  const int nb = std::min(grid_for(n, 256), 1024);
  lp_min_kernel<<<nb, 256, 0, s>>>(cut, size, n, blk);
  lp_final_kernel<<<1, 1024, 0, s>>>(blk, nb, st);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t uf_init(int* parent, int n, cudaStream_t s, int* launches) {
  uf_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(parent, n);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t uf_hook_pairs(int* parent, const int* pu, const int* pv, long long np, int n,
                          DevState* st, cudaStream_t s, int* launches) {
  if (np <= 0) return cudaSuccess;
  uf_pairs_kernel<<<grid_for(np, 256), 256, 0, s>>>(parent, pu, pv, np, n, st);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t uf_from_groups(int* parent, const int* group, int* gmin, int n, DevState* st,
                           cudaStream_t s, int* launches) {
  fill_i32_kernel<<<grid_for(n, 256), 256, 0, s>>>(gmin, n, 0x7fffffff);
  group_min_kernel<<<grid_for(n, 256), 256, 0, s>>>(group, n, gmin, st);
  group_parent_kernel<<<grid_for(n, 256), 256, 0, s>>>(group, gmin, n, parent);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t uf_relabel(int* parent, int* L, int* flags, int* rank, int* part, int n,
                       DevState* st, cudaStream_t s, int* launches) {
  uf_roots_kernel<<<grid_for(n, 256), 256, 0, s>>>(parent, n, flags);
  ++*launches;
  cudaError_t err = scan_exclusive_i32(flags, rank, n, part, &st->n_next, s, launches);
  if (err != cudaSuccess) return err;
  uf_label_kernel<<<grid_for(n, 256), 256, 0, s>>>(parent, n, rank, L);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t compose_map(int* map0, const int* L, int n0, cudaStream_t s, int* launches) {
  compose_map_kernel<<<grid_for(n0, 256), 256, 0, s>>>(map0, L, n0);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t side_from_vertex(uint8_t* side0, const int* map0, int n0, int x, cudaStream_t s,
                             int* launches) {
  side_vertex_kernel<<<grid_for(n0, 256), 256, 0, s>>>(side0, map0, n0, x);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t side_from_label(uint8_t* side0, const int* map0, int n0, const int* lab, int l,
                            cudaStream_t s, int* launches) {
  side_label_kernel<<<grid_for(n0, 256), 256, 0, s>>>(side0, map0, n0, lab, l);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t side_from_list(uint8_t* side0, const int* map0, int n0, uint8_t* cur, int n,
                           const int* list, int len, cudaStream_t s, int* launches) {
  cudaMemsetAsync(cur, 0, (size_t)n, s);
  if (len > 0) {
    mark_list_kernel<<<grid_for(len, 256), 256, 0, s>>>(cur, list, len);
    ++*launches;
  }
  side_cur_kernel<<<grid_for(n0, 256), 256, 0, s>>>(side0, map0, n0, cur);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t side_to_bitmap(const uint8_t* side0, int n0, u64* bitmap, cudaStream_t s,
                           int* launches) {
  bitmap_kernel<<<grid_for((n0 + 63) / 64, 256), 256, 0, s>>>(side0, n0, bitmap);
  ++*launches;
  return cudaGetLastError();
}

// ----------------------------------------------------- explicit instances
#define MC_INST(WT)                                                                              \
  template cudaError_t degrees_min<WT>(const WT*, int, unsigned long long*, DevState*,           \
                                       cudaStream_t, int*);                                      \
  template cudaError_t emit_pairs<WT>(int, long long, const int64_t*, const int*, const WT*,     \
                                      const int*, int, const int*, u64*, WT*, DevState*, int,    \
                                      cudaStream_t, int*, const int*);                           \
  template cudaError_t build_csr<WT>(const u64*, const WT*, int, int, int, int*, int*, int64_t*, \
                                     int*, WT*, DevState*, int*, int*, cudaStream_t, int*);      \
  template cudaError_t row_degrees<WT>(int, long long, const int64_t*, const WT*, int*, WT*,      \
                                       cudaStream_t, int*);                                      \
  template cudaError_t check_symmetric<WT>(int, long long, const int64_t*, const int*,           \
                                           const WT*, const int*, DevState*, cudaStream_t,       \
                                           int*);                                                \
  template cudaError_t pr_marks<WT>(int, long long, const int64_t*, const int*, const WT*,       \
                                    const WT*, const int*, uint32_t, long long, int*, uint8_t*,  \
                                    unsigned*, DevState*, cudaStream_t, int*, const BatchView*); \
  template cudaError_t lp_sweep<WT>(int, const int64_t*, const int*, const WT*, const int*,      \
                                    int*, int, const LpScratch&, DevState*, cudaStream_t, int*); \
  template cudaError_t lp_first_sweep<WT>(int, long long, const int64_t*, const int*, const WT*, \
                                          const int*, int, unsigned long long*, int*,           \
                                          cudaStream_t, int*);                                  \
  template cudaError_t lp_bound<WT>(int, long long, const int64_t*, const int*, const WT*,       \
                                    const int*, const int*, long long*, int*,                    \
                                    unsigned long long*, DevState*, cudaStream_t, int*);

MC_INST(int32_t)
MC_INST(int64_t)

}  // namespace mc
