// contract.cu -- row-wise contraction for rounds where most groups are
// single vertices.
//
// Contraction (Sec. 2: the vertices of a group become one vertex that
// inherits their edges; parallel edges are summed, self-loops dropped) with
// canonical labels L = rank of each group's smallest member.  On a singleton
// group's row u the relabelled entries keep their order wherever the
// neighbour y is itself a singleton: for singletons y1 < y2, L[y1] < L[y2].
// Only the entries towards multi-member groups ("moved" entries) can break
// the order or coincide.  So a singleton row is rebuilt in place: its clean
// entries are copied in order and the (few) distinct moved labels, summed
// and sorted, are merged in at their ranks.  Two forms: on graphs of
// kFlatMinEntries entries or more, kernels over the round's entry tiles that
// take the moved entries, by symmetry, from the other groups' contracted
// rows (the "flat rows" section below); on smaller graphs one warp per row
// that sums them itself (sr_count / sr_write).  Rows of multi-member groups,
// singleton rows of more than kSrMaxRow entries (and, in the warp form, those
// with more than kSrMoved distinct moved labels) are "general": their
// entries alone go through the relabel / radix sort / segmented sum path, or
// a dense accumulator for the largest groups, and the resulting rows are
// copied to their place.  The output is the same canonical CSR the full sort
// gives (rows ascending, parallel edges summed, self-loops dropped).
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"
#include "tiles.cuh"

namespace mc {

namespace {

constexpr int kSrWarps = 8;       // warps (rows) per block of the row kernels
constexpr int kSrSlots = 64;      // warp hash of moved labels (power of two)
constexpr int kSrMoved = 32;      // at most this many distinct moved labels per row
constexpr int kSrMaxRow = 4096;  // longer singleton rows take the general path
constexpr int kSrUnroll = 4;     // 32-entry chunks whose loads a warp issues together
constexpr int kMovedBit = (int)0x80000000u;  // vinfo: neighbour's group has several members

__device__ __forceinline__ unsigned sr_hash(int l) { return (unsigned)l * 0x9E3779B1u; }

// cnt[L[x]] += 1 for every vertex (one atomic per distinct label of a warp).
__global__ void group_count_kernel(const int* __restrict__ L, int n, int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int x = base + threadIdx.x;
    const int lab = x < n ? L[x] : -1;
    const unsigned peers = __match_any_sync(FULL, lab);
    if (lab >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[lab], __popc(peers));
  }
}

// After the counts: vinfo[x] = L[x], with kMovedBit set when x's group has
// several members; gen[g] for multi-member groups; single_entries += the
// entries of rows whose group is a single vertex.
__global__ void single_entries_kernel(const int64_t* __restrict__ rp, const int* __restrict__ L,
                                      int n, const int* __restrict__ cnt, int* __restrict__ gen,
                                      int* __restrict__ vinfo, int* __restrict__ rep,
                                      int* __restrict__ dsum, unsigned long long* single_entries) {
  unsigned long long s = 0;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int x = base + threadIdx.x;
    int g = -1, len = 0;
    if (x < n) {
      g = L[x];
      len = (int)(rp[x + 1] - rp[x]);
      if (cnt[g] == 1) {
        s += (unsigned long long)len;
        vinfo[x] = g;
        rep[g] = x;
        if (len > kSrMaxRow) gen[g] = 1;  // too long for the singleton-row kernels
      } else {
        gen[g] = 1;
        vinfo[x] = g | kMovedBit;
        rep[g] = -1;
      }
    }
    // entries per group (one atomic per distinct group of the warp)
    const unsigned peers = __match_any_sync(FULL, g);
    const int tot = (int)__reduce_add_sync(peers, (unsigned)len);
    if (g >= 0 && lane == __ffs(peers) - 1 && tot) atomicAdd(&dsum[g], tot);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(single_entries, s);
}

// Dense groups: big enough that an n2-slot accumulator (n2 slots read to
// count and to write, ~8 B each) costs less than sorting their entries
// (~120 B each through emit, radix passes and segmented sum).
// n2 is read on the device (the union-find relabel's vertex count), so the
// decision needs no synchronisation of its own; the capacity is
// dense_capacity(n2): min(n2, dense_slots / n2).
__global__ void dense_mark_kernel(const int* __restrict__ n2p, long long dense_slots,
                                  const int* __restrict__ dsum, int* __restrict__ gen,
                                  int* __restrict__ did, int* ndense,
                                  unsigned long long* dense_entries) {
  const int n2 = *n2p;
  if (n2 <= 1) return;
  const int max_dense = (int)min((long long)n2, dense_slots / n2);
  if (max_dense <= 0) return;
  const int thr = max(n2 / 16, 256);
  unsigned long long tot = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n2; g += gridDim.x * blockDim.x) {
    if (dsum[g] < thr) continue;
    const int d = atomicAdd(ndense, 1);
    if (d < max_dense) {
      gen[g] = 2;
      did[g] = d;
      tot += (unsigned long long)dsum[g];
    }
  }
  tot = warp_sum(tot);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(dense_entries, tot);
}

// Entry tiles: every entry of a dense group's member rows adds its weight to
// the group's accumulator slot of the far end's label (self-loops dropped).
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    dense_acc_kernel(int n, long long M, int n2, const int64_t* __restrict__ rp,
                     const int* __restrict__ col, const WT* __restrict__ w,
                     const int* __restrict__ L, const int* __restrict__ gen,
                     const int* __restrict__ did, const int* __restrict__ tile_row, int ntiles,
                     WT* __restrict__ acc) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rp, n, tile_row, ntiles, blockIdx.x);
  bool any = false;
  for (int r = tr.r0 + threadIdx.x; r <= tr.r1 && !any; r += blockDim.x) any = gen[L[r]] == 2;
  if (!__syncthreads_or(any)) return;
  const long long e0 = (long long)blockIdx.x * kET;
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    if (e >= M) break;
    const int u = tile_row_of(tr, rp, e);
    const int g = L[u];
    if (gen[g] != 2) continue;
    const int vp = L[col[e]];
    if (vp == g) continue;
    atomic_add_w(&acc[(long long)did[g] * n2 + vp], w[e]);
  }
}

// Per chunk of kDenseChunk accumulator slots: the nonzero slots (blockIdx.y =
// dense slot).  chunk[d * nchunks + c]; len[g] gets the total.

// flat != 0: the nonzero slots of multi-member dense groups towards single
// vertices are also transposed into those rows' moved lists (as in
// fr_fill_kernel: slot = kpc[label]++ inside the member's row span).
template <typename WT>
__global__ void __launch_bounds__(256)
    dense_count_kernel(int n2, const WT* __restrict__ acc, const int* ndense, int max_dense,
                       int* __restrict__ chunk, int nchunks, int flat,
                       const int* __restrict__ dense_group, const int64_t* __restrict__ rp,
                       const int* __restrict__ rep, const int* __restrict__ gen,
                       int* __restrict__ kpc, int* __restrict__ side_v, WT* __restrict__ side_w) {
  const int d = blockIdx.y;
  if (d >= min(*ndense, max_dense)) return;
  const int c = blockIdx.x;
  const long long base = (long long)d * n2;
  const int G = flat ? dense_group[d] : 0;
  const bool transpose = flat && rep[G] < 0;
  int cntv = 0;
  constexpr int kPer = kDenseChunk / 256;  // slots per thread (blocks of 256 threads)
  const int i0 = c * kDenseChunk + threadIdx.x, iend = min(n2, (c + 1) * kDenseChunk);
  WT v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = i0 + k * 256;
    v[k] = i < iend ? acc[base + i] : WT(0);
    cntv += v[k] != 0;
  }
  if (transpose) {
    // the gathers of a thread's slots go out together, level by level
    int m[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = i0 + k * 256;
      m[k] = -1;
      if (v[k] != 0) {
        const int r = rep[i];
        if (r >= 0 && gen[i] == 0) m[k] = r;
      }
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (m[k] < 0) continue;
      const int i = i0 + k * 256;
      const long long b = rp[m[k]];
      const long long len = rp[m[k] + 1] - b;
      const int slot = atomicAdd(&kpc[i], 1);
      if (slot < len) {
        side_v[b + slot] = G;
        side_w[b + slot] = v[k];
      }
    }
  }
  cntv = (int)__reduce_add_sync(FULL, (unsigned)cntv);
  __shared__ int s_w[8];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = cntv;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_w[k];
    chunk[(long long)d * nchunks + c] = t;
  }
}

// One block per dense group: chunk counts -> exclusive offsets, len[g].
__global__ void dense_scan_kernel(int n2, const int* __restrict__ gen, const int* __restrict__ did,
                                  const int* ndense, int max_dense, int* __restrict__ chunk,
                                  int nchunks, int* __restrict__ len) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n2; g += gridDim.x * blockDim.x) {
    if (gen[g] != 2) continue;
    int* ch = chunk + (long long)did[g] * nchunks;
    int run = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int v = ch[c];
      ch[c] = run;
      run += v;
    }
    len[g] = run;
  }
}

// Writes each dense group's nonzero slots in slot order (its canonical row)
// at rp2[g] + chunk offset + rank in the chunk, adds the row weight to
// deg2[g] and clears the slots for the next round.
template <typename WT>
__global__ void __launch_bounds__(256)
    dense_write_kernel(int n2, const int* __restrict__ gen, const int* __restrict__ did,
                       const int* ndense, int max_dense, const int* __restrict__ chunk,
                       int nchunks, WT* __restrict__ acc, const int* __restrict__ dense_group,
                       const int64_t* __restrict__ rp2, int* __restrict__ col2,
                       WT* __restrict__ w2, WT* __restrict__ deg2) {
  const int d = blockIdx.y;
  if (d >= min(*ndense, max_dense)) return;
  const int g = dense_group[d];
  const int c = blockIdx.x;
  const long long base = (long long)d * n2;
  __shared__ int s_w[8];
  __shared__ int s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  const long long out0 = rp2[g] + chunk[(long long)d * nchunks + c];
  long long dsumv = 0;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int i0 = c * kDenseChunk; i0 < min(n2, (c + 1) * kDenseChunk); i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    WT v = 0;
    if (i < n2 && i < (c + 1) * kDenseChunk) v = acc[base + i];
    const bool nz = v != 0;
    const unsigned b = __ballot_sync(FULL, nz);
    if (lane == 0) s_w[wp] = __popc(b);
    __syncthreads();
    int before = s_run;
    for (int k = 0; k < wp; ++k) before += s_w[k];
    if (nz) {
      const long long pos = out0 + before + __popc(b & lanemask_lt());
      col2[pos] = i;
      w2[pos] = v;
      acc[base + i] = 0;
      dsumv += (long long)v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_w[k];
      s_run += t;
    }
    __syncthreads();
  }
  dsumv = warp_sum(dsumv);
  if (lane == 0 && dsumv) atomic_add_w(&deg2[g], (WT)dsumv);
}

__global__ void dense_group_list_kernel(int n2, const int* __restrict__ gen,
                                        const int* __restrict__ did, int* __restrict__ dense_group) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n2; g += gridDim.x * blockDim.x)
    if (gen[g] == 2) dense_group[did[g]] = g;
}

// Pass A: one warp per singleton row u (g = L[u]).  Counts the clean entries,
// sums the moved entries per label in a warp hash, and stores the distinct
// moved labels ascending with their sums at side_v/side_w[rp[u] ...].
// len[g] = clean + distinct moved; kcnt[g] = distinct moved.  A row that
// does not fit (too long, too many moved labels) is marked general.
template <typename WT>
__global__ void __launch_bounds__(kSrWarps * 32)
    sr_count_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                    const WT* __restrict__ w, const int* __restrict__ vinfo,
                    int* __restrict__ gen, int* __restrict__ len,
                    int* __restrict__ kcnt, int* __restrict__ side_v, WT* __restrict__ side_w,
                    const int* __restrict__ list, const int* __restrict__ list_len) {
  __shared__ int hk[kSrWarps][kSrSlots];
  __shared__ unsigned long long hs[kSrWarps][kSrSlots];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nrows = list ? *list_len : n;
  // warp-uniform loop: the row kernels use no block barrier
  for (int wi = blockIdx.x * kSrWarps + wp; wi < nrows; wi += gridDim.x * kSrWarps) {
    const int u = list ? list[wi] : wi;
    const int vu = vinfo[u];
    const int b = (int)rp[u], e = (int)rp[u + 1];
    if (vu & kMovedBit) continue;
    const int g = vu;
    if (gen[g]) continue;  // dense
    if (e - b > kSrMaxRow) {
      if (lane == 0) gen[g] = 1;
      continue;
    }
    __syncwarp();  // the previous row's hash reads are done
    for (int i = lane; i < kSrSlots; i += 32) {
      hk[wp][i] = -1;
      hs[wp][i] = 0;
    }
    __syncwarp();
    int clean = 0;
    bool over = false;
    for (int base = b; base < e; base += 32 * kSrUnroll) {
      int vp[kSrUnroll];
      bool moved[kSrUnroll];
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) {
        const int idx = base + 32 * j + lane;
        vp[j] = idx < e ? col[idx] : 0;
      }
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) vp[j] = base + 32 * j + lane < e ? vinfo[vp[j]] : 0;
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) {
        const int idx = base + 32 * j + lane;
        moved[j] = idx < e && (vp[j] & kMovedBit);
        vp[j] &= ~kMovedBit;
        clean += __popc(__ballot_sync(FULL, idx < e && !moved[j]));
      }
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) {
        // lanes with the same moved label add their weights first; one lane
        // per label then updates the warp hash
        const unsigned mmask = __ballot_sync(FULL, moved[j]);
        if (!moved[j]) continue;
        unsigned long long c = (unsigned long long)(long long)w[base + 32 * j + lane];
        const unsigned peers = __match_any_sync(mmask, vp[j]);
        if (sizeof(WT) == 4) {
          // int32 weights: every partial sum of a graph's entries is below 2^31
          c = __reduce_add_sync(peers, (unsigned)c);
        } else {
          unsigned long long t = 0;
          for (unsigned m = peers; m; m &= m - 1) t += __shfl_sync(peers, c, __ffs(m) - 1);
          c = t;
        }
        if (lane != __ffs(peers) - 1) continue;
        unsigned h = sr_hash(vp[j]) & (kSrSlots - 1);
        int p = 0;
        for (; p < kSrSlots; ++p) {
          const int prev = atomicCAS(&hk[wp][h], -1, vp[j]);
          if (prev == -1 || prev == vp[j]) {
            atomicAdd(&hs[wp][h], c);
            break;
          }
          h = (h + 1) & (kSrSlots - 1);
        }
        if (p == kSrSlots) over = true;
      }
    }
    __syncwarp();
    const int k0 = hk[wp][lane], k1 = hk[wp][lane + 32];
    const int kp = __popc(__ballot_sync(FULL, k0 >= 0)) + __popc(__ballot_sync(FULL, k1 >= 0));
    if (__any_sync(FULL, over) || kp > kSrMoved) {
      if (lane == 0) gen[g] = 1;
      continue;
    }
    if (kp > 0) {
      // compact the stored labels (at most 32) into lanes, then rank each among
      // them: the labels are distinct
      const unsigned b0 = __ballot_sync(FULL, k0 >= 0);
      const unsigned b1 = __ballot_sync(FULL, k1 >= 0);
      const int n0 = __popc(b0);
      const unsigned long long s0 = k0 >= 0 ? hs[wp][lane] : 0ull;
      const unsigned long long s1 = k1 >= 0 ? hs[wp][lane + 32] : 0ull;
      __syncwarp();
      if (k0 >= 0) {
        const int slot = __popc(b0 & lanemask_lt());
        hk[wp][slot] = k0;
        hs[wp][slot] = s0;
      }
      if (k1 >= 0) {
        const int slot = n0 + __popc(b1 & lanemask_lt());
        hk[wp][slot] = k1;
        hs[wp][slot] = s1;
      }
      __syncwarp();
      if (lane < kp) {
        const int k = hk[wp][lane];
        int r = 0;
        for (int t = 0; t < kp; ++t) r += hk[wp][t] < k ? 1 : 0;
        side_v[b + r] = k;
        side_w[b + r] = (WT)(long long)hs[wp][lane];
      }
    }
    if (lane == 0) {
      len[g] = clean + kp;
      kcnt[g] = kp;
    }
  }
}

// General rows: len[g] from the general CSR.
__global__ void gen_len_kernel(const int64_t* __restrict__ rpG, const int* __restrict__ gen, int n2,
                               int* __restrict__ len) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n2; g += gridDim.x * blockDim.x)
    if (gen[g] == 1) len[g] = (int)(rpG[g + 1] - rpG[g]);
}

__global__ void rp_from_offsets_kernel(const int* __restrict__ off, const int* __restrict__ total,
                                       int n2, int64_t* __restrict__ rp2) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= n2; g += gridDim.x * blockDim.x)
    rp2[g] = g < n2 ? (int64_t)off[g] : (int64_t)*total;
}

// Pass B: one warp per non-general singleton row: clean entries at
// (clean index) + (moved labels below), moved labels at (their index) +
// (clean entries below); deg2[g] = the row's weight.
template <typename WT>
__global__ void __launch_bounds__(kSrWarps * 32)
    sr_write_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                    const WT* __restrict__ w, const int* __restrict__ vinfo,
                    const int* __restrict__ gen,
                    const int* __restrict__ kcnt, const int* __restrict__ side_v,
                    const WT* __restrict__ side_w, const int64_t* __restrict__ rp2,
                    int* __restrict__ col2, WT* __restrict__ w2, WT* __restrict__ deg2,
                    const int* __restrict__ list, const int* __restrict__ list_len) {
  __shared__ int mk[kSrWarps][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nrows = list ? *list_len : n;
  for (int wi = blockIdx.x * kSrWarps + wp; wi < nrows; wi += gridDim.x * kSrWarps) {
    const int u = list ? list[wi] : wi;
    // independent loads first
    const int vu = vinfo[u];
    const int b = (int)rp[u], e = (int)rp[u + 1];
    if (vu & kMovedBit) continue;
    const int g = vu;
    const int genr = gen[g], kp = kcnt[g];
    const long long out = rp2[g];
    if (genr) continue;
    int mv = INT_MAX;
    WT mw = 0;
    if (lane < kp) {
      mv = side_v[b + lane];
      mw = side_w[b + lane];
    }
    __syncwarp();  // the previous row's reads of mk are done
    mk[wp][lane] = mv;
    __syncwarp();
    int clean_before = 0, cless = 0;
    long long dsum = 0;
    for (int base = b; base < e; base += 32 * kSrUnroll) {
      int vp[kSrUnroll];
      WT c[kSrUnroll];
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) {
        const int idx = base + 32 * j + lane;
        vp[j] = idx < e ? col[idx] : 0;
        c[j] = idx < e ? w[idx] : WT(0);
      }
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) vp[j] = base + 32 * j + lane < e ? vinfo[vp[j]] : 0;
  #pragma unroll
      for (int j = 0; j < kSrUnroll; ++j) {
        const bool valid = base + 32 * j + lane < e;
        const bool moved = valid && (vp[j] & kMovedBit);
        vp[j] &= ~kMovedBit;
        dsum += (long long)c[j];
        const bool cl = valid && !moved;
        const unsigned bal = __ballot_sync(FULL, cl);
        if (cl) {
          int lo = 0, hi = kp;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (mk[wp][mid] < vp[j]) lo = mid + 1; else hi = mid;
          }
          const long long pos = out + clean_before + __popc(bal & lanemask_lt()) + lo;
          col2[pos] = vp[j];
          w2[pos] = c[j];
        }
        for (int t = 0; t < kp; ++t) {
          const unsigned bt = __ballot_sync(FULL, cl && vp[j] < mk[wp][t]);
          if (lane == t) cless += __popc(bt);
        }
        clean_before += __popc(bal);
      }
    }
    if (lane < kp) {
      const long long pos = out + lane + cless;
      col2[pos] = mv;
      w2[pos] = mw;
    }
    dsum = warp_sum(dsum);
    if (lane == 0) deg2[g] = (WT)dsum;
  }
}

// General rows: copy from the general CSR (rows of non-general groups are
// empty there) to their place; their degrees by segmented sums.
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    gen_copy_kernel(int n2, long long NG, const int64_t* __restrict__ rpG,
                    const int* __restrict__ colG, const WT* __restrict__ wG,
                    const int* __restrict__ tile_row, int ntiles,
                    const int64_t* __restrict__ rp2, int* __restrict__ col2, WT* __restrict__ w2,
                    WT* __restrict__ deg2) {
  __shared__ TileRowsSmem tr;
  tile_rows_load(tr, rpG, n2, tile_row, ntiles, blockIdx.x);
  const long long e0 = (long long)blockIdx.x * kET;
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    const bool valid = e < NG;
    int g = 0;
    WT c = 0;
    if (valid) {
      g = tile_row_of(tr, rpG, e);
      c = wG[e];
      const long long dst = rp2[g] + (e - rpG[g]);
      col2[dst] = colG[e];
      w2[dst] = c;
    }
    warp_segment_add<long long, WT>(g, g, (long long)c, valid, deg2);
  }
}


// ------------------------------------------------------------------ flat rows
// Entry-tiled form of the singleton-row rebuild, for large graphs.  A
// singleton row u (group g = L[u]) holds clean entries (neighbour a single
// vertex: label order kept) and moved entries (neighbour in a multi-member
// group G).  Its contracted moved entries (G, sum of w(u, y) over y in G) are,
// by the symmetry of the graph, exactly the entries (G, g) of the contracted
// rows of the multi-member groups, which the general (sorted) and dense
// (accumulator) paths build anyway: they are transposed into the row's own
// span of the side arrays (side_v / side_w at rp[u] ..., kp of them), sorted
// by G, and merged with the clean entries:
//   clean entry of rank k (among the row's clean entries), label l:
//     position base + k + #{j : G_j < l}
//   moved entry j: position base + j + #{clean entries with label < G_j}
// The second count is a histogram over the first one (side_c[rp[u] + b] =
// clean entries with exactly b moved labels below), summed by the writer.
// The tiles are the round's entry tiles (kET consecutive entries per block,
// tile_row = row of a tile's first entry); each thread owns a run of
// kETItems consecutive entries, so that its loads are whole 16-byte vectors
// and every lane works whatever the row lengths.  Clean ranks of a row that
// crosses tile boundaries continue from the tiles before: the counting pass
// stores per tile the clean entries of its first row (x) and last row (y).

constexpr int kTsortWarp = 32;     // moved labels a warp sorts in registers
constexpr int kStage = 32 * kETItems + kETItems;  // staging slots per warp of the writing pass
constexpr int kTsortBlock = 1024;  // threads of the block sort (up to kSrMaxRow labels)

// The row offsets an entry tile covers, in shared memory, for tiles of up to
// kFlatRows rows (the others search the global row offsets).  Offsets are
// below 2^31 (the entry count's limit).
constexpr int kFlatRows = 512;
struct FlatRowsSmem {
  int rp[kFlatRows + 2];
  int r0, r1, use;
};

// Loads them (without a first barrier: every thread reads the tile's row
// range itself).
__device__ __forceinline__ void tile_rows_load1(FlatRowsSmem& s, const int64_t* rp, int n,
                                                const int* tile_row, int ntiles, int t, int& r0,
                                                int& r1, bool& use) {
  r0 = tile_row[t];
  r1 = (t + 1 < ntiles) ? tile_row[t + 1] : n - 1;
  use = (r1 - r0 + 2) <= (kFlatRows + 2);
  if (threadIdx.x == 0) {
    s.r0 = r0;
    s.r1 = r1;
    s.use = use;
  }
  if (use)
    for (int i = threadIdx.x; i < r1 - r0 + 2; i += blockDim.x) s.rp[i] = (int)rp[r0 + i];
  __syncthreads();
}

__device__ __forceinline__ int tile_row_of(const FlatRowsSmem& s, const int64_t* rp, long long e) {
  return s.use ? s.r0 + row_in(s.rp, 0, s.r1 - s.r0 + 1, e) : row_in(rp, s.r0, s.r1 + 1, e);
}

__device__ __forceinline__ long long tile_rp(const FlatRowsSmem& s, const int64_t* rp, int r) {
  return s.use ? (long long)s.rp[r - s.r0] : (long long)rp[r];
}

// A thread's run of cnt <= kETItems column indices from eb (16-byte vector
// loads when whole and aligned).
__device__ __forceinline__ void load_col_run(const int* __restrict__ col, long long eb, int cnt,
                                             int (&c)[kETItems]) {
  if (cnt == kETItems && (reinterpret_cast<uintptr_t>(col) & 15) == 0) {
    const int4* cp = reinterpret_cast<const int4*>(col + eb);
    const int4 a = cp[0], b = cp[1];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < kETItems; ++k) c[k] = k < cnt ? col[eb + k] : 0;
  }
}

// Sum over the lanes of `peers` (all holding the same key).
template <typename T>
__device__ __forceinline__ T peer_sum(unsigned peers, T v) {
  if (sizeof(T) == 4) return (T)__reduce_add_sync(peers, (unsigned)v);
  T t = 0;
  for (unsigned m = peers; m; m &= m - 1) t += __shfl_sync(peers, v, __ffs(m) - 1);
  return t;
}

// Compact vertex map of the flat path, small enough to stay in L1 where the
// per-vertex words (4 bytes each) do not: per 32 consecutive vertices x0 ..
//   vmap.x  bit i: vertex x0 + i lies in a multi-member group (moved)
//   vmap.y  bit i: x0 + i is not its group's union-find root
//   vmap.z  vertices below x0 that are not roots
// and mvbits = vmap.x alone.  A single vertex y is a root, and its label (the
// rank of its root among the roots) is y - vmap.z - popc(vmap.y below y).
// It also clears the counters of the flat path (fcl, kpc: n; tile_ht:
// ntiles; list_len: 2).
__global__ void fr_vmap_kernel(int n, const int* __restrict__ vinfo,
                               const int* __restrict__ root_flags,
                               const int* __restrict__ root_rank, int4* __restrict__ vmap,
                               unsigned* __restrict__ mvbits, int* __restrict__ fcl,
                               int* __restrict__ kpc, int2* __restrict__ tile_ht, int ntiles,
                               int* __restrict__ list_len) {
  const int lane = threadIdx.x & 31;
  const int nw = (n + 31) >> 5;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    fcl[i] = 0;
    kpc[i] = 0;
    if (i < ntiles) tile_ht[i] = make_int2(0, 0);
    if (i < 2) list_len[i] = 0;
  }
  for (int i = n + blockIdx.x * blockDim.x + threadIdx.x; i < ntiles;
       i += gridDim.x * blockDim.x)
    tile_ht[i] = make_int2(0, 0);
  for (int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nw;
       wi += (gridDim.x * blockDim.x) >> 5) {
    const int x = (wi << 5) + lane;
    const bool in = x < n;
    const unsigned mv = __ballot_sync(FULL, in && (vinfo[x] & kMovedBit));
    const unsigned nm = __ballot_sync(FULL, in && root_flags[x] == 0);
    if (lane == 0) {
      const int x0 = wi << 5;
      vmap[wi] = make_int4((int)mv, (int)nm, x0 - root_rank[x0], 0);
      mvbits[wi] = mv;
    }
  }
}

__device__ __forceinline__ bool fr_moved(const unsigned* __restrict__ mvbits, int y) {
  return (__ldg(&mvbits[y >> 5]) >> (y & 31)) & 1u;
}

// Counting pass: clean entries of every row (fcl, zeroed before) and of each
// tile's first and last row (tile_ht, zeroed before).  A thread finds the row
// boundaries inside its run once; a row's clean entries in the run are the
// popcount of the clean mask over its segment.
__global__ void __launch_bounds__(kETThreads)
    fr_count_kernel(int n, long long M, const int64_t* __restrict__ rp,
                    const int* __restrict__ col, const unsigned* __restrict__ mvbits,
                    const int* __restrict__ tile_row, int ntiles, int* __restrict__ fcl,
                    int2* __restrict__ tile_ht) {
  __shared__ FlatRowsSmem tr;
  const int t = blockIdx.x;
  const long long e0 = (long long)t * kET;
  const long long eend = min(M, e0 + kET);
  const long long eb = e0 + (long long)threadIdx.x * kETItems;
  const int cnt = (int)max(0LL, min((long long)kETItems, eend - eb));
  // the entry loads and the neighbour gathers need no row: issued first
  int c[kETItems];
  load_col_run(col, eb, cnt, c);
  unsigned cm = 0;
#pragma unroll
  for (int k = 0; k < kETItems; ++k)
    if (k < cnt && !fr_moved(mvbits, c[k])) cm |= 1u << k;
  int r0, r1;
  bool use;
  tile_rows_load1(tr, rp, n, tile_row, ntiles, t, r0, r1, use);
  // the tile's last row (one search per warp)
  int rlast = 0;
  if ((threadIdx.x & 31) == 0) rlast = tile_row_of(tr, rp, eend - 1);
  rlast = __shfl_sync(FULL, rlast, 0);
  int ra = -1, rb = -1, ca = 0, cb = 0;
  if (cnt > 0) {
    int r = tile_row_of(tr, rp, eb);
    long long nx = tile_rp(tr, rp, r + 1);
    int k0 = 0;
    for (;;) {
      const int k1 = nx - eb < cnt ? (int)(nx - eb) : cnt;
      const int cc = __popc(cm & ((1u << k1) - 1u) & ~((1u << k0) - 1u));
      if (k0 == 0) {
        ra = r;
        ca = cc;
      } else if (k1 < cnt) {
        if (cc) fcl[r] = cc;  // a whole row inside the run
      } else {
        rb = r;
        cb = cc;
      }
      if (k1 >= cnt) break;
      k0 = k1;
      do {
        ++r;
        nx = tile_rp(tr, rp, r + 1);
      } while (nx <= eb + k0);  // (empty rows)
    }
  }
  // the first and last row of each run: one atomic per row and warp
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = h ? rb : ra;
    const unsigned peers = __match_any_sync(FULL, r);
    const unsigned s = __reduce_add_sync(peers, (unsigned)(h ? cb : ca));
    if (r >= 0 && s && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&fcl[r], (int)s);
  }
  int hcnt = (ra == r0 ? ca : 0) + (rb == r0 ? cb : 0);
  int tcnt = (ra == rlast ? ca : 0) + (rb == rlast ? cb : 0);
  hcnt = (int)__reduce_add_sync(FULL, (unsigned)hcnt);
  tcnt = (int)__reduce_add_sync(FULL, (unsigned)tcnt);
  if ((threadIdx.x & 31) == 0) {
    if (hcnt) atomicAdd(&tile_ht[t].x, hcnt);
    if (tcnt) atomicAdd(&tile_ht[t].y, tcnt);
  }
}

// The general CSR's rows of multi-member groups, transposed (entry tiles of
// the general CSR).  The gathers of a thread's entries go out together, one
// level at a time (column, then its member and group state, then the
// member's row offsets and the slot).
template <typename WT>
__global__ void __launch_bounds__(kETThreads)
    fr_fill_kernel(int n2, long long NG, const int64_t* __restrict__ rpG,
                   const int* __restrict__ colG, const WT* __restrict__ wG,
                   const int* __restrict__ tile_rowG, int ntiles, const int64_t* __restrict__ rp,
                   const int* __restrict__ rep, const int* __restrict__ gen,
                   int* __restrict__ kpc, int* __restrict__ side_v, WT* __restrict__ side_w) {
  __shared__ FlatRowsSmem tr;
  int r0, r1;
  bool use;
  tile_rows_load1(tr, rpG, n2, tile_rowG, ntiles, blockIdx.x, r0, r1, use);
  const long long e0 = (long long)blockIdx.x * kET;
  int G[kETItems], c[kETItems], u[kETItems];
  WT W[kETItems];
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    const long long e = e0 + i * kETThreads + threadIdx.x;
    G[i] = -1;
    c[i] = 0;
    W[i] = 0;
    if (e < NG) {
      G[i] = tile_row_of(tr, rpG, e);
      c[i] = colG[e];
      W[i] = wG[e];
    }
  }
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    u[i] = -1;
    // a single vertex's general row holds clean entries only
    if (G[i] >= 0 && rep[G[i]] < 0) {
      const int m = rep[c[i]];
      if (m >= 0 && gen[c[i]] == 0) u[i] = m;
    }
  }
#pragma unroll
  for (int i = 0; i < kETItems; ++i) {
    if (u[i] < 0) continue;
    const long long b = rp[u[i]];
    const long long len = rp[u[i] + 1] - b;
    const int slot = atomicAdd(&kpc[c[i]], 1);
    // (the slot stays inside the row's span: a row has at least as many
    // entries as moved labels)
    if (slot < len) {
      side_v[b + slot] = G[i];
      side_w[b + slot] = W[i];
    }
  }
}

// Per row of the flat path: len = clean + moved labels; the histogram slots
// cleared; rows with several moved labels listed for sorting (list[0 ..) up
// to kTsortWarp labels, list[n - 1] downwards above).
__global__ void fr_finalize_kernel(int n, const int64_t* __restrict__ rp,
                                   const int* __restrict__ vinfo, const int* __restrict__ gen,
                                   const int* __restrict__ fcl, const int* __restrict__ kpc,
                                   int* __restrict__ len, int* __restrict__ side_c,
                                   int* __restrict__ list, int* __restrict__ list_len, int n2,
                                   const int64_t* __restrict__ rpG) {
  const int lane = threadIdx.x & 31;
  // the general rows' lengths (from the general CSR)
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n2; g += gridDim.x * blockDim.x)
    if (gen[g] == 1) len[g] = (int)(rpG[g + 1] - rpG[g]);
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int u = base + threadIdx.x;
    int kind = 0;  // 1: warp sort, 2: block sort
    if (u < n) {
      const int v = vinfo[u];
      if (!(v & kMovedBit) && gen[v] == 0) {
        const long long b = rp[u];
        const int kp = (int)min((long long)kpc[v], rp[u + 1] - b);
        len[v] = fcl[u] + kp;
        for (int j = 0; j < kp; ++j) side_c[b + j] = 0;
        kind = kp < 2 ? 0 : kp <= kTsortWarp ? 1 : 2;
      }
    }
#pragma unroll
    for (int k = 1; k <= 2; ++k) {
      const unsigned bm = __ballot_sync(FULL, kind == k);
      if (!bm) continue;
      int at = 0;
      if (lane == __ffs(bm) - 1) at = atomicAdd(&list_len[k - 1], __popc(bm));
      at = __shfl_sync(FULL, at, __ffs(bm) - 1) + __popc(bm & lanemask_lt());
      if (kind == k) list[k == 1 ? at : n - 1 - at] = u;
    }
  }
}

// Sorts the moved list of each listed row with 2..kTsortWarp labels (one warp
// per row; the labels are distinct).
template <typename WT>
__global__ void fr_tsort_warp_kernel(const int64_t* __restrict__ rp, const int* __restrict__ vinfo,
                                     const int* __restrict__ kpc, const int* __restrict__ list,
                                     const int* __restrict__ list_len, int* __restrict__ side_v,
                                     WT* __restrict__ side_w) {
  const int lane = threadIdx.x & 31;
  const int nrows = list_len[0];
  for (int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nrows;
       wi += (gridDim.x * blockDim.x) >> 5) {
    const int u = list[wi];
    const long long b = rp[u];
    const int kp = (int)min((long long)kpc[vinfo[u]], rp[u + 1] - b);
    int G = INT_MAX;
    WT W = 0;
    if (lane < kp) {
      G = side_v[b + lane];
      W = side_w[b + lane];
    }
    int rank = 0;
    for (int j = 0; j < kp; ++j) rank += __shfl_sync(FULL, G, j) < G ? 1 : 0;
    __syncwarp();
    if (lane < kp) {
      side_v[b + rank] = G;
      side_w[b + rank] = W;
    }
  }
}

// The same for rows with more than kTsortWarp labels (at most kSrMaxRow): one
// block per row, bitonic sort in shared memory.
template <typename WT>
__global__ void __launch_bounds__(kTsortBlock)
    fr_tsort_block_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ vinfo,
                          const int* __restrict__ kpc, const int* __restrict__ list,
                          const int* __restrict__ list_len, int* __restrict__ side_v,
                          WT* __restrict__ side_w) {
  __shared__ int sk[kSrMaxRow];
  __shared__ WT sw[kSrMaxRow];
  const int nrows = list_len[1];
  for (int wi = blockIdx.x; wi < nrows; wi += gridDim.x) {
    const int u = list[n - 1 - wi];
    const long long b = rp[u];
    const int kp = (int)min(min((long long)kpc[vinfo[u]], rp[u + 1] - b), (long long)kSrMaxRow);
    int P = 1;
    while (P < kp) P <<= 1;
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      sk[i] = i < kp ? side_v[b + i] : INT_MAX;
      sw[i] = i < kp ? side_w[b + i] : WT(0);
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int p = i ^ j;
          if (p > i) {
            const bool up = (i & k) == 0;
            if ((sk[i] > sk[p]) == up) {
              const int tk = sk[i];
              sk[i] = sk[p];
              sk[p] = tk;
              const WT tw = sw[i];
              sw[i] = sw[p];
              sw[p] = tw;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < kp; i += blockDim.x) {
      side_v[b + i] = sk[i];
      side_w[b + i] = sw[i];
    }
  }
}

// Per row: the flat path's record {base = rp2[g] (-1: not flat; entries are
// below 2^31), kp, first moved label, g}.
struct __align__(16) FlatRec {
  int base;
  int kp;
  int g0;
  int g;
};

__global__ void fr_rowrec_kernel(int n, const int64_t* __restrict__ rp,
                                 const int* __restrict__ vinfo, const int* __restrict__ gen,
                                 const int* __restrict__ kpc, const int* __restrict__ side_v,
                                 const int* __restrict__ off, const int* __restrict__ total,
                                 int n2, int64_t* __restrict__ rp2, FlatRec* __restrict__ rec) {
  // the new row offsets (exclusive scan of the lengths, then the total)
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= n2; g += gridDim.x * blockDim.x)
    rp2[g] = g < n2 ? (int64_t)off[g] : (int64_t)*total;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const int v = vinfo[u];
    FlatRec o;
    o.base = -1;
    o.kp = 0;
    o.g0 = INT_MAX;
    o.g = v & ~kMovedBit;
    if (!(v & kMovedBit) && gen[v] == 0) {
      const long long b = rp[u];
      o.base = off[v];
      o.kp = (int)min((long long)kpc[v], rp[u + 1] - b);
      if (o.kp > 0) o.g0 = side_v[b];
    }
    rec[u] = o;
  }
}

// Exclusive scan over the block's threads, in order, of (brk, cnt) pairs
// under (a, b) -> b.brk ? b : (a.brk, a.cnt + b.cnt): the clean entries since
// the last row start before a thread's run.
__device__ __forceinline__ void seg_scan_block(int brk, int cnt, int* s_wb, int* s_wc,
                                               int& pbrk, int& pcnt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int b = brk, c = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int qb = __shfl_up_sync(FULL, b, o), qc = __shfl_up_sync(FULL, c, o);
    if (lane >= o && !b) {
      b = qb;
      c += qc;
    }
  }
  if (lane == 31) {
    s_wb[wid] = b;
    s_wc[wid] = c;
  }
  int xb = __shfl_up_sync(FULL, b, 1), xc = __shfl_up_sync(FULL, c, 1);
  if (lane == 0) xb = xc = 0;
  __syncthreads();
  int wb = 0, wc = 0;
  for (int k = 0; k < wid; ++k) {
    if (s_wb[k]) {
      wb = 1;
      wc = s_wc[k];
    } else {
      wc += s_wc[k];
    }
  }
  if (xb) {
    pbrk = 1;
    pcnt = xc;
  } else {
    pbrk = wb;
    pcnt = wc + xc;
  }
}

// Writing pass: the clean entries of flat rows at their positions, the row
// weights (deg2, zeroed before) and the histogram side_c.  Per run, the row
// boundaries are found once; within a row the moved labels below the current
// clean label advance monotonically (the clean labels of a row ascend).
template <typename WT>
__global__ void __launch_bounds__(kETThreads, sizeof(WT) == 4 ? 5 : 4)
    fr_write_kernel(int n, long long M, const int64_t* __restrict__ rp,
                    const int* __restrict__ col, const WT* __restrict__ w,
                    const int* __restrict__ vinfo, const int4* __restrict__ vmap,
                    const int* __restrict__ tile_row, int ntiles,
                    const FlatRec* __restrict__ rec, const int* __restrict__ fcl,
                    const int2* __restrict__ tile_ht, const int* __restrict__ side_v,
                    int* __restrict__ side_c, int* __restrict__ col2, WT* __restrict__ w2,
                    WT* __restrict__ deg2) {
  __shared__ FlatRowsSmem tr;
  __shared__ int s_wb[kETThreads / 32], s_wc[kETThreads / 32];
  // output staging of each warp (positions, labels, weights of its 256
  // entries; slot q + q / 32 for entry q, free of bank conflicts both ways)
  extern __shared__ __align__(16) unsigned char fr_stage[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* s_pos = reinterpret_cast<int*>(fr_stage) + wid * kStage;
  int* s_lab = reinterpret_cast<int*>(fr_stage) + (kETThreads / 32 + wid) * kStage;
  const int t = blockIdx.x;
  const long long e0 = (long long)t * kET;
  const long long eend = min(M, e0 + kET);
  const long long eb = e0 + (long long)threadIdx.x * kETItems;
  const int cnt = (int)max(0LL, min((long long)kETItems, eend - eb));
  int c[kETItems];
  WT x[kETItems];
  load_run<WT>(col, w, eb, cnt, c, x);
  const int q0 = lane * kETItems + (lane >> 2);  // staging slot of entry 0 of the run
  unsigned cm = 0;
#pragma unroll
  for (int k = 0; k < kETItems; ++k) {
    // c[] becomes the neighbours' labels (of single vertices; -1 for moved)
    const int y = c[k];
    const int4 v = k < cnt ? __ldg(&vmap[y >> 5]) : make_int4(-1, 0, 0, 0);
    const int bit = y & 31;
    if (((unsigned)v.x >> bit) & 1u) {
      c[k] = -1;
    } else {
      c[k] = y - v.z - __popc((unsigned)v.y & ((1u << bit) - 1u));
      cm |= 1u << k;
    }
  }
  int r0, r1;
  bool use;
  tile_rows_load1(tr, rp, n, tile_row, ntiles, t, r0, r1, use);
  // row boundaries inside the run (bit k: entry k starts a row)
  int r = 0;
  unsigned sm = 0;
  if (cnt > 0) {
    r = tile_row_of(tr, rp, eb);
    if (tile_rp(tr, rp, r) == eb) sm = 1u;
    long long p = tile_rp(tr, rp, r + 1);
    int q = r;
    while (p < eb + cnt) {
      sm |= 1u << (int)(p - eb);
      ++q;
      p = tile_rp(tr, rp, q + 1);
    }
  }
  const int brk = sm != 0;
  const int hi_start = brk ? 31 - __clz(sm) : 0;
  int pbrk, pcnt;
  seg_scan_block(brk, __popc(cm & ~((1u << hi_start) - 1u)), s_wb, s_wc, pbrk, pcnt);
  int running = 0;
  if (!pbrk) {
    // clean entries of the tile's first row in the tiles before (a flat row
    // has at most kSrMaxRow entries: it spans at most three tiles)
    const long long s0 = tile_rp(tr, rp, r0);
    int carry = 0;
    if (s0 < e0 && tile_rp(tr, rp, r0 + 1) - s0 <= kSrMaxRow) {
      const int ts = (int)(s0 / kET);
      carry = tile_ht[ts].y;
      for (int u = ts + 1; u < t; ++u) carry += tile_ht[u].x;
    }
    running = pcnt + carry;
  } else {
    running = pcnt;
  }
  int ra = -1, rb = -1, ga = 0, gb = 0;
  WT da = 0, db = 0;
  if (cnt > 0) {
#pragma unroll
    for (int k = 0; k < kETItems; ++k) s_pos[q0 + k] = -1;
    int k0 = 0;
    for (;;) {
      // segment [k0, k1) of row r
      unsigned rest = sm & ~((2u << k0) - 1u);
      const int k1 = rest ? __ffs(rest) - 1 : cnt;
      const unsigned seg = ((1u << k1) - 1u) & ~((1u << k0) - 1u);
      if ((sm >> k0) & 1u) running = 0;
      const FlatRec f = rec[r];
      WT dc = 0;
      if (f.base >= 0) {
        const long long rs = tile_rp(tr, rp, r);
        const int nc = fcl[r];
        int b = 0, nextG = f.g0, hn = 0;  // moved labels below; the next one; histogram run
#pragma unroll
        for (int k = 0; k < kETItems; ++k) {
          if ((seg >> k) & 1u) {
            dc += x[k];
            if ((cm >> k) & 1u) {
              const int l = c[k];
              while (l > nextG) {
                if (hn) atomicAdd(&side_c[rs + b], hn);
                hn = 0;
                ++b;
                nextG = b < f.kp ? side_v[rs + b] : INT_MAX;
              }
              if (running < nc) {  // (the count bounds every rank)
                s_pos[q0 + k] = f.base + running + b;  // (entries < 2^31)
                s_lab[q0 + k] = l;
                hn += b < f.kp ? 1 : 0;
              }
              ++running;
            }
          }
        }
        if (hn) atomicAdd(&side_c[rs + b], hn);
      } else {
        running += __popc(cm & seg);
      }
      const int g = f.g;
      if (k0 == 0) {
        ra = f.base >= 0 ? r : -1;
        ga = g;
        da = dc;
      } else if (k1 < cnt) {
        if (f.base >= 0 && dc) deg2[g] = dc;  // a whole row inside the run
      } else {
        rb = f.base >= 0 ? r : -1;
        gb = g;
        db = dc;
      }
      if (k1 >= cnt) break;
      k0 = k1;
      long long nx = tile_rp(tr, rp, r + 1);
      while (nx <= eb + k0) {  // the row that starts at entry k0 (empty rows skipped)
        ++r;
        nx = tile_rp(tr, rp, r + 1);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < kETItems; ++k) s_pos[q0 + k] = -1;
  }
  // the staged entries, 32 consecutive ones per store instruction (their
  // weights read again in that order)
  __syncwarp();
  const long long ew = e0 + (long long)wid * 32 * kETItems + lane;
#pragma unroll
  for (int j = 0; j < kETItems; ++j) {
    const int q = j * 32 + lane + j;
    const int p = s_pos[q];
    if (p >= 0) {
      col2[p] = s_lab[q];
      w2[p] = w[ew + 32 * j];
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rr = h ? rb : ra;
    const unsigned peers = __match_any_sync(FULL, rr);
    const WT d = peer_sum<WT>(peers, h ? db : da);
    if (rr >= 0 && d && lane == __ffs(peers) - 1) atomic_add_w(&deg2[h ? gb : ga], d);
  }
}

// The moved entries of the flat rows: blocks below `split` take the rows
// with one moved label (one thread per row); the others the listed rows with
// several (one warp per row; the clean entries below label j are the
// histogram's bins 0 .. j).
template <typename WT>
__global__ void fr_moved_kernel(int n, const int64_t* __restrict__ rp,
                                const FlatRec* __restrict__ rec, const int* __restrict__ list,
                                const int* __restrict__ list_len, const int* __restrict__ side_v,
                                const WT* __restrict__ side_w, const int* __restrict__ side_c,
                                int* __restrict__ col2, WT* __restrict__ w2, int split) {
  if ((int)blockIdx.x < split) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += split * blockDim.x) {
      const FlatRec f = rec[u];
      if (f.base < 0 || f.kp != 1) continue;
      const long long b = rp[u];
      const long long pos = (long long)f.base + side_c[b];
      col2[pos] = side_v[b];
      w2[pos] = side_w[b];
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int na = list_len[0], nrows = na + list_len[1];
  const int nb = (int)gridDim.x - split;
  for (int wi = (((int)blockIdx.x - split) * blockDim.x + threadIdx.x) >> 5; wi < nrows;
       wi += (nb * blockDim.x) >> 5) {
    const int u = wi < na ? list[wi] : list[n - 1 - (wi - na)];
    const FlatRec f = rec[u];
    const long long b = rp[u];
    int carry = 0;
    for (int j0 = 0; j0 < f.kp; j0 += 32) {
      const int j = j0 + lane;
      int h = j < f.kp ? side_c[b + j] : 0;
      int incl = h;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      if (j < f.kp) {
        const long long pos = (long long)f.base + j + carry + incl;
        col2[pos] = side_v[b + j];
        w2[pos] = side_w[b + j];
      }
      carry += __shfl_sync(FULL, incl, 31);
    }
  }
}

}  // namespace

cudaError_t rows_classify(int n, int n2, const int64_t* rp, const int* L, const RowScratch& rs,
                          cudaStream_t s, int* launches) {
  cudaMemsetAsync(rs.cnt, 0, (size_t)n2 * sizeof(int), s);
  cudaMemsetAsync(rs.gen, 0, (size_t)n2 * sizeof(int), s);
  cudaMemsetAsync(rs.single_entries, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(rs.dsum, 0, (size_t)n2 * sizeof(int), s);
  group_count_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(L, n, rs.cnt);
  single_entries_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(rp, L, n, rs.cnt, rs.gen, rs.vinfo,
                                                            rs.rep, rs.dsum, rs.single_entries);
  *launches += 2;
  return cudaGetLastError();
}

int dense_capacity(int n2, const RowScratch& rs) {
  return (int)std::min<long long>(n2, rs.dense_slots / std::max(n2, 1));
}

cudaError_t rows_dense_mark(int n_bound, const int* n2_dev, const RowScratch& rs, cudaStream_t s,
                            int* launches) {
  cudaMemsetAsync(rs.ndense, 0, sizeof(int), s);
  cudaMemsetAsync(rs.dense_entries, 0, sizeof(unsigned long long), s);
  dense_mark_kernel<<<grid_blocks(n_bound, 256), 256, 0, s>>>(
      n2_dev, rs.dense_slots, rs.dsum, rs.gen, rs.did, rs.ndense, rs.dense_entries);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t rows_dense_accumulate(int n, long long M, int n2, const int64_t* rp, const int* col,
                                  const WT* w, const int* L, const int* tile_row,
                                  const RowScratch& rs, int ndense, WT* side_w, cudaStream_t s,
                                  int* launches) {
  const int max_dense = std::min(dense_capacity(n2, rs), ndense);
  if (max_dense <= 0 || M <= 0) return cudaGetLastError();
  const int ntiles = (int)((M + kET - 1) / kET);
  dense_acc_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, n2, rp, col, w, L, rs.gen, rs.did,
                                                     tile_row, ntiles, (WT*)rs.acc);
  dense_group_list_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(n2, rs.gen, rs.did,
                                                               rs.dense_group);
  const int nchunks = (n2 + kDenseChunk - 1) / kDenseChunk;
  dense_count_kernel<WT><<<dim3(nchunks, max_dense), 256, 0, s>>>(
      n2, (const WT*)rs.acc, rs.ndense, max_dense, rs.chunk, nchunks, rows_flat(M) ? 1 : 0,
      rs.dense_group, rp, rs.rep, rs.gen, rs.kpc, rs.side_v, side_w);
  dense_scan_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(n2, rs.gen, rs.did, rs.ndense, max_dense,
                                                         rs.chunk, nchunks, rs.len);
  *launches += 4;
  return cudaGetLastError();
}

bool rows_flat(long long M) { return M >= kFlatMinEntries; }

template <typename WT>
cudaError_t rows_count(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                       const int* L, const int* root_flags, const int* root_rank,
                       const int* tile_row, const RowScratch& rs, WT* side_w, cudaStream_t s,
                       int* launches) {
  if (!rows_flat(M)) {
    const int blocks = (n + kSrWarps - 1) / kSrWarps;
    sr_count_kernel<WT><<<blocks, kSrWarps * 32, 0, s>>>(n, rp, col, w, rs.vinfo, rs.gen, rs.len,
                                                         rs.kcnt, rs.side_v, side_w, nullptr,
                                                         nullptr);
    ++*launches;
    return cudaGetLastError();
  }
  const int ntiles = (int)((M + kET - 1) / kET);
  fr_vmap_kernel<<<grid_blocks(std::max(n, ntiles), 256), 256, 0, s>>>(
      n, rs.vinfo, root_flags, root_rank, rs.vmap, rs.mvbits, rs.fcl, rs.kpc, rs.tile_ht, ntiles,
      rs.list_len);
  fr_count_kernel<<<ntiles, kETThreads, 0, s>>>(n, M, rp, col, rs.mvbits, tile_row, ntiles,
                                                rs.fcl, rs.tile_ht);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t rows_finish(int n, long long M, int n2, const int64_t* rp, const int* col,
                        const WT* w, const int* L, const RowScratch& rs, int ndense, WT* side_w,
                        const int64_t* rpG, const int* colG, const WT* wG, long long NG,
                        const int* tile_row, int64_t* rp2, int* col2, WT* w2, WT* deg2,
                        cudaStream_t s, int* launches) {
  const bool flat = rows_flat(M);
  const int ntilesG = (int)((NG + kET - 1) / kET);
  cudaError_t err = cudaSuccess;
  if (NG > 0) {
    err = tile_rows(rpG, n2, NG, rs.tile_rowG, s, launches);
    if (err != cudaSuccess) return err;
  }
  if (flat) {
    // the moved entries of the flat rows: transposed from the general rows,
    // sorted per row
    if (NG > 0) {
      fr_fill_kernel<WT><<<ntilesG, kETThreads, 0, s>>>(n2, NG, rpG, colG, wG, rs.tile_rowG,
                                                        ntilesG, rp, rs.rep, rs.gen, rs.kpc,
                                                        rs.side_v, side_w);
      ++*launches;
    }
    fr_finalize_kernel<<<grid_blocks(std::max(n, n2), 256), 256, 0, s>>>(
        n, rp, rs.vinfo, rs.gen, rs.fcl, rs.kpc, rs.len, rs.side_c, rs.list, rs.list_len, n2,
        rpG);
    fr_tsort_warp_kernel<WT><<<num_sms() * 4, 256, 0, s>>>(rp, rs.vinfo, rs.kpc, rs.list,
                                                           rs.list_len, rs.side_v, side_w);
    fr_tsort_block_kernel<WT><<<num_sms(), kTsortBlock, 0, s>>>(n, rp, rs.vinfo, rs.kpc, rs.list,
                                                                rs.list_len, rs.side_v, side_w);
    *launches += 3;
  }
  if (!flat) {
    gen_len_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(rpG, rs.gen, n2, rs.len);
    ++*launches;
  }
  err = scan_exclusive_i32(rs.len, rs.off, n2, rs.part, rs.total, s, launches);
  if (err != cudaSuccess) return err;
  if (!flat) {
    rp_from_offsets_kernel<<<grid_blocks(n2 + 1, 256), 256, 0, s>>>(rs.off, rs.total, n2, rp2);
    ++*launches;
  }
  cudaMemsetAsync(deg2, 0, (size_t)n2 * sizeof(WT), s);
  if (!flat) {
    const int blocks = (n + kSrWarps - 1) / kSrWarps;
    sr_write_kernel<WT><<<blocks, kSrWarps * 32, 0, s>>>(n, rp, col, w, rs.vinfo, rs.gen, rs.kcnt,
                                                         rs.side_v, side_w, rp2, col2, w2, deg2,
                                                         nullptr, nullptr);
    ++*launches;
  } else {
    // the round's entry tiles: tile_row still describes the round's graph
    const int ntiles = (int)((M + kET - 1) / kET);
    FlatRec* rec = static_cast<FlatRec*>(rs.rec);
    fr_rowrec_kernel<<<grid_blocks(std::max(n, n2 + 1), 256), 256, 0, s>>>(
        n, rp, rs.vinfo, rs.gen, rs.kpc, rs.side_v, rs.off, rs.total, n2, rp2, rec);
    const size_t stage = (size_t)(kETThreads / 32) * kStage * 2 * sizeof(int);
    static bool stage_attr = false;
    if (!stage_attr) {
      cudaFuncSetAttribute(fr_write_kernel<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)stage);
      stage_attr = true;
    }
    fr_write_kernel<WT><<<ntiles, kETThreads, stage, s>>>(n, M, rp, col, w, rs.vinfo, rs.vmap,
                                                      tile_row, ntiles,
                                                      rec, rs.fcl, rs.tile_ht, rs.side_v,
                                                      rs.side_c,
                                                      col2, w2, deg2);
    const int split = grid_blocks(n, 256);
    fr_moved_kernel<WT><<<split + num_sms() * 4, 256, 0, s>>>(n, rp, rec, rs.list, rs.list_len,
                                                              rs.side_v, side_w, rs.side_c, col2,
                                                              w2, split);
    *launches += 3;
  }
  const int max_dense = std::min(dense_capacity(n2, rs), ndense);
  if (max_dense > 0) {
    const int nchunks = (n2 + kDenseChunk - 1) / kDenseChunk;
    dense_write_kernel<WT><<<dim3(nchunks, max_dense), 256, 0, s>>>(
        n2, rs.gen, rs.did, rs.ndense, max_dense, rs.chunk, nchunks, (WT*)rs.acc,
        rs.dense_group, rp2, col2, w2, deg2);
    ++*launches;
  }
  if (NG > 0) {
    gen_copy_kernel<WT><<<ntilesG, kETThreads, 0, s>>>(n2, NG, rpG, colG, wG, rs.tile_rowG,
                                                       ntilesG, rp2, col2, w2, deg2);
    ++*launches;
  }
  return cudaGetLastError();
}

#define MC_ROWS_INST(WT)                                                                         \
  template cudaError_t rows_dense_accumulate<WT>(int, long long, int, const int64_t*, const int*, \
                                                 const WT*, const int*, const int*,              \
                                                 const RowScratch&, int, WT*, cudaStream_t,      \
                                                 int*);                                           \
  template cudaError_t rows_count<WT>(int, long long, const int64_t*, const int*, const WT*,      \
                                      const int*, const int*, const int*, const int*,            \
                                      const RowScratch&, WT*, cudaStream_t, int*);               \
  template cudaError_t rows_finish<WT>(int, long long, int, const int64_t*, const int*, const WT*,\
                                       const int*, const RowScratch&, int, WT*, const int64_t*,   \
                                       const int*, const WT*, long long, const int*, int64_t*,    \
                                       int*, WT*, WT*, cudaStream_t, int*);
MC_ROWS_INST(int32_t)
MC_ROWS_INST(int64_t)
#undef MC_ROWS_INST

}  // namespace mc
