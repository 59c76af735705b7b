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
// and sorted, are merged in at their ranks.  Rows of multi-member groups, and
// singleton rows with more than kSrMoved distinct moved labels or more than
// kSrMaxRow entries, are "general": their entries alone go through the
// relabel / radix sort / segmented sum path, and the resulting rows are
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
                                      int* __restrict__ vinfo, int* __restrict__ dsum,
                                      unsigned long long* single_entries) {
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
      } else {
        gen[g] = 1;
        vinfo[x] = g | kMovedBit;
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
template <typename WT>
__global__ void __launch_bounds__(256)
    dense_count_kernel(int n2, const WT* __restrict__ acc, const int* ndense, int max_dense,
                       int* __restrict__ chunk, int nchunks) {
  const int d = blockIdx.y;
  if (d >= min(*ndense, max_dense)) return;
  const int c = blockIdx.x;
  const long long base = (long long)d * n2;
  int cntv = 0;
  for (int i = c * kDenseChunk + threadIdx.x; i < min(n2, (c + 1) * kDenseChunk); i += blockDim.x)
    cntv += acc[base + i] != 0;
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
                    int* __restrict__ kcnt, int* __restrict__ side_v, WT* __restrict__ side_w) {
  __shared__ int hk[kSrWarps][kSrSlots];
  __shared__ unsigned long long hs[kSrWarps][kSrSlots];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int u = blockIdx.x * kSrWarps + wp;
  if (u >= n) return;  // warp-uniform: the row kernels use no block barrier
  const int vu = vinfo[u];
  const int b = (int)rp[u], e = (int)rp[u + 1];
  if (vu & kMovedBit) return;
  const int g = vu;
  if (gen[g]) return;  // dense
  if (e - b > kSrMaxRow) {
    if (lane == 0) gen[g] = 1;
    return;
  }
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
    return;
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
                    int* __restrict__ col2, WT* __restrict__ w2, WT* __restrict__ deg2) {
  __shared__ int mk[kSrWarps][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int u = blockIdx.x * kSrWarps + wp;
  if (u >= n) return;
  // independent loads first
  const int vu = vinfo[u];
  const int b = (int)rp[u], e = (int)rp[u + 1];
  if (vu & kMovedBit) return;
  const int g = vu;
  const int genr = gen[g], kp = kcnt[g];
  const long long out = rp2[g];
  if (genr) return;
  int mv = INT_MAX;
  WT mw = 0;
  if (lane < kp) {
    mv = side_v[b + lane];
    mw = side_w[b + lane];
  }
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

}  // namespace

cudaError_t rows_classify(int n, int n2, const int64_t* rp, const int* L, const RowScratch& rs,
                          cudaStream_t s, int* launches) {
  cudaMemsetAsync(rs.cnt, 0, (size_t)n2 * sizeof(int), s);
  cudaMemsetAsync(rs.gen, 0, (size_t)n2 * sizeof(int), s);
  cudaMemsetAsync(rs.single_entries, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(rs.dsum, 0, (size_t)n2 * sizeof(int), s);
  group_count_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(L, n, rs.cnt);
  single_entries_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(rp, L, n, rs.cnt, rs.gen, rs.vinfo,
                                                            rs.dsum, rs.single_entries);
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
                                  const RowScratch& rs, cudaStream_t s, int* launches) {
  const int max_dense = dense_capacity(n2, rs);
  if (max_dense <= 0 || M <= 0) return cudaGetLastError();
  const int ntiles = (int)((M + kET - 1) / kET);
  dense_acc_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n, M, n2, rp, col, w, L, rs.gen, rs.did,
                                                     tile_row, ntiles, (WT*)rs.acc);
  const int nchunks = (n2 + kDenseChunk - 1) / kDenseChunk;
  dense_count_kernel<WT><<<dim3(nchunks, max_dense), 256, 0, s>>>(
      n2, (const WT*)rs.acc, rs.ndense, max_dense, rs.chunk, nchunks);
  dense_scan_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(n2, rs.gen, rs.did, rs.ndense, max_dense,
                                                         rs.chunk, nchunks, rs.len);
  *launches += 3;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t rows_count(int n, const int64_t* rp, const int* col, const WT* w, const int* L,
                       const RowScratch& rs, WT* side_w, cudaStream_t s, int* launches) {
  const int blocks = (n + kSrWarps - 1) / kSrWarps;
  sr_count_kernel<WT><<<blocks, kSrWarps * 32, 0, s>>>(n, rp, col, w, rs.vinfo, rs.gen, rs.len,
                                                       rs.kcnt, rs.side_v, side_w);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t rows_finish(int n, int n2, const int64_t* rp, const int* col, const WT* w,
                        const int* L, const RowScratch& rs, const WT* side_w,
                        const int64_t* rpG, const int* colG, const WT* wG, long long NG,
                        int* tile_row, int64_t* rp2, int* col2, WT* w2, WT* deg2,
                        cudaStream_t s, int* launches) {
  gen_len_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(rpG, rs.gen, n2, rs.len);
  ++*launches;
  cudaError_t err = scan_exclusive_i32(rs.len, rs.off, n2, rs.part, rs.total, s, launches);
  if (err != cudaSuccess) return err;
  rp_from_offsets_kernel<<<grid_blocks(n2 + 1, 256), 256, 0, s>>>(rs.off, rs.total, n2, rp2);
  cudaMemsetAsync(deg2, 0, (size_t)n2 * sizeof(WT), s);
  const int blocks = (n + kSrWarps - 1) / kSrWarps;
  sr_write_kernel<WT><<<blocks, kSrWarps * 32, 0, s>>>(n, rp, col, w, rs.vinfo, rs.gen, rs.kcnt,
                                                       rs.side_v, side_w, rp2, col2, w2, deg2);
  *launches += 2;
  const int max_dense = dense_capacity(n2, rs);
  if (max_dense > 0) {
    const int nchunks = (n2 + kDenseChunk - 1) / kDenseChunk;
    dense_group_list_kernel<<<grid_blocks(n2, 256), 256, 0, s>>>(n2, rs.gen, rs.did,
                                                                 rs.dense_group);
    dense_write_kernel<WT><<<dim3(nchunks, max_dense), 256, 0, s>>>(
        n2, rs.gen, rs.did, rs.ndense, max_dense, rs.chunk, nchunks, (WT*)rs.acc,
        rs.dense_group, rp2, col2, w2, deg2);
    *launches += 2;
  }
  if (NG > 0) {
    err = tile_rows(rpG, n2, NG, tile_row, s, launches);
    if (err != cudaSuccess) return err;
    const int ntiles = (int)((NG + kET - 1) / kET);
    gen_copy_kernel<WT><<<ntiles, kETThreads, 0, s>>>(n2, NG, rpG, colG, wG, tile_row, ntiles,
                                                      rp2, col2, w2, deg2);
    ++*launches;
  }
  return cudaGetLastError();
}

#define MC_ROWS_INST(WT)                                                                         \
  template cudaError_t rows_dense_accumulate<WT>(int, long long, int, const int64_t*, const int*, \
                                                 const WT*, const int*, const int*,              \
                                                 const RowScratch&, cudaStream_t, int*);         \
  template cudaError_t rows_count<WT>(int, const int64_t*, const int*, const WT*, const int*,     \
                                      const RowScratch&, WT*, cudaStream_t, int*);               \
  template cudaError_t rows_finish<WT>(int, int, const int64_t*, const int*, const WT*,           \
                                       const int*, const RowScratch&, const WT*, const int64_t*,  \
                                       const int*, const WT*, long long, int*, int64_t*, int*,    \
                                       WT*, WT*, cudaStream_t, int*);
MC_ROWS_INST(int32_t)
MC_ROWS_INST(int64_t)
#undef MC_ROWS_INST

}  // namespace mc
