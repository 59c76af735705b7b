// batch_warp.cu -- small graphs of a batch, one warp per graph.
//
// A warp takes graphs from a work queue (largest first) and runs the whole
// of Algorithm 2 on each, its state in the warp's own scratch slot: per
// round the degree bound (Sec. 2.1), the PR1 / PR2 tests, one CAPFOREST pass
// from vertex 0 (Algorithm 1 with one process: a maximum-adjacency order
// with keys min(r(y), lambda-hat); marks where r(y) first reaches
// lambda-hat; alpha lowers the bound with the visited prefix as witness),
// the union-find of the marks and the contraction.  Of the PR tests only the
// per-edge PR1 / PR2 run: on one warp the PR3 / PR4 intersections measured
// several times the rest of a graph's solve, and the round's full pass marks
// anyway.  The contraction sums each contracted vertex's member rows into a
// dense accumulator of the new vertex count (the per-vertex dense
// accumulation of Sec. 4, parallel session (3)) and writes the row in label
// order, so the result is the same canonical CSR as every other
// contraction.  A full pass on a connected
// graph with lambda-hat > 0 marks at least one edge (its last vertex t has
// r(t) = c(t) >= lambda-hat), so every round but one whose pass lowered the
// bound shrinks the graph.
//
// Graphs of up to kBwMaxN vertices: the keys (r values, later the
// accumulator), the two-level max tree over them, the current row offsets,
// the degrees (later the labels), the group lists and the union-find live in
// the warp's shared memory; the columns, weights, visit positions and the
// map to the input vertices in its global slot.  All values are int: a
// batch's total weight is below 2^31.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace mc {

namespace {

constexpr int kBwWarps = 1;  // warps per block (each warp has its own graphs)
constexpr int kBwWarpSmemWords = kBwMaxN + (kBwMaxN + 1) + kBwMaxN + (kBwMaxN + 1) + kBwMaxN +
                                 kBwMaxN + kBwMaxN / 32 + kBwMaxN / 1024 + 32 + 1;
constexpr size_t kBwSmemBytes = (size_t)kBwWarps * kBwWarpSmemWords * sizeof(int);

__device__ __forceinline__ unsigned long long bw_warp_min(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(FULL, v, o);
    if (t < v) v = t;
  }
  return v;
}

__device__ __forceinline__ unsigned bw_key(int r, int lam) {
  // queued keys are min(r, lambda) + 1; 0 = not queued, r < 0 = visited
  return r > 0 ? (unsigned)min(r, lam) + 1u : 0u;
}

struct BwSlot {
  int* rp[2];
  int* col[2];
  int* w[2];
  int* pos;
  int* map;
};

__device__ BwSlot bw_slot(int* base, long long slot_words, int slot, int nmax, int mmax) {
  int* p = base + (long long)slot * slot_words;
  BwSlot s;
  for (int b = 0; b < 2; ++b) {
    s.rp[b] = p;
    p += nmax + 1;
    s.col[b] = p;
    p += mmax;
    s.w[b] = p;
    p += mmax;
  }
  s.pos = p;
  p += nmax;
  s.map = p;
  return s;
}

__global__ void __launch_bounds__(kBwWarps * 32)
    batch_warp_kernel(const int* __restrict__ list, int nlist, int* cursor,
                      const int* __restrict__ voff0, const int64_t* __restrict__ rp0,
                      const int* __restrict__ col0, const int* __restrict__ w0, int* scratch,
                      long long slot_words, int nmax, int mmax, uint32_t pr_mask,
                      unsigned long long* lam_g, uint8_t* side0, DevState* st) {
  // per warp, in dynamic shared memory (kBwWarpSmemWords ints each): the
  // keys (r values in a pass, then the accumulator), the current graph's row
  // offsets, its degrees (then the labels), the group counts and members,
  // the two tree levels, the row label list and count
  extern __shared__ int bw_smem[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const BwSlot S = bw_slot(scratch, slot_words, blockIdx.x * kBwWarps + wp, nmax, mmax);
  int* key = bw_smem + (long long)wp * kBwWarpSmemWords;
  int* srp = key + kBwMaxN;       // kBwMaxN + 1
  int* sdeg = srp + kBwMaxN + 1;  // kBwMaxN: degrees; labels once the pass is done
  int* lab = sdeg;
  int* scnt = sdeg + kBwMaxN;     // kBwMaxN + 1
  int* smem_members = scnt + kBwMaxN + 1;  // kBwMaxN
  int* parent = smem_members + kBwMaxN;    // kBwMaxN: the round's union-find
  unsigned* l1 = reinterpret_cast<unsigned*>(parent + kBwMaxN);  // kBwMaxN / 32
  unsigned* l2 = l1 + kBwMaxN / 32;                            // kBwMaxN / 1024
  int* tl = reinterpret_cast<int*>(l2 + kBwMaxN / 1024);       // 32
  int* tcount = tl + 32;                                       // 1
  int fail = 0;  // the first failed check: 1 rounds, 2 union-find, 3 / 4 tree descent
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(cursor, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= nlist) break;
    const int gi = list[item];
    const int v0 = voff0[gi], n0 = voff0[gi + 1] - v0;
    const long long e0 = rp0[v0];
    // the graph in local ids, buffer 0
    for (int i = lane; i <= n0; i += 32) S.rp[0][i] = (int)(rp0[v0 + i] - e0);
    const int m0 = (int)(rp0[v0 + n0] - e0);
    for (int e = lane; e < m0; e += 32) {
      S.col[0][e] = col0[e0 + e] - v0;
      S.w[0][e] = w0[e0 + e];
    }
    for (int i = lane; i < n0; i += 32) {
      S.map[i] = i;
      side0[v0 + i] = 0;
    }
    __syncwarp();
    long long lam = kInf;
    int n = n0, cur = 0;
    for (int round = 0;; ++round) {
      if (round > 2 * n0 + 8) {  // cannot happen (see the header); reported, not looped on
        fail = fail ? fail : 1;
        break;
      }
      // the current graph's row offsets into shared memory
      for (int i = lane; i <= n; i += 32) srp[i] = S.rp[cur][i];
      __syncwarp();
      const int* rp = srp;
      const int* col = S.col[cur];
      const int* w = S.w[cur];
      // ---- degree bound
      unsigned long long best = ~0ull;
      for (int v = lane; v < n; v += 32) {
        int d = 0;
        for (int e = rp[v]; e < rp[v + 1]; ++e) d += w[e];
        sdeg[v] = d;
        const unsigned long long k = ((unsigned long long)(unsigned)d << 32) | (unsigned)v;
        if (k < best) best = k;
      }
      best = bw_warp_min(best);
      __syncwarp();
      if (n >= 2 && (long long)(best >> 32) < lam) {
        lam = (long long)(best >> 32);
        const int x = (int)(best & 0xffffffffull);
        for (int i = lane; i < n0; i += 32) side0[v0 + i] = S.map[i] == x ? 1 : 0;
      }
      if (n <= 2 || lam == 0) break;
      // ---- PR1 / PR2, one lane per row, each edge once (u < v)
      for (int v = lane; v < n; v += 32) parent[v] = v;
      __syncwarp();
      if (pr_mask) {
        for (int u = lane; u < n; u += 32) {
          const int bu = rp[u], eu = rp[u + 1], du = sdeg[u];
          for (int e = bu; e < eu; ++e) {
            const int v = col[e];
            if (v <= u) continue;
            const int c = w[e], dv = sdeg[v];
            const bool f = ((pr_mask & 1u) && c >= lam) ||
                           ((pr_mask & 2u) && ((long long)du < 2ll * c || (long long)dv < 2ll * c));
            if (f && !uf_union(parent, u, v)) fail = fail ? fail : 2;
          }
        }
      }
      // ---- one CAPFOREST pass from vertex 0
      for (int i = lane; i < n; i += 32) {
        key[i] = 0;
        S.pos[i] = INT_MAX;
      }
      for (int i = lane; i < kBwMaxN / 32; i += 32) l1[i] = 0;
      if (lane < kBwMaxN / 1024) l2[lane] = 0;
      __syncwarp();
      int lam_p = (int)lam;  // lam <= min degree < 2^31
      int alpha = 0, best_len = -1;
      int x = 0, rx = 0;
      for (int it = 0; it < n; ++it) {
        if (it > 0) {
          const unsigned t2 = lane < kBwMaxN / 1024 ? l2[lane] : 0u;
          const unsigned m = __reduce_max_sync(FULL, t2);
          if (m == 0) break;  // nothing queued: the rest is not reachable
          const int i2 = __ffs(__ballot_sync(FULL, t2 == m)) - 1;  // m is some lane's t2
          const unsigned t1 = l1[i2 * 32 + lane];
          const unsigned b1 = __ballot_sync(FULL, t1 == m);
          if (b1 == 0) {  // a node below the maximum must hold it; checked, not trusted
            fail = fail ? fail : 3;
            break;
          }
          const int blk = i2 * 32 + (__ffs(b1) - 1);
          const int y = blk * 32 + lane;
          const int ry = y < n ? key[y] : -1;
          const unsigned b0 = __ballot_sync(FULL, bw_key(ry, lam_p) == m);
          if (b0 == 0) {
            fail = fail ? fail : 4;
            break;
          }
          const int wl = __ffs(b0) - 1;
          x = blk * 32 + wl;
          rx = __shfl_sync(FULL, ry, wl);
        }
        const int ns = it + 1;
        alpha += sdeg[x] - 2 * rx;
        if (ns < n && alpha < lam_p) {
          lam_p = alpha;
          best_len = ns;
        }
        if (lane == 0) {
          key[x] = -1;  // visited
          S.pos[x] = it;
        }
        __syncwarp();
        {  // x leaves the queue: its leaf block and the level above
          const int blk = x >> 5, y = blk * 32 + lane;
          const unsigned kb = __reduce_max_sync(FULL, bw_key(y < n ? key[y] : -1, lam_p));
          if (lane == 0) l1[blk] = kb;
          __syncwarp();
          const unsigned k2 = __reduce_max_sync(FULL, l1[(blk >> 5) * 32 + lane]);
          if (lane == 0) l2[blk >> 5] = k2;
          __syncwarp();
        }
        const int xb = rp[x], xe = rp[x + 1];
        for (int base = xb; base < xe; base += 32) {
          const int e = base + lane;
          if (e < xe) {
            const int y = col[e];
            const int r0 = key[y];
            if (r0 >= 0) {  // rows hold distinct neighbours: one lane per y
              const int r1 = r0 + w[e];
              key[y] = r1;
              if (r0 < lam_p && lam_p <= r1 && !uf_union(parent, x, y)) fail = fail ? fail : 2;
              const unsigned k = bw_key(r1, lam_p);
              atomicMax(&l1[y >> 5], k);
              atomicMax(&l2[y >> 10], k);
            }
          }
        }
        __syncwarp();
      }
      if (lam_p < lam) {
        lam = lam_p;
        for (int i = lane; i < n0; i += 32) side0[v0 + i] = S.pos[S.map[i]] < best_len ? 1 : 0;
      }
      if (lam == 0) break;
      // ---- union-find: label = rank of the root (the smallest member)
      __syncwarp();
      int n2 = 0;
      for (int base = 0; base < n; base += 32) {
        const int v = base + lane;
        const bool root = v < n && uf_find(parent, v) == v;
        const unsigned b = __ballot_sync(FULL, root);
        if (root) lab[v] = n2 + __popc(b & lanemask_lt());
        n2 += __popc(b);
      }
      __syncwarp();
      for (int v = lane; v < n; v += 32) {
        const int r = uf_find(parent, v);
        if (r != v) lab[v] = lab[r];
      }
      __syncwarp();
      if (n2 == n) continue;  // no marks (the pass lowered the bound): again, lower bound
      // ---- members of each group (counting sort by label)
      for (int g = lane; g <= n2; g += 32) scnt[g] = 0;
      __syncwarp();
      for (int v = lane; v < n; v += 32) atomicAdd(&scnt[lab[v]], 1);
      __syncwarp();
      int run = 0;  // exclusive scan of the counts
      for (int base = 0; base < n2; base += 32) {
        const int g = base + lane;
        const int c = g < n2 ? scnt[g] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += t;
        }
        if (g < n2) scnt[g] = run + incl - c;
        run += __shfl_sync(FULL, incl, 31);
      }
      __syncwarp();
      for (int v = lane; v < n; v += 32) smem_members[atomicAdd(&scnt[lab[v]], 1)] = v;
      __syncwarp();  // cnt[g] is now the end of group g's members
      // ---- contraction into the other buffer
      const int nb = cur ^ 1;
      int* rp2 = S.rp[nb];
      int* col2 = S.col[nb];
      int* w2 = S.w[nb];
      for (int i = lane; i < n2; i += 32) key[i] = 0;
      if (lane == 0) *tcount = 0;
      __syncwarp();
      int out = 0;
      for (int g = 0; g < n2; ++g) {
        const int mb = g == 0 ? 0 : scnt[g - 1], me = scnt[g];
        for (int k = mb; k < me; ++k) {
          const int m = smem_members[k];
          const int rb = rp[m], re = rp[m + 1];
          for (int base = rb; base < re; base += 32) {
            const int e = base + lane;
            if (e < re) {
              const int lv = lab[col[e]];
              if (lv != g && atomicAdd(&key[lv], w[e]) == 0) {  // weights are positive
                const int t = atomicAdd(&*tcount, 1);
                if (t < 32) tl[t] = lv;
              }
            }
          }
        }
        __syncwarp();
        const int tc = *tcount;
        if (tc <= 32) {
          // the few labels of the row, ranked among themselves
          const int my = lane < tc ? tl[lane] : INT_MAX;
          int rank = 0;
          for (int j = 0; j < tc; ++j) rank += __shfl_sync(FULL, my, j) < my ? 1 : 0;
          if (lane < tc) {
            col2[out + rank] = my;
            w2[out + rank] = key[my];
            key[my] = 0;
          }
        } else {
          // a long row: every label in order
          int o = out;
          for (int base = 0; base < n2; base += 32) {
            const int l = base + lane;
            const int val = l < n2 ? key[l] : 0;
            const unsigned b = __ballot_sync(FULL, val != 0);
            if (val != 0) {
              const int p = o + __popc(b & lanemask_lt());
              col2[p] = l;
              w2[p] = val;
              key[l] = 0;
            }
            o += __popc(b);
          }
        }
        if (lane == 0) {
          rp2[g] = out;
          *tcount = 0;
        }
        out += tc;
        __syncwarp();
      }
      if (lane == 0) rp2[n2] = out;
      for (int i = lane; i < n0; i += 32) S.map[i] = lab[S.map[i]];
      __syncwarp();
      cur = nb;
      n = n2;
      if (n2 <= 1) break;
    }
    if (lane == 0) lam_g[gi] = (unsigned long long)lam;
    __syncwarp();
  }
  if (fail) {
    atomicMax(&st->internal_code, 100 + fail);
    set_error(st, ERR_INTERNAL);
  }
}

__global__ void batch_mark_kernel(const int* __restrict__ list, int nlist, int* done_g,
                                  DevState* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlist; i += gridDim.x * blockDim.x)
    done_g[list[i]] = 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->batch_done, nlist);
}

}  // namespace

long long batch_warp_slot_words(int nmax, int mmax) {
  // two buffers of (rp, col, w), then pos, map
  return 2ll * ((long long)nmax + 1 + 2ll * mmax) + 2ll * nmax;
}

int batch_warp_block_warps() { return kBwWarps; }

bool bw_set_smem() {
  static const bool ok = cudaFuncSetAttribute(batch_warp_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kBwSmemBytes) == cudaSuccess;
  return ok;
}

int batch_warp_slots(int sms) {
  int per_sm = 0;
  if (!bw_set_smem() ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_warp_kernel, kBwWarps * 32,
                                                    kBwSmemBytes) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return std::max(1, sms) * per_sm * kBwWarps;
}

cudaError_t batch_warp_mark(const int* list, int nlist, int* done_g, DevState* st,
                            cudaStream_t s, int* launches) {
  if (nlist <= 0) return cudaSuccess;
  batch_mark_kernel<<<std::max(1, std::min(64, (nlist + 255) / 256)), 256, 0, s>>>(list, nlist,
                                                                               done_g, st);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_warp_solve(const int* list, int nlist, int* cursor, const int* voff0,
                             const int64_t* rp0, const int* col0, const int* w0, int* scratch,
                             int slots, int nmax, int mmax, uint32_t pr_mask,
                             unsigned long long* lam_g, uint8_t* side0, DevState* st,
                             cudaStream_t s, int* launches) {
  if (nlist <= 0) return cudaSuccess;
  if (nmax > kBwMaxN) return cudaErrorInvalidValue;
  cudaMemsetAsync(cursor, 0, sizeof(int), s);
  if (slots < kBwWarps || slots % kBwWarps) return cudaErrorInvalidValue;
  const int blocks = slots / kBwWarps;
  if (!bw_set_smem()) return cudaErrorInvalidValue;
  batch_warp_kernel<<<blocks, kBwWarps * 32, kBwSmemBytes, s>>>(
      list, nlist, cursor, voff0, rp0, col0, w0, scratch, batch_warp_slot_words(nmax, mmax), nmax,
      mmax, pr_mask, lam_g, side0, st);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace mc
