// capforest.cu -- CAPFOREST edge marking (Algorithm 1; Sec. 2.1).
//
// A pass grows a visited set S in maximum-adjacency order: it repeatedly takes
// the queued vertex x of highest bounded priority Q(x) = min(r(x), lambda)
// (ties: the smaller vertex id), adds it to S, updates
// alpha += c(x) - 2 r(x) (alpha = capacity of the cut (S, V \ S)) and lowers
// lambda to alpha while S != V, then scans x's edges to unvisited y:
// if r(y) < lambda <= r(y) + c(x, y) the edge is contractible (union-find
// hook), r(y) += c(x, y), Q(y) = min(r(y), lambda).
//
// With private visit sets (private_visit = 1, Sec. 4 parallel session (1))
// no vertex is claimed: every pass is its own maximum-adjacency ordering of
// G from its start vertex, up to its table's capacity.
//
// capforest_passes: Algorithm 1 proper.  Many passes run at once, one warp
// each, from seeded start vertices; the shared visit array T is `owner`
// (a vertex is claimed by CAS, so each vertex is scanned by one pass; a pass
// that pops a vertex claimed by another pass blacklists it).  An edge whose
// far end is already claimed by another pass is skipped when scanned; that
// only removes marks (marking fewer edges is always sound) and keeps the
// pass a maximum-adjacency prefix of G minus the vertices it saw claimed.
// Each pass keeps its queue in shared memory: an open-addressing table of
// `table` slots (vertex, r, packed priority) plus one max per 32 slots.  A
// pass stops when the next vertex's row might overflow the table (stopping
// early keeps every mark valid: the marks only depend on the prefix).
//
// capforest_sequential: one pass over the whole graph by one block (the
// sequential CAPFOREST of Algorithm 2, used when the concurrent passes mark
// nothing, and the deterministic mode).  A vertex's key crosses the bound
// at most once in a pass, so its marking edge is recorded per vertex and
// hooked after the pass, off the chain of pops.  Its queue is a 32-ary max tree over
// per-vertex keys (key + 1, 0 = not queued); the descent takes the leftmost
// maximum, i.e. the smallest vertex id among the largest keys.  Keys only
// grow between pops (when alpha lowers lambda, every queued r(y) is at most
// alpha, so no key exceeds the new bound), so the tree is maintained with
// atomicMax and recomputed only along the popped vertex's path.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mc {

namespace {

int num_sms_cf() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = kDefaultSms;
  }
  return sms;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned slot_hash(int v) { return (unsigned)v * 0x9E3779B1u; }

// Packed priority: (key + 1) in the high word, ~vertex in the low word, so
// the maximum is the largest key and, among equal keys, the smallest vertex.
__device__ __forceinline__ unsigned long long pack_key(long long key, int v) {
  return ((unsigned long long)(key + 1) << 32) | (unsigned long long)(0xffffffffu - (unsigned)v);
}

// ------------------------------------------------------ concurrent passes
template <typename WT>
__global__ void cf_passes_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                                 const WT* __restrict__ w, const WT* __restrict__ deg,
                                 int* owner, int* parent, int* __restrict__ visit_log,
                                 unsigned long long* __restrict__ pass_best,
                                 int* __restrict__ pass_len, int total_passes, int table,
                                 unsigned long long seed, int* pass_counter, DevState* st,
                                 BatchView bv, int batch, int priv, long long skip_pr) {
  if (skip_pr >= 0 && (long long)*(volatile unsigned long long*)&st->marks_pr >= skip_pr) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int nsum = table >> 5;
  const size_t per_warp = (size_t)table * (sizeof(int) + sizeof(WT) + 8) + (size_t)nsum * 8;
  unsigned char* base = smem + per_warp * warp;
  unsigned long long* pk = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* summ = pk + table;
  WT* rr = reinterpret_cast<WT*>(summ + nsum);
  int* vid = reinterpret_cast<int*>(rr + table);
  volatile int* vowner = owner;
  const int load_cap = table - (table >> 3);

  unsigned long long marks_total = 0, scanned_total = 0;
  bool uf_fail = false;
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(pass_counter, 1);
    p = __shfl_sync(FULL, p, 0);
    if (p >= total_passes) break;
    // ---- reset the table
    for (int i = lane; i < table; i += 32) { vid[i] = -1; rr[i] = 0; pk[i] = 0; }
    for (int i = lane; i < nsum; i += 32) summ[i] = 0;
    __syncwarp();
    long long lam = (long long)*(volatile unsigned long long*)&st->lambda;
    // ---- start vertex: hash(seed, p), then the first unclaimed of 32 probes
    int start = -1;
    {
      const unsigned long long h = mix64(seed ^ mix64((unsigned long long)p + 1));
      const int s0 = (int)(h % (unsigned long long)n);
      if (priv) start = s0;
      for (int tries = 0; tries < 4 && start < 0; ++tries) {
        const int c = (int)(((long long)s0 + tries * 32 + lane) % n);
        const unsigned free_mask = __ballot_sync(FULL, vowner[c] == 0);
        if (free_mask) start = __shfl_sync(FULL, c, __ffs(free_mask) - 1);
      }
    }
    unsigned long long best_alpha = ~0ull;
    int best_len = 0;
    int g = 0;
    long long n_here = n;  // vertices of the graph the pass runs in
    if (batch && start >= 0) {
      g = bv.gid[start];
      if (bv.done_g[g]) {
        start = -1;
      } else {
        lam = (long long)*(volatile unsigned long long*)&bv.lam_g[g];
        n_here = bv.voff[g + 1] - bv.voff[g];
      }
    }
    unsigned long long pass_marks = 0;
    if (start >= 0 && lam > 0) {
      if (lane == 0) {
        const int h = slot_hash(start) & (table - 1);
        vid[h] = start;
        pk[h] = pack_key(0, start);
        summ[h >> 5] = pk[h];
      }
      __syncwarp();
      int count = 1, nscanned = 0;
      long long alpha = 0;
      for (int it = 0; it < table; ++it) {
        // ---- pop the maximum packed priority
        unsigned long long m = 0;
        int mchunk = -1;
        for (int c = lane; c < nsum; c += 32) {
          const unsigned long long x = summ[c];
          if (x > m) { m = x; mchunk = c; }
        }
        const unsigned long long gm = warp_max(m);
        if (gm == 0) break;
        const unsigned hit = __ballot_sync(FULL, m == gm && mchunk >= 0);
        const int chunk = __shfl_sync(FULL, mchunk, __ffs(hit) - 1);
        const int slot_l = chunk * 32 + lane;
        const unsigned own = __ballot_sync(FULL, pk[slot_l] == gm);
        if (own == 0) {  // cannot happen: summaries are exact maxima
          if (lane == 0) set_error(st, ERR_INTERNAL);
          break;
        }
        const int wl = __ffs(own) - 1;
        const int slot = chunk * 32 + wl;
        const int x = vid[slot];
        const long long rx = (long long)rr[slot];
        __syncwarp();
        if (lane == wl) pk[slot] = 0;
        __syncwarp();
        {
          const unsigned long long y = warp_max(pk[slot_l]);
          if (lane == 0) summ[chunk] = y;
        }
        __syncwarp();
        const long long rb = rp[x], re = rp[x + 1];
        if (count + (re - rb) > load_cap) break;  // the row might not fit: stop
        int claimed = 1;
        if (!priv) {
          if (lane == 0) claimed = atomicCAS(&owner[x], 0, p + 1) == 0;
          claimed = __shfl_sync(FULL, claimed, 0);
        }
        if (!claimed) continue;  // blacklisted: visited by another pass
        ++nscanned;
        if (lane == 0) visit_log[(long long)p * table + nscanned - 1] = x;
        alpha += (long long)deg[x] - 2 * rx;
        if (nscanned < n_here && alpha < lam) {
          lam = alpha;
          best_alpha = (unsigned long long)alpha;
          best_len = nscanned;
          if (lane == 0) atomicMin(batch ? &bv.lam_g[g] : &st->lambda, (unsigned long long)alpha);
        }
        // ---- scan x's edges
        for (long long b = rb; b < re; b += 32) {
          const long long e = b + lane;
          bool ins = false;
          if (e < re) {
            const int y = col[e];
            if (priv || vowner[y] == 0) {
              unsigned h = slot_hash(y) & (table - 1);
              int s = -1;
              for (int probe = 0; probe < table; ++probe) {
                const int k = vid[h];
                if (k == y) { s = h; break; }
                if (k == -1) {
                  const int prev = atomicCAS(&vid[h], -1, y);
                  if (prev == -1) { s = h; ins = true; break; }
                  if (prev == y) { s = h; break; }
                }
                h = (h + 1) & (table - 1);
              }
              // a popped slot (priority cleared) belongs to a vertex this pass
              // already took; the owner check above normally skips it
              if (s >= 0 && (ins || pk[s] != 0)) {
                const long long c = (long long)w[e];
                const long long r0 = (long long)rr[s];
                const long long r1 = r0 + c;
                rr[s] = (WT)r1;
                if (r0 < lam && lam <= r1) {
                  if (!uf_union(parent, x, y)) uf_fail = true;
                  ++marks_total;
                  ++pass_marks;
                }
                const unsigned long long np = pack_key(r1 < lam ? r1 : lam, y);
                if (np > pk[s]) pk[s] = np;
                atomicMax(&summ[s >> 5], np);
              }
            }
          }
          count += __popc(__ballot_sync(FULL, ins));
          __syncwarp();
        }
      }
      scanned_total += nscanned;
    }
    if (batch) {
      pass_marks = warp_sum(pass_marks);
      if (lane == 0) {
        if (pass_marks) atomicAdd(&bv.marks_g[g], (int)pass_marks);
        if (best_alpha != ~0ull)
          atomicMin(&bv.cf_best[g], (best_alpha << 32) | (unsigned long long)(unsigned)p);
      }
    }
    if (lane == 0) {
      pass_best[p] = best_alpha;
      pass_len[p] = best_len;
    }
  }
  if (uf_fail) set_error(st, ERR_INTERNAL);
  marks_total = warp_sum(marks_total);
  if (lane == 0) {
    if (marks_total) atomicAdd(&st->marks_cf, marks_total);
    if (scanned_total) atomicAdd((unsigned long long*)&st->claimed, scanned_total);
  }
  (void)nwarps;
}

__global__ void cf_best_kernel(const unsigned long long* __restrict__ pass_best,
                               const int* __restrict__ pass_len, int passes, DevState* st,
                               long long skip_pr) {
  __shared__ unsigned long long sv[32];
  __shared__ int sp[32];
  if (skip_pr >= 0 && (long long)*(volatile unsigned long long*)&st->marks_pr >= skip_pr) {
    // the passes were skipped: their per-pass words are stale
    if (threadIdx.x == 0) {
      st->cf_val = ~0ull;
      st->cf_pass = -1;
      st->cf_len = 0;
    }
    return;
  }
  unsigned long long bv = ~0ull;
  int bp = 0x7fffffff;
  for (int p = threadIdx.x; p < passes; p += blockDim.x) {
    const unsigned long long v = pass_best[p];
    if (v < bv || (v == bv && p < bp)) { bv = v; bp = p; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v2 = __shfl_xor_sync(FULL, bv, o);
    const int p2 = __shfl_xor_sync(FULL, bp, o);
    if (v2 < bv || (v2 == bv && p2 < bp)) { bv = v2; bp = p2; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; sp[threadIdx.x >> 5] = bp; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2)
      if (sv[w2] < bv || (sv[w2] == bv && sp[w2] < bp)) { bv = sv[w2]; bp = sp[w2]; }
    st->cf_val = bv;
    st->cf_pass = bv == ~0ull ? -1 : bp;
    st->cf_len = bv == ~0ull ? 0 : pass_len[bp];
  }
}

// ------------------------------------------------------ sequential pass
// Queue of the sequential pass.  A queued vertex's key is min(r(y), lambda)
// + 1 (0 = not queued); because no queued r(y) ever exceeds the current bound
// (see the header comment), the key can be recomputed from r[] at any time,
// so the leaves of the max-tree are r[] itself (r = -1 marks a visited
// vertex, r = 0 an untouched one; the start vertex is popped first without a
// search).  Level 1 holds the maximum key of each 32 consecutive vertices,
// level 2 of each 32 level-1 nodes, and so on up to a level of at most 32
// nodes.  Levels that fit go to shared memory, from the top down.
struct SeqTree {
  int levels;            // number of node levels (>= 1)
  long long off[8];      // word offset of level l (l = 1..levels) in the level arena
  long long size[8];     // nodes of level l, padded to a multiple of 32
};

__host__ __device__ inline SeqTree seq_tree(int n) {
  SeqTree t{};
  long long below = ((long long)n + 31) / 32 * 32;  // padded leaves
  long long off = 0;
  int l = 1;
  for (;;) {
    const long long sz = (below / 32 + 31) / 32 * 32;
    t.off[l] = off;
    t.size[l] = sz;
    off += sz;
    t.levels = l;
    if (sz <= 32 || l == 7) break;
    below = sz;
    ++l;
  }
  return t;
}

template <typename KT>
__device__ __forceinline__ KT key_of(long long r, long long lam) {
  return r > 0 ? (KT)((r < lam ? r : lam) + 1) : (KT)0;
}

// One sequential pass over the graph of n vertices whose CSR rows are
// rp[0..n] (entry offsets into col/w), with neighbour ids col[e] - vbase.
// Parent hooks use ids + vbase.  lev[1..levels] and r point to shared or
// global memory as chosen by the caller.  Returns the results in the out
// references (thread 0's values are authoritative).
template <typename WT, typename KT>
__device__ void seq_pass_body(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                              int vbase, const WT* __restrict__ w, const WT* __restrict__ deg,
                              int start, int* parent, KT** lev, const SeqTree& tl, volatile WT* r,
                              int* __restrict__ order, int* __restrict__ mark_src,
                              int* __restrict__ marks_out,
                              long long marks_cap, long long lam0, long long* best_alpha_out,
                              int* best_len_out, int* ns_out, unsigned long long* marks_out_cnt,
                              bool* uf_fail_out) {
  __shared__ int s_x;
  __shared__ long long s_lam;
  __shared__ int s_done;
  __shared__ unsigned long long s_nmarks;
  __shared__ long long s_rb, s_re;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int l = 1; l <= tl.levels; ++l)
    for (long long i = tid; i < tl.size[l]; i += blockDim.x) lev[l][i] = 0;
  for (long long i = tid; i < n; i += blockDim.x) r[i] = 0;
  if (mark_src)
    for (long long i = tid; i < n; i += blockDim.x) mark_src[i] = -1;
  if (tid == 0) {
    s_lam = lam0;
    s_done = 0;
    s_nmarks = 0;
  }
  __syncthreads();
  long long alpha = 0, best_alpha = -1;
  int ns = 0, best_len = 0;
  bool uf_fail = false;
  unsigned long long my_marks = 0;
  for (int it = 0; it < n; ++it) {
    if (warp == 0) {
      int x = -1;
      long long rx = 0, xb = 0, xe = 0, xd = 0;
      const long long lam = s_lam;
      if (it == 0) {
        x = start;
        xb = rp[start];
        xe = rp[start + 1];
        xd = (long long)deg[start];
      } else {
        const int top = tl.levels;
        volatile KT* lt = lev[top];
        const KT tv = lane < tl.size[top] ? lt[lane] : (KT)0;
        const KT m = warp_max(tv);
        if (m != 0) {
          long long idx = __ffs(__ballot_sync(FULL, tv == m)) - 1;
          for (int l = top - 1; l >= 1; --l) {
            volatile KT* ll = lev[l];
            const KT cv = ll[idx * 32 + lane];
            idx = idx * 32 + (__ffs(__ballot_sync(FULL, cv == m)) - 1);
          }
          // leaves: keys recomputed from r of the 32 vertices under node idx
          // (row bounds and degrees of the 32 candidates load alongside r,
          // so the winner's row is known without another round trip)
          const long long v = idx * 32 + lane;
          long long rv = -1, vb = 0, ve = 0, vd = 0;
          if (v < n) {
            rv = (long long)r[v];
            vb = rp[v];
            ve = rp[v + 1];
            vd = (long long)deg[v];
          }
          const KT kv = key_of<KT>(rv, lam);
          const unsigned hit = __ballot_sync(FULL, kv == m);
          const int wl = __ffs(hit) - 1;
          x = (int)(idx * 32 + wl);
          rx = __shfl_sync(FULL, rv, wl);
          xb = __shfl_sync(FULL, vb, wl);
          xe = __shfl_sync(FULL, ve, wl);
          xd = __shfl_sync(FULL, vd, wl);
          // pop x and recompute its ancestors
          KT nk = lane == wl ? (KT)0 : kv;
          KT node = warp_max(nk);
          long long child = idx;
          if (lane == 0) lev[1][child] = node;
          __syncwarp();
          for (int l = 2; l <= tl.levels; ++l) {
            const long long p = child >> 5;
            volatile KT* lb = lev[l - 1];
            const KT cv = lb[p * 32 + lane];
            node = warp_max(cv);
            if (lane == 0) lev[l][p] = node;
            __syncwarp();
            child = p;
          }
        }
      }
      if (lane == 0) {
        if (x < 0) {
          s_done = 1;
        } else {
          r[x] = (WT)-1;  // visited
          order[ns] = x;
          ++ns;
          s_rb = xb;
          s_re = xe;
          alpha += xd - 2 * rx;
          if (ns < n && alpha < s_lam) {
            s_lam = alpha;
            best_alpha = alpha;
            best_len = ns;
          }
          s_x = x;
        }
      }
    }
    __syncthreads();
    if (s_done) break;
    const int x = s_x;
    const long long lam = s_lam;
    const long long rb = s_rb, re = s_re;
    for (long long e = rb + tid; e < re; e += blockDim.x) {
      const int y = col[e] - vbase;
      const long long r0 = (long long)r[y];
      if (r0 < 0) continue;  // visited
      const long long c = (long long)w[e];
      const long long r1 = r0 + c;
      r[y] = (WT)r1;
      if (r0 < lam && lam <= r1) {
        // r(y) crosses the bound once per pass (r grows, the bound only
        // falls), so each y has at most one marking edge: recorded here,
        // hooked after the pass, off the chain of pops
        if (mark_src) mark_src[y] = x;
        else if (!uf_union(parent, x + vbase, y + vbase)) uf_fail = true;
        ++my_marks;
        if (marks_out) {
          const unsigned long long k = atomicAdd(&s_nmarks, 1ull);
          if ((long long)k < marks_cap) {
            marks_out[2 * k] = x;
            marks_out[2 * k + 1] = y;
          }
        }
      }
      const KT key = key_of<KT>(r1, lam);
      long long idx = y >> 5;
      for (int l = 1; l <= tl.levels; ++l) {
        atomicMax(&lev[l][idx], key);
        idx >>= 5;
      }
    }
    __syncthreads();
  }
  if (mark_src) {
    for (long long i = tid; i < n; i += blockDim.x) {
      const int x = mark_src[i];
      if (x >= 0 && !uf_union(parent, x + vbase, (int)i + vbase)) uf_fail = true;
    }
  }
  *best_alpha_out = best_alpha;
  *best_len_out = best_len;
  *ns_out = ns;
  *marks_out_cnt = my_marks;
  *uf_fail_out = uf_fail;
}

// Places levels >= smem_from (and r when r_in_smem) in shared memory.
template <typename WT, typename KT>
__device__ __forceinline__ void seq_layout(const SeqTree& tl, int smem_from, int r_in_smem,
                                           unsigned char* smem, KT* g_levels, WT* g_r, KT** lev,
                                           WT** r_out) {
  long long soff = 0;
  for (int l = tl.levels; l >= 1; --l) {
    if (l >= smem_from) {
      lev[l] = reinterpret_cast<KT*>(smem) + soff;
      soff += tl.size[l];
    } else {
      lev[l] = g_levels + tl.off[l];
    }
  }
  const long long sbytes = ((soff * (long long)sizeof(KT)) + 15) / 16 * 16;
  *r_out = r_in_smem ? reinterpret_cast<WT*>(smem + sbytes) : g_r;
}

// A small graph's CSR copied into shared memory at byte offset `at` so that
// the pass's reads stay on chip; the pointers are redirected to the copies.
// Row offsets and degrees (read for the 32 candidates of every pop) come
// first; columns and weights (read for the popped row) only when `full`.
template <typename WT>
__device__ void seq_csr_to_smem(unsigned char* smem, long long at, int n, long long M, int full,
                                const int64_t*& rp, const int*& col, const WT*& w,
                                const WT*& deg) {
  int64_t* srp = reinterpret_cast<int64_t*>(smem + at);
  WT* sdeg = reinterpret_cast<WT*>(srp + (n + 1));
  WT* sw = sdeg + n;
  int* scol = reinterpret_cast<int*>(sw + M);
  for (long long i = threadIdx.x; i <= n; i += blockDim.x) srp[i] = rp[i];
  for (long long i = threadIdx.x; i < n; i += blockDim.x) sdeg[i] = deg[i];
  if (full) {
    for (long long i = threadIdx.x; i < M; i += blockDim.x) {
      scol[i] = col[i];
      sw[i] = w[i];
    }
  }
  __syncthreads();
  rp = srp;
  deg = sdeg;
  if (full) {
    col = scol;
    w = sw;
  }
}

template <typename WT, typename KT>
__global__ void __launch_bounds__(512)
    cf_seq_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                  const WT* __restrict__ w, const WT* __restrict__ deg, int start, int* parent,
                  WT* g_r, KT* g_levels, int* __restrict__ order, int* __restrict__ mark_src,
                  int* __restrict__ marks_out, long long marks_cap, int smem_from,
                  int r_in_smem, long long csr_at, int csr_full, long long M, DevState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SeqTree tl = seq_tree(n);
  KT* lev[8];
  WT* rr;
  seq_layout<WT, KT>(tl, smem_from, r_in_smem, smem, g_levels, g_r, lev, &rr);
  const int64_t* rp_ = rp;
  const int* col_ = col;
  const WT* w_ = w;
  const WT* deg_ = deg;
  if (csr_at >= 0) seq_csr_to_smem<WT>(smem, csr_at, n, M, csr_full, rp_, col_, w_, deg_);
  long long best_alpha;
  int best_len, ns;
  unsigned long long my_marks;
  bool uf_fail;
  seq_pass_body<WT, KT>(n, rp_, col_, 0, w_, deg_, start, parent, lev, tl, rr, order, mark_src,
                        marks_out,
                        marks_cap, (long long)st->lambda, &best_alpha, &best_len, &ns, &my_marks,
                        &uf_fail);
  const int lane = threadIdx.x & 31;
  if (uf_fail) set_error(st, ERR_INTERNAL);
  my_marks = warp_sum(my_marks);
  if (lane == 0 && my_marks) atomicAdd(&st->marks_cf, my_marks);
  if (threadIdx.x == 0) {
    st->cf_nscanned = ns;
    if (best_alpha >= 0) {  // below the bound this pass started from
      st->cf_val = (unsigned long long)best_alpha;
      st->cf_pass = -1;
      st->cf_len = best_len;
      atomicMin(&st->lambda, (unsigned long long)best_alpha);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) st->cf_nmarks = (long long)(*(volatile unsigned long long*)&st->marks_cf);
}

// Batch: block g runs the pass of graph g if it is not done and marked nothing.
template <typename WT, typename KT>
__global__ void __launch_bounds__(512)
    cf_seq_batch_kernel(int G, const int64_t* __restrict__ rp, const int* __restrict__ col,
                        const WT* __restrict__ w, const WT* __restrict__ deg, int* parent,
                        WT* g_r, KT* g_levels, const long long* __restrict__ level_off,
                        int* __restrict__ order, int all_smem, int always, BatchView bv,
                        DevState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = blockIdx.x;
  if (g >= G || bv.done_g[g] || (!always && *(volatile int*)&bv.marks_g[g] > 0)) return;
  const int vbase = bv.voff[g];
  const int n = bv.voff[g + 1] - vbase;
  if (n < 2) return;
  const SeqTree tl = seq_tree(n);
  KT* lev[8];
  WT* rr;
  seq_layout<WT, KT>(tl, all_smem ? 1 : tl.levels + 1, all_smem, smem, g_levels + level_off[g],
                     g_r + vbase, lev, &rr);
  long long best_alpha;
  int best_len, ns;
  unsigned long long my_marks;
  bool uf_fail;
  const long long lam0 = (long long)*(volatile unsigned long long*)&bv.lam_g[g];
  seq_pass_body<WT, KT>(n, rp + vbase, col, vbase, w, deg + vbase, 0, parent, lev, tl, rr,
                        order + vbase, nullptr, nullptr, 0, lam0, &best_alpha, &best_len, &ns,
                        &my_marks, &uf_fail);
  const int lane = threadIdx.x & 31;
  if (uf_fail) set_error(st, ERR_INTERNAL);
  my_marks = warp_sum(my_marks);
  if (lane == 0 && my_marks) atomicAdd(&bv.marks_g[g], (int)my_marks);
  if (threadIdx.x == 0 && best_alpha >= 0) {
    atomicMin(&bv.lam_g[g], (unsigned long long)best_alpha);
    atomicMin(&bv.cf_best[g], ((unsigned long long)best_alpha << 32) | 0xffffffffull);
    bv.cf_len[g] = best_len;
  }
}

// Best of the simultaneous sequential passes: when one of them lowered the
// bound it started from, cf_val / cf_pass / cf_len name it, with cf_pass =
// -2 - k for pass k (the earlier concurrent passes' best stays otherwise).
__global__ void cf_multi_best_kernel(const unsigned long long* __restrict__ pass_best,
                                     const int* __restrict__ pass_len, int passes, DevState* st) {
  __shared__ unsigned long long sv[32];
  __shared__ int sp[32];
  unsigned long long bv = ~0ull;
  int bp = 0x7fffffff;
  for (int p = threadIdx.x; p < passes; p += blockDim.x) {
    const unsigned long long v = pass_best[p];
    if (v < bv || (v == bv && p < bp)) { bv = v; bp = p; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v2 = __shfl_xor_sync(FULL, bv, o);
    const int p2 = __shfl_xor_sync(FULL, bp, o);
    if (v2 < bv || (v2 == bv && p2 < bp)) { bv = v2; bp = p2; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; sp[threadIdx.x >> 5] = bp; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2)
      if (sv[w2] < bv || (sv[w2] == bv && sp[w2] < bp)) { bv = sv[w2]; bp = sp[w2]; }
    if (bv != ~0ull) {
      st->cf_val = bv;
      st->cf_pass = -2 - bp;
      st->cf_len = pass_len[bp];
    }
  }
}

// Several sequential passes at once (private visit arrays): block k runs the
// pass of Algorithm 2 from its own start vertex over the whole graph with its
// own keys, tree and visit order (order + k*n), so each is a complete
// maximum-adjacency ordering of G and its marks are sound by themselves.  A
// pass lowers only its own copy of the bound; pass_best[k] / pass_len[k]
// give its best alpha and prefix length for the witness.
template <typename WT, typename KT>
__global__ void __launch_bounds__(512)
    cf_seq_multi_kernel(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                        const WT* __restrict__ w, const WT* __restrict__ deg,
                        unsigned long long seed, int* parent, WT* g_r, KT* g_levels,
                        long long tree_words, int* __restrict__ order,
                        int* __restrict__ mark_pool,
                        unsigned long long* __restrict__ pass_best, int* __restrict__ pass_len,
                        int smem_from, int r_in_smem, long long csr_at, int csr_full,
                        long long M,
                        DevState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const SeqTree tl = seq_tree(n);
  KT* lev[8];
  WT* rr;
  seq_layout<WT, KT>(tl, smem_from, r_in_smem, smem, g_levels + (long long)k * tree_words,
                     g_r + (long long)k * n, lev, &rr);
  const int64_t* rp_ = rp;
  const int* col_ = col;
  const WT* w_ = w;
  const WT* deg_ = deg;
  if (csr_at >= 0) seq_csr_to_smem<WT>(smem, csr_at, n, M, csr_full, rp_, col_, w_, deg_);
  const int start = k == 0 ? 0 : (int)(mix64(seed ^ mix64((unsigned long long)k)) % (unsigned long long)n);
  long long best_alpha;
  int best_len, ns;
  unsigned long long my_marks;
  bool uf_fail;
  seq_pass_body<WT, KT>(n, rp_, col_, 0, w_, deg_, start, parent, lev, tl, rr,
                        order + (long long)k * n, mark_pool + (long long)k * n, nullptr, 0,
                        (long long)*(volatile unsigned long long*)&st->lambda, &best_alpha,
                        &best_len, &ns, &my_marks, &uf_fail);
  const int lane = threadIdx.x & 31;
  if (uf_fail) set_error(st, ERR_INTERNAL);
  my_marks = warp_sum(my_marks);
  if (lane == 0 && my_marks) atomicAdd(&st->marks_cf, my_marks);
  if (threadIdx.x == 0) {
    pass_best[k] = best_alpha >= 0 ? (unsigned long long)best_alpha : ~0ull;
    pass_len[k] = best_len;
    if (best_alpha >= 0) atomicMin(&st->lambda, (unsigned long long)best_alpha);
  }
}

}  // namespace

// Bytes of a CSR copy in shared memory (int64 offsets, degrees, then with
// `full` the weights and int32 columns, in that order).
size_t seq_csr_bytes(int n, long long M, size_t wt, bool full) {
  return (size_t)(n + 1) * 8 + (size_t)n * wt + (full ? (size_t)M * (wt + 4) : 0);
}

// Where the CSR copy of a sequential pass goes: after `smem` bytes when r[]
// is on chip, whole if it fits under `limit`, else offsets and degrees only.
static void seq_csr_place(int n, long long M, size_t wt, int r_in_smem, size_t limit,
                          size_t* smem, long long* csr_at, int* csr_full) {
  *csr_at = -1;
  *csr_full = 0;
  if (!r_in_smem) return;
  const size_t at = (*smem + 15) / 16 * 16;
  for (int full = 1; full >= 0; --full) {
    const size_t b = seq_csr_bytes(n, M, wt, full != 0);
    if (at + b <= limit) {
      *csr_at = (long long)at;
      *csr_full = full;
      *smem = at + b;
      return;
    }
  }
}

template <typename WT>
cudaError_t capforest_passes(int n, const int64_t* rp, const int* col, const WT* w,
                             const WT* deg, int* owner, int* parent, int* visit_log,
                             unsigned long long* pass_best, int* pass_len, int* pass_counter,
                             PassConfig pc, DevState* st, cudaStream_t s, int* launches,
                             const BatchView* bv) {
  const int nsum = pc.table >> 5;
  const size_t per_warp = (size_t)pc.table * (sizeof(int) + sizeof(WT) + 8) + (size_t)nsum * 8;
  const size_t smem = per_warp * pc.warps_per_block;
  static size_t attr[2] = {0, 0};
  const int ai = sizeof(WT) == 8 ? 1 : 0;
  if (smem > attr[ai]) {
    cudaFuncSetAttribute(cf_passes_kernel<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)std::max<size_t>(smem, 48 * 1024));
    attr[ai] = std::max<size_t>(smem, 48 * 1024);
  }
  cudaMemsetAsync(pass_counter, 0, sizeof(int), s);
  const int blocks = std::max(1, std::min(pc.passes / pc.warps_per_block + 1,
                                          num_sms_cf() * 8));
  BatchView v{};
  if (bv) v = *bv;
  cf_passes_kernel<WT><<<blocks, pc.warps_per_block * 32, smem, s>>>(
      n, rp, col, w, deg, owner, parent, visit_log, pass_best, pass_len, pc.passes, pc.table,
      pc.seed, pass_counter, st, v, bv ? 1 : 0, pc.private_visit, bv ? -1ll : pc.skip_pr);
  ++*launches;
  if (!bv) {
    cf_best_kernel<<<1, 1024, 0, s>>>(pass_best, pass_len, pc.passes, st, pc.skip_pr);
    ++*launches;
  }
  return cudaGetLastError();
}

size_t capforest_pass_smem(int table, int warps_per_block, size_t wt_size) {
  return ((size_t)table * (sizeof(int) + wt_size + 8) + (size_t)(table >> 5) * 8) *
         (size_t)warps_per_block;
}

long long seq_tree_words(int n) {
  const SeqTree t = seq_tree(n);
  return t.off[t.levels] + t.size[t.levels];
}

template <typename WT>
cudaError_t capforest_sequential(int n, long long M, const int64_t* rp, const int* col,
                                 const WT* w, const WT* deg, int start, int* parent, WT* r,
                                 int* mark_src, unsigned long long* tree, int* order,
                                 int* marks_out, long long marks_cap, DevState* st,
                                 cudaStream_t s, int* launches) {
  using KT = typename std::conditional<sizeof(WT) == 4, unsigned, unsigned long long>::type;
  const size_t limit = 200 * 1024;
  const SeqTree t = seq_tree(n);
  // levels from the top down while they fit, then r[] if everything fits
  size_t used = 0;
  int smem_from = t.levels + 1;
  for (int l = t.levels; l >= 1; --l) {
    const size_t b = (size_t)t.size[l] * sizeof(KT);
    if (used + b > limit) break;
    used += b;
    smem_from = l;
  }
  const size_t lev_bytes = (used + 15) / 16 * 16;
  int r_in_smem = 0;
  size_t smem = used;
  if (smem_from == 1 && lev_bytes + (size_t)n * sizeof(WT) <= limit) {
    r_in_smem = 1;
    smem = lev_bytes + (size_t)n * sizeof(WT);
  }
  long long csr_at = -1;
  int csr_full = 0;
  seq_csr_place(n, M, sizeof(WT), r_in_smem, limit, &smem, &csr_at, &csr_full);
  static bool attr[2] = {false, false};
  const int ai = sizeof(WT) == 8 ? 1 : 0;
  if (!attr[ai]) {
    cudaFuncSetAttribute(cf_seq_kernel<WT, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)limit);
    attr[ai] = true;
  }
  cf_seq_kernel<WT, KT><<<1, 512, smem, s>>>(n, rp, col, w, deg, start, parent, r,
                                             reinterpret_cast<KT*>(tree), order, mark_src,
                                             marks_out,
                                             marks_cap, smem_from, r_in_smem, csr_at, csr_full,
                                             M, st);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t capforest_sequential_multi(int n, long long M, const int64_t* rp, const int* col,
                                       const WT* w, const WT* deg, int passes,
                                       unsigned long long seed,
                                       int* parent, WT* r_pool, unsigned long long* tree_pool,
                                       int* order_pool, int* mark_pool,
                                       unsigned long long* pass_best,
                                       int* pass_len, DevState* st, cudaStream_t s,
                                       int* launches) {
  using KT = typename std::conditional<sizeof(WT) == 4, unsigned, unsigned long long>::type;
  const size_t limit = 200 * 1024;
  const SeqTree t = seq_tree(n);
  size_t used = 0;
  int smem_from = t.levels + 1;
  for (int l = t.levels; l >= 1; --l) {
    const size_t b = (size_t)t.size[l] * sizeof(KT);
    if (used + b > limit) break;
    used += b;
    smem_from = l;
  }
  const size_t lev_bytes = (used + 15) / 16 * 16;
  int r_in_smem = 0;
  size_t smem = used;
  if (smem_from == 1 && lev_bytes + (size_t)n * sizeof(WT) <= limit) {
    r_in_smem = 1;
    smem = lev_bytes + (size_t)n * sizeof(WT);
  }
  long long csr_at = -1;
  int csr_full = 0;
  seq_csr_place(n, M, sizeof(WT), r_in_smem, limit, &smem, &csr_at, &csr_full);
  static bool attr[2] = {false, false};
  const int ai = sizeof(WT) == 8 ? 1 : 0;
  if (!attr[ai]) {
    cudaFuncSetAttribute(cf_seq_multi_kernel<WT, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)limit);
    attr[ai] = true;
  }
  cf_seq_multi_kernel<WT, KT><<<passes, 512, smem, s>>>(
      n, rp, col, w, deg, seed, parent, r_pool, reinterpret_cast<KT*>(tree_pool),
      seq_tree_words(n) * (long long)(sizeof(unsigned long long) / sizeof(KT)), order_pool,
      mark_pool, pass_best, pass_len, smem_from, r_in_smem, csr_at, csr_full, M, st);
  cf_multi_best_kernel<<<1, 1024, 0, s>>>(pass_best, pass_len, passes, st);
  *launches += 2;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t capforest_sequential_batch(int G, const int64_t* rp, const int* col, const WT* w,
                                       const WT* deg, int* parent, WT* r,
                                       unsigned long long* levels, const long long* level_off,
                                       int* order, int max_graph_n, int always,
                                       const BatchView& bv, DevState* st, cudaStream_t s,
                                       int* launches) {
  using KT = typename std::conditional<sizeof(WT) == 4, unsigned, unsigned long long>::type;
  const size_t limit = 200 * 1024;
  const SeqTree t = seq_tree(max_graph_n);
  size_t lev_words = 0;
  for (int l = 1; l <= t.levels; ++l) lev_words += (size_t)t.size[l];
  const size_t need = (lev_words * sizeof(KT) + 15) / 16 * 16 + (size_t)max_graph_n * sizeof(WT);
  const int all_smem = need <= limit ? 1 : 0;
  static bool attr[2] = {false, false};
  const int ai = sizeof(WT) == 8 ? 1 : 0;
  if (!attr[ai]) {
    cudaFuncSetAttribute(cf_seq_batch_kernel<WT, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)limit);
    attr[ai] = true;
  }
  if (G <= 0) return cudaSuccess;
  cf_seq_batch_kernel<WT, KT><<<G, 512, all_smem ? need : 0, s>>>(
      G, rp, col, w, deg, parent, r, reinterpret_cast<KT*>(levels), level_off, order, all_smem,
      always, bv, st);
  ++*launches;
  return cudaGetLastError();
}

#define MC_CF_INST(WT)                                                                        \
  template cudaError_t capforest_passes<WT>(int, const int64_t*, const int*, const WT*,       \
                                            const WT*, int*, int*, int*, unsigned long long*, \
                                            int*, int*, PassConfig, DevState*, cudaStream_t,  \
                                            int*, const BatchView*);                          \
  template cudaError_t capforest_sequential<WT>(int, long long, const int64_t*, const int*,     \
                                                const WT*,                                     \
                                                const WT*, int, int*, WT*, int*,              \
                                                unsigned long long*, int*, int*, long long,   \
                                                DevState*, cudaStream_t, int*);               \
  template cudaError_t capforest_sequential_multi<WT>(                                        \
      int, long long, const int64_t*, const int*, const WT*, const WT*, int,                   \
      unsigned long long, int*,                                                               \
      WT*, unsigned long long*, int*, int*, unsigned long long*, int*, DevState*, cudaStream_t, \
      int*);                                                                                  \
  template cudaError_t capforest_sequential_batch<WT>(                                        \
      int, const int64_t*, const int*, const WT*, const WT*, int*, WT*, unsigned long long*,   \
      const long long*, int*, int, int, const BatchView&, DevState*, cudaStream_t, int*);
MC_CF_INST(int32_t)
MC_CF_INST(int64_t)

}  // namespace mc
