// capforest_warp.cu -- whole-graph CAPFOREST passes, each driven by one warp
// (the sequential pass of Algorithm 2, run when a round's other marks do not
// suffice; with several blocks, several such passes from different start
// vertices at once, each with private keys and visit order).
//
// A pass is a bounded maximum-adjacency ordering (Sec. 2.1): repeatedly
// visit the unvisited vertex x of highest priority Q(x) = min(r(x), lambda),
// set alpha += c(x) - 2 r(x) (alpha = the cut of the visited set S) and
// lower lambda to alpha while S != V, then scan x's row: for each unvisited
// y, if r(y) < lambda <= r(y) + c(x, y) the edge {x, y} is contractible
// (Algorithm 1's union condition), r(y) += c(x, y).
//
// Order among the vertices of highest priority (a free choice, Sec. 2.1):
// neighbour first -- if some unvisited y of x's row now has the highest
// priority, the next vertex is the first such y in row order; otherwise the
// smallest vertex id among the highest.  The CPU oracle's tie = 1 mode
// implements the same rule, so one pass is comparable entry by entry.
//
// Design (one dependent chain of visits per pass, so the chain is short):
//  * one warp does everything: no block barrier on the path of a visit;
//  * the queue is a max tree of priorities over the vertices (key =
//    min(r, lambda) + 1, 0 = not queued): 128 leaves per level-1 node, 32
//    children per node above, 32-bit nodes in shared memory up to 6.4 M
//    vertices, so that a key update is one fire-and-forget atomicMax per
//    level; the leaves are r[] itself, in global memory (L2-resident) or,
//    for small graphs, in shared memory;
//  * a single warp pays the full latency of every dependent instruction, so
//    the chain of a visit is kept short: the row, then the gather of r, row
//    bounds and degree of its neighbours (L2 prefetch hints were measured to
//    gain nothing here); x's removal from the tree runs while that gather is
//    in flight, and yields the highest key without x;
//    if a neighbour's new key reaches it, that neighbour is next (no tree
//    descent); only otherwise does the warp descend the tree and read one
//    group of 128 leaves;
//  * each vertex is marked at most once per pass (r(y) crosses lambda once),
//    so marks are kept as mark[y] = x and hooked by a separate grid-wide
//    kernel after the passes.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mc {

namespace {

int num_sms_wp() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = kDefaultSms;
  }
  return sms;
}

__device__ __forceinline__ unsigned long long wp_mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The queue: a max tree of priorities.  A level-1 node holds the largest key
// of 128 consecutive vertices (key = min(r, lambda) + 1, 0 = not queued);
// a node of level l + 1 the largest of 32 nodes of level l, up to a level of
// 32 nodes.  Nodes are 32-bit, so a key update is one fire-and-forget
// atomicMax per level; with 128 leaves per level-1 node the levels of 6.4 M
// vertices fit in 200 KB of shared memory.
constexpr int kLeafShift = 7;                // 128 leaves per level-1 node
constexpr int kLeafFan = 1 << kLeafShift;
constexpr int kMaxLev = 6;                   // levels 1..5: enough for 2^31 vertices

struct WTree {
  int levels;
  long long size[8];  // nodes of level l, padded to a multiple of 32
};

__host__ __device__ inline WTree wtree(int n) {
  WTree t{};
  long long below = ((long long)n + kLeafFan - 1) / kLeafFan;
  int l = 1;
  for (;;) {
    const long long sz = (below + 31) / 32 * 32;
    t.size[l] = sz;
    t.levels = l;
    if (sz <= 32 || l == kMaxLev - 1) break;
    below = sz / 32;
    ++l;
  }
  return t;
}

__device__ __forceinline__ int lev_shift(int l) { return kLeafShift + 5 * (l - 1); }

// In the pass's weight type: r and lam fit it, and keys fit 32 bits.
template <typename WT>
__device__ __forceinline__ unsigned key_of_wp(WT r, WT lam) {
  return r > 0 ? (unsigned)(r < lam ? r : lam) + 1u : 0u;
}

struct WpArgs {
  int n;
  long long M;
  const int64_t* rp;
  const int* col;
  const void* w;
  const void* deg;
  int start0;               // start vertex of pass 0
  unsigned long long seed;  // start vertices of the other passes
  void* r_pool;             // [passes * n] (r, row start) pairs of WT (set by wp_init_kernel;
                            // unused when they live in shared memory)
  unsigned char* lev_pool;  // tree levels below smem_from, lev_stride bytes per pass, zero
  long long lev_stride;
  int* order_pool;          // [passes * n] visit order
  int* mark_pool;           // [passes * n] marking edge's far end, -1 = none
  unsigned long long* pass_best;  // [passes] best alpha below the start bound (~0: none)
  int* pass_len;            // [passes] its prefix length
  DevState* st;
  int smem_from;            // tree levels >= smem_from live in shared memory
  int r_smem;               // r in shared memory
  long long csr_at;         // byte offset of a shared-memory copy of the CSR (-1: none)
  int csr_full;             // the copy holds columns and weights too
  int stop_low;             // stop once the pass has marked and its highest priority falls
                            // below half the bound
};

// x has left the queue and its level-1 node holds the new maximum of its
// leaves: recompute the ancestors that change (a level whose node keeps its
// value leaves everything above unchanged).
__device__ __forceinline__ void tree_remove_up(unsigned* const* lev, int top, int x, int lane) {
#pragma unroll
  for (int l = 2; l < kMaxLev; ++l) {
    if (l > top) break;
    const int q = x >> lev_shift(l);
    const unsigned old = *(volatile unsigned*)&lev[l][q];
    const unsigned nv = __reduce_max_sync(FULL, *(volatile unsigned*)&lev[l - 1][q * 32 + lane]);
    if (nv == old) break;
    if (lane == 0) *(volatile unsigned*)&lev[l][q] = nv;
    __syncwarp();
  }
}

// Per-vertex state of a pass, one vector word per vertex so that a
// neighbour's gather is a single load: r (the connection to the visited set;
// -1 once visited) and the vertex's row start.  8 bytes for 32-bit weights,
// 16 for 64-bit.  In shared memory (RS) or in global memory, read and written
// at L2 (ld/st .cg): one warp owns it, and weak accesses ordered by
// __syncwarp let a visit's loads issue without waiting for the previous
// visit's stores.
template <typename WT>
struct RRT;
template <>
struct RRT<int32_t> {
  using V = int2;
};
template <>
struct RRT<int64_t> {
  using V = longlong2;
};

template <typename WT, bool RS>
struct RArr {
  using V = typename RRT<WT>::V;
  V* p;
  // (vertex ids are below 2^31)
  __device__ __forceinline__ V ld(int i) const { return RS ? p[i] : __ldcg(p + i); }
  __device__ __forceinline__ WT ld_r(int i) const {
    return RS ? p[i].x : __ldcg(reinterpret_cast<const WT*>(p + i));
  }
  __device__ __forceinline__ void st_r(int i, WT v) const {
    if (RS) p[i].x = v;
    else __stcg(reinterpret_cast<WT*>(p + i), v);
  }
};

// Per-pass state of the driving warp (uniform across its lanes).  A graph
// with 32-bit weights has a total weight below 2^31, so every r, degree, cut
// and bound of its passes fits the weight type WT.
template <typename WT>
struct PassState {
  int x, xb, xe;      // the vertex being visited and its row
  WT rx, xd;          // its r at the visit and its degree
  WT lam, alpha;
  unsigned kt;        // highest key without x, before x's row updates
  unsigned bk;        // highest key among x's updated neighbours ...
  int by, bb;         // ... the first such neighbour and its row start
  WT br;              // ... its r
};

// Updates of one chunk set of x's row: entries y[u] (-1: none) with weights
// c[u] and gathered state (r0[u], yb[u]): r, marks, tree, and the first entry
// with the highest new key.
template <int NCH, typename WT, bool RS>
__device__ __forceinline__ void apply_batch(PassState<WT>& ps, const int (&y)[NCH],
                                            const WT (&c)[NCH], const WT (&r0)[NCH],
                                            const int (&yb)[NCH], const RArr<WT, RS> rr,
                                            unsigned* const* lev, int top,
                                            int* __restrict__ mark, unsigned& nmarks,
                                            bool packed) {
  const int lane = threadIdx.x;
  unsigned lbk = 0;
  int lu = 0;
#pragma unroll
  for (int u = 0; u < NCH; ++u) {
    if (y[u] >= 0 && r0[u] >= 0) {
      const WT r1 = r0[u] + c[u];
      rr.st_r(y[u], r1);
      if (r0[u] < ps.lam && ps.lam <= r1) {
        mark[y[u]] = ps.x;
        ++nmarks;
      }
      const unsigned k1 = (unsigned)(r1 < ps.lam ? r1 : ps.lam) + 1u;
#pragma unroll
      for (int l = 1; l < kMaxLev; ++l)
        if (l <= top) atomicMax(&lev[l][y[u] >> lev_shift(l)], k1);
      if (k1 > lbk) {  // strictly larger: the earlier entry keeps ties
        lbk = k1;
        lu = u;
      }
    }
  }
  unsigned km, pos;
  if (packed) {  // key < 2^25: key and entry position in one reduction
    const unsigned pk = lbk ? (lbk << 7) | (127u - (unsigned)(lu * 32 + lane)) : 0u;
    const unsigned m = __reduce_max_sync(FULL, pk);
    km = m >> 7;
    pos = 127u - (m & 127u);
  } else {
    km = __reduce_max_sync(FULL, lbk);
    pos = __reduce_min_sync(FULL, (lbk == km && km) ? (unsigned)(lu * 32 + lane) : ~0u);
  }
  if (km > ps.bk) {
    const int wl = (int)(pos & 31);
    int sy = y[0], sb = yb[0];
    WT sr = r0[0] + c[0];
#pragma unroll
    for (int u = 1; u < NCH; ++u)
      if (lu == u) {
        sy = y[u];
        sb = yb[u];
        sr = r0[u] + c[u];
      }
    ps.bk = km;
    ps.by = __shfl_sync(FULL, sy, wl);
    ps.br = __shfl_sync(FULL, sr, wl);
    ps.bb = __shfl_sync(FULL, sb, wl);
  }
}

// The first entry with the highest new key among NCH chunks (no side
// effects; commit_batch then applies the same updates).
template <int NCH, typename WT>
__device__ __forceinline__ void best_batch(PassState<WT>& ps, const int (&y)[NCH],
                                           const WT (&c)[NCH], const WT (&r0)[NCH],
                                           const int (&yb)[NCH], bool packed, WT (&r1)[NCH],
                                           unsigned (&k1)[NCH]) {
  const int lane = threadIdx.x;
  unsigned lbk = 0;
  int lu = 0;
#pragma unroll
  for (int u = 0; u < NCH; ++u) {
    r1[u] = r0[u] + c[u];
    k1[u] = (y[u] >= 0 && r0[u] >= 0) ? (unsigned)(r1[u] < ps.lam ? r1[u] : ps.lam) + 1u : 0u;
    if (k1[u] > lbk) {
      lbk = k1[u];
      lu = u;
    }
  }
  unsigned km, pos;
  if (packed) {
    const unsigned pk = lbk ? (lbk << 7) | (127u - (unsigned)(lu * 32 + lane)) : 0u;
    const unsigned m = __reduce_max_sync(FULL, pk);
    km = m >> 7;
    pos = 127u - (m & 127u);
  } else {
    km = __reduce_max_sync(FULL, lbk);
    pos = __reduce_min_sync(FULL, (lbk == km && km) ? (unsigned)(lu * 32 + lane) : ~0u);
  }
  if (km > ps.bk) {
    const int wl = (int)(pos & 31);
    int sy = y[0], sb = yb[0];
    WT sr = r1[0];
#pragma unroll
    for (int u = 1; u < NCH; ++u)
      if (lu == u) {
        sy = y[u];
        sb = yb[u];
        sr = r1[u];
      }
    ps.bk = km;
    ps.by = __shfl_sync(FULL, sy, wl);
    ps.br = __shfl_sync(FULL, sr, wl);
    ps.bb = __shfl_sync(FULL, sb, wl);
  }
}

// The updates of NCH chunks (new r and keys from best_batch): r, marks and
// the tree.
template <int NCH, typename WT, bool RS>
__device__ __forceinline__ void commit_batch(const PassState<WT>& ps, const int (&y)[NCH],
                                             const WT (&r0)[NCH], const WT (&r1)[NCH],
                                             const unsigned (&k1)[NCH], const RArr<WT, RS> rr,
                                             unsigned* const* lev, int top,
                                             int* __restrict__ mark, unsigned& nmarks) {
#pragma unroll
  for (int u = 0; u < NCH; ++u) {
    if (k1[u]) {
      rr.st_r(y[u], r1[u]);
      if (r0[u] < ps.lam && ps.lam <= r1[u]) {
        mark[y[u]] = ps.x;
        ++nmarks;
      }
#pragma unroll
      for (int l = 1; l < kMaxLev; ++l)
        if (l <= top) atomicMax(&lev[l][y[u] >> lev_shift(l)], k1[u]);
    }
  }
}

// Gather of NCH chunks: r and row start of each valid entry's vertex.
template <int NCH, typename WT, bool RS>
__device__ __forceinline__ void gather_batch(const int (&y)[NCH], WT (&r0)[NCH], int (&yb)[NCH],
                                             const RArr<WT, RS> rr) {
#pragma unroll
  for (int u = 0; u < NCH; ++u) {
    r0[u] = -1;
    yb[u] = 0;
    if (y[u] >= 0) {
      const typename RRT<WT>::V v = rr.ld(y[u]);
      r0[u] = (WT)v.x;
      yb[u] = (int)v.y;
    }
  }
}

template <typename WT, bool RS>
__global__ void __launch_bounds__(32) cf_warp_pass_kernel(WpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using V = typename RRT<WT>::V;
  const int lane = threadIdx.x;
  const int k = blockIdx.x;
  const int n = a.n;
  const WTree tl = wtree(n);
  const int top = tl.levels;
  unsigned* lev[kMaxLev];
  long long soff = 0, goff = 0;
  unsigned char* gbase = a.lev_pool + (long long)k * a.lev_stride;
  lev[0] = nullptr;
#pragma unroll
  for (int l = kMaxLev - 1; l >= 1; --l) {
    lev[l] = nullptr;
    if (l <= top) {
      if (l >= a.smem_from) {
        lev[l] = reinterpret_cast<unsigned*>(smem + soff);
        soff += tl.size[l] * 4;
      } else {
        lev[l] = reinterpret_cast<unsigned*>(gbase + goff);
        goff += tl.size[l] * 4;
      }
    }
  }
  soff = (soff + 15) / 16 * 16;
  const RArr<WT, RS> rr{RS ? reinterpret_cast<V*>(smem + soff)
                           : reinterpret_cast<V*>(a.r_pool) + (long long)k * n};
#pragma unroll
  for (int l = 1; l < kMaxLev; ++l)
    if (l <= top && l >= a.smem_from)
      for (long long i = lane; i < tl.size[l]; i += 32) lev[l][i] = 0;
  const int64_t* rp = a.rp;
  const int* col = a.col;
  const WT* w = reinterpret_cast<const WT*>(a.w);
  const WT* deg = reinterpret_cast<const WT*>(a.deg);
  if (RS)  // global r_pool entries are set by wp_init_kernel
    for (long long i = lane; i < n; i += 32) {
      V v;
      v.x = 0;
      v.y = (WT)rp[i];
      rr.p[i] = v;
    }
  if (a.csr_at >= 0) {
    int64_t* srp = reinterpret_cast<int64_t*>(smem + a.csr_at);
    WT* sdeg = reinterpret_cast<WT*>(srp + (n + 1));
    WT* sw = sdeg + n;
    int* scol = reinterpret_cast<int*>(sw + a.M);
    for (long long i = lane; i <= n; i += 32) srp[i] = rp[i];
    for (long long i = lane; i < n; i += 32) sdeg[i] = deg[i];
    if (a.csr_full) {
      for (long long i = lane; i < a.M; i += 32) {
        scol[i] = col[i];
        sw[i] = w[i];
      }
      col = scol;
      w = sw;
    }
    rp = srp;
    deg = sdeg;
  }
  __syncwarp();
  unsigned* topl = lev[1];
#pragma unroll
  for (int l = 2; l < kMaxLev; ++l)
    if (l == top) topl = lev[l];
  volatile unsigned* vtop = topl;

  const int M = (int)a.M;
  int* order = a.order_pool + (long long)k * n;
  int* mark = a.mark_pool + (long long)k * n;
  PassState<WT> ps;
  ps.lam = (WT)*(volatile unsigned long long*)&a.st->lambda;
  const bool packed = (unsigned long long)ps.lam < (1ull << 24);
  ps.alpha = 0;
  WT best_alpha = -1;
  int best_len = 0, ns = 0;
  unsigned nmarks = 0;
  bool bad = false;
  ps.x = k == 0 ? a.start0
                : (int)(wp_mix64(a.seed ^ wp_mix64((unsigned long long)k)) % (unsigned long long)n);
  ps.rx = 0;
  ps.xb = (int)rp[ps.x];
  // the next vertex's first 64 row entries, row end and degree, loaded
  // ahead when the next vertex was known before x's updates were committed
  bool pre = false;
  int ny[2] = {-1, -1};
  WT nc[2] = {0, 0};
  int nxe = 0;
  WT nxd = 0;
  for (int it = 0; it < n; ++it) {
    // ---- visit x: its first 64 row entries, row end and degree in one round
    // trip (the row start came with x's gather)
    int y[2];
    WT c[2];
    if (pre) {
      y[0] = ny[0];
      y[1] = ny[1];
      c[0] = nc[0];
      c[1] = nc[1];
      ps.xe = nxe;
      ps.xd = nxd;
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = ps.xb + u * 32 + lane;
        y[u] = -1;
        c[u] = 0;
        if (e < M) {
          y[u] = col[e];
          c[u] = w[e];
        }
      }
      ps.xe = (int)rp[ps.x + 1];
      ps.xd = deg[ps.x];
    }
    // x's group of 128 leaves without x, for x's removal from the tree
    const int gb = ps.x & ~(kLeafFan - 1);
    WT g4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = gb + j * 32 + lane;
      g4[j] = (v < n && v != ps.x) ? rr.ld_r(v) : (WT)-1;
    }
    if (lane == 0) {
      rr.st_r(ps.x, (WT)-1);
      order[ns] = ps.x;
    }
    ++ns;
    ps.alpha += ps.xd - 2 * ps.rx;
    if (ns < n && ps.alpha < ps.lam) {
      ps.lam = ps.alpha;
      best_alpha = ps.alpha;
      best_len = ns;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (ps.xb + u * 32 + lane >= ps.xe) y[u] = -1;
    WT r0[2];
    int yb[2];
    gather_batch<2, WT, RS>(y, r0, yb, rr);
    // x leaves the queue (while the gather is in flight): its level-1 node
    // and the ancestors that change; then the highest key without x
    {
      unsigned gk = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) gk = max(gk, key_of_wp<WT>(g4[j], ps.lam));
      const unsigned node = __reduce_max_sync(FULL, gk);
      if (lane == 0) *(volatile unsigned*)&lev[1][ps.x >> kLeafShift] = node;
      __syncwarp();
      tree_remove_up(lev, top, ps.x, lane);
      ps.kt = __reduce_max_sync(FULL, vtop[lane]);
    }
    ps.bk = 0;
    ps.by = -1;
    ps.bb = 0;
    ps.br = 0;
    WT r1[2];
    unsigned k1[2];
    best_batch<2, WT>(ps, y, c, r0, yb, packed, r1, k1);
    // a row of at most 64 entries whose best neighbour holds the highest key:
    // that neighbour is next, and its row loads go out before this row's
    // updates are committed
    const bool single = ps.xe - ps.xb <= 64;
    const bool fast = single && ps.bk > 0 && ps.bk >= ps.kt &&
                      !(a.stop_low && 2ll * (long long)(ps.bk - 1) < (long long)ps.lam);
    if (fast) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = ps.bb + u * 32 + lane;
        ny[u] = -1;
        nc[u] = 0;
        if (e < M) {
          ny[u] = col[e];
          nc[u] = w[e];
        }
      }
      nxe = (int)rp[ps.by + 1];
      nxd = deg[ps.by];
    }
    commit_batch<2, WT, RS>(ps, y, r0, r1, k1, rr, lev, top, mark, nmarks);
    if (fast) {
      __syncwarp();  // this row's updates are visible to the next reads
      ps.x = ps.by;
      ps.rx = ps.br;
      ps.xb = ps.bb;
      pre = true;
      continue;
    }
    pre = false;
    // the rest of a long row, 128 entries per batch
    for (int e0 = ps.xb + 64; e0 < ps.xe; e0 += 128) {
      int y4[4];
      WT c4[4], r4[4];
      int b4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * 32 + lane;
        y4[u] = -1;
        c4[u] = 0;
        if (e < ps.xe) {
          y4[u] = col[e];
          c4[u] = w[e];
        }
      }
      gather_batch<4, WT, RS>(y4, r4, b4, rr);
      apply_batch<4, WT, RS>(ps, y4, c4, r4, b4, rr, lev, top, mark, nmarks, packed);
    }
    __syncwarp();  // this row's updates are visible to the next reads
    if (a.stop_low) {
      // the pass has left the region it marked (a prefix of a maximum-
      // adjacency order: its marks and its alpha stay valid)
      const unsigned kn = max(ps.bk, ps.kt);
      if (kn > 0 && 2ll * (long long)(kn - 1) < (long long)ps.lam &&
          __any_sync(FULL, nmarks != 0))
        break;
    }
    // ---- the next vertex: a neighbour holding the highest key, else the
    // smallest vertex id among the highest
    if (ps.bk > 0 && ps.bk >= ps.kt) {
      ps.x = ps.by;
      ps.rx = ps.br;
      ps.xb = ps.bb;
      continue;
    }
    const unsigned kt = ps.kt;
    if (kt == 0) break;  // nothing queued: every reachable vertex is visited
    int idx = __ffs(__ballot_sync(FULL, vtop[lane] == kt)) - 1;
#pragma unroll
    for (int l = kMaxLev - 1; l >= 1; --l) {
      if (l < top && !bad) {
        const unsigned hb =
            __ballot_sync(FULL, *(volatile unsigned*)&lev[l][idx * 32 + lane] == kt);
        if (!hb) bad = true;
        else idx = idx * 32 + (__ffs(hb) - 1);
      }
    }
    if (bad) break;
    WT rv[4];
    int bv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = idx * kLeafFan + j * 32 + lane;
      rv[j] = -1;
      bv[j] = 0;
      if (v < n) {
        const V q = rr.ld(v);
        rv[j] = (WT)q.x;
        bv[j] = (int)q.y;
      }
    }
    int found = -1;
    WT srv = 0;
    int sbv = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned hb = __ballot_sync(FULL, key_of_wp<WT>(rv[j], ps.lam) == kt);
      if (found < 0 && hb) {
        found = j * 32 + (__ffs(hb) - 1);
        srv = rv[j];
        sbv = bv[j];
      }
    }
    if (found < 0) {
      bad = true;
      break;
    }
    const int wl = found & 31;
    ps.x = idx * kLeafFan + found;
    ps.rx = __shfl_sync(FULL, srv, wl);
    ps.xb = __shfl_sync(FULL, sbv, wl);
  }
  nmarks = warp_sum(nmarks);
  if (lane == 0) {
    a.pass_best[k] = best_alpha >= 0 ? (unsigned long long)best_alpha : ~0ull;
    a.pass_len[k] = best_len;
    if (best_alpha >= 0) atomicMin(&a.st->lambda, (unsigned long long)best_alpha);
    if (k == 0) a.st->cf_nscanned = ns;
    if (nmarks) atomicAdd(&a.st->marks_cf, (unsigned long long)nmarks);
    if (bad) {
      set_error(a.st, ERR_INTERNAL);
      atomicMax(&a.st->internal_code, 41);
    }
  }
}

// Global per-vertex state of every pass: r = 0, row start from rp.
template <typename WT>
__global__ void wp_init_kernel(typename RRT<WT>::V* __restrict__ pool, int passes, int n,
                               const int64_t* __restrict__ rp) {
  const long long total = (long long)passes * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    typename RRT<WT>::V v;
    v.x = 0;
    v.y = (WT)rp[i % n];
    pool[i] = v;
  }
}

// Hook every pass's marks: mark_pool[k * n + y] = x >= 0 joins x and y.
__global__ void wp_hook_kernel(const int* __restrict__ mark_pool, long long total, int n,
                               int* parent, DevState* st) {
  bool fail = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = mark_pool[i];
    if (x >= 0 && !uf_union(parent, x, (int)(i % n))) fail = true;
  }
  if (fail) set_error(st, ERR_INTERNAL);
}

// Best pass: the smallest alpha below the start bound (ties: smaller pass)
// names the witness, cf_pass = -2 - k.
__global__ void wp_best_kernel(const unsigned long long* __restrict__ pass_best,
                               const int* __restrict__ pass_len, int passes, DevState* st) {
  unsigned long long bv = ~0ull;
  int bp = INT_MAX;
  for (int p = threadIdx.x; p < passes; p += 32) {
    const unsigned long long v = pass_best[p];
    if (v < bv || (v == bv && p < bp)) {
      bv = v;
      bp = p;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v2 = __shfl_xor_sync(FULL, bv, o);
    const int p2 = __shfl_xor_sync(FULL, bp, o);
    if (v2 < bv || (v2 == bv && p2 < bp)) {
      bv = v2;
      bp = p2;
    }
  }
  if (threadIdx.x == 0 && bv != ~0ull) {
    st->cf_val = bv;
    st->cf_pass = -2 - bp;
    st->cf_len = pass_len[bp];
  }
}

}  // namespace

// 4 when a pass starting from bound lam fits the 32-bit keys, else 0.
int warp_pass_key_bytes(long long lam) {
  return (lam >= 0 && lam <= 0xfffffffell) ? 4 : 0;
}

long long warp_pass_lev_bytes(int n) {
  const WTree t = wtree(n);
  long long b = 0;
  for (int l = 1; l <= t.levels; ++l) b += t.size[l] * 4;
  return (b + 255) / 256 * 256;
}

// Global-memory bytes one pass reads repeatedly (its r[] and the tree
// levels that stay in global memory): the L2 working set of a pass.
long long warp_pass_hot_bytes(int n, size_t wt, long long lam) {
  if (!warp_pass_key_bytes(lam)) return -1;
  const WTree t = wtree(n);
  long long lev = 0;
  for (int l = 1; l <= t.levels; ++l) lev += t.size[l] * 4;
  const long long rb = (long long)n * 2 * (long long)wt;
  if (lev + rb <= (long long)kWarpPassSmem) return 0;
  return rb + (lev <= (long long)kWarpPassSmem ? 0 : t.size[1] * 4);
}

template <typename WT>
cudaError_t capforest_warp_passes(int n, long long M, const int64_t* rp, const int* col,
                                  const WT* w, const WT* deg, int passes, int start0,
                                  unsigned long long seed, long long lam, int* parent,
                                  WT* r_pool, unsigned char* lev_pool, long long lev_stride,
                                  int* order_pool, int* mark_pool, unsigned long long* pass_best,
                                  int* pass_len, int stop_low, DevState* st, cudaStream_t s,
                                  int* launches) {
  if (!warp_pass_key_bytes(lam) || passes < 1 || n < 1) return cudaErrorInvalidValue;
  const WTree t = wtree(n);
  // tree levels from the top down while they fit, then r[], then the CSR
  const size_t limit = kWarpPassSmem;
  size_t used = 0;
  int smem_from = t.levels + 1;
  for (int l = t.levels; l >= 1; --l) {
    const size_t b = (size_t)t.size[l] * 4;
    if (used + b > limit) break;
    used += b;
    smem_from = l;
  }
  long long gl = 0;  // bytes of the global levels of a pass
  for (int l = 1; l < smem_from; ++l) gl += t.size[l] * 4;
  if (gl > lev_stride) return cudaErrorInvalidValue;
  size_t smem = (used + 15) / 16 * 16;
  int r_smem = 0;
  if (smem_from == 1 && smem + (size_t)n * 2 * sizeof(WT) <= limit) {
    r_smem = 1;
    smem += ((size_t)n * 2 * sizeof(WT) + 15) / 16 * 16;
  }
  long long csr_at = -1;
  int csr_full = 0;
  if (r_smem) {
    for (int full = 1; full >= 0; --full) {
      const size_t b = (size_t)(n + 1) * 8 + (size_t)n * sizeof(WT) +
                       (full ? (size_t)M * (sizeof(WT) + 4) : 0);
      if (smem + b <= limit) {
        csr_at = (long long)smem;
        csr_full = full;
        smem += b;
        break;
      }
    }
  }
  if (!r_smem) {
    const long long total = (long long)passes * n;
    const int ib = (int)std::min<long long>((total + 255) / 256, (long long)num_sms_wp() * 8);
    wp_init_kernel<WT><<<std::max(ib, 1), 256, 0, s>>>(
        reinterpret_cast<typename RRT<WT>::V*>(r_pool), passes, n, rp);
    ++*launches;
  }
  if (gl > 0) cudaMemsetAsync(lev_pool, 0, (size_t)passes * lev_stride, s);
  cudaMemsetAsync(mark_pool, 0xff, (size_t)passes * n * sizeof(int), s);
  WpArgs a{};
  a.n = n;
  a.M = M;
  a.rp = rp;
  a.col = col;
  a.w = w;
  a.deg = deg;
  a.start0 = start0;
  a.seed = seed;
  a.r_pool = r_pool;
  a.lev_pool = lev_pool;
  a.lev_stride = lev_stride;
  a.order_pool = order_pool;
  a.mark_pool = mark_pool;
  a.pass_best = pass_best;
  a.pass_len = pass_len;
  a.st = st;
  a.smem_from = smem_from;
  a.r_smem = r_smem;
  a.csr_at = csr_at;
  a.csr_full = csr_full;
  a.stop_low = stop_low;
  static bool attr[2][2] = {};
  const int wi = sizeof(WT) == 8 ? 1 : 0;
  if (!attr[wi][r_smem]) {
    cudaFuncSetAttribute(r_smem ? cf_warp_pass_kernel<WT, true> : cf_warp_pass_kernel<WT, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
    attr[wi][r_smem] = true;
  }
  if (r_smem) cf_warp_pass_kernel<WT, true><<<passes, 32, smem, s>>>(a);
  else cf_warp_pass_kernel<WT, false><<<passes, 32, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long total = (long long)passes * n;
  const int hb = (int)std::min<long long>((total + 255) / 256, (long long)num_sms_wp() * 8);
  wp_hook_kernel<<<std::max(hb, 1), 256, 0, s>>>(mark_pool, total, n, parent, st);
  wp_best_kernel<<<1, 32, 0, s>>>(pass_best, pass_len, passes, st);
  *launches += 3;
  return cudaGetLastError();
}

#define MC_WP_INST(WT)                                                                        \
  template cudaError_t capforest_warp_passes<WT>(                                             \
      int, long long, const int64_t*, const int*, const WT*, const WT*, int, int,              \
      unsigned long long, long long, int*, WT*, unsigned char*, long long, int*, int*,         \
      unsigned long long*, int*, int, DevState*, cudaStream_t, int*);
MC_WP_INST(int32_t)
MC_WP_INST(int64_t)

}  // namespace mc
