// batch.cu -- per-graph bookkeeping of a packed batch of graphs.
//
// A batch packs G independent graphs into one CSR: graph g owns the vertex
// range [voff[g], voff[g+1]) and no edge crosses ranges.  Every round runs the
// ordinary round kernels once over the whole batch; what differs is that each
// graph keeps its own upper bound lam_g[g] (Algorithm 2 runs per graph), its
// own stop test (n_g <= 2 or lam_g = 0, Sec. 2.1 / Algorithm 2) and its own
// witness.  A finished graph is collapsed into its first vertex, so its edges
// turn into self-loops and leave the next contraction.  Canonical relabelling
// keeps each graph's vertices contiguous and in graph order (contracted
// vertices are numbered by smallest member), so the new offsets are the ranks
// of the old first vertices.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mc {

namespace {

int sms_b() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = kDefaultSms;
  }
  return sms;
}

int gridb(long long work, int block) {
  long long g = (work + block - 1) / block;
  return (int)std::max<long long>(1, std::min<long long>(g, (long long)sms_b() * 32));
}

__device__ __forceinline__ int graph_of(const int* __restrict__ voff, int G, int v) {
  int lo = 0, hi = G;  // largest g with voff[g] <= v
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (voff[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void gid_fill_kernel(const int* __restrict__ voff, int G, int n, int* __restrict__ gid) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    gid[v] = graph_of(voff, G, v);
}

__global__ void batch_start_kernel(int G, unsigned long long* lam_g, int* done_g) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    lam_g[g] = (unsigned long long)kInf;
    done_g[g] = 0;
  }
}

__global__ void batch_round_reset_kernel(int G, const unsigned long long* lam_g,
                                         unsigned long long* lam_before,
                                         unsigned long long* deg_best,
                                         unsigned long long* cf_best, int* cf_len, int* marks_g,
                                         int* wit_kind) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    lam_before[g] = lam_g[g];
    deg_best[g] = ~0ull;
    cf_best[g] = ~0ull;
    cf_len[g] = 0;
    marks_g[g] = 0;
    wit_kind[g] = 0;
  }
}

// Per-graph minimum degree as deg << 32 | vertex (smallest vertex on ties).
template <typename WT>
__global__ void batch_degmin_kernel(int n, const WT* __restrict__ deg, const int* __restrict__ gid,
                                    const int* __restrict__ done_g,
                                    unsigned long long* deg_best) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int g = gid[v];
    if (done_g[g]) continue;
    atomicMin(&deg_best[g], ((unsigned long long)(unsigned)deg[v] << 32) | (unsigned)v);
  }
}

// Degree bound (graphs with at least 2 vertices), then the stop test.
__global__ void batch_apply_deg_kernel(int G, const int* __restrict__ voff,
                                       const unsigned long long* __restrict__ deg_best,
                                       unsigned long long* lam_g, int* done_g, int* newly_done) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    if (done_g[g]) continue;
    const int ng = voff[g + 1] - voff[g];
    if (ng >= 2) {
      const unsigned long long d = deg_best[g] >> 32;
      if (d < lam_g[g]) lam_g[g] = d;
    }
    if (ng <= 2 || lam_g[g] == 0) {
      done_g[g] = 1;
      atomicAdd(newly_done, 1);
    }
  }
}

// Which source set each improved bound: 1 degree (vertex), 2 a concurrent
// pass's visited prefix, 3 the sequential pass's prefix.
__global__ void batch_witness_decide_kernel(int G, const unsigned long long* __restrict__ lam_g,
                                            const unsigned long long* __restrict__ lam_before,
                                            const unsigned long long* __restrict__ deg_best,
                                            const unsigned long long* __restrict__ cf_best,
                                            int* wit_kind, int* wit_x, DevState* st) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const unsigned long long lam = lam_g[g];
    if (lam >= lam_before[g]) continue;
    if ((deg_best[g] >> 32) == lam) {
      wit_kind[g] = 1;
      wit_x[g] = (int)(deg_best[g] & 0xffffffffull);
    } else if ((cf_best[g] >> 32) == lam) {
      const unsigned p = (unsigned)(cf_best[g] & 0xffffffffull);
      wit_kind[g] = p == 0xffffffffu ? 3 : 2;
      wit_x[g] = (int)p;
    } else {
      set_error(st, ERR_INTERNAL);
    }
  }
}

// Block g: for a list witness, flag the listed current vertices of graph g.
__global__ void batch_witness_list_kernel(int G, const int* __restrict__ voff,
                                          const int* __restrict__ wit_kind,
                                          const int* __restrict__ wit_x,
                                          const int* __restrict__ cf_len,
                                          const int* __restrict__ visit_log, int table,
                                          const int* __restrict__ pass_len,
                                          const int* __restrict__ seq_order, uint8_t* cur) {
  const int g = blockIdx.x;
  if (g >= G) return;
  const int k = wit_kind[g];
  if (k < 2) return;
  const int b = voff[g], e = voff[g + 1];
  for (int v = b + threadIdx.x; v < e; v += blockDim.x) cur[v] = 0;
  __syncthreads();
  if (k == 2) {
    const int p = wit_x[g];
    const int len = pass_len[p];
    for (int i = threadIdx.x; i < len; i += blockDim.x) cur[visit_log[(long long)p * table + i]] = 1;
  } else {
    const int len = cf_len[g];
    for (int i = threadIdx.x; i < len; i += blockDim.x) cur[b + seq_order[b + i]] = 1;
  }
}

__global__ void batch_witness_apply_kernel(int n0, const int* __restrict__ gid0,
                                           const int* __restrict__ map0,
                                           const int* __restrict__ wit_kind,
                                           const int* __restrict__ wit_x,
                                           const uint8_t* __restrict__ cur, uint8_t* side0) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
    const int g = gid0[i];
    const int k = wit_kind[g];
    if (k == 1) side0[i] = map0[i] == wit_x[g] ? 1 : 0;
    else if (k >= 2) side0[i] = cur[map0[i]];
  }
}

// Finished graphs: every vertex joins the graph's first vertex.
__global__ void batch_collapse_kernel(int n, const int* __restrict__ gid,
                                      const int* __restrict__ voff,
                                      const int* __restrict__ done_g, int* parent) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int g = gid[v];
    if (done_g[g]) parent[v] = voff[g];
  }
}

__global__ void batch_new_offsets_kernel(int G, const int* __restrict__ voff,
                                         const int* __restrict__ rank, const DevState* st,
                                         int* __restrict__ voff_next) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
    voff_next[g] = g < G ? rank[voff[g]] : st->n_next;
}

// Bit i = side0[i] xor side0[first vertex of i's graph].
__global__ void batch_bitmap_kernel(const uint8_t* __restrict__ side0, int n0,
                                    const int* __restrict__ gid0, const int* __restrict__ voff0,
                                    u64* __restrict__ bitmap) {
  const int words = (n0 + 63) / 64;
  for (int wd = blockIdx.x * blockDim.x + threadIdx.x; wd < words; wd += gridDim.x * blockDim.x) {
    u64 x = 0;
    for (int b = 0; b < 64; ++b) {
      const int v = wd * 64 + b;
      if (v < n0 && (side0[v] ^ side0[voff0[gid0[v]]])) x |= 1ull << b;
    }
    bitmap[wd] = x;
  }
}

// Input check: no entry may leave its graph.
__global__ void batch_check_edges_kernel(int n, const int64_t* __restrict__ rp,
                                         const int* __restrict__ col,
                                         const int* __restrict__ gid, DevState* st) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nwarps) {
    const int gu = gid[u];
    bool bad = false;
    for (long long e = rp[u] + lane; e < rp[u + 1]; e += 32)
      if (gid[col[e]] != gu) bad = true;
    if (__any_sync(FULL, bad) && lane == 0) set_error(st, ERR_INPUT);
  }
}

__global__ void u64_to_i64_kernel(const unsigned long long* __restrict__ a, int G,
                                  long long* __restrict__ out) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    out[g] = (long long)a[g];
}

}  // namespace

cudaError_t batch_gid(const int* voff, int G, int n, int* gid, cudaStream_t s, int* launches) {
  gid_fill_kernel<<<gridb(n, 256), 256, 0, s>>>(voff, G, n, gid);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_start(int G, unsigned long long* lam_g, int* done_g, cudaStream_t s,
                        int* launches) {
  batch_start_kernel<<<gridb(G, 256), 256, 0, s>>>(G, lam_g, done_g);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_round_reset(int G, const BatchState& b, cudaStream_t s, int* launches) {
  batch_round_reset_kernel<<<gridb(G, 256), 256, 0, s>>>(G, b.lam_g, b.lam_before, b.deg_best,
                                                          b.cf_best, b.cf_len, b.marks_g,
                                                          b.wit_kind);
  ++*launches;
  return cudaGetLastError();
}

template <typename WT>
cudaError_t batch_degree_bound(int n, int G, const WT* deg, const BatchState& b, int* newly_done,
                               cudaStream_t s, int* launches) {
  batch_degmin_kernel<WT><<<gridb(n, 256), 256, 0, s>>>(n, deg, b.gid, b.done_g, b.deg_best);
  batch_apply_deg_kernel<<<gridb(G, 256), 256, 0, s>>>(G, b.voff, b.deg_best, b.lam_g, b.done_g,
                                                       newly_done);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t batch_witness(int G, int n0, const BatchState& b, const int* visit_log, int table,
                          const int* pass_len, const int* seq_order, uint8_t* cur,
                          const int* map0, uint8_t* side0, DevState* st, cudaStream_t s,
                          int* launches) {
  batch_witness_decide_kernel<<<gridb(G, 256), 256, 0, s>>>(G, b.lam_g, b.lam_before, b.deg_best,
                                                            b.cf_best, b.wit_kind, b.wit_x, st);
  batch_witness_list_kernel<<<G, 256, 0, s>>>(G, b.voff, b.wit_kind, b.wit_x, b.cf_len,
                                              visit_log, table, pass_len, seq_order, cur);
  batch_witness_apply_kernel<<<gridb(n0, 256), 256, 0, s>>>(n0, b.gid0, map0, b.wit_kind,
                                                            b.wit_x, cur, side0);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t batch_collapse(int n, const BatchState& b, int* parent, cudaStream_t s,
                           int* launches) {
  batch_collapse_kernel<<<gridb(n, 256), 256, 0, s>>>(n, b.gid, b.voff, b.done_g, parent);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_new_offsets(int G, const BatchState& b, const int* rank, const DevState* st,
                              cudaStream_t s, int* launches) {
  batch_new_offsets_kernel<<<gridb(G + 1, 256), 256, 0, s>>>(G, b.voff, rank, st, b.voff_next);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_bitmap(const uint8_t* side0, int n0, const BatchState& b, u64* bitmap,
                         cudaStream_t s, int* launches) {
  batch_bitmap_kernel<<<gridb((n0 + 63) / 64, 256), 256, 0, s>>>(side0, n0, b.gid0, b.voff0,
                                                                  bitmap);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_check_edges(int n, const int64_t* rp, const int* col, const int* gid,
                              DevState* st, cudaStream_t s, int* launches) {
  batch_check_edges_kernel<<<gridb((long long)n * 32, 256), 256, 0, s>>>(n, rp, col, gid, st);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t batch_values(const unsigned long long* lam_g, int G, long long* out, cudaStream_t s,
                         int* launches) {
  u64_to_i64_kernel<<<gridb(G, 256), 256, 0, s>>>(lam_g, G, out);
  ++*launches;
  return cudaGetLastError();
}

template cudaError_t batch_degree_bound<int32_t>(int, int, const int32_t*, const BatchState&, int*,
                                                 cudaStream_t, int*);
template cudaError_t batch_degree_bound<int64_t>(int, int, const int64_t*, const BatchState&, int*,
                                                 cudaStream_t, int*);

}  // namespace mc
