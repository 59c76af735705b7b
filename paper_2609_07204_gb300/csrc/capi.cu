// capi.cu -- C ABI and host driver of the contraction rounds (Algorithm 2).
//
// One graph object owns all device memory of a solve, allocated once at
// creation (sizes only shrink across rounds): the canonical input CSR, two
// ping-pong CSR buffers for the contracted graphs, sort buffers and the
// per-vertex arrays of the round kernels.  A round is a fixed sequence of
// kernels on the graph's stream with a few small device->host reads of the
// DevState block (bound, mark counts, new sizes) between phases.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mincut.h"
#include "common.cuh"
#include "kernels.h"

using namespace mc;

namespace {

thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return status;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(MINCUT_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,     \
                  cudaGetErrorString(e_));                                         \
  } while (0)

int bits_for(long long x) {  // bits to hold values in [0, x)
  int b = 1;
  while (b < 62 && (1ll << b) < x) ++b;
  return b;
}

__global__ void iota_kernel(int* a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}
__global__ void widen32_kernel(const int32_t* __restrict__ in, int64_t* __restrict__ out, long long M) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (int64_t)in[i];
}
// Device address of the host range [p, p + bytes) when the device can read
// it in place (pinned or registered host memory mapped into the device's
// address space, both ends in such memory at the same offset), else NULL.
const void* mapped_host_range(const void* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  const char* last = static_cast<const char*>(p) + bytes - 1;
  if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (b.type != cudaMemoryTypeHost || !b.devicePointer) return nullptr;
  if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) !=
      (ptrdiff_t)(bytes - 1))
    return nullptr;
  return a.devicePointer;
}

// Sum and minimum of the raw input weights; row_ptr monotonicity.
__global__ void input_stats_kernel(const int64_t* __restrict__ rp, int n, const int32_t* __restrict__ w,
                                   long long M, unsigned long long* out /* [sum, neg, badrp] */) {
  unsigned long long s = 0, neg = 0, bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x) {
    const int32_t x = w[i];
    if (x < 0) neg = 1; else s += (unsigned long long)x;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (rp[i] > rp[i + 1] || rp[i] < 0) bad = 1;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) {
    if (s) atomicAdd(&out[0], s);
    if (neg) atomicOr(&out[1], 1ull);
  }
  if (bad) atomicOr(&out[2], 1ull);
}
__global__ void reset_round_kernel(DevState* st) {
  st->marks_pr = 0;
  st->marks_cf = 0;
  st->emit_count = 0;
  st->deg_val = ~0ull;
  st->deg_arg = -1;
  st->lp_val = ~0ull;
  st->lp_label = -1;
  st->cf_val = ~0ull;
  st->cf_pass = -1;
  st->cf_len = 0;
  st->cf_nscanned = 0;
  st->cf_nmarks = 0;
  st->claimed = 0;
}

}  // namespace

struct Alloc {
  void* p;
  size_t bytes;
};

struct mincut_graph {
  cudaStream_t stream = nullptr;
  mincut_allocator alloc{};
  bool user_alloc = false;
  std::vector<Alloc> allocs;
  bool wt64 = false;
  int sms = kDefaultSms;
  // canonical input
  int n0 = 0;
  long long M0 = 0, Mraw = 0;
  int64_t* rp0 = nullptr;
  int* col0 = nullptr;
  void* w0 = nullptr;
  cudaMemPool_t pool = nullptr;  // library pool of the graph's device (no user allocator)
  bool rowwise = true;           // contraction may take the row-wise path
  // current state (cur < 0: the input)
  int n = 0;
  long long M = 0;
  int cur = -1;
  int64_t* rp[2]{};
  int* col[2]{};
  void* w[2]{};
  // scratch
  u64* keys[2]{};
  void* vals[2]{};
  int* tile_row = nullptr;
  void* deg0 = nullptr;     // degrees of the canonical input
  void* degb[2]{};          // degrees of the ping-pong CSRs
  unsigned long long* blk = nullptr;
  unsigned* short_bits = nullptr;  // n / 32: rows within the PR3/PR4 budget
  int *parent = nullptr, *L = nullptr, *flags = nullptr, *rank = nullptr, *part = nullptr,
      *uid = nullptr, *owner = nullptr, *gmin = nullptr, *map0 = nullptr;
  uint8_t *side0 = nullptr, *cur_side = nullptr;
  u64* bitmap_dev = nullptr;
  // label propagation (allocated on first use)
  int* lab[2]{};
  int* lp_chunk0 = nullptr;
  long long* lp_tbase = nullptr;
  unsigned long long* lp_best = nullptr;
  long long* lp_cut = nullptr;
  int *lp_size = nullptr, *long_rows = nullptr, *long_count = nullptr, *pool_lab = nullptr;
  // row-wise contraction (allocated at the first contraction that uses it)
  RowScratch rows{};
  long long acc_zeroed = 0;  // dense accumulator slots known to be zero
  bool m_pending = false;    // M of the current graph is in st->m_rows (not yet read)
  int64_t* rpG = nullptr;
  int* colG = nullptr;
  void* wG = nullptr;
  void* side_w = nullptr;
  long long* pool_sc = nullptr;
  long long pool_slots = 0;
  unsigned long long* pool_cursor = nullptr;
  // CAPFOREST
  int max_passes = 0, max_table = 0;
  int* visit_log = nullptr;
  unsigned long long* pass_best = nullptr;
  int *pass_len = nullptr, *pass_counter = nullptr;
  void* seq_r = nullptr;
  int* seq_mark = nullptr;  // the sequential pass's marks until the pass ends
  unsigned long long* seq_tree = nullptr;
  int* seq_order = nullptr;
  // several sequential passes at once (allocated at first use)
  int seq_multi_k = 0;
  void* seq_multi_r = nullptr;
  unsigned long long* seq_multi_tree = nullptr;
  int* seq_multi_order = nullptr;
  int* seq_multi_mark = nullptr;
  // sort
  SortScratch sort{};
  // state
  DevState* st = nullptr;
  DevState* hst = nullptr;  // pinned mirror
  int* m2_dev = nullptr;
  int launches = 0;
  Profiler* prof = nullptr;
  // packed batch (batch.G > 0)
  BatchState batch;
  std::vector<long long> voff0_h;
  std::vector<int> batch_m;  // entries of each graph of a batch (canonical input)
  int max_graph_n = 0;
  // graphs solved one per warp (batch_warp.cu)
  int bw_threshold = -1;      // the list below holds the graphs with n <= this
  int bw_auto = -1;           // threshold chosen by timing (batch_small_n = 0), -1: not yet
  int* bw_list = nullptr;     // graph ids, most entries first
  int bw_count = 0, bw_nmax = 0, bw_mmax = 0;
  int* bw_cursor = nullptr;
  int* bw_scratch = nullptr;
  long long bw_scratch_words = 0;
  int bw_slots = 0;
  // the launches of a solve whose graphs all take the one-warp solver,
  // captured as a CUDA graph at the second solve with the same split
  cudaGraphExec_t bw_exec = nullptr;
  cudaStream_t bw_capture = nullptr;  // private stream the launches are captured on
  int bw_exec_launches = 0;
  struct BwKey {
    int threshold = -1;
    const int* scratch = nullptr;
    const int* voff = nullptr;  // the offsets buffer in use (round solves swap it)
    unsigned pr = 0;
    bool operator==(const BwKey& o) const {
      return threshold == o.threshold && scratch == o.scratch && voff == o.voff && pr == o.pr;
    }
  } bw_key, bw_exec_key;
  int bw_key_runs = 0;
  unsigned long long* batch_levels = nullptr;
  long long* batch_vals = nullptr;
  long long spin_limit = 1ll << 22;

  const int64_t* crp() const { return cur < 0 ? rp0 : rp[cur]; }
  const int* ccol() const { return cur < 0 ? col0 : col[cur]; }
  const void* cw() const { return cur < 0 ? w0 : w[cur]; }
  void* cdeg() const { return cur < 0 ? deg0 : degb[cur]; }
};

namespace mc {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
Profiler* prof_create();
void prof_destroy(Profiler* p);
void prof_flush(Profiler* p);
void prof_read(const Profiler* p, int cat, double* ms, long long* launches, long long* units);
void prof_reset(Profiler* p);
}  // namespace mc

namespace {

// Concurrent CAPFOREST passes per round: one per 4 vertices, at least 256, at
// most 48 per SM (their visit logs are max_passes x 1024 ints).
int graph_max_passes(long long n, int sms) {
  return (int)std::max<long long>(256, std::min<long long>(n / 4, (long long)sms * 48));
}

// Installs the graph's profiler on this thread for the duration of a call.
struct ProfGuard {
  mincut_graph* g;
  bool on;
  ProfGuard(mincut_graph* gg, bool enable) : g(gg), on(enable) {
    if (on) {
      if (!g->prof) g->prof = prof_create();
      tl_prof = g->prof;
    }
  }
  ~ProfGuard() {
    if (on) {
      cudaStreamSynchronize(g->stream);
      prof_flush(g->prof);
      tl_prof = nullptr;
    }
  }
};

// Without a user allocator, device memory comes from a stream-ordered pool
// per device owned by the library.  The pool keeps the blocks that graphs
// free (no release threshold), so creating and destroying graphs of similar
// size reuses mapped memory instead of mapping it again for every graph;
// mincut_release_cached() hands the unused blocks back to the driver.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaMemPool_t lib_pool(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

// Pinned host mirrors of DevState, handed out from slabs that live as long
// as the process (a page-locking call per graph costs more than the graph's
// small solves).
std::mutex g_pin_mu;
std::vector<DevState*> g_pin_free;

DevState* pinned_state_get() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr int kSlab = 64;
    DevState* slab = nullptr;
    if (cudaMallocHost(&slab, kSlab * sizeof(DevState)) != cudaSuccess) return nullptr;
    for (int i = kSlab - 1; i >= 0; --i) g_pin_free.push_back(slab + i);
  }
  DevState* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_state_put(DevState* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

void* dev_alloc(mincut_graph* g, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  bytes = (bytes + 255) / 256 * 256;
  void* p = nullptr;
  if (g->user_alloc) {
    p = g->alloc.alloc(bytes, (void*)g->stream, g->alloc.ctx);
  } else {
    if (!g->pool) {
      int dev = 0;
      cudaGetDevice(&dev);
      g->pool = lib_pool(dev);
    }
    const cudaError_t rc = g->pool ? cudaMallocFromPoolAsync(&p, bytes, g->pool, g->stream)
                                   : cudaMallocAsync(&p, bytes, g->stream);
    if (rc != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) g->allocs.push_back({p, bytes});
  return p;
}

void dev_free(mincut_graph* g, void* p) {
  for (size_t i = 0; i < g->allocs.size(); ++i)
    if (g->allocs[i].p == p) {
      if (g->user_alloc) g->alloc.free(p, g->allocs[i].bytes, (void*)g->stream, g->alloc.ctx);
      else cudaFreeAsync(p, g->stream);
      g->allocs.erase(g->allocs.begin() + (long)i);
      return;
    }
}

template <typename T>
bool galloc(mincut_graph* g, T** out, long long count) {
  *out = static_cast<T*>(dev_alloc(g, (size_t)std::max<long long>(count, 1) * sizeof(T)));
  return *out != nullptr;
}

void free_all(mincut_graph* g) {
  if (g->bw_exec) {
    cudaStreamSynchronize(g->stream);
    cudaGraphExecDestroy(g->bw_exec);
    g->bw_exec = nullptr;
  }
  if (g->bw_capture) {
    cudaStreamDestroy(g->bw_capture);
    g->bw_capture = nullptr;
  }
  for (auto& a : g->allocs) {
    if (g->user_alloc) g->alloc.free(a.p, a.bytes, (void*)g->stream, g->alloc.ctx);
    else cudaFreeAsync(a.p, g->stream);
  }
  g->allocs.clear();
  if (g->hst) {
    // the mirror may still be the target of a copy on the graph's stream
    cudaStreamSynchronize(g->stream);
    pinned_state_put(g->hst);
  }
  g->hst = nullptr;
}

int sync_state(mincut_graph* g) {
  CK(cudaMemcpyAsync(g->hst, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  const unsigned e = g->hst->error;
  if (e & ERR_TIMEOUT) return fail(MINCUT_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
  if (e & ERR_INPUT) return fail(MINCUT_ERR_INVALID, "index out of range or negative weight");
  if (e & ERR_ASYM) return fail(MINCUT_ERR_INVALID, "input CSR is not symmetric");
  if (e & ERR_OVERFLOW) return fail(MINCUT_ERR_OVERFLOW, "a device capacity was exceeded");
  if (e & ERR_INTERNAL)
    return fail(MINCUT_ERR_INTERNAL, "internal consistency check failed (check %d)",
                g->hst->internal_code);
  return MINCUT_OK;
}

int set_lambda(mincut_graph* g, long long lam) {
  unsigned long long v = (unsigned long long)lam;
  CK(cudaMemcpyAsync(&g->st->lambda, &v, sizeof(v), cudaMemcpyHostToDevice, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  return MINCUT_OK;
}

int ensure_rows(mincut_graph* g) {
  if (g->rows.cnt) return MINCUT_OK;
  const size_t wsz = g->wt64 ? 8 : 4;
  const long long n = g->n0, M = std::max<long long>(g->M0, 1);
  RowScratch& r = g->rows;
  if (!galloc(g, &r.cnt, n + 1) || !galloc(g, &r.gen, n + 1) || !galloc(g, &r.len, n + 1) ||
      !galloc(g, &r.kcnt, n + 1) || !galloc(g, &r.off, n + 1) ||
      !galloc(g, &r.part, (n + 1) / 4096 + 3) ||
      !galloc(g, &r.side_v, M) || !galloc(g, &r.vinfo, n + 1) || !galloc(g, &g->rpG, n + 1) ||
      !galloc(g, &r.dsum, n + 1) || !galloc(g, &r.did, n + 1) ||
      !galloc(g, &r.chunk, 4 * M / kDenseChunk + n + 64) ||
      !galloc(g, &r.dense_group, n + 1) ||
      !(r.acc = dev_alloc(g, (size_t)4 * M * wsz)) ||
      !galloc(g, &g->colG, M) ||
      !(g->wG = dev_alloc(g, (size_t)M * wsz)) || !(g->side_w = dev_alloc(g, (size_t)M * wsz)) ||
      !galloc(g, &r.rep, n + 1) || !galloc(g, &r.fcl, n + 1) || !galloc(g, &r.kpc, n + 1) ||
      !galloc(g, &r.side_c, M) || !(r.rec = dev_alloc(g, (size_t)(n + 1) * 16)) ||
      !galloc(g, &r.tile_ht, M / kEntryTile + 2) || !galloc(g, &r.tile_rowG, M / kEntryTile + 2) ||
      !galloc(g, &r.list, n + 1) || !galloc(g, &r.list_len, 2) ||
      !galloc(g, &r.vmap, n / 32 + 2) || !galloc(g, &r.mvbits, n / 32 + 2)) {
    r.cnt = nullptr;
    return fail(MINCUT_ERR_OOM, "row-wise contraction buffers");
  }
  r.single_entries = &g->st->single_entries;
  r.dense_entries = &g->st->dense_entries;
  r.ndense = &g->st->ndense;
  r.total = &g->st->m_rows;
  r.dense_slots = 4 * M;
  g->acc_zeroed = 0;  // accumulator slots are cleared as rounds first need them
  return MINCUT_OK;
}

// Buffers of up to `want` simultaneous sequential passes over graphs of up
// to n0 vertices, capped at about 2 GB; returns the number of passes they
// hold (at least 1 when the allocation succeeded, 0 on failure).
int ensure_seq_multi(mincut_graph* g, int want) {
  if (g->seq_multi_k >= want) return want;
  const size_t wsz = g->wt64 ? 8 : 4;
  const long long n = g->n0;
  const long long per = n * (long long)(8 + 2 * wsz) + seq_tree_words((int)n) * 8;
  const long long cap = std::max<long long>(1, (2ll << 30) / std::max<long long>(per, 1));
  const int k = (int)std::min<long long>(want, cap);
  if (k <= g->seq_multi_k) return g->seq_multi_k;
  if (g->seq_multi_k > 0) {  // grow: the previous buffers go back to the allocator
    dev_free(g, g->seq_multi_r);
    dev_free(g, g->seq_multi_tree);
    dev_free(g, g->seq_multi_order);
    dev_free(g, g->seq_multi_mark);
    g->seq_multi_r = nullptr;
    g->seq_multi_tree = nullptr;
    g->seq_multi_order = nullptr;
    g->seq_multi_mark = nullptr;
    g->seq_multi_k = 0;
  }
  if (!(g->seq_multi_r = dev_alloc(g, (size_t)k * n * 2 * wsz)) ||
      !galloc(g, &g->seq_multi_tree, (long long)k * seq_tree_words((int)n)) ||
      !galloc(g, &g->seq_multi_order, (long long)k * n) ||
      !galloc(g, &g->seq_multi_mark, (long long)k * n))
    return 0;
  g->seq_multi_k = k;
  return k;
}

int ensure_lp(mincut_graph* g) {
  if (g->lab[0]) return MINCUT_OK;
  const size_t wsz = g->wt64 ? 8 : 4;
  (void)wsz;
  g->pool_slots = 2 * std::max<long long>(g->M0, 1);
  if (!galloc(g, &g->lab[0], g->n0) || !galloc(g, &g->lab[1], g->n0) ||
      !galloc(g, &g->lp_cut, g->n0) || !galloc(g, &g->lp_size, g->n0) ||
      !galloc(g, &g->long_rows, 2ll * g->n0) || !galloc(g, &g->long_count, 4) ||
      !galloc(g, &g->lp_chunk0, g->n0) || !galloc(g, &g->lp_tbase, g->n0) ||
      !galloc(g, &g->lp_best, g->n0) ||
      !galloc(g, &g->pool_lab, g->pool_slots) || !galloc(g, &g->pool_sc, g->pool_slots) ||
      !galloc(g, &g->pool_cursor, 1))
    return fail(MINCUT_ERR_OOM, "label propagation buffers");
  return MINCUT_OK;
}

// Contraction of the current graph by the union-find state in g->parent:
// relabel, emit, sort, build; the result becomes the current graph.
// Row-wise contraction of the current graph (most groups single vertices):
// singleton rows rebuilt in place, the other rows through emit / sort /
// build into a general CSR, then both placed into the next buffers.
template <typename WT>
int contract_rows(mincut_graph* g, int n2, int nxt, long long* m2_out, bool defer_m) {
  cudaStream_t s = g->stream;
  const int n = g->n;
  const long long M = g->M;
  const int vbits = bits_for(n2);
  RowScratch& rs = g->rows;
  const int ndense = g->hst->ndense;  // read with the relabel's synchronisation
  // (the emit of the general rows reads only their entries: it is timed
  // with the row-wise pass, whose algorithmic bytes cover every entry)
  { ProfScope ps(P_ROWS, M, s);
    CK(rows_count<WT>(n, M, g->crp(), g->ccol(), (const WT*)g->cw(), g->L, g->flags, g->rank,
                      g->tile_row, rs, (WT*)g->side_w, s, &g->launches));
    CK(rows_dense_accumulate<WT>(n, M, n2, g->crp(), g->ccol(), (const WT*)g->cw(), g->L,
                                 g->tile_row, rs, ndense, (WT*)g->side_w, s, &g->launches));
    CK(cudaMemsetAsync(&g->st->emit_count, 0, sizeof(long long), s));
    CK(emit_pairs<WT>(n, M, g->crp(), g->ccol(), (const WT*)g->cw(), g->L, vbits, g->tile_row,
                      g->keys[0], (WT*)g->vals[0], g->st, 0, s, &g->launches, rs.gen)); }
  int rc = sync_state(g);
  if (rc) return rc;
  const long long N = g->hst->emit_count;
  bool alt = false;
  CK(radix_sort_pairs<WT>(g->keys[0], (WT*)g->vals[0], g->keys[1], (WT*)g->vals[1], (int)N,
                          2 * vbits, g->sort, g->st, g->spin_limit, s, &alt, &g->launches));
  { ProfScope ps(P_BUILD, N, s);
    CK(build_csr<WT>(alt ? g->keys[1] : g->keys[0], (WT*)(alt ? g->vals[1] : g->vals[0]), (int)N,
                     vbits, n2, g->uid, g->part, g->rpG, g->colG, (WT*)g->wG, g->st, g->m2_dev,
                     reinterpret_cast<int*>(alt ? g->keys[0] : g->keys[1]), s, &g->launches)); }
  int mG = 0;
  CK(cudaMemcpyAsync(&mG, g->m2_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  { ProfScope ps(P_ROWS, M, s);
    CK(rows_finish<WT>(n, M, n2, g->crp(), g->ccol(), (const WT*)g->cw(), g->L, rs, ndense,
                       (WT*)g->side_w, g->rpG, g->colG, (const WT*)g->wG, mG, g->tile_row,
                       g->rp[nxt], g->col[nxt], (WT*)g->w[nxt], (WT*)g->degb[nxt], s,
                       &g->launches)); }
  if (defer_m) {
    // the entry count is read with the next synchronisation (st->m_rows)
    *m2_out = -1;
    return MINCUT_OK;
  }
  rc = sync_state(g);
  if (rc) return rc;
  *m2_out = g->hst->m_rows;
  return MINCUT_OK;
}

// Contraction of the current graph by the union-find state in g->parent:
// relabel, then either the row-wise path (when at least a quarter of the
// entries lie in rows of single-vertex groups or of dense groups) or emit /
// sort / build of all entries; the result becomes the current graph.
// defer_m: on the row-wise path, leave the new entry count in st->m_rows for
// the caller's next synchronisation (g->m_pending) instead of waiting here.
template <typename WT>
int contract_current(mincut_graph* g, int* n2_out, long long* m2_out, bool compose,
                     bool defer_m = false) {
  cudaStream_t s = g->stream;
  const int n = g->n;
  const long long M = g->M;
  { ProfScope ps(P_UF, n, s);
    CK(uf_relabel(g->parent, g->L, g->flags, g->rank, g->part, n, g->st, s, &g->launches)); }
  // the row classification runs before the vertex count n2 is known on the
  // host (n bounds it): one synchronisation serves both
  const bool try_rows = g->rowwise && M > 0 && n > 2;
  if (try_rows) {
    int rc = ensure_rows(g);
    if (rc) return rc;
    ProfScope ps(P_UF, n, s);
    CK(rows_classify(n, n, g->crp(), g->L, g->rows, s, &g->launches));
    CK(rows_dense_mark(n, &g->st->n_next, g->rows, s, &g->launches));
  }
  int rc = sync_state(g);
  if (rc) return rc;
  const int n2 = g->hst->n_next;
  const int nxt = g->cur == 0 ? 1 : 0;
  bool rowwise = false;
  if (try_rows && n2 > 1) {
    rowwise = 4 * (long long)(g->hst->single_entries + g->hst->dense_entries) >= M;
    if (rowwise) {
      // the dense accumulators this round uses must be zero: slots below
      // acc_zeroed are (the writing kernel clears what it read)
      const long long need =
          (long long)std::min(g->hst->ndense, dense_capacity(n2, g->rows)) * n2;
      if (need > g->acc_zeroed) {
        const size_t wsz = g->wt64 ? 8 : 4;
        CK(cudaMemsetAsync(static_cast<char*>(g->rows.acc) + (size_t)g->acc_zeroed * wsz, 0,
                           (size_t)(need - g->acc_zeroed) * wsz, s));
        g->acc_zeroed = need;
      }
    }
  }
  long long m2 = 0;
  if (rowwise) {
    rc = contract_rows<WT>(g, n2, nxt, &m2, defer_m);
    if (rc) return rc;
  } else {
    const int vbits = bits_for(n2);
    CK(cudaMemsetAsync(&g->st->emit_count, 0, sizeof(long long), s));
    { ProfScope ps(P_EMIT, M, s);
      CK(emit_pairs<WT>(n, M, g->crp(), g->ccol(), (const WT*)g->cw(), g->L, vbits, g->tile_row,
                        g->keys[0], (WT*)g->vals[0], g->st, 0, s, &g->launches)); }
    rc = sync_state(g);
    if (rc) return rc;
    const long long N = g->hst->emit_count;
    bool alt = false;
    CK(radix_sort_pairs<WT>(g->keys[0], (WT*)g->vals[0], g->keys[1], (WT*)g->vals[1], (int)N,
                            2 * vbits, g->sort, g->st, g->spin_limit, s, &alt, &g->launches));
    { ProfScope ps(P_BUILD, N, s);
      CK(build_csr<WT>(alt ? g->keys[1] : g->keys[0], (WT*)(alt ? g->vals[1] : g->vals[0]),
                       (int)N, vbits, n2, g->uid, g->part, g->rp[nxt], g->col[nxt],
                       (WT*)g->w[nxt], g->st, g->m2_dev,
                       reinterpret_cast<int*>(alt ? g->keys[0] : g->keys[1]), s, &g->launches)); }
    int m2i = 0;
    CK(cudaMemcpyAsync(&m2i, g->m2_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    rc = sync_state(g);
    if (rc) return rc;
    m2 = m2i;
    { ProfScope ps(P_DEGREE, m2, s);
      CK(row_degrees<WT>(n2, m2, g->rp[nxt], (const WT*)g->w[nxt], g->tile_row, (WT*)g->degb[nxt],
                         s, &g->launches)); }
  }
  if (compose) {
    ProfScope ps(P_UF, g->n0, s);
    CK(compose_map(g->map0, g->L, g->n0, s, &g->launches));
  }
  g->cur = nxt;
  g->n = n2;
  g->M = m2;
  g->m_pending = m2 < 0;
  *n2_out = n2;
  *m2_out = m2;
  return MINCUT_OK;
}

// Graphs of at most this many vertices skip the concurrent passes in the
// rounds after one where they marked almost nothing.
constexpr int kSkipConcurrentMaxN = 8192;

struct RoundCfg {
  int lp_iters, lp_min_n;
  bool lp_now;
  uint32_t pr_mask;
  long long pr_budget;
  int capforest;  // 0 none, 1 concurrent (+ sequential fallback), 2 sequential from cf_start
                  // (block pass, smaller-id ties), 4 one warp-driven pass from cf_start
                  // (neighbour-first ties)
  int cf_private = 0;  // concurrent passes with private visit sets
  int seq_passes = 1;  // sequential passes when the concurrent ones mark nothing (0: auto)
  int seq_kernel = 0;  // 0: warp-driven passes; 1: block passes (smaller-id ties)
  bool coarsen = false;  // heuristic round: also join every label-propagation cluster
  bool skip_concurrent = false;  // capforest 1: go straight to the whole-graph passes
  // capforest 1, >= 0: the concurrent passes stand down (decided on the
  // device) when the round's PR tests hooked at least this many edges
  long long cc_skip_pr = -1;
  // skip_concurrent rounds: run the whole passes without first reading the
  // PR count (set while the rounds barely shrink the graph)
  bool eager_seq = false;
  int cf_start;
  int passes, table;
  unsigned long long seed;
  uint8_t* pr_flags_host;
  int* cf_order_host;
  int* cf_marks_host;
  long long cf_marks_cap;
  int* lp_labels_host;
};

struct RoundOut {
  bool stopped = false;
  bool seq_pass = false;
  long long lambda = kInf;
  long long marks_pr = 0, marks_cf = 0;
  long long marks_cc = 0;  // of marks_cf, those of the concurrent passes
  bool cc_ran = false;     // the concurrent passes ran (were not skipped)
  long long cf_nscanned = 0, cf_nmarks = 0;
  int src = 0;  // which bound source set lambda this round
};

// Marking phase of one round on the current graph: degree bound, LP bound,
// PR marks and CAPFOREST marks (all hooked into g->parent).  Updates g->side0
// when lambda improves below lambda_before.
template <typename WT>
int mark_round(mincut_graph* g, const RoundCfg& c, long long lambda_before, RoundOut* o) {
  cudaStream_t s = g->stream;
  const int n = g->n;
  const int64_t* rp = g->crp();
  const int* col = g->ccol();
  const WT* w = (const WT*)g->cw();
  const WT* deg = (const WT*)g->cdeg();
  reset_round_kernel<<<1, 1, 0, s>>>(g->st);
  ++g->launches;
  if (n >= 2) {
    ProfScope ps(P_DEGREE, n, s);
    CK(degrees_min<WT>(deg, n, g->blk, g->st, s, &g->launches));
  }
  int rc = sync_state(g);
  if (rc) return rc;
  if (g->m_pending) {  // the previous contraction's entry count came with this sync
    g->M = g->hst->m_rows;
    g->m_pending = false;
  }
  const long long M = g->M;
  long long lam = (long long)g->hst->lambda;
  if (lam < lambda_before) {
    ProfScope ps(P_WITNESS, g->n0, s);
    CK(side_from_vertex(g->side0, g->map0, g->n0, g->hst->deg_arg, s, &g->launches));
    o->src = 1;
    lambda_before = lam;
  }
  o->lambda = lam;
  if (n <= 2 || lam == 0) {
    o->stopped = true;
    return MINCUT_OK;
  }
  { ProfScope ps(P_TILES, n, s);
    CK(tile_rows(rp, n, M, g->tile_row, s, &g->launches)); }
  const int* lab_final = nullptr;
  if (c.lp_now && c.lp_iters > 0 && n >= c.lp_min_n) {
    rc = ensure_lp(g);
    if (rc) return rc;
    for (int it = 0; it < c.lp_iters; ++it) {
      ProfScope ps(P_LP_SWEEP, M, s);
      if (it == 0 && sizeof(WT) == 4) {  // identity labels: heaviest-neighbour sweep
        CK(lp_first_sweep<WT>(n, M, rp, col, w, g->tile_row, 0,
                              reinterpret_cast<unsigned long long*>(g->lp_cut), g->lab[1], s,
                              &g->launches));
        continue;
      }
      if (it == 0) {
        iota_kernel<<<std::min((n + 255) / 256, g->sms * 8), 256, 0, s>>>(g->lab[0], n);
        ++g->launches;
      }
      LpScratch sc{g->long_rows, g->long_count, g->lp_chunk0, g->lp_tbase, g->lp_best,
                   g->pool_lab, g->pool_sc, g->pool_slots, g->pool_cursor};
      CK(lp_sweep<WT>(n, rp, col, w, g->lab[it & 1], g->lab[(it + 1) & 1], it, sc, g->st, s,
                      &g->launches));
    }
    lab_final = g->lab[c.lp_iters & 1];
    ProfScope ps(P_LP_BOUND, M, s);
    CK(lp_bound<WT>(n, M, rp, col, w, lab_final, g->tile_row, g->lp_cut, g->lp_size, g->blk,
                    g->st, s, &g->launches));
    if (c.lp_labels_host)
      CK(cudaMemcpyAsync(c.lp_labels_host, lab_final, (size_t)n * sizeof(int),
                         cudaMemcpyDeviceToHost, s));
  }
  { ProfScope ps(P_UF, n, s);
    CK(uf_init(g->parent, n, s, &g->launches));
    if (c.coarsen && lab_final)
      CK(uf_from_groups(g->parent, lab_final, g->gmin, n, g->st, s, &g->launches)); }
  uint8_t* flags_dev = c.pr_flags_host ? reinterpret_cast<uint8_t*>(g->vals[1]) : nullptr;
  if (c.pr_mask) {
    ProfScope ps(P_PR, M, s);
    CK(pr_marks<WT>(n, M, rp, col, w, deg, g->tile_row, c.pr_mask, c.pr_budget, g->parent,
                    flags_dev, g->short_bits, g->st, s, &g->launches));
  }
  if (c.capforest == 1 && n > 2 && !c.skip_concurrent) {
    CK(cudaMemsetAsync(g->owner, 0, (size_t)n * sizeof(int), s));
    PassConfig pc;
    pc.table = c.table;
    pc.warps_per_block = 4;
    pc.passes = std::min(c.passes, g->max_passes);
    pc.seed = c.seed;
    pc.private_visit = c.cf_private;
    pc.skip_pr = c.cc_skip_pr;
    ProfScope ps(P_CF_PASSES, M, s);
    CK(capforest_passes<WT>(n, rp, col, w, deg, g->owner, g->parent, g->visit_log,
                            g->pass_best, g->pass_len, g->pass_counter, pc, g->st, s,
                            &g->launches));
  }
  // a round whose concurrent passes stand down because the last one needed
  // the whole passes runs those again without first reading the PR count
  // (one host synchronisation less; nothing since the degree bound's
  // synchronisation has changed the bound: no LP, PR does not lower it)
  const bool eager_seq = c.eager_seq && c.capforest == 1 && n > 2 && c.skip_concurrent &&
                         !c.lp_now && !flags_dev;
  bool need_seq = eager_seq;
  if (!eager_seq) {
    rc = sync_state(g);
    if (rc) return rc;
    if (flags_dev && M > 0)
      CK(cudaMemcpyAsync(c.pr_flags_host, flags_dev, (size_t)M, cudaMemcpyDeviceToHost, s));
    const long long marks = (long long)(g->hst->marks_pr + g->hst->marks_cf);
    o->marks_pr = (long long)g->hst->marks_pr;
    o->marks_cc = (long long)g->hst->marks_cf;
    o->cc_ran = c.capforest == 1 && n > 2 && !c.skip_concurrent &&
                !(c.cc_skip_pr >= 0 && o->marks_pr >= c.cc_skip_pr);
    // the sequential pass when the round marked nothing (Algorithm 2), and on
    // small graphs (n <= 8192, where a pass costs a few rounds' fixed cost at
    // most) also when it marked so little (fewer edges than n / 64) that
    // contracting would spend a whole round on almost no vertices; its marks
    // only add
    need_seq = c.capforest == 2 || c.capforest == 4 ||
               (c.capforest == 1 && (marks == 0 || (n <= 8192 && marks * 64 < n)));
  }
  // whole passes driven by one warp each (the default), when the bound fits
  // their keys: one pass from cf_start in mode 4, else several from
  // different start vertices with private arrays, as many as keep their hot
  // arrays within a share of L2 (all SMs when they live in shared memory)
  const long long lam_seq = (long long)g->hst->lambda;
  if (need_seq && lam_seq > 0 && warp_pass_key_bytes(lam_seq) > 0 &&
      (c.capforest == 4 || (c.capforest == 1 && c.seq_kernel == 0))) {
    int want = 1;
    if (c.capforest == 1) {
      if (c.seq_passes > 0) {
        want = c.seq_passes;
      } else {
        // passes are independent chains on separate SMs: more of them cost
        // little time and mark more edges, so large graphs collapse in one
        // such round (measured on the planted cut: 4 passes leave one round
        // of whole passes, 2 leave two); the L2 share only raises the count
        const long long hot = warp_pass_hot_bytes(n, sizeof(WT), lam_seq);
        want = hot <= 0 ? g->sms
                        : (int)std::max<long long>(kWarpPassMin, kWarpPassL2Budget / hot);
      }
      want = std::max(1, std::min({want, g->sms, g->max_passes}));
    }
    const int k = ensure_seq_multi(g, want);
    if (k < 1) return fail(MINCUT_ERR_OOM, "sequential pass buffers");
    const int start = c.capforest == 4 ? c.cf_start : 0;
    {
      ProfScope ps(P_CF_SEQ, M, s);
      CK(capforest_warp_passes<WT>(n, M, rp, col, w, deg, k, start, c.seed, lam_seq, g->parent,
                                   (WT*)g->seq_multi_r,
                                   reinterpret_cast<unsigned char*>(g->seq_multi_tree),
                                   seq_tree_words((int)g->n0) * 8, g->seq_multi_order,
                                   g->seq_multi_mark, g->pass_best, g->pass_len,
                                   c.capforest == 1 && n >= kWarpStopMinN ? 1 : 0, g->st, s,
                                   &g->launches));
    }
    rc = sync_state(g);
    if (rc) return rc;
    o->seq_pass = true;
    o->cf_nscanned = g->hst->cf_nscanned;
    o->cf_nmarks = (long long)g->hst->marks_cf;
    if (c.capforest == 4 && (c.cf_order_host || c.cf_marks_host)) {
      // pass 0's visit order, and its marks as (x, y) pairs in scan order:
      // by x's visit position, then by y (rows are sorted by neighbour)
      std::vector<int> ord((size_t)o->cf_nscanned), mk((size_t)n);
      if (o->cf_nscanned > 0)
        CK(cudaMemcpyAsync(ord.data(), g->seq_multi_order, ord.size() * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(mk.data(), g->seq_multi_mark, (size_t)n * sizeof(int),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (c.cf_order_host && !ord.empty())
        memcpy(c.cf_order_host, ord.data(), ord.size() * sizeof(int));
      if (c.cf_marks_host) {
        std::vector<int> pos((size_t)n, INT32_MAX);
        for (size_t i = 0; i < ord.size(); ++i) pos[(size_t)ord[i]] = (int)i;
        std::vector<std::pair<long long, int>> pairs;
        for (int y = 0; y < n; ++y)
          if (mk[(size_t)y] >= 0)
            pairs.push_back({(long long)pos[(size_t)mk[(size_t)y]] * n + y, mk[(size_t)y]});
        std::sort(pairs.begin(), pairs.end());
        const long long cap = std::min<long long>(c.cf_marks_cap, (long long)pairs.size());
        for (long long i = 0; i < cap; ++i) {
          c.cf_marks_host[2 * i] = pairs[(size_t)i].second;
          c.cf_marks_host[2 * i + 1] = (int)(pairs[(size_t)i].first % n);
        }
      }
    }
    need_seq = false;
  }
  // several whole passes from different start vertices, each with private
  // arrays, when the concurrent passes found nothing (not in the modes that
  // report the single pass's order and marks)
  if (need_seq && (long long)g->hst->lambda > 0 && c.capforest == 1 && c.seq_passes != 1 &&
      !c.cf_marks_host && !c.cf_order_host) {
    const int want = c.seq_passes > 0 ? c.seq_passes : g->sms;
    const int k = ensure_seq_multi(g, std::min({want, std::max(2, n / 2), g->max_passes}));
    if (k > 1) {
      {
        ProfScope ps(P_CF_SEQ, M, s);
        CK(capforest_sequential_multi<WT>(n, M, rp, col, w, deg, k, c.seed, g->parent,
                                          (WT*)g->seq_multi_r, g->seq_multi_tree,
                                          g->seq_multi_order, g->seq_multi_mark, g->pass_best,
                                          g->pass_len, g->st, s,
                                          &g->launches));
      }
      rc = sync_state(g);
      if (rc) return rc;
      o->seq_pass = true;
      need_seq = false;
    }
  }
  // the sequential pass is only useful while the bound is positive
  if (need_seq && (long long)g->hst->lambda > 0) {
    const long long cap = c.cf_marks_host ? std::min(c.cf_marks_cap, M / 2 + 1) : 0;
    int* marks_dev = c.cf_marks_host ? reinterpret_cast<int*>(g->keys[1]) : nullptr;
    const int start = (c.capforest == 2 || c.capforest == 4) ? c.cf_start : 0;
    {
      ProfScope ps(P_CF_SEQ, M, s);
      CK(capforest_sequential<WT>(n, M, rp, col, w, deg, start, g->parent, (WT*)g->seq_r, g->seq_mark,
                                  g->seq_tree, g->seq_order, marks_dev, cap, g->st, s,
                                  &g->launches));
    }
    rc = sync_state(g);
    if (rc) return rc;
    o->seq_pass = true;
    o->cf_nscanned = g->hst->cf_nscanned;
    o->cf_nmarks = (long long)g->hst->marks_cf;
    if (c.cf_order_host && o->cf_nscanned > 0)
      CK(cudaMemcpyAsync(c.cf_order_host, g->seq_order, (size_t)o->cf_nscanned * sizeof(int),
                         cudaMemcpyDeviceToHost, s));
    if (marks_dev) {
      const long long k = std::min<long long>(o->cf_nmarks, cap);
      if (k > 0)
        CK(cudaMemcpyAsync(c.cf_marks_host, marks_dev, (size_t)k * 2 * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
  }
  if (eager_seq) {
    if (!o->seq_pass) {  // (no pass could run: the state is read here)
      rc = sync_state(g);
      if (rc) return rc;
    }
    o->marks_pr = (long long)g->hst->marks_pr;
    o->marks_cc = 0;
  }
  o->marks_cf = (long long)g->hst->marks_cf;
  lam = (long long)g->hst->lambda;
  if (lam < lambda_before) {
    const DevState& h = *g->hst;
    if (lab_final && h.lp_val == (unsigned long long)lam) {
      ProfScope ps(P_WITNESS, g->n0, s);
      CK(side_from_label(g->side0, g->map0, g->n0, lab_final, h.lp_label, s, &g->launches));
      o->src = 2;
    } else if (h.cf_val == (unsigned long long)lam) {
      const int* list = h.cf_pass <= -2 ? g->seq_multi_order + (long long)(-2 - h.cf_pass) * n
                        : h.cf_pass >= 0  ? g->visit_log + (long long)h.cf_pass * c.table
                                          : g->seq_order;
      ProfScope ps(P_WITNESS, g->n0, s);
      CK(side_from_list(g->side0, g->map0, g->n0, g->cur_side, n, list, h.cf_len, s,
                        &g->launches));
      o->src = 3;
    } else {
      return fail(MINCUT_ERR_INTERNAL, "bound improved without a witness");
    }
  }
  o->lambda = lam;
  return MINCUT_OK;
}

// Exact rounds (Algorithm 2 with the round of Sec. 2.1) from the graph's
// current state until it stops; lambda is the best bound so far (its witness
// already in side0).  cf_visit 2 runs the first round with the shared visit
// array and the second with private ones, then keeps the mode that removed
// more vertices per millisecond.
template <typename WT>
int exact_rounds(mincut_graph* g, const mincut_options& op, RoundCfg c, bool lp_allowed,
                 long long* lambda_io, mincut_stats* stl, int* round_io) {
  long long lambda = *lambda_io;
  double rate[2] = {-1.0, -1.0};
  int mode = op.cf_visit == 1 ? 1 : 0;
  bool skip_cc = false;
  // the concurrent passes marked fewer than n / 64 edges the last time they
  // ran: they stand down in rounds whose PR tests hook at least n / 64
  bool cc_low = false;
  bool barely = false;  // the last contraction kept at least half the vertices
  for (;; ++*round_io) {
    const int round = *round_io;
    if (op.max_rounds > 0 && round >= op.max_rounds) break;
    if (op.cf_visit == 2) {
      if (rate[0] < 0) mode = 0;
      else if (rate[1] < 0) mode = 1;
      else mode = rate[1] > rate[0] ? 1 : 0;
    }
    c.cf_private = mode;
    c.skip_concurrent = skip_cc && g->n <= kSkipConcurrentMaxN;
    c.eager_seq = c.skip_concurrent && barely;
    c.cc_skip_pr = cc_low && c.capforest == 1 && op.cf_visit != 2 ? (g->n + 63) / 64 : -1;
    c.lp_now = lp_allowed && (op.lp_every_round || round == 0);
    c.passes = op.passes > 0 ? op.passes : std::max(32, std::min(g->max_passes, g->n / 4));
    c.seed = op.seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(round + 1);
    const auto t0 = std::chrono::steady_clock::now();
    const int n_before = g->n;
    RoundOut o;
    int rc = mark_round<WT>(g, c, lambda, &o);
    if (rc) return rc;
    if (o.src) stl->lambda_source = o.src;
    // concurrent passes that marked almost nothing before the whole-graph
    // passes had to run: small graphs skip them in the next round
    // (and keep skipping them while those passes keep running)
    // (in a skipping round the whole passes run regardless: they were needed
    // if PR alone hooked fewer than n / 64 edges)
    skip_cc = c.skip_concurrent ? o.seq_pass && o.marks_pr * 64 < (long long)n_before
                                : c.capforest == 1 && o.seq_pass &&
                                      o.marks_cc * 64 < (long long)n_before;
    if (o.cc_ran) cc_low = o.marks_cc * 64 < (long long)n_before;
    const bool improved = o.lambda < lambda;
    lambda = std::min(lambda, o.lambda);
    if (o.stopped) break;
    stl->rounds++;
    stl->entries_processed += g->M;
    stl->marks_pr += o.marks_pr;
    stl->marks_cf += o.marks_cf;
    if (o.seq_pass) stl->seq_passes++;
    if (lambda == 0) break;
    if (o.marks_pr + o.marks_cf == 0) {
      if (!improved) return fail(MINCUT_ERR_INTERNAL, "round made no progress");
      continue;
    }
    int n2 = 0;
    long long m2 = 0;
    // (the visit-mode choice times each round to its end: no deferral then)
    rc = contract_current<WT>(g, &n2, &m2, true, op.cf_visit != 2);
    if (rc) return rc;
    barely = 2 * (long long)n2 >= (long long)n_before;
    if (op.cf_visit == 2 && rate[mode] < 0) {
      const double ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - t0).count();
      rate[mode] = (double)(n_before - n2) / std::max(ms, 1e-3);
    }
    if (n2 <= 1) break;
  }
  if (g->m_pending) {
    const int rc = sync_state(g);
    if (rc) return rc;
    g->M = g->hst->m_rows;
    g->m_pending = false;
  }
  *lambda_io = lambda;
  return MINCUT_OK;
}

// The coarsening heuristic of Sec. 2.1 ("Lowering the upper bound"): label
// propagation clusters and the PR tests are contracted repeatedly while the
// graph shrinks, then the coarse graph is solved exactly.  Every vertex of a
// coarse graph is a set of input vertices, so the result is a cut of the
// input graph (an upper bound, not necessarily minimum: a cluster may
// straddle a minimum cut).  Leaves the bound in *lambda_io, its witness in
// side0, and the graph reset to the input.
template <typename WT>
int coarsening_bound(mincut_graph* g, const mincut_options& op, const RoundCfg& base,
                     long long* lambda_io, mincut_stats* stl) {
  constexpr int kSmall = 1000;      // coarse graphs this small are solved exactly
  constexpr int kMaxLevels = 32;
  long long lambda = *lambda_io;
  RoundCfg h = base;
  h.lp_now = true;
  h.lp_min_n = 2;  // the clustering runs at every level, down to the small graph
  h.capforest = 0;
  h.coarsen = true;
  int src = 0;
  for (int level = 0; level < kMaxLevels && g->n > kSmall; ++level) {
    h.seed = op.seed ^ (0xC0A25E11ull * (unsigned long long)(level + 1));
    RoundOut o;
    int rc = mark_round<WT>(g, h, lambda, &o);
    if (rc) return rc;
    if (o.src) src = o.src;
    lambda = std::min(lambda, o.lambda);
    if (o.stopped || lambda == 0) break;
    const int n_before = g->n;
    int n2 = 0;
    long long m2 = 0;
    rc = contract_current<WT>(g, &n2, &m2, true);
    if (rc) return rc;
    if (n2 <= 1 || n2 > n_before - n_before / 10) break;  // clusters stopped shrinking it
  }
  if (g->n > 1 && lambda > 0) {
    mincut_stats inner{};
    int round = 0;
    const long long before = lambda;
    int rc = exact_rounds<WT>(g, op, base, false, &lambda, &inner, &round);
    if (rc) return rc;
    if (lambda < before) src = inner.lambda_source;
  }
  if (src) stl->lambda_source = 4;
  // back to the input graph; the bound and its witness (side0) stay
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  iota_kernel<<<std::min((g->n0 + 255) / 256, g->sms * 8), 256, 0, g->stream>>>(g->map0, g->n0);
  ++g->launches;
  int rc = set_lambda(g, lambda);
  if (rc) return rc;
  *lambda_io = lambda;
  return MINCUT_OK;
}

template <typename WT>
int solve_impl(mincut_graph* g, const mincut_options& op, int64_t* cut_value,
               uint64_t* side_bitmap, mincut_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = g->stream;
  g->launches = 0;
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  if (op.spin_limit > 0) g->spin_limit = op.spin_limit;
  CK(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
  int rc = set_lambda(g, kInf);
  if (rc) return rc;
  iota_kernel<<<std::min((g->n0 + 255) / 256, g->sms * 8), 256, 0, s>>>(g->map0, g->n0);
  ++g->launches;
  long long lambda = kInf;
  mincut_stats stl{};
  stl.n_input = g->n0;
  stl.m_input = g->M0 / 2;
  RoundCfg c{};
  c.lp_iters = op.lp_iters;
  c.lp_min_n = op.lp_min_n;
  c.pr_mask = op.pr_mask;
  c.pr_budget = op.pr_budget;
  c.capforest = op.deterministic ? 2 : 1;
  c.cf_start = 0;
  c.table = op.pass_table > 0 ? op.pass_table : g->max_table;
  c.table = std::min(c.table, g->max_table);
  c.seed = op.seed;
  c.seq_passes = std::max(0, op.seq_passes);
  c.seq_kernel = op.seq_kernel;
  const bool heuristic = op.init_bound == 1 && op.lp_iters > 0 && g->n0 >= op.lp_min_n;
  if (heuristic) {
    rc = coarsening_bound<WT>(g, op, c, &lambda, &stl);
    if (rc) return rc;
  }
  int round = 0;
  if (lambda > 0) {
    // with the heuristic's bound in hand, the rounds skip the LP bound
    rc = exact_rounds<WT>(g, op, c, !heuristic, &lambda, &stl, &round);
    if (rc) return rc;
  }
  *cut_value = lambda;
  if (side_bitmap) {
    cudaPointerAttributes attr{};
    bool dev = cudaPointerGetAttributes(&attr, side_bitmap) == cudaSuccess &&
               (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    u64* target = dev ? reinterpret_cast<u64*>(side_bitmap) : g->bitmap_dev;
    CK(side_to_bitmap(g->side0, g->n0, target, s, &g->launches));
    if (!dev)
      CK(cudaMemcpyAsync(side_bitmap, g->bitmap_dev, (size_t)((g->n0 + 63) / 64) * 8,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  stl.kernel_launches = g->launches;
  stl.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = stl;
  return MINCUT_OK;
}

template <typename WT>
int contract_round_impl(mincut_graph* g, const mincut_round_options* ro,
                        mincut_round_result* res) {
  cudaStream_t s = g->stream;
  memset(res, 0, sizeof(*res));
  res->n_in = g->n;
  res->m_in = g->M;
  res->lambda_out = ro->lambda_in;
  CK(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
  int rc = set_lambda(g, ro->lambda_in);
  if (rc) return rc;
  const int n = g->n;
  if (ro->groups || ro->pair_u) {
    CK(uf_init(g->parent, n, s, &g->launches));
    CK(tile_rows(g->crp(), n, g->M, g->tile_row, s, &g->launches));
    if (ro->groups) {
      int* gd = g->flags;  // n ints; consumed before uf_relabel reuses them
      CK(cudaMemcpyAsync(gd, ro->groups, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(uf_from_groups(g->parent, gd, g->gmin, n, g->st, s, &g->launches));
    } else {
      if (ro->npairs < 0 || ro->npairs > g->Mraw) return fail(MINCUT_ERR_INVALID, "npairs");
      int* pu = reinterpret_cast<int*>(g->keys[1]);
      int* pv = pu + ro->npairs;
      if (ro->npairs > 0) {
        CK(cudaMemcpyAsync(pu, ro->pair_u, (size_t)ro->npairs * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(pv, ro->pair_v, (size_t)ro->npairs * sizeof(int), cudaMemcpyHostToDevice, s));
      }
      CK(uf_hook_pairs(g->parent, pu, pv, ro->npairs, n, g->st, s, &g->launches));
    }
    rc = sync_state(g);
    if (rc) return rc;
    int n2;
    long long m2;
    rc = contract_current<WT>(g, &n2, &m2, false);
    if (rc) return rc;
    res->n_out = n2;
    res->m_out = m2;
    return MINCUT_OK;
  }
  RoundCfg c{};
  c.lp_iters = ro->lp_iters;
  c.lp_min_n = ro->lp_min_n;
  c.lp_now = true;
  c.pr_mask = ro->pr_mask;
  c.pr_budget = ro->pr_budget;
  c.capforest = ro->capforest == 3 ? 1 : ro->capforest;
  c.cf_private = ro->capforest == 3 ? 1 : 0;
  c.cf_start = ro->cf_start;
  if ((c.capforest == 2 || c.capforest == 4) && (c.cf_start < 0 || c.cf_start >= n))
    return fail(MINCUT_ERR_INVALID, "cf_start out of range");
  c.table = ro->pass_table > 0 ? std::min(ro->pass_table, g->max_table) : g->max_table;
  c.passes = ro->passes > 0 ? ro->passes : std::max(32, std::min(g->max_passes, n / 4));
  c.seed = ro->seed;
  c.pr_flags_host = ro->pr_flags_out;
  c.cf_order_host = ro->cf_order_out;
  c.cf_marks_host = ro->cf_marks_out;
  c.cf_marks_cap = ro->cf_marks_cap;
  c.lp_labels_host = ro->lp_labels_out;
  CK(cudaMemsetAsync(g->side0, 0, (size_t)g->n0, s));
  iota_kernel<<<std::min((g->n0 + 255) / 256, g->sms * 8), 256, 0, s>>>(g->map0, g->n0);
  RoundOut o;
  rc = mark_round<WT>(g, c, ro->lambda_in, &o);
  if (rc) return rc;
  res->lambda_out = o.lambda;
  res->marks_pr = o.marks_pr;
  res->marks_cf = o.marks_cf;
  res->seq_pass = o.seq_pass;
  res->cf_nscanned = o.cf_nscanned;
  res->cf_nmarks = o.cf_nmarks;
  if (o.stopped) {
    res->stopped = 1;
    res->n_out = g->n;
    res->m_out = g->M;
    return MINCUT_OK;
  }
  int n2;
  long long m2;
  rc = contract_current<WT>(g, &n2, &m2, false);
  if (rc) return rc;
  res->n_out = n2;
  res->m_out = m2;
  return MINCUT_OK;
}

// Degrees of the canonical input rp0/col0/w0 (M0 entries) and, with
// `validate`, the symmetry check.
template <typename WT>
int finish_input(mincut_graph* g, int n, bool validate, bool sym_checked) {
  cudaStream_t s = g->stream;
  const long long m = g->M0;
  CK(row_degrees<WT>(n, m, g->rp0, (const WT*)g->w0, g->tile_row, (WT*)g->deg0, s,
                     &g->launches));
  if (validate && !sym_checked && m > 0) {
    CK(check_symmetric<WT>(n, m, g->rp0, g->col0, (const WT*)g->w0, g->tile_row, g->st, s,
                           &g->launches));
    int rc = sync_state(g);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(s));
  return MINCUT_OK;
}

// Canonicalise the raw input already copied to rp[1]/col[1]/w[1] into
// rp0/col0/w0 (identity labels: sort, sum duplicates, drop self-loops).
template <typename WT>
int canonicalize_input(mincut_graph* g, int n, long long Mraw, bool validate) {
  cudaStream_t s = g->stream;
  CK(tile_rows(g->rp[1], n, Mraw, g->tile_row, s, &g->launches));
  const int vbits = bits_for(n);
  CK(emit_pairs<WT>(n, Mraw, g->rp[1], g->col[1], (const WT*)g->w[1], nullptr, vbits,
                    g->tile_row, g->keys[0], (WT*)g->vals[0], g->st, 1, s, &g->launches));
  int rc = sync_state(g);
  if (rc) return rc;
  const long long N = g->hst->emit_count;
  bool alt = false;
  CK(radix_sort_pairs<WT>(g->keys[0], (WT*)g->vals[0], g->keys[1], (WT*)g->vals[1], (int)N,
                          2 * vbits, g->sort, g->st, g->spin_limit, s, &alt, &g->launches));
  CK(build_csr<WT>(alt ? g->keys[1] : g->keys[0], (WT*)(alt ? g->vals[1] : g->vals[0]), (int)N,
                   vbits, n, g->uid, g->part, g->rp[0], g->col[0], (WT*)g->w[0], g->st,
                   g->m2_dev,
                   reinterpret_cast<int*>(alt ? g->keys[0] : g->keys[1]), s, &g->launches));
  int m2 = 0;
  CK(cudaMemcpyAsync(&m2, g->m2_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  rc = sync_state(g);
  if (rc) return rc;
  g->M0 = m2;
  if (!galloc(g, &g->rp0, n + 1) || !galloc(g, &g->col0, m2) ||
      !(g->w0 = dev_alloc(g, (size_t)std::max(m2, 1) * sizeof(WT))))
    return fail(MINCUT_ERR_OOM, "canonical input");
  CK(cudaMemcpyAsync(g->rp0, g->rp[0], (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (m2 > 0) {
    CK(cudaMemcpyAsync(g->col0, g->col[0], (size_t)m2 * sizeof(int), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(g->w0, g->w[0], (size_t)m2 * sizeof(WT), cudaMemcpyDeviceToDevice, s));
  }
  return finish_input<WT>(g, n, validate, false);
}

int create_impl(int64_t n64, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                uint32_t flags, void* stream, const mincut_allocator* alloc, mincut_graph** out) {
  if (!out) return fail(MINCUT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!row_ptr || (!col && n64 > 0) || (!w && n64 > 0))
    return fail(MINCUT_ERR_INVALID, "NULL input array");
  if (n64 < 2) return fail(MINCUT_ERR_INVALID, "n = %lld: a cut needs n >= 2", (long long)n64);
  if (n64 > 0x7ffffffell) return fail(MINCUT_ERR_OVERFLOW, "n = %lld exceeds 2^31-2", (long long)n64);
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(MINCUT_ERR_INVALID, "allocator");
  const int n = (int)n64;
  const bool dev_in = (flags & MINCUT_DEVICE_PTRS) != 0;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t rp_end[2] = {0, 0};
  if (dev_in) {
    CK(cudaMemcpyAsync(&rp_end[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&rp_end[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else {
    rp_end[0] = row_ptr[0];
    rp_end[1] = row_ptr[n];
  }
  const long long Mraw = rp_end[1];
  if (rp_end[0] != 0 || Mraw < 0) return fail(MINCUT_ERR_INVALID, "row_ptr[0] must be 0, row_ptr[n] >= 0");
  if (Mraw > 0x7fffffffll) return fail(MINCUT_ERR_OVERFLOW, "M = %lld exceeds 2^31-1", Mraw);

  mincut_graph* g = new mincut_graph();
  g->stream = s;
  if (alloc) { g->alloc = *alloc; g->user_alloc = true; }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](int rc) {
    cudaStreamSynchronize(s);
    free_all(g);
    delete g;
    return rc;
  };
  if (!(g->hst = pinned_state_get())) return bail(fail(MINCUT_ERR_OOM, "pinned state"));
  if (!galloc(g, &g->st, 1) || !galloc(g, &g->m2_dev, 1)) return bail(fail(MINCUT_ERR_OOM, "state"));
  if (cudaMemsetAsync(g->st, 0, sizeof(DevState), s) != cudaSuccess)
    return bail(fail(MINCUT_ERR_CUDA, "memset state"));
  // row_ptr first (checked before any entry is read through it), then one
  // ingestion pass over the entries: copy, weight statistics, canonical
  // test and symmetry fingerprint together
  int64_t* rp_raw = nullptr;
  int32_t* w_raw = nullptr;
  int* col_raw = nullptr;
  if (!galloc(g, &rp_raw, n + 1) || !galloc(g, &w_raw, Mraw) || !galloc(g, &col_raw, Mraw))
    return bail(fail(MINCUT_ERR_OOM, "raw input"));
  const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(rp_raw, row_ptr, (size_t)(n + 1) * sizeof(int64_t), kind, s) != cudaSuccess)
    return bail(fail(MINCUT_ERR_CUDA, "copy row_ptr: %s", cudaGetErrorString(cudaGetLastError())));
  unsigned long long* wst = nullptr;
  if (!galloc(g, &wst, 10)) return bail(fail(MINCUT_ERR_OOM, "stats"));
  cudaMemsetAsync(wst, 0, 10 * sizeof(unsigned long long), s);
  input_stats_kernel<<<std::max(1, std::min(g->sms * 8, (n + 255) / 256)), 256, 0, s>>>(
      rp_raw, n, w_raw, 0, wst);
  unsigned long long hws[6] = {0, 0, 0, 0, 0, 0};
  cudaMemcpyAsync(hws, wst, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return bail(fail(MINCUT_ERR_CUDA, "row_ptr check: %s", cudaGetErrorString(cudaGetLastError())));
  if (hws[2]) return bail(fail(MINCUT_ERR_INVALID, "row_ptr is not non-decreasing"));
  const long long ntiles = (std::max<long long>(Mraw, 1) + kEntryTile - 1) / kEntryTile + 2;
  if (!galloc(g, &g->tile_row, ntiles)) return bail(fail(MINCUT_ERR_OOM, "tile rows"));
  unsigned long long* ist = wst + 4;
  if (Mraw > 0) {
    // entries the device can address are read in place (device input, or
    // pinned host memory mapped into the device's address space); others
    // are copied first
    const int* col_src = dev_in ? col : (const int*)mapped_host_range(col, (size_t)Mraw * 4);
    const int* w_src = dev_in ? w : (const int*)mapped_host_range(w, (size_t)Mraw * 4);
    if (!col_src || !w_src) {
      if (cudaMemcpyAsync(w_raw, w, (size_t)Mraw * sizeof(int32_t), kind, s) != cudaSuccess ||
          cudaMemcpyAsync(col_raw, col, (size_t)Mraw * sizeof(int32_t), kind, s) != cudaSuccess)
        return bail(fail(MINCUT_ERR_CUDA, "copy input: %s", cudaGetErrorString(cudaGetLastError())));
      col_src = col_raw;
      w_src = w_raw;
    }
    if (tile_rows(rp_raw, n, Mraw, g->tile_row, s, &g->launches) != cudaSuccess ||
        ingest_csr(n, Mraw, rp_raw, col_src, w_src, col_raw, w_raw, g->tile_row, ist, s,
                   &g->launches) != cudaSuccess ||
        cudaMemcpyAsync(hws, ist, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return bail(fail(MINCUT_ERR_CUDA, "input pass: %s", cudaGetErrorString(cudaGetLastError())));
  }
  if (hws[1]) return bail(fail(MINCUT_ERR_INVALID, "negative weight"));
  g->wt64 = hws[0] > 0x7fffffffull;
  // An input already in canonical form (the form every contraction writes)
  // is adopted as is: no relabel/sort/sum pass; its symmetry is settled by
  // the fingerprint.
  const bool canonical = Mraw > 0 && hws[2] == 0;
  const bool sym_fingerprint_ok = hws[3] == 0 && hws[4] == 0 && hws[5] == 0;
  const size_t wsz = g->wt64 ? 8 : 4;
  g->n0 = n;
  g->Mraw = Mraw;
  const long long Mb = std::max<long long>(Mraw, 1);
  // buffers
  bool ok = true;
  for (int i = 0; i < 2; ++i) {
    ok = ok && galloc(g, &g->rp[i], n + 1) && galloc(g, &g->col[i], Mb) &&
         (g->w[i] = dev_alloc(g, (size_t)Mb * wsz)) && galloc(g, &g->keys[i], Mb) &&
         (g->vals[i] = dev_alloc(g, (size_t)Mb * wsz));
  }
  const long long scan_parts = (std::max<long long>(Mb, n) + 4095) / 4096 + 2;
  g->max_table = 1024;
  g->max_passes = graph_max_passes(n, g->sms);
  ok = ok && (g->deg0 = dev_alloc(g, (size_t)n * wsz)) &&
       (g->degb[0] = dev_alloc(g, (size_t)n * wsz)) && (g->degb[1] = dev_alloc(g, (size_t)n * wsz)) &&
       galloc(g, &g->blk, 2 * 1024) && galloc(g, &g->parent, n) && galloc(g, &g->L, n) &&
       galloc(g, &g->flags, n) && galloc(g, &g->rank, n) && galloc(g, &g->part, scan_parts) &&
       galloc(g, &g->uid, Mb) && galloc(g, &g->owner, n) && galloc(g, &g->gmin, n) &&
       galloc(g, &g->map0, n) && galloc(g, &g->side0, n) && galloc(g, &g->cur_side, n) &&
       galloc(g, &g->bitmap_dev, (n + 63) / 64) && galloc(g, &g->short_bits, n / 32 + 2) &&
       galloc(g, &g->visit_log, (long long)g->max_passes * g->max_table) &&
       galloc(g, &g->pass_best, g->max_passes) && galloc(g, &g->pass_len, g->max_passes) &&
       galloc(g, &g->pass_counter, 1) && (g->seq_r = dev_alloc(g, (size_t)n * wsz)) &&
       galloc(g, &g->seq_mark, n) && galloc(g, &g->seq_tree, seq_tree_words(n)) &&
       galloc(g, &g->seq_order, n) && galloc(g, &g->sort.hist, 8 * 256) &&
       galloc(g, &g->sort.goff, 8 * 256) &&
       galloc(g, &g->sort.lookback, sort_lookback_words(Mb));
  if (!ok) return bail(fail(MINCUT_ERR_OOM, "device buffers for n=%d M=%lld", n, Mraw));
  g->sort.lookback_words = sort_lookback_words(Mb);
  const bool validate = (flags & MINCUT_SKIP_VALIDATE) == 0;
  if (canonical) {
    g->rp0 = rp_raw;
    g->col0 = col_raw;
    if (g->wt64) {
      if (!(g->w0 = dev_alloc(g, (size_t)Mraw * 8))) return bail(fail(MINCUT_ERR_OOM, "weights"));
      widen32_kernel<<<std::max(1, std::min(g->sms * 8, (int)((Mraw + 255) / 256))), 256, 0, s>>>(
          w_raw, (int64_t*)g->w0, Mraw);
      dev_free(g, w_raw);
    } else {
      g->w0 = w_raw;
    }
    dev_free(g, wst);
    g->M0 = Mraw;
    if (validate && !sym_fingerprint_ok)
      return bail(fail(MINCUT_ERR_INVALID, "input CSR is not symmetric"));
    int rc = g->wt64 ? finish_input<int64_t>(g, n, validate, true)
                     : finish_input<int32_t>(g, n, validate, true);
    if (rc) return bail(rc);
    g->cur = -1;
    g->n = n;
    g->M = g->M0;
    *out = g;
    return MINCUT_OK;
  }
  // raw input into rp[1]/col[1]/w[1]
  if (cudaMemcpyAsync(g->rp[1], rp_raw, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      (Mraw > 0 && cudaMemcpyAsync(g->col[1], col_raw, (size_t)Mraw * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess))
    return bail(fail(MINCUT_ERR_CUDA, "stage input"));
  if (Mraw > 0) {
    if (g->wt64) {
      widen32_kernel<<<std::max(1, std::min(g->sms * 8, (int)((Mraw + 255) / 256))), 256, 0, s>>>(
          w_raw, (int64_t*)g->w[1], Mraw);
    } else if (cudaMemcpyAsync(g->w[1], w_raw, (size_t)Mraw * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      return bail(fail(MINCUT_ERR_CUDA, "stage weights"));
    }
  }
  cudaStreamSynchronize(s);
  dev_free(g, rp_raw);
  dev_free(g, w_raw);
  dev_free(g, col_raw);
  dev_free(g, wst);
  int rc = g->wt64 ? canonicalize_input<int64_t>(g, n, Mraw, validate)
                   : canonicalize_input<int32_t>(g, n, Mraw, validate);
  if (rc) return bail(rc);
  g->cur = -1;
  g->n = n;
  g->M = g->M0;
  g->m_pending = false;
  *out = g;
  return MINCUT_OK;
}

// The graphs of a batch with at most `threshold` vertices (and at most
// kBwMaxN), most entries first, for the one-warp-per-graph solver; its
// scratch (at most ~2 GB of slots).
int bw_prepare(mincut_graph* g, int threshold) {
  threshold = std::min(threshold, kBwMaxN);
  if (threshold == g->bw_threshold) return MINCUT_OK;
  const int G = g->batch.G;
  std::vector<int> ids;
  int nmax = 0, mmax = 0;
  for (int i = 0; i < G; ++i) {
    const int ng = (int)(g->voff0_h[i + 1] - g->voff0_h[i]);
    if (ng > threshold) continue;
    ids.push_back(i);
    nmax = std::max(nmax, ng);
    mmax = std::max(mmax, g->batch_m[i]);
  }
  std::stable_sort(ids.begin(), ids.end(),
                   [&](int a, int b) { return g->batch_m[a] > g->batch_m[b]; });
  g->bw_threshold = threshold;
  g->bw_count = (int)ids.size();
  g->bw_nmax = nmax;
  g->bw_mmax = std::max(mmax, 1);
  if (ids.empty()) return MINCUT_OK;
  if (!g->bw_list) {
    if (!galloc(g, &g->bw_list, G) || !galloc(g, &g->bw_cursor, 1))
      return fail(MINCUT_ERR_OOM, "batch warp list");
  }
  CK(cudaMemcpyAsync(g->bw_list, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice,
                     g->stream));
  // slots come in blocks of batch_warp_block_warps() (the kernel's block)
  const int bw = batch_warp_block_warps();
  const long long per = batch_warp_slot_words(nmax, g->bw_mmax);
  const long long cap = std::max<long long>(bw, (2ll << 30) / 4 / per / bw * bw);
  const long long need = ((long long)g->bw_count + bw - 1) / bw * bw;
  const int slots = (int)std::min<long long>({(long long)batch_warp_slots(g->sms), cap, need});
  const long long words = per * slots;
  if (words > g->bw_scratch_words) {
    if (g->bw_scratch) dev_free(g, g->bw_scratch);
    g->bw_scratch = nullptr;
    g->bw_scratch_words = 0;
    if (!galloc(g, &g->bw_scratch, words)) return fail(MINCUT_ERR_OOM, "batch warp scratch");
    g->bw_scratch_words = words;
  }
  g->bw_slots = slots;
  CK(cudaStreamSynchronize(g->stream));  // ids may go out of scope
  return MINCUT_OK;
}

// A solve whose graphs all take the one-warp solver: state reset, then the
// warp solver over the whole list (no round kernels, no host decisions
// before the completion check).  Only stream-ordered calls, so that it can
// be captured.
cudaError_t bw_enqueue(mincut_graph* g, uint32_t pr, cudaStream_t s, int* launches) {
  BatchState& b = g->batch;
  const int G = b.G;
  cudaError_t e = cudaMemsetAsync(g->st, 0, sizeof(DevState), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.voff, b.voff0, (size_t)(G + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                        s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.gid, b.gid0, (size_t)g->n0 * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = batch_start(G, b.lam_g, b.done_g, s, launches);
  if (e == cudaSuccess) {
    iota_kernel<<<std::min((g->n0 + 255) / 256, g->sms * 8), 256, 0, s>>>(g->map0, g->n0);
    ++*launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(g->side0, 0, (size_t)g->n0, s);
  if (e == cudaSuccess) e = batch_warp_mark(g->bw_list, g->bw_count, b.done_g, g->st, s, launches);
  if (e == cudaSuccess)
    e = batch_warp_solve(g->bw_list, g->bw_count, g->bw_cursor, b.voff0, g->rp0, g->col0,
                         (const int*)g->w0, g->bw_scratch, g->bw_slots, g->bw_nmax, g->bw_mmax,
                         pr, b.lam_g, g->side0, g->st, s, launches);
  return e;
}

template <typename WT>
int batch_solve_impl(mincut_graph* g, const mincut_options& op, int64_t* cut_values,
                     uint64_t* side_bitmap, mincut_stats* stats, int small_n,
                     bool allow_graph) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = g->stream;
  BatchState& b = g->batch;
  const int G = b.G;
  g->launches = 0;
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  if (op.spin_limit > 0) g->spin_limit = op.spin_limit;
  // the small graphs are the warp solver's: the round kernels treat them as done
  {
    const int rc0 = bw_prepare(g, small_n);
    if (rc0) return rc0;
  }
  mincut_stats stl{};
  stl.n_input = g->n0;
  stl.m_input = g->M0 / 2;
  const int max_rounds = op.max_rounds > 0 ? op.max_rounds : g->max_graph_n + 8;
  if (G > 0 && g->bw_count == G && !tl_prof) {
    // every graph on the one-warp solver (no profiling): the same launches
    // on every solve of this batch, replayed from a CUDA graph once the
    // same split comes a second time (a batch solved once pays no capture);
    // captured on a private stream, since the caller's may be the legacy one
    mincut_graph::BwKey key;
    key.threshold = g->bw_threshold;
    key.scratch = g->bw_scratch;
    key.voff = b.voff;
    key.pr = op.pr_mask & 3u;
    g->bw_key_runs = key == g->bw_key ? g->bw_key_runs + 1 : 1;
    g->bw_key = key;
    if (g->bw_exec && !(g->bw_exec_key == key)) {
      CK(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(g->bw_exec);
      g->bw_exec = nullptr;
    }
    if (!g->bw_exec && allow_graph && g->bw_key_runs >= 2) {
      if (!g->bw_capture) CK(cudaStreamCreateWithFlags(&g->bw_capture, cudaStreamNonBlocking));
      int nl = 0;
      CK(cudaStreamBeginCapture(g->bw_capture, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = bw_enqueue(g, key.pr, g->bw_capture, &nl);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(g->bw_capture, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g->bw_exec, graph, 0ull);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g->bw_exec = nullptr;
        return fail(MINCUT_ERR_CUDA, "capturing the batch's launches: %s", cudaGetErrorString(e));
      }
      g->bw_exec_key = key;
      g->bw_exec_launches = nl;
    }
    if (g->bw_exec) {
      CK(cudaGraphLaunch(g->bw_exec, s));
      g->launches += g->bw_exec_launches;
    } else {
      CK(bw_enqueue(g, key.pr, s, &g->launches));
    }
  } else {
    CK(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
    CK(cudaMemcpyAsync(b.voff, b.voff0, (size_t)(G + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(b.gid, b.gid0, (size_t)g->n0 * sizeof(int), cudaMemcpyDeviceToDevice, s));
    CK(batch_start(G, b.lam_g, b.done_g, s, &g->launches));
    iota_kernel<<<std::min((g->n0 + 255) / 256, g->sms * 8), 256, 0, s>>>(g->map0, g->n0);
    ++g->launches;
    CK(cudaMemsetAsync(g->side0, 0, (size_t)g->n0, s));
    if (g->bw_count > 0)
      CK(batch_warp_mark(g->bw_list, g->bw_count, b.done_g, g->st, s, &g->launches));
    const int table = op.pass_table > 0 ? std::min(op.pass_table, g->max_table) : g->max_table;
    for (int round = 0; g->bw_count < G && round < max_rounds; ++round) {
      const int n = g->n;
      const long long M = g->M;
      const int64_t* rp = g->crp();
      const int* col = g->ccol();
      const WT* w = (const WT*)g->cw();
      const WT* deg = (const WT*)g->cdeg();
      reset_round_kernel<<<1, 1, 0, s>>>(g->st);
      ++g->launches;
      CK(batch_round_reset(G, b, s, &g->launches));
      { ProfScope ps(P_DEGREE, n, s);
        CK(batch_degree_bound<WT>(n, G, deg, b, &g->st->batch_done, s, &g->launches)); }
      { ProfScope ps(P_TILES, n, s);
        CK(tile_rows(rp, n, M, g->tile_row, s, &g->launches)); }
      { ProfScope ps(P_UF, n, s);
        CK(uf_init(g->parent, n, s, &g->launches)); }
      const BatchView v = b.view();
      if (op.pr_mask) {
        ProfScope ps(P_PR, M, s);
        CK(pr_marks<WT>(n, M, rp, col, w, deg, g->tile_row, op.pr_mask, op.pr_budget, g->parent,
                        nullptr, g->short_bits, g->st, s, &g->launches, &v));
      }
      if (!op.deterministic) {
        ProfScope ps(P_CF_PASSES, M, s);
        CK(cudaMemsetAsync(g->owner, 0, (size_t)n * sizeof(int), s));
        PassConfig pc;
        pc.table = table;
        pc.warps_per_block = 4;
        pc.passes = op.passes > 0 ? std::min(op.passes, g->max_passes)
                                  : std::max(32, std::min(g->max_passes, n / 4));
        pc.seed = op.seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(round + 1);
        pc.private_visit = op.cf_visit == 1 ? 1 : 0;
        CK(capforest_passes<WT>(n, rp, col, w, deg, g->owner, g->parent, g->visit_log, g->pass_best,
                                g->pass_len, g->pass_counter, pc, g->st, s, &g->launches, &v));
      }
      { ProfScope ps(P_CF_SEQ, M, s);
        CK(capforest_sequential_batch<WT>(G, rp, col, w, deg, g->parent, (WT*)g->seq_r,
                                          g->batch_levels, b.level_off, g->seq_order,
                                          g->max_graph_n, op.deterministic ? 1 : 0, v, g->st, s,
                                          &g->launches)); }
      { ProfScope ps(P_WITNESS, g->n0, s);
        CK(batch_witness(G, g->n0, b, g->visit_log, table, g->pass_len, g->seq_order, g->cur_side,
                         g->map0, g->side0, g->st, s, &g->launches)); }
      CK(batch_collapse(n, b, g->parent, s, &g->launches));
      stl.rounds++;
      stl.entries_processed += M;
      int n2 = 0;
      long long m2 = 0;
      int rc = contract_current<WT>(g, &n2, &m2, true);
      if (rc) return rc;
      CK(batch_new_offsets(G, b, g->rank, g->st, s, &g->launches));
      std::swap(b.voff, b.voff_next);
      CK(batch_gid(b.voff, G, n2, b.gid, s, &g->launches));
      if (g->hst->batch_done >= G) break;
    }
    if (g->bw_count > 0) {
      ProfScope ps(P_BATCH_WARP, g->bw_count, s);
      // PR1 / PR2 only: on one warp the PR3 / PR4 intersections cost several
      // times the rest of a graph's solve (the pass of each round marks anyway)
      CK(batch_warp_solve(g->bw_list, g->bw_count, g->bw_cursor, b.voff0, g->rp0, g->col0,
                          (const int*)g->w0, g->bw_scratch, g->bw_slots, g->bw_nmax, g->bw_mmax,
                          op.pr_mask & 3u, b.lam_g, g->side0, g->st, s, &g->launches));
    }
  }
  int rc = sync_state(g);
  if (rc) return rc;
  if (g->hst->batch_done < G) return fail(MINCUT_ERR_INTERNAL, "batch did not finish in %d rounds", max_rounds);
  CK(batch_values(b.lam_g, G, g->batch_vals, s, &g->launches));
  CK(cudaMemcpyAsync(cut_values, g->batch_vals, (size_t)G * sizeof(long long), cudaMemcpyDeviceToHost, s));
  if (side_bitmap) {
    cudaPointerAttributes attr{};
    bool dev = cudaPointerGetAttributes(&attr, side_bitmap) == cudaSuccess &&
               (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    u64* target = dev ? reinterpret_cast<u64*>(side_bitmap) : g->bitmap_dev;
    CK(batch_bitmap(g->side0, g->n0, b, target, s, &g->launches));
    if (!dev)
      CK(cudaMemcpyAsync(side_bitmap, g->bitmap_dev, (size_t)((g->n0 + 63) / 64) * 8,
                         cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  stl.kernel_launches = g->launches;
  stl.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = stl;
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  return MINCUT_OK;
}

}  // namespace

extern "C" {

void mincut_default_options(mincut_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->lp_iters = 2;
  o->lp_min_n = 10000;
  o->lp_every_round = 0;
  o->pr_mask = 0xF;
  o->pr_budget = 16;
  o->seed = 0x5eed;
}

void mincut_default_round_options(mincut_round_options* ro) {
  if (!ro) return;
  memset(ro, 0, sizeof(*ro));
  ro->lambda_in = kInf;
  ro->lp_iters = 2;
  ro->lp_min_n = 10000;
  ro->pr_mask = 0xF;
  ro->pr_budget = 16;
  ro->capforest = 1;
  ro->seed = 0x5eed;
}

int mincut_graph_from_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                          uint32_t flags, void* cuda_stream, const mincut_allocator* alloc,
                          mincut_graph** out) {
  g_last_error.clear();
  return create_impl(n, row_ptr, col, w, flags, cuda_stream, alloc, out);
}

int mincut_solve(mincut_graph* g, const mincut_options* opts, int64_t* cut_value,
                 uint64_t* side_bitmap, mincut_stats* stats) {
  g_last_error.clear();
  if (!g || !cut_value) return fail(MINCUT_ERR_INVALID, "NULL graph or cut_value");
  mincut_options op;
  if (opts) op = *opts; else mincut_default_options(&op);
  if (op.pass_table != 0 && (op.pass_table < 256 || op.pass_table > 2048 ||
                             (op.pass_table & (op.pass_table - 1))))
    return fail(MINCUT_ERR_INVALID, "pass_table must be a power of two in [256, 2048]");
  int rc;
  {
    ProfGuard pg(g, op.profile != 0);
    rc = g->wt64 ? solve_impl<int64_t>(g, op, cut_value, side_bitmap, stats)
                 : solve_impl<int32_t>(g, op, cut_value, side_bitmap, stats);
  }
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  return rc;
}

int mincut_contract_round(mincut_graph* g, const mincut_round_options* ro,
                          mincut_round_result* res) {
  g_last_error.clear();
  if (!g || !ro || !res) return fail(MINCUT_ERR_INVALID, "NULL argument");
  if (ro->pass_table != 0 && (ro->pass_table < 256 || ro->pass_table > 2048 ||
                              (ro->pass_table & (ro->pass_table - 1))))
    return fail(MINCUT_ERR_INVALID, "pass_table must be a power of two in [256, 2048]");
  if (ro->capforest < 0 || ro->capforest > 4) return fail(MINCUT_ERR_INVALID, "capforest mode");
  return g->wt64 ? contract_round_impl<int64_t>(g, ro, res) : contract_round_impl<int32_t>(g, ro, res);
}

int mincut_graph_info(const mincut_graph* g, int64_t* n, int64_t* m_directed) {
  if (!g) return fail(MINCUT_ERR_INVALID, "NULL graph");
  if (n) *n = g->n;
  if (m_directed) *m_directed = g->M;
  return MINCUT_OK;
}

int mincut_graph_export_csr(const mincut_graph* g, int64_t* row_ptr, int32_t* col, int64_t* w) {
  if (!g || !row_ptr) return fail(MINCUT_ERR_INVALID, "NULL argument");
  mincut_graph* gg = const_cast<mincut_graph*>(g);
  cudaStream_t s = gg->stream;
  CK(cudaMemcpyAsync(row_ptr, g->crp(), (size_t)(g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (g->M > 0) {
    if (col) CK(cudaMemcpyAsync(col, g->ccol(), (size_t)g->M * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (w) {
      if (g->wt64) {
        CK(cudaMemcpyAsync(w, g->cw(), (size_t)g->M * 8, cudaMemcpyDeviceToHost, s));
      } else {
        int64_t* tmp = reinterpret_cast<int64_t*>(gg->keys[1]);
        widen32_kernel<<<std::max(1, std::min(g->sms * 8, (int)((g->M + 255) / 256))), 256, 0, s>>>(
            (const int32_t*)g->cw(), tmp, g->M);
        CK(cudaMemcpyAsync(w, tmp, (size_t)g->M * 8, cudaMemcpyDeviceToHost, s));
      }
    }
  }
  CK(cudaStreamSynchronize(s));
  return MINCUT_OK;
}

int mincut_graph_reset(mincut_graph* g) {
  if (!g) return fail(MINCUT_ERR_INVALID, "NULL graph");
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  return MINCUT_OK;
}

void mincut_graph_destroy(mincut_graph* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  prof_destroy(g->prof);
  g->prof = nullptr;
  free_all(g);
  cudaStreamSynchronize(g->stream);
  delete g;
}

const char* mincut_status_string(int status) {
  switch (status) {
    case MINCUT_OK: return "ok";
    case MINCUT_ERR_INVALID: return "invalid argument or graph";
    case MINCUT_ERR_OOM: return "device allocation failed";
    case MINCUT_ERR_OVERFLOW: return "size or sum out of the supported range";
    case MINCUT_ERR_DEVICE_TIMEOUT: return "bounded device wait ran out";
    case MINCUT_ERR_CUDA: return "CUDA runtime error";
    case MINCUT_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

const char* mincut_last_error(void) { return g_last_error.c_str(); }

int mincut_release_cached(int device) {
  if (device < 0 || device >= kMaxDevices) return fail(MINCUT_ERR_INVALID, "device %d", device);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pools[device] && cudaMemPoolTrimTo(g_pools[device], 0) != cudaSuccess)
    return fail(MINCUT_ERR_CUDA, "trim pool: %s", cudaGetErrorString(cudaGetLastError()));
  return MINCUT_OK;
}

int64_t mincut_graph_footprint(int64_t n, int64_t m_directed) {
  if (n < 0 || m_directed < 0) return -1;
  int dev = 0, sms = kDefaultSms;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = kDefaultSms;
  cudaGetLastError();
  const long long P = graph_max_passes(n, sms);
  // 8-byte weights and sums double the weight terms; this bound assumes
  // 4-byte ones (total weight < 2^31) plus the label-propagation and the
  // row-wise contraction buffers
  return (int64_t)(208 * n + 126 * m_directed + 4096 * P + (1 << 20));
}

int mincut_batch_from_csr(int64_t num_graphs, const int64_t* vertex_offsets,
                          const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                          uint32_t flags, void* cuda_stream, const mincut_allocator* alloc,
                          mincut_graph** out) {
  g_last_error.clear();
  if (!out || !vertex_offsets) return fail(MINCUT_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (num_graphs < 1 || num_graphs > 0x7ffffff) return fail(MINCUT_ERR_INVALID, "num_graphs");
  if (vertex_offsets[0] != 0) return fail(MINCUT_ERR_INVALID, "vertex_offsets[0] must be 0");
  int maxn = 0;
  for (int64_t i = 0; i < num_graphs; ++i) {
    const int64_t ng = vertex_offsets[i + 1] - vertex_offsets[i];
    if (ng < 2) return fail(MINCUT_ERR_INVALID, "graph %lld has fewer than 2 vertices", (long long)i);
    if (ng > maxn) maxn = (int)std::min<int64_t>(ng, 0x7fffffff);
  }
  const int64_t n = vertex_offsets[num_graphs];
  mincut_graph* g = nullptr;
  int rc = create_impl(n, row_ptr, col, w, flags, cuda_stream, alloc, &g);
  if (rc) return rc;
  auto bail = [&](int r) { mincut_graph_destroy(g); return r; };
  if (g->wt64) return bail(fail(MINCUT_ERR_OVERFLOW, "a batch needs a total weight below 2^31"));
  cudaStream_t s = g->stream;
  const int G = (int)num_graphs;
  BatchState& b = g->batch;
  b.G = G;
  g->max_graph_n = maxn;
  g->voff0_h.assign(vertex_offsets, vertex_offsets + G + 1);
  std::vector<int> v32(G + 1);
  std::vector<long long> loff(G);
  long long words = 0;
  for (int i = 0; i < G; ++i) {
    v32[i] = (int)vertex_offsets[i];
    loff[i] = words;
    words += seq_tree_words((int)(vertex_offsets[i + 1] - vertex_offsets[i]));
  }
  v32[G] = (int)n;
  if (!galloc(g, &b.voff0, G + 1) || !galloc(g, &b.gid0, n) || !galloc(g, &b.voff, G + 1) ||
      !galloc(g, &b.voff_next, G + 1) || !galloc(g, &b.gid, n) || !galloc(g, &b.lam_g, G) ||
      !galloc(g, &b.lam_before, G) || !galloc(g, &b.deg_best, G) || !galloc(g, &b.cf_best, G) ||
      !galloc(g, &b.cf_len, G) || !galloc(g, &b.marks_g, G) || !galloc(g, &b.done_g, G) ||
      !galloc(g, &b.wit_kind, G) || !galloc(g, &b.wit_x, G) || !galloc(g, &b.level_off, G) ||
      !galloc(g, &g->batch_levels, words) || !galloc(g, &g->batch_vals, G))
    return bail(fail(MINCUT_ERR_OOM, "batch arrays"));
  if (cudaMemcpyAsync(b.voff0, v32.data(), (size_t)(G + 1) * sizeof(int), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(b.level_off, loff.data(), (size_t)G * sizeof(long long), cudaMemcpyHostToDevice, s))
    return bail(fail(MINCUT_ERR_CUDA, "batch offsets"));
  if (batch_gid(b.voff0, G, (int)n, b.gid0, s, &g->launches) ||
      batch_check_edges((int)n, g->rp0, g->col0, b.gid0, g->st, s, &g->launches))
    return bail(fail(MINCUT_ERR_CUDA, "batch setup"));
  rc = sync_state(g);
  if (rc) {
    if (rc == MINCUT_ERR_INVALID) fail(rc, "an edge joins two different graphs of the batch");
    return bail(rc);
  }
  {  // entries per graph of the canonical input
    std::vector<int64_t> rp_h((size_t)n + 1);
    CK(cudaMemcpyAsync(rp_h.data(), g->rp0, (size_t)(n + 1) * sizeof(int64_t),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    g->batch_m.resize(G);
    for (int i = 0; i < G; ++i)
      g->batch_m[i] = (int)(rp_h[vertex_offsets[i + 1]] - rp_h[vertex_offsets[i]]);
  }
  CK(cudaStreamSynchronize(s));
  *out = g;
  return MINCUT_OK;
}

int mincut_batch_info(const mincut_graph* g, int32_t* small_n, int64_t* small_graphs) {
  g_last_error.clear();
  if (!g || g->batch.G <= 0) return fail(MINCUT_ERR_INVALID, "not a batch");
  if (small_n) *small_n = g->bw_threshold;
  if (small_graphs) *small_graphs = g->bw_threshold < 0 ? 0 : g->bw_count;
  return MINCUT_OK;
}

int mincut_batch_solve(mincut_graph* g, const mincut_options* opts, int64_t* cut_values,
                       uint64_t* side_bitmap, mincut_stats* stats) {
  g_last_error.clear();
  if (!g || !cut_values) return fail(MINCUT_ERR_INVALID, "NULL graph or cut_values");
  if (g->batch.G <= 0) return fail(MINCUT_ERR_INVALID, "not a batch (use mincut_batch_from_csr)");
  mincut_options op;
  if (opts) op = *opts; else mincut_default_options(&op);
  if (op.pass_table != 0 && (op.pass_table < 256 || op.pass_table > 2048 ||
                             (op.pass_table & (op.pass_table - 1))))
    return fail(MINCUT_ERR_INVALID, "pass_table must be a power of two in [256, 2048]");
  int small_n = op.batch_small_n > 0 ? std::min(op.batch_small_n, kBwMaxN)
                                      : (op.batch_small_n < 0 ? 0 : g->bw_auto);
  if (small_n < 0) {
    // autotuning: time the whole batch solve at each candidate threshold
    // (the largest first, which also sizes the scratch), keep the fastest
    const int cands[] = {kBwMaxN, 1024, 256, 64, 0};
    std::vector<int64_t> tmp((size_t)g->batch.G);
    double best_ms = 1e300;
    int best = 0, last_count = -1;
    for (int k = -1; k < 5; ++k) {
      const int t = cands[k < 0 ? 0 : k];
      if (k >= 0) {
        int cnt = 0;
        for (int i = 0; i < g->batch.G; ++i)
          cnt += (g->voff0_h[i + 1] - g->voff0_h[i]) <= t ? 1 : 0;
        if (cnt == last_count) continue;  // same graph split as the last candidate
        last_count = cnt;
      }
      const auto t0 = std::chrono::steady_clock::now();
      const int r = batch_solve_impl<int32_t>(g, op, tmp.data(), nullptr, nullptr, t, false);
      if (r) return r;
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (k >= 0 && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    g->bw_auto = best;
    small_n = best;
  }
  int rc;
  {
    ProfGuard pg(g, op.profile != 0);
    rc = batch_solve_impl<int32_t>(g, op, cut_values, side_bitmap, stats, small_n, true);
  }
  g->cur = -1;
  g->n = g->n0;
  g->M = g->M0;
  g->m_pending = false;
  return rc;
}


int mincut_profile_read(mincut_graph* g, mincut_profile_entry* out, int32_t cap, int32_t* count,
                        int32_t reset) {
  if (!g || !count) return fail(MINCUT_ERR_INVALID, "NULL argument");
  *count = 0;
  if (!g->prof) return MINCUT_OK;
  int k = 0;
  for (int c = 0; c < P_NCAT; ++c) {
    double ms;
    long long l, u;
    prof_read(g->prof, c, &ms, &l, &u);
    if (l == 0) continue;
    if (out && k < cap) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, prof_name(c), sizeof(out[k].name) - 1);
      out[k].launches = l;
      out[k].units = u;
      out[k].ms = ms;
    }
    ++k;
  }
  *count = k;
  if (reset) prof_reset(g->prof);
  return MINCUT_OK;
}

}  // extern "C"
