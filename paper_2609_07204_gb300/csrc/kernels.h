// kernels.h -- host-side launchers of the device kernels (internal interface
// between the C-ABI driver and the kernel translation units).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mc {

using u64 = unsigned long long;

// Per-graph view of a packed batch (many graphs in one CSR; graph g owns the
// current vertices [voff[g], voff[g+1])).  Kernels that take a BatchView use
// the graph's own bound lam_g[g] instead of DevState::lambda.
struct BatchView {
  const int* gid;                // [n] graph of each current vertex
  const int* voff;               // [G+1] current vertex offsets
  unsigned long long* lam_g;     // [G] per-graph upper bound
  unsigned long long* cf_best;   // [G] best CAPFOREST alpha << 32 | pass id (0xffffffff: sequential)
  int* cf_len;                   // [G] prefix length of the sequential pass's best alpha
  int* marks_g;                  // [G] marks of this round
  const int* done_g;             // [G] 1: graph finished
};

// Device arrays of a packed batch.
struct BatchState {
  int G = 0;
  int* voff0 = nullptr;   // [G+1] input vertex offsets
  int* gid0 = nullptr;    // [n0] graph of each input vertex
  int* voff = nullptr;    // [G+1] current offsets
  int* voff_next = nullptr;
  int* gid = nullptr;     // [n0] graph of each current vertex
  unsigned long long *lam_g = nullptr, *lam_before = nullptr, *deg_best = nullptr,
                     *cf_best = nullptr;
  int *cf_len = nullptr, *marks_g = nullptr, *done_g = nullptr, *wit_kind = nullptr,
      *wit_x = nullptr;
  long long* level_off = nullptr;  // [G] sequential-pass tree offsets
  BatchView view() const { return BatchView{gid, voff, lam_g, cf_best, cf_len, marks_g, done_g}; }
};

cudaError_t batch_gid(const int* voff, int G, int n, int* gid, cudaStream_t s, int* launches);
cudaError_t batch_start(int G, unsigned long long* lam_g, int* done_g, cudaStream_t s,
                        int* launches);
cudaError_t batch_round_reset(int G, const BatchState& b, cudaStream_t s, int* launches);
template <typename WT>
cudaError_t batch_degree_bound(int n, int G, const WT* deg, const BatchState& b, int* newly_done,
                               cudaStream_t s, int* launches);
cudaError_t batch_witness(int G, int n0, const BatchState& b, const int* visit_log, int table,
                          const int* pass_len, const int* seq_order, uint8_t* cur,
                          const int* map0, uint8_t* side0, DevState* st, cudaStream_t s,
                          int* launches);
cudaError_t batch_collapse(int n, const BatchState& b, int* parent, cudaStream_t s,
                           int* launches);
cudaError_t batch_new_offsets(int G, const BatchState& b, const int* rank, const DevState* st,
                              cudaStream_t s, int* launches);
// ---- batch_warp.cu: graphs of up to kBwMaxN vertices, one warp each (the
// whole of Algorithm 2 per graph, PR1 / PR2 of pr_mask).  list: the graph
// ids, largest first.
constexpr int kBwMaxN = 2048;
long long batch_warp_slot_words(int nmax, int mmax);  // ints of one warp's scratch slot
int batch_warp_slots(int sms);                        // warps resident at once
int batch_warp_block_warps();                          // warps (slots) per block
// done_g = 1 for the listed graphs, st->batch_done += nlist (the round
// kernels then leave them alone).
cudaError_t batch_warp_mark(const int* list, int nlist, int* done_g, DevState* st,
                            cudaStream_t s, int* launches);
// Solves the listed graphs of the packed input (voff0, rp0, col0, w0; int32
// weights, total below 2^31) into lam_g and side0.  scratch: slots slots (a
// multiple of batch_warp_block_warps()) of
// batch_warp_slot_words(nmax, mmax) ints; every listed graph has at most nmax
// vertices and mmax entries.  cursor: one int of work-queue state.
cudaError_t batch_warp_solve(const int* list, int nlist, int* cursor, const int* voff0,
                             const int64_t* rp0, const int* col0, const int* w0, int* scratch,
                             int slots, int nmax, int mmax, uint32_t pr_mask,
                             unsigned long long* lam_g, uint8_t* side0, DevState* st,
                             cudaStream_t s, int* launches);
cudaError_t batch_bitmap(const uint8_t* side0, int n0, const BatchState& b, u64* bitmap,
                         cudaStream_t s, int* launches);
cudaError_t batch_check_edges(int n, const int64_t* rp, const int* col, const int* gid,
                              DevState* st, cudaStream_t s, int* launches);
cudaError_t batch_values(const unsigned long long* lam_g, int G, long long* out, cudaStream_t s,
                         int* launches);

// Message returned by mincut_last_error() on the calling thread.
void set_last_error(const char* msg);

// ------------------------------------------------------------ profiling
// Optional per-kernel timing: when a Profiler is installed on the calling
// thread, every launcher brackets its kernels with CUDA events on the launch
// stream (category, units processed).  Resolved after the stream synchronises.
enum ProfCat {
  P_DEGREE, P_LP_SWEEP, P_LP_BOUND, P_PR, P_CF_PASSES, P_CF_SEQ, P_UF, P_EMIT,
  P_SORT_HIST, P_SORT_PASS, P_BUILD, P_TILES, P_WITNESS, P_OTHER, P_ROWS, P_BATCH_WARP, P_NCAT
};
const char* prof_name(int cat);
struct Profiler;
extern thread_local Profiler* tl_prof;
struct ProfScope {
  ProfScope(int cat, long long units, cudaStream_t s);
  ~ProfScope();
  int cat;
  long long units;
  cudaStream_t s;
  int idx;
};

// ------------------------------------------------------------- sort.cu
// Onesweep LSD radix sort of N (key, value) pairs on the low `bits` bits of
// the keys, 8 bits per pass.  Ping-pongs between (k0, v0) and (k1, v1);
// returns in *in_alt whether the result ended in (k1, v1).  hist and goff
// hold 8*256 unsigned, lookback sort_lookback_words(N) u64.
constexpr int kSortTile = 3072;  // keys per onesweep tile (256 threads x 12)

struct SortScratch {
  unsigned* hist;
  unsigned* goff;
  u64* lookback;
  long long lookback_words;
};
long long sort_lookback_words(long long maxN);
template <typename WT>
cudaError_t radix_sort_pairs(u64* k0, WT* v0, u64* k1, WT* v1, int N, int bits, SortScratch sc, DevState* st, long long spin_limit,
                             cudaStream_t s, bool* in_alt, int* launches);

// Exclusive scan of int flags/counts: out[i] = sum_{j<i} in[j]; *total = sum.
// part must hold ceil(N/4096)+1 ints.
cudaError_t scan_exclusive_i32(const int* in, int* out, int N, int* part, int* total,
                               cudaStream_t s, int* launches);

// ------------------------------------------------------------- round.cu
constexpr int kEntryTile = 2048;  // entries per block of the entry-parallel kernels

cudaError_t tile_rows(const int64_t* rp, int n, long long M, int* tile_row, cudaStream_t s,
                      int* launches);

// Minimum degree and its vertex (smallest id) -> st->deg_val/deg_arg; lowers
// st->lambda.  The degrees come with the CSR (build_csr).
template <typename WT>
cudaError_t degrees_min(const WT* deg, int n, unsigned long long* blk, DevState* st,
                        cudaStream_t s, int* launches);

// Relabelled entries (L[u] << vbits | L[v], w) appended to keys/vals
// (st->emit_count counts them); self-loops and zero weights dropped; with
// keep_row, only entries whose new row r = L[u] has keep_row[r] == 1.
template <typename WT>
cudaError_t emit_pairs(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                       const int* L, int vbits, const int* tile_row, u64* keys, WT* vals,
                       DevState* st, int validate, cudaStream_t s, int* launches,
                       const int* keep_row = nullptr);

// After sorting: unique keys -> canonical CSR (rp2[n2+1], col2, w2); the
// number of unique entries goes to *m2_dev.  uid/part: N and N/4096+1 ints;
// urow: N ints of scratch (row of each unique entry).
template <typename WT>
cudaError_t build_csr(const u64* keys, const WT* vals, int N, int vbits, int n2, int* uid,
                      int* part, int64_t* rp2, int* col2, WT* w2, DevState* st, int* m2_dev,
                      int* urow, cudaStream_t s, int* launches);

// Input pass over a CSR with non-decreasing rp (rp[0] = 0, rp[n] = M):
// copies col/w from *_src (device memory or mapped host memory) to *_dst
// (no copy when col_dst == col_src) and accumulates into stats (6 words,
// zeroed by the caller): [0] sum of the non-negative weights, [1] any
// negative weight, [2] any entry outside the canonical form, [3], [4] the
// signed symmetry fingerprints and [5] the (u < v) - (u > v) balance, all
// zero for a symmetric canonical graph.  tile_row: tile_rows() of rp.
cudaError_t ingest_csr(int n, long long M, const int64_t* rp, const int* col_src,
                       const int* w_src, int* col_dst, int* w_dst, const int* tile_row,
                       unsigned long long* stats, cudaStream_t s, int* launches);

template <typename WT>
cudaError_t check_symmetric(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                            const int* tile_row, DevState* st, cudaStream_t s, int* launches);

// short_bits: n / 32 + 1 words of scratch for the budget test's bit map.
// st->deg_val must hold the graph's minimum weighted degree (the round's
// degree bound) when bv is null.
template <typename WT>
cudaError_t pr_marks(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                     const WT* deg, const int* tile_row, uint32_t mask, long long budget,
                     int* parent, uint8_t* flags_out, unsigned* short_bits, DevState* st,
                     cudaStream_t s, int* launches, const BatchView* bv = nullptr);

// One label-propagation sweep (vertices with ((v ^ sweep) & 1) == 0 update).
// Rows up to 128 entries use a warp table, up to 4096 a block table, longer
// rows tables of 2d slots from the pool, split into 4096-entry chunks over
// many blocks.
struct LpScratch {
  int* long_rows;               // 2n ints: long-row list, then medium-row list
  int* counts;                  // 4 ints
  int* chunk0;                  // n ints
  long long* tbase;             // n
  unsigned long long* best;     // n
  int* pool_lab;                // pool_slots (>= 2M)
  long long* pool_sc;           // pool_slots
  long long pool_slots;
  unsigned long long* pool_cursor;
};
template <typename WT>
cudaError_t lp_sweep(int n, const int64_t* rp, const int* col, const WT* w, const int* lab_in,
                     int* lab_out, int sweep, const LpScratch& sc, DevState* st, cudaStream_t s,
                     int* launches);

// First LP sweep from identity labels (vertices of parity `sweep` adopt their
// heaviest neighbour, ties to the smaller id).  best: n u64 of scratch.
template <typename WT>
cudaError_t lp_first_sweep(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                           const int* tile_row, int sweep, unsigned long long* best, int* lab_out,
                           cudaStream_t s, int* launches);

// deg[u] = sum of the weights of row u (recomputes tile_row for this CSR).
template <typename WT>
cudaError_t row_degrees(int n, long long M, const int64_t* rp, const WT* w, int* tile_row,
                        WT* deg, cudaStream_t s, int* launches);

// Minimum cut value over the proper clusters of `lab` -> st->lp_val/lp_label.
template <typename WT>
cudaError_t lp_bound(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                     const int* lab, const int* tile_row, long long* cut, int* size,
                     unsigned long long* blk, DevState* st, cudaStream_t s, int* launches);

// union-find / relabel
cudaError_t uf_init(int* parent, int n, cudaStream_t s, int* launches);
cudaError_t uf_hook_pairs(int* parent, const int* pu, const int* pv, long long np, int n,
                          DevState* st, cudaStream_t s, int* launches);
cudaError_t uf_from_groups(int* parent, const int* group, int* gmin, int n, DevState* st,
                           cudaStream_t s, int* launches);
// L[v] = dense rank of find(v); st->n_next = number of roots.
cudaError_t uf_relabel(int* parent, int* L, int* flags, int* rank, int* part, int n,
                       DevState* st, cudaStream_t s, int* launches);
cudaError_t compose_map(int* map0, const int* L, int n0, cudaStream_t s, int* launches);

// witness sides over the original vertices
cudaError_t side_from_vertex(uint8_t* side0, const int* map0, int n0, int x, cudaStream_t s,
                             int* launches);
cudaError_t side_from_label(uint8_t* side0, const int* map0, int n0, const int* lab, int l,
                            cudaStream_t s, int* launches);
cudaError_t side_from_list(uint8_t* side0, const int* map0, int n0, uint8_t* cur, int n,
                           const int* list, int len, cudaStream_t s, int* launches);
cudaError_t side_to_bitmap(const uint8_t* side0, int n0, u64* bitmap, cudaStream_t s,
                           int* launches);

// ---------------------------------------------------------- capforest.cu
struct PassConfig {
  int passes;           // total passes run by the persistent warps
  int table;            // slots per pass (power of two, 256..2048)
  int warps_per_block;
  unsigned long long seed;
  int private_visit = 0;  // 1: each pass has its own visit set (owner is not used)
  // >= 0: the passes do nothing (no marks, no bound) when the round's PR
  // tests already hooked at least this many edges (read on the device from
  // st->marks_pr, so the choice needs no host synchronisation)
  long long skip_pr = -1;
};
// Concurrent CAPFOREST passes (Algorithm 1).  owner[n] must be zero on entry
// (the shared visit array T); visit_log[passes*table], pass_best/pass_len
// [passes]; pass_counter is one int of scratch.  Marks are hooked in parent;
// the best alpha goes to st->cf_val/cf_pass/cf_len.
template <typename WT>
cudaError_t capforest_passes(int n, const int64_t* rp, const int* col, const WT* w,
                             const WT* deg, int* owner, int* parent, int* visit_log,
                             unsigned long long* pass_best, int* pass_len, int* pass_counter,
                             PassConfig pc, DevState* st, cudaStream_t s, int* launches,
                             const BatchView* bv = nullptr);
size_t capforest_pass_smem(int table, int warps_per_block, size_t wt_size);

// One sequential CAPFOREST pass over the whole graph from `start` (one block).
// r[n], tree[seq_tree_words(n)] are scratch (unused when the pass fits in
// shared memory); order[n] receives the visit order; mark_src[n] (nullable)
// holds each vertex's marking edge until the pass ends, when the marks are
// hooked together (NULL: hooked as found); marks_out (nullable) up to
// marks_cap pairs.  The best alpha goes to st->cf_val/cf_len with
// st->cf_pass = -1; st->cf_nscanned counts the visited vertices.
template <typename WT>
cudaError_t capforest_sequential(int n, long long M, const int64_t* rp, const int* col,
                                 const WT* w, const WT* deg, int start, int* parent, WT* r,
                                 int* mark_src, unsigned long long* tree, int* order,
                                 int* marks_out, long long marks_cap, DevState* st,
                                 cudaStream_t s, int* launches);
long long seq_tree_words(int n);

// Batch form: one block per graph g of the view; a graph runs its sequential
// pass (from its first vertex) only if it is not done and marked nothing this
// round (always != 0: regardless of marks).  r[] is indexed by current
// vertex; levels at level_off[g] (words of the key type); order at the
// graph's vertex offset, as local ids.
// `passes` sequential passes at once, pass k from its own start vertex (pass
// 0 from vertex 0) with private keys and visit order: r_pool passes*n WT,
// tree_pool passes*seq_tree_words(n) u64 (only the parts that do not fit in
// shared memory are used), order_pool and mark_pool passes*n ints (mark_pool
// as mark_src of capforest_sequential).  A pass that lowers the
// bound lowers st->lambda; the best such pass k sets st->cf_val, cf_len and
// cf_pass = -2 - k (its visit order is order_pool + k*n).
template <typename WT>
cudaError_t capforest_sequential_multi(int n, long long M, const int64_t* rp, const int* col,
                                       const WT* w, const WT* deg, int passes,
                                       unsigned long long seed,
                                       int* parent, WT* r_pool, unsigned long long* tree_pool,
                                       int* order_pool, int* mark_pool,
                                       unsigned long long* pass_best, int* pass_len,
                                       DevState* st, cudaStream_t s, int* launches);

template <typename WT>
cudaError_t capforest_sequential_batch(int G, const int64_t* rp, const int* col, const WT* w,
                                       const WT* deg, int* parent, WT* r,
                                       unsigned long long* levels, const long long* level_off,
                                       int* order, int max_graph_n, int always,
                                       const BatchView& bv, DevState* st, cudaStream_t s,
                                       int* launches);

// ------------------------------------------------------ capforest_warp.cu
// Whole-graph CAPFOREST passes driven by one warp each (block k = pass k,
// pass 0 from start0, pass k > 0 from a seeded vertex), with private keys and
// visit order and the neighbour-first tie rule (see the file).  Keys are
// min(r, lambda) + 1 in 32 bits; warp_pass_key_bytes(lam) == 0 means lam
// (the bound at launch, which the device state also holds) is too large for
// these passes.  Scratch per pass: r_pool 2n WT,
// lev_pool lev_stride >= warp_pass_lev_bytes(n) bytes, order_pool and
// mark_pool n ints.  Marks are hooked in parent after the passes; the best
// alpha goes to st->lambda and, naming its pass (cf_pass = -2 - k, visit
// order order_pool + k * n), to st->cf_val / cf_len; st->cf_nscanned gets
// pass 0's visited count.  stop_low: a pass stops once it has marked an
// edge and the highest priority left in its queue is below half the bound
// (it has left the region it marked; the marks and alpha of a prefix of a
// maximum-adjacency order stay valid), else it visits every reachable vertex.
constexpr size_t kWarpPassSmem = 200 * 1024;
// global bytes the simultaneous warp passes of a round may keep hot in L2
constexpr long long kWarpPassL2Budget = 80ll << 20;
// passes a round runs at least (device memory and SMs permitting)
constexpr int kWarpPassMin = 4;
// graphs from this many vertices let the passes of a solve's round stop early
constexpr int kWarpStopMinN = 1 << 16;
int warp_pass_key_bytes(long long lam);
long long warp_pass_lev_bytes(int n);
// bytes of global memory a pass keeps reading (r and tree levels that do not
// fit in shared memory); -1 if lam is too large
long long warp_pass_hot_bytes(int n, size_t wt, long long lam);
template <typename WT>
cudaError_t capforest_warp_passes(int n, long long M, const int64_t* rp, const int* col,
                                  const WT* w, const WT* deg, int passes, int start0,
                                  unsigned long long seed, long long lam, int* parent,
                                  WT* r_pool, unsigned char* lev_pool, long long lev_stride,
                                  int* order_pool, int* mark_pool, unsigned long long* pass_best,
                                  int* pass_len, int stop_low, DevState* st, cudaStream_t s,
                                  int* launches);

// ------------------------------------------------------------- contract.cu
// Row-wise contraction when most groups are single vertices: singleton rows
// are rebuilt in place, the rows of multi-member groups (and singleton rows
// that do not fit) go through emit / sort / build as a general CSR.
struct RowScratch {
  int* cnt;     // n: members per group
  int* gen;     // n: group's row takes the general path
  int* len;     // n + 1: final row lengths
  int* kcnt;    // n: distinct moved labels of a singleton row
  int* off;     // n + 1: exclusive scan of len
  int* part;    // scan partials (n / 4096 + 2)
  int* total;   // 1: sum of len (the contracted entry count; in the device state)
  int* side_v;  // M: a singleton row's moved labels at the row's own offset
  int* vinfo;   // n: L[x], with the top bit set when x's group has several members
  unsigned long long* single_entries;  // entries of singleton groups' rows
  int* dsum;    // n: entries of each group's member rows
  int* did;     // n: dense accumulator slot of a dense group
  int* ndense;  // 1: dense groups asked for this round (in the device state)
  int* chunk;   // dense_slots / kDenseChunk + n + 64: per-chunk counts, then offsets
  void* acc;    // dense_slots weights: dense accumulators, n2 per dense group (the caller
                // zeroes slots before their first use; the writing kernel clears what
                // it read)
  long long dense_slots;
  int* dense_group;  // n: group of each dense slot
  unsigned long long* dense_entries;  // entries of the dense groups' rows
  int* rep;     // n: the member of a single-vertex group, -1 for the others
  // entry-tiled path of the singleton rows (graphs of kFlatMinEntries and more)
  int* fcl;       // n: clean entries of each row
  int* kpc;       // n: moved labels of each single-vertex group's row
  int* side_c;    // M: per row, clean entries by the number of moved labels below them
  void* rec;      // n: 16-byte record per row (output offset, moved labels, first label)
  int2* tile_ht;  // entry tiles: clean entries of each tile's first / last row
  int* tile_rowG; // entry tiles of the general CSR
  int* list;      // n: rows with several moved labels (two lists, from both ends)
  int* list_len;  // 2
  int4* vmap;        // n / 32 + 1: compact vertex map (moved, non-root bits, prefix)
  unsigned* mvbits;  // n / 32 + 1: the moved bits alone
};
constexpr int kDenseChunk = 2048;  // accumulator slots per block of the dense kernels
constexpr long long kFlatMinEntries = 1ll << 18;  // entry-tiled singleton rows from here

// Whether a graph of M entries takes the entry-tiled singleton-row path.
bool rows_flat(long long M);

// cnt, gen (multi-member groups) and *single_entries.  n2 only sizes the
// cleared arrays: any bound >= the relabelled vertex count will do.
cudaError_t rows_classify(int n, int n2, const int64_t* rp, const int* L, const RowScratch& rs,
                          cudaStream_t s, int* launches);

// Dense groups the accumulators hold for n2 vertices: min(n2, dense_slots / n2).
int dense_capacity(int n2, const RowScratch& rs);

// Groups whose member rows hold at least max(n2 / 16, 256) entries take a
// dense accumulator of n2 slots (gen = 2) while accumulators are left
// (min(n2, dense_slots / n2) of them); their entries go to *dense_entries.
// n2 is read from n2_dev on the device; n_bound >= n2 sizes the grid.
cudaError_t rows_dense_mark(int n_bound, const int* n2_dev, const RowScratch& rs, cudaStream_t s,
                            int* launches);

// Dense groups: accumulate their entries (acc must be zero), count the
// distinct labels into len.  ndense: the dense groups asked for (*rs.ndense,
// read by the host) size the grids.  On the entry-tiled path the slots of
// multi-member dense groups towards single vertices are transposed into those
// rows' moved lists (side_v / side_w).
template <typename WT>
cudaError_t rows_dense_accumulate(int n, long long M, int n2, const int64_t* rp, const int* col,
                                  const WT* w, const int* L, const int* tile_row,
                                  const RowScratch& rs, int ndense, WT* side_w, cudaStream_t s,
                                  int* launches);

// Singleton rows: len, kcnt and the moved labels with their summed weights
// (side_v / side_w); rows that do not fit are added to gen.  On the
// entry-tiled path (rows_flat(M)) only the clean entries of every row are
// counted here; the moved labels come from the other groups' contracted
// rows in rows_dense_accumulate / rows_finish.  tile_row: the entry tiles of
// this graph; root_flags / root_rank: the union-find roots behind L (1 per
// root) and their exclusive prefix sum.
template <typename WT>
cudaError_t rows_count(int n, long long M, const int64_t* rp, const int* col, const WT* w,
                       const int* L, const int* root_flags, const int* root_rank,
                       const int* tile_row, const RowScratch& rs, WT* side_w, cudaStream_t s,
                       int* launches);

// Final CSR (rp2, col2, w2) and degrees deg2 from the singleton rows and the
// general CSR (rpG over n2 rows, NG entries); rs.total = entries.
template <typename WT>
cudaError_t rows_finish(int n, long long M, int n2, const int64_t* rp, const int* col,
                        const WT* w, const int* L, const RowScratch& rs, int ndense, WT* side_w,
                        const int64_t* rpG, const int* colG, const WT* wG, long long NG,
                        const int* tile_row, int64_t* rp2, int* col2, WT* w2, WT* deg2,
                        cudaStream_t s, int* launches);

}  // namespace mc
