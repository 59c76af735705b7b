// server.cu -- continuous-batching solve server (host runtime of the library).
//
// Requests (host CSR graphs) arrive at any time through
// mincut_server_submit.  A request is admitted when a device worker is free
// and the summed footprint estimate of the admitted requests stays under the
// HBM cap.  Each worker owns a CUDA stream, so admitted requests run
// concurrently on the device; while some run, newly arrived ones are admitted
// as soon as a worker and memory free up (no waiting for a whole batch).  A
// worker that takes a small request also takes the small requests queued right
// behind it and solves them together as one packed batch
// (mincut_batch_from_csr / mincut_batch_solve); large requests are solved
// alone.  Every graph's contraction state stays on the device for the whole
// solve.  Results are exact, so a request's value is the same alone or in the
// mix.
#include <algorithm>
#include <chrono>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mincut.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  int64_t n = 0;
  std::vector<int64_t> rp;     // owned copy (mincut_server_submit) ...
  std::vector<int32_t> col, w;
  const int64_t* prp = nullptr;  // ... or the caller's arrays (submit_borrowed)
  const int32_t* pcol = nullptr;
  const int32_t* pw = nullptr;
  int64_t footprint = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
  int status = MINCUT_OK;
  int64_t value = -1;
  std::vector<uint64_t> bitmap;
  int packed = 0;
};

using ReqPtr = std::shared_ptr<Request>;

}  // namespace

struct mincut_server {
  mincut_server_options opt{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ReqPtr> queue;
  std::unordered_map<uint64_t, ReqPtr> live;
  int64_t inflight_bytes = 0;
  int inflight = 0;
  uint64_t next_id = 1;
  bool stopping = false;
  std::vector<std::thread> workers;
  mincut_server_stats st{};
  // warp-solver threshold of packed solves when solve.batch_small_n = 0: timed
  // on the first packed solve, then reused (0: not yet, -1: none)
  std::atomic<int> bw_small_n{0};
};

namespace {

void finish(mincut_server* S, const std::vector<ReqPtr>& reqs) {
  const double t = now_ms();
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto& r : reqs) {
    r->t_done = t;
    r->done = true;
    S->inflight_bytes -= r->footprint;
    S->inflight -= 1;
    S->st.completed += 1;
  }
  S->cv_done.notify_all();
  S->cv_work.notify_all();
}

void solve_alone(const mincut_server_options& o, cudaStream_t s, const ReqPtr& r) {
  mincut_graph* g = nullptr;
  r->status = mincut_graph_from_csr(r->n, r->prp, r->pcol, r->pw, MINCUT_HOST_PTRS, (void*)s,
                                    nullptr, &g);
  if (r->status != MINCUT_OK) return;
  if (o.want_bitmap) r->bitmap.assign((size_t)((r->n + 63) / 64), 0);
  r->status = mincut_solve(g, &o.solve, &r->value, o.want_bitmap ? r->bitmap.data() : nullptr,
                           nullptr);
  mincut_graph_destroy(g);
}

void solve_packed(mincut_server* S, const mincut_server_options& o, cudaStream_t s,
                  std::vector<ReqPtr>& reqs) {
  const size_t G = reqs.size();
  std::vector<int64_t> voff(G + 1, 0);
  int64_t entries = 0;
  for (size_t i = 0; i < G; ++i) {
    voff[i + 1] = voff[i] + reqs[i]->n;
    entries += reqs[i]->prp[reqs[i]->n];
  }
  std::vector<int64_t> rp((size_t)voff[G] + 1);
  std::vector<int32_t> col((size_t)std::max<int64_t>(entries, 1)), w((size_t)std::max<int64_t>(entries, 1));
  int64_t e0 = 0;
  for (size_t i = 0; i < G; ++i) {
    const Request& r = *reqs[i];
    for (int64_t v = 0; v < r.n; ++v) rp[(size_t)(voff[i] + v)] = e0 + r.prp[(size_t)v];
    const int64_t m = r.prp[r.n];
    for (int64_t e = 0; e < m; ++e) {
      col[(size_t)(e0 + e)] = r.pcol[(size_t)e] + (int32_t)voff[i];
      w[(size_t)(e0 + e)] = r.pw[(size_t)e];
    }
    e0 += m;
  }
  rp[(size_t)voff[G]] = e0;
  mincut_graph* g = nullptr;
  int rc = mincut_batch_from_csr((int64_t)G, voff.data(), rp.data(), col.data(), w.data(),
                                 MINCUT_HOST_PTRS, (void*)s, nullptr, &g);
  std::vector<int64_t> vals(G, -1);
  std::vector<uint64_t> bm;
  if (rc == MINCUT_OK) {
    if (o.want_bitmap) bm.assign((size_t)((voff[G] + 63) / 64), 0);
    mincut_options so = o.solve;
    const int tuned = S->bw_small_n.load();
    if (so.batch_small_n == 0 && tuned != 0) so.batch_small_n = tuned;
    rc = mincut_batch_solve(g, &so, vals.data(), o.want_bitmap ? bm.data() : nullptr, nullptr);
    if (rc == MINCUT_OK && so.batch_small_n == 0) {
      int32_t t = 0;
      int64_t k = 0;
      if (mincut_batch_info(g, &t, &k) == MINCUT_OK) S->bw_small_n.store(t > 0 ? t : -1);
    }
    mincut_graph_destroy(g);
  }
  if (rc != MINCUT_OK) {  // isolate the failing request(s)
    for (auto& r : reqs) solve_alone(o, s, r);
    return;
  }
  for (size_t i = 0; i < G; ++i) {
    Request& r = *reqs[i];
    r.status = MINCUT_OK;
    r.value = vals[i];
    r.packed = 1;
    if (o.want_bitmap) {
      r.bitmap.assign((size_t)((r.n + 63) / 64), 0);
      for (int64_t v = 0; v < r.n; ++v) {
        const int64_t gv = voff[i] + v;
        if ((bm[(size_t)(gv >> 6)] >> (gv & 63)) & 1ull) r.bitmap[(size_t)(v >> 6)] |= 1ull << (v & 63);
      }
    }
  }
}

void worker_loop(mincut_server* S, int wid) {
  (void)wid;
  cudaSetDevice(S->opt.device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  const mincut_server_options& o = S->opt;
  for (;;) {
    std::vector<ReqPtr> take;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (!S->queue.empty()) {
          const ReqPtr& h = S->queue.front();
          // admit the head if it fits under the cap (or nothing else runs)
          if (S->inflight == 0 || S->inflight_bytes + h->footprint <= o.hbm_cap_bytes) break;
        } else if (S->stopping) {
          break;
        }
        S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      }
      if (S->queue.empty()) break;  // stopping and drained
      ReqPtr h = S->queue.front();
      S->queue.pop_front();
      take.push_back(h);
      S->inflight_bytes += h->footprint;
      S->inflight += 1;
      if (h->n <= o.pack_max_n && o.pack_max_requests > 1) {
        int64_t verts = h->n;
        while (!S->queue.empty() && (int)take.size() < o.pack_max_requests) {
          const ReqPtr& q = S->queue.front();
          if (q->n > o.pack_max_n || verts + q->n > o.pack_max_vertices ||
              S->inflight_bytes + q->footprint > o.hbm_cap_bytes)
            break;
          verts += q->n;
          S->inflight_bytes += q->footprint;
          S->inflight += 1;
          take.push_back(q);
          S->queue.pop_front();
        }
      }
      S->st.peak_inflight_bytes = std::max(S->st.peak_inflight_bytes, S->inflight_bytes);
      S->st.peak_inflight = std::max<int32_t>(S->st.peak_inflight, S->inflight);
      if (take.size() > 1) {
        S->st.packed_batches += 1;
        S->st.packed_requests += (int64_t)take.size();
      } else {
        S->st.single_solves += 1;
      }
    }
    const double t = now_ms();
    for (auto& r : take) r->t_start = t;
    if (take.size() == 1) solve_alone(o, s, take[0]);
    else solve_packed(S, o, s, take);
    finish(S, take);
  }
  cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

void mincut_server_default_options(mincut_server_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->workers = 4;
  o->hbm_cap_bytes = 60ll << 30;
  o->pack_max_n = 4096;
  o->pack_max_requests = 256;
  o->pack_max_vertices = 1 << 20;
  o->want_bitmap = 1;
  o->device = 0;
  mincut_default_options(&o->solve);
}

int mincut_server_create(const mincut_server_options* opts, mincut_server** out) {
  if (!out) return MINCUT_ERR_INVALID;
  *out = nullptr;
  mincut_server* S = new mincut_server();
  if (opts) S->opt = *opts; else mincut_server_default_options(&S->opt);
  if (S->opt.workers < 1 || S->opt.workers > 64 || S->opt.hbm_cap_bytes <= 0) {
    delete S;
    return MINCUT_ERR_INVALID;
  }
  for (int i = 0; i < S->opt.workers; ++i) S->workers.emplace_back(worker_loop, S, i);
  *out = S;
  return MINCUT_OK;
}

static int submit_impl(mincut_server* S, int64_t n, const int64_t* row_ptr, const int32_t* col,
                       const int32_t* w, bool borrow, uint64_t* request_id) {
  if (!S || !row_ptr || !request_id || n < 2 || n > 0x7ffffffe) return MINCUT_ERR_INVALID;
  const int64_t m = row_ptr[n];
  if (row_ptr[0] != 0 || m < 0 || (m > 0 && (!col || !w))) return MINCUT_ERR_INVALID;
  auto r = std::make_shared<Request>();
  r->n = n;
  if (borrow && m > 0) {
    r->prp = row_ptr;
    r->pcol = col;
    r->pw = w;
  } else {
    r->rp.assign(row_ptr, row_ptr + n + 1);
    r->col.assign(col, col + m);
    r->w.assign(w, w + m);
    if (m == 0) { r->col.push_back(0); r->w.push_back(0); }
    r->prp = r->rp.data();
    r->pcol = r->col.data();
    r->pw = r->w.data();
  }
  r->footprint = mincut_graph_footprint(n, m);
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return MINCUT_ERR_INVALID;
    r->id = S->next_id++;
    S->live[r->id] = r;
    S->queue.push_back(r);
    S->st.submitted += 1;
  }
  S->cv_work.notify_one();
  *request_id = r->id;
  return MINCUT_OK;
}

int mincut_server_submit(mincut_server* S, int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* w, uint64_t* request_id) {
  return submit_impl(S, n, row_ptr, col, w, false, request_id);
}

int mincut_server_submit_borrowed(mincut_server* S, int64_t n, const int64_t* row_ptr,
                                  const int32_t* col, const int32_t* w, uint64_t* request_id) {
  return submit_impl(S, n, row_ptr, col, w, true, request_id);
}

int mincut_server_wait(mincut_server* S, uint64_t request_id, int64_t* cut_value,
                       double* latency_ms, uint64_t* side_bitmap) {
  if (!S) return MINCUT_ERR_INVALID;
  ReqPtr r;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(request_id);
    if (it == S->live.end()) return MINCUT_ERR_INVALID;
    r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    S->live.erase(it);
  }
  if (cut_value) *cut_value = r->value;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  if (side_bitmap && !r->bitmap.empty())
    memcpy(side_bitmap, r->bitmap.data(), r->bitmap.size() * sizeof(uint64_t));
  return r->status;
}

int mincut_server_stats_read(mincut_server* S, mincut_server_stats* out) {
  if (!S || !out) return MINCUT_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->inflight_bytes = S->inflight_bytes;
  out->queued = (int64_t)S->queue.size();
  return MINCUT_OK;
}

void mincut_server_destroy(mincut_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
