/*
 * oracle.c -- CPU oracle for the exact minimum-cut contraction round.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is called by tests/, by
 * __graft_entry__.smoke() and by the CPU-baseline leg of bench.py; the
 * product (the CUDA library and its Python binding) never links, loads or
 * calls it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Plain, slow and meant to be read against the paper:
 *   - every sum is int64; weights are int64 here whatever the caller stores;
 *   - no blocking, fusion or reordering beyond what the definition states;
 *   - each function names the passage of the paper it follows.
 *
 * Graph convention: CSR with row_ptr int64[n+1], col int32[M], w int64[M].
 * "Canonical" graphs (the only ones the round functions accept) are symmetric,
 * have every row sorted by neighbour id, no duplicate entries, no self-loops
 * and positive weights.  orc_contract() turns any graph into canonical form.
 *
 * Paper references: Sec. 2 "Basic Concepts" (cuts, degrees, contraction,
 * trivial-cut bound), Sec. 2.1 (NOI, CAPFOREST, bounded priority queue,
 * label propagation and the Padberg-Rinaldi tests, collapsed-vertex bound),
 * Algorithm 1 (Parallel CAPFOREST), Algorithm 2 (Parallel Minimum Cut),
 * App. A (Stoer-Wagner, Padberg-Rinaldi local tests), App. C (Stoer-Wagner
 * as an independent check that shares no code with NOI).
 *
 * Parity pins: brute force, closed forms and library cross-checks in
 * tests/test_oracle_*.py.  The label-propagation labels are pinned by
 * hand-traced sweeps (tests/golden/lp_trace.json: ties, the strictly-larger
 * rule and the parity order) and small rule checks; beyond those no closed
 * form fixes them.  The LP *bound* is pinned as a cut value of an explicit
 * vertex set.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF INT64_MAX

static void* xmalloc(size_t b) {
    void* p = malloc(b ? b : 1);
    if (!p) abort();
    return p;
}
static void* xcalloc(size_t n, size_t b) {
    void* p = calloc(n ? n : 1, b ? b : 1);
    if (!p) abort();
    return p;
}

/* ------------------------------------------------------------ degrees */
/* Degree of a vertex = total weight of its incident edges (Sec. 2, Basic
 * Concepts).  Self-loop entries, if present, are not incident edges of a cut
 * and are skipped. */
void orc_degrees(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                 int64_t* deg) {
    for (int32_t u = 0; u < n; ++u) {
        int64_t s = 0;
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
            if (col[e] != u) s += w[e];
        deg[u] = s;
    }
}

/* ---------------------------------------------------------- cut weight */
/* Capacity of the cut (A, V \ A): total weight of the edges between the two
 * sides (Sec. 2, Basic Concepts).  side[v] != 0 marks the vertices of one
 * side.  Each undirected edge appears twice in a symmetric CSR, so the
 * directed sum is halved. */
int64_t orc_cut_weight(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                       const uint8_t* side) {
    int64_t s = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
            if ((side[u] != 0) != (side[col[e]] != 0)) s += w[e];
    return s / 2;
}

/* -------------------------------------------------------- brute force */
/* lambda(G) straight from its definition (Sec. 2): the minimum capacity over
 * all partitions of V into two non-empty sides.  Vertex 0 is fixed on side 0;
 * every assignment of the other n-1 vertices except "all on side 0" is a
 * cut, 2^(n-1) - 1 of them.  Returns -1 when n < 2 (no cut exists) or n > 26.
 * best_side (nullable) receives a minimising side assignment (the first one
 * found in increasing mask order). */
int64_t orc_mincut_brute(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                         uint8_t* best_side) {
    if (n < 2 || n > 26) return -1;
    uint8_t* side = (uint8_t*)xcalloc((size_t)n, 1);
    int64_t best = ORC_INF;
    uint64_t lim = 1ull << (n - 1);
    for (uint64_t mask = 1; mask < lim; ++mask) {
        side[0] = 0;
        for (int32_t v = 1; v < n; ++v) side[v] = (uint8_t)((mask >> (v - 1)) & 1u);
        int64_t c = orc_cut_weight(n, rp, col, w, side);
        if (c < best) {
            best = c;
            if (best_side) memcpy(best_side, side, (size_t)n);
        }
    }
    free(side);
    return best;
}

/* Minimum s-t cut lambda(G, s, t) by brute force (Sec. 2): minimum capacity
 * over the cuts that put s and t on different sides.  n <= 26. */
int64_t orc_st_cut_brute(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                         int32_t s, int32_t t) {
    if (n < 2 || n > 26 || s == t) return -1;
    uint8_t* side = (uint8_t*)xcalloc((size_t)n, 1);
    int64_t best = ORC_INF;
    uint64_t lim = 1ull << (n - 1);
    for (uint64_t mask = 1; mask < lim; ++mask) {
        side[0] = 0;
        for (int32_t v = 1; v < n; ++v) side[v] = (uint8_t)((mask >> (v - 1)) & 1u);
        if (side[s] == side[t]) continue;
        int64_t c = orc_cut_weight(n, rp, col, w, side);
        if (c < best) best = c;
    }
    free(side);
    return best;
}

/* -------------------------------------------------- binary max-heap */
/* Entries (key, v) ordered by larger key first, then smaller vertex id.
 * Stale entries are skipped by the callers (lazy deletion). */
typedef struct {
    int64_t key;
    int32_t v;
} hent;
typedef struct {
    hent* a;
    int64_t n, cap;
} heap_t;

static int hbefore(hent x, hent y) { return x.key > y.key || (x.key == y.key && x.v < y.v); }
static void hpush(heap_t* h, int64_t key, int32_t v) {
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 64;
        h->a = (hent*)realloc(h->a, (size_t)h->cap * sizeof(hent));
        if (!h->a) abort();
    }
    int64_t i = h->n++;
    hent x = {key, v};
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hbefore(x, h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = x;
}
static hent hpop(heap_t* h) {
    hent top = h->a[0];
    hent x = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        hent bx = x;
        if (l < h->n && hbefore(h->a[l], bx)) { b = l; bx = h->a[l]; }
        if (r < h->n && hbefore(h->a[r], bx)) { b = r; bx = h->a[r]; }
        if (b == i) break;
        h->a[i] = h->a[b];
        i = b;
    }
    if (h->n > 0) h->a[i] = x;
    return top;
}

/* ------------------------------------------------------- Stoer-Wagner */
/* Stoer-Wagner (cited in App. A; used by the authors as an implementation
 * that shares no code with NOI, App. C).  Each phase grows a set A by
 * maximum adjacency from an arbitrary active vertex; the last vertex t added
 * gives the "cut of the phase" ({t's members}, rest) whose value is t's
 * connection weight to A; then t is merged into the vertex added before it.
 * The minimum cut-of-the-phase over n-1 phases is lambda(G).
 * Merged vertices are kept as member lists; rep[] maps every input vertex to
 * the merged vertex it belongs to.  best_side (nullable) gets the members of
 * the best phase's last vertex. */
int64_t orc_stoer_wagner(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                         uint8_t* best_side) {
    if (n < 2) return -1;
    int32_t* rep = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int32_t* nxt = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int32_t* tail = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    uint8_t* active = (uint8_t*)xmalloc((size_t)n);
    int64_t* key = (int64_t*)xmalloc((size_t)n * sizeof(int64_t));
    int64_t* inA = (int64_t*)xmalloc((size_t)n * sizeof(int64_t));
    for (int32_t v = 0; v < n; ++v) {
        rep[v] = v; nxt[v] = -1; tail[v] = v; active[v] = 1; inA[v] = -1;
    }
    heap_t h = {0};
    int32_t nact = n;
    int64_t best = ORC_INF;
    int64_t phase = 0;
    while (nact > 1) {
        h.n = 0;
        for (int32_t v = 0; v < n; ++v)
            if (active[v]) { key[v] = 0; hpush(&h, 0, v); }
        int32_t prev = -1, last = -1, cnt = 0;
        int64_t lastkey = 0;
        while (cnt < nact) {
            hent t = hpop(&h);
            int32_t v = t.v;
            if (!active[v] || inA[v] == phase || t.key != key[v]) continue;
            inA[v] = phase;
            ++cnt;
            prev = last;
            last = v;
            lastkey = key[v];
            for (int32_t m = v; m >= 0; m = nxt[m])
                for (int64_t e = rp[m]; e < rp[m + 1]; ++e) {
                    int32_t u = rep[col[e]];
                    if (u == v || inA[u] == phase) continue;
                    key[u] += w[e];
                    hpush(&h, key[u], u);
                }
        }
        if (lastkey < best) {
            best = lastkey;
            if (best_side) {
                memset(best_side, 0, (size_t)n);
                for (int32_t m = last; m >= 0; m = nxt[m]) best_side[m] = 1;
            }
        }
        /* merge last into prev */
        for (int32_t m = last; m >= 0; m = nxt[m]) rep[m] = prev;
        nxt[tail[prev]] = last;
        tail[prev] = tail[last];
        active[last] = 0;
        --nact;
        ++phase;
    }
    free(h.a);
    free(rep); free(nxt); free(tail); free(active); free(key); free(inA);
    return best;
}

/* ------------------------------------------------ canonical labelling */
/* Canonical labels of a grouping: vertices with equal group[] value form one
 * contracted vertex; contracted vertices are numbered 0, 1, ... in increasing
 * order of their smallest member.  Returns n' (the number of groups).
 * group[] values must lie in [0, n). */
int32_t orc_labels_from_groups(int32_t n, const int32_t* group, int32_t* L) {
    int32_t* id = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    for (int32_t g = 0; g < n; ++g) id[g] = -1;
    int32_t next = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t g = group[v];
        if (id[g] < 0) id[g] = next++;
        L[v] = id[g];
    }
    free(id);
    return next;
}

/* Canonical labels of the components of the marked-edge graph (V, pairs):
 * marking an edge contractible and merging its endpoints (Alg. 1, the
 * union-find U) groups V into these components.  Components are found by
 * breadth-first search and numbered by increasing smallest member. */
int32_t orc_labels_from_pairs(int32_t n, int64_t np, const int32_t* pu, const int32_t* pv,
                              int32_t* L) {
    int64_t* head = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < np; ++i) { head[pu[i] + 1]++; head[pv[i] + 1]++; }
    for (int32_t v = 0; v < n; ++v) head[v + 1] += head[v];
    int32_t* adj = (int32_t*)xmalloc((size_t)(2 * np + 1) * sizeof(int32_t));
    int64_t* cur = (int64_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int64_t));
    memcpy(cur, head, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < np; ++i) {
        adj[cur[pu[i]]++] = pv[i];
        adj[cur[pv[i]]++] = pu[i];
    }
    int32_t* q = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v) L[v] = -1;
    int32_t next = 0;
    for (int32_t s = 0; s < n; ++s) {
        if (L[s] >= 0) continue;
        int64_t qh = 0, qt = 0;
        L[s] = next;
        q[qt++] = s;
        while (qh < qt) {
            int32_t v = q[qh++];
            for (int64_t e = head[v]; e < head[v + 1]; ++e)
                if (L[adj[e]] < 0) { L[adj[e]] = next; q[qt++] = adj[e]; }
        }
        ++next;
    }
    free(head); free(adj); free(cur); free(q);
    return next;
}

/* --------------------------------------------------------- contraction */
static int cmp_colw(const void* a, const void* b) {
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

/* Contraction (Sec. 2, Basic Concepts): every group of vertices with equal
 * canonical label L[] (dense in [0, n2)) becomes one vertex that inherits the
 * group's edges; edges that become parallel are merged by summing weights,
 * edges inside a group vanish (self-loops dropped), and zero-weight entries
 * are dropped.  The output is canonical: row g lists its neighbours in
 * increasing id.  Outputs rp2[n2+1], col2[<=M], w2[<=M] are caller-allocated;
 * returns M2. */
int64_t orc_contract(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                     const int32_t* L, int32_t n2, int64_t* rp2, int32_t* col2, int64_t* w2) {
    int64_t* cnt = (int64_t*)xcalloc((size_t)n2 + 1, sizeof(int64_t));
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
            if (L[u] != L[col[e]] && w[e] != 0) cnt[L[u] + 1]++;
    for (int32_t g = 0; g < n2; ++g) cnt[g + 1] += cnt[g];
    int64_t tot = cnt[n2];
    int64_t* buf = (int64_t*)xmalloc((size_t)(2 * tot + 2) * sizeof(int64_t));
    int64_t* cur = (int64_t*)xmalloc((size_t)(n2 ? n2 : 1) * sizeof(int64_t));
    memcpy(cur, cnt, (size_t)n2 * sizeof(int64_t));
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t gu = L[u], gv = L[col[e]];
            if (gu == gv || w[e] == 0) continue;
            int64_t p = cur[gu]++;
            buf[2 * p] = gv;
            buf[2 * p + 1] = w[e];
        }
    int64_t out = 0;
    rp2[0] = 0;
    for (int32_t g = 0; g < n2; ++g) {
        int64_t b = cnt[g], e = cnt[g + 1];
        qsort(buf + 2 * b, (size_t)(e - b), 2 * sizeof(int64_t), cmp_colw);
        for (int64_t i = b; i < e; ++i) {
            if (out > rp2[g] && col2[out - 1] == (int32_t)buf[2 * i]) {
                w2[out - 1] += buf[2 * i + 1];
            } else {
                col2[out] = (int32_t)buf[2 * i];
                w2[out] = buf[2 * i + 1];
                ++out;
            }
        }
        rp2[g + 1] = out;
    }
    free(cnt); free(buf); free(cur);
    return out;
}

/* --------------------------------------------- Padberg-Rinaldi tests */
/* Local contraction tests of Padberg and Rinaldi (named in Sec. 2.1 and
 * App. A; the paper does not state them).  Reading used here, for an edge
 * e = {u, v} of a canonical graph and an upper bound lambda <= min degree:
 *   PR1: c(u,v) >= lambda                                   (threshold)
 *   PR2: c(u) < 2 c(u,v)  or  c(v) < 2 c(u,v)               (strict exchange)
 *   PR3: some common neighbour x with c(u) < 2 (c(u,v) + c(u,x)) and
 *        c(v) < 2 (c(u,v) + c(v,x))                         (strict exchange)
 *   PR4: c(u,v) + sum over common neighbours x of min(c(u,x), c(v,x))
 *        >= lambda                                          (threshold)
 * PR3/PR4 are evaluated only when min(|N(u)|, |N(v)|) <= budget (budget < 0:
 * always).  flags[e] gets bit 0..3 for PR1..PR4 (restricted to `mask`), the
 * same value on both directed entries of an edge. */
void orc_pr_marks(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                  int64_t lambda, uint32_t mask, int64_t budget, uint8_t* flags) {
    int64_t* deg = (int64_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int64_t));
    orc_degrees(n, rp, col, w, deg);
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = col[e];
            int64_t c = w[e];
            uint8_t f = 0;
            if ((mask & 1u) && c >= lambda) f |= 1;
            if ((mask & 2u) && (deg[u] < 2 * c || deg[v] < 2 * c)) f |= 2;
            int64_t du = rp[u + 1] - rp[u], dv = rp[v + 1] - rp[v];
            int64_t dmin = du < dv ? du : dv;
            if ((mask & 12u) && (budget < 0 || dmin <= budget)) {
                int64_t sum = c;
                int pr3 = 0;
                int64_t i = rp[u], j = rp[v];
                while (i < rp[u + 1] && j < rp[v + 1]) {
                    if (col[i] < col[j]) ++i;
                    else if (col[i] > col[j]) ++j;
                    else {
                        int32_t x = col[i];
                        if (x != u && x != v) {
                            int64_t cux = w[i], cvx = w[j];
                            sum += cux < cvx ? cux : cvx;
                            if (deg[u] < 2 * (c + cux) && deg[v] < 2 * (c + cvx)) pr3 = 1;
                        }
                        ++i; ++j;
                    }
                }
                if ((mask & 4u) && pr3) f |= 4;
                if ((mask & 8u) && sum >= lambda) f |= 8;
            }
            flags[e] = f;
        }
    free(deg);
}

/* ------------------------------------------------------------ CAPFOREST */
/* CAPFOREST as one process of Algorithm 1 (with a single process the shared
 * visit array T only records this pass, so the blacklist B stays empty).
 * Starting from `start`, repeatedly take the unvisited vertex x of highest
 * priority (the bounded priority queue of Sec. 2.1: keys are
 * Q(y) = min(r(y), lambda) as of y's last update; ties go to the smaller
 * vertex id), mark it visited, set alpha += c(x) - 2 r(x) and
 * lambda = min(lambda, alpha) while the visited set is a proper subset of V,
 * then scan every edge e = {x, y} to an unvisited y: if
 * r(y) < lambda <= r(y) + c(e) the edge is marked contractible; r(y) grows by
 * c(e); q(e) = r(y); Q(y) = min(r(y), lambda).
 * Outputs (all nullable): mark_u/mark_v (capacity M/2) and *nmarks, the visit
 * order (capacity n) and *nscanned, q_out[M] (q(e) on the entry x->y that was
 * scanned, -1 elsewhere), *best_len = length of the visited prefix whose cut
 * gave the returned lambda (0 if lambda never dropped below lambda_in).
 * Returns the final lambda.
 * Note: when alpha lowers lambda, every queued y has r(y) = c(y, S) <= c(S,
 * V \ S) = alpha, so no stored key exceeds the new bound; re-capping the queue
 * at that moment would change nothing. */
/* The same pass with a choice of tie rule among the vertices of highest
 * priority (Sec. 2.1 leaves the order inside a bucket of the bounded priority
 * queue open -- FIFO, LIFO, heap; any order keeps the pass a maximum-adjacency
 * ordering and every mark sound):
 *   tie = 0: the smaller vertex id;
 *   tie = 1: neighbour first -- after x's row has been scanned, if some
 *            unvisited y in x's row has the highest priority, the next vertex
 *            is the first such y in x's row order; otherwise the smaller
 *            vertex id among those of highest priority.
 * Everything else is as described above. */
int64_t orc_capforest_tie(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                          int64_t lambda, int32_t start, int32_t tie, int32_t* mark_u,
                          int32_t* mark_v, int64_t* nmarks, int32_t* order, int32_t* nscanned,
                          int64_t* q_out, int32_t* best_len) {
    int64_t* deg = (int64_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int64_t));
    orc_degrees(n, rp, col, w, deg);
    int64_t* r = (int64_t*)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));
    int64_t* key = (int64_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t* visited = (uint8_t*)xcalloc((size_t)(n ? n : 1), 1);
    for (int32_t v = 0; v < n; ++v) key[v] = -1;
    if (q_out)
        for (int64_t e = 0; e < rp[n]; ++e) q_out[e] = -1;
    heap_t h = {0};
    int64_t nm = 0, alpha = 0;
    int32_t ns = 0, blen = 0;
    int32_t x = n > 0 ? start : -1;  /* the next vertex to visit */
    while (x >= 0) {
        visited[x] = 1;
        if (order) order[ns] = x;
        ++ns;
        alpha += deg[x] - 2 * r[x];
        if (ns < n && alpha < lambda) {
            lambda = alpha;
            blen = ns;
        }
        for (int64_t e = rp[x]; e < rp[x + 1]; ++e) {
            int32_t y = col[e];
            if (visited[y]) continue;
            if (r[y] < lambda && lambda <= r[y] + w[e]) {
                if (mark_u) { mark_u[nm] = x; mark_v[nm] = y; }
                ++nm;
            }
            r[y] += w[e];
            if (q_out) q_out[e] = r[y];
            key[y] = r[y] < lambda ? r[y] : lambda;
            hpush(&h, key[y], y);
        }
        /* drop stale heap entries: the top is then the highest priority */
        while (h.n > 0 && (visited[h.a[0].v] || h.a[0].key != key[h.a[0].v])) hpop(&h);
        if (h.n == 0) break;
        int64_t top = h.a[0].key;
        int32_t next = -1;
        if (tie == 1) {
            for (int64_t e = rp[x]; e < rp[x + 1]; ++e) {
                int32_t y = col[e];
                if (!visited[y] && key[y] == top) { next = y; break; }
            }
        }
        if (next < 0) next = hpop(&h).v;
        x = next;
    }
    if (nmarks) *nmarks = nm;
    if (nscanned) *nscanned = ns;
    if (best_len) *best_len = blen;
    free(h.a);
    free(deg); free(r); free(key); free(visited);
    return lambda;
}

int64_t orc_capforest(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                      int64_t lambda, int32_t start, int32_t* mark_u, int32_t* mark_v,
                      int64_t* nmarks, int32_t* order, int32_t* nscanned, int64_t* q_out,
                      int32_t* best_len) {
    return orc_capforest_tie(n, rp, col, w, lambda, start, 0, mark_u, mark_v, nmarks, order,
                             nscanned, q_out, best_len);
}

/* ------------------------------------------------ label propagation */
/* Label propagation (Sec. 2.1, "Lowering the upper bound"; the paper gives
 * no details).  Reading used here: labels start as the vertex ids; sweep s
 * (s = 0 .. iters-1) updates the vertices v with ((v ^ s) & 1) == 0 from the
 * labels of the previous sweep: v adopts the neighbour label of largest total
 * edge weight to v (ties: the smaller label) if that weight is strictly
 * larger than the weight of v's own label among its neighbours. */
static int cmp_lw(const void* a, const void* b) {
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}
void orc_lp(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w, int32_t iters,
            int32_t* label) {
    int32_t* old = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        label[v] = v;
        if (rp[v + 1] - rp[v] > maxdeg) maxdeg = rp[v + 1] - rp[v];
    }
    int64_t* buf = (int64_t*)xmalloc((size_t)(2 * maxdeg + 2) * sizeof(int64_t));
    for (int32_t s = 0; s < iters; ++s) {
        memcpy(old, label, (size_t)n * sizeof(int32_t));
        for (int32_t v = 0; v < n; ++v) {
            if (((v ^ s) & 1) != 0) continue;
            int64_t k = 0;
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                buf[2 * k] = old[col[e]];
                buf[2 * k + 1] = w[e];
                ++k;
            }
            if (k == 0) continue;
            qsort(buf, (size_t)k, 2 * sizeof(int64_t), cmp_lw);
            int64_t own = 0, bestw = -1, bestl = -1;
            for (int64_t i = 0; i < k;) {
                int64_t l = buf[2 * i], sum = 0;
                while (i < k && buf[2 * i] == l) { sum += buf[2 * i + 1]; ++i; }
                if (l == old[v]) own = sum;
                if (sum > bestw) { bestw = sum; bestl = l; }
            }
            if (bestw > own) label[v] = (int32_t)bestl;
        }
    }
    free(old);
    free(buf);
}

/* Cluster bound (Sec. 2.1: any cut found by the heuristic is a valid upper
 * bound): for every label l whose cluster C_l = {v : label[v] = l} is a proper
 * non-empty subset of V, the cut value c(C_l, V \ C_l).  Returns the minimum
 * (ORC_INF when no proper cluster exists); *best_label gets the smallest label
 * attaining it. */
int64_t orc_lp_bound(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
                     const int32_t* label, int32_t* best_label) {
    int64_t* cut = (int64_t*)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));
    int64_t* size = (int64_t*)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));
    for (int32_t u = 0; u < n; ++u) {
        size[label[u]]++;
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
            if (label[col[e]] != label[u]) cut[label[u]] += w[e];
    }
    int64_t best = ORC_INF;
    int32_t bl = -1;
    for (int32_t l = 0; l < n; ++l)
        if (size[l] > 0 && size[l] < n && cut[l] < best) { best = cut[l]; bl = l; }
    if (best_label) *best_label = bl;
    free(cut);
    free(size);
    return best;
}

/* ---------------------------------------------------- one round */
typedef struct {
    int64_t lambda_in;  /* upper bound carried in (ORC_INF: none) */
    int32_t lp_iters;   /* label-propagation sweeps; 0 disables */
    int32_t lp_min_n;   /* run LP only when n >= lp_min_n */
    uint32_t pr_mask;   /* PR1..PR4 bits */
    int64_t pr_budget;  /* PR3/PR4 intersection budget (<0: none) */
    int32_t capforest;  /* 1: one sequential CAPFOREST pass from cf_start */
    int32_t cf_start;
} orc_round_opts;

typedef struct {
    int64_t lambda_out;
    int32_t n2;
    int64_t M2;
    int64_t marks_pr;
    int64_t marks_cf;
    int32_t stopped; /* 1: n <= 2 or lambda == 0 after the degree bound, no contraction */
} orc_round_res;

/* One deterministic contraction round: the degree bound (trivial cuts,
 * Sec. 2, and the collapsed-vertex bound, Sec. 2.1 "Overall algorithm"), the
 * label-propagation cluster bound when n >= lp_min_n, the PR marks on the
 * round's graph with that bound, one sequential CAPFOREST pass (Algorithm 1
 * with one process, started at cf_start), then contraction of the components
 * of all marked edges (Algorithm 2's contraction step).  If n <= 2 or the
 * bound is 0 after the degree bound the graph is returned unchanged.
 * Outputs rp2[n+1], col2[M], w2[M] are caller-allocated. */
int orc_round(int32_t n, const int64_t* rp, const int32_t* col, const int64_t* w,
              const orc_round_opts* o, int64_t* rp2, int32_t* col2, int64_t* w2,
              orc_round_res* res) {
    int64_t M = rp[n];
    int64_t lambda = o->lambda_in;
    memset(res, 0, sizeof(*res));
    if (n >= 2) {
        int64_t* deg = (int64_t*)xmalloc((size_t)n * sizeof(int64_t));
        orc_degrees(n, rp, col, w, deg);
        for (int32_t v = 0; v < n; ++v)
            if (deg[v] < lambda) lambda = deg[v];
        free(deg);
    }
    if (n <= 2 || lambda == 0) {
        memcpy(rp2, rp, (size_t)(n + 1) * sizeof(int64_t));
        memcpy(col2, col, (size_t)M * sizeof(int32_t));
        memcpy(w2, w, (size_t)M * sizeof(int64_t));
        res->lambda_out = lambda;
        res->n2 = n;
        res->M2 = M;
        res->stopped = 1;
        return 0;
    }
    if (o->lp_iters > 0 && n >= o->lp_min_n) {
        int32_t* lab = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
        orc_lp(n, rp, col, w, o->lp_iters, lab);
        int64_t b = orc_lp_bound(n, rp, col, w, lab, NULL);
        if (b < lambda) lambda = b;
        free(lab);
    }
    int32_t* pu = (int32_t*)xmalloc((size_t)(M + 1) * sizeof(int32_t));
    int32_t* pv = (int32_t*)xmalloc((size_t)(M + 1) * sizeof(int32_t));
    int64_t np = 0;
    if (o->pr_mask) {
        uint8_t* fl = (uint8_t*)xmalloc((size_t)(M + 1));
        orc_pr_marks(n, rp, col, w, lambda, o->pr_mask, o->pr_budget, fl);
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
                if (fl[e] && u < col[e]) { pu[np] = u; pv[np] = col[e]; ++np; }
        free(fl);
    }
    res->marks_pr = np;
    if (o->capforest) {
        int64_t nm = 0;
        lambda = orc_capforest(n, rp, col, w, lambda, o->cf_start, pu + np, pv + np, &nm, NULL,
                               NULL, NULL, NULL);
        np += nm;
        res->marks_cf = nm;
    }
    int32_t* L = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int32_t n2 = orc_labels_from_pairs(n, np, pu, pv, L);
    res->M2 = orc_contract(n, rp, col, w, L, n2, rp2, col2, w2);
    res->n2 = n2;
    res->lambda_out = lambda;
    free(L); free(pu); free(pv);
    return 0;
}

/* ------------------------------------------------------ sequential NOI */
/* The exact algorithm with one process (Algorithm 2 with Algorithm 1 run as
 * a single pass, no heuristic bound, no PR tests): lambda starts at the
 * minimum degree; each round runs one CAPFOREST pass from vertex 0, contracts
 * the components of the marked edges and applies the collapsed-vertex bound
 * (the degree of every contracted vertex is a cut value).  It stops when at
 * most two vertices remain or lambda = 0.  best_side (nullable, n entries)
 * receives the side of a cut of value lambda: 1 on the side not containing
 * vertex 0.  *rounds_out (nullable) gets the number of CAPFOREST rounds.
 * The input may be non-canonical; it is canonicalised first. */
int64_t orc_noi(int32_t n, const int64_t* rp_in, const int32_t* col_in, const int64_t* w_in,
                uint8_t* best_side, int32_t* rounds_out) {
    if (n < 2) return -1;
    int64_t M = rp_in[n];
    int32_t* L = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int32_t* map0 = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    uint8_t* side = (uint8_t*)xcalloc((size_t)n, 1);
    int64_t* rp = (int64_t*)xmalloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* col = (int32_t*)xmalloc((size_t)(M + 1) * sizeof(int32_t));
    int64_t* w = (int64_t*)xmalloc((size_t)(M + 1) * sizeof(int64_t));
    int64_t* rp2 = (int64_t*)xmalloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* col2 = (int32_t*)xmalloc((size_t)(M + 1) * sizeof(int32_t));
    int64_t* w2 = (int64_t*)xmalloc((size_t)(M + 1) * sizeof(int64_t));
    int32_t* pu = (int32_t*)xmalloc((size_t)(M / 2 + 1) * sizeof(int32_t));
    int32_t* pv = (int32_t*)xmalloc((size_t)(M / 2 + 1) * sizeof(int32_t));
    int32_t* order = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int64_t* deg = (int64_t*)xmalloc((size_t)n * sizeof(int64_t));
    uint8_t* inS = (uint8_t*)xcalloc((size_t)n, 1);
    for (int32_t v = 0; v < n; ++v) { L[v] = v; map0[v] = v; }
    int64_t Mc = orc_contract(n, rp_in, col_in, w_in, L, n, rp, col, w);
    (void)Mc;
    int32_t cn = n;
    int64_t lambda = ORC_INF;
    int32_t rounds = 0;
    for (;;) {
        if (cn >= 2) {
            orc_degrees(cn, rp, col, w, deg);
            int32_t arg = -1;
            for (int32_t v = 0; v < cn; ++v)
                if (deg[v] < lambda) { lambda = deg[v]; arg = v; }
            if (arg >= 0)
                for (int32_t v0 = 0; v0 < n; ++v0) side[v0] = (uint8_t)(map0[v0] == arg);
        }
        if (cn <= 2 || lambda == 0) break;
        int64_t nm = 0;
        int32_t ns = 0, blen = 0;
        int64_t lam2 = orc_capforest(cn, rp, col, w, lambda, 0, pu, pv, &nm, order, &ns, NULL,
                                     &blen);
        ++rounds;
        if (lam2 < lambda) {
            memset(inS, 0, (size_t)cn);
            for (int32_t i = 0; i < blen; ++i) inS[order[i]] = 1;
            for (int32_t v0 = 0; v0 < n; ++v0) side[v0] = inS[map0[v0]];
            lambda = lam2;
        }
        if (lambda == 0) break;
        int32_t n2 = orc_labels_from_pairs(cn, nm, pu, pv, L);
        int64_t M2 = orc_contract(cn, rp, col, w, L, n2, rp2, col2, w2);
        for (int32_t v0 = 0; v0 < n; ++v0) map0[v0] = L[map0[v0]];
        int64_t* t1 = rp; rp = rp2; rp2 = t1;
        int32_t* t2 = col; col = col2; col2 = t2;
        int64_t* t3 = w; w = w2; w2 = t3;
        (void)M2;
        cn = n2;
    }
    if (best_side) {
        uint8_t flip = side[0];
        for (int32_t v0 = 0; v0 < n; ++v0) best_side[v0] = (uint8_t)(side[v0] ^ flip);
    }
    if (rounds_out) *rounds_out = rounds;
    free(L); free(map0); free(side); free(rp); free(col); free(w); free(rp2); free(col2);
    free(w2); free(pu); free(pv); free(order); free(deg); free(inS);
    return lambda;
}
