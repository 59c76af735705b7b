/*
 * synth.c -- seeded synthetic graph generators (input construction only).
 *
 * These generators build the undirected, integer-weighted input graphs used by
 * the tests and the benchmark: Erdos-Renyi G(n, m), R-MAT, k-core reduction,
 * largest-connected-component extraction, the planted two-block cut instance
 * and the small "LP-support-like" graphs of the batched workload.  They hold
 * none of the minimum-cut arithmetic (no cut values, no contraction, no
 * CAPFOREST, no reductions): both the CPU oracle and the CUDA path consume the
 * graphs they produce.
 *
 * Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used as a counter-free sequential stream
 * seeded by the caller.  Bounded integers use the multiply-high reduction
 * (Lemire 2019), which is exactly reproducible on x86_64 and aarch64.
 *
 * Output format: symmetric CSR.  row_ptr int64[n+1], col int32[M], w int32[M],
 * M = 2m; every row sorted by neighbour id, no duplicates, no self-loops.
 * Memory returned by these functions is malloc'ed and released by synth_free.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int64_t n;
    int64_t m;        /* undirected edges */
    int64_t* row_ptr; /* n+1 */
    int32_t* col;     /* 2m */
    int32_t* w;       /* 2m */
} synth_graph;

/* ------------------------------------------------------------------ RNG */
static inline uint64_t sm64_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform integer in [0, range) */
static inline uint64_t sm64_below(uint64_t* s, uint64_t range) {
    unsigned __int128 p = (unsigned __int128)sm64_next(s) * (unsigned __int128)range;
    return (uint64_t)(p >> 64);
}
/* uniform double in [0, 1) with 53 random bits */
static inline double sm64_unit(uint64_t* s) {
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t synth_splitmix64(uint64_t state, uint64_t* next_state) {
    uint64_t v = sm64_next(&state);
    if (next_state) *next_state = state;
    return v;
}

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

/* ------------------------------------------------ LSD radix sort (u64) */
/* Sorts keys ascending over the low `bits` bits with 11-bit digits.  Used to
 * deduplicate pair lists; carries no payload. */
static void radix_sort_u64(uint64_t* a, int64_t n, int bits) {
    if (n < 2) return;
    uint64_t* tmp = (uint64_t*)xmalloc((size_t)n * sizeof(uint64_t));
    int64_t* cnt = (int64_t*)xmalloc(2048 * sizeof(int64_t));
    uint64_t* src = a;
    uint64_t* dst = tmp;
    for (int shift = 0; shift < bits; shift += 11) {
        memset(cnt, 0, 2048 * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 2047]++;
        int64_t s = 0;
        for (int d = 0; d < 2048; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 2047]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp);
    free(cnt);
}

static int bits_for(uint64_t x) { /* number of bits to represent values < x */
    int b = 0;
    while (b < 64 && (1ull << b) < x) ++b;
    return b;
}

/* Sort + unique a list of undirected pair keys (u << 32 | v with u < v). */
static int64_t sort_unique_pairs(uint64_t* keys, int64_t k, int64_t n) {
    int vb = bits_for((uint64_t)n);
    radix_sort_u64(keys, k, 32 + vb);
    int64_t out = 0;
    for (int64_t i = 0; i < k; ++i)
        if (out == 0 || keys[out - 1] != keys[i]) keys[out++] = keys[i];
    return out;
}

/* Build a symmetric CSR from sorted unique pairs (u < v) with weights. */
static void csr_from_pairs(int64_t n, const uint64_t* keys, const int32_t* wt, int64_t m,
                           synth_graph* g) {
    g->n = n;
    g->m = m;
    g->row_ptr = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
    g->col = (int32_t*)xmalloc((size_t)(2 * m) * sizeof(int32_t));
    g->w = (int32_t*)xmalloc((size_t)(2 * m) * sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) {
        int64_t u = (int64_t)(keys[i] >> 32), v = (int64_t)(keys[i] & 0xffffffffull);
        g->row_ptr[u + 1]++;
        g->row_ptr[v + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
    int64_t* cur = (int64_t*)xmalloc((size_t)n * sizeof(int64_t));
    memcpy(cur, g->row_ptr, (size_t)n * sizeof(int64_t));
    /* pass 1: lower neighbours (v's entry pointing at u < v), in increasing u */
    for (int64_t i = 0; i < m; ++i) {
        int64_t u = (int64_t)(keys[i] >> 32), v = (int64_t)(keys[i] & 0xffffffffull);
        int64_t p = cur[v]++;
        g->col[p] = (int32_t)u;
        g->w[p] = wt ? wt[i] : 1;
    }
    /* pass 2: upper neighbours (u's entry pointing at v > u), in increasing v */
    for (int64_t i = 0; i < m; ++i) {
        int64_t u = (int64_t)(keys[i] >> 32), v = (int64_t)(keys[i] & 0xffffffffull);
        int64_t p = cur[u]++;
        g->col[p] = (int32_t)v;
        g->w[p] = wt ? wt[i] : 1;
    }
    free(cur);
}

static inline uint64_t pair_key(int64_t a, int64_t b) {
    int64_t u = a < b ? a : b, v = a < b ? b : a;
    return ((uint64_t)u << 32) | (uint64_t)v;
}

static int32_t* draw_weights(uint64_t* s, int64_t m, int32_t wlo, int32_t whi) {
    int32_t* wt = (int32_t*)xmalloc((size_t)(m ? m : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i)
        wt[i] = (wlo == whi) ? wlo : (int32_t)(wlo + (int64_t)sm64_below(s, (uint64_t)(whi - wlo + 1)));
    return wt;
}

void synth_free(synth_graph* g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g->w);
    g->row_ptr = NULL;
    g->col = NULL;
    g->w = NULL;
}

/* --------------------------------------------------------------- G(n,m) */
/* m distinct unordered pairs drawn uniformly (rejecting self-loops and
 * duplicates), weights uniform in [wlo, whi]. */
int synth_er(int64_t n, int64_t m, int32_t wlo, int32_t whi, uint64_t seed, synth_graph* g) {
    if (n < 2 || m < 0 || m > n * (n - 1) / 2 || n > 0x7fffffff) return -1;
    uint64_t s = seed;
    uint64_t* keys = (uint64_t*)xmalloc((size_t)(m ? m : 1) * sizeof(uint64_t));
    int64_t have = 0;
    while (have < m) {
        int64_t need = m - have;
        for (int64_t i = 0; i < need; ++i) {
            int64_t a, b;
            do {
                a = (int64_t)sm64_below(&s, (uint64_t)n);
                b = (int64_t)sm64_below(&s, (uint64_t)n);
            } while (a == b);
            keys[have + i] = pair_key(a, b);
        }
        /* compacts in place: the sorted unique prefix stays, the tail is refilled */
        have = sort_unique_pairs(keys, m, n);
    }
    int32_t* wt = draw_weights(&s, m, wlo, whi);
    csr_from_pairs(n, keys, wt, m, g);
    free(keys);
    free(wt);
    return 0;
}

/* ---------------------------------------------------------------- R-MAT */
/* scale, edge_factor: 2^scale vertices, edge_factor * 2^scale generated
 * edges; quadrant probabilities (a, b, c, 1-a-b-c); then a seeded random
 * permutation of the vertex ids; duplicates and self-loops removed; weights
 * uniform in [wlo, whi] drawn after deduplication. */
int synth_rmat(int scale, int64_t edge_factor, double a, double b, double c, int32_t wlo,
               int32_t whi, uint64_t seed, synth_graph* g) {
    if (scale < 1 || scale > 30) return -1;
    int64_t n = (int64_t)1 << scale;
    int64_t k = edge_factor * n;
    uint64_t s = seed;
    uint64_t* keys = (uint64_t*)xmalloc((size_t)(k ? k : 1) * sizeof(uint64_t));
    int64_t kk = 0;
    double ab = a + b, abc = a + b + c;
    for (int64_t i = 0; i < k; ++i) {
        int64_t u = 0, v = 0;
        for (int lvl = 0; lvl < scale; ++lvl) {
            double r = sm64_unit(&s);
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        keys[kk++] = ((uint64_t)u << 32) | (uint64_t)v;
    }
    /* random permutation of ids (Fisher-Yates) */
    int32_t* perm = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&s, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    int64_t out = 0;
    for (int64_t i = 0; i < kk; ++i) {
        int64_t u = perm[keys[i] >> 32], v = perm[keys[i] & 0xffffffffull];
        if (u == v) continue;
        keys[out++] = pair_key(u, v);
    }
    free(perm);
    int64_t m = sort_unique_pairs(keys, out, n);
    int32_t* wt = draw_weights(&s, m, wlo, whi);
    csr_from_pairs(n, keys, wt, m, g);
    free(keys);
    free(wt);
    return 0;
}

/* ------------------------------------------- vertex-subset extraction */
/* Keep the vertices with keep[v] != 0, relabelled in increasing old id
 * (rows stay sorted).  old_id_out (optional, malloc'ed) maps new -> old. */
static void induced_subgraph(const synth_graph* in, const uint8_t* keep, synth_graph* out,
                             int32_t** old_id_out) {
    int64_t n = in->n;
    int32_t* nid = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    int64_t n2 = 0;
    for (int64_t v = 0; v < n; ++v) nid[v] = keep[v] ? (int32_t)(n2++) : -1;
    out->n = n2;
    out->row_ptr = (int64_t*)xcalloc((size_t)n2 + 1, sizeof(int64_t));
    int64_t M2 = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (!keep[v]) continue;
        for (int64_t e = in->row_ptr[v]; e < in->row_ptr[v + 1]; ++e)
            if (keep[in->col[e]]) M2++;
    }
    out->col = (int32_t*)xmalloc((size_t)(M2 ? M2 : 1) * sizeof(int32_t));
    out->w = (int32_t*)xmalloc((size_t)(M2 ? M2 : 1) * sizeof(int32_t));
    int64_t p = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (!keep[v]) continue;
        for (int64_t e = in->row_ptr[v]; e < in->row_ptr[v + 1]; ++e) {
            int32_t y = in->col[e];
            if (!keep[y]) continue;
            out->col[p] = nid[y];
            out->w[p] = in->w[e];
            ++p;
        }
        out->row_ptr[nid[v] + 1] = p;
    }
    out->m = M2 / 2;
    if (old_id_out) {
        int32_t* old = (int32_t*)xmalloc((size_t)(n2 ? n2 : 1) * sizeof(int32_t));
        for (int64_t v = 0; v < n; ++v)
            if (keep[v]) old[nid[v]] = (int32_t)v;
        *old_id_out = old;
    }
    free(nid);
}

/* k-core by peeling (vertices of current edge count < k removed until none
 * remain); the count is the number of incident edges, not their weight. */
static void kcore_keep(const synth_graph* g, int64_t k, uint8_t* keep) {
    int64_t n = g->n;
    int64_t* d = (int64_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int32_t* q = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t qh = 0, qt = 0;
    for (int64_t v = 0; v < n; ++v) {
        d[v] = g->row_ptr[v + 1] - g->row_ptr[v];
        keep[v] = 1;
        if (d[v] < k) { keep[v] = 0; q[qt++] = (int32_t)v; }
    }
    while (qh < qt) {
        int32_t v = q[qh++];
        for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            int32_t y = g->col[e];
            if (keep[y] && --d[y] < k) { keep[y] = 0; q[qt++] = y; }
        }
    }
    free(d);
    free(q);
}

/* keep[] restricted to the largest connected component (ties: the one
 * containing the smallest vertex id). */
static void lcc_keep(const synth_graph* g, uint8_t* keep) {
    int64_t n = g->n;
    int32_t* comp = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int32_t* q = (int32_t*)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v) comp[v] = -1;
    int32_t best = -1, nc = 0;
    int64_t bestsz = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (!keep[s] || comp[s] >= 0) continue;
        int64_t qh = 0, qt = 0, sz = 0;
        comp[s] = nc;
        q[qt++] = (int32_t)s;
        while (qh < qt) {
            int32_t v = q[qh++];
            ++sz;
            for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
                int32_t y = g->col[e];
                if (keep[y] && comp[y] < 0) { comp[y] = nc; q[qt++] = y; }
            }
        }
        if (sz > bestsz) { bestsz = sz; best = nc; }
        ++nc;
    }
    for (int64_t v = 0; v < n; ++v) keep[v] = (keep[v] && comp[v] == best) ? 1 : 0;
    free(comp);
    free(q);
}

/* k-core (k <= 0: none) followed by the largest connected component (lcc
 * != 0), relabelled densely in increasing old id. */
int synth_core_lcc(const synth_graph* in, int64_t k, int lcc, synth_graph* out,
                   int32_t** old_id_out) {
    uint8_t* keep = (uint8_t*)xmalloc((size_t)(in->n ? in->n : 1));
    if (k > 0) kcore_keep(in, k, keep);
    else memset(keep, 1, (size_t)in->n);
    if (lcc) lcc_keep(in, keep);
    induced_subgraph(in, keep, out, old_id_out);
    free(keep);
    return 0;
}

/* Vertices with id < nkeep, then (lcc != 0) the largest connected
 * component, relabelled densely in increasing old id. */
int synth_truncate_lcc(const synth_graph* in, int64_t nkeep, int lcc, synth_graph* out) {
    uint8_t* keep = (uint8_t*)xmalloc((size_t)(in->n ? in->n : 1));
    for (int64_t v = 0; v < in->n; ++v) keep[v] = v < nkeep ? 1 : 0;
    if (lcc) lcc_keep(in, keep);
    induced_subgraph(in, keep, out, NULL);
    free(keep);
    return 0;
}

/* ------------------------------------------------------- planted cut */
/* Two independent G(nb, mb) blocks with unit weights, each reduced to its
 * kcore-core, joined by `cross` random edges of weight `cross_w` between
 * uniformly chosen surviving vertices (a repeated pair sums its weight).
 * Vertex ids are then randomly permuted.  block_out (malloc'ed) gives 0/1
 * block membership per final vertex. */
int synth_planted(int64_t nb, int64_t mb, int64_t kcore, int64_t cross, int32_t cross_w,
                  uint64_t seed, synth_graph* g, uint8_t** block_out) {
    uint64_t s = seed;
    synth_graph blk[2], core[2];
    for (int i = 0; i < 2; ++i) {
        uint64_t bs = sm64_next(&s);
        if (synth_er(nb, mb, 1, 1, bs, &blk[i]) != 0) return -1;
        synth_core_lcc(&blk[i], kcore, 0, &core[i], NULL);
        synth_free(&blk[i]);
        if (core[i].n < 1) return -2;
    }
    int64_t n0 = core[0].n, n1 = core[1].n, n = n0 + n1;
    int64_t m_in = core[0].m + core[1].m;
    /* collect all undirected pairs (u < v) of both blocks, then cross pairs */
    uint64_t* keys = (uint64_t*)xmalloc((size_t)(m_in + cross + 1) * sizeof(uint64_t));
    int32_t* wt = (int32_t*)xmalloc((size_t)(m_in + cross + 1) * sizeof(int32_t));
    /* random permutation of the final ids */
    int32_t* perm = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&s, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    int64_t k = 0;
    for (int b = 0; b < 2; ++b) {
        int64_t off = b ? n0 : 0;
        for (int64_t u = 0; u < core[b].n; ++u)
            for (int64_t e = core[b].row_ptr[u]; e < core[b].row_ptr[u + 1]; ++e) {
                int64_t v = core[b].col[e];
                if (u < v) { keys[k] = pair_key(perm[u + off], perm[v + off]); wt[k] = 1; ++k; }
            }
    }
    /* cross edges, merged by pair */
    int64_t kc0 = k;
    for (int64_t i = 0; i < cross; ++i) {
        int64_t a = (int64_t)sm64_below(&s, (uint64_t)n0);
        int64_t b = n0 + (int64_t)sm64_below(&s, (uint64_t)n1);
        keys[k] = pair_key(perm[a], perm[b]);
        wt[k] = cross_w;
        ++k;
    }
    /* sort pairs with weights: encode index into a parallel sort */
    {
        /* simple approach: sort keys of inner edges, and merge cross pairs
         * (at most `cross`) afterwards */
        uint64_t* inner = keys;
        radix_sort_u64(inner, kc0, 32 + bits_for((uint64_t)n));
        /* aggregate cross pairs */
        int64_t nc = 0;
        uint64_t* ck = (uint64_t*)xmalloc((size_t)(cross + 1) * sizeof(uint64_t));
        int32_t* cw = (int32_t*)xmalloc((size_t)(cross + 1) * sizeof(int32_t));
        for (int64_t i = kc0; i < k; ++i) {
            int64_t j;
            for (j = 0; j < nc; ++j)
                if (ck[j] == keys[i]) break;
            if (j == nc) { ck[nc] = keys[i]; cw[nc] = 0; ++nc; }
            cw[j] += wt[i];
        }
        /* sort cross keys (insertion sort, nc <= cross) */
        for (int64_t i = 1; i < nc; ++i) {
            uint64_t kk = ck[i];
            int32_t ww = cw[i];
            int64_t j = i - 1;
            while (j >= 0 && ck[j] > kk) { ck[j + 1] = ck[j]; cw[j + 1] = cw[j]; --j; }
            ck[j + 1] = kk;
            cw[j + 1] = ww;
        }
        /* merge two sorted lists (cross pairs never coincide with inner ones) */
        uint64_t* mk = (uint64_t*)xmalloc((size_t)(kc0 + nc + 1) * sizeof(uint64_t));
        int32_t* mw = (int32_t*)xmalloc((size_t)(kc0 + nc + 1) * sizeof(int32_t));
        int64_t i = 0, j = 0, o = 0;
        while (i < kc0 || j < nc) {
            if (j >= nc || (i < kc0 && inner[i] < ck[j])) { mk[o] = inner[i++]; mw[o] = 1; }
            else { mk[o] = ck[j]; mw[o] = cw[j]; ++j; }
            ++o;
        }
        csr_from_pairs(n, mk, mw, o, g);
        free(mk); free(mw); free(ck); free(cw);
    }
    if (block_out) {
        uint8_t* bl = (uint8_t*)xmalloc((size_t)n);
        for (int64_t i = 0; i < n; ++i) bl[perm[i]] = (i >= n0) ? 1 : 0;
        *block_out = bl;
    }
    free(perm);
    free(keys);
    free(wt);
    synth_free(&core[0]);
    synth_free(&core[1]);
    return 0;
}

/* ------------------------------------------------ small batched graphs */
/* One graph of the batched workload: n vertices, a random Hamiltonian cycle
 * (connected, LP-support-like) plus extra distinct random pairs up to
 * m = ceil(n * d / 2) edges, weights uniform in [wlo, whi]. */
int synth_cycle_plus(int64_t n, double d, int32_t wlo, int32_t whi, uint64_t seed,
                     synth_graph* g) {
    if (n < 3) return -1;
    uint64_t s = seed;
    int64_t m = (int64_t)ceil((double)n * d / 2.0);
    int64_t mmax = n * (n - 1) / 2;
    if (m < n) m = n;
    if (m > mmax) m = mmax;
    int32_t* perm = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&s, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    uint64_t* keys = (uint64_t*)xmalloc((size_t)(m + n) * sizeof(uint64_t));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) keys[k++] = pair_key(perm[i], perm[(i + 1) % n]);
    k = sort_unique_pairs(keys, k, n);
    while (k < m) {
        int64_t need = m - k;
        for (int64_t i = 0; i < need; ++i) {
            int64_t a, b;
            do {
                a = (int64_t)sm64_below(&s, (uint64_t)n);
                b = (int64_t)sm64_below(&s, (uint64_t)n);
            } while (a == b);
            keys[k + i] = pair_key(a, b);
        }
        k = sort_unique_pairs(keys, m, n);
    }
    int32_t* wt = draw_weights(&s, m, wlo, whi);
    csr_from_pairs(n, keys, wt, m, g);
    free(perm);
    free(keys);
    free(wt);
    return 0;
}

/* ---- adversarial families: every edge fails the PR tests and each round
 * of a contraction algorithm that relies on them can merge only a few
 * vertices.  Both are built from pairs with weights, ids permuted by seed. */
typedef struct { uint64_t key; int32_t w; } wpair;

static int wpair_cmp(const void* a, const void* b) {
    const uint64_t x = ((const wpair*)a)->key, y = ((const wpair*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static void csr_from_wpairs(int64_t n, wpair* pr, int64_t m, uint64_t seed, synth_graph* g) {
    uint64_t s = seed;
    int32_t* perm = (int32_t*)xmalloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&s, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int64_t i = 0; i < m; ++i) {
        const int64_t u = (int64_t)(pr[i].key >> 32), v = (int64_t)(pr[i].key & 0xffffffffull);
        pr[i].key = pair_key(perm[u], perm[v]);
    }
    qsort(pr, (size_t)m, sizeof(wpair), wpair_cmp);
    uint64_t* keys = (uint64_t*)xmalloc((size_t)m * sizeof(uint64_t));
    int32_t* wt = (int32_t*)xmalloc((size_t)m * sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) { keys[i] = pr[i].key; wt[i] = pr[i].w; }
    csr_from_pairs(n, keys, wt, m, g);
    free(keys);
    free(wt);
    free(perm);
}

/* Wheel: hub plus a rim cycle of n-1 vertices; spokes of weight 2, rim edges
 * of weight n-2, so every vertex has weighted degree 2(n-1) and all n trivial
 * cuts are minimum: a cut that keeps the hub on one side and a proper part S
 * of the rim on the other crosses at least two rim edges, 2(n-2) + 2|S| >=
 * 2(n-1).  lambda = 2(n-1).  n >= 5. */
int synth_wheel(int64_t n, uint64_t seed, synth_graph* g) {
    if (n < 5 || 2 * (n - 1) > 0x7fffffffll) return -1;
    const int64_t r = n - 1, m = 2 * r;
    wpair* pr = (wpair*)xmalloc((size_t)m * sizeof(wpair));
    for (int64_t i = 0; i < r; ++i) {
        pr[i].key = pair_key(0, 1 + i);
        pr[i].w = 2;
        pr[r + i].key = pair_key(1 + i, 1 + (i + 1) % r);
        pr[r + i].w = (int32_t)(n - 2);
    }
    csr_from_wpairs(n, pr, m, seed, g);
    free(pr);
    return 0;
}

/* Two interleaved cycles: a Hamiltonian cycle 0-1-...-(n-1)-0 of weight
 * `heavy`, and on each half {0..h-1}, {h..n-1} (h = n/2, odd) the cycle
 * j -> j+2 (mod h) of weight `light`.  Any proper cut crosses the Hamiltonian
 * cycle at least twice; it avoids the light cycles only if each half lies on
 * one side, so the two halves are the unique minimum cut and lambda =
 * 2*heavy; every other cut is at least 2*heavy + 2*light.  n = 2h, h >= 5
 * odd. */
int synth_dblcyc(int64_t n, int32_t heavy, int32_t light, uint64_t seed, synth_graph* g) {
    const int64_t h = n / 2;
    if (n != 2 * h || h < 5 || (h & 1) == 0 || heavy < 1 || light < 1) return -1;
    const int64_t m = n + n;
    wpair* pr = (wpair*)xmalloc((size_t)m * sizeof(wpair));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        pr[k].key = pair_key(i, (i + 1) % n);
        pr[k++].w = heavy;
    }
    for (int64_t half = 0; half < 2; ++half)
        for (int64_t j = 0; j < h; ++j) {
            pr[k].key = pair_key(half * h + j, half * h + (j + 2) % h);
            pr[k++].w = light;
        }
    csr_from_wpairs(n, pr, m, seed, g);
    free(pr);
    return 0;
}

/* Parameters of graph i of the batched workload, drawn from seed: n
 * log-uniform in [nlo, nhi], average degree uniform in [dlo, dhi]. */
void synth_batch_params(uint64_t seed, int64_t i, int64_t nlo, int64_t nhi, double dlo,
                        double dhi, int64_t* n_out, double* d_out, uint64_t* seed_out) {
    uint64_t s = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(i + 1));
    sm64_next(&s);
    double u = sm64_unit(&s);
    double ln = log((double)nlo) + u * (log((double)nhi) - log((double)nlo));
    int64_t n = (int64_t)floor(exp(ln));
    if (n < nlo) n = nlo;
    if (n > nhi) n = nhi;
    *n_out = n;
    *d_out = dlo + sm64_unit(&s) * (dhi - dlo);
    *seed_out = sm64_next(&s);
}
