/*
 * Triangle-centrality oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the triangle
 * centrality path computes (P. Burkhardt, "Triangle Centrality"), in exact
 * 64-bit integers with one correctly rounded binary64 quotient at the end.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call it; the product library never links or loads it, and it shares no
 * code, header or table with the CUDA sources.
 *
 * Conventions (the paper is 1-based, section "Notation"; this file is
 * 0-based): vertices 0..n-1; the input is any list of (src, dst) pairs,
 * which is symmetrised, stripped of self-loops and de-duplicated to give the
 * simple undirected graph G of the paper's section "Comparison" set-up.
 * The canonical adjacency is a CSR whose rows are sorted ascending.
 *
 * What each routine follows:
 *   og_edge_triangles   t(v,u) = |N(v) ∩ N(u)| for every adjacency entry,
 *                       i.e. the graph triangle matrix T = A^2 ∘ A of the
 *                       Notation section, by sorted-list merge.
 *   og_vertex_triangles △(v) = ½ ||T_v||_1 (Theorem quoted in the "Algebraic Form" subsection; the
 *                       printed second equality "= T_v^T 1" drops the ½ and
 *                       is not used).
 *   og_total            △(G) = ⅙ 1^T T 1 = ⅓ Σ_v △(v).
 *   og_numer_definition Definition 1 multiplied through by 3△(G):
 *                       numer(v) = Σ_{u∈N△[v]} △(u) + 3 Σ_{w∈N(v)\N△(v)} △(w),
 *                       with N△(v) = {u ∈ N(v) : N(u) ∩ N(v) ≠ ∅}.
 *   og_numer_algebraic  Proposition 2: numerator ½ [(3A − 2T̂ + I) T 1]_v
 *                       over the denominator ½ 1^T T 1 = 3△(G).
 *   og_fast_edge_triangles  the same T restricted to degree-ordered
 *                       higher neighbourhoods N_H (Notation; Chiba–Nishizeki
 *                       listing, section "Algorithm"): each triangle is met once from
 *                       its lowest-ordered vertex and credited to its three
 *                       edges.  Used only to reach larger graphs; checked
 *                       against og_edge_triangles.
 *   og_sample_*         the definition evaluated at chosen vertices only,
 *                       with the marker-array membership test of Procedure 1
 *                       (mark N(v), scan N(u)); used for sampled checks on
 *                       graphs too large for the full routines.
 *   og_sample_tri       △(v) and the row of T = A² ∘ A at chosen vertices
 *                       only (marker test), for graphs whose hubs make the
 *                       sampled numerator too costly.
 *   og_div_rn           TC(v) = numer(v) / (3△(G)) rounded to nearest-even
 *                       binary64 (one exact rational, one rounding).
 *
 * Readings of the paper taken here: △(G) = 0 yields a NaN quotient (the
 * paper leaves TC undefined on triangle-free graphs); isolated vertices have
 * △ = 0 and numerator 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    int64_t m;        /* undirected edges */
    int64_t* ptr;     /* n + 1 */
    int32_t* adj;     /* 2m, each row ascending */
} og_graph;

static int og_cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Canonical simple undirected graph from arbitrary pairs: every pair (a, b)
 * with a != b is entered as b in row a and a in row b (counting sort by
 * row), each row is sorted and its repeats dropped.  Returns NULL if an id
 * is outside [0, n) or memory runs out. */
og_graph* og_build(const int32_t* src, const int32_t* dst, int64_t np, int64_t n) {
    if (n < 0 || np < 0 || n > INT32_MAX) return NULL;
    for (int64_t i = 0; i < np; ++i)
        if (src[i] < 0 || dst[i] < 0 || src[i] >= n || dst[i] >= n) return NULL;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return NULL;
    for (int64_t i = 0; i < np; ++i)
        if (src[i] != dst[i]) { cnt[src[i] + 1] += 1; cnt[dst[i] + 1] += 1; }   /* self-loops dropped */
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int64_t total = cnt[n];
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
    if (!buf || !fill || !g) { free(cnt); free(buf); free(fill); free(g); return NULL; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < np; ++i) {
        if (src[i] == dst[i]) continue;
        buf[fill[src[i]]++] = dst[i];          /* both directions */
        buf[fill[dst[i]]++] = src[i];
    }
    free(fill);
    g->n = n;
    g->ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->ptr) { free(cnt); free(buf); free(g); return NULL; }
    int64_t out = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = cnt[v], e = cnt[v + 1];
        qsort(buf + b, (size_t)(e - b), sizeof(int32_t), og_cmp_i32);
        g->ptr[v] = out;
        for (int64_t i = b; i < e; ++i)
            if (i == b || buf[i] != buf[i - 1]) buf[out++] = buf[i];   /* duplicates dropped */
    }
    g->ptr[n] = out;
    free(cnt);
    g->m = out / 2;
    g->adj = (int32_t*)realloc(buf, sizeof(int32_t) * (size_t)(out + 1));
    if (!g->adj) g->adj = buf;
    return g;
}

void og_free(og_graph* g) {
    if (!g) return;
    free(g->ptr);
    free(g->adj);
    free(g);
}

void og_info(const og_graph* g, int64_t* n, int64_t* m) { *n = g->n; *m = g->m; }

void og_copy_csr(const og_graph* g, int64_t* ptr, int32_t* adj) {
    memcpy(ptr, g->ptr, sizeof(int64_t) * (size_t)(g->n + 1));
    memcpy(adj, g->adj, sizeof(int32_t) * (size_t)(2 * g->m));
}

/* |N(a) ∩ N(b)| of two ascending rows by a two-pointer merge. */
static uint64_t og_common(const og_graph* g, int64_t a, int64_t b) {
    int64_t i = g->ptr[a], ie = g->ptr[a + 1], j = g->ptr[b], je = g->ptr[b + 1];
    uint64_t c = 0;
    while (i < ie && j < je) {
        if (g->adj[i] < g->adj[j]) ++i;
        else if (g->adj[i] > g->adj[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* t[p] = |N(v) ∩ N(u)| for the adjacency entry p = (v, u): T = A^2 ∘ A. */
void og_edge_triangles(const og_graph* g, uint64_t* t) {
    for (int64_t v = 0; v < g->n; ++v)
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p)
            t[p] = og_common(g, v, g->adj[p]);
}

/* △(v) = ½ Σ_u t(v,u).  Returns -1 if some row sum is odd (impossible for a
 * symmetric T), else 0. */
int og_vertex_triangles(const og_graph* g, const uint64_t* t, uint64_t* tri) {
    int bad = 0;
    for (int64_t v = 0; v < g->n; ++v) {
        uint64_t s = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) s += t[p];
        if (s & 1u) bad = 1;
        tri[v] = s / 2;
    }
    return bad ? -1 : 0;
}

/* △(G) = ⅓ Σ_v △(v); *rem gets Σ mod 3 (must be 0). */
uint64_t og_total(const og_graph* g, const uint64_t* tri, uint64_t* rem) {
    uint64_t s = 0;
    for (int64_t v = 0; v < g->n; ++v) s += tri[v];
    if (rem) *rem = s % 3;
    return s / 3;
}

/* Definition 1 times 3△(G):
 *   x = Σ_{u ∈ N△[v]} △(u)            (triangle core, v included)
 *   y = Σ_{w ∈ N(v) \ N△(v)} △(w)     (neighbours in no triangle with v)
 *   numer(v) = x + 3y                  so TC(v) = numer(v) / (3△(G)). */
void og_numer_definition(const og_graph* g, const uint64_t* t, const uint64_t* tri,
                         uint64_t* numer, uint64_t* core, uint64_t* noncore) {
    for (int64_t v = 0; v < g->n; ++v) {
        uint64_t x = tri[v], y = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) {
            int32_t u = g->adj[p];
            if (t[p] > 0) x += tri[u];      /* u ∈ N△(v): N(u) ∩ N(v) ≠ ∅ */
            else y += tri[u];
        }
        numer[v] = x + 3 * y;
        if (core) core[v] = x;
        if (noncore) noncore[v] = y;
    }
}

/* Proposition 2: z = T 1, r = (3A − 2T̂ + I) z with T̂ the 0/1 pattern of T;
 * numerator = r / 2, denominator = 1^T z / 2.  Returns -1 if r or 1^T z is
 * odd, else 0; *den gets 1^T z / 2. */
int og_numer_algebraic(const og_graph* g, const uint64_t* t, uint64_t* numer, uint64_t* den) {
    uint64_t* z = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(g->n + 1));
    if (!z) return -2;
    uint64_t total = 0;
    for (int64_t v = 0; v < g->n; ++v) {
        uint64_t s = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) s += t[p];
        z[v] = s;
        total += s;
    }
    int bad = 0;
    for (int64_t v = 0; v < g->n; ++v) {
        uint64_t a3 = 0, t2 = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) {
            int32_t u = g->adj[p];
            a3 += 3 * z[u];
            if (t[p] > 0) t2 += 2 * z[u];
        }
        uint64_t r = a3 - t2 + z[v];
        if (r & 1u) bad = 1;
        numer[v] = r / 2;
    }
    if (total & 1u) bad = 1;
    if (den) *den = total / 2;
    free(z);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Degree-ordered listing (larger graphs).                              */
/* ------------------------------------------------------------------ */

/* π(u) < π(v) iff d(u) < d(v), ties by label (Notation section). */
static int og_before(const og_graph* g, int64_t u, int64_t v) {
    int64_t du = g->ptr[u + 1] - g->ptr[u], dv = g->ptr[v + 1] - g->ptr[v];
    return du < dv || (du == dv && u < v);
}

static int64_t og_find(const og_graph* g, int64_t row, int32_t x) {
    int64_t lo = g->ptr[row], hi = g->ptr[row + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->adj[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < g->ptr[row + 1] && g->adj[lo] == x) ? lo : -1;
}

/* Same T as og_edge_triangles.  For every v and u ∈ N_H(v), every common
 * w ∈ N_H(v) ∩ N_H(u) closes the triangle {v, u, w} whose lowest-ordered
 * vertex is v; each such triangle is met exactly once and adds one to
 * t(v,u), t(v,w), t(u,w) and their mirror entries.  Returns 0, or -2 on
 * allocation failure. */
int og_fast_edge_triangles(const og_graph* g, uint64_t* t) {
    int64_t n = g->n, e2 = 2 * g->m;
    memset(t, 0, sizeof(uint64_t) * (size_t)(e2 ? e2 : 1));
    /* hp: positions p (in the symmetric CSR) of the higher neighbours of
     * each v, in ascending label order. */
    int64_t* hptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* hp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->m + 1));
    if (!hptr || !hp) { free(hptr); free(hp); return -2; }
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        hptr[v] = k;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p)
            if (og_before(g, v, g->adj[p])) hp[k++] = p;
    }
    hptr[n] = k;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t a = hptr[v]; a < hptr[v + 1]; ++a) {
            int64_t puv = hp[a];
            int32_t u = g->adj[puv];
            int64_t i = hptr[v], j = hptr[u];
            while (i < hptr[v + 1] && j < hptr[u + 1]) {
                int32_t wi = g->adj[hp[i]], wj = g->adj[hp[j]];
                if (wi < wj) ++i;
                else if (wi > wj) ++j;
                else {
                    t[puv] += 1;        /* edge {v,u} */
                    t[hp[i]] += 1;      /* edge {v,w} */
                    t[hp[j]] += 1;      /* edge {u,w} */
                    ++i; ++j;
                }
            }
        }
    }
    /* mirror each entry (v,u) with v before u onto (u,v) */
    for (int64_t v = 0; v < n; ++v)
        for (int64_t a = hptr[v]; a < hptr[v + 1]; ++a) {
            int64_t p = hp[a];
            int64_t q = og_find(g, g->adj[p], (int32_t)v);
            if (q < 0) { free(hptr); free(hp); return -1; }
            t[q] = t[p];
        }
    free(hptr);
    free(hp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sampled evaluation of the definition at chosen vertices.             */
/* ------------------------------------------------------------------ */

/* △(x) by the marker test: mark N(x), then Σ_{u∈N(x)} |{w ∈ N(u) : marked}|
 * counts each triangle at x twice. `mark` is an all-zero byte array of size
 * n and is left all-zero. */
static uint64_t og_tri_marked(const og_graph* g, int64_t x, uint8_t* mark) {
    for (int64_t p = g->ptr[x]; p < g->ptr[x + 1]; ++p) mark[g->adj[p]] = 1;
    uint64_t s = 0;
    for (int64_t p = g->ptr[x]; p < g->ptr[x + 1]; ++p) {
        int32_t u = g->adj[p];
        for (int64_t q = g->ptr[u]; q < g->ptr[u + 1]; ++q) s += mark[g->adj[q]];
    }
    for (int64_t p = g->ptr[x]; p < g->ptr[x + 1]; ++p) mark[g->adj[p]] = 0;
    return s / 2;
}

/* For each sampled vertex v = vs[i]: tri_out[i] = △(v), numer_out[i] =
 * numerator of Definition 1 times 3△(G).  If row_t is non-NULL, row_t gets,
 * for every adjacency entry of every sampled vertex (rows concatenated in
 * sample order), t(v,u) = |N(v) ∩ N(u)|.  Returns 0, -1 on a bad vertex id,
 * -2 on allocation failure. */
int og_sample(const og_graph* g, const int64_t* vs, int64_t k,
              uint64_t* tri_out, uint64_t* numer_out, uint64_t* row_t) {
    int64_t n = g->n;
    uint8_t* mark = (uint8_t*)calloc((size_t)n + 1, 1);
    uint64_t* cache = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    if (!mark || !cache) { free(mark); free(cache); return -2; }
    for (int64_t i = 0; i < n; ++i) cache[i] = UINT64_MAX;
    int64_t out = 0;
    for (int64_t s = 0; s < k; ++s) {
        int64_t v = vs[s];
        if (v < 0 || v >= n) { free(mark); free(cache); return -1; }
        if (cache[v] == UINT64_MAX) cache[v] = og_tri_marked(g, v, mark);
        uint64_t x = cache[v], y = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) mark[g->adj[p]] = 1;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) {
            int32_t u = g->adj[p];
            uint64_t common = 0;
            for (int64_t q = g->ptr[u]; q < g->ptr[u + 1]; ++q) common += mark[g->adj[q]];
            if (row_t) row_t[out++] = common;
            if (cache[u] == UINT64_MAX) {
                /* og_tri_marked needs a clean marker array */
                for (int64_t q = g->ptr[v]; q < g->ptr[v + 1]; ++q) mark[g->adj[q]] = 0;
                cache[u] = og_tri_marked(g, u, mark);
                for (int64_t q = g->ptr[v]; q < g->ptr[v + 1]; ++q) mark[g->adj[q]] = 1;
            }
            if (common > 0) x += cache[u]; else y += cache[u];
        }
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) mark[g->adj[p]] = 0;
        tri_out[s] = cache[v];
        numer_out[s] = x + 3 * y;
    }
    free(mark);
    free(cache);
    return 0;
}

/* The cheap half of og_sample, for graphs whose hubs make the numerator
 * too costly to sample: tri_out[i] = △(vs[i]) by the marker test, and
 * row_t (rows of the sampled vertices concatenated in sample order)
 * t(v,u) = |N(v) ∩ N(u)| for every u in N(v) (section "Notation": the
 * entries of T = A² ∘ A in row v).  Cost per vertex: Σ_{u∈N(v)} d(u).
 * Returns 0, -1 on a bad vertex id, -2 on allocation failure. */
int og_sample_tri(const og_graph* g, const int64_t* vs, int64_t k, uint64_t* tri_out, uint64_t* row_t) {
    int64_t n = g->n;
    uint8_t* mark = (uint8_t*)calloc((size_t)n + 1, 1);
    if (!mark) return -2;
    int64_t out = 0;
    for (int64_t s = 0; s < k; ++s) {
        int64_t v = vs[s];
        if (v < 0 || v >= n) { free(mark); return -1; }
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) mark[g->adj[p]] = 1;
        uint64_t twice = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) {
            int32_t u = g->adj[p];
            uint64_t common = 0;
            for (int64_t q = g->ptr[u]; q < g->ptr[u + 1]; ++q) common += mark[g->adj[q]];
            if (row_t) row_t[out++] = common;
            twice += common;
        }
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) mark[g->adj[p]] = 0;
        tri_out[s] = twice / 2;
    }
    free(mark);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Correctly rounded quotient.                                          */
/* ------------------------------------------------------------------ */

static int og_bitlen(unsigned __int128 x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

/* a / b rounded to nearest binary64, ties to even, by restoring long
 * division: integer part, then one quotient bit per step until 54
 * significant bits (53 kept + 1 rounding bit) are known; the remainder
 * gives the sticky bit.  b == 0 gives NaN. */
double og_div_rn_long(uint64_t a, uint64_t b) {
    if (b == 0) return NAN;
    if (a == 0) return 0.0;
    unsigned __int128 q = a / b;
    unsigned __int128 r = a % b;
    int exp2 = 0;                       /* value = q * 2^exp2 (+ remainder) */
    int sticky = 0;
    while (og_bitlen(q) < 54) {
        r <<= 1;
        q <<= 1;
        if (r >= b) { r -= b; q |= 1; }
        exp2 -= 1;
    }
    while (og_bitlen(q) > 54) {          /* only when a/b >= 2^54 */
        sticky |= (int)(q & 1);
        q >>= 1;
        exp2 += 1;
    }
    if (r != 0) sticky = 1;
    int round_bit = (int)(q & 1);
    q >>= 1;
    exp2 += 1;
    if (round_bit && (sticky || (q & 1))) q += 1;
    return ldexp((double)(uint64_t)q, exp2);
}

/* Exact operands below 2^53 make one IEEE division the correctly rounded
 * quotient; otherwise use the long division. */
double og_div_rn(uint64_t a, uint64_t b) {
    const uint64_t lim = (uint64_t)1 << 53;
    if (b == 0) return NAN;
    if (a < lim && b < lim) return (double)a / (double)b;
    return og_div_rn_long(a, b);
}

void og_tc(const uint64_t* numer, int64_t n, uint64_t den, double* out) {
    for (int64_t v = 0; v < n; ++v) out[v] = og_div_rn(numer[v], den);
}

/* ------------------------------------------------------------------ */
/* The same routines spread over host threads (CPU timing baseline).    */
/* ------------------------------------------------------------------ */
/* Each *_mt routine below computes exactly what its single-threaded
 * namesake computes: the outer loop over vertices is cut into chunks that
 * POSIX threads take in turn, the work per vertex is the same statements,
 * and where two vertices add into one entry (the three edges of a listed
 * triangle) the addition is atomic.  Integer addition in any order gives
 * the same sum, so the outputs are equal bit for bit (the tests check it).
 * They exist only to time the oracle on all host cores. */
#include <pthread.h>

typedef struct {
    int64_t n, chunk;
    int64_t next;               /* next chunk start (atomic) */
    void* ctx;
    void (*body)(void* ctx, int64_t lo, int64_t hi);
} og_pool;

static void* og_worker(void* arg) {
    og_pool* p = (og_pool*)arg;
    for (;;) {
        int64_t lo = __atomic_fetch_add(&p->next, p->chunk, __ATOMIC_RELAXED);
        if (lo >= p->n) break;
        int64_t hi = lo + p->chunk < p->n ? lo + p->chunk : p->n;
        p->body(p->ctx, lo, hi);
    }
    return NULL;
}

/* body(ctx, lo, hi) over [0, n) in chunks, on `threads` threads (the caller
 * is one of them). */
static void og_parallel(int64_t n, int threads, void* ctx, void (*body)(void*, int64_t, int64_t)) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    og_pool p = {n, 256, 0, ctx, body};
    pthread_t th[256];
    int ok[256];
    for (int k = 1; k < threads; ++k) ok[k] = pthread_create(&th[k], NULL, og_worker, &p) == 0;
    og_worker(&p);
    for (int k = 1; k < threads; ++k)
        if (ok[k]) pthread_join(th[k], NULL);
}

/* og_build with the per-row sort and de-duplication on threads. */
typedef struct {
    int32_t* buf;
    const int64_t* cnt;
    int64_t* len;
    int32_t* adj;
    const int64_t* ptr;
} og_build_ctx;

static void og_build_rows(void* c, int64_t lo, int64_t hi) {
    og_build_ctx* x = (og_build_ctx*)c;
    for (int64_t v = lo; v < hi; ++v) {
        int64_t b = x->cnt[v], e = x->cnt[v + 1], out = b;
        qsort(x->buf + b, (size_t)(e - b), sizeof(int32_t), og_cmp_i32);
        for (int64_t i = b; i < e; ++i)
            if (i == b || x->buf[i] != x->buf[i - 1]) x->buf[out++] = x->buf[i];
        x->len[v] = out - b;
    }
}

static void og_build_copy(void* c, int64_t lo, int64_t hi) {
    og_build_ctx* x = (og_build_ctx*)c;
    for (int64_t v = lo; v < hi; ++v)
        memcpy(x->adj + x->ptr[v], x->buf + x->cnt[v], sizeof(int32_t) * (size_t)(x->ptr[v + 1] - x->ptr[v]));
}

og_graph* og_build_mt(const int32_t* src, const int32_t* dst, int64_t np, int64_t n, int threads) {
    if (n < 0 || np < 0 || n > INT32_MAX) return NULL;
    for (int64_t i = 0; i < np; ++i)
        if (src[i] < 0 || dst[i] < 0 || src[i] >= n || dst[i] >= n) return NULL;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return NULL;
    for (int64_t i = 0; i < np; ++i)
        if (src[i] != dst[i]) { cnt[src[i] + 1] += 1; cnt[dst[i] + 1] += 1; }
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int64_t total = cnt[n];
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* len = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
    if (!buf || !fill || !len || !g) { free(cnt); free(buf); free(fill); free(len); free(g); return NULL; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < np; ++i) {
        if (src[i] == dst[i]) continue;
        buf[fill[src[i]]++] = dst[i];
        buf[fill[dst[i]]++] = src[i];
    }
    free(fill);
    og_build_ctx x = {buf, cnt, len, NULL, NULL};
    og_parallel(n, threads, &x, og_build_rows);
    g->n = n;
    g->ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->ptr) { free(cnt); free(buf); free(len); free(g); return NULL; }
    for (int64_t v = 0; v < n; ++v) g->ptr[v + 1] = g->ptr[v] + len[v];
    g->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->ptr[n] + 1));
    if (!g->adj) { free(cnt); free(buf); free(len); free(g->ptr); free(g); return NULL; }
    x.adj = g->adj;
    x.ptr = g->ptr;
    og_parallel(n, threads, &x, og_build_copy);
    g->m = g->ptr[n] / 2;
    free(cnt);
    free(buf);
    free(len);
    return g;
}

/* og_edge_triangles on threads (every entry is its own merge). */
typedef struct { const og_graph* g; uint64_t* t; } og_t_ctx;

static void og_edge_rows(void* c, int64_t lo, int64_t hi) {
    og_t_ctx* x = (og_t_ctx*)c;
    for (int64_t v = lo; v < hi; ++v)
        for (int64_t p = x->g->ptr[v]; p < x->g->ptr[v + 1]; ++p) x->t[p] = og_common(x->g, v, x->g->adj[p]);
}

void og_edge_triangles_mt(const og_graph* g, uint64_t* t, int threads) {
    og_t_ctx x = {g, t};
    og_parallel(g->n, threads, &x, og_edge_rows);
}

/* og_fast_edge_triangles on threads: the listing from each v in parallel
 * (atomic additions), then the mirror entries in parallel. */
typedef struct {
    const og_graph* g;
    uint64_t* t;
    const int64_t* hptr;
    const int64_t* hp;
    int bad;
} og_fast_ctx;

static void og_fast_list(void* c, int64_t lo, int64_t hi) {
    og_fast_ctx* x = (og_fast_ctx*)c;
    const og_graph* g = x->g;
    const int64_t* hptr = x->hptr;
    const int64_t* hp = x->hp;
    for (int64_t v = lo; v < hi; ++v) {
        for (int64_t a = hptr[v]; a < hptr[v + 1]; ++a) {
            int64_t puv = hp[a];
            int32_t u = g->adj[puv];
            int64_t i = hptr[v], j = hptr[u];
            while (i < hptr[v + 1] && j < hptr[u + 1]) {
                int32_t wi = g->adj[hp[i]], wj = g->adj[hp[j]];
                if (wi < wj) ++i;
                else if (wi > wj) ++j;
                else {
                    __atomic_fetch_add(&x->t[puv], 1, __ATOMIC_RELAXED);    /* edge {v,u} */
                    __atomic_fetch_add(&x->t[hp[i]], 1, __ATOMIC_RELAXED);  /* edge {v,w} */
                    __atomic_fetch_add(&x->t[hp[j]], 1, __ATOMIC_RELAXED);  /* edge {u,w} */
                    ++i; ++j;
                }
            }
        }
    }
}

static void og_fast_mirror(void* c, int64_t lo, int64_t hi) {
    og_fast_ctx* x = (og_fast_ctx*)c;
    for (int64_t v = lo; v < hi; ++v)
        for (int64_t a = x->hptr[v]; a < x->hptr[v + 1]; ++a) {
            int64_t p = x->hp[a];
            int64_t q = og_find(x->g, x->g->adj[p], (int32_t)v);
            if (q < 0) { __atomic_store_n(&x->bad, 1, __ATOMIC_RELAXED); continue; }
            x->t[q] = x->t[p];
        }
}

int og_fast_edge_triangles_mt(const og_graph* g, uint64_t* t, int threads) {
    int64_t n = g->n, e2 = 2 * g->m;
    memset(t, 0, sizeof(uint64_t) * (size_t)(e2 ? e2 : 1));
    int64_t* hptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* hp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->m + 1));
    if (!hptr || !hp) { free(hptr); free(hp); return -2; }
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        hptr[v] = k;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p)
            if (og_before(g, v, g->adj[p])) hp[k++] = p;
    }
    hptr[n] = k;
    og_fast_ctx x = {g, t, hptr, hp, 0};
    og_parallel(n, threads, &x, og_fast_list);
    og_parallel(n, threads, &x, og_fast_mirror);
    free(hptr);
    free(hp);
    return x.bad ? -1 : 0;
}

/* og_vertex_triangles, og_numer_definition and og_tc on threads (each
 * vertex writes only its own entries). */
typedef struct {
    const og_graph* g;
    const uint64_t* t;
    const uint64_t* tri;
    uint64_t* out;
    uint64_t* core;
    uint64_t* noncore;
    int bad;
} og_v_ctx;

static void og_tri_rows(void* c, int64_t lo, int64_t hi) {
    og_v_ctx* x = (og_v_ctx*)c;
    for (int64_t v = lo; v < hi; ++v) {
        uint64_t s = 0;
        for (int64_t p = x->g->ptr[v]; p < x->g->ptr[v + 1]; ++p) s += x->t[p];
        if (s & 1u) __atomic_store_n(&x->bad, 1, __ATOMIC_RELAXED);
        x->out[v] = s / 2;
    }
}

int og_vertex_triangles_mt(const og_graph* g, const uint64_t* t, uint64_t* tri, int threads) {
    og_v_ctx x = {g, t, NULL, tri, NULL, NULL, 0};
    og_parallel(g->n, threads, &x, og_tri_rows);
    return x.bad ? -1 : 0;
}

static void og_numer_rows(void* c, int64_t lo, int64_t hi) {
    og_v_ctx* x = (og_v_ctx*)c;
    const og_graph* g = x->g;
    for (int64_t v = lo; v < hi; ++v) {
        uint64_t cx = x->tri[v], y = 0;
        for (int64_t p = g->ptr[v]; p < g->ptr[v + 1]; ++p) {
            int32_t u = g->adj[p];
            if (x->t[p] > 0) cx += x->tri[u];
            else y += x->tri[u];
        }
        x->out[v] = cx + 3 * y;
        if (x->core) x->core[v] = cx;
        if (x->noncore) x->noncore[v] = y;
    }
}

void og_numer_definition_mt(const og_graph* g, const uint64_t* t, const uint64_t* tri, uint64_t* numer,
                            uint64_t* core, uint64_t* noncore, int threads) {
    og_v_ctx x = {g, t, tri, numer, core, noncore, 0};
    og_parallel(g->n, threads, &x, og_numer_rows);
}

typedef struct { const uint64_t* numer; uint64_t den; double* out; } og_tc_ctx;

static void og_tc_rows(void* c, int64_t lo, int64_t hi) {
    og_tc_ctx* x = (og_tc_ctx*)c;
    for (int64_t v = lo; v < hi; ++v) x->out[v] = og_div_rn(x->numer[v], x->den);
}

void og_tc_mt(const uint64_t* numer, int64_t n, uint64_t den, double* out, int threads) {
    og_tc_ctx x = {numer, den, out};
    og_parallel(n, threads, &x, og_tc_rows);
}
