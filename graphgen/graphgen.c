/*
 * Seeded synthetic graph generators shared by the CUDA path and the oracle.
 *
 * This file holds no triangle-centrality arithmetic: it only draws edge
 * lists.  Every random choice comes from a counter-based hash of
 * (seed, stream, counter) built on the splitmix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so
 * the output is a pure function of the arguments and does not depend on the
 * number of threads.
 *
 * Vertex ids are 0-based int32 values in [0, n).  Self-loops and duplicate
 * pairs are emitted as drawn; removing them is the consumer's job (the
 * triangle-centrality input is a simple undirected graph, built by
 * symmetrising and de-duplicating the drawn pairs).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based draw: a 64-bit value determined by (seed, stream, ctr). */
uint64_t gg_hash(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t s = gg_mix(seed + GG_GOLDEN * (stream + 1));
    return gg_mix(s + GG_GOLDEN * (ctr + 1));
}

/* Uniform integer in [0, bound) (bound >= 1); 64-bit modulo, bias < 2^-32
 * for every bound used here. */
static inline uint64_t gg_below(uint64_t seed, uint64_t stream, uint64_t ctr,
                                uint64_t bound) {
    return gg_hash(seed, stream, ctr) % bound;
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double gg_unit(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return (double)(gg_hash(seed, stream, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

enum { ST_RMAT = 1, ST_PERM = 2, ST_DIAG = 3, ST_CL_PERM = 4, ST_CL_EDGE = 5,
       ST_BA = 6, ST_HIER = 7, ST_NOISE = 8 };

/* ------------------------------------------------------------------ */
/* Random permutation of [0, n) by Fisher-Yates with seeded draws.     */
/* ------------------------------------------------------------------ */
int gg_permutation(uint64_t seed, uint64_t stream, int64_t n, int32_t* perm) {
    if (n < 0 || n > INT32_MAX) return -1;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)gg_below(seed, stream, (uint64_t)i, (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Thread helper                                                        */
/* ------------------------------------------------------------------ */
typedef void (*gg_range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { gg_range_fn fn; void* ctx; int64_t lo, hi; } gg_task;

static void* gg_task_main(void* p) {
    gg_task* t = (gg_task*)p;
    t->fn(t->ctx, t->lo, t->hi);
    return NULL;
}

static void gg_parallel(int64_t count, int threads, gg_range_fn fn, void* ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (count < 65536 || threads == 1) { fn(ctx, 0, count); return; }
    pthread_t th[256];
    gg_task tk[256];
    int64_t chunk = (count + threads - 1) / threads;
    int started = 0;
    for (int i = 0; i < threads; ++i) {
        int64_t lo = i * chunk, hi = lo + chunk < count ? lo + chunk : count;
        if (lo >= hi) break;
        tk[i].fn = fn; tk[i].ctx = ctx; tk[i].lo = lo; tk[i].hi = hi;
        if (pthread_create(&th[i], NULL, gg_task_main, &tk[i]) != 0) {
            fn(ctx, lo, hi);
            tk[i].fn = NULL;
        }
        started = i + 1;
    }
    for (int i = 0; i < started; ++i)
        if (tk[i].fn) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004)                            */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t seed; int scale; uint32_t ta, tab, tabc;
    int32_t* src; int32_t* dst; const int32_t* perm;
} rmat_ctx;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
    rmat_ctx* c = (rmat_ctx*)p;
    const int half = (c->scale + 1) / 2;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t s = 0, d = 0;
        for (int k = 0; k < half; ++k) {
            uint64_t h = gg_hash(c->seed, ST_RMAT, (uint64_t)i * (uint64_t)half + (uint64_t)k);
            for (int part = 0; part < 2; ++part) {
                int level = 2 * k + part;
                if (level >= c->scale) break;
                uint32_t u = part ? (uint32_t)(h >> 32) : (uint32_t)h;
                uint32_t sb, db;
                if (u < c->ta) { sb = 0; db = 0; }
                else if (u < c->tab) { sb = 0; db = 1; }
                else if (u < c->tabc) { sb = 1; db = 0; }
                else { sb = 1; db = 1; }
                s = (s << 1) | sb;
                d = (d << 1) | db;
            }
        }
        if (c->perm) { s = (uint32_t)c->perm[s]; d = (uint32_t)c->perm[d]; }
        c->src[i] = (int32_t)s;
        c->dst[i] = (int32_t)d;
    }
}

static uint32_t gg_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return (uint32_t)(p * 4294967296.0);
}

/*
 * Draw `samples` R-MAT pairs over n = 2^scale vertices with quadrant
 * probabilities (a, b, c, 1-a-b-c): a -> (0,0), b -> (0,1), c -> (1,0),
 * d -> (1,1), one level per bit from the most significant.  Each level uses
 * 32 random bits compared with fixed-point thresholds, so the draw is exact
 * integer work.  If `permute` is non-zero the vertex labels are then passed
 * through a seeded random permutation (breaks the id/degree correlation).
 */
int gg_rmat(uint64_t seed, int scale, int64_t samples, double a, double b, double c,
            int permute, int threads, int32_t* src, int32_t* dst) {
    if (scale < 1 || scale > 30 || samples < 0) return -1;
    rmat_ctx ctx;
    ctx.seed = seed; ctx.scale = scale;
    ctx.ta = gg_threshold(a);
    ctx.tab = gg_threshold(a + b);
    ctx.tabc = gg_threshold(a + b + c);
    ctx.src = src; ctx.dst = dst; ctx.perm = NULL;
    int32_t* perm = NULL;
    if (permute) {
        int64_t n = (int64_t)1 << scale;
        perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return -2;
        gg_permutation(seed, ST_PERM, n, perm);
        ctx.perm = perm;
    }
    gg_parallel(samples, threads, rmat_range, &ctx);
    free(perm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid + diagonals + Chung-Lu overlay                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t seed; int64_t pairs; const double* cdf; int64_t n;
    const int32_t* perm; int32_t* src; int32_t* dst;
} cl_ctx;

static int64_t cl_pick(const double* cdf, int64_t n, double x) {
    int64_t lo = 0, hi = n - 1;             /* first i with cdf[i] > x */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void cl_range(void* p, int64_t lo, int64_t hi) {
    cl_ctx* c = (cl_ctx*)p;
    double total = c->cdf[c->n - 1];
    for (int64_t i = lo; i < hi; ++i) {
        double x = gg_unit(c->seed, ST_CL_EDGE, 2 * (uint64_t)i) * total;
        double y = gg_unit(c->seed, ST_CL_EDGE, 2 * (uint64_t)i + 1) * total;
        c->src[i] = c->perm[cl_pick(c->cdf, c->n, x)];
        c->dst[i] = c->perm[cl_pick(c->cdf, c->n, y)];
    }
}

/*
 * side x side 4-neighbour grid (vertex (i,j) -> id i*side+j), plus the
 * diagonal (i,j)-(i+1,j+1) of each cell with probability pdiag, plus a
 * Chung-Lu overlay: vertex weights w = (k+1)^(-1/(gamma-1)) assigned to a
 * seeded random permutation of the vertices, side*side*mean_deg/2 pairs
 * whose two endpoints are drawn independently with probability
 * proportional to w.  Returns the number of pairs written (<= cap) or a
 * negative error.  Pass src = dst = NULL to get the exact count.
 */
int64_t gg_grid_cl(uint64_t seed, int64_t side, double pdiag, double gamma,
                   double mean_deg, int threads, int64_t cap,
                   int32_t* src, int32_t* dst) {
    if (side < 2) return -1;
    int64_t n = side * side;
    if (n > INT32_MAX) return -1;
    int64_t grid = 2 * side * (side - 1);
    int64_t ndiag = 0;
    uint32_t td = gg_threshold(pdiag);
    for (int64_t i = 0; i + 1 < side; ++i)
        for (int64_t j = 0; j + 1 < side; ++j)
            if ((uint32_t)gg_hash(seed, ST_DIAG, (uint64_t)(i * side + j)) < td) ++ndiag;
    int64_t ncl = (int64_t)((double)n * mean_deg / 2.0);
    int64_t total = grid + ndiag + ncl;
    if (!src || !dst) return total;
    if (cap < total) return -3;
    int64_t k = 0;
    for (int64_t i = 0; i < side; ++i)
        for (int64_t j = 0; j < side; ++j) {
            int64_t v = i * side + j;
            if (j + 1 < side) { src[k] = (int32_t)v; dst[k] = (int32_t)(v + 1); ++k; }
            if (i + 1 < side) { src[k] = (int32_t)v; dst[k] = (int32_t)(v + side); ++k; }
        }
    for (int64_t i = 0; i + 1 < side; ++i)
        for (int64_t j = 0; j + 1 < side; ++j)
            if ((uint32_t)gg_hash(seed, ST_DIAG, (uint64_t)(i * side + j)) < td) {
                src[k] = (int32_t)(i * side + j);
                dst[k] = (int32_t)((i + 1) * side + j + 1);
                ++k;
            }
    double* cdf = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!cdf || !perm) { free(cdf); free(perm); return -2; }
    double expo = -1.0 / (gamma - 1.0), acc = 0.0;
    for (int64_t v = 0; v < n; ++v) { acc += pow((double)(v + 1), expo); cdf[v] = acc; }
    gg_permutation(seed, ST_CL_PERM, n, perm);
    cl_ctx ctx = { seed, ncl, cdf, n, perm, src + k, dst + k };
    gg_parallel(ncl, threads, cl_range, &ctx);
    free(cdf);
    free(perm);
    return total;
}

/* ------------------------------------------------------------------ */
/* Barabasi-Albert preferential attachment                              */
/* ------------------------------------------------------------------ */
/*
 * n vertices, each new vertex v >= m0 attaches to `mm` targets drawn
 * proportionally to degree (uniform pick from the list of edge endpoints so
 * far; repeated targets are kept and vanish in de-duplication).  The first
 * mm+1 vertices form a clique seed.  Writes exactly gg_ba_count(n, mm)
 * pairs.
 */
int64_t gg_ba_count(int64_t n, int64_t mm) {
    if (n < mm + 1) return -1;
    return (mm + 1) * mm / 2 + (n - mm - 1) * mm;
}

int64_t gg_ba(uint64_t seed, int64_t n, int64_t mm, int32_t* src, int32_t* dst) {
    int64_t total = gg_ba_count(n, mm);
    if (total < 0 || n > INT32_MAX) return -1;
    int32_t* ends = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * total));
    if (!ends) return -2;
    int64_t k = 0, ne = 0;
    for (int64_t a = 0; a <= mm; ++a)
        for (int64_t b = a + 1; b <= mm; ++b) {
            src[k] = (int32_t)a; dst[k] = (int32_t)b; ++k;
            ends[ne++] = (int32_t)a; ends[ne++] = (int32_t)b;
        }
    for (int64_t v = mm + 1; v < n; ++v) {
        int64_t base = ne;
        for (int64_t j = 0; j < mm; ++j) {
            int64_t pick = (int64_t)gg_below(seed, ST_BA, (uint64_t)(v * mm + j), (uint64_t)base);
            int32_t t = ends[pick];
            src[k] = (int32_t)v; dst[k] = t; ++k;
            ends[ne++] = (int32_t)v; ends[ne++] = t;
        }
    }
    free(ends);
    return k;
}

/* ------------------------------------------------------------------ */
/* Planted hierarchy                                                    */
/* ------------------------------------------------------------------ */
/*
 * A root (vertex 0) joined to one member of each of `cliques` cliques of
 * size k, the clique members occupying ids 1 .. cliques*k; every remaining
 * vertex up to n-1 hangs as a leaf off a uniformly chosen clique member;
 * then every vertex, with probability pnoise, gets one extra edge to a
 * uniform random vertex.  Returns the number of pairs written, or the
 * upper bound if src == NULL.
 */
int64_t gg_hierarchy(uint64_t seed, int64_t n, int64_t cliques, int64_t k,
                     double pnoise, int32_t* src, int32_t* dst) {
    if (cliques < 1 || k < 2 || n < 1 + cliques * k || n > INT32_MAX) return -1;
    int64_t members = cliques * k;
    int64_t bound = cliques + cliques * k * (k - 1) / 2 + (n - 1 - members) + n;
    if (!src || !dst) return bound;
    int64_t e = 0;
    uint32_t tn = gg_threshold(pnoise);
    for (int64_t c = 0; c < cliques; ++c) {
        int64_t base = 1 + c * k;
        src[e] = 0; dst[e] = (int32_t)(base + (int64_t)gg_below(seed, ST_HIER, (uint64_t)c, (uint64_t)k)); ++e;
        for (int64_t a = 0; a < k; ++a)
            for (int64_t b = a + 1; b < k; ++b) {
                src[e] = (int32_t)(base + a); dst[e] = (int32_t)(base + b); ++e;
            }
    }
    for (int64_t v = 1 + members; v < n; ++v) {
        src[e] = (int32_t)v;
        dst[e] = (int32_t)(1 + (int64_t)gg_below(seed, ST_HIER, (uint64_t)(cliques + v), (uint64_t)members));
        ++e;
    }
    for (int64_t v = 0; v < n; ++v) {
        uint64_t h = gg_hash(seed, ST_NOISE, 2 * (uint64_t)v);
        if ((uint32_t)h < tn) {
            src[e] = (int32_t)v;
            dst[e] = (int32_t)gg_below(seed, ST_NOISE, 2 * (uint64_t)v + 1, (uint64_t)n);
            ++e;
        }
    }
    return e;
}
