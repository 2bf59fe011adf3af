/*
 * graphgen.c -- seeded synthetic graph generators (input plumbing only).
 *
 * This file builds the symmetric CSR graphs that both the CPU oracle and the
 * CUDA path consume.  It holds none of the connected-components arithmetic:
 * it only draws edges, symmetrises them, removes self-loops and duplicates,
 * and writes CSR arrays.
 *
 * Random numbers come from one counter-based generator built on the
 * SplitMix64 output function (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): word `idx` of stream
 * `stream` under key `seed` is
 *     mix(mix(seed * PHI + stream) + (idx + 1) * PHI),   PHI = 0x9E3779B97F4A7C15
 * where mix is the SplitMix64 finaliser.  Every draw is a pure function of
 * (seed, stream, idx), so generation is order-independent, parallel and
 * identical on x86_64 and aarch64 (integer arithmetic only; the few floating
 * point steps use basic IEEE operations compiled with -ffp-contract=off).
 *
 * Graph families (the workloads the FastSV paper evaluates on, Section 5 /
 * Table 1, are real graphs that are not available here; these stand in):
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with a/b/c/d quadrant
 *     probabilities, no noise, optional Fisher-Yates vertex relabelling;
 *   - a 2-D lattice with independent edge retention (near percolation) plus
 *     appended isolated vertices;
 *   - batches of Erdos-Renyi G(n, M) graphs with log-uniform sizes.
 *
 * All CSR outputs: row_ptr int64 (n+1), col_idx int32, rows sorted ascending,
 * no self-loops, no duplicates, symmetric.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PHI 0x9E3779B97F4A7C15ULL

enum {
    STREAM_RMAT = 1,
    STREAM_PERM = 2,
    STREAM_GRID_RIGHT = 3,
    STREAM_GRID_DOWN = 4,
    STREAM_ER_PARAM = 5,
    STREAM_ER_EDGE = 6,
    STREAM_TRACE = 7,
};

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t gg_word(uint64_t seed, uint64_t stream, uint64_t idx) {
    uint64_t key = sm64_mix(seed * PHI + stream);
    return sm64_mix(key + (idx + 1) * PHI);
}

/* uniform in [0, bound) by multiply-shift on 32 random bits (Lemire 2019). */
static inline uint32_t gg_bounded32(uint32_t r, uint32_t bound) {
    return (uint32_t)(((uint64_t)r * (uint64_t)bound) >> 32);
}

/* uniform in [0, bound) for 64-bit bounds, 128-bit multiply-shift. */
static inline uint64_t gg_bounded64(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)bound) >> 64);
}

/* uniform double in [0, 1) from the top 53 bits. */
static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* exp and log from basic IEEE operations only, so that both host
 * architectures produce the same bits (libm implementations may differ in
 * the last place).  exp: x = k ln2 + r, |r| <= ln2/2, Taylor series of e^r to
 * 24 terms.  log: m * 2^e with m in [1,2), atanh series for log(m). */
static const double GG_LN2 = 0.69314718055994530942;
static double gg_exp(double x) {
    double kf = x / GG_LN2;
    long k = (long)(kf >= 0 ? kf + 0.5 : kf - 0.5);
    double r = x - (double)k * GG_LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 24; ++i) {
        term = term * r / (double)i;
        sum = sum + term;
    }
    while (k > 0) { sum = sum * 2.0; --k; }
    while (k < 0) { sum = sum * 0.5; ++k; }
    return sum;
}
static double gg_log(double x) {
    if (x <= 0) return -1e300;
    int e = 0;
    while (x >= 2.0) { x = x * 0.5; ++e; }
    while (x < 1.0) { x = x * 2.0; --e; }
    double t = (x - 1.0) / (x + 1.0), t2 = t * t, term = t, sum = 0.0;
    for (int i = 1; i < 80; i += 2) {
        sum = sum + term / (double)i;
        term = term * t2;
    }
    return 2.0 * sum + (double)e * GG_LN2;
}
static int64_t gg_round(double x) { return (int64_t)(x + 0.5); }

double graphgen_exp(double x) { return gg_exp(x); }
double graphgen_log(double x) { return gg_log(x); }
uint64_t graphgen_word(uint64_t seed, uint64_t stream, uint64_t idx) { return gg_word(seed, stream, idx); }

/* ------------------------------------------------------------------ */
/* helpers: per-row sort + unique, compaction                          */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int64_t sort_unique(int32_t* a, int64_t len) {
    if (len <= 1) return len;
    if (len <= 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t v = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
            a[j + 1] = v;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
    int64_t w = 1;
    for (int64_t i = 1; i < len; ++i)
        if (a[i] != a[w - 1]) a[w++] = a[i];
    return w;
}

/* rows [0,n) live at col[rp_raw[u] .. rp_raw[u] + len[u]); pack them densely
 * in place (new offsets never exceed old ones) and write rp_out (n+1). */
static void compact_rows(int64_t n, const int64_t* rp_raw, const int64_t* len, int32_t* col, int64_t* rp_out) {
    int64_t w = 0;
    for (int64_t u = 0; u < n; ++u) {
        rp_out[u] = w;
        int64_t l = len[u];
        if (w != rp_raw[u] && l > 0) memmove(col + w, col + rp_raw[u], (size_t)l * sizeof(int32_t));
        w += l;
    }
    rp_out[n] = w;
}

/* ------------------------------------------------------------------ */
/* Fisher-Yates permutation                                            */
/* ------------------------------------------------------------------ */

void graphgen_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t j = gg_bounded64(gg_word(seed, STREAM_PERM, (uint64_t)i), (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* ------------------------------------------------------------------ */
/* R-MAT                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int scale;
    uint32_t ta, tab, tabc; /* cumulative quadrant thresholds on 32-bit uniforms */
    uint64_t seed;
    const int32_t* perm; /* NULL = identity */
} rmat_t;

static void rmat_init(rmat_t* r, int scale, double a, double b, double c, uint64_t seed, const int32_t* perm) {
    r->scale = scale;
    r->ta = (uint32_t)(a * 4294967296.0);
    r->tab = (uint32_t)((a + b) * 4294967296.0);
    r->tabc = (uint32_t)((a + b + c) * 4294967296.0);
    r->seed = seed;
    r->perm = perm;
}

/* draw i: level l (most significant bit first) takes 32 random bits from
 * word i*16 + l/2 (high half for even l, low half for odd l). */
static inline void rmat_draw(const rmat_t* r, uint64_t i, int32_t* pu, int32_t* pv) {
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int l = 0; l < r->scale; ++l) {
        uint32_t x;
        if ((l & 1) == 0) {
            w = gg_word(r->seed, STREAM_RMAT, i * 16 + (uint64_t)(l >> 1));
            x = (uint32_t)(w >> 32);
        } else {
            x = (uint32_t)w;
        }
        uint32_t bit = 1u << (r->scale - 1 - l);
        if (x < r->ta) {
        } else if (x < r->tab) {
            v |= bit;
        } else if (x < r->tabc) {
            u |= bit;
        } else {
            u |= bit;
            v |= bit;
        }
    }
    if (r->perm) {
        u = (uint32_t)r->perm[u];
        v = (uint32_t)r->perm[v];
    }
    *pu = (int32_t)u;
    *pv = (int32_t)v;
}

/* Pass 1: raw degrees (both directions, self-loops dropped, duplicates kept).
 * deg must hold n = 2^scale zeroed entries. Returns the raw entry count. */
int64_t graphgen_rmat_degrees(int scale, int64_t draws, double a, double b, double c, uint64_t seed,
                              const int32_t* perm, int64_t* deg) {
    rmat_t r;
    rmat_init(&r, scale, a, b, c, seed, perm);
    int64_t total = 0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t i = 0; i < draws; ++i) {
        int32_t u, v;
        rmat_draw(&r, (uint64_t)i, &u, &v);
        if (u == v) continue;
        __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
        total += 2;
    }
    return total;
}

/* Pass 2: scatter both directions into col (sized by the raw offsets
 * rp_raw, n+1 entries), then sort + unique every row and pack.  cursor is
 * scratch of n int64.  Writes the final rp (n+1); returns m. */
int64_t graphgen_rmat_fill(int scale, int64_t draws, double a, double b, double c, uint64_t seed,
                           const int32_t* perm, const int64_t* rp_raw, int64_t* cursor, int32_t* col,
                           int64_t* rp_out) {
    rmat_t r;
    rmat_init(&r, scale, a, b, c, seed, perm);
    int64_t n = (int64_t)1 << scale;
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) cursor[u] = rp_raw[u];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < draws; ++i) {
        int32_t u, v;
        rmat_draw(&r, (uint64_t)i, &u, &v);
        if (u == v) continue;
        int64_t pu = __atomic_fetch_add(&cursor[u], 1, __ATOMIC_RELAXED);
        int64_t pv = __atomic_fetch_add(&cursor[v], 1, __ATOMIC_RELAXED);
        col[pu] = v;
        col[pv] = u;
    }
    /* cursor now reused as per-row unique length */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; ++u) cursor[u] = sort_unique(col + rp_raw[u], rp_raw[u + 1] - rp_raw[u]);
    compact_rows(n, rp_raw, cursor, col, rp_out);
    return rp_out[n];
}

/* ------------------------------------------------------------------ */
/* 2-D lattice with edge retention + appended isolated vertices         */
/* ------------------------------------------------------------------ */

static inline int grid_keep(uint64_t seed, int stream, int64_t idx, uint32_t thr) {
    return (uint32_t)(gg_word(seed, (uint64_t)stream, (uint64_t)idx) >> 32) < thr;
}

/* vertex id = row * side + col for the lattice; ids side*side .. +extra-1
 * are isolated.  The right edge of (r,c) is kept iff word(seed, RIGHT, id)
 * falls under thr = floor(p * 2^32); the down edge likewise on stream DOWN.
 * rp must hold n+1 entries; if col is NULL only rp is written. Returns m. */
int64_t graphgen_grid(int64_t side, int64_t extra, double p, uint64_t seed, int64_t* rp, int32_t* col) {
    uint32_t thr = p >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(p * 4294967296.0);
    int all = p >= 1.0;
    int64_t nl = side * side, n = nl + extra;
    /* degrees */
#pragma omp parallel for schedule(static)
    for (int64_t id = 0; id < nl; ++id) {
        int64_t r = id / side, c = id % side, d = 0;
        if (r > 0 && (all || grid_keep(seed, STREAM_GRID_DOWN, id - side, thr))) ++d;
        if (c > 0 && (all || grid_keep(seed, STREAM_GRID_RIGHT, id - 1, thr))) ++d;
        if (c + 1 < side && (all || grid_keep(seed, STREAM_GRID_RIGHT, id, thr))) ++d;
        if (r + 1 < side && (all || grid_keep(seed, STREAM_GRID_DOWN, id, thr))) ++d;
        rp[id + 1] = d;
    }
    rp[0] = 0;
    for (int64_t id = 0; id < nl; ++id) rp[id + 1] += rp[id];
    for (int64_t id = nl; id < n; ++id) rp[id + 1] = rp[id];
    if (!col) return rp[n];
#pragma omp parallel for schedule(static)
    for (int64_t id = 0; id < nl; ++id) {
        int64_t r = id / side, c = id % side, w = rp[id];
        if (r > 0 && (all || grid_keep(seed, STREAM_GRID_DOWN, id - side, thr))) col[w++] = (int32_t)(id - side);
        if (c > 0 && (all || grid_keep(seed, STREAM_GRID_RIGHT, id - 1, thr))) col[w++] = (int32_t)(id - 1);
        if (c + 1 < side && (all || grid_keep(seed, STREAM_GRID_RIGHT, id, thr))) col[w++] = (int32_t)(id + 1);
        if (r + 1 < side && (all || grid_keep(seed, STREAM_GRID_DOWN, id, thr))) col[w++] = (int32_t)(id + side);
    }
    return rp[n];
}

/* ------------------------------------------------------------------ */
/* Batches of Erdos-Renyi G(n, M) graphs                                */
/* ------------------------------------------------------------------ */

/* Graph g: n_g = round(exp(U(ln nmin, ln nmax))), d_g = U(dmin, dmax) directed
 * entries per vertex, M_g = round(n_g d_g / 2) uniform pair draws. */
void graphgen_er_params(int64_t G, uint64_t seed, double nmin, double nmax, double dmin, double dmax, int64_t* n_out,
                        int64_t* draws_out) {
    double l0 = gg_log(nmin), l1 = gg_log(nmax);
    for (int64_t g = 0; g < G; ++g) {
        double u1 = gg_unit(gg_word(seed, STREAM_ER_PARAM, (uint64_t)(2 * g)));
        double u2 = gg_unit(gg_word(seed, STREAM_ER_PARAM, (uint64_t)(2 * g + 1)));
        int64_t ng = gg_round(gg_exp(l0 + u1 * (l1 - l0)));
        if (ng < 1) ng = 1;
        double d = dmin + u2 * (dmax - dmin);
        n_out[g] = ng;
        draws_out[g] = gg_round((double)ng * d * 0.5);
    }
}

/* Fill graph g of the batch.  Raw storage: col_raw[eoff_raw .. + 2*draws),
 * rp scratch of n_g+1 int64 (rp_tmp) and len scratch of n_g int64.
 * Output: local rows packed at the start of the raw region, local row_ptr
 * (int32, n_g+1 entries, starting at 0) into rp_out. Returns m_g. */
static int64_t er_fill_one(int64_t g, uint64_t seed, int64_t ng, int64_t draws, int32_t* col, int64_t* rp_tmp,
                           int64_t* len, int32_t* rp_out) {
    memset(rp_tmp, 0, (size_t)(ng + 1) * sizeof(int64_t));
    uint64_t base = (uint64_t)g << 34;
    for (int64_t j = 0; j < draws; ++j) {
        uint64_t w = gg_word(seed, STREAM_ER_EDGE, base + (uint64_t)j);
        uint32_t u = gg_bounded32((uint32_t)(w >> 32), (uint32_t)ng);
        uint32_t v = gg_bounded32((uint32_t)w, (uint32_t)ng);
        if (u == v) continue;
        rp_tmp[u + 1]++;
        rp_tmp[v + 1]++;
    }
    for (int64_t u = 0; u < ng; ++u) rp_tmp[u + 1] += rp_tmp[u];
    for (int64_t u = 0; u < ng; ++u) len[u] = rp_tmp[u];
    for (int64_t j = 0; j < draws; ++j) {
        uint64_t w = gg_word(seed, STREAM_ER_EDGE, base + (uint64_t)j);
        uint32_t u = gg_bounded32((uint32_t)(w >> 32), (uint32_t)ng);
        uint32_t v = gg_bounded32((uint32_t)w, (uint32_t)ng);
        if (u == v) continue;
        col[len[u]++] = (int32_t)v;
        col[len[v]++] = (int32_t)u;
    }
    for (int64_t u = 0; u < ng; ++u) len[u] = sort_unique(col + rp_tmp[u], rp_tmp[u + 1] - rp_tmp[u]);
    int64_t w = 0;
    for (int64_t u = 0; u < ng; ++u) {
        rp_out[u] = (int32_t)w;
        if (w != rp_tmp[u] && len[u] > 0) memmove(col + w, col + rp_tmp[u], (size_t)len[u] * sizeof(int32_t));
        w += len[u];
    }
    rp_out[ng] = (int32_t)w;
    return w;
}

/* Fill all G graphs.  col_raw holds sum(2*draws_g) int32, graph g's raw
 * region starting at sum_{h<g} 2*draws_h.  rp_out holds sum(n_g+1) int32
 * (graph g's local row_ptr at vtx_off[g] + g).  m_out[g] receives m_g.
 * The caller then packs col (see graphgen_er_pack). */
void graphgen_er_fill(int64_t G, uint64_t seed, const int64_t* n_g, const int64_t* draws_g, int32_t* col_raw,
                      int32_t* rp_out, int64_t* m_out) {
    int64_t* raw_off = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
    int64_t* rp_off = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
    int64_t nmax = 1;
    raw_off[0] = 0;
    rp_off[0] = 0;
    for (int64_t g = 0; g < G; ++g) {
        raw_off[g + 1] = raw_off[g] + 2 * draws_g[g];
        rp_off[g + 1] = rp_off[g] + n_g[g] + 1;
        if (n_g[g] > nmax) nmax = n_g[g];
    }
#pragma omp parallel
    {
        int64_t* rp_tmp = (int64_t*)malloc((size_t)(nmax + 1) * sizeof(int64_t));
        int64_t* len = (int64_t*)malloc((size_t)(nmax + 1) * sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t g = 0; g < G; ++g)
            m_out[g] = er_fill_one(g, seed, n_g[g], draws_g[g], col_raw + raw_off[g], rp_tmp, len, rp_out + rp_off[g]);
        free(rp_tmp);
        free(len);
    }
    free(raw_off);
    free(rp_off);
}

/* Pack the per-graph regions of col_raw densely (in place, ascending g).
 * Writes edge_off (G+1). */
void graphgen_er_pack(int64_t G, const int64_t* draws_g, const int64_t* m_g, int32_t* col_raw, int64_t* edge_off) {
    int64_t raw = 0, w = 0;
    for (int64_t g = 0; g < G; ++g) {
        edge_off[g] = w;
        if (w != raw && m_g[g] > 0) memmove(col_raw + w, col_raw + raw, (size_t)m_g[g] * sizeof(int32_t));
        w += m_g[g];
        raw += 2 * draws_g[g];
    }
    edge_off[G] = w;
}

/* ------------------------------------------------------------------ */
/* Serving trace: arrival times and per-request graph parameters        */
/* ------------------------------------------------------------------ */

/* Request i: inter-arrival -ln(U)/rate; undirected edge target E =
 * exp(U(ln emin, ln emax)); kind 0 = R-MAT (edge factor U{8..32}, scale =
 * round(log2(E/ef))), kind 1 = lattice (p = U(0.4, 0.9), side =
 * round(sqrt(E/(2p)))).  Outputs per request: t_arrival (s), kind, scale or
 * side, edge factor (R-MAT) and p (lattice), and a per-request seed. */
void graphgen_trace(int64_t R, uint64_t seed, double rate, double emin, double emax, double* t_out, int32_t* kind,
                    int64_t* size_param, int32_t* ef, double* p, uint64_t* req_seed) {
    double t = 0.0, l0 = gg_log(emin), l1 = gg_log(emax);
    for (int64_t i = 0; i < R; ++i) {
        uint64_t base = (uint64_t)i * 8;
        double ua = gg_unit(gg_word(seed, STREAM_TRACE, base + 0));
        double ue = gg_unit(gg_word(seed, STREAM_TRACE, base + 1));
        uint64_t wk = gg_word(seed, STREAM_TRACE, base + 2);
        double up = gg_unit(gg_word(seed, STREAM_TRACE, base + 3));
        uint64_t wf = gg_word(seed, STREAM_TRACE, base + 4);
        t = t + (-gg_log(1.0 - ua)) / rate;
        t_out[i] = t;
        double E = gg_exp(l0 + ue * (l1 - l0));
        kind[i] = (int32_t)(wk >> 63);
        req_seed[i] = gg_word(seed, STREAM_TRACE, base + 5);
        if (kind[i] == 0) {
            int32_t f = 8 + (int32_t)gg_bounded32((uint32_t)(wf >> 32), 25);
            double lg = gg_log(E / (double)f) / GG_LN2;
            int64_t s = gg_round(lg);
            if (s < 1) s = 1;
            ef[i] = f;
            size_param[i] = s;
            p[i] = 0.0;
        } else {
            double pp = 0.4 + up * 0.5;
            double x = E / (2.0 * pp), y = x > 1 ? x : 1.0;
            /* Newton iterations for sqrt with basic operations */
            for (int k = 0; k < 64; ++k) y = 0.5 * (y + x / y);
            int64_t side = gg_round(y);
            if (side < 2) side = 2;
            ef[i] = 0;
            size_param[i] = side;
            p[i] = pp;
        }
    }
}
