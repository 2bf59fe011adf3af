/*
 * oracle.c -- plain CPU reference for the FastSV connected-components method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * it is used by tests/, by the smoke check and by the CPU baseline leg of the
 * benchmark.  It shares no source, header or helper with the CUDA library.
 *
 * Paper: Y. Zhang, A. Azad, Z. Hu, "FastSV: A Distributed-Memory Connected
 * Component Algorithm with Fast Convergence" (arXiv:1910.05971).
 *
 * Contents (each function names the passage it follows):
 *   oracle_fastsv_alg2   Algorithm 2 (Section 3): edge-form stochastic hooking,
 *                        aggressive hooking, shortcutting, reads from f and
 *                        writes to f_next; stops when f[f] is unchanged
 *                        (Section 3.4, Lemma "early termination").
 *   oracle_fastsv_alg3   Algorithm 3 (Section 4.1): the same method written as
 *                        GraphBLAS operations (mxv on (select2nd,min) with MIN
 *                        accumulation, assign with MIN, two eWiseMult MIN,
 *                        extractTuples + extract, ISNE + reduce(+), dup).
 *   oracle_fastsv_sv     the convergence ablation sv1..sv5 of Section 5.2:
 *                        Algorithm 1, then the optimizations of Sections
 *                        3.1-3.4 added one at a time (sv5 = Algorithm 2).
 *   oracle_fastsv_omp    Algorithm 2 again with OpenMP parallel loops; every
 *                        min-update is an atomic min, so each iteration gives
 *                        exactly the sequential result.  Used for timing and
 *                        for large inputs.
 *   oracle_uf            Union-find (union by smaller root id, path halving):
 *                        labels[u] = smallest vertex id of u's component, the
 *                        converged state described in Section 3.4.
 *   oracle_bfs           Breadth-first search from every unvisited vertex in
 *                        ascending id order: the textbook definition of a
 *                        connected component (Section 2.1 notation).
 *
 * Graph input everywhere: CSR with int64 row pointers rp[0..n] and int32
 * neighbour ids ci[rp[u] .. rp[u+1]); the graph is undirected, so every edge
 * {u,v} appears as (u,v) and (v,u).  Self-loops and duplicate entries are
 * allowed.  INF (= INT32_MAX) stands for "no neighbour".
 *
 * Compile-time MUTANT (tests only): plants one deliberate mistake so that the
 * tests can show the pins catch it.  0 = correct code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef MUTANT
#define MUTANT 0
#endif

#define INF 0x7fffffff

static inline int32_t min32(int32_t a, int32_t b) { return a < b ? a : b; }

/* ---------------------------------------------------------------------- */
/* Algorithm 2 (Section 3): one iteration                                  */
/* ---------------------------------------------------------------------- */

/*
 * One pass of the repeat-loop body of Algorithm 2.
 *   f       parent vector, replaced by f_next on return
 *   fnext   scratch of n entries
 *   gf_prev scratch of n entries: receives f[f] as it was before the update
 * Returns the number of u with f[f[u]] after the update != f[f[u]] before it
 * (the termination test of Section 3.4; Algorithm 3 lines "ISNE" + "reduce").
 */
int64_t oracle_alg2_iteration(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int32_t* fnext,
                              int32_t* gf_prev) {
    /* grandparents of the current pointer graph */
    for (int64_t u = 0; u < n; ++u) gf_prev[u] = f[f[u]];
    /* f_next starts as a copy of f (Algorithm 2 initialises both to u, and
     * after every iteration f <- f_next makes them equal again) */
    memcpy(fnext, f, (size_t)n * sizeof(int32_t));

    /* Step 1, stochastic hooking: for every (u,v) in E,
     *   f_next[f[u]] <-min f[f[v]] */
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = ci[e];
            int32_t ffv = f[f[v]];
#if MUTANT == 1 /* hook onto the parent instead of the grandparent */
            ffv = f[v];
#endif
#if MUTANT == 2 /* index the hook by the vertex instead of its parent */
            int32_t target = (int32_t)u;
#else
            int32_t target = f[u];
#endif
            fnext[target] = min32(fnext[target], ffv);
        }
    }
    /* Step 2, aggressive hooking: for every (u,v) in E,
     *   f_next[u] <-min f[f[v]] */
#if MUTANT != 3 /* drop aggressive hooking */
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = ci[e];
            fnext[u] = min32(fnext[u], f[f[v]]);
        }
    }
#endif
    /* Step 3, shortcutting: for every u, f_next[u] <-min f[f[u]] */
#if MUTANT != 4 /* drop shortcutting */
    for (int64_t u = 0; u < n; ++u) fnext[u] = min32(fnext[u], f[f[u]]);
#endif
    /* f <- f_next */
    memcpy(f, fnext, (size_t)n * sizeof(int32_t));

    /* until f[f] remains unchanged */
    int64_t changed = 0;
    for (int64_t u = 0; u < n; ++u) {
#if MUTANT == 5 /* test f instead of the grandparent f[f] */
        changed += (f[u] != gf_prev[u]);
#else
        changed += (f[f[u]] != gf_prev[u]);
#endif
    }
    return changed;
}

/*
 * Algorithm 2: f[u] <- u, then repeat the iteration above until f[f] is
 * unchanged, or until max_iters iterations have run (max_iters <= 0 means no
 * limit).  f (n entries) receives the parent vector.  changed_trace (if not
 * NULL) receives the changed count of the first trace_cap iterations.
 * Returns the number of iterations executed; *converged = 1 if the last one
 * found f[f] unchanged.  n == 0 runs no iteration.
 */
int64_t oracle_fastsv_alg2(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int64_t max_iters,
                           int64_t* changed_trace, int64_t trace_cap, int32_t* converged) {
    *converged = 1;
    if (n <= 0) return 0;
    int32_t* fnext = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* gfp = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t u = 0; u < n; ++u) f[u] = (int32_t)u;
    int64_t it = 0, changed;
    do {
        changed = oracle_alg2_iteration(n, rp, ci, f, fnext, gfp);
        if (changed_trace && it < trace_cap) changed_trace[it] = changed;
        ++it;
    } while (changed != 0 && (max_iters <= 0 || it < max_iters));
    *converged = (changed == 0);
    free(fnext);
    free(gfp);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Convergence ablation sv1..sv5 (Section 3, Section 5.2 "Speed of          */
/* convergence"): Algorithm 1 with the optimizations of Section 3 added     */
/* one at a time, in the order of Sections 3.1-3.4                          */
/* ---------------------------------------------------------------------- */

/*
 * One iteration of variant sv<variant>, 1 <= variant <= 4 (sv5 is Algorithm 2
 * itself, oracle_fastsv_alg2).
 *   sv1  Algorithm 1: tree hooking f_next[f[u]] <- f[v] for every (u,v) in E
 *        whose f[u] is a root (f[u] == f[f[u]]) and f[v] < f[u]; f <- f_next;
 *        then shortcutting f_next[u] <- f[f[u]] where f[u] != f[f[u]];
 *        f <- f_next.  Several edges may write the same f_next[f[u]]: the
 *        smallest value is kept, which makes the iteration deterministic.
 *   sv2  sv1 hooking onto the grandparent f[f[v]] instead of f[v] (3.1).
 *   sv3  sv2 without the root test f[u] == f[f[u]]: stochastic hooking (3.2).
 *   sv4  the loop body of Algorithm 2: stochastic and aggressive hooking and
 *        shortcutting, all from the same f (3.3), still stopping when f is
 *        unchanged; sv5 adds the early termination of 3.4.
 *   f      parent vector, replaced by the iteration's result
 *   fnext  scratch of n entries;  fstart scratch of n entries
 * Returns the number of u whose f[u] changed over the iteration (Algorithm 1
 * stops when this is zero).
 */
int64_t oracle_sv_iteration(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int32_t* fnext,
                            int32_t* fstart, int variant) {
    memcpy(fstart, f, (size_t)n * sizeof(int32_t));
    memcpy(fnext, f, (size_t)n * sizeof(int32_t));
    if (variant <= 3) {
        /* Step 1: tree hooking */
        for (int64_t u = 0; u < n; ++u) {
            const int32_t fu = f[u];
#if MUTANT == 6 /* drop the root test of sv1/sv2 */
            const int root = 1;
#else
            const int root = (fu == f[fu]);
#endif
            if (variant <= 2 && !root) continue;
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t v = ci[e];
                const int32_t hv = variant == 1 ? f[v] : f[f[v]];
                if (hv < fu) fnext[fu] = min32(fnext[fu], hv);
            }
        }
        memcpy(f, fnext, (size_t)n * sizeof(int32_t));
        /* Step 2: shortcutting, on the hooked pointer graph */
        for (int64_t u = 0; u < n; ++u) {
#if MUTANT == 7 /* shortcut from the pointer graph before hooking */
            const int32_t gu = fstart[fstart[u]];
#else
            const int32_t gu = f[f[u]];
#endif
            if (f[u] != gu) fnext[u] = gu;
        }
        memcpy(f, fnext, (size_t)n * sizeof(int32_t));
    } else {
        /* the three steps of Algorithm 2, all reading the same f */
        for (int64_t u = 0; u < n; ++u)
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t ffv = f[f[ci[e]]];
                fnext[f[u]] = min32(fnext[f[u]], ffv); /* stochastic hooking */
                fnext[u] = min32(fnext[u], ffv);       /* aggressive hooking */
            }
        for (int64_t u = 0; u < n; ++u) fnext[u] = min32(fnext[u], f[f[u]]); /* shortcutting */
        memcpy(f, fnext, (size_t)n * sizeof(int32_t));
    }
    /* until f remains unchanged */
    int64_t changed = 0;
    for (int64_t u = 0; u < n; ++u) changed += (f[u] != fstart[u]);
    return changed;
}

/*
 * Variant sv<variant> (1..5) from f[u] = u until its stopping test holds, or
 * max_iters iterations (<= 0: no limit).  Same arguments and return as
 * oracle_fastsv_alg2; the trace holds the per-iteration count of the
 * variant's own test (changed f for sv1..sv4, changed f[f] for sv5).
 */
int64_t oracle_fastsv_sv(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int variant,
                         int64_t max_iters, int64_t* changed_trace, int64_t trace_cap, int32_t* converged) {
    if (variant == 5) return oracle_fastsv_alg2(n, rp, ci, f, max_iters, changed_trace, trace_cap, converged);
    *converged = 1;
    if (n <= 0) return 0;
    if (variant < 1 || variant > 5) {
        *converged = 0;
        return -1;
    }
    int32_t* fnext = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* fstart = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t u = 0; u < n; ++u) f[u] = (int32_t)u;
    int64_t it = 0, changed;
    do {
        changed = oracle_sv_iteration(n, rp, ci, f, fnext, fstart, variant);
        if (changed_trace && it < trace_cap) changed_trace[it] = changed;
        ++it;
    } while (changed != 0 && (max_iters <= 0 || it < max_iters));
    *converged = (changed == 0);
    free(fnext);
    free(fstart);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 3 (Section 4.1): GraphBLAS formulation, written out            */
/* ---------------------------------------------------------------------- */

/*
 * Each GraphBLAS call is spelled out as the loop its definition in
 * Section 4.1 gives.  mngf is carried across iterations (it is initialised
 * to gf and every mxv accumulates into it with MIN); a row with no entries
 * leaves mngf[u] as it was.  The assign uses the indices extracted from f
 * before this iteration's updates.  Same arguments and return as
 * oracle_fastsv_alg2.
 */
int64_t oracle_fastsv_alg3(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int64_t max_iters,
                           int64_t* changed_trace, int64_t trace_cap, int32_t* converged) {
    *converged = 1;
    if (n <= 0) return 0;
    size_t bytes = (size_t)n * sizeof(int32_t);
    int32_t* gf = (int32_t*)malloc(bytes);
    int32_t* dup = (int32_t*)malloc(bytes);
    int32_t* mngf = (int32_t*)malloc(bytes);
    int32_t* value = (int32_t*)malloc(bytes);
    /* the input parent vector: every vertex its own root */
    for (int64_t u = 0; u < n; ++u) f[u] = (int32_t)u;
    /* GrB_Vector_dup(&gf, f); dup(&dup, gf); dup(&mngf, gf) */
    memcpy(gf, f, bytes);
    memcpy(dup, gf, bytes);
    memcpy(mngf, gf, bytes);
    /* GrB_Vector_extractTuples(index, value, &n, f) */
    memcpy(value, f, bytes);
    int64_t it = 0, sum;
    do {
        /* Step 1: GrB_mxv(mngf, NULL, GrB_MIN, Sel2ndMin, A, gf, NULL) */
        for (int64_t u = 0; u < n; ++u) {
            if (rp[u + 1] == rp[u]) continue; /* empty row: no product, mngf[u] kept */
            int32_t t = INF;
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) t = min32(t, gf[ci[e]]); /* select2nd, then min */
            mngf[u] = min32(mngf[u], t);                                        /* accumulate with MIN */
        }
        /* GrB_assign(f, NULL, GrB_MIN, mngf, value, n, NULL): f[value[i]] min= mngf[i] */
        for (int64_t i = 0; i < n; ++i) f[value[i]] = min32(f[value[i]], mngf[i]);
        /* Step 2: GrB_eWiseMult(f, NULL, NULL, GrB_MIN, f, mngf, NULL) */
        for (int64_t u = 0; u < n; ++u) f[u] = min32(f[u], mngf[u]);
        /* Step 3: GrB_eWiseMult(f, NULL, NULL, GrB_MIN, f, gf, NULL) */
        for (int64_t u = 0; u < n; ++u) f[u] = min32(f[u], gf[u]);
        /* Step 4: extractTuples(index, value, &n, f); GrB_extract(gf, .., f, value, n, ..) */
        memcpy(value, f, bytes);
        for (int64_t i = 0; i < n; ++i) gf[i] = f[value[i]];
        /* Step 5: diff = ISNE(dup, gf); sum = reduce(+, diff); dup <- gf */
        sum = 0;
        for (int64_t u = 0; u < n; ++u) sum += (dup[u] != gf[u]);
        memcpy(dup, gf, bytes);
        if (changed_trace && it < trace_cap) changed_trace[it] = sum;
        ++it;
    } while (sum != 0 && (max_iters <= 0 || it < max_iters));
    *converged = (sum == 0);
    free(gf);
    free(dup);
    free(mngf);
    free(value);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 2 with OpenMP loops (same result per iteration)               */
/* ---------------------------------------------------------------------- */

static inline void atomic_min32(int32_t* p, int32_t v) {
    int32_t cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (v < cur && !__atomic_compare_exchange_n(p, &cur, v, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

/*
 * Algorithm 2 with the vertex loops split across nthreads OpenMP threads
 * (nthreads <= 0: the OpenMP default).  All writes to f_next are atomic mins
 * of values read from f, so the result of an iteration does not depend on
 * the schedule.  Same arguments and return as oracle_fastsv_alg2.
 */
int64_t oracle_fastsv_omp(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* f, int64_t max_iters,
                          int64_t* changed_trace, int64_t trace_cap, int32_t* converged, int nthreads) {
    *converged = 1;
    if (n <= 0) return 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int32_t* fnext = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* gfp = (int32_t*)malloc((size_t)n * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) f[u] = (int32_t)u;
    int64_t it = 0, changed;
    do {
#pragma omp parallel for schedule(static)
        for (int64_t u = 0; u < n; ++u) {
            gfp[u] = f[f[u]];
            fnext[u] = f[u];
        }
        /* stochastic hooking, then aggressive hooking (Algorithm 2 steps 1-2) */
#pragma omp parallel for schedule(dynamic, 512)
        for (int64_t u = 0; u < n; ++u) {
            /* min over the row first: applying the row minimum once is the
             * same as applying every f[f[v]] of the row */
            int32_t best = INF;
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) best = min32(best, f[f[ci[e]]]);
            if (best == INF) continue;
            atomic_min32(&fnext[f[u]], best);
            atomic_min32(&fnext[u], best);
        }
        /* shortcutting (step 3) */
#pragma omp parallel for schedule(static)
        for (int64_t u = 0; u < n; ++u) atomic_min32(&fnext[u], gfp[u]);
        changed = 0;
#pragma omp parallel for schedule(static)
        for (int64_t u = 0; u < n; ++u) f[u] = fnext[u];
#pragma omp parallel for schedule(static) reduction(+ : changed)
        for (int64_t u = 0; u < n; ++u) changed += (f[f[u]] != gfp[u]);
        if (changed_trace && it < trace_cap) changed_trace[it] = changed;
        ++it;
    } while (changed != 0 && (max_iters <= 0 || it < max_iters));
    *converged = (changed == 0);
    free(fnext);
    free(gfp);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Exact result: smallest vertex id per connected component                 */
/* ---------------------------------------------------------------------- */

static inline int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]]; /* path halving */
        x = parent[x];
    }
    return x;
}

/* Union-find with union by smaller root id: every root is the smallest id of
 * its tree, so labels[u] = min id of u's component. */
void oracle_uf(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* labels) {
    for (int64_t u = 0; u < n; ++u) labels[u] = (int32_t)u;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t a = uf_find(labels, (int32_t)u), b = uf_find(labels, ci[e]);
            if (a < b)
                labels[b] = a;
            else if (b < a)
                labels[a] = b;
        }
    }
    for (int64_t u = 0; u < n; ++u) labels[u] = uf_find(labels, (int32_t)u);
}

/* Breadth-first search from every unvisited vertex in ascending order; the
 * start vertex is the smallest id of the component it discovers. */
void oracle_bfs(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* labels) {
    int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t u = 0; u < n; ++u) labels[u] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (labels[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        labels[s] = (int32_t)s;
        queue[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t x = queue[head++];
            for (int64_t e = rp[x]; e < rp[x + 1]; ++e) {
                int32_t y = ci[e];
                if (labels[y] < 0) {
                    labels[y] = (int32_t)s;
                    queue[tail++] = y;
                }
            }
        }
    }
    free(queue);
}
