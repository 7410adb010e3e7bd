/*
 * cng_oracle.c -- plain, slow, FP64 CPU oracle for the alpha-CNG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  The CUDA library shares no code with it.
 *
 * Every routine below follows one passage of the paper (arXiv 2510.05975,
 * "Fast-Convergent Proximity Graphs for Approximate Nearest Neighbor Search"):
 *
 *   canonical distance      Sec. 2.1 (metric space); the numeric reading is ours:
 *                           D(x,y) = sqrt(sum_{i=0}^{d-1} (x_i - y_i)^2) in IEEE double,
 *                           summed left to right, one rounding per operation, no fused
 *                           multiply-add (compile with -ffp-contract=off).
 *   candidate lists         Alg. 3, phase 2 reads "the C closest points"; here the exact
 *                           L nearest points of P \ {p} ordered by (D, id).
 *   navigating node         Alg. 3, phase 1: nearest point to the centroid of P (exact
 *                           form: argmin over all points of (D(c, x), id)).
 *   pruning                 Def. 2 (Eq. 1) and Alg. 2, fixed alpha, stop at R kept; the
 *                           soundness check of whole kept lists follows the same rule.
 *   adaptive pruning        Alg. 4 with alpha_i = alpha0 + i * dalpha.
 *   reverse merge           Alg. 3, phase 3 and the lazy-pruning paragraph of Sec. 4.3.
 *   beam search             Alg. 1 (with a visited set; identical returned ids).
 *
 * Ties: every "sort by distance" orders by (D, id) lexicographically.
 * Parallelism: OpenMP over independent points / queries only; each point's arithmetic is
 * the sequential definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_E_INVAL -1
#define OR_E_NOMEM -2

/* ---- canonical distance (Sec. 2.1) -------------------------------------------------- */

/* Squared distance: left-to-right sum of squared differences, all in double. */
double or_sqdist(const float *x, const float *y, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = (double)x[i] - (double)y[i];
        s = s + t * t;
    }
    return s;
}

double or_dist(const float *x, const float *y, int d) { return sqrt(or_sqdist(x, y, d)); }

/* Distance from a double-precision point (the centroid) to a float point. */
double or_dist_dc(const double *c, const float *y, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = c[i] - (double)y[i];
        s = s + t * t;
    }
    return sqrt(s);
}

static int key_less(double da, int32_t ia, double db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

/* ---- exact candidate lists (Alg. 3 phase 2, exact form) ---------------------------- */

/*
 * For each of the m rows, the L points of `base` with the smallest (D, id), ascending.
 * If exclude_self, row i is base point i and is left out by id (duplicates stay).
 * Rows with fewer than L eligible points are padded with id -1 and distance +inf.
 */
int or_knn(const float *base, int64_t n, const float *rows, int64_t m, int d, int L,
           int exclude_self, int32_t *out_ids, double *out_d) {
    if (n < 0 || m < 0 || d <= 0 || L <= 0) return OR_E_INVAL;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
        int32_t *ids = out_ids + i * L;
        double *ds = out_d + i * L;
        int cnt = 0;
        const float *x = rows + i * (int64_t)d;
        for (int64_t j = 0; j < n; ++j) {
            if (exclude_self && j == i) continue;
            double D = or_dist(x, base + j * (int64_t)d, d);
            if (cnt < L || key_less(D, (int32_t)j, ds[cnt - 1], ids[cnt - 1])) {
                int pos = (cnt < L) ? cnt : L - 1;
                while (pos > 0 && key_less(D, (int32_t)j, ds[pos - 1], ids[pos - 1])) {
                    ds[pos] = ds[pos - 1];
                    ids[pos] = ids[pos - 1];
                    --pos;
                }
                ds[pos] = D;
                ids[pos] = (int32_t)j;
                if (cnt < L) ++cnt;
            }
        }
        for (int t = cnt; t < L; ++t) {
            ids[t] = -1;
            ds[t] = INFINITY;
        }
    }
    return err;
}

/* ---- navigating node (Alg. 3 phase 1, exact form) ---------------------------------- */

/*
 * Centroid: c_j = (sum_i x_ij) / n in double.  The paper fixes no summation order; ours:
 * rows are taken in consecutive blocks of OR_CENTROID_BLOCK, each block summed left to
 * right, then the block sums added left to right, then one division by n.
 */
#define OR_CENTROID_BLOCK 4096
void or_centroid(const float *X, int64_t n, int d, double *c) {
    for (int j = 0; j < d; ++j) {
        double total = 0.0;
        for (int64_t b = 0; b < n; b += OR_CENTROID_BLOCK) {
            int64_t e = b + OR_CENTROID_BLOCK < n ? b + OR_CENTROID_BLOCK : n;
            double s = 0.0;
            for (int64_t i = b; i < e; ++i) s = s + (double)X[i * (int64_t)d + j];
            total = total + s;
        }
        c[j] = total / (double)n;
    }
}

/* Navigating node s = argmin_i (D(c, x_i), i). */
int32_t or_entry(const float *X, int64_t n, int d) {
    if (n <= 0 || d <= 0) return -1;
    double *c = (double *)malloc(sizeof(double) * d);
    if (!c) return -1;
    or_centroid(X, n, d, c);
    double best = INFINITY;
    int32_t bi = -1;
    for (int64_t i = 0; i < n; ++i) {
        double D = or_dist_dc(c, X + i * (int64_t)d, d);
        if (bi < 0 || key_less(D, (int32_t)i, best, bi)) {
            best = D;
            bi = (int32_t)i;
        }
    }
    free(c);
    return bi;
}

/* ---- pruning (Def. 2, Alg. 2) ------------------------------------------------------ */

typedef struct {
    double D;
    int32_t id;
} or_pair;

static int pair_cmp(const void *a, const void *b) {
    const or_pair *x = (const or_pair *)a, *y = (const or_pair *)b;
    if (x->D < y->D) return -1;
    if (x->D > y->D) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Sort the ids in V by (D(p, .), id); writes the sorted pairs into `out`. */
static void sort_by_distance(const float *X, int d, int64_t p, const int32_t *V, int nv,
                             or_pair *out) {
    const float *xp = X + p * (int64_t)d;
    for (int i = 0; i < nv; ++i) {
        out[i].id = V[i];
        out[i].D = or_dist(xp, X + (int64_t)V[i] * d, d);
    }
    qsort(out, (size_t)nv, sizeof(or_pair), pair_cmp);
}

/*
 * Def. 2 / Eq. 1: u is pruned by v iff D(p,u) > alpha * D(u,v) + (alpha + 1) * tau.
 * Evaluated as t = (alpha + 1) * tau once, rhs = alpha * D(u,v) + t, strict '>'.
 */
static int rule_prunes(double Dpu, double Duv, double alpha, double t) {
    double rhs = alpha * Duv + t;
    return Dpu > rhs;
}

/* Alg. 2 on candidates already sorted by (D(p,.), id); stops when R points are kept. */
static int prune_sorted(const float *X, int d, const or_pair *V, int nv, double alpha,
                        double tau, int R, int32_t *S) {
    double t = (alpha + 1.0) * tau;
    int ns = 0;
    for (int i = 0; i < nv && ns < R; ++i) {
        int32_t u = V[i].id;
        int pruned = 0;
        for (int j = 0; j < ns && !pruned; ++j) {
            double Duv = or_dist(X + (int64_t)u * d, X + (int64_t)S[j] * d, d);
            pruned = rule_prunes(V[i].D, Duv, alpha, t);
        }
        if (!pruned) S[ns++] = u;
    }
    return ns;
}

/* pruning(p, V, alpha) of Alg. 2 with the out-degree cut at R.  Returns |S|. */
int or_prune(const float *X, int64_t n, int d, int64_t p, const int32_t *V, int nv,
             double alpha, double tau, int R, int32_t *S) {
    (void)n;
    if (nv < 0 || R <= 0) return OR_E_INVAL;
    or_pair *pv = (or_pair *)malloc(sizeof(or_pair) * (nv > 0 ? nv : 1));
    if (!pv) return OR_E_NOMEM;
    sort_by_distance(X, d, p, V, nv, pv);
    int ns = prune_sorted(X, d, pv, nv, alpha, tau, R, S);
    free(pv);
    return ns;
}

/*
 * adaptive-pruning of Alg. 4: alpha_i = alpha0 + i * dalpha for i = 0 .. imax with
 * imax = round((alpha_max - alpha0) / dalpha); stop at the first S_i with |S_i| >= R/2
 * (real division); return the R closest points of the last S_i computed.
 */
/* Alg. 4 on candidates already sorted by (D(p,.), id). */
static int prune_adaptive_sorted(const float *X, int d, const or_pair *pv, int nv, double alpha0,
                                 double alpha_max, double dalpha, double tau, int R, int32_t *S,
                                 double *alpha_used) {
    int imax = (int)floor((alpha_max - alpha0) / dalpha + 0.5);
    int ns = 0;
    double a = alpha0;
    for (int i = 0; i <= imax; ++i) {
        a = alpha0 + (double)i * dalpha;
        /* S_i in full is not needed: its R closest points are its first R members. */
        ns = prune_sorted(X, d, pv, nv, a, tau, R, S);
        if ((double)ns >= (double)R / 2.0) break;
    }
    if (alpha_used) *alpha_used = a;
    return ns;
}

int or_prune_adaptive(const float *X, int64_t n, int d, int64_t p, const int32_t *V, int nv,
                      double alpha0, double alpha_max, double dalpha, double tau, int R,
                      int32_t *S, double *alpha_used) {
    (void)n;
    if (nv < 0 || R <= 0 || dalpha <= 0.0) return OR_E_INVAL;
    or_pair *pv = (or_pair *)malloc(sizeof(or_pair) * (nv > 0 ? nv : 1));
    if (!pv) return OR_E_NOMEM;
    sort_by_distance(X, d, p, V, nv, pv);
    int ns = prune_adaptive_sorted(X, d, pv, nv, alpha0, alpha_max, dalpha, tau, R, S, alpha_used);
    free(pv);
    return ns;
}

/*
 * Soundness of kept lists under Def. 2 (Eq. 1) and Alg. 2: for every point p, its list
 * S = lists[p][0 .. cnt[p]) (row stride `stride`) must hold distinct valid ids other than p, in
 * ascending (D(p, .), id) order, and no member S[j] may be pruned by an earlier member S[i]
 * (i < j): D(p, S[j]) > alpha * D(S[j], S[i]) + (alpha + 1) * tau must be false for every such
 * pair, because Alg. 2 tests each candidate against every point kept before it.  bad[p] (if not
 * NULL) receives 0 for a sound row, 1 for a bad id or duplicate, 2 for an order violation, 3 for
 * a pair that the rule prunes.  Returns the number of unsound rows.
 */
int64_t or_check_rule(const float *X, int64_t n, int d, const int32_t *lists, const int32_t *cnt,
                      int stride, double alpha, double tau, int32_t *bad) {
    if (n <= 0 || stride <= 0) return OR_E_INVAL;
    const double t = (alpha + 1.0) * tau;
    int64_t nbad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nbad)
    for (int64_t p = 0; p < n; ++p) {
        const int32_t *S = lists + p * stride;
        const int c = cnt[p];
        const float *xp = X + p * (int64_t)d;
        int why = c < 0 || c > stride;
        double prevD = -1.0;
        for (int j = 0; j < c && !why; ++j) {
            const int32_t u = S[j];
            if (u < 0 || u >= n || u == p) {
                why = 1;
                break;
            }
            for (int i = 0; i < j; ++i)
                if (S[i] == u) why = 1;
            if (why) break;
            const double Dpu = or_dist(xp, X + (int64_t)u * d, d);
            if (j > 0 && !(Dpu > prevD || (Dpu == prevD && u > S[j - 1]))) {
                why = 2;
                break;
            }
            prevD = Dpu;
            for (int i = 0; i < j; ++i) {
                const double Duv = or_dist(X + (int64_t)u * d, X + (int64_t)S[i] * d, d);
                if (rule_prunes(Dpu, Duv, alpha, t)) {
                    why = 3;
                    break;
                }
            }
        }
        if (bad) bad[p] = why;
        nbad += why != 0;
    }
    return nbad;
}

/* ---- construction (Alg. 3 phases 1-3, exact candidates) ------------------------------ */

/* Pruning used by the build: fixed alpha (Alg. 2) or, with adaptive != 0, Alg. 4 over
 * alpha0, alpha0 + dalpha, ..., alpha_max -- in phase 2 and in phase 3's re-prune alike (Alg. 3
 * calls adaptive-pruning in both places). */
typedef struct {
    double alpha, tau;
    int adaptive;
    double alpha0, alpha_max, dalpha;
} or_rule;

static int build_prune(const float *X, int d, const or_pair *pv, int nv, const or_rule *r, int R,
                       int32_t *S) {
    if (r->adaptive)
        return prune_adaptive_sorted(X, d, pv, nv, r->alpha0, r->alpha_max, r->dalpha, r->tau, R,
                                     S, NULL);
    return prune_sorted(X, d, pv, nv, r->alpha, r->tau, R, S);
}

/*
 * Phases 2 and 3 of Alg. 3 from candidate lists cl [n][C] sorted by (D, id) with their canonical
 * distances cd, each row ending at its first -1 (at most C entries).
 */
static int build_from_lists(const float *X, int64_t n, int d, const or_rule *rp, int R, int C,
                            const int32_t *cl, const double *cd, int32_t *fwd, int32_t *fdeg,
                            int32_t *adj, int32_t *deg) {
    const or_rule rule = *rp;
    /* phase 2: prune every candidate list (already sorted by (D, id)) */
#pragma omp parallel
    {
        or_pair *pv = (or_pair *)malloc(sizeof(or_pair) * C);
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n; ++p) {
            int nv = 0;
            while (nv < C && cl[p * C + nv] >= 0) {
                pv[nv].id = cl[p * C + nv];
                pv[nv].D = cd[p * C + nv];
                ++nv;
            }
            int32_t *S = fwd + p * R;
            int ns = build_prune(X, d, pv, nv, &rule, R, S);
            for (int i = ns; i < R; ++i) S[i] = -1;
            fdeg[p] = ns;
        }
        free(pv);
    }

    /* phase 3: reverse edges from the phase-2 snapshot, then lazy pruning */
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off) return OR_E_NOMEM;
    for (int64_t u = 0; u < n; ++u)
        for (int j = 0; j < fdeg[u]; ++j) off[fwd[u * R + j] + 1] += 1;
    for (int64_t p = 0; p < n; ++p) off[p + 1] += off[p];
    int32_t *in = (int32_t *)malloc(sizeof(int32_t) * (off[n] > 0 ? off[n] : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!in || !cur) return OR_E_NOMEM;
    for (int64_t p = 0; p < n; ++p) cur[p] = off[p];
    for (int64_t u = 0; u < n; ++u) /* in-lists in ascending u */
        for (int j = 0; j < fdeg[u]; ++j) in[cur[fwd[u * R + j]]++] = (int32_t)u;

#pragma omp parallel
    {
        int cap = 0;
        int32_t *V = NULL;
        or_pair *pv = NULL;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n; ++p) {
            int nin = (int)(off[p + 1] - off[p]);
            int need = fdeg[p] + nin;
            if (need > cap) {
                cap = need * 2;
                V = (int32_t *)realloc(V, sizeof(int32_t) * cap);
                pv = (or_pair *)realloc(pv, sizeof(or_pair) * cap);
            }
            int nv = 0;
            for (int j = 0; j < fdeg[p]; ++j) V[nv++] = fwd[p * R + j];
            for (int j = 0; j < nin; ++j) {
                int32_t u = in[off[p] + j], dup = 0;
                for (int t = 0; t < fdeg[p] && !dup; ++t) dup = (fwd[p * R + t] == u);
                if (!dup) V[nv++] = u;
            }
            sort_by_distance(X, d, p, V, nv, pv);
            int32_t *A = adj + p * R;
            int na;
            if (nv <= R) { /* assigned directly, kept in (D, id) order */
                for (int i = 0; i < nv; ++i) A[i] = pv[i].id;
                na = nv;
            } else {
                na = build_prune(X, d, pv, nv, &rule, R, A);
            }
            for (int i = na; i < R; ++i) A[i] = -1;
            deg[p] = na;
        }
        free(V);
        free(pv);
    }
    free(in);
    free(cur);
    free(off);
    return OR_OK;
}

/*
 * Alg. 3 phases 1-3 with exact candidates:
 * entry            navigating node
 * cand  [n][L]     exact candidate lists (may be NULL)
 * fwd   [n][R]     phase-2 out-lists (pruned candidates), padded with -1
 * fdeg  [n]
 * adj   [n][R]     final out-lists after reverse merge + lazy pruning, padded with -1
 * deg   [n]
 * Returns 0, or a negative error.
 */
int or_build_ex(const float *X, int64_t n, int d, double alpha, double tau, int R, int L,
                int adaptive, double alpha0, double alpha_max, double dalpha, int32_t *entry,
                int32_t *cand, int32_t *fwd, int32_t *fdeg, int32_t *adj, int32_t *deg) {
    if (n < 2 || d <= 0 || R <= 0 || L <= 0 || L >= n) return OR_E_INVAL;
    if (adaptive && !(dalpha > 0.0)) return OR_E_INVAL;
    const or_rule rule = {alpha, tau, adaptive, alpha0, alpha_max, dalpha};
    int32_t *cl = cand ? cand : (int32_t *)malloc(sizeof(int32_t) * n * L);
    double *cd = (double *)malloc(sizeof(double) * n * L);
    if (!cl || !cd) return OR_E_NOMEM;
    *entry = or_entry(X, n, d);
    or_knn(X, n, X, n, d, L, 1, cl, cd);
    int rc = build_from_lists(X, n, d, &rule, R, L, cl, cd, fwd, fdeg, adj, deg);
    free(cd);
    if (!cand) free(cl);
    return rc;
}

int or_build(const float *X, int64_t n, int d, double alpha, double tau, int R, int L,
             int32_t *entry, int32_t *cand, int32_t *fwd, int32_t *fdeg, int32_t *adj,
             int32_t *deg) {
    return or_build_ex(X, n, d, alpha, tau, R, L, 0, 0.0, 0.0, 0.0, entry, cand, fwd, fdeg, adj,
                       deg);
}

/* ---- beam search (Alg. 1) ----------------------------------------------------------- */

typedef struct {
    double D;
    int32_t id;
    int32_t explored;
} or_qent;

/*
 * Alg. 1 from entry s with queue size L, returning the k closest entries of Q.
 * A visited set skips points whose distance was already computed; this returns the same
 * ids as the set-union form of Alg. 1 because a point dropped from Q can never re-enter
 * it (the L-th key of Q never increases once Q is full).
 * ndc counts distance computations (the entry included); hops counts hop vertices.
 * Rows of out_ids / out_d beyond |Q| are -1 / +inf.
 */
int or_search(const float *X, int64_t n, int d, const int32_t *adj, const int32_t *deg, int R,
              int32_t s, const float *Qv, int64_t nq, int k, int L, int32_t *out_ids,
              double *out_d, int32_t *ndc_out, int32_t *hops_out) {
    if (n <= 0 || k <= 0 || L < k || s < 0 || s >= n) return OR_E_INVAL;
    int err = 0;
#pragma omp parallel
    {
        unsigned char *vis = (unsigned char *)calloc((size_t)n, 1);
        int32_t *touched = NULL;
        int64_t tcap = 0;
        or_qent *Q = (or_qent *)malloc(sizeof(or_qent) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const float *q = Qv + qi * (int64_t)d;
            int64_t nt = 0;
            int len = 1;
            Q[0].D = or_dist(q, X + (int64_t)s * d, d);
            Q[0].id = s;
            Q[0].explored = 0;
            vis[s] = 1;
            if (nt >= tcap) {
                tcap = tcap ? tcap * 2 : 4096;
                touched = (int32_t *)realloc(touched, sizeof(int32_t) * tcap);
            }
            touched[nt++] = s;
            int32_t ndc = 1, hops = 0;
            for (;;) {
                int i = 0;
                while (i < len && Q[i].explored) ++i;
                if (i == len) break;
                Q[i].explored = 1;
                ++hops;
                int32_t u = Q[i].id;
                for (int j = 0; j < deg[u]; ++j) {
                    int32_t v = adj[(int64_t)u * R + j];
                    if (vis[v]) continue;
                    vis[v] = 1;
                    if (nt >= tcap) {
                        tcap *= 2;
                        touched = (int32_t *)realloc(touched, sizeof(int32_t) * tcap);
                    }
                    touched[nt++] = v;
                    ++ndc;
                    double D = or_dist(q, X + (int64_t)v * d, d);
                    if (len < L || key_less(D, v, Q[len - 1].D, Q[len - 1].id)) {
                        int pos = (len < L) ? len : L - 1;
                        while (pos > 0 && key_less(D, v, Q[pos - 1].D, Q[pos - 1].id)) {
                            Q[pos] = Q[pos - 1];
                            --pos;
                        }
                        Q[pos].D = D;
                        Q[pos].id = v;
                        Q[pos].explored = 0;
                        if (len < L) ++len;
                    }
                }
            }
            for (int t = 0; t < k; ++t) {
                out_ids[qi * k + t] = t < len ? Q[t].id : -1;
                out_d[qi * k + t] = t < len ? Q[t].D : INFINITY;
            }
            if (ndc_out) ndc_out[qi] = ndc;
            if (hops_out) hops_out[qi] = hops;
            for (int64_t t = 0; t < nt; ++t) vis[touched[t]] = 0;
        }
        free(vis);
        free(touched);
        free(Q);
    }
    return err;
}

/* ---- beam-search candidates (Alg. 3 phase 2, Sec. 4.1) ------------------------------- */

/*
 * For every point p: beam search (Alg. 1, queue size L) on the graph (adj [n][R], deg) from s
 * with x_p as the query; every point whose distance is computed is collected, and the C closest
 * by (D, id), p itself excluded by id, form p's candidate list out_ids [n][C] with canonical
 * distances out_d (rows padded with -1 / +inf); out_cnt [n] = entries in the row.
 */
int or_beam_candidates(const float *X, int64_t n, int d, const int32_t *adj, const int32_t *deg,
                       int R, int32_t s, int L, int C, int32_t *out_ids, double *out_d,
                       int32_t *out_cnt) {
    if (n <= 0 || L < 1 || C < 1 || s < 0 || s >= n) return OR_E_INVAL;
#pragma omp parallel
    {
        unsigned char *vis = (unsigned char *)calloc((size_t)n, 1);
        or_pair *seen = NULL;
        int64_t scap = 0;
        or_qent *Q = (or_qent *)malloc(sizeof(or_qent) * (L + 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n; ++p) {
            const float *q = X + p * (int64_t)d;
            int64_t ns = 0;
            if (scap == 0) {
                scap = 4096;
                seen = (or_pair *)malloc(sizeof(or_pair) * scap);
            }
            int len = 1;
            Q[0].D = or_dist(q, X + (int64_t)s * d, d);
            Q[0].id = s;
            Q[0].explored = 0;
            vis[s] = 1;
            seen[ns].D = Q[0].D;
            seen[ns++].id = s;
            for (;;) {
                int i = 0;
                while (i < len && Q[i].explored) ++i;
                if (i == len) break;
                Q[i].explored = 1;
                int32_t u = Q[i].id;
                for (int j = 0; j < deg[u]; ++j) {
                    int32_t v = adj[(int64_t)u * R + j];
                    if (vis[v]) continue;
                    vis[v] = 1;
                    double D = or_dist(q, X + (int64_t)v * d, d);
                    if (ns >= scap) {
                        scap *= 2;
                        seen = (or_pair *)realloc(seen, sizeof(or_pair) * scap);
                    }
                    seen[ns].D = D;
                    seen[ns++].id = v;
                    if (len < L || key_less(D, v, Q[len - 1].D, Q[len - 1].id)) {
                        int pos = (len < L) ? len : L - 1;
                        while (pos > 0 && key_less(D, v, Q[pos - 1].D, Q[pos - 1].id)) {
                            Q[pos] = Q[pos - 1];
                            --pos;
                        }
                        Q[pos].D = D;
                        Q[pos].id = v;
                        Q[pos].explored = 0;
                        if (len < L) ++len;
                    }
                }
            }
            for (int64_t t = 0; t < ns; ++t) vis[seen[t].id] = 0;
            qsort(seen, (size_t)ns, sizeof(or_pair), pair_cmp);
            int c = 0;
            for (int64_t t = 0; t < ns && c < C; ++t) {
                if (seen[t].id == (int32_t)p) continue;
                out_ids[p * C + c] = seen[t].id;
                out_d[p * C + c] = seen[t].D;
                ++c;
            }
            out_cnt[p] = c;
            for (int t = c; t < C; ++t) {
                out_ids[p * C + t] = -1;
                out_d[p * C + t] = INFINITY;
            }
        }
        free(vis);
        free(seen);
        free(Q);
    }
    return OR_OK;
}

/*
 * Alg. 3 phases 1-3 with the paper's candidate route: G0 = the K-NN graph given as knn [n][K]
 * (an approximate one in the paper; any K-NN graph here), s = the navigating node given,
 * candidates = or_beam_candidates on G0 (queue Lb, C entries), then phases 2 and 3 as for exact
 * candidates.  cand [n][C] receives the candidate lists (may be NULL).
 */
int or_build_beam(const float *X, int64_t n, int d, double alpha, double tau, int R,
                  int adaptive, double alpha0, double alpha_max, double dalpha,
                  const int32_t *knn, int K, int32_t s, int Lb, int C, int32_t *cand,
                  int32_t *fwd, int32_t *fdeg, int32_t *adj, int32_t *deg) {
    if (n < 2 || d <= 0 || R <= 0 || K <= 0 || C <= 0 || Lb <= 0 || s < 0 || s >= n)
        return OR_E_INVAL;
    if (adaptive && !(dalpha > 0.0)) return OR_E_INVAL;
    const or_rule rule = {alpha, tau, adaptive, alpha0, alpha_max, dalpha};
    int32_t *g0deg = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *cl = cand ? cand : (int32_t *)malloc(sizeof(int32_t) * n * C);
    double *cd = (double *)malloc(sizeof(double) * n * C);
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!g0deg || !cl || !cd || !cnt) return OR_E_NOMEM;
    for (int64_t p = 0; p < n; ++p) {
        int k = 0;
        while (k < K && knn[p * K + k] >= 0) ++k;
        g0deg[p] = k;
    }
    int rc = or_beam_candidates(X, n, d, knn, g0deg, K, s, Lb, C, cl, cd, cnt);
    if (rc == OR_OK) rc = build_from_lists(X, n, d, &rule, R, C, cl, cd, fwd, fdeg, adj, deg);
    free(g0deg);
    free(cd);
    free(cnt);
    if (!cand) free(cl);
    return rc;
}

/* ---- connectivity (Alg. 3 phase 4) ------------------------------------------------------ */

/*
 * The paper adds "necessary edges" from the DFS tree of s to every point outside it, in line
 * with NSG, without fixing which.  Our reading, in rounds until every point is reachable:
 *   reached = points reachable from s;
 *   for every unreached p: beam-search(G, x_p, s, Lc, Lc) on the current graph (all Lc results);
 *     r(p) = the first of its results (nearest first; all reached points) whose row has a free
 *     slot (deg < Rs, degrees as at the start of the round); none: p waits for a later round;
 *   if some unreached p without any in-edge has an r(p): each such p (ascending) gets the edge
 *     r(p) -> p while r(p)'s row has a free slot (such a p can be reached in no other way, so
 *     every one of these edges is necessary; the other unreached points wait, as the new edges
 *     may reach them);
 *   otherwise every reached r named by some r(p) gets the edge r -> (smallest such p).
 * adj rows have stride Rs; phase-3 rows use at most R < Rs of them.  Returns the number of
 * edges added (rounds in *rounds_out), or -3 if a round could add no edge.
 */
int or_connect(const float *X, int64_t n, int d, int32_t *adj, int32_t *deg, int Rs, int32_t s,
               int Lc, int32_t *rounds_out) {
    if (n <= 0 || s < 0 || s >= n || Lc < 1) return OR_E_INVAL;
    unsigned char *reach = (unsigned char *)malloc((size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *U = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * n);
    unsigned char *has_in = (unsigned char *)malloc((size_t)n);
    if (!reach || !stack || !U || !best || !has_in) return OR_E_NOMEM;
    for (int64_t i = 0; i < n; ++i) best[i] = -1;
    int total = 0, rounds = 0, rc = 0;
    for (;;) {
        memset(reach, 0, (size_t)n);
        int64_t top = 0;
        stack[top++] = s;
        reach[s] = 1;
        while (top > 0) {
            int32_t u = stack[--top];
            for (int j = 0; j < deg[u]; ++j) {
                int32_t v = adj[(int64_t)u * Rs + j];
                if (!reach[v]) {
                    reach[v] = 1;
                    stack[top++] = v;
                }
            }
        }
        int64_t nu = 0;
        for (int64_t i = 0; i < n; ++i)
            if (!reach[i]) U[nu++] = (int32_t)i;
        if (nu == 0) break;
        ++rounds;
        const int kc = Lc;
        float *Qm = (float *)malloc(sizeof(float) * nu * d);
        int32_t *rid = (int32_t *)malloc(sizeof(int32_t) * nu * kc);
        double *rd = (double *)malloc(sizeof(double) * nu * kc);
        if (!Qm || !rid || !rd) return OR_E_NOMEM;
        for (int64_t i = 0; i < nu; ++i) memcpy(Qm + i * d, X + (int64_t)U[i] * d, sizeof(float) * d);
        or_search(X, n, d, adj, deg, Rs, s, Qm, nu, kc, Lc, rid, rd, NULL, NULL);
        memset(has_in, 0, (size_t)n);
        for (int64_t u = 0; u < n; ++u)
            for (int j = 0; j < deg[u]; ++j) has_in[adj[u * Rs + j]] = 1;
        /* r(p) with the degrees at the start of the round, kept in rid[i * kc] */
        int64_t nz = 0;
        for (int64_t i = 0; i < nu; ++i) {
            int32_t r = -1;
            for (int t = 0; t < kc && r < 0; ++t) {
                int32_t c = rid[i * kc + t];
                if (c >= 0 && deg[c] < Rs) r = c;
            }
            rid[i * kc] = r;
            if (r >= 0 && !has_in[U[i]]) ++nz;
        }
        int added = 0;
        if (nz > 0) { /* U ascending: each r takes its points without in-edges, smallest first */
            for (int64_t i = 0; i < nu; ++i) {
                const int32_t r = rid[i * kc];
                if (r < 0 || has_in[U[i]] || deg[r] >= Rs) continue;
                adj[(int64_t)r * Rs + deg[r]] = U[i];
                deg[r] += 1;
                ++added;
            }
        } else {
            for (int64_t i = 0; i < nu; ++i) { /* the first p naming r is the smallest */
                const int32_t r = rid[i * kc];
                if (r >= 0 && best[r] < 0) best[r] = U[i];
            }
            for (int64_t r = 0; r < n; ++r) {
                if (best[r] < 0) continue;
                adj[r * Rs + deg[r]] = best[r];
                deg[r] += 1;
                ++added;
                best[r] = -1;
            }
        }
        free(Qm);
        free(rid);
        free(rd);
        if (added == 0) {
            rc = -3;
            break;
        }
        total += added;
    }
    free(reach);
    free(has_in);
    free(stack);
    free(U);
    free(best);
    if (rounds_out) *rounds_out = rounds;
    return rc < 0 ? rc : total;
}

/* ---- learned early stop (not in the paper): search-state features and traces ------------ */

/*
 * After hop t (t >= 1, the hop vertex u* explored and its neighbours merged into Q), with
 * lg(x) = ln(max(x, 1e-30)), D0 = D(q, s), D1 / Dk / DL the distances of Q[0], Q[min(k,|Q|)-1]
 * and Q[|Q|-1], du = D(q, u*), Dk_h[j] the Dk after hop j (Dk_h[0] = D0), tlc the last hop at
 * which the list of the first min(k, |Q|) ids changed (0 if never), U the unexplored entries
 * of Q and ins the points of this hop still in Q after it:
 *   f0 = lg D0          f1 = ln(1 + t)      f2 = lg D1 - lg D0   f3 = lg Dk - lg D0
 *   f4 = lg DL - lg D0  f5 = lg du - lg Dk
 *   f6..f11 = lg Dk_h[max(t - j, 0)] - lg Dk  for j = 1, 2, 4, 8, 16, 32
 *   f12 = ln(1 + t - tlc)   f13 = U / L   f14 = |Q| / L   f15 = ins / R
 * The label of hop t is 1 iff t >= tlc at the end of the search (the top-k list is final).
 */
#define OR_NF 16
#define OR_H 64
#define OR_NPARAMS (OR_H * OR_NF + OR_H + OR_H * OR_H + OR_H + OR_H + 1)

static double lgx(double x) { return log(x > 1e-30 ? x : 1e-30); }

/* model = params[OR_NPARAMS] followed by mu[16], sigma[16]; returns the logit. */
double or_mlp_logit(const double *model, const double *f) {
    const double *W1 = model, *b1 = W1 + OR_H * OR_NF, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H;
    const double *w3 = b2 + OR_H, *b3 = w3 + OR_H, *mu = model + OR_NPARAMS, *sg = mu + OR_NF;
    double x[OR_NF], h1[OR_H], h2[OR_H];
    for (int i = 0; i < OR_NF; ++i) x[i] = (f[i] - mu[i]) / sg[i];
    for (int o = 0; o < OR_H; ++o) {
        double a = b1[o];
        for (int i = 0; i < OR_NF; ++i) a = a + W1[o * OR_NF + i] * x[i];
        h1[o] = a > 0 ? a : 0;
    }
    for (int o = 0; o < OR_H; ++o) {
        double a = b2[o];
        for (int i = 0; i < OR_H; ++i) a = a + W2[o * OR_H + i] * h1[i];
        h2[o] = a > 0 ? a : 0;
    }
    double z = b3[0];
    for (int i = 0; i < OR_H; ++i) z = z + w3[i] * h2[i];
    return z;
}

/*
 * Alg. 1 as or_search, plus: per-hop features into feats[qi][t-1][16] for t <= max_trace
 * (when feats != NULL), the final tlc per query, and -- when model != NULL -- the learned stop:
 * after every hop t with t % check_every == 0 and t - tlc >= min_stable (the top-k ids unchanged
 * for min_stable hops) the search ends if or_mlp_logit >= zthr (stopped[qi] = 1).  Ids,
 * distances, ndc and hops as or_search.
 */
int or_search_ex(const float *X, int64_t n, int d, const int32_t *adj, const int32_t *deg, int R,
                 int32_t s, const float *Qv, int64_t nq, int k, int L, int max_trace, double *feats,
                 int32_t *tlc_out, const double *model, double zthr, int check_every,
                 int min_stable, int32_t *out_ids, double *out_d, int32_t *ndc_out, int32_t *hops_out,
                 int32_t *stopped) {
    if (n <= 0 || k <= 0 || L < k || s < 0 || s >= n || check_every < 1 || min_stable < 0)
        return OR_E_INVAL;
#pragma omp parallel
    {
        unsigned char *vis = (unsigned char *)calloc((size_t)n, 1);
        int32_t *touched = NULL;
        int64_t tcap = 0;
        or_qent *Q = (or_qent *)malloc(sizeof(or_qent) * (L + 1));
        int32_t *born = (int32_t *)malloc(sizeof(int32_t) * (L + 1));
        int32_t *prevk = (int32_t *)malloc(sizeof(int32_t) * k);
        int hcap = 1024;
        double *hist = (double *)malloc(sizeof(double) * hcap);
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const float *q = Qv + qi * (int64_t)d;
            int64_t nt = 0;
            int len = 1;
            Q[0].D = or_dist(q, X + (int64_t)s * d, d);
            Q[0].id = s;
            Q[0].explored = 0;
            born[0] = 0;
            vis[s] = 1;
            if (nt >= tcap) {
                tcap = tcap ? tcap * 2 : 4096;
                touched = (int32_t *)realloc(touched, sizeof(int32_t) * tcap);
            }
            touched[nt++] = s;
            const double D0 = Q[0].D;
            hist[0] = D0;
            int32_t ndc = 1, hops = 0, tlc = 0, stop = 0;
            for (;;) {
                int i = 0;
                while (i < len && Q[i].explored) ++i;
                if (i == len) break;
                Q[i].explored = 1;
                ++hops;
                const double du = Q[i].D;
                int32_t u = Q[i].id;
                int kk0 = len < k ? len : k;
                for (int t = 0; t < kk0; ++t) prevk[t] = Q[t].id;
                for (int j = 0; j < deg[u]; ++j) {
                    int32_t v = adj[(int64_t)u * R + j];
                    if (vis[v]) continue;
                    vis[v] = 1;
                    if (nt >= tcap) {
                        tcap *= 2;
                        touched = (int32_t *)realloc(touched, sizeof(int32_t) * tcap);
                    }
                    touched[nt++] = v;
                    ++ndc;
                    double D = or_dist(q, X + (int64_t)v * d, d);
                    if (len < L || key_less(D, v, Q[len - 1].D, Q[len - 1].id)) {
                        int pos = (len < L) ? len : L - 1;
                        while (pos > 0 && key_less(D, v, Q[pos - 1].D, Q[pos - 1].id)) {
                            Q[pos] = Q[pos - 1];
                            born[pos] = born[pos - 1];
                            --pos;
                        }
                        Q[pos].D = D;
                        Q[pos].id = v;
                        Q[pos].explored = 0;
                        born[pos] = hops;
                        if (len < L) ++len;
                    }
                }
                int kk = len < k ? len : k, changed = kk != kk0;
                for (int t = 0; t < kk && !changed; ++t) changed = Q[t].id != prevk[t];
                if (changed) tlc = hops;
                const double Dk = Q[kk - 1].D;
                if (hops >= hcap) {
                    hcap *= 2;
                    hist = (double *)realloc(hist, sizeof(double) * hcap);
                }
                hist[hops] = Dk;
                const int check = model && hops % check_every == 0 && hops - tlc >= min_stable;
                if ((feats && hops <= max_trace) || check) {
                    int U = 0, ins = 0;
                    for (int t = 0; t < len; ++t) {
                        U += !Q[t].explored;
                        ins += born[t] == hops;
                    }
                    double f[OR_NF];
                    const int lags[6] = {1, 2, 4, 8, 16, 32};
                    f[0] = lgx(D0);
                    f[1] = log(1.0 + hops);
                    f[2] = lgx(Q[0].D) - lgx(D0);
                    f[3] = lgx(Dk) - lgx(D0);
                    f[4] = lgx(Q[len - 1].D) - lgx(D0);
                    f[5] = lgx(du) - lgx(Dk);
                    for (int j = 0; j < 6; ++j) {
                        int h = hops - lags[j];
                        f[6 + j] = lgx(hist[h > 0 ? h : 0]) - lgx(Dk);
                    }
                    f[12] = log(1.0 + (hops - tlc));
                    f[13] = (double)U / L;
                    f[14] = (double)len / L;
                    f[15] = (double)ins / R;
                    if (feats && hops <= max_trace)
                        for (int j = 0; j < OR_NF; ++j)
                            feats[(qi * (int64_t)max_trace + (hops - 1)) * OR_NF + j] = f[j];
                    if (check && or_mlp_logit(model, f) >= zthr) {
                        stop = 1;
                        break;
                    }
                }
            }
            for (int t = 0; t < k; ++t) {
                if (out_ids) out_ids[qi * k + t] = t < len ? Q[t].id : -1;
                if (out_d) out_d[qi * k + t] = t < len ? Q[t].D : INFINITY;
            }
            if (ndc_out) ndc_out[qi] = ndc;
            if (hops_out) hops_out[qi] = hops;
            if (tlc_out) tlc_out[qi] = tlc;
            if (stopped) stopped[qi] = stop;
            for (int64_t t = 0; t < nt; ++t) vis[touched[t]] = 0;
        }
        free(vis);
        free(touched);
        free(Q);
        free(born);
        free(prevk);
        free(hist);
    }
    return OR_OK;
}

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
