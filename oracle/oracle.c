/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU oracle for graph-based
 * best-first approximate nearest-neighbour search (Speed-ANN, arXiv 2201.13007).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs load this library. The product library
 * (paper_2201_13007_gb300) never calls it, and the two share no code: no
 * header, no helper, no constant table.
 *
 * Every distance is evaluated in double precision on the float32 values the
 * caller passes (the stored, possibly already rounded, vectors). The total
 * order used everywhere (queue, top-M selection, ground truth, output) is
 * (key ascending, id ascending).
 *
 * What each function follows:
 *   orc_exact_knn   Def. 1 (NNS) and its K-NNS generalisation, Sec. 2.1:
 *                   the K points of P with the smallest distance to q,
 *                   by brute force over all n points.
 *   ALGO_BFIS       Algorithm 1 (Best-First Search, BFiS), Sec. 3.1.
 *   ALGO_TOPM       Sec. 4.1 parallel neighbour expansion: each step expands
 *                   the top-M unchecked candidates (bulk-synchronous, BFiS is
 *                   the M = 1 case), with the Sec. 4.2 staged schedule: M starts
 *                   at M0 and doubles every t steps up to M_max.
 *   ALGO_SPEEDANN   Algorithm 3 with Algorithm 2 (CheckMetrics, the
 *                   update-position test mean(U) >= L*R) as a deterministic
 *                   lock-step simulation of the walkers (Sec. 4.3); or, as
 *                   the merge test, the stall count (mean number of a
 *                   walker's expansions since the deal that inserted nothing
 *                   into its top L, against a patience P), one of the other
 *                   metrics Sec. 4.3 leaves open.
 *   orc_round_*     Storage formats for the reduced-precision variant:
 *                   IEEE binary16, bfloat16 (8-bit significand) and OCP FP8
 *                   E4M3 with a per-vector scale max|x|/448, each written from
 *                   the format's definition (round to nearest, ties to even).
 *   orc_rerank      Exact re-rank of a candidate list with FP32 base rows.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - the starting point P is marked visited when it is added (Alg. 1 adds P
 *     to S but never marks it);
 *   - ties in distance are broken by the smaller id;
 *   - distances are ranked and reported as squared L2; inner product uses
 *     key = -<q, x>;
 *   - "has unchecked vertices in S" is evaluated after the resize to L;
 *   - Alg. 3's deal is strided round-robin over the M active walkers in rank
 *     order; only unchecked entries move to the private queues; checked ones
 *     stay in S for the merge;
 *   - the update position is the 0-based rank of the best newly inserted
 *     candidate after the private queue's resize, or L when none survived;
 *     the mean is over walkers that received a non-empty deal; the checker is
 *     the (c mod #active)-th active walker and c advances by one each time the
 *     checker raises doMerge; the checker only tests in a sub-step in which it
 *     itself expanded a vertex (Alg. 3 places the test inside its loop body);
 *   - M doubles after every global step while M < T, capped at T.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_OOM -2

enum { ALGO_BFIS = 0, ALGO_TOPM = 1, ALGO_SPEEDANN = 2 };
enum { METRIC_L2 = 0, METRIC_IP = 1 };

typedef struct {
    const float *base; /* n x d row-major */
    int64_t n;
    int32_t d;
    const int32_t *adj; /* n x R, -1 = no edge */
    int32_t R;
    int64_t entry;
    int32_t metric;
} orc_graph;

typedef struct {
    int32_t L, K;
    int32_t M0, M_max, t;
    double R_ratio;    /* Alg. 2 position ratio; INFINITY = never merge early */
    int32_t merge_rule; /* 0 = Alg. 2 (mean update position >= L*R); 1 = stall count (below) */
    double patience;    /* rule 1: merge when the mean stall count reaches this; INFINITY = never */
    int64_t max_steps; /* stop after this many steps; < 0 = run to convergence */
    double tie_tol;    /* relative gap under which a boundary decision is logged */
    double tie_abs;    /* plus this absolute gap (inner-product keys can be near zero) */
} orc_params;

typedef struct {
    int64_t steps;      /* while-loop iterations (Alg. 1), BSP steps, or global steps (Alg. 3) */
    int64_t expansions; /* vertices marked checked and expanded */
    int64_t evals;      /* distance computations */
    int64_t merges;     /* Alg. 3 merges of the private queues */
    int64_t substeps;   /* Alg. 3 lock-step sub-steps */
    int64_t tie_events; /* near-ties at the selection, truncation or output boundary */
} orc_stats;

typedef struct {
    /* final queue S (capacity L) */
    int64_t *queue_ids;
    double *queue_keys;
    uint8_t *queue_checked;
    int32_t queue_len;
    /* visited vertices in visit order (capacity visited_cap) */
    int64_t *visited;
    int64_t n_visited;
    int64_t visited_cap;
    /* expanded vertices in expansion order (capacity expanded_cap) */
    int64_t *expanded;
    int64_t n_expanded;
    int64_t expanded_cap;
} orc_trace;

typedef struct {
    double key;
    int64_t id;
    int checked;
} entry_t;

/* ---------------------------------------------------------------- distances */

/* Sec. 2.1: delta(p, q) is the l2 distance; ranked here by its square.
 * Inner product (not in the paper) ranks by -<q, x>. */
static double key_of(const orc_graph *g, const float *q, int64_t u) {
    const float *x = g->base + (size_t)u * (size_t)g->d;
    double acc = 0.0;
    if (g->metric == METRIC_L2) {
        for (int32_t i = 0; i < g->d; ++i) {
            double diff = (double)q[i] - (double)x[i];
            acc += diff * diff;
        }
        return acc;
    }
    for (int32_t i = 0; i < g->d; ++i) acc += (double)q[i] * (double)x[i];
    return -acc;
}

static int entry_less(const entry_t *a, const entry_t *b) {
    if (a->key < b->key) return 1;
    if (a->key > b->key) return 0;
    return a->id < b->id;
}

static int entry_cmp(const void *pa, const void *pb) {
    const entry_t *a = (const entry_t *)pa, *b = (const entry_t *)pb;
    if (entry_less(a, b)) return -1;
    if (entry_less(b, a)) return 1;
    return 0;
}

static int near_tie_abs(double a, double b, double tol, double abs_tol) {
    double gap = fabs(b - a);
    double scale = fmax(fabs(a), fabs(b));
    return gap <= tol * scale + abs_tol;
}
#define near_tie(a, b, tol) near_tie_abs((a), (b), (tol), p->tie_abs)

/* Insert e into the sorted array q[0..*len) keeping (key, id) order. */
static void insert_sorted(entry_t *q, int32_t *len, entry_t e) {
    int32_t i = *len;
    while (i > 0 && entry_less(&e, &q[i - 1])) {
        q[i] = q[i - 1];
        --i;
    }
    q[i] = e;
    ++*len;
}

/* --------------------------------------------------------- per-query state */

typedef struct {
    uint8_t *visited_map; /* n bytes, all zero between queries */
    int64_t *visit_list;  /* vertices set in visited_map, for clearing */
    int64_t n_visit;
    int64_t visit_cap;
} vset_t;

static int vset_init(vset_t *v, int64_t n) {
    v->visited_map = (uint8_t *)calloc((size_t)n, 1);
    v->visit_cap = 1024;
    v->visit_list = (int64_t *)malloc(sizeof(int64_t) * (size_t)v->visit_cap);
    v->n_visit = 0;
    return (v->visited_map && v->visit_list) ? ORC_OK : ORC_ERR_OOM;
}

static void vset_free(vset_t *v) {
    free(v->visited_map);
    free(v->visit_list);
}

static void vset_clear(vset_t *v) {
    for (int64_t i = 0; i < v->n_visit; ++i) v->visited_map[v->visit_list[i]] = 0;
    v->n_visit = 0;
}

/* Marks u visited; returns 1 if it was not visited before. */
static int vset_add(vset_t *v, int64_t u) {
    if (v->visited_map[u]) return 0;
    v->visited_map[u] = 1;
    if (v->n_visit == v->visit_cap) {
        int64_t cap = v->visit_cap * 2;
        int64_t *p = (int64_t *)realloc(v->visit_list, sizeof(int64_t) * (size_t)cap);
        if (!p) return -1;
        v->visit_list = p;
        v->visit_cap = cap;
    }
    v->visit_list[v->n_visit++] = u;
    return 1;
}

static void trace_expanded(orc_trace *tr, int64_t v) {
    if (tr && tr->expanded && tr->n_expanded < tr->expanded_cap) tr->expanded[tr->n_expanded] = v;
    if (tr) tr->n_expanded++;
}

static void write_outputs(const entry_t *S, int32_t len, const orc_params *p, int64_t *ids,
                          double *keys, orc_stats *st, orc_trace *tr, const vset_t *vs) {
    for (int32_t i = 0; i < p->K; ++i) {
        if (i < len) {
            ids[i] = S[i].id;
            keys[i] = S[i].key;
        } else {
            ids[i] = -1;
            keys[i] = INFINITY;
        }
    }
    /* output boundary: rank K-1 vs rank K */
    if (len > p->K && p->K > 0 && near_tie(S[p->K - 1].key, S[p->K].key, p->tie_tol)) st->tie_events++;
    if (tr) {
        tr->queue_len = len;
        for (int32_t i = 0; i < len; ++i) {
            if (tr->queue_ids) tr->queue_ids[i] = S[i].id;
            if (tr->queue_keys) tr->queue_keys[i] = S[i].key;
            if (tr->queue_checked) tr->queue_checked[i] = (uint8_t)S[i].checked;
        }
        tr->n_visited = vs->n_visit;
        if (tr->visited) {
            int64_t m = vs->n_visit < tr->visited_cap ? vs->n_visit : tr->visited_cap;
            memcpy(tr->visited, vs->visit_list, sizeof(int64_t) * (size_t)m);
        }
    }
}

/* ------------------------------------------------------------- Algorithm 1 */

/* BFiS: repeatedly expand the first unchecked vertex of the sorted queue S,
 * add every not-yet-visited neighbour, then resize S to L (Algorithm 1). */
static int run_bfis(const orc_graph *g, const orc_params *p, const float *q, vset_t *vs,
                    int64_t *ids, double *keys, orc_stats *st, orc_trace *tr) {
    const int32_t L = p->L, R = g->R;
    entry_t *S = (entry_t *)malloc(sizeof(entry_t) * (size_t)(L + R + 1));
    if (!S) return ORC_ERR_OOM;
    int32_t len = 0;
    entry_t e0 = {key_of(g, q, g->entry), g->entry, 0};
    vset_add(vs, g->entry);
    st->evals++;
    insert_sorted(S, &len, e0);
    while (p->max_steps < 0 || st->steps < p->max_steps) {
        int32_t i = 0;
        while (i < len && S[i].checked) ++i;
        if (i == len) break; /* no unchecked vertex left */
        /* selection boundary: first vs second unchecked */
        for (int32_t j = i + 1; j < len; ++j)
            if (!S[j].checked) {
                if (near_tie(S[i].key, S[j].key, p->tie_tol)) st->tie_events++;
                break;
            }
        S[i].checked = 1;
        int64_t v = S[i].id;
        st->steps++;
        st->expansions++;
        trace_expanded(tr, v);
        for (int32_t r = 0; r < R; ++r) {
            int64_t u = g->adj[(size_t)v * (size_t)R + (size_t)r];
            if (u < 0) continue;
            int added = vset_add(vs, u);
            if (added < 0) { free(S); return ORC_ERR_OOM; }
            if (!added) continue;
            st->evals++;
            entry_t e = {key_of(g, q, u), u, 0};
            insert_sorted(S, &len, e);
        }
        if (len > L) {
            if (near_tie(S[L - 1].key, S[L].key, p->tie_tol)) st->tie_events++;
            len = L;
        }
    }
    write_outputs(S, len, p, ids, keys, st, tr, vs);
    free(S);
    return ORC_OK;
}

/* --------------------------------------------- Top-M with staged M (BSP) */

static int32_t next_m(int32_t M, const orc_params *p) {
    int64_t m2 = 2 * (int64_t)M;
    return (int32_t)(m2 < p->M_max ? m2 : p->M_max);
}

/* Each step: A = the first min(M, #unchecked) unchecked entries of S (rank
 * order) are marked checked; N = their neighbours not yet visited (a set);
 * S becomes the first L of S united with N in (key, id) order. M starts at M0
 * and doubles every t steps up to M_max (Sec. 4.1, 4.2). */
static int run_topm(const orc_graph *g, const orc_params *p, const float *q, vset_t *vs,
                    int64_t *ids, double *keys, orc_stats *st, orc_trace *tr) {
    const int32_t L = p->L, R = g->R, Mmax = p->M_max;
    entry_t *S = (entry_t *)malloc(sizeof(entry_t) * (size_t)(L + (int64_t)Mmax * R + 1));
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)Mmax);
    if (!S || !act) { free(S); free(act); return ORC_ERR_OOM; }
    int32_t len = 0;
    int32_t M = p->M0 < Mmax ? p->M0 : Mmax;
    S[len++] = (entry_t){key_of(g, q, g->entry), g->entry, 0};
    vset_add(vs, g->entry);
    st->evals++;
    while (p->max_steps < 0 || st->steps < p->max_steps) {
        int32_t na = 0, i = 0;
        for (; i < len && na < M; ++i)
            if (!S[i].checked) act[na++] = i;
        if (na == 0) break;
        /* selection boundary: the M-th chosen vs the next unchecked entry */
        for (; i < len; ++i)
            if (!S[i].checked) {
                if (near_tie(S[act[na - 1]].key, S[i].key, p->tie_tol)) st->tie_events++;
                break;
            }
        for (int32_t a = 0; a < na; ++a) {
            S[act[a]].checked = 1;
            st->expansions++;
            trace_expanded(tr, S[act[a]].id);
        }
        int32_t grown = len;
        for (int32_t a = 0; a < na; ++a) {
            int64_t v = S[act[a]].id;
            for (int32_t r = 0; r < R; ++r) {
                int64_t u = g->adj[(size_t)v * (size_t)R + (size_t)r];
                if (u < 0) continue;
                int added = vset_add(vs, u);
                if (added < 0) { free(S); free(act); return ORC_ERR_OOM; }
                if (!added) continue;
                st->evals++;
                S[grown++] = (entry_t){key_of(g, q, u), u, 0};
            }
        }
        qsort(S, (size_t)grown, sizeof(entry_t), entry_cmp);
        len = grown;
        if (len > L) {
            if (near_tie(S[L - 1].key, S[L].key, p->tie_tol)) st->tie_events++;
            len = L;
        }
        st->steps++;
        if (st->steps % p->t == 0) M = next_m(M, p);
    }
    write_outputs(S, len, p, ids, keys, st, tr, vs);
    free(S);
    free(act);
    return ORC_OK;
}

/* ------------------------------------------ Algorithm 3 (+ Algorithm 2) */

/* Algorithm 2, CheckMetrics: true when the mean update position reaches L*R. */
static int check_metrics(const int32_t *U, const uint8_t *active, int32_t M, int32_t L, double Rr) {
    double sum = 0.0;
    int32_t cnt = 0;
    for (int32_t w = 0; w < M; ++w)
        if (active[w]) {
            sum += (double)U[w];
            cnt++;
        }
    if (cnt == 0) return 0;
    return sum / (double)cnt >= (double)L * Rr;
}

/* The stall-count merge test (an alternative to CheckMetrics; Sec. 4.3 leaves
 * the choice of metric open): stall[w] counts the expansions walker w made
 * since the deal that put no new candidate into the first L entries of its
 * private queue (update position L). True when the mean over the walkers that
 * received a non-empty deal reaches the patience P. */
static int check_stall(const int32_t *stall, const uint8_t *active, int32_t M, double P) {
    double sum = 0.0;
    int32_t cnt = 0;
    for (int32_t w = 0; w < M; ++w)
        if (active[w]) {
            sum += (double)stall[w];
            cnt++;
        }
    if (cnt == 0) return 0;
    return sum / (double)cnt >= P;
}

/* Deterministic simulation of Algorithm 3: a global queue S and T private
 * queues. Each global step deals S's unchecked entries to the M walkers;
 * walkers then advance in lock-step sub-steps, in walker order, each running
 * one local best-first expansion against the shared visited set; after each
 * sub-step the checker evaluates CheckMetrics and may raise doMerge. When
 * doMerge is raised or every private queue is exhausted, the private queues
 * merge into S, S is resized to L and M doubles while M < T. */
static int run_speedann(const orc_graph *g, const orc_params *p, const float *q, vset_t *vs,
                        int64_t *ids, double *keys, orc_stats *st, orc_trace *tr) {
    const int32_t L = p->L, R = g->R, T = p->M_max;
    const int32_t cap = L + R + 1;
    entry_t *S = (entry_t *)malloc(sizeof(entry_t) * (size_t)(L + 1));
    entry_t *LS = (entry_t *)malloc(sizeof(entry_t) * (size_t)cap * (size_t)T);
    int32_t *lsn = (int32_t *)calloc((size_t)T, sizeof(int32_t));
    int32_t *U = (int32_t *)calloc((size_t)T, sizeof(int32_t));
    int32_t *stall = (int32_t *)calloc((size_t)T, sizeof(int32_t));
    uint8_t *active = (uint8_t *)calloc((size_t)T, 1);
    entry_t *pool = (entry_t *)malloc(sizeof(entry_t) * ((size_t)L + (size_t)cap * (size_t)T));
    int32_t *act_list = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
    int64_t *new_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    if (!S || !LS || !lsn || !U || !stall || !active || !pool || !act_list || !new_ids) {
        free(S); free(LS); free(lsn); free(U); free(stall); free(active); free(pool); free(act_list); free(new_ids);
        return ORC_ERR_OOM;
    }
    int32_t len = 0;
    int32_t M = p->M0 < T ? p->M0 : T;
    int64_t checker = 0;
    S[len++] = (entry_t){key_of(g, q, g->entry), g->entry, 0};
    vset_add(vs, g->entry);
    st->evals++;
    int rc = ORC_OK;
    while (p->max_steps < 0 || st->steps < p->max_steps) {
        /* deal: unchecked entries of S go round-robin, by rank, to the M walkers */
        for (int32_t w = 0; w < M; ++w) { lsn[w] = 0; U[w] = 0; stall[w] = 0; active[w] = 0; }
        int32_t kept = 0, dealt = 0;
        for (int32_t i = 0; i < len; ++i) {
            if (S[i].checked) {
                S[kept++] = S[i];
            } else {
                int32_t w = dealt % M;
                LS[(size_t)w * cap + lsn[w]++] = S[i];
                dealt++;
            }
        }
        len = kept;
        if (dealt == 0) break; /* all private queues empty */
        int32_t nactive = 0;
        for (int32_t w = 0; w < M; ++w)
            if (lsn[w] > 0) { active[w] = 1; act_list[nactive++] = w; }
        int32_t chk = act_list[checker % nactive];
        int do_merge = 0;
        while (!do_merge) {
            int any = 0, checker_expanded = 0;
            for (int32_t w = 0; w < M; ++w) {
                entry_t *Q = LS + (size_t)w * cap;
                int32_t i = 0;
                while (i < lsn[w] && Q[i].checked) ++i;
                if (i == lsn[w]) continue;
                any = 1;
                if (w == chk) checker_expanded = 1;
                Q[i].checked = 1;
                int64_t v = Q[i].id;
                st->expansions++;
                trace_expanded(tr, v);
                int32_t n_new = 0;
                for (int32_t r = 0; r < R; ++r) {
                    int64_t u = g->adj[(size_t)v * (size_t)R + (size_t)r];
                    if (u < 0) continue;
                    int added = vset_add(vs, u);
                    if (added < 0) { rc = ORC_ERR_OOM; goto done; }
                    if (!added) continue;
                    st->evals++;
                    insert_sorted(Q, &lsn[w], (entry_t){key_of(g, q, u), u, 0});
                    new_ids[n_new++] = u;
                }
                if (lsn[w] > L) lsn[w] = L;
                /* update position: best rank of a newly inserted entry, else L */
                int32_t upos = L;
                for (int32_t j = 0; j < lsn[w] && upos == L; ++j)
                    for (int32_t k = 0; k < n_new; ++k)
                        if (Q[j].id == new_ids[k]) { upos = j; break; }
                U[w] = upos;
                if (upos == L) stall[w]++;
            }
            if (!any) break;
            st->substeps++;
            const int test = p->merge_rule == 1 ? check_stall(stall, active, M, p->patience)
                                                : check_metrics(U, active, M, L, p->R_ratio);
            if (checker_expanded && test) {
                do_merge = 1;
                checker++;
            }
        }
        /* merge: S's checked entries with every private queue, dedupe by id
         * (a checked copy wins), sort, resize to L */
        int32_t np = 0;
        for (int32_t i = 0; i < len; ++i) pool[np++] = S[i];
        for (int32_t w = 0; w < M; ++w)
            for (int32_t i = 0; i < lsn[w]; ++i) pool[np++] = LS[(size_t)w * cap + i];
        qsort(pool, (size_t)np, sizeof(entry_t), entry_cmp);
        int32_t nu = 0;
        for (int32_t i = 0; i < np; ++i) {
            if (nu > 0 && pool[nu - 1].id == pool[i].id) {
                pool[nu - 1].checked |= pool[i].checked;
                continue;
            }
            pool[nu++] = pool[i];
        }
        len = nu < L ? nu : L;
        for (int32_t i = 0; i < len; ++i) S[i] = pool[i];
        st->merges++;
        st->steps++;
        if (M < T) M = (2 * M < T) ? 2 * M : T;
    }
    write_outputs(S, len, p, ids, keys, st, tr, vs);
done:
    free(S); free(LS); free(lsn); free(U); free(stall); free(active); free(pool); free(act_list); free(new_ids);
    return rc;
}

/* --------------------------------------------------------------- dispatch */

static int check_graph(const orc_graph *g) {
    if (!g || !g->base || !g->adj || g->n <= 0 || g->d <= 0 || g->R <= 0) return ORC_ERR_ARG;
    if (g->entry < 0 || g->entry >= g->n) return ORC_ERR_ARG;
    if (g->metric != METRIC_L2 && g->metric != METRIC_IP) return ORC_ERR_ARG;
    for (int64_t i = 0; i < g->n * (int64_t)g->R; ++i)
        if (g->adj[i] < -1 || (int64_t)g->adj[i] >= g->n) return ORC_ERR_ARG;
    return ORC_OK;
}

static int check_params(int32_t algo, const orc_params *p) {
    if (!p || p->L < 1 || p->K < 1 || p->K > p->L) return ORC_ERR_ARG;
    if (algo == ALGO_TOPM || algo == ALGO_SPEEDANN) {
        if (p->M0 < 1 || p->M_max < 1 || p->t < 1) return ORC_ERR_ARG;
    }
    if (algo == ALGO_SPEEDANN && !(p->R_ratio >= 0.0)) return ORC_ERR_ARG;
    if (algo == ALGO_SPEEDANN && (p->merge_rule < 0 || p->merge_rule > 1 || !(p->patience >= 0.0)))
        return ORC_ERR_ARG;
    if (algo < ALGO_BFIS || algo > ALGO_SPEEDANN) return ORC_ERR_ARG;
    return ORC_OK;
}

static int run_one(int32_t algo, const orc_graph *g, const orc_params *p, const float *q,
                   vset_t *vs, int64_t *ids, double *keys, orc_stats *st, orc_trace *tr) {
    memset(st, 0, sizeof(*st));
    if (tr) tr->n_expanded = 0;
    int rc;
    if (algo == ALGO_BFIS) rc = run_bfis(g, p, q, vs, ids, keys, st, tr);
    else if (algo == ALGO_TOPM) rc = run_topm(g, p, q, vs, ids, keys, st, tr);
    else rc = run_speedann(g, p, q, vs, ids, keys, st, tr);
    vset_clear(vs);
    return rc;
}

/* One query with a full trace (final queue, visited set, expansion order). */
int orc_search_trace(int32_t algo, const orc_graph *g, const orc_params *p, const float *q,
                     int64_t *ids, double *keys, orc_stats *st, orc_trace *tr) {
    int rc = check_graph(g);
    if (rc == ORC_OK) rc = check_params(algo, p);
    if (rc != ORC_OK) return rc;
    vset_t vs;
    if (vset_init(&vs, g->n) != ORC_OK) { vset_free(&vs); return ORC_ERR_OOM; }
    rc = run_one(algo, g, p, q, &vs, ids, keys, st, tr);
    vset_free(&vs);
    return rc;
}

typedef struct {
    int32_t algo;
    const orc_graph *g;
    const orc_params *p;
    const float *queries;
    int64_t nq;
    int64_t *ids;
    double *keys;
    orc_stats *stats;
    int32_t tid, nthreads;
    int rc;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *j = (batch_job *)arg;
    vset_t vs;
    if (vset_init(&vs, j->g->n) != ORC_OK) { vset_free(&vs); j->rc = ORC_ERR_OOM; return NULL; }
    for (int64_t i = j->tid; i < j->nq; i += j->nthreads) {
        int rc = run_one(j->algo, j->g, j->p, j->queries + (size_t)i * (size_t)j->g->d, &vs,
                         j->ids + (size_t)i * (size_t)j->p->K, j->keys + (size_t)i * (size_t)j->p->K,
                         &j->stats[i], NULL);
        if (rc != ORC_OK) { j->rc = rc; break; }
    }
    vset_free(&vs);
    return NULL;
}

/* nq independent queries, spread over nthreads host threads (strided). */
int orc_search(int32_t algo, const orc_graph *g, const orc_params *p, const float *queries,
               int64_t nq, int64_t *ids, double *keys, orc_stats *stats, int32_t nthreads) {
    int rc = check_graph(g);
    if (rc == ORC_OK) rc = check_params(algo, p);
    if (rc != ORC_OK) return rc;
    if (nq < 0) return ORC_ERR_ARG;
    if (nq == 0) return ORC_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nq) nthreads = (int32_t)nq;
    batch_job *jobs = (batch_job *)calloc((size_t)nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORC_ERR_OOM; }
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t] = (batch_job){algo, g, p, queries, nq, ids, keys, stats, t, nthreads, ORC_OK};
        if (nthreads == 1) batch_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    if (nthreads > 1)
        for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int32_t t = 0; t < nthreads; ++t)
        if (jobs[t].rc != ORC_OK) rc = jobs[t].rc;
    free(jobs);
    free(th);
    return rc;
}

/* ----------------------------------------------------- exact ground truth */

typedef struct {
    const orc_graph *g;
    const float *queries;
    int64_t nq;
    int32_t K;
    int64_t *ids;
    double *keys;
    int32_t tid, nthreads;
} knn_job;

static void *knn_worker(void *arg) {
    knn_job *j = (knn_job *)arg;
    entry_t *best = (entry_t *)malloc(sizeof(entry_t) * (size_t)(j->K + 1));
    if (!best) return NULL;
    for (int64_t qi = j->tid; qi < j->nq; qi += j->nthreads) {
        const float *q = j->queries + (size_t)qi * (size_t)j->g->d;
        int32_t len = 0;
        for (int64_t u = 0; u < j->g->n; ++u) {
            entry_t e = {key_of(j->g, q, u), u, 1};
            if (len == j->K && !entry_less(&e, &best[len - 1])) continue;
            insert_sorted(best, &len, e);
            if (len > j->K) len = j->K;
        }
        for (int32_t i = 0; i < j->K; ++i) {
            j->ids[(size_t)qi * j->K + i] = i < len ? best[i].id : -1;
            j->keys[(size_t)qi * j->K + i] = i < len ? best[i].key : INFINITY;
        }
    }
    free(best);
    return NULL;
}

/* Def. 1 (K-NNS): the K points of P nearest to q, by brute force. */
int orc_exact_knn(const orc_graph *g, const float *queries, int64_t nq, int32_t K, int64_t *ids,
                  double *keys, int32_t nthreads) {
    if (!g || !g->base || g->n <= 0 || g->d <= 0 || K < 1 || nq < 0) return ORC_ERR_ARG;
    if (g->metric != METRIC_L2 && g->metric != METRIC_IP) return ORC_ERR_ARG;
    if (nq == 0) return ORC_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nq) nthreads = (int32_t)nq;
    knn_job *jobs = (knn_job *)calloc((size_t)nthreads, sizeof(knn_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORC_ERR_OOM; }
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t] = (knn_job){g, queries, nq, K, ids, keys, t, nthreads};
        if (nthreads == 1) knn_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, knn_worker, &jobs[t]);
    }
    if (nthreads > 1)
        for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return ORC_OK;
}

/* ------------------------------------------------------------- re-rank */

/* Recompute each candidate's key from the FP32 rows in g->base, sort by
 * (key, id) and keep the first K; -1 candidates are skipped, missing slots
 * are padded with (-1, +inf). cand is nq x ncand. */
int orc_rerank(const orc_graph *g, const float *queries, int64_t nq, const int64_t *cand,
               int32_t ncand, int32_t K, int64_t *ids, double *keys) {
    if (!g || !g->base || g->n <= 0 || g->d <= 0 || K < 1 || ncand < 0 || nq < 0) return ORC_ERR_ARG;
    entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(ncand + 1));
    if (!buf) return ORC_ERR_OOM;
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = queries + (size_t)qi * (size_t)g->d;
        int32_t m = 0;
        for (int32_t c = 0; c < ncand; ++c) {
            int64_t u = cand[(size_t)qi * ncand + c];
            if (u < 0) continue;
            if (u >= g->n) { free(buf); return ORC_ERR_ARG; }
            buf[m++] = (entry_t){key_of(g, q, u), u, 1};
        }
        qsort(buf, (size_t)m, sizeof(entry_t), entry_cmp);
        for (int32_t i = 0; i < K; ++i) {
            ids[(size_t)qi * K + i] = i < m ? buf[i].id : -1;
            keys[(size_t)qi * K + i] = i < m ? buf[i].key : INFINITY;
        }
    }
    free(buf);
    return ORC_OK;
}

/* ------------------------------------------------------- storage formats */

/* Round x to a binary floating-point format with p significand bits
 * (including the implicit one), minimum normal exponent emin, to nearest with
 * ties to even. Values below 2^emin use the fixed subnormal quantum
 * 2^(emin - p + 1). x/quantum is exact (power-of-two scaling) and rint()
 * rounds ties to even in the default rounding mode. */
static double round_to_format(double x, int p, int emin) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(fabs(x), &e); /* |x| = f * 2^e, f in [0.5, 1) -> leading bit at 2^(e-1) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    double quantum = ldexp(1.0, lead - (p - 1));
    return rint(x / quantum) * quantum;
}

/* bfloat16: 8 significand bits, 8 exponent bits (same range as binary32). */
static float to_bf16(float x) {
    if (isnan(x) || isinf(x)) return x;
    double r = round_to_format((double)x, 8, -126);
    if (fabs(r) > 3.3895313892515355e38) return copysignf(INFINITY, x); /* above the largest finite bf16 */
    return (float)r;
}

/* IEEE binary16: 11 significand bits, emin = -14, largest finite 65504. */
static float to_fp16(float x) {
    if (isnan(x) || isinf(x)) return x;
    double r = round_to_format((double)x, 11, -14);
    if (fabs(r) > 65504.0) return copysignf(INFINITY, x);
    return (float)r;
}

/* OCP FP8 E4M3: 4 significand bits, emin = -6, largest finite 448, no
 * infinity; out-of-range values saturate to +-448. */
static float to_e4m3_sat(float x) {
    if (isnan(x)) return x;
    double r = round_to_format((double)x, 4, -6);
    if (r > 448.0) r = 448.0;
    if (r < -448.0) r = -448.0;
    return (float)r;
}

int orc_round_bf16(const float *x, int64_t cnt, float *out) {
    for (int64_t i = 0; i < cnt; ++i) out[i] = to_bf16(x[i]);
    return ORC_OK;
}

int orc_round_fp16(const float *x, int64_t cnt, float *out) {
    for (int64_t i = 0; i < cnt; ++i) out[i] = to_fp16(x[i]);
    return ORC_OK;
}

int orc_round_e4m3(const float *x, int64_t cnt, float *out) {
    for (int64_t i = 0; i < cnt; ++i) out[i] = to_e4m3_sat(x[i]);
    return ORC_OK;
}

/* Per-vector scaled FP8: scale_u = max_i |x_ui| / 448 (float32 division),
 * code = E4M3(x_ui / scale_u) (float32 division, then rounding), and the
 * value the search sees is the float32 product scale_u * code. A zero row
 * keeps scale 1 and codes 0. */
int orc_fp8_scaled(const float *x, int64_t n, int32_t d, float *dequant, float *scales) {
    for (int64_t u = 0; u < n; ++u) {
        const float *row = x + (size_t)u * (size_t)d;
        float mx = 0.0f;
        for (int32_t i = 0; i < d; ++i) {
            float a = fabsf(row[i]);
            if (a > mx) mx = a;
        }
        volatile float s = mx > 0.0f ? mx / 448.0f : 1.0f;
        scales[u] = s;
        for (int32_t i = 0; i < d; ++i) {
            volatile float ratio = row[i] / s;
            float code = to_e4m3_sat(ratio);
            volatile float v = s * code;
            dequant[(size_t)u * (size_t)d + i] = v;
        }
    }
    return ORC_OK;
}
