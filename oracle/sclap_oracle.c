/*
 * sclap_oracle.c -- plain, slow CPU oracle (one thread by default; built
 * with OpenMP, or_set_threads splits each sub-round's independent per-node
 * propose loop over threads, which cannot change any result).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by
 * the CPU-baseline leg of the benchmark; never by the product path.
 *
 * The code follows the paper's description step by step, with no blocking,
 * fusion or reordering beyond what the (deterministic) reading states:
 *
 *  - Sec. III.A: a node is moved to the eligible neighbouring block with the
 *    strongest connection; a block is eligible if it is not overloaded once
 *    the node has moved (bound U while clustering, L_max while refining);
 *    a node of an overloaded block ignores its own block.
 *  - Sec. IV.B: exact block weights when refining.
 *  - Sec. IV.C: contraction through the prefix-sum map q and C(v) = q(label).
 *  - Sec. IV.E: l rounds per coarsening level, initial partition of the
 *    coarsest graph, projection and r rounds per uncoarsening level.
 *
 * Deterministic reading (the paper visits nodes sequentially in random or
 * degree order and breaks ties randomly):
 *  R1  every round has S synchronous sub-rounds, a fresh random split of the
 *      nodes per round (the paper visits the nodes in a new random order
 *      each round): with h = mix64(seed ^ ((round+1) << 32) ^ v), node v
 *      belongs to sub-round colour(v) = (h >> 32) mod S and proposes against
 *      the state at the start of its sub-round.
 *  R2  candidates are the labels of v's neighbours other than its own; label
 *      L is eligible iff W(L) + c(v) <= B.  The best candidate maximises
 *      omega(v,L), then minimises tie(v,L) = high 32 bits of mix64(h ^ L),
 *      then L.
 *      v proposes iff gain = omega(v,best) - omega(v,own) > 0, or, when
 *      refining, iff its own block is overloaded (then gain may be <= 0).
 *  R3  departures from an overloaded block are admitted in (gain desc,
 *      id asc) order while the weight departed before them is below the
 *      excess W(own) - B.
 *  R4  proposals to a target T surviving R3 are admitted in (gain desc,
 *      id asc) order iff c(v) == 0 or the inclusive prefix of c in that
 *      order is <= B - W(T) (weights at sub-round start).
 *  R5  admitted moves are applied together; a round ends early after the
 *      first round without moves.
 *  R6  clustering only: nodes without neighbours are packed into clusters
 *      of weight <= U after the rounds (see pack_isolated).
 * mix64 is the SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
 */
#include "sclap_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* hashing (R1, R2)                                                     */
/* ------------------------------------------------------------------ */

uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* h(v, round): the per-round hash of node v that fixes its sub-round and
 * seeds its tie-breaks (R1, R2). */
static uint64_t node_hash(uint64_t seed, int32_t round, int64_t v)
{
    return or_mix64(seed ^ ((uint64_t)(round + 1) << 32) ^ (uint64_t)v);
}

uint32_t or_colour(uint64_t seed, int32_t round, int64_t v, int32_t S)
{
    return (uint32_t)(node_hash(seed, round, v) >> 32) % (uint32_t)S;
}

uint32_t or_tie(uint64_t seed, int32_t round, int64_t v, int64_t L)
{
    return (uint32_t)(or_mix64(node_hash(seed, round, v) ^ (uint64_t)L) >> 32);
}

/* Sec. II.A: L_max := (1 + eps) * ceil(c(V) / k), rounded down to an integer
 * because all weights are integers. */
int64_t or_lmax(int64_t cV, int32_t k, double eps)
{
    int64_t avg = (cV + k - 1) / k;
    return (int64_t)floor((1.0 + eps) * (double)avg);
}

/* ------------------------------------------------------------------ */
/* graph validation (Sec. II.A: undirected, omega > 0, c >= 0)          */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t u, v;
    int32_t w;
} edge_rec;

static int cmp_edge(const void *a, const void *b)
{
    const edge_rec *x = (const edge_rec *)a, *y = (const edge_rec *)b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

int or_validate(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *adjwgt, const int32_t *vwgt)
{
    if (n < 0) return OR_EINVAL;
    if (xadj[0] != 0) return OR_EGRAPH;
    for (int64_t v = 0; v < n; v++)
        if (xadj[v + 1] < xadj[v]) return OR_EGRAPH;
    int64_t nnz = xadj[n];
    for (int64_t v = 0; v < n; v++)
        if (vwgt[v] < 0) return OR_EGRAPH;
    edge_rec *e = (edge_rec *)malloc(sizeof(edge_rec) * (size_t)(nnz ? nnz : 1));
    if (!e) return OR_ENOMEM;
    int rc = OR_OK;
    for (int64_t v = 0; v < n && rc == OR_OK; v++)
        for (int64_t i = xadj[v]; i < xadj[v + 1]; i++) {
            int64_t u = adjncy[i];
            if (u < 0 || u >= n || u == v || adjwgt[i] <= 0) { rc = OR_EGRAPH; break; }
            e[i].u = v; e[i].v = u; e[i].w = adjwgt[i];
        }
    if (rc == OR_OK) {
        qsort(e, (size_t)nnz, sizeof(edge_rec), cmp_edge);
        for (int64_t i = 1; i < nnz; i++)
            if (e[i].u == e[i - 1].u && e[i].v == e[i - 1].v) { rc = OR_EGRAPH; break; }
    }
    if (rc == OR_OK) {
        /* symmetry: every (v,u,w) has its mirror (u,v,w) */
        for (int64_t i = 0; i < nnz; i++) {
            edge_rec key = {e[i].v, e[i].u, 0};
            edge_rec *m = (edge_rec *)bsearch(&key, e, (size_t)nnz, sizeof(edge_rec), cmp_edge);
            if (!m || m->w != e[i].w) { rc = OR_EGRAPH; break; }
        }
    }
    free(e);
    return rc;
}

/* ------------------------------------------------------------------ */
/* one synchronous round of size-constrained label propagation          */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t v;
    int64_t target, own;
    int64_t gain;
    int64_t c;
    int keep;
} proposal;

static int cmp_by_source(const void *a, const void *b)
{
    const proposal *x = (const proposal *)a, *y = (const proposal *)b;
    if (x->own != y->own) return x->own < y->own ? -1 : 1;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
    return x->v < y->v ? -1 : (x->v > y->v);
}

static int cmp_by_target(const void *a, const void *b)
{
    const proposal *x = (const proposal *)a, *y = (const proposal *)b;
    if (x->target != y->target) return x->target < y->target ? -1 : 1;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
    return x->v < y->v ? -1 : (x->v > y->v);
}

/* Runs of a batch refined together over the disjoint union of their graphs
 * (Sec. II.C / IV.E: the individuals of a population are independent).  Node
 * v of the union belongs to run run_of[v]; that run's nodes are off[r] ..
 * off[r] + n_r - 1 and its blocks r*k .. r*k + k - 1.  Its sub-rounds and
 * tie-breaks use its own seed seed[r] with its local node id v - off[r] and
 * local block id L - r*k, so a run's result does not depend on the other runs
 * of the batch or on its position in it.  NULL: one graph, one seed. */
typedef struct {
    const int32_t *run_of;
    const uint64_t *seed;
    const int64_t *off;
    int32_t k;
} run_map;

/* Workspace of the rounds.  The proposals of one sub-round are computed
 * node by node against the same state, so nodes are independent: with
 * OpenMP (or_set_threads) each of nthr threads takes a contiguous range of
 * nodes with its own acc / touched / proposal list, and the lists are joined
 * before arbitration, which orders proposals totally, so the result does not
 * depend on the number of threads. */
typedef struct {
    int nthr;
    int64_t **acc;      /* per thread: omega(v, L) for the node being visited, size nW */
    int64_t **touched;  /* per thread: labels with acc != 0                             */
    proposal **tp;      /* per thread: its proposals of the current sub-round           */
    int64_t *tnp;
    proposal *props;    /* all proposals of the sub-round                               */
} lp_ws;

static int g_threads = 1;

void or_set_threads(int t) { g_threads = t < 1 ? 1 : t; }

int or_get_threads(void)
{
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

static void ws_free(lp_ws *ws)
{
    for (int t = 0; t < ws->nthr; t++) {
        if (ws->acc) free(ws->acc[t]);
        if (ws->touched) free(ws->touched[t]);
        if (ws->tp) free(ws->tp[t]);
    }
    free(ws->acc); free(ws->touched); free(ws->tp); free(ws->tnp); free(ws->props);
    memset(ws, 0, sizeof(*ws));
}

static int ws_alloc(lp_ws *ws, int64_t n, int64_t nW)
{
    memset(ws, 0, sizeof(*ws));
    ws->nthr = or_get_threads();
    ws->acc = (int64_t **)calloc((size_t)ws->nthr, sizeof(int64_t *));
    ws->touched = (int64_t **)calloc((size_t)ws->nthr, sizeof(int64_t *));
    ws->tp = (proposal **)calloc((size_t)ws->nthr, sizeof(proposal *));
    ws->tnp = (int64_t *)calloc((size_t)ws->nthr, sizeof(int64_t));
    ws->props = (proposal *)malloc(sizeof(proposal) * (size_t)(n ? n : 1));
    if (!ws->acc || !ws->touched || !ws->tp || !ws->tnp || !ws->props) { ws_free(ws); return OR_ENOMEM; }
    int64_t per = n / ws->nthr + 2;
    for (int t = 0; t < ws->nthr; t++) {
        ws->acc[t] = (int64_t *)calloc((size_t)(nW ? nW : 1), sizeof(int64_t));
        ws->touched[t] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nW ? nW : 1));
        ws->tp[t] = (proposal *)malloc(sizeof(proposal) * (size_t)per);
        if (!ws->acc[t] || !ws->touched[t] || !ws->tp[t]) { ws_free(ws); return OR_ENOMEM; }
    }
    return OR_OK;
}

/* One round (R1-R5).  lab: label per node; W: weight per label (nW labels);
 * B: U (clustering) or L_max (refinement).  Returns the moves applied. */
/* Bound of label L: Bv[L] when per-label bounds are given (batched runs, one
 * L_max per run), else B. */
static int64_t bound_of(const int64_t *Bv, int64_t B, int64_t L)
{
    return Bv ? Bv[L] : B;
}

typedef struct {
    int64_t deg;
    uint32_t h;
    int64_t v;
} deg_key;

static int cmp_deg_key(const void *a, const void *b)
{
    const deg_key *x = (const deg_key *)a, *y = (const deg_key *)b;
    if (x->deg != y->deg) return x->deg < y->deg ? -1 : 1;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/* Degree-ordered sub-rounds of round r: the nodes in (degree asc, high 32
 * bits of h(v,r) asc, v asc) order; the node at position p acts in sub-round
 * floor(p * S / n), so low-degree nodes act first (Sec. III.A visits nodes
 * in increasing degree) and the S groups differ in size by at most one. */
int or_degree_colours(int64_t n, const int64_t *xadj, uint64_t seed, int32_t round, int32_t S,
                      int32_t *colour_out)
{
    deg_key *k = (deg_key *)malloc(sizeof(deg_key) * (size_t)(n ? n : 1));
    if (!k) return OR_ENOMEM;
    for (int64_t v = 0; v < n; v++) {
        k[v].deg = xadj[v + 1] - xadj[v];
        k[v].h = (uint32_t)(node_hash(seed, round, v) >> 32);
        k[v].v = v;
    }
    qsort(k, (size_t)n, sizeof(deg_key), cmp_deg_key);
    for (int64_t p = 0; p < n; p++) colour_out[k[p].v] = (int32_t)(p * S / n);
    free(k);
    return OR_OK;
}

static int64_t lp_round(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                        const int32_t *adjwgt, const int32_t *vwgt, int32_t *lab,
                        int64_t *W, int64_t B, const int64_t *Bv, int refine,
                        const int32_t *cp, uint64_t seed, int32_t round, int32_t S,
                        const uint8_t *active, const int32_t *colour, const run_map *rm,
                        int64_t *vis_best, int64_t *vis_own, lp_ws *ws)
{
    int64_t moves = 0;
    for (int32_t j = 0; j < S; j++) {
        /* --- every node of colour j proposes against the current state --- */
        for (int t = 0; t < ws->nthr; t++) ws->tnp[t] = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(ws->nthr)
#endif
        {
#ifdef _OPENMP
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
#else
        const int t = 0, T = 1;
#endif
        int64_t *acc = ws->acc[t], *touched = ws->touched[t];
        /* chunk c: nodes [n c / nthr, n (c + 1) / nthr), proposals into tp[c] */
        for (int c = t; c < ws->nthr; c += T) {
        int64_t tn = 0;
        for (int64_t v = n * c / ws->nthr; v < n * (c + 1) / ws->nthr; v++) {
            /* the seed, node id and block-id base that key v's hashes */
            uint64_t sv = seed;
            int64_t lv = v, lb = 0;
            if (rm) {
                int32_t r = rm->run_of[v];
                sv = rm->seed[r];
                lv = v - rm->off[r];
                lb = (int64_t)r * rm->k;
            }
            if ((colour ? colour[v] : (int32_t)or_colour(sv, round, lv, S)) != j) continue;
            if (xadj[v + 1] == xadj[v]) continue;  /* no neighbours: never moves */
            if (active && !active[v]) continue;    /* learned form: not visited */
            int64_t nt = 0;
            for (int64_t i = xadj[v]; i < xadj[v + 1]; i++) {
                int64_t u = adjncy[i];
                if (cp && cp[u] != cp[v]) continue;  /* V-cycle restriction */
                int64_t L = lab[u];
                if (acc[L] == 0) touched[nt++] = L;
                acc[L] += adjwgt[i];
            }
            int64_t own = lab[v];
            int64_t w_own = acc[own];
            int overloaded = refine && W[own] > bound_of(Bv, B, own);
            int64_t best = -1;
            uint32_t best_tie = 0;
            for (int64_t q = 0; q < nt; q++) {
                int64_t L = touched[q];
                if (L == own) continue;
                if (W[L] + vwgt[v] > bound_of(Bv, B, L)) continue; /* not eligible */
                uint32_t tl = or_tie(sv, round, lv, L - lb);
                int better;
                if (best < 0) better = 1;
                else if (acc[L] != acc[best]) better = acc[L] > acc[best];
                else if (tl != best_tie) better = tl < best_tie;
                else better = L < best;
                if (better) { best = L; best_tie = tl; }
            }
            if (vis_best) {  /* learned form: what this visit saw (R12) */
                vis_best[v] = best >= 0 ? acc[best] : 0;
                vis_own[v] = w_own;
            }
            if (best >= 0) {
                int64_t gain = acc[best] - w_own;
                if (gain > 0 || overloaded) {
                    proposal *p = &ws->tp[c][tn++];
                    p->v = v; p->target = best; p->own = own; p->gain = gain;
                    p->c = vwgt[v]; p->keep = 1;
                }
            }
            for (int64_t q = 0; q < nt; q++) acc[touched[q]] = 0;
        }
        ws->tnp[c] = tn;
        }
        }
        int64_t np = 0;
        for (int t = 0; t < ws->nthr; t++) {
            memcpy(ws->props + np, ws->tp[t], sizeof(proposal) * (size_t)ws->tnp[t]);
            np += ws->tnp[t];
        }
        /* --- R3: departures from overloaded blocks (refinement only) --- */
        if (refine && np > 0) {
            qsort(ws->props, (size_t)np, sizeof(proposal), cmp_by_source);
            int64_t i = 0;
            while (i < np) {
                int64_t b = ws->props[i].own, e = i;
                while (e < np && ws->props[e].own == b) e++;
                if (W[b] > bound_of(Bv, B, b)) {
                    int64_t excess = W[b] - bound_of(Bv, B, b), departed = 0;
                    for (int64_t q = i; q < e; q++) {
                        if (departed < excess) departed += ws->props[q].c;
                        else ws->props[q].keep = 0;
                    }
                }
                i = e;
            }
        }
        /* --- R4: capacity arbitration per target --- */
        if (np > 0) qsort(ws->props, (size_t)np, sizeof(proposal), cmp_by_target);
        int64_t i = 0;
        while (i < np) {
            int64_t T = ws->props[i].target, e = i;
            while (e < np && ws->props[e].target == T) e++;
            int64_t cap = bound_of(Bv, B, T) - W[T], sum = 0;
            for (int64_t q = i; q < e; q++) {
                proposal *p = &ws->props[q];
                if (!p->keep) continue;
                sum += p->c;
                if (!(p->c == 0 || sum <= cap)) p->keep = 0;
            }
            i = e;
        }
        /* --- R5: apply the admitted moves together --- */
        for (int64_t q = 0; q < np; q++) {
            proposal *p = &ws->props[q];
            if (!p->keep) continue;
            lab[p->v] = (int32_t)p->target;
            W[p->target] += p->c;
            W[p->own] -= p->c;
            moves++;
        }
    }
    return moves;
}

static int lp_run(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                  const int32_t *adjwgt, const int32_t *vwgt, int32_t *lab,
                  int64_t *W, int64_t nW, int64_t B, const int64_t *Bv, int refine,
                  const int32_t *cp, uint64_t seed, int32_t rounds, int32_t S,
                  int32_t degree_order, const run_map *rm, int32_t *rounds_done,
                  int64_t *moves_per_round)
{
    int32_t *colour = NULL;
    if (degree_order) {
        colour = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        if (!colour) return OR_ENOMEM;
    }
    lp_ws ws;
    if (ws_alloc(&ws, n, nW) != OR_OK) {
        free(colour);
        return OR_ENOMEM;
    }
    int32_t done = 0;
    for (int32_t r = 0; r < rounds; r++) {
        if (colour) or_degree_colours(n, xadj, seed, r, S, colour);
        int64_t m = lp_round(n, xadj, adjncy, adjwgt, vwgt, lab, W, B, Bv, refine, cp,
                             seed, r, S, NULL, colour, rm, NULL, NULL, &ws);
        if (moves_per_round) moves_per_round[r] = m;
        done = r + 1;
        if (m == 0) break;
    }
    if (rounds_done) *rounds_done = done;
    ws_free(&ws);
    free(colour);
    return OR_OK;
}

static int64_t total_weight(int64_t n, const int32_t *vwgt, int32_t *maxc)
{
    int64_t s = 0;
    int32_t m = 0;
    for (int64_t v = 0; v < n; v++) {
        s += vwgt[v];
        if (vwgt[v] > m) m = vwgt[v];
    }
    if (maxc) *maxc = m;
    return s;
}

typedef struct {
    int64_t v;
    int32_t block;
} iso_item;

static int cmp_iso(const void *a, const void *b)
{
    const iso_item *x = (const iso_item *)a, *y = (const iso_item *)b;
    if (x->block != y->block) return x->block < y->block ? -1 : 1;
    return x->v < y->v ? -1 : (x->v > y->v);
}

/* Reading R6 (the paper is silent on nodes without neighbours): label
 * propagation never moves them, so each would stay a singleton cluster and
 * coarsening would stall on graphs with many of them.  After the rounds the
 * nodes without neighbours are packed in id order, separately per block of the
 * constraint partition when one is given: with U' = U - cmax + 1 (cmax the
 * largest weight among them) and P(v) the total weight of the earlier ones in
 * the same block, v joins group floor(P(v) / U'); a group's label is its
 * smallest node id.  A group weighs at most U' - 1 + cmax = U. */
static int pack_isolated(int64_t n, const int64_t *xadj, const int32_t *vwgt, int64_t U,
                         const int32_t *cp, int32_t *lab)
{
    int64_t ni = 0;
    int32_t cmax = 0;
    for (int64_t v = 0; v < n; v++)
        if (xadj[v + 1] == xadj[v]) {
            ni++;
            if (vwgt[v] > cmax) cmax = vwgt[v];
        }
    if (ni == 0) return OR_OK;
    iso_item *it = (iso_item *)malloc(sizeof(iso_item) * (size_t)ni);
    if (!it) return OR_ENOMEM;
    ni = 0;
    for (int64_t v = 0; v < n; v++)
        if (xadj[v + 1] == xadj[v]) {
            it[ni].v = v;
            it[ni].block = cp ? cp[v] : 0;
            ni++;
        }
    qsort(it, (size_t)ni, sizeof(iso_item), cmp_iso);
    int64_t Up = U - cmax + 1;
    int64_t P = 0, group = -1, rep = 0;
    for (int64_t i = 0; i < ni; i++) {
        if (i == 0 || it[i].block != it[i - 1].block) { P = 0; group = -1; }
        int64_t gi = P / Up;
        if (gi != group) { group = gi; rep = it[i].v; }
        lab[it[i].v] = (int32_t)rep;
        P += vwgt[it[i].v];
    }
    free(it);
    return OR_OK;
}

/* Sec. III.A, clustering form: every node starts in its own cluster (label
 * = node id); cluster weights stay <= U. */
static int cluster_impl(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                        const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
                        int32_t rounds, int32_t S, uint64_t seed,
                        const int32_t *constraint_part, int32_t degree_order,
                        int32_t *labels_out, int32_t *rounds_done, int64_t *moves_per_round);

int or_cluster(int64_t n, const int64_t *xadj, const int32_t *adjncy,
               const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
               int32_t rounds, int32_t S, uint64_t seed,
               const int32_t *constraint_part, int32_t *labels_out,
               int32_t *rounds_done, int64_t *moves_per_round)
{
    return cluster_impl(n, xadj, adjncy, adjwgt, vwgt, U, rounds, S, seed, constraint_part, 0,
                        labels_out, rounds_done, moves_per_round);
}

/* Clustering with degree-ordered sub-rounds: the closest synchronous
 * analogue of the paper's traversal in increasing degree (Sec. III.A); see
 * or_degree_colours.  Otherwise as or_cluster. */
int or_cluster_degree_ordered(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                              const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
                              int32_t rounds, int32_t S, uint64_t seed,
                              const int32_t *constraint_part, int32_t *labels_out,
                              int32_t *rounds_done, int64_t *moves_per_round)
{
    return cluster_impl(n, xadj, adjncy, adjwgt, vwgt, U, rounds, S, seed, constraint_part, 1,
                        labels_out, rounds_done, moves_per_round);
}

static int cluster_impl(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                        const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
                        int32_t rounds, int32_t S, uint64_t seed,
                        const int32_t *constraint_part, int32_t degree_order,
                        int32_t *labels_out, int32_t *rounds_done, int64_t *moves_per_round)
{
    int32_t maxc;
    if (rounds < 0 || S < 1) return OR_EINVAL;
    total_weight(n, vwgt, &maxc);
    if (U < maxc) return OR_EINVAL;
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!W) return OR_ENOMEM;
    for (int64_t v = 0; v < n; v++) { labels_out[v] = (int32_t)v; W[v] = vwgt[v]; }
    int rc = lp_run(n, xadj, adjncy, adjwgt, vwgt, labels_out, W, n, U, NULL, 0,
                    constraint_part, seed, rounds, S, degree_order, NULL, rounds_done,
                    moves_per_round);
    free(W);
    if (rc) return rc;
    return pack_isolated(n, xadj, vwgt, U, constraint_part, labels_out);
}

/* Sec. III.A, local-search form with a bound on every block: Bv[b] when given,
 * else B. */
static int refine_bounds(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                         const int32_t *adjwgt, const int32_t *vwgt, int32_t nblocks,
                         int64_t B, const int64_t *Bv, int32_t rounds, int32_t S, uint64_t seed,
                         const run_map *rm, int32_t *part, int32_t *rounds_done,
                         int64_t *moves_per_round)
{
    if (nblocks < 1 || rounds < 0 || S < 1) return OR_EINVAL;
    for (int64_t v = 0; v < n; v++)
        if (part[v] < 0 || part[v] >= nblocks) return OR_EINVAL;
    int64_t *W = (int64_t *)calloc((size_t)nblocks, sizeof(int64_t));
    if (!W) return OR_ENOMEM;
    for (int64_t v = 0; v < n; v++) W[part[v]] += vwgt[v];
    int rc = lp_run(n, xadj, adjncy, adjwgt, vwgt, part, W, nblocks, B, Bv, 1, NULL,
                    seed, rounds, S, 0, rm, rounds_done, moves_per_round);
    free(W);
    return rc;
}

int or_refine_bound(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                    const int32_t *adjwgt, const int32_t *vwgt, int32_t nblocks,
                    int64_t B, int32_t rounds, int32_t S, uint64_t seed,
                    int32_t *part, int32_t *rounds_done, int64_t *moves_per_round)
{
    return refine_bounds(n, xadj, adjncy, adjwgt, vwgt, nblocks, B, NULL, rounds, S, seed,
                         NULL, part, rounds_done, moves_per_round);
}

int or_refine(int64_t n, const int64_t *xadj, const int32_t *adjncy,
              const int32_t *adjwgt, const int32_t *vwgt, int32_t k, double eps,
              int32_t rounds, int32_t S, uint64_t seed, int32_t *part,
              int64_t *cut_out, int64_t *block_w_out, int32_t *rounds_done,
              int64_t *moves_per_round)
{
    if (k < 1 || eps < 0) return OR_EINVAL;
    int64_t B = or_lmax(total_weight(n, vwgt, NULL), k, eps);
    int rc = or_refine_bound(n, xadj, adjncy, adjwgt, vwgt, k, B, rounds, S, seed,
                             part, rounds_done, moves_per_round);
    if (rc) return rc;
    if (cut_out) *cut_out = or_cut(n, xadj, adjncy, adjwgt, part);
    if (block_w_out) or_block_weights(n, vwgt, part, k, block_w_out);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* contraction (Sec. III, Sec. IV.C) and projection                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t cu, cv;
    int64_t w;
} triple;

static int cmp_triple(const void *a, const void *b)
{
    const triple *x = (const triple *)a, *y = (const triple *)b;
    if (x->cu != y->cu) return x->cu < y->cu ? -1 : 1;
    if (x->cv != y->cv) return x->cv < y->cv ? -1 : 1;
    return 0;
}

/* Each cluster becomes one node whose weight is the cluster's weight; two
 * coarse nodes are adjacent iff their clusters are, with the summed weight
 * of the edges between them.  Coarse ids: q maps the distinct cluster ids in
 * ascending order onto 0..n'-1 (the prefix-sum construction of Sec. IV.C),
 * C(v) = q(label(v)).  Output rows ascending, neighbours ascending. */
int or_contract(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *adjwgt, const int32_t *vwgt, const int32_t *labels,
                int64_t *cn_out, int64_t *cnnz_out, int64_t **cxadj_out,
                int32_t **cadjncy_out, int32_t **cadjwgt_out, int32_t **cvwgt_out,
                int32_t *f2c)
{
    for (int64_t v = 0; v < n; v++)
        if (labels[v] < 0 || labels[v] >= n) return OR_EINVAL;
    int64_t *q = (int64_t *)calloc(n > 0 ? (size_t)n : 1u, sizeof(int64_t));
    if (!q) return OR_ENOMEM;
    for (int64_t v = 0; v < n; v++) q[labels[v]] = 1;      /* mark used ids */
    int64_t cn = 0;
    for (int64_t L = 0; L < n; L++) {                        /* prefix sum    */
        int64_t used = q[L];
        q[L] = used ? cn : -1;
        cn += used;
    }
    for (int64_t v = 0; v < n; v++) f2c[v] = (int32_t)q[labels[v]];
    free(q);

    int32_t *cvwgt = (int32_t *)calloc((size_t)(cn ? cn : 1), sizeof(int32_t));
    int64_t *cxadj = (int64_t *)calloc((size_t)cn + 1, sizeof(int64_t));
    int64_t nnz = xadj[n];
    triple *t = (triple *)malloc(sizeof(triple) * (size_t)(nnz ? nnz : 1));
    if (!cvwgt || !cxadj || !t) { free(cvwgt); free(cxadj); free(t); return OR_ENOMEM; }
    for (int64_t v = 0; v < n; v++) cvwgt[f2c[v]] += vwgt[v];
    int64_t nt = 0;
    for (int64_t v = 0; v < n; v++)
        for (int64_t i = xadj[v]; i < xadj[v + 1]; i++) {
            int64_t cu = f2c[v], cv = f2c[adjncy[i]];
            if (cu == cv) continue;                 /* edge inside a cluster */
            t[nt].cu = cu; t[nt].cv = cv; t[nt].w = adjwgt[i];
            nt++;
        }
    if (nt > 0) qsort(t, (size_t)nt, sizeof(triple), cmp_triple);
    int64_t m = 0;                                   /* reduce equal pairs */
    for (int64_t i = 0; i < nt; i++) {
        if (m > 0 && t[m - 1].cu == t[i].cu && t[m - 1].cv == t[i].cv) t[m - 1].w += t[i].w;
        else t[m++] = t[i];
    }
    int32_t *cadj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t *cw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    if (!cadj || !cw) { free(cadj); free(cw); free(cvwgt); free(cxadj); free(t); return OR_ENOMEM; }
    for (int64_t i = 0; i < m; i++) {
        cxadj[t[i].cu + 1]++;
        cadj[i] = (int32_t)t[i].cv;
        cw[i] = (int32_t)t[i].w;
    }
    for (int64_t c = 0; c < cn; c++) cxadj[c + 1] += cxadj[c];
    free(t);
    *cn_out = cn; *cnnz_out = m;
    *cxadj_out = cxadj; *cadjncy_out = cadj; *cadjwgt_out = cw; *cvwgt_out = cvwgt;
    return OR_OK;
}

void or_free(void *p) { free(p); }

/* Uncoarsening: a fine node takes the block of its coarse representative. */
void or_project(int64_t n_fine, const int32_t *f2c, const int32_t *coarse_part,
                int32_t *fine_part)
{
    for (int64_t v = 0; v < n_fine; v++) fine_part[v] = coarse_part[f2c[v]];
}

/* Sec. II.A: cut = total weight of edges whose endpoints lie in different
 * blocks (each undirected edge is stored twice, hence the halving). */
int64_t or_cut(int64_t n, const int64_t *xadj, const int32_t *adjncy,
               const int32_t *adjwgt, const int32_t *part)
{
    int64_t s = 0;
    for (int64_t v = 0; v < n; v++)
        for (int64_t i = xadj[v]; i < xadj[v + 1]; i++)
            if (part[adjncy[i]] != part[v]) s += adjwgt[i];
    return s / 2;
}

void or_block_weights(int64_t n, const int32_t *vwgt, const int32_t *part,
                      int32_t k, int64_t *bw)
{
    for (int32_t b = 0; b < k; b++) bw[b] = 0;
    for (int64_t v = 0; v < n; v++) bw[part[v]] += vwgt[v];
}

/* ------------------------------------------------------------------ */
/* initial partition of the coarsest graph (stands in for KaFFPaE)      */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t v;
    int32_t c;
    uint32_t h;
} lpt_item;

static int cmp_lpt(const void *a, const void *b)
{
    const lpt_item *x = (const lpt_item *)a, *y = (const lpt_item *)b;
    if (x->c != y->c) return x->c > y->c ? -1 : 1;   /* heavier first */
    if (x->h != y->h) return x->h < y->h ? -1 : 1;   /* seeded shuffle */
    return x->v < y->v ? -1 : (x->v > y->v);
}

/* LPT start (the stand-in for an individual's initial assignment): the nodes
 * in (c desc, h(v) asc, v asc) order, h(v) = high 32 bits of mix64(seed ^ v),
 * each into the currently lightest of the k blocks (lowest id on ties). */
int or_lpt_start(int64_t n, const int32_t *vwgt, int32_t k, uint64_t seed, int32_t *part_out)
{
    if (k < 1) return OR_EINVAL;
    lpt_item *it = (lpt_item *)malloc(sizeof(lpt_item) * (size_t)(n ? n : 1));
    int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    if (!it || !bw) { free(it); free(bw); return OR_ENOMEM; }
    for (int64_t v = 0; v < n; v++) {
        it[v].v = v;
        it[v].c = vwgt[v];
        it[v].h = (uint32_t)(or_mix64(seed ^ (uint64_t)v) >> 32);
    }
    if (n > 0) qsort(it, (size_t)n, sizeof(lpt_item), cmp_lpt);
    for (int64_t i = 0; i < n; i++) {
        int32_t bb = 0;
        for (int32_t b = 1; b < k; b++)
            if (bw[b] < bw[bb]) bb = b;
        part_out[it[i].v] = bb;
        bw[bb] += it[i].c;
    }
    free(it);
    free(bw);
    return OR_OK;
}

/* Batched runs (the stand-in for the population of Sec. II.C / IV.E, whose
 * individuals are independent): run r refines graph run_graph[r] (bound
 * Bg[run_graph[r]] on each of its k blocks) from its own LPT start with its
 * own seed s_r = seeds[r].  It places its graph's nodes in (c desc, h_r(v)
 * asc, v asc) order into the currently lightest of its k blocks (lowest id
 * on ties), h_r(v) = high 32 bits of mix64(s_r ^ v) (or_lpt_start); then all
 * runs are refined together for `rounds` rounds as one SCLaP refinement of
 * the disjoint union of their graphs (run r: nodes off_r + v, blocks r*k ..
 * r*k+k-1), each run's sub-rounds and tie-breaks keyed by s_r, its local node
 * ids and its local block ids (run_map).  A run's result therefore equals
 * or_lpt_start followed by or_refine_bound on its graph alone with seed s_r
 * (a run that has converged stays unchanged while others go on).  Outputs per
 * run: its partition (block ids 0..k-1, concatenated in run order), cut and
 * largest block weight. */
int or_refine_batched(int32_t ngraphs, const int64_t *ns, const int64_t *const *xadjs,
                      const int32_t *const *adjncys, const int32_t *const *adjwgts,
                      const int32_t *const *vwgts, int32_t k, const int64_t *Bg,
                      int32_t rounds, int32_t S, const uint64_t *seeds, int32_t nruns,
                      const int32_t *run_graph, int32_t *parts_out, int64_t *cuts_out,
                      int64_t *maxbw_out)
{
    if (k < 1 || nruns < 1 || ngraphs < 1) return OR_EINVAL;
    int64_t un = 0, unnz = 0, nmax = 0;
    for (int32_t r = 0; r < nruns; r++) {
        int32_t g = run_graph[r];
        if (g < 0 || g >= ngraphs) return OR_EINVAL;
        un += ns[g];
        unnz += xadjs[g][ns[g]];
        if (ns[g] > nmax) nmax = ns[g];
    }
    int64_t *ux = (int64_t *)malloc(sizeof(int64_t) * (size_t)(un + 1));
    int32_t *ua = (int32_t *)malloc(sizeof(int32_t) * (size_t)(unnz ? unnz : 1));
    int32_t *uw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(unnz ? unnz : 1));
    int32_t *uc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(un ? un : 1));
    int32_t *up = (int32_t *)malloc(sizeof(int32_t) * (size_t)(un ? un : 1));
    int64_t *Bv = (int64_t *)malloc(sizeof(int64_t) * (size_t)nruns * (size_t)k);
    int64_t *bw = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int32_t *run_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(un ? un : 1));
    int64_t *roff = (int64_t *)malloc(sizeof(int64_t) * (size_t)nruns);
    int rc = OR_OK;
    if (!ux || !ua || !uw || !uc || !up || !Bv || !bw || !run_of || !roff) {
        rc = OR_ENOMEM;
        goto out;
    }

    int64_t off = 0, eoff = 0;
    for (int32_t r = 0; r < nruns; r++) {        /* the disjoint union */
        int32_t g = run_graph[r];
        int64_t n = ns[g];
        for (int64_t v = 0; v < n; v++) {
            ux[off + v] = eoff + xadjs[g][v];
            uc[off + v] = vwgts[g][v];
        }
        for (int64_t i = 0; i < xadjs[g][n]; i++) {
            ua[eoff + i] = (int32_t)(adjncys[g][i] + off);
            uw[eoff + i] = adjwgts[g][i];
        }
        for (int32_t b = 0; b < k; b++) Bv[(int64_t)r * k + b] = Bg[g];
        for (int64_t v = 0; v < n; v++) run_of[off + v] = r;
        roff[r] = off;
        /* LPT start of run r, its blocks shifted to r*k .. r*k+k-1 */
        rc = or_lpt_start(n, vwgts[g], k, seeds[r], up + off);
        if (rc) goto out;
        for (int64_t v = 0; v < n; v++) up[off + v] += r * k;
        off += n;
        eoff += xadjs[g][n];
    }
    ux[un] = unnz;

    run_map rm;
    rm.run_of = run_of;
    rm.seed = seeds;
    rm.off = roff;
    rm.k = k;
    rc = refine_bounds(un, ux, ua, uw, uc, k * nruns, 0, Bv, rounds, S, 0, &rm, up, NULL, NULL);
    if (rc) goto out;

    off = 0;
    for (int32_t r = 0; r < nruns; r++) {
        int32_t g = run_graph[r];
        int64_t n = ns[g];
        int64_t cut = 0;
        for (int64_t v = 0; v < n; v++)
            for (int64_t i = xadjs[g][v]; i < xadjs[g][v + 1]; i++)
                if (up[off + adjncys[g][i]] != up[off + v]) cut += adjwgts[g][i];
        for (int32_t b = 0; b < k; b++) bw[b] = 0;
        for (int64_t v = 0; v < n; v++) bw[up[off + v] - r * k] += vwgts[g][v];
        int64_t mx = 0;
        for (int32_t b = 0; b < k; b++) if (bw[b] > mx) mx = bw[b];
        if (cuts_out) cuts_out[r] = cut / 2;
        if (maxbw_out) maxbw_out[r] = mx;
        if (parts_out)
            for (int64_t v = 0; v < n; v++) parts_out[off + v] = up[off + v] - r * k;
        off += n;
    }
out:
    free(ux); free(ua); free(uw); free(uc); free(up); free(Bv); free(bw); free(run_of);
    free(roff);
    return rc;
}

/* Reading (the paper runs an evolutionary algorithm here): P independent
 * individuals, computed as P batched runs on the same graph with bound B (see
 * or_refine_batched), individual t with seed s_t = mix64(seed ^
 * (0xD1B54A32D192ED03 * (t + 1))).  The best individual has the lowest cut among those
 * with max block weight <= B (lowest t on ties); with none feasible, the
 * smallest max block weight, then cut, then t. */
int or_initial_partition(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                         const int32_t *adjwgt, const int32_t *vwgt, int32_t k,
                         int64_t B, int32_t P, int32_t rounds, int32_t S,
                         uint64_t seed, int32_t *part_out, int64_t *cuts_out,
                         int64_t *maxbw_out, int32_t *best_out)
{
    if (k < 1 || P < 1) return OR_EINVAL;
    int32_t *rg = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    uint64_t *seeds = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P);
    int32_t *parts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * P > 0 ? n * P : 1));
    int64_t *cuts = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
    int64_t *mxs = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
    int rc = OR_OK;
    if (!rg || !seeds || !parts || !cuts || !mxs) { rc = OR_ENOMEM; goto out; }
    for (int32_t t = 0; t < P; t++)
        seeds[t] = or_mix64(seed ^ (0xD1B54A32D192ED03ULL * (uint64_t)(t + 1)));
    rc = or_refine_batched(1, &n, &xadj, &adjncy, &adjwgt, &vwgt, k, &B, rounds, S, seeds, P,
                           rg, parts, cuts, mxs);
    if (rc) goto out;
    int32_t best = -1;
    int64_t best_cut = 0, best_max = 0;
    for (int32_t t = 0; t < P; t++) {
        int64_t cut = cuts[t], mx = mxs[t];
        if (cuts_out) cuts_out[t] = cut;
        if (maxbw_out) maxbw_out[t] = mx;
        int better;
        if (best < 0) better = 1;
        else {
            int f_new = mx <= B, f_old = best_max <= B;
            if (f_new != f_old) better = f_new;
            else if (f_new) better = cut < best_cut;
            else better = mx < best_max || (mx == best_max && cut < best_cut);
        }
        if (better) { best = t; best_cut = cut; best_max = mx; }
    }
    for (int64_t v = 0; v < n; v++) part_out[v] = parts[(int64_t)best * n + v];
    if (best_out) *best_out = best;
out:
    free(rg); free(seeds); free(parts); free(cuts); free(mxs);
    return rc;
}

/* ------------------------------------------------------------------ */
/* multilevel driver (Sec. IV.E)                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int64_t *xadj;
    int32_t *adjncy, *adjwgt, *vwgt;
    int32_t *f2c;   /* map to the next coarser level (NULL on the coarsest) */
    int own;        /* arrays malloc'ed here (all levels but the input) */
} level;

static uint64_t level_seed(uint64_t seed, int32_t l)
{
    return or_mix64(seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(l + 1)));
}

static int multilevel_impl(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                           const int32_t *adjwgt, const int32_t *vwgt, const or_ml_params *p,
                           const int32_t *seed_part, int32_t *part_out, or_ml_stats *st);

int or_multilevel(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                  const int32_t *adjwgt, const int32_t *vwgt,
                  const or_ml_params *p, int32_t *part_out, or_ml_stats *st)
{
    return multilevel_impl(n, xadj, adjncy, adjwgt, vwgt, p, NULL, part_out, st);
}

/* One iterated V-cycle (Sec. IV.E, the cycles of the fast and minimal
 * presets): the multilevel scheme seeded by the partition part_inout.  Every
 * clustering is restricted to the blocks of the current partition (the
 * constraint of Sec. III.A's coarsening), each coarse node inherits its
 * members' block, and the coarsest graph's inherited partition, refined
 * like every level, is the initial partition (init_best = -1; init_cut /
 * init_maxbw describe it after refinement).  part_inout: k blocks in, the
 * new partition out. */
int or_vcycle(int64_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
              const int32_t *vwgt, const or_ml_params *p, int32_t *part_inout, or_ml_stats *st)
{
    for (int64_t v = 0; v < n; v++)
        if (part_inout[v] < 0 || part_inout[v] >= p->k) return OR_EINVAL;
    int32_t *seed = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!seed) return OR_ENOMEM;
    memcpy(seed, part_inout, sizeof(int32_t) * (size_t)n);
    int rc = multilevel_impl(n, xadj, adjncy, adjwgt, vwgt, p, seed, part_inout, st);
    free(seed);
    return rc;
}

static int multilevel_impl(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                           const int32_t *adjwgt, const int32_t *vwgt, const or_ml_params *p,
                           const int32_t *seed_part, int32_t *part_out, or_ml_stats *st)
{
    if (p->k < 1 || p->eps < 0 || p->cluster_rounds < 0 || p->refine_rounds < 0 ||
        p->subrounds < 1 || p->init_seeds < 1 || p->init_rounds < 0)
        return OR_EINVAL;
    int32_t maxc;
    int64_t cV = total_weight(n, vwgt, &maxc);
    int64_t lmax = or_lmax(cV, p->k, p->eps);
    int64_t U = p->U > 0 ? p->U : (maxc > cV / (10 * (int64_t)p->k) ? maxc : cV / (10 * (int64_t)p->k));
    if (U < maxc) return OR_EINVAL;
    int32_t maxl = p->max_levels > 0 ? p->max_levels : 32;
    if (maxl > OR_MAX_LEVELS) maxl = OR_MAX_LEVELS;

    level lv[OR_MAX_LEVELS];
    int32_t *cpl[OR_MAX_LEVELS];  /* V-cycle: the seed partition on every level */
    memset(lv, 0, sizeof(lv));
    memset(cpl, 0, sizeof(cpl));
    lv[0].n = n; lv[0].xadj = (int64_t *)xadj; lv[0].adjncy = (int32_t *)adjncy;
    lv[0].adjwgt = (int32_t *)adjwgt; lv[0].vwgt = (int32_t *)vwgt;
    int32_t L = 0, rc = OR_OK;
    memset(st, 0, sizeof(*st));
    if (seed_part) {
        cpl[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        if (!cpl[0]) return OR_ENOMEM;
        memcpy(cpl[0], seed_part, sizeof(int32_t) * (size_t)n);
    }

    /* coarsening: l rounds of clustering, then contraction, recursively */
    while (lv[L].n >= p->n_stop && L + 1 < maxl) {
        level *g = &lv[L];
        int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n ? g->n : 1));
        g->f2c = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n ? g->n : 1));
        if (!lab || !g->f2c) { free(lab); rc = OR_ENOMEM; goto out; }
        int32_t rd = 0;
        rc = cluster_impl(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, U, p->cluster_rounds,
                          p->subrounds, level_seed(p->seed, L), cpl[L], p->degree_order != 0,
                          lab, &rd, NULL);
        if (rc) { free(lab); goto out; }
        st->cluster_rounds_done[L] = rd;
        level *c = &lv[L + 1];
        int64_t cnnz;
        rc = or_contract(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, lab, &c->n, &cnnz,
                         &c->xadj, &c->adjncy, &c->adjwgt, &c->vwgt, g->f2c);
        free(lab);
        if (rc) goto out;
        c->own = 1;
        if (c->n == g->n) {                       /* no shrink: drop the level */
            free(c->xadj); free(c->adjncy); free(c->adjwgt); free(c->vwgt);
            memset(c, 0, sizeof(*c));
            free(g->f2c); g->f2c = NULL;
            break;
        }
        if (seed_part) {  /* a cluster lies in one block: the coarse node inherits it */
            cpl[L + 1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->n ? c->n : 1));
            if (!cpl[L + 1]) { rc = OR_ENOMEM; goto out; }
            for (int64_t v = 0; v < g->n; v++) cpl[L + 1][g->f2c[v]] = cpl[L][v];
        }
        L++;
        if (20 * c->n > 19 * g->n) break;          /* stalled (< 5% shrink) */
    }

    /* initial partition of the coarsest graph */
    {
        level *g = &lv[L];
        int32_t *cp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n ? g->n : 1));
        int64_t *cuts = (int64_t *)malloc(sizeof(int64_t) * (size_t)p->init_seeds);
        int64_t *mx = (int64_t *)malloc(sizeof(int64_t) * (size_t)p->init_seeds);
        if (!cp || !cuts || !mx) { free(cp); free(cuts); free(mx); rc = OR_ENOMEM; goto out; }
        int32_t best = 0;
        if (seed_part) {
            memcpy(cp, cpl[L], sizeof(int32_t) * (size_t)g->n);
            int32_t rd = 0;
            rc = or_refine_bound(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, p->k, lmax,
                                 p->init_rounds, p->subrounds, level_seed(p->seed, L), cp, &rd,
                                 NULL);
            if (rc) { free(cp); free(cuts); free(mx); goto out; }
            int64_t *bw = (int64_t *)calloc((size_t)p->k, sizeof(int64_t));
            if (!bw) { free(cp); free(cuts); free(mx); rc = OR_ENOMEM; goto out; }
            or_block_weights(g->n, g->vwgt, cp, p->k, bw);
            st->init_best = -1;
            st->init_cut = or_cut(g->n, g->xadj, g->adjncy, g->adjwgt, cp);
            st->init_maxbw = 0;
            for (int32_t b = 0; b < p->k; b++) if (bw[b] > st->init_maxbw) st->init_maxbw = bw[b];
            free(bw);
        } else {
            rc = or_initial_partition(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, p->k, lmax,
                                      p->init_seeds, p->init_rounds, p->subrounds,
                                      level_seed(p->seed, L), cp, cuts, mx, &best);
            if (rc) { free(cp); free(cuts); free(mx); goto out; }
            st->init_best = best; st->init_cut = cuts[best]; st->init_maxbw = mx[best];
        }
        free(cuts); free(mx);
        /* uncoarsening: project, then r rounds of refinement per level */
        int32_t *cur = cp;
        for (int32_t l = L - 1; l >= 0; l--) {
            level *f = &lv[l];
            int32_t *fp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(f->n ? f->n : 1));
            if (!fp) { free(cur); rc = OR_ENOMEM; goto out; }
            or_project(f->n, f->f2c, cur, fp);
            free(cur);
            cur = fp;
            int32_t rd = 0;
            rc = or_refine_bound(f->n, f->xadj, f->adjncy, f->adjwgt, f->vwgt, p->k, lmax,
                                 p->refine_rounds, p->subrounds, level_seed(p->seed, l), cur,
                                 &rd, NULL);
            if (rc) { free(cur); goto out; }
            st->refine_rounds_done[l] = rd;
        }
        memcpy(part_out, cur, sizeof(int32_t) * (size_t)n);
        free(cur);
    }
    st->levels = L + 1;
    for (int32_t l = 0; l <= L; l++) { st->n[l] = lv[l].n; st->nnz[l] = lv[l].xadj[lv[l].n]; }
    st->U = U; st->lmax = lmax;
    st->cut = or_cut(n, xadj, adjncy, adjwgt, part_out);
    {
        int64_t *bw = (int64_t *)calloc((size_t)p->k, sizeof(int64_t));
        if (!bw) { rc = OR_ENOMEM; goto out; }
        or_block_weights(n, vwgt, part_out, p->k, bw);
        st->maxbw = 0;
        for (int32_t b = 0; b < p->k; b++) if (bw[b] > st->maxbw) st->maxbw = bw[b];
        free(bw);
    }
out:
    for (int32_t l = 0; l < OR_MAX_LEVELS; l++) {
        free(cpl[l]);
        free(lv[l].f2c);
        if (lv[l].own) { free(lv[l].xadj); free(lv[l].adjncy); free(lv[l].adjwgt); free(lv[l].vwgt); }
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* learned active set for refinement (not in the paper: a gate that    */
/* decides which nodes a refinement round visits; full sweeps every    */
/* full_every rounds and in the last round keep it a heuristic over    */
/* the plain method)                                                   */
/* ------------------------------------------------------------------ */

/* bfloat16 rounding of a finite float, round to nearest, ties to even: add
 * 0x7FFF plus the lowest kept bit to the 32-bit pattern and drop the low 16
 * bits. */
float or_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return f;
}

static float bf16_bits_to_float(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* 2^-e as a float, 0 <= e <= 62 (exact). */
static float pow2_neg(int e)
{
    uint32_t u = (uint32_t)(127 - e) << 23;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* Feature 1: log2 of x >= 1 by its piecewise-linear form e + (x - 2^e)/2^e,
 * e = floor(log2 x); exact at powers of two, every step IEEE-rounded. */
float or_log2_feature(int64_t x)
{
    int e = 0;
    while (e < 62 && (x >> (e + 1)) != 0) e++;
    float frac = (float)(x - ((int64_t)1 << e)) * pow2_neg(e);
    return (float)e + frac;
}

/* The six features of every node (row-major [n][6], each rounded to bf16),
 * wdeg = v's weighted degree, wb / wo = the weight to the best eligible
 * other block / to its own block that v's most recent visit saw (vis_best,
 * vis_own; 0 before any visit or when NULL):
 *   f1 log2-feature(1 + deg), f2 W(own)/L_max, f3 (wb - wo)/wdeg (the best
 *   external gain), f4 v moved in the previous round, f5 share of v's
 *   neighbours that moved in the previous round, f6 wo/wdeg.
 * Nodes without neighbours get zeros. */
void or_features(int64_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                 const int32_t *lab, const int64_t *W, int64_t Lmax, const uint8_t *moved,
                 const int64_t *vis_best, const int64_t *vis_own, float *x)
{
    for (int64_t v = 0; v < n; v++) {
        float *f = x + v * 6;
        int64_t deg = xadj[v + 1] - xadj[v];
        if (deg == 0) {
            for (int i = 0; i < 6; i++) f[i] = 0.0f;
            continue;
        }
        int64_t wdeg = 0, nmov = 0;
        for (int64_t i = xadj[v]; i < xadj[v + 1]; i++) {
            wdeg += adjwgt[i];
            if (moved && moved[adjncy[i]]) nmov++;
        }
        int64_t own = lab[v];
        int64_t wb = vis_best ? vis_best[v] : 0, wo = vis_own ? vis_own[v] : 0;
        f[0] = or_bf16(or_log2_feature(1 + deg));
        f[1] = or_bf16((float)W[own] / (float)Lmax);
        f[2] = or_bf16((float)(wb - wo) / (float)wdeg);
        f[3] = (moved && moved[v]) ? 1.0f : 0.0f;
        f[4] = or_bf16((float)nmov / (float)deg);
        f[5] = or_bf16((float)wo / (float)wdeg);
    }
}

/* Forward pass of the 6-32-32-1 scorer on one node's (bf16) features; the
 * parameters are 1313 bf16 values: W1[32][6], b1[32], W2[32][32], b2[32],
 * W3[32], b3.  Every output starts from its bias and adds w * x with one
 * fmaf per input in index order (float accumulator); hidden outputs go
 * through ReLU and are rounded to bf16.  Returns the logit z. */
float or_mlp_forward(const uint16_t *net, const float *x)
{
    float h1[32], h2[32];
    for (int j = 0; j < 32; j++) {
        float acc = bf16_bits_to_float(net[OR_MLP_B1 + j]);
        for (int i = 0; i < 6; i++)
            acc = fmaf(bf16_bits_to_float(net[OR_MLP_W1 + j * 6 + i]), x[i], acc);
        h1[j] = or_bf16(acc > 0.0f ? acc : 0.0f);
    }
    for (int j = 0; j < 32; j++) {
        float acc = bf16_bits_to_float(net[OR_MLP_B2 + j]);
        for (int i = 0; i < 32; i++)
            acc = fmaf(bf16_bits_to_float(net[OR_MLP_W2 + j * 32 + i]), h1[i], acc);
        h2[j] = or_bf16(acc > 0.0f ? acc : 0.0f);
    }
    float z = bf16_bits_to_float(net[OR_MLP_B3]);
    for (int i = 0; i < 32; i++) z = fmaf(bf16_bits_to_float(net[OR_MLP_W3 + i]), h2[i], z);
    return z;
}

/* BF16-in / FP32-accumulate training loss: the mean logistic loss of the
 * network inference runs (or_mlp_forward's arithmetic: parameters rounded to
 * bf16, one fmaf per input in index order from the bias, hidden outputs
 * ReLU then bf16) on the float master parameters prm, and its straight-through
 * gradient: the derivative of that loss with respect to the rounded
 * parameters, each rounding (of a parameter or a hidden output) passed as the
 * identity.  The loss and the backward sums are kept in double. */
double or_mlp_loss_grad_bf16(const float *X, const uint8_t *y, int64_t N, const float *prm,
                             double *grad)
{
    float q[OR_MLP_NPARAM];
    for (int i = 0; i < OR_MLP_NPARAM; i++) {
        q[i] = or_bf16(prm[i]);
        grad[i] = 0.0;
    }
    double loss = 0.0;
    for (int64_t s = 0; s < N; s++) {
        const float *x = X + s * 6;
        float a1[32], h1[32], a2[32], h2[32];
        for (int j = 0; j < 32; j++) {
            float acc = q[OR_MLP_B1 + j];
            for (int i = 0; i < 6; i++) acc = fmaf(q[OR_MLP_W1 + j * 6 + i], x[i], acc);
            a1[j] = acc;
            h1[j] = or_bf16(acc > 0.0f ? acc : 0.0f);
        }
        for (int j = 0; j < 32; j++) {
            float acc = q[OR_MLP_B2 + j];
            for (int i = 0; i < 32; i++) acc = fmaf(q[OR_MLP_W2 + j * 32 + i], h1[i], acc);
            a2[j] = acc;
            h2[j] = or_bf16(acc > 0.0f ? acc : 0.0f);
        }
        float zf = q[OR_MLP_B3];
        for (int i = 0; i < 32; i++) zf = fmaf(q[OR_MLP_W3 + i], h2[i], zf);
        double z = zf, t = y[s] ? 1.0 : 0.0;
        loss += (z > 0 ? z + log1p(exp(-z)) : log1p(exp(z))) - t * z;
        double dz = 1.0 / (1.0 + exp(-z)) - t;
        double d2[32], d1[32];
        grad[OR_MLP_B3] += dz;
        for (int i = 0; i < 32; i++) {
            grad[OR_MLP_W3 + i] += dz * h2[i];
            d2[i] = a2[i] > 0.0f ? dz * q[OR_MLP_W3 + i] : 0.0;
        }
        for (int i = 0; i < 32; i++) d1[i] = 0.0;
        for (int j = 0; j < 32; j++) {
            grad[OR_MLP_B2 + j] += d2[j];
            for (int i = 0; i < 32; i++) {
                grad[OR_MLP_W2 + j * 32 + i] += d2[j] * h1[i];
                d1[i] += d2[j] * q[OR_MLP_W2 + j * 32 + i];
            }
        }
        for (int j = 0; j < 32; j++) {
            double dj = a1[j] > 0.0f ? d1[j] : 0.0;
            grad[OR_MLP_B1 + j] += dj;
            for (int i = 0; i < 6; i++) grad[OR_MLP_W1 + j * 6 + i] += dj * x[i];
        }
    }
    if (N > 0) {
        for (int i = 0; i < OR_MLP_NPARAM; i++) grad[i] /= (double)N;
        loss /= (double)N;
    }
    return loss;
}

/* Refinement with the learned gate (Sec. III.A local search; the gate is not
 * in the paper).  Before round r the features are built from the state at
 * that point (or_features): block weights and labels now, moved flags of
 * round r - 1, and what each node's most recent visit saw (the weight to the
 * best eligible other block and to its own block, recorded by lp_round).  In
 * a gated round only nodes with logit >= z_min are visited; a round is full
 * (every node) when r == 0 (no visit has been recorded yet), r % full_every
 * == full_every - 1, r is the last round, or always when net is NULL.  The
 * run stops after a full round without moves.  trace_x [rounds][n][6] and
 * trace_y [rounds][n] (moved in round r) are written when non-NULL;
 * visited_out counts the visited nodes with neighbours over all rounds. */
int or_refine_learned(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                      const int32_t *adjwgt, const int32_t *vwgt, int32_t k, double eps,
                      int32_t rounds, int32_t S, uint64_t seed, const uint16_t *net,
                      float z_min, int32_t full_every, int32_t *part, int32_t *rounds_done,
                      int64_t *moves_per_round, int64_t *visited_out, float *trace_x,
                      uint8_t *trace_y)
{
    if (k < 1 || eps < 0 || rounds < 0 || S < 1 || full_every < 1) return OR_EINVAL;
    for (int64_t v = 0; v < n; v++)
        if (part[v] < 0 || part[v] >= k) return OR_EINVAL;
    int64_t B = or_lmax(total_weight(n, vwgt, NULL), k, eps);
    int64_t *W = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    uint8_t *moved = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    uint8_t *active = (uint8_t *)malloc((size_t)(n ? n : 1));
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    float *x = (float *)malloc(sizeof(float) * 6 * (size_t)(n ? n : 1));
    int64_t *vb = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    int64_t *vo = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    lp_ws ws;
    const int ws_rc = ws_alloc(&ws, n, k);
    int rc = OR_OK;
    if (!W || !moved || !active || !prev || !x || !vb || !vo || ws_rc != OR_OK) {
        rc = OR_ENOMEM;
        goto out;
    }
    for (int64_t v = 0; v < n; v++) W[part[v]] += vwgt[v];
    int64_t visited = 0;
    int32_t done = 0;
    for (int32_t r = 0; r < rounds; r++) {
        int full = !net || r == 0 || r % full_every == full_every - 1 || r == rounds - 1;
        or_features(n, xadj, adjncy, adjwgt, part, W, B, moved, vb, vo, x);
        if (trace_x) memcpy(trace_x + (size_t)r * n * 6, x, sizeof(float) * 6 * (size_t)n);
        for (int64_t v = 0; v < n; v++) {
            active[v] = full ? 1 : (or_mlp_forward(net, x + v * 6) >= z_min);
            if (active[v] && xadj[v + 1] > xadj[v]) visited++;
        }
        memcpy(prev, part, sizeof(int32_t) * (size_t)n);
        int64_t m = lp_round(n, xadj, adjncy, adjwgt, vwgt, part, W, B, NULL, 1, NULL, seed, r,
                             S, active, NULL, NULL, vb, vo, &ws);
        for (int64_t v = 0; v < n; v++) moved[v] = part[v] != prev[v];
        if (trace_y) memcpy(trace_y + (size_t)r * n, moved, (size_t)n);
        if (moves_per_round) moves_per_round[r] = m;
        done = r + 1;
        if (full && m == 0) break;
    }
    if (rounds_done) *rounds_done = done;
    if (visited_out) *visited_out = visited;
out:
    free(W); free(moved); free(active); free(prev); free(x); free(vb); free(vo);
    if (ws_rc == OR_OK) ws_free(&ws);
    return rc;
}

/* Loss and gradient of the scorer for training, in double: mean over the N
 * samples of the logistic loss log(1 + e^z) - y z of the float parameters
 * (same layout as the bf16 network, no rounding), with ReLU'(0) = 0.
 * grad [OR_MLP_NPARAM] is overwritten.  Returns the loss. */
double or_mlp_loss_grad(const float *X, const uint8_t *y, int64_t N, const float *prm,
                        double *grad)
{
    for (int i = 0; i < OR_MLP_NPARAM; i++) grad[i] = 0.0;
    double loss = 0.0;
    for (int64_t s = 0; s < N; s++) {
        const float *x = X + s * 6;
        double a1[32], h1[32], a2[32], h2[32];
        for (int j = 0; j < 32; j++) {
            double acc = prm[OR_MLP_B1 + j];
            for (int i = 0; i < 6; i++) acc += (double)prm[OR_MLP_W1 + j * 6 + i] * x[i];
            a1[j] = acc;
            h1[j] = acc > 0 ? acc : 0;
        }
        for (int j = 0; j < 32; j++) {
            double acc = prm[OR_MLP_B2 + j];
            for (int i = 0; i < 32; i++) acc += (double)prm[OR_MLP_W2 + j * 32 + i] * h1[i];
            a2[j] = acc;
            h2[j] = acc > 0 ? acc : 0;
        }
        double z = prm[OR_MLP_B3];
        for (int i = 0; i < 32; i++) z += (double)prm[OR_MLP_W3 + i] * h2[i];
        double t = y[s] ? 1.0 : 0.0;
        /* log(1 + e^z) - t z, written to avoid overflow */
        loss += (z > 0 ? z + log1p(exp(-z)) : log1p(exp(z))) - t * z;
        double dz = 1.0 / (1.0 + exp(-z)) - t;
        double d2[32], d1[32];
        grad[OR_MLP_B3] += dz;
        for (int i = 0; i < 32; i++) {
            grad[OR_MLP_W3 + i] += dz * h2[i];
            d2[i] = a2[i] > 0 ? dz * prm[OR_MLP_W3 + i] : 0.0;
        }
        for (int i = 0; i < 32; i++) d1[i] = 0.0;
        for (int j = 0; j < 32; j++) {
            grad[OR_MLP_B2 + j] += d2[j];
            for (int i = 0; i < 32; i++) {
                grad[OR_MLP_W2 + j * 32 + i] += d2[j] * h1[i];
                d1[i] += d2[j] * prm[OR_MLP_W2 + j * 32 + i];
            }
        }
        for (int j = 0; j < 32; j++) {
            double dj = a1[j] > 0 ? d1[j] : 0.0;
            grad[OR_MLP_B1 + j] += dj;
            for (int i = 0; i < 6; i++) grad[OR_MLP_W1 + j * 6 + i] += dj * x[i];
        }
    }
    if (N > 0) {
        for (int i = 0; i < OR_MLP_NPARAM; i++) grad[i] /= (double)N;
        loss /= (double)N;
    }
    return loss;
}

/* The logit of each of N feature rows (row-major [N][6]). */
void or_mlp_score(int64_t N, const float *X, const uint16_t *net, float *z)
{
    for (int64_t s = 0; s < N; s++) z[s] = or_mlp_forward(net, X + s * 6);
}
