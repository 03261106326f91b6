/*
 * CPU oracle for synchronous size-constrained label-propagation refinement under the
 * connectivity (lambda-1) metric.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential statement of what
 * the CUDA path must compute.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with the CUDA
 * library, and it never reads anything the CUDA library produced.
 *
 * Everything is integer arithmetic, so results are exact and must agree bit for bit with the
 * device path.  Weights, gains and block weights are int64.  Pin counts Phi(e, i) are int32:
 * 0 <= Phi(e, i) <= |e| <= P < 2^31 (the input bound), so every count is held exactly, and
 * the table of the largest workloads (m * k entries) takes half the host memory.
 *
 * Threads (oracle_set_threads, default 1): three loops whose items are independent may be
 * split into contiguous slices evaluated by separate threads: the eligibility of each vertex
 * (a function of the previous round's moved nets), the best move of each vertex (a function
 * of the state frozen at the start of the sub-round alone, Sec. 6 read synchronously), and
 * the objective (an integer sum of per-net terms).  Approval and application stay
 * sequential.  The results do not depend on the thread count.
 *
 * Definitions followed (paper Sec. 2 "Preliminaries"):
 *   H = (V, E, c, omega), positive integer weights; I(v) the incident nets of v.
 *   k-way partition Pi : V -> {0..k-1} (the paper numbers blocks 1..k).
 *   L_max = (1 + eps) * ceil(c(V) / k); read here as floor((1+eps)*ceil(c(V)/k)) computed
 *   in IEEE double, since block weights are integers.
 *   Phi(e, V_i) = |V_i intersect e|; Lambda(e) = {i : Phi(e,i) > 0}; lambda(e) = |Lambda(e)|.
 *   (lambda - 1)(Pi) = sum_e (lambda(e) - 1) * omega(e); an empty net (lambda = 0) counts 0.
 * Gain (Sec. 5, "Parallel Gain Calculation"):
 *   g_i(u) = b(u) - p_i(u),  b(u) = omega({e in I(u) : Phi(e, Pi(u)) = 1}),
 *                            p_i(u) = omega({e in I(u) : Phi(e, i) = 0}).
 * Label propagation (Sec. 6), in the deterministic synchronous form:
 *   round r: a vertex is eligible if it is the first round since creation, or if one of its
 *   incident nets had a pin moved in round r-1 (the paper's "u and its neighbours").
 *   The round is split into S sub-rounds; vertex u is active in sub-round
 *   splitmix64_finalizer(seed ^ (r << 32 | u)) mod S.  In a sub-round, every active eligible
 *   vertex picks the block with the highest positive gain whose weight (frozen at the start
 *   of the sub-round) plus c(u) stays within L_max; ties go to the smaller block id.
 *   Candidates are then approved per target block in (gain desc, vertex id asc) order while
 *   the inclusive prefix of their weights fits into L_max - w(t).  All approved moves are
 *   applied, Phi and the block weights are updated, and the objective is recomputed.
 * Variants (Sec. 6), both off by default:
 *   balance moves: a vertex without a feasible positive-gain target may move with gain 0 to a
 *   block t with room and w(t) + c(u) < w(Pi(u)) (the lightest such block, then the smaller id).
 *   revert of negative attributed gains (Sec. 5.2, Sec. 6): the attributed gain of a move is
 *   read as its gain when the sub-round's approved moves are performed one at a time in
 *   ascending vertex id (each net then sees its moves in that order, and crediting +omega(e)
 *   to the move that takes Phi(e, from) to 0 and -omega(e) to the one that takes Phi(e, to)
 *   to 1 gives exactly this gain).  After the sub-round, every move whose attributed gain is
 *   negative is undone.  A reverted move still counts as a move for eligibility.
 *
 * Build: gcc -O2 -shared -fPIC -pthread -o liboracle.so hgp_oracle.c -lm
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef struct {
    /* hypergraph (copied) */
    int32_t n, m, k;
    int64_t *net_off;      /* [m+1] */
    int32_t *pins;         /* [P]   */
    int64_t *vw;           /* [n]   vertex weights c(v) */
    int64_t *nw;           /* [m]   net weights omega(e) */
    int64_t *vtx_off;      /* [n+1] incident-net lists I(v) */
    int32_t *inc;          /* [P]   */
    /* parameters */
    int64_t lmax;
    int32_t subrounds;
    uint64_t seed;
    /* state */
    int32_t *part;         /* Pi */
    int32_t *phi;          /* [m*k] Phi(e,i) */
    int64_t *bw;           /* [k]  block weights c(V_i) */
    int64_t round;         /* global round counter */
    int32_t balance_moves; /* variant: zero-gain moves that improve the balance (Sec. 6) */
    int32_t revert_negative; /* variant: undo moves whose exact gain is negative (Sec. 6) */
    int all_eligible;      /* 1 until the first round has run */
    uint8_t *moved_prev;   /* [m]  net had a pin moved in the previous round */
    uint8_t *moved_cur;    /* [m]  net had a pin moved in the current round */
    /* sub-round scratch */
    int32_t *cand_t;       /* [n]  chosen target or -1 */
    int64_t *cand_g;       /* [n]  its gain */
    uint8_t *approved;     /* [n]  */
    int32_t *order;        /* [n]  */
    int32_t *from;         /* [n]  block an approved vertex left */
    int64_t *attr;         /* [n]  attributed gain of an approved move */
    uint8_t *selected;     /* [n]  rebalancing: passed the source-side selection */
    int32_t threads;       /* threads for the per-vertex candidate loop (1 = sequential) */
} oracle_t;

/* Per-round statistics, in this order: objective after the round, number of candidates,
 * number of approved moves, number of eligible vertices, heaviest block weight, number of
 * reverted moves. */
enum { ST_OBJ = 0, ST_CAND, ST_APPROVED, ST_ELIGIBLE, ST_MAXW, ST_REVERTED, ST_COUNT };

int64_t oracle_lmax(int64_t total_weight, int32_t k, double eps)
{
    int64_t avg = (total_weight + k - 1) / k;             /* ceil(c(V)/k), Sec. 2 */
    return (int64_t)floor((1.0 + eps) * (double)avg);
}

/* SplitMix64 output function (Steele, Lea, Flood: "Fast splittable pseudorandom number
 * generators", OOPSLA 2014). */
uint64_t oracle_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Sub-round of vertex u in round r: mix64(seed ^ (r << 32 | u)) mod S. */
int32_t oracle_subround_of(uint64_t seed, int64_t round, int32_t u, int32_t S)
{
    uint64_t z = oracle_mix64(seed ^ (((uint64_t)round << 32) | (uint64_t)(uint32_t)u));
    return (int32_t)(z % (uint64_t)S);
}

/* Runs fn(ctx, lo, hi, &acc) over `threads` contiguous slices of [0, count) and returns the
 * sum of the slices' acc.  Used only where every item's result is independent of the others
 * (an integer sum does not depend on how it is split); a slice whose thread cannot be started
 * runs in the calling thread. */
typedef void (*slice_fn)(void *ctx, int64_t lo, int64_t hi, int64_t *acc);
typedef struct {
    slice_fn fn;
    void *ctx;
    int64_t lo, hi, acc;
} slice_t;

static void *slice_worker(void *arg)
{
    slice_t *sl = (slice_t *)arg;
    sl->acc = 0;
    sl->fn(sl->ctx, sl->lo, sl->hi, &sl->acc);
    return NULL;
}

static int64_t for_slices(int32_t threads, int64_t count, slice_fn fn, void *ctx)
{
    enum { MAX_THREADS = 256 };
    const int32_t T = threads < 1 ? 1 : (threads > MAX_THREADS ? MAX_THREADS : threads);
    if (T == 1 || count < 4096) {
        int64_t acc = 0;
        fn(ctx, 0, count, &acc);
        return acc;
    }
    pthread_t th[MAX_THREADS];
    slice_t sl[MAX_THREADS];
    int started[MAX_THREADS];
    for (int32_t t = 0; t < T; ++t) {
        sl[t].fn = fn;
        sl[t].ctx = ctx;
        sl[t].lo = count * t / T;
        sl[t].hi = count * (t + 1) / T;
        started[t] = pthread_create(&th[t], NULL, slice_worker, &sl[t]) == 0;
        if (!started[t]) slice_worker(&sl[t]);
    }
    int64_t total = 0;
    for (int32_t t = 0; t < T; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        total += sl[t].acc;
    }
    return total;
}

/* (lambda(e) - 1) * omega(e) summed over the nets lo <= e < hi (an empty net counts 0). */
static void objective_slice(void *ctx, int64_t lo, int64_t hi, int64_t *acc)
{
    const oracle_t *o = (const oracle_t *)ctx;
    for (int64_t e = lo; e < hi; ++e) {
        int64_t lambda = 0;
        for (int32_t i = 0; i < o->k; ++i)
            if (o->phi[e * o->k + i] > 0) lambda++;
        if (lambda > 0) *acc += (lambda - 1) * o->nw[e];
    }
}

static int64_t objective_from_phi(const oracle_t *o)
{
    return for_slices(o->threads, o->m, objective_slice, (void *)o);
}

void oracle_destroy(oracle_t *o)
{
    if (!o) return;
    free(o->net_off); free(o->pins); free(o->vw); free(o->nw); free(o->vtx_off);
    free(o->inc); free(o->part); free(o->phi); free(o->bw); free(o->moved_prev);
    free(o->moved_cur); free(o->cand_t); free(o->cand_g); free(o->approved); free(o->order);
    free(o->from); free(o->attr); free(o->selected);
    free(o);
}

/* Returns NULL on allocation failure or invalid input. vertex_w / net_w may be NULL
 * (unit weights).  part is copied. */
oracle_t *oracle_create(int32_t n, int32_t m, const int64_t *net_off, const int32_t *pins,
                        const int32_t *vertex_w, const int32_t *net_w, int32_t k, double eps,
                        const int32_t *part, int32_t subrounds, uint64_t seed)
{
    if (n < 0 || m < 0 || k < 2 || subrounds < 1) return NULL;
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    if (!o) return NULL;
    int64_t P = net_off[m];
    o->n = n; o->m = m; o->k = k; o->subrounds = subrounds; o->seed = seed;
    o->net_off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    o->pins = (int32_t *)malloc(sizeof(int32_t) * ((size_t)P + 1));
    o->vw = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    o->nw = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    o->vtx_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    o->inc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)P + 1));
    o->part = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    o->phi = (int32_t *)calloc((size_t)m * k + 1, sizeof(int32_t));
    o->bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    o->moved_prev = (uint8_t *)calloc((size_t)m + 1, 1);
    o->moved_cur = (uint8_t *)calloc((size_t)m + 1, 1);
    o->cand_t = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    o->cand_g = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    o->approved = (uint8_t *)calloc((size_t)n + 1, 1);
    o->order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    o->from = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    o->attr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    o->selected = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!o->net_off || !o->pins || !o->vw || !o->nw || !o->vtx_off || !o->inc || !o->part ||
        !o->phi || !o->bw || !o->moved_prev || !o->moved_cur || !o->cand_t || !o->cand_g ||
        !o->approved || !o->order || !o->from || !o->attr || !o->selected) {
        oracle_destroy(o);
        return NULL;
    }
    memcpy(o->net_off, net_off, sizeof(int64_t) * ((size_t)m + 1));
    if (P) memcpy(o->pins, pins, sizeof(int32_t) * (size_t)P);
    for (int32_t v = 0; v < n; ++v) o->vw[v] = vertex_w ? vertex_w[v] : 1;
    for (int32_t e = 0; e < m; ++e) o->nw[e] = net_w ? net_w[e] : 1;
    for (int32_t v = 0; v < n; ++v) {
        if (part[v] < 0 || part[v] >= k) { oracle_destroy(o); return NULL; }
        o->part[v] = part[v];
    }

    /* incident nets I(v): count degrees, prefix sum, fill in net order */
    for (int64_t j = 0; j < P; ++j) o->vtx_off[pins[j] + 1]++;
    for (int32_t v = 0; v < n; ++v) o->vtx_off[v + 1] += o->vtx_off[v];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
        if (!fill) { oracle_destroy(o); return NULL; }
        memcpy(fill, o->vtx_off, sizeof(int64_t) * ((size_t)n + 1));
        for (int32_t e = 0; e < m; ++e)
            for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j)
                o->inc[fill[pins[j]]++] = e;
        free(fill);
    }

    /* Phi(e, i) by counting pins; block weights c(V_i) */
    for (int32_t e = 0; e < m; ++e)
        for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j)
            o->phi[(int64_t)e * k + o->part[pins[j]]]++;
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) { o->bw[o->part[v]] += o->vw[v]; total += o->vw[v]; }
    o->lmax = oracle_lmax(total, k, eps);
    o->round = 0;
    o->all_eligible = 1;
    o->threads = 1;
    return o;
}

/* g_i(u) = b(u) - p_i(u), Sec. 5, against the current Phi. */
int64_t oracle_gain(const oracle_t *o, int32_t u, int32_t i)
{
    int32_t a = o->part[u];
    int64_t b = 0, p = 0;
    for (int64_t j = o->vtx_off[u]; j < o->vtx_off[u + 1]; ++j) {
        int32_t e = o->inc[j];
        if (o->phi[(int64_t)e * o->k + a] == 1) b += o->nw[e];
        if (o->phi[(int64_t)e * o->k + i] == 0) p += o->nw[e];
    }
    return b - p;
}

static int eligible(const oracle_t *o, int32_t u)
{
    if (o->all_eligible) return 1;
    for (int64_t j = o->vtx_off[u]; j < o->vtx_off[u + 1]; ++j)
        if (o->moved_prev[o->inc[j]]) return 1;
    return 0;
}

/* Best feasible positive-gain target of u against the frozen state (Sec. 6): the block
 * with the highest gain, smallest id on ties; -1 if no block has positive gain and room.
 * With the balance-move variant, a vertex without such a block may instead take a zero-gain
 * move that improves the balance (Sec. 6): to a block t with room and w(t) + c(u) < w(a), the
 * lightest such block (smallest id among equally light ones). */
static void best_move(const oracle_t *o, int32_t u, int32_t *t_out, int64_t *g_out)
{
    int32_t a = o->part[u];
    int32_t best_t = -1;
    int64_t best_g = 0;
    for (int32_t i = 0; i < o->k; ++i) {
        if (i == a) continue;
        int64_t g = oracle_gain(o, u, i);
        if (g > best_g && o->bw[i] + o->vw[u] <= o->lmax) { best_t = i; best_g = g; }
    }
    if (best_t < 0 && o->balance_moves) {
        for (int32_t i = 0; i < o->k; ++i) {
            if (i == a) continue;
            const int64_t wi = o->bw[i] + o->vw[u];
            if (wi > o->lmax || wi >= o->bw[a] || oracle_gain(o, u, i) != 0) continue;
            if (best_t < 0 || o->bw[i] < o->bw[best_t]) best_t = i;
        }
    }
    *t_out = best_t;
    *g_out = best_g;
}

void oracle_set_variant(oracle_t *o, int32_t balance_moves, int32_t revert_negative)
{
    o->balance_moves = balance_moves;
    o->revert_negative = revert_negative;
}

static const oracle_t *g_sort_ctx;
static int by_gain_desc_id_asc(const void *x, const void *y)
{
    int32_t u = *(const int32_t *)x, v = *(const int32_t *)y;
    int64_t gu = g_sort_ctx->cand_g[u], gv = g_sort_ctx->cand_g[v];
    if (gu != gv) return gu > gv ? -1 : 1;
    return (u > v) - (u < v);
}

/* Candidates of sub-round s of the NEXT round against the current state, without
 * applying anything.  target[u] = -1 for inactive, ineligible or non-candidate vertices. */
void oracle_candidates(const oracle_t *o, int32_t s, int32_t *target, int64_t *gain)
{
    for (int32_t u = 0; u < o->n; ++u) {
        target[u] = -1;
        gain[u] = 0;
        if (oracle_subround_of(o->seed, o->round, u, o->subrounds) != s) continue;
        if (!eligible(o, u)) continue;
        best_move(o, u, &target[u], &gain[u]);
    }
}

/* Best moves (Sec. 6) of the vertices lo <= u < hi that are eligible and active in sub-round s
 * of round r, against the current (frozen) state; cand_t[u] = -1 for the others. */
typedef struct {
    oracle_t *o;
    const uint8_t *elig;
    int64_t r;
    int32_t s;
} cand_ctx_t;

static void candidates_slice(void *ctx, int64_t lo, int64_t hi, int64_t *acc)
{
    cand_ctx_t *c = (cand_ctx_t *)ctx;
    oracle_t *o = c->o;
    for (int64_t u = lo; u < hi; ++u) {
        o->cand_t[u] = -1;
        o->cand_g[u] = 0;
        if (!c->elig[u] || oracle_subround_of(o->seed, c->r, (int32_t)u, o->subrounds) != c->s) continue;
        best_move(o, (int32_t)u, &o->cand_t[u], &o->cand_g[u]);
        if (o->cand_t[u] >= 0) (*acc)++;
    }
}

static void sub_round_candidates(oracle_t *o, const uint8_t *elig, int64_t r, int32_t s)
{
    cand_ctx_t c = {o, elig, r, s};
    for_slices(o->threads, o->n, candidates_slice, &c);
}

/* elig[u] = eligible(u) for lo <= u < hi; acc counts the eligible vertices. */
typedef struct {
    const oracle_t *o;
    uint8_t *elig;
} elig_ctx_t;

static void eligible_slice(void *ctx, int64_t lo, int64_t hi, int64_t *acc)
{
    elig_ctx_t *c = (elig_ctx_t *)ctx;
    for (int64_t u = lo; u < hi; ++u) {
        c->elig[u] = (uint8_t)eligible(c->o, (int32_t)u);
        *acc += c->elig[u];
    }
}

/* Threads used by the candidate step of oracle_refine (1 = sequential; results identical). */
void oracle_set_threads(oracle_t *o, int32_t threads) { o->threads = threads < 1 ? 1 : threads; }

/* Moves u from its block to t: partition, block weights, Phi, and (mark != 0) the moved-net
 * marks that decide the next LP round's eligibility. */
static void move_vertex_marked(oracle_t *o, int32_t u, int32_t t, int mark)
{
    const int32_t a = o->part[u], k = o->k;
    o->part[u] = t;
    o->bw[a] -= o->vw[u];
    o->bw[t] += o->vw[u];
    for (int64_t j = o->vtx_off[u]; j < o->vtx_off[u + 1]; ++j) {
        const int32_t e = o->inc[j];
        o->phi[(int64_t)e * k + a]--;
        o->phi[(int64_t)e * k + t]++;
        if (mark) o->moved_cur[e] = 1;
    }
}

static void move_vertex(oracle_t *o, int32_t u, int32_t t) { move_vertex_marked(o, u, t, 1); }

/* Runs `rounds` synchronous LP rounds.  stats: NULL or [rounds * ST_COUNT].
 * moves: NULL or [max_moves * 4] receiving (global sub-round index, u, from, to) for each
 * applied move in application order; *num_moves receives the count (may exceed max_moves,
 * in which case the log is truncated). */
int oracle_refine(oracle_t *o, int32_t rounds, int64_t *stats, int64_t *moves,
                  int64_t max_moves, int64_t *num_moves)
{
    const int32_t n = o->n, m = o->m, k = o->k, S = o->subrounds;
    int64_t logged = 0;
    for (int32_t rr = 0; rr < rounds; ++rr) {
        const int64_t r = o->round;
        int64_t n_cand = 0, n_appr = 0, n_elig = 0, n_rev = 0;
        memset(o->moved_cur, 0, (size_t)m);
        /* eligibility is fixed for the whole round: it depends only on the previous round */
        uint8_t *elig_copy = (uint8_t *)malloc((size_t)n + 1);
        if (!elig_copy) return -1;
        {
            elig_ctx_t c = {o, elig_copy};
            n_elig = for_slices(o->threads, n, eligible_slice, &c);
        }

        for (int32_t s = 0; s < S; ++s) {
            /* (1) candidates against the state frozen at the start of the sub-round */
            sub_round_candidates(o, elig_copy, r, s);
            int32_t cnt = 0;
            for (int32_t u = 0; u < n; ++u)
                if (o->cand_t[u] >= 0) { o->order[cnt++] = u; n_cand++; }
            /* (2) approval per target block: (gain desc, id asc), inclusive prefix sums */
            g_sort_ctx = o;
            qsort(o->order, (size_t)cnt, sizeof(int32_t), by_gain_desc_id_asc);
            for (int32_t u = 0; u < n; ++u) o->approved[u] = 0;
            for (int32_t t = 0; t < k; ++t) {
                int64_t acc = 0;
                for (int32_t j = 0; j < cnt; ++j) {
                    int32_t u = o->order[j];
                    if (o->cand_t[u] != t) continue;
                    acc += o->vw[u];
                    if (o->bw[t] + acc <= o->lmax) o->approved[u] = 1;
                }
            }
            /* (3) apply every approved move (ascending vertex id); with the revert variant,
             * the attributed gain of each is its gain just before it is performed */
            for (int32_t u = 0; u < n; ++u) {
                if (!o->approved[u]) continue;
                int32_t a = o->part[u], t = o->cand_t[u];
                if (o->revert_negative) {
                    o->from[u] = a;
                    o->attr[u] = oracle_gain(o, u, t);
                }
                move_vertex(o, u, t);
                if (moves && logged < max_moves) {
                    int64_t *mv = moves + 4 * logged;
                    mv[0] = r * S + s; mv[1] = u; mv[2] = a; mv[3] = t;
                }
                logged++;
                n_appr++;
            }
            /* (4) revert variant: undo every move with a negative attributed gain */
            if (o->revert_negative) {
                for (int32_t u = 0; u < n; ++u) {
                    if (!o->approved[u] || o->attr[u] >= 0) continue;
                    const int32_t t = o->part[u], a = o->from[u];
                    move_vertex(o, u, a);
                    if (moves && logged < max_moves) {
                        int64_t *mv = moves + 4 * logged;
                        mv[0] = r * S + s; mv[1] = u; mv[2] = t; mv[3] = a;
                    }
                    logged++;
                    n_rev++;
                }
            }
        }
        free(elig_copy);
        memcpy(o->moved_prev, o->moved_cur, (size_t)m);
        o->all_eligible = 0;
        o->round++;
        if (stats) {
            int64_t maxw = 0;
            for (int32_t i = 0; i < k; ++i) if (o->bw[i] > maxw) maxw = o->bw[i];
            int64_t *st = stats + (int64_t)rr * ST_COUNT;
            st[ST_OBJ] = objective_from_phi(o);
            st[ST_CAND] = n_cand;
            st[ST_APPROVED] = n_appr;
            st[ST_ELIGIBLE] = n_elig;
            st[ST_MAXW] = maxw;
            st[ST_REVERTED] = n_rev;
        }
    }
    if (num_moves) *num_moves = logged;
    return 0;
}

static int64_t heaviest_block(const oracle_t *o)
{
    int64_t w = 0;
    for (int32_t i = 0; i < o->k; ++i) if (o->bw[i] > w) w = o->bw[i];
    return w;
}

/* Rebalancing (Sec. 8), in a synchronous form.  A pass splits the vertices into the S
 * sub-rounds of the hash with round number 2^30 + pass (so it never coincides with an LP
 * round).  In a sub-round, against the frozen state, a vertex u of an overloaded block a
 * (w(a) > L_max) picks the block t != a with room (w(t) + c(u) <= L_max) of highest gain,
 * smaller id on ties; in phase 1 only a gain >= 0 makes it a candidate (the paper's immediate
 * non-negative moves), in phase 2 any gain does (the paper's second step, least connectivity
 * increase first).  Candidates are ordered by (gain desc, id asc).  Source side: a candidate
 * is selected while the weight that left its block before it, in that order, is still below
 * w(a) - L_max (its block is still overloaded when it leaves).  Target side: selected
 * candidates are approved while the inclusive prefix of their weights fits L_max - w(t).
 * Approved moves are applied; they do not count as moves for LP eligibility.
 * Passes run while a block is overloaded and at most max_passes times: the first pass is
 * phase 1 (one sweep over all vertices, as in the paper), every later pass is phase 2, and a
 * phase-2 pass without moves ends it.
 * stats: NULL or [max_passes * ST_COUNT] per pass; phases: NULL or [max_passes].
 * moves as in oracle_refine (first field = pass * S + sub-round).  Returns 0, -1 on failure. */
int oracle_rebalance(oracle_t *o, int32_t max_passes, int64_t *stats, int32_t *phases,
                     int32_t *num_passes, int64_t *moves, int64_t max_moves, int64_t *num_moves)
{
    const int32_t n = o->n, k = o->k, S = o->subrounds;
    int32_t phase = 1, pass = 0;
    int64_t logged = 0;
    while (pass < max_passes && heaviest_block(o) > o->lmax) {
        const int64_t rid = ((int64_t)1 << 30) + pass;
        int64_t n_cand = 0, n_appr = 0, n_cons = 0;
        for (int32_t s = 0; s < S; ++s) {
            /* (1) candidates of overloaded blocks against the frozen state */
            int32_t cnt = 0;
            for (int32_t u = 0; u < n; ++u) {
                o->cand_t[u] = -1;
                o->cand_g[u] = 0;
                o->selected[u] = 0;
                o->approved[u] = 0;
                const int32_t a = o->part[u];
                if (oracle_subround_of(o->seed, rid, u, S) != s || o->bw[a] <= o->lmax) continue;
                n_cons++;
                int32_t best_t = -1;
                int64_t best_g = 0;
                for (int32_t i = 0; i < k; ++i) {
                    if (i == a || o->bw[i] + o->vw[u] > o->lmax) continue;
                    const int64_t g = oracle_gain(o, u, i);
                    if (best_t < 0 || g > best_g) { best_t = i; best_g = g; }
                }
                if (best_t < 0 || (phase == 1 && best_g < 0)) continue;
                o->cand_t[u] = best_t;
                o->cand_g[u] = best_g;
                o->order[cnt++] = u;
                n_cand++;
            }
            g_sort_ctx = o;
            qsort(o->order, (size_t)cnt, sizeof(int32_t), by_gain_desc_id_asc);
            /* (2) source side: leave while the block is still overloaded */
            for (int32_t a = 0; a < k; ++a) {
                int64_t left = 0;
                for (int32_t j = 0; j < cnt; ++j) {
                    const int32_t u = o->order[j];
                    if (o->part[u] != a) continue;
                    if (left < o->bw[a] - o->lmax) o->selected[u] = 1;
                    left += o->vw[u];
                }
            }
            /* (3) target side: inclusive prefix of the selected candidates fits */
            for (int32_t t = 0; t < k; ++t) {
                int64_t acc = 0;
                for (int32_t j = 0; j < cnt; ++j) {
                    const int32_t u = o->order[j];
                    if (!o->selected[u] || o->cand_t[u] != t) continue;
                    acc += o->vw[u];
                    if (o->bw[t] + acc <= o->lmax) o->approved[u] = 1;
                }
            }
            /* (4) apply (ascending id), no eligibility marks */
            for (int32_t u = 0; u < n; ++u) {
                if (!o->approved[u]) continue;
                const int32_t a = o->part[u], t = o->cand_t[u];
                move_vertex_marked(o, u, t, 0);
                if (moves && logged < max_moves) {
                    int64_t *mv = moves + 4 * logged;
                    mv[0] = (int64_t)pass * S + s; mv[1] = u; mv[2] = a; mv[3] = t;
                }
                logged++;
                n_appr++;
            }
        }
        if (stats) {
            int64_t *st = stats + (int64_t)pass * ST_COUNT;
            st[ST_OBJ] = objective_from_phi(o);
            st[ST_CAND] = n_cand;
            st[ST_APPROVED] = n_appr;
            st[ST_ELIGIBLE] = n_cons;
            st[ST_MAXW] = heaviest_block(o);
            st[ST_REVERTED] = 0;
        }
        if (phases) phases[pass] = phase;
        pass++;
        if (phase == 1) phase = 2;
        else if (n_appr == 0) break;
    }
    if (num_passes) *num_passes = pass;
    if (num_moves) *num_moves = logged;
    return 0;
}

int64_t oracle_objective(const oracle_t *o) { return objective_from_phi(o); }
int64_t oracle_lmax_of(const oracle_t *o) { return o->lmax; }
int64_t oracle_round_of(const oracle_t *o) { return o->round; }

void oracle_get_partition(const oracle_t *o, int32_t *out)
{
    memcpy(out, o->part, sizeof(int32_t) * (size_t)o->n);
}

void oracle_get_block_weights(const oracle_t *o, int64_t *out)
{
    memcpy(out, o->bw, sizeof(int64_t) * (size_t)o->k);
}

void oracle_get_phi(const oracle_t *o, int64_t *out)
{
    const int64_t cnt = (int64_t)o->m * o->k;
    for (int64_t x = 0; x < cnt; ++x) out[x] = o->phi[x];
}

/* Rows e0 <= e < e1 of Phi into out[(e1 - e0) * k] (for instances too large to copy whole). */
void oracle_get_phi_rows(const oracle_t *o, int32_t e0, int32_t e1, int32_t *out)
{
    memcpy(out, o->phi + (int64_t)e0 * o->k, sizeof(int32_t) * (size_t)(e1 - e0) * (size_t)o->k);
}

/* Candidates of round 0, sub-round s, for a sample of vertices, straight from the input
 * (no full Phi table): Phi(e, .) is counted from the pins of each net incident to a
 * sampled vertex.  Used to check full-size instances whose Phi table would not fit the
 * host.  Requires the sampled vertices to be distinct.  Returns 0, or -1 on allocation
 * failure. */
int oracle_sample_candidates(int32_t n, int32_t m, const int64_t *net_off, const int32_t *pins,
                             const int32_t *vertex_w, const int32_t *net_w, int32_t k,
                             double eps, const int32_t *part, int32_t subrounds, uint64_t seed,
                             int32_t s, int32_t count, const int32_t *sample,
                             int32_t *target, int64_t *gain)
{
    int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t *phi_row = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    /* per sampled vertex: b, and p_i accumulated over its incident nets */
    int64_t *b = (int64_t *)calloc((size_t)count + 1, sizeof(int64_t));
    int64_t *p = (int64_t *)calloc(((size_t)count + 1) * (size_t)k, sizeof(int64_t));
    if (!bw || !slot || !phi_row || !b || !p) {
        free(bw); free(slot); free(phi_row); free(b); free(p);
        return -1;
    }
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t c = vertex_w ? vertex_w[v] : 1;
        bw[part[v]] += c;
        total += c;
        slot[v] = -1;
    }
    int64_t lmax = oracle_lmax(total, k, eps);
    for (int32_t j = 0; j < count; ++j) slot[sample[j]] = j;
    for (int32_t e = 0; e < m; ++e) {
        int any = 0;
        for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) if (slot[pins[j]] >= 0) { any = 1; break; }
        if (!any) continue;
        for (int32_t i = 0; i < k; ++i) phi_row[i] = 0;
        for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) phi_row[part[pins[j]]]++;
        int64_t w = net_w ? net_w[e] : 1;
        for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) {
            int32_t q = slot[pins[j]];
            if (q < 0) continue;
            if (phi_row[part[pins[j]]] == 1) b[q] += w;
            for (int32_t i = 0; i < k; ++i) if (phi_row[i] == 0) p[(int64_t)q * k + i] += w;
        }
    }
    for (int32_t q = 0; q < count; ++q) {
        int32_t u = sample[q];
        target[q] = -1;
        gain[q] = 0;
        if (oracle_subround_of(seed, 0, u, subrounds) != s) continue;
        int32_t a = part[u];
        int64_t c = vertex_w ? vertex_w[u] : 1;
        for (int32_t i = 0; i < k; ++i) {
            if (i == a) continue;
            int64_t g = b[q] - p[(int64_t)q * k + i];
            if (g > gain[q] && bw[i] + c <= lmax) { target[q] = i; gain[q] = g; }
        }
    }
    free(bw); free(slot); free(phi_row); free(b); free(p);
    return 0;
}

/* Exact gains of a move sequence (Sec. 5.4): moves[3*j..3*j+2] = (u, from, to), performed in
 * order j = 0..count-1; gain[j] = g_to(u) (Sec. 5) against the state after moves 0..j-1.
 * The oracle's own state is not changed.  Returns -1 if a move is invalid (u out of range,
 * from != Pi(u) at that point, to out of range or equal to from, a vertex moved twice). */
int oracle_exact_gains(const oracle_t *o, int32_t count, const int32_t *moves, int64_t *gain)
{
    const int32_t n = o->n, m = o->m, k = o->k;
    int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m * k + 1));
    int32_t *part = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint8_t *seen = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!phi || !part || !seen) { free(phi); free(part); free(seen); return -1; }
    memcpy(phi, o->phi, sizeof(int32_t) * (size_t)m * k);
    memcpy(part, o->part, sizeof(int32_t) * (size_t)n);
    int rc = 0;
    for (int32_t j = 0; j < count && rc == 0; ++j) {
        const int32_t u = moves[3 * j], a = moves[3 * j + 1], b = moves[3 * j + 2];
        if (u < 0 || u >= n || seen[u] || a != part[u] || b < 0 || b >= k || b == a) { rc = -1; break; }
        seen[u] = 1;
        int64_t bu = 0, pb = 0;
        for (int64_t x = o->vtx_off[u]; x < o->vtx_off[u + 1]; ++x) {
            const int32_t e = o->inc[x];
            if (phi[(int64_t)e * k + a] == 1) bu += o->nw[e];
            if (phi[(int64_t)e * k + b] == 0) pb += o->nw[e];
        }
        gain[j] = bu - pb;
        for (int64_t x = o->vtx_off[u]; x < o->vtx_off[u + 1]; ++x) {
            const int32_t e = o->inc[x];
            phi[(int64_t)e * k + a]--;
            phi[(int64_t)e * k + b]++;
        }
        part[u] = b;
    }
    free(phi); free(part); free(seen);
    return rc;
}

/* ---------------------------------------------------------------------------------------
 * Contraction (Sec. 3.2): coarse hypergraph of a vertex clustering.
 *   cluster ids (values in [0, n)) are remapped to 0..n'-1 in increasing order (a prefix sum
 *   over the used ids); c'(C) = sum of c(u) over the cluster; every net's pins are mapped to
 *   their clusters, sorted and de-duplicated; nets left with fewer than two pins are removed;
 *   identical nets (equal sorted pin lists) become one net whose weight is the sum of theirs,
 *   kept at the position of the smallest original net id; the coarse nets keep the order of
 *   those representatives.  map[u] = coarse id of u.
 */
typedef struct {
    int32_t n, m;
    int64_t P;
    int64_t *net_off;   /* [m+1] */
    int32_t *pins;      /* [P] */
    int64_t *vw;        /* [n] */
    int64_t *nw;        /* [m] */
    int32_t *map;       /* [fine n] */
    int32_t fine_n;
} oracle_coarse_t;

static int cmp_i32(const void *x, const void *y)
{
    const int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* context for ordering nets by (size, pin list, original id) */
static const int64_t *g_ct_off;
static const int32_t *g_ct_pins;
static int by_pin_list(const void *x, const void *y)
{
    const int32_t e = *(const int32_t *)x, f = *(const int32_t *)y;
    const int64_t se = g_ct_off[e + 1] - g_ct_off[e], sf = g_ct_off[f + 1] - g_ct_off[f];
    if (se != sf) return se < sf ? -1 : 1;
    for (int64_t j = 0; j < se; ++j) {
        const int32_t a = g_ct_pins[g_ct_off[e] + j], b = g_ct_pins[g_ct_off[f] + j];
        if (a != b) return a < b ? -1 : 1;
    }
    return (e > f) - (e < f);
}

void oracle_coarse_destroy(oracle_coarse_t *c)
{
    if (!c) return;
    free(c->net_off); free(c->pins); free(c->vw); free(c->nw); free(c->map);
    free(c);
}

/* Returns 0, -1 on allocation failure, -2 on a cluster id outside [0, n). */
int oracle_contract(int32_t n, int32_t m, const int64_t *net_off, const int32_t *pins,
                    const int32_t *vertex_w, const int32_t *net_w, const int32_t *cluster,
                    oracle_coarse_t **out)
{
    *out = NULL;
    for (int32_t u = 0; u < n; ++u) if (cluster[u] < 0 || cluster[u] >= n) return -2;
    const int64_t P = net_off[m];
    oracle_coarse_t *c = (oracle_coarse_t *)calloc(1, sizeof(oracle_coarse_t));
    int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t *off1 = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    int32_t *pins1 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)P + 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    int32_t *rep = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    int64_t *wsum = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    if (!c || !cid || !off1 || !pins1 || !order || !rep || !wsum) goto oom;
    c->fine_n = n;
    /* (1) remap the used cluster ids by a prefix sum */
    for (int32_t i = 0; i <= n; ++i) cid[i] = 0;
    for (int32_t u = 0; u < n; ++u) cid[cluster[u]] = 1;
    {
        int32_t run = 0;
        for (int32_t i = 0; i < n; ++i) { const int32_t used = cid[i]; cid[i] = run; run += used; }
        c->n = run;
    }
    c->map = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    c->vw = (int64_t *)calloc((size_t)c->n + 1, sizeof(int64_t));
    if (!c->map || !c->vw) goto oom;
    /* (2) cluster weights */
    for (int32_t u = 0; u < n; ++u) {
        c->map[u] = cid[cluster[u]];
        c->vw[c->map[u]] += vertex_w ? vertex_w[u] : 1;
    }
    /* (3) pins mapped, sorted and de-duplicated per net */
    off1[0] = 0;
    for (int32_t e = 0; e < m; ++e) {
        int64_t w = off1[e];
        for (int64_t j = net_off[e]; j < net_off[e + 1]; ++j) pins1[w++] = c->map[pins[j]];
        qsort(pins1 + off1[e], (size_t)(w - off1[e]), sizeof(int32_t), cmp_i32);
        int64_t k = off1[e];
        for (int64_t j = off1[e]; j < w; ++j)
            if (j == off1[e] || pins1[j] != pins1[j - 1]) pins1[k++] = pins1[j];
        off1[e + 1] = k;
    }
    /* (4) nets with at least two pins, grouped by identical pin lists */
    int32_t kept = 0;
    for (int32_t e = 0; e < m; ++e) {
        rep[e] = -1;
        if (off1[e + 1] - off1[e] >= 2) order[kept++] = e;
    }
    g_ct_off = off1;
    g_ct_pins = pins1;
    qsort(order, (size_t)kept, sizeof(int32_t), by_pin_list);
    for (int32_t i = 0; i < kept; ++i) {
        const int32_t e = order[i];
        int same = 0;
        if (i > 0) {
            const int32_t f = order[i - 1];
            const int64_t s = off1[e + 1] - off1[e];
            same = s == off1[f + 1] - off1[f] &&
                   memcmp(pins1 + off1[e], pins1 + off1[f], sizeof(int32_t) * (size_t)s) == 0;
        }
        rep[e] = same ? rep[order[i - 1]] : e;   /* the group's first = its smallest id */
        wsum[rep[e]] += net_w ? net_w[e] : 1;
    }
    /* (5) coarse nets: the representatives in original order */
    {
        int32_t m2 = 0;
        int64_t P2 = 0;
        for (int32_t e = 0; e < m; ++e)
            if (rep[e] == e) { m2++; P2 += off1[e + 1] - off1[e]; }
        c->m = m2;
        c->P = P2;
        c->net_off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m2 + 1));
        c->pins = (int32_t *)malloc(sizeof(int32_t) * ((size_t)P2 + 1));
        c->nw = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m2 + 1));
        if (!c->net_off || !c->pins || !c->nw) goto oom;
        int32_t i2 = 0;
        c->net_off[0] = 0;
        for (int32_t e = 0; e < m; ++e) {
            if (rep[e] != e) continue;
            const int64_t s = off1[e + 1] - off1[e];
            memcpy(c->pins + c->net_off[i2], pins1 + off1[e], sizeof(int32_t) * (size_t)s);
            c->nw[i2] = wsum[e];
            c->net_off[i2 + 1] = c->net_off[i2] + s;
            i2++;
        }
    }
    free(cid); free(off1); free(pins1); free(order); free(rep); free(wsum);
    *out = c;
    return 0;
oom:
    free(cid); free(off1); free(pins1); free(order); free(rep); free(wsum);
    oracle_coarse_destroy(c);
    return -1;
}

void oracle_coarse_sizes(const oracle_coarse_t *c, int32_t *n, int32_t *m, int64_t *P)
{
    *n = c->n; *m = c->m; *P = c->P;
}

void oracle_coarse_copy(const oracle_coarse_t *c, int64_t *net_off, int32_t *pins, int64_t *vw,
                        int64_t *nw, int32_t *map)
{
    memcpy(net_off, c->net_off, sizeof(int64_t) * ((size_t)c->m + 1));
    memcpy(pins, c->pins, sizeof(int32_t) * (size_t)c->P);
    memcpy(vw, c->vw, sizeof(int64_t) * (size_t)c->n);
    memcpy(nw, c->nw, sizeof(int64_t) * (size_t)c->m);
    memcpy(map, c->map, sizeof(int32_t) * (size_t)c->fine_n);
}
