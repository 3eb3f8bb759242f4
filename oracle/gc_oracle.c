/*
 * gc_oracle.c -- plain, single-threaded CPU oracle for speculative distance-1
 * graph coloring with iterative recoloring (Sariyuce, Saule, Catalyurek,
 * "On Distributed Graph Coloring with Iterative Recoloring", arXiv 1407.6745).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline load it.  It shares no code with the CUDA path: it has its own
 * Philox generator, its own graph walk and its own permutation logic.
 *
 * Every routine follows the paper's steps literally, without blocking, fusion
 * or reordering beyond what the paper states:
 *
 *   - Alg. 1 (Sec. 2.1, sequential greedy): forbiddenColors marker array,
 *     color[v] = min{ i > 0 : forbiddenColors[i] != v }.
 *   - First Fit (Sec. 2.1): the smallest permissible color.
 *   - Random-X Fit (Sec. 3.2): a color drawn uniformly among the first X
 *     permissible colors.
 *   - Speculative rounds (Sec. 2.2): all uncolored vertices are tentatively
 *     colored, conflicts are detected, one endpoint of each conflicting edge
 *     keeps its color, chosen by a random total order fixed beforehand, the
 *     other is colored again in the next round, until no conflict remains.
 *   - Recoloring (Sec. 2.1 Culberson's iterated greedy; Sec. 3 RC): color
 *     classes of the previous coloring are recolored one class after the
 *     other, in a chosen class permutation (RV, NI, ND, RAND with Knuth's
 *     shuffle, Sec. 3), each vertex by First Fit against the new colors of
 *     the classes already recolored.
 *
 * Readings where the paper is silent (the one-GPU data-parallel reading):
 *   - a round is Jacobi: every tentative color is chosen against the colors
 *     fixed before the round (a snapshot), never against other tentative
 *     colors of the same round;
 *   - a vertex loses iff some neighbor has the same tentative color and a
 *     larger (priority, id) pair; prio(v) = Philox4x32-10(key = seed,
 *     counter = (v_lo, v_hi, 0, 1)).w0;
 *   - Random-X Fit takes the j-th permissible color (0-based) with
 *     j = floor(w0 * X / 2^32), w0 = Philox(seed, (v_lo, v_hi, r, 2)).w0,
 *     r the round number; permissible colors are those not used by a colored
 *     neighbor in the snapshot, the palette is unbounded;
 *   - recoloring uses First Fit; absent colors form no class; NI/ND ties go
 *     to the smaller color; RAND is Fisher-Yates from the ascending list of
 *     present colors, i = k-1 .. 1, j = floor(w0 * (i+1) / 2^32) with
 *     w0 = Philox(seed, (i, it, 0, 3)).w0, it the iteration number;
 *   - within a class, vertices are visited in increasing id (any order gives
 *     the same result, a class being an independent set);
 *   - vertex-visit orderings become the first key of the conflict priority
 *     (one GPU thread per vertex leaves no visit order): Largest First
 *     (Sec. 2.2.1) uses min(deg(v), 65535); asynchronous recoloring (aRC,
 *     Sec. 3) colors again from scratch by the speculative rounds with First
 *     Fit, the first key being 65535 - min(rank, 65535), rank the position
 *     of v's previous color class in the iteration's class permutation; the
 *     second key is the upper 16 bits of the Philox priority, then the id;
 *   - permutation schedules (Sec. 4.2.1): ND-RAND%x uses RAND at iterations
 *     x, 2x, 3x, ... and ND at the others; ND-RAND%2^i uses RAND at the
 *     iterations that are powers of two from 2 on (2, 4, 8, ...) and ND at
 *     the others; iterations are counted from 1 there, so iteration t uses
 *     the RAND draws of iteration number t - 1 above.
 *
 * The Philox4x32-10 generator is written from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): a 10-round Feistel-like network on four 32-bit words using the two
 * multipliers 0xD2511F53 and 0xCD9E8D57 and the Weyl key increments
 * 0x9E3779B9 and 0xBB67AE85.  It is pinned against an independent
 * implementation, PyTorch's open-source at::Philox4_32 engine, whole blocks
 * and the three counter layouts below (tests/test_philox_pin.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID_ARG 1
#define OR_ERR_BAD_GRAPH 2
#define OR_ERR_IMPROPER_INPUT 3
#define OR_ERR_OOM 4
#define OR_ERR_ROUND_LIMIT 7

#define PERM_REVERSE 0
#define PERM_NONINC 1
#define PERM_NONDEC 2
#define PERM_RANDOM 3
/* schedules: 4 = ND-RAND%2^i; 256 + x = ND-RAND%x, 1 <= x <= 65535 */
#define SCHED_POW2 4
#define SCHED_EVERY_BASE 256
#define SCHED_EVERY_MAX (256 + 65535)

#define TAG_PRIO 1u
#define TAG_RXF 2u
#define TAG_PERM 3u

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11)                                               */
/* ------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0, p1;
        uint32_t n0, n1, n2, n3;
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        n1 = (uint32_t)p1;
        n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_w0(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                          uint32_t tag)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = a; ctr[1] = b; ctr[2] = c; ctr[3] = tag;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* floor(w * m / 2^32): an index in [0, m) from a 32-bit draw. */
static uint32_t scale_draw(uint32_t w, uint32_t m)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)m) >> 32);
}

uint32_t oracle_priority(uint64_t seed, int64_t v)
{
    return philox_w0(seed, (uint32_t)v, (uint32_t)((uint64_t)v >> 32), 0u, TAG_PRIO);
}

uint32_t oracle_rxf_draw(uint64_t seed, int64_t v, int32_t round)
{
    return philox_w0(seed, (uint32_t)v, (uint32_t)((uint64_t)v >> 32),
                     (uint32_t)round, TAG_RXF);
}

uint32_t oracle_perm_draw(uint64_t seed, int32_t i, int32_t iteration)
{
    return philox_w0(seed, (uint32_t)i, (uint32_t)iteration, 0u, TAG_PERM);
}

/* ------------------------------------------------------------------ */
/* Graph checks                                                        */
/* ------------------------------------------------------------------ */

/* Offsets must start at 0, never decrease and end at nnz; every neighbor id
 * must be a vertex.  (Self-loops are reported by oracle_validate as a
 * conflict; the coloring routines simply never let v constrain itself.) */
static int check_graph(int64_t n, const int64_t* off, const int32_t* idx)
{
    int64_t v, e;
    if (n < 0) return OR_ERR_INVALID_ARG;
    if (n == 0) return OR_OK;
    if (!off) return OR_ERR_INVALID_ARG;
    if (off[0] != 0) return OR_ERR_BAD_GRAPH;
    for (v = 0; v < n; ++v)
        if (off[v + 1] < off[v]) return OR_ERR_BAD_GRAPH;
    if (off[n] > 0 && !idx) return OR_ERR_INVALID_ARG;
    for (e = 0; e < off[n]; ++e)
        if (idx[e] < 0 || (int64_t)idx[e] >= n) return OR_ERR_BAD_GRAPH;
    return OR_OK;
}

/* The graph to be colored must have no self-loop: C(u) != C(v) cannot hold on
 * an edge (v, v) (Sec. 1).  (Validation instead counts a loop as a conflict.) */
static int check_colorable(int64_t n, const int64_t* off, const int32_t* idx)
{
    int64_t v, e;
    int status = check_graph(n, off, idx);
    if (status != OR_OK) return status;
    for (v = 0; v < n; ++v)
        for (e = off[v]; e < off[v + 1]; ++e)
            if ((int64_t)idx[e] == v) return OR_ERR_BAD_GRAPH;
    return OR_OK;
}

static int64_t max_degree(int64_t n, const int64_t* off)
{
    int64_t v, d = 0;
    for (v = 0; v < n; ++v)
        if (off[v + 1] - off[v] > d) d = off[v + 1] - off[v];
    return d;
}

/* ------------------------------------------------------------------ */
/* Speculative coloring (Sec. 2.2 rounds, Alg. 1 selection, Sec. 3.2)  */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t rounds;            /* rounds until no conflict remained        */
    int32_t max_color;         /* max_v C(v), the paper's color count      */
    int64_t edges_examined;    /* adjacency entries scanned (both phases)  */
    int64_t conflicts;         /* vertices sent back, summed over rounds   */
} oracle_color_stats;

/* Where a round's random numbers come from: either Philox keyed by the seed,
 * or tables handed in by a test (prio[n]; draws[r * n + v] for r < rounds). */
typedef struct {
    uint64_t seed;
    const uint32_t* prio_tab;
    const uint32_t* draw_tab;
    int32_t draw_rounds;
    int64_t n;
} rng_source;

static uint32_t src_prio(const rng_source* s, int64_t v)
{
    return s->prio_tab ? s->prio_tab[v] : oracle_priority(s->seed, v);
}

static int src_draw(const rng_source* s, int64_t v, int32_t r, uint32_t* w)
{
    if (s->draw_tab) {
        if (r >= s->draw_rounds) return 0;
        *w = s->draw_tab[(int64_t)r * s->n + v];
        return 1;
    }
    *w = oracle_rxf_draw(s->seed, v, r);
    return 1;
}

/* u beats v in the random total order: larger priority, then larger id. */
static int beats(uint32_t pu, int64_t u, uint32_t pv, int64_t v)
{
    if (pu != pv) return pu > pv;
    return u > v;
}

static int color_core(int64_t n, const int64_t* off, const int32_t* idx,
                      int32_t X, const rng_source* src, int32_t* color,
                      oracle_color_stats* st)
{
    int64_t *W = NULL, *W_next = NULL, *forbidden = NULL;
    int32_t *tent = NULL;
    unsigned char *in_W = NULL, *lost = NULL;
    int64_t w, w_next, i, e, v, cap;
    int32_t r = 0;
    int status = OR_OK;
    oracle_color_stats local;

    memset(&local, 0, sizeof(local));
    if (X < 1) return OR_ERR_INVALID_ARG;
    status = check_colorable(n, off, idx);
    if (status != OR_OK) return status;
    if (n == 0) { if (st) *st = local; return OR_OK; }

    /* The chosen color never exceeds deg(v) + X (at most deg(v) colors are
     * forbidden), so markers up to max degree + X suffice. */
    cap = max_degree(n, off) + (int64_t)X + 1;
    W = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    W_next = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    forbidden = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap + 1));
    tent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    in_W = (unsigned char*)malloc((size_t)n);
    lost = (unsigned char*)malloc((size_t)n);
    if (!W || !W_next || !forbidden || !tent || !in_W || !lost) {
        status = OR_ERR_OOM;
        goto done;
    }
    for (i = 0; i <= cap; ++i) forbidden[i] = -1;

    /* Every vertex starts uncolored and in the work set, in id order. */
    for (v = 0; v < n; ++v) { color[v] = 0; tent[v] = 0; W[v] = v; in_W[v] = 1; }
    w = n;

    while (w > 0) {
        if ((int64_t)r > n) { status = OR_ERR_ROUND_LIMIT; goto done; }

        /* Tentative coloring: Alg. 1 against the snapshot `color`. */
        for (i = 0; i < w; ++i) {
            uint32_t j = 0, seen = 0;
            int32_t c;
            v = W[i];
            for (e = off[v]; e < off[v + 1]; ++e) {
                int32_t cu = color[idx[e]];
                if (cu > 0 && (int64_t)cu <= cap) forbidden[cu] = v;
            }
            local.edges_examined += off[v + 1] - off[v];
            if (X > 1) {
                uint32_t wdraw;
                if (!src_draw(src, v, r, &wdraw)) { status = OR_ERR_INVALID_ARG; goto done; }
                j = scale_draw(wdraw, (uint32_t)X);
            }
            /* Enumerate permissible colors 1, 2, ... and take the j-th. */
            c = 0;
            for (;;) {
                ++c;
                if (forbidden[c] != v) {
                    if (seen == j) break;
                    ++seen;
                }
            }
            tent[v] = c;
        }

        /* Conflict detection against the tentative colors of the round;
         * a vertex outside the work set shows its fixed color. */
        w_next = 0;
        for (i = 0; i < w; ++i) {
            int32_t tv;
            uint32_t pv;
            v = W[i];
            tv = tent[v];
            pv = src_prio(src, v);
            lost[v] = 0;
            for (e = off[v]; e < off[v + 1]; ++e) {
                int64_t u = idx[e];
                int32_t tu;
                if (u == v) continue;
                tu = in_W[u] ? tent[u] : color[u];
                if (tu == tv && beats(src_prio(src, u), u, pv, v)) {
                    lost[v] = 1;
                    break;
                }
            }
            local.edges_examined += off[v + 1] - off[v];
            if (lost[v]) W_next[w_next++] = v;
        }

        /* Apply the round: winners keep their tentative color, losers stay
         * uncolored and form the next work set (still in id order). */
        for (i = 0; i < w; ++i) {
            v = W[i];
            if (!lost[v]) { color[v] = tent[v]; in_W[v] = 0; }
        }
        local.conflicts += w_next;
        { int64_t* t = W; W = W_next; W_next = t; }
        w = w_next;
        ++r;
    }

    local.rounds = r;
    local.max_color = 0;
    for (v = 0; v < n; ++v)
        if (color[v] > local.max_color) local.max_color = color[v];
    if (st) *st = local;

done:
    free(W); free(W_next); free(forbidden); free(tent); free(in_W); free(lost);
    return status;
}

/* Speculative coloring with Philox priorities and draws.  X = 1 is First
 * Fit; X > 1 is Random-X Fit. */
int oracle_color(int64_t n, const int64_t* off, const int32_t* idx, int32_t X,
                 uint64_t seed, int32_t* colors_out, oracle_color_stats* st)
{
    rng_source src;
    if (n > 0 && !colors_out) return OR_ERR_INVALID_ARG;
    src.seed = seed; src.prio_tab = NULL; src.draw_tab = NULL;
    src.draw_rounds = 0; src.n = n;
    return color_core(n, off, idx, X, &src, colors_out, st);
}

/* The same rounds with priorities and draws given as tables (hand-traced
 * tests).  draws may be NULL when X == 1. */
int oracle_color_tables(int64_t n, const int64_t* off, const int32_t* idx,
                        int32_t X, const uint32_t* prio, const uint32_t* draws,
                        int32_t draw_rounds, int32_t* colors_out,
                        oracle_color_stats* st)
{
    rng_source src;
    if (n > 0 && (!colors_out || !prio)) return OR_ERR_INVALID_ARG;
    if (X > 1 && !draws) return OR_ERR_INVALID_ARG;
    src.seed = 0; src.prio_tab = prio; src.draw_tab = draws;
    src.draw_rounds = draw_rounds; src.n = n;
    return color_core(n, off, idx, X, &src, colors_out, st);
}

/* ------------------------------------------------------------------ */
/* Validation (Sec. 1 problem statement)                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n_conflicts;      /* entries (v,u), u in adj(v), C(u) == C(v)   */
    int64_t n_uncolored;      /* vertices with C(v) < 1                     */
    int32_t max_color;        /* max_v C(v)                                 */
    int32_t n_distinct;       /* number of distinct colors >= 1             */
    int64_t first_bad_vertex; /* smallest such v, or -1                     */
} oracle_validation;

int oracle_validate(int64_t n, const int64_t* off, const int32_t* idx,
                    const int32_t* colors, oracle_validation* out)
{
    int64_t v, e;
    int32_t maxc = 0;
    unsigned char* seen;
    int status = check_graph(n, off, idx);
    if (status != OR_OK) return status;
    if (!out || (n > 0 && !colors)) return OR_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->first_bad_vertex = -1;
    for (v = 0; v < n; ++v) {
        int bad = 0;
        if (colors[v] < 1) { out->n_uncolored++; bad = 1; }
        for (e = off[v]; e < off[v + 1]; ++e) {
            if (colors[idx[e]] == colors[v]) { out->n_conflicts++; bad = 1; }
        }
        if (bad && out->first_bad_vertex < 0) out->first_bad_vertex = v;
        if (colors[v] > maxc) maxc = colors[v];
    }
    out->max_color = maxc;
    seen = (unsigned char*)calloc((size_t)maxc + 1, 1);
    if (!seen) return OR_ERR_OOM;
    for (v = 0; v < n; ++v)
        if (colors[v] >= 1) seen[colors[v]] = 1;
    for (v = 1; v <= maxc; ++v) out->n_distinct += seen[v];
    free(seen);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Class permutations (Sec. 3: RV, NI, ND, RAND)                       */
/* ------------------------------------------------------------------ */

/* Given class sizes size[c] for colors c = 1..maxc (size[0] unused), write
 * the present colors (size > 0) into order[0..k-1] in the order they are to
 * be recolored and return k.  For RAND, draws[i] (i = 1..k-1) may be given
 * by a test; with draws == NULL they come from Philox(seed, (i, it, 0, 3)). */
int32_t oracle_class_order(int32_t maxc, const int64_t* size, int32_t perm,
                           uint64_t seed, int32_t iteration,
                           const uint32_t* draws, int32_t* order)
{
    int32_t k = 0, c, a, b, i;
    for (c = 1; c <= maxc; ++c)
        if (size[c] > 0) order[k++] = c;       /* ascending list */

    if (perm == PERM_REVERSE) {
        for (a = 0, b = k - 1; a < b; ++a, --b) {
            int32_t t = order[a]; order[a] = order[b]; order[b] = t;
        }
    } else if (perm == PERM_NONINC || perm == PERM_NONDEC) {
        /* insertion sort: stable, so equal sizes keep ascending color */
        for (a = 1; a < k; ++a) {
            int32_t key = order[a];
            b = a - 1;
            while (b >= 0) {
                int move;
                if (perm == PERM_NONINC) move = size[order[b]] < size[key];
                else                     move = size[order[b]] > size[key];
                if (!move) break;
                order[b + 1] = order[b];
                --b;
            }
            order[b + 1] = key;
        }
    } else if (perm == PERM_RANDOM) {
        /* Knuth (Fisher-Yates) shuffle of the ascending list */
        for (i = k - 1; i >= 1; --i) {
            uint32_t w = draws ? draws[i] : oracle_perm_draw(seed, i, iteration);
            int32_t j = (int32_t)scale_draw(w, (uint32_t)(i + 1));
            int32_t t = order[i]; order[i] = order[j]; order[j] = t;
        }
    } else {
        return -1;
    }
    return k;
}

/* The permutation that recoloring iteration `it` (0-based) uses under a
 * permutation or schedule code (Sec. 4.2.1), or -1 if the code is unknown. */
int32_t oracle_perm_of_iteration(int32_t code, int32_t it)
{
    int32_t t = it + 1;                 /* the paper counts iterations from 1 */
    if (code >= PERM_REVERSE && code <= PERM_RANDOM) return code;
    if (code == SCHED_POW2) {
        int32_t p = 2;
        while (p < t && p <= (1 << 29)) p *= 2;
        return p == t ? PERM_RANDOM : PERM_NONDEC;
    }
    if (code > SCHED_EVERY_BASE && code <= SCHED_EVERY_MAX) {
        int32_t x = code - SCHED_EVERY_BASE;
        return t % x == 0 ? PERM_RANDOM : PERM_NONDEC;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Iterative recoloring (Culberson's iterated greedy, Sec. 2.1; RC Sec. 3) */
/* ------------------------------------------------------------------ */

/* ncolors (may be NULL) receives iterations + 1 entries: max color of the
 * input, then the max color after each iteration.  colors_out may alias
 * colors_in. */
int oracle_recolor(int64_t n, const int64_t* off, const int32_t* idx,
                   const int32_t* colors_in, int32_t perm, int32_t iterations,
                   uint64_t seed, int32_t* colors_out, int32_t* ncolors)
{
    int32_t *old = NULL, *nw = NULL, *order = NULL;
    int64_t *size = NULL, *start = NULL, *fill = NULL, *members = NULL;
    int64_t *forbidden = NULL;
    int64_t v, e, cap;
    int32_t it, maxc, c, k, p;
    int status;
    oracle_validation val;

    if (iterations < 0 || oracle_perm_of_iteration(perm, 0) < 0)
        return OR_ERR_INVALID_ARG;
    status = oracle_validate(n, off, idx, colors_in, &val);
    if (status != OR_OK) return status;
    if (val.n_conflicts > 0 || val.n_uncolored > 0) return OR_ERR_IMPROPER_INPUT;
    if (ncolors) ncolors[0] = val.max_color;
    if (n == 0) {
        for (it = 0; it < iterations; ++it) if (ncolors) ncolors[it + 1] = 0;
        return OR_OK;
    }

    cap = max_degree(n, off) + 2;
    old = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    nw = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    members = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    forbidden = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap + 1));
    if (!old || !nw || !members || !forbidden) { status = OR_ERR_OOM; goto done; }
    memcpy(old, colors_in, sizeof(int32_t) * (size_t)n);
    maxc = val.max_color;

    for (it = 0; it < iterations; ++it) {
        int32_t newmax = 0;
        /* class sizes and, per class, its members in increasing id */
        size = (int64_t*)calloc((size_t)maxc + 1, sizeof(int64_t));
        start = (int64_t*)calloc((size_t)maxc + 2, sizeof(int64_t));
        fill = (int64_t*)calloc((size_t)maxc + 2, sizeof(int64_t));
        order = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxc + 1));
        if (!size || !start || !fill || !order) { status = OR_ERR_OOM; goto done; }
        for (v = 0; v < n; ++v) size[old[v]]++;
        for (c = 1; c <= maxc; ++c) start[c + 1] = start[c] + size[c];
        for (v = 0; v < n; ++v) {
            c = old[v];
            members[start[c] + fill[c]] = v;
            fill[c]++;
        }
        k = oracle_class_order(maxc, size, oracle_perm_of_iteration(perm, it), seed, it, NULL, order);

        /* Alg. 1 over the vertices taken class after class in the order
         * chosen; a vertex not recolored yet has new color 0 and so does not
         * constrain anybody. */
        for (v = 0; v < n; ++v) nw[v] = 0;
        for (v = 0; v <= cap; ++v) forbidden[v] = -1;
        for (p = 0; p < k; ++p) {
            int64_t m;
            c = order[p];
            for (m = start[c]; m < start[c] + size[c]; ++m) {
                int32_t cc;
                v = members[m];
                for (e = off[v]; e < off[v + 1]; ++e) {
                    int32_t cu = nw[idx[e]];
                    if (cu > 0) forbidden[cu] = v;
                }
                cc = 1;
                while (forbidden[cc] == v) ++cc;
                nw[v] = cc;
                if (cc > newmax) newmax = cc;
            }
        }
        memcpy(old, nw, sizeof(int32_t) * (size_t)n);
        maxc = newmax;
        if (ncolors) ncolors[it + 1] = newmax;
        free(size); free(start); free(fill); free(order);
        size = NULL; start = NULL; fill = NULL; order = NULL;
    }
    memcpy(colors_out, old, sizeof(int32_t) * (size_t)n);
    status = OR_OK;

done:
    free(old); free(nw); free(members); free(forbidden);
    free(size); free(start); free(fill); free(order);
    return status;
}

/* ------------------------------------------------------------------ */
/* Vertex-visit orders as conflict priorities: Largest First            */
/* (Sec. 2.2.1) and asynchronous recoloring (aRC, Sec. 3)              */
/* ------------------------------------------------------------------ */

/* A visit-order key (clamped to 16 bits) above the upper half of the
 * Philox priority; equal pairs fall back to the id, as in every round. */
static uint32_t ordered_priority(uint32_t first_key, uint64_t seed, int64_t v)
{
    if (first_key > 65535u) first_key = 65535u;
    return (first_key << 16) | (oracle_priority(seed, v) >> 16);
}

uint32_t oracle_ordered_priority(uint32_t first_key, uint64_t seed, int64_t v)
{
    return ordered_priority(first_key, seed, v);
}

/* Speculative coloring in which a larger degree wins a conflict. */
int oracle_color_lf(int64_t n, const int64_t* off, const int32_t* idx, int32_t X,
                    uint64_t seed, int32_t* colors_out, oracle_color_stats* st)
{
    rng_source src;
    uint32_t* prio;
    int64_t v;
    int status;
    if (n > 0 && !colors_out) return OR_ERR_INVALID_ARG;
    status = check_colorable(n, off, idx);
    if (status != OR_OK) return status;
    prio = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!prio) return OR_ERR_OOM;
    for (v = 0; v < n; ++v) {
        int64_t d = off[v + 1] - off[v];
        prio[v] = ordered_priority((uint32_t)(d > 65535 ? 65535 : d), seed, v);
    }
    src.seed = seed; src.prio_tab = prio; src.draw_tab = NULL;
    src.draw_rounds = 0; src.n = n;
    status = color_core(n, off, idx, X, &src, colors_out, st);
    free(prio);
    return status;
}

/* aRC: each iteration colors the graph again by speculative First-Fit
 * rounds, a vertex of an earlier class (in the iteration's permutation of
 * the previous coloring's classes) winning its conflicts.  ncolors as for
 * oracle_recolor; rounds (may be NULL) receives each iteration's rounds. */
int oracle_recolor_async(int64_t n, const int64_t* off, const int32_t* idx,
                         const int32_t* colors_in, int32_t perm, int32_t iterations,
                         uint64_t seed, int32_t* colors_out, int32_t* ncolors,
                         int32_t* rounds)
{
    int32_t *old = NULL, *nw = NULL, *order = NULL, *rank = NULL;
    int64_t *size = NULL;
    uint32_t* prio = NULL;
    int64_t v;
    int32_t it, maxc, c, k, p;
    int status;
    oracle_validation val;
    oracle_color_stats st;
    rng_source src;

    if (iterations < 0 || oracle_perm_of_iteration(perm, 0) < 0) return OR_ERR_INVALID_ARG;
    status = oracle_validate(n, off, idx, colors_in, &val);
    if (status != OR_OK) return status;
    if (val.n_conflicts > 0 || val.n_uncolored > 0) return OR_ERR_IMPROPER_INPUT;
    if (ncolors) ncolors[0] = val.max_color;
    if (n == 0) {
        for (it = 0; it < iterations; ++it) {
            if (ncolors) ncolors[it + 1] = 0;
            if (rounds) rounds[it] = 0;
        }
        return OR_OK;
    }
    old = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    nw = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    prio = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!old || !nw || !prio) { status = OR_ERR_OOM; goto done; }
    memcpy(old, colors_in, sizeof(int32_t) * (size_t)n);
    maxc = val.max_color;
    for (it = 0; it < iterations; ++it) {
        size = (int64_t*)calloc((size_t)maxc + 1, sizeof(int64_t));
        order = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxc + 1));
        rank = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxc + 1));
        if (!size || !order || !rank) { status = OR_ERR_OOM; goto done; }
        for (v = 0; v < n; ++v) size[old[v]]++;
        k = oracle_class_order(maxc, size, oracle_perm_of_iteration(perm, it), seed, it, NULL, order);
        for (c = 0; c <= maxc; ++c) rank[c] = 0;
        for (p = 0; p < k; ++p) rank[order[p]] = p;
        for (v = 0; v < n; ++v) {
            int32_t r = rank[old[v]];
            prio[v] = ordered_priority(65535u - (uint32_t)(r > 65535 ? 65535 : r), seed, v);
        }
        src.seed = seed; src.prio_tab = prio; src.draw_tab = NULL;
        src.draw_rounds = 0; src.n = n;
        status = color_core(n, off, idx, 1, &src, nw, &st);
        if (status != OR_OK) goto done;
        memcpy(old, nw, sizeof(int32_t) * (size_t)n);
        maxc = st.max_color;
        if (ncolors) ncolors[it + 1] = maxc;
        if (rounds) rounds[it] = st.rounds;
        free(size); free(order); free(rank);
        size = NULL; order = NULL; rank = NULL;
    }
    memcpy(colors_out, old, sizeof(int32_t) * (size_t)n);
    status = OR_OK;

done:
    free(old); free(nw); free(prio); free(size); free(order); free(rank);
    return status;
}

/* ------------------------------------------------------------------ */
/* Sequential greedy (Alg. 1, Sec. 2.1) in a vertex-visit order         */
/* (Sec. 2.2.1): Natural (id order) or Largest First (non-increasing    */
/* degree, equal degrees in id order).  The columns NAT and LF of       */
/* Tables 1 and 2.                                                      */
/* ------------------------------------------------------------------ */

int oracle_greedy_sequential(int64_t n, const int64_t* off, const int32_t* idx, int32_t order_kind,
                             int32_t* colors_out)
{
    int64_t *order = NULL, *forbidden = NULL, *count = NULL;
    int64_t v, e, i, maxd, d;
    int status;
    if (order_kind != 0 && order_kind != 1) return OR_ERR_INVALID_ARG;
    status = check_colorable(n, off, idx);
    if (status != OR_OK) return status;
    if (n == 0) return OR_OK;
    maxd = max_degree(n, off);
    order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    forbidden = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxd + 2));
    count = (int64_t*)calloc((size_t)maxd + 2, sizeof(int64_t));
    if (!order || !forbidden || !count) { status = OR_ERR_OOM; goto done; }
    if (order_kind == 0) {
        for (v = 0; v < n; ++v) order[v] = v;
    } else {
        /* counting sort by degree, largest first, stable in id */
        for (v = 0; v < n; ++v) count[off[v + 1] - off[v]]++;
        {
            int64_t pos = 0;
            for (d = maxd; d >= 0; --d) { int64_t c = count[d]; count[d] = pos; pos += c; }
        }
        for (v = 0; v < n; ++v) order[count[off[v + 1] - off[v]]++] = v;
    }
    for (i = 0; i <= maxd + 1; ++i) forbidden[i] = -1;
    for (v = 0; v < n; ++v) colors_out[v] = 0;
    for (i = 0; i < n; ++i) {
        int32_t c;
        v = order[i];
        for (e = off[v]; e < off[v + 1]; ++e) {
            int32_t cu = colors_out[idx[e]];
            if (cu > 0) forbidden[cu] = v;
        }
        c = 1;
        while (forbidden[c] == v) ++c;
        colors_out[v] = c;
    }
    status = OR_OK;
done:
    free(order); free(forbidden); free(count);
    return status;
}
