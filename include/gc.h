/*
 * gc.h -- C ABI of the GB300 speculative graph-coloring library (libgc.so).
 *
 * Distance-1 coloring of an undirected graph G = (V, E): a map C: V -> N with
 * C(u) != C(v) for every edge (u, v); the number of colors is max_u C(u)
 * (Sec. 1 of Sariyuce, Saule, Catalyurek, "On Distributed Graph Coloring with
 * Iterative Recoloring", arXiv 1407.6745).  The library runs, on one GPU:
 *
 *   gc_color    speculative rounds (Sec. 2.2): every uncolored vertex picks a
 *               tentative color -- First Fit (Alg. 1, Sec. 2.1) or Random-X
 *               Fit (Sec. 3.2) -- then conflicts are detected and the endpoint
 *               lower in a random total order is uncolored for the next
 *               round, until no conflict is left;
 *   gc_recolor  iterative recoloring (Culberson's iterated greedy, Sec. 2.1;
 *               RC, Sec. 3): the classes of a proper coloring are recolored
 *               one class after another in a class permutation (RV, NI, ND,
 *               RAND), each vertex First Fit against the classes already
 *               recolored; the color count never increases;
 *   gc_validate the definition of Sec. 1 checked on the device.
 *
 * Determinism: results depend only on (graph, arguments, seed), never on
 * thread scheduling.  Tentative colors are chosen against the colors fixed
 * before the round; a vertex loses iff a neighbor has the same tentative
 * color and a larger (priority, id), priority = Philox4x32-10 word 0 of
 * counter (v_lo, v_hi, 0, 1) under key (seed_lo, seed_hi); Random-X Fit takes
 * the j-th permissible color (0-based), j = floor(w * X / 2^32), w = Philox
 * word 0 of counter (v_lo, v_hi, round, 2); RAND shuffles the ascending list
 * of present colors (Knuth/Fisher-Yates, i = k-1..1, j = floor(w * (i+1) /
 * 2^32), w = Philox word 0 of counter (i, iteration, 0, 3)).
 *
 * Graph layout: symmetric CSR, offsets int64[n+1] with offsets[0] = 0,
 * non-decreasing, offsets[n] = nnz; idx int32[nnz] neighbor ids in [0, n).
 * Every undirected edge appears in both rows; duplicates are tolerated.  A
 * self-loop makes a graph uncolorable: the coloring calls report it as
 * GC_ERR_BAD_GRAPH, and a coloring given to gc_recolor / gc_validate counts
 * it as a conflict.
 * Colors are int32, 1-based.
 *
 * Memory: every pointer argument of a call (graph arrays, colors in and out)
 * lives in the memory space named by gc_graph.mem: GC_MEM_DEVICE (device
 * memory of the current CUDA device, e.g. torch tensors) or GC_MEM_HOST
 * (host memory; the call copies to the device, runs, and copies the result
 * back; pinned memory makes those copies faster).  Statistics and per-iteration
 * color counts are always host memory.  The caller owns all buffers; the
 * library allocates its scratch from its own stream-ordered pool and frees it
 * before returning.
 *
 * Streams and synchronisation: `stream` is a cudaStream_t (NULL = the legacy
 * default stream).  Work is enqueued on it and every call waits for that
 * stream before returning, so outputs are ready and device-side errors are
 * reported by the return value.
 *
 * Errors: a call returns GC_OK or an error code and never aborts.  The
 * kernels bounds-check every offset and neighbor id they read, so a malformed
 * graph yields GC_ERR_BAD_GRAPH, not a memory fault.  On error the output
 * contents are unspecified.
 */
#ifndef GC_H_
#define GC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GC_OK = 0,
    GC_ERR_INVALID_ARG = 1,    /* NULL pointer, n < 0, X < 1, unknown enum   */
    GC_ERR_BAD_GRAPH = 2,      /* offsets not monotone / out of range, id not in [0, n) */
    GC_ERR_IMPROPER_INPUT = 3, /* gc_recolor input not a proper coloring     */
    GC_ERR_OOM = 4,            /* device or pinned host allocation failed    */
    GC_ERR_CUDA = 5,           /* a CUDA runtime call failed                 */
    GC_ERR_TIMEOUT = 6,        /* a bounded device-side wait ran out         */
    GC_ERR_ROUND_LIMIT = 7,    /* more than n+1 speculative rounds (cannot happen
                                  for a valid graph: the top-priority vertex of the
                                  work set always keeps its color)           */
    GC_ERR_BUDGET = 8,         /* a server request larger than its memory budget */
    GC_PENDING = 9             /* a server request not finished yet (not an error) */
} gc_status;

typedef enum { GC_FIRST_FIT = 0, GC_RANDOM_X_FIT = 1 } gc_strategy;

typedef enum {
    GC_PERM_REVERSE = 0, /* RV: decreasing color                              */
    GC_PERM_NONINC = 1,  /* NI: non-increasing class size, ties smaller color */
    GC_PERM_NONDEC = 2,  /* ND: non-decreasing class size, ties smaller color */
    GC_PERM_RANDOM = 3,  /* RAND: seeded Knuth shuffle                        */
    /* Schedules (Sec. 4.2.1), iterations counted from 1: ND at every iteration
     * except 2, 4, 8, 16, ..., which use RAND (ND-RAND%2^i) */
    GC_PERM_ND_RAND_POW2 = 4
} gc_perm;
/* ND-RAND%x (Sec. 4.2.1): RAND at iterations x, 2x, 3x, ..., ND at the
 * others; 1 <= x <= 65535.  Accepted wherever a gc_perm is.  An iteration
 * that uses RAND draws its shuffle with its own iteration number, as plain
 * RAND does. */
#define GC_PERM_ND_RAND_EVERY(x) (256 + (x))

/* Parameter sets of Sec. 4.3 and Sec. 5: "speed" is First Fit with no
 * recoloring (FIxxND0); "quality" is Random-5 Fit (or Random-10 Fit) with
 * one ND recoloring iteration (R(5|10)IxxND1).  The internal-first vertex
 * order of those names is a distributed-memory notion with no counterpart on
 * one GPU, where every vertex is its own processor. */
typedef enum { GC_PRESET_SPEED = 0, GC_PRESET_QUALITY = 1, GC_PRESET_QUALITY_X10 = 2 } gc_preset;

typedef enum { GC_MEM_DEVICE = 0, GC_MEM_HOST = 1 } gc_memspace;

/* Symmetric CSR graph (see layout above).  Read-only for the library. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* offsets; /* n + 1 entries */
    const int32_t* idx;     /* nnz entries   */
    int32_t mem;            /* gc_memspace of every pointer argument of the call */
} gc_graph;

/* Optional statistics (host memory; pass NULL to skip). */
typedef struct {
    int32_t rounds;         /* speculative rounds (gc_color)                     */
    int32_t iterations;     /* recoloring iterations done                        */
    int32_t max_color;      /* max_v C(v) of the output                          */
    int32_t reserved;
    int64_t edges_examined; /* adjacency entries scanned by the hot kernels       */
    int64_t conflicts;      /* vertices uncolored by conflict resolution, summed  */
    float ms_color;         /* device time of the speculative coloring            */
    float ms_recolor;       /* device time of all recoloring iterations           */
} gc_stats;

/* Result of gc_validate (host memory). */
typedef struct {
    int64_t n_conflicts;      /* directed entries (v, u), u in adj(v), C(u) == C(v) */
    int64_t n_uncolored;      /* vertices with C(v) < 1                               */
    int32_t max_color;        /* max_v C(v)                                           */
    int32_t n_distinct;       /* distinct colors >= 1                                 */
    int64_t first_bad_vertex; /* smallest v uncolored or in a conflict, -1 if none    */
} gc_validation;

/*
 * Speculative coloring to convergence (Sec. 2.2 rounds; Alg. 1 First Fit,
 * Sec. 2.1; Random-X Fit, Sec. 3.2).
 *   strategy   GC_FIRST_FIT (X ignored, treated as 1) or GC_RANDOM_X_FIT (X >= 1).
 *   seed       keys the priorities and the Random-X draws.
 *   colors_out int32[n]: the coloring, each C(v) in [1, deg(v) + X].
 *   stats      may be NULL.
 */
gc_status gc_color(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                   int32_t* colors_out, gc_stats* stats, void* stream);

/*
 * Iterative recoloring (Sec. 2.1, Culberson; Sec. 3, RC and the class
 * permutations).  colors_in must be a proper coloring with colors in
 * [1, 2^28] (checked: GC_ERR_IMPROPER_INPUT).  iterations >= 0; 0 copies the
 * input.  seed is used by GC_PERM_RANDOM only.  colors_out may alias
 * colors_in.  ncolors_per_iter (host, may be NULL) receives iterations + 1
 * entries: the max color of the input, then after each iteration.
 */
gc_status gc_recolor(const gc_graph* g, const int32_t* colors_in, gc_perm perm,
                     int32_t iterations, uint64_t seed, int32_t* colors_out,
                     int32_t* ncolors_per_iter, gc_stats* stats, void* stream);

/*
 * Speculative coloring with a vertex-visit order as the conflict priority
 * (Sec. 2.2.1).  GC_ORDER_RANDOM is gc_color.  GC_ORDER_LARGEST_FIRST: of two
 * neighbors with the same tentative color the one of larger degree keeps
 * it; the priority is (min(deg, 65535) << 16) | (random priority >> 16),
 * ties to the larger id.  One thread per vertex leaves no visit order, so
 * the order acts where a distributed processor's local order would: on
 * conflicts.  Arguments, memory and errors as gc_color.
 */
typedef enum { GC_ORDER_RANDOM = 0, GC_ORDER_LARGEST_FIRST = 1 } gc_order;
/* GC_ERR_INVALID_ARG for an unknown order; otherwise as gc_color. */
gc_status gc_color_ordered(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_order order, int32_t* colors_out, gc_stats* stats, void* stream);

/*
 * Asynchronous recoloring, aRC (Sec. 3): each iteration colors the graph
 * again from scratch by the speculative First-Fit rounds, with the class
 * permutation of the previous coloring (perm, schedules included, RAND keyed
 * by seed and the iteration number) as the first key of the conflict
 * priority: (65535 - min(rank, 65535)) << 16 | (random priority >> 16), so a
 * vertex of an earlier class wins; conflicts make it take rounds, and unlike
 * gc_recolor the color count may grow.  colors_in must be proper
 * (GC_ERR_IMPROPER_INPUT); colors_out may alias it; ncolors_per_iter as for
 * gc_recolor; stats->rounds sums the rounds of all iterations.
 */
gc_status gc_recolor_async(const gc_graph* g, const int32_t* colors_in, gc_perm perm,
                           int32_t iterations, uint64_t seed, int32_t* colors_out,
                           int32_t* ncolors_per_iter, gc_stats* stats, void* stream);

/*
 * The paper's full method in one call: gc_color followed by `iterations`
 * recoloring iterations of gc_recolor on its (proper by construction)
 * output, with no input re-validation and no intermediate host round trip.
 * Same arguments as the two calls; perm_seed keys GC_PERM_RANDOM.  check
 * (host, may be NULL) receives gc_validate of the final coloring, computed on
 * the device before the result is copied out.
 */
gc_status gc_color_recolor(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_perm perm, int32_t iterations, uint64_t perm_seed,
                           int32_t* colors_out, int32_t* ncolors_per_iter, gc_stats* stats,
                           gc_validation* check, void* stream);

/* The random total order of Sec. 2.2 as used by gc_color: out[v] =
 * prio(v) = Philox4x32-10 word 0 of counter (v_lo, v_hi, 0, 1) under key
 * (seed_lo, seed_hi), for v in [0, n).  out is device memory (uint32[n]). */
gc_status gc_priorities(uint64_t seed, int64_t n, uint32_t* out, void* stream);

/*
 * Batches: many independent graphs colored and recolored together in the
 * same launches.  The batch is one concatenated CSR (gc_graph) whose vertices
 * are numbered globally; graph i owns the vertices [vertex_base, vertex_base +
 * n) and every edge of a vertex stays inside its graph (caller's contract).
 * The descriptors must tile [0, g->n) in order: vertex_base of the first is
 * 0 and each next one starts where the previous one ends.  Priorities and
 * Random-X draws use graph-local ids and the graph's own seed, so every
 * graph's colors are exactly those gc_color / gc_recolor give it alone.
 * (Not in the paper: a library extension for many-graph workloads.)
 */
typedef struct {
    int64_t vertex_base;  /* first vertex of the graph in the batch            */
    int64_t n;            /* vertices of the graph                             */
    uint64_t seed;        /* keys priorities and Random-X draws                 */
    int32_t X;            /* 1 = First Fit, > 1 = Random-X Fit                  */
    int32_t perm;         /* gc_perm of its recoloring                          */
    int32_t iterations;   /* recoloring iterations (>= 0)                       */
    int32_t reserved;
    uint64_t perm_seed;   /* keys GC_PERM_RANDOM                                */
} gc_batch_graph;

/*
 * Speculative coloring of every graph of a batch (host descriptors).
 * rounds_out / max_color_out (host, ngraphs entries each, may be NULL)
 * receive each graph's round count and max color.
 */
gc_status gc_color_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                         int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                         gc_stats* stats, void* stream);

/*
 * Recoloring of every graph of a batch, each with its own permutation,
 * seed and iteration count; colors_in must be proper.  max_color_out (host,
 * ngraphs entries, may be NULL) receives each graph's final max color.
 * colors_out may alias colors_in.
 */
gc_status gc_recolor_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                           const int32_t* colors_in, int32_t* colors_out, int32_t* max_color_out,
                           gc_stats* stats, void* stream);

/*
 * Batch pipeline: gc_color_batch followed by gc_recolor_batch on its output
 * (proper by construction: not re-validated), each graph with its own
 * recoloring settings.  rounds_out / max_color_out as above (final colors).
 */
gc_status gc_color_recolor_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                                 int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                                 gc_stats* stats, void* stream);

/*
 * Serving: a request loop that colors graphs as they arrive (a library
 * extension, not in the paper), with continuous batching.  Submitted
 * requests are queued and admitted first come first served while they fit
 * the device-memory budget and the batch limit; the requests admitted
 * together form a cohort, laid out as one concatenated CSR on the device.
 * Each worker (one host thread and CUDA stream) keeps up to four cohorts
 * resident and advances them in turn, one step at a time -- the speculative
 * coloring of a cohort's graphs, then its recoloring iterations -- with CSR,
 * colors and work lists resident on the device throughout.  Between steps a
 * worker admits the requests that arrived meanwhile as a new cohort, as soon
 * as memory is free, so they do not wait for the graphs already on the GPU;
 * and a request retires as soon as its own iterations are done: its result
 * is ready, its latency taken and its scratch share of the budget returned
 * (its CSR share when its cohort is compacted, once half of the cohort's CSR
 * belongs to retired requests, or ends).  Workers run their steps on their
 * own streams, so the work of several cohorts overlaps on the device.  Every
 * request gets exactly the colors, round count and final max color that
 * gc_color_recolor gives it alone.
 */
typedef struct gc_server gc_server;

typedef struct {
    gc_graph graph;      /* host or device memory; copied by gc_server_submit */
    int32_t strategy;    /* gc_strategy */
    int32_t X;           /* Random-X Fit's X (>= 1); ignored for First Fit */
    uint64_t seed;
    int32_t perm;        /* gc_perm */
    int32_t iterations;
    uint64_t perm_seed;
} gc_request;

typedef struct {
    int32_t status;      /* gc_status of the request */
    int32_t rounds;      /* speculative rounds */
    int32_t max_color;   /* after the last recoloring iteration */
    int32_t batch_size;  /* requests admitted in its cohort */
    double submit_ms;    /* server clock (ms since gc_server_create) */
    double start_ms;     /* its cohort was admitted */
    double done_ms;      /* its own iterations done, result available */
} gc_request_result;

typedef struct {
    int64_t submitted, completed, rejected;
    int64_t batches;                 /* cohorts admitted */
    double p50_ms, p99_ms, mean_ms;  /* submit-to-done latency, completed requests */
    double graphs_per_s;             /* completed / (last done - first submit)     */
    int64_t bytes_in_use, bytes_peak;/* admitted device-memory estimate            */
} gc_server_info;

/* Starts a server on the calling thread's current CUDA device.
 * mem_budget: bytes of device memory the admitted requests may hold at once
 *   (an estimate per request: its CSR and colors plus the larger of the
 *   coloring and the recoloring scratch);
 * max_batch: requests per cohort (1..65535); workers: one host thread and
 *   CUDA stream each (1..64), each with its own cohorts.  The workers use the
 *   tuning in force at creation.  One worker gives the lowest tail latency
 *   (its cohorts take turns, the one with the highest response ratio
 *   first); several overlap their steps on the device.
 * Errors: GC_ERR_INVALID_ARG, GC_ERR_CUDA (no usable device).
 * Every gc_server_* call is thread-safe. */
gc_status gc_server_create(size_t mem_budget, int32_t max_batch, int32_t workers, gc_server** out);
/* Queues a request; *ticket identifies it.  The graph is NOT copied: its
 * offsets and ids (host memory -- pinned memory uploads fastest -- or device
 * memory, complete before the call) must stay valid and unchanged until the
 * request's result has been claimed or the server destroyed.  The offsets are
 * checked here, the ids when its cohort is staged on the device.  Errors, with
 * nothing queued: GC_ERR_INVALID_ARG, GC_ERR_BAD_GRAPH (offsets),
 * GC_ERR_BUDGET (its estimate exceeds mem_budget), GC_ERR_CUDA (reading
 * device offsets).  A request whose ids are malformed finishes with
 * GC_ERR_BAD_GRAPH.  A graph without vertices finishes at once. */
gc_status gc_server_submit(gc_server* s, const gc_request* r, uint64_t* ticket);
/* GC_PENDING while queued or running.  Otherwise returns the request's status
 * and fills colors_out (host, n entries; may be NULL; written only for GC_OK)
 * and res (may be NULL); the server then forgets the ticket, so a second
 * poll or wait on it returns GC_ERR_INVALID_ARG (as does an unknown ticket). */
gc_status gc_server_poll(gc_server* s, uint64_t ticket, int32_t* colors_out, gc_request_result* res);
/* As gc_server_poll, blocking up to timeout_ms (< 0: until it finishes). */
gc_status gc_server_wait(gc_server* s, uint64_t ticket, int32_t* colors_out, gc_request_result* res,
                         int32_t timeout_ms);
/* Counters and latency percentiles (nearest rank) since creation. */
gc_status gc_server_stats(gc_server* s, gc_server_info* out);
/* Finishes the queued requests, stops the workers and frees the server with
 * any results not yet claimed. */
void gc_server_destroy(gc_server* s);

/* Checks the coloring against the definition of Sec. 1 and the graph's
 * structure (GC_ERR_BAD_GRAPH if malformed). */
gc_status gc_validate(const gc_graph* g, const int32_t* colors, gc_validation* out, void* stream);

/*
 * gc_validate that allocates nothing (the paper has no counterpart: this is
 * a library convenience).  For callers that cannot allocate device memory:
 * a process whose own caching allocator has reserved the device's memory up
 * front, so that a cudaMalloc would fail or fragment it; a caller checking a
 * result right after an out-of-memory error; a latency-critical path that
 * must not wait on the driver's allocator.  The call uses a fixed scratch
 * array of about 8.3 KB in the library's static device memory instead of the
 * pool; every GPU that loads libgc.so holds that array until the process
 * exits.
 *   - Same result as gc_validate; the graph and colors must be device memory
 *     (GC_MEM_HOST is rejected with GC_ERR_INVALID_ARG: staging would allocate).
 *   - Colors must be below 65536: the array's presence bitmap counts distinct
 *     colors up to there; a larger color gives GC_ERR_INVALID_ARG.
 *   - Like gc_validate it copies its result to the host and synchronizes
 *     `stream` before returning.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - All calls share the array, which each call clears before use; calls
 *     that overlap on the GPU (two streams, two host threads) race on it and
 *     must be serialised by the caller.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.  Its
 *     launches are counted by gc_kernel_launches but not timed by
 *     gc_profile_enable.
 */
gc_status gc_validate_noalloc(const gc_graph* g, const int32_t* colors, gc_validation* out,
                              void* stream);

/* Structure check of a CSR: offsets start at 0, never decrease, end at nnz;
 * ids in [0, n); no self-loop.  GC_OK or GC_ERR_BAD_GRAPH; first_bad_vertex
 * (may be NULL) receives the smallest offending row, or -1. */
gc_status gc_check_graph(const gc_graph* g, int64_t* first_bad_vertex, void* stream);

/*
 * Scheduling knobs (not part of the method: results are identical for every
 * setting).  A vertex of degree d with d + X <= 64 is handled by a group of
 * 2 lanes if d <= g2_max_deg, 4 lanes if d <= g4_max_deg, 8 if d <= g8_max_deg, 16 if d <= g16_max_deg,
 * else 32; otherwise by one warp with a shared-memory bitmap if
 * d <= warp_max_deg (default 1024; a graph with no row longer than 12288
 * entries runs the coloring with no limit while warp_max_deg is at its
 * default), else by a whole block (coloring) or split into chunks
 * of 256 neighbors (recoloring, where rc_warp_max_deg takes the place of
 * warp_max_deg and rc_g2_max_deg, capped at g4_max_deg, that of g2_max_deg;
 * while rc_g2_max_deg holds its default of 16, a recoloring launch bound by
 * its class chain, one given fewer blocks than fit, takes 8).  grid_blocks = 0 sizes every
 * grid to the blocks that fit on the GPU at once.  recolor_mode 0 runs each recoloring iteration as one dataflow
 * launch (vertices wait, with a bounded spin of spin_limit polls, for their
 * earlier-class neighbors); 1 launches one grid per color class.
 * spec_graph 1 (default) runs the speculative rounds as a CUDA graph whose
 * WHILE node repeats {tentative, conflict} until a kernel reports an empty
 * work set (no host round trip per round); 0 drives the rounds from the
 * host.  gc_set_tuning sets the process-wide knobs (change them only while
 * no call is running); a plan's knobs apply to its own calls only.
 */
typedef struct {
    int32_t g4_max_deg;
    int32_t g8_max_deg;
    int32_t g16_max_deg;
    int32_t warp_max_deg;
    int32_t grid_blocks;
    int32_t recolor_mode;
    int32_t spin_limit;
    int32_t spec_graph;
    int32_t rc_warp_max_deg;
    int32_t g2_max_deg;
    int32_t rc_g2_max_deg;
} gc_tuning;

/* Sets the scheduling knobs (NULL restores the defaults).  GC_ERR_INVALID_ARG
 * if a threshold is out of order or negative. */
gc_status gc_set_tuning(const gc_tuning* t);
/* Reads the knobs in force. */
gc_status gc_get_tuning(gc_tuning* out);

/*
 * Autotuner: times gc_color_recolor on the caller's graph (device memory) for
 * candidate scheduling knobs, by coordinate descent from the knobs in force
 * for the calling thread (lane-group thresholds, warp_max_deg,
 * rc_warp_max_deg, g2_max_deg, rc_g2_max_deg, recolor_mode, spec_graph,
 * grid size),
 * `repeats` timed runs each after one warm-up, and returns the fastest in
 * `best` with its time.  Results are identical for every candidate, so only
 * speed is compared.  The candidates are applied to the calling thread only:
 * the process-wide knobs, and calls running on other threads, are never
 * touched.  The caller applies `best` with gc_set_tuning or keeps it in a
 * plan (below).  GC_ERR_INVALID_ARG unless the graph is in device memory
 * with n >= 1 and repeats >= 1.  (A library convenience, not in the paper.)
 */
gc_status gc_autotune(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed, gc_perm perm,
                      int32_t iterations, int32_t repeats, gc_tuning* best, float* best_ms,
                      void* stream);

/*
 * Plans (a library convenience, not in the paper).  A plan is an opaque,
 * library-owned object holding the settings of a coloring + recoloring run
 * (strategy, X, permutation, iteration count) and the scheduling knobs to run
 * it with.  gc_plan_color_recolor applies the plan's knobs to that call alone
 * (on the calling thread), so plans tuned for different graph shapes can run
 * side by side on several threads while the process-wide knobs stay as they
 * are.  The graph is not kept: a plan runs on any graph, and results never
 * depend on the knobs, only the speed does.  A plan may be used by several
 * threads at once; free it once no call using it is running.
 */
typedef struct gc_plan gc_plan;

typedef struct {
    gc_tuning tuning;    /* the knobs the plan runs with */
    int32_t strategy;    /* gc_strategy */
    int32_t X;           /* 1 for First Fit */
    int32_t perm;        /* gc_perm code (schedule codes included) */
    int32_t iterations;  /* recoloring iterations */
    float tuned_ms;      /* time of one run at the tuned knobs (0: not tuned) */
    int64_t tuned_n;     /* shape of the graph tuned on (0: not tuned) */
    int64_t tuned_nnz;
} gc_plan_info;

/* Tunes the knobs for these settings on the caller's graph (gc_autotune, from
 * the calling thread's knobs) and returns a new plan holding them in *out.
 * Errors as gc_autotune; *out is untouched on error. */
gc_status gc_plan_autotune(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_perm perm, int32_t iterations, int32_t repeats, gc_plan** out,
                           void* stream);
/* A plan from given knobs (NULL: the defaults), e.g. knobs cached from an
 * earlier tuning.  GC_ERR_INVALID_ARG for knobs gc_set_tuning would reject,
 * an unknown strategy or permutation, X < 1 for Random-X Fit, iterations < 0
 * or out == NULL; GC_ERR_OOM if the host allocation fails.  Host only. */
gc_status gc_plan_create(const gc_tuning* t, gc_strategy strategy, int32_t X, gc_perm perm,
                         int32_t iterations, gc_plan** out);
/* Copies a plan's settings and knobs into *out (host only). */
gc_status gc_plan_get_info(const gc_plan* p, gc_plan_info* out);
/* gc_color_recolor with the plan's settings, run with the plan's knobs: the
 * arguments and results are those of gc_color_recolor; `seed` seeds the
 * random total order and the Random-X Fit draws, `perm_seed` the RAND
 * permutations. */
gc_status gc_plan_color_recolor(const gc_plan* p, const gc_graph* g, uint64_t seed,
                                uint64_t perm_seed, int32_t* colors_out, int32_t* ncolors_per_iter,
                                gc_stats* stats, gc_validation* check, void* stream);
/* Releases a plan (NULL is a no-op). */
void gc_plan_free(gc_plan* p);

/* Testing aid (host-side fault injection; not in the paper): the scratch
 * allocation after the next `after` ones fails once, so the call making it
 * returns GC_ERR_OOM; after < 0 disables.  Process-wide. */
void gc_inject_alloc_failure(int64_t after);

/* Number of kernel launches the library has made in this process. */
int64_t gc_kernel_launches(void);

/*
 * Kernel timing (tracing aid, off by default).  While enabled, the library
 * brackets each of its kernel launches with CUDA events on the launching
 * stream and accumulates, per kernel, the launch count and the summed
 * device time, read back after the calls return.  Enabling resets the
 * counters.  Not for use inside stream capture.
 */
typedef struct {
    char name[40];
    int64_t launches;
    double ms;
} gc_kernel_time;

/* on != 0 starts (and resets) the per-kernel timing, 0 stops it. */
void gc_profile_enable(int32_t on);
/* Copies up to max entries (kernels launched at least once) into out and
 * returns how many there are. */
int32_t gc_profile_read(gc_kernel_time* out, int32_t max);

/* The strategy, X, permutation and iteration count of a preset (host only;
 * any pointer may be NULL).  GC_ERR_INVALID_ARG for an unknown preset. */
gc_status gc_preset_params(gc_preset preset, int32_t* strategy, int32_t* X, int32_t* perm,
                           int32_t* iterations);

/* A static, human-readable description of a status code (never NULL). */
const char* gc_status_string(gc_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t gc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GC_H_ */
