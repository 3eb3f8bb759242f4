// gc_internal.h -- host-side plumbing shared by the library's translation
// units: the scratch pool, launch accounting, error mapping and the internal
// (device-pointer) implementations behind the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gc.h"
#include "gc_common.cuh"

namespace gc {

// Stream-ordered scratch from a library-owned memory pool (kept warm across
// calls).  Returns nullptr on failure.
void* scratch_alloc(size_t bytes, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

// Number of SMs of the current device (cached).
int sm_count();
// Default persistent grid: blocks_per_sm resident blocks on every SM.
int persistent_grid(const Tuning& t, int blocks_per_sm = 8);

// Resident blocks per SM of a kernel at `threads` threads and `dyn_smem`
// bytes of dynamic shared memory (cached).
int occupancy_of(const void* kernel, int threads, size_t dyn_smem = 0);

// Grid of a persistent (grid-stride) kernel: every block resident at once,
// unless the tuning fixes the grid size.
template <class K>
int resident_grid(K kernel, const Tuning& t, int threads = kBlock) {
    if (t.grid_blocks > 0) return t.grid_blocks;
    return sm_count() * occupancy_of(reinterpret_cast<const void*>(kernel), threads);
}

// Process-wide count of kernel launches made by the library.
void note_launches(int64_t k);

// Kernel timing (gc_profile_enable): events around each launch.
enum KernelId {
    KID_SPEC_SETUP, KID_SPEC_FILL, KID_TENTATIVE, KID_CONFLICT, KID_PRIORITIES,
    KID_RC_BUCKET, KID_RC_VALIDATE, KID_RC_HIST, KID_RC_ORDER, KID_RC_SCATTER,
    KID_RC_RECOLOR, KID_RC_STEP, KID_VALIDATE, KID_VALIDATE_HEAVY, KID_MARK_PRESENT,
    KID_COUNT_BITS, KID_CHECK_GRAPH, KID_SPEC_GRAPH, KID_BATCH, KID_BRC_HIST, KID_BRC_ORDER,
    KID_BRC_SEGMENTS, KID_MARK, KID_COUNT_
};
void prof_begin(KernelId k, cudaStream_t s);
void prof_end(KernelId k, cudaStream_t s);
// Folds the finished launches into the totals (call after a stream sync).
void prof_collect();

#define GC_LAUNCH(kid, stream, ...)              \
    do {                                          \
        ::gc::prof_begin((kid), (stream));        \
        __VA_ARGS__;                              \
        ::gc::prof_end((kid), (stream));          \
        ::gc::note_launches(1);                   \
    } while (0)

// The tuning in force: the calling thread's own (set_thread_tuning), else the
// process-wide one (gc_set_tuning).
Tuning current_tuning();
// Gives the calling thread its own tuning (nullptr: back to the process-wide one).
void set_thread_tuning(const Tuning* t);
// The calling thread's own tuning, if it has one (false: none).
bool thread_tuning(Tuning* out);

// Gives the calling thread a tuning for the scope's lifetime, then puts back
// what the thread had before.
struct ThreadTuningScope {
    bool had;
    Tuning prev;
    explicit ThreadTuningScope(const Tuning& t) {
        had = thread_tuning(&prev);
        set_thread_tuning(&t);
    }
    ThreadTuningScope(const ThreadTuningScope&) = delete;
    ThreadTuningScope& operator=(const ThreadTuningScope&) = delete;
    ~ThreadTuningScope() { set_thread_tuning(had ? &prev : nullptr); }
};

gc_status cuda_status(cudaError_t e);
gc_status status_from_err_bits(uint32_t bits);

// RAII holder for one scratch buffer.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() { if (p) scratch_free(p, s); }
    bool alloc(size_t bytes, cudaStream_t st) {
        s = st;
        p = scratch_alloc(bytes ? bytes : 16, st);
        return p != nullptr;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
    void reset() {
        if (p) scratch_free(p, s);
        p = nullptr;
    }
};

// Speculative coloring on device pointers; writes colors_out (device) and,
// if given, stats.  maxc_out receives the max color (host).
gc_status color_device(const Graph& g, int32_t X, uint64_t seed, int32_t* colors_out,
                       gc_stats* stats, cudaStream_t s);

// Recoloring on device pointers.  When `trusted` the input is known proper
// (our own gc_color output) and maxc_in is its max color; otherwise the
// input is validated first.  colors_out may alias colors_in.
gc_status recolor_device(const Graph& g, const int32_t* colors_in, int32_t maxc_in, bool trusted,
                         int32_t perm, int32_t iterations, uint64_t seed, int32_t* colors_out,
                         int32_t* ncolors_per_iter, gc_stats* stats, cudaStream_t s);

// Speculative coloring where the larger degree wins a conflict (Largest
// First as the first key of the priority, Sec. 2.2.1).
gc_status color_lf_device(const Graph& g, int32_t X, uint64_t seed, int32_t* colors_out,
                          gc_stats* stats, cudaStream_t s);

// Asynchronous recoloring (aRC, Sec. 3) on device pointers; colors_out may
// alias colors_in.  The input is validated.
gc_status recolor_async_device(const Graph& g, const int32_t* colors_in, int32_t perm, int32_t iterations,
                               uint64_t seed, int32_t* colors_out, int32_t* ncolors_per_iter,
                               gc_stats* stats, cudaStream_t s);

// The class permutation of iteration `iteration` of a proper coloring:
// rank_out[c] (max color + 1 entries; nullptr: none) is the position of color
// c in it, *maxc_out the max color.  Unless `trusted`, the coloring is
// validated first (GC_ERR_IMPROPER_INPUT).
gc_status class_ranks_device(const Graph& g, const int32_t* colors, bool trusted, int32_t perm,
                             int32_t iteration, uint64_t seed, int32_t* rank_out, int32_t* maxc_out,
                             cudaStream_t s);

// Batches (see gc_batch_graph): descriptor checks, graph of each vertex,
// per-graph statistics.
gc_status batch_layout(const Graph& g, const gc_batch_graph* graphs, int32_t ng, int32_t* max_x);
gc_status batch_graph_of(const Graph& g, const BatchDesc* d_desc, int32_t ng, int32_t* graph_of,
                         cudaStream_t s);
gc_status batch_max_colors(const Graph& g, const int32_t* graph_of, const int32_t* colors,
                           const int32_t* win_round, int32_t ng, int32_t* max_color_out,
                           int32_t* rounds_out, cudaStream_t s);
gc_status color_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                             int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                             gc_stats* stats, cudaStream_t s);
gc_status recolor_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                               const int32_t* colors_in, int32_t* colors_out, int32_t* max_color_out,
                               gc_stats* stats, cudaStream_t s);
// Recoloring iterations [it_begin, it_end) of a batch in place, on a proper
// coloring whose per-graph max colors are max_in (trusted: not validated);
// max_color_out (host, ng entries) receives each graph's max color after.
gc_status recolor_batch_range(const Graph& g, const gc_batch_graph* graphs, int32_t ng, int32_t* colors,
                              const int32_t* max_in, int32_t it_begin, int32_t it_end,
                              int32_t* max_color_out, cudaStream_t s);
gc_status color_recolor_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                                     int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                                     gc_stats* stats, cudaStream_t s);

gc_status priorities_device(uint64_t seed, int64_t n, uint32_t* out, cudaStream_t s);

gc_status validate_device(const Graph& g, const int32_t* colors, gc_validation* out,
                          cudaStream_t s);

gc_status validate_noalloc_device(const Graph& g, const int32_t* colors, gc_validation* out,
                                  cudaStream_t s);

gc_status check_graph_device(const Graph& g, int64_t* first_bad, cudaStream_t s);

}  // namespace gc
