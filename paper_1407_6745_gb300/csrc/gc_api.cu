// gc_api.cu -- the C ABI (include/gc.h): argument checks, host-memory
// staging, the scratch pool, tuning and launch accounting.
#include <atomic>
#include <climits>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gc_internal.h"

namespace gc {

// ---------------------------------------------------------------------------
// Scratch pool: one library-owned stream-ordered pool per device, kept warm
// (release threshold = unlimited) so repeated calls do not hit the driver.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;
std::vector<int> g_sms;

cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (static_cast<int>(g_pools.size()) <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

std::atomic<long long> g_launches{0};

std::mutex g_tune_mu;
Tuning default_tuning() {
    Tuning t;
    t.g4_max_deg = 64;
    t.g8_max_deg = 64;
    t.g16_max_deg = 64;
    t.warp_max_deg = kDefaultWarpMaxDeg;
    t.grid_blocks = 0;
    t.recolor_mode = 0;
    t.spin_limit = 1 << 20;
    t.spec_graph = 1;
    t.rc_warp_max_deg = 512;
    // 2 lanes up to degree 32 when coloring, 16 when recoloring (measured:
    // stencil coloring 1.32 -> 1.15 ms at 32, its recoloring 3.24 -> 4.61 ms)
    t.g2_max_deg = 32;
    t.rc_g2_max_deg = kDefaultRcG2MaxDeg;
    return t;
}
Tuning g_tune = default_tuning();
}  // namespace

namespace {
// Host-side fault injection (gc_inject_alloc_failure): the allocation after
// the next `g_fail_after` ones fails once.
std::atomic<long long> g_fail_after{-1};
}  // namespace

void* scratch_alloc(size_t bytes, cudaStream_t s) {
    if (g_fail_after.load(std::memory_order_relaxed) >= 0 &&
        g_fail_after.fetch_sub(1, std::memory_order_relaxed) == 0)
        return nullptr;
    cudaMemPool_t p = pool_for_current_device();
    if (!p) return nullptr;
    void* ptr = nullptr;
    if (cudaMallocFromPoolAsync(&ptr, bytes, p, s) == cudaSuccess) return ptr;
    cudaGetLastError();
    // The pool keeps freed memory for reuse; give it back to the device and
    // try once more before reporting GC_ERR_OOM.
    cudaStreamSynchronize(s);
    cudaMemPoolTrimTo(p, 0);
    if (cudaMallocFromPoolAsync(&ptr, bytes, p, s) == cudaSuccess) return ptr;
    cudaGetLastError();
    return nullptr;
}

void scratch_free(void* p, cudaStream_t s) { cudaFreeAsync(p, s); }

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (static_cast<int>(g_sms.size()) <= dev) g_sms.resize(dev + 1, 0);
    if (!g_sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = v > 0 ? v : 1;
    }
    return g_sms[dev];
}

int occupancy_of(const void* kernel, int threads, size_t dyn_smem) {
    struct Entry {
        const void* k;
        int dev;
        size_t dyn;
        int nb;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& e : cache)
        if (e.k == kernel && e.dev == dev && e.dyn == dyn_smem) return e.nb;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, dyn_smem) != cudaSuccess || nb < 1)
        nb = 1;
    cache.push_back({kernel, dev, dyn_smem, nb});
    return nb;
}

int persistent_grid(const Tuning& t, int blocks_per_sm) {
    if (t.grid_blocks > 0) return t.grid_blocks;
    return sm_count() * blocks_per_sm;
}

void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Kernel timing
// ---------------------------------------------------------------------------
namespace {
const char* const kKernelNames[] = {
    "k_spec_setup", "k_spec_fill", "k_tentative", "k_conflict", "k_priorities",
    "k_rc_bucket", "k_rc_validate", "k_rc_hist", "k_rc_order", "k_rc_scatter",
    "k_rc_recolor_coop", "k_rc_recolor_step", "k_validate", "k_validate_heavy",
    "k_mark_present", "k_count_bits", "k_check_graph", "spec_rounds_graph", "k_batch", "k_brc_hist",
    "k_brc_order", "k_brc_segments", "k_mark_colors"};
static_assert(sizeof(kKernelNames) / sizeof(kKernelNames[0]) == KID_COUNT_,
              "one name per KernelId");
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
long long g_prof_launches[KID_COUNT_];
double g_prof_ms[KID_COUNT_];
struct Pending {
    KernelId k;
    cudaEvent_t e0, e1;
};
thread_local std::vector<Pending> t_pending;
thread_local cudaEvent_t t_open = nullptr;
}  // namespace

void prof_begin(KernelId, cudaStream_t s) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    t_open = e;
}

void prof_end(KernelId k, cudaStream_t s) {
    if (!t_open) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaEventDestroy(t_open);
        t_open = nullptr;
        return;
    }
    cudaEventRecord(e, s);
    t_pending.push_back({k, t_open, e});
    t_open = nullptr;
}

void prof_collect() {
    if (t_pending.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const Pending& p : t_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            g_prof_launches[p.k] += 1;
            g_prof_ms[p.k] += ms;
        }
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    t_pending.clear();
}

namespace {
thread_local bool t_tune_set = false;
thread_local Tuning t_tune;
}  // namespace

void set_thread_tuning(const Tuning* t) {
    t_tune_set = t != nullptr;
    if (t) t_tune = *t;
}

bool thread_tuning(Tuning* out) {
    if (t_tune_set && out) *out = t_tune;
    return t_tune_set;
}

Tuning current_tuning() {
    if (t_tune_set) return t_tune;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

gc_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GC_OK;
    if (e == cudaErrorMemoryAllocation) return GC_ERR_OOM;
    return GC_ERR_CUDA;
}

gc_status status_from_err_bits(uint32_t bits) {
    if (bits & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    if (bits & kErrImproper) return GC_ERR_IMPROPER_INPUT;
    if (bits & kErrTimeout) return GC_ERR_TIMEOUT;
    if (bits & kErrRoundLimit) return GC_ERR_ROUND_LIMIT;
    return GC_OK;
}

namespace {

gc_status check_graph_args(const gc_graph* g) {
    if (!g) return GC_ERR_INVALID_ARG;
    if (g->n < 0 || g->n > INT32_MAX || g->nnz < 0) return GC_ERR_INVALID_ARG;
    if (g->mem != GC_MEM_DEVICE && g->mem != GC_MEM_HOST) return GC_ERR_INVALID_ARG;
    if (g->n > 0 && !g->offsets) return GC_ERR_INVALID_ARG;
    if (g->nnz > 0 && !g->idx) return GC_ERR_INVALID_ARG;
    return GC_OK;
}

// Device view of the caller's graph; host graphs are staged into scratch.
struct DeviceGraph {
    Graph g{};
    Scratch off, idx;
    gc_status stage(const gc_graph* h, cudaStream_t s) {
        g.n = static_cast<int32_t>(h->n);
        g.nnz = h->nnz;
        if (h->mem == GC_MEM_DEVICE) {
            g.off = h->offsets;
            g.idx = h->idx;
            g.vec = (reinterpret_cast<uintptr_t>(g.idx) & 15u) == 0;
            return GC_OK;
        }
        if (!off.alloc((h->n + 1) * sizeof(int64_t), s) || !idx.alloc(h->nnz * sizeof(int32_t), s))
            return GC_ERR_OOM;
        if (h->n > 0 || h->offsets)
            if (cudaMemcpyAsync(off.p, h->offsets, (h->n + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s) != cudaSuccess)
                return GC_ERR_CUDA;
        if (h->nnz > 0)
            if (cudaMemcpyAsync(idx.p, h->idx, h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice,
                                s) != cudaSuccess)
                return GC_ERR_CUDA;
        g.off = off.as<int64_t>();
        g.idx = idx.as<int32_t>();
        g.vec = (reinterpret_cast<uintptr_t>(g.idx) & 15u) == 0;
        return GC_OK;
    }
};

// A colors buffer of n entries in the caller's memory space, seen on the device.
struct DeviceColors {
    int32_t* d = nullptr;
    Scratch sc;
    gc_status stage(int32_t* user, int64_t n, int32_t mem, bool copy_in, cudaStream_t s) {
        if (mem == GC_MEM_DEVICE) {
            d = user;
            return GC_OK;
        }
        if (!sc.alloc(n * sizeof(int32_t), s)) return GC_ERR_OOM;
        d = sc.as<int32_t>();
        if (copy_in && n > 0 &&
            cudaMemcpyAsync(d, user, n * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return GC_ERR_CUDA;
        return GC_OK;
    }
    gc_status unstage(int32_t* user, int64_t n, int32_t mem, cudaStream_t s) {
        if (mem == GC_MEM_DEVICE || n == 0) return GC_OK;
        cudaError_t e = cudaMemcpyAsync(user, d, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return cuda_status(e);
    }
};

}  // namespace
}  // namespace gc

using namespace gc;

extern "C" {

static gc_status gc_color_impl(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                   int32_t* colors_out, gc_stats* stats, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (strategy != GC_FIRST_FIT && strategy != GC_RANDOM_X_FIT) return GC_ERR_INVALID_ARG;
    if (strategy == GC_FIRST_FIT) X = 1;
    if (X < 1) return GC_ERR_INVALID_ARG;
    if (g->n > 0 && !colors_out) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(colors_out, g->n, g->mem, false, s)) != GC_OK) return st;
    st = color_device(dg.g, X, seed, dc.d, stats, s);
    if (st != GC_OK) return st;
    return dc.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_color_ordered_impl(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                                       gc_order order, int32_t* colors_out, gc_stats* stats, void* stream) {
    if (order == GC_ORDER_RANDOM) return gc_color_impl(g, strategy, X, seed, colors_out, stats, stream);
    if (order != GC_ORDER_LARGEST_FIRST) return GC_ERR_INVALID_ARG;
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (strategy != GC_FIRST_FIT && strategy != GC_RANDOM_X_FIT) return GC_ERR_INVALID_ARG;
    if (strategy == GC_FIRST_FIT) X = 1;
    if (X < 1) return GC_ERR_INVALID_ARG;
    if (g->n > 0 && !colors_out) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(colors_out, g->n, g->mem, false, s)) != GC_OK) return st;
    st = color_lf_device(dg.g, X, seed, dc.d, stats, s);
    if (st != GC_OK) return st;
    return dc.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_recolor_async_impl(const gc_graph* g, const int32_t* colors_in, gc_perm perm,
                                       int32_t iterations, uint64_t seed, int32_t* colors_out,
                                       int32_t* ncolors_per_iter, gc_stats* stats, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!perm_valid(perm) || iterations < 0) return GC_ERR_INVALID_ARG;
    if (g->n > 0 && (!colors_in || !colors_out)) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors din;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = din.stage(const_cast<int32_t*>(colors_in), g->n, g->mem, true, s)) != GC_OK) return st;
    int32_t* dout = g->mem == GC_MEM_HOST ? din.d : colors_out;
    st = recolor_async_device(dg.g, din.d, perm, iterations, seed, dout, ncolors_per_iter, stats, s);
    if (st != GC_OK) return st;
    return din.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_recolor_impl(const gc_graph* g, const int32_t* colors_in, gc_perm perm, int32_t iterations,
                     uint64_t seed, int32_t* colors_out, int32_t* ncolors_per_iter, gc_stats* stats,
                     void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!perm_valid(perm) || iterations < 0) return GC_ERR_INVALID_ARG;
    if (g->n > 0 && (!colors_in || !colors_out)) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors din, dout;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = din.stage(const_cast<int32_t*>(colors_in), g->n, g->mem, true, s)) != GC_OK) return st;
    if (g->mem == GC_MEM_HOST) {
        dout.d = din.d;  // recolor in place on the staged copy
    } else {
        dout.d = colors_out;
    }
    st = recolor_device(dg.g, din.d, 0, false, perm, iterations, seed, dout.d, ncolors_per_iter,
                        stats, s);
    if (st != GC_OK) return st;
    return din.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_color_recolor_impl(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_perm perm, int32_t iterations, uint64_t perm_seed, int32_t* colors_out,
                           int32_t* ncolors_per_iter, gc_stats* stats, gc_validation* check,
                           void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (strategy != GC_FIRST_FIT && strategy != GC_RANDOM_X_FIT) return GC_ERR_INVALID_ARG;
    if (strategy == GC_FIRST_FIT) X = 1;
    if (X < 1 || !perm_valid(perm) || iterations < 0)
        return GC_ERR_INVALID_ARG;
    if (g->n > 0 && !colors_out) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(colors_out, g->n, g->mem, false, s)) != GC_OK) return st;
    gc_stats cs;
    st = color_device(dg.g, X, seed, dc.d, &cs, s);
    if (st != GC_OK) return st;
    gc_stats rs;
    st = recolor_device(dg.g, dc.d, cs.max_color, true, perm, iterations, perm_seed, dc.d,
                        ncolors_per_iter, &rs, s);
    if (st != GC_OK) return st;
    if (stats) {
        *stats = cs;
        stats->iterations = iterations;
        stats->max_color = iterations > 0 ? rs.max_color : cs.max_color;
        stats->edges_examined = cs.edges_examined + rs.edges_examined;
        stats->ms_recolor = rs.ms_recolor;
    }
    if (check && (st = validate_device(dg.g, dc.d, check, s)) != GC_OK) return st;
    return dc.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_validate_impl(const gc_graph* g, const int32_t* colors, gc_validation* out, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!out || (g->n > 0 && !colors)) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(const_cast<int32_t*>(colors), g->n, g->mem, true, s)) != GC_OK) return st;
    return validate_device(dg.g, dc.d, out, s);
}

static gc_status gc_check_graph_impl(const gc_graph* g, int64_t* first_bad_vertex, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    return check_graph_device(dg.g, first_bad_vertex, s);
}

static gc_status gc_priorities_impl(uint64_t seed, int64_t n, uint32_t* out, void* stream) {
    if (n < 0 || n > INT32_MAX || (n > 0 && !out)) return GC_ERR_INVALID_ARG;
    return priorities_device(seed, n, out, static_cast<cudaStream_t>(stream));
}

gc_status gc_color(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                   int32_t* colors_out, gc_stats* stats, void* stream) {
    const gc_status st = gc_color_impl(g, strategy, X, seed, colors_out, stats, stream);
    prof_collect();
    return st;
}

gc_status gc_color_ordered(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_order order, int32_t* colors_out, gc_stats* stats, void* stream) {
    const gc_status st = gc_color_ordered_impl(g, strategy, X, seed, order, colors_out, stats, stream);
    prof_collect();
    return st;
}

gc_status gc_recolor_async(const gc_graph* g, const int32_t* colors_in, gc_perm perm,
                           int32_t iterations, uint64_t seed, int32_t* colors_out,
                           int32_t* ncolors_per_iter, gc_stats* stats, void* stream) {
    const gc_status st = gc_recolor_async_impl(g, colors_in, perm, iterations, seed, colors_out,
                                               ncolors_per_iter, stats, stream);
    prof_collect();
    return st;
}

gc_status gc_recolor(const gc_graph* g, const int32_t* colors_in, gc_perm perm, int32_t iterations,
                     uint64_t seed, int32_t* colors_out, int32_t* ncolors_per_iter, gc_stats* stats,
                     void* stream) {
    const gc_status st = gc_recolor_impl(g, colors_in, perm, iterations, seed, colors_out, ncolors_per_iter, stats, stream);
    prof_collect();
    return st;
}

gc_status gc_color_recolor(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_perm perm, int32_t iterations, uint64_t perm_seed, int32_t* colors_out,
                           int32_t* ncolors_per_iter, gc_stats* stats, gc_validation* check,
                           void* stream) {
    const gc_status st = gc_color_recolor_impl(g, strategy, X, seed, perm, iterations, perm_seed, colors_out, ncolors_per_iter, stats, check, stream);
    prof_collect();
    return st;
}

gc_status gc_validate(const gc_graph* g, const int32_t* colors, gc_validation* out, void* stream) {
    const gc_status st = gc_validate_impl(g, colors, out, stream);
    prof_collect();
    return st;
}

gc_status gc_check_graph(const gc_graph* g, int64_t* first_bad_vertex, void* stream) {
    const gc_status st = gc_check_graph_impl(g, first_bad_vertex, stream);
    prof_collect();
    return st;
}

gc_status gc_priorities(uint64_t seed, int64_t n, uint32_t* out, void* stream) {
    const gc_status st = gc_priorities_impl(seed, n, out, stream);
    prof_collect();
    return st;
}

void gc_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < KID_COUNT_; ++k) {
        g_prof_launches[k] = 0;
        g_prof_ms[k] = 0.0;
    }
    g_prof_on.store(on != 0);
}

int32_t gc_profile_read(gc_kernel_time* out, int32_t max) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int32_t cnt = 0;
    for (int k = 0; k < KID_COUNT_; ++k) {
        if (g_prof_launches[k] == 0) continue;
        if (out && cnt < max) {
            std::memset(out[cnt].name, 0, sizeof(out[cnt].name));
            std::strncpy(out[cnt].name, kKernelNames[k], sizeof(out[cnt].name) - 1);
            out[cnt].launches = g_prof_launches[k];
            out[cnt].ms = g_prof_ms[k];
        }
        ++cnt;
    }
    return cnt;
}

static gc_status gc_color_batch_impl(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                                     int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                                     gc_stats* stats, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!graphs || ngraphs < 1 || (g->n > 0 && !colors_out)) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(colors_out, g->n, g->mem, false, s)) != GC_OK) return st;
    st = color_batch_device(dg.g, graphs, ngraphs, dc.d, rounds_out, max_color_out, stats, s);
    if (st != GC_OK) return st;
    return dc.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_recolor_batch_impl(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                                       const int32_t* colors_in, int32_t* colors_out,
                                       int32_t* max_color_out, gc_stats* stats, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!graphs || ngraphs < 1 || (g->n > 0 && (!colors_in || !colors_out))) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors din;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = din.stage(const_cast<int32_t*>(colors_in), g->n, g->mem, true, s)) != GC_OK) return st;
    int32_t* dout = g->mem == GC_MEM_HOST ? din.d : colors_out;
    st = recolor_batch_device(dg.g, graphs, ngraphs, din.d, dout, max_color_out, stats, s);
    if (st != GC_OK) return st;
    return din.unstage(colors_out, g->n, g->mem, s);
}

static gc_status gc_color_recolor_batch_impl(const gc_graph* g, const gc_batch_graph* graphs,
                                             int32_t ngraphs, int32_t* colors_out, int32_t* rounds_out,
                                             int32_t* max_color_out, gc_stats* stats, void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!graphs || ngraphs < 1 || (g->n > 0 && !colors_out)) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGraph dg;
    DeviceColors dc;
    if ((st = dg.stage(g, s)) != GC_OK) return st;
    if ((st = dc.stage(colors_out, g->n, g->mem, false, s)) != GC_OK) return st;
    st = color_recolor_batch_device(dg.g, graphs, ngraphs, dc.d, rounds_out, max_color_out, stats, s);
    if (st != GC_OK) return st;
    return dc.unstage(colors_out, g->n, g->mem, s);
}

gc_status gc_color_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                         int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                         gc_stats* stats, void* stream) {
    const gc_status st = gc_color_batch_impl(g, graphs, ngraphs, colors_out, rounds_out, max_color_out,
                                             stats, stream);
    prof_collect();
    return st;
}

gc_status gc_recolor_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                           const int32_t* colors_in, int32_t* colors_out, int32_t* max_color_out,
                           gc_stats* stats, void* stream) {
    const gc_status st = gc_recolor_batch_impl(g, graphs, ngraphs, colors_in, colors_out, max_color_out,
                                               stats, stream);
    prof_collect();
    return st;
}

gc_status gc_color_recolor_batch(const gc_graph* g, const gc_batch_graph* graphs, int32_t ngraphs,
                                 int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                                 gc_stats* stats, void* stream) {
    const gc_status st = gc_color_recolor_batch_impl(g, graphs, ngraphs, colors_out, rounds_out,
                                                     max_color_out, stats, stream);
    prof_collect();
    return st;
}

gc_status gc_validate_noalloc(const gc_graph* g, const int32_t* colors, gc_validation* out,
                              void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (g->mem != GC_MEM_DEVICE || !out || (g->n > 0 && !colors)) return GC_ERR_INVALID_ARG;
    Graph dg;
    dg.n = static_cast<int32_t>(g->n);
    dg.nnz = g->nnz;
    dg.off = g->offsets;
    dg.idx = g->idx;
    dg.vec = (reinterpret_cast<uintptr_t>(dg.idx) & 15u) == 0;
    return validate_noalloc_device(dg, colors, out, static_cast<cudaStream_t>(stream));
}

static gc_status tuning_from(const gc_tuning* t, Tuning* out) {
    Tuning v = default_tuning();
    if (t) {
        if (t->g2_max_deg < 0 || t->g4_max_deg < t->g2_max_deg || t->g8_max_deg < t->g4_max_deg || t->g16_max_deg < t->g8_max_deg ||
            t->warp_max_deg < 0 || t->grid_blocks < 0 || t->recolor_mode < 0 ||
            t->recolor_mode > 1 || t->spin_limit < 1 || t->spec_graph < 0 || t->spec_graph > 1 ||
            t->rc_warp_max_deg < 0 || t->rc_g2_max_deg < 0)
            return GC_ERR_INVALID_ARG;
        v.g4_max_deg = t->g4_max_deg;
        v.g8_max_deg = t->g8_max_deg;
        v.g16_max_deg = t->g16_max_deg;
        v.warp_max_deg = t->warp_max_deg;
        v.grid_blocks = t->grid_blocks;
        v.recolor_mode = t->recolor_mode;
        v.spin_limit = t->spin_limit;
        v.spec_graph = t->spec_graph;
        v.rc_warp_max_deg = t->rc_warp_max_deg;
        v.g2_max_deg = t->g2_max_deg;
        v.rc_g2_max_deg = t->rc_g2_max_deg;
    }
    *out = v;
    return GC_OK;
}

static gc_tuning tuning_to(const Tuning& t) {
    gc_tuning out;
    out.g4_max_deg = t.g4_max_deg;
    out.g8_max_deg = t.g8_max_deg;
    out.g16_max_deg = t.g16_max_deg;
    out.warp_max_deg = t.warp_max_deg;
    out.grid_blocks = t.grid_blocks;
    out.recolor_mode = t.recolor_mode;
    out.spin_limit = t.spin_limit;
    out.spec_graph = t.spec_graph;
    out.rc_warp_max_deg = t.rc_warp_max_deg;
    out.g2_max_deg = t.g2_max_deg;
    out.rc_g2_max_deg = t.rc_g2_max_deg;
    return out;
}

gc_status gc_set_tuning(const gc_tuning* t) {
    Tuning v;
    gc_status st = tuning_from(t, &v);
    if (st != GC_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = v;
    return GC_OK;
}

gc_status gc_get_tuning(gc_tuning* out) {
    if (!out) return GC_ERR_INVALID_ARG;
    *out = tuning_to(current_tuning());
    return GC_OK;
}

gc_status gc_autotune(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed, gc_perm perm,
                      int32_t iterations, int32_t repeats, gc_tuning* best, float* best_ms,
                      void* stream) {
    gc_status st = check_graph_args(g);
    if (st != GC_OK) return st;
    if (!best || g->mem != GC_MEM_DEVICE || repeats < 1 || g->n < 1) return GC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gc_tuning orig = tuning_to(current_tuning());
    int32_t* colors = nullptr;
    Scratch sc;
    if (!sc.alloc(g->n * sizeof(int32_t), s)) return GC_ERR_OOM;
    colors = sc.as<int32_t>();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // each candidate runs on this thread only (the process-wide knobs stay)
    auto time_it = [&](const gc_tuning& t, float* ms) -> gc_status {
        Tuning v;
        gc_status r = tuning_from(&t, &v);
        if (r != GC_OK) return r;
        ThreadTuningScope scope(v);
        r = gc_color_recolor_impl(g, strategy, X, seed, perm, iterations, 0, colors, nullptr, nullptr,
                                  nullptr, stream);  // warm-up
        if (r != GC_OK) return r;
        cudaEventRecord(e0, s);
        for (int32_t i = 0; i < repeats && r == GC_OK; ++i)
            r = gc_color_recolor_impl(g, strategy, X, seed, perm, iterations, 0, colors, nullptr,
                                      nullptr, nullptr, stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t_ms = 0.f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        *ms = t_ms / repeats;
        return r;
    };
    gc_tuning cur = orig;
    float cur_ms = 0.f;
    st = time_it(cur, &cur_ms);
    // one knob at a time, keeping any improvement
    const int32_t groups[][3] = {{64, 64, 64}, {4, 8, 16}, {0, 0, 0}, {0, 64, 64}, {16, 32, 64}};
    const int32_t warp_max[] = {256, 1024, 2048};
    const int32_t rc_warp_max[] = {256, 512, 1024};
    const int32_t g2_max[] = {0, 16, 32};
    const int32_t rc_g2_max[] = {0, 8, 32};
    const int32_t blocks_per_sm[] = {0, 2, 4};
    for (int step = 0; step < 8 && st == GC_OK; ++step) {
        const int variants = step == 0 ? 5 : step == 1 ? 3 : step == 2 ? 2 : step == 3 ? 2 : 3;
        for (int i = 0; i < variants && st == GC_OK; ++i) {
            gc_tuning t = cur;
            if (step == 0) {
                t.g4_max_deg = groups[i][0];
                t.g8_max_deg = groups[i][1];
                t.g16_max_deg = groups[i][2];
                t.g2_max_deg = std::min(t.g2_max_deg, t.g4_max_deg);
            }
            else if (step == 1) t.warp_max_deg = warp_max[i];
            else if (step == 2) t.recolor_mode = i;
            else if (step == 3) t.spec_graph = i;
            else if (step == 4) t.grid_blocks = blocks_per_sm[i] * sm_count();
            else if (step == 5) t.rc_warp_max_deg = rc_warp_max[i];
            else if (step == 6) t.g2_max_deg = std::min(g2_max[i], t.g4_max_deg);
            else t.rc_g2_max_deg = rc_g2_max[i];
            if (std::memcmp(&t, &cur, sizeof(t)) == 0) continue;
            float ms = 0.f;
            st = time_it(t, &ms);
            if (st == GC_OK && ms < cur_ms) { cur = t; cur_ms = ms; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GC_OK) return st;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return GC_OK;
}

}  // extern "C"

// A plan: run settings plus the knobs to run them with (see gc.h).
struct gc_plan {
    Tuning tune;
    gc_plan_info info;
};

extern "C" {

gc_status gc_plan_create(const gc_tuning* t, gc_strategy strategy, int32_t X, gc_perm perm,
                         int32_t iterations, gc_plan** out) {
    if (!out) return GC_ERR_INVALID_ARG;
    Tuning v;
    if (tuning_from(t, &v) != GC_OK) return GC_ERR_INVALID_ARG;
    if (strategy != GC_FIRST_FIT && strategy != GC_RANDOM_X_FIT) return GC_ERR_INVALID_ARG;
    if (strategy == GC_FIRST_FIT) X = 1;
    if (X < 1 || !perm_valid(perm) || iterations < 0) return GC_ERR_INVALID_ARG;
    gc_plan* p = new (std::nothrow) gc_plan;
    if (!p) return GC_ERR_OOM;
    p->tune = v;
    std::memset(&p->info, 0, sizeof(p->info));
    p->info.tuning = tuning_to(v);
    p->info.strategy = strategy;
    p->info.X = X;
    p->info.perm = perm;
    p->info.iterations = iterations;
    *out = p;
    return GC_OK;
}

gc_status gc_plan_autotune(const gc_graph* g, gc_strategy strategy, int32_t X, uint64_t seed,
                           gc_perm perm, int32_t iterations, int32_t repeats, gc_plan** out,
                           void* stream) {
    if (!out) return GC_ERR_INVALID_ARG;
    gc_tuning best;
    float ms = 0.f;
    gc_status st = gc_autotune(g, strategy, X, seed, perm, iterations, repeats, &best, &ms, stream);
    if (st != GC_OK) return st;
    gc_plan* p = nullptr;
    if ((st = gc_plan_create(&best, strategy, X, perm, iterations, &p)) != GC_OK) return st;
    p->info.tuned_ms = ms;
    p->info.tuned_n = g->n;
    p->info.tuned_nnz = g->nnz;
    *out = p;
    return GC_OK;
}

gc_status gc_plan_get_info(const gc_plan* p, gc_plan_info* out) {
    if (!p || !out) return GC_ERR_INVALID_ARG;
    *out = p->info;
    return GC_OK;
}

gc_status gc_plan_color_recolor(const gc_plan* p, const gc_graph* g, uint64_t seed,
                                uint64_t perm_seed, int32_t* colors_out, int32_t* ncolors_per_iter,
                                gc_stats* stats, gc_validation* check, void* stream) {
    if (!p) return GC_ERR_INVALID_ARG;
    gc_status st;
    {
        ThreadTuningScope scope(p->tune);
        st = gc_color_recolor_impl(g, static_cast<gc_strategy>(p->info.strategy), p->info.X, seed,
                                   static_cast<gc_perm>(p->info.perm), p->info.iterations, perm_seed,
                                   colors_out, ncolors_per_iter, stats, check, stream);
    }
    prof_collect();
    return st;
}

void gc_plan_free(gc_plan* p) { delete p; }

gc_status gc_preset_params(gc_preset preset, int32_t* strategy, int32_t* X, int32_t* perm,
                           int32_t* iterations) {
    int32_t s_, x_, p_, i_;
    switch (preset) {
    case GC_PRESET_SPEED: s_ = GC_FIRST_FIT; x_ = 1; p_ = GC_PERM_NONDEC; i_ = 0; break;
    case GC_PRESET_QUALITY: s_ = GC_RANDOM_X_FIT; x_ = 5; p_ = GC_PERM_NONDEC; i_ = 1; break;
    case GC_PRESET_QUALITY_X10: s_ = GC_RANDOM_X_FIT; x_ = 10; p_ = GC_PERM_NONDEC; i_ = 1; break;
    default: return GC_ERR_INVALID_ARG;
    }
    if (strategy) *strategy = s_;
    if (X) *X = x_;
    if (perm) *perm = p_;
    if (iterations) *iterations = i_;
    return GC_OK;
}

void gc_inject_alloc_failure(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }

int64_t gc_kernel_launches(void) { return g_launches.load(); }

const char* gc_status_string(gc_status s) {
    switch (s) {
    case GC_OK: return "ok";
    case GC_ERR_INVALID_ARG: return "invalid argument";
    case GC_ERR_BAD_GRAPH: return "malformed CSR graph";
    case GC_ERR_IMPROPER_INPUT: return "input coloring is not proper";
    case GC_ERR_OOM: return "out of memory";
    case GC_ERR_CUDA: return "CUDA runtime error";
    case GC_ERR_TIMEOUT: return "bounded device wait expired";
    case GC_ERR_ROUND_LIMIT: return "speculative round limit exceeded";
    case GC_ERR_BUDGET: return "request larger than the server's memory budget";
    case GC_PENDING: return "request pending";
    }
    return "unknown status";
}

int32_t gc_version(void) { return 100; }

}  // extern "C"
