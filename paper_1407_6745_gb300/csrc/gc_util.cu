// gc_util.cu -- validation of a coloring (the definition of Sec. 1:
// C(u) != C(v) on every edge, #colors = max_u C(u)) and the CSR structure
// check.  Both are one pass over the adjacency, warp per vertex.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "gc_internal.h"

namespace gc {

struct ValCtrl {
    unsigned long long conflicts;
    unsigned long long uncolored;
    long long first_bad;
    int32_t max_color;
    uint32_t err;
    unsigned long long distinct;
    int32_t heavy;          // rows deferred to the block-per-row pass (gc_validate: to the warp-per-row one)
    int32_t big_colors;     // vertices with a color >= kPresColors
    int32_t big;            // gc_validate: pieces of the rows beyond kValWarpDeg
};

constexpr int kValG = 4;                 // lanes per light row (measured: 8 -> 4 saves 30 us on the stencil)
constexpr int32_t kHeavyDeg = 256;       // heavier rows: one block each (gc_validate_noalloc)
// gc_validate: rows of up to kValLightDeg entries take kValG lanes (one
// pass of loads), up to kValWarpDeg a warp, longer ones a block.  (R-MAT
// scale 24: 2.77 + 1.60 ms with the noalloc form's split at 256 entries.)
constexpr int32_t kValLightDeg = 64;
constexpr int32_t kValWarpDeg = 4096;
// Rows beyond kValWarpDeg are cut into pieces of kValPiece entries, a block
// each (the largest R-MAT rows hold hundreds of thousands of entries; one
// block per row left a single block walking the largest).
constexpr int32_t kValPiece = 4096;
constexpr int kPresWords = 2048;         // presence bitmap of colors < 65536
constexpr int32_t kPresColors = kPresWords * 32;

struct ValArgs {
    Graph g;
    const int32_t* colors;
    ValCtrl* c;
    uint32_t* pres;    // kPresWords
    int32_t* heavy;    // n
    int2* pieces;      // gc_validate: (row, piece index) of the rows beyond kValWarpDeg
    int64_t piece_cap;
};

// Count of neighbors with v's color in this lane's stripe.
template <int UC>
__device__ __forceinline__ int32_t same_color(const ValArgs& a, int64_t beg, int32_t deg, int32_t cv,
                                              int32_t lane0, int32_t stride) {
    int32_t cnt = 0;
    for_each_nbr<UC, int32_t, true>(
        a.g, beg, deg, lane0, stride, [&](int32_t u) { return __ldg(a.colors + u); },
        [&](int32_t, int32_t x) { cnt += x == cv; }, &a.c->err);
    return cnt;
}

__device__ __forceinline__ void account(const ValArgs& a, int32_t v, int32_t cv, int32_t same,
                                        uint32_t* s_pres, unsigned long long& conf,
                                        unsigned long long& unc, int32_t& my_max) {
    conf += static_cast<unsigned long long>(same);
    if (cv < 1) ++unc;
    if (cv < 1 || same > 0) atomicMin(&a.c->first_bad, static_cast<long long>(v));
    my_max = max(my_max, cv);
    if (cv >= 1 && cv < kPresColors) atomicOr(&s_pres[cv >> 5], 1u << (cv & 31));
    else if (cv >= kPresColors) atomicAdd(&a.c->big_colors, 1);
}

// One piece of a row: its same-colored neighbors; the row's own accounting
// (uncolored, max color, presence) with its first piece only.
__device__ __forceinline__ void account_piece(const ValArgs& a, int32_t v, int32_t cv, int32_t same, bool first,
                                              uint32_t* s_pres, unsigned long long& conf,
                                              unsigned long long& unc, int32_t& my_max) {
    if (first) {
        account(a, v, cv, same, s_pres, conf, unc, my_max);
        return;
    }
    conf += static_cast<unsigned long long>(same);
    if (same > 0) atomicMin(&a.c->first_bad, static_cast<long long>(v));
}

__device__ __forceinline__ void flush_presence(const ValArgs& a, uint32_t* s_pres) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPresWords; i += kBlock)
        if (s_pres[i]) atomicOr(&a.pres[i], s_pres[i]);
}

// Light rows: kValG lanes per vertex; longer rows are listed for the next
// pass, from the front of `heavy` up to kValWarpDeg entries, from the back
// beyond.
__global__ void __launch_bounds__(kBlock) k_validate(ValArgs a) {
    __shared__ uint32_t s_pres[kPresWords];
    for (int i = threadIdx.x; i < kPresWords; i += kBlock) s_pres[i] = 0u;
    __syncthreads();
    const int gi = threadIdx.x / kValG, gl = threadIdx.x % kValG;
    const int64_t groups = static_cast<int64_t>(gridDim.x) * (kBlock / kValG);
    int32_t my_max = 0;
    unsigned long long conf = 0, unc = 0;
    const int64_t n_pad = (a.g.n + groups - 1) / groups * groups;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * (kBlock / kValG) + gi; v < n_pad; v += groups) {
        const bool valid = v < a.g.n;
        int64_t beg = 0;
        int32_t deg = 0, cv = 0;
        bool heavy = false;
        if (valid) {
            row_of(a.g, static_cast<int32_t>(v), beg, deg, &a.c->err);
            cv = a.colors[v];
            heavy = deg > kValLightDeg;
        }
        int32_t same = same_color<1>(a, beg, heavy ? 0 : deg, cv, gl, kValG);
#pragma unroll
        for (int d = kValG / 2; d >= 1; d >>= 1) same += __shfl_xor_sync(kFull, same, d);
        if (valid && gl == 0) {
            if (!heavy) account(a, static_cast<int32_t>(v), cv, same, s_pres, conf, unc, my_max);
            else if (deg <= kValWarpDeg) a.heavy[atomicAdd(&a.c->heavy, 1)] = static_cast<int32_t>(v);
            else {
                const int32_t np = (deg + kValPiece - 1) / kValPiece;
                const int32_t p0 = atomicAdd(&a.c->big, np);
                for (int32_t i = 0; i < np && p0 + i < a.piece_cap; ++i)
                    a.pieces[p0 + i] = make_int2(static_cast<int32_t>(v), i);
            }
        }
    }
    warp_add(&a.c->conflicts, conf);
    warp_add(&a.c->uncolored, unc);
    warp_max(&a.c->max_color, my_max);
    flush_presence(a, s_pres);
}

// The rows k_validate listed: a warp each up to kValWarpDeg entries, then a
// block per piece of kValPiece entries beyond.
__global__ void __launch_bounds__(kBlock) k_validate_heavy(ValArgs a) {
    __shared__ uint32_t s_pres[kPresWords];
    __shared__ int32_t s_sum[kWarps];
    for (int i = threadIdx.x; i < kPresWords; i += kBlock) s_pres[i] = 0u;
    __syncthreads();
    int32_t my_max = 0;
    unsigned long long conf = 0, unc = 0;
    const int32_t nmid = a.c->heavy, nbig = a.c->big;
    const int w = threadIdx.x >> 5, l = lane_id();
    for (int32_t h = blockIdx.x * kWarps + w; h < nmid; h += gridDim.x * kWarps) {
        const int32_t v = a.heavy[h];
        int64_t beg;
        int32_t deg;
        row_of(a.g, v, beg, deg, &a.c->err);
        const int32_t cv = a.colors[v];
        int32_t same = same_color<2>(a, beg, deg, cv, l, 32);
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) same += __shfl_xor_sync(kFull, same, d);
        if (l == 0) account(a, v, cv, same, s_pres, conf, unc, my_max);
    }
    const int64_t npieces = nbig < a.piece_cap ? nbig : a.piece_cap;
    for (int64_t k = blockIdx.x; k < npieces; k += gridDim.x) {
        const int2 pc = a.pieces[k];
        const int32_t v = pc.x;
        int64_t beg;
        int32_t deg;
        row_of(a.g, v, beg, deg, &a.c->err);
        const int64_t off = static_cast<int64_t>(pc.y) * kValPiece;
        const int32_t len = static_cast<int32_t>(min(static_cast<int64_t>(kValPiece), deg - off));
        const int32_t cv = a.colors[v];
        int32_t same = same_color<1>(a, beg + off, len, cv, threadIdx.x, kBlock);
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) same += __shfl_xor_sync(kFull, same, d);
        if (lane_id() == 0) s_sum[threadIdx.x >> 5] = same;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int q = 0; q < kWarps; ++q) tot += s_sum[q];
            account_piece(a, v, cv, tot, pc.y == 0, s_pres, conf, unc, my_max);
        }
        __syncthreads();
    }
    warp_add(&a.c->conflicts, conf);
    warp_add(&a.c->uncolored, unc);
    warp_max(&a.c->max_color, my_max);
    flush_presence(a, s_pres);
}

__global__ void __launch_bounds__(kBlock) k_mark_present(int64_t n, const int32_t* colors,
                                                         uint32_t* bits) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < n; v += stride) {
        const int32_t cv = colors[v];
        if (cv >= 1) atomicOr(&bits[cv >> 5], 1u << (cv & 31));
    }
}

__global__ void __launch_bounds__(kBlock) k_count_bits(int64_t words, const uint32_t* bits,
                                                       ValCtrl* c) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    unsigned long long s = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; i < words; i += stride)
        s += __popc(bits[i]);
    warp_add(&c->distinct, s);
}

gc_status validate_device(const Graph& g, const int32_t* colors, gc_validation* out,
                          cudaStream_t s) {
    std::memset(out, 0, sizeof(*out));
    out->first_bad_vertex = -1;
    if (g.n == 0) return GC_OK;
    Scratch sc, sp, shv, spc;
    // pieces: at most one per kValPiece entries, plus one per row beyond kValWarpDeg
    const int64_t piece_cap = g.nnz / kValPiece + g.nnz / kValWarpDeg + 1;
    if (!sc.alloc(sizeof(ValCtrl), s) || !sp.alloc(kPresWords * 4, s) || !shv.alloc(static_cast<int64_t>(g.n) * 4, s) ||
        !spc.alloc(piece_cap * sizeof(int2), s))
        return GC_ERR_OOM;
    ValArgs a{g, colors, sc.as<ValCtrl>(), sp.as<uint32_t>(), shv.as<int32_t>(), spc.as<int2>(), piece_cap};
    ValCtrl h;
    std::memset(&h, 0, sizeof(h));
    h.first_bad = LLONG_MAX;
    cudaMemcpyAsync(a.c, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(a.pres, 0, kPresWords * 4, s);
    const Tuning t = current_tuning();
    const int grid = persistent_grid(t);
    GC_LAUNCH(KID_VALIDATE, s, k_validate<<<resident_grid(k_validate, t), kBlock, 0, s>>>(a));
    GC_LAUNCH(KID_VALIDATE_HEAVY, s,
              k_validate_heavy<<<resident_grid(k_validate_heavy, t), kBlock, 0, s>>>(a));
    GC_LAUNCH(KID_COUNT_BITS, s, k_count_bits<<<8, kBlock, 0, s>>>(kPresWords, a.pres, a.c));
    cudaError_t ce = cudaMemcpyAsync(&h, a.c, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    int64_t distinct = static_cast<int64_t>(h.distinct);
    if (h.big_colors > 0) {
        // colors beyond the shared bitmap: one bit per color up to the max
        const int64_t words = (static_cast<int64_t>(h.max_color) >> 5) + 1;
        Scratch sb;
        if (!sb.alloc(words * 4, s)) return GC_ERR_OOM;
        cudaMemsetAsync(sb.p, 0, words * 4, s);
        cudaMemsetAsync(&a.c->distinct, 0, sizeof(unsigned long long), s);
        const int vg = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(g.n) + kBlock - 1) / kBlock, grid));
        GC_LAUNCH(KID_MARK_PRESENT, s, k_mark_present<<<vg, kBlock, 0, s>>>(g.n, colors, sb.as<uint32_t>()));
        const int wg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((words + kBlock - 1) / kBlock, grid)));
        GC_LAUNCH(KID_COUNT_BITS, s, k_count_bits<<<wg, kBlock, 0, s>>>(words, sb.as<uint32_t>(), a.c));
        ce = cudaMemcpyAsync(&h, a.c, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_status(ce);
        distinct = static_cast<int64_t>(h.distinct);
    }
    out->n_conflicts = static_cast<int64_t>(h.conflicts);
    out->n_uncolored = static_cast<int64_t>(h.uncolored);
    out->max_color = h.max_color;
    out->n_distinct = static_cast<int32_t>(distinct);
    out->first_bad_vertex = h.first_bad == LLONG_MAX ? -1 : static_cast<int64_t>(h.first_bad);
    return GC_OK;
}

// ---------------------------------------------------------------------------
// Validation without allocation (gc_validate_noalloc).  For callers that
// cannot allocate device memory: a process whose own caching allocator has
// reserved the device's memory up front (a cudaMalloc would fail or fragment
// it), a caller checking a result after an out-of-memory error, or a
// latency-critical path that must not wait on the driver's allocator.  Its
// scratch is a file-scope device array, held by every device that loads the
// library until the process exits; every call shares it, so two calls that
// overlap on the GPU (e.g. on two streams) race on it and must be serialised
// by the caller.  The call reads its result back and synchronizes the
// caller's stream.  The presence bitmap covers colors below kPresColors
// (65536); a coloring with a larger color is rejected, since counting its
// distinct colors would need scratch beyond the array.
// ---------------------------------------------------------------------------
struct NoAllocScratch {
    ValCtrl ctrl;
    uint32_t pres[kPresWords];
};

static __device__ __align__(256) NoAllocScratch g_validate_scratch;

// Clears what every call must start from: counters, the first bad vertex
// (LLONG_MAX = none yet) and the presence bitmap.
__global__ void __launch_bounds__(kBlock) k_validate_na_clear(NoAllocScratch* sc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->ctrl.conflicts = 0;
        sc->ctrl.uncolored = 0;
        sc->ctrl.first_bad = LLONG_MAX;
        sc->ctrl.max_color = 0;
        sc->ctrl.err = 0;
        sc->ctrl.distinct = 0;
        sc->ctrl.heavy = 0;
        sc->ctrl.big_colors = 0;
    }
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < kPresWords; i += gridDim.x * kBlock)
        sc->pres[i] = 0u;
}

// Light rows, kValG lanes per vertex; heavy rows are left to the next kernel
// (which finds them again by degree instead of through a list).
__global__ void __launch_bounds__(kBlock) k_validate_na_light(ValArgs a) {
    __shared__ uint32_t s_pres[kPresWords];
    for (int i = threadIdx.x; i < kPresWords; i += kBlock) s_pres[i] = 0u;
    __syncthreads();
    const int gi = threadIdx.x / kValG, gl = threadIdx.x % kValG;
    const int64_t groups = static_cast<int64_t>(gridDim.x) * (kBlock / kValG);
    int32_t my_max = 0;
    unsigned long long conf = 0, unc = 0;
    const int64_t n_pad = (a.g.n + groups - 1) / groups * groups;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * (kBlock / kValG) + gi; v < n_pad; v += groups) {
        const bool valid = v < a.g.n;
        int64_t beg = 0;
        int32_t deg = 0, cv = 0;
        bool heavy = false;
        if (valid) {
            row_of(a.g, static_cast<int32_t>(v), beg, deg, &a.c->err);
            cv = a.colors[v];
            heavy = deg > kHeavyDeg;
        }
        int32_t same = same_color<1>(a, beg, heavy ? 0 : deg, cv, gl, kValG);
#pragma unroll
        for (int d = kValG / 2; d >= 1; d >>= 1) same += __shfl_xor_sync(kFull, same, d);
        if (valid && gl == 0 && !heavy) account(a, static_cast<int32_t>(v), cv, same, s_pres, conf, unc, my_max);
    }
    warp_add(&a.c->conflicts, conf);
    warp_add(&a.c->uncolored, unc);
    warp_max(&a.c->max_color, my_max);
    flush_presence(a, s_pres);
}

// Heavy rows (degree > kHeavyDeg), one block per row, found by a scan of the
// degrees.
__global__ void __launch_bounds__(kBlock) k_validate_na_heavy(ValArgs a) {
    __shared__ uint32_t s_pres[kPresWords];
    __shared__ int32_t s_sum[kWarps];
    for (int i = threadIdx.x; i < kPresWords; i += kBlock) s_pres[i] = 0u;
    __syncthreads();
    int32_t my_max = 0;
    unsigned long long conf = 0, unc = 0;
    for (int64_t v0 = static_cast<int64_t>(blockIdx.x) * kBlock; v0 < a.g.n;
         v0 += static_cast<int64_t>(gridDim.x) * kBlock) {
        // the block's threads look at kBlock vertices, then walk the heavy ones
        const int64_t mine = v0 + threadIdx.x;
        bool heavy = false;
        if (mine < a.g.n) {
            const int64_t b = a.g.off[mine], e = a.g.off[mine + 1];
            heavy = e - b > kHeavyDeg;
        }
        uint32_t mask = __ballot_sync(kFull, heavy);
        __shared__ uint32_t s_mask[kWarps];
        if (lane_id() == 0) s_mask[threadIdx.x >> 5] = mask;
        __syncthreads();
        for (int w = 0; w < kWarps; ++w) {
            uint32_t m = s_mask[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int32_t v = static_cast<int32_t>(v0 + w * 32 + bit);
                int64_t beg;
                int32_t deg;
                row_of(a.g, v, beg, deg, &a.c->err);
                const int32_t cv = a.colors[v];
                int32_t same = same_color<1>(a, beg, deg, cv, threadIdx.x, kBlock);
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) same += __shfl_xor_sync(kFull, same, d);
                if (lane_id() == 0) s_sum[threadIdx.x >> 5] = same;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int32_t tot = 0;
                    for (int q = 0; q < kWarps; ++q) tot += s_sum[q];
                    account(a, v, cv, tot, s_pres, conf, unc, my_max);
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
    warp_add(&a.c->conflicts, conf);
    warp_add(&a.c->uncolored, unc);
    warp_max(&a.c->max_color, my_max);
    flush_presence(a, s_pres);
}

namespace {
constexpr int kNoAllocDevices = 64;
std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[kNoAllocDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in).
gc_status noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return GC_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocDevices) return GC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_validate_scratch);
        if (e != cudaSuccess || !p) return GC_ERR_CUDA;
        g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_na_ptr[dev];
    return GC_OK;
}

int noalloc_grid(const void* kernel) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max(1, sms) * per_sm;
}
}  // namespace

gc_status validate_noalloc_device(const Graph& g, const int32_t* colors, gc_validation* out,
                                  cudaStream_t s) {
    std::memset(out, 0, sizeof(*out));
    out->first_bad_vertex = -1;
    if (g.n == 0) return GC_OK;
    NoAllocScratch* sc = nullptr;
    gc_status st = noalloc_scratch(&sc);
    if (st != GC_OK) return st;
    ValArgs a{g, colors, &sc->ctrl, sc->pres, nullptr};
    // Each launch is checked before the next is enqueued: a clear that failed
    // to launch must not let the read-back return the previous call's counts.
    // (Not bracketed by the profiling events, which would create events.)
    cudaError_t ce;
    k_validate_na_clear<<<8, kBlock, 0, s>>>(sc);
    note_launches(1);
    if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_status(ce);
    k_validate_na_light<<<noalloc_grid(reinterpret_cast<const void*>(k_validate_na_light)), kBlock, 0, s>>>(a);
    note_launches(1);
    if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_status(ce);
    k_validate_na_heavy<<<noalloc_grid(reinterpret_cast<const void*>(k_validate_na_heavy)), kBlock, 0, s>>>(a);
    note_launches(1);
    if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_status(ce);
    k_count_bits<<<8, kBlock, 0, s>>>(kPresWords, sc->pres, &sc->ctrl);
    note_launches(1);
    if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_status(ce);
    ValCtrl h;
    ce = cudaMemcpyAsync(&h, &sc->ctrl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    if (h.big_colors > 0) return GC_ERR_INVALID_ARG;  // a color >= 65536: beyond the scratch
    out->n_conflicts = static_cast<int64_t>(h.conflicts);
    out->n_uncolored = static_cast<int64_t>(h.uncolored);
    out->max_color = h.max_color;
    out->n_distinct = static_cast<int32_t>(h.distinct);
    out->first_bad_vertex = h.first_bad == LLONG_MAX ? -1 : static_cast<int64_t>(h.first_bad);
    return GC_OK;
}

// ---------------------------------------------------------------------------
// CSR structure check
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_check_graph(Graph g, long long* first_bad) {
    const int w = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int nw = (gridDim.x * kBlock) >> 5;
    const int l = lane_id();
    for (int64_t v = w; v < g.n; v += nw) {
        const int64_t beg = g.off[v], end = g.off[v + 1];
        bool bad = beg < 0 || end < beg || end > g.nnz || (v == 0 && beg != 0) ||
                   (v == g.n - 1 && end != g.nnz);
        if (!bad) {
            for (int64_t e = beg + l; e < end; e += 32) {
                const int32_t u = g.idx[e];
                if (u < 0 || u >= g.n || u == v) bad = true;
            }
        }
        if (__any_sync(kFull, bad) && l == 0) atomicMin(first_bad, static_cast<long long>(v));
    }
}

gc_status check_graph_device(const Graph& g, int64_t* first_bad, cudaStream_t s) {
    if (first_bad) *first_bad = -1;
    if (g.n == 0) return g.nnz == 0 ? GC_OK : GC_ERR_BAD_GRAPH;
    Scratch sc;
    if (!sc.alloc(sizeof(long long), s)) return GC_ERR_OOM;
    long long h = LLONG_MAX;
    cudaMemcpyAsync(sc.p, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    GC_LAUNCH(KID_CHECK_GRAPH, s,
              k_check_graph<<<persistent_grid(current_tuning()), kBlock, 0, s>>>(g, sc.as<long long>()));
    cudaError_t ce = cudaMemcpyAsync(&h, sc.p, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h == LLONG_MAX) return GC_OK;
    if (first_bad) *first_bad = static_cast<int64_t>(h);
    return GC_ERR_BAD_GRAPH;
}

}  // namespace gc
