// gc_util.cu -- validation of a coloring (the definition of Sec. 1:
// C(u) != C(v) on every edge, #colors = max_u C(u)) and the CSR structure
// check.  Both are one pass over the adjacency, warp per vertex.
#include <algorithm>
#include <climits>
#include <cstring>

#include "gc_internal.h"

namespace gc {

struct ValCtrl {
    unsigned long long conflicts;
    unsigned long long uncolored;
    long long first_bad;
    int32_t max_color;
    uint32_t err;
    unsigned long long distinct;
};

__global__ void __launch_bounds__(kBlock) k_validate(Graph g, const int32_t* colors, ValCtrl* c) {
    const int w = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int nw = (gridDim.x * kBlock) >> 5;
    const int l = lane_id();
    int32_t my_max = 0;
    unsigned long long conf = 0, unc = 0;
    for (int64_t v = w; v < g.n; v += nw) {
        const int32_t cv = colors[v];
        int64_t beg, end;
        row_range(g, static_cast<int32_t>(v), beg, end, &c->err);
        int32_t mine = 0;
        for (int64_t e = beg + l; e < end; e += 32) {
            const int32_t u = load_nbr(g, e, &c->err);
            if (u >= 0 && colors[u] == cv) ++mine;
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) mine += __shfl_xor_sync(kFull, mine, d);
        if (l == 0) {
            conf += static_cast<unsigned long long>(mine);
            if (cv < 1) ++unc;
            if (cv < 1 || mine > 0) atomicMin(&c->first_bad, static_cast<long long>(v));
            my_max = max(my_max, cv);
        }
    }
    warp_add(&c->conflicts, conf);
    warp_add(&c->uncolored, unc);
    warp_max(&c->max_color, my_max);
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
    Scratch sc;
    if (!sc.alloc(sizeof(ValCtrl), s)) return GC_ERR_OOM;
    ValCtrl* c = sc.as<ValCtrl>();
    ValCtrl h;
    std::memset(&h, 0, sizeof(h));
    h.first_bad = LLONG_MAX;
    cudaMemcpyAsync(c, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    const Tuning t = current_tuning();
    const int grid = persistent_grid(t);
    GC_LAUNCH(KID_VALIDATE, s, k_validate<<<grid, kBlock, 0, s>>>(g, colors, c));
    cudaError_t ce = cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    int64_t distinct = 0;
    if (h.max_color >= 1) {
        const int64_t words = (static_cast<int64_t>(h.max_color) >> 5) + 1;
        Scratch sb;
        if (!sb.alloc(words * 4, s)) return GC_ERR_OOM;
        cudaMemsetAsync(sb.p, 0, words * 4, s);
        const int vg = static_cast<int>(std::min<int64_t>((g.n + kBlock - 1) / kBlock, grid));
        GC_LAUNCH(KID_MARK_PRESENT, s, k_mark_present<<<vg, kBlock, 0, s>>>(g.n, colors, sb.as<uint32_t>()));
        const int wg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((words + kBlock - 1) / kBlock, grid)));
        GC_LAUNCH(KID_COUNT_BITS, s, k_count_bits<<<wg, kBlock, 0, s>>>(words, sb.as<uint32_t>(), c));
        ce = cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s);
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
