// gc_recolor.cu -- iterative recoloring on one GPU.
//
// Culberson's iterated greedy (Sec. 2.1) as synchronous recoloring RC
// (Sec. 3): the classes of the previous coloring are taken one after the
// other in a class permutation (RV, NI, ND or RAND, Sec. 3) and every vertex
// takes the smallest color not used by a neighbor of an earlier class.  A
// class is an independent set, so all its vertices can choose at once and
// the result equals the sequential greedy run in class order (Sec. 3).
//
// One iteration = four launches, with no host round trip:
//   k_rc_hist     histogram of (class, degree bucket) pairs;
//   k_rc_order    the class permutation, computed on the device (one block):
//                 present classes, RV/NI/ND order or a Fisher-Yates shuffle,
//                 rank of every color, segment starts and tile counts;
//   k_rc_scatter  counting sort of the vertices into class-major,
//                 bucket-minor segments; new[v] = -(rank(v) + 1);
//   k_rc_recolor  the class steps.  Dataflow form: blocks claim tiles in
//                 class order from an atomic counter; a neighbor u of an
//                 earlier class whose new color is not yet written (still
//                 negative) is waited for, with a bounded spin; a neighbor of
//                 a later class (negative, rank above v's) is ignored.  All
//                 earlier tiles were claimed by running blocks, and the
//                 earliest unfinished tile waits on nothing, so the waits
//                 always end.  The alternative form launches one grid per
//                 class and needs no waits.
// The negative encoding makes one 4-byte gather per edge serve both "is u
// earlier than v" and "what color did u take".
#include <algorithm>
#include <cstring>
#include <vector>

#include "gc_internal.h"

namespace gc {

constexpr int32_t kMaxInputColor = 1 << 28;
constexpr int kOrderThreads = 1024;
constexpr int kShuffleSmem = 4096;

struct RcCtrl {
    int32_t k;            // present classes this iteration
    int32_t total_tiles;
    int32_t claim;        // next tile to claim (dataflow)
    int32_t max_deg;
    int32_t max_in;       // max input color (validation)
    uint32_t err;
    unsigned long long edges;
};

struct RcArgs {
    Graph g;
    Tuning tune;
    uint64_t seed;
    int32_t perm;
    int32_t iteration;
    int32_t cap;          // colors are in [1, cap]
    const int32_t* old_c;
    int32_t* new_c;
    uint8_t* bucket;
    int32_t* cls_cnt;     // (cap + 1) * kNB
    int32_t* present;     // cap + 1
    int32_t* psize;       // cap + 1
    int32_t* order;       // cap + 1 (class order, colors)
    int32_t* jtab;        // cap + 1 (shuffle indices)
    int32_t* rank_of;     // cap + 1
    int32_t* seg_start;   // (cap + 1) * kNB + 1
    int32_t* tile_prefix; // (cap + 1) * kNB + 1
    int32_t* fill;        // (cap + 1) * kNB
    WorkItem* list;       // n, vertices in class-major order
    int32_t* ncolors;     // iterations + 1
    RcCtrl* ctrl;
};

__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
    int32_t x;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(x) : "l"(p));
    return x;
}
__device__ __forceinline__ void st_relaxed(int32_t* p, int32_t x) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

// ---------------------------------------------------------------------------
// Per-call set-up: degree buckets (X = 1) and, for untrusted input, the
// proper-coloring check of Sec. 1 plus the max color.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_rc_bucket(RcArgs a) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    int32_t my_max = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; i < a.g.n; i += stride) {
        int64_t beg, end;
        row_range(a.g, static_cast<int32_t>(i), beg, end, &a.ctrl->err);
        const int64_t deg = end - beg;
        my_max = max(my_max, static_cast<int32_t>(deg < INT32_MAX ? deg : INT32_MAX));
        a.bucket[i] = static_cast<uint8_t>(bucket_of(deg, 1, a.tune));
    }
    warp_max(&a.ctrl->max_deg, my_max);
}

__global__ void __launch_bounds__(kBlock) k_rc_validate(RcArgs a) {
    const int w = (blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int nw = (gridDim.x * kBlock) >> 5;
    const int l = lane_id();
    int32_t my_max = 0;
    for (int64_t v = w; v < a.g.n; v += nw) {
        const int32_t cv = a.old_c[v];
        if (cv < 1 || cv > kMaxInputColor) {
            if (l == 0) atomicOr(&a.ctrl->err, kErrImproper);
            continue;
        }
        my_max = max(my_max, cv);
        int64_t beg, end;
        row_range(a.g, static_cast<int32_t>(v), beg, end, &a.ctrl->err);
        bool bad = false;
        for (int64_t e = beg + l; e < end; e += 32) {
            const int32_t u = load_nbr(a.g, e, &a.ctrl->err);
            if (u >= 0 && a.old_c[u] == cv) bad = true;
        }
        if (__any_sync(kFull, bad) && l == 0) atomicOr(&a.ctrl->err, kErrImproper);
    }
    warp_max(&a.ctrl->max_in, my_max);
}

// ---------------------------------------------------------------------------
// Histogram of (class, bucket)
// ---------------------------------------------------------------------------
constexpr int kHistSmem = 8192;

__global__ void __launch_bounds__(kBlock) k_rc_hist(RcArgs a) {
    __shared__ int32_t sh[kHistSmem];
    const int32_t entries = (a.cap + 1) * kNB;
    const bool local = entries <= kHistSmem;
    if (local) {
        for (int i = threadIdx.x; i < entries; i += kBlock) sh[i] = 0;
        __syncthreads();
    }
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < a.g.n; v += stride) {
        const int32_t c = a.old_c[v];
        if (c < 1 || c > a.cap) {
            atomicOr(&a.ctrl->err, kErrImproper);
            continue;
        }
        const int32_t key = c * kNB + a.bucket[v];
        if (local) atomicAdd(&sh[key], 1);
        else atomicAdd(&a.cls_cnt[key], 1);
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < entries; i += kBlock)
            if (sh[i]) atomicAdd(&a.cls_cnt[i], sh[i]);
    }
}

// ---------------------------------------------------------------------------
// Class order (one block of 1024 threads)
// ---------------------------------------------------------------------------
struct OrderShared {
    int32_t wsum[kOrderThreads / 32];
    int32_t carry;
    int32_t shuffle[kShuffleSmem];
};

// Exclusive scan over the block; returns the prefix, writes the total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, OrderShared& s, int32_t& total) {
    const int l = lane_id(), w = threadIdx.x >> 5;
    const int32_t incl = static_cast<int32_t>(warp_inclusive_scan(static_cast<uint32_t>(x)));
    if (l == 31) s.wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int32_t y = s.wsum[l];
        const int32_t yi = static_cast<int32_t>(warp_inclusive_scan(static_cast<uint32_t>(y)));
        s.wsum[l] = yi - y;
        if (l == 31) s.carry = yi;
    }
    __syncthreads();
    const int32_t r = s.wsum[w] + incl - x;
    total = s.carry;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kOrderThreads) k_rc_order(RcArgs a) {
    __shared__ OrderShared s;
    const int t = threadIdx.x;
    // present classes in ascending color, with their sizes
    int32_t k = 0;
    for (int32_t c0 = 1; c0 <= a.cap; c0 += kOrderThreads) {
        const int32_t c = c0 + t;
        int32_t size = 0;
        if (c <= a.cap)
            for (int b = 0; b < kNB; ++b) size += a.cls_cnt[c * kNB + b];
        int32_t total;
        const int32_t pos = block_exclusive_scan(size > 0 ? 1 : 0, s, total);
        if (size > 0) {
            a.present[k + pos] = c;
            a.psize[k + pos] = size;
        }
        k += total;
    }
    __syncthreads();
    if (a.iteration == 0 && t == 0) a.ncolors[0] = k > 0 ? a.present[k - 1] : 0;

    // the permutation (Sec. 3)
    if (a.perm == 0) {  // RV
        for (int32_t i = t; i < k; i += kOrderThreads) a.order[i] = a.present[k - 1 - i];
    } else if (a.perm == 1 || a.perm == 2) {  // NI / ND, ties to the smaller color
        const bool noninc = a.perm == 1;
        for (int32_t i = t; i < k; i += kOrderThreads) {
            const int32_t si = a.psize[i];
            int32_t r = 0;
            for (int32_t j = 0; j < k; ++j) {
                const int32_t sj = a.psize[j];
                const bool before = noninc ? (sj > si || (sj == si && j < i))
                                           : (sj < si || (sj == si && j < i));
                r += before;
            }
            a.order[r] = a.present[i];
        }
    } else {  // RAND: Fisher-Yates from the ascending list, i = k-1 .. 1
        for (int32_t i = t; i < k; i += kOrderThreads) {
            a.jtab[i] = i == 0 ? 0
                               : static_cast<int32_t>(scale_index(perm_word(a.seed, i, a.iteration),
                                                                  static_cast<uint32_t>(i + 1)));
            if (k <= kShuffleSmem) s.shuffle[i] = a.present[i];
            else a.order[i] = a.present[i];
        }
        __syncthreads();
        if (t == 0) {
            int32_t* L = k <= kShuffleSmem ? s.shuffle : a.order;
            for (int32_t i = k - 1; i >= 1; --i) {
                const int32_t j = a.jtab[i];
                const int32_t x = L[i];
                L[i] = L[j];
                L[j] = x;
            }
        }
        __syncthreads();
        if (k <= kShuffleSmem)
            for (int32_t i = t; i < k; i += kOrderThreads) a.order[i] = s.shuffle[i];
    }
    __syncthreads();

    // rank of every present color; segments (class-major, bucket-minor)
    for (int32_t p = t; p < k; p += kOrderThreads) a.rank_of[a.order[p]] = p;
    const int32_t nseg = k * kNB;
    int32_t vbase = 0, tbase = 0;
    for (int32_t s0 = 0; s0 < nseg; s0 += kOrderThreads) {
        const int32_t sg = s0 + t;
        int32_t cnt = 0, tiles = 0;
        if (sg < nseg) {
            const int b = sg % kNB;
            cnt = a.cls_cnt[a.order[sg / kNB] * kNB + b];
            tiles = (cnt + bucket_tile(b) - 1) / bucket_tile(b);
            a.fill[sg] = 0;
        }
        int32_t vt, tt;
        const int32_t vp = block_exclusive_scan(cnt, s, vt);
        const int32_t tp = block_exclusive_scan(tiles, s, tt);
        if (sg < nseg) {
            a.seg_start[sg] = vbase + vp;
            a.tile_prefix[sg] = tbase + tp;
        }
        vbase += vt;
        tbase += tt;
    }
    if (t == 0) {
        a.seg_start[nseg] = vbase;
        a.tile_prefix[nseg] = tbase;
        a.ctrl->k = k;
        a.ctrl->total_tiles = tbase;
        a.ctrl->claim = 0;
    }
}

// ---------------------------------------------------------------------------
// Counting-sort scatter into class-major segments.  Each block takes a
// contiguous slice of vertices, counts its vertices per segment in shared
// memory, reserves its ranges with one global atomic per (block, segment),
// then places the vertices.  (Order inside a segment is free: a class is an
// independent set.)
// ---------------------------------------------------------------------------
constexpr int kScatterSegs = 4096;

__device__ __forceinline__ int32_t segment_of(const RcArgs& a, int32_t v) {
    return a.rank_of[a.old_c[v]] * kNB + a.bucket[v];
}

__device__ __forceinline__ void place(const RcArgs& a, int32_t v, int32_t sg, int32_t pos) {
    int64_t beg;
    int32_t deg;
    row_of(a.g, v, beg, deg, &a.ctrl->err);
    store_item(a.list + pos, beg, v, deg);
    a.new_c[v] = -(sg / kNB + 1);
}

__global__ void __launch_bounds__(kBlock) k_rc_scatter(RcArgs a) {
    __shared__ int32_t s_cnt[kScatterSegs];
    __shared__ int32_t s_base[kScatterSegs];
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    const int32_t nseg = a.ctrl->k * kNB;
    const int64_t chunk = (a.g.n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = a.g.n < lo + chunk ? a.g.n : lo + chunk;
    if (nseg > kScatterSegs) {
        // many classes: warp-aggregated global atomics
        for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
            const int32_t v = static_cast<int32_t>(i);
            const int32_t sg = segment_of(a, v);
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, sg);
            const int leader = __ffs(peers) - 1;
            int32_t base = 0;
            if (lane_id() == leader) base = atomicAdd(&a.fill[sg], __popc(peers));
            base = __shfl_sync(peers, base, leader);
            place(a, v, sg, a.seg_start[sg] + base + __popc(peers & ((1u << lane_id()) - 1u)));
        }
        return;
    }
    for (int i = threadIdx.x; i < nseg; i += kBlock) s_cnt[i] = 0;
    __syncthreads();
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        const int32_t sg = segment_of(a, static_cast<int32_t>(i));
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, sg);
        if (lane_id() == __ffs(peers) - 1) atomicAdd(&s_cnt[sg], __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nseg; i += kBlock) {
        const int32_t c = s_cnt[i];
        if (c) s_base[i] = a.seg_start[i] + atomicAdd(&a.fill[i], c);
        s_cnt[i] = 0;
    }
    __syncthreads();
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        const int32_t v = static_cast<int32_t>(i);
        const int32_t sg = segment_of(a, v);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, sg);
        const int leader = __ffs(peers) - 1;
        int32_t base = 0;
        if (lane_id() == leader) base = atomicAdd(&s_cnt[sg], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        place(a, v, sg, s_base[sg] + base + __popc(peers & ((1u << lane_id()) - 1u)));
    }
}

// ---------------------------------------------------------------------------
// The class steps
// ---------------------------------------------------------------------------
// Color of neighbor u as seen by a vertex of class rank p (< 1 = ignore).
template <bool kDataflow>
struct RecolorFetch {
    int32_t* new_c;
    int32_t p;
    int32_t spin_limit;
    uint32_t* err;
    __device__ __forceinline__ int32_t raw(int32_t u) const {
        return kDataflow ? ld_relaxed(new_c + u) : __ldcg(new_c + u);
    }
    __device__ __forceinline__ int32_t resolve(int32_t u, int32_t x) const {
        if (x > 0) return x;
        if (!kDataflow || -x - 1 >= p) return 0;  // later class: not recolored yet
        // Earlier class, still in flight: bounded wait.  Once any wait of the
        // launch has run out, every other wait gives up at once, so a launch
        // never spends more than about one spin_limit in waits.
        unsigned ns = 32;
        for (int32_t it = 0; it < spin_limit; ++it) {
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            x = ld_relaxed(new_c + u);
            if (x > 0) return x;
            if ((it & 63) == 0 &&
                (ld_relaxed(reinterpret_cast<const int32_t*>(err)) & static_cast<int32_t>(kErrTimeout)))
                return 0;
        }
        atomicOr(err, kErrTimeout);
        return 0;
    }
};

union RcShared {
    BlockScratch blk;
    uint32_t warp_bm[kWarps][kWarpBitmapWords];
};

template <int G, bool kDataflow>
__device__ __forceinline__ void recolor_group_tile(const RcArgs& a, const RecolorFetch<kDataflow>& f,
                                                   int32_t first, int32_t last, int32_t& my_max,
                                                   unsigned long long& edges) {
    const int gi = threadIdx.x / G, gl = threadIdx.x % G;
    const int32_t k = first + gi;
    const bool valid = k < last;
    WorkItem it{0, 0, 0};
    if (valid) it = load_item(a.list + k);
    const int32_t c = choose_reg<G, LanesUnroll<G>::U>(a.g, it.beg, it.deg, gl, 0u, f, &a.ctrl->err);
    if (valid && gl == 0) {
        st_relaxed(a.new_c + it.v, c);
        my_max = max(my_max, c);
        edges += static_cast<unsigned long long>(it.deg);
    }
}

template <bool kDataflow>
__device__ __forceinline__ void recolor_tile(const RcArgs& a, RcShared& sm, int32_t sg,
                                             int32_t seg_first, int32_t seg_last, int32_t tile_in_seg,
                                             int32_t& my_max, unsigned long long& edges) {
    const int32_t p = sg / kNB;
    const int b = sg % kNB;
    const int32_t first = seg_first + tile_in_seg * bucket_tile(b);
    const RecolorFetch<kDataflow> f{a.new_c, p, a.tune.spin_limit, &a.ctrl->err};
    switch (b) {
    case 0: {
        const WorkItem it = load_item(a.list + first);
        const int32_t c = choose_block<4>(a.g, it.beg, it.deg, 0u, f, sm.blk, &a.ctrl->err);
        if (threadIdx.x == 0) {
            st_relaxed(a.new_c + it.v, c);
            my_max = max(my_max, c);
            edges += static_cast<unsigned long long>(it.deg);
        }
        break;
    }
    case 1: {
        const int w = threadIdx.x >> 5;
        const int32_t k = first + w;
        if (k < seg_last) {
            const WorkItem it = load_item(a.list + k);
            const int32_t c = choose_warp<4>(a.g, it.beg, it.deg, 0u, f, sm.warp_bm[w], &a.ctrl->err);
            if (lane_id() == 0) {
                st_relaxed(a.new_c + it.v, c);
                my_max = max(my_max, c);
                edges += static_cast<unsigned long long>(it.deg);
            }
        }
        break;
    }
    case 2: recolor_group_tile<32, kDataflow>(a, f, first, seg_last, my_max, edges); break;
    case 3: recolor_group_tile<16, kDataflow>(a, f, first, seg_last, my_max, edges); break;
    case 4: recolor_group_tile<8, kDataflow>(a, f, first, seg_last, my_max, edges); break;
    default: recolor_group_tile<4, kDataflow>(a, f, first, seg_last, my_max, edges); break;
    }
}

// Segment lookup: the segment table is staged in shared memory when it fits.
constexpr int kSegSmem = 2048;

struct SegTable {
    int32_t tile_prefix[kSegSmem + 1];
    int32_t seg_start[kSegSmem + 1];
};

// Dataflow form: tiles claimed in class order; the next claim is taken while
// the current tile is processed.
__global__ void __launch_bounds__(kBlock) k_rc_recolor_dataflow(RcArgs a) {
    __shared__ RcShared sm;
    __shared__ SegTable st;
    __shared__ int32_t s_tile, s_seg;
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    const int32_t total = a.ctrl->total_tiles;
    const int32_t nseg = a.ctrl->k * kNB;
    const bool staged = nseg <= kSegSmem;
    if (staged) {
        for (int i = threadIdx.x; i <= nseg; i += kBlock) {
            st.tile_prefix[i] = a.tile_prefix[i];
            st.seg_start[i] = a.seg_start[i];
        }
    }
    const int32_t* tp = staged ? st.tile_prefix : a.tile_prefix;
    const int32_t* ss = staged ? st.seg_start : a.seg_start;
    int32_t my_max = 0;
    unsigned long long edges = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctrl->claim, 1);
    __syncthreads();
    for (;;) {
        const int32_t t = s_tile;
        if (t >= total) break;
        int32_t next = 0;
        if (threadIdx.x == 0) {
            next = atomicAdd(&a.ctrl->claim, 1);
            s_seg = find_segment(tp, nseg, t);
        }
        __syncthreads();
        const int32_t sg = s_seg;
        recolor_tile<true>(a, sm, sg, ss[sg], ss[sg + 1], t - tp[sg], my_max, edges);
        __syncthreads();
        if (threadIdx.x == 0) s_tile = next;
        __syncthreads();
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ncolors[a.iteration + 1], my_max);
}

// Stepwise form: one launch per class p over its tiles [t0, t1).
__global__ void __launch_bounds__(kBlock) k_rc_recolor_step(RcArgs a, int32_t p, int32_t t0,
                                                            int32_t t1) {
    __shared__ RcShared sm;
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    int32_t my_max = 0;
    unsigned long long edges = 0;
    const int32_t seg0 = p * kNB;
    for (int32_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        int sg = seg0;
        while (sg + 1 < seg0 + kNB && a.tile_prefix[sg + 1] <= t) ++sg;
        recolor_tile<false>(a, sm, sg, a.seg_start[sg], a.seg_start[sg + 1], t - a.tile_prefix[sg],
                            my_max, edges);
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ncolors[a.iteration + 1], my_max);
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
gc_status recolor_device(const Graph& g, const int32_t* colors_in, int32_t maxc_in, bool trusted,
                         int32_t perm, int32_t iterations, uint64_t seed, int32_t* colors_out,
                         int32_t* ncolors_per_iter, gc_stats* stats, cudaStream_t s) {
    const int64_t n = g.n;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const Tuning tune = current_tuning();
    const int grid = persistent_grid(tune);
    const int vgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, grid)));
    const int grid_rc = resident_grid(k_rc_recolor_dataflow, tune);
    const int grid_step = resident_grid(k_rc_recolor_step, tune);
    const int grid_sc = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((n + kBlock - 1) / kBlock, resident_grid(k_rc_scatter, tune))));
    cudaError_t ce;

    Scratch sc_ctrl, sc_bucket;
    if (!sc_ctrl.alloc(sizeof(RcCtrl), s) || !sc_bucket.alloc(n + 1, s)) return GC_ERR_OOM;
    RcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.tune = tune;
    a.seed = seed;
    a.perm = perm;
    a.old_c = colors_in;
    a.bucket = sc_bucket.as<uint8_t>();
    a.ctrl = sc_ctrl.as<RcCtrl>();
    cudaMemsetAsync(a.ctrl, 0, sizeof(RcCtrl), s);
    RcCtrl h;
    if (n > 0) {
        GC_LAUNCH(KID_RC_BUCKET, s, k_rc_bucket<<<vgrid, kBlock, 0, s>>>(a));
        if (!trusted) GC_LAUNCH(KID_RC_VALIDATE, s, k_rc_validate<<<grid, kBlock, 0, s>>>(a));
    }
    ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    if (h.err & kErrImproper) return GC_ERR_IMPROPER_INPUT;
    if (!trusted) maxc_in = h.max_in;
    if (n == 0) {
        if (ncolors_per_iter)
            for (int32_t i = 0; i <= iterations; ++i) ncolors_per_iter[i] = 0;
        return GC_OK;
    }
    if (iterations == 0) {
        if (colors_out != colors_in)
            cudaMemcpyAsync(colors_out, colors_in, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
        ce = cudaStreamSynchronize(s);
        if (ncolors_per_iter) ncolors_per_iter[0] = maxc_in;
        if (stats) stats->max_color = maxc_in;
        return ce == cudaSuccess ? GC_OK : cuda_status(ce);
    }

    const int32_t cap = std::max(maxc_in, h.max_deg + 1);
    const int64_t ent = static_cast<int64_t>(cap + 1) * kNB;
    Scratch sc_cls, sc_present, sc_psize, sc_order, sc_jtab, sc_rank, sc_seg, sc_tiles, sc_fill,
        sc_list, sc_alt, sc_ncol;
    if (!sc_cls.alloc(ent * 4, s) || !sc_present.alloc((cap + 1) * 4, s) ||
        !sc_psize.alloc((cap + 1) * 4, s) || !sc_order.alloc((cap + 1) * 4, s) ||
        !sc_jtab.alloc((cap + 1) * 4, s) || !sc_rank.alloc((cap + 1) * 4, s) ||
        !sc_seg.alloc((ent + 1) * 4, s) || !sc_tiles.alloc((ent + 1) * 4, s) ||
        !sc_fill.alloc(ent * 4, s) || !sc_list.alloc(n * sizeof(WorkItem), s) ||
        !sc_alt.alloc(n * 4, s) ||
        !sc_ncol.alloc((iterations + 1) * 4, s))
        return GC_ERR_OOM;
    a.cap = cap;
    a.cls_cnt = sc_cls.as<int32_t>();
    a.present = sc_present.as<int32_t>();
    a.psize = sc_psize.as<int32_t>();
    a.order = sc_order.as<int32_t>();
    a.jtab = sc_jtab.as<int32_t>();
    a.rank_of = sc_rank.as<int32_t>();
    a.seg_start = sc_seg.as<int32_t>();
    a.tile_prefix = sc_tiles.as<int32_t>();
    a.fill = sc_fill.as<int32_t>();
    a.list = sc_list.as<WorkItem>();
    a.ncolors = sc_ncol.as<int32_t>();
    cudaMemsetAsync(a.ncolors, 0, (iterations + 1) * 4, s);

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int32_t* alt = sc_alt.as<int32_t>();
    const int32_t* cur = colors_in;
    gc_status st = GC_OK;
    std::vector<int32_t> tp;
    for (int32_t it = 0; it < iterations && st == GC_OK; ++it) {
        int32_t* dst = (it % 2 == 0) ? alt : colors_out;
        a.iteration = it;
        a.old_c = cur;
        a.new_c = dst;
        cudaMemsetAsync(a.cls_cnt, 0, ent * 4, s);
        GC_LAUNCH(KID_RC_HIST, s, k_rc_hist<<<vgrid, kBlock, 0, s>>>(a));
        GC_LAUNCH(KID_RC_ORDER, s, k_rc_order<<<1, kOrderThreads, 0, s>>>(a));
        GC_LAUNCH(KID_RC_SCATTER, s, k_rc_scatter<<<grid_sc, kBlock, 0, s>>>(a));
        if (tune.recolor_mode == 0) {
            GC_LAUNCH(KID_RC_RECOLOR, s, k_rc_recolor_dataflow<<<grid_rc, kBlock, 0, s>>>(a));
        } else {
            RcCtrl hc;
            ce = cudaMemcpyAsync(&hc, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            tp.resize(static_cast<size_t>(hc.k) * kNB + 1);
            ce = cudaMemcpy(tp.data(), a.tile_prefix, tp.size() * 4, cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            for (int32_t p = 0; p < hc.k; ++p) {
                const int32_t t0 = tp[p * kNB], t1 = tp[(p + 1) * kNB];
                if (t1 <= t0) continue;
                const int g2 = std::min(grid_step, t1 - t0);
                GC_LAUNCH(KID_RC_STEP, s, k_rc_recolor_step<<<g2, kBlock, 0, s>>>(a, p, t0, t1));
            }
        }
        cur = dst;
    }
    if (st == GC_OK && cur != colors_out)
        cudaMemcpyAsync(colors_out, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    cudaEventRecord(e1, s);
    std::vector<int32_t> nc(iterations + 1);
    ce = cudaMemcpyAsync(nc.data(), a.ncolors, (iterations + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess && st == GC_OK) st = cuda_status(ce);
    if (st == GC_OK) st = status_from_err_bits(h.err);
    if (ncolors_per_iter) std::copy(nc.begin(), nc.end(), ncolors_per_iter);
    if (stats) {
        stats->iterations = iterations;
        stats->max_color = nc[iterations];
        stats->edges_examined = static_cast<int64_t>(h.edges);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_recolor = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace gc
