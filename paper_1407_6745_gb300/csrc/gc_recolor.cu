// gc_recolor.cu -- iterative recoloring on one GPU.
//
// Culberson's iterated greedy (Sec. 2.1) as synchronous recoloring RC
// (Sec. 3): the classes of the previous coloring are taken one after the
// other in a class permutation (RV, NI, ND or RAND, Sec. 3) and every vertex
// takes the smallest color not used by a neighbor of an earlier class.  A
// class is an independent set, so all its vertices can choose at once and
// the result equals the sequential greedy run in class order (Sec. 3).
//
// One iteration = three launches, with no host round trip:
//   k_rc_hist     histogram of (class, degree bucket) pairs (first iteration
//                 only; later ones get it from the previous recoloring);
//   k_rc_order    the class permutation, computed on the device (one block):
//                 present classes, RV/NI/ND order or a Fisher-Yates shuffle,
//                 rank of every color, segment starts and tile counts;
//   k_rc_scatter  counting sort of the vertices into class-major,
//                 bucket-minor segments; new[v] = -(rank(v) + 1);
//   k_rc_recolor  the class steps, as one cooperative launch: warp tiles are
//                 dealt out statically in class order; a neighbor u of an
//                 earlier class whose new color is not yet written (still
//                 negative) is waited for, with a bounded spin; a neighbor of
//                 a later class (negative, rank above v's) is ignored.  The
//                 alternative form launches one grid per class and needs no
//                 waits.
// The negative encoding makes one 4-byte gather per edge serve both "is u
// earlier than v" and "what color did u take".  Rows longer than
// rc_warp_max_deg are cut into chunks of 256 neighbors handled by different
// warps; the chunks OR their forbidden colors into a per-row bitmap and the
// warp that finishes the last chunk picks the color.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gc_internal.h"

namespace gc {

constexpr int32_t kMaxInputColor = 1 << 28;
constexpr int kOrderThreads = 1024;
constexpr int kShuffleSmem = 4096;
constexpr int32_t kChunk = 256;   // neighbors per chunk of a split (heavy) row (measured best on R-MAT)

// An isolated vertex (no neighbor) takes color 1 in every iteration and no
// vertex waits on it: it gets bucket kIsoBucket, no list entry and no tile;
// the scatter writes its color and it is counted in iso_cnt (class sizes
// only).  (R-MAT 24: 47 % of the vertices; the recoloring kernel went from
// 5.07 to 4.91 ms per iteration.)
constexpr int kIsoBucket = 7;

// Vertices (or, bucket 0, row chunks) per warp tile.
__host__ __device__ constexpr int warp_tile(int b) {
    return b <= 2 ? 1 : b == 3 ? 2 : b == 4 ? 4 : b == 5 ? 8 : 16;
}

struct RcCtrl {
    int32_t k;            // present classes this iteration
    int32_t total_tiles;  // warp tiles this iteration
    int32_t hub_next;     // next free split-row slot
    int32_t max_deg;
    int32_t max_in;       // max input color (validation)
    int32_t n_heavy;      // rows in bucket 0 (split into chunks)
    uint32_t err;
    int32_t hot_sg;       // the largest segment of single-entry vertices (scatter)
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
    int32_t* cls_cnt;     // (cap + 1) * kNB vertices per (class, bucket)
    int32_t* cls_units;   // cap + 1: row chunks of the bucket-0 vertices per class
    int32_t* nxt_cnt;     // the same two histograms of the new colors, filled by
    int32_t* nxt_units;   //   the recoloring kernel for the next iteration
    int32_t* iso_cnt;     // cap + 1 (batch: per (graph, color)): isolated vertices per class
    int32_t* nxt_iso;     // the same of the new colors, filled by the scatter (one graph)
    int32_t* present;     // cap + 1
    int32_t* psize;       // cap + 1
    int32_t* order;       // cap + 1 (class order, colors)
    int32_t* jtab;        // cap + 1 (shuffle indices)
    int32_t* rank_of;     // cap + 1
    int32_t* seg_start;   // (cap + 1) * kNB + 1, in list entries
    int32_t* tile_prefix; // (cap + 1) * kNB + 1, in warp tiles
    int32_t* fill;        // (cap + 1) * kNB
    WorkItem* list;       // list entries in class-major order
    int32_t* ncolors;     // iterations + 1
    int32_t* hub_v;       // split rows: vertex, chunk count, finished chunks,
    int32_t* hub_nch;     //   and a forbidden-color bitmap of hub_words words
    int32_t* hub_done;
    uint32_t* hub_bm;
    int32_t hub_words;
    RcCtrl* ctrl;
    // batches (nullptr for one graph): graph of every vertex, descriptors,
    // and the start of each graph's colors in the (graph, color) tables
    // cls_cnt / cls_units / rank_of / g*
    const int32_t* graph_of;
    const BatchDesc* desc;
    const int64_t* cls_base;
    int32_t ngraphs;
    int32_t fuse_hist;    // 1: the recoloring kernel fills nxt_cnt (one graph only)
    int32_t hist_smem;    // entries of its dynamic shared-memory histogram (0: global)
    int32_t* gpresent;    // per (graph, color): present colors, sizes, order, shuffle
    int32_t* gpsize;
    int32_t* gorder;
    int32_t* gjtab;
    int32_t* seg_cnt;     // list entries per global segment (rank, bucket)
};

__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
    int32_t x;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(x) : "l"(p));
    return x;
}
__device__ __forceinline__ void st_relaxed(int32_t* p, int32_t x) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}
// Adds 1 with acquire-release semantics at GPU scope; returns the old value.
__device__ __forceinline__ int32_t add_acq_rel(int32_t* p) {
    int32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__device__ __forceinline__ int32_t chunks_of(int32_t deg) { return (deg + kChunk - 1) / kChunk; }

// ---------------------------------------------------------------------------
// Per-call set-up: degree buckets (X = 1) and, for untrusted input, the
// proper-coloring check of Sec. 1 plus the max color.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_rc_bucket(RcArgs a) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    int32_t my_max = 0, heavy = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; i < a.g.n; i += stride) {
        int64_t beg;
        int32_t deg;
        row_of(a.g, static_cast<int32_t>(i), beg, deg, &a.ctrl->err);
        my_max = max(my_max, deg);
        const int b = deg == 0 ? kIsoBucket : bucket_of(deg, 1, a.tune);
        a.bucket[i] = static_cast<uint8_t>(b);
        heavy += b == 0;
    }
    warp_max(&a.ctrl->max_deg, my_max);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) heavy += __shfl_xor_sync(kFull, heavy, d);
    if (lane_id() == 0 && heavy) atomicAdd(&a.ctrl->n_heavy, heavy);
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
        int64_t beg;
        int32_t deg;
        row_of(a.g, static_cast<int32_t>(v), beg, deg, &a.ctrl->err);
        bool bad = false;
        for (int32_t k = l; k < deg; k += 32) {
            const int32_t u = load_nbr(a.g, beg + k, &a.ctrl->err);
            if (u >= 0 && a.old_c[u] == cv) bad = true;
        }
        if (__any_sync(kFull, bad) && l == 0) atomicOr(&a.ctrl->err, kErrImproper);
    }
    warp_max(&a.ctrl->max_in, my_max);
}

// Max color of a coloring known to be proper (colors outside [1, max input
// color] still flag it improper).
__global__ void __launch_bounds__(kBlock) k_rc_maxin(RcArgs a) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    int32_t my_max = 0;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < a.g.n; v += stride) {
        const int32_t cv = a.old_c[v];
        if (cv < 1 || cv > kMaxInputColor) atomicOr(&a.ctrl->err, kErrImproper);
        else my_max = max(my_max, cv);
    }
    warp_max(&a.ctrl->max_in, my_max);
}

// ---------------------------------------------------------------------------
// Histogram of (class, bucket); bucket-0 rows also count their chunks
// ---------------------------------------------------------------------------
constexpr int kHistSmem = 8192;

constexpr int kIsoSmem = 1024;  // isolated vertices per class, colors below this counted in shared memory

__global__ void __launch_bounds__(kBlock) k_rc_hist(RcArgs a) {
    __shared__ int32_t sh[kHistSmem];
    __shared__ int32_t s_iso[kIsoSmem];
    const int32_t entries = (a.cap + 1) * kNB;
    const bool local = entries <= kHistSmem;
    for (int i = threadIdx.x; i < kIsoSmem; i += kBlock) s_iso[i] = 0;
    if (local)
        for (int i = threadIdx.x; i < entries; i += kBlock) sh[i] = 0;
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < a.g.n; v += stride) {
        const int32_t c = a.old_c[v];
        if (c < 1 || c > a.cap) {
            atomicOr(&a.ctrl->err, kErrImproper);
            continue;
        }
        const int b = a.bucket[v];
        if (b == kIsoBucket) {
            if (c < kIsoSmem) atomicAdd(&s_iso[c], 1);
            else atomicAdd(&a.iso_cnt[c], 1);
            continue;
        }
        const int32_t key = c * kNB + b;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, key);
        if (lane_id() == __ffs(peers) - 1) {
            if (local) atomicAdd(&sh[key], __popc(peers));
            else atomicAdd(&a.cls_cnt[key], __popc(peers));
        }
        if (b == 0) {
            int64_t beg;
            int32_t deg;
            row_of(a.g, static_cast<int32_t>(v), beg, deg, &a.ctrl->err);
            atomicAdd(&a.cls_units[c], chunks_of(deg));
        }
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < entries; i += kBlock)
            if (sh[i]) atomicAdd(&a.cls_cnt[i], sh[i]);
    for (int i = threadIdx.x; i < kIsoSmem && i <= a.cap; i += kBlock)
        if (s_iso[i]) atomicAdd(&a.iso_cnt[i], s_iso[i]);
}

// ---------------------------------------------------------------------------
// Class order (one block of 1024 threads)
// ---------------------------------------------------------------------------
struct OrderShared {
    int32_t wsum[kOrderThreads / 32];
    int32_t carry;
    unsigned long long best[kOrderThreads / 32];
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

// Segment starts (list entries) and tile prefix (warp tiles) of the k
// ranks x kNB buckets, class-major; units(sg) gives a segment's entries.
template <class Units>
__device__ __forceinline__ void build_segments(const RcArgs& a, int32_t k, OrderShared& s, Units&& units) {
    const int t = threadIdx.x;
    const int32_t nseg = k * kNB;
    int32_t vbase = 0, tbase = 0;
    unsigned long long best = 0;  // (entries << 32) | segment, over the single-entry buckets
    for (int32_t s0 = 0; s0 < nseg; s0 += kOrderThreads) {
        const int32_t sg = s0 + t;
        int32_t cnt = 0, tiles = 0;
        if (sg < nseg) {
            const int b = sg % kNB;
            cnt = units(sg);
            tiles = (cnt + warp_tile(b) - 1) / warp_tile(b);
            a.fill[sg] = 0;
            if (b != 0) {
                const unsigned long long key = (static_cast<unsigned long long>(cnt) << 32) | static_cast<uint32_t>(sg);
                best = key > best ? key : best;
            }
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
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, d);
        best = o > best ? o : best;
    }
    if (lane_id() == 0) s.best[t >> 5] = best;
    __syncthreads();
    if (t == 0) {
        for (int w = 0; w < kOrderThreads / 32; ++w) best = s.best[w] > best ? s.best[w] : best;
        a.seg_start[nseg] = vbase;
        a.tile_prefix[nseg] = tbase;
        a.ctrl->k = k;
        a.ctrl->total_tiles = tbase;
        a.ctrl->hub_next = 0;
        a.ctrl->hot_sg = (best >> 32) ? static_cast<int32_t>(best & 0xffffffffu) : -1;
    }
}

__global__ void __launch_bounds__(kOrderThreads) k_rc_order(RcArgs a) {
    __shared__ OrderShared s;
    const int t = threadIdx.x;
    // present classes in ascending color, with their sizes
    int32_t k = 0;
    for (int32_t c0 = 1; c0 <= a.cap; c0 += kOrderThreads) {
        const int32_t c = c0 + t;
        int32_t size = 0;
        if (c <= a.cap) {
            for (int b = 0; b < kNB; ++b) size += a.cls_cnt[c * kNB + b];
            size += a.iso_cnt[c];
        }
        int32_t total;
        const int32_t pos = block_exclusive_scan(size > 0 ? 1 : 0, s, total);
        if (size > 0) {
            a.present[k + pos] = c;
            a.psize[k + pos] = size;
        }
        k += total;
    }
    __syncthreads();
    if (a.ncolors && a.iteration == 0 && t == 0) a.ncolors[0] = k > 0 ? a.present[k - 1] : 0;

    // the permutation (Sec. 3) of this iteration (Sec. 4.2.1 schedules)
    const int32_t perm = perm_at(a.perm, a.iteration);
    if (perm == 0) {  // RV
        for (int32_t i = t; i < k; i += kOrderThreads) a.order[i] = a.present[k - 1 - i];
    } else if (perm == 1 || perm == 2) {  // NI / ND, ties to the smaller color
        const bool noninc = perm == 1;
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

    // rank of every present color; segments (class-major, bucket-minor) in
    // list entries and in warp tiles
    for (int32_t p = t; p < k; p += kOrderThreads) a.rank_of[a.order[p]] = p;
    build_segments(a, k, s, [&](int32_t sg) {
        const int b = sg % kNB;
        const int32_t c = a.order[sg / kNB];
        return b == 0 ? a.cls_units[c] : a.cls_cnt[c * kNB + b];
    });
}

// ---------------------------------------------------------------------------
// Counting-sort scatter into class-major segments.  Each block takes a
// contiguous slice of vertices, counts its list entries per segment in
// shared memory, reserves its ranges with one global atomic per (block,
// segment), then places them.  A bucket-0 row takes one entry per chunk and
// a split-row slot.  (Order inside a segment is free: a class is an
// independent set.)
// ---------------------------------------------------------------------------
constexpr int kScatterSegs = 4096;

struct ScatterInfo {
    int32_t sg;
    int32_t units;
    int64_t beg;
    int32_t deg;
};

__device__ __forceinline__ ScatterInfo scatter_info(const RcArgs& a, int32_t v) {
    ScatterInfo si;
    const int b = a.bucket[v];
    int64_t key = a.old_c[v];
    if (a.graph_of) {  // batch: the graph's own class ranks; a finished graph keeps its colors
        const int32_t gi = a.graph_of[v];
        if (a.iteration >= a.desc[gi].iterations) {
            si.sg = -1;
            si.units = 0;
            si.beg = 0;
            si.deg = 0;
            return si;
        }
        key += a.cls_base[gi];
    }
    if (b == kIsoBucket) {  // color 1, no list entry
        si.sg = -2;
        si.units = 0;
        si.beg = 0;
        si.deg = 0;
        return si;
    }
    si.sg = a.rank_of[key] * kNB + b;
    row_of(a.g, v, si.beg, si.deg, &a.ctrl->err);
    si.units = b == 0 ? chunks_of(si.deg) : 1;
    return si;
}

// A vertex without a list entry: a finished graph's (sg -1) keeps its color,
// an isolated one (sg -2) takes color 1 and is counted in `iso`.
__device__ __forceinline__ void place_unlisted(const RcArgs& a, int32_t v, int32_t sg, int32_t& iso) {
    if (sg == -2) {
        a.new_c[v] = 1;
        ++iso;
    } else {
        a.new_c[v] = a.old_c[v];
    }
}

// The isolated vertices placed by a block: counted in the next iteration's
// class 1 (one graph), and the iteration's max color is at least 1.
__device__ __forceinline__ void flush_isolated(const RcArgs& a, int32_t iso) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) iso += __shfl_xor_sync(kFull, iso, d);
    if (lane_id() == 0 && iso > 0) {
        if (a.nxt_iso) atomicAdd(&a.nxt_iso[1], iso);
        if (a.ncolors) atomicMax(&a.ncolors[a.iteration + 1], 1);
    }
}

__device__ __forceinline__ void place(const RcArgs& a, int32_t v, const ScatterInfo& si, int32_t pos) {
    a.new_c[v] = -(si.sg / kNB + 1);
    if (si.sg % kNB != 0) {
        store_item(a.list + pos, si.beg, v, si.deg);
        return;
    }
    const int32_t slot = atomicAdd(&a.ctrl->hub_next, 1);
    a.hub_v[slot] = v;
    a.hub_nch[slot] = si.units;
    a.hub_done[slot] = 0;
    for (int32_t w = 0; w < a.hub_words; ++w) a.hub_bm[static_cast<int64_t>(slot) * a.hub_words + w] = 0u;
    for (int32_t c = 0; c < si.units; ++c) {
        const int32_t len = min(kChunk, si.deg - c * kChunk);
        store_item(a.list + pos + c, si.beg + static_cast<int64_t>(c) * kChunk, -(slot + 1), len);
    }
}

// Reserve `units` entries of segment sg from a counter (warp-aggregated
// when all peers reserve one entry).
__device__ __forceinline__ int32_t reserve(int32_t* counter_base, const ScatterInfo& si) {
    if (si.units != 1) return atomicAdd(&counter_base[si.sg], si.units);
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, si.sg);
    const int leader = __ffs(peers) - 1;
    int32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(&counter_base[si.sg], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane_id()) - 1u));
}

// Reserve `units` entries of s_cnt[sg]: the active lanes whose segment is
// `hot` share one atomic (ballot, not a match), the others take their own.
__device__ __forceinline__ int32_t hot_or_own(int32_t* s_cnt, int32_t sg, int32_t units, int32_t hot) {
    const unsigned act = __activemask();
    const bool is_hot = sg == hot && units == 1;
    const unsigned hm = __ballot_sync(act, is_hot);
    if (!is_hot) return atomicAdd(&s_cnt[sg], units);
    const int l = lane_id();
    const int leader = __ffs(hm) - 1;
    int32_t base = 0;
    if (l == leader) base = atomicAdd(&s_cnt[sg], __popc(hm));
    base = __shfl_sync(hm, base, leader);
    return base + __popc(hm & ((1u << l) - 1u));
}

__global__ void __launch_bounds__(kBlock) k_rc_scatter(RcArgs a) {
    __shared__ int32_t s_cnt[kScatterSegs];
    __shared__ int32_t s_base[kScatterSegs];
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    const int32_t nseg = a.ctrl->k * kNB;
    const int64_t chunk = (static_cast<int64_t>(a.g.n) + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = a.g.n < lo + chunk ? a.g.n : lo + chunk;
    if (nseg > kScatterSegs) {
        // many classes: global atomics
        int32_t iso = 0;
        for (int64_t i0 = lo; i0 < hi; i0 += kBlock) {  // whole warps: flush_isolated shuffles
            const int64_t i = i0 + threadIdx.x;
            if (i >= hi) continue;
            const int32_t v = static_cast<int32_t>(i);
            const ScatterInfo si = scatter_info(a, v);
            if (si.sg < 0) {
                place_unlisted(a, v, si.sg, iso);
                continue;
            }
            const int32_t off = reserve(a.fill, si);
            place(a, v, si, a.seg_start[si.sg] + off);
        }
        flush_isolated(a, iso);
        return;
    }
    for (int i = threadIdx.x; i < nseg; i += kBlock) s_cnt[i] = 0;
    const int32_t hot = a.ctrl->hot_sg;
    __syncthreads();
    // count: the segment and, for a split row, its chunk count (no row read
    // for the others); shared-memory atomics, positions inside a segment are
    // free (a class is an independent set).  The lanes of a warp that fall
    // into the largest segment (on a skewed graph most vertices do) take
    // their entries with one atomic.
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        const int32_t v = static_cast<int32_t>(i);
        const int b = a.bucket[v];
        if (b == kIsoBucket) continue;
        int64_t key = a.old_c[v];
        if (a.graph_of) {
            const int32_t gi = a.graph_of[v];
            if (a.iteration >= a.desc[gi].iterations) continue;
            key += a.cls_base[gi];
        }
        const int32_t sg = a.rank_of[key] * kNB + b;
        int32_t units = 1;
        if (b == 0) {
            int64_t beg;
            int32_t deg;
            row_of(a.g, v, beg, deg, &a.ctrl->err);
            units = chunks_of(deg);
        }
        hot_or_own(s_cnt, sg, units, hot);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nseg; i += kBlock) {
        const int32_t c = s_cnt[i];
        if (c) s_base[i] = a.seg_start[i] + atomicAdd(&a.fill[i], c);
        s_cnt[i] = 0;
    }
    __syncthreads();
    int32_t iso = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        const int32_t v = static_cast<int32_t>(i);
        const ScatterInfo si = scatter_info(a, v);
        if (si.sg < 0) {
            place_unlisted(a, v, si.sg, iso);
            continue;
        }
        const int32_t off = hot_or_own(s_cnt, si.sg, si.units, hot);
        place(a, v, si, s_base[si.sg] + off);
    }
    flush_isolated(a, iso);
}

// ---------------------------------------------------------------------------
// The class steps
// ---------------------------------------------------------------------------
// Color of neighbor u as seen by a vertex of class rank p (< 1 = ignore).
//
// In the dataflow form an entry of new_c changes once in the launch, from
// -(rank + 1) to the final color, so a stale copy can only be the negative
// placeholder.  On graphs with split (hub) rows the first read is an
// L1-cached weak load: millions of light rows read the same few hub colors,
// which as GPU-scope loads all queue at the few L2 lines holding them
// (R-MAT scale 24: 6.14 -> 5.17 ms per iteration).  A positive value read
// that way is final; a negative one of an earlier class is read again from
// L2 (relaxed) while waiting.  Without hub rows the gathers are scattered
// and gain nothing from L1 (the shuffled stencil: 0.325 -> 0.335 ms), so they
// stay GPU-scope loads.
__device__ __forceinline__ int32_t ld_weak_l1(const int32_t* p) {
    int32_t x;
    asm volatile("ld.global.ca.s32 %0, [%1];" : "=r"(x) : "l"(p));
    return x;
}

template <bool kDataflow>
struct RecolorFetch {
    int32_t* new_c;
    int32_t p;
    int32_t spin_limit;
    uint32_t* err;
    bool cached;  // first read through L1 (dataflow form, graphs with hub rows)
    __device__ __forceinline__ int32_t raw(int32_t u) const {
        if (!kDataflow) return __ldcg(new_c + u);
        return cached ? ld_weak_l1(new_c + u) : ld_relaxed(new_c + u);
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
            if (ns < 256) ns <<= 1;
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

// Histogram of the new colors for the next iteration: counts in dynamic
// shared memory sized to the colors (up to 1023 colors), flushed once per
// block; beyond that, global counts, where the lanes of a warp that add to
// the same (color, bucket) are merged into one atomic (most vertices of a
// skewed graph take the same few colors, and unmerged adds to one global
// counter serialise in L2).
constexpr int kRcHistSmem = 6144;

struct NextHist {
    int32_t* sh;     // nullptr: count in global memory
    int32_t* glob;
    int32_t* units;
    int32_t cap;
    __device__ __forceinline__ void add(int32_t c, int b, int32_t chunks) const {
        if (c < 1 || c > cap) return;
        const int32_t key = c * kNB + b;
        if (sh) {
            atomicAdd(&sh[key], 1);
        } else {
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, key);
            if (lane_id() == __ffs(peers) - 1) atomicAdd(&glob[key], __popc(peers));
        }
        if (b == 0) atomicAdd(&units[c], chunks);
    }
};

template <int G, bool kDataflow>
__device__ __forceinline__ void recolor_group_tile(const RcArgs& a, const RecolorFetch<kDataflow>& f,
                                                   const NextHist& nh, int b, int32_t first,
                                                   int32_t last, int32_t& my_max,
                                                   unsigned long long& edges) {
    const int gi = lane_id() / G, gl = lane_id() % G;
    const int32_t k = first + gi;
    const bool valid = k < last;
    WorkItem it{0, 0, 0};
    if (valid) it = load_item(a.list + k);
    const int32_t c = choose_reg<G, LanesUnroll<G>::U>(a.g, it.beg, it.deg, gl, 0u, f, &a.ctrl->err);
    if (valid && gl == 0) {
        st_relaxed(a.new_c + it.v, c);
        my_max = max(my_max, c);
        edges += static_cast<unsigned long long>(it.deg);
        nh.add(c, b, 0);
    }
}

// One chunk of a split row: the chunk's forbidden colors are OR-ed into the
// row's bitmap; the warp finishing the last chunk picks the First-Fit color.
//
// Ordering: the lanes' OR-s into the row's bitmap precede a warp barrier,
// and lane 0 then counts the chunk with one acquire-release atomic.  Its
// release covers the warp's OR-s (the barrier orders them before it); the
// last chunk's acquire reads the end of the counter's chain of increments,
// so it sees every chunk's OR-s, and the barrier after it orders the lanes'
// bitmap reads after it.  (One atomic by one lane instead of a fence by all
// 32: R-MAT 24 4.86 -> 4.37 ms per iteration, RXF-4 5.17 -> 4.62 ms.)
template <bool kDataflow>
__device__ __forceinline__ void recolor_chunk(const RcArgs& a, const RecolorFetch<kDataflow>& f,
                                              const NextHist& nh, const WorkItem& it, uint32_t* bm,
                                              int32_t& my_max, unsigned long long& edges) {
    const int l = lane_id();
    const int32_t slot = -it.v - 1;
    uint32_t* hb = a.hub_bm + static_cast<int64_t>(slot) * a.hub_words;
    // written by the scatter (an earlier launch): read-only here, loaded early
    const int32_t nch = l == 0 ? __ldg(a.hub_nch + slot) : 0;
    const int32_t hv = l == 0 ? __ldg(a.hub_v + slot) : 0;
    static_assert(kWarpBitmapWords == 64, "two bitmap words per lane");
    for (int32_t w0 = 0; w0 < a.hub_words; w0 += kWarpBitmapWords) {
        // The row's bits already merged (read before the scan, in the shadow
        // of its loads): a word adding no new bit is not merged again.  Bits
        // are only ever set during the launch, so skipping is exact; the
        // chunks of one row otherwise all send atomics to the same few words
        // (R-MAT 24: 4.91 -> 4.84 ms per iteration).
        const uint32_t have0 = w0 + l < a.hub_words ? __ldcg(hb + w0 + l) : 0u;
        const uint32_t have1 = w0 + l + 32 < a.hub_words ? __ldcg(hb + w0 + l + 32) : 0u;
        bm[l] = 0u;
        bm[l + 32] = 0u;
        __syncwarp();
        const int32_t base = w0 * 32 + 1;
        scan_row<2>(a.g, it.beg, it.deg, l, 32, f,
                    [&](int32_t c) {
                        const uint32_t d = static_cast<uint32_t>(c - base);
                        if (c > 0 && d < 32u * kWarpBitmapWords) atomicOr(&bm[d >> 5], 1u << (d & 31));
                    },
                    &a.ctrl->err);
        __syncwarp();
        if (w0 + l < a.hub_words && (bm[l] & ~have0)) atomicOr(&hb[w0 + l], bm[l]);
        if (w0 + l + 32 < a.hub_words && (bm[l + 32] & ~have1)) atomicOr(&hb[w0 + l + 32], bm[l + 32]);
        __syncwarp();
    }
    if (l == 0) edges += static_cast<unsigned long long>(it.deg);
    __syncwarp();
    int last = 0;
    if (l == 0) last = add_acq_rel(a.hub_done + slot) == nch - 1;
    last = __shfl_sync(kFull, last, 0);
    __syncwarp();
    if (!last) return;
    // First Fit over the merged bitmap: the first clear bit
    for (int32_t w0 = 0; w0 < a.hub_words; w0 += 32) {
        const int32_t i = w0 + l;
        const uint32_t free_bits = i < a.hub_words ? ~__ldcg(hb + i) : 0u;
        const uint32_t any = __ballot_sync(kFull, free_bits != 0u);
        if (any) {
            const int src = __ffs(any) - 1;
            const uint32_t fw = __shfl_sync(kFull, free_bits, src);
            const int32_t c = (w0 + src) * 32 + __ffs(fw);
            if (l == 0) {
                st_relaxed(a.new_c + hv, c);
                my_max = max(my_max, c);
                nh.add(c, 0, nch);
            }
            return;
        }
    }
}

template <bool kDataflow>
__device__ __forceinline__ void recolor_warp_tile(const RcArgs& a, const NextHist& nh, uint32_t* bm,
                                                  int32_t sg, int32_t seg_first, int32_t seg_last,
                                                  int32_t tile_in_seg, bool cached, int32_t& my_max,
                                                  unsigned long long& edges) {
    const int32_t p = sg / kNB;
    const int b = sg % kNB;
    const int32_t first = seg_first + tile_in_seg * warp_tile(b);
    const RecolorFetch<kDataflow> f{a.new_c, p, a.tune.spin_limit, &a.ctrl->err, cached};
    switch (b) {
    case 0: recolor_chunk<kDataflow>(a, f, nh, load_item(a.list + first), bm, my_max, edges); break;
    case 1: {
        const WorkItem it = load_item(a.list + first);
        const int32_t c = choose_warp<4>(a.g, it.beg, it.deg, 0u, f, bm, &a.ctrl->err);
        if (lane_id() == 0) {
            st_relaxed(a.new_c + it.v, c);
            my_max = max(my_max, c);
            edges += static_cast<unsigned long long>(it.deg);
            nh.add(c, 1, 0);
        }
        break;
    }
    case 2: recolor_group_tile<32, kDataflow>(a, f, nh, 2, first, seg_last, my_max, edges); break;
    case 3: recolor_group_tile<16, kDataflow>(a, f, nh, 3, first, seg_last, my_max, edges); break;
    case 4: recolor_group_tile<8, kDataflow>(a, f, nh, 4, first, seg_last, my_max, edges); break;
    case 5: recolor_group_tile<4, kDataflow>(a, f, nh, 5, first, seg_last, my_max, edges); break;
    default: recolor_group_tile<2, kDataflow>(a, f, nh, 6, first, seg_last, my_max, edges); break;
    }
}

// Segment table in shared memory when it fits.
constexpr int kSegSmem = 1024;

// Blocks of the dataflow launch: about one per 400 adjacency entries per
// color class, at least 16, at most all that fit.  An iteration is bound by
// its class chain when the classes are small (each class waits for the ones
// before it, and more warps only add pollers) and by throughput when they
// are large.  Measured on GB300, per iteration: G(10^4, 16) 86 -> 50 us,
// R-MAT 16 746 -> 537 us, R-MAT 18 1.12 -> 0.85 ms, R-MAT 20 1.64 -> 1.45
// ms, 27-point stencil 64^3 133 -> 102 us; R-MAT 22 and 24 and the stencil
// 128^3 keep the full grid.
inline int coop_grid(int64_t nnz, int32_t classes, int capacity) {
    const int64_t want = nnz / (400 * static_cast<int64_t>(std::max(classes, 1)));
    return static_cast<int>(std::max<int64_t>(std::min<int64_t>(16, capacity), std::min<int64_t>(want, capacity)));
}

// Dataflow form, cooperative launch (every block resident): warp w takes the
// warp tiles w, w + W, w + 2W, ... in class order, W = all warps of the
// grid.  A tile waits only on tiles before it, and the owner of the first
// unfinished tile has finished all its earlier tiles, so it is working on
// that tile: the waits always end.
__device__ __forceinline__ NextHist setup_next_hist(const RcArgs& a, int32_t* s_hist) {
    if (!a.fuse_hist) return NextHist{nullptr, nullptr, nullptr, 0};  // cap 0: add() is a no-op
    const bool local = a.hist_smem > 0;  // (cap + 1) * kNB entries of dynamic shared memory
    if (local)
        for (int i = threadIdx.x; i < a.hist_smem; i += kBlock) s_hist[i] = 0;
    return NextHist{local ? s_hist : nullptr, a.nxt_cnt, a.nxt_units, a.cap};
}

__device__ __forceinline__ void flush_next_hist(const RcArgs& a, const NextHist& nh) {
    if (!nh.sh) return;
    __syncthreads();
    const int32_t entries = (a.cap + 1) * kNB;
    for (int i = threadIdx.x; i < entries; i += kBlock)
        if (nh.sh[i]) atomicAdd(&a.nxt_cnt[i], nh.sh[i]);
}

__global__ void __launch_bounds__(kBlock, 5) k_rc_recolor_coop(RcArgs a) {
    __shared__ uint32_t s_bm[kWarps][kWarpBitmapWords];
    __shared__ int32_t s_tp[kSegSmem + 1], s_ss[kSegSmem + 1];
    extern __shared__ int32_t s_hist[];
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    const int32_t total = a.ctrl->total_tiles;
    const int32_t nseg = a.ctrl->k * kNB;
    const bool staged = nseg <= kSegSmem;
    if (staged) {
        for (int i = threadIdx.x; i <= nseg; i += kBlock) {
            s_tp[i] = a.tile_prefix[i];
            s_ss[i] = a.seg_start[i];
        }
    }
    const NextHist nh = setup_next_hist(a, s_hist);
    __syncthreads();
    const int32_t* tp = staged ? s_tp : a.tile_prefix;
    const int32_t* ss = staged ? s_ss : a.seg_start;
    const int warp = threadIdx.x >> 5;
    const int32_t W = gridDim.x * kWarps;
    const bool cached = a.ctrl->n_heavy > 0;
    int32_t my_max = 0;
    unsigned long long edges = 0;
    int32_t sg = 0;
    for (int32_t t = blockIdx.x * kWarps + warp; t < total; t += W) {
        if (tp[sg + 1] <= t) sg = find_segment(tp, nseg, t);
        recolor_warp_tile<true>(a, nh, s_bm[warp], sg, ss[sg], ss[sg + 1], t - tp[sg], cached, my_max,
                                edges);
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ncolors[a.iteration + 1], my_max);
    flush_next_hist(a, nh);
}

// Stepwise form: one launch per class p over its warp tiles [t0, t1).
__global__ void __launch_bounds__(kBlock, 5) k_rc_recolor_step(RcArgs a, int32_t p, int32_t t0,
                                                               int32_t t1) {
    __shared__ uint32_t s_bm[kWarps][kWarpBitmapWords];
    extern __shared__ int32_t s_hist[];
    if (a.ctrl->err & (kErrImproper | kErrBadGraph)) return;
    const NextHist nh = setup_next_hist(a, s_hist);
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    int32_t my_max = 0;
    unsigned long long edges = 0;
    const int32_t seg0 = p * kNB;
    for (int32_t t = t0 + blockIdx.x * kWarps + warp; t < t1; t += gridDim.x * kWarps) {
        int sg = seg0;
        while (sg + 1 < seg0 + kNB && a.tile_prefix[sg + 1] <= t) ++sg;
        recolor_warp_tile<false>(a, nh, s_bm[warp], sg, a.seg_start[sg], a.seg_start[sg + 1],
                                 t - a.tile_prefix[sg], false, my_max, edges);
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ncolors[a.iteration + 1], my_max);
    flush_next_hist(a, nh);
}

// ---------------------------------------------------------------------------
// Class ranks of a coloring (for aRC): the histogram and permutation kernels
// of one iteration, without the scatter and the class steps.
// ---------------------------------------------------------------------------
gc_status class_ranks_device(const Graph& g, const int32_t* colors, bool trusted, int32_t perm,
                             int32_t iteration, uint64_t seed, int32_t* rank_out, int32_t* maxc_out,
                             cudaStream_t s) {
    const int64_t n = g.n;
    *maxc_out = 0;
    if (n == 0) return GC_OK;
    const Tuning tune = recolor_tuning(current_tuning());
    const int grid = persistent_grid(tune);
    const int vgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, grid)));
    Scratch sc_ctrl, sc_bucket;
    if (!sc_ctrl.alloc(sizeof(RcCtrl), s) || !sc_bucket.alloc(n + 1, s)) return GC_ERR_OOM;
    RcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.tune = tune;
    a.seed = seed;
    a.perm = perm;
    a.iteration = iteration;
    a.old_c = colors;
    a.bucket = sc_bucket.as<uint8_t>();
    a.ctrl = sc_ctrl.as<RcCtrl>();
    cudaMemsetAsync(a.ctrl, 0, sizeof(RcCtrl), s);
    GC_LAUNCH(KID_RC_BUCKET, s, k_rc_bucket<<<vgrid, kBlock, 0, s>>>(a));
    if (!trusted) GC_LAUNCH(KID_RC_VALIDATE, s, k_rc_validate<<<grid, kBlock, 0, s>>>(a));
    else GC_LAUNCH(KID_RC_VALIDATE, s, k_rc_maxin<<<vgrid, kBlock, 0, s>>>(a));
    RcCtrl h;
    cudaError_t ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    if (h.err & kErrImproper) return GC_ERR_IMPROPER_INPUT;
    *maxc_out = h.max_in;
    if (!rank_out) return GC_OK;
    const int32_t cap = std::max(h.max_in, 1);
    const int64_t ent = static_cast<int64_t>(cap + 1) * kNB;
    Scratch sc_cls, sc_units, sc_present, sc_psize, sc_order, sc_jtab, sc_seg, sc_tiles, sc_fill, sc_iso;
    if (!sc_cls.alloc(ent * 4, s) || !sc_units.alloc((cap + 1) * 4, s) || !sc_iso.alloc((cap + 1) * 4, s) ||
        !sc_present.alloc((cap + 1) * 4, s) || !sc_psize.alloc((cap + 1) * 4, s) ||
        !sc_order.alloc((cap + 1) * 4, s) || !sc_jtab.alloc((cap + 1) * 4, s) ||
        !sc_seg.alloc((ent + 1) * 4, s) || !sc_tiles.alloc((ent + 1) * 4, s) || !sc_fill.alloc(ent * 4, s))
        return GC_ERR_OOM;
    a.cap = cap;
    a.cls_cnt = sc_cls.as<int32_t>();
    a.cls_units = sc_units.as<int32_t>();
    a.present = sc_present.as<int32_t>();
    a.psize = sc_psize.as<int32_t>();
    a.order = sc_order.as<int32_t>();
    a.jtab = sc_jtab.as<int32_t>();
    a.rank_of = rank_out;
    a.seg_start = sc_seg.as<int32_t>();
    a.tile_prefix = sc_tiles.as<int32_t>();
    a.fill = sc_fill.as<int32_t>();
    a.iso_cnt = sc_iso.as<int32_t>();
    cudaMemsetAsync(a.cls_cnt, 0, ent * 4, s);
    cudaMemsetAsync(a.cls_units, 0, (cap + 1) * 4, s);
    cudaMemsetAsync(a.iso_cnt, 0, (cap + 1) * 4, s);
    cudaMemsetAsync(rank_out, 0, (cap + 1) * 4, s);
    GC_LAUNCH(KID_RC_HIST, s, k_rc_hist<<<vgrid, kBlock, 0, s>>>(a));
    GC_LAUNCH(KID_RC_ORDER, s, k_rc_order<<<1, kOrderThreads, 0, s>>>(a));
    ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    return status_from_err_bits(h.err);
}

// ---------------------------------------------------------------------------
// Batches: per-graph class histograms and orders, global (rank, bucket)
// segments.  A vertex waits only on neighbors of its own graph of a smaller
// rank, and ranks are global segment keys, so the cooperative launch above
// serves the whole batch unchanged.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_brc_hist(RcArgs a) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < a.g.n; v += stride) {
        const int32_t gi = a.graph_of[v];
        if (a.iteration >= a.desc[gi].iterations) continue;
        const int64_t base = a.cls_base[gi];
        const int32_t maxc = static_cast<int32_t>(a.cls_base[gi + 1] - base - 1);
        const int32_t c = a.old_c[v];
        if (c < 1 || c > maxc) {
            atomicOr(&a.ctrl->err, kErrImproper);
            continue;
        }
        const int b = a.bucket[v];
        const int64_t key = base + c;
        if (b == kIsoBucket) {
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, static_cast<uint32_t>(key));
            if (lane_id() == __ffs(peers) - 1) atomicAdd(&a.iso_cnt[key], __popc(peers));
            continue;
        }
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, static_cast<uint32_t>(key * kNB + b));
        if (lane_id() == __ffs(peers) - 1) atomicAdd(&a.cls_cnt[key * kNB + b], __popc(peers));
        if (b == 0) {
            int64_t rb;
            int32_t deg;
            row_of(a.g, static_cast<int32_t>(v), rb, deg, &a.ctrl->err);
            atomicAdd(&a.cls_units[key], chunks_of(deg));
        }
    }
}

// One warp per graph: present classes, the graph's permutation (the rules of
// k_rc_order), the rank of each color, and the global segment counts.
__global__ void __launch_bounds__(kBlock) k_brc_order(RcArgs a) {
    const int l = lane_id();
    const int32_t warps = gridDim.x * kWarps;
    for (int32_t gi = blockIdx.x * kWarps + (threadIdx.x >> 5); gi < a.ngraphs; gi += warps) {
        const BatchDesc d = a.desc[gi];
        if (a.iteration >= d.iterations) continue;
        const int64_t base = a.cls_base[gi];
        const int32_t maxc = static_cast<int32_t>(a.cls_base[gi + 1] - base - 1);
        int32_t* present = a.gpresent + base;
        int32_t* psize = a.gpsize + base;
        int32_t* order = a.gorder + base;
        int32_t k = 0;
        for (int32_t c0 = 1; c0 <= maxc; c0 += 32) {
            const int32_t c = c0 + l;
            int32_t size = 0;
            if (c <= maxc) {
                for (int b = 0; b < kNB; ++b) size += a.cls_cnt[(base + c) * kNB + b];
                size += a.iso_cnt[base + c];
            }
            const uint32_t bal = __ballot_sync(kFull, size > 0);
            if (size > 0) {
                const int32_t pos = k + __popc(bal & ((1u << l) - 1u));
                present[pos] = c;
                psize[pos] = size;
            }
            k += __popc(bal);
        }
        __syncwarp();
        const int32_t perm = perm_at(d.perm, a.iteration);
        if (perm == 0) {
            for (int32_t i = l; i < k; i += 32) order[i] = present[k - 1 - i];
        } else if (perm == 1 || perm == 2) {
            const bool noninc = perm == 1;
            for (int32_t i = l; i < k; i += 32) {
                const int32_t si = psize[i];
                int32_t r = 0;
                for (int32_t j = 0; j < k; ++j) {
                    const int32_t sj = psize[j];
                    r += noninc ? (sj > si || (sj == si && j < i)) : (sj < si || (sj == si && j < i));
                }
                order[r] = present[i];
            }
        } else {
            int32_t* jtab = a.gjtab + base;
            for (int32_t i = l; i < k; i += 32) {
                jtab[i] = i == 0 ? 0
                                 : static_cast<int32_t>(scale_index(perm_word(d.perm_seed, i, a.iteration),
                                                                    static_cast<uint32_t>(i + 1)));
                order[i] = present[i];
            }
            __syncwarp();
            if (l == 0)
                for (int32_t i = k - 1; i >= 1; --i) {
                    const int32_t j = jtab[i];
                    const int32_t x = order[i];
                    order[i] = order[j];
                    order[j] = x;
                }
        }
        __syncwarp();
        for (int32_t p = l; p < k; p += 32) {
            const int32_t c = order[p];
            a.rank_of[base + c] = p;
            for (int b = 0; b < kNB; ++b) {
                const int32_t u = b == 0 ? a.cls_units[base + c] : a.cls_cnt[(base + c) * kNB + b];
                if (u) atomicAdd(&a.seg_cnt[p * kNB + b], u);
            }
        }
        if (l == 0) atomicMax(&a.ctrl->k, k);
    }
}

__global__ void __launch_bounds__(kOrderThreads) k_brc_segments(RcArgs a) {
    __shared__ OrderShared s;
    const int32_t k = a.ctrl->k;
    build_segments(a, k, s, [&](int32_t sg) { return a.seg_cnt[sg]; });
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
gc_status recolor_device(const Graph& g, const int32_t* colors_in, int32_t maxc_in, bool trusted,
                         int32_t perm, int32_t iterations, uint64_t seed, int32_t* colors_out,
                         int32_t* ncolors_per_iter, gc_stats* stats, cudaStream_t s) {
    const int64_t n = g.n;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const Tuning tune = recolor_tuning(current_tuning());
    const int grid = persistent_grid(tune);
    const int vgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, grid)));
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
    // A launch that gets fewer blocks than fit is bound by its class chain
    // (coop_grid); there a row of 9 to 16 entries takes 4 lanes (one batch of
    // loads) instead of 2 (two batches), unless the caller set the 2-lane
    // threshold.  Per iteration, G(10^4, 16): 86 -> 51 us; a large graph is
    // bound by tile throughput and keeps 2 lanes (RMAT-ER at scale 24 went
    // 2.08 -> 3.09 ms with 4).
    const bool g2_default = current_tuning().rc_g2_max_deg == kDefaultRcG2MaxDeg;
    const int coop_fit = sm_count() * occupancy_of(reinterpret_cast<const void*>(k_rc_recolor_coop), kBlock);
    auto chain_bound = [&](int32_t maxc) {
        return g2_default && coop_grid(g.nnz, std::max(maxc, 1), coop_fit) < coop_fit;
    };
    if (trusted && chain_bound(maxc_in)) a.tune.g2_max_deg = std::min(kChainRcG2MaxDeg, a.tune.g4_max_deg);
    RcCtrl h;
    std::memset(&h, 0, sizeof(h));
    if (n > 0) {
        GC_LAUNCH(KID_RC_BUCKET, s, k_rc_bucket<<<vgrid, kBlock, 0, s>>>(a));
        if (!trusted) GC_LAUNCH(KID_RC_VALIDATE, s, k_rc_validate<<<grid, kBlock, 0, s>>>(a));
    }
    // A trusted input (our own coloring) has a known max color; the split
    // rows are then sized by a bound (a bucket-0 row has more than
    // max(rc_warp_max_deg, 63) entries) instead of a read-back, when the
    // bound's scratch is small.
    const int64_t heavy_min = std::max<int64_t>(tune.warp_max_deg, 63) + 1;
    const int64_t heavy_bound = std::min<int64_t>(n, static_cast<int64_t>(g.nnz) / heavy_min);
    const int64_t bound_words = (static_cast<int64_t>(std::max(maxc_in, 1)) + 1 + 31) / 32;
    const bool read_back = !trusted || n == 0 || heavy_bound * bound_words * 4 > (int64_t(64) << 20);
    if (read_back) {
        ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_status(ce);
        if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
        if (h.err & kErrImproper) return GC_ERR_IMPROPER_INPUT;
        if (!trusted) {
            maxc_in = h.max_in;
            if (n > 0 && chain_bound(maxc_in)) {  // the buckets again, with the chain-bound threshold
                a.tune.g2_max_deg = std::min(kChainRcG2MaxDeg, a.tune.g4_max_deg);
                cudaMemsetAsync(&a.ctrl->n_heavy, 0, sizeof(int32_t), s);
                GC_LAUNCH(KID_RC_BUCKET, s, k_rc_bucket<<<vgrid, kBlock, 0, s>>>(a));
            }
        }
    } else {
        h.n_heavy = static_cast<int32_t>(heavy_bound);
    }
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

    // Colors stay within [1, maxc_in]: a vertex of the class of rank p takes
    // at most color p + 1 <= k <= maxc_in.
    const int32_t cap = std::max(maxc_in, 1);
    const int64_t ent = static_cast<int64_t>(cap + 1) * kNB;
    const int32_t hub_words = (cap + 1 + 31) / 32;
    const int64_t hubs = std::max<int64_t>(1, h.n_heavy);
    Scratch sc_cls, sc_units, sc_cls2, sc_units2, sc_present, sc_psize, sc_order, sc_jtab, sc_rank, sc_seg, sc_tiles,
        sc_fill, sc_list, sc_alt, sc_ncol, sc_hv, sc_hn, sc_hd, sc_hb, sc_iso, sc_iso2;
    // list entries: one per vertex, one per chunk of a bucket-0 row
    const int64_t list_len = n + (static_cast<int64_t>(g.nnz) / kChunk) + h.n_heavy;
    if (!sc_cls.alloc(ent * 4, s) || !sc_units.alloc((cap + 1) * 4, s) ||
        !sc_cls2.alloc(ent * 4, s) || !sc_units2.alloc((cap + 1) * 4, s) ||
        !sc_present.alloc((cap + 1) * 4, s) || !sc_psize.alloc((cap + 1) * 4, s) ||
        !sc_order.alloc((cap + 1) * 4, s) || !sc_jtab.alloc((cap + 1) * 4, s) ||
        !sc_rank.alloc((cap + 1) * 4, s) || !sc_seg.alloc((ent + 1) * 4, s) ||
        !sc_tiles.alloc((ent + 1) * 4, s) || !sc_fill.alloc(ent * 4, s) ||
        !sc_list.alloc(list_len * sizeof(WorkItem), s) || !sc_alt.alloc(n * 4, s) ||
        !sc_ncol.alloc((iterations + 1) * 4, s) || !sc_hv.alloc(hubs * 4, s) ||
        !sc_hn.alloc(hubs * 4, s) || !sc_hd.alloc(hubs * 4, s) ||
        !sc_hb.alloc(hubs * hub_words * 4, s) || !sc_iso.alloc((cap + 1) * 4, s) ||
        !sc_iso2.alloc((cap + 1) * 4, s))
        return GC_ERR_OOM;
    a.cap = cap;
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
    a.hub_v = sc_hv.as<int32_t>();
    a.hub_nch = sc_hn.as<int32_t>();
    a.hub_done = sc_hd.as<int32_t>();
    a.hub_bm = sc_hb.as<uint32_t>();
    a.hub_words = hub_words;
    a.fuse_hist = 1;
    const int32_t hist_entries = static_cast<int32_t>(ent);
    const size_t hist_dyn = hist_entries <= kRcHistSmem ? static_cast<size_t>(hist_entries) * 4 : 0;
    a.hist_smem = hist_dyn ? hist_entries : 0;
    const int coop_capacity =
        sm_count() * occupancy_of(reinterpret_cast<const void*>(k_rc_recolor_coop), kBlock, hist_dyn);
    const int grid_rc = tune.grid_blocks > 0 ? std::min(tune.grid_blocks, coop_capacity)
                                             : coop_grid(g.nnz, cap, coop_capacity);
    const int step_capacity =
        sm_count() * occupancy_of(reinterpret_cast<const void*>(k_rc_recolor_step), kBlock, hist_dyn);
    const int grid_step = tune.grid_blocks > 0 ? tune.grid_blocks : step_capacity;
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
        // histograms: of the input (iteration 0), else filled by the previous
        // iteration's recoloring kernel
        a.cls_cnt = (it % 2 == 0) ? sc_cls.as<int32_t>() : sc_cls2.as<int32_t>();
        a.cls_units = (it % 2 == 0) ? sc_units.as<int32_t>() : sc_units2.as<int32_t>();
        a.nxt_cnt = (it % 2 == 0) ? sc_cls2.as<int32_t>() : sc_cls.as<int32_t>();
        a.nxt_units = (it % 2 == 0) ? sc_units2.as<int32_t>() : sc_units.as<int32_t>();
        a.iso_cnt = (it % 2 == 0) ? sc_iso.as<int32_t>() : sc_iso2.as<int32_t>();
        a.nxt_iso = (it % 2 == 0) ? sc_iso2.as<int32_t>() : sc_iso.as<int32_t>();
        if (it == 0) {
            cudaMemsetAsync(a.cls_cnt, 0, ent * 4, s);
            cudaMemsetAsync(a.cls_units, 0, (cap + 1) * 4, s);
            cudaMemsetAsync(a.iso_cnt, 0, (cap + 1) * 4, s);
            GC_LAUNCH(KID_RC_HIST, s, k_rc_hist<<<vgrid, kBlock, 0, s>>>(a));
        }
        cudaMemsetAsync(a.nxt_cnt, 0, ent * 4, s);
        cudaMemsetAsync(a.nxt_units, 0, (cap + 1) * 4, s);
        cudaMemsetAsync(a.nxt_iso, 0, (cap + 1) * 4, s);
        GC_LAUNCH(KID_RC_ORDER, s, k_rc_order<<<1, kOrderThreads, 0, s>>>(a));
        GC_LAUNCH(KID_RC_SCATTER, s, k_rc_scatter<<<grid_sc, kBlock, 0, s>>>(a));
        if (tune.recolor_mode == 0) {
            void* args[] = {&a};
            cudaError_t le;
            GC_LAUNCH(KID_RC_RECOLOR, s,
                      le = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_rc_recolor_coop),
                                                       dim3(grid_rc), dim3(kBlock), args, hist_dyn, s));
            if (le != cudaSuccess) { st = cuda_status(le); break; }
        } else {
            RcCtrl hc;
            ce = cudaMemcpyAsync(&hc, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            tp.resize(static_cast<size_t>(hc.k) * kNB + 1);
            ce = cudaMemcpyAsync(tp.data(), a.tile_prefix, tp.size() * 4, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            for (int32_t p = 0; p < hc.k; ++p) {
                const int32_t t0 = tp[p * kNB], t1 = tp[(p + 1) * kNB];
                if (t1 <= t0) continue;
                const int g2 = std::min(grid_step, (t1 - t0 + kWarps - 1) / kWarps);
                GC_LAUNCH(KID_RC_STEP, s, k_rc_recolor_step<<<g2, kBlock, hist_dyn, s>>>(a, p, t0, t1));
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

// Batch recoloring: every graph recolored with its own permutation, seed and
// iteration count; a graph past its count keeps its colors.
// Iterations [it_begin, it_end) of every graph (it_end < 0: to the largest
// count); a graph whose count is reached keeps its colors.  Running the
// iterations in several calls gives the same colors as one call: an
// iteration's class order depends only on the colors it starts from and its
// own number.
static gc_status recolor_batch_impl(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                                    const int32_t* colors_in, bool trusted, const int32_t* max_in,
                                    int32_t* colors_out, int32_t* max_color_out, gc_stats* stats,
                                    cudaStream_t s, int32_t it_begin = 0, int32_t it_end = -1) {
    int32_t max_x = 1;
    gc_status st = batch_layout(g, graphs, ng, &max_x);
    if (st != GC_OK) return st;
    const int64_t n = g.n;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int32_t iters = 0;
    for (int32_t i = 0; i < ng; ++i) iters = std::max(iters, graphs[i].iterations);
    if (it_end >= 0) iters = std::min(iters, it_end);
    it_begin = std::max(it_begin, 0);
    if (iters < it_begin) iters = it_begin;
    const Tuning tune = recolor_tuning(current_tuning());
    const int grid = persistent_grid(tune);
    const int vgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, grid)));
    const int coop_capacity = sm_count() * occupancy_of(reinterpret_cast<const void*>(k_rc_recolor_coop), kBlock);
    const int grid_step = resident_grid(k_rc_recolor_step, tune);
    const int grid_sc = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((n + kBlock - 1) / kBlock, resident_grid(k_rc_scatter, tune))));
    const int grid_go = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((ng + kWarps - 1) / kWarps, grid)));
    cudaError_t ce;

    Scratch sc_ctrl, sc_bucket, sc_desc, sc_gof;
    if (!sc_ctrl.alloc(sizeof(RcCtrl), s) || !sc_bucket.alloc(n + 1, s) ||
        !sc_desc.alloc(static_cast<size_t>(ng) * sizeof(BatchDesc), s) || !sc_gof.alloc(n * 4 + 4, s))
        return GC_ERR_OOM;
    ce = cudaMemcpyAsync(sc_desc.p, graphs, static_cast<size_t>(ng) * sizeof(BatchDesc), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_status(ce);
    RcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.tune = tune;
    a.old_c = colors_in;
    a.bucket = sc_bucket.as<uint8_t>();
    a.ctrl = sc_ctrl.as<RcCtrl>();
    a.desc = sc_desc.as<BatchDesc>();
    a.graph_of = sc_gof.as<int32_t>();
    a.ngraphs = ng;
    batch_graph_of(g, a.desc, ng, sc_gof.as<int32_t>(), s);
    cudaMemsetAsync(a.ctrl, 0, sizeof(RcCtrl), s);
    if (n > 0) {
        GC_LAUNCH(KID_RC_BUCKET, s, k_rc_bucket<<<vgrid, kBlock, 0, s>>>(a));
        if (!trusted) GC_LAUNCH(KID_RC_VALIDATE, s, k_rc_validate<<<grid, kBlock, 0, s>>>(a));
    }
    RcCtrl h;
    ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (h.err & kErrBadGraph) return GC_ERR_BAD_GRAPH;
    if (h.err & kErrImproper) return GC_ERR_IMPROPER_INPUT;
    // each graph's max input color sizes its rows of the (graph, color) tables
    std::vector<int32_t> gmax(ng, 0);
    if (trusted && max_in) {
        std::copy(max_in, max_in + ng, gmax.begin());
    } else {
        st = batch_max_colors(g, a.graph_of, colors_in, nullptr, ng, gmax.data(), nullptr, s);
        if (st != GC_OK) return st;
    }
    std::vector<int64_t> base(static_cast<size_t>(ng) + 1, 0);
    int32_t cap = 1;
    for (int32_t i = 0; i < ng; ++i) {
        base[i + 1] = base[i] + gmax[i] + 1;
        cap = std::max(cap, gmax[i]);
    }
    const int64_t T = base[ng];
    if (iters == it_begin || n == 0) {
        if (colors_out != colors_in && n > 0)
            cudaMemcpyAsync(colors_out, colors_in, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (max_color_out) std::copy(gmax.begin(), gmax.end(), max_color_out);
        return cuda_status(cudaStreamSynchronize(s));
    }
    const int64_t ent = static_cast<int64_t>(cap + 1) * kNB;
    const int32_t hub_words = (cap + 1 + 31) / 32;
    const int64_t hubs = std::max<int64_t>(1, h.n_heavy);
    const int64_t list_len = n + (static_cast<int64_t>(g.nnz) / kChunk) + h.n_heavy;
    const int grid_rc = tune.grid_blocks > 0 ? std::min(tune.grid_blocks, coop_capacity)
                                             : coop_grid(g.nnz, cap, coop_capacity);
    Scratch sc_base, sc_cls, sc_units, sc_rank, sc_gp, sc_gs, sc_go, sc_gj, sc_segc, sc_seg, sc_tiles,
        sc_fill, sc_list, sc_alt, sc_ncol, sc_hv, sc_hn, sc_hd, sc_hb, sc_iso;
    if (!sc_base.alloc((ng + 1) * 8, s) || !sc_cls.alloc(T * kNB * 4, s) || !sc_units.alloc(T * 4, s) ||
        !sc_rank.alloc(T * 4, s) || !sc_gp.alloc(T * 4, s) || !sc_gs.alloc(T * 4, s) ||
        !sc_go.alloc(T * 4, s) || !sc_gj.alloc(T * 4, s) || !sc_segc.alloc(ent * 4, s) ||
        !sc_seg.alloc((ent + 1) * 4, s) || !sc_tiles.alloc((ent + 1) * 4, s) || !sc_fill.alloc(ent * 4, s) ||
        !sc_list.alloc(list_len * sizeof(WorkItem), s) || !sc_alt.alloc(n * 4, s) ||
        !sc_ncol.alloc((iters + 1) * 4, s) || !sc_hv.alloc(hubs * 4, s) || !sc_hn.alloc(hubs * 4, s) ||
        !sc_hd.alloc(hubs * 4, s) || !sc_hb.alloc(hubs * hub_words * 4, s) || !sc_iso.alloc(T * 4, s))
        return GC_ERR_OOM;
    ce = cudaMemcpyAsync(sc_base.p, base.data(), (ng + 1) * 8, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_status(ce);
    a.cap = cap;
    a.cls_base = sc_base.as<int64_t>();
    a.cls_cnt = sc_cls.as<int32_t>();
    a.cls_units = sc_units.as<int32_t>();
    a.rank_of = sc_rank.as<int32_t>();
    a.gpresent = sc_gp.as<int32_t>();
    a.gpsize = sc_gs.as<int32_t>();
    a.gorder = sc_go.as<int32_t>();
    a.gjtab = sc_gj.as<int32_t>();
    a.seg_cnt = sc_segc.as<int32_t>();
    a.seg_start = sc_seg.as<int32_t>();
    a.tile_prefix = sc_tiles.as<int32_t>();
    a.fill = sc_fill.as<int32_t>();
    a.list = sc_list.as<WorkItem>();
    a.ncolors = sc_ncol.as<int32_t>();
    a.hub_v = sc_hv.as<int32_t>();
    a.hub_nch = sc_hn.as<int32_t>();
    a.hub_done = sc_hd.as<int32_t>();
    a.hub_bm = sc_hb.as<uint32_t>();
    a.hub_words = hub_words;
    a.iso_cnt = sc_iso.as<int32_t>();
    a.fuse_hist = 0;
    cudaMemsetAsync(a.ncolors, 0, (iters + 1) * 4, s);

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int32_t* alt = sc_alt.as<int32_t>();
    const int32_t* cur = colors_in;
    std::vector<int32_t> tp;
    for (int32_t it = it_begin; it < iters && st == GC_OK; ++it) {
        int32_t* dst = ((it - it_begin) % 2 == 0) ? alt : colors_out;
        a.iteration = it;
        a.old_c = cur;
        a.new_c = dst;
        cudaMemsetAsync(a.cls_cnt, 0, T * kNB * 4, s);
        cudaMemsetAsync(a.cls_units, 0, T * 4, s);
        cudaMemsetAsync(a.iso_cnt, 0, T * 4, s);
        cudaMemsetAsync(a.seg_cnt, 0, ent * 4, s);
        cudaMemsetAsync(&a.ctrl->k, 0, sizeof(int32_t), s);
        GC_LAUNCH(KID_BRC_HIST, s, k_brc_hist<<<vgrid, kBlock, 0, s>>>(a));
        GC_LAUNCH(KID_BRC_ORDER, s, k_brc_order<<<grid_go, kBlock, 0, s>>>(a));
        GC_LAUNCH(KID_BRC_SEGMENTS, s, k_brc_segments<<<1, kOrderThreads, 0, s>>>(a));
        GC_LAUNCH(KID_RC_SCATTER, s, k_rc_scatter<<<grid_sc, kBlock, 0, s>>>(a));
        if (tune.recolor_mode == 0) {
            void* args[] = {&a};
            cudaError_t le;
            GC_LAUNCH(KID_RC_RECOLOR, s,
                      le = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_rc_recolor_coop),
                                                       dim3(grid_rc), dim3(kBlock), args, 0, s));
            if (le != cudaSuccess) { st = cuda_status(le); break; }
        } else {
            RcCtrl hc;
            ce = cudaMemcpyAsync(&hc, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            tp.resize(static_cast<size_t>(hc.k) * kNB + 1);
            ce = cudaMemcpyAsync(tp.data(), a.tile_prefix, tp.size() * 4, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            for (int32_t p = 0; p < hc.k; ++p) {
                const int32_t t0 = tp[p * kNB], t1 = tp[(p + 1) * kNB];
                if (t1 <= t0) continue;
                const int g2 = std::min(grid_step, (t1 - t0 + kWarps - 1) / kWarps);
                GC_LAUNCH(KID_RC_STEP, s, k_rc_recolor_step<<<g2, kBlock, 0, s>>>(a, p, t0, t1));
            }
        }
        cur = dst;
    }
    if (st == GC_OK && cur != colors_out)
        cudaMemcpyAsync(colors_out, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    cudaEventRecord(e1, s);
    ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(RcCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess && st == GC_OK) st = cuda_status(ce);
    if (st == GC_OK) st = status_from_err_bits(h.err);
    if (st == GC_OK && max_color_out)
        st = batch_max_colors(g, a.graph_of, colors_out, nullptr, ng, max_color_out, nullptr, s);
    if (stats) {
        stats->iterations = iters - it_begin;
        stats->edges_examined = static_cast<int64_t>(h.edges);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_recolor = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

gc_status recolor_batch_range(const Graph& g, const gc_batch_graph* graphs, int32_t ng, int32_t* colors,
                              const int32_t* max_in, int32_t it_begin, int32_t it_end,
                              int32_t* max_color_out, cudaStream_t s) {
    return recolor_batch_impl(g, graphs, ng, colors, true, max_in, colors, max_color_out, nullptr, s,
                              it_begin, it_end);
}

gc_status recolor_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                               const int32_t* colors_in, int32_t* colors_out, int32_t* max_color_out,
                               gc_stats* stats, cudaStream_t s) {
    return recolor_batch_impl(g, graphs, ng, colors_in, false, nullptr, colors_out, max_color_out,
                              stats, s);
}

gc_status color_recolor_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                                     int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                                     gc_stats* stats, cudaStream_t s) {
    std::vector<int32_t> cmax(std::max(ng, 1));
    gc_stats cs;
    gc_status st = color_batch_device(g, graphs, ng, colors_out, rounds_out, cmax.data(), &cs, s);
    if (st != GC_OK) return st;
    gc_stats rs;
    st = recolor_batch_impl(g, graphs, ng, colors_out, true, cmax.data(), colors_out, max_color_out,
                            &rs, s);
    if (stats) {
        *stats = cs;
        stats->iterations = rs.iterations;
        stats->edges_examined = cs.edges_examined + rs.edges_examined;
        stats->ms_recolor = rs.ms_recolor;
    }
    return st;
}

}  // namespace gc
