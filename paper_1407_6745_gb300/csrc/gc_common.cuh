// gc_common.cuh -- device building blocks shared by the coloring kernels.
//
// Degree-bucketed scheduling: every vertex to (re)color is handled by a group
// of lanes sized to its degree.  A vertex whose answer is known to lie in the
// first 64 colors (deg + X <= 64: at most deg colors are forbidden, and the
// pick is among the first X permissible ones) keeps its forbidden set in a
// 64-bit register mask, OR-reduced over a group of 4, 8, 16 or 32 lanes; a
// larger one uses a bitmap in shared memory, per warp (deg <= warp_max_deg)
// or per block.  The color picked is the j-th clear bit of the mask (First
// Fit: j = 0), located with popc/ffs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gc {

constexpr int kBlock = 256;          // threads per block, every kernel
constexpr int kWarps = kBlock / 32;
constexpr int kNB = 7;               // degree buckets
// bucket b: 0 block/vertex, 1 warp/vertex + smem bitmap, 2..6 group of
// 32/16/8/4/2 lanes per vertex with a 64-bit register mask
__host__ __device__ constexpr int bucket_group(int b) {
    return b == 0 ? kBlock : b == 1 ? 32 : b == 2 ? 32 : b == 3 ? 16 : b == 4 ? 8 : b == 5 ? 4 : 2;
}
// vertices per block tile
__host__ __device__ constexpr int bucket_tile(int b) {
    return b == 0 ? 1 : kBlock / bucket_group(b);
}
constexpr int kWarpBitmapWords = 64;    // 2048 colors per window, per warp

// error bits accumulated on the device
constexpr uint32_t kErrBadGraph = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrImproper = 4u;
constexpr uint32_t kErrRoundLimit = 8u;

// Default warp threshold of the coloring phase (rows above it take a whole
// block); on a graph whose largest row has at most kPullAllMaxDeg entries the
// default is lifted so that every heavy row is a warp row (see color_impl).
constexpr int32_t kDefaultWarpMaxDeg = 1024;
constexpr int32_t kPullAllMaxDeg = 12288;
// Default 2-lane threshold of the recoloring phase, and the one a recoloring
// launch bound by its class chain takes instead (see recolor_device).
constexpr int32_t kDefaultRcG2MaxDeg = 16;
constexpr int32_t kChainRcG2MaxDeg = 8;

// Scheduling thresholds (runtime; tuned per workload).
struct Tuning {
    int32_t g4_max_deg;    // deg <= this -> 4 lanes
    int32_t g8_max_deg;    // -> 8 lanes
    int32_t g16_max_deg;   // -> 16 lanes
    int32_t warp_max_deg;  // deg + X > 64 and deg <= this -> warp + smem bitmap
    int32_t grid_blocks;   // persistent grid size (0 = 8 per SM)
    int32_t recolor_mode;  // 0 = dataflow (one launch), 1 = one launch per class
    int32_t spin_limit;    // bounded wait iterations in the dataflow recolor
    int32_t spec_graph;    // 1: speculative rounds in a CUDA graph WHILE node; 0: host loop
    int32_t rc_warp_max_deg;  // warp_max_deg of the recoloring phase
    int32_t g2_max_deg;    // deg <= this -> 2 lanes (0: none)
    int32_t rc_g2_max_deg;  // g2_max_deg of the recoloring phase (capped at g4_max_deg)
};

// The recoloring phase's view of the knobs: its own warp and 2-lane thresholds.
__host__ __device__ inline Tuning recolor_tuning(Tuning t) {
    t.warp_max_deg = t.rc_warp_max_deg;
    t.g2_max_deg = t.rc_g2_max_deg < t.g4_max_deg ? t.rc_g2_max_deg : t.g4_max_deg;
    return t;
}

__host__ __device__ inline int bucket_of(int64_t deg, int32_t X, const Tuning& t) {
    if (deg + (int64_t)X <= 64) {
        if (deg <= t.g2_max_deg) return 6;
        if (deg <= t.g4_max_deg) return 5;
        if (deg <= t.g8_max_deg) return 4;
        if (deg <= t.g16_max_deg) return 3;
        return 2;
    }
    return deg <= t.warp_max_deg ? 1 : 0;
}

// The permutation (RV/NI/ND/RAND = 0..3) of recoloring iteration `it`
// (0-based) under a gc_perm code, schedules included (Sec. 4.2.1: the paper
// counts iterations from 1); -1 for an unknown code.
constexpr int32_t kSchedPow2 = 4, kSchedEveryBase = 256, kSchedEveryMax = 256 + 65535;
__host__ __device__ inline int32_t perm_at(int32_t code, int32_t it) {
    if (code >= 0 && code <= 3) return code;
    const int32_t t = it + 1;
    if (code == kSchedPow2) return (t >= 2 && (t & (t - 1)) == 0) ? 3 : 2;
    if (code > kSchedEveryBase && code <= kSchedEveryMax) return t % (code - kSchedEveryBase) == 0 ? 3 : 2;
    return -1;
}
__host__ __device__ inline bool perm_valid(int32_t code) { return perm_at(code, 0) >= 0; }

// One graph of a batch (same layout as gc_batch_graph).
struct BatchDesc {
    int64_t base;
    int64_t n;
    uint64_t seed;
    int32_t X;
    int32_t perm;
    int32_t iterations;
    int32_t reserved;
    uint64_t perm_seed;
};

struct Graph {
    const int64_t* off;
    const int32_t* idx;
    int32_t n;
    int64_t nnz;
    int32_t vec;  // idx is 16-byte aligned: rows are read as aligned 4-id chunks
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), word 0 only.  Device copy written for
// this library; the key is bumped by the two Weyl constants after each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t philox_word0(uint64_t seed, uint32_t x0, uint32_t x1,
                                                 uint32_t x2, uint32_t x3) {
    uint32_t key_lo = static_cast<uint32_t>(seed);
    uint32_t key_hi = static_cast<uint32_t>(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a_hi = __umulhi(0xD2511F53u, x0), a_lo = 0xD2511F53u * x0;
        const uint32_t b_hi = __umulhi(0xCD9E8D57u, x2), b_lo = 0xCD9E8D57u * x2;
        const uint32_t y0 = b_hi ^ x1 ^ key_lo;
        const uint32_t y2 = a_hi ^ x3 ^ key_hi;
        x0 = y0;
        x1 = b_lo;
        x2 = y2;
        x3 = a_lo;
        key_lo += 0x9E3779B9u;
        key_hi += 0xBB67AE85u;
    }
    return x0;
}

__device__ __forceinline__ uint32_t prio_of(uint64_t seed, int32_t v) {
    return philox_word0(seed, static_cast<uint32_t>(v), 0u, 0u, 1u);
}
__device__ __forceinline__ uint32_t rxf_word(uint64_t seed, int32_t v, int32_t round) {
    return philox_word0(seed, static_cast<uint32_t>(v), 0u, static_cast<uint32_t>(round), 2u);
}
__device__ __forceinline__ uint32_t perm_word(uint64_t seed, int32_t i, int32_t iteration) {
    return philox_word0(seed, static_cast<uint32_t>(i), static_cast<uint32_t>(iteration), 0u, 3u);
}
// index in [0, m) from a 32-bit word: floor(w * m / 2^32)
__device__ __forceinline__ uint32_t scale_index(uint32_t w, uint32_t m) {
    return static_cast<uint32_t>((static_cast<uint64_t>(w) * m) >> 32);
}

// ---------------------------------------------------------------------------
// Warp / group helpers
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <int G>
__device__ __forceinline__ uint64_t group_or(uint64_t m) {
    uint32_t lo = static_cast<uint32_t>(m), hi = static_cast<uint32_t>(m >> 32);
    if constexpr (G == 32) {
        lo = __reduce_or_sync(kFull, lo);
        hi = __reduce_or_sync(kFull, hi);
    } else {
#pragma unroll
        for (int d = G / 2; d >= 1; d >>= 1) {
            lo |= __shfl_xor_sync(kFull, lo, d);
            hi |= __shfl_xor_sync(kFull, hi, d);
        }
    }
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

template <int G>
__device__ __forceinline__ bool group_any(bool p) {
    const uint32_t b = __ballot_sync(kFull, p);
    if constexpr (G == 32) {
        return b != 0;
    } else {
        const int shift = lane_id() & ~(G - 1);
        const uint32_t gm = (G == 32) ? kFull : ((1u << G) - 1u);
        return ((b >> shift) & gm) != 0;
    }
}

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x) {
    const int l = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (l >= d) x += y;
    }
    return x;
}

// Position (0-based) of the j-th set bit of x; requires j < popc(x).
__device__ __forceinline__ int select_bit32(uint32_t x, uint32_t j) {
    int pos = 0;
    uint32_t c = __popc(x & 0xFFFFu);
    if (j >= c) { j -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xFFu);
    if (j >= c) { j -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xFu);
    if (j >= c) { j -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (j >= c) { j -= c; x >>= 2; pos += 2; }
    c = x & 1u;
    if (j >= c) pos += 1;
    return pos;
}

__device__ __forceinline__ int select_bit64(uint64_t x, uint32_t j) {
    const uint32_t lo = static_cast<uint32_t>(x);
    const uint32_t pl = __popc(lo);
    if (j < pl) return select_bit32(lo, j);
    return 32 + select_bit32(static_cast<uint32_t>(x >> 32), j - pl);
}

// Adjacency range of v with the structure checks that keep every later load
// in bounds: a bad row is flagged and treated as empty.
__device__ __forceinline__ void row_range(const Graph& g, int32_t v, int64_t& beg, int64_t& end,
                                          uint32_t* err) {
    beg = __ldg(g.off + v);
    end = __ldg(g.off + v + 1);
    if (beg < 0 || end < beg || end > g.nnz) {
        atomicOr(err, kErrBadGraph);
        beg = end = 0;
    }
}

// Streamed data (adjacency, work items) is read once per pass: it is loaded
// with an L2 evict-first policy and without L1 allocation, so it does not
// push the gathered color arrays out of L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t* ptr) {
    int32_t x;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
        : "=r"(x)
        : "l"(ptr), "l"(policy_evict_first()));
    return x;
}

__device__ __forceinline__ int4 ld_stream4(const void* ptr) {
    int4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(ptr), "l"(policy_evict_first()));
    return r;
}

__device__ __forceinline__ int32_t load_nbr(const Graph& g, int64_t e, uint32_t* err) {
    const int32_t u = ld_stream(g.idx + e);
    if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(g.n)) {
        atomicOr(err, kErrBadGraph);
        return -1;
    }
    return u;
}

// ---------------------------------------------------------------------------
// Work items: a vertex with its adjacency row, so a kernel reaches the row
// without a dependent load of the offsets.  16 bytes, one vector load.
// ---------------------------------------------------------------------------
struct __align__(16) WorkItem {
    int64_t beg;
    int32_t v;
    int32_t deg;
};

__device__ __forceinline__ WorkItem load_item(const WorkItem* p) {
    const int4 r = ld_stream4(p);
    WorkItem w;
    w.beg = (static_cast<int64_t>(static_cast<uint32_t>(r.y)) << 32) | static_cast<uint32_t>(r.x);
    w.v = r.z;
    w.deg = r.w;
    return w;
}

__device__ __forceinline__ void store_item(WorkItem* p, int64_t beg, int32_t v, int32_t deg) {
    int4 r;
    r.x = static_cast<int32_t>(static_cast<uint64_t>(beg));
    r.y = static_cast<int32_t>(static_cast<uint64_t>(beg) >> 32);
    r.z = v;
    r.w = deg;
    *reinterpret_cast<int4*>(p) = r;
}

// Row of v as (beg, deg) with the checks that keep every later load in
// bounds: a malformed row is flagged and treated as empty.
__device__ __forceinline__ void row_of(const Graph& g, int32_t v, int64_t& beg, int32_t& deg,
                                       uint32_t* err) {
    int64_t b = __ldg(g.off + v), e = __ldg(g.off + v + 1);
    if (b < 0 || e < b || e > g.nnz || e - b > INT32_MAX) {
        atomicOr(err, kErrBadGraph);
        b = e = 0;
    }
    beg = b;
    deg = static_cast<int32_t>(e - b);
}

// ---------------------------------------------------------------------------
// Color choice: the j-th (0-based) color >= 1 not used by a neighbor.
//
// A Fetch gives a neighbor's color in two steps: raw(u) issues the load (no
// branch, so a batch of U loads is in flight at once) and resolve(u, x)
// turns the loaded word into a color, or a value < 1 to ignore the neighbor.
// Each lane takes the neighbors lane0, lane0 + stride, ...; U per batch.
// ---------------------------------------------------------------------------
// Visits the neighbors of a row, lane `lane0` of a group of `stride` lanes
// taking every stride-th piece.  (kVec selects the chunked reads; color
// selection keeps single-id reads, measured faster there: the chunked form
// holds more registers per gather batch.)  load(u) issues the gather for neighbor u
// (called for a whole batch before any visit, so the batch's gathers are in
// flight together); visit(u, x) consumes it.  With an aligned idx the row is
// read as aligned 16-byte chunks of 4 ids (UC chunks per lane per batch),
// the entries outside the row masked off; otherwise 4 * UC single ids.
template <int UC, class T, bool kVec, class Load, class Visit>
__device__ __forceinline__ void for_each_nbr(const Graph& g, int64_t beg, int32_t deg,
                                             int32_t lane0, int32_t stride, Load&& load,
                                             Visit&& visit, uint32_t* err) {
    constexpr int U = 4 * UC;
    if (deg <= 0) return;
    if (kVec && g.vec) {
        const int64_t a0 = beg & ~static_cast<int64_t>(3);
        const int64_t end = beg + deg;
        const int32_t nch = static_cast<int32_t>((end - a0 + 3) >> 2);
        for (int32_t c0 = lane0; c0 < nch; c0 += stride * UC) {
            int32_t u[U];
#pragma unroll
            for (int i = 0; i < UC; ++i) {
                const int32_t c = c0 + i * stride;
                const int64_t e0 = a0 + 4 * static_cast<int64_t>(c);
                int4 q = make_int4(-1, -1, -1, -1);
                if (c < nch) {
                    if (e0 + 4 <= g.nnz) {
                        q = ld_stream4(g.idx + e0);
                    } else {  // the last ids of the array: no read past its end
                        q.x = e0 < g.nnz ? ld_stream(g.idx + e0) : -1;
                        q.y = e0 + 1 < g.nnz ? ld_stream(g.idx + e0 + 1) : -1;
                        q.z = e0 + 2 < g.nnz ? ld_stream(g.idx + e0 + 2) : -1;
                        q.w = e0 + 3 < g.nnz ? ld_stream(g.idx + e0 + 3) : -1;
                    }
                }
                const int32_t qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t e = e0 + j;
                    int32_t v = -1;
                    if (c < nch && e >= beg && e < end) {
                        v = qq[j];
                        if (static_cast<uint32_t>(v) >= static_cast<uint32_t>(g.n)) {
                            atomicOr(err, kErrBadGraph);
                            v = -1;
                        }
                    }
                    u[4 * i + j] = v;
                }
            }
            T x[U];
#pragma unroll
            for (int i = 0; i < U; ++i) x[i] = load(u[i] >= 0 ? u[i] : 0);
#pragma unroll
            for (int i = 0; i < U; ++i)
                if (u[i] >= 0) visit(u[i], x[i]);
        }
    } else {
        for (int32_t k0 = lane0; k0 < deg; k0 += stride * U) {
            int32_t u[U];
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const int32_t k = k0 + i * stride;
                u[i] = k < deg ? load_nbr(g, beg + k, err) : -1;
            }
            T x[U];
#pragma unroll
            for (int i = 0; i < U; ++i) x[i] = load(u[i] >= 0 ? u[i] : 0);
#pragma unroll
            for (int i = 0; i < U; ++i)
                if (u[i] >= 0) visit(u[i], x[i]);
        }
    }
}

// Colors of the neighbors through a Fetch: raw(u) issues the load (no
// branch), resolve(u, x) turns it into a color, or a value < 1 to ignore.
template <int UC, class Fetch, class Mark, bool kVec = false>
__device__ __forceinline__ void scan_row(const Graph& g, int64_t beg, int32_t deg, int32_t lane0,
                                         int32_t stride, const Fetch& fetch, Mark&& mark,
                                         uint32_t* err) {
    for_each_nbr<UC, int32_t, kVec>(
        g, beg, deg, lane0, stride, [&](int32_t u) { return fetch.raw(u); },
        [&](int32_t u, int32_t x) { mark(fetch.resolve(u, x)); }, err);
}

// Register path, G lanes per vertex; requires deg + j < 64.  All 32 lanes of
// the warp must call it (lanes without a vertex pass deg = 0).
template <int G, int U, class Fetch, bool kVec = false>
__device__ __forceinline__ int32_t choose_reg(const Graph& g, int64_t beg, int32_t deg, int gl,
                                              uint32_t j, const Fetch& fetch, uint32_t* err) {
    uint64_t m = 0;
    auto mark = [&](int32_t c) {
        if (static_cast<uint32_t>(c - 1) < 64u) m |= 1ull << (c - 1);
    };
    scan_row<U, Fetch, decltype(mark)&, kVec>(g, beg, deg, gl, G, fetch, mark, err);
    m = group_or<G>(m);
    const uint64_t free_bits = ~m;
    if (j == 0) return __ffsll(static_cast<long long>(free_bits));
    return select_bit64(free_bits, j) + 1;
}

// Warp path with a 64-word shared bitmap (2048 colors per window); windows
// advance until the j-th permissible color is found.  Whole warp, one vertex.
template <int U, class Fetch>
__device__ __forceinline__ int32_t choose_warp(const Graph& g, int64_t beg, int32_t deg,
                                               uint32_t j, const Fetch& fetch, uint32_t* bm,
                                               uint32_t* err) {
    const int l = lane_id();
    int32_t base = 1;
    for (;;) {
        bm[l] = 0u;
        bm[l + 32] = 0u;
        __syncwarp();
        scan_row<1>(g, beg, deg, l, 32, fetch,
                    [&](int32_t c) {
                        const uint32_t d = static_cast<uint32_t>(c - base);
                        if (c > 0 && d < 32u * kWarpBitmapWords) atomicOr(&bm[d >> 5], 1u << (d & 31));
                    },
                    err);
        __syncwarp();
        const uint32_t w0 = ~bm[2 * l], w1 = ~bm[2 * l + 1];
        const uint32_t cnt = __popc(w0) + __popc(w1);
        const uint32_t incl = warp_inclusive_scan(cnt);
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        if (j < total) {
            const uint32_t excl = incl - cnt;
            const bool mine = j >= excl && j < incl;
            const int owner = __ffs(__ballot_sync(kFull, mine)) - 1;
            int32_t color = 0;
            if (mine) {
                const uint32_t jj = j - excl;
                const uint32_t p0 = __popc(w0);
                const int bit = jj < p0 ? select_bit32(w0, jj) : 32 + select_bit32(w1, jj - p0);
                color = base + 64 * l + bit;
            }
            color = __shfl_sync(kFull, color, owner);
            __syncwarp();
            return color;
        }
        j -= total;
        base += 32 * kWarpBitmapWords;
        __syncwarp();
    }
}

// Single ids per lane per batch in the recoloring scans, in units of 4, per
// group size (32/16/8/4/2 lanes).  (2 lanes: 4 ids each, rows of at most 16
// entries; 8 in flight were measured 1-3 % slower on R-MAT, where most of
// those rows have 1 or 2 entries.)
template <int G> struct LanesUnroll { static constexpr int U = (G == 4) ? 2 : 1; };

// ---------------------------------------------------------------------------
// Tiles: a list is cut into segments (one bucket each); segment s holds
// tiles tile_prefix[s] .. tile_prefix[s+1]-1 of bucket_tile(bucket) vertices.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_segment(const int32_t* prefix, int nseg, int32_t t) {
    int lo = 0, hi = nseg - 1;  // largest s with prefix[s] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Warp-aggregated append of the items of the lanes with `want` into
// list[start + counter++].  The whole warp must call it.
__device__ __forceinline__ void warp_append(bool want, int64_t beg, int32_t v, int32_t deg,
                                            int32_t* counter, WorkItem* list, int32_t start) {
    const uint32_t b = __ballot_sync(kFull, want);
    if (b == 0) return;
    const int l = lane_id();
    const int leader = __ffs(b) - 1;
    int32_t base = 0;
    if (l == leader) base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(kFull, base, leader);
    if (want) store_item(list + start + base + __popc(b & ((1u << l) - 1u)), beg, v, deg);
}

// Warp-wide sum of a per-thread count added to a global counter (one atomic
// per warp).  The whole warp must call it.
__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned long long x) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    if (lane_id() == 0 && x != 0) atomicAdd(dst, x);
}

// Max of non-negative values into *dst (which starts at 0): a warp whose
// values are all 0 adds nothing.
__device__ __forceinline__ void warp_max(int32_t* dst, int32_t x) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) x = max(x, __shfl_xor_sync(kFull, x, d));
    if (lane_id() == 0 && x > 0) atomicMax(dst, x);
}

}  // namespace gc
