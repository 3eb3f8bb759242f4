// gc_color.cu -- speculative distance-1 coloring on one GPU.
//
// The rounds of Sec. 2.2 in a data-parallel (Jacobi) form: in round r every
// vertex of the work set W_r chooses a tentative color against the colors
// fixed before the round (First Fit, Alg. 1 / Sec. 2.1, or Random-X Fit,
// Sec. 3.2); then every vertex of W_r compares its tentative color with its
// neighbors' and loses if one of them has the same color and a larger
// (priority, id) -- the random total order of Sec. 2.2.  Winners keep their
// color, losers form W_{r+1}.  The vertex of W_r with the largest (priority,
// id) always wins, so the loop ends within |V| rounds.
//
// Layout in HBM: colors int32[n] (the output, 0 = uncolored), key uint64[n]
// = (tentative color << 32 | priority), so one 8-byte gather gives conflict
// detection both the color and the priority of a neighbor; two work lists of
// 16-byte items (vertex, row start, degree) used as
// ping-pong buffers, each cut into six degree-bucket regions whose starts are
// fixed in round 0 (a loser stays in its bucket, so a region never
// overflows).  All per-round state (round number, bucket counts) lives in a
// small device control block, so a round's two launches take no host input.
//
// Heavy rows (the block- and warp-bucket rows, degree above 64 - X) are not
// re-read every round.  Each keeps a bitmap of the colors of its fixed
// neighbors, which those neighbors mark when they are fixed (a fixed vertex
// walks its row once and sets its color's bit in each heavy neighbor's
// bitmap; a block-bucket winner's row is marked by the whole grid in a third
// launch of the round), so its tentative color is a search of its bitmap.
// For the conflict test it keeps a list of its neighbors above it in the
// total order that were not fixed at its last look, built from the row in
// round 0; only those can beat it, so a round scans the list, dropping the
// entries fixed since.  The forbidden set and the conflict candidates are
// exactly those of a full row scan.  Where the block-bucket rows hold under
// 1/16 of the entries, marks would cost more than they save for the warp-
// bucket rows: those keep the list of all their neighbors not fixed and
// fold the fixed ones' colors into their bitmaps themselves each round.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gc_internal.h"

namespace gc {

struct SpecCtrl {
    int32_t cnt[2][kNB];    // bucket counts of the work list of parity p
    int32_t start[kNB];     // region starts (fixed)
    int32_t init_cnt[kNB];  // round-0 bucket sizes
    int32_t round;
    int32_t active;         // |W| for the coming round
    int32_t max_color;
    int32_t max_deg;
    uint32_t err;
    uint32_t done_blocks;
    int32_t mark_cnt;       // marking items of the round (block-bucket winners)
    unsigned long long edges;
    unsigned long long conflicts;
    long long heavy_entries;  // pending-list entries over all heavy rows
    unsigned long long block_entries;  // adjacency entries of the block-bucket rows
    long long heavy_words;    // bitmap words over all heavy rows
};

// Heavy rows (the block- and warp-bucket rows): index of each, its list
// (start, length) of the neighbors that were not fixed at its last look
// (those above it in the total order, except for pulling warp-bucket rows)
// and its forbidden bitmap (start, words), which the marking vertices reach
// through bref.
struct HeavyRows {
    int32_t* hid;
    int64_t* h_pbeg;
    int32_t* h_pcnt;
    int64_t* h_bbeg;
    int32_t* h_bwords;
    int32_t* pend;
    uint32_t* hbm;
    uint64_t* bref;  // per vertex: bitmap_ref of its row, or all ones
    // the rows of the round's block-bucket winners, in pieces of kMarkChunk
    // entries (item: row piece start, winner's color, length), marked by
    // the whole grid after the conflict launch
    WorkItem* mark;
    int64_t mark_cap;
    // 1: the warp-bucket rows keep lists of all their neighbors not fixed and
    // fold their bitmaps themselves (few block-bucket rows: marks would cost
    // more than they save); only the block-bucket rows are marked then
    int32_t pull_warp;
    int32_t mark_bucket;  // the largest bucket that is marked
    uint8_t* near;        // with pull_warp: 1 for a neighbor of a block-bucket row (it marks)
};

constexpr int32_t kMarkChunk = 2048;
constexpr uint8_t kBucketFixed = 0xFE;  // bucket byte of a fixed heavy row (marks skip it)
constexpr unsigned long long kPullShare = 16;    // block-bucket rows below 1/16 of the entries: warp rows pull

struct SpecArgs {
    Graph g;
    int32_t X;
    uint64_t seed;
    Tuning tune;
    int32_t* color;    // fixed colors (0 = in the work set)
    uint64_t* key;     // (tentative color << 32) | priority
    uint8_t* bucket;   // degree bucket per vertex
    WorkItem* list0;   // work lists (ping-pong), bucket regions
    WorkItem* list1;
    SpecCtrl* ctrl;
    unsigned long long cond;  // WHILE-node handle (graph mode)
    int32_t use_cond;
    int32_t round_limit;
    // batches: graph of every vertex and the graphs' descriptors (nullptr for
    // one graph), and the round in which every vertex kept its color
    const int32_t* graph_of;
    const BatchDesc* desc;
    int32_t* win_round;
    int32_t* graph_heavy;  // batches: nonzero for a graph with heavy rows (its vertices mark)
    // heavy rows (bucket 0), in device memory so that the arrays can be
    // sized after the CUDA graph of the rounds has been built
    struct HeavyRows* heavy;
    // priority rule: 0 the random order; 1 Largest First (degree first);
    // 2 aRC (rank of the vertex's previous class first, from prio_rank[prio_old[v]])
    int32_t prio_kind;
    const int32_t* prio_rank;
    const int32_t* prio_old;
};

// A vertex-visit key (16 bits, clamped) above the upper half of the random
// priority; equal keys still fall back to the id.
__device__ __forceinline__ uint32_t ordered_prio(int64_t first_key, uint32_t p) {
    const uint32_t k = static_cast<uint32_t>(first_key < 0 ? 0 : first_key > 65535 ? 65535 : first_key);
    return (k << 16) | (p >> 16);
}

// Bitmap words of a heavy row: colors 1 .. 32 * words, at least deg + 64.
__host__ __device__ __forceinline__ int32_t heavy_words(int32_t deg) { return (deg + 64) / 32 + 2; }

// Per-vertex reference to a heavy row's bitmap: (first word << 24) | words,
// the words clamped to 2^24 - 1 on the marking and the reading side alike;
// kNoBitmap for every other row.
constexpr uint64_t kNoBitmap = ~0ull;
constexpr uint32_t kRefWords = (1u << 24) - 1u;
__device__ __forceinline__ uint64_t bitmap_ref(long long first_word, long long words) {
    return (static_cast<uint64_t>(first_word) << 24) |
           static_cast<uint32_t>(words < kRefWords ? words : kRefWords);
}

// Random-X index of v in `round`: the graph's own seed, X and local id.
__device__ __forceinline__ uint32_t draw_index(const SpecArgs& a, int32_t v, int32_t round) {
    if (a.graph_of) {
        const BatchDesc& d = a.desc[a.graph_of[v]];
        if (d.X <= 1) return 0u;
        return scale_index(rxf_word(d.seed, static_cast<int32_t>(v - d.base), round),
                           static_cast<uint32_t>(d.X));
    }
    return scale_index(rxf_word(a.seed, v, round), static_cast<uint32_t>(a.X));
}

// ---------------------------------------------------------------------------
// Set-up: priorities, bucket sizes, then the round-0 work list (all vertices)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_spec_setup(SpecArgs a) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    int32_t my_max_deg = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; i < a.g.n; i += stride) {
        const int32_t v = static_cast<int32_t>(i);
        int64_t beg;
        int32_t deg;
        row_of(a.g, v, beg, deg, &a.ctrl->err);
        my_max_deg = max(my_max_deg, deg);
        int32_t X = a.X, vl = v;
        uint64_t seed = a.seed;
        if (a.graph_of) {
            const BatchDesc& d = a.desc[a.graph_of[v]];
            X = d.X;
            seed = d.seed;
            vl = static_cast<int32_t>(v - d.base);
        }
        const int b = bucket_of(deg, X, a.tune);
        a.bucket[v] = static_cast<uint8_t>(b);
        if (b == 0) atomicAdd(&a.ctrl->block_entries, static_cast<unsigned long long>(deg));
        if (b <= 1 && a.graph_of) {
            int32_t* gh = a.graph_heavy + a.graph_of[v];
            if (!*gh) atomicOr(gh, 1);
        }
        uint32_t p = prio_of(seed, vl);
        if (a.prio_kind == 1) p = ordered_prio(deg, p);
        else if (a.prio_kind == 2) p = ordered_prio(65535 - static_cast<int64_t>(a.prio_rank[a.prio_old[v]]), p);
        // round 0's tentative color: nothing is colored yet, so the j-th
        // permissible color is j + 1 (First Fit: 1)
        const uint32_t j0 = (a.graph_of || a.X > 1) ? draw_index(a, v, 0) : 0u;
        a.key[v] = (static_cast<uint64_t>(j0 + 1u) << 32) | p;
        a.color[v] = 0;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        const int leader = __ffs(peers) - 1;
        if (lane_id() == leader) atomicAdd(&a.ctrl->init_cnt[b], __popc(peers));
    }
    warp_max(&a.ctrl->max_deg, my_max_deg);
}

__global__ void __launch_bounds__(kBlock) k_spec_fill(SpecArgs a) {
    __shared__ int32_t s_start[kNB];
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int b = 0; b < kNB; ++b) {
            s_start[b] = acc;
            acc += a.ctrl->init_cnt[b];
        }
        if (blockIdx.x == 0) {
            for (int b = 0; b < kNB; ++b) a.ctrl->start[b] = s_start[b];
            a.ctrl->active = acc;
        }
    }
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; i < a.g.n; i += stride) {
        const int32_t v = static_cast<int32_t>(i);
        const int b = a.bucket[v];
        int64_t beg;
        int32_t deg;
        row_of(a.g, v, beg, deg, &a.ctrl->err);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        const int leader = __ffs(peers) - 1;
        int32_t base = 0;
        if (lane_id() == leader) base = atomicAdd(&a.ctrl->cnt[0][b], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        store_item(a.list0 + s_start[b] + base + __popc(peers & ((1u << lane_id()) - 1u)), beg, v, deg);
    }
}

// Heavy rows: index, pending-list and bitmap offsets (exclusive scans over
// the bucket-0 region of the round-0 list), one block.
constexpr int kHeavyThreads = 1024;
constexpr int kHeavyChunk = 8 * kHeavyThreads;  // rows per block of the two set-up kernels

__device__ __forceinline__ void heavy_sizes(const SpecArgs& a, int32_t h, int32_t nh, int32_t& v,
                                            long long& e, long long& wd) {
    v = 0;
    e = 0;
    wd = 0;
    if (h < nh) {
        const WorkItem it = load_item(a.list0 + a.ctrl->start[0] + h);
        v = it.v;
        e = (static_cast<long long>(it.deg) + 3) & ~3ll;  // 16-byte aligned list starts
        wd = heavy_words(it.deg);
    }
}

// Block sums of the list entries and bitmap words of its chunk of rows.
__global__ void __launch_bounds__(kHeavyThreads) k_heavy_sums(SpecArgs a, int32_t nh, long long* sums) {
    __shared__ long long s_e[kHeavyThreads / 32], s_w[kHeavyThreads / 32];
    const int l = lane_id(), w = threadIdx.x >> 5;
    long long te = 0, tw = 0;
    const int32_t lo = blockIdx.x * kHeavyChunk;
    for (int32_t h = lo + static_cast<int32_t>(threadIdx.x); h < min(nh, lo + kHeavyChunk); h += kHeavyThreads) {
        int32_t v;
        long long e, wd;
        heavy_sizes(a, h, nh, v, e, wd);
        te += e;
        tw += wd;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        te += __shfl_xor_sync(kFull, te, d);
        tw += __shfl_xor_sync(kFull, tw, d);
    }
    if (l == 0) {
        s_e[w] = te;
        s_w[w] = tw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long be = 0, bw = 0;
        for (int k = 0; k < kHeavyThreads / 32; ++k) {
            be += s_e[k];
            bw += s_w[k];
        }
        sums[2 * blockIdx.x] = be;
        sums[2 * blockIdx.x + 1] = bw;
    }
}

// Heavy rows: index, pending-list and bitmap offsets (exclusive scans over
// the block- and warp-bucket regions of the round-0 list), a chunk of rows
// per block, based at the sums of the chunks before it.
__global__ void __launch_bounds__(kHeavyThreads) k_heavy_setup(SpecArgs a, int32_t nh, const long long* sums) {
    __shared__ long long s_e[kHeavyThreads / 32], s_w[kHeavyThreads / 32];
    __shared__ long long s_base_e, s_base_w;
    const int l = lane_id(), w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        long long be = 0, bw = 0;
        for (uint32_t b = 0; b < blockIdx.x; ++b) {
            be += sums[2 * b];
            bw += sums[2 * b + 1];
        }
        s_base_e = be;
        s_base_w = bw;
        if (blockIdx.x == gridDim.x - 1) {
            a.ctrl->heavy_entries = be + sums[2 * blockIdx.x];
            a.ctrl->heavy_words = bw + sums[2 * blockIdx.x + 1];
        }
    }
    __syncthreads();
    const int32_t lo = blockIdx.x * kHeavyChunk;
    const int32_t hi = min(nh, lo + kHeavyChunk);
    for (int32_t h0 = lo; h0 < hi; h0 += kHeavyThreads) {
        const int32_t h = h0 + static_cast<int32_t>(threadIdx.x);
        int32_t v;
        long long e, wd;
        heavy_sizes(a, h < hi ? h : nh, nh, v, e, wd);
        long long ie = e, iw = wd;  // warp inclusive scans
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long ye = __shfl_up_sync(kFull, ie, d), yw = __shfl_up_sync(kFull, iw, d);
            if (l >= d) {
                ie += ye;
                iw += yw;
            }
        }
        if (l == 31) {
            s_e[w] = ie;
            s_w[w] = iw;
        }
        __syncthreads();
        long long be = s_base_e, bw = s_base_w, te = 0, tw = 0;
        for (int k = 0; k < kHeavyThreads / 32; ++k) {
            if (k < w) {
                be += s_e[k];
                bw += s_w[k];
            }
            te += s_e[k];
            tw += s_w[k];
        }
        if (h < hi) {
            const HeavyRows& hr = *a.heavy;
            hr.hid[v] = h;
            hr.h_pbeg[h] = be + ie - e;
            hr.h_pcnt[h] = -1;
            hr.h_bbeg[h] = bw + iw - wd;
            hr.h_bwords[h] = static_cast<int32_t>(wd);
            if (hr.bref && (h < a.ctrl->init_cnt[0] || !hr.pull_warp)) hr.bref[v] = bitmap_ref(bw + iw - wd, wd);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base_e += te;
            s_base_w += tw;
        }
        __syncthreads();
    }
}

// Tile bookkeeping of one round, loaded by every block at kernel start.  In
// the tentative launch a block-bucket row needs only one warp (its color
// comes from its bitmap), so its tiles hold one row per warp there.
struct RoundTiles {
    int32_t cnt[kNB];
    int32_t start[kNB];
    int32_t prefix[kNB + 1];
};

__device__ __forceinline__ int round_tile(int b, bool warp_heavy) {
    return b == 0 && warp_heavy ? kWarps : bucket_tile(b);
}

__device__ __forceinline__ void load_round_tiles(const SpecCtrl* c, int par, bool warp_heavy,
                                                 RoundTiles& rt) {
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int b = 0; b < kNB; ++b) {
            rt.cnt[b] = c->cnt[par][b];
            rt.start[b] = c->start[b];
            rt.prefix[b] = acc;
            const int tile = round_tile(b, warp_heavy);
            acc += (rt.cnt[b] + tile - 1) / tile;
        }
        rt.prefix[kNB] = acc;
    }
    __syncthreads();
}

__device__ __forceinline__ int tile_bucket(const RoundTiles& rt, int32_t t) {
    int b = 0;
    while (t >= rt.prefix[b + 1]) ++b;
    return b;
}

// Colors fixed before the round (the snapshot); 0 = in the work set.
struct SnapshotFetch {
    const int32_t* color;
    __device__ __forceinline__ int32_t raw(int32_t u) const { return __ldg(color + u); }
    __device__ __forceinline__ int32_t resolve(int32_t, int32_t x) const { return x; }
};

// ---------------------------------------------------------------------------
// Keys, the total order and the heavy rows' bitmaps
// ---------------------------------------------------------------------------
// Bit 63 of a key marks a fixed vertex.  The conflict launch that fixes a
// vertex sets it while other blocks of that launch may still read the key,
// so every conflict test compares tentative colors with the bit masked off.
// A neighbor fixed before the round never matches a tentative color (the
// color was chosen against it), so the bit only tells the list scans which
// entries to drop.
constexpr uint64_t kKeyFixed = 1ull << 63;
__device__ __forceinline__ uint32_t key_tent(uint64_t k) {
    return static_cast<uint32_t>(k >> 32) & 0x7FFFFFFFu;
}
// u is above v in the random total order of Sec. 2.2: the larger priority,
// then the larger id.
__device__ __forceinline__ bool above(uint64_t ku, int32_t u, uint64_t kv, int32_t v) {
    const uint32_t pu = static_cast<uint32_t>(ku), pv = static_cast<uint32_t>(kv);
    return pu > pv || (pu == pv && u > v);
}

constexpr int kHeavyU = 4;  // list entries per thread per step of a heavy row
constexpr int kCompactEvery = 16;  // power of two
constexpr int kProbeMin = 4;       // lists longer than this many probes are probed
constexpr int kHeavyStep = kHeavyU * kBlock;

// Per-thread asynchronous 16-byte global -> shared copies (cp.async): a
// thread stages the 4 list entries it will process next while it works on
// the current ones, and waits only for its own copies (no barrier, no spin).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stages step `step` of a 16-byte aligned list (entries [i0, i0 +
// kHeavyStep), thread t the 4 at i0 + 4t) into buf.  A copy may read up to 3
// entries past cnt: lists are padded to 4 entries.
__device__ __forceinline__ void stage_step(int32_t* buf, const int32_t* lst, int64_t i0, int64_t cnt) {
    const int64_t i = i0 + 4 * static_cast<int64_t>(threadIdx.x);
    if (i < cnt) cp_async16(buf + 4 * threadIdx.x, lst + i);
    cp_async_commit();
}

// A vertex fixed at color c marks c in the bitmap of each heavy neighbor,
// where it stays forbidden for the neighbor's later rounds (a neighbor's
// bitmap thus holds the colors of all its neighbors fixed before the
// round).  Lanes lane0, lane0 + stride, ... take the row's entries; a bit
// already set is not written again.
__device__ __forceinline__ void mark_color(const SpecArgs& a, const HeavyRows& hr, int64_t beg,
                                           int32_t deg, int32_t c, int32_t lane0, int32_t stride) {
    const uint32_t bit = static_cast<uint32_t>(c - 1);
    const uint32_t mask = 1u << (bit & 31u);
    // the bucket bytes (L2-resident) first; the bitmap reference only for
    // heavy rows not fixed yet (a fixed heavy row's byte is kBucketFixed)
    for_each_nbr<2, uint32_t, false>(
        a.g, beg, deg, lane0, stride, [&](int32_t u) { return static_cast<uint32_t>(__ldcg(a.bucket + u)); },
        [&](int32_t u, uint32_t b) {
            if (b > hr.mark_bucket) return;
            const uint64_t r = __ldg(hr.bref + u);
            if (r == kNoBitmap || bit >= 32u * static_cast<uint32_t>(r & kRefWords)) return;
            uint32_t* w = hr.hbm + (r >> 24) + (bit >> 5);
            if (!(__ldcg(w) & mask)) atomicOr(w, mask);
        },
        &a.ctrl->err);
}

// ---------------------------------------------------------------------------
// Tentative coloring of W_r against the snapshot `color`
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_tent(const SpecArgs& a, int32_t v, int32_t c) {
    const uint64_t k = a.key[v];
    a.key[v] = (static_cast<uint64_t>(static_cast<uint32_t>(c)) << 32) | (k & 0xFFFFFFFFull);
}
template <int G, bool kRXF>
__device__ __forceinline__ void tentative_group_tile(const SpecArgs& a, const RoundTiles& rt,
                                                     const WorkItem* list, int b, int32_t first,
                                                     int32_t round, unsigned long long& edges) {
    const int gi = threadIdx.x / G, gl = threadIdx.x % G;
    const int32_t k = first + gi;
    const bool valid = k < rt.cnt[b];
    WorkItem it{0, 0, 0};
    uint32_t j = 0;
    if (valid) {
        it = load_item(list + rt.start[b] + k);
        if (kRXF) j = draw_index(a, it.v, round);
    }
    const SnapshotFetch fetch{a.color};
    // aligned 4-id reads, one chunk per lane per batch (measured: stencil coloring 1.40 ->
    // 1.35 ms, RMAT-Good 30.5 -> 28.6 ms; the recoloring keeps single-id reads)
    const int32_t c = choose_reg<G, 1, SnapshotFetch, true>(a.g, it.beg, it.deg, gl, j, fetch, &a.ctrl->err);
    if (valid && gl == 0) {
        set_tent(a, it.v, c);
        edges += static_cast<unsigned long long>(it.deg);
    }
}

// The j-th clear bit of a bitmap (bit b = color b + 1), one warp; -1: past it.
__device__ __forceinline__ int32_t choose_from_bitmap(const uint32_t* bm, int32_t words, uint32_t j) {
    const int l = lane_id();
    for (int32_t w0 = 0; w0 < words; w0 += 32) {
        const int32_t wi = w0 + l;
        const uint32_t f = wi < words ? ~__ldcg(bm + wi) : 0u;
        const uint32_t cnt_f = static_cast<uint32_t>(__popc(f));
        const uint32_t incl = warp_inclusive_scan(cnt_f);
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        if (j < total) {
            const uint32_t excl = incl - cnt_f;
            const bool mine = j >= excl && j < incl;
            const int owner = __ffs(__ballot_sync(kFull, mine)) - 1;
            int32_t color = 0;
            if (mine) color = 32 * wi + select_bit32(f, j - excl) + 1;
            return __shfl_sync(kFull, color, owner);
        }
        j -= total;
    }
    return -1;
}

// Heavy row v in round >= 1 (one warp): its bitmap holds the colors of
// every neighbor fixed before the round (marked by those neighbors).
__device__ int32_t choose_bitmap_warp(const HeavyRows& hr, int32_t v, uint32_t j) {
    const uint64_t r = hr.bref[v];
    return choose_from_bitmap(hr.hbm + (r >> 24), static_cast<int32_t>(r & kRefWords), j);
}

// Warp-bucket row v in round >= 1 (the whole warp): it keeps the list of its
// neighbors not fixed at its last look (the row itself before the first
// look) and a bitmap of the colors of the others.  It folds the neighbors
// fixed since into the bitmap (a shared window of 2048 colors, merged once)
// and drops them from the list, compacted in place with ballots (a batch's
// reads precede its writes, which land at or below every position the batch
// read); then it takes the j-th permissible color from the bitmap.  -1: past
// the bitmap.  The forbidden set is exactly that of a full row scan.
__device__ int32_t choose_warp_pending(const SpecArgs& a, const WorkItem& it, uint32_t j, uint32_t* sbm) {
    const int l = lane_id();
    const HeavyRows& hr = *a.heavy;
    const int32_t h = hr.hid[it.v];
    const int32_t pc = hr.h_pcnt[h];
    const int64_t cnt = pc < 0 ? static_cast<int64_t>(it.deg) : static_cast<int64_t>(pc);
    const int32_t* src = pc < 0 ? a.g.idx + it.beg : hr.pend + hr.h_pbeg[h];
    int32_t* dst = hr.pend + hr.h_pbeg[h];
    uint32_t* bm = hr.hbm + hr.h_bbeg[h];
    const int32_t words = hr.h_bwords[h];
    const uint32_t bits = 32u * static_cast<uint32_t>(words);
    const int32_t sw = min(words, kWarpBitmapWords);
    const uint32_t sbits = 32u * static_cast<uint32_t>(sw);
    for (int i = l; i < sw; i += 32) sbm[i] = 0u;
    __syncwarp();
    int32_t kept = 0;
    for (int64_t i0 = 0; i0 < cnt; i0 += kHeavyU * 32) {
        int32_t u[kHeavyU], c[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int64_t i = i0 + k * 32 + l;
            u[k] = i < cnt ? src[i] : -1;
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int64_t i = i0 + k * 32 + l;
            c[k] = -1;
            if (i < cnt) {
                if (u[k] < 0 || u[k] >= a.g.n) atomicOr(&a.ctrl->err, kErrBadGraph);
                else c[k] = __ldg(a.color + u[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            if (c[k] > 0) {
                const uint32_t b = static_cast<uint32_t>(c[k] - 1);
                if (b < sbits) atomicOr(&sbm[b >> 5], 1u << (b & 31));
                else if (b < bits) atomicOr(bm + (b >> 5), 1u << (b & 31));
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const unsigned bal = __ballot_sync(kFull, c[k] == 0);
            if (c[k] == 0) dst[kept + __popc(bal & ((1u << l) - 1u))] = u[k];
            kept += __popc(bal);
        }
    }
    if (l == 0) hr.h_pcnt[h] = kept;
    __syncwarp();
    for (int i = l; i < sw; i += 32) {
        const uint32_t x = sbm[i];
        if (x) bm[i] = __ldcg(bm + i) | x;  // the warp owns these words this round
    }
    __syncwarp();
    return choose_from_bitmap(bm, words, j);
}

template <bool kRXF>
__global__ void __launch_bounds__(kBlock, 5) k_tentative(SpecArgs a) {
    __shared__ uint32_t s_bm[kWarps][kWarpBitmapWords];
    __shared__ RoundTiles rt;
    const int32_t round = a.ctrl->round;
    const int par = round & 1;
    const WorkItem* list = par ? a.list1 : a.list0;
    if (blockIdx.x == 0 && threadIdx.x < kNB) a.ctrl->cnt[par ^ 1][threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->mark_cnt = 0;  // the last round's were marked
    if (round == 0) {  // tentative colors set with the priorities (every row counted once)
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicAdd(&a.ctrl->edges, static_cast<unsigned long long>(a.g.nnz));
        return;
    }
    load_round_tiles(a.ctrl, par, true, rt);
    unsigned long long edges = 0;
    const SnapshotFetch fetch{a.color};
    for (int32_t t = blockIdx.x; t < rt.prefix[kNB]; t += gridDim.x) {
        const int b = tile_bucket(rt, t);
        const int32_t first = (t - rt.prefix[b]) * round_tile(b, true);
        switch (b) {
        case 0:
        case 1: {  // heavy rows, one warp each
            const int w = threadIdx.x >> 5;
            const int32_t k = first + w;
            if (k < rt.cnt[b]) {
                const WorkItem it = load_item(list + rt.start[b] + k);
                const uint32_t j = kRXF ? draw_index(a, it.v, round) : 0u;
                // a marking row's item holds its list (ListItem), and the
                // conflict launch counts this visit's entries with its own
                const bool marked = b == 0 || !a.heavy->pull_warp;
                int32_t c = marked ? choose_bitmap_warp(*a.heavy, it.v, j) : choose_warp_pending(a, it, j, s_bm[w]);
                // past the bitmap's free colors (Random-X with a large X): the row in full
                if (c < 0) {
                    int64_t rbeg = it.beg;
                    int32_t rdeg = it.deg;
                    if (marked) row_of(a.g, it.v, rbeg, rdeg, &a.ctrl->err);
                    c = choose_warp<4>(a.g, rbeg, rdeg, j, fetch, s_bm[w], &a.ctrl->err);
                }
                if (lane_id() == 0) {
                    set_tent(a, it.v, c);
                    if (!marked) edges += static_cast<unsigned long long>(it.deg);
                }
            }
            break;
        }
        case 2: tentative_group_tile<32, kRXF>(a, rt, list, 2, first, round, edges); break;
        case 3: tentative_group_tile<16, kRXF>(a, rt, list, 3, first, round, edges); break;
        case 4: tentative_group_tile<8, kRXF>(a, rt, list, 4, first, round, edges); break;
        case 5: tentative_group_tile<4, kRXF>(a, rt, list, 5, first, round, edges); break;
        default: tentative_group_tile<2, kRXF>(a, rt, list, 6, first, round, edges); break;
        }
    }
    warp_add(&a.ctrl->edges, edges);
}

// ---------------------------------------------------------------------------
// Conflict detection; winners fix their color, losers go to W_{r+1}
// ---------------------------------------------------------------------------
// Does some neighbor in this lane's stripe have v's tentative color and a
// larger (priority, id)?  U gathers in flight.  Without heavy rows no key
// carries the fixed bit, and equal tentative colors make the keys order as
// the priorities.
template <int UC, bool kHeavy = true>
__device__ __forceinline__ bool loses(const SpecArgs& a, const WorkItem& it, int32_t lane0,
                                      int32_t stride) {
    if (it.deg == 0) return false;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint64_t kv = __ldg(key + it.v);
    const uint32_t tv = key_tent(kv);
    bool lose = false, loop = false;
    for_each_nbr<UC, uint64_t, true>(
        a.g, it.beg, it.deg, lane0, stride, [&](int32_t u) { return __ldg(key + u); },
        [&](int32_t u, uint64_t ku) {
            if (u == it.v) loop = true;  // uncolorable (Sec. 1): reported as a malformed graph
            else if (kHeavy ? key_tent(ku) == tv && above(ku, u, kv, it.v)
                            : static_cast<uint32_t>(ku >> 32) == tv && (ku > kv || (ku == kv && u > it.v)))
                lose = true;
        },
        &a.ctrl->err);
    if (loop) atomicOr(&a.ctrl->err, kErrBadGraph);
    return lose;
}

// ListItem: from round 1 on, the work item of a marking heavy row (a
// block-bucket row, or a warp-bucket row where the warp rows do not pull)
// holds its list instead of its row: beg = the list's start in pend, deg =
// its length.  A visit then reads the item, the list and the listed keys
// with no index lookups in between (before: item, heavy index, list start
// and length, list, keys); the row's bounds, needed only for the edge count
// and a winner's marks, are loaded beside the list (the conflict launch
// counts both launches' entries of such a row: every row of a round's work
// set is visited by both).  Round 0 reads rows from items of the usual form,
// and its losers write the new one.

// Round 0, a block-bucket row (the whole block): the conflict test over the
// full row, which also writes the row's list: its neighbors above it in the
// total order that are not fixed.  Only these can beat it in a later round.
// lbeg, lcnt: the list's start in pend and its length (block-uniform).
__device__ bool above_build_block(const SpecArgs& a, const HeavyRows& hr, const WorkItem& it,
                                  uint32_t* wsum, int64_t& lbeg, int32_t& lcnt) {
    const int t = threadIdx.x, l = lane_id(), w = t >> 5;
    const int32_t h = hr.hid[it.v];
    lbeg = hr.h_pbeg[h];
    int32_t* dst = hr.pend + lbeg;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint64_t kv = __ldg(key + it.v);
    const uint32_t tv = key_tent(kv);
    bool lose = false, loop = false;
    int32_t kept = 0;
    for (int64_t i0 = 0; i0 < it.deg; i0 += kHeavyStep) {
        int32_t u[kHeavyU];
        uint64_t ku[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int64_t i = i0 + static_cast<int64_t>(k) * kBlock + t;
            u[k] = i < it.deg ? load_nbr(a.g, it.beg + i, &a.ctrl->err) : -1;
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) ku[k] = u[k] >= 0 ? __ldg(key + u[k]) : 0ull;
        int32_t mine = 0;
        bool keep[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            keep[k] = false;
            if (u[k] < 0) continue;
            if (u[k] == it.v) {
                loop = true;
                continue;
            }
            const bool up = above(ku[k], u[k], kv, it.v);
            if (up && key_tent(ku[k]) == tv) lose = true;
            keep[k] = up && !(ku[k] & kKeyFixed);
            mine += keep[k];
        }
        const int32_t incl_w = static_cast<int32_t>(warp_inclusive_scan(static_cast<uint32_t>(mine)));
        if (l == 31) wsum[w] = static_cast<uint32_t>(incl_w);
        __syncthreads();
        int32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const int32_t x = static_cast<int32_t>(wsum[k]);
            if (k < w) before += x;
            total += x;
        }
        int32_t pos = kept + before + incl_w - mine;
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k)
            if (keep[k]) dst[pos++] = u[k];
        kept += total;
        __syncthreads();
    }
    lcnt = kept;
    if (loop) atomicOr(&a.ctrl->err, kErrBadGraph);
    return lose;
}

// Round >= 1, a block-bucket row: the conflict test over its list (the
// neighbors above it not fixed at its last look), dropping the entries fixed
// since, compacted in place (a kept entry moves to a position at or below
// the one it was read from, after the step's entries are staged).  The
// list's next step is staged while this one runs.  On a list longer
// than kProbeMin probes, a probe of the first kBlock entries comes first:
// most rows of a dense core lose every round,
// usually to one of the first entries, and a loss found there leaves the
// list as it is (still a superset of the neighbors above v not fixed).
// Every kCompactEvery-th round skips the probe, so that no list goes long
// uncompacted.  The item holds the list (see ListItem); lcnt: its length
// after the scan (block-uniform).
__device__ bool above_scan_block(const SpecArgs& a, const WorkItem& it, int32_t (*stage)[kHeavyStep],
                                 uint32_t* wsum, int32_t& lcnt) {
    const int t = threadIdx.x, l = lane_id(), w = t >> 5;
    const int64_t pc = it.deg;
    int32_t* lst = a.heavy->pend + it.beg;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint32_t tv = key_tent(__ldg(key + it.v));
    lcnt = static_cast<int32_t>(pc);
    if (pc > kProbeMin * kBlock && (a.ctrl->round & (kCompactEvery - 1)) != 0) {  // the probe
        bool hit = false;
        const int32_t u = lst[t];
        if (static_cast<uint32_t>(u) < static_cast<uint32_t>(a.g.n)) hit = key_tent(__ldg(key + u)) == tv;
        if (__syncthreads_or(hit)) return true;
    }
    bool lose = false;
    int32_t kept = 0;
    if (pc > 0) stage_step(stage[0], lst, 0, pc);
    int parity = 0;
    for (int64_t i0 = 0; i0 < pc; i0 += kHeavyStep, parity ^= 1) {
        const bool more = i0 + kHeavyStep < pc;
        if (more) stage_step(stage[parity ^ 1], lst, i0 + kHeavyStep, pc);
        if (more) cp_async_wait<1>(); else cp_async_wait<0>();
        int32_t u[kHeavyU];
        uint64_t ku[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int64_t i = i0 + 4 * static_cast<int64_t>(t) + k;
            u[k] = i < pc ? stage[parity][4 * t + k] : -1;
            ku[k] = 0;
            if (i < pc) {
                if (static_cast<uint32_t>(u[k]) >= static_cast<uint32_t>(a.g.n)) {
                    atomicOr(&a.ctrl->err, kErrBadGraph);
                    u[k] = -1;
                } else {
                    ku[k] = __ldg(key + u[k]);
                }
            }
        }
        int32_t mine = 0;
        bool keep[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            keep[k] = u[k] >= 0 && !(ku[k] & kKeyFixed);
            if (u[k] >= 0 && key_tent(ku[k]) == tv) lose = true;
            mine += keep[k];
        }
        const int32_t incl_w = static_cast<int32_t>(warp_inclusive_scan(static_cast<uint32_t>(mine)));
        if (l == 31) wsum[w] = static_cast<uint32_t>(incl_w);
        __syncthreads();  // also: the whole step is staged before any write
        int32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const int32_t x = static_cast<int32_t>(wsum[k]);
            if (k < w) before += x;
            total += x;
        }
        int32_t pos = kept + before + incl_w - mine;
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k)
            if (keep[k]) lst[pos++] = u[k];
        kept += total;
        __syncthreads();  // frees stage[parity] for the step after next
    }
    lcnt = kept;
    return lose;
}

// The two list passes of a warp-bucket row (the whole warp): round 0 builds
// the list from the row, later rounds scan and compact it (ballots; a
// batch's reads precede its writes, which land at or below every position
// the batch read), after a probe of the first 32 entries as in
// above_scan_block.
__device__ bool above_build_warp(const SpecArgs& a, const HeavyRows& hr, const WorkItem& it, int64_t& lbeg,
                                 int32_t& lcnt) {
    const int l = lane_id();
    const int32_t h = hr.hid[it.v];
    lbeg = hr.h_pbeg[h];
    int32_t* dst = hr.pend + lbeg;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint64_t kv = __ldg(key + it.v);
    const uint32_t tv = key_tent(kv);
    bool lose = false, loop = false;
    int32_t kept = 0;
    for (int32_t i0 = 0; i0 < it.deg; i0 += kHeavyU * 32) {
        int32_t u[kHeavyU];
        uint64_t ku[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int32_t i = i0 + k * 32 + l;
            u[k] = i < it.deg ? load_nbr(a.g, it.beg + i, &a.ctrl->err) : -1;
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) ku[k] = u[k] >= 0 ? __ldg(key + u[k]) : 0ull;
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            bool keep = false;
            if (u[k] == it.v) {
                loop = true;
            } else if (u[k] >= 0) {
                const bool up = above(ku[k], u[k], kv, it.v);
                if (up && key_tent(ku[k]) == tv) lose = true;
                keep = up && !(ku[k] & kKeyFixed);
            }
            const unsigned bal = __ballot_sync(kFull, keep);
            if (keep) dst[kept + __popc(bal & ((1u << l) - 1u))] = u[k];
            kept += __popc(bal);
        }
    }
    lcnt = kept;
    if (loop) atomicOr(&a.ctrl->err, kErrBadGraph);
    return __any_sync(kFull, lose);
}

__device__ bool above_scan_warp(const SpecArgs& a, const WorkItem& it, int32_t& lcnt) {
    const int l = lane_id();
    const int32_t pc = it.deg;
    int32_t* lst = a.heavy->pend + it.beg;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint32_t tv = key_tent(__ldg(key + it.v));
    lcnt = pc;
    if (pc > kProbeMin * 32 && (a.ctrl->round & (kCompactEvery - 1)) != 0) {  // the probe
        const int32_t u = lst[l];
        const bool hit = static_cast<uint32_t>(u) < static_cast<uint32_t>(a.g.n) &&
                         key_tent(__ldg(key + u)) == tv;
        if (__any_sync(kFull, hit)) return true;
    }
    bool lose = false;
    int32_t kept = 0;
    for (int32_t i0 = 0; i0 < pc; i0 += kHeavyU * 32) {
        int32_t u[kHeavyU];
        uint64_t ku[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int32_t i = i0 + k * 32 + l;
            u[k] = i < pc ? lst[i] : -1;
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            ku[k] = 0;
            if (u[k] >= a.g.n) {
                atomicOr(&a.ctrl->err, kErrBadGraph);
                u[k] = -1;
            } else if (u[k] >= 0) {
                ku[k] = __ldg(key + u[k]);
            }
        }
        __syncwarp();  // every read of the batch before any write
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            if (u[k] >= 0 && key_tent(ku[k]) == tv) lose = true;
            const bool keep = u[k] >= 0 && !(ku[k] & kKeyFixed);
            const unsigned bal = __ballot_sync(kFull, keep);
            if (keep) lst[kept + __popc(bal & ((1u << l) - 1u))] = u[k];
            kept += __popc(bal);
        }
    }
    lcnt = kept;
    return __any_sync(kFull, lose);
}

// The conflict test of a warp-bucket row after round 0 (the whole warp),
// over its list, which the round's tentative launch has just compacted: the
// neighbors not fixed before the round, the only ones that can share its
// tentative color.
__device__ bool loses_pending_warp(const SpecArgs& a, const WorkItem& it) {
    const HeavyRows& hr = *a.heavy;
    const int32_t h = hr.hid[it.v];
    const int32_t pc = hr.h_pcnt[h];
    const int32_t* lst = hr.pend + hr.h_pbeg[h];
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint64_t kv = __ldg(key + it.v);
    const uint32_t tv = key_tent(kv);
    const int l = lane_id();
    bool lose = false;
    for (int32_t i0 = 0; i0 < pc; i0 += kHeavyU * 32) {
        int32_t u[kHeavyU];
        uint64_t ku[kHeavyU];
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            const int32_t i = i0 + k * 32 + l;
            u[k] = i < pc ? __ldg(lst + i) : -1;
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k) {
            ku[k] = 0;
            if (u[k] >= a.g.n) {
                atomicOr(&a.ctrl->err, kErrBadGraph);
                u[k] = -1;
            } else if (u[k] >= 0) {
                ku[k] = __ldg(key + u[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kHeavyU; ++k)
            if (u[k] >= 0 && u[k] != it.v && key_tent(ku[k]) == tv && above(ku[k], u[k], kv, it.v))
                lose = true;
    }
    return __any_sync(kFull, lose);
}

// Whether a fixed vertex marks its heavy neighbors' bitmaps: only where the
// graph has heavy rows (in a batch, its own graph).
__device__ __forceinline__ bool marks_of(const SpecArgs& a, const HeavyRows& hr, int32_t v) {
    return hr.bref && (!hr.near || hr.near[v]) && (!a.graph_of || a.graph_heavy[a.graph_of[v]]);
}

// A winner (leader lane) fixes its color c, its key's tentative color: the
// color array and the fixed bit of its key.
template <bool kHeavy>
__device__ __forceinline__ void fix_color(const SpecArgs& a, int32_t v, int32_t c, bool leader,
                                          int32_t& my_max, int32_t round) {
    if (!leader) return;
    a.color[v] = c;
    if (kHeavy) {  // the fixed bit: read by the heavy rows' list scans only
        const HeavyRows& hr = *a.heavy;
        if (hr.bref && (!hr.near || hr.near[v])) a.key[v] |= kKeyFixed;
    }
    my_max = max(my_max, c);
    if (a.win_round) a.win_round[v] = round;
}

template <int G, bool kHeavy, bool kPending = false>
__device__ __forceinline__ void conflict_group_tile(const SpecArgs& a, const HeavyRows& hr,
                                                    const RoundTiles& rt, const WorkItem* list,
                                                    WorkItem* next, int par, int b, int32_t first,
                                                    int32_t round, int32_t& my_max,
                                                    unsigned long long& edges) {
    const int gi = threadIdx.x / G, gl = threadIdx.x % G;
    const int32_t k = first + gi;
    const bool valid = k < rt.cnt[b];
    WorkItem it{0, 0, 0};
    if (valid) it = load_item(list + rt.start[b] + k);
    bool lose;
    if constexpr (kPending) lose = valid && loses_pending_warp(a, it);  // G == 32: one warp per row
    else lose = group_any<G>(loses<1, kHeavy>(a, it, gl, G));  // one 4-id chunk per lane per batch
    const bool leader = valid && gl == 0;
    const bool win = valid && !lose;
    int32_t c = 0;
    if (leader) {
        edges += static_cast<unsigned long long>(it.deg);
        if (win) c = static_cast<int32_t>(key_tent(a.key[it.v])) * (kHeavy && marks_of(a, hr, it.v) ? -1 : 1);
    }
    fix_color<kHeavy>(a, it.v, c < 0 ? -c : c, leader && win, my_max, round);
    if (kHeavy && hr.bref) {  // c < 0: fixed at -c, marks
        c = __shfl_sync(kFull, c, lane_id() & ~(G - 1));
        if (win && c < 0) mark_color(a, hr, it.beg, it.deg, -c, gl, G);
    }
    warp_append(leader && lose, it.beg, it.v, it.deg, &a.ctrl->cnt[par ^ 1][b], next, rt.start[b]);
}

// Warp-bucket rows: one warp per row, over its list after round 0.
__device__ __forceinline__ void conflict_warp_tile(const SpecArgs& a, const HeavyRows& hr,
                                                   const RoundTiles& rt, const WorkItem* list,
                                                   WorkItem* next, int par, int32_t first,
                                                   int32_t round, int32_t& my_max,
                                                   unsigned long long& edges) {
    const int32_t k = first + (threadIdx.x >> 5);
    const bool valid = k < rt.cnt[1];  // the same for the whole warp
    WorkItem it{0, 0, 0};
    bool lose = false;
    int64_t rbeg = 0, lbeg = 0;  // the row (edge count, marks) and the list (next round's item)
    int32_t rdeg = 0, lcnt = 0;
    if (valid) {
        it = load_item(list + rt.start[1] + k);
        if (round == 0) {
            rbeg = it.beg;
            rdeg = it.deg;
            lose = above_build_warp(a, hr, it, lbeg, lcnt);
        } else {
            row_of(a.g, it.v, rbeg, rdeg, &a.ctrl->err);  // loaded beside the list
            lbeg = it.beg;
            lose = above_scan_warp(a, it, lcnt);
        }
    }
    const bool leader = valid && lane_id() == 0;
    const bool win = valid && !lose;
    int32_t c = 0;
    if (leader) {
        // from round 1 on also the round's tentative visit (ListItem)
        edges += static_cast<unsigned long long>(rdeg) * (round == 0 ? 1u : 2u);
        if (win) c = static_cast<int32_t>(key_tent(a.key[it.v]));
    }
    fix_color<true>(a, it.v, c, leader && win, my_max, round);
    if (leader && win) a.bucket[it.v] = kBucketFixed;
    if (hr.bref) {  // a warp-bucket row's graph has heavy rows: it marks
        c = __shfl_sync(kFull, c, 0);
        if (win) mark_color(a, hr, rbeg, rdeg, c, lane_id(), 32);
    }
    warp_append(leader && lose, lbeg, it.v, lcnt, &a.ctrl->cnt[par ^ 1][1], next, rt.start[1]);
}

// kHeavy = false: the form for graphs without heavy rows (buckets 0 and 1
// empty), with none of their code, nor marks or fixed bits.  kMinBlocks:
// resident blocks per SM the registers are budgeted for (measured: the
// light form and the pulling warp rows gain from 64 registers without
// spills, the marking form from the fifth block).
template <bool kHeavy, int kMinBlocks>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_conflict(SpecArgs a) {
    __shared__ RoundTiles rt;
    __shared__ bool s_last;
    __shared__ uint32_t s_wsum[kWarps];
    __shared__ int32_t s_c, s_pos, s_rdeg;
    __shared__ int64_t s_rbeg;
    __shared__ __align__(16) int32_t stage[2][kHeavyStep];  // block-bucket rows' next list step
    const int32_t round = a.ctrl->round;
    const int par = round & 1;
    const WorkItem* list = par ? a.list1 : a.list0;
    WorkItem* next = par ? a.list0 : a.list1;
    load_round_tiles(a.ctrl, par, false, rt);
    // only the blocks with a tile take part in closing the round (a round has
    // at least one tile: the rounds stop when the work set is empty)
    const uint32_t participants = static_cast<uint32_t>(min(static_cast<int32_t>(gridDim.x), rt.prefix[kNB]));
    if (blockIdx.x >= participants) return;
    const HeavyRows& hr = *a.heavy;  // bref == nullptr: no heavy rows, nothing to mark
    unsigned long long edges = 0;
    int32_t my_max = 0;
    for (int32_t t = blockIdx.x; t < rt.prefix[kNB]; t += gridDim.x) {
        const int b = tile_bucket(rt, t);
        const int32_t first = (t - rt.prefix[b]) * bucket_tile(b);
        if constexpr (kHeavy) {
            if (b == 0) {
            const WorkItem it = load_item(list + rt.start[0] + first);
            int64_t rbeg = it.beg, lbeg = it.beg;  // the row and the list (see ListItem)
            int32_t rdeg = it.deg, lcnt = 0;
            if (round != 0 && threadIdx.x == 0) row_of(a.g, it.v, rbeg, rdeg, &a.ctrl->err);
            const bool mine = round == 0 ? above_build_block(a, hr, it, s_wsum, lbeg, lcnt)
                                         : above_scan_block(a, it, stage, s_wsum, lcnt);
            const bool lose = __syncthreads_or(mine);
            if (threadIdx.x == 0) {
                // from round 1 on also the round's tentative visit (ListItem)
                edges += static_cast<unsigned long long>(rdeg) * (round == 0 ? 1u : 2u);
                s_rdeg = rdeg;
                s_rbeg = rbeg;
                if (lose) {
                    const int32_t pos = atomicAdd(&a.ctrl->cnt[par ^ 1][0], 1);
                    store_item(next + rt.start[0] + pos, lbeg, it.v, lcnt);
                } else {
                    s_c = static_cast<int32_t>(key_tent(a.key[it.v]));
                    fix_color<true>(a, it.v, s_c, true, my_max, round);
                    a.bucket[it.v] = kBucketFixed;
                    // the row's marks go to the grid-wide marking launch
                    const int32_t pieces = (rdeg + kMarkChunk - 1) / kMarkChunk;
                    s_pos = pieces ? atomicAdd(&a.ctrl->mark_cnt, pieces) : 0;
                }
            }
            __syncthreads();
            if (!lose) {
                const int32_t pieces = (s_rdeg + kMarkChunk - 1) / kMarkChunk;
                for (int32_t q = threadIdx.x; q < pieces && s_pos + q < hr.mark_cap; q += kBlock) {
                    const int32_t len = min(kMarkChunk, s_rdeg - q * kMarkChunk);
                    store_item(hr.mark + s_pos + q, s_rbeg + static_cast<int64_t>(q) * kMarkChunk, s_c, len);
                }
            }
            __syncthreads();  // s_c, s_pos and the stage buffers are reused by the next tile
            continue;
            }
            if (b == 1) {
                if (!hr.pull_warp) conflict_warp_tile(a, hr, rt, list, next, par, first, round, my_max, edges);
                else if (round == 0) conflict_group_tile<32, true>(a, hr, rt, list, next, par, 1, first, round, my_max, edges);
                else conflict_group_tile<32, true, true>(a, hr, rt, list, next, par, 1, first, round, my_max, edges);
                continue;
            }
        }
        switch (b) {
        case 2: conflict_group_tile<32, kHeavy>(a, hr, rt, list, next, par, 2, first, round, my_max, edges); break;
        case 3: conflict_group_tile<16, kHeavy>(a, hr, rt, list, next, par, 3, first, round, my_max, edges); break;
        case 4: conflict_group_tile<8, kHeavy>(a, hr, rt, list, next, par, 4, first, round, my_max, edges); break;
        case 5: conflict_group_tile<4, kHeavy>(a, hr, rt, list, next, par, 5, first, round, my_max, edges); break;
        default: conflict_group_tile<2, kHeavy>(a, hr, rt, list, next, par, 6, first, round, my_max, edges); break;
        }
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ctrl->max_color, my_max);

    // The last block to finish closes the round.
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.ctrl->done_blocks, 1u) == participants - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        volatile SpecCtrl* c = a.ctrl;
        int32_t total = 0;
        for (int b = 0; b < kNB; ++b) total += c->cnt[par ^ 1][b];
        c->active = total;
        c->conflicts += static_cast<unsigned long long>(total);
        c->round = round + 1;
        c->done_blocks = 0u;
        const bool over = total > 0 && round + 1 >= a.round_limit;
        if (over) c->err |= kErrRoundLimit;
        if (a.use_cond) cudaGraphSetConditional(a.cond, (total > 0 && !over) ? 1u : 0u);
    }
}

// Neighbors of the block-bucket rows (one block per row): the vertices that
// mark when only those rows are marked.
__global__ void __launch_bounds__(kBlock) k_near_block(SpecArgs a, uint8_t* near) {
    const int32_t rows = a.ctrl->init_cnt[0];
    for (int32_t q = blockIdx.x; q < rows; q += gridDim.x) {
        const WorkItem it = load_item(a.list0 + a.ctrl->start[0] + q);
        for (int32_t i = threadIdx.x; i < it.deg; i += kBlock) {
            const int32_t u = ld_stream(a.g.idx + it.beg + i);
            if (static_cast<uint32_t>(u) < static_cast<uint32_t>(a.g.n)) near[u] = 1;
        }
    }
}

// The marks of the round's block-bucket winners (their rows in pieces, one
// block per piece), before the next round's tentative launch reads them.
__global__ void __launch_bounds__(kBlock) k_mark_colors(SpecArgs a) {
    const int32_t pending = a.ctrl->mark_cnt;
    if (pending == 0) return;
    const HeavyRows& hr = *a.heavy;
    // (the capacity holds every piece of every block-bucket row: never cut)
    const int32_t cnt = static_cast<int32_t>(min(static_cast<int64_t>(pending), hr.mark_cap));
    for (int32_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const WorkItem it = load_item(hr.mark + q);  // v: the color, deg: the piece's length
        mark_color(a, hr, it.beg, it.deg, it.v, threadIdx.x, kBlock);
    }
}

__global__ void __launch_bounds__(kBlock) k_priorities(uint64_t seed, int64_t n, uint32_t* out) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < n; v += stride)
        out[v] = prio_of(seed, static_cast<int32_t>(v));
}

gc_status priorities_device(uint64_t seed, int64_t n, uint32_t* out, cudaStream_t s) {
    if (n == 0) return GC_OK;
    const int grid = static_cast<int>(std::min<int64_t>((n + kBlock - 1) / kBlock,
                                                        persistent_grid(current_tuning())));
    GC_LAUNCH(KID_PRIORITIES, s, k_priorities<<<grid, kBlock, 0, s>>>(seed, n, out));
    return cuda_status(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
namespace {
struct PinnedWord {
    int32_t* p = nullptr;
    PinnedWord() { cudaMallocHost(&p, sizeof(int32_t) * 16); }
};
thread_local PinnedWord t_pinned;
}  // namespace

// The rounds as one CUDA graph: a WHILE node whose body is {tentative,
// conflict}; the last block of the conflict kernel sets the condition from
// the size of the next work set, so no round waits for the host.
struct RoundsGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~RoundsGraph() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
};

// The conflict kernel's form: without heavy rows, with pulling warp rows, or
// with marks for both heavy buckets.
void* conflict_kernel(bool heavy, bool pull) {
    if (!heavy) return reinterpret_cast<void*>(k_conflict<false, 4>);
    return pull ? reinterpret_cast<void*>(k_conflict<true, 4>) : reinterpret_cast<void*>(k_conflict<true, 5>);
}

// heavy: the conflict kernel with the heavy rows' code, and the marking node.
gc_status build_rounds_graph(const SpecArgs& a, int32_t X, int grid_t, int grid_c, int grid_m,
                             bool heavy, bool pull, RoundsGraph& rg) {
    cudaGraph_t& graph = rg.graph;
    cudaGraphExec_t& exec = rg.exec;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle handle = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)];
    std::memset(cp_buf, 0, sizeof(cp_buf));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_buf);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    SpecArgs ga = a;
    ga.cond = handle;
    ga.use_cond = 1;
    void* args[] = {&ga};
    cudaGraphNode_t n1 = nullptr, n2 = nullptr, n3 = nullptr;
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaKernelNodeParams k1;
        std::memset(&k1, 0, sizeof(k1));
        k1.func = X > 1 ? reinterpret_cast<void*>(k_tentative<true>) : reinterpret_cast<void*>(k_tentative<false>);
        k1.gridDim = dim3(grid_t);
        k1.blockDim = dim3(kBlock);
        k1.kernelParams = args;
        cudaKernelNodeParams k2 = k1;
        k2.func = conflict_kernel(heavy, pull);
        k2.gridDim = dim3(grid_c);
        cudaKernelNodeParams k3 = k1;
        k3.func = reinterpret_cast<void*>(k_mark_colors);
        k3.gridDim = dim3(grid_m);
        e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2);
        if (e == cudaSuccess && heavy) e = cudaGraphAddKernelNode(&n3, body, &n2, 1, &k3);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    return cuda_status(e);
}

gc_status launch_rounds_graph(RoundsGraph& rg, cudaStream_t s) {
    prof_begin(KID_SPEC_GRAPH, s);
    const cudaError_t e = cudaGraphLaunch(rg.exec, s);
    prof_end(KID_SPEC_GRAPH, s);
    return cuda_status(e);  // the caller's read-back of the round state waits for it
}

// The speculative coloring; with graph_of / desc / win_round set, a batch.
struct PrioRule {
    int32_t kind = 0;
    const int32_t* rank = nullptr;
    const int32_t* old = nullptr;
};

static gc_status color_impl(const Graph& g, int32_t X, uint64_t seed, const int32_t* graph_of,
                            const BatchDesc* desc, int32_t ng, int32_t* win_round, const PrioRule& rule,
                            int32_t* colors_out, gc_stats* stats, cudaStream_t s) {
    if (g.n == 0) {
        if (stats) { std::memset(stats, 0, sizeof(*stats)); }
        return GC_OK;
    }
    if (!t_pinned.p) return GC_ERR_OOM;
    const int64_t n = g.n;
    Scratch sc_key, sc_l0, sc_l1, sc_bucket, sc_ctrl;
    if (!sc_key.alloc(n * 8, s) ||
        !sc_l0.alloc(n * sizeof(WorkItem), s) || !sc_l1.alloc(n * sizeof(WorkItem), s) ||
        !sc_bucket.alloc(n, s) || !sc_ctrl.alloc(sizeof(SpecCtrl), s))
        return GC_ERR_OOM;
    SpecArgs a;
    std::memset(&a, 0, sizeof(a));  // use_cond = 0: no WHILE node unless rounds_in_graph sets it
    a.g = g;
    a.X = X;
    a.seed = seed;
    a.tune = current_tuning();
    a.color = colors_out;
    a.key = sc_key.as<uint64_t>();
    a.bucket = sc_bucket.as<uint8_t>();
    a.list0 = sc_l0.as<WorkItem>();
    a.list1 = sc_l1.as<WorkItem>();
    a.ctrl = sc_ctrl.as<SpecCtrl>();
    a.graph_of = graph_of;
    a.desc = desc;
    a.win_round = win_round;
    Scratch sc_gh;
    if (graph_of) {
        if (!sc_gh.alloc(static_cast<size_t>(ng) * 4 + 4, s)) return GC_ERR_OOM;
        a.graph_heavy = sc_gh.as<int32_t>();
        cudaMemsetAsync(a.graph_heavy, 0, static_cast<size_t>(ng) * 4 + 4, s);
    }
    a.prio_kind = rule.kind;
    a.prio_rank = rule.rank;
    a.prio_old = rule.old;

    struct Events {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        Events() {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
        }
        ~Events() {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    } ev;
    const cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    cudaEventRecord(e0, s);
    cudaMemsetAsync(a.ctrl, 0, sizeof(SpecCtrl), s);
    const int grid_t = resident_grid(X > 1 ? k_tentative<true> : k_tentative<false>, a.tune);
    const int grid_cl = resident_grid(k_conflict<false, 4>, a.tune);
    const int grid_m = resident_grid(k_mark_colors, a.tune);
    const int setup_grid = static_cast<int>(
        std::min<int64_t>((n + kBlock - 1) / kBlock, resident_grid(k_spec_setup, a.tune)));
    Scratch sc_heavy;
    if (!sc_heavy.alloc(sizeof(HeavyRows), s)) return GC_ERR_OOM;
    a.heavy = sc_heavy.as<HeavyRows>();
    cudaMemsetAsync(a.heavy, 0, sizeof(HeavyRows), s);
    GC_LAUNCH(KID_SPEC_SETUP, s, k_spec_setup<<<setup_grid, kBlock, 0, s>>>(a));
    GC_LAUNCH(KID_SPEC_FILL, s, k_spec_fill<<<setup_grid, kBlock, 0, s>>>(a));
    gc_status st = GC_OK;
    a.round_limit = static_cast<int32_t>(std::min<int64_t>(n + 2, INT32_MAX));
    // the rounds' CUDA graph is built while the set-up kernels run
    RoundsGraph rg;
    if (a.tune.spec_graph && (st = build_rounds_graph(a, X, grid_t, grid_cl, grid_m, false, false, rg)) != GC_OK) return st;
    // heavy rows: their pending lists and bitmaps (sizes read back)
    Scratch sc_hid, sc_pbeg, sc_pcnt, sc_bbeg, sc_bwords, sc_pend, sc_hbm, sc_hsums, sc_bref, sc_mark, sc_near;
    bool heavy = false, pull = false;
    int grid_ch = 0;
    {
        SpecCtrl h0;
        cudaError_t ce = cudaMemcpyAsync(&h0, a.ctrl, sizeof(SpecCtrl), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_status(ce);
        if (h0.err) return status_from_err_bits(h0.err);
        if (h0.init_cnt[0] > 0 && h0.max_deg <= kPullAllMaxDeg && a.tune.warp_max_deg == kDefaultWarpMaxDeg) {
            // No row longer than kPullAllMaxDeg: every heavy row is a warp row
            // that pulls (folds its list of neighbors not yet fixed each
            // round) instead of being marked.  The marks' extra launch per
            // round and one pass per fixed vertex cost more than the folds
            // on such graphs (coloring on GB300: R-MAT 14 2.53 -> 1.93 ms,
            // R-MAT 16 4.28 -> 3.71 ms, RMAT-Bad 16 1.49 -> 1.36 ms; R-MAT 17,
            // max degree 15.7 K, 4.97 -> 5.48 ms the other way).  The set-up
            // runs again with the lifted threshold.
            a.tune.warp_max_deg = INT32_MAX;
            cudaMemsetAsync(a.ctrl, 0, sizeof(SpecCtrl), s);
            GC_LAUNCH(KID_SPEC_SETUP, s, k_spec_setup<<<setup_grid, kBlock, 0, s>>>(a));
            GC_LAUNCH(KID_SPEC_FILL, s, k_spec_fill<<<setup_grid, kBlock, 0, s>>>(a));
            ce = cudaMemcpyAsync(&h0, a.ctrl, sizeof(SpecCtrl), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return cuda_status(ce);
            if (h0.err) return status_from_err_bits(h0.err);
        }
        const int32_t nh = h0.init_cnt[0] + h0.init_cnt[1];  // block- and warp-bucket rows
        heavy = nh > 0;
        if (heavy) {
            // a small share of the entries in block-bucket rows: the warp-bucket
            // rows fold their own bitmaps, and only the block-bucket rows'
            // neighbors mark
            const bool pull_warp = h0.block_entries * kPullShare < static_cast<unsigned long long>(g.nnz);
            pull = pull_warp;
            grid_ch = pull ? resident_grid(k_conflict<true, 4>, a.tune) : resident_grid(k_conflict<true, 5>, a.tune);
            const bool marks = !pull_warp || h0.init_cnt[0] > 0;
            const bool near = pull_warp && h0.init_cnt[0] > 0;
            if (!sc_hid.alloc(n * 4, s) || !sc_pbeg.alloc(static_cast<int64_t>(nh) * 8, s) ||
                !sc_pcnt.alloc(static_cast<int64_t>(nh) * 4, s) || !sc_bbeg.alloc(static_cast<int64_t>(nh) * 8, s) ||
                !sc_bwords.alloc(static_cast<int64_t>(nh) * 4, s) || (marks && !sc_bref.alloc(n * 8, s)) ||
                (near && !sc_near.alloc(n, s)))
                return GC_ERR_OOM;
            HeavyRows hr1{};
            hr1.pull_warp = pull_warp ? 1 : 0;
            hr1.mark_bucket = pull_warp ? 0 : 1;
            hr1.near = sc_near.as<uint8_t>();
            if (near) {
                cudaMemsetAsync(hr1.near, 0, static_cast<size_t>(n), s);
                const int grid = std::min(h0.init_cnt[0], resident_grid(k_near_block, a.tune));
                GC_LAUNCH(KID_SPEC_FILL, s, k_near_block<<<grid, kBlock, 0, s>>>(a, hr1.near));
            }
            hr1.hid = sc_hid.as<int32_t>();
            hr1.h_pbeg = sc_pbeg.as<int64_t>();
            hr1.h_pcnt = sc_pcnt.as<int32_t>();
            hr1.h_bbeg = sc_bbeg.as<int64_t>();
            hr1.h_bwords = sc_bwords.as<int32_t>();
            hr1.bref = sc_bref.as<uint64_t>();  // nullptr: nothing is marked
            ce = marks ? cudaMemsetAsync(hr1.bref, 0xFF, static_cast<size_t>(n) * 8, s) : cudaSuccess;  // kNoBitmap
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(a.heavy, &hr1, sizeof(HeavyRows), cudaMemcpyHostToDevice, s);
            if (ce != cudaSuccess) return cuda_status(ce);
            const int hblocks = static_cast<int>((static_cast<int64_t>(nh) + kHeavyChunk - 1) / kHeavyChunk);
            if (!sc_hsums.alloc(static_cast<int64_t>(hblocks) * 16, s)) return GC_ERR_OOM;
            GC_LAUNCH(KID_SPEC_FILL, s, k_heavy_sums<<<hblocks, kHeavyThreads, 0, s>>>(a, nh, sc_hsums.as<long long>()));
            GC_LAUNCH(KID_SPEC_FILL, s,
                      k_heavy_setup<<<hblocks, kHeavyThreads, 0, s>>>(a, nh, sc_hsums.as<long long>()));
            ce = cudaMemcpyAsync(&h0, a.ctrl, sizeof(SpecCtrl), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return cuda_status(ce);
            // marking pieces: at most one per kMarkChunk entries, plus one, per row
            const int64_t mark_cap = h0.heavy_entries / kMarkChunk + h0.init_cnt[0] + 1;
            if (!sc_pend.alloc(static_cast<size_t>(h0.heavy_entries) * 4, s) ||
                !sc_hbm.alloc(static_cast<size_t>(h0.heavy_words) * 4, s) ||
                !sc_mark.alloc(static_cast<size_t>(mark_cap) * sizeof(WorkItem), s))
                return GC_ERR_OOM;
            HeavyRows hr2 = hr1;
            hr2.pend = sc_pend.as<int32_t>();
            hr2.hbm = sc_hbm.as<uint32_t>();
            hr2.mark = sc_mark.as<WorkItem>();
            hr2.mark_cap = mark_cap;
            ce = cudaMemsetAsync(hr2.hbm, 0, static_cast<size_t>(h0.heavy_words) * 4, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(a.heavy, &hr2, sizeof(HeavyRows), cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return cuda_status(ce);
            if (a.tune.spec_graph) {  // the graph of the heavy form instead
                rg.reset();
                if ((st = build_rounds_graph(a, X, grid_t, grid_ch, grid_m, true, pull, rg)) != GC_OK) return st;
            }
        }
    }
    if (a.tune.spec_graph) {
        st = launch_rounds_graph(rg, s);
    } else {
        int32_t rounds = 0;
        for (;;) {
            if (X > 1) GC_LAUNCH(KID_TENTATIVE, s, k_tentative<true><<<grid_t, kBlock, 0, s>>>(a));
            else GC_LAUNCH(KID_TENTATIVE, s, k_tentative<false><<<grid_t, kBlock, 0, s>>>(a));
            if (heavy && pull) GC_LAUNCH(KID_CONFLICT, s, k_conflict<true, 4><<<grid_ch, kBlock, 0, s>>>(a));
            else if (heavy) GC_LAUNCH(KID_CONFLICT, s, k_conflict<true, 5><<<grid_ch, kBlock, 0, s>>>(a));
            else GC_LAUNCH(KID_CONFLICT, s, k_conflict<false, 4><<<grid_cl, kBlock, 0, s>>>(a));
            if (heavy) GC_LAUNCH(KID_MARK, s, k_mark_colors<<<grid_m, kBlock, 0, s>>>(a));
            ++rounds;
            cudaMemcpyAsync(t_pinned.p, &a.ctrl->active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            cudaError_t ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) { st = cuda_status(ce); break; }
            if (t_pinned.p[0] == 0) break;
            if (rounds >= a.round_limit) { st = GC_ERR_ROUND_LIMIT; break; }
        }
    }
    cudaEventRecord(e1, s);
    SpecCtrl h;
    cudaError_t ce = cudaMemcpyAsync(&h, a.ctrl, sizeof(SpecCtrl), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess && st == GC_OK) st = cuda_status(ce);
    if (st == GC_OK) st = status_from_err_bits(h.err);
    if (a.tune.spec_graph) note_launches((heavy ? 3 : 2) * static_cast<int64_t>(h.round));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = h.round;
        stats->max_color = h.max_color;
        stats->edges_examined = static_cast<int64_t>(h.edges);
        stats->conflicts = static_cast<int64_t>(h.conflicts);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_color = ms;
    }
    return st;
}

gc_status color_device(const Graph& g, int32_t X, uint64_t seed, int32_t* colors_out,
                       gc_stats* stats, cudaStream_t s) {
    return color_impl(g, X, seed, nullptr, nullptr, 0, nullptr, PrioRule{}, colors_out, stats, s);
}

gc_status color_lf_device(const Graph& g, int32_t X, uint64_t seed, int32_t* colors_out,
                          gc_stats* stats, cudaStream_t s) {
    PrioRule r;
    r.kind = 1;
    return color_impl(g, X, seed, nullptr, nullptr, 0, nullptr, r, colors_out, stats, s);
}

// aRC (Sec. 3): every iteration colors the graph again by the speculative
// First-Fit rounds, the vertices of earlier classes (in the iteration's
// permutation of the previous coloring's classes) winning their conflicts.
gc_status recolor_async_device(const Graph& g, const int32_t* colors_in, int32_t perm, int32_t iterations,
                               uint64_t seed, int32_t* colors_out, int32_t* ncolors_per_iter,
                               gc_stats* stats, cudaStream_t s) {
    const int64_t n = g.n;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    Scratch sc_old;
    if (!sc_old.alloc(n * 4, s)) return GC_ERR_OOM;
    int32_t* old = sc_old.as<int32_t>();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    gc_status st = GC_OK;
    int32_t maxc = 0;
    // the input: proper, and its max color (no iteration: copied through)
    st = class_ranks_device(g, colors_in, false, perm, 0, seed, nullptr, &maxc, s);
    if (st == GC_OK && ncolors_per_iter) ncolors_per_iter[0] = n > 0 ? maxc : 0;
    const int32_t* cur = colors_in;
    for (int32_t it = 0; it < iterations && st == GC_OK && n > 0; ++it) {
        cudaError_t ce = cudaMemcpyAsync(old, cur, n * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) { st = cuda_status(ce); break; }
        Scratch sc_rank;
        if (!sc_rank.alloc((static_cast<int64_t>(maxc) + 1) * 4, s)) { st = GC_ERR_OOM; break; }
        int32_t m = 0;
        st = class_ranks_device(g, old, true, perm, it, seed, sc_rank.as<int32_t>(), &m, s);
        if (st != GC_OK) break;
        PrioRule r;
        r.kind = 2;
        r.rank = sc_rank.as<int32_t>();
        r.old = old;
        gc_stats cs;
        st = color_impl(g, 1, seed, nullptr, nullptr, 0, nullptr, r, colors_out, &cs, s);
        if (st != GC_OK) break;
        maxc = cs.max_color;
        if (ncolors_per_iter) ncolors_per_iter[it + 1] = maxc;
        if (stats) {
            stats->rounds += cs.rounds;
            stats->edges_examined += cs.edges_examined;
            stats->conflicts += cs.conflicts;
        }
        cur = colors_out;
    }
    if (st == GC_OK && iterations == 0 && n > 0 && colors_out != colors_in) {
        const cudaError_t ce = cudaMemcpyAsync(colors_out, colors_in, n * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) st = cuda_status(ce);
    }
    if (st == GC_OK && n == 0 && ncolors_per_iter)
        for (int32_t i = 0; i <= iterations; ++i) ncolors_per_iter[i] = 0;
    cudaEventRecord(e1, s);
    const cudaError_t ce = cudaEventSynchronize(e1);
    if (st == GC_OK && ce != cudaSuccess) st = cuda_status(ce);
    if (stats) {
        stats->iterations = iterations;
        stats->max_color = maxc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_recolor = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
// Graph of every vertex, by binary search over the graphs' first vertices.
__global__ void __launch_bounds__(kBlock) k_graph_of(int64_t n, const BatchDesc* desc, int32_t ng,
                                                     int32_t* graph_of) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < n; v += stride) {
        int lo = 0, hi = ng - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (desc[mid].base <= v) lo = mid; else hi = mid - 1;
        }
        graph_of[v] = lo;
    }
}

// Per-graph max of a color array and of the winning rounds (+1); graphs are
// contiguous, so a warp mostly covers one or two of them.
__global__ void __launch_bounds__(kBlock) k_batch_stats(int64_t n, const int32_t* graph_of,
                                                        const int32_t* colors, const int32_t* win_round,
                                                        int32_t* g_maxc, int32_t* g_rounds) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; v < n; v += stride) {
        const int32_t gi = graph_of[v];
        int32_t c = colors[v];
        int32_t r = win_round ? win_round[v] + 1 : 0;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, gi);
        c = __reduce_max_sync(peers, c);
        r = __reduce_max_sync(peers, r);
        if (lane_id() == __ffs(peers) - 1) {
            atomicMax(&g_maxc[gi], c);
            if (g_rounds) atomicMax(&g_rounds[gi], r);
        }
    }
}

gc_status batch_layout(const Graph& g, const gc_batch_graph* graphs, int32_t ng, int32_t* max_x) {
    if (ng < 1 || !graphs) return GC_ERR_INVALID_ARG;
    int64_t next = 0;
    int32_t mx = 1;
    for (int32_t i = 0; i < ng; ++i) {
        const gc_batch_graph& d = graphs[i];
        if (d.vertex_base != next || d.n < 0 || d.X < 1 || d.iterations < 0 || !perm_valid(d.perm))
            return GC_ERR_INVALID_ARG;
        next += d.n;
        mx = std::max(mx, d.X);
    }
    if (next != g.n) return GC_ERR_INVALID_ARG;
    *max_x = mx;
    return GC_OK;
}

gc_status batch_graph_of(const Graph& g, const BatchDesc* d_desc, int32_t ng, int32_t* graph_of,
                         cudaStream_t s) {
    if (g.n == 0) return GC_OK;
    const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(g.n) + kBlock - 1) / kBlock,
                                                        persistent_grid(current_tuning())));
    GC_LAUNCH(KID_BATCH, s, k_graph_of<<<grid, kBlock, 0, s>>>(g.n, d_desc, ng, graph_of));
    return GC_OK;
}

gc_status batch_max_colors(const Graph& g, const int32_t* graph_of, const int32_t* colors,
                           const int32_t* win_round, int32_t ng, int32_t* max_color_out,
                           int32_t* rounds_out, cudaStream_t s) {
    Scratch sm, sr;
    if (!sm.alloc(ng * 4, s) || !sr.alloc(ng * 4, s)) return GC_ERR_OOM;
    cudaMemsetAsync(sm.p, 0, ng * 4, s);
    cudaMemsetAsync(sr.p, 0, ng * 4, s);
    if (g.n > 0) {
        const int grid = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(g.n) + kBlock - 1) / kBlock,
                                                            persistent_grid(current_tuning())));
        GC_LAUNCH(KID_BATCH, s,
                  k_batch_stats<<<grid, kBlock, 0, s>>>(g.n, graph_of, colors, win_round,
                                                         sm.as<int32_t>(), win_round ? sr.as<int32_t>() : nullptr));
    }
    cudaError_t e = cudaSuccess;
    if (max_color_out) e = cudaMemcpyAsync(max_color_out, sm.p, ng * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && rounds_out)
        e = cudaMemcpyAsync(rounds_out, sr.p, ng * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

gc_status color_batch_device(const Graph& g, const gc_batch_graph* graphs, int32_t ng,
                             int32_t* colors_out, int32_t* rounds_out, int32_t* max_color_out,
                             gc_stats* stats, cudaStream_t s) {
    int32_t max_x = 1;
    gc_status st = batch_layout(g, graphs, ng, &max_x);
    if (st != GC_OK) return st;
    static_assert(sizeof(BatchDesc) == sizeof(gc_batch_graph), "descriptor layout");
    Scratch sd, sgo, swr;
    if (!sd.alloc(static_cast<size_t>(ng) * sizeof(BatchDesc), s) || !sgo.alloc(static_cast<int64_t>(g.n) * 4 + 4, s) ||
        !swr.alloc(static_cast<int64_t>(g.n) * 4 + 4, s))
        return GC_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(sd.p, graphs, static_cast<size_t>(ng) * sizeof(BatchDesc),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    const BatchDesc* d_desc = sd.as<BatchDesc>();
    int32_t* graph_of = sgo.as<int32_t>();
    batch_graph_of(g, d_desc, ng, graph_of, s);
    st = color_impl(g, max_x, 0, graph_of, d_desc, ng, swr.as<int32_t>(), PrioRule{}, colors_out, stats, s);
    if (st != GC_OK) return st;
    if (rounds_out || max_color_out)
        st = batch_max_colors(g, graph_of, colors_out, swr.as<int32_t>(), ng, max_color_out, rounds_out, s);
    return st;
}

}  // namespace gc
