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
// Rows longer than warp_max_deg ("hubs") are split into chunks of 1024
// neighbors, one work item and one block tile each, so a hub's scan is spread
// over many blocks.  In the tentative phase every chunk ORs the colors it sees
// into the hub's forbidden bitmap in global memory and the block finishing the
// last chunk picks the color; in the conflict phase the chunks OR a lose flag
// and the last one decides (keep the color, or re-queue every chunk).
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
    unsigned long long edges;
    unsigned long long conflicts;
    int32_t hub_cnt[2];     // hub vertices in the work list of parity p
    int32_t n_hubs;         // rows split into chunks (set-up)
    int32_t hub_next;       // slot bump (fill)
    unsigned long long hub_words;       // bitmap words needed (set-up)
    unsigned long long hub_words_used;  // bitmap bump (fill)
    int32_t bad_where;                  // first failed internal check: site and index
    int32_t pad2;
    long long bad_index;
};

constexpr int32_t kSpecChunk = 1024;  // neighbors per chunk of a hub row

__host__ __device__ inline int32_t spec_chunks(int32_t deg) { return (deg + kSpecChunk - 1) / kSpecChunk; }
// Forbidden-bitmap words of a hub: the color chosen is at most deg + X.
__host__ __device__ inline int64_t hub_bitmap_words(int32_t deg, int32_t X) {
    return (static_cast<int64_t>(deg) + X + 31) / 32 + 1;
}

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
    // hub rows: vertex, row start, degree, chunk count, bitmap offset, chunks
    // finished in the current phase, lose flag, forbidden bitmaps
    int32_t* hub_v;
    int64_t* hub_beg;
    int32_t* hub_deg;
    int32_t* hub_nch;
    int64_t* hub_off;
    int32_t* hub_done;
    int32_t* hub_lose;
    uint32_t* hub_bm;
    int32_t n_hubs;           // slots allocated
    int64_t hub_words_total;  // bitmap words allocated
    int64_t list_len;         // entries of each work list
};

// Internal index checks: a failed one records where, skips the access and
// makes the call return GC_ERR_CUDA-free GC_ERR_BAD_GRAPH-like status.
__device__ __forceinline__ bool check_index(const SpecArgs& a, bool ok, int where, long long idx) {
    if (ok) return true;
    if (atomicOr(&a.ctrl->err, kErrInternal) == 0u || true) {
        if (atomicCAS(&a.ctrl->bad_where, 0, where) == 0) a.ctrl->bad_index = idx;
    }
    return false;
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
        const int b = bucket_of(deg, a.X, a.tune);
        a.bucket[v] = static_cast<uint8_t>(b);
        a.key[v] = prio_of(a.seed, v);  // tentative color 0
        a.color[v] = 0;
        if (b == 0) {
            atomicAdd(&a.ctrl->init_cnt[0], spec_chunks(deg));
            atomicAdd(&a.ctrl->n_hubs, 1);
            atomicAdd(&a.ctrl->hub_words, static_cast<unsigned long long>(hub_bitmap_words(deg, a.X)));
        } else {
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, b);
            const int leader = __ffs(peers) - 1;
            if (lane_id() == leader) atomicAdd(&a.ctrl->init_cnt[b], __popc(peers));
        }
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
            a.ctrl->active = static_cast<int32_t>(a.g.n);
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
        if (b == 0) {
            const int32_t slot = atomicAdd(&a.ctrl->hub_next, 1);
            const int32_t nch = spec_chunks(deg);
            if (!check_index(a, slot < a.n_hubs, 1, slot)) continue;
            a.hub_v[slot] = v;
            a.hub_beg[slot] = beg;
            a.hub_deg[slot] = deg;
            a.hub_nch[slot] = nch;
            a.hub_off[slot] = static_cast<int64_t>(
                atomicAdd(&a.ctrl->hub_words_used, static_cast<unsigned long long>(hub_bitmap_words(deg, a.X))));
            a.hub_done[slot] = 0;
            a.hub_lose[slot] = 0;
            const int32_t pos = atomicAdd(&a.ctrl->cnt[0][0], nch);
            if (!check_index(a, a.hub_off[slot] + hub_bitmap_words(deg, a.X) <= a.hub_words_total, 2,
                             a.hub_off[slot]))
                continue;
            if (!check_index(a, pos + nch <= a.ctrl->init_cnt[0] &&
                                    s_start[0] + static_cast<int64_t>(pos) + nch <= a.list_len, 3, pos))
                continue;
            for (int32_t c = 0; c < nch; ++c)
                store_item(a.list0 + s_start[0] + pos + c, beg + static_cast<int64_t>(c) * kSpecChunk,
                           -(slot + 1), min(kSpecChunk, deg - c * kSpecChunk));
            atomicAdd(&a.ctrl->hub_cnt[0], 1);
        } else {
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, b);
            const int leader = __ffs(peers) - 1;
            int32_t base = 0;
            if (lane_id() == leader) base = atomicAdd(&a.ctrl->cnt[0][b], __popc(peers));
            base = __shfl_sync(peers, base, leader);
            const int64_t at = s_start[b] + static_cast<int64_t>(base) + __popc(peers & ((1u << lane_id()) - 1u));
            if (check_index(a, at < a.list_len, 4, at)) store_item(a.list0 + at, beg, v, deg);
        }
    }
}

// Tile bookkeeping of one round, loaded by every block at kernel start.
struct RoundTiles {
    int32_t cnt[kNB];
    int32_t start[kNB];
    int32_t prefix[kNB + 1];
};

__device__ __forceinline__ void load_round_tiles(const SpecCtrl* c, int par, RoundTiles& rt) {
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int b = 0; b < kNB; ++b) {
            rt.cnt[b] = c->cnt[par][b];
            rt.start[b] = c->start[b];
            rt.prefix[b] = acc;
            acc += (rt.cnt[b] + bucket_tile(b) - 1) / bucket_tile(b);
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

union SpecShared {
    BlockScratch blk;
    uint32_t warp_bm[kWarps][kWarpBitmapWords];
};

// Colors fixed before the round (the snapshot); 0 = in the work set.
struct SnapshotFetch {
    const int32_t* color;
    __device__ __forceinline__ int32_t raw(int32_t u) const { return __ldg(color + u); }
    __device__ __forceinline__ int32_t resolve(int32_t, int32_t x) const { return x; }
};

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
        if (kRXF) j = scale_index(rxf_word(a.seed, it.v, round), static_cast<uint32_t>(a.X));
    }
    const SnapshotFetch fetch{a.color};
    const int32_t c = choose_reg<G, LanesUnroll<G>::U>(a.g, it.beg, it.deg, gl, j, fetch, &a.ctrl->err);
    if (valid && gl == 0) {
        set_tent(a, it.v, c);
        edges += static_cast<unsigned long long>(it.deg);
    }
}

// j-th (0-based) clear bit of a global bitmap of `words` words, as a color
// (bit c-1 <-> color c).  Whole block.
__device__ __forceinline__ int32_t select_zero_global(const uint32_t* bm, int64_t words, uint32_t j,
                                                      BlockScratch& s) {
    const int t = threadIdx.x, l = lane_id(), w = t >> 5;
    for (int64_t w0 = 0; w0 < words; w0 += kBlock) {
        const int64_t wi = w0 + t;
        const uint32_t f = wi < words ? ~__ldcg(bm + wi) : 0u;
        const uint32_t cnt = __popc(f);
        const uint32_t incl_w = warp_inclusive_scan(cnt);
        if (l == 31) s.wsum[w] = incl_w;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int i = 0; i < kWarps; ++i) {
            const uint32_t x = s.wsum[i];
            if (i < w) before += x;
            total += x;
        }
        const uint32_t incl = incl_w + before, excl = incl - cnt;
        if (j < total) {
            if (j >= excl && j < incl) s.result = static_cast<int32_t>(wi * 32) + select_bit32(f, j - excl) + 1;
            __syncthreads();
            const int32_t c = s.result;
            __syncthreads();
            return c;
        }
        j -= total;
        __syncthreads();
    }
    return static_cast<int32_t>(words * 32);  // unreachable: the bitmap has more than j clear bits
}

// One chunk of a hub row in the tentative phase (whole block).
template <bool kRXF>
__device__ __forceinline__ void tentative_chunk(const SpecArgs& a, const WorkItem& it, int32_t round,
                                                BlockScratch& s, unsigned long long& edges) {
    const int t = threadIdx.x;
    const int32_t slot = -it.v - 1;
    // a bad slot or bitmap range is recorded and the chunk skipped (uniform)
    if (!(slot >= 0 && slot < a.n_hubs)) {
        if (t == 0) check_index(a, false, 5, slot);
        return;
    }
    const int32_t v = a.hub_v[slot];
    const int64_t words = hub_bitmap_words(a.hub_deg[slot], a.X);
    if (!(a.hub_off[slot] >= 0 && a.hub_off[slot] + words <= a.hub_words_total &&
          static_cast<uint32_t>(v) < static_cast<uint32_t>(a.g.n))) {
        if (t == 0) check_index(a, false, 6, a.hub_off[slot]);
        return;
    }
    uint32_t* bm = a.hub_bm + a.hub_off[slot];
    const SnapshotFetch fetch{a.color};
    for (int64_t w0 = 0; w0 < words; w0 += kBlockBitmapWords) {
        for (int i = t; i < kBlockBitmapWords; i += kBlock) s.bm[i] = 0u;
        __syncthreads();
        const int64_t base = w0 * 32 + 1;
        scan_row<1>(a.g, it.beg, it.deg, t, kBlock, fetch,
                    [&](int32_t c) {
                        const int64_t d = static_cast<int64_t>(c) - base;
                        if (c > 0 && d >= 0 && d < 32 * kBlockBitmapWords)
                            atomicOr(&s.bm[d >> 5], 1u << (d & 31));
                    },
                    &a.ctrl->err);
        __syncthreads();
        for (int i = t; i < kBlockBitmapWords && w0 + i < words; i += kBlock)
            if (s.bm[i]) atomicOr(&bm[w0 + i], s.bm[i]);
        __syncthreads();
    }
    __threadfence();
    if (t == 0) s.result = atomicAdd(&a.hub_done[slot], 1) == a.hub_nch[slot] - 1;
    __syncthreads();
    const bool last = s.result != 0;
    __syncthreads();
    if (t == 0) edges += static_cast<unsigned long long>(it.deg);
    if (!last) return;
    __threadfence();
    const uint32_t j = kRXF ? scale_index(rxf_word(a.seed, v, round), static_cast<uint32_t>(a.X)) : 0u;
    const int32_t c = select_zero_global(bm, words, j, s);
    if (t == 0) {
        set_tent(a, v, c);
        a.hub_done[slot] = 0;
    }
}

template <bool kRXF>
__global__ void __launch_bounds__(kBlock, 5) k_tentative(SpecArgs a) {
    __shared__ SpecShared sm;
    __shared__ RoundTiles rt;
    const int32_t round = a.ctrl->round;
    const int par = round & 1;
    const WorkItem* list = par ? a.list1 : a.list0;
    if (blockIdx.x == 0 && threadIdx.x < kNB) a.ctrl->cnt[par ^ 1][threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->hub_cnt[par ^ 1] = 0;
    load_round_tiles(a.ctrl, par, rt);
    unsigned long long edges = 0;
    const SnapshotFetch fetch{a.color};
    for (int32_t t = blockIdx.x; t < rt.prefix[kNB]; t += gridDim.x) {
        const int b = tile_bucket(rt, t);
        const int32_t first = (t - rt.prefix[b]) * bucket_tile(b);
        switch (b) {
        case 0:
            tentative_chunk<kRXF>(a, load_item(list + rt.start[0] + first), round, sm.blk, edges);
            break;
        case 1: {
            const int w = threadIdx.x >> 5;
            const int32_t k = first + w;
            if (k < rt.cnt[1]) {
                const WorkItem it = load_item(list + rt.start[1] + k);
                const uint32_t j = kRXF ? scale_index(rxf_word(a.seed, it.v, round), a.X) : 0u;
                const int32_t c = choose_warp<4>(a.g, it.beg, it.deg, j, fetch, sm.warp_bm[w], &a.ctrl->err);
                if (lane_id() == 0) {
                    set_tent(a, it.v, c);
                    edges += static_cast<unsigned long long>(it.deg);
                }
            }
            break;
        }
        case 2: tentative_group_tile<32, kRXF>(a, rt, list, 2, first, round, edges); break;
        case 3: tentative_group_tile<16, kRXF>(a, rt, list, 3, first, round, edges); break;
        case 4: tentative_group_tile<8, kRXF>(a, rt, list, 4, first, round, edges); break;
        default: tentative_group_tile<4, kRXF>(a, rt, list, 5, first, round, edges); break;
        }
    }
    warp_add(&a.ctrl->edges, edges);
}

// ---------------------------------------------------------------------------
// Conflict detection; winners fix their color, losers go to W_{r+1}
// ---------------------------------------------------------------------------
// Does some neighbor in this lane's stripe have v's tentative color and a
// larger (priority, id)?  With equal tentative colors the 64-bit keys order
// as the priorities; equal keys fall back to the id.  U gathers in flight.
template <int UC>
__device__ __forceinline__ bool loses_v(const SpecArgs& a, int32_t v, int64_t beg, int32_t deg,
                                        int32_t lane0, int32_t stride) {
    if (deg == 0) return false;
    const unsigned long long* key = reinterpret_cast<const unsigned long long*>(a.key);
    const uint64_t kv = __ldg(key + v);
    const uint32_t tv = static_cast<uint32_t>(kv >> 32);
    bool lose = false;
    for_each_nbr<UC, uint64_t, true>(
        a.g, beg, deg, lane0, stride, [&](int32_t u) { return __ldg(key + u); },
        [&](int32_t u, uint64_t ku) {
            if (u != v && static_cast<uint32_t>(ku >> 32) == tv && (ku > kv || (ku == kv && u > v)))
                lose = true;
        },
        &a.ctrl->err);
    return lose;
}

template <int UC>
__device__ __forceinline__ bool loses(const SpecArgs& a, const WorkItem& it, int32_t lane0,
                                      int32_t stride) {
    return loses_v<UC>(a, it.v, it.beg, it.deg, lane0, stride);
}

// One chunk of a hub row in the conflict phase (whole block): the chunks OR
// a lose flag; the block finishing the last chunk fixes the color or
// re-queues all the chunks (clearing the hub's bitmap for the next round).
__device__ __forceinline__ void conflict_chunk(const SpecArgs& a, const WorkItem& it, int par,
                                               WorkItem* next, int32_t start0, int32_t& my_max,
                                               unsigned long long& edges, int32_t* s_flag) {
    const int t = threadIdx.x;
    const int32_t slot = -it.v - 1;
    if (!(slot >= 0 && slot < a.n_hubs) || static_cast<uint32_t>(a.hub_v[slot]) >= static_cast<uint32_t>(a.g.n)) {
        if (t == 0) check_index(a, false, 7, slot);
        return;
    }
    const int32_t v = a.hub_v[slot];
    const bool lose = __syncthreads_or(loses_v<1>(a, v, it.beg, it.deg, t, kBlock));
    if (t == 0) {
        if (lose) atomicOr(&a.hub_lose[slot], 1);
        edges += static_cast<unsigned long long>(it.deg);
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_flag[0] = atomicAdd(&a.hub_done[slot], 1) == a.hub_nch[slot] - 1;
    __syncthreads();
    const bool last = s_flag[0] != 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int32_t lost = *reinterpret_cast<volatile int32_t*>(a.hub_lose + slot);
    const int32_t nch = a.hub_nch[slot];
    if (lost) {
        const int64_t words = hub_bitmap_words(a.hub_deg[slot], a.X);
        uint32_t* bm = a.hub_bm + a.hub_off[slot];
        if (a.hub_off[slot] >= 0 && a.hub_off[slot] + words <= a.hub_words_total)
            for (int64_t i = t; i < words; i += kBlock) bm[i] = 0u;
        if (t == 0) {
            a.hub_lose[slot] = 0;
            a.hub_done[slot] = 0;
            s_flag[1] = atomicAdd(&a.ctrl->cnt[par ^ 1][0], nch);
            atomicAdd(&a.ctrl->hub_cnt[par ^ 1], 1);
        }
        __syncthreads();
        const int64_t beg = a.hub_beg[slot];
        const int32_t deg = a.hub_deg[slot];
        const bool fits = s_flag[1] + nch <= a.ctrl->init_cnt[0] &&
                          start0 + static_cast<int64_t>(s_flag[1]) + nch <= a.list_len;
        if (!fits && t == 0) check_index(a, false, 8, s_flag[1]);
        if (fits)
            for (int32_t c = t; c < nch; c += kBlock)
                store_item(next + start0 + s_flag[1] + c, beg + static_cast<int64_t>(c) * kSpecChunk,
                           -(slot + 1), min(kSpecChunk, deg - c * kSpecChunk));
        __syncthreads();
    } else if (t == 0) {
        const int32_t c = static_cast<int32_t>(a.key[v] >> 32);
        a.color[v] = c;
        my_max = max(my_max, c);
        a.hub_done[slot] = 0;
    }
}

template <int G>
__device__ __forceinline__ void conflict_group_tile(const SpecArgs& a, const RoundTiles& rt,
                                                    const WorkItem* list, WorkItem* next, int par,
                                                    int b, int32_t first, int32_t& my_max,
                                                    unsigned long long& edges) {
    const int gi = threadIdx.x / G, gl = threadIdx.x % G;
    const int32_t k = first + gi;
    const bool valid = k < rt.cnt[b];
    WorkItem it{0, 0, 0};
    if (valid) it = load_item(list + rt.start[b] + k);
    const bool lose = group_any<G>(loses<LanesUnroll<G>::U>(a, it, gl, G));
    const bool leader = valid && gl == 0;
    if (leader) {
        edges += static_cast<unsigned long long>(it.deg);
        if (!lose) {
            const int32_t c = static_cast<int32_t>(a.key[it.v] >> 32);
            a.color[it.v] = c;
            my_max = max(my_max, c);
        }
    }
    warp_append(leader && lose, it.beg, it.v, it.deg, &a.ctrl->cnt[par ^ 1][b], next, rt.start[b]);
}

__global__ void __launch_bounds__(kBlock) k_conflict(SpecArgs a) {
    __shared__ RoundTiles rt;
    __shared__ bool s_last;
    __shared__ int32_t s_flag[2];
    const int32_t round = a.ctrl->round;
    const int par = round & 1;
    const WorkItem* list = par ? a.list1 : a.list0;
    WorkItem* next = par ? a.list0 : a.list1;
    load_round_tiles(a.ctrl, par, rt);
    unsigned long long edges = 0;
    int32_t my_max = 0;
    for (int32_t t = blockIdx.x; t < rt.prefix[kNB]; t += gridDim.x) {
        const int b = tile_bucket(rt, t);
        const int32_t first = (t - rt.prefix[b]) * bucket_tile(b);
        switch (b) {
        case 0:
            conflict_chunk(a, load_item(list + rt.start[0] + first), par, next, rt.start[0], my_max,
                           edges, s_flag);
            break;
        case 1:
        case 2: conflict_group_tile<32>(a, rt, list, next, par, b, first, my_max, edges); break;
        case 3: conflict_group_tile<16>(a, rt, list, next, par, 3, first, my_max, edges); break;
        case 4: conflict_group_tile<8>(a, rt, list, next, par, 4, first, my_max, edges); break;
        default: conflict_group_tile<4>(a, rt, list, next, par, 5, first, my_max, edges); break;
        }
    }
    warp_add(&a.ctrl->edges, edges);
    warp_max(&a.ctrl->max_color, my_max);

    // The last block to finish closes the round.
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.ctrl->done_blocks, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        volatile SpecCtrl* c = a.ctrl;
        int32_t total = c->hub_cnt[par ^ 1];  // vertices, not chunks, for the hubs
        for (int b = 1; b < kNB; ++b) total += c->cnt[par ^ 1][b];
        c->active = total;
        c->conflicts += static_cast<unsigned long long>(total);
        c->round = round + 1;
        c->done_blocks = 0u;
        const bool over = total > 0 && round + 1 >= a.round_limit;
        if (over) c->err |= kErrRoundLimit;
        if (a.use_cond) cudaGraphSetConditional(a.cond, (total > 0 && !over) ? 1u : 0u);
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
gc_status rounds_in_graph(SpecArgs& a, int32_t X, int grid_t, int grid_c, cudaStream_t s) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
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
    cudaGraphNode_t n1 = nullptr, n2 = nullptr;
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaKernelNodeParams k1;
        std::memset(&k1, 0, sizeof(k1));
        k1.func = X > 1 ? reinterpret_cast<void*>(k_tentative<true>) : reinterpret_cast<void*>(k_tentative<false>);
        k1.gridDim = dim3(grid_t);
        k1.blockDim = dim3(kBlock);
        k1.kernelParams = args;
        cudaKernelNodeParams k2 = k1;
        k2.func = reinterpret_cast<void*>(k_conflict);
        k2.gridDim = dim3(grid_c);
        e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) {
        prof_begin(KID_SPEC_GRAPH, s);
        e = cudaGraphLaunch(exec, s);
        prof_end(KID_SPEC_GRAPH, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return cuda_status(e);
}

gc_status color_device(const Graph& g, int32_t X, uint64_t seed, int32_t* colors_out,
                       gc_stats* stats, cudaStream_t s) {
    if (g.n == 0) {
        if (stats) { std::memset(stats, 0, sizeof(*stats)); }
        return GC_OK;
    }
    if (!t_pinned.p) return GC_ERR_OOM;
    const int64_t n = g.n;
    Scratch sc_key, sc_l0, sc_l1, sc_bucket, sc_ctrl;
    // one list entry per vertex, plus the extra chunks of hub rows
    const int64_t list_len = n + g.nnz / kSpecChunk + 1;
    if (!sc_key.alloc(n * 8, s) ||
        !sc_l0.alloc(list_len * sizeof(WorkItem), s) || !sc_l1.alloc(list_len * sizeof(WorkItem), s) ||
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

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaMemsetAsync(a.ctrl, 0, sizeof(SpecCtrl), s);
    const int grid_t = resident_grid(X > 1 ? k_tentative<true> : k_tentative<false>, a.tune);
    const int grid_c = resident_grid(k_conflict, a.tune);
    const int setup_grid = static_cast<int>(
        std::min<int64_t>((n + kBlock - 1) / kBlock, resident_grid(k_spec_setup, a.tune)));
    GC_LAUNCH(KID_SPEC_SETUP, s, k_spec_setup<<<setup_grid, kBlock, 0, s>>>(a));
    // hub rows need their slots and bitmaps before the fill
    SpecCtrl hs;
    cudaError_t ce0 = cudaMemcpyAsync(&hs, a.ctrl, sizeof(SpecCtrl), cudaMemcpyDeviceToHost, s);
    if (ce0 == cudaSuccess) ce0 = cudaStreamSynchronize(s);
    if (ce0 != cudaSuccess) return cuda_status(ce0);
    const int64_t hubs = std::max<int32_t>(hs.n_hubs, 1);
    const int64_t hub_words = std::max<int64_t>(static_cast<int64_t>(hs.hub_words), 1);
    Scratch sh_v, sh_beg, sh_deg, sh_nch, sh_off, sh_done, sh_lose, sh_bm;
    if (!sh_v.alloc(hubs * 4, s) || !sh_beg.alloc(hubs * 8, s) || !sh_deg.alloc(hubs * 4, s) ||
        !sh_nch.alloc(hubs * 4, s) || !sh_off.alloc(hubs * 8, s) || !sh_done.alloc(hubs * 4, s) ||
        !sh_lose.alloc(hubs * 4, s) || !sh_bm.alloc(hub_words * 4, s))
        return GC_ERR_OOM;
    a.hub_v = sh_v.as<int32_t>();
    a.hub_beg = sh_beg.as<int64_t>();
    a.hub_deg = sh_deg.as<int32_t>();
    a.hub_nch = sh_nch.as<int32_t>();
    a.hub_off = sh_off.as<int64_t>();
    a.hub_done = sh_done.as<int32_t>();
    a.hub_lose = sh_lose.as<int32_t>();
    a.hub_bm = sh_bm.as<uint32_t>();
    a.n_hubs = hs.n_hubs;
    a.hub_words_total = hub_words;
    a.list_len = list_len;
    if (hs.n_hubs > 0) cudaMemsetAsync(a.hub_bm, 0, hub_words * 4, s);
    GC_LAUNCH(KID_SPEC_FILL, s, k_spec_fill<<<setup_grid, kBlock, 0, s>>>(a));
    gc_status st = GC_OK;
    a.round_limit = static_cast<int32_t>(std::min<int64_t>(n + 2, INT32_MAX));
    if (a.tune.spec_graph) {
        st = rounds_in_graph(a, X, grid_t, grid_c, s);
    } else {
        int32_t rounds = 0;
        for (;;) {
            if (X > 1) GC_LAUNCH(KID_TENTATIVE, s, k_tentative<true><<<grid_t, kBlock, 0, s>>>(a));
            else GC_LAUNCH(KID_TENTATIVE, s, k_tentative<false><<<grid_t, kBlock, 0, s>>>(a));
            GC_LAUNCH(KID_CONFLICT, s, k_conflict<<<grid_c, kBlock, 0, s>>>(a));
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
    if (h.err & kErrInternal) {
        std::fprintf(stderr, "libgc: internal check %d failed at index %lld (access skipped)\n",
                     h.bad_where, h.bad_index);
        if (st == GC_OK) st = GC_ERR_CUDA;
    }
    if (a.tune.spec_graph) note_launches(2 * static_cast<int64_t>(h.round));
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
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace gc
