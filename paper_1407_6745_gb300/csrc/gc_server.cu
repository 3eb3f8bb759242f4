// gc_server.cu -- the serving loop (gc_server_*): a request queue, admission
// by a device-memory budget, continuous batching onto worker streams.
//
// A request refers to the caller's CSR (host or device memory, left in place
// until its result is claimed); submit checks the offsets on the host and
// queues it.  Workers -- one host thread and one non-blocking CUDA stream
// each -- admit the queue's head requests first come first served while they
// fit the memory budget and the batch limit, as a cohort: one concatenated
// CSR on the device (one copy per array and request, then a staging kernel
// that checks every row and shifts each graph's ids and offsets to its
// place).  A worker keeps several cohorts resident and advances them in
// turn, one step at a time: the speculative coloring of a cohort's graphs,
// then recoloring iterations, with CSR, colors and work lists resident on the
// device throughout.  Between steps it admits the requests that arrived
// meanwhile as a new cohort (as soon as memory is free), so a request does
// not wait for the graphs already on the GPU to finish, and a request
// retires as soon as its own iterations are done: its colors come back, its
// latency is taken and its scratch share of the budget is returned at once.
// The CSR of retired requests is returned when its cohort is compacted (once
// half of its CSR belongs to retired requests) or ends.  A step is the
// coloring or up to four recoloring iterations, never past the cohort's next
// retirement, and goes to the worker's cohort with the highest response
// ratio, (time waited + work left) / work left: a small request admitted
// behind large ones finishes first, and a large one is not starved.
//
// Workers use the tuning in force at creation.  The dataflow recoloring
// launch is cooperative: with several workers, one worker's launch waits
// until every one of its blocks can be resident, so launches of different
// workers never wait on each other's blocks.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gc_internal.h"

namespace gc {
namespace {

struct Slot {
    int64_t vbase, ebase, n, nnz;
};

// Stages a cohort: graph y's local offsets (n + 1 of them) sit at
// loff[vbase + y ...] and its ids at idx[ebase ...].  One warp per vertex
// checks the row (the rules of gc_check_graph: offsets from 0 to nnz, never
// decreasing; ids in [0, n), no self-loop), writes the global offset and
// shifts the ids by the graph's vertex base.  A graph with a bad row gets
// bad[y] = 1 (its rows are left unshifted: the cohort is staged again
// without it).
__global__ void __launch_bounds__(kBlock) k_srv_stage(const int64_t* loff, int64_t* off, int32_t* idx,
                                                      const Slot* slots, int32_t ng, int64_t n_total,
                                                      int64_t nnz_total, int32_t* bad) {
    const int lane = lane_id();
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * kBlock) >> 5;
    int32_t y = 0;
    for (int64_t v = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) >> 5; v < n_total; v += nw) {
        while (y + 1 < ng && slots[y + 1].vbase <= v) ++y;
        const Slot sl = slots[y];
        const int64_t lv = v - sl.vbase;
        const int64_t b = loff[v + y], e = loff[v + y + 1];
        bool ok = b >= 0 && e >= b && e <= sl.nnz && (lv != 0 || b == 0) && (lv != sl.n - 1 || e == sl.nnz);
        if (lane == 0) off[v] = b + sl.ebase;
        if (ok) {
            const int32_t vb = static_cast<int32_t>(sl.vbase);
            for (int64_t k = b + lane; k < e; k += 32) {
                const int32_t u = idx[sl.ebase + k];
                if (u < 0 || u >= sl.n || u == lv) ok = false;
                idx[sl.ebase + k] = u + vb;
            }
        }
        if (__any_sync(kFull, !ok) && lane == 0) bad[y] = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[n_total] = nnz_total;
}

// Where a graph kept by a compaction was (o*) and goes (n*).
struct MoveSlot {
    int64_t ovbase, oebase, nvbase, nebase, n;
};

// Compacts a cohort: the graphs kept move to their new vertex and entry
// bases; one warp per new vertex copies its row with the ids shifted by the
// change of vertex base, its offset shifted by the change of entry base, and
// its color.  (The rows were checked when the cohort was staged.)
__global__ void __launch_bounds__(kBlock) k_srv_compact(const int64_t* off_o, const int32_t* idx_o,
                                                        const int32_t* col_o, int64_t* off_n, int32_t* idx_n,
                                                        int32_t* col_n, const MoveSlot* mv, int32_t ng,
                                                        int64_t n_total, int64_t nnz_total) {
    const int lane = lane_id();
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * kBlock) >> 5;
    int32_t y = 0;
    for (int64_t v = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) >> 5; v < n_total; v += nw) {
        while (y + 1 < ng && mv[y + 1].nvbase <= v) ++y;
        const MoveSlot m = mv[y];
        const int64_t ov = m.ovbase + (v - m.nvbase);
        const int64_t b = off_o[ov], e = off_o[ov + 1];
        const int64_t nb = b - m.oebase + m.nebase;
        const int32_t dv = static_cast<int32_t>(m.nvbase - m.ovbase);
        if (lane == 0) {
            off_n[v] = nb;
            col_n[v] = col_o[ov];
        }
        for (int64_t k = b + lane; k < e; k += 32) idx_n[nb + (k - b)] = idx_o[k] + dv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off_n[n_total] = nnz_total;
}

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const int64_t* off = nullptr;  // the caller's CSR, n + 1 offsets and nnz ids
    const int32_t* idx = nullptr;
    int64_t n = 0, nnz = 0;
    int64_t bytes = 0;             // admitted device-memory estimate
    int64_t resident = 0;          // of which its CSR and colors in its cohort
    bool solo = false;             // admit alone (a shared cohort ran out of memory)
    gc_batch_graph desc{};
    // result; `status` is read by waiters and written under the server lock
    // only (finish), from the worker's `outcome`
    int32_t outcome = GC_OK;
    int32_t status = GC_PENDING;
    std::vector<int32_t> colors;
    gc_request_result res{};
};

// Device bytes one request holds while its cohort runs: its CSR and colors,
// the coloring scratch (priority keys, two work lists, buckets, per-vertex
// graph index and win round) or the recoloring scratch (work list, alternate
// colors, per-class tables over at most min(n, max degree + X) + 1 classes),
// whichever is larger, with room to spare.
int64_t request_bytes(int64_t n, int64_t nnz, int64_t max_deg, int32_t X) {
    const int64_t classes = std::min<int64_t>(n, max_deg + X) + 2;
    return 16 * (n + 1) + 4 * nnz + 4 * n + 64 * n + 16 * (nnz / 256 + 1) + 256 * classes + 1024;
}
// The part of it that stays with the cohort until compaction: offsets, ids, colors.
int64_t resident_bytes(int64_t n, int64_t nnz) { return 8 * (n + 1) + 4 * nnz + 4 * n; }

// Requests admitted together, laid out as one concatenated CSR on the device.
struct Cohort {
    std::vector<Request*> reqs;
    std::vector<Slot> slots;
    std::vector<gc_batch_graph> desc;
    std::vector<char> live;
    std::vector<int32_t> rounds, maxc;
    int32_t iters_done = -1;   // -1: not colored yet; else recoloring iterations done
    int64_t N = 0, E = 0;
    Scratch off, idx, col;
    int64_t resident = 0;          // resident bytes of its requests, live or not
    int64_t retired_resident = 0;  // of which held for retired requests
    int32_t admitted = 0;          // requests at admission
    double start_ms = 0.0;
    int32_t n_live() const { return static_cast<int32_t>(std::count(live.begin(), live.end(), 1)); }
    // Work left, in adjacency entries to scan: every live graph's remaining
    // recoloring iterations, plus its coloring (weighted as a few iterations:
    // the speculative rounds rescan the rows) if not done yet.
    double oldest_submit() const {
        double t = 1e300;
        for (size_t i = 0; i < reqs.size(); ++i)
            if (live[i]) t = std::min(t, reqs[i]->res.submit_ms);
        return t;
    }
    double work_left() const {
        double w = 0.0;
        for (size_t i = 0; i < reqs.size(); ++i) {
            if (!live[i]) continue;
            const double its = desc[i].iterations - std::max(iters_done, 0) + (iters_done < 0 ? 3.0 : 0.0);
            w += static_cast<double>(slots[i].nnz + slots[i].n) * its;
        }
        return w;
    }
    Graph graph() const {
        Graph g{};
        g.off = off.as<int64_t>();
        g.idx = idx.as<int32_t>();
        g.n = static_cast<int32_t>(N);
        g.nnz = E;
        g.vec = (reinterpret_cast<uintptr_t>(g.idx) & 15u) == 0;
        return g;
    }
};

constexpr int kCohortsPerWorker = 4;
// Recoloring iterations in a step at most: a request that arrives meanwhile
// waits at most that long to be admitted and to take the next step.
constexpr int32_t kStepIters = 4;

}  // namespace
}  // namespace gc

using namespace gc;

struct gc_server {
    int device = 0;
    int64_t budget = 0;
    int32_t max_batch = 1;
    Tuning tune{};
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work;  // workers: queue changed / memory freed / stop
    std::condition_variable cv_done;  // waiters: a request finished
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> live;  // queued, running or unclaimed
    uint64_t next_ticket = 1;
    bool stopping = false;
    int64_t in_use = 0, peak = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0;
    double first_submit = -1.0, last_done = 0.0;
    std::vector<double> latencies;

    std::vector<std::thread> workers;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
    void worker_main();
    Cohort* stage(std::vector<Request*> reqs, cudaStream_t s);
    bool step(Cohort* c, cudaStream_t s);
    void compact(Cohort* c, cudaStream_t s);
    // Finishes requests (status, colors already in place) and returns
    // `release` bytes to the budget.  Takes the lock.
    void finish(const std::vector<Request*>& done, int64_t release, double start, int32_t size);
    // Puts requests back at the head of the queue, to be admitted alone.
    void requeue_solo(const std::vector<Request*>& rs, int64_t release);
};

void gc_server::finish(const std::vector<Request*>& done, int64_t release, double start, int32_t size) {
    const double t = now_ms();
    {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= release;
        for (Request* r : done) {
            r->status = r->outcome;
            r->res.status = r->outcome;
            r->res.batch_size = size;
            r->res.start_ms = start;
            r->res.done_ms = t;
            if (r->status != GC_OK) r->colors.clear();
            ++completed;
            latencies.push_back(t - r->res.submit_ms);
        }
        if (!done.empty()) last_done = std::max(last_done, t);
    }
    cv_work.notify_all();
    cv_done.notify_all();
}

void gc_server::requeue_solo(const std::vector<Request*>& rs, int64_t release) {
    {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= release;
        for (auto it = rs.rbegin(); it != rs.rend(); ++it) {
            (*it)->solo = true;
            queue.push_front(*it);
        }
    }
    cv_work.notify_all();
}

// Admits batches of the queue as cohorts and advances its cohorts in turn
// until the server stops and nothing is left.
void gc_server::worker_main() {
    cudaSetDevice(device);
    set_thread_tuning(&tune);
    cudaStream_t s = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    std::deque<Cohort*> mine;
    double ms_per_unit = 0.0;  // measured step time per unit of work (Cohort::work_left)
    for (;;) {
        std::vector<Request*> batch;
        int64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            auto can_admit = [&] {
                return !queue.empty() && static_cast<int>(mine.size()) < kCohortsPerWorker &&
                       in_use + queue.front()->bytes <= budget;
            };
            cv_work.wait(lk, [&] { return can_admit() || !mine.empty() || (stopping && queue.empty()); });
            if (!can_admit() && mine.empty()) break;  // stopping, nothing left
            if (can_admit()) {
                int64_t n_sum = 0;
                while (!queue.empty() && static_cast<int32_t>(batch.size()) < max_batch) {
                    Request* r = queue.front();
                    if (in_use + bytes + r->bytes > budget) break;
                    if (n_sum + r->n > INT32_MAX) break;  // the cohort CSR numbers vertices in int32
                    if (r->solo && !batch.empty()) break;
                    queue.pop_front();
                    batch.push_back(r);
                    bytes += r->bytes;
                    n_sum += r->n;
                    if (r->solo) break;
                }
                in_use += bytes;
                peak = std::max(peak, in_use);
                ++batches;
            }
        }
        if (!batch.empty()) {
            if (have_stream) {
                Cohort* c = stage(batch, s);
                if (c) mine.push_back(c);
            } else {
                for (Request* r : batch) r->outcome = GC_ERR_CUDA;
                finish(batch, bytes, now_ms(), static_cast<int32_t>(batch.size()));
            }
        }
        if (mine.empty()) continue;
        // highest response ratio next: (time waited + work left) / work left,
        // the work in ms at the rate this worker has measured.  A small
        // request admitted behind large ones goes first, and a large one's
        // ratio grows while it waits, so it is not starved.
        const double now = now_ms();
        auto ratio = [&](const Cohort* x) {
            const double est = std::max(x->work_left() * ms_per_unit, 1e-3);
            return (now - x->oldest_submit() + est) / est;
        };
        auto pick = std::max_element(mine.begin(), mine.end(),
                                     [&](const Cohort* x, const Cohort* y) { return ratio(x) < ratio(y); });
        Cohort* c = *pick;
        mine.erase(pick);
        const double w0 = c->work_left(), t0 = now_ms();
        const bool more = step(c, s);
        const double done_units = w0 - (more ? c->work_left() : 0.0);
        if (done_units > 0) {  // exponential average of the measured rate
            const double rate = (now_ms() - t0) / done_units;
            ms_per_unit = ms_per_unit > 0 ? 0.8 * ms_per_unit + 0.2 * rate : rate;
        }
        if (more) mine.push_back(c);
        else delete c;
        prof_collect();
    }
    if (have_stream) cudaStreamDestroy(s);
    set_thread_tuning(nullptr);
}

// Lays requests out as a cohort on the device.  Requests whose CSR fails the
// staging check finish with GC_ERR_BAD_GRAPH and the rest are staged again
// without them; if the cohort does not fit the device's free memory (memory
// held outside the server), its requests go back to the queue to be admitted
// one at a time.  Returns nullptr when no request is left to run.
Cohort* gc_server::stage(std::vector<Request*> reqs, cudaStream_t s) {
    const double start = now_ms();
    const int32_t admitted = static_cast<int32_t>(reqs.size());
    for (;;) {
        const int32_t ng = static_cast<int32_t>(reqs.size());
        int64_t bytes = 0;
        for (Request* r : reqs) bytes += r->bytes;
        auto fail_all = [&](gc_status st) {
            for (Request* r : reqs) r->outcome = st;
            finish(reqs, bytes, start, admitted);
            return nullptr;
        };
        Cohort* c = new Cohort();
        c->reqs = reqs;
        c->slots.resize(ng);
        c->desc.resize(ng);
        for (int32_t i = 0; i < ng; ++i) {
            const Request* r = reqs[i];
            c->slots[i] = Slot{c->N, c->E, r->n, r->nnz};
            c->desc[i] = r->desc;
            c->desc[i].vertex_base = c->N;
            c->N += r->n;
            c->E += r->nnz;
            c->resident += r->resident;
        }
        c->live.assign(ng, 1);
        c->rounds.assign(ng, 0);
        c->maxc.assign(ng, 0);
        c->admitted = admitted;
        c->start_ms = start;
        Scratch s_loff, s_slot, s_bad;
        if (!s_loff.alloc((c->N + ng) * sizeof(int64_t), s) || !c->off.alloc((c->N + 1) * sizeof(int64_t), s) ||
            !c->idx.alloc(c->E * sizeof(int32_t), s) || !c->col.alloc(c->N * sizeof(int32_t), s) ||
            !s_slot.alloc(ng * sizeof(Slot), s) || !s_bad.alloc(ng * sizeof(int32_t), s)) {
            delete c;
            if (ng == 1) return fail_all(GC_ERR_OOM);
            requeue_solo(reqs, bytes);
            return nullptr;
        }
        int64_t* loff = s_loff.as<int64_t>();
        int32_t* bad = s_bad.as<int32_t>();
        cudaError_t e = cudaMemsetAsync(bad, 0, ng * sizeof(int32_t), s);
        for (int32_t i = 0; i < ng && e == cudaSuccess; ++i) {
            const Request* r = reqs[i];
            e = cudaMemcpyAsync(loff + c->slots[i].vbase + i, r->off, (r->n + 1) * sizeof(int64_t),
                                cudaMemcpyDefault, s);
            if (e == cudaSuccess && r->nnz > 0)
                e = cudaMemcpyAsync(c->idx.as<int32_t>() + c->slots[i].ebase, r->idx, r->nnz * sizeof(int32_t),
                                    cudaMemcpyDefault, s);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s_slot.p, c->slots.data(), ng * sizeof(Slot), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            delete c;
            return fail_all(cuda_status(e));
        }
        const int grid = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>((c->N * 32 + kBlock - 1) / kBlock, persistent_grid(tune))));
        GC_LAUNCH(KID_BATCH, s,
                  k_srv_stage<<<grid, kBlock, 0, s>>>(loff, c->off.as<int64_t>(), c->idx.as<int32_t>(),
                                                       s_slot.as<Slot>(), ng, c->N, c->E, bad));
        std::vector<int32_t> hbad(ng, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hbad.data(), bad, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            delete c;
            return fail_all(cuda_status(e));
        }
        if (std::count(hbad.begin(), hbad.end(), 1) == 0) return c;
        // bad rows: those requests finish now, the others are staged again
        delete c;
        std::vector<Request*> good, badr;
        int64_t bad_bytes = 0;
        for (int32_t i = 0; i < ng; ++i) {
            if (hbad[i]) {
                reqs[i]->outcome = GC_ERR_BAD_GRAPH;
                badr.push_back(reqs[i]);
                bad_bytes += reqs[i]->bytes;
            } else {
                good.push_back(reqs[i]);
            }
        }
        finish(badr, bad_bytes, start, admitted);
        if (good.empty()) return nullptr;
        reqs.swap(good);
    }
}

// One step of a cohort: its coloring, or up to kStepIters recoloring
// iterations, never past its next retirement; then the requests whose own
// iterations are done retire.  Returns false once the cohort is over (it is
// then to be deleted: its memory is returned to the budget here).
bool gc_server::step(Cohort* c, cudaStream_t s) {
    const int32_t ng = static_cast<int32_t>(c->reqs.size());
    const Graph g = c->graph();
    gc_status st;
    std::vector<int32_t> maxc_out(ng, 0);
    if (c->iters_done < 0) {
        st = color_batch_device(g, c->desc.data(), ng, c->col.as<int32_t>(), c->rounds.data(), maxc_out.data(),
                                nullptr, s);
        if (st == GC_OK) c->iters_done = 0;
    } else {
        int32_t next = INT32_MAX;
        for (int32_t i = 0; i < ng; ++i)
            if (c->live[i]) next = std::min(next, c->desc[i].iterations);
        const int32_t it1 = std::min(next, c->iters_done + kStepIters);
        st = recolor_batch_range(g, c->desc.data(), ng, c->col.as<int32_t>(), c->maxc.data(), c->iters_done, it1,
                                 maxc_out.data(), s);
        if (st == GC_OK) c->iters_done = it1;
    }
    std::vector<Request*> done;
    int64_t release = 0;
    if (st != GC_OK) {
        std::vector<Request*> rest;
        for (int32_t i = 0; i < ng; ++i)
            if (c->live[i]) {
                rest.push_back(c->reqs[i]);
                release += c->reqs[i]->bytes;
            }
        release += c->retired_resident;
        if (st == GC_ERR_OOM && rest.size() > 1) {
            requeue_solo(rest, release);  // they start again alone: their results do not depend on it
        } else {
            for (Request* r : rest) r->outcome = st;
            finish(rest, release, c->start_ms, c->admitted);
        }
        return false;
    }
    c->maxc = maxc_out;
    cudaError_t e = cudaSuccess;
    for (int32_t i = 0; i < ng && e == cudaSuccess; ++i) {
        if (!c->live[i] || c->desc[i].iterations > c->iters_done) continue;
        Request* r = c->reqs[i];
        r->colors.resize(static_cast<size_t>(r->n));
        e = cudaMemcpyAsync(r->colors.data(), c->col.as<int32_t>() + c->slots[i].vbase, r->n * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s);
        r->res.rounds = c->rounds[i];
        r->res.max_color = c->maxc[i];
        r->outcome = GC_OK;
        c->live[i] = 0;
        done.push_back(r);
        release += r->bytes - r->resident;
        c->retired_resident += r->resident;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        for (int32_t i = 0; i < ng; ++i)
            if (c->live[i]) {
                done.push_back(c->reqs[i]);
                release += c->reqs[i]->bytes - c->reqs[i]->resident;
                c->retired_resident += c->reqs[i]->resident;
                c->live[i] = 0;
            }
        for (Request* r : done) r->outcome = cuda_status(e);
    }
    const bool over = c->n_live() == 0;
    if (over) release += c->retired_resident;
    finish(done, release, c->start_ms, c->admitted);
    if (over) return false;
    if (2 * c->retired_resident >= c->resident) compact(c, s);
    return true;
}

// Drops the retired requests from a cohort: the kept graphs move into new,
// smaller device arrays and the retired ones' CSR returns to the budget.  If
// the new arrays cannot be had, the cohort stays as it is.
void gc_server::compact(Cohort* c, cudaStream_t s) {
    const int32_t ng = static_cast<int32_t>(c->reqs.size());
    std::vector<MoveSlot> mv;
    std::vector<int32_t> keep;
    int64_t N = 0, E = 0;
    for (int32_t i = 0; i < ng; ++i) {
        if (!c->live[i]) continue;
        const Slot& sl = c->slots[i];
        mv.push_back(MoveSlot{sl.vbase, sl.ebase, N, E, sl.n});
        keep.push_back(i);
        N += sl.n;
        E += sl.nnz;
    }
    const int32_t nk = static_cast<int32_t>(keep.size());
    Scratch off, idx, col, smv;
    if (!off.alloc((N + 1) * sizeof(int64_t), s) || !idx.alloc(E * sizeof(int32_t), s) ||
        !col.alloc(N * sizeof(int32_t), s) || !smv.alloc(nk * sizeof(MoveSlot), s))
        return;
    if (cudaMemcpyAsync(smv.p, mv.data(), nk * sizeof(MoveSlot), cudaMemcpyHostToDevice, s) != cudaSuccess) return;
    const int grid = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>((N * 32 + kBlock - 1) / kBlock, persistent_grid(tune))));
    GC_LAUNCH(KID_BATCH, s,
              k_srv_compact<<<grid, kBlock, 0, s>>>(c->off.as<int64_t>(), c->idx.as<int32_t>(),
                                                     c->col.as<int32_t>(), off.as<int64_t>(), idx.as<int32_t>(),
                                                     col.as<int32_t>(), smv.as<MoveSlot>(), nk, N, E));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return;
    std::swap(c->off.p, off.p);
    std::swap(c->idx.p, idx.p);
    std::swap(c->col.p, col.p);
    Cohort k;
    for (int32_t j = 0; j < nk; ++j) {
        const int32_t i = keep[j];
        k.reqs.push_back(c->reqs[i]);
        k.slots.push_back(Slot{mv[j].nvbase, mv[j].nebase, c->slots[i].n, c->slots[i].nnz});
        gc_batch_graph d = c->desc[i];
        d.vertex_base = mv[j].nvbase;
        k.desc.push_back(d);
        k.rounds.push_back(c->rounds[i]);
        k.maxc.push_back(c->maxc[i]);
    }
    c->reqs.swap(k.reqs);
    c->slots.swap(k.slots);
    c->desc.swap(k.desc);
    c->rounds.swap(k.rounds);
    c->maxc.swap(k.maxc);
    c->live.assign(nk, 1);
    c->N = N;
    c->E = E;
    const int64_t freed = c->retired_resident;
    c->resident -= freed;
    c->retired_resident = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= freed;
    }
    cv_work.notify_all();
}

namespace {

// Host check of a request's offsets (the ids are checked on the device when
// its batch is staged); *max_deg receives the largest row.
gc_status check_offsets(const int64_t* off, int64_t n, int64_t nnz, int64_t* max_deg) {
    if (off[0] != 0 || off[n] != nnz) return GC_ERR_BAD_GRAPH;
    int64_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = off[v + 1] - off[v];
        if (d < 0) return GC_ERR_BAD_GRAPH;
        md = std::max(md, d);
    }
    *max_deg = md;
    return GC_OK;
}

gc_status finish_poll(gc_server* s, std::unordered_map<uint64_t, Request*>::iterator it, int32_t* colors_out,
                      gc_request_result* res) {
    Request* r = it->second;
    if (colors_out && r->status == GC_OK && r->n > 0)
        std::memcpy(colors_out, r->colors.data(), r->n * sizeof(int32_t));
    if (res) *res = r->res;
    const gc_status st = static_cast<gc_status>(r->status);
    s->live.erase(it);
    delete r;
    return st;
}

}  // namespace

extern "C" {

gc_status gc_server_create(size_t mem_budget, int32_t max_batch, int32_t workers, gc_server** out) {
    if (!out || mem_budget == 0 || max_batch < 1 || max_batch > 65535 || workers < 1 || workers > 64)
        return GC_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    gc_server* s = new gc_server();
    s->device = dev;
    s->budget = static_cast<int64_t>(std::min<size_t>(mem_budget, static_cast<size_t>(INT64_MAX)));
    s->max_batch = max_batch;
    s->tune = current_tuning();
    s->t0 = Clock::now();
    for (int32_t i = 0; i < workers; ++i) s->workers.emplace_back([s] { s->worker_main(); });
    *out = s;
    return GC_OK;
}

gc_status gc_server_submit(gc_server* s, const gc_request* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return GC_ERR_INVALID_ARG;
    const gc_graph& g = q->graph;
    if (g.n < 0 || g.n > INT32_MAX || g.nnz < 0 ||
        (g.mem != GC_MEM_DEVICE && g.mem != GC_MEM_HOST) || !g.offsets || (g.nnz > 0 && !g.idx))
        return GC_ERR_INVALID_ARG;
    if ((q->strategy != GC_FIRST_FIT && q->strategy != GC_RANDOM_X_FIT) ||
        (q->strategy == GC_RANDOM_X_FIT && q->X < 1) || q->iterations < 0 || !perm_valid(q->perm))
        return GC_ERR_INVALID_ARG;
    Request* r = new Request();
    r->n = g.n;
    r->nnz = g.nnz;
    r->off = g.offsets;
    r->idx = g.idx;
    int64_t max_deg = 0;
    gc_status st = GC_OK;
    if (g.mem == GC_MEM_HOST) {
        st = check_offsets(g.offsets, g.n, g.nnz, &max_deg);
    } else {
        std::vector<int64_t> off(static_cast<size_t>(g.n) + 1);
        cudaSetDevice(s->device);
        const cudaError_t e =
            cudaMemcpy(off.data(), g.offsets, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost);
        st = e == cudaSuccess ? check_offsets(off.data(), g.n, g.nnz, &max_deg) : cuda_status(e);
    }
    const int32_t X = q->strategy == GC_FIRST_FIT ? 1 : q->X;
    r->bytes = request_bytes(g.n, g.nnz, max_deg, X);
    r->resident = resident_bytes(g.n, g.nnz);
    if (st == GC_OK && r->bytes > s->budget) st = GC_ERR_BUDGET;
    if (st != GC_OK) {
        delete r;
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->rejected;
        return st;
    }
    r->desc.n = g.n;
    r->desc.seed = q->seed;
    r->desc.X = X;
    r->desc.perm = q->perm;
    r->desc.iterations = q->iterations;
    r->desc.perm_seed = q->perm_seed;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete r;
            return GC_ERR_INVALID_ARG;
        }
        r->ticket = s->next_ticket++;
        r->res.submit_ms = s->now_ms();
        if (s->first_submit < 0) s->first_submit = r->res.submit_ms;
        ++s->submitted;
        s->live[r->ticket] = r;
        *ticket = r->ticket;
        if (r->n == 0) {  // nothing to color: done at once
            r->status = GC_OK;
            r->res.status = GC_OK;
            r->res.start_ms = r->res.done_ms = r->res.submit_ms;
            ++s->completed;
            s->latencies.push_back(0.0);
            s->last_done = std::max(s->last_done, r->res.done_ms);
        } else {
            s->queue.push_back(r);
        }
    }
    s->cv_work.notify_one();
    s->cv_done.notify_all();
    return GC_OK;
}

gc_status gc_server_poll(gc_server* s, uint64_t ticket, int32_t* colors_out, gc_request_result* res) {
    if (!s) return GC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return GC_ERR_INVALID_ARG;
    if (it->second->status == GC_PENDING) return GC_PENDING;
    return finish_poll(s, it, colors_out, res);
}

gc_status gc_server_wait(gc_server* s, uint64_t ticket, int32_t* colors_out, gc_request_result* res,
                         int32_t timeout_ms) {
    if (!s) return GC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->live.find(ticket);
        return it == s->live.end() || it->second->status != GC_PENDING;
    };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return GC_ERR_INVALID_ARG;
    if (it->second->status == GC_PENDING) return GC_PENDING;
    return finish_poll(s, it, colors_out, res);
}

gc_status gc_server_stats(gc_server* s, gc_server_info* out) {
    if (!s || !out) return GC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->bytes_in_use = s->in_use;
    out->bytes_peak = s->peak;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {  // nearest rank
            size_t k = static_cast<size_t>(std::ceil(p * l.size()));
            return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : l) sum += x;
        out->mean_ms = sum / l.size();
        const double span = s->last_done - s->first_submit;
        out->graphs_per_s = span > 0 ? 1e3 * s->completed / span : 0.0;
    }
    return GC_OK;
}

void gc_server_destroy(gc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (auto& kv : s->live) delete kv.second;
    delete s;
}

}  // extern "C"
