// gc_server.cu -- the serving loop (gc_server_*): a request queue, admission
// by a device-memory budget, continuous batching onto worker streams.
//
// A request refers to the caller's CSR (host or device memory, left in place
// until its result is claimed); submit checks the offsets on the host and
// queues it.  Workers -- one host thread and one non-blocking CUDA stream
// each -- take the queue's head requests first come first served while they
// fit the memory budget and the batch limit, lay them out as one
// concatenated CSR on the device (one copy per array and request, then a
// staging kernel that checks every row and shifts each graph's ids and
// offsets to its place), and run the batch pipeline on it: coloring, then the
// recoloring iterations with CSR, colors and work lists resident on the
// device throughout.  The colors come back per request.  While one worker's
// batch is on the GPU the requests that arrive meanwhile are admitted by the
// next free worker, so batches overlap on the device and the batch size
// follows the load.
//
// Several batches on the device at once share the SMs, so the workers use the
// stepwise recoloring form (one launch per class step, no inter-block waits);
// a single-worker server keeps the tuning it was created with.
#include <algorithm>
#include <chrono>
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

// Stages a batch: graph y's local offsets (n + 1 of them) sit at
// loff[vbase + y ...] and its ids at idx[ebase ...].  One warp per vertex
// checks the row (the rules of gc_check_graph: offsets from 0 to nnz, never
// decreasing; ids in [0, n), no self-loop), writes the global offset and
// shifts the ids by the graph's vertex base.  A graph with a bad row gets
// bad[y] = 1 (its rows are left unshifted: the batch is run again without it).
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

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const int64_t* off = nullptr;  // the caller's CSR, n + 1 offsets and nnz ids
    const int32_t* idx = nullptr;
    int64_t n = 0, nnz = 0;
    int64_t bytes = 0;             // admitted device-memory estimate
    gc_batch_graph desc{};
    // result
    int32_t status = GC_PENDING;
    std::vector<int32_t> colors;
    gc_request_result res{};
};

// Device bytes one request holds while its batch runs: its CSR and colors,
// the coloring scratch (priority keys, two work lists, buckets, per-vertex
// graph index and win round) or the recoloring scratch (work list, alternate
// colors, per-class tables over at most min(n, max degree + X) + 1 classes),
// whichever is larger, with room to spare.
int64_t request_bytes(int64_t n, int64_t nnz, int64_t max_deg, int32_t X) {
    const int64_t classes = std::min<int64_t>(n, max_deg + X) + 2;
    return 16 * (n + 1) + 4 * nnz + 4 * n + 64 * n + 16 * (nnz / 256 + 1) + 256 * classes + 1024;
}

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
    void run_batch(const std::vector<Request*>& batch, cudaStream_t s, std::vector<gc_status>& each);
};

// Takes batches off the queue until the server stops and the queue is empty.
void gc_server::worker_main() {
    cudaSetDevice(device);
    set_thread_tuning(&tune);
    cudaStream_t s = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    for (;;) {
        std::vector<Request*> batch;
        int64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                return (!queue.empty() && in_use + queue.front()->bytes <= budget) ||
                       (stopping && queue.empty());
            });
            if (queue.empty()) break;  // stopping
            int64_t n_sum = 0;
            while (!queue.empty() && static_cast<int32_t>(batch.size()) < max_batch) {
                Request* r = queue.front();
                if (in_use + bytes + r->bytes > budget) break;
                if (n_sum + r->n > INT32_MAX) break;  // the batch CSR numbers vertices in int32
                queue.pop_front();
                batch.push_back(r);
                bytes += r->bytes;
                n_sum += r->n;
            }
            in_use += bytes;
            peak = std::max(peak, in_use);
            ++batches;
        }
        const double start = now_ms();
        std::vector<gc_status> each(batch.size(), GC_ERR_CUDA);
        if (have_stream) run_batch(batch, s, each);
        prof_collect();
        const double done = now_ms();
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use -= bytes;
            for (size_t i = 0; i < batch.size(); ++i) {
                Request* r = batch[i];
                const gc_status st = each[i];
                r->status = st;
                r->res.status = st;
                r->res.batch_size = static_cast<int32_t>(batch.size());
                r->res.start_ms = start;
                r->res.done_ms = done;
                if (st != GC_OK) r->colors.clear();
                ++completed;
                latencies.push_back(done - r->res.submit_ms);
            }
            last_done = std::max(last_done, done);
        }
        cv_work.notify_all();
        cv_done.notify_all();
    }
    if (have_stream) cudaStreamDestroy(s);
    set_thread_tuning(nullptr);
}

// Runs one batch; each[i] receives request i's status.  Requests whose CSR
// fails the staging check get GC_ERR_BAD_GRAPH and the rest run again
// without them; if the batch does not fit the device's free memory (memory
// held outside the server), its requests run one at a time.
void gc_server::run_batch(const std::vector<Request*>& batch, cudaStream_t s,
                          std::vector<gc_status>& each) {
    const int32_t ng = static_cast<int32_t>(batch.size());
    auto fail_all = [&](gc_status st) { std::fill(each.begin(), each.end(), st); };
    int64_t N = 0, E = 0;
    std::vector<Slot> slots(ng);
    std::vector<gc_batch_graph> desc(ng);
    for (int32_t i = 0; i < ng; ++i) {
        const Request* r = batch[i];
        slots[i] = Slot{N, E, r->n, r->nnz};
        desc[i] = r->desc;
        desc[i].vertex_base = N;
        N += r->n;
        E += r->nnz;
    }
    Scratch s_loff, s_off, s_idx, s_col, s_slot, s_bad;
    auto release = [&] {
        for (Scratch* x : {&s_loff, &s_off, &s_idx, &s_col, &s_slot, &s_bad}) x->reset();
    };
    auto one_at_a_time = [&] {
        release();
        for (int32_t i = 0; i < ng; ++i) {
            std::vector<gc_status> one(1);
            run_batch(std::vector<Request*>{batch[i]}, s, one);
            each[i] = one[0];
        }
    };
    if (!s_loff.alloc((N + ng) * sizeof(int64_t), s) || !s_off.alloc((N + 1) * sizeof(int64_t), s) ||
        !s_idx.alloc(E * sizeof(int32_t), s) || !s_col.alloc(N * sizeof(int32_t), s) ||
        !s_slot.alloc(ng * sizeof(Slot), s) || !s_bad.alloc(ng * sizeof(int32_t), s)) {
        if (ng == 1) return fail_all(GC_ERR_OOM);
        return one_at_a_time();
    }
    int64_t* loff = s_loff.as<int64_t>();
    int64_t* off = s_off.as<int64_t>();
    int32_t* idx = s_idx.as<int32_t>();
    int32_t* col = s_col.as<int32_t>();
    int32_t* bad = s_bad.as<int32_t>();
    cudaError_t e = cudaMemsetAsync(bad, 0, ng * sizeof(int32_t), s);
    for (int32_t i = 0; i < ng && e == cudaSuccess; ++i) {
        const Request* r = batch[i];
        e = cudaMemcpyAsync(loff + slots[i].vbase + i, r->off, (r->n + 1) * sizeof(int64_t),
                            cudaMemcpyDefault, s);
        if (e == cudaSuccess && r->nnz > 0)
            e = cudaMemcpyAsync(idx + slots[i].ebase, r->idx, r->nnz * sizeof(int32_t), cudaMemcpyDefault, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s_slot.p, slots.data(), ng * sizeof(Slot), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_all(cuda_status(e));
    const int grid = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((N * 32 + kBlock - 1) / kBlock, persistent_grid(tune))));
    GC_LAUNCH(KID_BATCH, s,
              k_srv_stage<<<grid, kBlock, 0, s>>>(loff, off, idx, s_slot.as<Slot>(), ng, N, E, bad));
    std::vector<int32_t> hbad(ng, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hbad.data(), bad, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_all(cuda_status(e));
    if (std::count(hbad.begin(), hbad.end(), 1) > 0) {
        std::vector<Request*> good;
        std::vector<int32_t> where;
        for (int32_t i = 0; i < ng; ++i) {
            if (hbad[i]) {
                each[i] = GC_ERR_BAD_GRAPH;
            } else {
                good.push_back(batch[i]);
                where.push_back(i);
            }
        }
        release();
        if (!good.empty()) {
            std::vector<gc_status> sub(good.size());
            run_batch(good, s, sub);
            for (size_t j = 0; j < good.size(); ++j) each[where[j]] = sub[j];
        }
        return;
    }

    Graph g{};
    g.off = off;
    g.idx = idx;
    g.n = static_cast<int32_t>(N);
    g.nnz = E;
    g.vec = (reinterpret_cast<uintptr_t>(idx) & 15u) == 0;
    std::vector<int32_t> rounds(ng, 0), maxc(ng, 0);
    const gc_status st = color_recolor_batch_device(g, desc.data(), ng, col, rounds.data(), maxc.data(),
                                                    nullptr, s);
    if (st == GC_ERR_OOM && ng > 1) return one_at_a_time();
    if (st != GC_OK) return fail_all(st);
    for (int32_t i = 0; i < ng && e == cudaSuccess; ++i) {
        Request* r = batch[i];
        r->colors.resize(static_cast<size_t>(r->n));
        e = cudaMemcpyAsync(r->colors.data(), col + slots[i].vbase, r->n * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s);
        r->res.rounds = rounds[i];
        r->res.max_color = maxc[i];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    fail_all(cuda_status(e));
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
    if (workers > 1) s->tune.recolor_mode = 1;
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
