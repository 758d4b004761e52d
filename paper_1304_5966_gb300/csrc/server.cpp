// server.cpp -- sw_server_*: continuous batching of alignment requests.
//
// Requests (score-only or full alignment, any size) are submitted from any host
// thread and queued with host copies of their sequences.  W worker threads, each
// with its own context, CUDA stream and slice of the parent context's device
// workspace, repeatedly take every queued request that fits their memory slice
// (first come first served, same scoring scheme) and run them as one batch
// (sw_align_batch: one persistent launch over all their row bands).  Requests
// that arrive while a worker is busy are picked up by the next free worker, whose
// kernels run concurrently on its own stream, so new work overlaps work already
// on the device instead of waiting for it.  Admission is by device-memory
// budget: a request whose estimated footprint exceeds a worker's slice is
// refused (SW_EBUSY), as is a submit that would push the queued footprint past
// the queue limit.  Results are bit-identical to the same request run alone: the
// batch path computes each pair independently.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "ctx.h"

namespace {

struct Req {
    uint64_t id = 0;
    std::vector<uint8_t> a, b;
    int32_t flags = 0;
    sw_scheme scheme{};
    std::vector<int8_t> matrix;
    size_t need = 0;
    sw_result res{};
    int status = SW_EPENDING;
    bool done = false;
    bool running = false;
};

bool same_scheme(const Req &x, const Req &y)
{
    return x.scheme.alphabet == y.scheme.alphabet && x.scheme.match == y.scheme.match &&
           x.scheme.mismatch == y.scheme.mismatch && x.scheme.gap_open == y.scheme.gap_open &&
           x.scheme.gap_extend == y.scheme.gap_extend && x.matrix == y.matrix &&
           (x.flags & SW_FLAG_NO_PRUNE) == (y.flags & SW_FLAG_NO_PRUNE);
}

// device footprint estimate of one request inside a batch (bytes)
size_t footprint(int64_t n, int64_t m, bool align)
{
    const int64_t mn = std::min(n, m), mx = std::max(n, m);
    size_t f = (size_t)(n + m) * 2 + (size_t)mn * 8 + (size_t)mx / 16 + (64u << 10);
    if (align) {
        // reverse copies + label bus + checkpoint rows of the level-0 pass (one per
        // 256 rows, bounded by the driver's choice of spacing) + leaves
        f += (size_t)(n + m) + (size_t)mn * 16 + std::min<size_t>((size_t)(mx / 256) * mn * 16, 1ull << 30);
        f += (size_t)(n + m) * 8;
    }
    return f;
}

}  // namespace

struct sw_server {
    sw_ctx *parent = nullptr;
    std::vector<sw_ctx *> workers;
    std::vector<cudaStream_t> streams;
    std::vector<void *> slices;
    std::vector<std::thread> threads;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> all;
    uint64_t next_id = 1;
    bool stop = false;
    size_t slice_bytes = 0;
    size_t queued_bytes = 0;
    size_t queue_limit = 0;

    void worker_loop(int w);
};

void sw_server::worker_loop(int w)
{
    sw_ctx *ctx = workers[w];
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<Req *> batch;
        {
            std::unique_lock<std::mutex> g(mu);
            cv_work.wait(g, [&] { return stop || !queue.empty(); });
            if (stop && queue.empty()) return;
            // everything queued that fits this worker's slice, same scheme as the head
            size_t used = 0;
            Req *head = queue.front();
            for (auto it = queue.begin(); it != queue.end();) {
                Req *r = *it;
                if (same_scheme(*r, *head) && used + r->need <= slice_bytes) {
                    used += r->need;
                    r->running = true;
                    batch.push_back(r);
                    queued_bytes -= r->need;
                    it = queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        // one batch call per kind: score-only, then alignments
        for (int kind = 0; kind < 2; ++kind) {
            std::vector<Req *> grp;
            for (Req *r : batch)
                if (((r->flags & SW_FLAG_SCORE_ONLY) != 0) == (kind == 0)) grp.push_back(r);
            if (grp.empty()) continue;
            std::vector<sw_pair> pairs(grp.size());
            for (size_t k = 0; k < grp.size(); ++k)
                pairs[k] = sw_pair{grp[k]->a.data(), (int64_t)grp[k]->a.size(), grp[k]->b.data(),
                                   (int64_t)grp[k]->b.size()};
            std::vector<sw_result> outs(grp.size());
            sw_scheme sch = grp[0]->scheme;
            sch.matrix = grp[0]->matrix.empty() ? nullptr : grp[0]->matrix.data();
            const int32_t fl = (kind == 0 ? SW_FLAG_SCORE_ONLY : 0) | (grp[0]->flags & SW_FLAG_NO_PRUNE);
            const int st = sw_align_batch(ctx, pairs.data(), (int32_t)pairs.size(), &sch, fl, outs.data());
            std::lock_guard<std::mutex> g(mu);
            for (size_t k = 0; k < grp.size(); ++k) {
                if (st == SW_OK) grp[k]->res = outs[k];
                else sw_result_free(&outs[k]);
                grp[k]->status = st;
                grp[k]->done = true;
                grp[k]->running = false;
            }
            cv_done.notify_all();
        }
    }
}

extern "C" {

int sw_server_create(sw_ctx *ctx, int32_t workers, uint64_t device_budget, sw_server **out)
{
    if (!ctx || !out || workers < 1 || workers > 16) return SW_EINVAL;
    *out = nullptr;
    sw_server *s = new (std::nothrow) sw_server();
    if (!s) return SW_ENOMEM;
    s->parent = ctx;
    cudaSetDevice(ctx->device);
    const size_t avail = ctx->arena.largest_free();
    size_t budget = device_budget ? (size_t)device_budget : avail;
    budget = std::min(budget, avail);
    s->slice_bytes = (budget / (size_t)workers) & ~(size_t)255;
    if (s->slice_bytes < (64u << 20)) { delete s; return SW_ENOMEM; }
    s->queue_limit = s->slice_bytes * (size_t)workers * 4;
    for (int w = 0; w < workers; ++w) {
        void *slice = ctx->arena.alloc(s->slice_bytes);
        cudaStream_t st = nullptr;
        sw_ctx *wc = nullptr;
        if (!slice || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            sw_ctx_create(ctx->device, st, slice, s->slice_bytes, &wc) != SW_OK) {
            if (slice) ctx->arena.release(slice);
            if (st) cudaStreamDestroy(st);
            for (size_t k = 0; k < s->workers.size(); ++k) {
                sw_ctx_destroy(s->workers[k]);
                cudaStreamDestroy(s->streams[k]);
                ctx->arena.release(s->slices[k]);
            }
            delete s;
            return SW_ENOMEM;
        }
        wc->opt = ctx->opt;
        s->workers.push_back(wc);
        s->streams.push_back(st);
        s->slices.push_back(slice);
    }
    for (int w = 0; w < workers; ++w) s->threads.emplace_back([s, w] { s->worker_loop(w); });
    *out = s;
    return SW_OK;
}

int sw_server_submit(sw_server *s, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                     const sw_scheme *scheme, int32_t flags, uint64_t *ticket)
{
    if (!s || !scheme || !ticket || n < 0 || m < 0 || (n && !a) || (m && !b)) return SW_EINVAL;
    if (flags & SW_FLAG_DEVICE_INPUT) return SW_EINVAL;          // requests are host data
    if (scheme->alphabet < 1 || scheme->alphabet > 8) return SW_EINVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return SW_ENOMEM;
    r->a.assign(a, a + n);
    r->b.assign(b, b + m);
    r->flags = flags;
    r->scheme = *scheme;
    if (scheme->matrix) r->matrix.assign(scheme->matrix, scheme->matrix + scheme->alphabet * scheme->alphabet);
    r->scheme.matrix = nullptr;
    r->need = footprint(n, m, !(flags & SW_FLAG_SCORE_ONLY));
    std::lock_guard<std::mutex> g(s->mu);
    if (r->need > s->slice_bytes || s->queued_bytes + r->need > s->queue_limit) { delete r; return SW_EBUSY; }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
    s->queued_bytes += r->need;
    *ticket = r->id;
    s->cv_work.notify_one();
    return SW_OK;
}

int sw_server_poll(sw_server *s, uint64_t ticket, sw_result *out, int64_t timeout_us)
{
    if (!s || !out) return SW_EINVAL;
    std::unique_lock<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SW_EINVAL;
    Req *r = it->second;
    if (!r->done) {
        if (timeout_us < 0) s->cv_done.wait(g, [&] { return r->done; });
        else s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    }
    if (!r->done) return SW_EPENDING;
    const int st = r->status;
    *out = r->res;                     // the caller now owns the CIGAR
    s->all.erase(it);
    delete r;
    return st;
}

int sw_server_cancel(sw_server *s, uint64_t ticket)
{
    if (!s) return SW_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SW_EINVAL;
    Req *r = it->second;
    if (r->running || r->done) return SW_EBUSY;
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
    s->queued_bytes -= r->need;
    s->all.erase(it);
    delete r;
    return SW_OK;
}

void sw_server_destroy(sw_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    for (size_t k = 0; k < s->workers.size(); ++k) {
        sw_ctx_destroy(s->workers[k]);
        cudaStreamDestroy(s->streams[k]);
        s->parent->arena.release(s->slices[k]);
    }
    for (auto &kv : s->all) { sw_result_free(&kv.second->res); delete kv.second; }
    delete s;
}

}  // extern "C"
