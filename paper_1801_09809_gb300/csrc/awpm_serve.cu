// Request server of a context: awpm_submit / awpm_poll / awpm_wait.
//
// Continuous batching of independent matching requests.  A scheduler thread
// owns `slots` solve slots; each slot is an internal context with its own
// stream, workspace and instantiated solve graph.  Requests queue in arrival
// order; whenever a slot is free and the device bytes held by all slots plus
// what the request needs stay within the context's budget, the head of the
// queue (or, when the head does not fit, one of the next few requests that
// does) is admitted: its inputs are staged, its descriptor written and its
// graph launched on the slot's stream without waiting.  Requests therefore
// run concurrently on the device, and a new one starts as soon as an earlier
// one frees its slot; completion is detected by polling each slot's event.
// Each request is solved exactly as by awpm_improve on its own, so its
// result does not depend on what else is running.
//
// Memory: a request's need is estimated from n and nnz (nnz read from a
// device colptr at admission when the caller did not give it); a slot is
// given, for the solve it starts, a budget of what the other slots leave,
// so its workspace can never push the total past the context's budget;
// idle slots give their workspaces back when that lets a waiting request
// in.  Fairness: a request that later ones have overtaken kMaxPassed times
// is the only one admitted until it fits.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "awpm.h"
#include "awpm_ctx.h"

using namespace awpm;

namespace {

constexpr int kDefaultSlots = 4;
constexpr int kAdmitLookahead = 8;
constexpr int kMaxPassed = 16;

struct Item {
    uint64_t ticket = 0;
    awpm_problem p{};
    int state = 0;  // 0 queued, 1 running, 2 done
    int rc = AWPM_OK;
    awpm_stats st{};
    size_t need = 0;
    bool sized = false;  // nnz known (given, or read from colptr[n])
    bool host_in = true;
    int passed = 0;      // times a later request was admitted before this one
};

}  // namespace

struct awpm_server_impl {
    awpm_ctx *owner = nullptr;
    std::vector<awpm_ctx *> slots;
    std::vector<cudaStream_t> streams;  // non-blocking, one per slot
    std::vector<Item *> running;  // per slot
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Item *> queue;
    std::unordered_map<uint64_t, Item *> items;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t budget = 0;
    size_t peak = 0;               // most device bytes all slots held at once
    cudaStream_t aux = nullptr;    // reads colptr[n] of device inputs at admission
    std::thread th;
};

namespace {

bool host_side(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

size_t held_total(const awpm_server_impl *s)
{
    size_t h = 0;
    for (const awpm_ctx *c : s->slots)
        h += ctx_bytes_held(c);
    return h;
}

void finish_item(awpm_server_impl *s, Item *it, int rc)
{
    it->rc = rc;
    it->state = 2;
    s->cv_done.notify_all();
}

// Start `it` on free slot k (server lock held by the caller; released around
// the CUDA calls).  cap: the device bytes the slot may hold for this solve
// (0 = no limit).
void start(awpm_server_impl *s, std::unique_lock<std::mutex> &lk, int k, Item *it, size_t cap)
{
    NvtxRange nvtx_range("admit");
    it->state = 1;
    s->running[k] = it;
    awpm_ctx *c = s->slots[k];
    lk.unlock();
    Request r;
    r.n = it->p.n;
    r.nnz = it->p.nnz;
    r.colptr = it->p.colptr;
    r.rowidx = it->p.rowidx;
    r.weight = it->p.weight;
    r.mate_in = it->p.mate_in;
    r.mate_out = it->p.mate_out;
    int rc;
    {
        std::lock_guard<std::mutex> cl(c->mu);
        c->opt.mem_budget_bytes = cap;
        rc = ctx_enqueue(c, r);
        if (rc != AWPM_OK) {
            cudaStreamSynchronize(c->stream);
            cudaGetLastError();
            c->pend.active = false;
        }
        if (rc == AWPM_ERR_BUDGET && cap) {
            // buffers kept from earlier, differently shaped problems can
            // leave too little room: start again from an empty workspace
            // (the request's estimate fits the cap)
            ctx_trim(c);
            rc = ctx_enqueue(c, r);
            if (rc != AWPM_OK) {
                cudaStreamSynchronize(c->stream);
                cudaGetLastError();
                c->pend.active = false;
            }
        }
    }
    lk.lock();
    const size_t h = held_total(s);
    if (h > s->peak)
        s->peak = h;
    if (rc != AWPM_OK) {
        s->running[k] = nullptr;
        finish_item(s, it, rc);
    }
}

// Make the request's need exact: with nnz not given and colptr in device
// memory, read colptr[n] (a 4-byte copy on the server's own stream).
void size_item(awpm_server_impl *s, Item *it)
{
    if (it->sized)
        return;
    it->sized = true;
    int32_t nnz = it->p.nnz;
    if (nnz < 0 && it->p.n > 0 && it->p.colptr) {
        int32_t v = -1;
        if (cudaMemcpyAsync(&v, it->p.colptr + it->p.n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            s->aux) == cudaSuccess &&
            cudaStreamSynchronize(s->aux) == cudaSuccess) {
            nnz = v;
            it->p.nnz = v;
        } else {
            cudaGetLastError();  // the solve itself reports the bad pointer
        }
    }
    it->need = ctx_bytes_needed(it->p.n, nnz > 0 ? nnz : 0, it->host_in, s->owner->opt.lookup,
                                s->owner->opt.select);
}

// Pick the queued request to start on free slot k, or -1.  Requests that can
// never fit the budget are finished with AWPM_ERR_BUDGET on the way.
int pick_request(awpm_server_impl *s, int k, bool *progress)
{
    for (;;) {
        const int look = (int)s->queue.size() < kAdmitLookahead ? (int)s->queue.size()
                                                                 : kAdmitLookahead;
        bool failed = false;
        for (int x = 0; x < look; ++x) {
            Item *it = s->queue[x];
            size_item(s, it);
            if (s->budget && it->need > s->budget) {
                s->queue.erase(s->queue.begin() + x);
                finish_item(s, it, AWPM_ERR_BUDGET);
                *progress = true;
                failed = true;
                break;
            }
        }
        if (!failed)
            break;
    }
    if (s->queue.empty())
        return -1;
    if (!s->budget)
        return 0;
    // a head overtaken often enough goes next, alone
    const int look = s->queue.front()->passed >= kMaxPassed
                         ? 1
                         : ((int)s->queue.size() < kAdmitLookahead ? (int)s->queue.size()
                                                                   : kAdmitLookahead);
    const size_t held = held_total(s);
    const size_t mine = ctx_bytes_held(s->slots[k]);
    size_t idle = 0;  // workspace of the other idle slots (can be given back)
    for (size_t q = 0; q < s->slots.size(); ++q)
        if ((int)q != k && !s->running[q])
            idle += ctx_bytes_held(s->slots[q]);
    for (int x = 0; x < look; ++x) {
        const Item *it = s->queue[x];
        const size_t grow = it->need > mine ? it->need - mine : 0;
        if (held + grow <= s->budget)
            return x;
        if (held - idle + grow <= s->budget) {
            // it fits once the idle slots free their workspaces
            for (size_t q = 0; q < s->slots.size(); ++q)
                if ((int)q != k && !s->running[q] && ctx_bytes_held(s->slots[q])) {
                    std::lock_guard<std::mutex> cl(s->slots[q]->mu);
                    ctx_trim(s->slots[q]);
                }
            return x;
        }
    }
    return -1;
}

void scheduler(awpm_server_impl *s)
{
    cudaSetDevice(s->owner->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        // reap finished slots
        for (size_t k = 0; k < s->slots.size(); ++k) {
            Item *it = s->running[k];
            if (!it)
                continue;
            awpm_ctx *c = s->slots[k];
            const cudaError_t q = cudaEventQuery(c->ev_b);
            if (q == cudaErrorNotReady)
                continue;
            if (q != cudaSuccess)
                cudaGetLastError();
            int rc;
            {
                std::lock_guard<std::mutex> cl(c->mu);
                rc = ctx_finish(c, &it->st, nullptr);
            }
            s->running[k] = nullptr;
            finish_item(s, it, rc);
            progress = true;
        }
        // admit queued requests onto free slots within the budget
        for (size_t k = 0; k < s->slots.size() && !s->queue.empty(); ++k) {
            if (s->running[k])
                continue;
            const int pick = pick_request(s, (int)k, &progress);
            if (pick < 0)
                continue;
            Item *it = s->queue[pick];
            if (pick > 0)
                s->queue.front()->passed += 1;
            s->queue.erase(s->queue.begin() + pick);
            // the slot may hold what the other slots leave of the budget
            const size_t others = held_total(s) - ctx_bytes_held(s->slots[k]);
            const size_t cap = s->budget ? (s->budget > others ? s->budget - others : 1) : 0;
            start(s, lk, (int)k, it, cap);
            progress = true;
        }
        bool busy = false;
        for (Item *it : s->running)
            busy |= it != nullptr;
        if (s->stop && !busy)
            break;
        if (!busy && s->queue.empty()) {
            s->cv_work.wait(lk);
        } else if (!progress) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

awpm_server_impl *server_of(awpm_ctx *ctx, int *rc)
{
    *rc = AWPM_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->server)
        return ctx->server;
    awpm_server_impl *s = new (std::nothrow) awpm_server_impl();
    if (!s) {
        *rc = AWPM_ERR_OOM;
        return nullptr;
    }
    s->owner = ctx;
    s->budget = ctx->opt.mem_budget_bytes;
    const int nslots = ctx->opt.slots > 0 ? ctx->opt.slots : kDefaultSlots;
    cudaSetDevice(ctx->device);
    if (cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        *rc = AWPM_ERR_CUDA;
        return nullptr;
    }
    for (int k = 0; k < nslots; ++k) {
        // slot streams do not synchronise with the legacy default stream:
        // requests run beside whatever the caller's threads do
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (awpm_ctx *x : s->slots)
                awpm_destroy(x);
            for (cudaStream_t y : s->streams)
                cudaStreamDestroy(y);
            cudaStreamDestroy(s->aux);
            delete s;
            *rc = AWPM_ERR_CUDA;
            return nullptr;
        }
        s->streams.push_back(st);
        awpm_options o = ctx->opt;
        o.stream = st;
        o.mem_budget_bytes = 0;  // the server enforces the budget over all slots
        o.flags = 0;
        o.slots = 0;
        o.device = ctx->device;
        awpm_ctx *c = nullptr;
        int r = awpm_create(&c, &o);
        if (r != AWPM_OK) {
            for (awpm_ctx *x : s->slots)
                awpm_destroy(x);
            for (cudaStream_t y : s->streams)
                cudaStreamDestroy(y);
            cudaStreamDestroy(s->aux);
            delete s;
            *rc = r;
            return nullptr;
        }
        s->slots.push_back(c);
    }
    s->running.assign(s->slots.size(), nullptr);
    s->th = std::thread(scheduler, s);
    ctx->server = s;
    return s;
}

}  // namespace

extern "C" {

void awpm_server_shutdown(awpm_ctx *ctx)
{
    awpm_server_impl *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s = ctx->server;
        ctx->server = nullptr;
    }
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests that never started are dropped: their arrays are released
        for (Item *it : s->queue)
            finish_item(s, it, AWPM_ERR_NOT_FOUND);
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->th.join();
    for (awpm_ctx *c : s->slots)
        awpm_destroy(c);
    for (cudaStream_t st : s->streams)
        cudaStreamDestroy(st);
    if (s->aux)
        cudaStreamDestroy(s->aux);
    for (auto &kv : s->items)
        delete kv.second;
    delete s;
}

void awpm_server_memory(awpm_ctx *ctx, size_t *held, size_t *peak)
{
    *held = 0;
    *peak = 0;
    awpm_server_impl *s;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s = ctx->server;
    }
    if (!s)
        return;
    std::lock_guard<std::mutex> lk(s->mu);
    *held = held_total(s);
    *peak = s->peak;
}

int awpm_submit(awpm_ctx *ctx, const awpm_problem *p, uint64_t *ticket)
{
    NvtxRange nvtx_range("awpm_submit");
    if (!ctx || !p || !ticket || p->n < 0)
        return AWPM_ERR_INVALID_ARG;
    int rc;
    awpm_server_impl *s = server_of(ctx, &rc);
    if (!s)
        return rc;
    Item *it = new (std::nothrow) Item();
    if (!it)
        return AWPM_ERR_OOM;
    it->p = *p;
    it->host_in = host_side(p->rowidx);
    if (it->p.nnz < 0 && p->colptr && host_side(p->colptr))
        it->p.nnz = p->colptr[p->n];
    // a device colptr without nnz is read at admission (size_item)
    it->sized = it->p.nnz >= 0 || p->n == 0 || !p->colptr;
    it->need = ctx_bytes_needed(p->n, it->p.nnz > 0 ? it->p.nnz : 0, it->host_in,
                                ctx->opt.lookup, ctx->opt.select);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        it->ticket = s->next_ticket++;
        s->items[it->ticket] = it;
        s->queue.push_back(it);
    }
    s->cv_work.notify_all();
    *ticket = it->ticket;
    return AWPM_OK;
}

int awpm_poll(awpm_ctx *ctx, uint64_t ticket, int *done, awpm_stats *stats)
{
    if (!ctx || !done)
        return AWPM_ERR_INVALID_ARG;
    awpm_server_impl *s;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s = ctx->server;
    }
    if (!s)
        return AWPM_ERR_NOT_FOUND;
    std::lock_guard<std::mutex> lk(s->mu);
    auto f = s->items.find(ticket);
    if (f == s->items.end())
        return AWPM_ERR_NOT_FOUND;
    Item *it = f->second;
    if (it->state != 2) {
        *done = 0;
        return AWPM_OK;
    }
    *done = 1;
    if (stats)
        *stats = it->st;
    const int rc = it->rc;
    s->items.erase(f);
    delete it;
    return rc;
}

int awpm_cancel(awpm_ctx *ctx, uint64_t ticket, int *cancelled)
{
    if (!ctx || !cancelled)
        return AWPM_ERR_INVALID_ARG;
    *cancelled = 0;
    awpm_server_impl *s;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s = ctx->server;
    }
    if (!s)
        return AWPM_ERR_NOT_FOUND;
    std::lock_guard<std::mutex> lk(s->mu);
    auto f = s->items.find(ticket);
    if (f == s->items.end())
        return AWPM_ERR_NOT_FOUND;
    Item *it = f->second;
    if (it->state == 0) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == it) {
                s->queue.erase(q);
                break;
            }
        finish_item(s, it, AWPM_ERR_CANCELLED);
        *cancelled = 1;
    }
    return AWPM_OK;
}

int awpm_wait(awpm_ctx *ctx, uint64_t ticket, awpm_stats *stats)
{
    if (!ctx)
        return AWPM_ERR_INVALID_ARG;
    awpm_server_impl *s;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s = ctx->server;
    }
    if (!s)
        return AWPM_ERR_NOT_FOUND;
    std::unique_lock<std::mutex> lk(s->mu);
    auto f = s->items.find(ticket);
    if (f == s->items.end())
        return AWPM_ERR_NOT_FOUND;
    Item *it = f->second;
    s->cv_done.wait(lk, [it] { return it->state == 2; });
    if (stats)
        *stats = it->st;
    const int rc = it->rc;
    s->items.erase(ticket);
    delete it;
    return rc;
}

}  // extern "C"
