// Serving: continuous batching of gridding requests on one context.
//
// bg_submit returns a ticket for a request. When nothing is queued ahead of
// it and a stream slot and the context's HBM budget are free, the calling
// thread issues it at once; otherwise it is queued, and a dispatcher thread
// admits queued requests in arrival order whenever a slot is free and the
// budget covers the request's estimated device memory; each admitted request
// runs on its slot's stream (host copy into pinned staging + bounding box on
// the host, async upload and hash build, interpolation, async copy of the
// grids back), so requests that arrive while others run overlap with them on
// the device. An event recorded behind the work marks the request's end; a
// completion thread polls the events of the running slots, copies each
// finished request's grids into the caller's buffers and completes its ticket
// (a polled event ends a request sooner than a host function queued on the
// stream, which waits for a driver thread to wake). While the device works,
// the completion thread writes one byte of every page of the caller's output
// arrays, so that fresh arrays take their page faults then rather than in
// the copy-out; the copy-out of large grids is shared with three helper
// threads, which spin while requests are in flight and sleep otherwise (one
// core copies about 20 GB/s: a 512 x 512 kriging tile's 2 MB took 60 us
// alone, 18 us shared). bg_poll never blocks, bg_wait blocks up to a timeout.
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bg_internal.h"

namespace bg {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kDefaultSlots = 8;

struct Slot;

struct Ticket {
    uint64_t id = 0;
    bg_request req{};
    int64_t nodes = 0;
    size_t reserve = 0;          // device bytes reserved at admission
    bg_status status = BG_PENDING;
    double t_submit = 0, t_start = 0, t_done = 0;
    bool done = false;
    Slot* slot = nullptr;
    bg_soundings_s* snd = nullptr;
    void* d_out = nullptr;
    size_t d_out_bytes = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;  // recorded behind the request's last copy
    bool busy = false;
    bool inflight = false;       // issued, end event not yet seen (server lock)
    bool touched = false;        // the caller's output pages written once (completion thread)
    char* pin_in = nullptr;      // pinned staging: x, y, z
    size_t pin_in_bytes = 0;
    float* pin_out = nullptr;    // pinned staging: depth (+ variance)
    size_t pin_out_bytes = 0;
    Ticket* ticket = nullptr;
    Server* server = nullptr;
};

}  // namespace

struct Server {
    bg_ctx_s* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work;   // dispatcher: new request or a slot freed
    std::condition_variable cv_done;   // waiters: a ticket completed
    std::condition_variable cv_flight; // completion thread: a request was issued
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, Ticket*> tickets;
    std::vector<Slot> slots;
    uint64_t next_id = 1;
    size_t reserved = 0;               // device bytes reserved by running requests
    int inflight = 0;                  // slots issued and not yet completed
    int issuing = 0;                   // slots admitted, still being issued
    bool stop = false;
    bool stop_completer = false;
    std::thread worker;
    std::thread completer;
    // copy-out helpers: each copies one share of a finished request's grids
    // beside the completion thread (copy_gen announces a copy, copy_pending
    // counts the helpers still copying)
    static constexpr int kHelpers = 3;
    std::thread helpers[kHelpers];
    std::atomic<int> copy_gen{0}, copy_pending{0};
    std::atomic<bool> helpers_spin{false}, helpers_stop{false};
    std::mutex hmu;
    std::condition_variable cv_helpers;
    char* cdst[2] = {nullptr, nullptr};
    const char* csrc[2] = {nullptr, nullptr};
    size_t cbytes = 0;
    Clock::time_point t0;
    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }
};

namespace {

size_t request_bytes(const bg_request& r) {
    const int64_t m = (int64_t)r.nx * r.ny;
    size_t b = soundings_bytes_estimate(r.n, r.n) + (size_t)m * 4 * (r.var_out ? 2 : 1);
    if (r.method == 1) {
        // kriging keeps a neighbour-id buffer of at most ~1 GiB (2^28 ids)
        const int64_t ids = std::min<int64_t>(m * r.k, ((int64_t)1 << 28) + (int64_t)8 * r.nx * r.k);
        b += (size_t)ids * 4;
    }
    return b + 4096;
}

// Write one byte of every page of [p, p + bytes): a caller's output array
// fresh from the allocator takes its page faults here, while the device still
// works, instead of in the copy-out. Output contents are unspecified until the
// ticket completes.
void touch_pages(void* p, size_t bytes) {
    static const size_t ps = (size_t)std::max(4096L, sysconf(_SC_PAGESIZE));
    if (!p || bytes == 0) return;
    volatile char* c = static_cast<volatile char*>(p);
    for (size_t off = 0; off < bytes; off += ps) c[off] = 0;
    c[bytes - 1] = 0;
}

// Copier j of kHelpers + 1 copies its share (64-byte multiples, the last
// share takes the rest) of each of the announced arrays.
void copy_share(Server* sv, int j) {
    constexpr int P = Server::kHelpers + 1;
    const size_t n = sv->cbytes, q = (n / P) & ~(size_t)63;
    const size_t a = q * j, b = (j == P - 1) ? n : q * (j + 1);
    if (b <= a) return;
    for (int k = 0; k < 2; ++k)
        if (sv->cdst[k]) std::memcpy(sv->cdst[k] + a, sv->csrc[k] + a, b - a);
}

// Helper j: sleeps until requests are in flight, then spins (yielding) and
// takes its share of every copy announced, until the completion thread goes
// idle again.
void helper(Server* sv, int j) {
    int seen = sv->copy_gen.load(std::memory_order_acquire);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(sv->hmu);
            sv->cv_helpers.wait(lk, [&] { return sv->helpers_spin.load() || sv->helpers_stop.load(); });
        }
        if (sv->helpers_stop.load()) return;
        while (sv->helpers_spin.load(std::memory_order_acquire)) {
            const int g = sv->copy_gen.load(std::memory_order_acquire);
            if (g != seen) {
                seen = g;
                copy_share(sv, j + 1);
                sv->copy_pending.fetch_sub(1, std::memory_order_acq_rel);
            } else {
                std::this_thread::yield();
            }
        }
    }
}

// dst0 <- src0 and, when dst1 is not null, dst1 <- src1 (bytes each): alone
// below 256 KB, else shared with the helpers (completion thread only; the
// helpers are spinning whenever a request is in flight).
void copy_out(Server* sv, char* dst0, const char* src0, char* dst1, const char* src1, size_t bytes) {
    if (bytes < ((size_t)256 << 10) || !sv->helpers_spin.load()) {
        std::memcpy(dst0, src0, bytes);
        if (dst1) std::memcpy(dst1, src1, bytes);
        return;
    }
    sv->cdst[0] = dst0;
    sv->csrc[0] = src0;
    sv->cdst[1] = dst1;
    sv->csrc[1] = src1;
    sv->cbytes = bytes;
    sv->copy_pending.store(Server::kHelpers, std::memory_order_relaxed);
    sv->copy_gen.fetch_add(1, std::memory_order_acq_rel);
    copy_share(sv, 0);
    while (sv->copy_pending.load(std::memory_order_acquire) > 0) {
    }
}

// A slot's request has finished on the device (or failed): copy its grids
// out of pinned staging into the caller's buffers, then free the slot and
// complete the ticket. Completion thread, server lock not held.
void complete_slot(Slot* sl) {
    Server* sv = sl->server;
    Ticket* t = sl->ticket;
    const int64_t m = t->nodes;
    if (t->status == BG_PENDING) {
        copy_out(sv, (char*)t->req.depth_out, (const char*)sl->pin_out, (char*)t->req.var_out,
                 (const char*)(sl->pin_out + m), (size_t)m * 4);
        t->status = BG_OK;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    t->t_done = sv->now_us();
    t->done = true;
    sl->busy = false;
    sl->inflight = false;
    sl->ticket = nullptr;
    sv->inflight -= 1;
    sv->reserved -= t->reserve;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

// Poll the end events of the issued slots while any is in flight (the copy
// helpers spinning beside); sleep on cv_flight otherwise (and the helpers).
void completer(Server* sv) {
    cudaSetDevice(sv->ctx->device);
    std::vector<Slot*> live;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (sv->inflight == 0) sv->helpers_spin.store(false);
        while (sv->inflight == 0 && (sv->issuing > 0 || !sv->stop_completer))
            sv->cv_flight.wait(lk);
        if (sv->inflight == 0) break;  // stopping, nothing left or being issued
        if (!sv->helpers_spin.load()) {
            {
                std::lock_guard<std::mutex> hl(sv->hmu);
                sv->helpers_spin.store(true);
            }
            sv->cv_helpers.notify_all();
        }
        live.clear();
        for (auto& s : sv->slots)
            if (s.inflight) live.push_back(&s);
        lk.unlock();
        bool any = false;
        for (Slot* sl : live) {
            if (!sl->touched) {
                const size_t mb = (size_t)sl->ticket->nodes * 4;
                touch_pages(sl->ticket->req.depth_out, mb);
                touch_pages(sl->ticket->req.var_out, mb);
                sl->touched = true;
            }
            const cudaError_t e = cudaEventQuery(sl->done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess && sl->ticket->status == BG_PENDING)
                sl->ticket->status = cuda_fail(e, "request on the device");
            complete_slot(sl);
            any = true;
        }
        if (!any) std::this_thread::yield();
        lk.lock();
    }
}

bg_status grow_pinned(void** p, size_t* have, size_t need) {
    if (*have >= need) return BG_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    const size_t sz = need + need / 4;
    const cudaError_t e = cudaHostAlloc(p, sz, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc");
    *have = sz;
    return BG_OK;
}

// Bounding box, valid count and out-of-range count of the valid soundings
// (depth not NaN). Branch-free, so the compiler can vectorize it.
__attribute__((optimize("O3"))) HostBBox host_bbox(const int32_t* x, const int32_t* y,
                                                    const float* z, int64_t n) {
    const int32_t lim = 1 << 30;
    int32_t x0 = INT32_MAX, y0 = INT32_MAX, x1 = INT32_MIN, y1 = INT32_MIN;
    int64_t nv = 0, oor = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t xi = x[i], yi = y[i];
        const bool v = z[i] == z[i];
        x0 = std::min(x0, v ? xi : INT32_MAX);
        y0 = std::min(y0, v ? yi : INT32_MAX);
        x1 = std::max(x1, v ? xi : INT32_MIN);
        y1 = std::max(y1, v ? yi : INT32_MIN);
        nv += v;
        oor += v & ((xi <= -lim) | (xi >= lim) | (yi <= -lim) | (yi >= lim));
    }
    return HostBBox{x0, y0, x1, y1, nv, (int32_t)oor};
}

// Issue one request on its slot (dispatcher thread, server lock not held).
bg_status launch_request(Server* sv, Slot* sl, Ticket* t) {
    NvtxRange nvtx("serve request");
    bg_ctx_s* ctx = sv->ctx;
    const bg_request& r = t->req;
    const int64_t n = r.n, m = t->nodes;
    cudaStream_t st = sl->stream;
    bg_status rc = grow_pinned((void**)&sl->pin_in, &sl->pin_in_bytes, (size_t)std::max<int64_t>(n, 1) * 12);
    if (rc != BG_OK) return rc;
    rc = grow_pinned((void**)&sl->pin_out, &sl->pin_out_bytes, (size_t)m * 8);
    if (rc != BG_OK) return rc;

    // copy into pinned staging, then the bounding box of the valid soundings
    int32_t* px = (int32_t*)sl->pin_in;
    int32_t* py = px + n;
    float* pz = (float*)(py + n);
    if (n > 0) {
        std::memcpy(px, r.x_cm, (size_t)n * 4);
        std::memcpy(py, r.y_cm, (size_t)n * 4);
        std::memcpy(pz, r.z_m, (size_t)n * 4);
    }
    HostBBox bb = host_bbox(px, py, pz, n);
    t->snd = new (std::nothrow) bg_soundings_s();
    if (!t->snd) return BG_ERR_INTERNAL;
    t->snd->ctx = ctx;
    rc = build_soundings(ctx, px, py, pz, n, 0, 0, st, t->snd, &bb);
    if (rc != BG_OK) return rc;
    t->d_out_bytes = (size_t)m * 4 * (r.var_out ? 2 : 1);
    rc = dalloc(ctx, &t->d_out, t->d_out_bytes, st);
    if (rc != BG_OK) return rc;
    float* d_depth = (float*)t->d_out;
    float* d_var = r.var_out ? d_depth + m : nullptr;
    const GridView g{r.x0_cm, r.y0_cm, r.cell_cm, r.nx, r.ny};
    if (r.method == 0) {
        rc = launch_idw(t->snd, g, r.k, r.power, d_depth, nullptr, st);
    } else {
        const bg_variogram& v = r.variogram;
        const OkParams p{v.model, v.nugget_m2, v.sill_m2 - v.nugget_m2, v.sill_m2, 1.0f / v.range_m};
        rc = launch_okrige(t->snd, g, r.k, p, d_depth, d_var, nullptr, st);
    }
    if (rc != BG_OK) return rc;
    BG_CUDA(cudaMemcpyAsync(sl->pin_out, t->d_out, t->d_out_bytes, cudaMemcpyDeviceToHost, st));
    return BG_OK;
}

// Launch an admitted request on its slot and hand the slot to the completion
// thread (server lock not held; the slot is already marked busy).
void issue(Server* sv, Slot* sl, Ticket* t) {
    bg_status rc = launch_request(sv, sl, t);
    cudaStream_t st = sl->stream;
    if (rc != BG_OK) {
        t->status = rc;  // the completion skips the copy-out
        cudaStreamSynchronize(st);
    }
    // stream-ordered releases queued behind the copy-out
    if (t->snd) {
        free_soundings(t->snd, st);
        delete t->snd;
        t->snd = nullptr;
    }
    if (t->d_out) {
        dfree(sv->ctx, t->d_out, t->d_out_bytes, st);
        t->d_out = nullptr;
    }
    const cudaError_t e = cudaEventRecord(sl->done, st);
    if (e != cudaSuccess) {
        t->status = cuda_fail(e, "cudaEventRecord");
        cudaStreamSynchronize(st);
    }
    {
        // hand the slot to the completion thread (an event that could not
        // be recorded is complete at once: the stream was synchronized)
        std::lock_guard<std::mutex> g(sv->mu);
        sl->touched = false;
        sl->inflight = true;
        sv->inflight += 1;
        sv->issuing -= 1;
    }
    sv->cv_flight.notify_one();
}

// A free slot for the request at the head of the queue, if one is free and
// the budget admits it (server lock held); marks the slot busy.
Slot* admit(Server* sv, Ticket* t) {
    Slot* free_slot = nullptr;
    for (auto& s : sv->slots)
        if (!s.busy) {
            free_slot = &s;
            break;
        }
    if (!free_slot) return nullptr;
    const size_t budget = sv->ctx->budget;
    if (!(budget == 0 || sv->reserved == 0 || sv->reserved + t->reserve <= budget)) return nullptr;
    free_slot->busy = true;
    free_slot->ticket = t;
    t->slot = free_slot;
    sv->reserved += t->reserve;
    sv->issuing += 1;
    t->t_start = sv->now_us();
    return free_slot;
}

void dispatcher(Server* sv) {
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (sv->stop && sv->queue.empty()) break;
        Ticket* t = sv->queue.empty() ? nullptr : sv->queue.front();
        Slot* free_slot = t ? admit(sv, t) : nullptr;
        if (!free_slot) {
            sv->cv_work.wait(lk);
            continue;
        }
        sv->queue.pop_front();
        lk.unlock();

        issue(sv, free_slot, t);
        lk.lock();
    }
}

Server* get_server(bg_ctx_s* ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->server) return ctx->server;
    Server* sv = new Server();
    sv->ctx = ctx;
    sv->t0 = Clock::now();
    sv->slots.resize(kDefaultSlots);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    for (auto& s : sv->slots) {
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        s.server = sv;
    }
    cudaSetDevice(prev);
    sv->worker = std::thread(dispatcher, sv);
    sv->completer = std::thread(completer, sv);
    for (int j = 0; j < Server::kHelpers; ++j) sv->helpers[j] = std::thread(helper, sv, j);
    ctx->server = sv;
    return sv;
}

}  // namespace
}  // namespace bg

using namespace bg;

extern "C" {

bg_status bg_submit(bg_ctx_t ctx, const bg_request* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket) {
        set_error("NULL argument");
        return BG_ERR_INVALID_ARG;
    }
    const bg_request& r = *req;
    const char* bad = nullptr;
    if (r.n < 0 || r.n >= ((int64_t)1 << 31) - 1) bad = "n out of range";
    else if (r.n > 0 && (!r.x_cm || !r.y_cm || !r.z_m)) bad = "NULL input pointer";
    else if (r.cell_cm <= 0 || r.cell_cm % 2 || r.nx <= 0 || r.ny <= 0) bad = "bad grid";
    else if ((int64_t)r.nx * r.ny > ((int64_t)1 << 36)) bad = "grid too large";
    else if (!r.depth_out) bad = "depth_out is NULL";
    else if (r.method != 0 && r.method != 1) bad = "method must be 0 (IDW) or 1 (kriging)";
    else if (r.k < 1 || r.k > 32) bad = "k must be in [1, 32]";
    else if (r.method == 0 && !(r.power > 0.0f && std::isfinite(r.power))) bad = "power must be > 0";
    else if (r.method == 1) {
        const bg_variogram& v = r.variogram;
        if (v.model != 0 && v.model != 1) bad = "unknown variogram model";
        else if (!(v.nugget_m2 >= 0.0f) || !(v.sill_m2 > v.nugget_m2) || !(v.range_m > 0.0f))
            bad = "bad variogram";
    }
    {
        const int64_t lim = (int64_t)1 << 30;
        const int64_t xa = (int64_t)r.x0_cm + r.cell_cm / 2;
        const int64_t xb = (int64_t)r.x0_cm + (int64_t)(r.nx - 1) * r.cell_cm + r.cell_cm / 2;
        const int64_t ya = (int64_t)r.y0_cm + r.cell_cm / 2;
        const int64_t yb = (int64_t)r.y0_cm + (int64_t)(r.ny - 1) * r.cell_cm + r.cell_cm / 2;
        if (!bad && !(xa > -lim && xb < lim && ya > -lim && yb < lim))
            bad = "grid node coordinates must lie in (-2^30, 2^30) cm";
    }
    if (bad) {
        set_error(bad);
        return BG_ERR_INVALID_ARG;
    }
    Server* sv = get_server(ctx);
    Ticket* t = new (std::nothrow) Ticket();
    if (!t) return BG_ERR_INTERNAL;
    Slot* inline_slot = nullptr;
    t->req = r;
    t->nodes = (int64_t)r.nx * r.ny;
    t->reserve = request_bytes(r);
    if (ctx->budget && t->reserve > ctx->budget) {
        delete t;
        set_error("the request alone needs more device memory than the context's budget");
        return BG_ERR_OOM_BUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete t;
            set_error("context is shutting down");
            return BG_ERR_CANCELLED;
        }
        t->id = sv->next_id++;
        t->t_submit = sv->now_us();
        sv->tickets[t->id] = t;
        // nothing queued ahead and a slot free: issue it on this thread (no
        // hand-off to the dispatcher), else queue it in arrival order
        if (sv->queue.empty()) inline_slot = admit(sv, t);
        if (!inline_slot) sv->queue.push_back(t);
        *ticket = t->id;
    }
    if (inline_slot) {
        int prev = 0;
        cudaGetDevice(&prev);
        if (prev != ctx->device) cudaSetDevice(ctx->device);
        issue(sv, inline_slot, t);
        if (prev != ctx->device) cudaSetDevice(prev);
    } else {
        sv->cv_work.notify_all();
    }
    return BG_OK;
}

static bg_status take_result(Server* sv, uint64_t ticket, bg_result* out, bool erase) {
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) {
        set_error("unknown ticket");
        return BG_ERR_NOT_FOUND;
    }
    Ticket* t = it->second;
    if (!t->done) return BG_PENDING;
    if (out) {
        out->status = t->status;
        out->nodes = t->nodes;
        out->t_submit_us = t->t_submit;
        out->t_start_us = t->t_start;
        out->t_done_us = t->t_done;
    }
    if (erase) {
        sv->tickets.erase(it);
        delete t;
    }
    return BG_OK;
}

bg_status bg_poll(bg_ctx_t ctx, uint64_t ticket, bg_result* out) {
    if (!ctx) {
        set_error("NULL argument");
        return BG_ERR_INVALID_ARG;
    }
    Server* sv = get_server(ctx);
    std::lock_guard<std::mutex> lk(sv->mu);
    return take_result(sv, ticket, out, true);
}

bg_status bg_wait(bg_ctx_t ctx, uint64_t ticket, int timeout_ms, bg_result* out) {
    if (!ctx) {
        set_error("NULL argument");
        return BG_ERR_INVALID_ARG;
    }
    Server* sv = get_server(ctx);
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        const bg_status rc = take_result(sv, ticket, out, true);
        if (rc != BG_PENDING) return rc;
        if (timeout_ms >= 0 && sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            const bg_status r2 = take_result(sv, ticket, out, true);
            if (r2 != BG_PENDING) return r2;
            set_error("bg_wait timed out");
            return BG_ERR_TIMEOUT;
        }
        if (timeout_ms < 0) sv->cv_done.wait(lk);
    }
}

bg_status bg_cancel(bg_ctx_t ctx, uint64_t ticket) {
    if (!ctx) {
        set_error("NULL argument");
        return BG_ERR_INVALID_ARG;
    }
    Server* sv = get_server(ctx);
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) {
        set_error("unknown ticket");
        return BG_ERR_NOT_FOUND;
    }
    Ticket* t = it->second;
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q) {
        if (*q == t) {
            sv->queue.erase(q);
            t->status = BG_ERR_CANCELLED;
            t->t_done = sv->now_us();
            t->done = true;
            sv->cv_done.notify_all();
            return BG_OK;
        }
    }
    set_error(t->done ? "ticket already finished" : "ticket already running");
    return BG_ERR_INVALID_ARG;
}

bg_status bg_serve_stats(bg_ctx_t ctx, int64_t* queued, int64_t* running, int64_t* reserved_bytes) {
    if (!ctx) {
        set_error("NULL argument");
        return BG_ERR_INVALID_ARG;
    }
    Server* sv = get_server(ctx);
    std::lock_guard<std::mutex> lk(sv->mu);
    int64_t run = 0;
    for (auto& s : sv->slots) run += s.busy ? 1 : 0;
    if (queued) *queued = (int64_t)sv->queue.size();
    if (running) *running = run;
    if (reserved_bytes) *reserved_bytes = (int64_t)sv->reserved;
    return BG_OK;
}

bg_status bg_serve_shutdown(bg_ctx_t ctx) {
    Server* sv = ctx ? ctx->server : nullptr;
    if (!sv) return BG_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Ticket* t : sv->queue) {
            t->status = BG_ERR_CANCELLED;
            t->done = true;
        }
        sv->queue.clear();
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    {
        // the completion thread drains what is still running, then ends
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop_completer = true;
    }
    sv->cv_flight.notify_all();
    if (sv->completer.joinable()) sv->completer.join();
    {
        std::lock_guard<std::mutex> hl(sv->hmu);
        sv->helpers_spin.store(false);
        sv->helpers_stop.store(true);
    }
    sv->cv_helpers.notify_all();
    for (auto& h : sv->helpers)
        if (h.joinable()) h.join();
    for (auto& s : sv->slots) {
        if (s.stream) {
            cudaStreamSynchronize(s.stream);
            cudaStreamDestroy(s.stream);
        }
        if (s.done) cudaEventDestroy(s.done);
        if (s.pin_in) cudaFreeHost(s.pin_in);
        if (s.pin_out) cudaFreeHost(s.pin_out);
    }
    for (auto& kv : sv->tickets) delete kv.second;
    delete sv;
    ctx->server = nullptr;
    return BG_OK;
}

}  // extern "C"
