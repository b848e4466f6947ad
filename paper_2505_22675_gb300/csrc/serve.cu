// Serving: continuous batching of gridding requests on one context.
//
// bg_submit queues a request and returns a ticket at once. A dispatcher
// thread admits queued requests in arrival order whenever a stream slot is
// free and the context's HBM budget covers the request's estimated device
// memory; each admitted request runs on its slot's stream (host copy into
// pinned staging + bounding box on the host, async upload and hash build,
// interpolation, async copy of the grids back), so requests that arrive while
// others run overlap with them on the device. A host function queued behind
// the work copies the grids into the caller's buffers and completes the
// ticket; bg_poll never blocks, bg_wait blocks up to a timeout.
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
    bool busy = false;
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
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, Ticket*> tickets;
    std::vector<Slot> slots;
    uint64_t next_id = 1;
    size_t reserved = 0;               // device bytes reserved by running requests
    bool stop = false;
    std::thread worker;
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

void CUDART_CB on_done(void* arg) {
    // runs on a driver thread once the slot's stream reached this point
    Slot* sl = static_cast<Slot*>(arg);
    Server* sv = sl->server;
    Ticket* t = sl->ticket;
    const int64_t m = t->nodes;
    if (t->status == BG_PENDING) {
        std::memcpy(t->req.depth_out, sl->pin_out, (size_t)m * 4);
        if (t->req.var_out) std::memcpy(t->req.var_out, sl->pin_out + m, (size_t)m * 4);
        t->status = BG_OK;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    t->t_done = sv->now_us();
    t->done = true;
    sl->busy = false;
    sl->ticket = nullptr;
    sv->reserved -= t->reserve;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
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

    // copy into pinned staging and take the bounding box on the way
    int32_t* px = (int32_t*)sl->pin_in;
    int32_t* py = px + n;
    float* pz = (float*)(py + n);
    HostBBox bb{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, 0, 0};
    const int32_t lim = 1 << 30;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t xi = r.x_cm[i], yi = r.y_cm[i];
        const float zi = r.z_m[i];
        px[i] = xi;
        py[i] = yi;
        pz[i] = zi;
        if (!std::isnan(zi)) {
            bb.x0 = std::min(bb.x0, xi);
            bb.y0 = std::min(bb.y0, yi);
            bb.x1 = std::max(bb.x1, xi);
            bb.y1 = std::max(bb.y1, yi);
            ++bb.n_valid;
            bb.out_of_range += (xi <= -lim || xi >= lim || yi <= -lim || yi >= lim);
        }
    }
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

void dispatcher(Server* sv) {
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (sv->stop && sv->queue.empty()) break;
        Slot* free_slot = nullptr;
        for (auto& s : sv->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        Ticket* t = nullptr;
        if (free_slot && !sv->queue.empty()) {
            Ticket* head = sv->queue.front();
            const size_t budget = sv->ctx->budget;
            const bool fits = budget == 0 || sv->reserved == 0 || sv->reserved + head->reserve <= budget;
            if (fits) {
                t = head;
                sv->queue.pop_front();
            }
        }
        if (!t) {
            sv->cv_work.wait(lk);
            continue;
        }
        free_slot->busy = true;
        free_slot->ticket = t;
        t->slot = free_slot;
        sv->reserved += t->reserve;
        t->t_start = sv->now_us();
        lk.unlock();

        bg_status rc = launch_request(sv, free_slot, t);
        cudaStream_t st = free_slot->stream;
        if (rc != BG_OK) {
            t->status = rc;  // on_done skips the copy-out
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
        const cudaError_t e = cudaLaunchHostFunc(st, on_done, free_slot);
        if (e != cudaSuccess) {
            t->status = cuda_fail(e, "cudaLaunchHostFunc");
            cudaStreamSynchronize(st);
            on_done(free_slot);
        }
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
        s.server = sv;
    }
    cudaSetDevice(prev);
    sv->worker = std::thread(dispatcher, sv);
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
        sv->queue.push_back(t);
    }
    sv->cv_work.notify_all();
    *ticket = t->id;
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
    for (auto& s : sv->slots) {
        if (s.stream) {
            cudaStreamSynchronize(s.stream);
            cudaStreamDestroy(s.stream);
        }
        if (s.pin_in) cudaFreeHost(s.pin_in);
        if (s.pin_out) cudaFreeHost(s.pin_out);
    }
    for (auto& kv : sv->tickets) delete kv.second;
    delete sv;
    ctx->server = nullptr;
    return BG_OK;
}

}  // extern "C"
