// Serving loop with continuous batching (E2).
//
// A host thread owns a FIFO of requests.  Each pass it
//  1. completes launches whose CUDA event has fired (results are copied from
//     the lane's pinned buffers into the requests, latency recorded);
//  2. admits work into idle lanes: the oldest queued request picks the
//     (catalog, flags) key, and every queued request with the same key is
//     appended, in arrival order, while the batch stays within MAX_BATCH
//     points; the lane's workspace must fit the HBM budget, otherwise the
//     batch waits until running lanes release memory (and fails with
//     CHIMERA_ERR_ADMISSION when nothing is running);
//  3. launches the batch on the lane's own stream (K1..K6, plus the adjoint
//     for gradient requests) and records an event.
// Lanes run concurrently on separate streams, so requests that arrive while
// others are on the GPU start as soon as a lane is free.  Every point of a
// batch is computed independently of the others, so a request's result does
// not depend on what it was batched with.  No kernel waits on a device flag.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "runtime.cuh"

namespace chim {

namespace {

constexpr int MAX_LANES = 4;
constexpr int MAX_BATCH = 512;

using Clock = std::chrono::steady_clock;

enum class RState { Queued, Running, Done, Cancelled, Failed };

struct Request {
    uint64_t ticket;
    int32_t cat;
    int32_t n;
    int32_t flags;
    std::vector<double> theta;
    std::vector<double> lnL, dlnL;
    std::vector<int32_t> status;
    RState state = RState::Queued;
    int err = CHIMERA_OK;
    Clock::time_point t_submit, t_done;
};

struct Lane {
    Workspace ws;
    bool busy = false;
    std::vector<std::shared_ptr<Request>> batch;
    int H = 0;
    bool grad = false;
    cudaEvent_t done = nullptr;
    double *h_lnL = nullptr, *h_grad = nullptr;
    int32_t *h_status = nullptr;
    int hcap = 0;
};

}  // namespace

struct Server {
    Ctx *ctx = nullptr;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    Lane lanes[MAX_LANES];
    // stats
    std::vector<double> lat_ms;
    int64_t batches = 0, points = 0;
    int64_t admitted_peak = 0;

    void loop();
    bool complete_lanes();
    bool admit_and_launch();
    int launch(Lane &L, std::vector<std::shared_ptr<Request>> &b);
};

static int lane_buffers(Lane &L, int H) {
    if (H <= L.hcap) return CHIMERA_OK;
    if (L.h_lnL) cudaFreeHost(L.h_lnL);
    if (L.h_grad) cudaFreeHost(L.h_grad);
    if (L.h_status) cudaFreeHost(L.h_status);
    L.h_lnL = nullptr; L.h_grad = nullptr; L.h_status = nullptr;
    if (cudaMallocHost(&L.h_lnL, sizeof(double) * H) != cudaSuccess ||
        cudaMallocHost(&L.h_grad, sizeof(double) * 12 * H) != cudaSuccess ||
        cudaMallocHost(&L.h_status, sizeof(int32_t) * H) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocHost failed for serve lane buffers");
        return CHIMERA_ERR_CUDA;
    }
    L.hcap = H;
    return CHIMERA_OK;
}

int Server::launch(Lane &L, std::vector<std::shared_ptr<Request>> &b) {
    Ctx &c = *ctx;
    std::lock_guard<std::recursive_mutex> lk(c.mu);
    cudaSetDevice(c.device);
    auto cat = find_catalog(c, b[0]->cat);
    if (!cat) {
        set_error("unknown catalog id");
        return CHIMERA_ERR_NOT_FOUND;
    }
    int H = 0;
    for (auto &r : b) H += r->n;
    std::vector<double> th;
    th.reserve(12 * (size_t)H);
    for (auto &r : b) th.insert(th.end(), r->theta.begin(), r->theta.end());
    const int prec = (b[0]->flags & CHIMERA_SERVE_MIXED) ? CHIMERA_MIXED : CHIMERA_FP64;
    const bool grad = (b[0]->flags & CHIMERA_SERVE_GRAD) != 0;
    int rc = lane_buffers(L, H);
    if (rc) return rc;
    if (!L.ws.st) {
        int prio_lo = 0, prio_hi = 0;
        cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (cudaStreamCreateWithPriority(&L.ws.st, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaStreamCreate failed");
            return CHIMERA_ERR_CUDA;
        }
    }
    if (!L.done && cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return CHIMERA_ERR_CUDA;
    }
    rc = forward(c, *cat, L.ws, H, th.data(), grad ? prec | PREC_WITH_GRAD : prec);
    if (rc) return rc;
    if (grad) {
        rc = backward(c, *cat, L.ws, H, prec);
        if (rc) return rc;
    }
    CallPtrs p = L.ws.ptrs(H, cat->d);
    cudaMemcpyAsync(L.h_lnL, L.ws.lnL, sizeof(double) * H, cudaMemcpyDeviceToHost, L.ws.st);
    cudaMemcpyAsync(L.h_status, p.status, sizeof(int32_t) * H, cudaMemcpyDeviceToHost, L.ws.st);
    if (grad) cudaMemcpyAsync(L.h_grad, L.ws.grad, sizeof(double) * 12 * H, cudaMemcpyDeviceToHost, L.ws.st);
    if (cudaEventRecord(L.done, L.ws.st) != cudaSuccess) return cuda_check(cudaGetLastError(), "event");
    int64_t adm = 0;
    for (auto &l : lanes) adm += (int64_t)l.ws.bytes;
    admitted_peak = std::max(admitted_peak, adm);
    L.H = H;
    L.grad = grad;
    return CHIMERA_OK;
}

bool Server::complete_lanes() {
    bool any = false;
    for (auto &L : lanes) {
        if (!L.busy) continue;
        cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        auto now = Clock::now();
        std::lock_guard<std::mutex> lk(m);
        int off = 0;
        for (auto &r : L.batch) {
            if (q != cudaSuccess) {
                r->state = RState::Failed;
                r->err = CHIMERA_ERR_CUDA;
            } else if (r->state != RState::Cancelled) {
                r->lnL.assign(L.h_lnL + off, L.h_lnL + off + r->n);
                r->status.assign(L.h_status + off, L.h_status + off + r->n);
                if (L.grad) r->dlnL.assign(L.h_grad + 12 * off, L.h_grad + 12 * (off + r->n));
                r->state = RState::Done;
                r->t_done = now;
                lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
            }
            off += r->n;
        }
        points += off;
        batches++;
        L.batch.clear();
        L.busy = false;
        any = true;
        if (q != cudaSuccess) cudaGetLastError();
    }
    if (any) cv_done.notify_all();
    return any;
}

bool Server::admit_and_launch() {
    bool launched = false;
    for (auto &L : lanes) {
        if (L.busy) continue;
        std::vector<std::shared_ptr<Request>> b;
        {
            std::lock_guard<std::mutex> lk(m);
            while (!queue.empty() && queue.front()->state == RState::Cancelled) queue.pop_front();
            if (queue.empty()) break;
            auto head = queue.front();
            int H = 0;
            for (auto it = queue.begin(); it != queue.end();) {
                auto &r = *it;
                if (r->state == RState::Cancelled) { it = queue.erase(it); continue; }
                if (r->cat == head->cat && r->flags == head->flags && H + r->n <= std::max(MAX_BATCH, head->n)) {
                    H += r->n;
                    r->state = RState::Running;
                    b.push_back(r);
                    it = queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (b.empty()) break;
        int rc = launch(L, b);
        if (rc == CHIMERA_ERR_ADMISSION) {
            bool others = false;
            for (auto &l2 : lanes) others |= l2.busy;
            if (others) {  // wait for memory: put the batch back at the front, in order
                std::lock_guard<std::mutex> lk(m);
                for (auto it = b.rbegin(); it != b.rend(); ++it) {
                    (*it)->state = RState::Queued;
                    queue.push_front(*it);
                }
                break;
            }
        }
        if (rc) {
            std::lock_guard<std::mutex> lk(m);
            for (auto &r : b) {
                r->state = RState::Failed;
                r->err = rc;
            }
            cv_done.notify_all();
            continue;
        }
        L.batch = std::move(b);
        L.busy = true;
        launched = true;
    }
    return launched;
}

void Server::loop() {
    while (true) {
        {
            std::unique_lock<std::mutex> lk(m);
            if (stop) break;
        }
        bool a = complete_lanes();
        bool b = admit_and_launch();
        if (!a && !b) {
            std::unique_lock<std::mutex> lk(m);
            bool busy = false;
            for (auto &L : lanes) busy |= L.busy;
            if (stop) break;
            if (busy) cv_work.wait_for(lk, std::chrono::microseconds(50));
            else cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return stop || !queue.empty(); });
        }
    }
}

static Server *get_server(Ctx &ctx) {
    std::lock_guard<std::recursive_mutex> lk(ctx.mu);
    if (!ctx.server) {
        ctx.server = new Server();
        ctx.server->ctx = &ctx;
        Server *s = ctx.server;
        int dev = ctx.device;
        s->th = std::thread([s, dev] {
            cudaSetDevice(dev);
            s->loop();
        });
    }
    return ctx.server;
}

int serve_submit(Ctx &ctx, int32_t cat, int32_t n, const double *theta, int32_t flags, uint64_t *ticket) {
    {
        std::lock_guard<std::recursive_mutex> lk(ctx.mu);
        if (!find_catalog(ctx, cat)) {
            set_error("unknown catalog id");
            return CHIMERA_ERR_NOT_FOUND;
        }
    }
    if (flags & ~(CHIMERA_SERVE_GRAD | CHIMERA_SERVE_MIXED)) {
        set_error("unknown serve flags");
        return CHIMERA_ERR_INVALID_ARG;
    }
    Server *s = get_server(ctx);
    auto r = std::make_shared<Request>();
    r->cat = cat;
    r->n = n;
    r->flags = flags;
    r->theta.assign(theta, theta + 12 * (size_t)n);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->m);
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return CHIMERA_OK;
}

int serve_poll(Ctx &ctx, uint64_t ticket, int64_t timeout_us, double *lnL, double *dlnL, int32_t *status) {
    Server *s = get_server(ctx);
    std::unique_lock<std::mutex> lk(s->m);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("unknown ticket");
        return CHIMERA_ERR_NOT_FOUND;
    }
    auto r = it->second;
    auto finished = [&] {
        return r->state == RState::Done || r->state == RState::Cancelled || r->state == RState::Failed;
    };
    if (!finished()) {
        if (timeout_us == 0) return CHIMERA_ERR_TIMEOUT;
        if (timeout_us < 0) s->cv_done.wait(lk, finished);
        else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished))
            return CHIMERA_ERR_TIMEOUT;
    }
    s->all.erase(ticket);
    if (r->state == RState::Cancelled) return CHIMERA_ERR_CANCELLED;
    if (r->state == RState::Failed) {
        set_error("serve request failed");
        return r->err ? r->err : CHIMERA_ERR_CUDA;
    }
    std::copy(r->lnL.begin(), r->lnL.end(), lnL);
    if (status) std::copy(r->status.begin(), r->status.end(), status);
    if (dlnL && !r->dlnL.empty()) std::copy(r->dlnL.begin(), r->dlnL.end(), dlnL);
    return CHIMERA_OK;
}

int serve_cancel(Ctx &ctx, uint64_t ticket) {
    Server *s = get_server(ctx);
    std::lock_guard<std::mutex> lk(s->m);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("unknown ticket");
        return CHIMERA_ERR_NOT_FOUND;
    }
    auto &r = it->second;
    if (r->state == RState::Queued || r->state == RState::Running) r->state = RState::Cancelled;
    s->cv_done.notify_all();
    return CHIMERA_OK;
}

size_t serve_ws_bytes(Ctx &ctx) {
    if (!ctx.server) return 0;
    size_t b = 0;
    for (auto &L : ctx.server->lanes) b += L.ws.bytes + L.ws.gscr_bytes;
    return b;
}

int serve_stats(Ctx &ctx, chimera_serve_stats_t *out) {
    Server *s = get_server(ctx);
    std::lock_guard<std::mutex> lk(s->m);
    std::vector<double> v = s->lat_ms;
    out->completed = (int64_t)v.size();
    out->batches = s->batches;
    out->points = s->points;
    out->admitted_bytes_peak = s->admitted_peak;
    out->p50_ms = out->p99_ms = out->mean_ms = 0.0;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto q = [&](double f) {
            double pos = f * (v.size() - 1);
            size_t i = (size_t)pos;
            double fr = pos - i;
            return i + 1 < v.size() ? v[i] * (1 - fr) + v[i + 1] * fr : v[i];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        double m = 0;
        for (double x : v) m += x;
        out->mean_ms = m / v.size();
    }
    return CHIMERA_OK;
}

int serve_reset_stats(Ctx &ctx) {
    Server *s = get_server(ctx);
    std::lock_guard<std::mutex> lk(s->m);
    s->lat_ms.clear();
    s->batches = 0;
    s->points = 0;
    s->admitted_peak = 0;
    return CHIMERA_OK;
}

void serve_shutdown(Ctx &ctx) {
    Server *s = ctx.server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(ctx.device);
    for (auto &L : s->lanes) {
        if (L.ws.st) cudaStreamSynchronize(L.ws.st);
        ws_release(ctx, L.ws);
        ws_destroy_streams(L.ws);
        if (L.ws.st) cudaStreamDestroy(L.ws.st);
        if (L.done) cudaEventDestroy(L.done);
        if (L.h_lnL) cudaFreeHost(L.h_lnL);
        if (L.h_grad) cudaFreeHost(L.h_grad);
        if (L.h_status) cudaFreeHost(L.h_status);
    }
    delete s;
    ctx.server = nullptr;
}

}  // namespace chim
