// The solve server (bae_server_*): continuous admission of BAE solves of
// mixed N, kappa, geometry and layer into concurrent slots.
//
// Each slot is a context with its own CUDA stream and work space, driven by
// one host worker thread, so the device work of different requests
// overlaps. A queued request is admitted as soon as a slot is free and its
// device-memory estimate fits next to the requests in flight. All slots
// share one LGF spectrum cache. A request's arithmetic is exactly that of
// bae_solve on a fresh context: the kernels and reductions do not depend on
// the other slots.
//
// Priority classes: with two or more slots, the first half of the slots run
// on streams of the device's highest priority and prefer small requests
// (N <= 64), the others on the lowest priority and prefer large ones; a slot
// with no request of its class queued takes the first one that fits, so no
// slot idles while work waits. Small solves are latency-bound (a few
// hundred short launches), large ones fill the GPU for tens of
// milliseconds; with the same priority the small ones wait behind the large
// ones' kernels (an N = 32 solve of ~1 ms alone took ~9 ms in the mix).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

struct Req {
    int64_t id = 0;
    bae_request rq{};
    int status = BAE_PENDING;
    bae_result res{};
    std::vector<double> density;
    int64_t footprint = 0;
};

// Device-memory estimate of one solve at grid size N (float64-sized
// convolution buffers A and B, volume buffers, Krylov basis for a boundary
// of at most 6 N^2 nodes).
int64_t footprint(int N, int restart) {
    const int64_t n = N, n1 = N + 1;
    const int64_t conv = 16 * n * n * n1 * 3;            // A + B (B is twice A)
    const int64_t vol = 8 * n * n * n * 4 + 4 * n * n * n;  // v64, u_p, staging x2, v32
    const int64_t ngm = 6 * n * n;
    const int64_t kry = 8 * ngm * (int64_t)(restart + 8);
    return conv + vol + kry + ((int64_t)64 << 20);
}

}  // namespace

struct bae_server {
    int device = 0;
    int64_t budget = 0;
    int64_t in_use = 0;
    std::vector<bae_ctx*> slots;
    std::vector<cudaStream_t> streams;   // one per slot, owned by the server
    std::vector<int> small_class;        // per slot: 1 = high priority, prefers N <= 64
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // runs one request on a slot; the caller publishes the code under the lock
    int run(Req* r, bae_ctx* ctx) {
        const bae_request& q = r->rq;
        bae_problem* P = nullptr;
        int rc = bae_problem_create(ctx, q.N, q.h, q.origin, q.phi, q.kappa2, q.layer, &P);
        if (rc != BAE_OK) return rc;
        int64_t n_gm = 0;
        bae_problem_sizes(P, &n_gm, nullptr, nullptr);
        std::vector<double> xyz((size_t)n_gm * 3), g((size_t)n_gm);
        rc = bae_boundary_points(P, xyz.data());
        if (rc == BAE_OK) {
            if (q.boundary) q.boundary(xyz.data(), n_gm, g.data(), q.user);
            int64_t n_unk = 0;
            bae_problem_unknowns(P, &n_unk);
            r->density.assign((size_t)n_unk, 0.0);
            rc = bae_solve(P, q.f, g.data(), &q.opts, r->density.data(), q.u_out, &r->res.stats);
        }
        r->res.n_gm = (int64_t)r->density.size();   // the density's length
        bae_problem_destroy(P);
        return rc;
    }

    void worker(int slot) {
        cudaSetDevice(device);
        for (;;) {
            Req* r = nullptr;
            {
                std::unique_lock<std::mutex> lock(mu);
                for (;;) {
                    if (stop) return;
                    // the first request of this slot's class that fits, else
                    // the first that fits; a request larger than the whole
                    // budget runs alone rather than never
                    auto pick = queue.end();
                    for (int pass = 0; pass < 2 && pick == queue.end(); ++pass)
                        for (auto it = queue.begin(); it != queue.end(); ++it) {
                            const bool fits = in_use + (*it)->footprint <= budget || in_use == 0;
                            const bool mine = ((*it)->rq.N <= 64) == (small_class[slot] != 0);
                            if (fits && (pass == 1 || mine)) {
                                pick = it;
                                break;
                            }
                        }
                    if (pick != queue.end()) {
                        r = *pick;
                        queue.erase(pick);
                    }
                    if (r) break;
                    cv_work.wait(lock);
                }
                in_use += r->footprint;
                r->res.t_admit = now();
            }
            const int rc = run(r, slots[slot]);
            {
                std::lock_guard<std::mutex> lock(mu);
                in_use -= r->footprint;
                r->res.t_done = now();
                r->res.status = rc;
                r->status = rc;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

extern "C" {

int bae_server_create(int device, int slots, int64_t hbm_budget_bytes, bae_server** out) {
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes <= 0) {
        bae::set_last_error("bae_server_create: need out, 1 <= slots <= 64 and a positive budget");
        return BAE_ERR_INVALID_ARG;
    }
    auto s = std::make_unique<bae_server>();
    s->device = device;
    s->budget = hbm_budget_bytes;
    int least = 0, greatest = 0;
    {
        bae::DeviceGuard dg;
        if (cudaSetDevice(device) != cudaSuccess || cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            bae::set_last_error("bae_server_create: no such CUDA device");
            return BAE_ERR_INVALID_ARG;
        }
        for (int i = 0; i < slots; ++i) {
            const int small = (slots >= 2 && i < slots / 2) ? 1 : 0;
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, small ? greatest : least) != cudaSuccess) {
                cudaGetLastError();
                for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
                bae::set_last_error("bae_server_create: stream creation failed");
                return BAE_ERR_CUDA;
            }
            s->streams.push_back(st);
            s->small_class.push_back(small);
        }
    }
    for (int i = 0; i < slots; ++i) {
        bae_ctx* c = nullptr;
        const int rc = bae_ctx_create(device, s->streams[i], &c);
        if (rc != BAE_OK) {
            for (bae_ctx* x : s->slots) bae_ctx_destroy(x);
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            return rc;
        }
        if (!s->slots.empty()) bae::ctx_share_cache(c, s->slots.front());
        bae::ctx_set_shared_gpu(c);
        s->slots.push_back(c);
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back([srv = s.get(), i]() { srv->worker(i); });
    *out = s.release();
    return BAE_OK;
}

int bae_server_submit(bae_server* srv, const bae_request* req, int64_t* ticket) {
    if (!srv || !req || !ticket || !req->phi || !req->f) {
        bae::set_last_error("bae_server_submit: null argument");
        return BAE_ERR_INVALID_ARG;
    }
    auto r = std::make_unique<Req>();
    r->rq = *req;
    r->footprint = footprint(req->N, req->opts.restart > 0 ? req->opts.restart : 200);
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        r->id = srv->next_id++;
        r->res.t_submit = srv->now();
        r->res.status = BAE_PENDING;
        *ticket = r->id;
        srv->queue.push_back(r.get());
        srv->reqs[r->id] = std::move(r);
    }
    srv->cv_work.notify_all();
    return BAE_OK;
}

int bae_server_poll(bae_server* srv, int64_t ticket, int timeout_ms, bae_result* out) {
    if (!srv) return BAE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) {
        bae::set_last_error("bae_server_poll: unknown ticket");
        return BAE_ERR_INVALID_ARG;
    }
    Req* r = it->second.get();
    auto done = [&]() { return r->status != BAE_PENDING; };
    if (!done()) {
        if (timeout_ms < 0) srv->cv_done.wait(lock, done);
        else if (timeout_ms > 0) srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done);
    }
    if (!done()) return BAE_PENDING;
    if (out) *out = r->res;
    return BAE_OK;
}

int bae_server_density(bae_server* srv, int64_t ticket, double* out, int64_t capacity) {
    if (!srv || !out) return BAE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end() || it->second->status == BAE_PENDING) {
        bae::set_last_error("bae_server_density: unknown or unfinished ticket");
        return BAE_ERR_INVALID_ARG;
    }
    const auto& d = it->second->density;
    if ((int64_t)d.size() > capacity) {
        bae::set_last_error("bae_server_density: capacity too small");
        return BAE_ERR_INVALID_ARG;
    }
    if (cudaMemcpy(out, d.data(), d.size() * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
        bae::set_last_error("bae_server_density: copy failed");
        return BAE_ERR_CUDA;
    }
    return BAE_OK;
}

int bae_server_release(bae_server* srv, int64_t ticket) {
    if (!srv) return BAE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end() || it->second->status == BAE_PENDING) {
        bae::set_last_error("bae_server_release: unknown or unfinished ticket");
        return BAE_ERR_INVALID_ARG;
    }
    srv->reqs.erase(it);
    return BAE_OK;
}

double bae_server_clock(bae_server* srv) { return srv ? srv->now() : 0.0; }

void bae_server_destroy(bae_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    for (bae_ctx* c : srv->slots) bae_ctx_destroy(c);
    {
        bae::DeviceGuard dg;
        cudaSetDevice(srv->device);
        for (cudaStream_t x : srv->streams) cudaStreamDestroy(x);
    }
    delete srv;
}

}  // extern "C"
