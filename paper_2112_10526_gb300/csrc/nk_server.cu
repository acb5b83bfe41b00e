// nk_server_*: a persistent request loop for VMC expectation values and SR
// steps on one GPU (declared in include/nk.h).
//
// Requests arrive from any host thread (nk_server_submit) and wait in a FIFO.
// A scheduler thread admits the head request as soon as a worker slot is free
// and the HBM budget has room for the request's device state plus the growth
// of the slot's context workspace (estimated by a plan-only pass of the same
// entry points).  Each slot is one host thread with its own nk_ctx and
// non-blocking stream; admitted requests therefore run concurrently and their
// kernels overlap on the device, while new requests keep being admitted as
// slots and memory free up.  A request's parameters, edges, chains, samples
// and solver workspace stay on the device until it completes; its results
// (statistics, updated parameters) are copied back and the device state is
// released.  Results depend only on the request (its own Philox stream and
// fixed-order reductions), not on what runs beside it.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/nk.h"
#include "nk_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    uint64_t id = 0;
    nk_request r{};
    std::vector<double> params;
    std::vector<int32_t> edges;
    double *params_out = nullptr;
    size_t state_bytes = 0, ws_bytes = 0;
    size_t reserved = 0;
    Clock::time_point t_submit, t_admit, t_done;
    nk_result res{};
    bool done = false;
};

struct Slot {
    nk_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    std::thread th;
    Req *job = nullptr;
    size_t ws_reserved = 0;  // high-water mark of the context workspace
};

int64_t n_params(int N, int M) { return (int64_t)N + M + (int64_t)M * N; }

size_t state_bytes_of(const nk_request &r) {
    const int64_t Np = n_params(r.N, r.M), Ns = (int64_t)r.n_chains * r.cfg.n_samples;
    return (size_t)Np * 8 + (size_t)r.n_edges * 8 + (size_t)r.n_chains * r.N + (size_t)r.n_chains * 8 +
           (size_t)Ns * r.N + (size_t)Ns * 8 + 256 + 8 * 256;
}

}  // namespace

struct nk_server {
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_work;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::vector<Slot> slots;
    std::thread sched;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t submitted = 0, completed = 0, failed = 0;
    std::vector<double> latencies;
    nk_ctx *planner = nullptr;
};

namespace {

// Workspace one request needs in a context, by a plan-only pass (no device work).
nk_status plan_ws(nk_ctx *planner, const nk_request &r, size_t *out) {
    planner->plan_bytes = 0;
    nk::set_plan_only(true);
    double *fake_d = reinterpret_cast<double *>(256);
    nk_rbm rbm{r.N, r.M, fake_d};
    nk_ham ham{r.ham_kind, r.J, r.h, r.marshall, r.n_edges, reinterpret_cast<const int32_t *>(256), r.J2,
               r.n_edges2};
    nk_status st;
    if (r.kind == NK_REQ_SR_STEP) {
        nk_chains ch{r.n_chains, reinterpret_cast<int8_t *>(256), 0, nullptr};
        st = nk_sr_step(planner, &rbm, &ham, &ch, &r.cfg, nullptr, nullptr, nullptr, nullptr);
    } else {
        const int64_t Ns = (int64_t)r.n_chains * r.cfg.n_samples;
        st = nk_metropolis_sweep(planner, &rbm, r.cfg.precision, nk::effective_rule(r.cfg.rule, r.ham_kind), r.n_edges,
                                 reinterpret_cast<const int32_t *>(256), r.n_chains, reinterpret_cast<int8_t *>(256),
                                 0, r.cfg.n_discard, r.cfg.n_samples, r.cfg.seed, r.cfg.stream_id,
                                 reinterpret_cast<int8_t *>(256), nullptr, nullptr, nullptr, nullptr);
        if (st == NK_OK)
            st = nk_local_energy(planner, &rbm, r.cfg.precision, &ham, reinterpret_cast<const int8_t *>(256), Ns,
                                 fake_d, nullptr, nullptr);
    }
    nk::set_plan_only(false);
    *out = planner->plan_bytes;
    return st;
}

// Runs one admitted request on its slot (blocking on the slot's stream).
void run_request(nk_server *srv, Slot &slot, Req &q) {
    const nk_request &r = q.r;
    cudaStream_t st = slot.st;
    const int N = r.N, M = r.M, C = r.n_chains;
    const int64_t Np = n_params(N, M), Ns = (int64_t)C * r.cfg.n_samples;
    nk_result &res = q.res;
    res.status = NK_OK;
    double *d_params = nullptr, *d_stats = nullptr, *d_eloc = nullptr;
    int32_t *d_edges = nullptr;
    int8_t *d_s = nullptr, *d_samples = nullptr;
    uint64_t *d_acc = nullptr;
    res.message[0] = '\0';
    // code from an entry point (message from nk_last_error) or from a
    // runtime call here (message given)
    auto fail = [&](nk_status code, const char *what = nullptr) {
        if (res.status == NK_OK) {
            res.status = code;
            std::snprintf(res.message, sizeof res.message, "%s", what ? what : nk_last_error());
        }
    };
    auto alloc = [&](void **p, size_t bytes) {
        if (res.status != NK_OK) return;
        if (cudaMallocAsync(p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            fail(NK_ERR_OOM, "cudaMallocAsync of the request state failed");
        }
    };
    alloc((void **)&d_params, (size_t)Np * 8);
    alloc((void **)&d_edges, (size_t)r.n_edges * 8);
    alloc((void **)&d_s, (size_t)C * N);
    alloc((void **)&d_acc, (size_t)C * 8);
    alloc((void **)&d_stats, 16 * 8);
    alloc((void **)&d_samples, (size_t)Ns * N);
    alloc((void **)&d_eloc, (size_t)Ns * 8);
    if (res.status == NK_OK) {
        if (cudaMemcpyAsync(d_params, q.params.data(), (size_t)Np * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_edges, q.edges.data(), (size_t)r.n_edges * 8, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemsetAsync(d_acc, 0, (size_t)C * 8, st) != cudaSuccess)
            fail(NK_ERR_CUDA, "upload of the request state failed");
    }
    nk_rbm rbm{N, M, d_params};
    nk_ham ham{r.ham_kind, r.J, r.h, r.marshall, r.n_edges, d_edges, r.J2, r.n_edges2};
    if (res.status == NK_OK) {
        nk_status s0 = nk_chains_init(slot.ctx, N, C, nk::effective_rule(r.cfg.rule, r.ham_kind), r.cfg.seed,
                                      r.cfg.stream_id, d_s, st);
        if (s0 != NK_OK) fail(s0);
    }
    double host_stats[16] = {0};
    if (res.status == NK_OK && r.kind == NK_REQ_SR_STEP) {
        nk_chains ch{C, d_s, 0, d_acc};
        nk_status s1 = nk_sr_step(slot.ctx, &rbm, &ham, &ch, &r.cfg, reinterpret_cast<nk_sr_stats *>(d_stats),
                                  d_samples, d_eloc, st);
        if (s1 != NK_OK && s1 != NK_ERR_NOT_CONVERGED) fail(s1);
    } else if (res.status == NK_OK) {
        nk_status s1 = nk_metropolis_sweep(slot.ctx, &rbm, r.cfg.precision, nk::effective_rule(r.cfg.rule, r.ham_kind),
                                           r.n_edges, d_edges, C, d_s,
                                           0, r.cfg.n_discard, r.cfg.n_samples, r.cfg.seed, r.cfg.stream_id,
                                           d_samples, nullptr, d_acc, nullptr, st);
        if (s1 == NK_OK) s1 = nk_local_energy(slot.ctx, &rbm, r.cfg.precision, &ham, d_samples, Ns, d_eloc, nullptr, st);
        if (s1 == NK_OK) s1 = nk_stats(slot.ctx, d_eloc, Ns, C, d_stats, st);
        if (s1 != NK_OK) fail(s1);
    }
    if (res.status == NK_OK) {
        const size_t nstat = r.kind == NK_REQ_SR_STEP ? sizeof(nk_sr_stats) : 3 * sizeof(double);
        if (cudaMemcpyAsync(host_stats, d_stats, nstat, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            fail(NK_ERR_CUDA, "download of the statistics failed");
        if (q.params_out &&
            cudaMemcpyAsync(q.params_out, d_params, (size_t)Np * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            fail(NK_ERR_CUDA, "download of the parameters failed");
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        fail(NK_ERR_CUDA, "the request's stream reported an error");
    }
    if (res.status == NK_OK) {
        if (r.kind == NK_REQ_SR_STEP) {
            nk_sr_stats ss;
            std::memcpy(&ss, host_stats, sizeof ss);
            res.energy = ss.energy;
            res.variance = ss.variance;
            res.error = ss.error;
            res.acceptance = ss.acceptance;
            res.cg_iters = ss.cg_iters;
            res.solver_status = ss.solver_status;
        } else {
            res.energy = host_stats[0];
            res.variance = host_stats[1];
            res.error = host_stats[2];
        }
    }
    void *frees[] = {d_params, d_edges, d_s, d_acc, d_stats, d_samples, d_eloc};
    for (void *p : frees)
        if (p) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    cudaGetLastError();
    (void)srv;
}

void worker_loop(nk_server *srv, int k) {
    cudaSetDevice(srv->device);
    Slot &slot = srv->slots[k];
    for (;;) {
        Req *q = nullptr;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || slot.job; });
            if (!slot.job) return;
            q = slot.job;
        }
        run_request(srv, slot, *q);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            q->t_done = Clock::now();
            q->res.queue_ms = ms_between(q->t_submit, q->t_admit);
            q->res.run_ms = ms_between(q->t_admit, q->t_done);
            q->res.latency_ms = ms_between(q->t_submit, q->t_done);
            q->res.slot = k;
            q->res.device_bytes = q->reserved;
            q->done = true;
            srv->used -= q->state_bytes;
            if (slot.ctx->ws_size > slot.ws_reserved) {
                srv->used += slot.ctx->ws_size - slot.ws_reserved;
                slot.ws_reserved = slot.ctx->ws_size;
            }
            ++srv->completed;
            if (q->res.status != NK_OK) ++srv->failed;
            srv->latencies.push_back(q->res.latency_ms);
            slot.job = nullptr;
        }
        srv->cv_done.notify_all();
        srv->cv_sched.notify_all();
    }
}

void scheduler_loop(nk_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        srv->cv_sched.wait(lk, [&] {
            if (srv->stop) return true;
            if (srv->queue.empty()) return false;
            for (auto &s : srv->slots)
                if (!s.job) return true;
            return false;
        });
        if (srv->stop) return;
        Req *q = srv->queue.front();
        // the free slot whose workspace already covers most of the request
        int best = -1;
        size_t best_extra = SIZE_MAX;
        for (size_t k = 0; k < srv->slots.size(); ++k) {
            if (srv->slots[k].job) continue;
            const size_t have = srv->slots[k].ws_reserved;
            // a context workspace grows to bytes + bytes/8 + 1 MiB (ensure_ws)
            const size_t alloc = q->ws_bytes + q->ws_bytes / 8 + (1u << 20);
            const size_t extra = q->ws_bytes > have ? alloc - have : 0;
            if (extra < best_extra) {
                best_extra = extra;
                best = (int)k;
            }
        }
        size_t need = q->state_bytes + best_extra;
        int inflight = 0;
        for (auto &s : srv->slots) inflight += s.job ? 1 : 0;
        if (srv->used + need > srv->budget) {
            // release the workspaces of idle slots (largest first) before
            // making the request wait or fail
            for (;;) {
                int victim = -1;
                for (size_t k = 0; k < srv->slots.size(); ++k) {
                    const Slot &sl = srv->slots[k];
                    if (sl.job || (int)k == best || sl.ws_reserved == 0) continue;
                    if (victim < 0 || sl.ws_reserved > srv->slots[victim].ws_reserved) victim = (int)k;
                }
                if (victim < 0 || srv->used + need <= srv->budget) break;
                Slot &sl = srv->slots[victim];
                if (sl.ctx->ws) cudaFree(sl.ctx->ws);
                sl.ctx->ws = nullptr;
                sl.ctx->ws_size = 0;
                srv->used -= sl.ws_reserved;
                sl.ws_reserved = 0;
            }
            if (srv->used + need > srv->budget && srv->slots[best].ws_reserved > 0) {
                // the chosen slot's own workspace is also reclaimable
                Slot &sl = srv->slots[best];
                if (sl.ctx->ws) cudaFree(sl.ctx->ws);
                sl.ctx->ws = nullptr;
                sl.ctx->ws_size = 0;
                srv->used -= sl.ws_reserved;
                sl.ws_reserved = 0;
                best_extra = q->ws_bytes + q->ws_bytes / 8 + (1u << 20);
                need = q->state_bytes + best_extra;
            }
        }
        if (srv->used + need > srv->budget && inflight == 0) {
            // does not fit even with nothing in flight: fail it instead of
            // blocking the queue
            srv->queue.pop_front();
            q->res.status = NK_ERR_OOM;
            std::snprintf(q->res.message, sizeof q->res.message,
                          "needs %zu bytes, the HBM budget is %zu", need, srv->budget);
            q->t_admit = q->t_done = Clock::now();
            q->res.latency_ms = ms_between(q->t_submit, q->t_done);
            q->done = true;
            ++srv->completed;
            ++srv->failed;
            srv->cv_done.notify_all();
            continue;
        }
        if (srv->used + need > srv->budget) {
            // wait for a request to complete and return its memory
            const int64_t done_before = srv->completed;
            srv->cv_sched.wait(lk, [&] { return srv->stop || srv->completed != done_before; });
            continue;
        }
        srv->queue.pop_front();
        Slot &slot = srv->slots[best];
        srv->used += need;
        slot.ws_reserved += best_extra;
        q->reserved = need;
        q->t_admit = Clock::now();
        slot.job = q;
        srv->cv_work.notify_all();
    }
}

double quantile(std::vector<double> v, double qn) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t idx = (size_t)std::ceil(qn * (double)v.size());
    if (idx > 0) --idx;
    if (idx >= v.size()) idx = v.size() - 1;
    return v[idx];
}

}  // namespace

extern "C" {

nk_status nk_server_create(int32_t device, size_t hbm_budget, int32_t slots, nk_server **out) {
    if (!out || slots < 1 || slots > 256 || hbm_budget == 0) return nk::report_error(NK_ERR_INVALID_ARG, "bad server arguments");
    *out = nullptr;
    auto *srv = new nk_server();
    srv->device = device;
    srv->budget = hbm_budget;
    nk_status st = nk_ctx_create(device, &srv->planner);
    if (st != NK_OK) {
        delete srv;
        return st;
    }
    srv->slots.resize(slots);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    for (int k = 0; k < slots; ++k) {
        st = nk_ctx_create(device, &srv->slots[k].ctx);
        if (st == NK_OK && cudaStreamCreateWithFlags(&srv->slots[k].st, cudaStreamNonBlocking) != cudaSuccess)
            st = nk::report_error(NK_ERR_CUDA, "stream creation failed");
        if (st != NK_OK) break;
    }
    cudaSetDevice(prev);
    if (st != NK_OK) {
        for (auto &s : srv->slots) {
            if (s.ctx) nk_ctx_destroy(s.ctx);
            if (s.st) cudaStreamDestroy(s.st);
        }
        nk_ctx_destroy(srv->planner);
        delete srv;
        return st;
    }
    for (int k = 0; k < slots; ++k) srv->slots[k].th = std::thread(worker_loop, srv, k);
    srv->sched = std::thread(scheduler_loop, srv);
    *out = srv;
    return NK_OK;
}

size_t nk_request_bytes(const nk_request *req) {
    if (!req) return 0;
    // plan-only calls touch no device resource, so a bare context suffices
    nk_ctx planner{};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        planner.device = dev;
    else
        cudaGetLastError();
    size_t ws = 0;
    if (plan_ws(&planner, *req, &ws) != NK_OK) return 0;
    return ws + ws / 8 + (1u << 20) + state_bytes_of(*req);
}

nk_status nk_server_submit(nk_server *srv, const nk_request *req, double *params_out, uint64_t *id) {
    if (!srv || !req || !id) return nk::report_error(NK_ERR_INVALID_ARG, "NULL argument");
    const nk_request &r = *req;
    if (r.kind != NK_REQ_SR_STEP && r.kind != NK_REQ_EXPECT) return nk::report_error(NK_ERR_INVALID_ARG, "request kind");
    if (r.N < 1 || r.N > 4096 || r.M < 1 || r.M > 8192 || r.n_chains < 1 || r.cfg.n_samples < 1 || !r.params ||
        r.n_edges < 1 || !r.edges || r.n_edges2 < 0 || r.n_edges2 > r.n_edges)
        return nk::report_error(NK_ERR_INVALID_ARG, "request sizes or pointers");
    auto q = std::make_unique<Req>();
    q->r = r;
    const int64_t Np = n_params(r.N, r.M);
    q->params.assign(r.params, r.params + Np);
    q->edges.assign(r.edges, r.edges + 2 * (size_t)r.n_edges);
    for (int32_t e : q->edges)
        if (e < 0 || e >= r.N) return nk::report_error(NK_ERR_INVALID_ARG, "edge index outside [0, N)");
    q->r.params = nullptr;
    q->r.edges = nullptr;
    q->params_out = params_out;
    size_t ws = 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        nk_status st = plan_ws(srv->planner, r, &ws);
        if (st != NK_OK) return st;
    }
    q->ws_bytes = ws;
    q->state_bytes = state_bytes_of(r);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        q->id = srv->next_id++;
        *id = q->id;
        srv->queue.push_back(q.get());
        srv->reqs.emplace(q->id, std::move(q));
        ++srv->submitted;
    }
    srv->cv_sched.notify_all();
    return NK_OK;
}

nk_status nk_server_poll(nk_server *srv, uint64_t id, int32_t *done, nk_result *out) {
    if (!srv || !done) return nk::report_error(NK_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return nk::report_error(NK_ERR_INVALID_ARG, "unknown request id");
    *done = it->second->done ? 1 : 0;
    if (it->second->done && out) *out = it->second->res;
    return NK_OK;
}

nk_status nk_server_wait(nk_server *srv, uint64_t id, nk_result *out) {
    if (!srv) return nk::report_error(NK_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return nk::report_error(NK_ERR_INVALID_ARG, "unknown request id");
    Req *q = it->second.get();
    srv->cv_done.wait(lk, [&] { return q->done; });
    if (out) *out = q->res;
    return NK_OK;
}

nk_status nk_server_stats_get(nk_server *srv, nk_server_stats *out) {
    if (!srv || !out) return nk::report_error(NK_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    int64_t inflight = 0;
    for (auto &s : srv->slots) inflight += s.job ? 1 : 0;
    out->inflight = inflight;
    out->queued = (int64_t)srv->queue.size();
    out->hbm_in_use = srv->used;
    out->hbm_budget = srv->budget;
    out->p50_ms = quantile(srv->latencies, 0.50);
    out->p99_ms = quantile(srv->latencies, 0.99);
    return NK_OK;
}

nk_status nk_server_destroy(nk_server *srv) {
    if (!srv) return NK_OK;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->queue.clear();
        // let in-flight requests finish
        srv->cv_done.wait(lk, [&] {
            for (auto &s : srv->slots)
                if (s.job) return false;
            return true;
        });
        srv->stop = true;
    }
    srv->cv_sched.notify_all();
    srv->cv_work.notify_all();
    if (srv->sched.joinable()) srv->sched.join();
    for (auto &s : srv->slots)
        if (s.th.joinable()) s.th.join();
    for (auto &s : srv->slots) {
        if (s.ctx) nk_ctx_destroy(s.ctx);
        if (s.st) cudaStreamDestroy(s.st);
    }
    nk_ctx_destroy(srv->planner);
    delete srv;
    return NK_OK;
}

}  // extern "C"
