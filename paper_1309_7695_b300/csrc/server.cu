// Serving loop: continuous batching of simulation requests.
//
// Requests (one network + one batch of simulations each) are queued by
// ssa_server_submit.  A dispatcher thread admits queued requests, in arrival
// order, whenever a stream slot is free and the request's HBM footprint fits
// the remaining budget; all requests admitted together form one
// multi-network persistent launch on that slot's stream, so batches on
// different slots overlap on the device.  Each request of a launch is one
// group of the launch and completes on its own: the kernel counts the
// group's finished simulations and its last one raises the request's flag
// in host-mapped memory, which the dispatcher polls, so a short request does
// not wait for the long ones it was batched with.  Results stay resident in
// device memory until ssa_server_fetch copies them out (on a stream of its
// own, not behind later launches on the slot) and frees them, which returns
// their bytes to the budget.  Each simulation's random stream is keyed by
// (request seed, replicate index) and every launch uses the same kernel, so
// a request's result does not depend on what it was batched or overlapped
// with.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

namespace {

thread_local std::string g_srv_error;

int sfail(int code, const std::string &msg)
{
    g_srv_error = msg;
    return code;
}

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
    int64_t ticket = 0;
    ssa_model_t model = nullptr;
    int32_t N = 0, M = 0;
    int64_t n_sims = 0;
    std::vector<double> params, T;
    std::vector<int32_t> x0;
    double t_end = 0.0;
    uint64_t seed = 0;
    size_t bytes = 0;  // device footprint
    int state = SSA_JOB_RUNNING;
    double t_submit = 0, t_admit = -1, t_done = -1;
    int32_t batch_size = 0;
    int slot = -1;
    int flag = -1;   // index of its completion flag / counter while its launch runs
    // device buffers (valid from admission until fetch)
    double *d_params = nullptr, *d_T = nullptr;
    int32_t *d_x0 = nullptr, *d_samples = nullptr;
    ssa_sim_stats *d_stats = nullptr;
    std::string error;
};

struct Batch {
    int slot = -1;
    std::vector<std::shared_ptr<Request>> reqs;
    std::atomic<bool> done{false};
};

}  // namespace

struct ssa_server {
    ssa_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<int64_t, std::shared_ptr<Request>> all;
    std::vector<std::shared_ptr<Batch>> inflight;
    int64_t next_ticket = 1;
    size_t budget = 0, used = 0;
    bool shutdown = false;
    std::thread worker;
    int64_t launches = 0;
    // completion signals, max_batch per slot: flags in host-mapped memory
    // (h_flags, seen by the device as d_flags), counters in device memory
    int32_t *h_flags = nullptr;
    int32_t *d_flags = nullptr;
    unsigned long long *d_counts = nullptr;

    void run();
};

static void CUDART_CB batch_done_cb(void *p)
{
    // host callback: no CUDA calls here, only flag the batch and wake the dispatcher
    auto *pair = static_cast<std::pair<ssa_server *, Batch *> *>(p);
    {
        std::lock_guard<std::mutex> lock(pair->first->mu);
        pair->second->done = true;
    }
    pair->first->cv.notify_all();
    delete pair;
}

void ssa_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        cv.wait_for(lock, inflight.empty() ? std::chrono::milliseconds(5) : std::chrono::milliseconds(1));
        bool woke = false;
        // per-request completions: flags raised by the kernel for finished groups
        for (auto &bp : inflight)
            for (auto &r : bp->reqs)
                if (r->t_done < 0 && r->flag >= 0 && reinterpret_cast<volatile int32_t *>(h_flags)[r->flag] != 0) {
                    r->t_done = now_s(t0);
                    r->state = SSA_JOB_DONE;
                    woke = true;
                }
        // whole launches: free the slot; requests without a raised flag (no
        // simulations, or a failed launch) complete here
        for (size_t k = 0; k < inflight.size();) {
            Batch &b = *inflight[k];
            if (!b.done) {
                ++k;
                continue;
            }
            cudaError_t e = cudaStreamQuery(streams[(size_t)b.slot]);
            const double t = now_s(t0);
            for (auto &r : b.reqs) {
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    r->state = SSA_JOB_FAILED;
                    r->error = cudaGetErrorString(e);
                    if (r->t_done < 0) r->t_done = t;
                } else if (r->t_done < 0) {
                    r->state = SSA_JOB_DONE;
                    r->t_done = t;
                }
                r->flag = -1;
            }
            slot_busy[(size_t)b.slot] = false;
            inflight.erase(inflight.begin() + (long)k);
            woke = true;
        }
        if (woke) cv.notify_all();
        if (shutdown && pending.empty() && inflight.empty()) break;
        // admission: FIFO, as many queued requests as fit one free slot and the budget
        int slot = -1;
        for (size_t s = 0; s < slot_busy.size(); ++s)
            if (!slot_busy[s]) {
                slot = (int)s;
                break;
            }
        if (slot < 0 || pending.empty()) continue;
        std::vector<std::shared_ptr<Request>> take;
        size_t add = 0;
        while (!pending.empty() && (int)take.size() < cfg.max_batch) {
            auto &r = pending.front();
            if (used + add + r->bytes > budget) break;
            add += r->bytes;
            take.push_back(r);
            pending.pop_front();
        }
        if (take.empty()) continue;
        used += add;
        slot_busy[(size_t)slot] = true;
        auto batch = std::make_shared<Batch>();
        batch->slot = slot;
        batch->reqs = take;
        cudaStream_t st = streams[(size_t)slot];
        const int fbase = slot * cfg.max_batch;
        lock.unlock();
        // allocate, copy in, launch (outside the lock: copies from pageable memory block this thread)
        std::vector<ssa_group> groups;
        cudaError_t e = cudaSuccess;
        const double t_adm = now_s(t0);
        for (size_t k = 0; k < take.size(); ++k) {
            auto &r = take[k];
            r->t_admit = t_adm;
            r->slot = slot;
            r->batch_size = (int32_t)take.size();
            // the slot's previous launch has finished, so its flags are free to clear
            reinterpret_cast<volatile int32_t *>(h_flags)[fbase + (int)k] = 0;
            const size_t S = r->T.size();
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->d_params, sizeof(double) * r->params.size() + 8, st);
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->d_x0, sizeof(int32_t) * r->x0.size() + 8, st);
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->d_T, sizeof(double) * S + 8, st);
            if (e == cudaSuccess)
                e = cudaMallocAsync((void **)&r->d_samples, sizeof(int32_t) * (size_t)r->n_sims * S * r->N + 8, st);
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->d_stats, sizeof(ssa_sim_stats) * (size_t)r->n_sims + 8, st);
            if (e == cudaSuccess && !r->params.empty())
                e = cudaMemcpyAsync(r->d_params, r->params.data(), sizeof(double) * r->params.size(),
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && !r->x0.empty())
                e = cudaMemcpyAsync(r->d_x0, r->x0.data(), sizeof(int32_t) * r->x0.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && S) e = cudaMemcpyAsync(r->d_T, r->T.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st);
            ssa_group g{};
            g.model = r->model;
            g.n_sims = r->n_sims;
            g.sim_offset = 0;
            g.params = r->d_params;
            g.x0 = r->d_x0;
            g.t_end = r->t_end;
            g.sample_times = r->d_T;
            g.n_samples = (int32_t)S;
            g.seed = r->seed;
            g.samples = r->d_samples;
            g.stats = r->d_stats;
            groups.push_back(g);
        }
        if (e == cudaSuccess)
            e = cudaMemsetAsync(d_counts + fbase, 0, sizeof(unsigned long long) * take.size(), st);
        int rc = SSA_ECUDA;
        std::string msg = e == cudaSuccess ? "" : cudaGetErrorString(e);
        if (e == cudaSuccess) {
            rc = tl::simulate_multi_impl((int32_t)groups.size(), groups.data(), &cfg.opts, st, d_counts + fbase,
                                         d_flags + fbase);
            if (rc != SSA_OK) msg = ssa_last_error();
        }
        if (rc == SSA_OK) {
            e = cudaLaunchHostFunc(st, batch_done_cb, new std::pair<ssa_server *, Batch *>(this, batch.get()));
            if (e != cudaSuccess) {
                rc = SSA_ECUDA;
                msg = cudaGetErrorString(e);
            }
        }
        lock.lock();
        ++launches;
        if (rc == SSA_OK) {
            for (size_t k = 0; k < take.size(); ++k) take[k]->flag = fbase + (int)k;
            inflight.push_back(batch);
        } else {
            for (auto &r : take) {
                r->state = SSA_JOB_FAILED;
                r->error = msg;
                r->t_done = now_s(t0);
            }
            slot_busy[(size_t)slot] = false;
            cv.notify_all();
        }
    }
}

extern "C" {

const char *ssa_server_last_error(void) { return g_srv_error.c_str(); }

void ssa_server_default_config(ssa_server_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->max_device_bytes = 0;
    c->n_streams = 4;
    c->max_batch = 16;
    ssa_default_options(&c->opts);
    c->opts.precision = SSA_FAST;
}

int ssa_server_create(const ssa_server_config *cfg, ssa_server_t *out)
{
    g_srv_error.clear();
    if (!out) return sfail(SSA_EINVAL, "null argument");
    *out = nullptr;
    ssa_server_config c;
    if (cfg) c = *cfg;
    else ssa_server_default_config(&c);
    if (c.n_streams < 1 || c.n_streams > 16) return sfail(SSA_EINVAL, "n_streams must be in 1..16");
    if (c.max_batch < 1 || c.max_batch > 256) return sfail(SSA_EINVAL, "max_batch must be in 1..256");
    if (c.max_device_bytes < 0) return sfail(SSA_EINVAL, "max_device_bytes < 0");
    if (c.opts.layout == SSA_LAYOUT_WARP) return sfail(SSA_EUNSUPPORTED, "the server uses the lane layout");
    auto srv = std::make_unique<ssa_server>();
    srv->cfg = c;
    if (cudaGetDevice(&srv->device) != cudaSuccess) return sfail(SSA_ECUDA, "no CUDA device");
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return sfail(SSA_ECUDA, "cudaMemGetInfo failed");
    srv->budget = c.max_device_bytes > 0 ? (size_t)c.max_device_bytes : (size_t)(0.8 * (double)free_b);
    srv->streams.resize((size_t)c.n_streams);
    srv->slot_busy.assign((size_t)c.n_streams, false);
    for (auto &s : srv->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return sfail(SSA_ECUDA, "stream create failed");
    const size_t n_sig = (size_t)c.n_streams * (size_t)c.max_batch;
    if (cudaHostAlloc((void **)&srv->h_flags, sizeof(int32_t) * n_sig, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&srv->d_flags, srv->h_flags, 0) != cudaSuccess ||
        cudaMalloc((void **)&srv->d_counts, sizeof(unsigned long long) * n_sig) != cudaSuccess) {
        if (srv->h_flags) cudaFreeHost(srv->h_flags);
        if (srv->d_counts) cudaFree(srv->d_counts);
        for (auto &s : srv->streams) cudaStreamDestroy(s);
        return sfail(SSA_ECUDA, "completion-signal allocation failed");
    }
    std::memset(srv->h_flags, 0, sizeof(int32_t) * n_sig);
    srv->t0 = std::chrono::steady_clock::now();
    srv->worker = std::thread([p = srv.get()] { p->run(); });
    *out = srv.release();
    return SSA_OK;
}

int ssa_server_submit(ssa_server_t srv, ssa_model_t model, int64_t n_sims, const double *params, const int32_t *x0,
                      double t_end, const double *sample_times, int32_t n_samples, uint64_t seed, int64_t *ticket)
{
    g_srv_error.clear();
    if (!srv || !model || !ticket) return sfail(SSA_EINVAL, "null argument");
    int32_t N = 0, M = 0;
    ssa_model_info(model, &N, &M);
    if (n_sims < 0 || n_sims > (1ll << 32) || n_samples < 0) return sfail(SSA_EINVAL, "bad sizes");
    if (!(t_end >= 0.0) || t_end > 1e300) return sfail(SSA_EINVAL, "t_end must be finite and >= 0");
    if ((n_sims > 0 && (!params || !x0)) || (n_samples > 0 && !sample_times)) return sfail(SSA_EINVAL, "null host array");
    for (int32_t k = 0; k < n_samples; ++k)
        if (!(sample_times[k] >= 0.0) || !(sample_times[k] <= t_end) || (k && sample_times[k] < sample_times[k - 1]))
            return sfail(SSA_EINVAL, "sample_times must be non-decreasing within [0, t_end]");
    for (int64_t i = 0; i < n_sims * (int64_t)M; ++i)
        if (!(params[i] >= 0.0) || params[i] > 1e300) return sfail(SSA_EINVAL, "params must be finite and >= 0");
    for (int64_t i = 0; i < n_sims * (int64_t)N; ++i)
        if (x0[i] < 0) return sfail(SSA_EINVAL, "x0 must be >= 0");
    auto r = std::make_shared<Request>();
    r->model = model;
    r->N = N;
    r->M = M;
    r->n_sims = n_sims;
    r->params.assign(params, params + n_sims * (int64_t)M);
    r->x0.assign(x0, x0 + n_sims * (int64_t)N);
    r->T.assign(sample_times, sample_times + n_samples);
    r->t_end = t_end;
    r->seed = seed;
    r->bytes = sizeof(double) * r->params.size() + sizeof(int32_t) * r->x0.size() + sizeof(double) * r->T.size() +
               sizeof(int32_t) * (size_t)n_sims * n_samples * N + sizeof(ssa_sim_stats) * (size_t)n_sims + 5 * 512;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (r->bytes > srv->budget)
        return sfail(SSA_ENOMEM, "request needs " + std::to_string(r->bytes) + " bytes, budget " + std::to_string(srv->budget));
    if (srv->shutdown) return sfail(SSA_EINVAL, "server is shutting down");
    r->ticket = srv->next_ticket++;
    r->t_submit = now_s(srv->t0);
    srv->pending.push_back(r);
    srv->all[r->ticket] = r;
    *ticket = r->ticket;
    srv->cv.notify_all();
    return SSA_OK;
}

static void fill_info(const Request &r, ssa_request_info *info)
{
    if (!info) return;
    info->state = r.t_admit < 0 ? 0 : r.state;
    info->batch_size = r.batch_size;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
}

int ssa_server_poll(ssa_server_t srv, int64_t ticket, ssa_request_info *info)
{
    g_srv_error.clear();
    if (!srv) return sfail(SSA_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return sfail(SSA_EINVAL, "unknown ticket");
    fill_info(*it->second, info);
    return SSA_OK;
}

int ssa_server_wait(ssa_server_t srv, int64_t ticket, ssa_request_info *info)
{
    g_srv_error.clear();
    if (!srv) return sfail(SSA_EINVAL, "null server");
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return sfail(SSA_EINVAL, "unknown ticket");
    auto r = it->second;
    srv->cv.wait(lock, [&] { return r->t_done >= 0; });
    fill_info(*r, info);
    return r->state == SSA_JOB_DONE ? SSA_OK : sfail(SSA_ECUDA, r->error);
}

int ssa_server_fetch(ssa_server_t srv, int64_t ticket, int32_t *samples, ssa_sim_stats *stats)
{
    g_srv_error.clear();
    if (!srv) return sfail(SSA_EINVAL, "null server");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        auto it = srv->all.find(ticket);
        if (it == srv->all.end()) return sfail(SSA_EINVAL, "unknown ticket");
        r = it->second;
        srv->cv.wait(lock, [&] { return r->t_done >= 0; });
        srv->all.erase(it);
    }
    int rc = SSA_OK;
    std::string msg;
    cudaSetDevice(srv->device);
    // a stream of this fetch's own: the copies and frees wait for nothing
    // else that runs on the device (the request's results are complete; its
    // launch may still be running other requests)
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess && r->state == SSA_JOB_DONE) {
        const size_t bs = sizeof(int32_t) * (size_t)r->n_sims * r->T.size() * r->N;
        if (samples && bs) e = cudaMemcpyAsync(samples, r->d_samples, bs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && stats && r->n_sims)
            e = cudaMemcpyAsync(stats, r->d_stats, sizeof(ssa_sim_stats) * (size_t)r->n_sims, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = SSA_ECUDA;
            msg = cudaGetErrorString(e);
        }
    } else if (e != cudaSuccess) {
        rc = SSA_ECUDA;
        msg = cudaGetErrorString(e);
    } else {
        rc = SSA_ECUDA;
        msg = r->error;
    }
    for (void *p : {(void *)r->d_params, (void *)r->d_x0, (void *)r->d_T, (void *)r->d_samples, (void *)r->d_stats})
        if (p) cudaFreeAsync(p, st ? st : srv->streams[(size_t)r->slot]);
    if (st) cudaStreamDestroy(st);   // its frees complete on the device afterwards
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (r->t_admit >= 0) srv->used -= r->bytes;
    }
    srv->cv.notify_all();
    return rc == SSA_OK ? SSA_OK : sfail(rc, msg);
}

int ssa_server_stats(ssa_server_t srv, int64_t *launches, int64_t *queued, int64_t *device_bytes_in_use)
{
    if (!srv) return sfail(SSA_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(srv->mu);
    if (launches) *launches = srv->launches;
    if (queued) *queued = (int64_t)srv->pending.size();
    if (device_bytes_in_use) *device_bytes_in_use = (int64_t)srv->used;
    return SSA_OK;
}

int ssa_server_destroy(ssa_server_t srv)
{
    g_srv_error.clear();
    if (!srv) return SSA_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->shutdown = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (auto &kv : srv->all) {
        Request &r = *kv.second;
        cudaStream_t st = r.slot >= 0 ? srv->streams[(size_t)r.slot] : nullptr;
        for (void *p : {(void *)r.d_params, (void *)r.d_x0, (void *)r.d_T, (void *)r.d_samples, (void *)r.d_stats})
            if (p) cudaFreeAsync(p, st);
    }
    for (auto &s : srv->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaFreeHost(srv->h_flags);
    cudaFree(srv->d_counts);
    delete srv;
    return SSA_OK;
}

}  // extern "C"
