// Serving loop for EIG requests (host C++): continuous batching with admission by
// device-memory footprint.
//
// Requests are queued in arrival order.  Up to max_active worker threads take the
// head of the queue as soon as it fits in the free part of the memory budget;
// each runs its request on its own CUDA stream through the public calls
// (oed_create, oed_hessian, oed_eig), so requests admitted while others are on the
// GPU overlap on the device.  A request's footprint is its context workspace plus
// its node, weight and Hessian arrays; a request larger than the whole budget is
// refused at submission.  Launch shapes are autotuned once per grid shape and
// reused.  Timestamps (submission, admission, completion) come from one monotonic
// clock so the caller can form latency percentiles.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/oed.h"

namespace {

struct Request {
    unsigned long long id;
    oed_problem p;
    std::vector<double> z_top, vp, vs, rho, theta, w, lo, hi;
    std::vector<int> rec;
    double rel_step, sigma;
    int jacobian, n, chunk;
    size_t footprint;
    double t_submit;
};

struct Result {
    oed_result r;
    bool done = false;
};

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct oed_server {
    int device = 0;
    size_t budget = 0, in_use = 0;
    int max_active = 1, chunk_nodes = 64;
    bool autotune = true;
    bool stop = false;
    unsigned long long next_id = 1;
    std::deque<Request> queue;
    std::map<unsigned long long, Result> results;
    std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int>> tuning;   // shape -> tune
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    int active = 0;
};

static int run_request(oed_server *srv, Request &rq, oed_result *res)
{
    cudaSetDevice(srv->device);
    const int per_node = rq.jacobian == OED_JAC_PAIRS ? 15 : 7;
    oed_ctx *ctx = nullptr;
    int rc = oed_create(&ctx, &rq.p, per_node * rq.chunk);
    if (rc) return rc;
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    double *d = nullptr;
    const size_t n = (size_t)rq.n;
    const size_t doubles = n * 7 + n + n * 49 + 1;
    cudaError_t e = cudaMallocAsync((void **)&d, doubles * sizeof(double) + 64, st);
    if (e != cudaSuccess) {
        oed_destroy(ctx);
        cudaStreamDestroy(st);
        return OED_ENOMEM;
    }
    double *d_theta = d, *d_w = d + n * 7, *d_H = d_w + n, *d_eig = d_H + n * 49;
    int *d_bad = (int *)(d_eig + 1);
    rc = oed_set_jacobian(ctx, rq.jacobian);
    if (!rc) {
        const auto key = std::make_tuple(rq.p.nx, rq.p.nz, rq.p.precision, rq.jacobian, rq.chunk);
        std::tuple<int, int, int> tune;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            auto it = srv->tuning.find(key);
            if (it != srv->tuning.end()) {
                tune = it->second;
                have = true;
            }
        }
        if (have) {
            rc = oed_set_tuning(ctx, std::get<0>(tune), std::get<1>(tune), std::get<2>(tune));
        } else if (srv->autotune) {
            rc = oed_autotune(ctx, per_node * rq.chunk, st);
            int c, z, wz;
            oed_get_tuning(ctx, &c, &z, &wz);
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->tuning[key] = std::make_tuple(c, z, wz);
        }
    }
    if (!rc) {
        cudaMemcpyAsync(d_theta, rq.theta.data(), sizeof(double) * n * 7, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_w, rq.w.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
        rc = oed_hessian(ctx, d_theta, rq.n, rq.lo.data(), rq.hi.data(), rq.rel_step, rq.sigma, nullptr,
                         0, d_H, nullptr, nullptr, st);
    }
    if (!rc)
        rc = oed_eig(ctx, d_H, rq.n, d_w, rq.lo.data(), rq.hi.data(), d_eig, nullptr, nullptr, d_bad, st);
    if (!rc) {
        cudaMemcpyAsync(&res->eig, d_eig, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&res->n_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = OED_ECUDA;
    cudaStreamDestroy(st);
    oed_destroy(ctx);
    return rc;
}

static void worker_loop(oed_server *srv)
{
    for (;;) {
        Request rq;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                return srv->stop ||
                       (!srv->queue.empty() && srv->in_use + srv->queue.front().footprint <= srv->budget);
            });
            if (srv->stop) return;
            rq = std::move(srv->queue.front());
            srv->queue.pop_front();
            srv->in_use += rq.footprint;
            srv->active++;
            Result &r = srv->results[rq.id];
            r.r.t_admit = now_s();
        }
        oed_result out;
        std::memset(&out, 0, sizeof(out));
        const int rc = run_request(srv, rq, &out);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            Result &r = srv->results[rq.id];
            r.r.status = rc;
            r.r.eig = rc ? 0.0 : out.eig;
            r.r.n_bad = rc ? 0 : out.n_bad;
            r.r.t_done = now_s();
            r.done = true;
            srv->in_use -= rq.footprint;
            srv->active--;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
}

extern "C" {

int oed_server_create(oed_server **out, size_t hbm_budget_bytes, int max_active, int chunk_nodes,
                      int flags)
{
    if (!out || max_active < 1 || max_active > 64 || chunk_nodes < 1 || hbm_budget_bytes == 0)
        return OED_EINVAL;
    oed_server *srv = new oed_server();
    cudaGetDevice(&srv->device);
    srv->budget = hbm_budget_bytes;
    srv->max_active = max_active;
    srv->chunk_nodes = chunk_nodes;
    srv->autotune = !(flags & OED_SERVER_NO_AUTOTUNE);
    for (int k = 0; k < max_active; k++) srv->workers.emplace_back(worker_loop, srv);
    *out = srv;
    return OED_OK;
}

size_t oed_server_request_bytes(const oed_request *req, int chunk_nodes)
{
    if (!req || req->n < 1 || chunk_nodes < 1) return 0;
    const int per_node = req->jacobian == OED_JAC_PAIRS ? 15 : 7;
    const int chunk = req->n < chunk_nodes ? req->n : chunk_nodes;
    if (req->jacobian == OED_JAC_SENSITIVITY && req->problem.stf != OED_STF_GAUSS) return 0;
    const size_t ws = oed_workspace_bytes(&req->problem, per_node * chunk);
    if (!ws) return 0;
    return ws + (size_t)req->n * (7 + 1 + 49) * sizeof(double) + 4096;
}

int oed_server_submit(oed_server *srv, const oed_request *req, unsigned long long *id)
{
    if (!srv || !req || !id || req->n < 1 || !req->theta || !req->w || !req->lo || !req->hi)
        return OED_EINVAL;
    if (req->jacobian != OED_JAC_PAIRS && req->jacobian != OED_JAC_DIFFERENCE &&
        req->jacobian != OED_JAC_SENSITIVITY)
        return OED_EINVAL;
    Request rq;
    rq.chunk = req->n < srv->chunk_nodes ? req->n : srv->chunk_nodes;
    rq.footprint = oed_server_request_bytes(req, srv->chunk_nodes);
    if (!rq.footprint) return OED_EINVAL;
    if (rq.footprint > srv->budget) return OED_ENOMEM;   // can never be admitted
    const oed_problem &p = req->problem;
    rq.p = p;
    rq.z_top.assign(p.z_top, p.z_top + p.nlayers);
    rq.vp.assign(p.vp, p.vp + p.nlayers);
    rq.vs.assign(p.vs, p.vs + p.nlayers);
    rq.rho.assign(p.rho, p.rho + p.nlayers);
    rq.rec.assign(p.rec_ix, p.rec_ix + p.nrec);
    rq.p.z_top = rq.z_top.data();
    rq.p.vp = rq.vp.data();
    rq.p.vs = rq.vs.data();
    rq.p.rho = rq.rho.data();
    rq.p.rec_ix = rq.rec.data();
    rq.n = req->n;
    rq.theta.assign(req->theta, req->theta + (size_t)req->n * 7);
    rq.w.assign(req->w, req->w + req->n);
    rq.lo.assign(req->lo, req->lo + 7);
    rq.hi.assign(req->hi, req->hi + 7);
    rq.rel_step = req->rel_step;
    rq.sigma = req->sigma;
    rq.jacobian = req->jacobian;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        rq.id = srv->next_id++;
        rq.t_submit = now_s();
        Result &r = srv->results[rq.id];
        std::memset(&r.r, 0, sizeof(r.r));
        r.r.status = OED_PENDING;
        r.r.t_submit = rq.t_submit;
        r.r.footprint_bytes = rq.footprint;
        *id = rq.id;
        srv->queue.push_back(std::move(rq));
    }
    srv->cv_work.notify_all();
    return OED_OK;
}

int oed_server_poll(oed_server *srv, unsigned long long id, oed_result *out)
{
    if (!srv || !out) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->results.find(id);
    if (it == srv->results.end()) return OED_EINVAL;
    *out = it->second.r;
    if (!it->second.done) out->status = OED_PENDING;
    return OED_OK;
}

int oed_server_wait(oed_server *srv, unsigned long long id, double timeout_s, oed_result *out)
{
    if (!srv || !out) return OED_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->results.find(id);
    if (it == srv->results.end()) return OED_EINVAL;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                          [&] { return srv->results[id].done; });
    *out = srv->results[id].r;
    if (!ok) {
        out->status = OED_PENDING;
        return OED_ETIMEOUT;
    }
    return OED_OK;
}

int oed_server_stats(oed_server *srv, size_t *in_use, int *active, int *queued)
{
    if (!srv) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (in_use) *in_use = srv->in_use;
    if (active) *active = srv->active;
    if (queued) *queued = (int)srv->queue.size();
    return OED_OK;
}

int oed_server_destroy(oed_server *srv)
{
    if (!srv) return OED_OK;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        // queued requests are cancelled; running ones finish
        for (auto &rq : srv->queue) {
            Result &r = srv->results[rq.id];
            r.r.status = OED_ECANCELED;
            r.done = true;
        }
        srv->queue.clear();
        srv->cv_done.wait(lk, [&] { return srv->active == 0; });
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (auto &t : srv->workers) t.join();
    delete srv;
    return OED_OK;
}

}  // extern "C"
