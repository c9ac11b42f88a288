// Serving loop for EIG requests (host C++): continuous batching with admission by
// device-memory footprint, a pool of resident workspaces, cancellation with
// per-node checkpoints, and one JSON metrics line per request.
//
// Requests are queued in arrival order.  Up to max_active worker threads each take
// a request as soon as it fits in the free part of the memory budget and run it on
// the worker's own CUDA stream through the public calls (oed_rebind or oed_create,
// oed_hessian, oed_eig), so requests admitted while others are on the GPU overlap
// on the device.  A request's footprint is a context workspace for chunks of its
// nodes plus its node, weight and Hessian arrays; a request whose footprint exceeds
// the whole budget at the configured chunk is run in smaller chunks, down to one
// node, and refused at submission only if even that does not fit.
//
// Workspaces stay resident: when a request finishes, its context goes back to an
// idle pool, and the next request of the same grid shape and precision whose
// workspace fits re-targets it with oed_rebind instead of allocating.  Idle
// workspaces count against the budget and are released, oldest first, when a
// request of another shape needs the room.
//
// Admission takes the oldest queued request that fits; a younger request may be
// admitted ahead of the queue's head (which may be waiting for memory) only while
// the head has waited less than max_wait_s, so a large request cannot starve.
//
// A request runs chunk by chunk; after every chunk its per-node Hessians are copied
// to the host.  A running request can be cancelled between chunks: the nodes
// finished so far stay available (oed_server_checkpoint) and a later request can
// resume from them (oed_request.n_done / H_done), recomputing only the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/oed.h"
#include "nvtx_range.h"

namespace {

struct Request {
    unsigned long long id = 0, tag = 0;
    oed_problem p{};
    std::vector<double> z_top, vp, vs, rho, theta, w, lo, hi, H_done;
    std::vector<int> rec;
    double rel_step = 0.0, sigma = 0.0;
    int jacobian = 0, n = 0, chunk = 1, n_done = 0, per_node = 15;
    size_t ws_bytes = 0;    // context workspace for chunks of `chunk` nodes
    size_t arr_bytes = 0;   // node, weight and Hessian arrays
    double t_submit = 0.0;
};

// An idle context, kept for the next request of its grid shape and precision.
struct Slot {
    oed_ctx *ctx = nullptr;
    size_t bytes = 0;
    int nx = 0, nz = 0, precision = 0, max_solves = 0;
    double t_idle = 0.0;
};

struct Entry {
    oed_result r{};
    bool done = false, cancel = false;
    std::vector<double> H;   // per-node Hessians finished so far, node order, [nodes_done][49]
    std::string json;        // the metrics line, once done
};

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int per_node_of(int jacobian) { return jacobian == OED_JAC_PAIRS ? 15 : 7; }

size_t arrays_bytes(int n) { return (size_t)n * (7 + 1 + 49) * sizeof(double) + 4096; }

}  // namespace

struct oed_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;   // reservations of running requests plus idle workspaces
    int max_active = 1, chunk_nodes = 64;
    bool autotune = true;
    bool stop = false;
    double max_wait_s = 10.0;
    unsigned long long next_id = 1;
    std::deque<Request> queue;
    std::map<unsigned long long, Entry> results;
    std::vector<Slot> idle;
    std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int>> tuning;   // shape, form -> tune
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    int active = 0;
    std::mutex log_mu;
    FILE *log = nullptr;
};

namespace {

bool slot_fits(const Slot &s, const Request &rq)
{
    if (s.nx != rq.p.nx || s.nz != rq.p.nz || s.precision != rq.p.precision) return false;
    if (s.max_solves < rq.per_node * rq.chunk) return false;
    const size_t need = oed_workspace_bytes(&rq.p, s.max_solves);
    return need && need <= s.bytes;
}

// How a request would be admitted: reuse idle slot `slot` (or -1 for a new context),
// releasing the idle slots in `evict` first.
struct Plan {
    size_t k = 0;
    int slot = -1;
    std::vector<int> evict;
};

bool plan_for(const oed_server *srv, const Request &rq, Plan &pl)
{
    pl.slot = -1;
    pl.evict.clear();
    const size_t free_b = srv->budget - srv->in_use;
    for (int i = 0; i < (int)srv->idle.size(); i++)
        if (slot_fits(srv->idle[i], rq) && rq.arr_bytes <= free_b) {
            pl.slot = i;
            return true;
        }
    const size_t need = rq.ws_bytes + rq.arr_bytes;
    size_t avail = free_b;
    if (avail >= need) return true;
    // release idle workspaces, oldest first, until the new one fits
    std::vector<int> order((size_t)srv->idle.size());
    for (int i = 0; i < (int)order.size(); i++) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return srv->idle[a].t_idle < srv->idle[b].t_idle; });
    for (int i : order) {
        pl.evict.push_back(i);
        avail += srv->idle[i].bytes;
        if (avail >= need) return true;
    }
    return false;
}

// The request to admit next, under the lock: the oldest that fits, where younger
// requests may pass the head only while it has waited less than max_wait_s.
bool pick(const oed_server *srv, Plan &pl)
{
    if (srv->queue.empty()) return false;
    const double now = now_s();
    const bool head_old = now - srv->queue.front().t_submit > srv->max_wait_s;
    for (size_t k = 0; k < srv->queue.size(); k++) {
        if (k > 0 && head_old) break;
        if (plan_for(srv, srv->queue[k], pl)) {
            pl.k = k;
            return true;
        }
    }
    return false;
}

const char *status_name(int s)
{
    switch (s) {
    case OED_OK: return "OED_OK";
    case OED_EINVAL: return "OED_EINVAL";
    case OED_ENOMEM: return "OED_ENOMEM";
    case OED_ENOTPD: return "OED_ENOTPD";
    case OED_ECUDA: return "OED_ECUDA";
    case OED_ETIMEOUT: return "OED_ETIMEOUT";
    case OED_PENDING: return "OED_PENDING";
    case OED_ECANCELED: return "OED_ECANCELED";
    default: return "unknown";
    }
}

std::string metrics_json(const Request &rq, const oed_result &r)
{
    const char *jac = rq.jacobian == OED_JAC_PAIRS ? "pairs" : rq.jacobian == OED_JAC_DIFFERENCE ? "difference"
                                                                                                   : "sensitivity";
    const double cells = (double)rq.p.nx * rq.p.nz * rq.p.nsteps * rq.per_node *
                         (double)std::max(0, r.nodes_done - rq.n_done);
    const double run = r.t_done - r.t_admit;
    char buf[1024];
    snprintf(buf, sizeof(buf),
             "{\"id\": %llu, \"tag\": %llu, \"status\": \"%s\", \"grid\": \"%dx%d\", \"h\": %.17g, "
             "\"nsteps\": %d, \"layers\": %d, \"receivers\": %d, \"nodes\": %d, \"nodes_resumed\": %d, "
             "\"nodes_done\": %d, \"chunk_nodes\": %d, \"precision\": \"%s\", \"jacobian\": \"%s\", "
             "\"eig\": %.17g, \"n_bad\": %d, \"t_submit\": %.6f, \"queue_s\": %.6f, \"run_s\": %.6f, "
             "\"latency_s\": %.6f, \"cell_updates\": %.17g, \"gcell_upd_per_s\": %.6g, "
             "\"footprint_bytes\": %zu, \"workspace\": \"%s\"}",
             rq.id, rq.tag, status_name(r.status), rq.p.nx, rq.p.nz, rq.p.h, rq.p.nsteps, rq.p.nlayers,
             rq.p.nrec, rq.n, rq.n_done, r.nodes_done, rq.chunk, rq.p.precision == OED_FP64 ? "f64" : "f32",
             jac, r.status == OED_OK ? r.eig : 0.0, r.n_bad, r.t_submit, r.t_admit - r.t_submit, run,
             r.t_done - r.t_submit, cells, run > 0 ? cells / run / 1e9 : 0.0, r.footprint_bytes,
             r.workspace_reused ? "reused" : "new");
    return buf;
}

// Run one request on stream st with context ctx (already bound to its problem).
int run_request(oed_server *srv, Request &rq, oed_ctx *ctx, cudaStream_t st, Entry *ent)
{
    const size_t n = (size_t)rq.n;
    double *d = nullptr;
    const size_t doubles = n * 7 + n + n * 49 + 1;
    if (cudaMallocAsync((void **)&d, doubles * sizeof(double) + 64, st) != cudaSuccess) {
        cudaGetLastError();
        return OED_ENOMEM;
    }
    double *d_theta = d, *d_w = d + n * 7, *d_H = d_w + n, *d_eig = d_H + n * 49;
    int *d_bad = (int *)(d_eig + 1);
    int rc = oed_set_jacobian(ctx, rq.jacobian);
    if (!rc) {
        const auto key = std::make_tuple(rq.p.nx, rq.p.nz, rq.p.precision, rq.jacobian);
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
            rc = oed_autotune(ctx, rq.per_node * rq.chunk, st);
            int c, z, wz;
            oed_get_tuning(ctx, &c, &z, &wz);
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->tuning[key] = std::make_tuple(c, z, wz);
        }
    }
    std::vector<double> Hc;
    bool cancelled = false;
    if (!rc) {
        cudaMemcpyAsync(d_theta, rq.theta.data(), sizeof(double) * n * 7, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_w, rq.w.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
        if (rq.n_done > 0)   // resumed nodes: their Hessians as the earlier request left them
            cudaMemcpyAsync(d_H, rq.H_done.data(), sizeof(double) * rq.n_done * 49, cudaMemcpyHostToDevice, st);
        for (int off = rq.n_done; off < rq.n && !rc; off += rq.chunk) {
            const int nb = std::min(rq.chunk, rq.n - off);
            oed::NvtxRange chunk_range("oed_server: chunk of nodes");
            rc = oed_hessian(ctx, d_theta + (size_t)off * 7, nb, rq.lo.data(), rq.hi.data(), rq.rel_step,
                             rq.sigma, nullptr, 0, d_H + (size_t)off * 49, nullptr, nullptr, st);
            if (!rc) {
                Hc.resize((size_t)nb * 49);
                cudaMemcpyAsync(Hc.data(), d_H + (size_t)off * 49, sizeof(double) * nb * 49, cudaMemcpyDeviceToHost,
                                st);
                if (cudaStreamSynchronize(st) != cudaSuccess) rc = OED_ECUDA;
            }
            if (rc) break;
            std::lock_guard<std::mutex> lk(srv->mu);
            ent->H.insert(ent->H.end(), Hc.begin(), Hc.end());
            ent->r.nodes_done = off + nb;
            if (ent->cancel && off + nb < rq.n) {
                cancelled = true;
                break;
            }
        }
    }
    double eig = 0.0;
    int bad = 0;
    if (!rc && !cancelled) {
        rc = oed_eig(ctx, d_H, rq.n, d_w, rq.lo.data(), rq.hi.data(), d_eig, nullptr, nullptr, d_bad, st);
        if (!rc) {
            cudaMemcpyAsync(&eig, d_eig, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        }
    }
    cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = OED_ECUDA;
    if (!rc && !cancelled) {
        std::lock_guard<std::mutex> lk(srv->mu);
        ent->r.eig = eig;
        ent->r.n_bad = bad;
    }
    return rc ? rc : (cancelled ? OED_ECANCELED : OED_OK);
}

// Bind the pooled context (or create one) and run the request on it.
int serve_one(oed_server *srv, Request &rq, Slot &slot, bool reuse, cudaStream_t st, Entry *ent)
{
    oed::NvtxRange range("oed_server: request");
    int rc = OED_OK;
    if (reuse) {
        rc = oed_rebind(slot.ctx, &rq.p);
    } else {
        slot.ctx = nullptr;
        rc = oed_create(&slot.ctx, &rq.p, rq.per_node * rq.chunk);
        slot.bytes = rq.ws_bytes;
        slot.nx = rq.p.nx;
        slot.nz = rq.p.nz;
        slot.precision = rq.p.precision;
        slot.max_solves = rq.per_node * rq.chunk;
    }
    return rc ? rc : run_request(srv, rq, slot.ctx, st, ent);
}

void worker_loop(oed_server *srv)
{
    cudaSetDevice(srv->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request rq;
        Slot slot;
        bool reuse = false;
        std::vector<Slot> evicted;
        Entry *ent = nullptr;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            Plan pl;
            srv->cv_work.wait(lk, [&] { return srv->stop || pick(srv, pl); });
            if (srv->stop) break;
            rq = std::move(srv->queue[pl.k]);
            srv->queue.erase(srv->queue.begin() + (long)pl.k);
            if (pl.slot >= 0) {
                slot = srv->idle[pl.slot];
                reuse = true;
            }
            // release the planned idle workspaces (indices refer to the current list)
            std::vector<int> gone = pl.evict;
            if (pl.slot >= 0) gone.push_back(pl.slot);
            std::sort(gone.begin(), gone.end(), std::greater<int>());
            for (int i : gone) {
                if (i != pl.slot) {
                    srv->in_use -= srv->idle[i].bytes;
                    evicted.push_back(srv->idle[i]);
                }
                srv->idle.erase(srv->idle.begin() + i);
            }
            srv->in_use += reuse ? rq.arr_bytes : rq.ws_bytes + rq.arr_bytes;
            srv->active++;
            ent = &srv->results[rq.id];
            ent->r.t_admit = now_s();
            ent->r.footprint_bytes = (reuse ? slot.bytes : rq.ws_bytes) + rq.arr_bytes;
            ent->r.workspace_reused = reuse ? 1 : 0;
        }
        for (Slot &s : evicted) oed_destroy(s.ctx);
        const int rc = serve_one(srv, rq, slot, reuse, st, ent);
        bool keep = !rc || rc == OED_ECANCELED || rc == OED_ENOTPD;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            ent->r.status = rc;
            if (rc) ent->r.eig = 0.0;
            ent->r.t_done = now_s();
            ent->done = true;
            ent->json = metrics_json(rq, ent->r);
            srv->in_use -= rq.arr_bytes;
            if (!slot.ctx || srv->stop) keep = false;
            if (keep) {
                slot.t_idle = ent->r.t_done;
                srv->idle.push_back(slot);
            } else {
                srv->in_use -= reuse ? slot.bytes : rq.ws_bytes;
            }
            srv->active--;
        }
        if (!keep && slot.ctx) oed_destroy(slot.ctx);
        {
            std::lock_guard<std::mutex> lk(srv->log_mu);
            if (srv->log) {
                fprintf(srv->log, "%s\n", ent->json.c_str());
                fflush(srv->log);
            }
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

}  // namespace

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

int oed_server_set_admission(oed_server *srv, double max_wait_s)
{
    if (!srv || !(max_wait_s >= 0.0)) return OED_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->max_wait_s = max_wait_s;
    }
    srv->cv_work.notify_all();
    return OED_OK;
}

int oed_server_set_log(oed_server *srv, const char *path)
{
    if (!srv) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->log_mu);
    if (srv->log && srv->log != stderr) fclose(srv->log);
    srv->log = nullptr;
    if (!path) return OED_OK;
    if (!strcmp(path, "-")) {
        srv->log = stderr;
        return OED_OK;
    }
    srv->log = fopen(path, "a");
    return srv->log ? OED_OK : OED_EINVAL;
}

static size_t footprint(const oed_request *req, int chunk)
{
    const int per_node = per_node_of(req->jacobian);
    const size_t ws = oed_workspace_bytes(&req->problem, per_node * chunk);
    return ws ? ws + arrays_bytes(req->n) : 0;
}

size_t oed_server_request_bytes(const oed_request *req, int chunk_nodes)
{
    if (!req || req->n < 1 || chunk_nodes < 1) return 0;
    if (req->jacobian == OED_JAC_SENSITIVITY && req->problem.stf != OED_STF_GAUSS) return 0;
    return footprint(req, req->n < chunk_nodes ? req->n : chunk_nodes);
}

int oed_server_submit(oed_server *srv, const oed_request *req, unsigned long long *id)
{
    if (!srv || !req || !id || req->n < 1 || !req->theta || !req->w || !req->lo || !req->hi)
        return OED_EINVAL;
    if (req->jacobian != OED_JAC_PAIRS && req->jacobian != OED_JAC_DIFFERENCE &&
        req->jacobian != OED_JAC_SENSITIVITY)
        return OED_EINVAL;
    if (req->jacobian == OED_JAC_SENSITIVITY && req->problem.stf != OED_STF_GAUSS) return OED_EINVAL;
    if (req->n_done < 0 || req->n_done > req->n || (req->n_done > 0 && !req->H_done)) return OED_EINVAL;
    Request rq;
    rq.per_node = per_node_of(req->jacobian);
    // nodes per chunk: the configured count, halved until the footprint fits the budget
    int chunk = req->n < srv->chunk_nodes ? req->n : srv->chunk_nodes;
    size_t fp = footprint(req, chunk);
    if (!fp) return OED_EINVAL;
    while (fp > srv->budget && chunk > 1) {
        chunk = (chunk + 1) / 2;
        fp = footprint(req, chunk);
    }
    if (fp > srv->budget) return OED_ENOMEM;   // can never be admitted
    rq.chunk = chunk;
    rq.arr_bytes = arrays_bytes(req->n);
    rq.ws_bytes = fp - rq.arr_bytes;
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
    rq.n_done = req->n_done;
    if (req->n_done > 0) rq.H_done.assign(req->H_done, req->H_done + (size_t)req->n_done * 49);
    rq.tag = req->tag;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        rq.id = srv->next_id++;
        rq.t_submit = now_s();
        Entry &e = srv->results[rq.id];
        std::memset(&e.r, 0, sizeof(e.r));
        e.r.status = OED_PENDING;
        e.r.t_submit = rq.t_submit;
        e.r.footprint_bytes = fp;
        e.r.nodes_done = rq.n_done;
        e.H = rq.H_done;
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
    Entry &e = it->second;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return e.done; });
    *out = e.r;
    if (!ok) {
        out->status = OED_PENDING;
        return OED_ETIMEOUT;
    }
    return OED_OK;
}

int oed_server_cancel(oed_server *srv, unsigned long long id)
{
    if (!srv) return OED_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->results.find(id);
        if (it == srv->results.end()) return OED_EINVAL;
        Entry &e = it->second;
        if (e.done) return OED_OK;
        for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
            if (q->id == id) {   // still queued: never runs
                e.r.status = OED_ECANCELED;
                e.r.t_admit = e.r.t_done = now_s();
                e.done = true;
                e.json = metrics_json(*q, e.r);
                srv->queue.erase(q);
                break;
            }
        e.cancel = true;   // running: stops after its current chunk
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    return OED_OK;
}

int oed_server_checkpoint(oed_server *srv, unsigned long long id, double *H, int cap, int *nodes_done)
{
    if (!srv || !nodes_done || cap < 0) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->results.find(id);
    if (it == srv->results.end()) return OED_EINVAL;
    const Entry &e = it->second;
    const int nd = (int)(e.H.size() / 49);
    *nodes_done = nd;
    if (!H) return OED_OK;
    if (cap < nd) return OED_ENOMEM;
    std::copy(e.H.begin(), e.H.end(), H);
    return OED_OK;
}

int oed_server_metrics(oed_server *srv, unsigned long long id, char *buf, size_t cap)
{
    if (!srv || !buf || cap == 0) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->results.find(id);
    if (it == srv->results.end()) return OED_EINVAL;
    if (!it->second.done) return OED_PENDING;
    const std::string &j = it->second.json;
    if (j.size() + 1 > cap) return OED_ENOMEM;
    memcpy(buf, j.c_str(), j.size() + 1);
    return OED_OK;
}

int oed_server_release(oed_server *srv, unsigned long long id)
{
    if (!srv) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->results.find(id);
    if (it == srv->results.end()) return OED_EINVAL;
    if (!it->second.done) return OED_PENDING;
    srv->results.erase(it);
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

int oed_server_pool(oed_server *srv, int *idle, size_t *idle_bytes)
{
    if (!srv) return OED_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    size_t b = 0;
    for (const Slot &s : srv->idle) b += s.bytes;
    if (idle) *idle = (int)srv->idle.size();
    if (idle_bytes) *idle_bytes = b;
    return OED_OK;
}

int oed_server_destroy(oed_server *srv)
{
    if (!srv) return OED_OK;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        // queued requests are cancelled; running ones finish
        for (auto &rq : srv->queue) {
            Entry &e = srv->results[rq.id];
            e.r.status = OED_ECANCELED;
            e.done = true;
        }
        srv->queue.clear();
        srv->cv_done.wait(lk, [&] { return srv->active == 0; });
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (auto &t : srv->workers) t.join();
    for (Slot &s : srv->idle) oed_destroy(s.ctx);
    srv->idle.clear();
    oed_server_set_log(srv, nullptr);
    delete srv;
    return OED_OK;
}

}  // extern "C"
