// C ABI of liboed (include/oed.h): context, workspace, validation, chunking and
// the captured CUDA graph that replays the time loop of a batch of solves.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "nvtx_range.h"
#include "oed_internal.cuh"

namespace oed {

int set_err(oed_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_err(oed_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return OED_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_err(ctx, OED_ENOMEM, m);
    return set_err(ctx, OED_ECUDA, m);
}

void hessian_init(cudaStream_t);
int hsub_threads(int nrec);

static bool problem_ok(const oed_problem *p, std::string *why)
{
    auto fail = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (!p) return fail("problem is NULL");
    if (p->nx < 8 || p->nz < 8) return fail("nx and nz must be >= 8");
    if ((long long)p->nx * p->nz > (1LL << 30)) return fail("grid too large");
    if (!(p->h > 0) || !(p->dt > 0) || !std::isfinite(p->h) || !std::isfinite(p->dt))
        return fail("h and dt must be positive");
    if (p->nsteps < 1 || p->nsteps > 1000000) return fail("nsteps must be in 1..1e6");
    if (p->nlayers < 1 || p->nlayers > 64 || !p->z_top || !p->vp || !p->vs || !p->rho)
        return fail("need 1..64 layers with z_top, vp, vs, rho");
    if (p->z_top[0] != 0.0) return fail("z_top[0] must be 0");
    for (int l = 0; l < p->nlayers; l++) {
        if (l > 0 && !(p->z_top[l] > p->z_top[l - 1])) return fail("z_top must increase");
        if (!(p->vp[l] > 0) || !(p->vs[l] > 0) || !(p->rho[l] > 0))
            return fail("vp, vs, rho must be positive");
        if (!(p->vp[l] * p->vp[l] >= 2.0 * p->vs[l] * p->vs[l]))
            return fail("vp^2 >= 2 vs^2 required (lambda >= 0)");
    }
    if (p->nrec < 1 || p->nrec > kMaxRec || !p->rec_ix) return fail("nrec must be in 1..4096");
    for (int r = 0; r < p->nrec; r++)
        if (p->rec_ix[r] < 0 || p->rec_ix[r] >= p->nx) return fail("receiver index outside 0..nx-1");
    if (p->precision != OED_FP32 && p->precision != OED_FP64) return fail("precision must be OED_FP32 or OED_FP64");
    if (p->stf != OED_STF_GAUSS && p->stf != OED_STF_RICKER) return fail("stf must be OED_STF_GAUSS or OED_STF_RICKER");
    return true;
}

static Geometry make_geometry(const oed_problem *p)
{
    Geometry g;
    g.nx = p->nx;
    g.nz = p->nz;
    g.xp = (p->nx + 31) / 32 * 32;
    g.nsteps = p->nsteps;
    g.nlev = p->nsteps + 1;
    g.nrec = p->nrec;
    g.h = p->h;
    g.dt = p->dt;
    g.comp_stride = (size_t)g.nz * g.xp;
    g.solve_stride = 2 * g.comp_stride;
    return g;
}

struct Sizes {
    size_t u, u2, kp, src, stf, trace, theta, rows, rec, hseg, err, total;
};

static Sizes sizes(const Geometry &g, int precision, int max_solves)
{
    const size_t e = precision == OED_FP64 ? 8 : 4;
    const int chunk = std::max(1, max_solves / kND);   // the larger of the two node chunks
    Sizes s;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    // FP32 grids that do not fit on chip keep a second pair of levels for the two-step
    // kernel (it reads one pair and writes the other), whose paired layout may need a
    // little more than the planar one per solve
    const bool two_step = precision == OED_FP32 && !resident_fits(g);
    const size_t per = two_step ? std::max(g.solve_stride, paired_stride(g)) : g.solve_stride;
    s.u = al((size_t)max_solves * per * e);
    s.u2 = two_step ? 2 * s.u : 0;
    s.kp = s.u2 ? al((size_t)g.nz * 16 * sizeof(float)) : 0;   // packed row coefficients
    s.src = al((size_t)max_solves * (precision == OED_FP64 ? sizeof(SourceDesc<double>)
                                                           : sizeof(SourceDesc<float>)));
    s.stf = al((size_t)max_solves * g.nsteps * e);
    s.trace = al((size_t)max_solves * g.nlev * g.nrec * 2 * e);
    s.theta = al((size_t)max_solves * kNT * sizeof(double));
    s.rows = al((size_t)g.nz * (precision == OED_FP64 ? sizeof(RowCoef<double>) : sizeof(RowCoef<float>)));
    s.rows += al((size_t)g.nz * (precision == OED_FP64 ? sizeof(FacCoef<double>) : sizeof(FacCoef<float>)));
    s.rec = al((size_t)g.nrec * sizeof(int));
    s.hseg = al((size_t)chunk * 16 * g.nrec * 28 * sizeof(double));
    s.err = 256;
    s.total = 2 * s.u + s.u2 + s.kp + s.src + s.stf + s.trace + s.theta + s.rows + s.rec + s.hseg + s.err;
    return s;
}

static void drop_graphs(oed_ctx *ctx)
{
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
}

// Run the time loop for nsolve solves on stream st, replaying a captured graph
// (built on first use for this batch size).
static int run_steps(oed_ctx *ctx, int nsolve, cudaStream_t st)
{
    // the expiry flag describes this time loop only
    cudaError_t ez = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
    if (ez != cudaSuccess) return cuda_err(ctx, ez, "cudaMemsetAsync");
    if (ctx->tune.C > 0) {
        // one persistent launch integrates every step; no wavefield in HBM
        ctx->last_steps_launches = ctx->g.nsteps;
        return cuda_err(ctx, launch_resident(ctx, ctx->tune.C, nsolve, st, ctx->ev_steps[0],
                                             ctx->ev_steps[1], 0),
                        "cluster-resident launch");
    }
    auto it = ctx->graphs.find(nsolve);
    if (it == ctx->graphs.end()) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamCreate");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_err(ctx, e, "cudaStreamBeginCapture");
        }
        const cudaError_t el = launch_forward_steps(ctx, nsolve, cap, ctx->ev_steps[0], ctx->ev_steps[1]);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (el != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_err(ctx, el, "time loop launch");
        }
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphInstantiate");
        it = ctx->graphs.emplace(nsolve, ex).first;
    }
    ctx->last_steps_launches = ctx->g.nsteps;
    return cuda_err(ctx, cudaGraphLaunch(it->second, st), "cudaGraphLaunch");
}

// Lay the workspace arrays out in the single allocation starting at base.
static void carve(oed_ctx *ctx, char *base, const Sizes &s)
{
    char *q = base;
    ctx->d_u0 = q; q += s.u;
    ctx->d_u1 = q; q += s.u;
    ctx->d_u2 = s.u2 ? q : nullptr;
    ctx->d_u3 = s.u2 ? q + s.u : nullptr;
    q += s.u2;
    ctx->d_kp = s.kp ? q : nullptr;
    q += s.kp;
    ctx->d_src = q; q += s.src;
    ctx->d_stf = q; q += s.stf;
    ctx->d_trace = q; q += s.trace;
    ctx->d_theta = (double *)q; q += s.theta;
    ctx->d_rows = q;
    ctx->d_fac = q + ((size_t)ctx->g.nz * (ctx->precision == OED_FP64 ? sizeof(RowCoef<double>)
                                                                       : sizeof(RowCoef<float>)) +
                      255) / 256 * 256;
    q += s.rows;
    ctx->d_rec = (int *)q; q += s.rec;
    ctx->d_hseg = (double *)q; q += s.hseg;
    ctx->d_err = (int *)q; q += s.err;
}

// Problem-dependent contents of the workspace: error flag, defined source descriptors,
// receiver indices and the rows' stencil coefficients (on the context's own stream).
static void fill_problem(oed_ctx *ctx)
{
    cudaMemsetAsync(ctx->d_err, 0, 256, ctx->own_stream);
    cudaMemsetAsync(ctx->d_src, 0, (size_t)ctx->max_solves * (ctx->precision == OED_FP64
                                                                  ? sizeof(SourceDesc<double>)
                                                                  : sizeof(SourceDesc<float>)),
                    ctx->own_stream);   // defined descriptors before first use
    cudaMemcpyAsync(ctx->d_rec, ctx->rec_ix.data(), sizeof(int) * ctx->rec_ix.size(), cudaMemcpyHostToDevice,
                    ctx->own_stream);
    launch_rows(ctx, ctx->own_stream);   // synchronises the stream
    launch_pack_kp(ctx, ctx->own_stream);
}

}  // namespace oed

using namespace oed;

extern "C" {

const char *oed_status_string(int status)
{
    switch (status) {
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

size_t oed_workspace_bytes(const oed_problem *p, int max_solves)
{
    if (!problem_ok(p, nullptr) || max_solves < 1) return 0;
    return sizes(make_geometry(p), p->precision, max_solves).total;
}

int oed_create(oed_ctx **out, const oed_problem *p, int max_solves)
{
    if (!out) return OED_EINVAL;
    *out = nullptr;
    std::string why;
    if (!problem_ok(p, &why)) {
        fprintf(stderr, "oed_create: %s\n", why.c_str());
        return OED_EINVAL;
    }
    if (max_solves < 1 || max_solves > 65535) {
        fprintf(stderr, "oed_create: max_solves must be in 1..65535\n");
        return OED_EINVAL;
    }
    oed_ctx *ctx = new (std::nothrow) oed_ctx();
    if (!ctx) return OED_ENOMEM;
    ctx->g = make_geometry(p);
    ctx->precision = p->precision;
    ctx->stf = p->stf;
    ctx->elem = p->precision == OED_FP64 ? 8 : 4;
    ctx->max_solves = max_solves;
    cudaGetDevice(&ctx->device);
    ctx->z_top.assign(p->z_top, p->z_top + p->nlayers);
    ctx->vp.assign(p->vp, p->vp + p->nlayers);
    ctx->vs.assign(p->vs, p->vs + p->nlayers);
    ctx->rho.assign(p->rho, p->rho + p->nlayers);
    ctx->rec_ix.assign(p->rec_ix, p->rec_ix + p->nrec);

    const Sizes s = sizes(ctx->g, ctx->precision, max_solves);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete ctx;
        return OED_ECUDA;
    }
    if (s.total > free_b) {
        fprintf(stderr, "oed_create: workspace %zu B exceeds free device memory %zu B\n", s.total, free_b);
        delete ctx;
        return OED_ENOMEM;
    }
    char *base = nullptr;
    cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    cudaError_t e = cudaMallocAsync((void **)&base, s.total, ctx->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->own_stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(ctx->own_stream);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? OED_ENOMEM : OED_ECUDA;
    }
    ctx->bytes = s.total;
    carve(ctx, base, s);
    cudaEventCreate(&ctx->ev_steps[0]);
    cudaEventCreate(&ctx->ev_steps[1]);
    hessian_init(ctx->own_stream);
    fill_problem(ctx);
    e = cudaStreamSynchronize(ctx->own_stream);
    if (e != cudaSuccess) {
        int rc = cuda_err(ctx, e, "oed_create");
        oed_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return OED_OK;
}

int oed_destroy(oed_ctx *ctx)
{
    if (!ctx) return OED_OK;
    drop_graphs(ctx);
    if (ctx->d_u0) {   // base of the single workspace allocation
        cudaFreeAsync(ctx->d_u0, ctx->own_stream);
        cudaStreamSynchronize(ctx->own_stream);
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    for (int k = 0; k < 2; k++)
        if (ctx->ev_steps[k]) cudaEventDestroy(ctx->ev_steps[k]);
    cudaFree(ctx->h_stage_theta);
    cudaFree(ctx->h_stage_w);
    cudaFree(ctx->h_stage_H);
    cudaFree(ctx->h_stage_dkl);
    cudaFree(ctx->h_stage_eig);
    cudaFree(ctx->h_stage_bad);
    cudaFree(ctx->d_adj);
    delete ctx;
    return OED_OK;
}

int oed_rebind(oed_ctx *ctx, const oed_problem *p)
{
    if (!ctx) return OED_EINVAL;
    std::string why;
    if (!problem_ok(p, &why)) return set_err(ctx, OED_EINVAL, "oed_rebind: " + why);
    if (p->nx != ctx->g.nx || p->nz != ctx->g.nz || p->precision != ctx->precision)
        return set_err(ctx, OED_EINVAL, "oed_rebind: the grid shape and precision must be the context's");
    const Geometry g = make_geometry(p);
    const Sizes s = sizes(g, p->precision, ctx->max_solves);
    if (s.total > ctx->bytes)
        return set_err(ctx, OED_ENOMEM, "oed_rebind: the problem's workspace exceeds the context's");
    if (p->stf != OED_STF_GAUSS && ctx->jac_mode == OED_JAC_SENSITIVITY)
        return set_err(ctx, OED_EINVAL, "oed_rebind: sensitivity solves need the Gaussian time function");
    // the caller has synchronised the streams of its earlier calls on this context
    cudaError_t e = cudaStreamSynchronize(ctx->own_stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "oed_rebind");
    drop_graphs(ctx);   // captured time loops hold the old problem's sizes
    ctx->g = g;
    ctx->stf = p->stf;
    ctx->z_top.assign(p->z_top, p->z_top + p->nlayers);
    ctx->vp.assign(p->vp, p->vp + p->nlayers);
    ctx->vs.assign(p->vs, p->vs + p->nlayers);
    ctx->rho.assign(p->rho, p->rho + p->nlayers);
    ctx->rec_ix.assign(p->rec_ix, p->rec_ix + p->nrec);
    carve(ctx, (char *)ctx->d_u0, s);
    fill_problem(ctx);
    return cuda_err(ctx, cudaStreamSynchronize(ctx->own_stream), "oed_rebind");
}

const char *oed_last_error(const oed_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

int oed_last_step_time(const oed_ctx *ctx, float *ms, int *launches)
{
    if (!ctx || !ms) return OED_EINVAL;
    *ms = 0.0f;
    if (launches) *launches = ctx->last_steps_launches;
    if (!ctx->last_steps_launches) return OED_OK;
    cudaError_t e = cudaEventElapsedTime(ms, ctx->ev_steps[0], ctx->ev_steps[1]);
    if (e != cudaSuccess) {
        const_cast<oed_ctx *>(ctx)->err = std::string("oed_last_step_time: ") + cudaGetErrorString(e);
        return OED_ECUDA;
    }
    return OED_OK;
}

int oed_autotune(oed_ctx *ctx, int nsolve, void *stream)
{
    if (!ctx || nsolve < 1 || nsolve > ctx->max_solves)
        return set_err(ctx, OED_EINVAL, "oed_autotune: nsolve must be in 1..max_solves");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // streaming kernel: enough launches for ~20 ms per candidate, at least 4
    const double cells = (double)nsolve * ctx->g.nx * ctx->g.nz;
    int nrep = (int)(2e9 / (cells * ctx->elem * 6 + 1.0));
    nrep = nrep < 4 ? 4 : (nrep > 200 ? 200 : nrep);
    const StepTuning keep = ctx->tune;
    StepTuning best = keep;
    float best_ms = 1e30f;   // per time step
    launch_fill_probe(ctx, nsolve, st);   // the probes' scratch levels hold non-zero data
    auto fail = [&](cudaError_t e) {
        ctx->tune = keep;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_err(ctx, e, "oed_autotune");
    };
    const int zs_list[] = {2, 4, 8};
    const int wz_list[] = {1, 2, 4, 8};
    for (int zs : zs_list)
        for (int wz : wz_list) {
            ctx->tune = StepTuning{zs, wz, 0};
            launch_step_probe(ctx, nsolve, 2, st, e0, e1);   // warm
            launch_step_probe(ctx, nsolve, nrep, st, e0, e1);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) return fail(e);
            ms /= nrep;
            if (ms < best_ms) {
                best_ms = ms;
                best = ctx->tune;
            }
        }
    // TMA streaming kernel (FP32)
    if (tma_supported(ctx) && tma_prepare(ctx) > 0) {
        ctx->tune = StepTuning{best.zs, best.wz, -1};
        // at least 16 steps: a persistent kernel's few first passes fill its copy ring
        const int probe = std::min(ctx->g.nsteps, std::max(nrep, 16));
        cudaError_t e = launch_steps_tma(ctx, nsolve, st, e0, e1, 2);   // warm
        if (e == cudaSuccess) e = launch_steps_tma(ctx, nsolve, st, e0, e1, probe);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return fail(e);
        ms /= probe;
        if (ms < best_ms) {
            best_ms = ms;
            best = ctx->tune;
        }
    }
    // two-step TMA streaming kernel (FP32 grids that do not fit on chip).  It is taken
    // whenever it runs: short probes time it well below its rate in a real time loop
    // (801x401, 1792 solves: 211 Gcell-upd/s in a 16- or 64-step probe, on zero, random
    // or smooth data alike, against 304 in a 1200-step solve, where the one-step kernel
    // probes and runs at 230), so the probe only checks that it launches.
    if (ctx->d_u2 && tma_supported(ctx) && tma_prepare(ctx) > 0 && tma2_prepare(ctx) > 0) {
        ctx->tune = StepTuning{best.zs, best.wz, -2};
        int probe = std::min(ctx->g.nsteps, std::max(nrep, 16));
        probe = probe < 4 ? probe : probe / 2 * 2;
        const float *last = nullptr;
        cudaError_t e = launch_steps_tma2(ctx, nsolve, st, e0, e1, 2, &last);   // warm
        if (e == cudaSuccess) e = launch_steps_tma2(ctx, nsolve, st, e0, e1, probe, &last);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return fail(e);
        ms /= probe;
        best_ms = ms;
        best = ctx->tune;
    }
    // cluster-resident kernel (FP32 grids whose two levels fit in 1..8 CTAs)
    const int cmin = resident_cluster_size(ctx);
    if (cmin > 0) {
        const int probe_steps = ctx->g.nsteps < 64 ? ctx->g.nsteps : 64;
        for (int C = cmin; C <= 8; C++) {
            if (resident_max_active_clusters(ctx, C) < 1) continue;
            ctx->tune = StepTuning{best.zs, best.wz, C};
            cudaError_t e = launch_resident(ctx, C, nsolve, st, e0, e1, probe_steps);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) return fail(e);
            ms /= probe_steps;
            if (ms < best_ms) {
                best_ms = ms;
                best = ctx->tune;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune = best;
    drop_graphs(ctx);   // captured loops used the previous shape
    return OED_OK;
}

int oed_wait_selftest(oed_ctx *ctx, double seconds, void *stream)
{
    if (!ctx) return OED_EINVAL;
    if (!(seconds > 0.0) || seconds > 2.0)
        return set_err(ctx, OED_EINVAL, "oed_wait_selftest: seconds must be in (0, 2]");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_wait_selftest(ctx, (unsigned long long)(seconds * 1e9), st);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "oed_wait_selftest");
    return flag ? set_err(ctx, OED_ETIMEOUT, "oed_wait_selftest: the bounded wait expired as intended")
                : set_err(ctx, OED_ECUDA, "oed_wait_selftest: the wait ended without an arrival");
}

int oed_get_tuning(const oed_ctx *ctx, int *cluster_size, int *rows_per_thread, int *warps_per_block)
{
    if (!ctx) return OED_EINVAL;
    if (cluster_size) *cluster_size = ctx->tune.C;
    if (rows_per_thread) *rows_per_thread = ctx->tune.zs;
    if (warps_per_block) *warps_per_block = ctx->tune.wz;
    return OED_OK;
}

int oed_set_tuning(oed_ctx *ctx, int cluster_size, int rows_per_thread, int warps_per_block)
{
    if (!ctx) return OED_EINVAL;
    if ((rows_per_thread != 2 && rows_per_thread != 4 && rows_per_thread != 8) ||
        (warps_per_block != 1 && warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8))
        return set_err(ctx, OED_EINVAL, "oed_set_tuning: rows 2/4/8, warps 1/2/4/8");
    if (cluster_size == -1) {
        if (!tma_supported(ctx) || tma_prepare(ctx) < 1)
            return set_err(ctx, OED_EINVAL, "oed_set_tuning: the TMA kernel needs FP32");
    } else if (cluster_size == -2) {
        if (!ctx->d_u2 || !tma_supported(ctx) || tma_prepare(ctx) < 1 || tma2_prepare(ctx) < 1)
            return set_err(ctx, OED_EINVAL,
                           "oed_set_tuning: the two-step TMA kernel needs FP32 and a grid that does not fit on chip");
    } else if (cluster_size != 0) {
        const int cmin = resident_cluster_size(ctx);
        if (cmin == 0 || cluster_size < cmin || cluster_size > 8 ||
            resident_max_active_clusters(ctx, cluster_size) < 1)
            return set_err(ctx, OED_EINVAL, "oed_set_tuning: the grid does not fit that cluster");
    }
    ctx->tune = StepTuning{rows_per_thread, warps_per_block, cluster_size};
    drop_graphs(ctx);
    return OED_OK;
}

int oed_set_jacobian(oed_ctx *ctx, int mode)
{
    if (!ctx) return OED_EINVAL;
    if (mode != OED_JAC_PAIRS && mode != OED_JAC_DIFFERENCE && mode != OED_JAC_SENSITIVITY)
        return set_err(ctx, OED_EINVAL, "oed_set_jacobian: unknown Jacobian form");
    if (mode == OED_JAC_SENSITIVITY && ctx->stf != OED_STF_GAUSS)
        return set_err(ctx, OED_EINVAL, "oed_set_jacobian: sensitivity solves need the Gaussian time function");
    ctx->jac_mode = mode;
    return OED_OK;
}

int oed_get_jacobian(const oed_ctx *ctx)
{
    return ctx ? ctx->jac_mode : -1;
}

int oed_resident_min_cluster(const oed_ctx *ctx)
{
    return ctx ? resident_cluster_size(ctx) : 0;
}

int oed_chunk_nodes(const oed_ctx *ctx)
{
    return ctx ? std::max(1, ctx->max_solves / solves_per_node(ctx)) : 0;
}

int oed_forward(oed_ctx *ctx, const double *theta, int n, double *g, void *stream)
{
    if (!ctx) return OED_EINVAL;
    if (n < 0 || (n > 0 && (!theta || !g))) return set_err(ctx, OED_EINVAL, "oed_forward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)ctx->g.nlev * ctx->g.nrec * 2;
    NvtxRange r("oed_forward");
    for (int off = 0; off < n; off += ctx->max_solves) {
        const int nb = std::min(ctx->max_solves, n - off);
        launch_sources(ctx, theta + (size_t)off * kNT, nb, 1, nullptr, st);
        int rc = run_steps(ctx, nb, st);
        if (rc) return rc;
        launch_trace_to_f64(ctx, nb, g + (size_t)off * per, st);
    }
    return cuda_err(ctx, cudaGetLastError(), "oed_forward");
}

int oed_hessian(oed_ctx *ctx, const double *theta, int n, const double *lo, const double *hi,
                double rel_step, double sigma, const int *win_levels, int nwin, double *H,
                double *H_rec, int *status, void *stream)
{
    if (!ctx) return OED_EINVAL;
    if (n < 0 || (n > 0 && (!theta || !H)) || !lo || !hi)
        return set_err(ctx, OED_EINVAL, "oed_hessian: bad pointer arguments");
    if (!(rel_step > 0) || !(sigma > 0) || !std::isfinite(rel_step) || !std::isfinite(sigma))
        return set_err(ctx, OED_EINVAL, "oed_hessian: rel_step and sigma must be positive");
    if (ctx->g.nrec > kMaxRecHessian)
        return set_err(ctx, OED_EINVAL, "oed_hessian: at most 256 receivers");
    if (ctx->max_solves < solves_per_node(ctx))
        return set_err(ctx, OED_EINVAL, "oed_hessian: max_solves below the solves of one node");
    if (nwin < 0 || nwin > 15 || (nwin > 0 && !win_levels) || (H_rec && nwin == 0))
        return set_err(ctx, OED_EINVAL, "oed_hessian: 0..15 windows; H_rec needs windows");
    double inv2d[kNT], d[kNT];
    for (int j = 0; j < kNT; j++) {
        if (!(hi[j] > lo[j])) return set_err(ctx, OED_EINVAL, "oed_hessian: need hi > lo");
        d[j] = rel_step * (hi[j] - lo[j]);
        // sensitivity solves give the Jacobian columns directly
        inv2d[j] = ctx->jac_mode == OED_JAC_SENSITIVITY ? 1.0 : 1.0 / (2.0 * d[j]);
    }
    // segment ends: the window ends (increasing), then all levels
    std::vector<int> seg_end;
    std::vector<int> win_seg(nwin);
    for (int w = 0; w < nwin; w++) {
        const int L = win_levels[w];
        if (L < 1 || L > ctx->g.nlev || (w > 0 && L <= win_levels[w - 1]))
            return set_err(ctx, OED_EINVAL, "oed_hessian: window levels must increase within 1..nsteps+1");
        seg_end.push_back(L);
        win_seg[w] = (int)seg_end.size() - 1;
    }
    if (seg_end.empty() || seg_end.back() != ctx->g.nlev) seg_end.push_back(ctx->g.nlev);
    cudaStream_t st = (cudaStream_t)stream;
    const int chunk = oed_chunk_nodes(ctx);
    NvtxRange all("oed_hessian");
    for (int off = 0; off < n; off += chunk) {
        const int nb = std::min(chunk, n - off);
        const int P = solves_per_node(ctx);
        {
            NvtxRange r("oed_hessian: sources and perturbations");
            launch_sources(ctx, theta + (size_t)off * kNT, nb, P, d, st);
        }
        {
            NvtxRange r("oed_hessian: stencil time steps");
            int rc = run_steps(ctx, nb * P, st);
            if (rc) return rc;
        }
        NvtxRange r("oed_hessian: FD Jacobian and J^T J reduction");
        launch_hessian(ctx, nb, inv2d, sigma, seg_end.data(), (int)seg_end.size(), win_seg.data(),
                       nwin, H + (size_t)off * 49,
                       H_rec ? H_rec + (size_t)off * ctx->g.nrec * nwin * 28 : nullptr,
                       status ? status + off : nullptr, st);
    }
    return cuda_err(ctx, cudaGetLastError(), "oed_hessian");
}

int oed_hessian_ii(oed_ctx *ctx, const double *theta, int n, const double *y, double sigma, double *H,
                   double *grad, int *status, void *stream)
{
    if (!ctx) return OED_EINVAL;
    if (n < 0 || (n > 0 && (!theta || !y || !H)))
        return set_err(ctx, OED_EINVAL, "oed_hessian_ii: bad pointer arguments");
    if (!(sigma > 0) || !std::isfinite(sigma)) return set_err(ctx, OED_EINVAL, "oed_hessian_ii: sigma must be positive");
    if (ctx->g.nrec > kMaxRecHessian) return set_err(ctx, OED_EINVAL, "oed_hessian_ii: at most 256 receivers");
    if (ctx->stf != OED_STF_GAUSS)
        return set_err(ctx, OED_EINVAL, "oed_hessian_ii: the dual solve needs the Gaussian time function");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)ctx->g.nlev * ctx->g.nrec * 2;
    const int chunk = ctx->max_solves;
    const size_t need = ((size_t)chunk * per + (size_t)chunk * 6 * 2 * kPatch * kPatch) * sizeof(double);
    if (ctx->adj_bytes < need) {
        cudaStreamSynchronize(st);
        cudaFree(ctx->d_adj);
        ctx->d_adj = nullptr;
        ctx->adj_bytes = 0;
        if (cudaMalloc((void **)&ctx->d_adj, need) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, OED_ENOMEM, "oed_hessian_ii: no device memory for the dual solve");
        }
        ctx->adj_bytes = need;
    }
    double *w = ctx->d_adj, *acc = ctx->d_adj + (size_t)chunk * per;
    for (int off = 0; off < n; off += chunk) {
        const int nb = std::min(chunk, n - off);
        launch_sources(ctx, theta + (size_t)off * kNT, nb, 1, nullptr, st);   // step 6: primal
        int rc = run_steps(ctx, nb, st);
        if (rc) return rc;
        launch_adjoint(ctx, nb, y + (size_t)off * per, sigma, w, acc, st);     // steps 7-8: dual
        launch_hii_combine(ctx, nb, acc, H + (size_t)off * 49, grad ? grad + (size_t)off * kNT : nullptr,
                           status ? status + off : nullptr, st);              // steps 9-10
    }
    return cuda_err(ctx, cudaGetLastError(), "oed_hessian_ii");
}

int oed_newton_step(const double *H, const double *grad, int n, const double *lo, const double *hi, int param_mask,
                    double *theta, int *status, void *stream)
{
    if (n < 0 || (n > 0 && (!H || !grad || !theta)) || !lo || !hi) return OED_EINVAL;
    if (param_mask < 1 || param_mask > 127) return OED_EINVAL;
    double lh[2 * kNT];
    for (int j = 0; j < kNT; j++) {
        if (!(hi[j] > lo[j])) return OED_EINVAL;
        lh[j] = lo[j];
        lh[kNT + j] = hi[j];
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *d_lh = nullptr;
    if (cudaMallocAsync((void **)&d_lh, sizeof(lh), st) != cudaSuccess) return OED_ENOMEM;
    cudaMemcpyAsync(d_lh, lh, sizeof(lh), cudaMemcpyHostToDevice, st);
    launch_newton(H, grad, n, param_mask, d_lh, theta, status, st);
    cudaFreeAsync(d_lh, st);
    const cudaError_t e = cudaStreamSynchronize(st);   // the host array lh must outlive the copy
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? OED_OK : OED_ECUDA;
}

int oed_hessian_map(oed_ctx *ctx, double *theta, int n, const double *y, const double *lo, const double *hi,
                    double rel_step, double sigma, int param_mask, int iters, double *H, double *grad,
                    int *status, void *stream)
{
    if (ctx && (param_mask < 1 || param_mask > 127))
        return set_err(ctx, OED_EINVAL, "oed_hessian_map: param_mask must be in 1..127");
    if (!ctx) return OED_EINVAL;
    if (ctx->stf != OED_STF_GAUSS)
        return set_err(ctx, OED_EINVAL, "oed_hessian_map: the dual solve needs the Gaussian time function");
    if (iters < 0 || iters > 100) return set_err(ctx, OED_EINVAL, "oed_hessian_map: iters must be in 0..100");
    if (n < 0 || (n > 0 && (!theta || !y || !H || !grad))) return set_err(ctx, OED_EINVAL, "oed_hessian_map: bad pointers");
    for (int it = 0; it <= iters; it++) {
        int rc = oed_hessian(ctx, theta, n, lo, hi, rel_step, sigma, nullptr, 0, H, nullptr, status, stream);
        if (rc) return rc;
        rc = oed_hessian_ii(ctx, theta, n, y, sigma, H, grad, status, stream);
        if (rc) return rc;
        if (it == iters) break;
        rc = oed_newton_step(H, grad, n, lo, hi, param_mask, theta, nullptr, stream);
        if (rc) return set_err(ctx, rc, "oed_hessian_map: Newton step");
    }
    return OED_OK;
}

static double log_volume(const double *lo, const double *hi)
{
    double v = 0.0;
    for (int j = 0; j < kNT; j++) v += std::log(hi[j] - lo[j]);
    return v;
}

int oed_eig_subset(oed_ctx *ctx, const double *H, int n, const double *w, const double *lo,
                   const double *hi, int param_mask, double *eig, double *dkl, int *status, int *n_bad,
                   void *stream)
{
    if (n < 0 || (n > 0 && (!H || !w)) || !eig || !lo || !hi)
        return set_err(ctx, OED_EINVAL, "oed_eig: bad arguments");
    if (param_mask < 1 || param_mask > 127)
        return set_err(ctx, OED_EINVAL, "oed_eig_subset: param_mask must be in 1..127");
    double logvol = 0.0;
    for (int j = 0; j < kNT; j++) {
        if (!(param_mask >> j & 1)) continue;
        if (!(hi[j] > lo[j])) return set_err(ctx, OED_EINVAL, "oed_eig: need hi > lo");
        logvol += log(hi[j] - lo[j]);
    }
    NvtxRange r("oed_eig: scaled Cholesky log-det, D_KL-hat, weighted sum");
    launch_eig(H, n, w, logvol, param_mask, eig, dkl, status, n_bad, (cudaStream_t)stream);
    return cuda_err(ctx, cudaGetLastError(), "oed_eig");
}

int oed_eig(oed_ctx *ctx, const double *H, int n, const double *w, const double *lo,
            const double *hi, double *eig, double *dkl, int *status, int *n_bad, void *stream)
{
    return oed_eig_subset(ctx, H, n, w, lo, hi, 127, eig, dkl, status, n_bad, stream);
}

int oed_eig_designs(oed_ctx *ctx, const double *H_rec, int n, int nrec, int nwin, int win,
                    const unsigned char *mask, int ndesign, const double *w, const double *lo,
                    const double *hi, double *eig, int *n_bad, void *stream)
{
    if (n < 0 || nrec < 1 || nrec > kMaxRecHessian || nwin < 1 || win < 0 || win >= nwin || ndesign < 0 ||
        (n > 0 && (!H_rec || !w)) || (ndesign > 0 && (!mask || !eig)) || !lo || !hi)
        return set_err(ctx, OED_EINVAL, "oed_eig_designs: bad arguments");
    for (int j = 0; j < kNT; j++)
        if (!(hi[j] > lo[j])) return set_err(ctx, OED_EINVAL, "oed_eig_designs: need hi > lo");
    NvtxRange r("oed_eig_designs: per-design H, scaled Cholesky log-det, weighted sum");
    launch_eig_designs(H_rec, n, nrec, nwin, win, mask, ndesign, w, log_volume(lo, hi), eig, n_bad,
                       (cudaStream_t)stream);
    return cuda_err(ctx, cudaGetLastError(), "oed_eig_designs");
}

int oed_nodes_mc(const double *u, int M, const double *lo, const double *hi, double *theta,
                 double *w, void *stream)
{
    if (M < 0 || (M > 0 && (!u || !theta || !w)) || !lo || !hi) return OED_EINVAL;
    launch_nodes_mc(u, M, lo, hi, theta, w, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? OED_OK : OED_ECUDA;
}

int oed_eig_host(oed_ctx *ctx, const double *theta, const double *w, int n, const double *lo,
                 const double *hi, double rel_step, double sigma, double *eig, double *dkl,
                 int *n_bad)
{
    if (!ctx) return OED_EINVAL;
    if (n < 1 || !theta || !w || !eig || !lo || !hi)
        return set_err(ctx, OED_EINVAL, "oed_eig_host: bad arguments");
    cudaStream_t st = ctx->own_stream;
    if (n > ctx->h_stage_cap) {
        cudaFree(ctx->h_stage_theta);
        cudaFree(ctx->h_stage_w);
        cudaFree(ctx->h_stage_H);
        cudaFree(ctx->h_stage_dkl);
        cudaFree(ctx->h_stage_eig);
        cudaFree(ctx->h_stage_bad);
        ctx->h_stage_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->h_stage_theta, sizeof(double) * kNT * n);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_stage_w, sizeof(double) * n);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_stage_H, sizeof(double) * 49 * n);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_stage_dkl, sizeof(double) * n);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_stage_eig, sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_stage_bad, sizeof(int));
        if (e != cudaSuccess) return cuda_err(ctx, e, "oed_eig_host staging");
        ctx->h_stage_cap = n;
    }
    cudaMemcpyAsync(ctx->h_stage_theta, theta, sizeof(double) * kNT * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ctx->h_stage_w, w, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    int rc = oed_hessian(ctx, ctx->h_stage_theta, n, lo, hi, rel_step, sigma, nullptr, 0,
                         ctx->h_stage_H, nullptr, nullptr, st);
    if (rc) return rc;
    rc = oed_eig(ctx, ctx->h_stage_H, n, ctx->h_stage_w, lo, hi, ctx->h_stage_eig,
                 dkl ? ctx->h_stage_dkl : nullptr, nullptr, ctx->h_stage_bad, st);
    if (rc) return rc;
    cudaMemcpyAsync(eig, ctx->h_stage_eig, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (dkl) cudaMemcpyAsync(dkl, ctx->h_stage_dkl, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (n_bad) cudaMemcpyAsync(n_bad, ctx->h_stage_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    return cuda_err(ctx, cudaStreamSynchronize(st), "oed_eig_host");
}

}  // extern "C"
