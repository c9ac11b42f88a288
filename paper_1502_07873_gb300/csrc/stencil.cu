// Batched leap-frog time stepping of the 2-D elastic wave equation
// (Sec. 3.3.1: Eqs. interior_disc, absorbing_disc, full_discrete, Full_Disc).
//
// One launch advances every solve of the batch by one step:
//   interior and surface nodes:  u^{m+1} = 2u^m - u^{m-1} + dt^2/nu (A_h u^m + f^m)
//   absorbing nodes (sides, bottom; first-order Clayton-Engquist, forward in time,
//   upwind in space):            u^{m+1} = u^m + c dt/h (u_inward^m - u^m)
// with A_h the second-order operator built from D+, D-, D0 and a summation-by-parts
// closure on the free surface, and f^m = S(t_m) M grad(delta) on the 7x7 source patch.
//
// Memory layout: u[solve][component][z][xp] with xp a multiple of 32, so every warp
// reads and writes whole 128-byte lines.  u^{m+1} overwrites u^{m-1} in place (each
// node reads only its own u^{m-1}), so a solve needs two level buffers.
// Each thread owns one column i and ZS consecutive rows.  It issues all of its
// loads first (rows j-1 .. j+ZS of u^m at columns i-1, i, i+1, both components,
// and its ZS values of u^{m-1}), so each thread keeps ~8 ZS independent loads in
// flight, then computes and stores its ZS nodes.  Horizontal neighbours are L1
// hits and the two halo rows of a segment are L2 hits, so HBM traffic is the
// algorithmic minimum: read u^m and u^{m-1}, write u^{m+1}, two components each
// (24 B per cell-update in FP32).
//
// The same launch gathers the receiver samples of level m from its input u^m
// (Eq. forward_model), so the seismograms need no extra pass over the field.
#include "stencil_cell.cuh"

namespace oed {

template <typename real>
struct StepArgs {
    const real *cur;               // u^m
    real *nxt;                     // u^{m-1} in, u^{m+1} out
    const FacCoef<real> *fac;      // [nz]
    const SourceDesc<real> *src;   // [nsolve]
    const real *stf;               // [nsolve][nsteps]
    real *trace;                   // [nsolve][nlev][nrec][2]
    const int *rec;                // [nrec]
    Geometry g;
    int m;
};

template <typename real>
__device__ __forceinline__ void load3(const real *__restrict__ p, int im, int i, int ip, real *v)
{
    v[0] = __ldg(p + im);
    v[1] = __ldg(p + i);
    v[2] = __ldg(p + ip);
}

template <typename real, int ZS>
__global__ void __launch_bounds__(256) k_step(StepArgs<real> a)
{
    const Geometry &g = a.g;
    const int s = blockIdx.z;
    const size_t base = (size_t)s * g.solve_stride;
    const real *__restrict__ cx = a.cur + base;
    const real *__restrict__ cz = cx + g.comp_stride;

    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // receiver samples of level m (the input field)
        const int t = threadIdx.y * blockDim.x + threadIdx.x;
        real *tr = a.trace + ((size_t)s * g.nlev + a.m) * g.nrec * 2;
        for (int q = t; q < 2 * g.nrec; q += blockDim.x * blockDim.y)
            tr[q] = (q & 1 ? cz : cx)[a.rec[q >> 1]];
    }

    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int jb = (blockIdx.y * blockDim.y + threadIdx.y) * ZS;
    if (i >= g.nx || jb >= g.nz) return;

    real *__restrict__ px = a.nxt + base;
    real *__restrict__ pz = px + g.comp_stride;
    const int im = i > 0 ? i - 1 : 0;
    const int ip = i < g.nx - 1 ? i + 1 : g.nx - 1;
    const int side = (i == 0) ? 1 : ((i == g.nx - 1) ? 2 : 0);
    const int jlast = g.nz - 1;

    // Issue every load of this thread before any arithmetic: rows jb-1 .. jb+ZS of
    // u^m (three columns, two components) and rows jb .. jb+ZS-1 of u^{m-1}.  Rows
    // outside the grid are clamped (their values are never used).
    real X[ZS + 2][3], Z[ZS + 2][3], XM[ZS], ZM[ZS];
#pragma unroll
    for (int k = 0; k < ZS + 2; k++) {
        int j = jb - 1 + k;
        j = j < 0 ? 0 : (j > jlast ? jlast : j);
        const size_t o = (size_t)j * g.xp;
        load3(cx + o, im, i, ip, X[k]);
        load3(cz + o, im, i, ip, Z[k]);
    }
#pragma unroll
    for (int k = 0; k < ZS; k++) {
        const int j = jb + k < jlast ? jb + k : jlast;
        const size_t o = (size_t)j * g.xp + i;
        XM[k] = __ldcs(px + o);   // read once, never reused: streaming
        ZM[k] = __ldcs(pz + o);
    }
    const int si = i - a.src[s].i0;
    const int sj = a.src[s].j0;
    const bool scol = (unsigned)si < (unsigned)kPatch;
    const real S = scol ? a.stf[(size_t)s * g.nsteps + a.m] : (real)0;

#pragma unroll
    for (int k = 0; k < ZS; k++) {
        const int j = jb + k;
        if (j > jlast) break;
        const FacCoef<real> K = a.fac[j];
        real ux, uz;
        node_update(K, X[k], X[k + 1], X[k + 2], Z[k], Z[k + 1], Z[k + 2], XM[k], ZM[k], side,
                    j == jlast, j == 0, ux, uz);
        const int b = j - sj;
        if (scol && (unsigned)b < (unsigned)kPatch && !side && j != jlast) {
            ux = add_force(ux, S, a.src[s].wx[b * kPatch + si]);
            uz = add_force(uz, S, a.src[s].wz[b * kPatch + si]);
        }
        const size_t o = (size_t)j * g.xp + i;
        __stcs(px + o, ux);   // u^{m+1} is next read one full step later: streaming
        __stcs(pz + o, uz);
    }
}

// Receiver samples of one level (used for the last level after the final step).
template <typename real>
__global__ void k_gather(const real *__restrict__ cur, real *__restrict__ trace,
                         const int *__restrict__ rec, Geometry g, int m, int nsolve)
{
    const int s = blockIdx.x;
    if (s >= nsolve) return;
    const real *cx = cur + (size_t)s * g.solve_stride;
    const real *cz = cx + g.comp_stride;
    real *tr = trace + ((size_t)s * g.nlev + m) * g.nrec * 2;
    for (int q = threadIdx.x; q < 2 * g.nrec; q += blockDim.x)
        tr[q] = (q & 1 ? cz : cx)[rec[q >> 1]];
}

template <typename real, int ZS>
static void launch_steps_zs(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                            cudaEvent_t ev1)
{
    const Geometry &g = ctx->g;
    const int wz = ctx->tune.wz;
    dim3 block(32, wz);
    const int rows_per_block = wz * ZS;
    dim3 grid((g.nx + 31) / 32, (g.nz + rows_per_block - 1) / rows_per_block, nsolve);
    real *u0 = (real *)ctx->d_u0, *u1 = (real *)ctx->d_u1;
    StepArgs<real> a;
    a.fac = (const FacCoef<real> *)ctx->d_fac;
    a.src = (const SourceDesc<real> *)ctx->d_src;
    a.stf = (const real *)ctx->d_stf;
    a.trace = (real *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.g = g;
    // external event records so they become event nodes of a captured graph
    if (ev0) cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal);
    for (int m = 0; m < g.nsteps; m++) {
        a.cur = (m & 1) ? u1 : u0;
        a.nxt = (m & 1) ? u0 : u1;
        a.m = m;
        k_step<real, ZS><<<grid, block, 0, st>>>(a);
    }
    if (ev1) cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    const real *last = (g.nsteps & 1) ? u1 : u0;
    k_gather<real><<<nsolve, 128, 0, st>>>(last, (real *)ctx->d_trace, ctx->d_rec, g, g.nsteps,
                                           nsolve);
}

template <typename real>
static void launch_steps(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                         cudaEvent_t ev1)
{
    switch (ctx->tune.zs) {
    case 2: launch_steps_zs<real, 2>(ctx, nsolve, st, ev0, ev1); break;
    case 8: launch_steps_zs<real, 8>(ctx, nsolve, st, ev0, ev1); break;
    default: launch_steps_zs<real, 4>(ctx, nsolve, st, ev0, ev1); break;
    }
}

// Autotuner probe: nrep stencil launches for nsolve solves with the context's
// current tuning, bracketed by ev0 / ev1 (fields and traces are scratch here).
template <typename real, int ZS>
static void probe_zs(const oed_ctx *ctx, int nsolve, int nrep, cudaStream_t st, cudaEvent_t ev0,
                     cudaEvent_t ev1)
{
    const Geometry &g = ctx->g;
    const int wz = ctx->tune.wz;
    dim3 block(32, wz);
    const int rows_per_block = wz * ZS;
    dim3 grid((g.nx + 31) / 32, (g.nz + rows_per_block - 1) / rows_per_block, nsolve);
    StepArgs<real> a;
    a.fac = (const FacCoef<real> *)ctx->d_fac;
    a.src = (const SourceDesc<real> *)ctx->d_src;
    a.stf = (const real *)ctx->d_stf;
    a.trace = (real *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.g = g;
    cudaEventRecord(ev0, st);
    for (int m = 0; m < nrep; m++) {
        a.cur = (real *)((m & 1) ? ctx->d_u1 : ctx->d_u0);
        a.nxt = (real *)((m & 1) ? ctx->d_u0 : ctx->d_u1);
        a.m = m % g.nsteps;
        k_step<real, ZS><<<grid, block, 0, st>>>(a);
    }
    cudaEventRecord(ev1, st);
}

template <typename real>
static void probe_real(const oed_ctx *ctx, int nsolve, int nrep, cudaStream_t st, cudaEvent_t ev0,
                       cudaEvent_t ev1)
{
    switch (ctx->tune.zs) {
    case 2: probe_zs<real, 2>(ctx, nsolve, nrep, st, ev0, ev1); break;
    case 8: probe_zs<real, 8>(ctx, nsolve, nrep, st, ev0, ev1); break;
    default: probe_zs<real, 4>(ctx, nsolve, nrep, st, ev0, ev1); break;
    }
}

// Fill the level buffers the autotuner's probes run on with a deterministic pattern of
// order-one values (a hash of the index): the probes then time the kernels on data like
// a running solve's rather than on zeros, on which some kernels run at another speed.
template <typename real>
__global__ void k_fill_probe(real *__restrict__ u, size_t n, unsigned salt)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned h = ((unsigned)i ^ salt) * 2654435761u;
        u[i] = (real)((double)(h >> 8) * (1.0 / 16777216.0) - 0.5);
    }
}

void launch_fill_probe(const oed_ctx *ctx, int nsolve, cudaStream_t st)
{
    size_t per = ctx->g.solve_stride;
    if (ctx->d_u2) per = per > paired_stride(ctx->g) ? per : paired_stride(ctx->g);
    const size_t n = (size_t)nsolve * per;
    void *lv[4] = {ctx->d_u0, ctx->d_u1, ctx->d_u2, ctx->d_u3};
    for (int k = 0; k < 4; k++) {
        if (!lv[k]) continue;
        if (ctx->precision == OED_FP64)
            k_fill_probe<double><<<152 * 8, 256, 0, st>>>((double *)lv[k], n, 0x9e3779b9u * (k + 1));
        else
            k_fill_probe<float><<<152 * 8, 256, 0, st>>>((float *)lv[k], n, 0x9e3779b9u * (k + 1));
    }
}

void launch_step_probe(const oed_ctx *ctx, int nsolve, int nrep, cudaStream_t st, cudaEvent_t ev0,
                       cudaEvent_t ev1)
{
    if (ctx->precision == OED_FP64)
        probe_real<double>(ctx, nsolve, nrep, st, ev0, ev1);
    else
        probe_real<float>(ctx, nsolve, nrep, st, ev0, ev1);
}

// Zero both level buffers (u^0 = u^{-1} = 0, Eq. elastic_2nd) and run all steps;
// ev0 / ev1 (may be null) bracket the stencil launches.
cudaError_t launch_forward_steps(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                                 cudaEvent_t ev1)
{
    if (ctx->tune.C == -2) {   // the two-step kernel's paired layout
        const size_t pb = (size_t)nsolve * paired_stride(ctx->g) * sizeof(float);
        cudaMemsetAsync(ctx->d_u0, 0, pb, st);
        cudaMemsetAsync(ctx->d_u1, 0, pb, st);
        cudaMemsetAsync(ctx->d_u2, 0, pb, st);
        cudaMemsetAsync(ctx->d_u3, 0, pb, st);
        const float *last = nullptr;
        const cudaError_t e = launch_steps_tma2(ctx, nsolve, st, ev0, ev1, 0, &last);
        if (e != cudaSuccess) return e;
        launch_tma2_gather(ctx, nsolve, last, ctx->g.nsteps, st);
        return cudaGetLastError();
    }
    const size_t bytes = (size_t)nsolve * ctx->g.solve_stride * ctx->elem;
    cudaMemsetAsync(ctx->d_u0, 0, bytes, st);
    cudaMemsetAsync(ctx->d_u1, 0, bytes, st);
    if (ctx->tune.C == -1) {
        const cudaError_t e = launch_steps_tma(ctx, nsolve, st, ev0, ev1, 0);
        if (e != cudaSuccess) return e;
        const float *last = (const float *)((ctx->g.nsteps & 1) ? ctx->d_u1 : ctx->d_u0);
        k_gather<float><<<nsolve, 128, 0, st>>>(last, (float *)ctx->d_trace, ctx->d_rec, ctx->g,
                                                ctx->g.nsteps, nsolve);
        return cudaGetLastError();
    }
    if (ctx->precision == OED_FP64)
        launch_steps<double>(ctx, nsolve, st, ev0, ev1);
    else
        launch_steps<float>(ctx, nsolve, st, ev0, ev1);
    return cudaGetLastError();
}

template <typename real>
__global__ void k_trace_f64(const real *__restrict__ trace, const SourceDesc<real> *__restrict__ src,
                            Geometry g, int nsolve, double *__restrict__ out)
{
    const size_t per = (size_t)g.nlev * g.nrec * 2;
    const size_t n = per * nsolve;
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(k / per);
        out[k] = src[s].ok ? (double)trace[k] : nan;
    }
}

void launch_trace_to_f64(const oed_ctx *ctx, int nsolve, double *g, cudaStream_t st)
{
    const size_t n = (size_t)ctx->g.nlev * ctx->g.nrec * 2 * nsolve;
    const int blocks = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    if (ctx->precision == OED_FP64)
        k_trace_f64<double><<<blocks, 256, 0, st>>>((const double *)ctx->d_trace,
                                                    (const SourceDesc<double> *)ctx->d_src,
                                                    ctx->g, nsolve, g);
    else
        k_trace_f64<float><<<blocks, 256, 0, st>>>((const float *)ctx->d_trace,
                                                   (const SourceDesc<float> *)ctx->d_src, ctx->g,
                                                   nsolve, g);
}

}  // namespace oed
