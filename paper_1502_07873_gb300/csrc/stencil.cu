// Batched leap-frog time stepping of the 2-D elastic wave equation
// (Sec. 3.3.1: Eqs. interior_disc, absorbing_disc, full_discrete, Full_Disc).
//
// One launch advances every solve of the batch by one step:
//   interior and surface nodes:  u^{m+1} = 2u^m - u^{m-1} + dt^2/nu (A_h u^m + f^m)
//   absorbing nodes (sides, bottom; first-order Clayton-Engquist, forward in time,
//   upwind in space):            u^{m+1} = u^m + c dt/h (u_inward^m - u^m)
// with A_h the second-order operator built from D+, D-, D0 and a summation-by-parts
// closure on the free surface, and f^m = S(t_m) M grad(delta) on the 6x6 source patch.
//
// Memory layout: u[solve][component][z][xp] with xp a multiple of 32, so every warp
// reads and writes whole 128-byte lines.  u^{m+1} overwrites u^{m-1} in place (each
// node reads only its own u^{m-1}), so a solve needs two level buffers.
// Each thread owns one column i and marches ZS rows downward, keeping a 3x3
// register window of u_x and u_z (rows j-1, j, j+1; columns i-1, i, i+1): every
// value of u^m is fetched from L2/HBM once and re-read from L1 by its two
// horizontal neighbours.  HBM traffic is the algorithmic minimum: read u^m and
// u^{m-1}, write u^{m+1}, two components each (24 B per cell-update in FP32).
//
// The same launch gathers the receiver samples of level m from its input u^m
// (Eq. forward_model), so the seismograms need no extra pass over the field.
#include "oed_internal.cuh"

namespace oed {

template <typename real>
struct StepArgs {
    const real *cur;               // u^m
    real *nxt;                     // u^{m-1} in, u^{m+1} out
    const RowCoef<real> *rows;     // [nz]
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
    const bool left = (i == 0), right = (i == g.nx - 1);

    const int si = i - a.src[s].i0;
    const int sj = a.src[s].j0;
    const bool scol = (unsigned)si < 6u;
    const real S = scol ? a.stf[(size_t)s * g.nsteps + a.m] : (real)0;

    real xn[3], xc[3], xs[3], zn[3], zc[3], zs[3];
    {
        const size_t on = (size_t)(jb > 0 ? jb - 1 : 0) * g.xp;
        const size_t oc = (size_t)jb * g.xp;
        load3(cx + on, im, i, ip, xn);
        load3(cz + on, im, i, ip, zn);
        load3(cx + oc, im, i, ip, xc);
        load3(cz + oc, im, i, ip, zc);
    }
#pragma unroll
    for (int k = 0; k < ZS; k++) {
        const int j = jb + k;
        if (j >= g.nz) break;
        {
            const size_t os = (size_t)(j < g.nz - 1 ? j + 1 : j) * g.xp;
            load3(cx + os, im, i, ip, xs);
            load3(cz + os, im, i, ip, zs);
        }
        const size_t o = (size_t)j * g.xp + i;
        const real uxm = px[o], uzm = pz[o];
        const RowCoef<real> R = a.rows[j];
        real ux, uz;
        if (left || right) {
            const real xi = left ? xc[2] : xc[0];
            const real zi = left ? zc[2] : zc[0];
            ux = xc[1] + R.cp * (xi - xc[1]);
            uz = zc[1] + R.cs * (zi - zc[1]);
        } else if (j == g.nz - 1) {
            ux = xc[1] + R.cs * (xn[1] - xc[1]);
            uz = zc[1] + R.cp * (zn[1] - zc[1]);
        } else {
            real Ax = R.axx * (xc[2] - (real)2 * xc[1] + xc[0]) + R.axzp * (xs[1] - xc[1]);
            real Az = R.azx * (zc[2] - (real)2 * zc[1] + zc[0]) + R.azzp * (zs[1] - zc[1]);
            if (j > 0) {
                Ax += -R.axzm * (xc[1] - xn[1]) + R.lx * ((zs[2] - zn[2]) - (zs[0] - zn[0])) +
                      R.mxp * (zs[2] - zs[0]) - R.mxm * (zn[2] - zn[0]);
                Az += -R.azzm * (zc[1] - zn[1]) + R.mz * ((xs[2] - xn[2]) - (xs[0] - xn[0])) +
                      R.lzp * (xs[2] - xs[0]) - R.lzm * (xn[2] - xn[0]);
            } else {
                Ax += R.lx * ((zs[2] - zc[2]) - (zs[0] - zc[0])) + R.mxm * (zc[2] - zc[0]) +
                      R.mxp * (zs[2] - zs[0]);
                Az += R.mz * ((xs[2] - xc[2]) - (xs[0] - xc[0])) + R.lzm * (xc[2] - xc[0]) +
                      R.lzp * (xs[2] - xs[0]);
            }
            const int b = j - sj;
            if (scol && (unsigned)b < 6u) {
                Ax += S * a.src[s].wx[b * 6 + si];
                Az += S * a.src[s].wz[b * 6 + si];
            }
            ux = (real)2 * xc[1] - uxm + Ax;
            uz = (real)2 * zc[1] - uzm + Az;
        }
        px[o] = ux;
        pz[o] = uz;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            xn[q] = xc[q];
            xc[q] = xs[q];
            zn[q] = zc[q];
            zc[q] = zs[q];
        }
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
    a.rows = (const RowCoef<real> *)ctx->d_rows;
    a.src = (const SourceDesc<real> *)ctx->d_src;
    a.stf = (const real *)ctx->d_stf;
    a.trace = (real *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.g = g;
    if (ev0) cudaEventRecord(ev0, st);
    for (int m = 0; m < g.nsteps; m++) {
        a.cur = (m & 1) ? u1 : u0;
        a.nxt = (m & 1) ? u0 : u1;
        a.m = m;
        k_step<real, ZS><<<grid, block, 0, st>>>(a);
    }
    if (ev1) cudaEventRecord(ev1, st);
    const real *last = (g.nsteps & 1) ? u1 : u0;
    k_gather<real><<<nsolve, 128, 0, st>>>(last, (real *)ctx->d_trace, ctx->d_rec, g, g.nsteps,
                                           nsolve);
}

template <typename real>
static void launch_steps(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                         cudaEvent_t ev1)
{
    switch (ctx->tune.zs) {
    case 4: launch_steps_zs<real, 4>(ctx, nsolve, st, ev0, ev1); break;
    case 16: launch_steps_zs<real, 16>(ctx, nsolve, st, ev0, ev1); break;
    case 32: launch_steps_zs<real, 32>(ctx, nsolve, st, ev0, ev1); break;
    default: launch_steps_zs<real, 8>(ctx, nsolve, st, ev0, ev1); break;
    }
}

// Zero both level buffers (u^0 = u^{-1} = 0, Eq. elastic_2nd) and run all steps;
// ev0 / ev1 (may be null) bracket the stencil launches.
void launch_forward_steps(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                          cudaEvent_t ev1)
{
    const size_t bytes = (size_t)nsolve * ctx->g.solve_stride * ctx->elem;
    cudaMemsetAsync(ctx->d_u0, 0, bytes, st);
    cudaMemsetAsync(ctx->d_u1, 0, bytes, st);
    if (ctx->precision == OED_FP64)
        launch_steps<double>(ctx, nsolve, st, ev0, ev1);
    else
        launch_steps<float>(ctx, nsolve, st, ev0, ev1);
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
