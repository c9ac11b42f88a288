// The dual (adjoint) problem of Eq. Dual_problems for Alg. 1 steps 6-10: the
// transpose of the discrete scheme, run backwards in time from receiver weights.
//
// For J = sum_m sum_{r,c} w^m_{r,c} g^m_{r,c} (w = C^-1 r, the data-side derivative
// of the cost) the derivative of J with respect to every value of the forcing is
// obtained from
//   lambda^m = R^T w^m + B^T lambda^{m+1} + E^T lambda^{m+2},   m = nsteps .. 1,
//   lambda^{nsteps+1} = lambda^{nsteps+2} = 0,   dJ/d(S W)^{m-1} = lambda^m,
// where u^{m+1} = B u^m + E u^{m-1} + (forcing) is the node update of
// stencil_cell.cuh (E = -I on interior and surface nodes, 0 on absorbing nodes) and
// R samples the receivers.  B^T is applied in gather form: node j collects, from
// every node i whose update reads u_j, the coefficient of u_j in that update times
// lambda_i, with the coefficients of node i's row (FacCoef).  Interior node i reads
// its 3x3 neighbourhood; the surface row reads its own row in place of the row
// above; an absorbing node reads itself and its inward neighbour.
//
// Like the forward kernels, lambda^m overwrites lambda^{m+2} in place (a node reads
// only its own lambda^{m+2}).  After each step a small kernel per solve adds the
// receiver weights and accumulates, for the source patch, the time sums
//   acc[s][c][node] += lambda^m(node, c) * S_s(t_{m-1}),   s = S, S_t, S_w, S_tt, S_tw, S_ww,
// from which the forcing's first and second parameter derivatives give the cost
// gradient and H_II (source.cu, k_hii_combine).
#include "oed_internal.cuh"

namespace oed {

template <typename real>
struct AdjArgs {
    const real *cur;    // lambda^{m+1}
    real *nxt;          // lambda^{m+2} in, lambda^m out
    const FacCoef<real> *fac;
    Geometry g;
};

template <typename real>
__device__ __forceinline__ bool interior(const Geometry &g, int i, int j)
{
    return i >= 1 && i <= g.nx - 2 && j >= 0 && j <= g.nz - 2;
}

// (B^T lambda)(i, j) for both components plus E^T lambda^{m+2}.
template <typename real>
__global__ void __launch_bounds__(256) k_adjoint_step(AdjArgs<real> a)
{
    const Geometry &g = a.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int s = blockIdx.z;
    if (i >= g.nx || j >= g.nz) return;
    const real *lx = a.cur + (size_t)s * g.solve_stride;
    const real *lz = lx + g.comp_stride;
    real *ox = a.nxt + (size_t)s * g.solve_stride;
    real *oz = ox + g.comp_stride;
    auto LX = [&](int ii, int jj) { return lx[(size_t)jj * g.xp + ii]; };
    auto LZ = [&](int ii, int jj) { return lz[(size_t)jj * g.xp + ii]; };
    const FacCoef<real> *F = a.fac;
    const bool side = (i == 0 || i == g.nx - 1);
    const bool bottom = !side && j == g.nz - 1;
    const bool inner = !side && !bottom;
    real sx = 0, sz = 0;
    // the node's own update
    if (inner) {
        const FacCoef<real> &K = F[j];
        sx = ((real)2 - (real)2 * K.axx - K.axzp + K.naxzm) * LX(i, j);
        sz = ((real)2 - (real)2 * K.azx - K.azzp + K.nazzm) * LZ(i, j);
    } else if (side) {
        sx = ((real)1 - F[j].cp) * LX(i, j);
        sz = ((real)1 - F[j].cs) * LZ(i, j);
    } else {
        sx = ((real)1 - F[g.nz - 1].cs) * LX(i, j);
        sz = ((real)1 - F[g.nz - 1].cp) * LZ(i, j);
    }
    // west / east neighbours on the same row (this node is their east / west)
    if (interior<real>(g, i - 1, j)) {
        sx += F[j].axx * LX(i - 1, j);
        sz += F[j].azx * LZ(i - 1, j);
    }
    if (interior<real>(g, i + 1, j)) {
        sx += F[j].axx * LX(i + 1, j);
        sz += F[j].azx * LZ(i + 1, j);
    }
    // the row above (this node is its south) and the row below (this node is its north)
    if (j >= 1 && interior<real>(g, i, j - 1)) {
        sx += F[j - 1].axzp * LX(i, j - 1);
        sz += F[j - 1].azzp * LZ(i, j - 1);
    }
    if (interior<real>(g, i, j + 1)) {
        sx -= F[j + 1].naxzm * LX(i, j + 1);
        sz -= F[j + 1].nazzm * LZ(i, j + 1);
    }
    // cross terms: u_x(i,j) enters the u_z update of the diagonal neighbours and vice versa
    if (j >= 1) {
        if (interior<real>(g, i - 1, j - 1)) {   // this node is their south-east
            sx += F[j - 1].pz * LZ(i - 1, j - 1);
            sz += F[j - 1].px * LX(i - 1, j - 1);
        }
        if (interior<real>(g, i + 1, j - 1)) {   // south-west
            sx -= F[j - 1].pz * LZ(i + 1, j - 1);
            sz -= F[j - 1].px * LX(i + 1, j - 1);
        }
    }
    if (interior<real>(g, i - 1, j + 1)) {       // north-east of the row below
        sx += F[j + 1].nqz * LZ(i - 1, j + 1);
        sz += F[j + 1].nqx * LX(i - 1, j + 1);
    }
    if (interior<real>(g, i + 1, j + 1)) {       // north-west
        sx -= F[j + 1].nqz * LZ(i + 1, j + 1);
        sz -= F[j + 1].nqx * LX(i + 1, j + 1);
    }
    if (j == 0) {   // the surface row's cross terms read its own row: east / west of row 0
        if (interior<real>(g, i - 1, 0)) {
            sx += F[0].nqz * LZ(i - 1, 0);
            sz += F[0].nqx * LX(i - 1, 0);
        }
        if (interior<real>(g, i + 1, 0)) {
            sx -= F[0].nqz * LZ(i + 1, 0);
            sz -= F[0].nqx * LX(i + 1, 0);
        }
    }
    // absorbing nodes whose inward neighbour is this node
    if (i == 1) {
        sx += F[j].cp * LX(0, j);
        sz += F[j].cs * LZ(0, j);
    }
    if (i == g.nx - 2) {
        sx += F[j].cp * LX(g.nx - 1, j);
        sz += F[j].cs * LZ(g.nx - 1, j);
    }
    if (j == g.nz - 2 && i >= 1 && i <= g.nx - 2) {
        sx += F[g.nz - 1].cs * LX(i, g.nz - 1);
        sz += F[g.nz - 1].cp * LZ(i, g.nz - 1);
    }
    const size_t o = (size_t)j * g.xp + i;
    if (inner) {   // E^T lambda^{m+2}
        sx -= ox[o];
        sz -= oz[o];
    }
    ox[o] = sx;
    oz[o] = sz;
}

// S and its first and second derivatives in (t_s, omega_s): tau = t - t_s,
// L = log S, dL/dt_s = w^2 tau, dL/dw = 1/w - w tau^2, d2L/dt_s2 = -w^2,
// d2L/dt_s dw = 2 w tau, d2L/dw2 = -1/w^2 - tau^2, d2S = S (dL dL + d2L).
__device__ void stf_derivs(double t, double ts, double w, double *out)
{
    const double tau = t - ts;
    const double S = w * 0.3989422804014327 * exp(-0.5 * w * w * tau * tau);   // w / sqrt(2 pi)
    const double Lt = w * w * tau, Lw = 1.0 / w - w * tau * tau;
    out[0] = S;
    out[1] = S * Lt;
    out[2] = S * Lw;
    out[3] = S * (Lt * Lt - w * w);
    out[4] = S * (Lt * Lw + 2.0 * w * tau);
    out[5] = S * (Lw * Lw - 1.0 / (w * w) - tau * tau);
}

// One block per solve: add R^T w^m (duplicate receivers summed by the first of them,
// in receiver order), then accumulate the patch's time sums.
template <typename real>
__global__ void __launch_bounds__(128) k_adjoint_post(real *lam, const double *__restrict__ w,
                                                      const int *__restrict__ rec,
                                                      const SourceDesc<real> *__restrict__ src,
                                                      const double *__restrict__ theta, double *acc,
                                                      Geometry g, int m)
{
    const int s = blockIdx.x;
    real *lx = lam + (size_t)s * g.solve_stride;
    real *lz = lx + g.comp_stride;
    const double *wm = w + ((size_t)s * g.nlev + m) * g.nrec * 2;
    for (int q = threadIdx.x; q < 2 * g.nrec; q += blockDim.x) {
        const int r = q >> 1, c = q & 1, node = rec[r];
        bool first = true;
        for (int k = 0; k < r; k++) first = first && rec[k] != node;
        if (!first) continue;
        double v = 0.0;
        for (int k = r; k < g.nrec; k++)
            if (rec[k] == node) v += wm[k * 2 + c];
        real *p = (c ? lz : lx) + node;
        *p = (real)((double)*p + v);
    }
    __syncthreads();
    __shared__ double sd[6];
    const SourceDesc<real> *sdesc = src + s;
    if (!sdesc->ok) return;
    if (threadIdx.x == 0) stf_derivs((m - 1) * g.dt, theta[(size_t)s * kNT + 2], theta[(size_t)s * kNT + 3], sd);
    __syncthreads();
    const int k = threadIdx.x;
    if (k < 2 * kPatch * kPatch) {
        const int c = k / (kPatch * kPatch), ab = k % (kPatch * kPatch);
        const int b = ab / kPatch, a2 = ab % kPatch;
        const int ii = sdesc->i0 + a2, jj = sdesc->j0 + b;
        if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.nz) {
            const double v = (double)(c ? lz : lx)[(size_t)jj * g.xp + ii];
            double *ac = acc + (size_t)s * 6 * 2 * kPatch * kPatch;
#pragma unroll
            for (int t = 0; t < 6; t++) ac[(t * 2 + c) * kPatch * kPatch + ab] += v * sd[t];
        }
    }
}

// w = (y - g) / sigma^2 in FP64 from the traces of the primal solves
template <typename real>
__global__ void k_residual(const real *__restrict__ trace, const double *__restrict__ y, double inv_s2,
                           size_t count, double *__restrict__ w)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x)
        w[k] = (y[k] - (double)trace[k]) * inv_s2;
}

template <typename real>
static void adjoint_impl(const oed_ctx *ctx, int nsolve, const double *y, double sigma, double *w,
                         double *acc, cudaStream_t st)
{
    const Geometry &g = ctx->g;
    const size_t cnt = (size_t)nsolve * g.nlev * g.nrec * 2;
    k_residual<real><<<(int)std::min<size_t>((cnt + 255) / 256, 4096), 256, 0, st>>>(
        (const real *)ctx->d_trace, y, 1.0 / (sigma * sigma), cnt, w);
    const size_t bytes = (size_t)nsolve * g.solve_stride * sizeof(real);
    cudaMemsetAsync(ctx->d_u0, 0, bytes, st);
    cudaMemsetAsync(ctx->d_u1, 0, bytes, st);
    cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)nsolve * 6 * 2 * kPatch * kPatch, st);
    AdjArgs<real> a;
    a.fac = (const FacCoef<real> *)ctx->d_fac;
    a.g = g;
    const dim3 blk(32, 8, 1), grd((g.nx + 31) / 32, (g.nz + 7) / 8, nsolve);
    real *A = (real *)ctx->d_u0, *B = (real *)ctx->d_u1;
    for (int m = g.nsteps; m >= 1; m--) {
        const int k = g.nsteps - m;
        a.cur = (k & 1) ? B : A;   // lambda^{m+1}
        a.nxt = (k & 1) ? A : B;   // lambda^{m+2} -> lambda^m
        k_adjoint_step<real><<<grd, blk, 0, st>>>(a);
        k_adjoint_post<real><<<nsolve, 128, 0, st>>>(a.nxt, w, ctx->d_rec, (const SourceDesc<real> *)ctx->d_src,
                                                     ctx->d_theta, acc, g, m);
    }
}

void launch_adjoint(const oed_ctx *ctx, int nsolve, const double *y, double sigma, double *w, double *acc,
                    cudaStream_t st)
{
    if (ctx->precision == OED_FP64)
        adjoint_impl<double>(ctx, nsolve, y, sigma, w, acc, st);
    else
        adjoint_impl<float>(ctx, nsolve, y, sigma, w, acc, st);
}

}  // namespace oed
