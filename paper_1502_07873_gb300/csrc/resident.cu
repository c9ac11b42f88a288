// Cluster-resident time stepping: one thread-block cluster integrates one solve
// through all of its time steps with the wavefield held in distributed shared
// memory (Sec. 3.3.1, Eq. Full_Disc; the node update is the one of the streaming
// kernel, stencil_cell.cuh).
//
// CTA r of a cluster of C owns rows [r R, min((r+1) R, nz)) of the grid, both
// components and both time levels, in its shared memory:
//     A_x, A_z, B_x, B_z : [R][xp] floats,   coef : [R] RowCoef
// Level m lives in A (m even) or B (m odd); u^{m+1} overwrites u^{m-1} in place.
// The rows just above and below a CTA's slab are read straight from the
// neighbouring CTA's shared memory (mapa + ld.shared::cluster).  One cluster
// barrier (arrive.release / wait.acquire) per step orders the writes of step m
// before the reads of step m+1 and the reads of step m before the overwrites of
// step m+1.  Every thread of every CTA executes the same number of barriers.
// HBM traffic is only the seismogram samples and the source time function: the
// wavefield never leaves the chip, so this kernel is bound by shared-memory
// traffic and FP32 issue, not by HBM.
#include "stencil_cell.cuh"

namespace oed {

struct ResArgs {
    const RowCoef<float> *rows;    // [nz]
    const SourceDesc<float> *src;  // [nsolve]
    const float *stf;              // [nsolve][nsteps]
    float *trace;                  // [nsolve][nlev][nrec][2]
    const int *rec;                // [nrec]
    Geometry g;
    int R;                         // rows per CTA
    int nseg;                      // row segments per column (blockDim.y)
    int rps;                       // rows per segment
};

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// shared::cta address of a local pointer, and its image in CTA `rank` of the cluster
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned remote_addr(unsigned local, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

__device__ __forceinline__ float ld_cluster(unsigned addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// three horizontal neighbours of row `l` (local index, may be -1 or nrows) of one
// component buffer; rows outside the slab come from the neighbouring CTA
__device__ __forceinline__ void load_row(const float *buf, int l, int nrows, int Rfull, int xp, int im,
                                         int i, int ip, unsigned rank, float *v)
{
    if (l >= 0 && l < nrows) {
        const float *p = buf + l * xp;
        v[0] = p[im];
        v[1] = p[i];
        v[2] = p[ip];
    } else {
        // l == -1: last row of CTA rank-1 (always a full slab); l == nrows: first row of rank+1
        const int lr = (l < 0) ? Rfull - 1 : 0;
        const unsigned nb = (l < 0) ? rank - 1 : rank + 1;
        const unsigned base = remote_addr(smem_addr(buf + lr * xp), nb);
        v[0] = ld_cluster(base + 4u * im);
        v[1] = ld_cluster(base + 4u * i);
        v[2] = ld_cluster(base + 4u * ip);
    }
}

__global__ void __launch_bounds__(1024, 1) k_resident(ResArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const Geometry &g = a.g;
    const unsigned rank = cluster_rank();
    const int s = blockIdx.y;
    const int R = a.R, xp = g.xp;
    const int j0 = (int)rank * R;
    const int nrows = max(0, min(R, g.nz - j0));
    float *Ax = sm, *Az = sm + R * xp, *Bx = sm + 2 * R * xp, *Bz = sm + 3 * R * xp;
    RowCoef<float> *coef = reinterpret_cast<RowCoef<float> *>(sm + 4 * R * xp);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;

    for (int k = tid; k < 4 * R * xp; k += nthr) sm[k] = 0.0f;   // u^0 = u^{-1} = 0
    for (int k = tid; k < nrows; k += nthr) coef[k] = a.rows[j0 + k];

    const int i = threadIdx.x + 32 * (threadIdx.y % ((g.nx + 31) / 32));
    const int seg = threadIdx.y / ((g.nx + 31) / 32);
    const bool active = i < g.nx && seg < a.nseg;
    const int im = i > 0 ? i - 1 : 0;
    const int ip = i < g.nx - 1 ? i + 1 : g.nx - 1;
    const int side = (i == 0) ? 1 : ((i == g.nx - 1) ? 2 : 0);
    const int l0 = seg * a.rps;
    const int l1 = min(l0 + a.rps, nrows);
    const SourceDesc<float> *sd = a.src + s;
    const int si = i - sd->i0;
    const int sj = sd->j0;
    const bool scol = (unsigned)si < 6u;
    const float *stf = a.stf + (size_t)s * g.nsteps;
    float *trace = a.trace + (size_t)s * g.nlev * g.nrec * 2;
    cluster_barrier();

    for (int m = 0; m < g.nsteps; m++) {
        const float *cx = (m & 1) ? Bx : Ax, *cz = (m & 1) ? Bz : Az;
        float *nx_ = (m & 1) ? Ax : Bx, *nz_ = (m & 1) ? Az : Bz;
        if (rank == 0)
            for (int q = tid; q < 2 * g.nrec; q += nthr)
                trace[(size_t)m * g.nrec * 2 + q] = (q & 1 ? cz : cx)[a.rec[q >> 1]];
        if (active && l0 < l1) {
            const float S = scol ? stf[m] : 0.0f;
            float xn[3], xc[3], xs[3], zn[3], zc[3], zs[3];
            // j - 1 of the first row: for the surface row (j = 0) it is never used
            const int ln = (j0 + l0 == 0) ? l0 : l0 - 1;
            load_row(cx, ln, nrows, R, xp, im, i, ip, rank, xn);
            load_row(cz, ln, nrows, R, xp, im, i, ip, rank, zn);
            load_row(cx, l0, nrows, R, xp, im, i, ip, rank, xc);
            load_row(cz, l0, nrows, R, xp, im, i, ip, rank, zc);
            for (int l = l0; l < l1; l++) {
                const int j = j0 + l;
                // j + 1 of the bottom row is never used
                const int ls = (j == g.nz - 1) ? l : l + 1;
                load_row(cx, ls, nrows, R, xp, im, i, ip, rank, xs);
                load_row(cz, ls, nrows, R, xp, im, i, ip, rank, zs);
                const int o = l * xp + i;
                const int b = j - sj;
                float fx = 0.0f, fz = 0.0f;
                if (scol && (unsigned)b < 6u) {
                    fx = S * sd->wx[b * 6 + si];
                    fz = S * sd->wz[b * 6 + si];
                }
                const RowCoef<float> Rc = coef[l];   // four 16-byte broadcast loads
                float ux, uz;
                cell_update(Rc, xn, xc, xs, zn, zc, zs, nx_[o], nz_[o], side, j == g.nz - 1, j == 0,
                            fx, fz, ux, uz);
                nx_[o] = ux;
                nz_[o] = uz;
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    xn[q] = xc[q];
                    xc[q] = xs[q];
                    zn[q] = zc[q];
                    zc[q] = zs[q];
                }
            }
        }
        cluster_barrier();
    }
    if (rank == 0) {
        const float *cx = (g.nsteps & 1) ? Bx : Ax, *cz = (g.nsteps & 1) ? Bz : Az;
        for (int q = tid; q < 2 * g.nrec; q += nthr)
            trace[(size_t)g.nsteps * g.nrec * 2 + q] = (q & 1 ? cz : cx)[a.rec[q >> 1]];
    }
}

// Shape of the resident launch for a grid: cluster size C (1..8) and rows per CTA,
// or C = 0 when the two levels do not fit in C CTAs of shared memory.
struct ResShape {
    int C, R, nseg, rps, threads_x, threads_y;
    size_t smem;
};

static ResShape resident_shape(const Geometry &g, int C)
{
    ResShape r{};
    const int ncolw = (g.nx + 31) / 32;
    if (ncolw > 32 || C < 1 || C > 8) return r;
    const int R = (g.nz + C - 1) / C;
    if ((C - 1) * R >= g.nz) return r;   // a CTA would own no rows
    const size_t smem = (size_t)4 * R * g.xp * sizeof(float) + (size_t)R * sizeof(RowCoef<float>);
    if (smem > 227 * 1024) return r;
    int nseg = 32 / ncolw;
    if (nseg < 1) nseg = 1;
    if (nseg > R) nseg = R;
    r.C = C;
    r.R = R;
    r.nseg = nseg;
    r.rps = (R + nseg - 1) / nseg;
    r.threads_x = 32;
    r.threads_y = ncolw * nseg;
    r.smem = smem;
    return r;
}

// Smallest cluster that holds the grid, or 0 if none does (or the context is FP64).
int resident_cluster_size(const oed_ctx *ctx)
{
    if (ctx->precision != OED_FP32) return 0;
    for (int C = 1; C <= 8; C++)
        if (resident_shape(ctx->g, C).C) return C;
    return 0;
}

int resident_max_active_clusters(const oed_ctx *ctx, int C)
{
    const ResShape r = resident_shape(ctx->g, C);
    if (!r.C) return 0;
    cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(r.C, 1, 1);
    cfg.blockDim = dim3(r.threads_x, r.threads_y, 1);
    cfg.dynamicSmemBytes = r.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = r.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_resident, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// All nsteps steps of nsolve solves in one launch (grid: C CTAs per solve).
cudaError_t launch_resident(const oed_ctx *ctx, int C, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                            cudaEvent_t ev1, int nsteps_override)
{
    const ResShape r = resident_shape(ctx->g, C);
    if (!r.C) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);
    ResArgs a;
    a.rows = (const RowCoef<float> *)ctx->d_rows;
    a.src = (const SourceDesc<float> *)ctx->d_src;
    a.stf = (const float *)ctx->d_stf;
    a.trace = (float *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.g = ctx->g;
    if (nsteps_override > 0 && nsteps_override < a.g.nsteps) a.g.nsteps = nsteps_override;
    a.R = r.R;
    a.nseg = r.nseg;
    a.rps = r.rps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(r.C, nsolve, 1);
    cfg.blockDim = dim3(r.threads_x, r.threads_y, 1);
    cfg.dynamicSmemBytes = r.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = r.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (ev0) cudaEventRecord(ev0, st);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_resident, a);
    if (ev1) cudaEventRecord(ev1, st);
    return e;
}

}  // namespace oed
