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
// Each thread owns a pair of adjacent columns (64-bit shared loads and stores)
// and marches down a segment of the slab's rows with a 3-row x 4-column register
// window per component; the surface row, the bottom row and the rows whose
// neighbour lives in another CTA are peeled off the main loop, and the source
// term is added after the sweep to the few patch nodes.
// HBM traffic is only the seismogram samples and the source time function: the
// wavefield never leaves the chip, so this kernel is bound by instruction issue
// and shared-memory traffic, not by HBM.
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

// Row access for a thread owning the column pair (c, c+1), c even: the values at
// columns c-1, c, c+1, c+2 of one component of a local row (v[0..3]).
__device__ __forceinline__ void row4_local(const float *row, int c, int cm, int cp2, float *v)
{
    const float2 mid = *reinterpret_cast<const float2 *>(row + c);
    v[0] = row[cm];
    v[1] = mid.x;
    v[2] = mid.y;
    v[3] = row[cp2];
}

// The same for row l of the slab, where l may be -1 (last row of CTA rank-1) or
// nrows (first row of CTA rank+1): those come from the neighbour's shared memory.
__device__ __forceinline__ void row4_any(const float *buf, int l, int nrows, int Rfull, int xp, int c,
                                         int cm, int cp2, unsigned rank, float *v)
{
    if (l >= 0 && l < nrows) {
        row4_local(buf + l * xp, c, cm, cp2, v);
    } else {
        const int lr = (l < 0) ? Rfull - 1 : 0;
        const unsigned nb = (l < 0) ? rank - 1 : rank + 1;
        const unsigned base = remote_addr(smem_addr(buf + lr * xp), nb);
        v[0] = ld_cluster(base + 4u * cm);
        v[1] = ld_cluster(base + 4u * c);
        v[2] = ld_cluster(base + 4u * (c + 1));
        v[3] = ld_cluster(base + 4u * cp2);
    }
}

// Update of the two nodes (c, c+1) of one row from 3x4 windows of u_x and u_z
// (node c uses window columns 0..2, node c+1 columns 1..3).  ux, uz hold u^{m-1}
// on entry and u^{m+1} on exit.  TOP / BOTTOM select the surface closure and the
// absorbing bottom row.
template <bool TOP, bool BOTTOM>
__device__ __forceinline__ void pair_update(const RowCoef<float> &R, const float *xn, const float *xc,
                                            const float *xs, const float *zn, const float *zc,
                                            const float *zs, float2 &ux, float2 &uz, int sideA,
                                            int sideB)
{
    float a, b;
    cell_update(R, xn, xc, xs, zn, zc, zs, ux.x, uz.x, sideA, BOTTOM, TOP, 0.0f, 0.0f, a, b);
    ux.x = a;
    uz.x = b;
    cell_update(R, xn + 1, xc + 1, xs + 1, zn + 1, zc + 1, zs + 1, ux.y, uz.y, sideB, BOTTOM, TOP, 0.0f,
                0.0f, a, b);
    ux.y = a;
    uz.y = b;
}

#define OED_ROTATE()                                                                               \
    _Pragma("unroll") for (int q = 0; q < 4; q++)                                                  \
    {                                                                                              \
        xn[q] = xc[q];                                                                             \
        xc[q] = xs[q];                                                                             \
        zn[q] = zc[q];                                                                             \
        zc[q] = zs[q];                                                                             \
    }

__global__ void __launch_bounds__(768, 1) k_resident(ResArgs a)
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

    // thread -> column pair (c, c+1) and row segment [l0, l1) of the slab
    const int ncolw = (g.nx + 63) / 64;
    const int c = 2 * (threadIdx.x + 32 * (threadIdx.y % ncolw));
    const int seg = threadIdx.y / ncolw;
    const bool active = c < g.nx && seg < a.nseg;
    const int cm = c > 0 ? c - 1 : 0;
    const int cp2 = c + 2 < g.nx ? c + 2 : g.nx - 1;
    const int sideA = (c == 0) ? 1 : ((c == g.nx - 1) ? 2 : 0);
    const int sideB = (c + 1 == g.nx - 1) ? 2 : 0;
    const bool validB = c + 1 < g.nx;
    const int l0 = seg * a.rps;
    const int l1 = min(l0 + a.rps, nrows);
    const bool top = (j0 + l0 == 0);
    const SourceDesc<float> *sd = a.src + s;
    const int sj = sd->j0;
    const int siA = c - sd->i0, siB = c + 1 - sd->i0;
    const bool scolA = (unsigned)siA < (unsigned)kPatch;
    const bool scolB = validB && (unsigned)siB < (unsigned)kPatch;
    const float *stf = a.stf + (size_t)s * g.nsteps;
    float *trace = a.trace + (size_t)s * g.nlev * g.nrec * 2;
    cluster_barrier();

    for (int m = 0; m < g.nsteps; m++) {
        const float *cx = (m & 1) ? Bx : Ax, *cz = (m & 1) ? Bz : Az;
        float *nxb = (m & 1) ? Ax : Bx, *nzb = (m & 1) ? Az : Bz;
        if (rank == 0)
            for (int q = tid; q < 2 * g.nrec; q += nthr)
                trace[(size_t)m * g.nrec * 2 + q] = (q & 1 ? cz : cx)[a.rec[q >> 1]];
        if (active && l0 < l1) {
            float xn[4], xc[4], xs[4], zn[4], zc[4], zs[4];
            // row above the first node (not used on the surface row)
            const int ln = top ? l0 : l0 - 1;
            row4_any(cx, ln, nrows, R, xp, c, cm, cp2, rank, xn);
            row4_any(cz, ln, nrows, R, xp, c, cm, cp2, rank, zn);
            row4_local(cx + l0 * xp, c, cm, cp2, xc);
            row4_local(cz + l0 * xp, c, cm, cp2, zc);
            int l = l0;
            if (top) {   // surface row
                row4_any(cx, l + 1, nrows, R, xp, c, cm, cp2, rank, xs);
                row4_any(cz, l + 1, nrows, R, xp, c, cm, cp2, rank, zs);
                const RowCoef<float> Rc = coef[l];
                float2 *px = reinterpret_cast<float2 *>(nxb + l * xp + c);
                float2 *pz = reinterpret_cast<float2 *>(nzb + l * xp + c);
                float2 ux = *px, uz = *pz;
                pair_update<true, false>(Rc, xn, xc, xs, zn, zc, zs, ux, uz, sideA, sideB);
                *px = ux;
                *pz = uz;
                OED_ROTATE();
                l++;
            }
            // rows whose lower neighbour is a local row and that are not the bottom row:
            // unrolled by three with the three window rows taking turns (no register
            // moves), pointers advanced by one row per step
            const int lstop = min(l1, nrows - 1);
            {
                const float *sx = cx + (l + 1) * xp, *sz = cz + (l + 1) * xp;
                float *ox = nxb + l * xp + c, *oz = nzb + l * xp + c;
                const RowCoef<float> *cf = coef + l;
                auto row = [&](const float *an, const float *ac, float *as, const float *bn,
                               const float *bc, float *bs) {
                    row4_local(sx, c, cm, cp2, as);
                    row4_local(sz, c, cm, cp2, bs);
                    const RowCoef<float> Rc = *cf;
                    float2 ux = *reinterpret_cast<float2 *>(ox), uz = *reinterpret_cast<float2 *>(oz);
                    pair_update<false, false>(Rc, an, ac, as, bn, bc, bs, ux, uz, sideA, sideB);
                    *reinterpret_cast<float2 *>(ox) = ux;
                    *reinterpret_cast<float2 *>(oz) = uz;
                    sx += xp;
                    sz += xp;
                    ox += xp;
                    oz += xp;
                    cf++;
                };
                for (; l + 3 <= lstop; l += 3) {
                    row(xn, xc, xs, zn, zc, zs);   // window (n, c, s)
                    row(xc, xs, xn, zc, zs, zn);   // window (c, s, n): row l+2 lands in n
                    row(xs, xn, xc, zs, zn, zc);   // window (s, n, c): row l+3 lands in c
                }
                // the loop left rows (l-1, l) in (xn, xc) again; up to two more rows
                for (; l < lstop; l++) {
                    row(xn, xc, xs, zn, zc, zs);
                    OED_ROTATE();
                }
            }
            // what is left: a last interior row whose lower neighbour sits in CTA rank+1,
            // or the absorbing bottom row
            for (; l < l1; l++) {
                const RowCoef<float> Rc = coef[l];
                float2 *px = reinterpret_cast<float2 *>(nxb + l * xp + c);
                float2 *pz = reinterpret_cast<float2 *>(nzb + l * xp + c);
                float2 ux = *px, uz = *pz;
                if (j0 + l == g.nz - 1) {
                    pair_update<false, true>(Rc, xn, xc, xc, zn, zc, zc, ux, uz, sideA, sideB);
                } else {
                    row4_any(cx, l + 1, nrows, R, xp, c, cm, cp2, rank, xs);
                    row4_any(cz, l + 1, nrows, R, xp, c, cm, cp2, rank, zs);
                    pair_update<false, false>(Rc, xn, xc, xs, zn, zc, zs, ux, uz, sideA, sideB);
                }
                *px = ux;
                *pz = uz;
                OED_ROTATE();
            }
            // source term: u^{m+1} += dt^2/nu f^m on the patch nodes this thread owns,
            // added last as in the node update of the streaming kernel
            if (scolA || scolB) {
                const float S = stf[m];
                for (int bb = 0; bb < kPatch; bb++) {
                    const int lj = sj + bb - j0;
                    if (lj < l0 || lj >= l1) continue;
                    const int o = lj * xp + c;
                    if (scolA) {
                        nxb[o] += S * sd->wx[bb * kPatch + siA];
                        nzb[o] += S * sd->wz[bb * kPatch + siA];
                    }
                    if (scolB) {
                        nxb[o + 1] += S * sd->wx[bb * kPatch + siB];
                        nzb[o + 1] += S * sd->wz[bb * kPatch + siB];
                    }
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
    const int ncolw = (g.nx + 63) / 64;   // warps of 32 column pairs
    if (ncolw > 24 || C < 1 || C > 8) return r;
    const int R = (g.nz + C - 1) / C;
    if ((C - 1) * R >= g.nz) return r;   // a CTA would own no rows
    const size_t smem = (size_t)4 * R * g.xp * sizeof(float) + (size_t)R * sizeof(RowCoef<float>);
    if (smem > 227 * 1024) return r;
    int nseg = 24 / ncolw;   // at most 768 threads: 85 registers per thread
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

// The kernel's dynamic shared-memory limit is always set to the device's opt-in
// maximum (launches may use less): a fixed value, so concurrent callers with
// different grids never lower it under each other.
static cudaError_t set_smem_limit()
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

int resident_max_active_clusters(const oed_ctx *ctx, int C)
{
    const ResShape r = resident_shape(ctx->g, C);
    if (!r.C) return 0;
    set_smem_limit();
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
    set_smem_limit();
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
