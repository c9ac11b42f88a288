// Cluster-resident time stepping: one thread-block cluster integrates one solve
// through all of its time steps with the wavefield held in distributed shared
// memory (Sec. 3.3.1, Eq. Full_Disc, in the factored form of FacCoef).
//
// CTA r of a cluster of C owns rows [r R, min((r+1) R, nz)) of the grid, both
// components and both time levels, in its shared memory:
//     A_x, A_z, B_x, B_z : [R][sxp] floats,   coef : [R] FacCoef
// Column i of a row sits at offset i + kGhost; the columns -1, nx and nx + 1 are
// zero ghosts, so every thread reads its west and east neighbours at fixed
// offsets.  Level m lives in A (m even) or B (m odd); u^{m+1} overwrites u^{m-1}
// in place.  The rows just above and below a CTA's slab are read straight from the
// neighbouring CTA's shared memory (mapa + ld.shared::cluster).  One cluster
// barrier (arrive.release / wait.acquire) per step orders the writes of step m
// before the reads of step m+1 and the reads of step m before the overwrites of
// step m+1.  Every thread of every CTA executes the same number of barriers.
// Each thread owns a pair of adjacent columns (64-bit shared loads and stores)
// and marches down a segment of the slab's rows.  A row enters the register
// window once, as the south row, where its centre values, west + east sums and
// east - west differences are formed; they serve it again as the centre row and
// as the north row, so a node costs six multiply-adds per component.  The
// surface row, the bottom row and the rows whose neighbour lives in another CTA
// are peeled off the main loop; the absorbing side columns are patched by the
// threads that own them; the source term is added after the sweep to the few
// patch nodes.  HBM traffic is only the seismogram samples and the source time
// function: the wavefield never leaves the chip, so this kernel is bound by
// instruction issue and shared-memory traffic, not by HBM.
#include "stencil_cell.cuh"

namespace oed {

constexpr int kGhost = 2;   // offset of column 0 in a shared row (keeps pairs 8-byte aligned)
// Block size and register budget: registers are split over the SM's four
// schedulers (16 K each), so 20 warps of 96 registers is the most one CTA can hold
// with the row window in registers.
constexpr int kResThreads = 640;
constexpr int kResRegs = 96;

struct ResArgs {
    const FacCoef<float> *fac;     // [nz]
    const SourceDesc<float> *src;  // [nsolve]
    const float *stf;              // [nsolve][nsteps]
    float *trace;                  // [nsolve][nlev][nrec][2]
    const int *rec;                // [nrec]
    Geometry g;
    int R;                         // rows per CTA
    int sxp;                       // shared row stride (floats)
    int npair;                     // column pairs per row, (nx + 1) / 2
    int nseg;                      // row segments per column pair
    int rps;                       // rows per segment
};

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
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

// One grid row as seen by the thread owning columns (c, c+1): per component the
// two centre values, the two (e - c) - (c - w) second differences, the two
// east - west differences (cross terms of the other component) and, once the row
// below is known, the two south differences (row below minus this row).
struct Row2 {
    float xa, xb, za, zb;
    float lxa, lxb, lza, lzb;
    float dxa, dxb, dza, dzb;
    float vxa, vxb, vza, vzb;
};

__device__ __forceinline__ void row_from(float w, float2 m, float e, float &va, float &vb, float &la,
                                         float &lb, float &da, float &db)
{
    va = m.x;
    vb = m.y;
    la = (m.y - m.x) - (m.x - w);
    lb = (e - m.y) - (m.y - m.x);
    da = m.y - w;
    db = e - m.x;
}

// px, pz point at column c of a local row of each component
__device__ __forceinline__ void load_row(const float *px, const float *pz, Row2 &r)
{
    const float2 mx = *reinterpret_cast<const float2 *>(px);
    const float2 mz = *reinterpret_cast<const float2 *>(pz);
    row_from(px[-1], mx, px[2], r.xa, r.xb, r.lxa, r.lxb, r.dxa, r.dxb);
    row_from(pz[-1], mz, pz[2], r.za, r.zb, r.lza, r.lzb, r.dza, r.dzb);
}

// the same row in CTA `nb` of the cluster (local pointers are mapped)
__device__ __forceinline__ void load_row_remote(const float *px, const float *pz, unsigned nb, Row2 &r)
{
    const unsigned bx = remote_addr(smem_addr(px), nb), bz = remote_addr(smem_addr(pz), nb);
    const float2 mx = make_float2(ld_cluster(bx), ld_cluster(bx + 4u));
    const float2 mz = make_float2(ld_cluster(bz), ld_cluster(bz + 4u));
    row_from(ld_cluster(bx - 4u), mx, ld_cluster(bx + 8u), r.xa, r.xb, r.lxa, r.lxb, r.dxa, r.dxb);
    row_from(ld_cluster(bz - 4u), mz, ld_cluster(bz + 8u), r.za, r.zb, r.lza, r.lzb, r.dza, r.dzb);
}

// south differences of row c once its south row s is loaded
__device__ __forceinline__ void south(Row2 &c, const Row2 &s)
{
    c.vxa = s.xa - c.xa;
    c.vxb = s.xb - c.xb;
    c.vza = s.za - c.za;
    c.vzb = s.zb - c.zb;
}

// u^{m+1} of the pair from the rows n, c, s (the node update of stencil_cell.cuh);
// n supplies the north differences (its south ones) and the north cross terms.
// ux, uz hold u^{m-1} on entry.
__device__ __forceinline__ void pair_update(const FacCoef<float> &K, const Row2 &n, const Row2 &c,
                                            const Row2 &s, float2 &ux, float2 &uz)
{
    ux.x = leap(c.xa, ux.x, op_x(K, c.lxa, c.vxa, n.vxa, s.dza, n.dza));
    ux.y = leap(c.xb, ux.y, op_x(K, c.lxb, c.vxb, n.vxb, s.dzb, n.dzb));
    uz.x = leap(c.za, uz.x, op_z(K, c.lza, c.vza, n.vza, s.dxa, n.dxa));
    uz.y = leap(c.zb, uz.y, op_z(K, c.lzb, c.vzb, n.vzb, s.dxb, n.dxb));
}

// Absorbing rows: the bottom row from its north neighbour, then the side columns
// (which take precedence at the corners) from their interior neighbour.  kind:
// bit 0 node c is column 0, bit 1 node c+1 is column nx-1, bit 2 node c is column
// nx-1 (node c+1 is then the ghost and stays zero).
__device__ __forceinline__ void absorbing(float cp, float cs, const Row2 &n, const Row2 &c, bool bottom,
                                          int kind, float2 &ux, float2 &uz)
{
    if (bottom) {
        ux.x = absorb(c.xa, n.xa, cs);
        ux.y = absorb(c.xb, n.xb, cs);
        uz.x = absorb(c.za, n.za, cp);
        uz.y = absorb(c.zb, n.zb, cp);
    }
    if (kind & 1) {
        ux.x = absorb(c.xa, c.xb, cp);
        uz.x = absorb(c.za, c.zb, cs);
    }
    if (kind & 2) {
        ux.y = absorb(c.xb, c.xa, cp);
        uz.y = absorb(c.zb, c.za, cs);
    }
    if (kind & 4) {   // column nx-1: its east - west difference is -west (the ghost east is 0)
        ux.x = absorb(c.xa, -c.dxa, cp);
        uz.x = absorb(c.za, -c.dza, cs);
        ux.y = 0.0f;
        uz.y = 0.0f;
    }
}

__global__ void __maxnreg__(kResRegs) k_resident(ResArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const Geometry &g = a.g;
    const unsigned rank = cluster_rank();
    const int s = blockIdx.y;
    const int R = a.R, sxp = a.sxp;
    const int j0 = (int)rank * R;
    const int nrows = max(0, min(R, g.nz - j0));
    const int lvl = R * sxp;   // floats per component and level
    float *Ax = sm, *Az = sm + lvl, *Bx = sm + 2 * lvl, *Bz = sm + 3 * lvl;
    FacCoef<float> *coef = reinterpret_cast<FacCoef<float> *>(sm + 4 * lvl);
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;

    for (int k = tid; k < lvl; k += nthr) {   // u^0 = u^{-1} = 0, ghosts 0
        Ax[k] = 0.0f;
        Az[k] = 0.0f;
        Bx[k] = 0.0f;
        Bz[k] = 0.0f;
    }
    for (int k = tid; k < nrows; k += nthr) coef[k] = a.fac[j0 + k];

    // thread -> column pair (c, c+1) and row segment [l0, l1) of the slab
    // threads are packed densely over (segment, pair): a warp may straddle two segments
    const int c = 2 * (tid % a.npair);
    const int seg = tid / a.npair;
    const bool active = seg < a.nseg;
    const int kind = (c == 0 ? 1 : 0) | (c + 1 == g.nx - 1 ? 2 : 0) | (c == g.nx - 1 ? 4 : 0);
    const int l0 = seg * a.rps;
    const int l1 = min(l0 + a.rps, nrows);
    const bool top = (j0 + l0 == 0);
    const SourceDesc<float> *sd = a.src + s;
    const int sj = sd->j0;
    const int siA = c - sd->i0, siB = c + 1 - sd->i0;
    const bool scolA = (unsigned)siA < (unsigned)kPatch;
    const bool scolB = c + 1 < g.nx && (unsigned)siB < (unsigned)kPatch;
    const float *stf = a.stf + (size_t)s * g.nsteps;
    float *trace = a.trace + (size_t)s * g.nlev * g.nrec * 2;
    const int col = c + kGhost;
    cluster_barrier();

    for (int m = 0; m < g.nsteps; m++) {
        const float *cx = (m & 1) ? Bx : Ax, *cz = (m & 1) ? Bz : Az;
        float *nxb = (m & 1) ? Ax : Bx, *nzb = (m & 1) ? Az : Bz;
        if (rank == 0)
            for (int q = tid; q < 2 * g.nrec; q += nthr)
                trace[(size_t)m * g.nrec * 2 + q] = (q & 1 ? cz : cx)[a.rec[q >> 1] + kGhost];
        if (active && l0 < l1) {
            Row2 rn, rc, rs;
            int l = l0;
            load_row(cx + l * sxp + col, cz + l * sxp + col, rc);
            if (top) {   // surface row: its "north" terms are the row itself
                if (l + 1 < nrows)
                    load_row(cx + (l + 1) * sxp + col, cz + (l + 1) * sxp + col, rs);
                else   // a one-row slab
                    load_row_remote(cx + col, cz + col, rank + 1, rs);
                south(rc, rs);
                Row2 nt = rc;   // no north differences; cross terms on the row itself
                nt.vxa = nt.vxb = nt.vza = nt.vzb = 0.0f;
                float2 *px = reinterpret_cast<float2 *>(nxb + l * sxp + col);
                float2 *pz = reinterpret_cast<float2 *>(nzb + l * sxp + col);
                float2 ux = *px, uz = *pz;
                const FacCoef<float> K = coef[l];
                pair_update(K, nt, rc, rs, ux, uz);
                if (kind) absorbing(K.cp, K.cs, nt, rc, false, kind, ux, uz);
                *px = ux;
                *pz = uz;
                rn = rc;
                rc = rs;
                l++;
            } else {
                if (l > 0)
                    load_row(cx + (l - 1) * sxp + col, cz + (l - 1) * sxp + col, rn);
                else
                    load_row_remote(cx + (R - 1) * sxp + col, cz + (R - 1) * sxp + col, rank - 1, rn);
                south(rn, rc);
            }
            // rows whose south neighbour is a local row and that are not the bottom row:
            // unrolled by three with the three window rows taking turns
            const int lstop = min(l1, nrows - 1);
            {
                const float *sx = cx + (l + 1) * sxp + col, *sz = cz + (l + 1) * sxp + col;
                float *ox = nxb + l * sxp + col, *oz = nzb + l * sxp + col;
                const FacCoef<float> *cf = coef + l;
                auto row = [&](const Row2 &wn, Row2 &wc, Row2 &ws) {
                    load_row(sx, sz, ws);
                    south(wc, ws);
                    const FacCoef<float> K = *cf;
                    float2 ux = *reinterpret_cast<float2 *>(ox), uz = *reinterpret_cast<float2 *>(oz);
                    pair_update(K, wn, wc, ws, ux, uz);
                    if (kind) absorbing(K.cp, K.cs, wn, wc, false, kind, ux, uz);
                    *reinterpret_cast<float2 *>(ox) = ux;
                    *reinterpret_cast<float2 *>(oz) = uz;
                    sx += sxp;
                    sz += sxp;
                    ox += sxp;
                    oz += sxp;
                    cf++;
                };
                for (; l + 3 <= lstop; l += 3) {
                    row(rn, rc, rs);   // window (n, c, s)
                    row(rc, rs, rn);   // row l+2 lands in rn
                    row(rs, rn, rc);   // row l+3 lands in rc
                }
                for (; l < lstop; l++) {
                    row(rn, rc, rs);
                    rn = rc;
                    rc = rs;
                }
            }
            // what is left: a last interior row whose south neighbour sits in CTA rank+1,
            // or the absorbing bottom row
            for (; l < l1; l++) {
                const FacCoef<float> K = coef[l];
                float2 *px = reinterpret_cast<float2 *>(nxb + l * sxp + col);
                float2 *pz = reinterpret_cast<float2 *>(nzb + l * sxp + col);
                float2 ux = *px, uz = *pz;
                if (j0 + l == g.nz - 1) {
                    absorbing(K.cp, K.cs, rn, rc, true, kind, ux, uz);
                } else {
                    load_row_remote(cx + col, cz + col, rank + 1, rs);
                    south(rc, rs);
                    pair_update(K, rn, rc, rs, ux, uz);
                    if (kind) absorbing(K.cp, K.cs, rn, rc, false, kind, ux, uz);
                }
                *px = ux;
                *pz = uz;
                rn = rc;
                rc = rs;
            }
            // source term: u^{m+1} += dt^2/nu f^m on the patch nodes this thread owns,
            // added last as in the node update of the streaming kernel
            if (scolA || scolB) {
                const float S = stf[m];
                for (int bb = 0; bb < kPatch; bb++) {
                    const int lj = sj + bb - j0;
                    if (lj < l0 || lj >= l1) continue;
                    const int o = lj * sxp + col;
                    if (scolA) {
                        nxb[o] = add_force(nxb[o], S, sd->wx[bb * kPatch + siA]);
                        nzb[o] = add_force(nzb[o], S, sd->wz[bb * kPatch + siA]);
                    }
                    if (scolB) {
                        nxb[o + 1] = add_force(nxb[o + 1], S, sd->wx[bb * kPatch + siB]);
                        nzb[o + 1] = add_force(nzb[o + 1], S, sd->wz[bb * kPatch + siB]);
                    }
                }
            }
        }
        cluster_barrier();
    }
    if (rank == 0) {
        const float *cx = (g.nsteps & 1) ? Bx : Ax, *cz = (g.nsteps & 1) ? Bz : Az;
        for (int q = tid; q < 2 * g.nrec; q += nthr)
            trace[(size_t)g.nsteps * g.nrec * 2 + q] = (q & 1 ? cz : cx)[a.rec[q >> 1] + kGhost];
    }
}

// Shape of the resident launch for a grid: cluster size C (1..8) and rows per CTA,
// or C = 0 when the two levels do not fit in C CTAs of shared memory.
struct ResShape {
    int C, R, sxp, npair, nseg, rps, threads;
    size_t smem;
};

static ResShape resident_shape(const Geometry &g, int C)
{
    ResShape r{};
    const int npair = (g.nx + 1) / 2;
    if (npair > kResThreads || C < 1 || C > 8) return r;
    const int R = (g.nz + C - 1) / C;
    if ((C - 1) * R >= g.nz) return r;   // a CTA would own no rows
    const int sxp = (g.nx + kGhost + 2 + 3) / 4 * 4;   // ghosts at -1, nx, nx + 1
    const size_t smem = (size_t)4 * R * sxp * sizeof(float) + (size_t)R * sizeof(FacCoef<float>);
    if (smem > 227 * 1024) return r;
    int nseg = kResThreads / npair;
    if (nseg > R) nseg = R;
    r.C = C;
    r.R = R;
    r.sxp = sxp;
    r.npair = npair;
    r.nseg = nseg;
    r.rps = (R + nseg - 1) / nseg;
    r.threads = (npair * nseg + 31) / 32 * 32;
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
    cfg.blockDim = dim3(r.threads, 1, 1);
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
    a.fac = (const FacCoef<float> *)ctx->d_fac;
    a.src = (const SourceDesc<float> *)ctx->d_src;
    a.stf = (const float *)ctx->d_stf;
    a.trace = (float *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.g = ctx->g;
    if (nsteps_override > 0 && nsteps_override < a.g.nsteps) a.g.nsteps = nsteps_override;
    a.R = r.R;
    a.sxp = r.sxp;
    a.npair = r.npair;
    a.nseg = r.nseg;
    a.rps = r.rps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(r.C, nsolve, 1);
    cfg.blockDim = dim3(r.threads, 1, 1);
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
