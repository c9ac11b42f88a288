// Cluster-resident time stepping: one thread-block cluster integrates one solve
// through all of its time steps with the wavefield held in distributed shared
// memory (Sec. 3.3.1, Eq. Full_Disc; the node update of stencil_cell.cuh).
//
// CTA r of a cluster of C owns rows [r R, min((r+1) R, nz)) of the grid, both
// components and both time levels, in its shared memory:
//     A, B : [R][npair + 2] float4,   coef : [R] KP (FacCoef in (x, z) pairs),   the solve's 2 x 49
//     source weights (kept on chip: read from global memory every step they put an L1
//     round trip on the critical path of the warps that own the patch columns)
// A row stores the even columns' (x, z) in sq = npair + 2 float2 slots, then the odd
// columns' in sq more; slot q of each half belongs to the column pair p = q - 1, and
// slots 0 and npair + 1 (columns -2, -1, nx.., and column nx when nx is odd) are zero
// ghosts.  A thread owning pair p reads its whole neighbourhood, both components at
// once, with four 64-bit loads (its two columns, the west column from the odd half
// and the east column from the even half), each at an 8-byte stride across the
// warp: no bank conflicts.  Level m lives in A (m
// even) or B (m odd); u^{m+1} overwrites u^{m-1} in place.  The rows just above
// and below a CTA's slab are read straight from the neighbouring CTA's shared
// memory (mapa + ld.shared::cluster).  One cluster barrier (arrive.release /
// wait.acquire) per step orders the writes of step m before the reads of step
// m+1 and the reads of step m before the overwrites of step m+1; every thread of
// every CTA executes the same number of barriers.  Threads are packed densely
// over (row segment, column pair); each marches down its segment.  A row enters
// the register window once, as the south row, where its second differences and
// east - west differences are formed; its south differences are formed when the
// next row arrives, and all of them serve it again as the centre and north row.
// The surface row, the bottom row and the rows whose neighbour lives in another
// CTA are peeled off the main loop, and so are the march's last one to three rows
// (the only ones that do not prefetch): the unrolled march body has no branch.  The
// absorbing side columns are left out of the march (its stores to them go to ghost
// slots that no thread reads) and written by a separate edge warp from u^m alone, so
// the warps that hold a side column march exactly like the others; the same warp adds
// the source term to the patch nodes once the march warps that own them have stored
// them (named barrier 1).  The arithmetic runs on packed
// (x, z) pairs (.f32x2).  HBM traffic is only the seismogram samples and the source
// time function: the wavefield never leaves the chip, so this kernel is bound by
// shared-memory latency and throughput and the per-step barrier, not by HBM.
#include <type_traits>

#include "pair_math.cuh"

namespace oed {

// Block size and register cap: registers are split over the SM's four schedulers
// (16 K each), so 20 warps of 96 registers is the most one CTA can hold (the packed
// update needs about 90).  The last warp is the edge warp; three row segments of about
// twelve rows per column pair (19 march warps at 401 columns) measured faster than one,
// two, four or five.
constexpr int kResThreads = 640;
constexpr int kResRegs = 96;
constexpr bool kPS = true;   // the packed-subtract form of the pair arithmetic

struct ResArgs {
    const FacCoef<float> *fac;     // [nz]
    const SourceDesc<float> *src;  // [nsolve]
    const float *stf;              // [nsolve][nsteps]
    float *trace;                  // [nsolve][nlev][nrec][2]
    const int *rec;                // [nrec]
    Geometry g;
    int R;                         // rows per CTA
    int sq;                        // float2 slots per half row (npair + 2); a row is 2 sq
    int npair;                     // column pairs per row, (nx + 1) / 2
    int nseg;                      // row segments per column pair
    int rps;                       // rows per segment
    int nmarch;                    // threads of the march warps; the last warp is the edge warp
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

__device__ __forceinline__ float2 ld_cluster2(unsigned addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// A shared row holds the even columns' (x, z) in its first sq float2 slots and the odd
// columns' in the next sq: slot q of each half belongs to the column pair p = q - 1, so
// the pair of a thread is (E[q], O[q]), its west column O[q-1] and its east column
// E[q+1] -- four 64-bit loads at an 8-byte stride across the warp, no bank conflicts.
// q points at the thread's even slot of the row.
__device__ __forceinline__ float4 pair_at(const float2 *q, int sq)
{
    const float2 e = q[0], o = q[sq];
    return make_float4(e.x, e.y, o.x, o.y);
}

// The pair's slots in the level being written (u^{m-1} in, u^{m+1} out), at per-thread
// offsets offE (column c) and offO (column c + 1) from q: 0 and sq for interior pairs.  A
// side column (or the ghost column nx) is written by the edge warp, not by the march, so
// its thread's slot is moved to a ghost slot that no thread reads (even slot 0, or slot
// npair + 1 of either half): the march's stores stay unconditional.
__device__ __forceinline__ float4 pair_at_n(const float2 *q, int offE, int offO)
{
    const float2 e = q[offE], o = q[offO];
    return make_float4(e.x, e.y, o.x, o.y);
}

__device__ __forceinline__ void pair_put_n(float2 *q, int offE, int offO, float4 u)
{
    q[offE] = make_float2(u.x, u.y);
    q[offO] = make_float2(u.z, u.w);
}

__device__ __forceinline__ void load_row(const float2 *q, int sq, Row2P &r)
{
    row_fromP<kPS>(q[sq - 1], pair_at(q, sq), q[1], r);
}

// the same slots of a row in CTA `nb` of the cluster
__device__ __forceinline__ float4 pair_at_remote(const float2 *q, int sq, unsigned nb)
{
    const unsigned b = remote_addr(smem_addr(q), nb);
    const float2 e = ld_cluster2(b), o = ld_cluster2(b + 8u * (unsigned)sq);
    return make_float4(e.x, e.y, o.x, o.y);
}

__device__ __forceinline__ void load_row_remote(const float2 *q, int sq, unsigned nb, Row2P &r)
{
    const unsigned b = remote_addr(smem_addr(q), nb);
    const float2 e = ld_cluster2(b), o = ld_cluster2(b + 8u * (unsigned)sq);
    row_fromP<kPS>(ld_cluster2(b + 8u * (unsigned)(sq - 1)), make_float4(e.x, e.y, o.x, o.y), ld_cluster2(b + 8u), r);
}

// float offset of node (column i, component comp) within a shared row
__device__ __forceinline__ int node_off(int i, int comp, int sq)
{
    return 2 * ((i & 1) ? sq + (i >> 1) + 1 : (i >> 1) + 1) + comp;
}

__global__ void __maxnreg__(kResRegs) k_resident(ResArgs a)
{
    extern __shared__ float4 smem4[];
    const Geometry &g = a.g;
    const unsigned rank = cluster_rank();
    const int s = blockIdx.y;
    const int R = a.R, sq = a.sq;
    const int j0 = (int)rank * R;
    const int nrows = max(0, min(R, g.nz - j0));
    const int lvl = R * sq;   // 16-byte units per level
    const int RS = 2 * sq;    // float2 slots per row
    float2 *A = reinterpret_cast<float2 *>(smem4), *B = A + R * RS;
    KP *coef = reinterpret_cast<KP *>(smem4 + 2 * lvl);
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;

    for (int k = tid; k < 2 * lvl; k += nthr) smem4[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = tid; k < nrows; k += nthr) coef[k] = pack_coef(a.fac[j0 + k]);
    float *sw = reinterpret_cast<float *>(coef + R);   // this solve's source weights, x then z
    for (int k = tid; k < 2 * kPatch * kPatch; k += nthr)
        sw[k] = k < kPatch * kPatch ? a.src[blockIdx.y].wx[k] : a.src[blockIdx.y].wz[k - kPatch * kPatch];

    // march threads are packed densely over (segment, pair): a warp may straddle two
    // segments.  The last warp (the edge warp) takes the absorbing side columns, which
    // the march does not store, and the receiver samples: side columns read only u^m, so
    // this needs no synchronisation with the march, and no march warp is slowed down by
    // the absorbing patch of a side column.
    const bool edge = tid >= a.nmarch;
    const int p = tid % a.npair;
    const int c = 2 * p;
    const int seg = tid / a.npair;
    const bool active = !edge && seg < a.nseg;
    const int kind = (c == 0 ? 1 : 0) | (c + 1 == g.nx - 1 ? 2 : 0) | (c == g.nx - 1 ? 4 : 0);
    const int offE = (kind & 1) ? -1 : ((kind & 4) ? 1 : 0);
    const int offO = a.sq + ((kind & 6) ? 1 : 0);
    const int l0 = seg * a.rps;
    const int l1 = min(l0 + a.rps, nrows);
    const bool top = (j0 + l0 == 0);
    const SourceDesc<float> *sd = a.src + s;
    const int sj = sd->j0, si0 = sd->i0;
    const int siA = c - sd->i0, siB = c + 1 - sd->i0;
    const bool scolA = (unsigned)siA < (unsigned)kPatch;
    const bool scolB = c + 1 < g.nx && (unsigned)siB < (unsigned)kPatch;
    const float *stf = a.stf + (size_t)s * g.nsteps;
    // The source term of the patch nodes is added by the edge warp once the march warps
    // that own patch nodes of this CTA have stored them: those warps arrive at named
    // barrier 1 after their march (without waiting), the edge warp waits there.  The
    // count is fixed per CTA, so every step's barrier completes.
    const int srow0 = max(sj, j0), srow1 = min(sj + kPatch, j0 + nrows);   // patch rows in this CTA
    const bool patch = active && (scolA || scolB) && sj + kPatch > j0 + l0 && sj < j0 + l1;
    const bool patch_warp = __any_sync(0xffffffffu, patch);
    float *trace = a.trace + (size_t)s * g.nlev * g.nrec * 2;
    // when every row the march visits in this CTA (rows 1 or 0 .. nrows-2: the surface and
    // the last row are peeled) has the coefficients of the first, as in a homogeneous
    // medium, the march keeps them in registers instead of reloading them row by row
    const int kfirst = (j0 == 0) ? 1 : 0;
    __syncthreads();
    bool same = true;
    for (int k = kfirst + 1 + tid; k < nrows - 1; k += nthr) same &= kp_equal(coef[k], coef[kfirst]);
    const bool unif = __syncthreads_and(same) != 0 && kfirst < nrows - 1;
    const KP K0 = coef[min(kfirst, nrows - 1)];
    const int npw = __syncthreads_count(patch_warp && (tid & 31) == 0);
    cluster_barrier();

    for (int m = 0; m < g.nsteps; m++) {
        const float2 *cur = ((m & 1) ? B : A) + p + 1;   // this thread's even slot in row 0
        float2 *nxt = ((m & 1) ? A : B) + p + 1;
        if (edge) {
            const int e = tid - a.nmarch;
            const float *cf = reinterpret_cast<const float *>((m & 1) ? B : A);   // u^m
            float *nf = reinterpret_cast<float *>((m & 1) ? A : B);               // u^{m+1}
            if (rank == 0)
                for (int q = e; q < 2 * g.nrec; q += 32)
                    trace[(size_t)m * g.nrec * 2 + q] = cf[node_off(a.rec[q >> 1], q & 1, sq)];
            // side columns 0 and nx-1 (first-order absorbing, from the inward neighbour;
            // they take precedence at the surface and bottom corners)
            const int oL = node_off(0, 0, sq), oL1 = node_off(1, 0, sq);
            const int oR = node_off(g.nx - 1, 0, sq), oR1 = node_off(g.nx - 2, 0, sq);
            for (int l = e; l < nrows; l += 32) {
                const float2 cpcs = coef[l].c;
                const float *cr = cf + (size_t)l * RS * 2;
                float *nr = nf + (size_t)l * RS * 2;
                nr[oL] = absorb(cr[oL], cr[oL1], cpcs.x);
                nr[oL + 1] = absorb(cr[oL + 1], cr[oL1 + 1], cpcs.y);
                nr[oR] = absorb(cr[oR], cr[oR1], cpcs.x);
                nr[oR + 1] = absorb(cr[oR + 1], cr[oR1 + 1], cpcs.y);
            }
        }
        if (active && l0 < l1) {
            Row2P rn, rc, rs;
            int l = l0;
            load_row(cur + l * RS, sq, rc);
            if (top) {   // surface row: no north differences, cross terms on the row itself
                if (l + 1 < nrows)
                    load_row(cur + (l + 1) * RS, sq, rs);
                else   // a one-row slab
                    load_row_remote(cur, sq, rank + 1, rs);
                southP<kPS>(rc, rs);
                Row2P nt = rc;
                nt.va = nt.vb = make_float2(0.0f, 0.0f);
                float2 *o = nxt + l * RS;
                float4 u = pair_at_n(o, offE, offO);
                const KP K = coef[l];
                pair_updateP<kPS>(K, nt, rc, rs, u);
                pair_put_n(o, offE, offO, u);
                rn = rc;
                rc = rs;
                l++;
            } else {
                if (l > 0)
                    load_row(cur + (l - 1) * RS, sq, rn);
                else
                    load_row_remote(cur + (R - 1) * RS, sq, rank - 1, rn);
                southP<kPS>(rn, rc);
            }
            // rows whose south neighbour is a local row and that are not the bottom row:
            // unrolled by three with the three window rows taking turns
            const int lstop = min(l1, nrows - 1);
            if (l < lstop) {
                // the loads of the next row are issued before the update of this one
                const float2 *sp = cur + (l + 1) * RS;
                float2 *o = nxt + l * RS;
                const KP *cf = coef + l;
                float4 pm = pair_at(sp, sq), pu = pair_at_n(o, offE, offO);
                float2 pw = sp[sq - 1];
                float2 pe = sp[1];
                // pf: a row below the south row exists, prefetch it (every row but the last)
                // unifK: the CTA's march rows share K0 (no coefficient loads)
                auto march = [&](auto unifK) {
                    auto row = [&](auto pf, const Row2P &wn, Row2P &wc, Row2P &ws) {
                        row_fromP<kPS>(pw, pm, pe, ws);
                        float4 u = pu;
                        if constexpr (decltype(pf)::value) {
                            sp += RS;
                            pm = pair_at(sp, sq);
                            pw = sp[sq - 1];
                            pe = sp[1];
                            pu = pair_at_n(o + RS, offE, offO);
                        }
                        southP<kPS>(wc, ws);
                        const KP K = decltype(unifK)::value ? K0 : *cf;
                        pair_updateP<kPS>(K, wn, wc, ws, u);
                        pair_put_n(o, offE, offO, u);
                        o += RS;
                        cf++;
                    };
                    const std::true_type P{};
                    const std::false_type N{};
                    for (; l + 3 < lstop; l += 3) {
                        row(P, rn, rc, rs);   // window (n, c, s)
                        row(P, rc, rs, rn);   // row l+2 lands in rn
                        row(P, rs, rn, rc);   // row l+3 lands in rc
                    }
                    // one to three rows left, the last without prefetch; the window ends
                    // as (rn, rc) = (north, centre) of the row after the march
                    const int r = lstop - l;
                    if (r == 3) {
                        row(P, rn, rc, rs);
                        row(P, rc, rs, rn);
                        row(N, rs, rn, rc);
                    } else if (r == 2) {
                        row(P, rn, rc, rs);
                        row(N, rc, rs, rn);
                        const Row2P t = rn;
                        rn = rs;
                        rc = t;
                    } else {
                        row(N, rn, rc, rs);
                        rn = rc;
                        rc = rs;
                    }
                    l = lstop;
                };
                // a CTA-uniform choice: a branch inside the march body would split the
                // unrolled rows into separate blocks and cost the scheduler its overlap
                if (unif)
                    march(std::true_type{});
                else
                    march(std::false_type{});
            }
            // what is left: a last interior row whose south neighbour sits in CTA rank+1,
            // or the absorbing bottom row
            for (; l < l1; l++) {
                const KP K = coef[l];
                float2 *o = nxt + l * RS;
                float4 u = pair_at_n(o, offE, offO);
                if (j0 + l == g.nz - 1) {
                    const float4 nv = l > 0 ? pair_at(cur + (l - 1) * RS, sq)
                                            : pair_at_remote(cur + (R - 1) * RS, sq, rank - 1);
                    absorbingP(K.c, nv, rc, true, 0, u);
                } else {
                    load_row_remote(cur, sq, rank + 1, rs);
                    southP<kPS>(rc, rs);
                    pair_updateP<kPS>(K, rn, rc, rs, u);
                }
                pair_put_n(o, offE, offO, u);
                rn = rc;
                rc = rs;
            }
        }
        if (patch_warp)
            asm volatile("bar.arrive 1, %0;" :: "r"(32 * (npw + 1)) : "memory");
        if (edge && npw > 0) {
            // source term: u^{m+1} += dt^2/nu f^m on the patch nodes of this CTA, added last
            // as in the node update of the streaming kernel (one node per lane)
            asm volatile("bar.sync 1, %0;" :: "r"(32 * (npw + 1)) : "memory");
            float *nf = reinterpret_cast<float *>((m & 1) ? A : B);
            const float S = stf[m];
            for (int k = tid - a.nmarch; k < kPatch * kPatch; k += 32) {
                const int bb = k / kPatch, ai = k - bb * kPatch;
                const int j = sj + bb;
                if (j < srow0 || j >= srow1) continue;
                float *row = nf + (size_t)(j - j0) * RS * 2;
                const int o = node_off(si0 + ai, 0, sq);
                row[o] = add_force(row[o], S, sw[k]);
                row[o + 1] = add_force(row[o + 1], S, sw[kPatch * kPatch + k]);
            }
        }
        cluster_barrier();
    }
    if (rank == 0) {
        const float *row0 = reinterpret_cast<const float *>((g.nsteps & 1) ? B : A);
        for (int q = tid; q < 2 * g.nrec; q += nthr)
            trace[(size_t)g.nsteps * g.nrec * 2 + q] = row0[node_off(a.rec[q >> 1], q & 1, sq)];
    }
}

// Shape of the resident launch for a grid: cluster size C (1..8) and rows per CTA,
// or C = 0 when the two levels do not fit in C CTAs of shared memory.
struct ResShape {
    int C, R, sq, npair, nseg, rps, nmarch, threads;
    size_t smem;
};

static ResShape resident_shape(const Geometry &g, int C)
{
    ResShape r{};
    const int npair = (g.nx + 1) / 2;
    if (npair > kResThreads - 32 || C < 1 || C > 8) return r;
    const int R = (g.nz + C - 1) / C;
    if ((C - 1) * R >= g.nz) return r;   // a CTA would own no rows
    const int sq = npair + 2;   // ghost slots on both sides
    const size_t smem = (size_t)2 * R * sq * sizeof(float4) + (size_t)R * sizeof(KP) +
                        2 * kPatch * kPatch * sizeof(float);
    if (smem > 227 * 1024) return r;
    int nseg = (kResThreads - 32) / npair;   // the last warp is the edge warp
    if (nseg > R) nseg = R;
    r.C = C;
    r.R = R;
    r.sq = sq;
    r.npair = npair;
    r.nseg = nseg;
    r.rps = (R + nseg - 1) / nseg;
    r.nmarch = (npair * nseg + 31) / 32 * 32;
    r.threads = r.nmarch + 32;
    r.smem = smem;
    return r;
}

// Smallest cluster that holds an FP32 grid, or 0 if none does.
int resident_fits(const Geometry &g)
{
    for (int C = 1; C <= 8; C++)
        if (resident_shape(g, C).C) return C;
    return 0;
}

// The same for a context (0 for FP64 contexts).
int resident_cluster_size(const oed_ctx *ctx)
{
    return ctx->precision == OED_FP32 ? resident_fits(ctx->g) : 0;
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
    a.sq = r.sq;
    a.npair = r.npair;
    a.nseg = r.nseg;
    a.rps = r.rps;
    a.nmarch = r.nmarch;
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
