// Two leap-frog steps per pass for grids whose wavefield does not fit the
// cluster-resident kernel (Sec. 3.3.1, Eq. Full_Disc; the packed node update of
// pair_math.cuh, so the bits are those of every other stencil kernel).
//
// The levels are kept in the paired layout (oed_internal.cuh): a row holds the even
// columns' (x, z) pairs, then the odd columns', as the cluster-resident kernel keeps its
// rows in shared memory.  A persistent CTA walks tiles (solve, 20-row band, 60-column
// band).  For each tile its producer warp loads, with one 4-D cp.async.bulk.tensor copy
// per level (34 slots of both halves, i.e. columns x0-4 .. x0+63, by the rows below),
// into one stage of a 4-stage shared-memory ring:
//   HM  u^m,     rows z0-2 .. z0+21
//   HP  u^{m-1}, rows z0-1 .. z0+20
// and, with cp.async.bulk, the coefficient rows z0-1 .. z0+20 that lie in the grid, as
// (x, z) pairs packed once per problem
// (x0 is a multiple of 60, so every copy starts on a 16-byte boundary; rows and
// columns outside the grid read as zeros and are never used).  Completion is tracked
// per stage by an mbarrier with the stage's byte count.  Two groups of four consumer
// warps take the tiles in turn, each owning two stages.  In a tile, lane p owns the
// column pair x0-2+2p and reads its pair, its west and its east column as four
// conflict-free 64-bit (x, z) loads, and a warp a segment of rows (the tests for the
// surface and bottom rows, the side columns and the source patch run only in the
// tiles that hold them):
//   step 1  u^{m+1} on rows z0-1 .. z0+20, columns x0-2 .. x0+61 (the tile and a
//           one-node ring), written in place over u^{m-1} in HP (a node reads only
//           its own u^{m-1}), and, for the tile's own nodes, to global memory;
//   group barrier (the ring values of other warps' rows are needed next);
//   step 2  u^{m+2} on the tile's own nodes, from u^{m+1} in HP and u^m in HM, to
//           global memory (skipped in the single-step pass of an odd step count).
// The receiver samples of levels m and m+1 are taken from HM and HP on the surface
// band.  Levels live in two pairs of buffers used in alternation: a pass reads
// (u^{m-1}, u^m) from one pair and writes (u^{m+1}, u^{m+2}) to the other, so no
// tile overwrites what a neighbouring tile still reads.  HBM traffic per
// cell-update is 16 B (two levels read and two written per two steps) against the
// one-step kernel's 24 B; the halo re-reads come from L2.  Every wait is bounded as
// in the one-step kernel and raises the same device flag on expiry.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "pair_math.cuh"
#include "tma_sync.cuh"

namespace oed {

constexpr int kT2X = 60, kT2Z = 20;                  // output tile
constexpr int kS2 = (kT2X + 8) / 2;                  // 34 slots per half row: columns x0-4 .. x0+63
constexpr int kR2 = 2 * kS2;                         // float2 slots per tile row
constexpr int kM2Z = kT2Z + 4;                       // 24 rows of u^m: z0-2 .. z0+21
constexpr int kP2Z = kT2Z + 2;                       // 22 rows of u^{m-1}, u^{m+1}: z0-1 .. z0+20
constexpr int k2Groups = 2, k2GroupStages = 2, k2Stages = k2Groups * k2GroupStages;
constexpr int k2GroupWarps = 4, k2ConsumerWarps = k2Groups * k2GroupWarps;
constexpr int k2PlaneM = kR2 * kM2Z * 8;                        // 13056 = 102 x 128
constexpr int k2PlaneP = kR2 * kP2Z * 8;                        // 11968
constexpr int k2PlanePPad = (k2PlaneP + 127) / 128 * 128;       // 12032
constexpr int k2Coef = kP2Z * (int)sizeof(KP);                  // 1408
constexpr int k2StageBytes = k2PlaneM + k2PlanePPad + k2Coef;
constexpr unsigned k2TileTx = k2PlaneM + k2PlaneP;
constexpr int k2SmemBytes = k2Stages * k2StageBytes + 128 /* alignment slack */ + 128 /* barriers */;
// rows of step 1 per warp (22 = 6 + 6 + 5 + 5) and of step 2 (20 = 4 x 5)
__device__ __constant__ int k2Seg1[k2GroupWarps + 1] = {0, 6, 12, 17, 22};
constexpr int k2Seg1Max = 6;
constexpr int k2Rows2 = kT2Z / k2GroupWarps;

struct Tma2Args {
    float *outA;                  // u^{m+1} (global, paired layout, the other pair's older level)
    float *outB;                  // u^{m+2} (global, paired layout, the other pair's newer level)
    const KP *kp;                 // [nz] the rows' coefficients as (x, z) pairs
    const SourceDesc<float> *src;
    const float *stf;
    float *trace;
    const int *rec;
    int *err;
    Geometry g;
    int m, nsolve, nbx, nbz;
    int sq;                       // slots per half row of the paired layout
    size_t pst;                   // floats per solve of the paired layout
    int single;                   // 1: step 1 only (the last pass of an odd step count)
};

__device__ __forceinline__ int stage2(unsigned k)
{
    return (int)(k % k2Groups) * k2GroupStages + (int)((k / k2Groups) % k2GroupStages);
}
__device__ __forceinline__ unsigned phase2(unsigned k)
{
    return ((k / k2Groups) / k2GroupStages) & 1u;
}

// q points at a lane's even slot in a tile row: its pair is (q[0], q[kS2]), its west
// column q[kS2 - 1] (odd half), its east column q[1] (even half); 64-bit loads at an
// 8-byte stride across the warp, no bank conflicts
__device__ __forceinline__ void tile_row(const float2 *q, Row2P &row)
{
    const float2 e = q[0], o = q[kS2];
    row_fromP(q[kS2 - 1], make_float4(e.x, e.y, o.x, o.y), q[1], row);
}

__device__ __forceinline__ float4 tile_pair(const float2 *q)
{
    const float2 e = q[0], o = q[kS2];
    return make_float4(e.x, e.y, o.x, o.y);
}

__device__ __forceinline__ void tile_put(float2 *q, float4 u)
{
    q[0] = make_float2(u.x, u.y);
    q[kS2] = make_float2(u.z, u.w);
}

// float offset of (column x, component comp) in a tile row whose first column is x0 - 4
__device__ __forceinline__ int tile_off(int x, int x0, int comp)
{
    return 2 * ((x & 1) * kS2 + (x >> 1) + 2 - (x0 >> 1)) + comp;
}

// One node-pair update at grid row z: the interior, surface or bottom form, the
// absorbing side columns, then the force on the source patch (added last, as in
// every kernel).  u holds u^{m-1} of the pair on entry.
struct PairCtx {
    int kind;          // side-column flags (stencil_cell.cuh)
    int siA, siB;      // column offsets in the source patch
    int j0;            // first row of the source patch
    bool scolA, scolB; // the pair's columns lie in the patch
};

struct TileFlags {
    bool rows;   // the surface or the bottom row is among the tile's rows
    bool side;   // a side column is among the tile's columns
    bool src;    // the source patch meets the tile
};

__device__ __forceinline__ void update_at(const KP &K, int z, int nz, const Row2P &rn, const Row2P &rc,
                                          const Row2P &rs, const PairCtx &pc, const TileFlags &tf,
                                          const SourceDesc<float> *sd, float S, float4 &u)
{
    if (tf.rows && z == nz - 1) {
        absorbingP(K.c, make_float4(rn.ca.x, rn.ca.y, rn.cb.x, rn.cb.y), rc, true, pc.kind, u);
    } else if (tf.rows && z == 0) {   // surface row: no north differences, cross terms on the row itself
        Row2P nt = rc;
        nt.va = nt.vb = make_float2(0.0f, 0.0f);
        pair_updateP(K, nt, rc, rs, u);
        if (pc.kind) absorbingP(K.c, u, rc, false, pc.kind, u);
    } else {
        pair_updateP(K, rn, rc, rs, u);
        if (tf.side && pc.kind) absorbingP(K.c, u, rc, false, pc.kind, u);
    }
    if (!tf.src) return;
    const int b = z - pc.j0;
    if ((unsigned)b < (unsigned)kPatch && (pc.scolA || pc.scolB)) {
        if (pc.scolA) {
            u.x = add_force(u.x, S, sd->wx[b * kPatch + pc.siA]);
            u.y = add_force(u.y, S, sd->wz[b * kPatch + pc.siA]);
        }
        if (pc.scolB) {
            u.z = add_force(u.z, S, sd->wx[b * kPatch + pc.siB]);
            u.w = add_force(u.w, S, sd->wz[b * kPatch + pc.siB]);
        }
    }
}

// named barrier 1 + grp over the group's 128 threads
__device__ __forceinline__ void group_sync(int grp)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(32 * k2GroupWarps) : "memory");
}

// the same barrier, returning whether pred holds in every thread of the group
__device__ __forceinline__ bool group_all(int grp, bool pred)
{
    unsigned r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
                 " bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((unsigned)pred), "r"(1 + grp), "r"(32 * k2GroupWarps)
                 : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(32 * (k2ConsumerWarps + 1), 2)
    k_step2_tma(Tma2Args a, const __grid_constant__ CUtensorMap cur_m, const __grid_constant__ CUtensorMap cur_p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const unsigned raw = (unsigned)__cvta_generic_to_shared(smem_raw);
    unsigned char *smem = smem_raw + (((raw + 127u) & ~127u) - raw);
    uint64_t *full_bar = reinterpret_cast<uint64_t *>(smem + k2Stages * k2StageBytes);
    uint64_t *empty_bar = full_bar + k2Stages;
    const Geometry &g = a.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned ntile = (unsigned)a.nsolve * (unsigned)a.nbz * (unsigned)a.nbx;
    if (threadIdx.x == 0) {
        for (int s = 0; s < k2Stages; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], k2GroupWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // producer
        if (lane == 0) {
            unsigned k = 0;
            bool ok = true;
            for (unsigned t = blockIdx.x; t < ntile; t += gridDim.x, k++) {
                const int stage = stage2(k);
                if (k / k2Groups >= k2GroupStages && !mbar_wait(&empty_bar[stage], phase2(k) ^ 1u)) {
                    ok = false;
                    break;
                }
                const unsigned q = t / (unsigned)a.nbx;
                const int bx = (int)(t - q * (unsigned)a.nbx);
                const int s = (int)(q / (unsigned)a.nbz);
                const int bz = (int)(q - (unsigned)s * (unsigned)a.nbz);
                const int x0 = bx * kT2X, z0 = bz * kT2Z;
                unsigned char *st = smem + stage * k2StageBytes;
                // coefficient rows z0-1 .. z0+20 inside the grid
                const int c0 = max(0, z0 - 1), c1 = min(g.nz, z0 + kT2Z + 1);
                const unsigned cbytes = (unsigned)((c1 - c0) * (int)sizeof(KP));
                mbar_expect_tx(&full_bar[stage], k2TileTx + cbytes);
                // slot x0 / 2 of each half is column x0 - 4: the float coordinate x0 is a
                // multiple of four, a 16-byte boundary
                tma_load4(st, &cur_m, x0, 0, z0 - 2, s, &full_bar[stage]);
                tma_load4(st + k2PlaneM, &cur_p, x0, 0, z0 - 1, s, &full_bar[stage]);
                bulk_load(st + k2PlaneM + k2PlanePPad + (c0 - (z0 - 1)) * (int)sizeof(KP), a.kp + c0, cbytes,
                          &full_bar[stage]);
            }
            if (!ok) {
                atomicExch(a.err, 1);
                // copies already issued for the last stages must land before the CTA exits
                for (unsigned j = (k > k2Stages ? k - k2Stages : 0); j < k; j++)
                    mbar_wait(&full_bar[stage2(j)], phase2(j));
            }
        }
        return;
    }

    const int grp = (warp - 1) / k2GroupWarps, wig = (warp - 1) % k2GroupWarps;
    const int gt = wig * 32 + lane;
    const size_t grow = 4 * (size_t)a.sq;   // floats per row of the paired layout
    for (unsigned k = grp, t = blockIdx.x + grp * gridDim.x; t < ntile; k += k2Groups, t += k2Groups * gridDim.x) {
        const int stage = stage2(k);
        // the group leaves together or not at all: one thread's wait may run out while
        // another's sees the phase complete, and a thread that left alone would stop the
        // rest at the group barrier below for good
        if (!group_all(grp, mbar_wait(&full_bar[stage], phase2(k)))) {
            if (gt == 0) atomicExch(a.err, 1);
            return;
        }
        const unsigned qq = t / (unsigned)a.nbx;
        const int bx = (int)(t - qq * (unsigned)a.nbx);
        const int s = (int)(qq / (unsigned)a.nbz);
        const int bz = (int)(qq - (unsigned)s * (unsigned)a.nbz);
        const int x0 = bx * kT2X, z0 = bz * kT2Z;
        unsigned char *st = smem + stage * k2StageBytes;
        const float2 *hm = reinterpret_cast<const float2 *>(st);
        float2 *hp = reinterpret_cast<float2 *>(st + k2PlaneM);
        const KP *kp = reinterpret_cast<const KP *>(st + k2PlaneM + k2PlanePPad);
        const float2 *hmq = hm + lane + 1;   // this lane's even slot in tile row 0
        float2 *hpq = hp + lane + 1;
        const SourceDesc<float> *sd = a.src + s;
        const int c = x0 - 2 + 2 * lane;   // the pair's first column
        // the pair's even slot in row 0 of the solve's outputs (its odd slot is sq float2 on)
        const size_t co = (size_t)s * a.pst + 2 * (size_t)((c >> 1) + 2);
        float *gA = a.outA + co, *gB = a.outB + co;
        const int si0 = sd->i0, sj0 = sd->j0;
        // tile-uniform flags: the tile (with its ring) holds the surface or bottom row, a
        // side column, or part of the source patch; the tests of each are skipped
        // elsewhere, which is most tiles
        TileFlags tf;
        tf.rows = z0 < 2 || z0 + kT2Z > g.nz - 2;
        tf.side = x0 < 3 || x0 + kT2X + 1 > g.nx - 2;
        tf.src = !(sj0 + kPatch <= z0 - 1 || sj0 >= z0 + kT2Z + 1 || si0 + kPatch <= x0 - 2 ||
                   si0 >= x0 + kT2X + 2);
        const size_t tr0 = (size_t)s * g.nlev * g.nrec * 2;
        // receiver samples of level m (HM row 2 is grid row 0 on the surface band)
        if (z0 == 0)
            for (int r = gt; r < 2 * g.nrec; r += 32 * k2GroupWarps) {
                const int xr = a.rec[r >> 1];
                if (xr >= x0 && xr < x0 + kT2X)
                    a.trace[tr0 + (size_t)a.m * g.nrec * 2 + r] =
                        reinterpret_cast<const float *>(hm + 2 * kR2)[tile_off(xr, x0, r & 1)];
            }
        const bool valid = c >= 0 && c < g.nx;
        PairCtx pc;
        pc.kind = (c == 0 ? 1 : 0) | (c + 1 == g.nx - 1 ? 2 : 0) | (c == g.nx - 1 ? 4 : 0);
        pc.siA = c - si0;
        pc.siB = c + 1 - si0;
        pc.j0 = sj0;
        pc.scolA = (unsigned)pc.siA < (unsigned)kPatch;
        pc.scolB = c + 1 < g.nx && (unsigned)pc.siB < (unsigned)kPatch;
        const bool own = lane >= 1 && lane <= kT2X / 2 && valid;   // a pair of the tile itself
        const float S1 = (pc.scolA || pc.scolB) ? a.stf[(size_t)s * g.nsteps + a.m] : 0.0f;
        const float S2 = (pc.scolA || pc.scolB) && a.m + 1 < g.nsteps ? a.stf[(size_t)s * g.nsteps + a.m + 1] : 0.0f;

        // step 1: u^{m+1} on HP rows [r_a, r_b) (grid row z0 - 1 + r)
        if (valid) {
            const int ra = k2Seg1[wig], nr = k2Seg1[wig + 1] - ra;
            Row2P rn, rc, rs;
            tile_row(hmq + ra * kR2, rn);       // HM row r is grid row z0 - 2 + r
            tile_row(hmq + (ra + 1) * kR2, rc);
            southP(rn, rc);
            // unrolled to the longest segment, so the window rows stay in place in the
            // registers instead of being copied row after row
#pragma unroll
            for (int i = 0; i < k2Seg1Max; i++) {
                if (i >= nr) break;
                const int r = ra + i;
                const int z = z0 - 1 + r;
                tile_row(hmq + (r + 2) * kR2, rs);
                southP(rc, rs);
                if (z >= 0 && z < g.nz) {
                    float4 u = tile_pair(hpq + r * kR2);
                    update_at(kp[r], z, g.nz, rn, rc, rs, pc, tf, sd, S1, u);
                    tile_put(hpq + r * kR2, u);
                    if (own && r >= 1 && r <= kT2Z) {
                        float *o = gA + (size_t)z * grow;
                        __stcs(reinterpret_cast<float2 *>(o), make_float2(u.x, u.y));
                        __stcs(reinterpret_cast<float2 *>(o + 2 * a.sq), make_float2(u.z, u.w));
                    }
                }
                rn = rc;
                rc = rs;
            }
        }
        group_sync(grp);
        // receiver samples of level m+1 (HP row 1 is grid row 0)
        if (z0 == 0)
            for (int r = gt; r < 2 * g.nrec; r += 32 * k2GroupWarps) {
                const int xr = a.rec[r >> 1];
                if (xr >= x0 && xr < x0 + kT2X)
                    a.trace[tr0 + (size_t)(a.m + 1) * g.nrec * 2 + r] =
                        reinterpret_cast<const float *>(hp + kR2)[tile_off(xr, x0, r & 1)];
            }
        // step 2: u^{m+2} on the tile's rows [5 wig, 5 wig + 5) (grid row z0 + r)
        if (own && !a.single) {
            const int ra = wig * k2Rows2;
            Row2P rn, rc, rs;
            tile_row(hpq + ra * kR2, rn);       // HP row r + 1 is grid row z0 + r
            tile_row(hpq + (ra + 1) * kR2, rc);
            southP(rn, rc);
#pragma unroll
            for (int r = ra; r < ra + k2Rows2; r++) {
                const int z = z0 + r;
                if (z >= g.nz) break;
                tile_row(hpq + (r + 2) * kR2, rs);
                southP(rc, rs);
                float4 u = tile_pair(hmq + (r + 2) * kR2);   // u^m of the node
                update_at(kp[r + 1], z, g.nz, rn, rc, rs, pc, tf, sd, S2, u);
                float *o = gB + (size_t)z * grow;
                __stcs(reinterpret_cast<float2 *>(o), make_float2(u.x, u.y));
                __stcs(reinterpret_cast<float2 *>(o + 2 * a.sq), make_float2(u.z, u.w));
                rn = rc;
                rc = rs;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[stage]);
    }
}

// The rows' coefficients as (x, z) pairs, the form the packed update reads.
__global__ void k_pack_kp(const FacCoef<float> *__restrict__ fac, int nz, KP *__restrict__ kp)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nz) kp[j] = pack_coef(fac[j]);
}

// ---------------------------------------------------------------- host side

void launch_pack_kp(const oed_ctx *ctx, cudaStream_t st)
{
    if (!ctx->d_kp) return;
    k_pack_kp<<<(ctx->g.nz + 127) / 128, 128, 0, st>>>((const FacCoef<float> *)ctx->d_fac, ctx->g.nz,
                                                       (KP *)ctx->d_kp);
}

int tma2_prepare(oed_ctx *ctx)
{
    if (cudaFuncSetAttribute(k_step2_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, k2SmemBytes) != cudaSuccess)
        return 0;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step2_tma, 32 * (k2ConsumerWarps + 1),
                                                      k2SmemBytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    ctx->tma2_ctas = nsm * per_sm;
    return ctx->tma2_ctas;
}

// Receiver samples of one level in the paired layout (the final level after the last pass).
__global__ void k_gather_paired(const float *__restrict__ cur, float *__restrict__ trace,
                                const int *__restrict__ rec, Geometry g, int sq, size_t pst, int m, int nsolve)
{
    const int s = blockIdx.x;
    if (s >= nsolve) return;
    const float *row0 = cur + (size_t)s * pst;   // grid row 0
    float *tr = trace + ((size_t)s * g.nlev + m) * g.nrec * 2;
    for (int q = threadIdx.x; q < 2 * g.nrec; q += blockDim.x) {
        const int x = rec[q >> 1];
        tr[q] = row0[2 * ((x & 1) * sq + (x >> 1) + 2) + (q & 1)];
    }
}

void launch_tma2_gather(const oed_ctx *ctx, int nsolve, const float *last, int m, cudaStream_t st)
{
    k_gather_paired<<<nsolve, 128, 0, st>>>(last, (float *)ctx->d_trace, ctx->d_rec, ctx->g, paired_sq(ctx->g),
                                            paired_stride(ctx->g), m, nsolve);
}

// nsteps (or nsteps_override) steps of nsolve solves: two-step passes over the level
// pairs (d_u0, d_u1) and (d_u2, d_u3) in alternation, all in the paired layout, and a
// last single-step pass when the count is odd.  *last is set to the buffer that holds
// the final level.  The caller zeroes all four levels (paired_stride floats per solve).
cudaError_t launch_steps_tma2(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                              int nsteps_override, const float **last)
{
    const Geometry &g = ctx->g;
    if (ctx->tma2_ctas < 1 || !ctx->d_u2 || !ctx->d_kp) return cudaErrorInvalidConfiguration;
    float *lv[4] = {(float *)ctx->d_u0, (float *)ctx->d_u1, (float *)ctx->d_u2, (float *)ctx->d_u3};
    CUtensorMap mmap[2], pmap[2];   // per pair: u^m (newer level, 2-row halo), u^{m-1} (older, 1-row)
    for (int pr = 0; pr < 2; pr++)
        if (!tma_make_paired_map(&mmap[pr], lv[2 * pr + 1], g, nsolve, kS2, kM2Z) ||
            !tma_make_paired_map(&pmap[pr], lv[2 * pr], g, nsolve, kS2, kP2Z))
            return cudaErrorInvalidValue;
    Tma2Args a;
    a.kp = (const KP *)ctx->d_kp;
    a.src = (const SourceDesc<float> *)ctx->d_src;
    a.stf = (const float *)ctx->d_stf;
    a.trace = (float *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.err = ctx->d_err;
    a.g = g;
    a.nsolve = nsolve;
    a.nbx = (g.nx + kT2X - 1) / kT2X;
    a.nbz = (g.nz + kT2Z - 1) / kT2Z;
    a.sq = paired_sq(g);
    a.pst = paired_stride(g);
    a.single = 0;
    const long long ntile = (long long)nsolve * a.nbx * a.nbz;
    if (ntile >= (1LL << 31) - 2LL * ctx->tma2_ctas) return cudaErrorInvalidValue;   // 32-bit tile indices
    const int grid = (int)(ntile < (long long)ctx->tma2_ctas ? ntile : (long long)ctx->tma2_ctas);
    const int nsteps = (nsteps_override > 0 && nsteps_override < g.nsteps) ? nsteps_override : g.nsteps;
    tma_record(ev0, st);
    int pr = 0;   // the pair holding (u^{m-1}, u^m)
    int m = 0;
    for (; m < nsteps; m += 2, pr ^= 1) {
        a.outA = lv[2 * (pr ^ 1)];
        a.outB = lv[2 * (pr ^ 1) + 1];
        a.m = m;
        a.single = m + 1 == nsteps;   // an odd count: the last pass takes one step
        k_step2_tma<<<grid, 32 * (k2ConsumerWarps + 1), k2SmemBytes, st>>>(a, mmap[pr], pmap[pr]);
        *last = a.single ? a.outA : a.outB;
    }
    tma_record(ev1, st);
    return cudaGetLastError();
}

}  // namespace oed
