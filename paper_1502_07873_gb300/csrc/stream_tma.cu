// Streaming leap-frog step with TMA tile loads (one launch per time step, for
// grids whose wavefield does not fit the cluster-resident kernel; Sec. 3.3.1,
// Eq. Full_Disc; the column-pair node update of stencil_cell.cuh).
//
// A persistent CTA walks tiles (solve, 20-row band, 64-column band) of the batch.
// Its producer warp issues, for each tile, four cp.async.bulk.tensor loads into one
// stage of a shared-memory ring -- u_x and u_z of level m with a halo (rows z0-1 ..
// z0+20, columns x0-4 .. x0+67; the x start stays a multiple of four floats so
// every copy starts on a 16-byte boundary, the grid edges read as zeros and are
// never used) and u_x, u_z of level m-1 without halo -- and one cp.async.bulk of the
// band's per-row coefficients.  Completion is tracked by an mbarrier per stage
// (expect_tx of the stage's bytes).  Two groups of four consumer warps take the
// tiles in turn, each with two stages of its own, so each barrier is waited on
// phase after phase by one group only (a group that waited on another group's
// stage could see a phase two uses old and read a stage still being filled).  In
// a tile a thread owns a column pair and marches five rows with the register
// window of the resident kernel (each row's differences formed once), stores
// u^{m+1} with streaming stores over u^{m-1}, and the group releases the stage on
// a second mbarrier.  Every wait is bounded: on expiry the kernel raises a device
// flag, the producer waits (bounded) for its copies in flight, and the threads
// return; the flag turns the affected nodes' status into OED_ETIMEOUT.  HBM traffic
// per cell-update is the algorithmic 24 B (FP32); the halo re-reads come from L2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "stencil_cell.cuh"
#include "tma_sync.cuh"

namespace oed {

constexpr int kTX = 64, kTZ = 20, kHX = 4;
constexpr int kWX = kTX + 2 * kHX, kWZ = kTZ + 2;
constexpr int kGroups = 2;                               // consumer groups, tiles taken in turn
constexpr int kGroupStages = 2;                          // ring stages owned by each group
constexpr int kStages = kGroups * kGroupStages;
constexpr int kGroupWarps = 4;                           // 32 column pairs x 4 segments
constexpr int kConsumerWarps = kGroups * kGroupWarps;
constexpr int kRowsPerSeg = kTZ / kGroupWarps;           // 5
constexpr int kHaloBytes = kWX * kWZ * 4;                // 6336
constexpr int kHaloPad = (kHaloBytes + 127) / 128 * 128; // 6400
constexpr int kPlainBytes = kTX * kTZ * 4;               // 5120
constexpr int kCoefBytes = kTZ * (int)sizeof(FacCoef<float>);   // 1280
constexpr int kStageBytes = 2 * kHaloPad + 2 * kPlainBytes + kCoefBytes;
constexpr unsigned kTileTxBytes = 2 * kHaloBytes + 2 * kPlainBytes;
constexpr int kSmemBytes = kStages * kStageBytes + 128 /* alignment slack */ + 128 /* barriers */;

struct TmaArgs {
    float *nxt;                   // u^{m-1} in, u^{m+1} out (global)
    const FacCoef<float> *fac;
    const SourceDesc<float> *src;
    const float *stf;
    float *trace;
    const int *rec;
    int *err;                     // set to 1 if a bounded wait expired
    Geometry g;
    int m, nsolve, nbx, nbz;
};

// Self-test of the bounded wait: one CTA waits for the first phase of a barrier that
// expects one arrival and never gets it, so the wait can only end by its limit; it
// then raises the same device flag as the streaming kernel does.
__global__ void k_wait_selftest(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0 && !ok) atomicExch(err, 1);
}

// stage and phase of the CTA's k-th tile: group k % kGroups takes it as its i-th
// tile, i = k / kGroups, in one of the group's own stages
__device__ __forceinline__ int tile_stage(unsigned k)
{
    return (int)(k % kGroups) * kGroupStages + (int)((k / kGroups) % kGroupStages);
}
__device__ __forceinline__ unsigned tile_phase(unsigned k)
{
    return ((k / kGroups) / kGroupStages) & 1u;
}

// (column band, row band, solve) of tile t; 32-bit arithmetic (the host keeps the tile
// count below 2^31)
__device__ __forceinline__ void tile_coords(unsigned t, const TmaArgs &a, int &bx, int &bz, int &s)
{
    const unsigned q = t / (unsigned)a.nbx;
    bx = (int)(t - q * (unsigned)a.nbx);
    s = (int)(q / (unsigned)a.nbz);
    bz = (int)(q - (unsigned)s * (unsigned)a.nbz);
}

// the row of a tile seen by the thread owning pair p (columns x0 + 2p, x0 + 2p + 1)
__device__ __forceinline__ void tile_row(const float *hx, const float *hz, int r, int p, Row2 &row)
{
    const float *qx = hx + r * kWX + kHX + 2 * p, *qz = hz + r * kWX + kHX + 2 * p;
    const float2 mx = *reinterpret_cast<const float2 *>(qx), mz = *reinterpret_cast<const float2 *>(qz);
    row_from(make_float2(qx[-1], qz[-1]), make_float4(mx.x, mz.x, mx.y, mz.y), make_float2(qx[2], qz[2]), row);
}

__global__ void __launch_bounds__(32 * (kConsumerWarps + 1), 2)
    k_step_tma(TmaArgs a, const __grid_constant__ CUtensorMap cur_halo,
               const __grid_constant__ CUtensorMap nxt_plain)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // stages start on a 128-byte boundary of the shared window (TMA destinations);
    // the two barrier arrays follow the stages
    const unsigned raw = (unsigned)__cvta_generic_to_shared(smem_raw);
    unsigned char *smem = smem_raw + (((raw + 127u) & ~127u) - raw);
    uint64_t *full_bar = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty_bar = full_bar + kStages;
    const Geometry &g = a.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned ntile = (unsigned)a.nsolve * (unsigned)a.nbz * (unsigned)a.nbx;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], kGroupWarps);
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
                const int stage = tile_stage(k);
                const unsigned phase = tile_phase(k);
                if (k / kGroups >= kGroupStages && !mbar_wait(&empty_bar[stage], phase ^ 1u)) {
                    ok = false;
                    break;
                }
                int bx, bz, s;
                tile_coords(t, a, bx, bz, s);
                const int x0 = bx * kTX, z0 = bz * kTZ;
                unsigned char *st = smem + stage * kStageBytes;
                const int nrow = min(kTZ, g.nz - z0);   // coefficient rows of the band
                mbar_expect_tx(&full_bar[stage], kTileTxBytes + (unsigned)(nrow * (int)sizeof(FacCoef<float>)));
                tma_load3(st, &cur_halo, x0 - kHX, z0 - 1, 2 * s, &full_bar[stage]);
                tma_load3(st + kHaloPad, &cur_halo, x0 - kHX, z0 - 1, 2 * s + 1, &full_bar[stage]);
                tma_load3(st + 2 * kHaloPad, &nxt_plain, x0, z0, 2 * s, &full_bar[stage]);
                tma_load3(st + 2 * kHaloPad + kPlainBytes, &nxt_plain, x0, z0, 2 * s + 1, &full_bar[stage]);
                bulk_load(st + 2 * kHaloPad + 2 * kPlainBytes, a.fac + z0, (unsigned)(nrow * (int)sizeof(FacCoef<float>)),
                          &full_bar[stage]);
            }
            if (!ok) {
                atomicExch(a.err, 1);
                // copies already issued for the last stages must land before the CTA exits
                for (unsigned j = (k > kStages ? k - kStages : 0); j < k; j++)
                    mbar_wait(&full_bar[tile_stage(j)], tile_phase(j));
            }
        }
        return;
    }

    // consumers: group grp takes the CTA's tiles k = grp, grp + kGroups, ...; within a
    // tile, lane p owns the column pair p and warp wig the rows [5 wig, 5 wig + 5)
    const int grp = (warp - 1) / kGroupWarps, wig = (warp - 1) % kGroupWarps;
    const int gt = wig * 32 + lane;   // thread index within the group
    const int p = lane;
    for (unsigned k = grp, t = blockIdx.x + grp * gridDim.x; t < ntile; k += kGroups, t += kGroups * gridDim.x) {
        const int stage = tile_stage(k);
        if (!mbar_wait(&full_bar[stage], tile_phase(k))) {
            atomicExch(a.err, 1);
            return;
        }
        int bx, bz, s;
        tile_coords(t, a, bx, bz, s);
        const int x0 = bx * kTX, z0 = bz * kTZ;
        const float *hx = reinterpret_cast<const float *>(smem + stage * kStageBytes);
        const float *hz = hx + kHaloPad / 4;
        const float *px = hx + 2 * kHaloPad / 4;
        const float *pz = px + kPlainBytes / 4;
        const FacCoef<float> *cf = reinterpret_cast<const FacCoef<float> *>(px + 2 * kPlainBytes / 4);
        // receiver samples of level m on the surface band (halo row 1 is grid row 0)
        if (z0 == 0)
            for (int q = gt; q < 2 * g.nrec; q += 32 * kGroupWarps) {
                const int xr = a.rec[q >> 1] - x0;
                if (xr >= 0 && xr < kTX)
                    a.trace[((size_t)s * g.nlev + a.m) * g.nrec * 2 + q] = ((q & 1) ? hz : hx)[kWX + xr + kHX];
            }
        const int x = x0 + 2 * p;
        if (x < g.nx) {
            const int kind = (x == 0 ? 1 : 0) | (x + 1 == g.nx - 1 ? 2 : 0) | (x == g.nx - 1 ? 4 : 0);
            const SourceDesc<float> *sd = a.src + s;
            const int siA = x - sd->i0, siB = x + 1 - sd->i0;
            const bool scolA = (unsigned)siA < (unsigned)kPatch;
            const bool scolB = x + 1 < g.nx && (unsigned)siB < (unsigned)kPatch;
            const float S = (scolA || scolB) ? a.stf[(size_t)s * g.nsteps + a.m] : 0.0f;
            float *gx = a.nxt + (size_t)s * g.solve_stride;
            float *gz = gx + g.comp_stride;
            const int r0 = wig * kRowsPerSeg;
            Row2 rn, rc, rs;
            tile_row(hx, hz, r0, p, rn);       // grid row z0 + r0 - 1
            tile_row(hx, hz, r0 + 1, p, rc);   // grid row z0 + r0
            south(rn, rc);
#pragma unroll
            for (int r = r0; r < r0 + kRowsPerSeg; r++) {
                const int z = z0 + r;
                if (z >= g.nz) break;
                tile_row(hx, hz, r + 2, p, rs);
                south(rc, rs);
                const float2 ux = *reinterpret_cast<const float2 *>(px + r * kTX + 2 * p);
                const float2 uz = *reinterpret_cast<const float2 *>(pz + r * kTX + 2 * p);
                float4 u = make_float4(ux.x, uz.x, ux.y, uz.y);
                const FacCoef<float> K = cf[r];
                if (z == g.nz - 1) {
                    absorbing(K.cp, K.cs, make_float4(rn.xa, rn.za, rn.xb, rn.zb), rc, true, kind, u);
                } else if (z == 0) {   // surface row: no north differences, cross terms on the row itself
                    Row2 nt = rc;
                    nt.vxa = nt.vxb = nt.vza = nt.vzb = 0.0f;
                    pair_update(K, nt, rc, rs, u);
                    if (kind) absorbing(K.cp, K.cs, u, rc, false, kind, u);
                } else {
                    pair_update(K, rn, rc, rs, u);
                    if (kind) absorbing(K.cp, K.cs, u, rc, false, kind, u);
                }
                const int b = z - sd->j0;
                if ((unsigned)b < (unsigned)kPatch) {   // force term on the patch nodes (zero off it)
                    if (scolA) {
                        u.x = add_force(u.x, S, sd->wx[b * kPatch + siA]);
                        u.y = add_force(u.y, S, sd->wz[b * kPatch + siA]);
                    }
                    if (scolB) {
                        u.z = add_force(u.z, S, sd->wx[b * kPatch + siB]);
                        u.w = add_force(u.w, S, sd->wz[b * kPatch + siB]);
                    }
                }
                const size_t o = (size_t)z * g.xp + x;
                __stcs(reinterpret_cast<float2 *>(gx + o), make_float2(u.x, u.z));
                __stcs(reinterpret_cast<float2 *>(gz + o), make_float2(u.y, u.w));
                rn = rc;
                rc = rs;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[stage]);
    }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map over the [2 nsolve][nz][xp] FP32 planes of one wavefield level, with
// copy boxes of bx columns by bz rows.
bool tma_make_map(CUtensorMap *map, void *base, const Geometry &g, int nsolve, int bx, int bz)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.xp, (cuuint64_t)g.nz, (cuuint64_t)(2 * nsolve)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.xp * 4, (cuuint64_t)g.xp * g.nz * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)bz, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_make_paired_map(CUtensorMap *map, void *base, const Geometry &g, int nsolve, int bslots, int bz)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const int sq = paired_sq(g);
    const cuuint64_t dims[4] = {(cuuint64_t)(2 * sq), 2, (cuuint64_t)g.nz, (cuuint64_t)nsolve};
    const cuuint64_t strides[3] = {(cuuint64_t)sq * 8, (cuuint64_t)sq * 16, (cuuint64_t)paired_stride(g) * 4};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * bslots), 2, (cuuint32_t)bz, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_wait_selftest(const oed_ctx *ctx, unsigned long long limit_ns, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(ctx->d_err, limit_ns);
    return cudaGetLastError();
}

bool tma_supported(const oed_ctx *ctx)
{
    return ctx->precision == OED_FP32 && encode_fn() != nullptr;
}

// Launch limits and the persistent grid size (outside any stream capture).
int tma_prepare(oed_ctx *ctx)
{
    const int smem = kSmemBytes;
    if (cudaFuncSetAttribute(k_step_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_tma, 32 * (kConsumerWarps + 1), smem) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    ctx->tma_ctas = nsm * per_sm;
    return ctx->tma_ctas;
}

// Record ev on st, as an external event node when st is being captured into a graph.
void tma_record(cudaEvent_t ev, cudaStream_t st)
{
    if (!ev) return;
    cudaStreamCaptureStatus cs;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

static void tma_args(const oed_ctx *ctx, int nsolve, TmaArgs &a)
{
    a.fac = (const FacCoef<float> *)ctx->d_fac;
    a.src = (const SourceDesc<float> *)ctx->d_src;
    a.stf = (const float *)ctx->d_stf;
    a.trace = (float *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.err = ctx->d_err;
    a.g = ctx->g;
    a.nsolve = nsolve;
    a.nbx = (ctx->g.nx + kTX - 1) / kTX;
    a.nbz = (ctx->g.nz + kTZ - 1) / kTZ;
}

// One step m of nsolve solves with the one-step kernel on explicit levels: u^m in cur,
// u^{m-1} in nxt, overwritten with u^{m+1}.
cudaError_t launch_tma_one_step(const oed_ctx *ctx, int nsolve, cudaStream_t st, float *cur, float *nxt, int m)
{
    CUtensorMap halo, plain;
    if (!tma_make_map(&halo, cur, ctx->g, nsolve, kWX, kWZ) || !tma_make_map(&plain, nxt, ctx->g, nsolve, kTX, kTZ))
        return cudaErrorInvalidValue;
    if (ctx->tma_ctas < 1) return cudaErrorInvalidConfiguration;
    TmaArgs a;
    tma_args(ctx, nsolve, a);
    const long long ntile = (long long)nsolve * a.nbx * a.nbz;
    if (ntile >= (1LL << 31) - 2LL * ctx->tma_ctas) return cudaErrorInvalidValue;
    const int grid = (int)(ntile < (long long)ctx->tma_ctas ? ntile : (long long)ctx->tma_ctas);
    a.nxt = nxt;
    a.m = m;
    k_step_tma<<<grid, 32 * (kConsumerWarps + 1), kSmemBytes, st>>>(a, halo, plain);
    return cudaGetLastError();
}

// All steps of nsolve solves with the TMA kernel (the caller zeroes the levels).
cudaError_t launch_steps_tma(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                             cudaEvent_t ev1, int nsteps_override)
{
    const Geometry &g = ctx->g;
    CUtensorMap halo0, halo1, plain0, plain1;
    if (!tma_make_map(&halo0, ctx->d_u0, g, nsolve, kWX, kWZ) || !tma_make_map(&halo1, ctx->d_u1, g, nsolve, kWX, kWZ) ||
        !tma_make_map(&plain0, ctx->d_u0, g, nsolve, kTX, kTZ) || !tma_make_map(&plain1, ctx->d_u1, g, nsolve, kTX, kTZ))
        return cudaErrorInvalidValue;
    const int smem = kSmemBytes;
    if (ctx->tma_ctas < 1) return cudaErrorInvalidConfiguration;
    TmaArgs a;
    a.fac = (const FacCoef<float> *)ctx->d_fac;
    a.src = (const SourceDesc<float> *)ctx->d_src;
    a.stf = (const float *)ctx->d_stf;
    a.trace = (float *)ctx->d_trace;
    a.rec = ctx->d_rec;
    a.err = ctx->d_err;
    a.g = g;
    a.nsolve = nsolve;
    a.nbx = (g.nx + kTX - 1) / kTX;
    a.nbz = (g.nz + kTZ - 1) / kTZ;
    const long long ntile = (long long)nsolve * a.nbx * a.nbz;
    if (ntile >= (1LL << 31) - 2LL * ctx->tma_ctas) return cudaErrorInvalidValue;   // 32-bit tile indices
    const int grid = (int)(ntile < (long long)ctx->tma_ctas ? ntile : (long long)ctx->tma_ctas);
    const int nsteps = (nsteps_override > 0 && nsteps_override < g.nsteps) ? nsteps_override : g.nsteps;
    float *u0 = (float *)ctx->d_u0, *u1 = (float *)ctx->d_u1;
    if (ev0) {
        cudaStreamCaptureStatus cs;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal);
        else
            cudaEventRecord(ev0, st);
    }
    for (int m = 0; m < nsteps; m++) {
        a.nxt = (m & 1) ? u0 : u1;
        a.m = m;
        k_step_tma<<<grid, 32 * (kConsumerWarps + 1), smem, st>>>(a, (m & 1) ? halo1 : halo0,
                                                                  (m & 1) ? plain0 : plain1);
    }
    if (ev1) {
        cudaStreamCaptureStatus cs;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
        else
            cudaEventRecord(ev1, st);
    }
    return cudaGetLastError();
}

}  // namespace oed
