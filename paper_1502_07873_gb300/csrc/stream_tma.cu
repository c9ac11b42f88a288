// Streaming leap-frog step with TMA tile loads (one launch per time step, for
// grids whose wavefield does not fit the cluster-resident kernel; Sec. 3.3.1,
// Eq. Full_Disc; node update from stencil_cell.cuh).
//
// A persistent CTA walks tiles (solve, 16-row band, 64-column band) of the batch.
// Its producer warp issues, for each tile, four cp.async.bulk.tensor loads into one
// stage of a shared-memory ring: u_x and u_z of level m with a halo (rows z0-1 ..
// z0+16, columns x0-4 .. x0+67; the x start stays a multiple of four floats so
// every copy starts on a 16-byte boundary, the grid edges read as zeros and are
// never used) and u_x, u_z of level m-1 without halo.  Completion is tracked by
// an mbarrier per stage (expect_tx of the stage's bytes); the consumer warps wait
// on it, compute the tile from shared memory with a register window per column,
// store u^{m+1} with streaming stores over u^{m-1}, and release the stage on a
// second mbarrier.  Every wait is bounded: on expiry the kernel raises a device
// flag, the producer waits (bounded) for its copies in flight, and the threads
// return; the flag turns the affected nodes' status into OED_ETIMEOUT.
// HBM traffic per cell-update is the algorithmic 24 B (FP32); the halo re-reads
// come from L2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "stencil_cell.cuh"

namespace oed {

constexpr int kTX = 64, kTZ = 16, kHX = 4;
constexpr int kWX = kTX + 2 * kHX, kWZ = kTZ + 2;
constexpr int kStages = 4;
constexpr int kConsumerWarps = 8;                       // 64 columns x 4 segments of 4 rows
constexpr int kRowsPerSeg = kTZ / (kConsumerWarps / 2); // 4
constexpr int kHaloBytes = kWX * kWZ * 4;               // 5184
constexpr int kHaloPad = (kHaloBytes + 127) / 128 * 128;  // 5248
constexpr int kPlainBytes = kTX * kTZ * 4;              // 4096
constexpr int kStageBytes = 2 * kHaloPad + 2 * kPlainBytes;
constexpr unsigned kTxBytes = 2 * kHaloBytes + 2 * kPlainBytes;
constexpr unsigned long long kWaitLimitNs = 2000000000ULL;   // 2 s per wait
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

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((unsigned)__cvta_generic_to_shared(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase with the given parity, bounded by kWaitLimitNs; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int y, int z,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z),
        "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
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
    const long long ntile = (long long)a.nsolve * a.nbz * a.nbx;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // producer
        if (lane == 0) {
            long long k = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntile; t += gridDim.x, k++) {
                const int stage = (int)(k % kStages);
                const unsigned phase = (unsigned)((k / kStages) & 1);
                if (k >= kStages && !mbar_wait(&empty_bar[stage], phase ^ 1u)) {
                    ok = false;
                    break;
                }
                const int bx = (int)(t % a.nbx);
                const int bz = (int)((t / a.nbx) % a.nbz);
                const int s = (int)(t / ((long long)a.nbx * a.nbz));
                const int x0 = bx * kTX, z0 = bz * kTZ;
                unsigned char *st = smem + stage * kStageBytes;
                mbar_expect_tx(&full_bar[stage], kTxBytes);
                tma_load3(st, &cur_halo, x0 - kHX, z0 - 1, 2 * s, &full_bar[stage]);
                tma_load3(st + kHaloPad, &cur_halo, x0 - kHX, z0 - 1, 2 * s + 1, &full_bar[stage]);
                tma_load3(st + 2 * kHaloPad, &nxt_plain, x0, z0, 2 * s, &full_bar[stage]);
                tma_load3(st + 2 * kHaloPad + kPlainBytes, &nxt_plain, x0, z0, 2 * s + 1, &full_bar[stage]);
            }
            if (!ok) {
                atomicExch(a.err, 1);
                // copies already issued for the last stages must land before the CTA exits
                for (long long j = (k > kStages ? k - kStages : 0); j < k; j++)
                    mbar_wait(&full_bar[j % kStages], (unsigned)((j / kStages) & 1));
            }
        }
        return;
    }

    // consumers: thread -> column cx of the tile and a segment of kRowsPerSeg rows
    const int ct = threadIdx.x - 32;
    const int cx = ct % kTX;
    const int seg = ct / kTX;
    long long k = 0;
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x, k++) {
        const int stage = (int)(k % kStages);
        const unsigned phase = (unsigned)((k / kStages) & 1);
        if (!mbar_wait(&full_bar[stage], phase)) {
            atomicExch(a.err, 1);
            return;
        }
        const int bx = (int)(t % a.nbx);
        const int bz = (int)((t / a.nbx) % a.nbz);
        const int s = (int)(t / ((long long)a.nbx * a.nbz));
        const int x0 = bx * kTX, z0 = bz * kTZ;
        const float *hx = reinterpret_cast<const float *>(smem + stage * kStageBytes);
        const float *hz = hx + kHaloPad / 4;
        const float *px = hx + 2 * kHaloPad / 4;
        const float *pz = px + kPlainBytes / 4;
        // receiver samples of level m on the surface band
        if (z0 == 0)
            for (int q = ct; q < 2 * g.nrec; q += 32 * kConsumerWarps) {
                const int xr = a.rec[q >> 1] - x0;
                if (xr >= 0 && xr < kTX)
                    a.trace[((size_t)s * g.nlev + a.m) * g.nrec * 2 + q] = ((q & 1) ? hz : hx)[kWX + xr + kHX];
            }
        const int x = x0 + cx;
        if (x < g.nx) {
            const int side = (x == 0) ? 1 : ((x == g.nx - 1) ? 2 : 0);
            const SourceDesc<float> *sd = a.src + s;
            const int si = x - sd->i0;
            const bool scol = (unsigned)si < (unsigned)kPatch;
            const float S = scol ? a.stf[(size_t)s * g.nsteps + a.m] : 0.0f;
            float *gx = a.nxt + (size_t)s * g.solve_stride;
            float *gz = gx + g.comp_stride;
            const int r0 = seg * kRowsPerSeg;
            float W[3][3], Z[3][3];
            // halo rows r0 and r0 + 1 (grid rows z0 + r0 - 1, z0 + r0)
#pragma unroll
            for (int q = 0; q < 2; q++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    W[q][c] = hx[(r0 + q) * kWX + cx + kHX - 1 + c];
                    Z[q][c] = hz[(r0 + q) * kWX + cx + kHX - 1 + c];
                }
#pragma unroll
            for (int r = r0; r < r0 + kRowsPerSeg; r++) {
                const int z = z0 + r;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    W[2][c] = hx[(r + 2) * kWX + cx + kHX - 1 + c];
                    Z[2][c] = hz[(r + 2) * kWX + cx + kHX - 1 + c];
                }
                if (z < g.nz) {
                    const FacCoef<float> K = a.fac[z];
                    float ux, uz;
                    node_update(K, W[0], W[1], W[2], Z[0], Z[1], Z[2], px[r * kTX + cx], pz[r * kTX + cx],
                                side, z == g.nz - 1, z == 0, ux, uz);
                    const int b = z - sd->j0;
                    if (scol && (unsigned)b < (unsigned)kPatch && !side && z != g.nz - 1) {
                        ux = add_force(ux, S, sd->wx[b * kPatch + si]);
                        uz = add_force(uz, S, sd->wz[b * kPatch + si]);
                    }
                    const size_t o = (size_t)z * g.xp + x;
                    __stcs(gx + o, ux);
                    __stcs(gz + o, uz);
                }
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    W[0][c] = W[1][c];
                    W[1][c] = W[2][c];
                    Z[0][c] = Z[1][c];
                    Z[1][c] = Z[2][c];
                }
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

static bool make_map(CUtensorMap *map, void *base, const Geometry &g, int nsolve, int bx, int bz)
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

// All steps of nsolve solves with the TMA kernel (the caller zeroes the levels).
cudaError_t launch_steps_tma(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                             cudaEvent_t ev1, int nsteps_override)
{
    const Geometry &g = ctx->g;
    CUtensorMap halo0, halo1, plain0, plain1;
    if (!make_map(&halo0, ctx->d_u0, g, nsolve, kWX, kWZ) || !make_map(&halo1, ctx->d_u1, g, nsolve, kWX, kWZ) ||
        !make_map(&plain0, ctx->d_u0, g, nsolve, kTX, kTZ) || !make_map(&plain1, ctx->d_u1, g, nsolve, kTX, kTZ))
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
