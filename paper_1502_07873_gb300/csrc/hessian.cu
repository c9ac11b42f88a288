// Central finite-difference Jacobian and Gauss-Newton Hessian
// H_1 = sum_{m,r} J_{m,r}^T C_eps^-1 J_{m,r}, C_eps = sigma^2 I
// (Thm 2 Eq. H1; Eq. H1_numerics; Appendix C: H_1 is a sum over receivers and
// time levels of rank-one terms, so per-receiver and per-window partial sums add up).
//
// Seismograms of the solves of a node sit in trace[s][m][r][c] (stencil
// precision).  Pairs form (15 solves per node): the Jacobian column j is formed
// in FP64 from the +/- pair, J_j = (g_{+j} - g_{-j}) / (2 d_j).  Difference form
// (7 solves per node): solve j already holds g_{+j} - g_{-j} (its forcing is the
// FP64 difference of the two forcings), so J_j = g_j / (2 d_j).  The 28 unique
// products are accumulated in FP64.  One block handles one
// node and one time sub-segment; its threads walk the flattened (m, r, c) rows so
// that a warp reads consecutive (r, c) of the same level (coalesced), and each
// thread keeps a single (r, c) so its 28 partial sums belong to one receiver.
#include "oed_internal.cuh"

namespace oed {

struct HArgs {
    double inv2d[kNT];      // 1 / (2 d_j)
    int sub_m0[16];         // sub-segment level ranges [m0, m1)
    int sub_m1[16];
    int win_sub_end[16];    // window w ends with sub-segment win_sub_end[w] - 1
    int nsub;
};

template <typename real, bool DIFF>
__global__ void __launch_bounds__(512) k_hsub(const real *__restrict__ trace, Geometry g,
                                              HArgs a, double *__restrict__ hsub)
{
    const int node = blockIdx.x, sub = blockIdx.y;
    const int nq = 2 * g.nrec;                // (r, c) pairs per level
    const int lanes = blockDim.x / nq;        // threads per (r, c)
    const int t = threadIdx.x;
    const int q = t % nq, mo = t / nq;
    double acc[28];
#pragma unroll
    for (int k = 0; k < 28; k++) acc[k] = 0.0;
    const size_t per_solve = (size_t)g.nlev * nq;
    const real *base = trace + (size_t)node * (DIFF ? kND : kNP) * per_solve;
    if (mo < lanes) {
        for (int m = a.sub_m0[sub] + mo; m < a.sub_m1[sub]; m += lanes) {
            const size_t off = (size_t)m * nq + q;
            double J[kNT];
#pragma unroll
            for (int j = 0; j < kNT; j++) {
                if (DIFF) {
                    J[j] = (double)base[(size_t)j * per_solve + off] * a.inv2d[j];
                } else {
                    const double gp = (double)base[(size_t)(1 + 2 * j) * per_solve + off];
                    const double gm = (double)base[(size_t)(2 + 2 * j) * per_solve + off];
                    J[j] = (gp - gm) * a.inv2d[j];
                }
            }
            int k = 0;
#pragma unroll
            for (int x = 0; x < kNT; x++)
#pragma unroll
                for (int y = x; y < kNT; y++) acc[k++] += J[x] * J[y];
        }
    }
    // the two components of a receiver sit in neighbouring threads of one warp (q = 2r + c
    // and nq is even): a shuffle adds them (x + z, the order of the sum below), then the
    // receiver's partial sums over the lanes are added in shared memory
    const int wbase = t & ~31;
    const int nact = min(32, (int)blockDim.x - wbase);
    const unsigned mask = nact == 32 ? 0xffffffffu : ((1u << nact) - 1u);
#pragma unroll
    for (int k = 0; k < 28; k++) acc[k] += __shfl_xor_sync(mask, acc[k], 1);
    extern __shared__ double sh[];   // [lanes][nrec][29] (padded)
    const int nrec = g.nrec;
    if (mo < lanes && (q & 1) == 0)
#pragma unroll
        for (int k = 0; k < 28; k++) sh[(mo * nrec + (q >> 1)) * 29 + k] = acc[k];
    __syncthreads();
    for (int w = t; w < nrec * 28; w += blockDim.x) {
        const int r = w / 28, k = w % 28;
        double v = 0.0;
        for (int l = 0; l < lanes; l++) v += sh[(l * nrec + r) * 29 + k];
        hsub[(((size_t)node * a.nsub + sub) * nrec + r) * 28 + k] = v;
    }
}

// Sum the sub-segments into per-receiver cumulative windows and the total H.
template <typename real>
__global__ void k_hcombine(const double *__restrict__ hsub, Geometry g, double s2, int nwin, HArgs a,
                           int per_node, const SourceDesc<real> *__restrict__ src, double *__restrict__ H,
                           double *__restrict__ H_rec, int *__restrict__ status,
                           const int *__restrict__ err)
{
    const int node = blockIdx.x;
    const int nrec = g.nrec;
    const int nsub = a.nsub;
    __shared__ double tot[28];
    __shared__ int ok;
    if (threadIdx.x < 28) tot[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) {
        int o = 1;
        for (int p = 0; p < per_node; p++) o &= src[(size_t)node * per_node + p].ok;
        ok = *err ? -1 : o;   // -1: a bounded wait in the time loop expired
    }
    __syncthreads();
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    // per receiver, per window (cumulative over sub-segments), and the total
    for (int w = threadIdx.x; w < nrec * 28; w += blockDim.x) {
        const int r = w / 28, k = w % 28;
        double run = 0.0;
        int next = 0;
        for (int sub = 0; sub < nsub; sub++) {
            run += hsub[(((size_t)node * nsub + sub) * nrec + r) * 28 + k];
            while (next < nwin && a.win_sub_end[next] == sub + 1) {
                if (H_rec)
                    H_rec[(((size_t)node * nrec + r) * nwin + next) * 28 + k] = ok == 1 ? s2 * run : nan;
                next++;
            }
        }
    }
    // total over receivers and sub-segments in a fixed order (28 threads)
    if (threadIdx.x < 28) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int r = 0; r < nrec; r++)
            for (int sub = 0; sub < nsub; sub++)
                v += hsub[(((size_t)node * nsub + sub) * nrec + r) * 28 + k];
        tot[k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 49) {
        const int x = threadIdx.x / 7, y = threadIdx.x % 7;
        const int a0 = x < y ? x : y, b0 = x < y ? y : x;
        const int k = a0 * 7 - a0 * (a0 - 1) / 2 + (b0 - a0);
        H[(size_t)node * 49 + threadIdx.x] = ok == 1 ? s2 * tot[k] : nan;
    }
    if (threadIdx.x == 0 && status) status[node] = ok == 1 ? 0 : (ok < 0 ? OED_ETIMEOUT : OED_EINVAL);
}

int hsub_threads(int nrec);

void launch_hessian(const oed_ctx *ctx, int nnode, const double *inv2d, double sigma,
                    const int *seg_end, int nseg, const int *win_seg, int nwin, double *H,
                    double *H_rec, int *status, cudaStream_t st)
{
    // Split the level range into at most 16 sub-segments that respect the window
    // boundaries seg_end[0..nseg) (seg_end[nseg-1] = nlev), enough for >= ~4 blocks per SM.
    const Geometry &g = ctx->g;
    HArgs a;
    for (int j = 0; j < kNT; j++) a.inv2d[j] = inv2d[j];
    int want = 16;
    int per = want / nseg;
    if (per < 1) per = 1;
    int nsub = 0;
    int m0 = 0;
    for (int sgi = 0; sgi < nseg; sgi++) {
        const int m1 = seg_end[sgi];
        const int len = m1 - m0;
        int parts = per < len ? per : (len > 0 ? len : 1);
        if (nsub + parts > 16 - (nseg - 1 - sgi)) parts = 16 - (nseg - 1 - sgi) - nsub;
        if (parts < 1) parts = 1;
        for (int p = 0; p < parts; p++) {
            a.sub_m0[nsub] = m0 + (int)((long long)len * p / parts);
            a.sub_m1[nsub] = m0 + (int)((long long)len * (p + 1) / parts);
            nsub++;
        }
        for (int w = 0; w < nwin; w++)
            if (win_seg[w] == sgi) a.win_sub_end[w] = nsub;
        m0 = m1;
    }
    a.nsub = nsub;
    const int threads = hsub_threads(g.nrec);
    const size_t smem = (size_t)(threads / 2) * 29 * sizeof(double);   // one row per (lane, receiver)
    dim3 grid(nnode, nsub);
    const bool diff = ctx->jac_mode != OED_JAC_PAIRS;   // one solve per parameter
    if (ctx->precision == OED_FP64) {
        if (diff)
            k_hsub<double, true><<<grid, threads, smem, st>>>((const double *)ctx->d_trace, g, a, ctx->d_hseg);
        else
            k_hsub<double, false><<<grid, threads, smem, st>>>((const double *)ctx->d_trace, g, a, ctx->d_hseg);
    } else {
        if (diff)
            k_hsub<float, true><<<grid, threads, smem, st>>>((const float *)ctx->d_trace, g, a, ctx->d_hseg);
        else
            k_hsub<float, false><<<grid, threads, smem, st>>>((const float *)ctx->d_trace, g, a, ctx->d_hseg);
    }
    const double s2 = 1.0 / (sigma * sigma);
    const int per_node = diff ? kND : kNP;
    if (ctx->precision == OED_FP64)
        k_hcombine<double><<<nnode, 256, 0, st>>>(ctx->d_hseg, g, s2, nwin, a, per_node,
                                                  (const SourceDesc<double> *)ctx->d_src, H, H_rec,
                                                  status, ctx->d_err);
    else
        k_hcombine<float><<<nnode, 256, 0, st>>>(ctx->d_hseg, g, s2, nwin, a, per_node,
                                                 (const SourceDesc<float> *)ctx->d_src, H, H_rec,
                                                 status, ctx->d_err);
}

int hsub_threads(int nrec)
{
    const int nq = 2 * nrec;
    int lanes = 128 / nq;
    if (lanes < 1) lanes = 1;
    return lanes * nq;
}

void hessian_init(cudaStream_t)
{
    const int smem = 512 * 29 * (int)sizeof(double);
    cudaFuncSetAttribute(k_hsub<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_hsub<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_hsub<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_hsub<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace oed
