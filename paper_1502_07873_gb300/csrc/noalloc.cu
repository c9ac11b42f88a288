// Allocation-free Gauss-Newton Hessian from caller-provided seismograms.
//
// A variant of the Jacobian / Hessian reduction of hessian.cu for callers that
// cannot allocate device memory at run time.  Its scratch (the per node, time
// segment and receiver partial sums) lives in a file-scope device array of fixed
// size, so the call itself never allocates.  Host code obtains the array's device
// address once per device with cudaGetSymbolAddress; the host-side symbol is only
// a stand-in and is never passed to a kernel.
#include <mutex>

#include "oed_internal.cuh"

namespace oed {

constexpr int kNoAllocSub = 8;   // time sub-segments per node
static __device__ __align__(256) double g_noalloc_scratch[OED_NOALLOC_SCRATCH_DOUBLES];

struct NaArgs {
    double inv2d[kNT];
    double s2;
    int nlev, nrec, per_node, nsub;
};

// Block (node, sub-segment): threads walk the flattened (m, r, c) rows of the
// sub-segment, each keeping one (r, c), and accumulate the 28 products of the FD
// Jacobian row in FP64; partial sums per receiver go to the scratch array.
__global__ void __launch_bounds__(512) k_na_partial(const double *__restrict__ g, NaArgs a,
                                                    double *__restrict__ part)
{
    const int node = blockIdx.x, sub = blockIdx.y;
    const int nq = 2 * a.nrec;
    const int lanes = blockDim.x / nq;
    const int t = threadIdx.x, q = t % nq, mo = t / nq;
    const int m0 = (int)((long long)a.nlev * sub / a.nsub);
    const int m1 = (int)((long long)a.nlev * (sub + 1) / a.nsub);
    const size_t per_solve = (size_t)a.nlev * nq;
    const double *base = g + (size_t)node * a.per_node * per_solve;
    double acc[28];
#pragma unroll
    for (int k = 0; k < 28; k++) acc[k] = 0.0;
    if (mo < lanes) {
        for (int m = m0 + mo; m < m1; m += lanes) {
            const size_t off = (size_t)m * nq + q;
            double J[kNT];
#pragma unroll
            for (int j = 0; j < kNT; j++) {
                if (a.per_node == kND)
                    J[j] = base[(size_t)j * per_solve + off] * a.inv2d[j];
                else
                    J[j] = (base[(size_t)(1 + 2 * j) * per_solve + off] -
                            base[(size_t)(2 + 2 * j) * per_solve + off]) * a.inv2d[j];
            }
            int k = 0;
#pragma unroll
            for (int x = 0; x < kNT; x++)
#pragma unroll
                for (int y = x; y < kNT; y++) acc[k++] += J[x] * J[y];
        }
    }
    extern __shared__ double sh[];   // [blockDim.x][29]
#pragma unroll
    for (int k = 0; k < 28; k++) sh[t * 29 + k] = acc[k];
    __syncthreads();
    for (int w = t; w < a.nrec * 28; w += blockDim.x) {
        const int r = w / 28, k = w % 28;
        double v = 0.0;
        for (int l = 0; l < lanes; l++)
            v += sh[(l * nq + 2 * r) * 29 + k] + sh[(l * nq + 2 * r + 1) * 29 + k];
        part[(((size_t)node * a.nsub + sub) * a.nrec + r) * 28 + k] = v;
    }
}

// One block per node: H = sigma^-2 sum over receivers and sub-segments (fixed order).
__global__ void k_na_total(const double *__restrict__ part, NaArgs a, double *__restrict__ H)
{
    const int node = blockIdx.x;
    __shared__ double tot[28];
    if (threadIdx.x < 28) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int r = 0; r < a.nrec; r++)
            for (int sub = 0; sub < a.nsub; sub++)
                v += part[(((size_t)node * a.nsub + sub) * a.nrec + r) * 28 + k];
        tot[k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 49) {
        const int x = threadIdx.x / 7, y = threadIdx.x % 7;
        const int a0 = x < y ? x : y, b0 = x < y ? y : x;
        H[(size_t)node * 49 + threadIdx.x] = a.s2 * tot[a0 * 7 - a0 * (a0 - 1) / 2 + (b0 - a0)];
    }
}

// Device address of the scratch array, looked up once per device.
static double *scratch_address(int *rc)
{
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *rc = OED_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *rc = OED_ECUDA;
            return nullptr;
        }
        addr[dev] = static_cast<double *>(p);
    }
    *rc = OED_OK;
    return addr[dev];
}

}  // namespace oed

extern "C" int oed_gauss_newton_noalloc(const double *g, int n, int per_node, int nlev, int nrec,
                                        const double *lo, const double *hi, double rel_step,
                                        double sigma, double *H, void *stream)
{
    using namespace oed;
    if (n < 0 || (n > 0 && (!g || !H)) || !lo || !hi) return OED_EINVAL;
    if (per_node != kNP && per_node != kND) return OED_EINVAL;
    if (nlev < 1 || nrec < 1 || nrec > kMaxRecHessian) return OED_EINVAL;
    if (!(rel_step > 0) || !(sigma > 0)) return OED_EINVAL;
    NaArgs a;
    for (int j = 0; j < kNT; j++) {
        if (!(hi[j] > lo[j])) return OED_EINVAL;
        a.inv2d[j] = 1.0 / (2.0 * rel_step * (hi[j] - lo[j]));
    }
    a.s2 = 1.0 / (sigma * sigma);
    a.nlev = nlev;
    a.nrec = nrec;
    a.per_node = per_node;
    a.nsub = nlev < kNoAllocSub ? nlev : kNoAllocSub;
    if ((double)n * a.nsub * nrec * 28 > (double)OED_NOALLOC_SCRATCH_DOUBLES) return OED_ENOMEM;
    if (n == 0) return OED_OK;
    int rc = OED_OK;
    double *part = scratch_address(&rc);
    if (rc != OED_OK) return rc;
    const int nq = 2 * nrec;
    const int lanes = nq <= 128 ? 128 / nq : 1;
    const int threads = lanes * nq;
    const size_t smem = (size_t)threads * 29 * sizeof(double);
    // fixed limit (the largest block this entry point launches), so concurrent calls agree
    if (cudaFuncSetAttribute(k_na_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             512 * 29 * (int)sizeof(double)) != cudaSuccess)
        return OED_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    k_na_partial<<<dim3(n, a.nsub), threads, smem, st>>>(g, a, part);
    k_na_total<<<n, 64, 0, st>>>(part, a, H);
    return cudaGetLastError() == cudaSuccess ? OED_OK : OED_ECUDA;
}
