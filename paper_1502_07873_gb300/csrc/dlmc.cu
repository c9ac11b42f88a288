// Double-loop (nested) Monte Carlo estimate of the expected information gain, the
// direct sampling of Eq. expected_I that the Laplace method of Thm 4 replaces
// (Sec. 4.4 compares the two).  With y_n = g(theta_n) + eps_n and Gaussian noise
// C_eps = sigma^2 I,
//   log_ev[n] = log( (1/M) sum_m exp(-|y_n - g(theta'_m)|^2 / (2 sigma^2)) )
//   I_DL      = (1/N) sum_n [ -|eps_n|^2 / (2 sigma^2) - log_ev[n] ]
// (the normalising constant of the Gaussian likelihood cancels).  All in FP64, the
// squared distances summed from the differences themselves (no |y|^2 + |g|^2 - 2 y.g
// expansion, which cancels catastrophically when the noise is small).
//
// k_log_evidence: a block owns 32 outer samples and streams all inner samples in
// tiles of 64, the data dimension in chunks of 32 through shared memory; each
// thread accumulates a 2 x 4 tile of squared distances, then folds them into a
// running (max, sum of exponentials) per outer sample; the 16 threads sharing an
// outer sample combine their partial sums with shuffles at the end.
#include <math.h>

#include "oed_internal.cuh"

namespace oed {

constexpr int kDN = 32, kDM = 64, kDD = 32;

__global__ void __launch_bounds__(256) k_log_evidence(const double *__restrict__ g_out,
                                                      const double *__restrict__ eps, int N,
                                                      const double *__restrict__ g_in, int M, int D,
                                                      double inv2s2, double *__restrict__ log_ev)
{
    __shared__ double ys[kDD][kDN];
    __shared__ double gs[kDD][kDM + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int n0 = blockIdx.x * kDN;
    double mx[2] = {-INFINITY, -INFINITY}, sm[2] = {0.0, 0.0};
    for (int m0 = 0; m0 < M; m0 += kDM) {
        double acc[2][4];
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[r][q] = 0.0;
        for (int d0 = 0; d0 < D; d0 += kDD) {
            // y tile (32 x 32): y = g(theta_n) + eps_n, zero outside the data
            for (int k = tid; k < kDN * kDD; k += 256) {
                const int nn = k / kDD, dd = k % kDD;
                const int n = n0 + nn, d = d0 + dd;
                double v = 0.0;
                if (n < N && d < D) v = g_out[(size_t)n * D + d] + eps[(size_t)n * D + d];
                ys[dd][nn] = v;
            }
            for (int k = tid; k < kDM * kDD; k += 256) {
                const int mm = k / kDD, dd = k % kDD;
                const int m = m0 + mm, d = d0 + dd;
                gs[dd][mm] = (m < M && d < D) ? g_in[(size_t)m * D + d] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int dd = 0; dd < kDD; dd++) {
                const double a0 = ys[dd][2 * ty], a1 = ys[dd][2 * ty + 1];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const double b = gs[dd][tx + 16 * q];
                    const double e0 = a0 - b, e1 = a1 - b;
                    acc[0][q] = fma(e0, e0, acc[0][q]);
                    acc[1][q] = fma(e1, e1, acc[1][q]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (m0 + tx + 16 * q >= M) continue;
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const double l = -acc[r][q] * inv2s2;
                if (l > mx[r]) {
                    sm[r] = sm[r] * exp(mx[r] - l) + 1.0;
                    mx[r] = l;
                } else {
                    sm[r] += exp(l - mx[r]);
                }
            }
        }
    }
    // combine the 16 threads of each outer sample (lanes differing in the low four bits)
#pragma unroll
    for (int r = 0; r < 2; r++) {
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) {
            const double om = __shfl_xor_sync(0xffffffffu, mx[r], off);
            const double os = __shfl_xor_sync(0xffffffffu, sm[r], off);
            const double nm = fmax(mx[r], om);
            double ns = 0.0;
            if (nm > -INFINITY) ns = sm[r] * exp(mx[r] - nm) + os * exp(om - nm);
            mx[r] = nm;
            sm[r] = ns;
        }
        const int n = n0 + 2 * ty + r;
        if (tx == 0 && n < N) log_ev[n] = mx[r] + log(sm[r]) - log((double)M);
    }
}

// I_DL = (1/N) sum_n [-|eps_n|^2 inv2s2 - log_ev[n]]: one block, fixed summation order.
__global__ void __launch_bounds__(512) k_dlmc_sum(const double *__restrict__ eps, const double *__restrict__ log_ev,
                                                  int N, int D, double inv2s2, double *__restrict__ eig)
{
    __shared__ double sv[512];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (N + T - 1) / T;
    double v = 0.0;
    for (int n = t * per; n < (t + 1) * per && n < N; n++) {
        double e2 = 0.0;
        for (int d = 0; d < D; d++) e2 = fma(eps[(size_t)n * D + d], eps[(size_t)n * D + d], e2);
        v += -e2 * inv2s2 - log_ev[n];
    }
    sv[t] = v;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if (t < s) sv[t] += sv[t + s];
        __syncthreads();
    }
    if (t == 0) *eig = sv[0] / N;
}

}  // namespace oed

extern "C" int oed_dlmc(const double *g_outer, const double *eps, int N, const double *g_inner, int M, int D,
                        double sigma, double *log_ev, double *eig, void *stream)
{
    using namespace oed;
    if (N < 1 || M < 1 || D < 1 || !g_outer || !eps || !g_inner || !log_ev || !(sigma > 0.0))
        return OED_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    k_log_evidence<<<(N + kDN - 1) / kDN, 256, 0, st>>>(g_outer, eps, N, g_inner, M, D, inv2s2, log_ev);
    if (eig) k_dlmc_sum<<<1, 512, 0, st>>>(eps, log_ev, N, D, inv2s2, eig);
    return cudaGetLastError() == cudaSuccess ? OED_OK : OED_ECUDA;
}
