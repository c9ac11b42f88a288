// Scaled log-determinant, per-node information gain and quadrature sums (FP64).
//
//   S = sqrt(diag H_1), Ht = S^-1 H_1 S^-1 (Sec. 3.3.3: the scaling that takes the
//   condition number from ~1e30 to O(10)), Ht = L L^T (Cholesky),
//   log det H_1 = sum_i log H_ii + 2 sum_i log L_ii,
//   D_KL-hat = 1/2 log det H_1 - N/2 log(2 pi) - N/2 - h(theta)   (Thm 4, Eq. DKL_hat)
//   with the uniform-prior log-density h = -sum_j log(hi_j - lo_j),
//   EIG = sum_i w_i D_i                                          (Eqs. intpoly / mcs).
// Sums run in a fixed order, so a result does not depend on scheduling.
#include "oed_internal.cuh"

namespace oed {

// Returns 0 and *logdet, or 1 if H is not positive definite (or not finite).
// H is read through an accessor so both the full 7x7 and the packed 28 forms work;
// K is the order (7, or the number of unknown parameters of a subset).
template <int K, typename Get>
__device__ int scaled_logdet_k(Get Hij, double *logdet)
{
    double S[K], L[K][K];
    double ld = 0.0;
#pragma unroll
    for (int i = 0; i < K; i++) {
        const double d = Hij(i, i);
        if (!(d > 0.0) || !isfinite(d)) return 1;
        S[i] = sqrt(d);
        ld += log(d);
    }
#pragma unroll
    for (int j = 0; j < K; j++) {
        double s = Hij(j, j) / (S[j] * S[j]);
#pragma unroll
        for (int k = 0; k < j; k++) s -= L[j][k] * L[j][k];
        if (!(s > 0.0) || !isfinite(s)) return 1;
        const double ljj = sqrt(s);
        L[j][j] = ljj;
        ld += 2.0 * log(ljj);
#pragma unroll
        for (int i = j + 1; i < K; i++) {
            double t = Hij(i, j) / (S[i] * S[j]);
#pragma unroll
            for (int k = 0; k < j; k++) t -= L[i][k] * L[j][k];
            L[i][j] = t / ljj;
        }
    }
    *logdet = ld;
    return 0;
}

template <typename Get>
__device__ int scaled_logdet7(Get Hij, double *logdet)
{
    return scaled_logdet_k<kNT>(Hij, logdet);
}

// log det of the sub-block of the unknown parameters idx[0..k) of a 7x7 H
template <typename Get>
__device__ int scaled_logdet_sub(Get Hij, const int *idx, int k, double *logdet)
{
    auto sub = [&](int a, int b) { return Hij(idx[a], idx[b]); };
    switch (k) {
    case 1: return scaled_logdet_k<1>(sub, logdet);
    case 2: return scaled_logdet_k<2>(sub, logdet);
    case 3: return scaled_logdet_k<3>(sub, logdet);
    case 4: return scaled_logdet_k<4>(sub, logdet);
    case 5: return scaled_logdet_k<5>(sub, logdet);
    case 6: return scaled_logdet_k<6>(sub, logdet);
    default: return scaled_logdet_k<7>(sub, logdet);
    }
}

__device__ __forceinline__ int upper_index(int a, int b)
{
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    return a * kNT - a * (a - 1) / 2 + (b - a);
}

// D_KL-hat from log det H_1 of k unknown parameters: 1/2 logdet - k/2 (log 2 pi + 1) + logvol
__device__ __forceinline__ double dkl_from_logdet(double ld, double logvol, int k = kNT)
{
    const double c = 0.5 * k * (1.8378770664093453 + 1.0);   // k/2 (log(2 pi) + 1)
    return 0.5 * ld - c + logvol;
}

// Whole quadrature in one block, deterministic: thread t takes the contiguous node
// slice [t*per, (t+1)*per), computes each node's log-determinant and gain in order,
// then the block adds the per-thread sums with a fixed tree.
// pmask: bit j set = parameter j unknown (the others are known and drop out).
__global__ void __launch_bounds__(1024) k_eig(const double *__restrict__ H, int n,
                                              const double *__restrict__ w, double logvol, int pmask,
                                              double *__restrict__ eig, double *__restrict__ dkl,
                                              int *__restrict__ status, int *__restrict__ n_bad)
{
    __shared__ double sv[1024];
    __shared__ int sb[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (n + T - 1) / T;
    int idx[kNT], k = 0;
#pragma unroll
    for (int j = 0; j < kNT; j++)
        if (pmask >> j & 1) idx[k++] = j;
    double v = 0.0;
    int b = 0;
    for (int i = t * per; i < (t + 1) * per && i < n; i++) {
        const double *h = H + (size_t)i * 49;
        double ld = 0.0;
        const int bad = k == kNT ? scaled_logdet7([&](int x, int y) { return h[x * 7 + y]; }, &ld)
                                 : scaled_logdet_sub([&](int x, int y) { return h[x * 7 + y]; }, idx, k, &ld);
        const double D = bad ? 0.0 : dkl_from_logdet(ld, logvol, k);
        if (!bad) v += w[i] * D;
        b += bad;
        if (dkl) dkl[i] = D;
        if (status) status[i] = bad ? OED_ENOTPD : 0;
    }
    sv[t] = v;
    sb[t] = b;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if (t < s) {
            sv[t] += sv[t + s];
            sb[t] += sb[t + s];
        }
        __syncthreads();
    }
    if (t == 0) {
        *eig = sv[0];
        if (n_bad) *n_bad = sb[0];
    }
}

// One block per design: every thread takes nodes i = t, t + T, ..., builds
// H = sum over the design's receivers of H_rec[i][r][win], and accumulates w_i D_i.
__global__ void __launch_bounds__(256) k_designs(const double *__restrict__ H_rec, int n, int nrec,
                                                 int nwin, int win,
                                                 const unsigned char *__restrict__ mask,
                                                 const double *__restrict__ w, double logvol,
                                                 double *__restrict__ eig, int *__restrict__ n_bad)
{
    const int d = blockIdx.x;
    extern __shared__ int sel[];   // receivers of this design, then reduction scratch
    __shared__ int nsel;
    __shared__ double sv[256];
    __shared__ int sb[256];
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < nrec; r++)
            if (mask[(size_t)d * nrec + r]) sel[c++] = r;
        nsel = c;
    }
    __syncthreads();
    double v = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double h[28];
#pragma unroll
        for (int k = 0; k < 28; k++) h[k] = 0.0;
        for (int q = 0; q < nsel; q++) {
            const double *p = H_rec + (((size_t)i * nrec + sel[q]) * nwin + win) * 28;
#pragma unroll
            for (int k = 0; k < 28; k++) h[k] += p[k];
        }
        double ld = 0.0;
        const int b = scaled_logdet7([&](int a, int c) { return h[upper_index(a, c)]; }, &ld);
        if (b)
            bad++;
        else
            v += w[i] * dkl_from_logdet(ld, logvol);
    }
    sv[threadIdx.x] = v;
    sb[threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sv[threadIdx.x] += sv[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        eig[d] = sv[0];
        if (n_bad) n_bad[d] = sb[0];
    }
}

// One Newton step per node on the cost L (Thm 1's estimator) over the unknown
// parameters F (bit j of pmask): solve H_FF d = -grad_F with the scaled Cholesky of
// H_FF (S^-1 H_FF S^-1 = L L^T), theta_F += d, clamped to the prior box; the known
// parameters are left alone.  A node whose H_FF is not positive definite keeps its
// theta (status OED_ENOTPD).
__global__ void k_newton(const double *__restrict__ H, const double *__restrict__ grad, int n, int pmask,
                         const double *__restrict__ lohi, double *__restrict__ theta, int *__restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int idx[kNT], k = 0;
    for (int j = 0; j < kNT; j++)
        if (pmask >> j & 1) idx[k++] = j;
    const double *h = H + (size_t)i * 49;
    auto Hf = [&](int a, int b) { return h[idx[a] * kNT + idx[b]]; };
    double S[kNT], L[kNT][kNT], y[kNT];
    int bad = 0;
    for (int a = 0; a < k; a++) {
        const double d = Hf(a, a);
        bad |= !(d > 0.0) || !isfinite(d);
        S[a] = bad ? 1.0 : sqrt(d);
    }
    for (int j = 0; j < k && !bad; j++) {
        double s = Hf(j, j) / (S[j] * S[j]);
        for (int c = 0; c < j; c++) s -= L[j][c] * L[j][c];
        if (!(s > 0.0) || !isfinite(s)) {
            bad = 1;
            break;
        }
        L[j][j] = sqrt(s);
        for (int r = j + 1; r < k; r++) {
            double t = Hf(r, j) / (S[r] * S[j]);
            for (int c = 0; c < j; c++) t -= L[r][c] * L[j][c];
            L[r][j] = t / L[j][j];
        }
    }
    if (!bad) {
        // (S L L^T S) d = -grad_F:  L z = -S^-1 grad_F, L^T e = z, d = S^-1 e
        for (int a = 0; a < k; a++) {
            double t = -grad[(size_t)i * kNT + idx[a]] / S[a];
            for (int c = 0; c < a; c++) t -= L[a][c] * y[c];
            y[a] = t / L[a][a];
        }
        for (int a = k - 1; a >= 0; a--) {
            double t = y[a];
            for (int c = a + 1; c < k; c++) t -= L[c][a] * y[c];
            y[a] = t / L[a][a];
        }
        for (int a = 0; a < k; a++) {
            const int j = idx[a];
            const double v = theta[(size_t)i * kNT + j] + y[a] / S[a];
            theta[(size_t)i * kNT + j] = fmin(fmax(v, lohi[j]), lohi[kNT + j]);
        }
    }
    if (status) status[i] = bad ? OED_ENOTPD : 0;
}

void launch_newton(const double *H, const double *grad, int n, int pmask, const double *lohi, double *theta,
                   int *status, cudaStream_t s)
{
    if (n > 0) k_newton<<<(n + 127) / 128, 128, 0, s>>>(H, grad, n, pmask, lohi, theta, status);
}

struct LoHi {
    double v[2 * kNT];
};

__global__ void k_nodes_mc_v(const double *__restrict__ u, int M, LoHi lh, double *__restrict__ theta,
                             double *__restrict__ w)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * kNT) return;
    const int j = k % kNT;
    theta[k] = lh.v[j] + (lh.v[kNT + j] - lh.v[j]) * u[k];
    if (j == 0) w[k / kNT] = 1.0 / M;
}

void launch_eig(const double *H, int n, const double *w, double logvol, int pmask, double *eig,
                double *dkl, int *status, int *n_bad, cudaStream_t s)
{
    k_eig<<<1, 1024, 0, s>>>(H, n, w, logvol, pmask, eig, dkl, status, n_bad);
}

void launch_eig_designs(const double *H_rec, int n, int nrec, int nwin, int win,
                        const unsigned char *mask, int ndesign, const double *w, double logvol,
                        double *eig, int *n_bad, cudaStream_t s)
{
    if (ndesign <= 0) return;
    k_designs<<<ndesign, 256, sizeof(int) * nrec, s>>>(H_rec, n, nrec, nwin, win, mask, w, logvol,
                                                      eig, n_bad);
}

void launch_nodes_mc(const double *u, int M, const double *lo, const double *hi, double *theta,
                     double *w, cudaStream_t s)
{
    LoHi lh;
    for (int j = 0; j < kNT; j++) {
        lh.v[j] = lo[j];
        lh.v[kNT + j] = hi[j];
    }
    if (M > 0) k_nodes_mc_v<<<(M * kNT + 255) / 256, 256, 0, s>>>(u, M, lh, theta, w);
}

}  // namespace oed
