// Internal declarations shared by the CUDA translation units of liboed.
// Kernels and host launchers for the Laplace expected-information-gain path
// (arXiv:1502.07873); the public C ABI is include/oed.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/oed.h"

namespace oed {

constexpr int kNT = 7;    // source parameters
constexpr int kNP = 15;   // solves per node, pairs Jacobian: centre and +/- d_j e_j
constexpr int kND = 7;    // solves per node, difference Jacobian: one per parameter
constexpr int kPatch = 7; // source patch edge: the 6-point delta support, widened by one
                          // node so the difference of two shifted patches fits
constexpr int kMaxRec = 4096;      // receivers of a forward solve
constexpr int kMaxRecHessian = 256; // receivers of oed_hessian / oed_eig_designs

// Per-row stencil coefficients of the leap-frog update (Eq. Full_Disc) for a
// medium that is constant along each grid row (layered in depth).  Every
// coefficient is premultiplied by dt^2 / nu_j so the kernel adds
// coefficient * (difference of neighbours) directly to 2u^m - u^{m-1}.
//   interior rows 1..nz-2:
//     Ax = axx (x_e - 2x_c + x_w) + axzp (x_s - x_c) - axzm (x_c - x_n)
//        + lx ((z_se - z_ne) - (z_sw - z_nw)) + mxp (z_se - z_sw) - mxm (z_ne - z_nw)
//     Az = azx (z_e - 2z_c + z_w) + azzp (z_s - z_c) - azzm (z_c - z_n)
//        + mz ((x_se - x_ne) - (x_sw - x_nw)) + lzp (x_se - x_sw) - lzm (x_ne - x_nw)
//   surface row 0 (summation-by-parts closure, "s" = row 1):
//     Ax = axx (..) + axzp (x_s - x_c) + lx ((z_se - z_e) - (z_sw - z_w))
//        + mxm (z_e - z_w) + mxp (z_se - z_sw)
//     Az = azx (..) + azzp (z_s - z_c) + mz ((x_se - x_e) - (x_sw - x_w))
//        + lzm (x_e - x_w) + lzp (x_se - x_sw)
//   rf = dt^2/nu_j multiplies the force density; cp, cs = c dt / h for the
//   absorbing rows (side columns of this row; the whole bottom row).
template <typename real>
struct __align__(16 * sizeof(real)) RowCoef {
    real axx, azx, axzp, axzm, azzp, azzm, lx, mxp, mxm, mz, lzp, lzm, rf, cp, cs, pad;
};

// The same update regrouped so that FP32 rounds as little as possible at the
// scale of u itself: every neighbour enters through a difference, the operator
// term is summed at the (small) scale of those differences, onto u^m - u^{m-1},
// and u^{m+1} is formed as u^m + that sum: one rounding at the scale of u per step.
//   A_x = axx lap_x + axzp dv_s + naxzm dv_n + px dz_s + nqx dz_n
//   A_z = azx lap_z + azzp dw_s + nazzm dw_n + pz dx_s + nqz dx_n
// with lap_x = (x_e - x_c) - (x_c - x_w), dv_s = x_s - x_c, dv_n = x_c - x_n (dw for
// u_z likewise), dz_r = z_re - z_rw and dx_r = x_re - x_rw on row r, and
//   naxzm = -axzm, px = lx + mxp, nqx = -(lx + mxm),
//   nazzm = -azzm, pz = mz + lzp, nqz = -(mz + lzm)
// on interior rows.  On the surface row the north terms vanish (naxzm = nazzm = 0)
// and the cross terms use the row itself: dz_n -> dz_c, dx_n -> dx_c, with
// nqx = mxm - lx, nqz = lzm - mz.  cp, cs as in RowCoef.  Built from the FP64
// coefficients by the same kernel.
template <typename real>
struct __align__(16 * sizeof(real)) FacCoef {
    real axx, axzp, naxzm, px, nqx, azx, azzp, nazzm, pz, nqz, cp, cs, pad0, pad1, pad2, pad3;
};

// Source of one solve: corner of the 7x7 patch and the spatial force density
// f_x, f_z (Eq. source with the regularised delta / delta' of Sec. 3.3.2),
// already multiplied by dt^2/nu of the patch rows.  The forcing at step m is
// stf[m] * w.  For a difference solve w (or stf) is the FP64 difference of the
// +d_j and -d_j forcings.
template <typename real>
struct SourceDesc {
    int i0, j0, ok, pad;
    real wx[kPatch * kPatch];
    real wz[kPatch * kPatch];
};

struct Geometry {
    int nx, nz, xp;        // nodes, padded row stride (multiple of 32)
    int nsteps, nlev;      // steps, levels = nsteps + 1
    int nrec;
    double h, dt;
    size_t comp_stride;    // elements per component of one solve (nz * xp)
    size_t solve_stride;   // 2 * comp_stride
};

// The paired level layout of the two-step TMA kernel (FP32): row z of a solve holds the
// even columns' (x, z) in sq float2 slots, then the odd columns' in sq more; column c sits
// in slot (c >> 1) + 2 of its half, and the slots of columns -4 .. -1 and past nx - 1 are
// zero.  sq is even, so each half row is a multiple of 16 bytes (a TMA stride).
__host__ __device__ inline int paired_sq(const Geometry &g) { return ((g.nx + 1) / 2 + 4 + 1) & ~1; }
__host__ __device__ inline size_t paired_stride(const Geometry &g) { return (size_t)g.nz * 4 * paired_sq(g); }

struct StepTuning {
    int zs;      // streaming kernel: rows marched per thread
    int wz;      // streaming kernel: warps along z in a block
    int C;       // > 0: cluster-resident kernel with clusters of C CTAs (FP32 only);
                 // -1: TMA streaming kernel (FP32 only); -2: two-step TMA streaming
                 // kernel (FP32, grids that do not fit on chip); 0: register streaming kernel
};

}  // namespace oed

struct oed_ctx {
    oed::Geometry g;
    int precision;
    int stf = OED_STF_GAUSS;   // source time function of the problem
    int max_solves;
    int device;
    size_t elem;               // 4 or 8
    std::vector<double> z_top, vp, vs, rho;
    std::vector<int> rec_ix;
    // device workspace
    void *d_rows = nullptr;    // RowCoef<real>[nz]
    void *d_fac = nullptr;     // FacCoef<real>[nz] (same rows, factored form)
    int *d_rec = nullptr;      // [nrec]
    int *d_err = nullptr;      // device flag: a bounded wait in a kernel expired (cleared
                               // before every time loop, read when the Hessians are combined)
    void *d_u0 = nullptr;      // wavefield level buffer A [max_solves][2][nz][xp]
    void *d_u1 = nullptr;      // wavefield level buffer B
    void *d_u2 = nullptr;      // second level pair of the two-step kernel (FP32 grids
    void *d_u3 = nullptr;      // that do not fit on chip; NULL otherwise)
    void *d_kp = nullptr;      // [nz] the rows' coefficients as (x, z) pairs (two-step kernel)
    void *d_src = nullptr;     // SourceDesc<real>[max_solves]
    void *d_stf = nullptr;     // real [max_solves][nsteps]
    void *d_trace = nullptr;   // real [max_solves][nlev][nrec][2]
    double *d_theta = nullptr; // [max_solves][7] perturbed parameters
    double *d_hseg = nullptr;  // [chunk][nrec][nseg_max][28] partial Hessians
    int nseg_max = 0;
    size_t bytes = 0;
    oed::StepTuning tune{4, 4, 0};
    int jac_mode = OED_JAC_PAIRS;   // Jacobian form of oed_hessian
    int tma_ctas = 0;               // persistent grid of the TMA streaming kernel
    int tma2_ctas = 0;              // persistent grid of the two-step TMA kernel
    // host-path staging
    cudaStream_t own_stream = nullptr;
    double *h_stage_theta = nullptr, *h_stage_w = nullptr, *h_stage_H = nullptr,
           *h_stage_dkl = nullptr, *h_stage_eig = nullptr;
    int *h_stage_bad = nullptr;
    int h_stage_cap = 0;
    std::map<int, cudaGraphExec_t> graphs;   // nsolve -> captured time loop
    cudaEvent_t ev_steps[2] = {nullptr, nullptr};   // recorded around the stencil launches
    int last_steps_launches = 0;
    double *d_adj = nullptr;        // oed_hessian_ii: residual weights, then patch sums
    size_t adj_bytes = 0;
    std::string err;
};

namespace oed {

int set_err(oed_ctx *ctx, int code, const std::string &msg);
int cuda_err(oed_ctx *ctx, cudaError_t e, const char *what);

// source.cu: per_node 1 (forward), kNP (pairs Jacobian) or kND (difference Jacobian)
void launch_sources(const oed_ctx *ctx, const double *theta_nodes, int nnode, int per_node,
                    const double *step, cudaStream_t s);
inline int solves_per_node(const oed_ctx *ctx)
{
    return ctx->jac_mode == OED_JAC_PAIRS ? kNP : kND;
}
void launch_rows(oed_ctx *ctx, cudaStream_t s);

// stencil.cu
cudaError_t launch_forward_steps(const oed_ctx *ctx, int nsolve, cudaStream_t s, cudaEvent_t ev0,
                                 cudaEvent_t ev1);
void launch_trace_to_f64(const oed_ctx *ctx, int nsolve, double *g, cudaStream_t s);
void launch_step_probe(const oed_ctx *ctx, int nsolve, int nrep, cudaStream_t st, cudaEvent_t ev0,
                       cudaEvent_t ev1);

// stream_tma.cu
bool tma_supported(const oed_ctx *ctx);
int tma_prepare(oed_ctx *ctx);
cudaError_t launch_steps_tma(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                             cudaEvent_t ev1, int nsteps_override);
cudaError_t launch_wait_selftest(const oed_ctx *ctx, unsigned long long limit_ns, cudaStream_t st);
void tma_record(cudaEvent_t ev, cudaStream_t st);
cudaError_t launch_tma_one_step(const oed_ctx *ctx, int nsolve, cudaStream_t st, float *cur, float *nxt, int m);

// stream_tma2.cu
int tma2_prepare(oed_ctx *ctx);
void launch_pack_kp(const oed_ctx *ctx, cudaStream_t st);
cudaError_t launch_steps_tma2(const oed_ctx *ctx, int nsolve, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                              int nsteps_override, const float **last);
void launch_tma2_gather(const oed_ctx *ctx, int nsolve, const float *last, int m, cudaStream_t st);
void launch_fill_probe(const oed_ctx *ctx, int nsolve, cudaStream_t st);

// resident.cu
int resident_cluster_size(const oed_ctx *ctx);
int resident_fits(const Geometry &g);   // smallest cluster holding an FP32 grid, 0 if none
int resident_max_active_clusters(const oed_ctx *ctx, int C);
cudaError_t launch_resident(const oed_ctx *ctx, int C, int nsolve, cudaStream_t st, cudaEvent_t ev0,
                            cudaEvent_t ev1, int nsteps_override);

// adjoint.cu: residual weights w = (y - g)/sigma^2 from the primal traces, then the
// dual solve into the patch time sums acc[nsolve][6][2][49]
void launch_adjoint(const oed_ctx *ctx, int nsolve, const double *y, double sigma, double *w, double *acc,
                    cudaStream_t st);
// source.cu: gradient and H_II (added to H) from those sums
void launch_hii_combine(const oed_ctx *ctx, int nsolve, const double *acc, double *H, double *grad, int *status,
                        cudaStream_t st);

// hessian.cu
void launch_hessian(const oed_ctx *ctx, int nnode, const double *inv2d, double sigma,
                    const int *seg_end, int nseg, const int *win_seg, int nwin, double *H,
                    double *H_rec, int *status, cudaStream_t s);

// logdet.cu
void launch_eig(const double *H, int n, const double *w, double logvol, int pmask, double *eig,
                double *dkl, int *status, int *n_bad, cudaStream_t s);
void launch_eig_designs(const double *H_rec, int n, int nrec, int nwin, int win,
                        const unsigned char *mask, int ndesign, const double *w, double logvol,
                        double *eig, int *n_bad, cudaStream_t s);
void launch_newton(const double *H, const double *grad, int n, int pmask, const double *lohi, double *theta,
                   int *status, cudaStream_t s);
void launch_nodes_mc(const double *u, int M, const double *lo, const double *hi, double *theta,
                     double *w, cudaStream_t s);

}  // namespace oed
