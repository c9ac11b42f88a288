/*
 * oed.h - C ABI of the GB300 (sm_103a) library for the Laplace-approximated
 * expected information gain (EIG) of seismic source inversion, after
 * Long, Motamed & Tempone, "Fast Bayesian optimal experimental design for
 * seismic source inversion" (arXiv:1502.07873).
 *
 * The path: source parameters theta = (x_s, z_s, t_s, omega_s, m_xx, m_xz, m_zz)
 * (Sec. 2.1, paper order, N_theta = 7) -> 2-D elastic finite-difference forward
 * solves (Sec. 3.3.1, Eq. Full_Disc) -> receiver seismograms (Eq. forward_model)
 * -> central finite-difference Jacobian -> Gauss-Newton Hessian
 * H_1 = sum_{r,m} J^T C_eps^-1 J (Thm 2, Eq. H1; Eq. H1_numerics; Appendix C)
 * -> scaled log-determinant (Sec. 3.3.3) -> D_KL-hat (Thm 4, Eq. DKL_hat)
 * -> EIG = sum_i w_i D_KL-hat(theta_i) (Eqs. intpoly and mcs).
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: OED_OK (0) or one of the OED_E* codes
 *    below.  oed_last_error() gives a message for the last failure on a context.
 *  - Array arguments marked "device" are device pointers on the context's
 *    device (e.g. from torch.empty(..., device="cuda")); "host" arrays are plain
 *    host memory.  The caller owns every array it passes; the library owns only
 *    the context and the device workspace it allocates in oed_create().
 *  - Calls taking a stream enqueue work on that stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream) and return before the work ends;
 *    results are ready once the stream is synchronised.  Calls on one context
 *    must not overlap (they share its workspace).
 *  - Grid: nodes x_i = i h (0 <= i < nx), depth z_j = j h (0 <= j < nz); j = 0 is
 *    the free surface, the two sides and the bottom are absorbing.  The medium is
 *    piecewise constant in depth.
 *  - Seismogram layout (time-major): g[solve][m][r][c], m = 0..nsteps time
 *    levels t_m = m dt, r = receiver, c = 0 (u_x) or 1 (u_z, positive down).
 */
#ifndef OED_H
#define OED_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OED_OK 0
#define OED_EINVAL 1   /* invalid argument (sizes, pointers, source outside the grid) */
#define OED_ENOMEM 2   /* device allocation failed, or a request exceeds the workspace */
#define OED_ENOTPD 3   /* some H_1 is not positive definite (see the per-node status) */
#define OED_ECUDA 4    /* a CUDA runtime call failed */
#define OED_ETIMEOUT 5 /* a bounded wait gave up */
#define OED_PENDING 6  /* (serving) the request has not finished yet */
#define OED_ECANCELED 7 /* (serving) the request was cancelled (before it ran, or between chunks) */

#define OED_FP32 0 /* stencil time stepping in FP32 (Jacobian, H_1, log-det in FP64) */
#define OED_FP64 1 /* everything in FP64 */

#define OED_JAC_PAIRS 0      /* 2 N_theta + 1 solves per node: centre, theta +/- d_j e_j */
#define OED_JAC_DIFFERENCE 1 /* N_theta solves per node, each driven by the FP64 forcing
                                difference f(theta + d_j e_j) - f(theta - d_j e_j) */
#define OED_JAC_SENSITIVITY 2 /* N_theta sensitivity solves per node driven by the
                                 analytic df/dtheta_j (Alg. 1 steps 1-5) */

#define OED_STF_GAUSS 0  /* the paper's source time function (Sec. 4.1):
                            S(t) = omega_s / sqrt(2 pi) exp(-omega_s^2 (t - t_s)^2 / 2) */
#define OED_STF_RICKER 1 /* Ricker wavelet (1 - 2a) exp(-a), a = (pi f (t - t_s))^2, with the
                            fourth source parameter read as the peak frequency f in Hz */

#define OED_NTHETA 7
#define OED_NH 28 /* unique entries of a symmetric 7x7 matrix, row-major upper triangle */

typedef struct oed_ctx oed_ctx;

/* The discretised problem (Sec. 3.3.1 and Sec. 4.1).  All pointers are host
 * pointers; the library copies what it needs during oed_create(). */
typedef struct {
    int nx, nz;        /* grid nodes along x and depth, nx >= 8, nz >= 8 */
    double h;          /* grid spacing in metres, > 0 */
    double dt;         /* time step in seconds, > 0 (CFL: dt <= h / max vp is the
                          caller's responsibility; the synthetic workloads use 0.5) */
    int nsteps;        /* leap-frog steps; seismograms hold nsteps + 1 levels */
    int nlayers;       /* >= 1 layers, piecewise constant in depth */
    const double *z_top; /* [nlayers] layer tops, z_top[0] = 0, increasing; a node on
                            an interface belongs to the deeper layer */
    const double *vp, *vs, *rho; /* [nlayers] P and S speed (m/s), density (kg/m^3) */
    int nrec;          /* receivers, 1..4096 (oed_hessian accepts at most 256) */
    const int *rec_ix; /* [nrec] surface node index i of each receiver (0 <= i < nx);
                          repeats allowed */
    int precision;     /* OED_FP32 or OED_FP64 */
    int stf;           /* source time function: OED_STF_GAUSS (0, the paper's) or
                          OED_STF_RICKER.  The analytic derivatives of the time function
                          (OED_JAC_SENSITIVITY, oed_hessian_ii, oed_hessian_map) exist
                          for the Gaussian only: with OED_STF_RICKER those return
                          OED_EINVAL.  Other values make the problem invalid. */
} oed_problem;

/* Create a context on the current CUDA device with device workspace for up to
 * max_solves (1..65535) simultaneous forward solves (oed_hessian uses 15 or 7
 * per node, see oed_set_jacobian, and processes nodes in chunks).  Returns OED_ENOMEM if the
 * workspace does not fit.  *ctx is set to NULL on failure. */
int oed_create(oed_ctx **ctx, const oed_problem *p, int max_solves);

/* Device bytes oed_create() would allocate for this problem and max_solves
 * (used for admission by HBM footprint).  Returns 0 for an invalid problem. */
size_t oed_workspace_bytes(const oed_problem *p, int max_solves);

/* Release the context and its workspace.  NULL is accepted.  The streams used
 * with the context must be synchronised first.  The workspace is allocated and
 * released stream-ordered (cudaMallocAsync / cudaFreeAsync on the context's own
 * stream), so creating and destroying contexts does not stall other streams. */
int oed_destroy(oed_ctx *ctx);

/* Re-target a context at another problem with the same nx, nz and precision,
 * reusing its device workspace (no allocation): the time-step count, medium,
 * receivers and time function may differ, as long as the new problem's workspace
 * for the context's max_solves (oed_workspace_bytes) fits in the context's.  This
 * is how a server keeps one workspace per grid shape resident across requests.
 * Captured time loops are dropped; the kernel choice (oed_autotune /
 * oed_set_tuning), which depends only on the grid shape, is kept.  Streams that
 * ran earlier calls on the context must be synchronised first.  Returns OED_OK,
 * OED_EINVAL (malformed problem, another shape or precision, or sensitivity
 * solves with a non-Gaussian time function), OED_ENOMEM (the workspace does not
 * fit; the context is unchanged) or OED_ECUDA.  Not in the paper: a systems
 * call of the serving layer. */
int oed_rebind(oed_ctx *ctx, const oed_problem *p);

/* Message of the last failing call on ctx (never NULL). */
const char *oed_last_error(const oed_ctx *ctx);

/* Static name of a status code. */
const char *oed_status_string(int status);

/* Diagnostics: device time of the stencil launches of the last replayed time
 * loop (the nsteps leap-frog launches of the last batch of solves run by
 * oed_forward / oed_hessian on this context), from CUDA events recorded on the
 * stream that ran them.  Call after that stream has been synchronised.
 *   ms        host [1] milliseconds
 *   launches  host [1] or NULL: stencil launches in that interval (0 if none yet) */
int oed_last_step_time(const oed_ctx *ctx, float *ms, int *launches);

/* Time stepping runs in one of four kernels:
 *  - streaming: one launch per step over all solves, wavefields in HBM
 *    (any grid, FP32 or FP64), replayed from a captured CUDA graph;
 *  - TMA streaming (FP32): the same, with halo tiles moved by the tensor-memory
 *    accelerator into a persistent CTA's mbarrier ring (cluster_size -1);
 *  - two-step TMA streaming (FP32, grids that do not fit on chip): two steps per
 *    pass over a paired level layout (cluster_size -2);
 *  - cluster-resident (FP32, grids whose two time levels fit in the shared
 *    memory of a cluster of C <= 8 CTAs, e.g. 401x201): one launch for all
 *    steps, one thread-block cluster per solve, wavefield kept on chip.
 * All give the same node updates, bit for bit.  oed_autotune times every streaming launch
 * shape (rows marched per thread 2/4/8 x warps per block 1/2/4/8), the TMA kernel and
 * every feasible cluster size on nsolve solves of this context's grid, keeps the
 * fastest for later calls, and synchronises the stream; where the two-step kernel
 * runs it is chosen (short probes under-rate it against its rate in a full time
 * loop).  It overwrites the
 * context's workspace (no caller data).  nsolve in 1..max_solves, typically
 * 15 * oed_chunk_nodes(ctx). */
int oed_autotune(oed_ctx *ctx, int nsolve, void *stream);

/* Failure-detection self-test of the bounded waits.  Every wait in the library's
 * kernels on another agent's progress (the TMA kernel's mbarrier waits) gives up
 * after a time limit (2 s), raises the context's device flag, lets its copies in
 * flight land and returns; the flag turns the affected nodes' status into
 * OED_ETIMEOUT and is cleared before the next time loop, so the context stays usable.
 * This call launches one CTA that waits, with a limit of `seconds` (0 < seconds <= 2),
 * for a barrier phase nothing completes, and reads the flag back after synchronising
 * the stream.  Returns OED_ETIMEOUT when the wait expired and the flag arrived (the
 * expected outcome), OED_ECUDA otherwise, OED_EINVAL for a bad argument. */
int oed_wait_selftest(oed_ctx *ctx, double seconds, void *stream);

/* Current / forced choice: cluster_size 0 = streaming kernel with the given
 * rows_per_thread (2, 4, 8) and warps_per_block (1, 2, 4, 8); cluster_size > 0 =
 * cluster-resident kernel (OED_EINVAL if the grid does not fit). */
int oed_get_tuning(const oed_ctx *ctx, int *cluster_size, int *rows_per_thread,
                   int *warps_per_block);
int oed_set_tuning(oed_ctx *ctx, int cluster_size, int rows_per_thread, int warps_per_block);

/* Jacobian form of oed_hessian (default OED_JAC_PAIRS).  Both give the same
 * central difference J_j = (g(theta + d_j e_j) - g(theta - d_j e_j)) / (2 d_j):
 *  - OED_JAC_PAIRS runs the 2 N_theta + 1 perturbed solves of each node and
 *    subtracts the +/- seismograms in FP64;
 *  - OED_JAC_DIFFERENCE runs N_theta solves per node, solve j driven by the
 *    difference of the two forcings formed in FP64 (on the 7x7 union of the two
 *    source patches, or as a difference of time functions for t_s, omega_s).
 *    The scheme (Eq. Full_Disc) is linear in the forcing with theta-independent
 *    coefficients, so its seismogram equals g(theta + d_j e_j) - g(theta - d_j e_j)
 *    exactly in exact arithmetic; in FP32 it avoids the cancellation of the pairs
 *    form and halves the solves.  Requires 2 d_j < h for j = x_s, z_s (else the
 *    node's status is OED_EINVAL).
 *  - OED_JAC_SENSITIVITY is Algorithm 1 steps 1-5 of the paper: solve j is driven
 *    by df/dtheta_j, the analytic derivative of the discrete source (of the
 *    delta / delta' weights for x_s, z_s; of S(t) for t_s, omega_s; the unit
 *    moment patches for m_ij), so its seismogram is the Jacobian column itself
 *    (no step d_j; lo, hi and rel_step are then unused).  It differs from the
 *    central difference by O(d_j^2).
 * The node chunk (oed_chunk_nodes) is max_solves / 15 (pairs) or / 7. */
int oed_set_jacobian(oed_ctx *ctx, int mode);
int oed_get_jacobian(const oed_ctx *ctx);

/* Smallest cluster size of the resident kernel for this context, 0 if none. */
int oed_resident_min_cluster(const oed_ctx *ctx);

/* Largest node chunk oed_hessian processes per pass (max_solves / 15, or / 7 in
 * the difference form). */
int oed_chunk_nodes(const oed_ctx *ctx);

/* Forward map (Eq. forward_model): seismograms of n source vectors.
 *   theta  device [n][7] FP64, paper order (x_s, z_s, t_s, omega_s, m_xx, m_xz, m_zz)
 *   g      device [n][nsteps+1][nrec][2] FP64 (time-major layout above)
 * n may exceed max_solves (processed in chunks).  A source whose 6x6 stencil
 * patch (Sec. 3.3.2 item 2) leaves the interior nodes 1 <= i <= nx-2,
 * 0 <= j <= nz-2 yields NaN seismograms. */
int oed_forward(oed_ctx *ctx, const double *theta, int n, double *g, void *stream);

/* Gauss-Newton Hessians H_1 at n nodes (Thm 2 Eq. H1; Eq. H1_numerics) with
 * C_eps = sigma^2 I and a central-FD Jacobian:
 *   J_{m,r,c; j} = (g(theta + d_j e_j) - g(theta - d_j e_j)) / (2 d_j),
 *   d_j = rel_step * (hi_j - lo_j).
 * The 2*7 perturbed solves of every node run batched; the FP64 Jacobian
 * subtraction and the FP64 J^T J accumulation are fused.
 *   theta       device [n][7]
 *   lo, hi      host [7] prior box (sets the FD steps)
 *   win_levels  host [nwin] or NULL: window w covers levels m < win_levels[w]
 *               (1 <= win_levels[w] <= nsteps+1, increasing)
 *   H           device [n][7][7] FP64 over all levels (full symmetric matrix)
 *   H_rec       device [n][nrec][nwin][28] or NULL: per receiver and window,
 *               upper triangle row-major (requires win_levels)
 *   status      device [n] or NULL: 0, or OED_EINVAL if a perturbed source
 *               leaves the interior (its H is then NaN). */
int oed_hessian(oed_ctx *ctx, const double *theta, int n, const double *lo, const double *hi,
                double rel_step, double sigma, const int *win_levels, int nwin, double *H,
                double *H_rec, int *status, void *stream);

/* Per-node gain and quadrature sum (Sec. 3.3.3, Thm 4, Eqs. intpoly / mcs):
 *   S = sqrt(diag H_1), Ht = S^-1 H_1 S^-1 = L L^T (Cholesky, FP64),
 *   log det H_1 = sum log H_ii + 2 sum log L_ii,
 *   D_i = 1/2 log det H_1 - 7/2 (1 + log 2 pi) + sum_j log(hi_j - lo_j),
 *   eig = sum over positive-definite nodes of w_i D_i (deterministic order).
 *   H       device [n][7][7]
 *   w       device [n] quadrature weights (may be negative for sparse grids)
 *   lo, hi  host [7]
 *   eig     device [1]
 *   dkl     device [n] or NULL (0 for rejected nodes)
 *   status  device [n] or NULL: 0 or OED_ENOTPD
 *   n_bad   device [1] or NULL: number of rejected nodes
 * ctx may be NULL (no workspace is used). */
int oed_eig(oed_ctx *ctx, const double *H, int n, const double *w, const double *lo,
            const double *hi, double *eig, double *dkl, int *status, int *n_bad, void *stream);

/* The same for a problem in which only some parameters are unknown and the others
 * are known (the three-parameter studies of Sec. 4.3 and 4.4): the Laplace gain of
 * Thm 4 with N_theta = k, the number of unknowns,
 *   D_i = 1/2 log det H_FF - k/2 (1 + log 2 pi) + sum_{j in F} log(hi_j - lo_j),
 * where H_FF is the sub-block of H_1 over the unknown set F (rows and columns of
 * known parameters drop out; the scaling and Cholesky act on H_FF).
 *   param_mask  bit j set = parameter j (paper order) is unknown; 1..127
 *               (127 is oed_eig).  Other arguments as for oed_eig; lo, hi are
 *               read only at the unknown indices.
 * Errors: OED_EINVAL for a mask outside 1..127 or hi_j <= lo_j at an unknown j. */
int oed_eig_subset(oed_ctx *ctx, const double *H, int n, const double *w, const double *lo,
                   const double *hi, int param_mask, double *eig, double *dkl, int *status,
                   int *n_bad, void *stream);

/* Second part of the Hessian of the cost L = 1/2 sum_m sum_r r^T C^-1 r,
 * r = y - g(theta), C = sigma^2 I, from one primal and one dual solve per node
 * (Alg. 1 steps 6-10; Eq. H2_numerics; Thm 2's H_2):
 *   step 6-7:  primal solve at theta, w = C^-1 (y - g(theta)) at the receivers,
 *   step 8:    dual problem (Eq. Dual_problems), the transpose of the scheme run
 *              backwards from w: lambda = dJ/d(forcing) for J = sum w . g,
 *   step 9-10: H_II = -sum lambda . d2f/dtheta2 with the analytic second
 *              derivatives of the discrete source (delta weights in x_s, z_s;
 *              S(t) in t_s, omega_s; d2f/dm dm = 0).
 * H_II is ADDED to H (pass H_1 from oed_hessian to get H_1 + H_II, Eq.
 * Hessian_Y with a uniform prior); grad receives dL/dtheta = -J^T C^-1 r.
 *   theta   device [n][7]
 *   y       device [n][nsteps+1][nrec][2] FP64 data (e.g. g(theta*) + eps)
 *   H       device [n][7][7] in/out
 *   grad    device [n][7] or NULL
 *   status  device [n] or NULL: 0, or OED_EINVAL if the source leaves the
 *           interior (H and grad of that node become NaN)
 * nrec <= 256.  The first call on a context allocates FP64 scratch for
 * max_solves nodes (cudaMalloc; OED_ENOMEM if it fails).  Asynchronous on
 * `stream` apart from that first allocation. */
int oed_hessian_ii(oed_ctx *ctx, const double *theta, int n, const double *y, double sigma, double *H,
                   double *grad, int *status, void *stream);

/* One Newton step per node toward the minimiser of the cost (Thm 1) over the
 * unknown parameters (bit j of param_mask, 1..127; the others are known and
 * stay put): solve H_FF d = -grad_F with the scaled Cholesky of H_FF,
 * theta_F += d, clamped to the prior box [lo, hi].  A node whose H_FF is not
 * positive definite keeps its theta (status OED_ENOTPD).  H [n][7][7],
 * grad [n][7], theta [n][7] (in/out), status [n] or NULL, all device; lo, hi
 * host [7].  Synchronises `stream`. */
int oed_newton_step(const double *H, const double *grad, int n, const double *lo, const double *hi, int param_mask,
                    double *theta, int *status, void *stream);

/* The estimate theta-hat of Thm 1 and the Hessian of Thm 2 at it, for Thm 3's
 * refined gain: starting from theta (device [n][7], in/out), `iters` Newton steps
 * over the unknown parameters of param_mask (as oed_newton_step) on the cost with
 * H = H_1 + H_II (H_1 from oed_hessian in the context's Jacobian
 * form, H_II from oed_hessian_ii), then H (device [n][7][7]) = H_1 + H_II and grad
 * (device [n][7]) at the final theta.  Thm 3's per-node gain is then
 * 1/2 log det H - 7/2 (1 + log 2 pi) - h, which oed_eig (oed_eig_subset for a
 * subset) computes from H.
 * iters in 0..100 (0: H_1 + H_II at the given theta). */
int oed_hessian_map(oed_ctx *ctx, double *theta, int n, const double *y, const double *lo, const double *hi,
                    double rel_step, double sigma, int param_mask, int iters, double *H, double *grad,
                    int *status, void *stream);

/* Double-loop (nested) Monte Carlo estimate of the expected information gain:
 * Eq. expected_I sampled directly, the estimator the Laplace method replaces
 * (Sec. 4.4 compares the two).  With y_n = g_outer[n] + eps[n] and noise sigma^2 I,
 *   log_ev[n] = log( (1/M) sum_m exp(-|y_n - g_inner[m]|^2 / (2 sigma^2)) )
 *   eig       = (1/N) sum_n ( -|eps_n|^2 / (2 sigma^2) - log_ev[n] )
 * (the Gaussian normalising constant cancels).  FP64 throughout; distances are
 * summed from the differences (no |y|^2 + |g|^2 - 2 y.g expansion).
 *   g_outer  device [N][D]  noise-free data of the outer samples, e.g. seismograms
 *                           from oed_forward (D = (nsteps+1) * nrec * 2)
 *   eps      device [N][D]  the noise realisations (the caller draws them)
 *   g_inner  device [M][D]  data of the inner (evidence) samples; passing the
 *                           outer set again gives the sample-reusing variant
 *   log_ev   device [N]; eig device [1] or NULL
 * N, M, D >= 1, sigma > 0, else OED_EINVAL.  Asynchronous on `stream`. */
int oed_dlmc(const double *g_outer, const double *eps, int N, const double *g_inner, int M, int D,
             double sigma, double *log_ev, double *eig, void *stream);

/* EIG of many receiver designs from per-receiver partial Hessians (H_1 is
 * additive over receivers and levels, Appendix C):
 *   H_d(theta_i) = sum_{r : mask[d][r] != 0} H_rec[i][r][win]
 *   H_rec   device [n][nrec][nwin][28] from oed_hessian
 *   mask    device [ndesign][nrec] bytes
 *   eig     device [ndesign]
 *   n_bad   device [ndesign] or NULL */
int oed_eig_designs(oed_ctx *ctx, const double *H_rec, int n, int nrec, int nwin, int win,
                    const unsigned char *mask, int ndesign, const double *w, const double *lo,
                    const double *hi, double *eig, int *n_bad, void *stream);

/* Monte Carlo nodes (Eq. mcs): theta_i = lo + (hi - lo) u_i, w_i = 1/M.
 *   u      device [M][7] uniform variates in [0, 1)
 *   theta  device [M][7], w device [M] */
int oed_nodes_mc(const double *u, int M, const double *lo, const double *hi, double *theta,
                 double *w, void *stream);

/* Smolyak sparse grid on [lo, hi] (Eq. intpoly): 1-D Gauss-Legendre rules of
 * l + 1 points (l >= 0), total-degree index set level - dim + 1 <= |l| <= level,
 * combination coefficients (-1)^(level-|l|) C(dim-1, level-|l|), coinciding
 * nodes merged, weights for the uniform probability measure (sum 1).  Host call.
 *   theta host [max_nodes][dim], w host [max_nodes] (may be NULL to count only)
 *   count receives the number of nodes; OED_ENOMEM if it exceeds max_nodes. */
int oed_nodes_smolyak(int dim, int level, const double *lo, const double *hi, int max_nodes,
                      double *theta, double *w, int *count);

/* Whole path with HOST buffers: copies theta and w to the device, runs
 * oed_hessian and oed_eig on the context's own stream, copies the results back
 * and synchronises.  theta host [n][7], w host [n], eig host [1], dkl host [n]
 * or NULL, n_bad host [1] or NULL.  The device staging buffers live in the
 * context and grow on demand. */
int oed_eig_host(oed_ctx *ctx, const double *theta, const double *w, int n, const double *lo,
                 const double *hi, double rel_step, double sigma, double *eig, double *dkl,
                 int *n_bad);

/* ------------------------------------------------------------------------
 * Serving: a request loop for EIG queries with continuous batching.
 *
 * Requests (a problem, its quadrature nodes and weights, the prior box, the FD
 * step, the noise level and the Jacobian form) are queued in arrival order.  Up
 * to max_active requests run at once, each on a worker thread with its own CUDA
 * stream through the public calls (oed_rebind or oed_create, oed_hessian,
 * oed_eig), so a request admitted while others are on the GPU overlaps with them
 * on the device.  A request's device footprint (oed_server_request_bytes) is a
 * context workspace for chunks of chunk_nodes of its nodes plus its node, weight
 * and Hessian arrays; a request whose footprint exceeds the whole budget is run in
 * smaller chunks (halved down to one node) and refused only if even one node does
 * not fit.
 *
 * Workspaces stay resident: a finished request's context goes to an idle pool and
 * the next request with the same grid shape and precision whose workspace fits
 * re-targets it (oed_rebind) instead of allocating.  Idle workspaces count against
 * hbm_budget_bytes and are released, oldest first, when a request of another shape
 * needs the room.
 *
 * Admission takes the oldest queued request that fits in the free budget.  A
 * younger request may be admitted ahead of the queue's head (which may be waiting
 * for memory) only while the head has waited less than max_wait_s seconds
 * (oed_server_set_admission, default 10 s); after that nothing passes it, so no
 * request starves.
 *
 * A request runs chunk by chunk; after each chunk its per-node Hessians are copied
 * to the host.  oed_server_cancel stops a running request after its current chunk
 * (a queued one never runs); oed_server_checkpoint returns the nodes finished so
 * far, and a new request with n_done / H_done set from them resumes the work,
 * recomputing only the remaining nodes, with the same EIG.
 *
 * Every finished request has a one-line JSON record (oed_server_metrics; appended
 * to a file with oed_server_set_log): id, tag, status, grid, steps, layers,
 * receivers, nodes, precision, Jacobian form, EIG, queue / run / total seconds,
 * cell-updates and Gcell-updates/s, footprint, and whether its workspace was
 * reused.  Launch shapes are autotuned on the first request of each grid shape,
 * precision and Jacobian form (on that request's chunk of solves) and reused
 * (unless OED_SERVER_NO_AUTOTUNE).  The server
 * uses the CUDA device current at creation.  None of this is in the paper: it is
 * the serving layer around the paper's computation.
 * ------------------------------------------------------------------------ */
typedef struct oed_server oed_server;

#define OED_SERVER_NO_AUTOTUNE 1

typedef struct {
    oed_problem problem;   /* host arrays, copied at submission */
    int n;                 /* quadrature nodes, >= 1 */
    const double *theta;   /* host [n][7] */
    const double *w;       /* host [n] weights */
    const double *lo, *hi; /* host [7] prior box */
    double rel_step;       /* FD step as a fraction of the prior width */
    double sigma;          /* noise standard deviation (C_eps = sigma^2 I) */
    int jacobian;          /* OED_JAC_PAIRS, OED_JAC_DIFFERENCE or OED_JAC_SENSITIVITY */
    int n_done;            /* resume: the first n_done nodes are already done (0..n) */
    const double *H_done;  /* host [n_done][7][7] their Hessians (oed_server_checkpoint
                              of a request on the same nodes); NULL when n_done == 0 */
    unsigned long long tag;/* caller's label, echoed in the metrics line (e.g. a seed) */
} oed_request;

typedef struct {
    int status;            /* OED_OK, OED_PENDING, OED_ECANCELED or the failing call's code */
    double eig;            /* expected information gain (valid when status == OED_OK) */
    int n_bad;             /* nodes rejected as not positive definite */
    double t_submit, t_admit, t_done; /* seconds on the server's monotonic clock */
    size_t footprint_bytes;           /* device memory reserved while it ran */
    int nodes_done;        /* nodes whose Hessians are finished (resumed ones included) */
    int workspace_reused;  /* 1 if it ran in a pooled workspace, 0 if it allocated one */
} oed_result;

int oed_server_create(oed_server **srv, size_t hbm_budget_bytes, int max_active, int chunk_nodes,
                      int flags);
/* Admission policy: requests may pass the queue's head only while it has waited
 * less than max_wait_s seconds (>= 0; 0 = strictly first come, first served). */
int oed_server_set_admission(oed_server *srv, double max_wait_s);
/* Append each finished request's JSON metrics line to the file at path ("-" =
 * stderr, NULL = stop logging).  OED_EINVAL if the file cannot be opened. */
int oed_server_set_log(oed_server *srv, const char *path);
/* Device bytes a request reserves while it runs at chunks of chunk_nodes nodes
 * (0 if the request is invalid). */
size_t oed_server_request_bytes(const oed_request *req, int chunk_nodes);
/* Queue a request (all of its host data is copied).  OED_ENOMEM if even one node
 * at a time exceeds the whole budget (it could never be admitted), OED_EINVAL if
 * malformed. */
int oed_server_submit(oed_server *srv, const oed_request *req, unsigned long long *id);
/* Current result of request id (status OED_PENDING until it finishes). */
int oed_server_poll(oed_server *srv, unsigned long long id, oed_result *out);
/* Wait up to timeout_s seconds for request id; OED_ETIMEOUT if it is still pending. */
int oed_server_wait(oed_server *srv, unsigned long long id, double timeout_s, oed_result *out);
/* Cancel request id: a queued request finishes at once with OED_ECANCELED; a running
 * one stops after its current chunk with OED_ECANCELED (its finished nodes stay
 * available to oed_server_checkpoint); a finished one is left as it is.  OED_EINVAL
 * for an unknown id. */
int oed_server_cancel(oed_server *srv, unsigned long long id);
/* The per-node Hessians of request id finished so far, in node order: *nodes_done
 * is set to their count k; if H is not NULL it receives them, host [k][7][7]
 * (OED_ENOMEM if cap < k).  Valid while the request runs and after it ends. */
int oed_server_checkpoint(oed_server *srv, unsigned long long id, double *H, int cap, int *nodes_done);
/* The JSON metrics line of finished request id, NUL-terminated, into buf[cap];
 * OED_PENDING if it has not finished, OED_ENOMEM if cap is too small. */
int oed_server_metrics(oed_server *srv, unsigned long long id, char *buf, size_t cap);
/* Drop the record of finished request id (its result, per-node checkpoint and metrics
 * line), which the server otherwise keeps until it is destroyed; the id is unknown
 * afterwards.  OED_PENDING if the request has not finished, OED_EINVAL if unknown. */
int oed_server_release(oed_server *srv, unsigned long long id);
/* Device bytes reserved (running requests and idle workspaces), running and queued
 * request counts. */
int oed_server_stats(oed_server *srv, size_t *in_use, int *active, int *queued);
/* Idle pooled workspaces: their count and bytes. */
int oed_server_pool(oed_server *srv, int *idle, size_t *idle_bytes);
/* Cancel queued requests, wait for running ones, stop the workers, release the
 * pooled workspaces, free the server. */
int oed_server_destroy(oed_server *srv);

/* Allocation-free Gauss-Newton Hessian from seismograms the caller already has.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory while they run, e.g. code that records work into a
 * CUDA graph or a stream-ordered pipeline where cudaMalloc would synchronise the
 * device or is not permitted, or an embedding application that fixes its device
 * memory budget up front.  It computes the same H_1 as oed_hessian from given
 * seismograms, with no context, and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   g        device [n][per_node][nlev][nrec][2] FP64, time-major seismograms of the
 *            node's solves: per_node = 15 for the pairs form (solve 0 the centre,
 *            1 + 2j at theta + d_j e_j, 2 + 2j at theta - d_j e_j) or 7 for the
 *            difference form (solve j = g(theta + d_j e_j) - g(theta - d_j e_j))
 *   lo, hi   host [7] prior box; d_j = rel_step (hi_j - lo_j); sigma the noise std
 *   H        device [n][7][7]
 * Its scratch is one fixed device array of OED_NOALLOC_SCRATCH_DOUBLES doubles
 * (4 MiB) in the library, held by every GPU that loads the library until the
 * process exits; a call needs n * min(8, nlev) * nrec * 28 of them (n * nrec <= 2340
 * when nlev >= 8) and returns OED_ENOMEM, without launching anything, above that.
 * Every call on a device shares that array: calls that can overlap on the GPU
 * (different streams, or host threads) race and must be serialised by the caller.
 * Each call writes every scratch entry it reads, so no clearing is needed.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream capture.
 * Returns OED_OK, OED_EINVAL (bad sizes or pointers), OED_ENOMEM or OED_ECUDA. */
#define OED_NOALLOC_SCRATCH_DOUBLES (1 << 19)
int oed_gauss_newton_noalloc(const double *g, int n, int per_node, int nlev, int nrec,
                             const double *lo, const double *hi, double rel_step, double sigma,
                             double *H, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OED_H */
