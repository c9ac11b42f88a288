/*
 * Plain FP64 CPU oracle for the Laplace-approximated expected information gain
 * (EIG) of Long, Motamed & Tempone, "Fast Bayesian optimal experimental design
 * for seismic source inversion" (arXiv:1502.07873).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition the CUDA path is checked against.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or table with the CUDA library.
 *
 * Every routine follows the paper's steps in the paper's order, written out
 * plainly, with no blocking, fusion or reordering:
 *   ref_delta_1d       regularised delta / delta' weights   (Sec. 3.3.2, item 2)
 *   ref_stf            Gaussian source time function          (Sec. 4.1)
 *   ref_ricker         Ricker wavelet, the optional alternative
 *   ref_media          Lame parameters from velocities        (Sec. 2.1, c_p, c_s)
 *   ref_source_patch   f = S(t) M grad(delta)                 (Eq. source, item 2)
 *   ref_step           one leap-frog step of the FD scheme    (Eqs. interior_disc,
 *                      absorbing_disc, full_discrete, Full_Disc)
 *   ref_forward        seismograms g_r(t_m)                   (Eq. forward_model)
 *   ref_node_hessian   central-FD Jacobian and H_1            (Eq. H1, Eq. H1_numerics,
 *                      Appendix C)
 *   ref_node_hessian_sens  H_I from sensitivity solves        (Alg. 1 steps 1-5)
 *   ref_scaled_logdet  S = sqrt(diag H_1), S^-T H_1 S^-1      (Sec. 3.3.3)
 *   ref_dkl            D_KL-hat                               (Thm 4, Eq. DKL_hat)
 *   ref_eig            sum_i w_i D_KL-hat(theta_i)            (Eqs. intpoly, mcs)
 *   ref_scaled_logdet_sub  the same log-det for the unknown parameters of a
 *                      subset (the known ones drop out)       (Sec. 4.3, 4.4)
 *   ref_dlmc           double-loop Monte Carlo EIG, the direct sampling of
 *                      the definition                         (Eq. expected_I, Sec. 4.4)
 *   ref_adjoint        the dual problem: gradient of sum_m w^m . g^m with respect
 *                      to every forcing value, by the transposed scheme
 *                                                             (Eq. Dual_problems)
 *   ref_hessian_ii     H_II and the cost gradient from one primal and one dual
 *                      solve                                  (Alg. 1 steps 6-10,
 *                                                             Eq. H2_numerics, Thm 2)
 *
 * Readings of points the paper leaves open (the paper cites Nilsson et al. for
 * A_h and B_h without printing them):
 *   - grid x_i = i h, depth z_j = j h, j = 0 is the free surface;
 *   - A_h is the second-order variable-coefficient operator
 *       (Au)_x = D+x((l+2m) D-x ux) + D+z(m D-z ux) + D0x(l D0z uz) + D0z(m D0x uz)
 *       (Au)_z = D+x(m D-x uz) + D+z((l+2m) D-z uz) + D0x(m D0z ux) + D0z(l D0x ux)
 *     with arithmetic-mean half-point coefficients;
 *   - the free surface j = 0 uses the summation-by-parts closure of that
 *     operator: A_h is minus the gradient of a discrete strain energy whose
 *     surface row has quadrature weight 1/2 and a one-sided z-derivative, so
 *     the traction-free conditions hold naturally and the discrete energy
 *     cannot grow (a ghost-row closure that applies the interior formula at
 *     j = 0 has spectral radius above one and is not used);
 *   - the absorbing rows are first-order Clayton-Engquist, forward in time and
 *     upwind in space (normal component with c_p, tangential with c_s); the
 *     leap-frog form with a one-sided B_h is unstable at the boundary node, so
 *     the forward-Euler upwind form is used; all four corners take the
 *     left/right rule;
 *   - S(t) = w/sqrt(2 pi) exp(-w^2 (t - t_s)^2 / 2), i.e. omega_0 = omega_s;
 *   - delta and delta' have six-point support k-2..k+3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NT 7
#define REF_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Regularised delta and delta' (Sec. 3.3.2, item 2).  x_k <= x_s < x_{k+1},
 * alpha = (x_s - x_k)/h.  d[0..5] and dp[0..5] are the weights at nodes
 * k-2, ..., k+3.
 * ------------------------------------------------------------------------- */
void ref_delta_1d(double a, double h, double *d, double *dp)
{
    double a2 = a * a, a3 = a2 * a, a4 = a3 * a, a5 = a4 * a, a6 = a5 * a,
           a7 = a6 * a, a8 = a7 * a, a9 = a8 * a;
    double P = 5.0 * a5 / 3.0 - 7.0 * a6 / 24.0 - 17.0 * a7 / 12.0 + 9.0 * a8 / 8.0 - a9 / 4.0;
    double R = -25.0 * a4 / 12.0 - 3.0 * a5 / 4.0 + 59.0 * a6 / 12.0 - 4.0 * a7 + a8;

    d[0] = (a / 12.0 - a2 / 24.0 - a3 / 12.0 - 19.0 * a4 / 24.0 + P) / h;
    d[1] = (-2.0 * a / 3.0 + 2.0 * a2 / 3.0 + a3 / 6.0 + 4.0 * a4 - 5.0 * P) / h;
    d[2] = (1.0 - 5.0 * a2 / 4.0 - 97.0 * a4 / 12.0 + 10.0 * P) / h;
    d[3] = (2.0 * a / 3.0 + 2.0 * a2 / 3.0 - a3 / 6.0 + 49.0 * a4 / 6.0 - 10.0 * P) / h;
    d[4] = (-a / 12.0 - a2 / 24.0 + a3 / 12.0 - 33.0 * a4 / 8.0 + 5.0 * P) / h;
    d[5] = (5.0 * a4 / 6.0 - P) / h;

    double h2 = h * h;
    dp[0] = (-1.0 / 12.0 + a / 12.0 + a2 / 4.0 + 2.0 * a3 / 3.0 + R) / h2;
    dp[1] = (2.0 / 3.0 - 4.0 * a / 3.0 - a2 / 2.0 - 7.0 * a3 / 2.0 - 5.0 * R) / h2;
    dp[2] = (5.0 * a / 2.0 + 22.0 * a3 / 3.0 + 10.0 * R) / h2;
    dp[3] = (-2.0 / 3.0 - 4.0 * a / 3.0 + a2 / 2.0 - 23.0 * a3 / 3.0 - 10.0 * R) / h2;
    dp[4] = (1.0 / 12.0 + a / 12.0 - a2 / 4.0 + 4.0 * a3 + 5.0 * R) / h2;
    dp[5] = (-5.0 * a3 / 6.0 - R) / h2;
}

/* Derivatives of the delta / delta' weights with respect to the source position
 * x_s (Alg. 1 step 2: the forcing of a sensitivity solve is df/dtheta_j).  With
 * alpha = (x_s - x_k)/h, d/dx_s = (1/h) d/dalpha applied to each printed
 * polynomial; P'(alpha) and R'(alpha) are the derivatives of P and R. */
void ref_delta_1d_dxs(double a, double h, double *dd, double *ddp)
{
    double a2 = a * a, a3 = a2 * a, a4 = a3 * a, a5 = a4 * a, a6 = a5 * a, a7 = a6 * a, a8 = a7 * a;
    double Pp = 25.0 * a4 / 3.0 - 7.0 * a5 / 4.0 - 119.0 * a6 / 12.0 + 9.0 * a7 - 9.0 * a8 / 4.0;
    double Rp = -25.0 * a3 / 3.0 - 15.0 * a4 / 4.0 + 59.0 * a5 / 2.0 - 28.0 * a6 + 8.0 * a7;
    double h2 = h * h, h3 = h2 * h;
    dd[0] = (1.0 / 12.0 - a / 12.0 - a2 / 4.0 - 19.0 * a3 / 6.0 + Pp) / h2;
    dd[1] = (-2.0 / 3.0 + 4.0 * a / 3.0 + a2 / 2.0 + 16.0 * a3 - 5.0 * Pp) / h2;
    dd[2] = (-5.0 * a / 2.0 - 97.0 * a3 / 3.0 + 10.0 * Pp) / h2;
    dd[3] = (2.0 / 3.0 + 4.0 * a / 3.0 - a2 / 2.0 + 98.0 * a3 / 3.0 - 10.0 * Pp) / h2;
    dd[4] = (-1.0 / 12.0 - a / 12.0 + a2 / 4.0 - 33.0 * a3 / 2.0 + 5.0 * Pp) / h2;
    dd[5] = (10.0 * a3 / 3.0 - Pp) / h2;
    ddp[0] = (1.0 / 12.0 + a / 2.0 + 2.0 * a2 + Rp) / h3;
    ddp[1] = (-4.0 / 3.0 - a - 21.0 * a2 / 2.0 - 5.0 * Rp) / h3;
    ddp[2] = (5.0 / 2.0 + 22.0 * a2 + 10.0 * Rp) / h3;
    ddp[3] = (-4.0 / 3.0 + a - 23.0 * a2 - 10.0 * Rp) / h3;
    ddp[4] = (1.0 / 12.0 - a / 2.0 + 12.0 * a2 + 5.0 * Rp) / h3;
    ddp[5] = (-5.0 * a2 / 2.0 - Rp) / h3;
}

/* Second derivatives of the same weights with respect to x_s (Alg. 1 step 9: the
 * forcing's second derivatives, which exist because the regularised delta is C^2
 * in x_s): (1/h^2) d^2/dalpha^2 of each printed polynomial. */
void ref_delta_1d_dxs2(double a, double h, double *dd, double *ddp)
{
    double a2 = a * a, a3 = a2 * a, a4 = a3 * a, a5 = a4 * a, a6 = a5 * a, a7 = a6 * a;
    double Ppp = 100.0 * a3 / 3.0 - 35.0 * a4 / 4.0 - 119.0 * a5 / 2.0 + 63.0 * a6 - 18.0 * a7;
    double Rpp = -25.0 * a2 - 15.0 * a3 + 295.0 * a4 / 2.0 - 168.0 * a5 + 56.0 * a6;
    double h3 = h * h * h, h4 = h3 * h;
    dd[0] = (-1.0 / 12.0 - a / 2.0 - 19.0 * a2 / 2.0 + Ppp) / h3;
    dd[1] = (4.0 / 3.0 + a + 48.0 * a2 - 5.0 * Ppp) / h3;
    dd[2] = (-5.0 / 2.0 - 97.0 * a2 + 10.0 * Ppp) / h3;
    dd[3] = (4.0 / 3.0 - a + 98.0 * a2 - 10.0 * Ppp) / h3;
    dd[4] = (-1.0 / 12.0 + a / 2.0 - 99.0 * a2 / 2.0 + 5.0 * Ppp) / h3;
    dd[5] = (10.0 * a2 - Ppp) / h3;
    ddp[0] = (1.0 / 2.0 + 4.0 * a + Rpp) / h4;
    ddp[1] = (-1.0 - 21.0 * a - 5.0 * Rpp) / h4;
    ddp[2] = (44.0 * a + 10.0 * Rpp) / h4;
    ddp[3] = (1.0 - 46.0 * a - 10.0 * Rpp) / h4;
    ddp[4] = (-1.0 / 2.0 + 24.0 * a + 5.0 * Rpp) / h4;
    ddp[5] = (-5.0 * a - Rpp) / h4;
}

/* Gaussian source time function of Sec. 4.1 with omega_0 read as omega_s. */
double ref_stf(double t, double ts, double ws)
{
    double s = t - ts;
    return ws / sqrt(2.0 * REF_PI) * exp(-ws * ws * s * s / 2.0);
}

/* Ricker wavelet with peak frequency f (Hz) centred at t_s, the conventional
 * alternative source time function: r = (1 - 2a) exp(-a), a = (pi f (t - t_s))^2. */
double ref_ricker(double t, double ts, double f)
{
    double a = REF_PI * f * (t - ts);
    a = a * a;
    return (1.0 - 2.0 * a) * exp(-a);
}

/* the time function of kind 0 (the paper's Gaussian) or 1 (Ricker) */
static double stf_kind(int kind, double t, double ts, double w)
{
    return kind == 1 ? ref_ricker(t, ts, w) : ref_stf(t, ts, w);
}

/* Node media from a depth-layered model: layer l covers z_top[l] <= z < z_top[l+1];
 * a node exactly on an interface belongs to the deeper layer.  lambda = rho (vp^2 - 2 vs^2),
 * mu = rho vs^2 (from c_p = sqrt((lambda + 2 mu)/rho), c_s = sqrt(mu/rho), Sec. 2.1).
 * Outputs are [nz][nx]. */
void ref_media(int nx, int nz, double h, int nlayers, const double *z_top, const double *vp,
               const double *vs, const double *rho, double *lam, double *mu, double *nu)
{
    for (int j = 0; j < nz; j++) {
        double z = j * h;
        int l = 0;
        for (int q = 0; q < nlayers; q++)
            if (z >= z_top[q]) l = q;
        for (int i = 0; i < nx; i++) {
            lam[j * nx + i] = rho[l] * (vp[l] * vp[l] - 2.0 * vs[l] * vs[l]);
            mu[j * nx + i] = rho[l] * vs[l] * vs[l];
            nu[j * nx + i] = rho[l];
        }
    }
}

/* Spatial part of f = S(t) M grad(delta(x - x_s)) on the 6x6 patch of nodes
 * (i0 + a, j0 + b), a, b = 0..5:
 *   f_x = m_xx delta'(x) delta(z) + m_xz delta(x) delta'(z)
 *   f_z = m_xz delta'(x) delta(z) + m_zz delta(x) delta'(z)
 * fx[b*6 + a], fz[b*6 + a].  Returns 0, or -1 if the patch leaves the nodes where
 * the interior formula applies (1 <= i <= nx-2, 0 <= j <= nz-2). */
int ref_source_patch(const double *theta, int nx, int nz, double h, int *i0, int *j0,
                     double *fx, double *fz)
{
    double xs = theta[0], zs = theta[1];
    double mxx = theta[4], mxz = theta[5], mzz = theta[6];
    double qx = xs / h, qz = zs / h;
    int kx = (int)floor(qx), kz = (int)floor(qz);
    double dx[6], dpx[6], dz[6], dpz[6];
    ref_delta_1d(qx - kx, h, dx, dpx);
    ref_delta_1d(qz - kz, h, dz, dpz);
    *i0 = kx - 2;
    *j0 = kz - 2;
    for (int b = 0; b < 6; b++)
        for (int a = 0; a < 6; a++) {
            fx[b * 6 + a] = mxx * dpx[a] * dz[b] + mxz * dx[a] * dpz[b];
            fz[b * 6 + a] = mxz * dpx[a] * dz[b] + mzz * dx[a] * dpz[b];
        }
    if (*i0 < 1 || *i0 + 5 > nx - 2 || *j0 < 0 || *j0 + 5 > nz - 2) return -1;
    return 0;
}

/* ---------------------------------------------------------------------------
 * One leap-frog step (Eq. Full_Disc):
 *   interior and free-surface nodes:  u^{m+1} = 2u^m - u^{m-1} + dt^2/nu (A_h u^m + f^m)
 *   absorbing nodes:                   (u^{m+1} - u^m)/dt = B_h u^m
 * All fields are [nz][nx]; fx, fz is the full forcing field at t_m (may be NULL).
 * ------------------------------------------------------------------------- */
typedef struct {
    int nx, nz;
    double h, dt;
    const double *lam, *mu, *nu;   /* [nz][nx] */
} ref_grid;

/* node value of a [nz][nx] array */
#define AT(a, i, j) ((a)[(size_t)(j) * nx + (i)])

void ref_step(const ref_grid *g, const double *ux, const double *uz, const double *uxm,
              const double *uzm, const double *fx, const double *fz, double *uxn, double *uzn)
{
    int nx = g->nx, nz = g->nz;
    double h = g->h, dt = g->dt, h2 = h * h;
    const double *lam = g->lam, *mu = g->mu, *nu = g->nu;

    for (int j = 0; j < nz; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)j * nx + i;
            if (i == 0 || i == nx - 1 || j == nz - 1) {
                double cp = sqrt((lam[c] + 2.0 * mu[c]) / nu[c]), cs = sqrt(mu[c] / nu[c]);
                if (i == 0 || i == nx - 1) {
                /* left / right (all rows, corners included): d_t u = -/+ c d_x u,
                 * upwind in space, forward in time; normal ux with c_p, tangential uz with c_s */
                    size_t in = (i == 0) ? c + 1 : c - 1;
                    uxn[c] = ux[c] + cp * dt / h * (ux[in] - ux[c]);
                    uzn[c] = uz[c] + cs * dt / h * (uz[in] - uz[c]);
                } else {
                    /* bottom: normal uz with c_p, tangential ux with c_s */
                    size_t in = c - nx;
                    uxn[c] = ux[c] + cs * dt / h * (ux[in] - ux[c]);
                    uzn[c] = uz[c] + cp * dt / h * (uz[in] - uz[c]);
                }
                continue;
            }
            double pc = AT(lam, i, j) + 2.0 * AT(mu, i, j);
            double pe = AT(lam, i + 1, j) + 2.0 * AT(mu, i + 1, j);
            double pw = AT(lam, i - 1, j) + 2.0 * AT(mu, i - 1, j);
            double ps = AT(lam, i, j + 1) + 2.0 * AT(mu, i, j + 1);
            double mc = AT(mu, i, j), me = AT(mu, i + 1, j), mw = AT(mu, i - 1, j);
            double ms = AT(mu, i, j + 1);
            double le = AT(lam, i + 1, j), lw = AT(lam, i - 1, j), ls = AT(lam, i, j + 1);

            /* D+x((l+2m)_{i-1/2} D-x ux) and D+x(m_{i-1/2} D-x uz): every row */
            double Ax = (0.5 * (pc + pe) * (AT(ux, i + 1, j) - AT(ux, i, j))
                       - 0.5 * (pw + pc) * (AT(ux, i, j) - AT(ux, i - 1, j))) / h2;
            double Az = (0.5 * (mc + me) * (AT(uz, i + 1, j) - AT(uz, i, j))
                       - 0.5 * (mw + mc) * (AT(uz, i, j) - AT(uz, i - 1, j))) / h2;
            if (j > 0) {
                double pn = AT(lam, i, j - 1) + 2.0 * AT(mu, i, j - 1);
                double mn = AT(mu, i, j - 1), ln = AT(lam, i, j - 1);
                /* D+z(m_{j-1/2} D-z ux), D+z((l+2m)_{j-1/2} D-z uz) */
                Ax += (0.5 * (mc + ms) * (AT(ux, i, j + 1) - AT(ux, i, j))
                     - 0.5 * (mn + mc) * (AT(ux, i, j) - AT(ux, i, j - 1))) / h2;
                Az += (0.5 * (pc + ps) * (AT(uz, i, j + 1) - AT(uz, i, j))
                     - 0.5 * (pn + pc) * (AT(uz, i, j) - AT(uz, i, j - 1))) / h2;
                /* D0x(l D0z uz) + D0z(m D0x uz) */
                Ax += (le * (AT(uz, i + 1, j + 1) - AT(uz, i + 1, j - 1))
                     - lw * (AT(uz, i - 1, j + 1) - AT(uz, i - 1, j - 1))) / (4.0 * h2)
                    + (ms * (AT(uz, i + 1, j + 1) - AT(uz, i - 1, j + 1))
                     - mn * (AT(uz, i + 1, j - 1) - AT(uz, i - 1, j - 1))) / (4.0 * h2);
                /* D0x(m D0z ux) + D0z(l D0x ux) */
                Az += (me * (AT(ux, i + 1, j + 1) - AT(ux, i + 1, j - 1))
                     - mw * (AT(ux, i - 1, j + 1) - AT(ux, i - 1, j - 1))) / (4.0 * h2)
                    + (ls * (AT(ux, i + 1, j + 1) - AT(ux, i - 1, j + 1))
                     - ln * (AT(ux, i + 1, j - 1) - AT(ux, i - 1, j - 1))) / (4.0 * h2);
            } else {
                /* free surface j = 0: summation-by-parts closure.  The operator is minus the
                 * gradient of a discrete strain energy whose surface row carries weight 1/2
                 * and whose z-derivative is one-sided there (D~z u = (u_1 - u_0)/h); the
                 * traction-free conditions sigma_xz = sigma_zz = 0 hold naturally.
                 *   z-edge:   (2/h^2) m_{1/2} (ux_1 - ux_0),  (2/h^2) (l+2m)_{1/2} (uz_1 - uz_0)
                 *   mixed x:  D0x(l D~z uz) + (m_0 D0x uz_0 + m_1 D0x uz_1)/h
                 *   mixed z:  D0x(m D~z ux) + (l_0 D0x ux_0 + l_1 D0x ux_1)/h */
                double l1 = AT(lam, i, 1);
                Ax += 2.0 * 0.5 * (mc + ms) * (AT(ux, i, 1) - AT(ux, i, 0)) / h2;
                Az += 2.0 * 0.5 * (pc + ps) * (AT(uz, i, 1) - AT(uz, i, 0)) / h2;
                double dzuz_e = (AT(uz, i + 1, 1) - AT(uz, i + 1, 0)) / h;
                double dzuz_w = (AT(uz, i - 1, 1) - AT(uz, i - 1, 0)) / h;
                double dzux_e = (AT(ux, i + 1, 1) - AT(ux, i + 1, 0)) / h;
                double dzux_w = (AT(ux, i - 1, 1) - AT(ux, i - 1, 0)) / h;
                double dxuz0 = (AT(uz, i + 1, 0) - AT(uz, i - 1, 0)) / (2.0 * h);
                double dxuz1 = (AT(uz, i + 1, 1) - AT(uz, i - 1, 1)) / (2.0 * h);
                double dxux0 = (AT(ux, i + 1, 0) - AT(ux, i - 1, 0)) / (2.0 * h);
                double dxux1 = (AT(ux, i + 1, 1) - AT(ux, i - 1, 1)) / (2.0 * h);
                Ax += (le * dzuz_e - lw * dzuz_w) / (2.0 * h) + (mc * dxuz0 + ms * dxuz1) / h;
                Az += (me * dzux_e - mw * dzux_w) / (2.0 * h) + (AT(lam, i, 0) * dxux0 + l1 * dxux1) / h;
            }
            if (fx) Ax += fx[c];
            if (fz) Az += fz[c];
            double r = dt * dt / nu[c];
            uxn[c] = 2.0 * ux[c] - uxm[c] + r * Ax;
            uzn[c] = 2.0 * uz[c] - uzm[c] + r * Az;
        }
}
#undef AT

/* ---------------------------------------------------------------------------
 * Forward solve: zero initial levels u^0 = u^{-1} = 0 (Eq. elastic_2nd), nsteps
 * leap-frog steps with forcing f^m = S(t_m) f_patch at t_m = m dt, receiver
 * samples g[m][r][c] = u_c(x_r, t_m) for m = 0..nsteps (Eq. forward_model).
 * Returns 0, or -1 if the source patch leaves the interior.
 * ------------------------------------------------------------------------- */
int ref_forward_stf(int kind, int nx, int nz, double h, double dt, int nsteps, const double *lam,
                    const double *mu, const double *nu, int nrec, const int *rec_ix,
                    const double *theta, double *g);

int ref_forward(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                const double *mu, const double *nu, int nrec, const int *rec_ix,
                const double *theta, double *g)
{
    return ref_forward_stf(0, nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, theta, g);
}

/* The same with the time function of the given kind (0 Gaussian, 1 Ricker). */
int ref_forward_stf(int kind, int nx, int nz, double h, double dt, int nsteps, const double *lam,
                    const double *mu, const double *nu, int nrec, const int *rec_ix,
                    const double *theta, double *g)
{
    ref_grid G = {nx, nz, h, dt, lam, mu, nu};
    int i0, j0;
    double px[36], pz[36];
    if (ref_source_patch(theta, nx, nz, h, &i0, &j0, px, pz) != 0) return -1;
    size_t n = (size_t)nx * nz;
    double *ux = calloc(n, sizeof(double)), *uz = calloc(n, sizeof(double));
    double *uxm = calloc(n, sizeof(double)), *uzm = calloc(n, sizeof(double));
    double *uxn = calloc(n, sizeof(double)), *uzn = calloc(n, sizeof(double));
    double *fx = calloc(n, sizeof(double)), *fz = calloc(n, sizeof(double));

    for (int r = 0; r < nrec; r++) {
        g[(0 * nrec + r) * 2 + 0] = 0.0;
        g[(0 * nrec + r) * 2 + 1] = 0.0;
    }
    for (int m = 0; m < nsteps; m++) {
        double s = stf_kind(kind, m * dt, theta[2], theta[3]);
        for (int b = 0; b < 6; b++)
            for (int a = 0; a < 6; a++) {
                size_t c = (size_t)(j0 + b) * nx + (i0 + a);
                fx[c] = s * px[b * 6 + a];
                fz[c] = s * pz[b * 6 + a];
            }
        ref_step(&G, ux, uz, uxm, uzm, fx, fz, uxn, uzn);
        /* rotate levels: (m-1, m, m+1) -> (m, m+1, free) */
        double *t;
        t = uxm; uxm = ux; ux = uxn; uxn = t;
        t = uzm; uzm = uz; uz = uzn; uzn = t;
        for (int r = 0; r < nrec; r++) {
            g[((size_t)(m + 1) * nrec + r) * 2 + 0] = ux[rec_ix[r]];
            g[((size_t)(m + 1) * nrec + r) * 2 + 1] = uz[rec_ix[r]];
        }
    }
    free(ux); free(uz); free(uxm); free(uzm); free(uxn); free(uzn); free(fx); free(fz);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Forward solve driven by a given 6x6 patch (corner i0, j0) and one of three time
 * functions of (t_s, w_s): kind 0 S(t), kind 1 dS/dt_s = S(t) w^2 (t - t_s),
 * kind 2 dS/dw_s = S(t) (1/w - w (t - t_s)^2).  Same time stepping as ref_forward.
 * ------------------------------------------------------------------------- */
int ref_forward_forcing(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                        const double *mu, const double *nu, int nrec, const int *rec_ix, int i0,
                        int j0, const double *px, const double *pz, int kind, double ts, double ws,
                        double *g)
{
    ref_grid G = {nx, nz, h, dt, lam, mu, nu};
    if (i0 < 1 || i0 + 5 > nx - 2 || j0 < 0 || j0 + 5 > nz - 2) return -1;
    size_t n = (size_t)nx * nz;
    double *ux = calloc(n, sizeof(double)), *uz = calloc(n, sizeof(double));
    double *uxm = calloc(n, sizeof(double)), *uzm = calloc(n, sizeof(double));
    double *uxn = calloc(n, sizeof(double)), *uzn = calloc(n, sizeof(double));
    double *fx = calloc(n, sizeof(double)), *fz = calloc(n, sizeof(double));
    for (int r = 0; r < nrec; r++) g[r * 2] = g[r * 2 + 1] = 0.0;
    for (int m = 0; m < nsteps; m++) {
        double t = m * dt, sv = ref_stf(t, ts, ws);
        if (kind == 1) sv = sv * ws * ws * (t - ts);
        if (kind == 2) sv = sv * (1.0 / ws - ws * (t - ts) * (t - ts));
        for (int b = 0; b < 6; b++)
            for (int a = 0; a < 6; a++) {
                size_t c = (size_t)(j0 + b) * nx + (i0 + a);
                fx[c] = sv * px[b * 6 + a];
                fz[c] = sv * pz[b * 6 + a];
            }
        ref_step(&G, ux, uz, uxm, uzm, fx, fz, uxn, uzn);
        double *t2;
        t2 = uxm; uxm = ux; ux = uxn; uxn = t2;
        t2 = uzm; uzm = uz; uz = uzn; uzn = t2;
        for (int r = 0; r < nrec; r++) {
            g[((size_t)(m + 1) * nrec + r) * 2 + 0] = ux[rec_ix[r]];
            g[((size_t)(m + 1) * nrec + r) * 2 + 1] = uz[rec_ix[r]];
        }
    }
    free(ux); free(uz); free(uxm); free(uzm); free(uxn); free(uzn); free(fx); free(fz);
    return 0;
}

/* ---------------------------------------------------------------------------
 * H_I of Alg. 1 steps 1-5 with sensitivity solves: the seismograms of the
 * solves driven by df/dtheta_j (step 2, analytic derivatives of the discrete
 * source) are the Jacobian columns J_j (step 3), and
 * H = sigma^-2 sum_{m,r,c} J^T J (steps 4-5, Eq. H1_numerics).
 *   x_s, z_s: derivative of the delta / delta' weights; t_s, w_s: derivative of
 *   S(t); m_xx, m_xz, m_zz: the unit-moment patches.
 * ------------------------------------------------------------------------- */
static int sens_solves(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                       const double *mu, const double *nu, int nrec, const int *rec_ix,
                       const double *theta, double sigma, double *H, double *Jout);

int ref_node_hessian_sens(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                          const double *mu, const double *nu, int nrec, const int *rec_ix,
                          const double *theta, double sigma, double *H)
{
    return sens_solves(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, theta, sigma, H, NULL);
}

/* The Jacobian columns themselves, J[j][m][r][c] = dg_{m,r,c}/dtheta_j (step 3). */
int ref_jacobian_sens(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                      const double *mu, const double *nu, int nrec, const int *rec_ix,
                      const double *theta, double *J)
{
    return sens_solves(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, theta, 1.0, NULL, J);
}

static int sens_solves(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                       const double *mu, const double *nu, int nrec, const int *rec_ix,
                       const double *theta, double sigma, double *H, double *Jout)
{
    double xs = theta[0], zs = theta[1], mxx = theta[4], mxz = theta[5], mzz = theta[6];
    double qx = xs / h, qz = zs / h;
    int kx = (int)floor(qx), kz = (int)floor(qz);
    double dx[6], dpx[6], dz[6], dpz[6], ex[6], epx[6], ez[6], epz[6];
    ref_delta_1d(qx - kx, h, dx, dpx);
    ref_delta_1d(qz - kz, h, dz, dpz);
    ref_delta_1d_dxs(qx - kx, h, ex, epx);
    ref_delta_1d_dxs(qz - kz, h, ez, epz);
    size_t nrow = (size_t)(nsteps + 1) * nrec * 2;
    double *gall = malloc(sizeof(double) * nrow * NT);
    int rc = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc) if (!omp_in_parallel())
#endif
    for (int j = 0; j < NT; j++) {
        double px[36], pz[36];
        int kind = 0;
        for (int b = 0; b < 6; b++)
            for (int a = 0; a < 6; a++) {
                double vx = 0.0, vz = 0.0;
                if (j == 0) {          /* d/dx_s */
                    vx = mxx * epx[a] * dz[b] + mxz * ex[a] * dpz[b];
                    vz = mxz * epx[a] * dz[b] + mzz * ex[a] * dpz[b];
                } else if (j == 1) {   /* d/dz_s */
                    vx = mxx * dpx[a] * ez[b] + mxz * dx[a] * epz[b];
                    vz = mxz * dpx[a] * ez[b] + mzz * dx[a] * epz[b];
                } else if (j == 2 || j == 3) {   /* time function derivatives */
                    vx = mxx * dpx[a] * dz[b] + mxz * dx[a] * dpz[b];
                    vz = mxz * dpx[a] * dz[b] + mzz * dx[a] * dpz[b];
                    kind = j - 1;
                } else if (j == 4) {   /* d/dm_xx */
                    vx = dpx[a] * dz[b];
                } else if (j == 5) {   /* d/dm_xz */
                    vx = dx[a] * dpz[b];
                    vz = dpx[a] * dz[b];
                } else {               /* d/dm_zz */
                    vz = dx[a] * dpz[b];
                }
                px[b * 6 + a] = vx;
                pz[b * 6 + a] = vz;
            }
        rc |= ref_forward_forcing(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, kx - 2, kz - 2, px,
                                  pz, kind, theta[2], theta[3], gall + (size_t)j * nrow);
    }
    if (rc == 0 && H) {
        double s2 = 1.0 / (sigma * sigma);
        for (int a = 0; a < NT * NT; a++) H[a] = 0.0;
        for (size_t k = 0; k < nrow; k++)
            for (int a = 0; a < NT; a++)
                for (int b = 0; b < NT; b++)
                    H[a * NT + b] += s2 * gall[(size_t)a * nrow + k] * gall[(size_t)b * nrow + k];
    }
    if (rc == 0 && Jout) memcpy(Jout, gall, sizeof(double) * nrow * NT);
    free(gall);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Gauss-Newton Hessian H_1 at one node from the 2*N_theta central-FD solves
 * (Eq. H1 with C_eps = sigma^2 I; Eq. H1_numerics; Appendix C):
 *   J_{m,r,c; j} = (g(theta + d_j e_j) - g(theta - d_j e_j)) / (2 d_j),
 *   d_j = rel_step (hi_j - lo_j),
 *   H_rec[r][w] = sigma^-2 sum_{m < win_levels[w]} sum_c J_{m,r,c}^T J_{m,r,c}
 *   H = sigma^-2 sum_{m <= nsteps} sum_r sum_c J^T J.
 * H_rec ([nrec][nwin][49]) may be NULL.  Returns 0 or -1 (source out of range).
 * ------------------------------------------------------------------------- */
int ref_node_hessian_stf(int kind, int nx, int nz, double h, double dt, int nsteps, const double *lam,
                         const double *mu, const double *nu, int nrec, const int *rec_ix,
                         const double *theta, const double *lo, const double *hi, double rel_step,
                         double sigma, int nwin, const int *win_levels, double *H, double *H_rec);

int ref_node_hessian(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                     const double *mu, const double *nu, int nrec, const int *rec_ix,
                     const double *theta, const double *lo, const double *hi, double rel_step,
                     double sigma, int nwin, const int *win_levels, double *H, double *H_rec)
{
    return ref_node_hessian_stf(0, nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, theta, lo, hi,
                                rel_step, sigma, nwin, win_levels, H, H_rec);
}

/* The same with the time function of the given kind (0 Gaussian, 1 Ricker). */
int ref_node_hessian_stf(int kind, int nx, int nz, double h, double dt, int nsteps, const double *lam,
                         const double *mu, const double *nu, int nrec, const int *rec_ix,
                         const double *theta, const double *lo, const double *hi, double rel_step,
                         double sigma, int nwin, const int *win_levels, double *H, double *H_rec)
{
    size_t nrow = (size_t)(nsteps + 1) * nrec * 2;
    double *gall = malloc(sizeof(double) * nrow * 2 * NT);
    double *J = malloc(sizeof(double) * nrow * NT);
    int rc = 0;
    /* the 2 N_theta perturbed solves are independent (run in parallel when this is
     * not already inside a parallel region) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc) if (!omp_in_parallel())
#endif
    for (int q = 0; q < 2 * NT; q++) {
        int j = q / 2;
        double d = rel_step * (hi[j] - lo[j]);
        double t[NT];
        for (int k = 0; k < NT; k++) t[k] = theta[k];
        t[j] += (q % 2 == 0) ? d : -d;
        rc |= ref_forward_stf(kind, nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, t,
                              gall + (size_t)q * nrow);
    }
    for (int j = 0; j < NT && rc == 0; j++) {
        double d = rel_step * (hi[j] - lo[j]);
        const double *gp = gall + (size_t)(2 * j) * nrow, *gm = gall + (size_t)(2 * j + 1) * nrow;
        for (size_t k = 0; k < nrow; k++) J[k * NT + j] = (gp[k] - gm[k]) / (2.0 * d);
    }
    if (rc == 0) {
        double s2 = 1.0 / (sigma * sigma);
        for (int a = 0; a < NT * NT; a++) H[a] = 0.0;
        for (size_t k = 0; k < nrow; k++)
            for (int a = 0; a < NT; a++)
                for (int b = 0; b < NT; b++) H[a * NT + b] += s2 * J[k * NT + a] * J[k * NT + b];
        if (H_rec) {
            for (int r = 0; r < nrec; r++)
                for (int w = 0; w < nwin; w++) {
                    double *Hw = H_rec + ((size_t)r * nwin + w) * NT * NT;
                    for (int a = 0; a < NT * NT; a++) Hw[a] = 0.0;
                    for (int m = 0; m < win_levels[w] && m <= nsteps; m++)
                        for (int c = 0; c < 2; c++) {
                            const double *row = J + (((size_t)m * nrec + r) * 2 + c) * NT;
                            for (int a = 0; a < NT; a++)
                                for (int b = 0; b < NT; b++) Hw[a * NT + b] += s2 * row[a] * row[b];
                        }
                }
        }
    }
    free(gall); free(J);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Scaled log-determinant (Sec. 3.3.3): S = sqrt(diag H), Ht = S^-1 H S^-1,
 * textbook Cholesky Ht = L L^T, log det H = sum log H_ii + 2 sum log L_ii.
 * Ht (49 values) is written if non-NULL.  Returns 0, or 1 if H is not
 * positive definite.
 * ------------------------------------------------------------------------- */
int ref_scaled_logdet(const double *H, double *logdet, double *Ht)
{
    double S[NT], A[NT * NT], L[NT * NT];
    for (int i = 0; i < NT; i++) {
        if (!(H[i * NT + i] > 0.0)) return 1;
        S[i] = sqrt(H[i * NT + i]);
    }
    for (int i = 0; i < NT; i++)
        for (int j = 0; j < NT; j++) A[i * NT + j] = H[i * NT + j] / (S[i] * S[j]);
    if (Ht) memcpy(Ht, A, sizeof(A));
    memset(L, 0, sizeof(L));
    for (int j = 0; j < NT; j++) {
        double s = A[j * NT + j];
        for (int k = 0; k < j; k++) s -= L[j * NT + k] * L[j * NT + k];
        if (!(s > 0.0)) return 1;
        L[j * NT + j] = sqrt(s);
        for (int i = j + 1; i < NT; i++) {
            double t = A[i * NT + j];
            for (int k = 0; k < j; k++) t -= L[i * NT + k] * L[j * NT + k];
            L[i * NT + j] = t / L[j * NT + j];
        }
    }
    double ld = 0.0;
    for (int i = 0; i < NT; i++) ld += log(H[i * NT + i]) + 2.0 * log(L[i * NT + i]);
    *logdet = ld;
    return 0;
}

/* D_KL-hat (Thm 4, Eq. DKL_hat):
 *   -1/2 log((2 pi)^n |H^-1|) - n/2 - h(theta*) = 1/2 log det H - n/2 log(2 pi) - n/2 - h,
 * with h = log of the prior density at theta*. */
double ref_dkl(double logdet, int n, double log_prior_density)
{
    return 0.5 * logdet - 0.5 * n * log(2.0 * REF_PI) - 0.5 * n - log_prior_density;
}

/* ---------------------------------------------------------------------------
 * Whole path for one design: for each node i (OpenMP over nodes only),
 * H_1(theta_i) by ref_node_hessian, log det by ref_scaled_logdet, D_KL-hat by
 * ref_dkl with the uniform prior density h = -sum_j log(hi_j - lo_j), then
 * EIG = sum_i w_i D_i over positive-definite nodes, in node order with Kahan
 * compensation (Eqs. intpoly / mcs).  dkl[i], status[i] (0 ok, 1 not PD,
 * -1 source out of range) and H[i][49] are written if non-NULL.
 * nthreads <= 0 keeps the OpenMP default.  Returns the number of threads used.
 * ------------------------------------------------------------------------- */
int ref_eig(int nx, int nz, double h, double dt, int nsteps, const double *lam,
            const double *mu, const double *nu, int nrec, const int *rec_ix, int nnode,
            const double *theta, const double *w, const double *lo, const double *hi,
            double rel_step, double sigma, int nthreads, double *eig, double *dkl, int *status,
            double *Hout)
{
    double logprior = 0.0;
    for (int j = 0; j < NT; j++) logprior -= log(hi[j] - lo[j]);
    double *D = malloc(sizeof(double) * (nnode > 0 ? nnode : 1));
    int *st = malloc(sizeof(int) * (nnode > 0 ? nnode : 1));
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nnode; i++) {
        double H[NT * NT], ld = 0.0;
        int rc = ref_node_hessian(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix,
                                  theta + (size_t)i * NT, lo, hi, rel_step, sigma, 0, NULL, H, NULL);
        if (rc != 0) {
            st[i] = -1;
            D[i] = 0.0;
            continue;
        }
        if (Hout) memcpy(Hout + (size_t)i * NT * NT, H, sizeof(H));
        st[i] = ref_scaled_logdet(H, &ld, NULL);
        D[i] = st[i] == 0 ? ref_dkl(ld, NT, logprior) : 0.0;
    }
    double sum = 0.0, comp = 0.0;
    for (int i = 0; i < nnode; i++) {
        if (st[i] != 0) continue;
        double y = w[i] * D[i] - comp;
        double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    *eig = sum;
    if (dkl) memcpy(dkl, D, sizeof(double) * nnode);
    if (status) memcpy(status, st, sizeof(int) * nnode);
    free(D);
    free(st);
    return used;
}

/* ---------------------------------------------------------------------------
 * Scaled log-det of the sub-block of H_1 (7x7, row-major) over the parameters
 * whose bit is set in mask (Sec. 3.3.3 applied to the unknown parameters only;
 * the known parameters are fixed and their rows and columns drop out).
 * Returns 0, or 1 if the sub-block is not positive definite.
 * ------------------------------------------------------------------------- */
int ref_scaled_logdet_sub(const double *H, int mask, double *logdet)
{
    int idx[NT], k = 0;
    for (int j = 0; j < NT; j++)
        if (mask >> j & 1) idx[k++] = j;
    if (k == 0) return 1;
    double S[NT], L[NT * NT];
    for (int a = 0; a < k; a++) {
        double d = H[idx[a] * NT + idx[a]];
        if (!(d > 0.0)) return 1;
        S[a] = sqrt(d);
    }
    memset(L, 0, sizeof(L));
    for (int j = 0; j < k; j++) {
        double s = H[idx[j] * NT + idx[j]] / (S[j] * S[j]);
        for (int c = 0; c < j; c++) s -= L[j * NT + c] * L[j * NT + c];
        if (!(s > 0.0)) return 1;
        L[j * NT + j] = sqrt(s);
        for (int i = j + 1; i < k; i++) {
            double t = H[idx[i] * NT + idx[j]] / (S[i] * S[j]);
            for (int c = 0; c < j; c++) t -= L[i * NT + c] * L[j * NT + c];
            L[i * NT + j] = t / L[j * NT + j];
        }
    }
    double ld = 0.0;
    for (int a = 0; a < k; a++) ld += 2.0 * log(S[a]) + 2.0 * log(L[a * NT + a]);
    *logdet = ld;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Double-loop Monte Carlo estimate of the expected information gain (Eq.
 * expected_I by direct sampling; Sec. 4.4).  Outer samples: y_n = g_out[n] +
 * eps[n] (n < N), inner samples g_in[m] (m < M), each a vector of D data values,
 * Gaussian noise sigma^2 I:
 *   log_ev[n] = log( (1/M) sum_m exp(-|y_n - g_in[m]|^2 / (2 sigma^2)) )
 *   *eig      = (1/N) sum_n ( -|eps_n|^2 / (2 sigma^2) - log_ev[n] )
 * The Gaussian normalising constant cancels between the two terms.  The sum of
 * exponentials is taken relative to its largest term (log-sum-exp) so it does
 * not underflow; otherwise the definition is written out as it reads.
 * ------------------------------------------------------------------------- */
void ref_dlmc(const double *g_out, const double *eps, int N, const double *g_in, int M, int D,
              double sigma, double *log_ev, double *eig)
{
    const double s2 = 2.0 * sigma * sigma;
    double *l = malloc(sizeof(double) * (M > 0 ? M : 1));
    double total = 0.0;
    for (int n = 0; n < N; n++) {
        double lmax = -INFINITY;
        for (int m = 0; m < M; m++) {
            double q = 0.0;
            for (int d = 0; d < D; d++) {
                double r = g_out[(size_t)n * D + d] + eps[(size_t)n * D + d] - g_in[(size_t)m * D + d];
                q += r * r;
            }
            l[m] = -q / s2;
            if (l[m] > lmax) lmax = l[m];
        }
        double sum = 0.0;
        for (int m = 0; m < M; m++) sum += exp(l[m] - lmax);
        log_ev[n] = lmax + log(sum) - log((double)M);
        double e2 = 0.0;
        for (int d = 0; d < D; d++) e2 += eps[(size_t)n * D + d] * eps[(size_t)n * D + d];
        total += -e2 / s2 - log_ev[n];
    }
    *eig = total / N;
    free(l);
}

/* ---------------------------------------------------------------------------
 * Source time function and its derivatives with respect to (t_s, omega_s) up to
 * second order (Alg. 1 steps 2 and 9), tau = t - t_s, L = log S:
 *   dL/dt_s = w^2 tau, dL/dw = 1/w - w tau^2, d2L/dt_s2 = -w^2,
 *   d2L/dt_s dw = 2 w tau, d2L/dw2 = -1/w^2 - tau^2,
 * and d2S = S (dL dL + d2L).  out = (S, S_t, S_w, S_tt, S_tw, S_ww).
 * ------------------------------------------------------------------------- */
void ref_stf_derivs(double t, double ts, double w, double *out)
{
    double tau = t - ts, S = ref_stf(t, ts, w);
    double Lt = w * w * tau, Lw = 1.0 / w - w * tau * tau;
    out[0] = S;
    out[1] = S * Lt;
    out[2] = S * Lw;
    out[3] = S * (Lt * Lt - w * w);
    out[4] = S * (Lt * Lw + 2.0 * w * tau);
    out[5] = S * (Lw * Lw - 1.0 / (w * w) - tau * tau);
}

/* ---------------------------------------------------------------------------
 * The leap-frog step as a linear map on the state u = (u_x, u_z), 2 nx nz values:
 *   u^{m+1} = B u^m + E u^{m-1} + F f^m   (Eq. Full_Disc)
 * The j-th column of B (E, F) is the output of ref_step for a unit input at
 * entry j of u^m (u^{m-1}, f^m) and zero elsewhere; its nonzero entries are kept.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n;
    int *start;     /* [n + 1] */
    int *row;
    double *val;
} ref_cols;

static void probe_columns(const ref_grid *G, int which, ref_cols *C)
{
    int nx = G->nx, nz = G->nz;
    size_t nn = (size_t)nx * nz;
    int n = (int)(2 * nn);
    double *in = calloc(2 * nn, sizeof(double)), *zero = calloc(2 * nn, sizeof(double));
    double *out = calloc(2 * nn, sizeof(double));
    size_t cap = (size_t)n * 24, used = 0;
    C->n = n;
    C->start = malloc(sizeof(int) * (n + 1));
    C->row = malloc(sizeof(int) * cap);
    C->val = malloc(sizeof(double) * cap);
    for (int j = 0; j < n; j++) {
        in[j] = 1.0;
        const double *ux = which == 0 ? in : zero, *uz = which == 0 ? in + nn : zero + nn;
        const double *uxm = which == 1 ? in : zero, *uzm = which == 1 ? in + nn : zero + nn;
        const double *fx = which == 2 ? in : NULL, *fz = which == 2 ? in + nn : NULL;
        ref_step(G, ux, uz, uxm, uzm, fx, fz, out, out + nn);
        C->start[j] = (int)used;
        for (int i = 0; i < n; i++) {
            if (out[i] == 0.0) continue;
            if (used == cap) {
                cap *= 2;
                C->row = realloc(C->row, sizeof(int) * cap);
                C->val = realloc(C->val, sizeof(double) * cap);
            }
            C->row[used] = i;
            C->val[used] = out[i];
            used++;
        }
        in[j] = 0.0;
    }
    C->start[n] = (int)used;
    free(in);
    free(zero);
    free(out);
}

static void free_cols(ref_cols *C)
{
    free(C->start);
    free(C->row);
    free(C->val);
}

/* (M^T v)_j = sum over the stored entries of column j of M_ij v_i */
static void apply_transpose(const ref_cols *C, const double *v, double *out)
{
    for (int j = 0; j < C->n; j++) {
        double s = 0.0;
        for (int k = C->start[j]; k < C->start[j + 1]; k++) s += C->val[k] * v[C->row[k]];
        out[j] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Forward solve driven by a full forcing sequence f[m][c][nz][nx], m < nsteps
 * (c = 0: x, 1: z), zero initial levels; receiver samples g[m][r][c], m <= nsteps.
 * ------------------------------------------------------------------------- */
void ref_forward_field(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                       const double *mu, const double *nu, int nrec, const int *rec_ix,
                       const double *f, double *g)
{
    ref_grid G = {nx, nz, h, dt, lam, mu, nu};
    size_t nn = (size_t)nx * nz;
    double *ux = calloc(nn, sizeof(double)), *uz = calloc(nn, sizeof(double));
    double *uxm = calloc(nn, sizeof(double)), *uzm = calloc(nn, sizeof(double));
    double *uxn = calloc(nn, sizeof(double)), *uzn = calloc(nn, sizeof(double));
    for (int r = 0; r < nrec; r++) g[r * 2] = g[r * 2 + 1] = 0.0;
    for (int m = 0; m < nsteps; m++) {
        const double *fm = f + (size_t)m * 2 * nn;
        ref_step(&G, ux, uz, uxm, uzm, fm, fm + nn, uxn, uzn);
        double *t;
        t = uxm; uxm = ux; ux = uxn; uxn = t;
        t = uzm; uzm = uz; uz = uzn; uzn = t;
        for (int r = 0; r < nrec; r++) {
            g[((size_t)(m + 1) * nrec + r) * 2 + 0] = ux[rec_ix[r]];
            g[((size_t)(m + 1) * nrec + r) * 2 + 1] = uz[rec_ix[r]];
        }
    }
    free(ux); free(uz); free(uxm); free(uzm); free(uxn); free(uzn);
}

/* ---------------------------------------------------------------------------
 * The dual problem (Eq. Dual_problems): for the functional J = sum_{m=0}^{nsteps}
 * sum_{r,c} w[m][r][c] g_{r,c}(t_m), the derivative of J with respect to every
 * forcing value, gradf[m][c][nz][nx] = dJ/df^m (m < nsteps), from the transposed
 * scheme run backwards:
 *   lambda^m = R^T w^m + B^T lambda^{m+1} + E^T lambda^{m+2},  m = nsteps .. 1,
 *   lambda^{nsteps+1} = lambda^{nsteps+2} = 0,   dJ/df^m = F^T lambda^{m+1},
 * with R the receiver sampling.  B, E, F are read off the step by probing.
 * ------------------------------------------------------------------------- */
void ref_adjoint(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                 const double *mu, const double *nu, int nrec, const int *rec_ix, const double *w,
                 double *gradf)
{
    ref_grid G = {nx, nz, h, dt, lam, mu, nu};
    size_t nn = (size_t)nx * nz;
    int n = (int)(2 * nn);
    ref_cols B, E, F;
    probe_columns(&G, 0, &B);
    probe_columns(&G, 1, &E);
    probe_columns(&G, 2, &F);
    double *l1 = calloc(n, sizeof(double)), *l2 = calloc(n, sizeof(double));   /* m+1, m+2 */
    double *l0 = calloc(n, sizeof(double)), *tmp = calloc(n, sizeof(double));
    for (int m = nsteps; m >= 1; m--) {
        apply_transpose(&B, l1, l0);
        apply_transpose(&E, l2, tmp);
        for (int j = 0; j < n; j++) l0[j] += tmp[j];
        for (int r = 0; r < nrec; r++) {
            l0[rec_ix[r]] += w[((size_t)m * nrec + r) * 2 + 0];
            l0[nn + rec_ix[r]] += w[((size_t)m * nrec + r) * 2 + 1];
        }
        apply_transpose(&F, l0, gradf + (size_t)(m - 1) * n);
        double *t = l2;
        l2 = l1;
        l1 = l0;
        l0 = t;
    }
    free(l0); free(l1); free(l2); free(tmp);
    free_cols(&B); free_cols(&E); free_cols(&F);
}

/* ---------------------------------------------------------------------------
 * H_II and the cost gradient at theta for data y (Alg. 1 steps 6-10, Eq.
 * H2_numerics, Thm 2's H_2), cost L = 1/2 sum_m sum_r r^T C^-1 r, r = y - g(theta),
 * C = sigma^2 I:
 *   step 6-7: primal solve, w = C^-1 r (the data-side derivative of L, sign aside),
 *   step 8:   dual solve, dJ/df^m for J = sum w . g (ref_adjoint),
 *   step 9-10: with f^m = S(t_m) P(x_s, z_s, M) on the 6x6 patch,
 *     H_II[a][b] = - sum_m sum_patch dJ/df^m d2 f^m / dtheta_a dtheta_b,
 *     grad[a]    = - sum_m sum_patch dJ/df^m d f^m / dtheta_a   (= dL/dtheta_a).
 * d f / d(x_s, z_s) act on the delta / delta' weights of that axis, d f / dm_k
 * select the k-th moment term, d f / d(t_s, w_s) act on S; d2 f / dm dm = 0.
 * Returns 0, or -1 if the source patch leaves the interior.
 * ------------------------------------------------------------------------- */
int ref_hessian_ii(int nx, int nz, double h, double dt, int nsteps, const double *lam,
                   const double *mu, const double *nu, int nrec, const int *rec_ix,
                   const double *theta, const double *y, double sigma, double *H2, double *grad)
{
    size_t nn = (size_t)nx * nz, nrow = (size_t)(nsteps + 1) * nrec * 2;
    int i0, j0;
    double px[36], pz[36];
    if (ref_source_patch(theta, nx, nz, h, &i0, &j0, px, pz) != 0) return -1;
    double *g = malloc(sizeof(double) * nrow), *w = malloc(sizeof(double) * nrow);
    ref_forward(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, theta, g);
    for (size_t k = 0; k < nrow; k++) w[k] = (y[k] - g[k]) / (sigma * sigma);
    double *gf = malloc(sizeof(double) * (size_t)nsteps * 2 * nn);
    ref_adjoint(nx, nz, h, dt, nsteps, lam, mu, nu, nrec, rec_ix, w, gf);

    /* weights of both axes and their first and second derivatives in x_s / z_s:
     * W[axis][order][kind][a]: kind 0 delta, 1 delta' */
    double W[2][3][2][6];
    for (int axis = 0; axis < 2; axis++) {
        double q = theta[axis] / h, al = q - floor(q);
        ref_delta_1d(al, h, W[axis][0][0], W[axis][0][1]);
        ref_delta_1d_dxs(al, h, W[axis][1][0], W[axis][1][1]);
        ref_delta_1d_dxs2(al, h, W[axis][2][0], W[axis][2][1]);
    }
    /* P_c = sum_k m_k X_k Z_k: c = x: (m_xx: delta' x delta), (m_xz: delta x delta');
     *                          c = z: (m_xz: delta' x delta), (m_zz: delta x delta') */
    const int term_m[2][2] = {{4, 5}, {5, 6}};
    const int term_xk[2][2] = {{1, 0}, {1, 0}};   /* kind of the x factor */
    double Hs[NT * NT], gs[NT];
    memset(Hs, 0, sizeof(Hs));
    memset(gs, 0, sizeof(gs));
    for (int m = 0; m < nsteps; m++) {
        double sd[6];
        ref_stf_derivs(m * dt, theta[2], theta[3], sd);
        for (int c = 0; c < 2; c++)
            for (int b = 0; b < 6; b++)
                for (int a = 0; a < 6; a++) {
                    double lamv = gf[(size_t)m * 2 * nn + (size_t)c * nn + (size_t)(j0 + b) * nx + (i0 + a)];
                    if (lamv == 0.0) continue;
                    /* dP/dtheta and d2P/dtheta2 of this node for the spatial parameters
                     * (x_s, z_s, m_xx, m_xz, m_zz), S-derivatives for t_s, w_s */
                    for (int p = 0; p < NT; p++)
                        for (int q = p; q < NT; q++) {
                            int ordx = (p == 0) + (q == 0), ordz = (p == 1) + (q == 1);
                            int nt = (p == 2 || p == 3) + (q == 2 || q == 3);
                            int nm = (p >= 4) + (q >= 4);
                            if (nm == 2) continue;
                            double P = 0.0;
                            for (int k = 0; k < 2; k++) {
                                int mk = term_m[c][k];
                                double coef = theta[mk];
                                if (nm == 1) coef = (p == mk || q == mk) ? 1.0 : 0.0;
                                int xk = term_xk[c][k], zk = 1 - xk;
                                P += coef * W[0][ordx][xk][a] * W[1][ordz][zk][b];
                            }
                            double S;
                            if (nt == 0)
                                S = sd[0];
                            else if (nt == 1)
                                S = ((p == 2 || q == 2) ? sd[1] : sd[2]);
                            else
                                S = (p == 2 && q == 2) ? sd[3] : ((p == 3 && q == 3) ? sd[5] : sd[4]);
                            Hs[p * NT + q] += lamv * S * P;
                        }
                    for (int p = 0; p < NT; p++) {
                        int ordx = (p == 0), ordz = (p == 1);
                        double P = 0.0;
                        for (int k = 0; k < 2; k++) {
                            int mk = term_m[c][k];
                            double coef = p >= 4 ? (p == mk ? 1.0 : 0.0) : theta[mk];
                            int xk = term_xk[c][k], zk = 1 - xk;
                            P += coef * W[0][ordx][xk][a] * W[1][ordz][zk][b];
                        }
                        double S = p == 2 ? sd[1] : (p == 3 ? sd[2] : sd[0]);
                        gs[p] += lamv * S * P;
                    }
                }
    }
    for (int p = 0; p < NT; p++) {
        if (grad) grad[p] = -gs[p];
        for (int q = p; q < NT; q++) H2[p * NT + q] = H2[q * NT + p] = -Hs[p * NT + q];
    }
    free(g); free(w); free(gf);
    return 0;
}
