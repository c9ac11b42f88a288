// Source discretisation and medium coefficients (device side).
//
//  - k_sources: for every solve, the perturbed parameter vector theta +/- d_j e_j
//    (central finite differences, 2*7 + 1 solves per node), the regularised
//    delta / delta' weights of Sec. 3.3.2 item 2 (six points k-2..k+3, fourth-order
//    moments, C^2 in x_s) combined into the force density f = M grad(delta)
//    (Eq. source), and the Gaussian source time function of Sec. 4.1
//    S(t) = w/sqrt(2 pi) exp(-w^2 (t - t_s)^2 / 2) sampled at every step.
//    All of it in FP64, stored in the stencil's precision.
//  - k_rows: per-row stencil coefficients of the leap-frog update for a medium
//    layered in depth (lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2, Sec. 2.1).
#include "oed_internal.cuh"

namespace oed {

// Regularised delta and delta' at nodes k-2..k+3 for offset a = (x_s - x_k)/h
// (Sec. 3.3.2 item 2).  Horner form of the printed polynomials.
__device__ void delta_weights(double a, double h, double *d, double *dp)
{
    const double P = a * a * a * a * a *
                     (5.0 / 3.0 + a * (-7.0 / 24.0 + a * (-17.0 / 12.0 + a * (9.0 / 8.0 - a / 4.0))));
    const double R = a * a * a * a * (-25.0 / 12.0 + a * (-3.0 / 4.0 + a * (59.0 / 12.0 + a * (-4.0 + a))));
    const double ih = 1.0 / h, ih2 = ih * ih;
    d[0] = (a * (1.0 / 12.0 + a * (-1.0 / 24.0 + a * (-1.0 / 12.0 - 19.0 / 24.0 * a))) + P) * ih;
    d[1] = (a * (-2.0 / 3.0 + a * (2.0 / 3.0 + a * (1.0 / 6.0 + 4.0 * a))) - 5.0 * P) * ih;
    d[2] = (1.0 + a * a * (-5.0 / 4.0 - 97.0 / 12.0 * a * a) + 10.0 * P) * ih;
    d[3] = (a * (2.0 / 3.0 + a * (2.0 / 3.0 + a * (-1.0 / 6.0 + 49.0 / 6.0 * a))) - 10.0 * P) * ih;
    d[4] = (a * (-1.0 / 12.0 + a * (-1.0 / 24.0 + a * (1.0 / 12.0 - 33.0 / 8.0 * a))) + 5.0 * P) * ih;
    d[5] = (5.0 / 6.0 * a * a * a * a - P) * ih;
    dp[0] = (-1.0 / 12.0 + a * (1.0 / 12.0 + a * (1.0 / 4.0 + 2.0 / 3.0 * a)) + R) * ih2;
    dp[1] = (2.0 / 3.0 + a * (-4.0 / 3.0 + a * (-1.0 / 2.0 - 7.0 / 2.0 * a)) - 5.0 * R) * ih2;
    dp[2] = (a * (5.0 / 2.0 + 22.0 / 3.0 * a * a) + 10.0 * R) * ih2;
    dp[3] = (-2.0 / 3.0 + a * (-4.0 / 3.0 + a * (1.0 / 2.0 - 23.0 / 3.0 * a)) - 10.0 * R) * ih2;
    dp[4] = (1.0 / 12.0 + a * (1.0 / 12.0 + a * (-1.0 / 4.0 + 4.0 * a)) + 5.0 * R) * ih2;
    dp[5] = (-5.0 / 6.0 * a * a * a - R) * ih2;
}

// d/dx_s of the six delta and delta' weights (the forcing derivative of a
// sensitivity solve, Alg. 1 step 2): (1/h) d/dalpha of the printed polynomials.
__device__ void delta_weights_dxs(double a, double h, double *d, double *dp)
{
    const double Pp = a * a * a * a * (25.0 / 3.0 + a * (-7.0 / 4.0 + a * (-119.0 / 12.0 + a * (9.0 - 9.0 / 4.0 * a))));
    const double Rp = a * a * a * (-25.0 / 3.0 + a * (-15.0 / 4.0 + a * (59.0 / 2.0 + a * (-28.0 + 8.0 * a))));
    const double ih2 = 1.0 / (h * h), ih3 = ih2 / h;
    d[0] = (1.0 / 12.0 + a * (-1.0 / 12.0 + a * (-1.0 / 4.0 - 19.0 / 6.0 * a)) + Pp) * ih2;
    d[1] = (-2.0 / 3.0 + a * (4.0 / 3.0 + a * (1.0 / 2.0 + 16.0 * a)) - 5.0 * Pp) * ih2;
    d[2] = (a * (-5.0 / 2.0 - 97.0 / 3.0 * a * a) + 10.0 * Pp) * ih2;
    d[3] = (2.0 / 3.0 + a * (4.0 / 3.0 + a * (-1.0 / 2.0 + 98.0 / 3.0 * a)) - 10.0 * Pp) * ih2;
    d[4] = (-1.0 / 12.0 + a * (-1.0 / 12.0 + a * (1.0 / 4.0 - 33.0 / 2.0 * a)) + 5.0 * Pp) * ih2;
    d[5] = (10.0 / 3.0 * a * a * a - Pp) * ih2;
    dp[0] = (1.0 / 12.0 + a * (1.0 / 2.0 + 2.0 * a) + Rp) * ih3;
    dp[1] = (-4.0 / 3.0 + a * (-1.0 - 21.0 / 2.0 * a) - 5.0 * Rp) * ih3;
    dp[2] = (5.0 / 2.0 + 22.0 * a * a + 10.0 * Rp) * ih3;
    dp[3] = (-4.0 / 3.0 + a * (1.0 - 23.0 * a) - 10.0 * Rp) * ih3;
    dp[4] = (1.0 / 12.0 + a * (-1.0 / 2.0 + 12.0 * a) + 5.0 * Rp) * ih3;
    dp[5] = (-5.0 / 2.0 * a * a - Rp) * ih3;
}

// d2/dx_s2 of the six delta and delta' weights (the forcing's second derivatives,
// Alg. 1 step 9; the regularised delta is C^2 in x_s): (1/h^2) d2/dalpha2 of the
// printed polynomials.
__device__ void delta_weights_dxs2(double a, double h, double *d, double *dp)
{
    const double Ppp = a * a * a * (100.0 / 3.0 + a * (-35.0 / 4.0 + a * (-119.0 / 2.0 + a * (63.0 - 18.0 * a))));
    const double Rpp = a * a * (-25.0 + a * (-15.0 + a * (295.0 / 2.0 + a * (-168.0 + 56.0 * a))));
    const double h3 = h * h * h, h4 = h3 * h;
    d[0] = (-1.0 / 12.0 + a * (-1.0 / 2.0 - 19.0 / 2.0 * a) + Ppp) / h3;
    d[1] = (4.0 / 3.0 + a * (1.0 + 48.0 * a) - 5.0 * Ppp) / h3;
    d[2] = (-5.0 / 2.0 - 97.0 * a * a + 10.0 * Ppp) / h3;
    d[3] = (4.0 / 3.0 + a * (-1.0 + 98.0 * a) - 10.0 * Ppp) / h3;
    d[4] = (-1.0 / 12.0 + a * (1.0 / 2.0 - 99.0 / 2.0 * a) + 5.0 * Ppp) / h3;
    d[5] = (10.0 * a * a - Ppp) / h3;
    dp[0] = (1.0 / 2.0 + 4.0 * a + Rpp) / h4;
    dp[1] = (-1.0 - 21.0 * a - 5.0 * Rpp) / h4;
    dp[2] = (44.0 * a + 10.0 * Rpp) / h4;
    dp[3] = (1.0 - 46.0 * a - 10.0 * Rpp) / h4;
    dp[4] = (-1.0 / 2.0 + 24.0 * a + 5.0 * Rpp) / h4;
    dp[5] = (-5.0 * a - Rpp) / h4;
}

struct FdStep {
    double d[kNT];
};

// Spatial part of M grad(delta) for one parameter vector on its 6x6 support:
// corner (kx - 2, kz - 2); f[b][a] at node (kx - 2 + a, kz - 2 + b).
//   f_x = m_xx delta'(x) delta(z) + m_xz delta(x) delta'(z)
//   f_z = m_xz delta'(x) delta(z) + m_zz delta(x) delta'(z)
// Returns false if x_s / h or z_s / h is not a usable number.
__device__ bool source_patch6(const double *th, double h, int *kx, int *kz, double *fx, double *fz)
{
    const double qx = th[0] / h, qz = th[1] / h;
    const double flx = floor(qx), flz = floor(qz);
    if (!(isfinite(qx) && isfinite(qz) && fabs(flx) < 1e9 && fabs(flz) < 1e9)) return false;
    double dx[6], dpx[6], dz[6], dpz[6];
    delta_weights(qx - flx, h, dx, dpx);
    delta_weights(qz - flz, h, dz, dpz);
    *kx = (int)flx;
    *kz = (int)flz;
    for (int b = 0; b < 6; b++)
        for (int a = 0; a < 6; a++) {
            fx[b * 6 + a] = th[4] * dpx[a] * dz[b] + th[5] * dx[a] * dpz[b];
            fz[b * 6 + a] = th[5] * dpx[a] * dz[b] + th[6] * dx[a] * dpz[b];
        }
    return true;
}

// S(t) of the given kind: OED_STF_GAUSS (Sec. 4.1, w = omega_s) or OED_STF_RICKER
// ((1 - 2a) e^{-a}, a = (pi w (t - ts))^2, w the peak frequency)
__device__ __forceinline__ double stf_value(int kind, double t, double ts, double ws)
{
    const double u = t - ts;
    if (kind == OED_STF_RICKER) {
        double a = 3.141592653589793 * ws * u;
        a = a * a;
        return (1.0 - 2.0 * a) * exp(-a);
    }
    return ws * 0.3989422804014327 * exp(-0.5 * ws * ws * u * u);   // w / sqrt(2 pi) e^{...}
}

// One thread block per solve.  per_node = 1: the node itself (forward map);
// per_node = 15: centre and theta +/- d_j e_j (pairs Jacobian); per_node = 7:
// solve j carries the FP64 difference of the theta + d_j e_j and theta - d_j e_j
// forcings (difference Jacobian; by linearity of the scheme in the forcing its
// seismogram is exactly g(theta + d_j e_j) - g(theta - d_j e_j)).  For j = x_s, z_s
// and the moments the spatial patch differs (the two 6x6 patches are subtracted
// on their 7x7 union); for j = t_s, omega_s the time function differs.
template <typename real>
__global__ void k_sources(const double *__restrict__ theta_nodes, int nsolve, int per_node, int sens,
                          int stf_kind, FdStep step, Geometry g, const RowCoef<real> *__restrict__ rows,
                          SourceDesc<real> *__restrict__ src, real *__restrict__ stf,
                          double *__restrict__ theta_out)
{
    const int s = blockIdx.x;
    if (s >= nsolve) return;
    const int node = s / per_node, p = s % per_node;
    const bool diff = per_node == kND && !sens;
    __shared__ double th[kNT], tp[kNT], tm[kNT];
    __shared__ double w7x[kPatch * kPatch], w7z[kPatch * kPatch];
    __shared__ int corner[3];
    __shared__ int time_diff;
    __shared__ int time_kind;   // sensitivity solves: 0 S, 1 dS/dt_s, 2 dS/domega_s
    if (threadIdx.x < kNT) {
        const int j = threadIdx.x;
        const double v = theta_nodes[(size_t)node * kNT + j];
        double vs = v;
        // pairs form: p = 0 centre, p = 1 + 2j: +d_j, p = 2 + 2j: -d_j
        if (per_node == kNP && p > 0 && j == (p - 1) / 2) vs += ((p - 1) & 1) ? -step.d[j] : step.d[j];
        th[j] = vs;
        tp[j] = v + ((diff && j == p) ? step.d[j] : 0.0);
        tm[j] = v - ((diff && j == p) ? step.d[j] : 0.0);
        theta_out[(size_t)s * kNT + j] = vs;
    }
    for (int k = threadIdx.x; k < kPatch * kPatch; k += blockDim.x) w7x[k] = w7z[k] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double fx[36], fz[36];
        int kx = 0, kz = 0, ok;
        int i0, j0, span;   // span: 6 or 7 nodes of the patch actually used
        time_diff = diff && (p == 2 || p == 3);
        time_kind = (sens && (p == 2 || p == 3)) ? p - 1 : 0;
        if (sens) {
            // Alg. 1 step 2: the forcing of solve j is df/dtheta_j of the discrete source
            const double qx = th[0] / g.h, qz = th[1] / g.h;
            const double flx = floor(qx), flz = floor(qz);
            ok = isfinite(qx) && isfinite(qz) && fabs(flx) < 1e9 && fabs(flz) < 1e9;
            double dx[6], dpx[6], dz[6], dpz[6], ex[6], epx[6], ez[6], epz[6];
            delta_weights(qx - flx, g.h, dx, dpx);
            delta_weights(qz - flz, g.h, dz, dpz);
            delta_weights_dxs(qx - flx, g.h, ex, epx);
            delta_weights_dxs(qz - flz, g.h, ez, epz);
            kx = ok ? (int)flx : 0;
            kz = ok ? (int)flz : 0;
            i0 = kx - 2;
            j0 = kz - 2;
            span = 6;
            const double mxx = th[4], mxz = th[5], mzz = th[6];
            for (int b = 0; b < 6; b++)
                for (int a2 = 0; a2 < 6; a2++) {
                    double vx = 0.0, vz = 0.0;
                    if (p == 0) {
                        vx = mxx * epx[a2] * dz[b] + mxz * ex[a2] * dpz[b];
                        vz = mxz * epx[a2] * dz[b] + mzz * ex[a2] * dpz[b];
                    } else if (p == 1) {
                        vx = mxx * dpx[a2] * ez[b] + mxz * dx[a2] * epz[b];
                        vz = mxz * dpx[a2] * ez[b] + mzz * dx[a2] * epz[b];
                    } else if (p == 2 || p == 3) {
                        vx = mxx * dpx[a2] * dz[b] + mxz * dx[a2] * dpz[b];
                        vz = mxz * dpx[a2] * dz[b] + mzz * dx[a2] * dpz[b];
                    } else if (p == 4) {
                        vx = dpx[a2] * dz[b];
                    } else if (p == 5) {
                        vx = dx[a2] * dpz[b];
                        vz = dpx[a2] * dz[b];
                    } else {
                        vz = dx[a2] * dpz[b];
                    }
                    w7x[b * kPatch + a2] = vx;
                    w7z[b * kPatch + a2] = vz;
                }
        } else if (!diff || time_diff) {
            ok = source_patch6(th, g.h, &kx, &kz, fx, fz);
            i0 = kx - 2;
            j0 = kz - 2;
            span = 6;
            for (int b = 0; b < 6; b++)
                for (int a = 0; a < 6; a++) {
                    w7x[b * kPatch + a] = fx[b * 6 + a];
                    w7z[b * kPatch + a] = fz[b * 6 + a];
                }
        } else {
            double gx[36], gz[36];
            int kx2 = 0, kz2 = 0;
            ok = source_patch6(tp, g.h, &kx, &kz, fx, fz) && source_patch6(tm, g.h, &kx2, &kz2, gx, gz);
            const int kxm = min(kx, kx2), kzm = min(kz, kz2);
            ok = ok && max(kx, kx2) - kxm <= 1 && max(kz, kz2) - kzm <= 1;
            i0 = kxm - 2;
            j0 = kzm - 2;
            span = (kx != kx2 || kz != kz2) ? 7 : 6;
            if (ok) {
                const int ox = kx - kxm, oz = kz - kzm, ox2 = kx2 - kxm, oz2 = kz2 - kzm;
                for (int b = 0; b < 6; b++)
                    for (int a = 0; a < 6; a++) {
                        w7x[(b + oz) * kPatch + a + ox] += fx[b * 6 + a];
                        w7z[(b + oz) * kPatch + a + ox] += fz[b * 6 + a];
                        w7x[(b + oz2) * kPatch + a + ox2] -= gx[b * 6 + a];
                        w7z[(b + oz2) * kPatch + a + ox2] -= gz[b * 6 + a];
                    }
            }
        }
        ok = ok && i0 >= 1 && i0 + span - 1 <= g.nx - 2 && j0 >= 0 && j0 + span - 1 <= g.nz - 2;
        corner[0] = ok ? i0 : -100;
        corner[1] = ok ? j0 : -100;
        corner[2] = ok;
        src[s].i0 = corner[0];
        src[s].j0 = corner[1];
        src[s].ok = ok;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kPatch * kPatch; k += blockDim.x) {
        const int b = k / kPatch;
        const int j = corner[1] + b;
        const double rf = (corner[2] && j <= g.nz - 1) ? (double)rows[j].rf : 0.0;
        src[s].wx[k] = (real)(w7x[k] * rf);
        src[s].wz[k] = (real)(w7z[k] * rf);
    }
    for (int m = threadIdx.x; m < g.nsteps; m += blockDim.x) {
        const double t = m * g.dt;
        double v = time_diff ? stf_value(stf_kind, t, tp[2], tp[3]) - stf_value(stf_kind, t, tm[2], tm[3])
                             : stf_value(stf_kind, t, th[2], th[3]);
        // (sensitivity solves: Gaussian only, the host refuses them for any other kind)
        if (time_kind == 1) v *= th[3] * th[3] * (t - th[2]);                 // dS/dt_s
        if (time_kind == 2) v *= 1.0 / th[3] - th[3] * (t - th[2]) * (t - th[2]);   // dS/domega_s
        stf[(size_t)s * g.nsteps + m] = (real)v;
    }
}

// Per-row coefficients (one thread per row).
template <typename real>
__global__ void k_rows(Geometry g, int nlayers, const double *__restrict__ lay,
                       RowCoef<real> *__restrict__ rows, FacCoef<real> *__restrict__ fac)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.nz) return;
    auto layer_of = [&](int jj) {
        const double z = (jj < 0 ? 0 : (jj >= g.nz ? g.nz - 1 : jj)) * g.h;
        int l = 0;
        for (int q = 0; q < nlayers; q++)
            if (z >= lay[q]) l = q;
        return l;
    };
    auto lam = [&](int jj) {
        int l = layer_of(jj);
        double vp = lay[nlayers + l], vs = lay[2 * nlayers + l], rho = lay[3 * nlayers + l];
        return rho * (vp * vp - 2.0 * vs * vs);
    };
    auto mu = [&](int jj) {
        int l = layer_of(jj);
        double vs = lay[2 * nlayers + l], rho = lay[3 * nlayers + l];
        return rho * vs * vs;
    };
    const int l = layer_of(j);
    const double vp = lay[nlayers + l], vs = lay[2 * nlayers + l], rho = lay[3 * nlayers + l];
    const double h2 = g.h * g.h;
    const double r = g.dt * g.dt / rho;
    const double lc = lam(j), mc = mu(j), pc = lc + 2.0 * mc;
    RowCoef<double> c;
    c.axx = pc * r / h2;
    c.azx = mc * r / h2;
    c.rf = r;
    c.cp = vp * g.dt / g.h;
    c.cs = vs * g.dt / g.h;
    c.pad = 0.0;
    if (j == 0) {
        const double l1 = lam(1), m1 = mu(1), p1 = l1 + 2.0 * m1;
        c.axzp = 2.0 * 0.5 * (mc + m1) * r / h2;
        c.axzm = 0.0;
        c.azzp = 2.0 * 0.5 * (pc + p1) * r / h2;
        c.azzm = 0.0;
        c.lx = lc * r / (2.0 * h2);
        c.mxp = m1 * r / (2.0 * h2);
        c.mxm = mc * r / (2.0 * h2);
        c.mz = mc * r / (2.0 * h2);
        c.lzp = l1 * r / (2.0 * h2);
        c.lzm = lc * r / (2.0 * h2);
    } else {
        const double ls = lam(j + 1), ms = mu(j + 1), ps = ls + 2.0 * ms;
        const double ln = lam(j - 1), mn = mu(j - 1), pn = ln + 2.0 * mn;
        c.axzp = 0.5 * (mc + ms) * r / h2;
        c.axzm = 0.5 * (mn + mc) * r / h2;
        c.azzp = 0.5 * (pc + ps) * r / h2;
        c.azzm = 0.5 * (pn + pc) * r / h2;
        c.lx = lc * r / (4.0 * h2);
        c.mxp = ms * r / (4.0 * h2);
        c.mxm = mn * r / (4.0 * h2);
        c.mz = mc * r / (4.0 * h2);
        c.lzp = ls * r / (4.0 * h2);
        c.lzm = ln * r / (4.0 * h2);
    }
    RowCoef<real> o;
    o.axx = (real)c.axx; o.azx = (real)c.azx; o.axzp = (real)c.axzp; o.axzm = (real)c.axzm;
    o.azzp = (real)c.azzp; o.azzm = (real)c.azzm; o.lx = (real)c.lx; o.mxp = (real)c.mxp;
    o.mxm = (real)c.mxm; o.mz = (real)c.mz; o.lzp = (real)c.lzp; o.lzm = (real)c.lzm;
    o.rf = (real)c.rf; o.cp = (real)c.cp; o.cs = (real)c.cs; o.pad = (real)0;
    rows[j] = o;
    FacCoef<double> f;
    f.axx = c.axx; f.axzp = c.axzp; f.naxzm = -c.axzm;
    f.azx = c.azx; f.azzp = c.azzp; f.nazzm = -c.azzm;
    f.px = c.lx + c.mxp;
    f.pz = c.mz + c.lzp;
    f.nqx = j == 0 ? c.mxm - c.lx : -(c.lx + c.mxm);
    f.nqz = j == 0 ? c.lzm - c.mz : -(c.mz + c.lzm);
    FacCoef<real> q;
    q.axx = (real)f.axx; q.axzp = (real)f.axzp; q.naxzm = (real)f.naxzm; q.px = (real)f.px;
    q.nqx = (real)f.nqx; q.azx = (real)f.azx; q.azzp = (real)f.azzp; q.nazzm = (real)f.nazzm;
    q.pz = (real)f.pz; q.nqz = (real)f.nqz; q.cp = (real)c.cp; q.cs = (real)c.cs;
    q.pad0 = q.pad1 = q.pad2 = q.pad3 = (real)0;
    fac[j] = q;
}

void launch_rows(oed_ctx *ctx, cudaStream_t s)
{
    const int nl = (int)ctx->z_top.size();
    std::vector<double> lay(4 * nl);
    for (int l = 0; l < nl; l++) {
        lay[l] = ctx->z_top[l];
        lay[nl + l] = ctx->vp[l];
        lay[2 * nl + l] = ctx->vs[l];
        lay[3 * nl + l] = ctx->rho[l];
    }
    double *d_lay = nullptr;
    cudaMallocAsync((void **)&d_lay, sizeof(double) * lay.size(), s);
    cudaMemcpyAsync(d_lay, lay.data(), sizeof(double) * lay.size(), cudaMemcpyHostToDevice, s);
    const int nb = (ctx->g.nz + 127) / 128;
    if (ctx->precision == OED_FP64)
        k_rows<double><<<nb, 128, 0, s>>>(ctx->g, nl, d_lay, (RowCoef<double> *)ctx->d_rows,
                                           (FacCoef<double> *)ctx->d_fac);
    else
        k_rows<float><<<nb, 128, 0, s>>>(ctx->g, nl, d_lay, (RowCoef<float> *)ctx->d_rows,
                                          (FacCoef<float> *)ctx->d_fac);
    cudaFreeAsync(d_lay, s);
    cudaStreamSynchronize(s);   // the host vector `lay` must outlive the copy
}

// Cost gradient and H_II from the dual solve (Alg. 1 steps 9-10, Eq. H2_numerics).
// The forcing of a solve is S(t) W on the 6x6 patch, W = dt^2/nu_row P(x_s, z_s, M),
//   P_x = m_xx d'(x) d(z) + m_xz d(x) d'(z),   P_z = m_xz d'(x) d(z) + m_zz d(x) d'(z),
// with d, d' the delta / delta' weights.  acc[t][c][node] = sum_m lambda^{m+1} S_t(t_m)
// (t = S, S_ts, S_w, S_tsts, S_tsw, S_ww), so with dJ/d(S W)^m = lambda^{m+1}
//   d2J/dth_p dth_q = sum_c sum_node acc[time part of (p,q)] * d^k W / (space part of (p,q))
// where t_s, omega_s differentiate S, x_s and z_s the weights of their axis, m_k
// select their moment term (d2/dm dm = 0).  H_II = -d2J (added to H), grad = -dJ.
// One block per solve; thread t < 28 takes the upper-triangle pair t, 28 <= t < 35
// the gradient entry t - 28.
template <typename real>
__global__ void __launch_bounds__(64) k_hii_combine(const double *__restrict__ theta, const double *__restrict__ acc,
                                                    const SourceDesc<real> *__restrict__ src,
                                                    const RowCoef<real> *__restrict__ rows, Geometry g,
                                                    double *__restrict__ H, double *__restrict__ grad,
                                                    int *__restrict__ status)
{
    const int s = blockIdx.x, t = threadIdx.x;
    const double *th = theta + (size_t)s * kNT;
    __shared__ double W[2][3][2][6];   // axis, derivative order, delta / delta', node
    __shared__ double rf[6];
    const bool ok = src[s].ok;
    if (t == 0 && ok) {
        for (int axis = 0; axis < 2; axis++) {
            const double q = th[axis] / g.h, al = q - floor(q);
            delta_weights(al, g.h, W[axis][0][0], W[axis][0][1]);
            delta_weights_dxs(al, g.h, W[axis][1][0], W[axis][1][1]);
            delta_weights_dxs2(al, g.h, W[axis][2][0], W[axis][2][1]);
        }
        for (int b = 0; b < 6; b++) rf[b] = (double)rows[src[s].j0 + b].rf;
    }
    __syncthreads();
    if (t >= 35) return;
    int p, q;
    if (t < 28) {   // upper-triangle pair number t
        p = 0;
        int r = t;
        while (r >= kNT - p) {
            r -= kNT - p;
            p++;
        }
        q = p + r;
    } else {
        p = t - 28;
        q = -1;
    }
    if (!ok) {
        if (t < 28) {
            H[(size_t)s * 49 + p * kNT + q] = NAN;
            H[(size_t)s * 49 + q * kNT + p] = NAN;
        } else if (grad) {
            grad[(size_t)s * kNT + p] = NAN;
        }
        if (t == 0 && status) status[s] = OED_EINVAL;
        return;
    }
    // derivative orders of the two axes, the time part and the moment selection
    const int ordx = (p == 0) + (q == 0), ordz = (p == 1) + (q == 1);
    const int nt = (p == 2 || p == 3) + (q == 2 || q == 3);
    const int nm = (p >= 4) + (q >= 4);
    double v = 0.0;
    if (nm < 2) {
        int tk;   // S-derivative index of acc
        if (nt == 0)
            tk = 0;
        else if (nt == 1)
            tk = (p == 2 || q == 2) ? 1 : 2;
        else
            tk = (p == 2 && q == 2) ? 3 : ((p == 3 && q == 3) ? 5 : 4);
        const double *ac = acc + (size_t)s * 6 * 2 * kPatch * kPatch + (size_t)tk * 2 * kPatch * kPatch;
        // moment terms of each component: (moment index, kind of the x factor; z factor the other)
        const int tm[2][2] = {{4, 5}, {5, 6}};
        const int xk[2][2] = {{1, 0}, {1, 0}};
        for (int c = 0; c < 2; c++)
            for (int b = 0; b < 6; b++)
                for (int a = 0; a < 6; a++) {
                    double P = 0.0;
                    for (int k = 0; k < 2; k++) {
                        const int mk = tm[c][k];
                        double coef = th[mk];
                        if (nm == 1) coef = (p == mk || q == mk) ? 1.0 : 0.0;
                        P += coef * W[0][ordx][xk[c][k]][a] * W[1][ordz][1 - xk[c][k]][b];
                    }
                    v += ac[c * kPatch * kPatch + b * kPatch + a] * rf[b] * P;
                }
    }
    if (t < 28) {
        H[(size_t)s * 49 + p * kNT + q] -= v;
        if (q != p) H[(size_t)s * 49 + q * kNT + p] -= v;
    } else if (grad) {
        grad[(size_t)s * kNT + p] = -v;
    }
    if (t == 0 && status) status[s] = 0;
}

void launch_hii_combine(const oed_ctx *ctx, int nsolve, const double *acc, double *H, double *grad, int *status,
                        cudaStream_t st)
{
    if (nsolve <= 0) return;
    if (ctx->precision == OED_FP64)
        k_hii_combine<double><<<nsolve, 64, 0, st>>>(ctx->d_theta, acc, (const SourceDesc<double> *)ctx->d_src,
                                                     (const RowCoef<double> *)ctx->d_rows, ctx->g, H, grad,
                                                     status);
    else
        k_hii_combine<float><<<nsolve, 64, 0, st>>>(ctx->d_theta, acc, (const SourceDesc<float> *)ctx->d_src,
                                                    (const RowCoef<float> *)ctx->d_rows, ctx->g, H, grad, status);
}

void launch_sources(const oed_ctx *ctx, const double *theta_nodes, int nnode, int per_node,
                    const double *step, cudaStream_t s)
{
    const int sens = (per_node == kND && ctx->jac_mode == OED_JAC_SENSITIVITY) ? 1 : 0;
    FdStep st;
    for (int j = 0; j < kNT; j++) st.d[j] = step ? step[j] : 0.0;
    const int nsolve = nnode * per_node;
    if (nsolve <= 0) return;
    if (ctx->precision == OED_FP64)
        k_sources<double><<<nsolve, 128, 0, s>>>(
            theta_nodes, nsolve, per_node, sens, ctx->stf, st, ctx->g, (const RowCoef<double> *)ctx->d_rows,
            (SourceDesc<double> *)ctx->d_src, (double *)ctx->d_stf, ctx->d_theta);
    else
        k_sources<float><<<nsolve, 128, 0, s>>>(
            theta_nodes, nsolve, per_node, sens, ctx->stf, st, ctx->g, (const RowCoef<float> *)ctx->d_rows,
            (SourceDesc<float> *)ctx->d_src, (float *)ctx->d_stf, ctx->d_theta);
}

}  // namespace oed
