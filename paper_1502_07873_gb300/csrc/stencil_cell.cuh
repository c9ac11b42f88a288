// The node update of the leap-frog scheme (Sec. 3.3.1, Eq. Full_Disc) in the
// regrouped form of FacCoef, shared by every stencil kernel.  Each rounding step is
// spelled out (explicit multiply-adds, the force term multiplied and added with
// round-to-nearest intrinsics that the compiler may not contract), so the
// streaming, TMA and cluster-resident kernels produce the same bits for the same
// solve.
#pragma once
#include "oed_internal.cuh"

namespace oed {

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float add_force(float u, float S, float w) { return __fadd_rn(u, __fmul_rn(S, w)); }
__device__ __forceinline__ double add_force(double u, double S, double w) { return __dadd_rn(u, __dmul_rn(S, w)); }

__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }

// Operator term A_x of FacCoef (dt^2/nu times (A_h u)_x) from the differences
// around the node: lap = (x_e - x_c) - (x_c - x_w), dvs = x_s - x_c, dvn = x_c - x_n,
// dzs / dzn = east - west of u_z on the south / north row.
template <typename real>
__device__ __forceinline__ real op_x(const FacCoef<real> &K, real lap, real dvs, real dvn, real dzs, real dzn)
{
    real a = mul_(K.axx, lap);
    a = fma_(K.axzp, dvs, a);
    a = fma_(K.naxzm, dvn, a);
    a = fma_(K.px, dzs, a);
    return fma_(K.nqx, dzn, a);
}

// the same for u_z (roles of the components exchanged)
template <typename real>
__device__ __forceinline__ real op_z(const FacCoef<real> &K, real lap, real dws, real dwn, real dxs, real dxn)
{
    real a = mul_(K.azx, lap);
    a = fma_(K.azzp, dws, a);
    a = fma_(K.nazzm, dwn, a);
    a = fma_(K.pz, dxs, a);
    return fma_(K.nqz, dxn, a);
}

// u^{m+1} = u^m + ((u^m - u^{m-1}) + A): the only rounding at the scale of u is the last
template <typename real>
__device__ __forceinline__ real leap(real u, real um, real A)
{
    return u + ((u - um) + A);
}

// first-order absorbing node, forward in time: u + c dt/h (u_inward - u)
template <typename real>
__device__ __forceinline__ real absorb(real u, real inward, real c)
{
    return fma_(c, inward - u, u);
}

// u^{m+1} at one node from the 3x3 neighbourhood of u^m (rows n = j-1, c = j,
// s = j+1; columns [0] = i-1, [1] = i, [2] = i+1) and its u^{m-1} (xm, zm),
// without the force term.
//   side:   0 interior column, 1 left (i = 0), 2 right (i = nx-1): absorbing rule
//           (it takes precedence at the corners)
//   bottom: j = nz-1 (absorbing), top: j = 0 (free-surface closure: the north
//           terms are taken on the row itself, with the surface-row coefficients)
template <typename real>
__device__ __forceinline__ void node_update(const FacCoef<real> &K, const real *xn, const real *xc,
                                            const real *xs, const real *zn, const real *zc,
                                            const real *zs, real xm, real zm, int side, bool bottom,
                                            bool top, real &ux, real &uz)
{
    if (side) {
        const real xi = side == 1 ? xc[2] : xc[0];
        const real zi = side == 1 ? zc[2] : zc[0];
        ux = absorb(xc[1], xi, K.cp);
        uz = absorb(zc[1], zi, K.cs);
        return;
    }
    if (bottom) {
        ux = absorb(xc[1], xn[1], K.cs);
        uz = absorb(zc[1], zn[1], K.cp);
        return;
    }
    const real *xr = top ? xc : xn, *zr = top ? zc : zn;   // top: dv_n = 0, cross terms on row 0
    const real lx = (xc[2] - xc[1]) - (xc[1] - xc[0]);
    const real lz = (zc[2] - zc[1]) - (zc[1] - zc[0]);
    ux = leap(xc[1], xm, op_x(K, lx, xs[1] - xc[1], xc[1] - xr[1], zs[2] - zs[0], zr[2] - zr[0]));
    uz = leap(zc[1], zm, op_z(K, lz, zs[1] - zc[1], zc[1] - zr[1], xs[2] - xs[0], xr[2] - xr[0]));
}

}  // namespace oed
