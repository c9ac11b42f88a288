// The node update of the leap-frog scheme (Sec. 3.3.1, Eq. Full_Disc), shared by
// the HBM-streaming and the cluster-resident stencil kernels.
#pragma once
#include "oed_internal.cuh"

namespace oed {

// u^{m+1} at one node from the 3x3 neighbourhood of u^m (rows n = j-1, c = j,
// s = j+1; columns [0] = i-1, [1] = i, [2] = i+1), its u^{m-1} (xm, zm) and the
// force density already scaled by dt^2/nu (fx, fz).
//   side:   0 interior column, 1 left (i = 0), 2 right (i = nx-1): absorbing rule
//   bottom: j = nz-1 (absorbing), top: j = 0 (free surface closure)
template <typename real>
__device__ __forceinline__ void cell_update(const RowCoef<real> &R, const real *xn, const real *xc,
                                            const real *xs, const real *zn, const real *zc,
                                            const real *zs, real xm, real zm, int side, bool bottom,
                                            bool top, real fx, real fz, real &ux, real &uz)
{
    if (side) {
        const real xi = side == 1 ? xc[2] : xc[0];
        const real zi = side == 1 ? zc[2] : zc[0];
        ux = xc[1] + R.cp * (xi - xc[1]);
        uz = zc[1] + R.cs * (zi - zc[1]);
        return;
    }
    if (bottom) {
        ux = xc[1] + R.cs * (xn[1] - xc[1]);
        uz = zc[1] + R.cp * (zn[1] - zc[1]);
        return;
    }
    real Ax = R.axx * (xc[2] - (real)2 * xc[1] + xc[0]) + R.axzp * (xs[1] - xc[1]);
    real Az = R.azx * (zc[2] - (real)2 * zc[1] + zc[0]) + R.azzp * (zs[1] - zc[1]);
    if (!top) {
        Ax += -R.axzm * (xc[1] - xn[1]) + R.lx * ((zs[2] - zn[2]) - (zs[0] - zn[0])) +
              R.mxp * (zs[2] - zs[0]) - R.mxm * (zn[2] - zn[0]);
        Az += -R.azzm * (zc[1] - zn[1]) + R.mz * ((xs[2] - xn[2]) - (xs[0] - xn[0])) +
              R.lzp * (xs[2] - xs[0]) - R.lzm * (xn[2] - xn[0]);
    } else {
        Ax += R.lx * ((zs[2] - zc[2]) - (zs[0] - zc[0])) + R.mxm * (zc[2] - zc[0]) +
              R.mxp * (zs[2] - zs[0]);
        Az += R.mz * ((xs[2] - xc[2]) - (xs[0] - xc[0])) + R.lzm * (xc[2] - xc[0]) +
              R.lzp * (xs[2] - xs[0]);
    }
    ux = (real)2 * xc[1] - xm + Ax + fx;
    uz = (real)2 * zc[1] - zm + Az + fz;
}

}  // namespace oed
