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


// Operator term A_x of FacCoef (dt^2/nu times (A_h u)_x) from the differences
// around the node, accumulated onto d = u^m - u^{m-1}: lap = (x_e - x_c) - (x_c - x_w),
// dvs = x_s - x_c, dvn = x_c - x_n, dzs / dzn = east - west of u_z on the south / north row.
template <typename real>
__device__ __forceinline__ real op_x(const FacCoef<real> &K, real d, real lap, real dvs, real dvn, real dzs,
                                     real dzn)
{
    real a = fma_(K.axx, lap, d);
    a = fma_(K.axzp, dvs, a);
    a = fma_(K.naxzm, dvn, a);
    a = fma_(K.px, dzs, a);
    return fma_(K.nqx, dzn, a);
}

// the same for u_z (roles of the components exchanged)
template <typename real>
__device__ __forceinline__ real op_z(const FacCoef<real> &K, real d, real lap, real dws, real dwn, real dxs,
                                     real dxn)
{
    real a = fma_(K.azx, lap, d);
    a = fma_(K.azzp, dws, a);
    a = fma_(K.nazzm, dwn, a);
    a = fma_(K.pz, dxs, a);
    return fma_(K.nqz, dxn, a);
}

// u^{m+1} = u^m + ((u^m - u^{m-1}) + A), with A accumulated onto u^m - u^{m-1} (op_x,
// op_z): every rounding before the last is at the scale of the increment, not of u
template <typename real>
__device__ __forceinline__ real leap(real u, real dA)
{
    return u + dA;
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
    ux = leap(xc[1], op_x(K, xc[1] - xm, lx, xs[1] - xc[1], xc[1] - xr[1], zs[2] - zs[0], zr[2] - zr[0]));
    uz = leap(zc[1], op_z(K, zc[1] - zm, lz, zs[1] - zc[1], zc[1] - zr[1], xs[2] - xs[0], xr[2] - xr[0]));
}

// ------------------------------------------------------------------------------
// The same update for a thread owning the column pair (c, c+1), FP32, as used by the
// cluster-resident and the TMA streaming kernels: every value below is computed by
// the same operations, in the same order, as node_update above.

// One grid row as seen by the thread owning columns (c, c+1): per component the
// two centre values, the two (e - c) - (c - w) second differences, the two
// east - west differences (cross terms of the other component) and, once the row
// below is known, the two south differences (row below minus this row).
struct Row2 {
    float xa, xb, za, zb;
    float lxa, lxb, lza, lzb;
    float dxa, dxb, dza, dzb;
    float vxa, vxb, vza, vzb;
};

// w = (x, z) of the west column, m = the pair, e = (x, z) of the east column
__device__ __forceinline__ void row_from(float2 w, float4 m, float2 e, Row2 &r)
{
    r.xa = m.x;
    r.za = m.y;
    r.xb = m.z;
    r.zb = m.w;
    r.lxa = (m.z - m.x) - (m.x - w.x);
    r.lxb = (e.x - m.z) - (m.z - m.x);
    r.lza = (m.w - m.y) - (m.y - w.y);
    r.lzb = (e.y - m.w) - (m.w - m.y);
    r.dxa = m.z - w.x;
    r.dxb = e.x - m.x;
    r.dza = m.w - w.y;
    r.dzb = e.y - m.y;
}

// south differences of row c once its south row s is loaded
__device__ __forceinline__ void south(Row2 &c, const Row2 &s)
{
    c.vxa = s.xa - c.xa;
    c.vxb = s.xb - c.xb;
    c.vza = s.za - c.za;
    c.vzb = s.zb - c.zb;
}

// u^{m+1} of the pair from the rows n, c, s (the node update of stencil_cell.cuh);
// n supplies the north differences (its south ones) and the north cross terms.
// u holds u^{m-1} on entry, in slot order (x_a, z_a, x_b, z_b).
__device__ __forceinline__ void pair_update(const FacCoef<float> &K, const Row2 &n, const Row2 &c,
                                            const Row2 &s, float4 &u)
{
    u.x = leap(c.xa, op_x(K, c.xa - u.x, c.lxa, c.vxa, n.vxa, s.dza, n.dza));
    u.z = leap(c.xb, op_x(K, c.xb - u.z, c.lxb, c.vxb, n.vxb, s.dzb, n.dzb));
    u.y = leap(c.za, op_z(K, c.za - u.y, c.lza, c.vza, n.vza, s.dxa, n.dxa));
    u.w = leap(c.zb, op_z(K, c.zb - u.w, c.lzb, c.vzb, n.vzb, s.dxb, n.dxb));
}

// Absorbing rows: the bottom row from its north neighbour, then the side columns
// (which take precedence at the corners) from their interior neighbour.  kind:
// bit 0 node c is column 0, bit 1 node c+1 is column nx-1, bit 2 node c is column
// nx-1 (node c+1 is then the ghost and stays zero).
// (nv: the north row's slot, used by the bottom row only)
__device__ __forceinline__ void absorbing(float cp, float cs, float4 nv, const Row2 &c, bool bottom,
                                          int kind, float4 &u)
{
    if (bottom) {
        u.x = absorb(c.xa, nv.x, cs);
        u.z = absorb(c.xb, nv.z, cs);
        u.y = absorb(c.za, nv.y, cp);
        u.w = absorb(c.zb, nv.w, cp);
    }
    if (kind & 1) {
        u.x = absorb(c.xa, c.xb, cp);
        u.y = absorb(c.za, c.zb, cs);
    }
    if (kind & 2) {
        u.z = absorb(c.xb, c.xa, cp);
        u.w = absorb(c.zb, c.za, cs);
    }
    if (kind & 4) {   // column nx-1: its east - west difference is -west (the ghost east is 0)
        u.x = absorb(c.xa, -c.dxa, cp);
        u.y = absorb(c.za, -c.dza, cs);
        u.z = 0.0f;
        u.w = 0.0f;
    }
}

}  // namespace oed
