// The node update of stencil_cell.cuh on packed FP32 pairs (Sec. 3.3.1, Eq.
// Full_Disc), shared by the cluster-resident kernel and the two-step TMA kernel.
// A column's two components (x, z) sit side by side in a slot, and the update of u_x and of u_z
// runs through the same sequence of operations with their own coefficients, so
// each step of it is one two-wide instruction (fma/mul/add .f32x2, rounded per
// component exactly like the scalar fmaf/fmul/fadd).  Every value is computed by
// the same operations in the same order as pair_update, so the bits are those of
// the streaming kernels.
#pragma once

#include "stencil_cell.cuh"

namespace oed {

// a row's coefficients as (x, z) pairs: operator term A = a*lap + vs*dv_s +
// vn*dv_n + ds*d_s + dn*d_n, and the absorbing speeds (c_p, c_s) dt/h
struct __align__(16) KP {
    float2 a, vs, vn, ds, dn, c, pad0, pad1;
};

__device__ __forceinline__ KP pack_coef(const FacCoef<float> &f)
{
    KP k;
    k.a = make_float2(f.axx, f.azx);
    k.vs = make_float2(f.axzp, f.azzp);
    k.vn = make_float2(f.naxzm, f.nazzm);
    k.ds = make_float2(f.px, f.pz);
    k.dn = make_float2(f.nqx, f.nqz);
    k.c = make_float2(f.cp, f.cs);
    k.pad0 = k.pad1 = make_float2(0.0f, 0.0f);
    return k;
}

// the coefficients that the update and the absorbing rows read are equal
__device__ __forceinline__ bool kp_equal(const KP &a, const KP &b)
{
    return a.a.x == b.a.x && a.a.y == b.a.y && a.vs.x == b.vs.x && a.vs.y == b.vs.y && a.vn.x == b.vn.x &&
           a.vn.y == b.vn.y && a.ds.x == b.ds.x && a.ds.y == b.ds.y && a.dn.x == b.dn.x && a.dn.y == b.dn.y &&
           a.c.x == b.c.x && a.c.y == b.c.y;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once per component, in two forms with the same bits: fma(b, -1, a) (the
// product b * -1 is exact) and the packed subtract sub.rn.f32x2.  The cluster-resident
// kernel runs faster with the second (PS), the two-step TMA kernel with the first.
template <bool PS>
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    if constexpr (PS) {
        float2 d;
        asm("{\n\t.reg .b64 x, y, z;\n\t"
            "mov.b64 x, {%2, %3};\n\t"
            "mov.b64 y, {%4, %5};\n\t"
            "sub.rn.f32x2 z, x, y;\n\t"
            "mov.b64 {%0, %1}, z;\n\t}"
            : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return d;
    } else {
        return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
    }
}

// Row2 with each quantity as a (x, z) pair per column a = c, b = c+1; the east - west
// differences, which enter the other component's update, are stored swapped (z, x)
struct Row2P {
    float2 ca, cb;   // centre values
    float2 la, lb;   // (e - c) - (c - w)
    float2 da, db;   // (dz, dx): east - west differences, swapped
    float2 va, vb;   // south row minus this row
};

template <bool PS = false>
__device__ __forceinline__ void row_fromP(float2 w, float4 m, float2 e, Row2P &r)
{
    r.ca = make_float2(m.x, m.y);
    r.cb = make_float2(m.z, m.w);
    const float2 t = sub2<PS>(r.cb, r.ca);
    r.la = sub2<PS>(t, sub2<PS>(r.ca, w));
    r.lb = sub2<PS>(sub2<PS>(e, r.cb), t);
    r.da = make_float2(m.w - w.y, m.z - w.x);
    r.db = make_float2(e.y - m.y, e.x - m.x);
}

template <bool PS = false>
__device__ __forceinline__ void southP(Row2P &c, const Row2P &s)
{
    c.va = sub2<PS>(s.ca, c.ca);
    c.vb = sub2<PS>(s.cb, c.cb);
}

// u^{m+1} of the pair (u holds u^{m-1} on entry, slot order x_a, z_a, x_b, z_b)
template <bool PS = false>
__device__ __forceinline__ void pair_updateP(const KP &K, const Row2P &n, const Row2P &c, const Row2P &s,
                                             float4 &u)
{
    float2 A = fma2(K.a, c.la, sub2<PS>(c.ca, make_float2(u.x, u.y)));
    A = fma2(K.vs, c.va, A);
    A = fma2(K.vn, n.va, A);
    A = fma2(K.ds, s.da, A);
    A = fma2(K.dn, n.da, A);
    float2 B = fma2(K.a, c.lb, sub2<PS>(c.cb, make_float2(u.z, u.w)));
    B = fma2(K.vs, c.vb, B);
    B = fma2(K.vn, n.vb, B);
    B = fma2(K.ds, s.db, B);
    B = fma2(K.dn, n.db, B);
    const float2 xa = add2(c.ca, A);
    const float2 xb = add2(c.cb, B);
    u = make_float4(xa.x, xa.y, xb.x, xb.y);
}

// the absorbing rows and side columns of stencil_cell.cuh's absorbing()
__device__ __forceinline__ void absorbingP(float2 cpcs, float4 nv, const Row2P &c, bool bottom, int kind, float4 &u)
{
    const float cp = cpcs.x, cs = cpcs.y;
    if (bottom) {
        u.x = absorb(c.ca.x, nv.x, cs);
        u.z = absorb(c.cb.x, nv.z, cs);
        u.y = absorb(c.ca.y, nv.y, cp);
        u.w = absorb(c.cb.y, nv.w, cp);
    }
    if (kind & 1) {
        u.x = absorb(c.ca.x, c.cb.x, cp);
        u.y = absorb(c.ca.y, c.cb.y, cs);
    }
    if (kind & 2) {
        u.z = absorb(c.cb.x, c.ca.x, cp);
        u.w = absorb(c.cb.y, c.ca.y, cs);
    }
    if (kind & 4) {   // column nx-1: its east - west difference is -west (the ghost east is 0)
        u.x = absorb(c.ca.x, -c.da.y, cp);
        u.y = absorb(c.ca.y, -c.da.x, cs);
        u.z = 0.0f;
        u.w = 0.0f;
    }
}

}  // namespace oed
