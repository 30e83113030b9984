// reed_physics.cuh -- interatomic potentials and stopping used inside the
// track step.  All functions are generic over the arithmetic type R (float
// for the mixed-precision form, double for the plain FP64 path) and read the
// parameters from a HotParams<R> block, so the FP32 form runs without any
// double-precision instruction.
#pragma once

#include "reed_common.cuh"

// ZBL universal screening (Sec. 2 "First"; Ziegler, Biersack, Littmark 1985):
// phi(x) = sum_i c_i exp(-d_i x) with x = r / a_U,
// c = {0.18175, 0.50986, 0.28022, 0.02817}, d = {3.1998, 0.94229, 0.4029, 0.20162}.
// Exponentials are evaluated as 2^(-d_i log2(e) x).
template <typename R> struct Zbl {
    __device__ static __forceinline__ void eval(R r, R ir, R k, R ia, R& V, R& dV)
    {
        const R x = r * ia;
        const R e0 = Mth<R>::exp2n(R(-3.19980 * 1.4426950408889634) * x);
        const R e1 = Mth<R>::exp2n(R(-0.94229 * 1.4426950408889634) * x);
        const R e2 = Mth<R>::exp2n(R(-0.40290 * 1.4426950408889634) * x);
        const R e3 = Mth<R>::exp2n(R(-0.20162 * 1.4426950408889634) * x);
        const R phi = R(0.18175) * e0 + R(0.50986) * e1 + R(0.28022) * e2 + R(0.02817) * e3;
        const R dphi = -(R(0.18175 * 3.19980) * e0 + R(0.50986 * 0.94229) * e1 +
                         R(0.28022 * 0.40290) * e2 + R(0.02817 * 0.20162) * e3);
        const R kr = k * ir;
        V = kr * phi;
        dV = kr * (dphi * ia - phi * ir);
    }
};

// C2 quintic taper S(r): 1 below lo, 0 above lo + 1/inv_w.  Writes dS/dr.
template <typename R> __device__ __forceinline__ R taper(R r, R lo, R inv_w, R& dS)
{
    const R t = (r - lo) * inv_w;
    if (t <= R(0)) { dS = R(0); return R(1); }
    if (t >= R(1)) { dS = R(0); return R(0); }
    const R t2 = t * t, u = R(1) - t;
    dS = R(-30) * t2 * u * u * inv_w;
    return R(1) - t2 * t * (R(10) - R(15) * t + R(6) * t2);
}

// Centred cubic B-spline of unit knot spacing and its derivative.
template <typename R> __device__ __forceinline__ R bspline3(R u, R& du)
{
    const R au = fabs(u), sg = u < R(0) ? R(-1) : R(1);
    if (au >= R(2)) { du = R(0); return R(0); }
    if (au >= R(1)) {
        const R q = R(2) - au;
        du = -sg * R(0.5) * q * q;
        return q * q * q * R(1.0 / 6.0);
    }
    du = sg * (R(-2) * au + R(1.5) * au * au);
    return R(2.0 / 3.0) - au * au + R(0.5) * au * au * au;
}

// Ion-target pair energy U = V_ZBL(r) exp(c(r)) S(r), c(r) = sum_i c_i
// B_i(ln r) (Sec. 2 "First" with a smooth correction).  Returns dU/dr / r
// (force on the atom = -that * d, on the ion = +that * d, d = x_atom - x_ion);
// writes U and the local-density weight S(r) exp(-r / lam).
template <typename R>
__device__ __forceinline__ R ion_pair(const HotParams<R>& H, int spline_on, int rho_on, int s, R r2, R& U,
                                      R& rho_w)
{
    const R ir = Mth<R>::rsqrt(r2);
    const R r = r2 * ir;
    R V, dV;
    Zbl<R>::eval(r, ir, H.zk[s], H.zia[s], V, dV);
    if (spline_on) {
        const R lr = Mth<R>::log(r);
        R c = R(0), dc = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            R du;
            const R b = bspline3<R>((lr - H.spline_ctr[i]) * H.spline_invh, du);
            c += H.spline_c[i] * b;
            dc += H.spline_c[i] * du;
        }
        dc *= H.spline_invh * ir;
        const R ec = Mth<R>::exp(c);
        dV = (dV + V * dc) * ec;
        V *= ec;
    }
    R dS;
    const R S = taper<R>(r, H.rt, H.inv_tw, dS);
    U = V * S;
    rho_w = rho_on ? S * Mth<R>::exp(-r * H.lam_inv) : R(0);
    return (dV * S + V * dS) * ir;
}

// ---------------------------------------------------------------------------
// Tersoff Si(C) (PRB 38, 9902) blended into Si-Si ZBL at short range:
//   V_ab = (1 - s) fc (fR + b_ab fA) + s Z,   E = 1/2 sum_{a != b} V_ab,
//   b_ab = (1 + beta^n zeta_ab^n)^(-1/2n),
//   zeta_ab = sum_{k != a,b} fc(r_ak) g(cos theta_bak),
//   g(c) = 1 + C^2/d^2 - C^2 / (d^2 + (h - c)^2).
// ---------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R ters_fc(const HotParams<R>& H, R r, R& dfc)
{
    if (r <= H.tRmD) { dfc = R(0); return R(1); }
    if (r >= H.tcut) { dfc = R(0); return R(0); }
    const R q = H.tq * (r - H.tR);
    dfc = H.tdq * Mth<R>::cos(q);
    return R(0.5) - R(0.5) * Mth<R>::sin(q);
}

// g is evaluated as 1 + (C^2/d^2) q^2 / (d^2 + q^2), q = h - cos theta, which
// equals the textbook form without its cancellation (C^2/d^2 ~ 4e7 for Si).
template <typename R> __device__ __forceinline__ R ters_g(const HotParams<R>& H, R c, R& dg)
{
    const R q = H.th - c;
    const R iden = Mth<R>::rcp(H.td2 + q * q);
    dg = R(-2) * H.tc2 * q * iden * iden;
    return R(1) + H.tc2d2 * q * q * iden;
}

template <typename R> __device__ __forceinline__ R ters_b(const HotParams<R>& H, R zeta, R& db)
{
    if (zeta <= R(0)) { db = R(0); return R(1); }
    const R zn = Mth<R>::pow(zeta, H.tn);          // zeta^n
    const R q = R(1) + H.tbn * zn;                 // 1 + beta^n zeta^n
    const R b = Mth<R>::pow(q, H.tmhn);            // q^(-1/2n)
    db = R(-0.5) * H.tbn * zn * Mth<R>::rcp(zeta * q) * b;
    return b;
}

// V_ab at fixed bond order b, given fc(r) and its derivative: value V,
// radial derivative dV, and pre_fA = (1 - s) fc fA (the coefficient of b in V_ab).
template <typename R>
__device__ __forceinline__ void ters_pair(const HotParams<R>& H, R r, R fc, R dfc, R b, R& V, R& dV, R& pre_fA)
{
    const R fR = H.tA * Mth<R>::exp(-H.tl1 * r);
    const R fA = -H.tB * Mth<R>::exp(-H.tl2 * r);
    const R VT = fc * (fR + b * fA);
    const R dVT = dfc * (fR + b * fA) - fc * (H.tl1 * fR + b * H.tl2 * fA);
    R ds;
    const R s = taper<R>(r, H.t_blo, H.t_binvw, ds);
    pre_fA = (R(1) - s) * fc * fA;
    if (s > R(0)) {
        R Vz, dVz;
        Zbl<R>::eval(r, Mth<R>::rcp(r), H.t_zk, H.t_zia, Vz, dVz);
        V = (R(1) - s) * VT + s * Vz;
        dV = (R(1) - s) * dVT + ds * (Vz - VT) + s * dVz;
    } else {
        V = VT;
        dV = dVT;
    }
}

// Buckingham pair A exp(-r/rho) - C/r^6 for species pair p = s_i + s_j, with
// ZBL below b_lo (quintic blend to b_hi) and a taper to zero at b_rc.
// Returns dU/dr / r, writes U.
template <typename R> __device__ __forceinline__ R buck_pair(const HotParams<R>& H, int p, R r2, R& U)
{
    const R ir = Mth<R>::rsqrt(r2);
    const R r = r2 * ir;
    R Vb = R(0), dVb = R(0);
    if (H.bA[p] != R(0) || H.bC[p] != R(0)) {
        const R e = H.bA[p] * Mth<R>::exp(-r * H.brho_inv[p]);
        const R ir2 = ir * ir, ir6 = ir2 * ir2 * ir2;
        Vb = e - H.bC[p] * ir6;
        dVb = -e * H.brho_inv[p] + R(6) * H.bC[p] * ir6 * ir;
    }
    R ds;
    const R s = taper<R>(r, H.b_lo, H.b_binvw, ds);
    R V = Vb, dV = dVb;
    if (s > R(0)) {
        R Vz, dVz;
        Zbl<R>::eval(r, ir, H.b_zk[p], H.b_zia[p], Vz, dVz);
        V = (R(1) - s) * Vb + s * Vz;
        dV = (R(1) - s) * dVb + ds * (Vz - Vb) + s * dVz;
    }
    R dS;
    const R S = taper<R>(r, H.b_rt, H.b_rinvw, dS);
    U = V * S;
    return (dV * S + V * dS) * ir;
}
