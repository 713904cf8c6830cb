// pair2.cuh -- the penalty norm of two states at once with paired FP32
// arithmetic (fma.rn.f32x2 and friends, one instruction for two lanes of a
// 64-bit register pair).  The formula of penalty_norm in dg_device.cuh, term
// by term; where a product and a sum are contracted into one fused
// multiply-add may differ, so the results agree to FP32 rounding, not bit for
// bit.  The square roots and reciprocals stay scalar; the trigonometric step
// of the eigenvalue, cos(acos(r) / 3), is a polynomial evaluated in pairs
// (2 % faster per step at p = 4 than the arccosine and cosine).
#pragma once
#include <cuda_runtime.h>

#include "dg_stage.cuh"

namespace dg {

struct pf2 {
    float2 v;
};

__device__ __forceinline__ pf2 mk(float a, float b) { return pf2{make_float2(a, b)}; }
__device__ __forceinline__ pf2 sp(float a) { return pf2{make_float2(a, a)}; }
__device__ __forceinline__ pf2 operator+(pf2 a, pf2 b) { return pf2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ pf2 operator-(pf2 a, pf2 b) { return pf2{__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))}; }
__device__ __forceinline__ pf2 operator*(pf2 a, pf2 b) { return pf2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ pf2 fma2(pf2 a, pf2 b, pf2 c) { return pf2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ pf2 neg(pf2 a) { return mk(-a.v.x, -a.v.y); }

// largest eigenvalue of two symmetric 3x3 matrices (sym3_max_eig, paired)
__device__ __forceinline__ pf2 sym3_max_eig2(pf2 a11, pf2 a12, pf2 a13, pf2 a22, pf2 a23, pf2 a33)
{
    const pf2 p1 = fma2(a23, a23, fma2(a13, a13, a12 * a12));
    const pf2 q = (a11 + a22 + a33) * sp(1.0f / 3.0f);
    pf2 b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
    const pf2 p2 = fma2(sp(2.0f), p1, fma2(b33, b33, fma2(b22, b22, b11 * b11)));
    const float ppx = sqrtf(p2.v.x * (1.0f / 6.0f)), ppy = sqrtf(p2.v.y * (1.0f / 6.0f));
    const pf2 ip = mk(1.0f / ppx, 1.0f / ppy);
    b11 = b11 * ip;
    b22 = b22 * ip;
    b33 = b33 * ip;
    const pf2 c12 = a12 * ip, c13 = a13 * ip, c23 = a23 * ip;
    const pf2 m1 = b22 * b33 - c23 * c23, m2 = c12 * b33 - c23 * c13, m3 = c12 * c23 - b22 * c13;
    const pf2 det = fma2(c13, m3, b11 * m1 - c12 * m2);
    const pf2 r = det * sp(0.5f);
    // cos(acos(r) / 3) = cos(2/3 acos(w)) with w = cos(acos(r) / 2) =
    // sqrt((1 + r) / 2) in [0, 1], where it is analytic: a polynomial of
    // degree 7 in w, interpolated at the 8 Chebyshev nodes of [0, 1]
    // (|error| < 3e-8; 1.2e-7 with FP32 Horner steps)
    const pf2 w2 = fma2(sp(0.5f), r, sp(0.5f));
    const pf2 w = mk(sqrtf(fminf(fmaxf(w2.v.x, 0.0f), 1.0f)), sqrtf(fminf(fmaxf(w2.v.y, 0.0f), 1.0f)));
    pf2 c = fma2(sp(0.0011276363f), w, sp(-0.0060893456f));
    c = fma2(c, w, sp(0.016047280f));
    c = fma2(c, w, sp(-0.030235397f));
    c = fma2(c, w, sp(0.052841410f));
    c = fma2(c, w, sp(-0.11103851f));
    c = fma2(c, w, sp(0.57734692f));
    c = fma2(c, w, sp(0.5f));
    const pf2 l = fma2(mk(2.0f * ppx, 2.0f * ppy), c, q);
    // a matrix with p2 = 0 is a multiple of the identity
    return mk(p2.v.x > 0.0f ? l.v.x : q.v.x, p2.v.y > 0.0f ? l.v.y : q.v.y);
}

// penalty_norm of two states (rho, v1, v2, e) with one normal
__device__ __forceinline__ pf2 penalty_norm2(pf2 rho, pf2 v1, pf2 v2, pf2 e, float n1, float n2, const Phys<float> &ph)
{
    const pf2 N1 = sp(n1), N2 = sp(n2), g = sp(ph.gPr);
    const pf2 vn = fma2(v1, N1, v2 * N2), vt = fma2(v2, N1, neg(v1 * N2));
    const pf2 vsq = fma2(v1, v1, v2 * v2);
    const pf2 a41 = neg(fma2(vn * vn, sp(1.0f / 3.0f), vsq)) - g * (e - vsq);
    const pf2 c42 = (sp(4.0f / 3.0f) - g) * vn, c43 = (sp(1.0f) - g) * vt;
    const pf2 s11 = sp(16.0f / 9.0f) * fma2(vn, vn, sp(1.0f));
    const pf2 s12 = sp(4.0f / 3.0f) * (vn * vt);
    const pf2 s13 = sp(4.0f / 3.0f) * (c42 - vn * a41);
    const pf2 s22 = fma2(vt, vt, sp(1.0f));
    const pf2 s23 = c43 - vt * a41;
    const pf2 s33 = fma2(g, g, fma2(c43, c43, fma2(c42, c42, a41 * a41)));
    const pf2 lam = sym3_max_eig2(s11, s12, s13, s22, s23, s33);
    const float lx = sqrtf(lam.v.x > 0.0f ? lam.v.x : 0.0f), ly = sqrtf(lam.v.y > 0.0f ? lam.v.y : 0.0f);
    return mk(ph.mu / rho.v.x * lx, ph.mu / rho.v.y * ly);
}

// Gbar_e's two terms at one face node (Sec. 2.2): the larger penalty norm of
// the own trace u (1 / rho = ir, pressure pw) and of the other side, which is
// the neighbour's trace w on an interior face, the far-field state, or the
// wall ghost (rho+, v_w, pressure p+).  w is read on interior faces only.
__device__ __forceinline__ float trace_norms_max(const float u[4], float ir, float pw, int bt, const float w[4],
                                                 float n1, float n2, const Phys<float> &ph)
{
    float rb, vb1, vb2, eb;
    if (bt == BCT_INTERIOR) {
        const float iw = 1.0f / w[0];
        rb = w[0]; vb1 = w[1] * iw; vb2 = w[2] * iw; eb = w[3] * iw;
    } else if (bt == BCT_FARFIELD) {
        const float iw = 1.0f / ph.Uinf[0];
        rb = ph.Uinf[0]; vb1 = ph.Uinf[1] * iw; vb2 = ph.Uinf[2] * iw; eb = ph.Uinf[3] * iw;
    } else {
        rb = u[0]; vb1 = ph.vw1; vb2 = ph.vw2;
        eb = (pw / ph.gm1 + 0.5f * u[0] * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2)) * ir;
    }
    const pf2 nab = penalty_norm2(mk(u[0], rb), mk(u[1] * ir, vb1), mk(u[2] * ir, vb2), mk(u[3] * ir, eb), n1, n2, ph);
    return fmaxf(nab.v.x, nab.v.y);
}

}  // namespace dg
