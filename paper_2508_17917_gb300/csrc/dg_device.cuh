// dg_device.cuh -- device-side physics of the nodal IP-DG right-hand side.
//
// Templated on the arithmetic type `real`: double for the plain FP64 path,
// float for the mixed path.  In the mixed path the state stays FP64 in HBM;
// it is converted to FP32 on load, the pressure is recovered in FP64
// (p = (gamma-1)(eps - rho|v|^2/2), Sec. 2.1) and the Runge-Kutta registers
// are updated in FP64 (Algorithm 1).  On GB300 the FP64<->FP32 conversion
// instructions run on the FP64 pipe at the FP64 FMA rate, so the mixed path
// converts with integer operations instead (cvt_d2f / cvt_f2d below).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dg {

// ---------------------------------------------------------------- conversions

// FP64 -> FP32 by integer operations, rounding half away from zero in
// magnitude.  |x| < 2^-126 flushes to zero, overflow gives infinity, NaN stays
// NaN.  Uses no FP64 instruction.
__device__ __forceinline__ float cvt_d2f(double d)
{
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
    unsigned long long mag = b & 0x7fffffffffffffffull;
    bool nan = mag > 0x7ff0000000000000ull;
    mag += 0x10000000ull;                      // round at bit 28 (first dropped bit)
    unsigned hi = static_cast<unsigned>(mag >> 32), lo = static_cast<unsigned>(mag);
    int ef = static_cast<int>(hi >> 20) - 896;   // rebias 1023 -> 127
    unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned out = (static_cast<unsigned>(ef) << 23) | m23;
    out = (ef <= 0) ? 0u : out;
    out = (ef >= 255) ? 0x7f800000u : out;
    out = nan ? 0x7fc00000u : out;
    return __uint_as_float(sign | out);
}

// FP32 -> FP64 by integer operations; exact for normal numbers, subnormals
// flush to zero, infinities and NaN are kept.  Uses no FP64 instruction.
__device__ __forceinline__ double cvt_f2d(float f)
{
    unsigned b = __float_as_uint(f);
    unsigned sign = b & 0x80000000u;
    unsigned e = (b >> 23) & 0xffu;
    unsigned m = b & 0x7fffffu;
    unsigned he = (e == 255u) ? 2047u : e + 896u;
    he = (e == 0u) ? 0u : he;
    m = (e == 0u) ? 0u : m;
    unsigned hi = sign | (he << 20) | (m >> 3);
    unsigned lo = m << 29;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

template <typename real> __device__ __forceinline__ real to_real(double d);
template <> __device__ __forceinline__ double to_real<double>(double d) { return d; }
template <> __device__ __forceinline__ float to_real<float>(double d) { return cvt_d2f(d); }

template <typename real> __device__ __forceinline__ double to_f64(real x);
template <> __device__ __forceinline__ double to_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return cvt_f2d(x); }

// ---------------------------------------------------------------- physics

template <typename real>
struct Phys {
    real gamma, gm1, mu, gPr;      // gamma, gamma-1, viscosity, gamma/Pr
    real vw1, vw2;                 // mesh velocity
    real Uinf[4];                  // far-field state
    real pinf;
    int adiabatic;
};

// Pressure, p = (gamma-1)(eps - rho|v|^2/2).  In the mixed path the
// cancellation runs in FP64 on the FP64 energy `Ed`, as one FMA:
// p = (gamma-1) Ed - (gamma-1) ke with (gamma-1) ke formed in FP32 (the
// kinetic energy is an FP32 value already) and widened exactly; one FP64
// instruction instead of a subtraction and a product, on a pipe that runs at
// about 1/60 of the FP32 rate on GB300 (-1 % per step at p = 3 and 4).
template <typename real>
__device__ __forceinline__ real pressure(const real u[4], double Ed, double gm1d)
{
    real ke = real(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0];
    return to_real<real>(gm1d * (Ed - to_f64<real>(ke)));
}
template <>
__device__ __forceinline__ float pressure<float>(const float u[4], double Ed, double gm1d)
{
    const float gke = cvt_d2f(gm1d) * (0.5f * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    return cvt_d2f(fma(gm1d, Ed, -cvt_f2d(gke)));
}

// Advective flux minus mesh motion, F_c - v_w (x) U, in both directions.
template <typename real>
__device__ __forceinline__ void adv_flux(const real u[4], real p, const Phys<real> &ph,
                                         real Fx[4], real Fy[4])
{
    real ir = real(1) / u[0];
    real v1 = u[1] * ir, v2 = u[2] * ir;
    Fx[0] = u[1] - ph.vw1 * u[0];
    Fx[1] = u[1] * v1 + p - ph.vw1 * u[1];
    Fx[2] = u[2] * v1 - ph.vw1 * u[2];
    Fx[3] = v1 * (p + u[3]) - ph.vw1 * u[3];
    Fy[0] = u[2] - ph.vw2 * u[0];
    Fy[1] = u[1] * v2 - ph.vw2 * u[1];
    Fy[2] = u[2] * v2 + p - ph.vw2 * u[2];
    Fy[3] = v2 * (p + u[3]) - ph.vw2 * u[3];
}

// Viscous flux F_v = G(U) grad U.  The four blocks of G (Sec. 2.1) applied to
// grad U reduce to the Newtonian stress tau = mu (grad v + grad v^T - 2/3 div v I)
// and the heat flux mu gamma/Pr grad(eps/rho - |v|^2/2); this factored form
// is evaluated here with (rho, v, e = eps/rho) taken from (rho, m, e) and the
// gradient from gu.  For the wall flux the caller passes the ghost state's
// velocity and energy with the interior gradient.
template <typename real>
__device__ __forceinline__ void visc_flux_prim(real rho, real v1, real v2, real e,
                                               const real gx[4], const real gy[4],
                                               const Phys<real> &ph, real Fx[4], real Fy[4],
                                               real *qx_out = nullptr, real *qy_out = nullptr)
{
    real ir = real(1) / rho;
    real dv1x = (gx[1] - v1 * gx[0]) * ir, dv1y = (gy[1] - v1 * gy[0]) * ir;
    real dv2x = (gx[2] - v2 * gx[0]) * ir, dv2y = (gy[2] - v2 * gy[0]) * ir;
    real dex = (gx[3] - e * gx[0]) * ir, dey = (gy[3] - e * gy[0]) * ir;
    real mu = ph.mu;
    real txx = mu * (real(4.0 / 3.0) * dv1x - real(2.0 / 3.0) * dv2y);
    real tyy = mu * (real(4.0 / 3.0) * dv2y - real(2.0 / 3.0) * dv1x);
    real txy = mu * (dv1y + dv2x);
    real k = mu * ph.gPr;
    real qx = k * (dex - v1 * dv1x - v2 * dv2x);
    real qy = k * (dey - v1 * dv1y - v2 * dv2y);
    Fx[0] = real(0);
    Fx[1] = txx;
    Fx[2] = txy;
    Fx[3] = v1 * txx + v2 * txy + qx;
    Fy[0] = real(0);
    Fy[1] = txy;
    Fy[2] = tyy;
    Fy[3] = v1 * txy + v2 * tyy + qy;
    if (qx_out) { *qx_out = qx; *qy_out = qy; }
}

template <typename real>
__device__ __forceinline__ void visc_flux(const real u[4], const real gx[4], const real gy[4],
                                          const Phys<real> &ph, real Fx[4], real Fy[4])
{
    real ir = real(1) / u[0];
    visc_flux_prim(u[0], u[1] * ir, u[2] * ir, u[3] * ir, gx, gy, ph, Fx, Fy);
}

// Theta term of the interior-penalty flux (Eq. ip_flux; H_theta of Eq.
// dg_on_K) at one face node: t_l[k] = sum_j n_j (G_jl^T d)_k, l = x, y, for
// the jump d = U+ - U- and G at (rho, v, e).  Because G(U) grad U is linear
// in grad U, t_l[k] is d . (n . F_v) for the gradient that is the unit
// vector e_k along x_l and zero along the other axis.  With a = (d1 + v1 d3,
// d2 + v2 d3) weighting the momentum rows and d3 the energy row, a unit
// gradient of field k gives the velocity gradient w = (dv1, dv2) and energy
// gradient de along x_l:
//   k = 0: w = -(v1, v2)/rho, de = -e/rho;  k = 1: w = (1/rho, 0);
//   k = 2: w = (0, 1/rho);                  k = 3: de = 1/rho,
// and d . (n . F_v) = w1 alpha_1 + w2 alpha_2 + de beta with the
// coefficients below (Newtonian stress with the -2/3 div v term, heat flux
// mu gamma/Pr grad(e - |v|^2/2)).
template <typename real>
__device__ __forceinline__ void theta_vec(real rho, real v1, real v2, real e, const real d[4],
                                          real n1, real n2, const Phys<real> &ph, real tx[4], real ty[4])
{
    const real mu = ph.mu, kq = ph.mu * ph.gPr;
    const real a1 = d[1] + v1 * d[3], a2 = d[2] + v2 * d[3];
    const real sh = mu * (a1 * n2 + a2 * n1);
    const real ax1 = mu * (real(4.0 / 3.0) * a1 * n1 - real(2.0 / 3.0) * a2 * n2) - kq * d[3] * n1 * v1;
    const real ax2 = sh - kq * d[3] * n1 * v2;
    const real bx = kq * d[3] * n1;
    const real ay1 = sh - kq * d[3] * n2 * v1;
    const real ay2 = mu * (real(4.0 / 3.0) * a2 * n2 - real(2.0 / 3.0) * a1 * n1) - kq * d[3] * n2 * v2;
    const real by = kq * d[3] * n2;
    const real ir = real(1) / rho;
    tx[0] = -(v1 * ax1 + v2 * ax2 + e * bx) * ir;
    tx[1] = ax1 * ir;
    tx[2] = ax2 * ir;
    tx[3] = bx * ir;
    ty[0] = -(v1 * ay1 + v2 * ay2 + e * by) * ir;
    ty[1] = ay1 * ir;
    ty[2] = ay2 * ir;
    ty[3] = by * ir;
}

// Largest eigenvalue of a symmetric 3x3 matrix by the trigonometric solution
// of its characteristic cubic.
template <typename real>
__device__ __forceinline__ real sym3_max_eig(real a11, real a12, real a13, real a22, real a23, real a33)
{
    real p1 = a12 * a12 + a13 * a13 + a23 * a23;
    real q = (a11 + a22 + a33) / real(3);
    real b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
    real p2 = b11 * b11 + b22 * b22 + b33 * b33 + real(2) * p1;
    if (!(p2 > real(0))) return q;
    real pp = sqrt(p2 / real(6));
    real ip = real(1) / pp;
    b11 *= ip; b22 *= ip; b33 *= ip;
    real c12 = a12 * ip, c13 = a13 * ip, c23 = a23 * ip;
    real det = b11 * (b22 * b33 - c23 * c23) - c12 * (c12 * b33 - c23 * c13) + c13 * (c12 * c23 - b22 * c13);
    real r = det * real(0.5);
    r = r < real(-1) ? real(-1) : (r > real(1) ? real(1) : r);
    real phi = acos(r) / real(3);
    return q + real(2) * pp * cos(phi);
}

// || n1^2 G11 + n1 n2 (G12 + G21) + n2^2 G22 ||_2 at the state (rho, m, e)
// (Sec. 2.2, definition of Gbar_e).  Rotating the momentum rows and columns
// to the (normal, tangential) frame turns the matrix into G11 evaluated with
// (v.n, v.t); its first row is zero, so the norm is the square root of the
// largest eigenvalue of B B^T with B the remaining 3x4 block.
template <typename real>
__device__ __forceinline__ real penalty_norm(real rho, real v1, real v2, real e, real n1, real n2,
                                             const Phys<real> &ph)
{
    real vn = v1 * n1 + v2 * n2, vt = -v1 * n2 + v2 * n1;
    real vsq = v1 * v1 + v2 * v2, g = ph.gPr;
    real a41 = -vn * vn / real(3) - vsq - g * (e - vsq);
    real c42 = (real(4.0 / 3.0) - g) * vn, c43 = (real(1) - g) * vt;
    real s11 = real(16.0 / 9.0) * (vn * vn + real(1));
    real s12 = real(4.0 / 3.0) * vn * vt;
    real s13 = real(4.0 / 3.0) * (-vn * a41 + c42);
    real s22 = vt * vt + real(1);
    real s23 = -vt * a41 + c43;
    real s33 = a41 * a41 + c42 * c42 + c43 * c43 + g * g;
    real lam = sym3_max_eig(s11, s12, s13, s22, s23, s33);
    return ph.mu / rho * sqrt(lam > real(0) ? lam : real(0));
}

// Normal advective flux n.(F_c - v_w (x) U).
template <typename real>
__device__ __forceinline__ void flux_n(const real u[4], real p, real n1, real n2,
                                       const Phys<real> &ph, real F[4])
{
    real ir = real(1) / u[0];
    real vn = (u[1] * n1 + u[2] * n2) * ir - (ph.vw1 * n1 + ph.vw2 * n2);
    F[0] = u[0] * vn;
    F[1] = u[1] * vn + p * n1;
    F[2] = u[2] * vn + p * n2;
    F[3] = u[3] * vn + p * (u[1] * n1 + u[2] * n2) * ir;
}

// Upwind part of the Roe flux, D = |A~| (U+ - U-), with Roe averages weighted
// by sqrt(rho), eigenvalues (v~ - v_w).n - c~, (v~ - v_w).n (twice),
// (v~ - v_w).n + c~ (Eq. roe_flux) and the wave strengths of U+ - U- along
// the right eigenvectors written with the primitive jumps.
template <typename real>
__device__ __forceinline__ void roe_dissipation(const real up[4], real pp, const real um[4], real pm,
                                                real n1, real n2, const Phys<real> &ph, real D[4])
{
    real rp = up[0], rm = um[0];
    real sp = sqrt(rp), sm = sqrt(rm);
    real irp = real(1) / rp, irm = real(1) / rm;
    real v1p = up[1] * irp, v2p = up[2] * irp, v1m = um[1] * irm, v2m = um[2] * irm;
    real Hp = (up[3] + pp) * irp, Hm = (um[3] + pm) * irm;
    real iw = real(1) / (sp + sm);
    real v1 = (sp * v1p + sm * v1m) * iw, v2 = (sp * v2p + sm * v2m) * iw;
    real H = (sp * Hp + sm * Hm) * iw;
    real q2 = v1 * v1 + v2 * v2;
    real c2 = ph.gm1 * (H - real(0.5) * q2);
    real c = sqrt(c2);
    real un = v1 * n1 + v2 * n2, ut = -v1 * n2 + v2 * n1;
    real vwn = ph.vw1 * n1 + ph.vw2 * n2;
    real rt = sp * sm;
    real dr = rp - rm, dp = pp - pm;
    real dun = (v1p - v1m) * n1 + (v2p - v2m) * n2;
    real dut = -(v1p - v1m) * n2 + (v2p - v2m) * n1;
    real ic2 = real(1) / c2;
    real a1 = real(0.5) * (dp - rt * c * dun) * ic2;
    real a4 = real(0.5) * (dp + rt * c * dun) * ic2;
    real a2 = dr - dp * ic2;
    real a3 = rt * dut;
    real l1 = fabs(un - c - vwn), l2 = fabs(un - vwn), l4 = fabs(un + c - vwn);
    real w1 = l1 * a1, w2 = l2 * a2, w3 = l2 * a3, w4 = l4 * a4;
    D[0] = w1 + w2 + w4;
    D[1] = w1 * (v1 - c * n1) + w2 * v1 - w3 * n2 + w4 * (v1 + c * n1);
    D[2] = w1 * (v2 - c * n2) + w2 * v2 + w3 * n1 + w4 * (v2 + c * n2);
    D[3] = w1 * (H - c * un) + w2 * real(0.5) * q2 + w3 * ut + w4 * (H + c * un);
}

}  // namespace dg
