// aux_kernels.cu -- time step, wall forces and finiteness kernels (FP64).
#include <math.h>

#include "dg_stage.cuh"
#include "launch.h"
#include "rigid.h"

namespace dg {
namespace {

__device__ __forceinline__ void load_node(const double *U, int Np, long long k, int i, double u[4])
{
#pragma unroll
    for (int c = 0; c < 4; ++c) u[c] = U[(k * 4 + c) * Np + i];
}

// One thread per element: Lambda_K of Eq. rayleigh_bound,
//   Lambda_K = 3/2 C_inv,2(K) G_K + (d+1) C_inv,K (3 sigma_K + beta_K) + beta'_K,
// with C_inv,2 = p^4 / rho_K^2 (rho_K the inradius 2|K| / perimeter); G_K the
// largest diffusivity of the system, max(4/3, gamma/Pr) mu / rho, over the
// face-node traces of both sides of the faces of K (the largest eigenvalue of
// N G N^T, which does not depend on the normal); sigma_K the largest penalty
// sigma_e of Eq. penalty_final over the faces of K and C_inv,K the largest
// C_inv; beta_K = max over nodes of |b_ns|_2, (b_ns)_j = |v_j - v_w,j| + c
// (Eq. cfl_general), beta'_K = 0.
__global__ void dt_lambda_kernel(AuxMesh m, Phys<double> ph, double sig_fac, double *lam)
{
    long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (k >= m.K) return;
    if (m.elem_case) {            // batch: the element's case sets mu and v_b
        const BatchCase &cs = m.cases[m.elem_case[k]];
        ph.mu = cs.mu;
        ph.vw2 = cs.vb;
    }
    const int p = m.p, Np = (p + 1) * (p + 2) / 2, Nfp = p + 1;
    const double *g = m.geo + k * 16;
    const int4 cn = m.conn[k];
    double GK = 0, sigK = 0, ciK = 0, perim = 0;
    const double pp = (p + 1.0) * (p + 2.0);
    const double gdiff = fmax(4.0 / 3.0, ph.gPr);
    for (int f = 0; f < 3; ++f) {
        long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
        int f2 = (cn.w >> (2 * f)) & 3;
        int bt = (cn.w >> (8 + 2 * f)) & 3;
        double n1 = g[G_NX + f], n2 = g[G_NY + f], fs = g[G_FS + f];
        double gbar = 0, rmin = INFINITY;
        for (int i = 0; i < Nfp; ++i) {
            int vm = m.fmask[f * Nfp + i];
            double u[4];
            load_node(m.U, Np, k, vm, u);
            double a = penalty_norm(u[0], u[1] / u[0], u[2] / u[0], u[3] / u[0], n1, n2, ph);
            double b;
            rmin = fmin(rmin, u[0]);
            if (bt == BCT_INTERIOR) {
                double w[4];
                load_node(m.U, Np, nb, m.fmask[f2 * Nfp + (Nfp - 1 - i)], w);
                b = penalty_norm(w[0], w[1] / w[0], w[2] / w[0], w[3] / w[0], n1, n2, ph);
                rmin = fmin(rmin, w[0]);
            } else if (bt == BCT_FARFIELD) {
                const double *w = ph.Uinf;
                b = penalty_norm(w[0], w[1] / w[0], w[2] / w[0], w[3] / w[0], n1, n2, ph);
                rmin = fmin(rmin, w[0]);
            } else {   // wall ghost: the interior density
                double pw = pressure<double>(u, u[3], ph.gm1);
                double eb = (pw / ph.gm1 + 0.5 * u[0] * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2)) / u[0];
                b = penalty_norm(u[0], ph.vw1, ph.vw2, eb, n1, n2, ph);
            }
            gbar = fmax(gbar, fmax(a, b));
        }
        double ci = pp * fs * 0.5;
        double cmax = ci;
        if (bt == BCT_INTERIOR) cmax = fmax(ci, pp * m.geo[nb * 16 + G_FS + f2] * 0.5);
        double sig = sig_fac * gbar * cmax;
        GK = fmax(GK, gdiff * ph.mu / rmin);
        sigK = fmax(sigK, sig);
        ciK = fmax(ciK, ci);
        perim += 2.0 * fs * g[G_J];     // |e| = 2 sJ = 2 Fscale J
    }
    double area = 2.0 * g[G_J];
    double rhoK = 2.0 * area / perim;
    double cinv2 = double(p) * p * p * p / (rhoK * rhoK);
    double beta = 0;
    for (int i = 0; i < Np; ++i) {
        double u[4];
        load_node(m.U, Np, k, i, u);
        double pr = pressure<double>(u, u[3], ph.gm1);
        double c = sqrt(ph.gamma * pr / u[0]);
        double b1 = fabs(u[1] / u[0] - ph.vw1) + c, b2 = fabs(u[2] / u[0] - ph.vw2) + c;
        beta = fmax(beta, sqrt(b1 * b1 + b2 * b2));
    }
    lam[k] = 1.5 * cinv2 * GK + 3.0 * ciK * (3.0 * sigK + beta);
}

// Single-block maximum; non-finite entries propagate as NaN.
__global__ void max_reduce_kernel(const double *x, long long n, double *out)
{
    __shared__ double s[1024];
    double m = 0.0;
    bool bad = false;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        double v = x[i];
        if (!isfinite(v)) bad = true;
        m = fmax(m, v);
    }
    s[threadIdx.x] = bad ? NAN : m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double a = s[threadIdx.x], b = s[threadIdx.x + w];
            s[threadIdx.x] = (isnan(a) || isnan(b)) ? NAN : fmax(a, b);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Force and moment of one wall face: traction p n - tau n at its face nodes
// (interior trace, n the element's outward normal), integrated with the LGL
// weights scaled by sJ; moment about (xc, yc).  xy: the face nodes'
// coordinates (x, y interleaved).
__device__ void wall_face_force(const AuxMesh &m, Phys<double> ph, long long k, int f, const double *xy,
                                const double *wface, double xc, double yc, double out[3])
{
    const int p = m.p, Np = (p + 1) * (p + 2) / 2, Nfp = p + 1;
    if (m.elem_case) ph.mu = m.cases[m.elem_case[k]].mu;
    const double *g = m.geo + k * 16;
    const double rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
    const double n1 = g[G_NX + f], n2 = g[G_NY + f], sJ = g[G_FS + f] * g[G_J];
    double F0 = 0, F1 = 0, Mz = 0;
    for (int i = 0; i < Nfp; ++i) {
        int vm = m.fmask[f * Nfp + i];
        double ur[4] = {0, 0, 0, 0}, us[4] = {0, 0, 0, 0}, u[4];
        for (int j = 0; j < Np; ++j) {
            double dr = m.Dr[vm * Np + j], ds = m.Ds[vm * Np + j];
            for (int c = 0; c < 4; ++c) {
                double uj = m.U[(k * 4 + c) * Np + j];
                ur[c] += dr * uj;
                us[c] += ds * uj;
            }
        }
        double gx[4], gy[4];
        for (int c = 0; c < 4; ++c) {
            gx[c] = rx * ur[c] + sx * us[c];
            gy[c] = ry * ur[c] + sy * us[c];
        }
        load_node(m.U, Np, k, vm, u);
        double vx[4], vy[4];
        visc_flux(u, gx, gy, ph, vx, vy);
        double pr = pressure<double>(u, u[3], ph.gm1);
        double tx = pr * n1 - (vx[1] * n1 + vy[1] * n2);
        double ty = pr * n2 - (vx[2] * n1 + vy[2] * n2);
        double x = xy[2 * i] - xc;
        double y = xy[2 * i + 1] - yc;
        double wq = sJ * wface[i];
        F0 += wq * tx;
        F1 += wq * ty;
        Mz += wq * (x * ty - y * tx);
    }
    out[0] = F0;
    out[1] = F1;
    out[2] = Mz;
}

// One thread per wall face of one mesh: partial[w] = (Fx, Fy, Mz) of face w.
__global__ void wall_force_kernel(AuxMesh m, Phys<double> ph, const int2 *faces, const double *face_xy,
                                  const double *wface, int nwall, double xc, double yc, double *partial)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwall) return;
    const int Nfp = m.p + 1;
    wall_face_force(m, ph, faces[w].x, faces[w].y, face_xy + static_cast<long long>(w) * Nfp * 2, wface, xc, yc,
                    partial + w * 3);
}

// One thread per wall face of every degree group of a batch: the groups'
// faces are numbered consecutively (group g from wg.g[g].base), and face w
// writes partial[w].
__global__ void batch_wall_force_kernel(WallGroups wg, Phys<double> ph, double *partial)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= wg.total) return;
    int gi = 0;
    while (gi + 1 < wg.n && w >= wg.g[gi + 1].base) ++gi;
    const WallGroup &G = wg.g[gi];
    const int i = w - G.base, Nfp = G.m.p + 1;
    wall_face_force(G.m, ph, G.faces[i].x, G.faces[i].y, G.face_xy + static_cast<long long>(i) * Nfp * 2,
                    G.wface, 0.0, 0.0, partial + static_cast<long long>(w) * 3);
}

// Deterministic single-block sum of n triples.
__global__ void sum3_kernel(const double *partial, int n, double *out)
{
    __shared__ double s[3][256];
    double a[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int c = 0; c < 3; ++c) a[c] += partial[i * 3 + c];
    for (int c = 0; c < 3; ++c) s[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) out[c] = s[c][0];
}

__global__ void nonfinite_kernel(const double *x, long long n, int *flag)
{
    long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

// ---- batch of independent cases (Algorithm 3 per case, on the device)

// One block per case: max_K Lambda_K over the case's elements, then
// dt = cfl / max (Eq. rayleigh_bound), or the case's entry of `fixed` when
// the caller fixed the steps (the bound is still evaluated and recorded); a
// bound that is not finite freezes the case (dt = 0, bad = 1) instead of
// spreading NaN.  Thread 0 then takes the case's Newmark step with the lift
// of the previous force evaluation (Algorithm 3: F_r = lift / m), giving v_b
// for the coming RK step.
__global__ void batch_dt_newmark_kernel(const double *lam, const long long *seg, BatchCase *cases, double cfl,
                                        const double *fixed)
{
    __shared__ double s[256];
    const int i = blockIdx.x;
    const long long b = seg[2 * i], e = seg[2 * i + 1];
    double m = 0.0;
    bool bad = false;
    for (long long k = b + threadIdx.x; k < e; k += blockDim.x) {
        const double v = lam[k];
        bad |= !isfinite(v);
        m = fmax(m, v);
    }
    s[threadIdx.x] = bad ? NAN : m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double x = s[threadIdx.x], y = s[threadIdx.x + w];
            s[threadIdx.x] = (isnan(x) || isnan(y)) ? NAN : fmax(x, y);
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    BatchCase &cs = cases[i];
    const double l = s[0];
    cs.lam = l;
    if (cs.bad || !isfinite(l) || !(l > 0.0)) {
        cs.bad = 1;
        cs.dt = 0.0;
        cs.vb = 0.0;
        return;
    }
    cs.dt = fixed ? fixed[i] : cfl / l;
    double y = cs.y, yd = cs.yd, ydd = cs.ydd, vb = 0.0;
    if (newmark_step(cs.Mr, cs.Cr, cs.Kr, cs.Fy / cs.mass, cs.dt, y, yd, ydd, vb)) {
        cs.y = y;
        cs.yd = yd;
        cs.ydd = ydd;
        cs.vb = vb;
        cs.t += cs.dt;
    } else {
        cs.bad = 1;
        cs.vb = 0.0;
    }
}

// One block per case: deterministic tree sum of its wall-face partials into
// the case's (Fx, Fy, Mz); with a history, row *counter of hist gets
// (t, dt, y, y', v_b, Fx, Fy, lam) of the case (rows beyond cap are dropped).
// The last block to finish (ticket) advances the row counter once every
// block has read it.
__global__ void batch_forces_record_kernel(const double *partial, const int *wseg, BatchCase *cases,
                                           double *hist, int cap, int *counter, unsigned *ticket)
{
    __shared__ double s[3][256];
    const int i = blockIdx.x, n = gridDim.x;
    const int b = wseg[2 * i], e = wseg[2 * i + 1];
    double a[3] = {0, 0, 0};
    for (int w = b + threadIdx.x; w < e; w += blockDim.x)
        for (int c = 0; c < 3; ++c) a[c] += partial[static_cast<long long>(w) * 3 + c];
    for (int c = 0; c < 3; ++c) s[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    BatchCase &cs = cases[i];
    cs.Fx = s[0][0];
    cs.Fy = s[1][0];
    cs.Mz = s[2][0];
    if (!hist) return;
    const int row = *counter;
    if (row < cap) {
        double *h = hist + (static_cast<long long>(row) * n + i) * 8;
        h[0] = cs.t; h[1] = cs.dt; h[2] = cs.y; h[3] = cs.yd;
        h[4] = cs.vb; h[5] = cs.Fx; h[6] = cs.Fy; h[7] = cs.lam;
    }
    __threadfence();
    if (atomicAdd(ticket, 1u) == static_cast<unsigned>(n - 1)) {
        *ticket = 0u;
        *counter = row + 1;
    }
}

// Viscous source of the advected isentropic vortex, S = -div F_v(U_v), in
// closed form.  With (dx, dy) the offset of the node from the nearest
// periodic image of the centre (x0 + u0 t, y0 + v0 t), r^2 = dx^2 + dy^2,
// f = beta / (2 pi) exp((1 - r^2) / 2) and (du, dv) = f (-dy, dx) the
// velocity perturbation: the perturbation is divergence free and its
// Laplacian is -(4 - r^2)(du, dv), the stress work tau : grad v is
// mu f^2 r^4 and the Laplacian of T = 1 - a exp(1 - r^2) is
// 4 a exp(1 - r^2)(1 - r^2), so
//   S_rho = 0,   S_m = mu (4 - r^2) (du, dv),
//   S_E = mu (4 - r^2)(u0 du + v0 dv)
//         + mu beta^2 / (2 pi^2) exp(1 - r^2) (r^2 (2 - r^2) - (1 - r^2) / Pr).
// One thread per node; (xc, yc) is the centre at the stage's time (host,
// FP64); `real` is the arithmetic after the FP64 offsets (FP64 path: double;
// mixed: float).  The constants come precomputed (VortexSource).
template <typename real>
__device__ __forceinline__ void vortex_source_node(const double *xy, long long nn, long long n, int Np,
                                                   const VortexSource &v, double xc, double yc, double *S)
{
    real dx = real(xy[n] - xc), dy = real(xy[nn + n] - yc);
    dx -= real(v.L) * rint(dx * real(v.invL));
    dy -= real(v.L) * rint(dy * real(v.invL));
    const real r2 = dx * dx + dy * dy;
    const real e1 = exp(real(1) - r2);
    const real f = real(v.f0) * sqrt(e1);
    const real du = -f * dy, dv = f * dx;
    const real mu = real(v.mu), w = mu * (real(4) - r2);
    const real sE = w * (real(v.u0) * du + real(v.v0) * dv) +
                    mu * real(v.c2) * e1 * (r2 * (real(2) - r2) - (real(1) - r2) * real(v.invPr));
    const long long k = n / Np;
    const int i = static_cast<int>(n - k * Np);
    double *o = S + k * 4 * Np + i;
    o[0] = 0.0;
    o[Np] = static_cast<double>(w * du);
    o[2 * Np] = static_cast<double>(w * dv);
    o[3 * Np] = static_cast<double>(sE);
}

// ns source arrays (one per stage time, centres (xc[s], yc[s]) given) in one
// launch: S + s * 4 nn holds the source at stage time s.
template <typename real>
__global__ void vortex_source_kernel(const double *xy, long long nn, int Np, VortexSource v, VortexCentres cen,
                                     double *S)
{
    const long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (n >= nn) return;
    for (int s = 0; s < cen.ns; ++s)
        vortex_source_node<real>(xy, nn, n, Np, v, cen.xc[s], cen.yc[s], S + s * 4 * nn);
}

}  // namespace

cudaError_t launch_vortex_source(bool fp64, const double *xy, long long nn, int Np, const VortexSource &v,
                                 const double *t, int ns, double *S, cudaStream_t st)
{
    if (ns < 1 || ns > 5) return cudaErrorInvalidValue;
    const unsigned blocks = static_cast<unsigned>((nn + 255) / 256);
    VortexCentres cen{};
    cen.ns = ns;
    for (int s = 0; s < ns; ++s) {
        cen.xc[s] = v.x0 + v.u0 * t[s];
        cen.yc[s] = v.y0 + v.v0 * t[s];
    }
    if (fp64)
        vortex_source_kernel<double><<<blocks, 256, 0, st>>>(xy, nn, Np, v, cen, S);
    else
        vortex_source_kernel<float><<<blocks, 256, 0, st>>>(xy, nn, Np, v, cen, S);
    return cudaGetLastError();
}

cudaError_t launch_batch_dt_newmark(const double *lam, const long long *seg, BatchCase *cases, int ncases,
                                    double cfl, const double *fixed, cudaStream_t st)
{
    batch_dt_newmark_kernel<<<ncases, 256, 0, st>>>(lam, seg, cases, cfl, fixed);
    return cudaGetLastError();
}

cudaError_t launch_batch_wall_forces(const WallGroups &wg, const Phys<double> &ph, double *partial,
                                     cudaStream_t st)
{
    if (wg.total < 1) return cudaSuccess;
    batch_wall_force_kernel<<<(wg.total + 127) / 128, 128, 0, st>>>(wg, ph, partial);
    return cudaGetLastError();
}

cudaError_t launch_batch_forces_record(const double *partial, const int *wseg, BatchCase *cases, int ncases,
                                       double *hist, int cap, int *counter, unsigned *ticket, cudaStream_t st)
{
    batch_forces_record_kernel<<<ncases, 256, 0, st>>>(partial, wseg, cases, hist, cap, counter, ticket);
    return cudaGetLastError();
}

cudaError_t launch_dt_lambda(const AuxMesh &m, const Phys<double> &ph, double sig_fac, double *lam,
                             cudaStream_t st)
{
    int threads = 128;
    long long blocks = (m.K + threads - 1) / threads;
    dt_lambda_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(m, ph, sig_fac, lam);
    return cudaGetLastError();
}

cudaError_t launch_max_reduce(const double *lam, long long K, double *out, cudaStream_t st)
{
    max_reduce_kernel<<<1, 1024, 0, st>>>(lam, K, out);
    return cudaGetLastError();
}

cudaError_t launch_wall_force_faces(const AuxMesh &m, const Phys<double> &ph, const int2 *faces,
                                    const double *face_xy, const double *wface, int nwall,
                                    double xc, double yc, double *partial, cudaStream_t st)
{
    int threads = 128;
    int blocks = (nwall + threads - 1) / threads;
    wall_force_kernel<<<blocks, threads, 0, st>>>(m, ph, faces, face_xy, wface, nwall, xc, yc, partial);
    return cudaGetLastError();
}

cudaError_t launch_sum3(const double *partial, int n, double *out, cudaStream_t st)
{
    sum3_kernel<<<1, 256, 0, st>>>(partial, n, out);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite(const double *x, long long n, int *flag, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (n + 255) / 256;
    long long blocks = want < 4LL * sms ? want : 4LL * sms;
    if (blocks < 1) blocks = 1;
    nonfinite_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(x, n, flag);
    return cudaGetLastError();
}

}  // namespace dg
