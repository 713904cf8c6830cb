// dg_stage.cuh -- fused right-hand side + low-storage RK stage kernel.
//
// One launch evaluates, for every element, the nodal residual of Eq. dg_on_K
// in strong form
//     dU/dt = -(rx Dr + sx Ds) F_x - (ry Dr + sy Ds) F_y + LIFT (Fscale (F.n - H))
// with F = F_c - v_w (x) U - G(U) grad_h U (Sec. 2.1), H the Roe + interior-
// penalty face flux with the penalty of Eq. penalty_final, and then applies
// one stage of Algorithm 1:  K1 <- A K1 + dt R;  K0_out <- K0_in + B K1.
// For theta != 0 (SIP, NIPG) the terms -S_x H_theta,x - S_y H_theta,y of
// Eq. dg_on_K add
//     Wr (rx Lx + ry Ly) + Ws (sx Lx + sy Ly),  L_l = LIFT (Fscale theta w t_l),
// with Wr = M^-1 Dr^T M, Ws = M^-1 Ds^T M, t_l the theta vector of each face
// node (theta_vec) and w = 1/2 on interior faces (the average), 1 on boundary
// faces; G is taken at U+ on interior and far-field faces, at U^b on walls.
// (The strong form equals the paper's weak form exactly for collocated
// fluxes on affine elements: the weak volume term integrated by parts gives
// the strong divergence plus the lifted interior trace F.n.)
//
// Work decomposition: a CTA of NT threads owns a tile of E elements at a
// time (persistent loop over tiles).  Thread t is volume node (t / Np, t % Np)
// and face node (t / 3Nfp, t % 3Nfp) of the tile.  The neighbour's broken
// gradient at a shared face node is recomputed from the neighbour's state,
// staged in shared memory, so one pass over the state serves the volume and
// the face terms (the paper's halo exchange of {U, grad U} traces becomes a
// read of the neighbour's state from L2).  K0 is read from one buffer and
// written to another so that neighbours always see the stage's input state.
#pragma once
#include "dg_device.cuh"

namespace dg {

enum { STAGE_UPDATE = 0, STAGE_RHS_ONLY = 1 };
enum { BCT_INTERIOR = 0, BCT_WALL = 1, BCT_FARFIELD = 2 };

// Per-case quantities of a batch of independent cases (Algorithm 3 state kept
// on the device): time step and time, rigid-body state with its mesh
// velocity v_b, oscillator coefficients, latest wall forces, viscosity.
struct BatchCase {
    double dt, t;
    double y, yd, ydd, vb;        // transverse displacement, velocity, acceleration; v_b
    double Mr, Cr, Kr, mass;      // M_r y'' + C_r y' + K_r y = F_r with F_r = lift / mass
    double Fx, Fy, Mz;            // drag, lift, moment of the last force evaluation
    double mu;                    // viscosity of the case
    double lam;                   // max_K Lambda_K of the last time-step bound
    int bad;                      // set once the bound was not finite (the case is frozen)
    int pad;
};

// Time-step bound of a batch: one degree group's inputs (FP32 state copy,
// pressures, geometry, connectivity, face table, tile table) and where its
// Lambda_K go; first_block is the group's first block of the launch.
struct DtGroup {
    const float4 *S;
    const float *Pr;
    const float *geo;
    const int4 *conn;
    const int *fmask;
    const int4 *tiles;
    long long K, ntiles, first_block;
    double *lam;
    int p;
};
struct DtGroups {
    DtGroup g[8];
    int n;
    long long blocks;
};

struct StageParams {
    const double *K0in;
    double *K0out;
    double *K1;
    double *Rout;              // STAGE_RHS_ONLY output
    const void *geo;           // real[16] per element
    const int4 *conn;          // (nbr0, nbr1, nbr2, packed faces/bc)
    const void *ops;           // real Dr, Ds [Np*Np], LIFT [Np*3Nfp], Wr, Ws [Np*Np]
    const int *fmask;          // 3*Nfp, counter-clockwise along each face
    const double *src;         // optional nodal source [K][4][Np] or null
    const float4 *Sin;         // mixed path: FP32 copy of K0in, [K][Np] (rho, m1, m2, E)
    const float *Pin;          // mixed path: pressure of K0in, [K][NpP]
    float4 *Sout;              // mixed path: FP32 copy of K0out
    float *Pout;               // mixed path: pressure of K0out
    long long K;
    double A, B, dt;
    double gm1;                // gamma - 1 in FP64 for the pressure
    double sig_fac;            // C1 (1+theta)^2 (d+1) of Eq. penalty_final
    double theta;              // IP variant (Eq. ip_flux): 1 SIP, 0 IIP, -1 NIPG
    double uinf[4];            // far-field conserved state in FP64 (mixed theta variant)
    int mode;
    int first_stage;           // A == 0: K1 is not read
    // batch variant: tile table (first element, element count, case, 0), the
    // per-case quantities (dt, v_b, mu are read per tile) and the tile count
    const int4 *tiles;
    const BatchCase *cases;
    long long ntiles;
    // fused variant: the five stages of one step (Algorithm 1) in one
    // cooperative launch, a grid barrier between stages; the K0 / FP32-copy /
    // pressure buffers swap roles after every stage
    double A5[5], B5[5];
    unsigned *bar;             // [0] arrivals, [1] generation
    int *bar_err;              // set to 1 when a barrier wait gave up
    unsigned bar_limit;        // waits of about 100 ns before giving up
};

template <int P>
struct Shape {
    static constexpr int Np = (P + 1) * (P + 2) / 2;
    static constexpr int Nfp = P + 1;
    static constexpr int NF = 3 * Nfp;
    static constexpr int NT = 256;
    static constexpr int W = Np > NF ? Np : NF;
    static constexpr int E = NT / W;
};

// geometry record (real[16]) per element
enum { G_RX = 0, G_RY = 1, G_SX = 2, G_SY = 3, G_J = 4, G_NX = 5, G_NY = 8, G_FS = 11 };

// Over-integration rule of degree p: collapsed Gauss rule of degree
// min(3p, 15), N = deg / 2 + 1 points per direction, Nq = N^2 <= 64.
template <int P>
struct OIShape {
    static constexpr int deg = (3 * P < 15) ? 3 * P : 15;
    static constexpr int N = deg / 2 + 1;
    static constexpr int Nq = N * N;
};

template <int P, typename real, bool TH = false, bool OI = false>
struct Smem {
    using S = Shape<P>;
    static constexpr int Np = S::Np, NF = S::NF, E = S::E;
    static constexpr int Nq = OI ? OIShape<P>::Nq : 0;
    // sizes in elements of `real`
    static constexpr int ops = 2 * Np * Np + Np * NF + (TH ? 2 * Np * Np : 0);
    static constexpr int oiops = 5 * Nq * Np;           // Vq, Vqr, Vqs [Nq][Np]; Sr, Ss [Np][Nq]
    static constexpr int fq = 2 * E * 4 * Nq;           // contravariant fluxes at the cubature points
    static constexpr int u = E * 4 * Np;
    static constexpr int gx = E * 4 * Np;
    static constexpr int gy = E * 4 * Np;
    static constexpr int fr = E * 4 * Np;
    static constexpr int fs = E * 4 * Np;
    static constexpr int pr = E * Np;
    static constexpr int nb = E * 3 * 4 * Np;
    static constexpr int norm = E * NF;
    static constexpr int dh = E * NF * 4;
    static constexpr int geo = E * 16;
    static constexpr int ngeo = E * 3 * 8;
    static constexpr int th = TH ? E * NF * 8 : 0;
    static constexpr int total_real = ops + u + gx + gy + fr + fs + pr + nb + norm + dh + geo + ngeo + th + oiops + fq;
    static constexpr size_t bytes = total_real * sizeof(real) + NF * sizeof(int) + 16;
};

template <int P, typename real, bool TH, bool OI = false>
__global__ void __launch_bounds__(Shape<P>::NT)
stage_kernel(StageParams sp, Phys<real> ph)
{
    using S = Shape<P>;
    constexpr int Np = S::Np, Nfp = S::Nfp, NF = S::NF, E = S::E, NT = S::NT;
    using L = Smem<P, real, TH, OI>;
    constexpr int Nq = L::Nq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sDr = reinterpret_cast<real *>(smem_raw);
    real *sDs = sDr + Np * Np;
    real *sLIFT = sDs + Np * Np;
    real *sWr = sLIFT + Np * NF;               // theta variant only
    real *sWs = sWr + Np * Np;
    real *sU = sDr + L::ops;
    real *sGx = sU + L::u;
    real *sGy = sGx + L::gx;
    real *sFr = sGy + L::gy;
    real *sFs = sFr + L::fr;
    real *sP = sFs + L::fs;
    real *sN = sP + L::pr;
    real *sNorm = sN + L::nb;
    real *sDH = sNorm + L::norm;
    real *sGeo = sDH + L::dh;
    real *sNGeo = sGeo + L::geo;
    real *sTH = sNGeo + L::ngeo;               // theta variant: Fscale theta w (t_x, t_y)
    real *sVq = sTH + L::th;                   // over-integration: Vq | Vqr | Vqs | Sr | Ss
    real *sVqr = sVq + Nq * Np;
    real *sVqs = sVqr + Nq * Np;
    real *sSr = sVqs + Nq * Np;
    real *sSs = sSr + Np * Nq;
    real *sFq = sVq + L::oiops;                // [E][4][Nq] x (r, s)
    int *sFm = reinterpret_cast<int *>(sFq + L::fq);

    const int tid = threadIdx.x;
    {
        const real *ops = static_cast<const real *>(sp.ops);
        for (int i = tid; i < L::ops; i += NT) sDr[i] = ops[i];
        for (int i = tid; i < NF; i += NT) sFm[i] = sp.fmask[i];
        if constexpr (OI) {
            // the operator buffer holds Dr | Ds | LIFT | Wr | Ws | Vq | Vqr | Vqs | Sr | Ss
            const real *oi = ops + 4 * Np * Np + Np * NF;
            for (int i = tid; i < L::oiops; i += NT) sVq[i] = oi[i];
        }
    }
    const real *geo = static_cast<const real *>(sp.geo);
    const long long K = sp.K;
    const long long ntiles = (K + E - 1) / E;
    const double gm1d = sp.gm1;
    const real p1 = real(P + 1), p2 = real(P + 2);
    const real sig_fac = static_cast<real>(sp.sig_fac);
    const real theta = static_cast<real>(sp.theta);

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long k0 = tile * E;
        const int ne = static_cast<int>((K - k0) < E ? (K - k0) : E);
        __syncthreads();   // operators loaded / previous tile's face reads done

        // ---- P1: stage the tile's state, geometry and neighbour states
        const double *K0 = sp.K0in;
        for (int idx = tid; idx < ne * 4 * Np; idx += NT)
            sU[idx] = to_real<real>(K0[k0 * 4 * Np + idx]);
        for (int idx = tid; idx < ne * 16; idx += NT)
            sGeo[idx] = geo[k0 * 16 + idx];
        for (int idx = tid; idx < ne * 3 * 4 * Np; idx += NT) {
            int e = idx / (3 * 4 * Np), rem = idx - e * (3 * 4 * Np);
            int f = rem / (4 * Np), j = rem - f * (4 * Np);
            int4 cn = sp.conn[k0 + e];
            long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            sN[idx] = to_real<real>(K0[nb * 4 * Np + j]);
        }
        for (int idx = tid; idx < ne * 3; idx += NT) {
            int e = idx / 3, f = idx - 3 * e;
            int4 cn = sp.conn[k0 + e];
            long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            int f2 = (cn.w >> (2 * f)) & 3;
            const real *g = geo + nb * 16;
            real *d = sNGeo + idx * 8;
            d[0] = g[G_RX]; d[1] = g[G_RY]; d[2] = g[G_SX]; d[3] = g[G_SY];
            d[4] = g[G_FS + f2];
        }
        __syncthreads();

        // ---- P2: volume gradient, volume flux; face-node penalty norms
        const int ve = tid / Np, vi = tid - (tid / Np) * Np;
        const bool vol = ve < ne;
        if (vol) {
            const real *u_e = sU + ve * 4 * Np;
            real ur[4] = {0, 0, 0, 0}, us[4] = {0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                real dr = sDr[vi * Np + j], ds = sDs[vi * Np + j];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    real uj = u_e[c * Np + j];
                    ur[c] += dr * uj;
                    us[c] += ds * uj;
                }
            }
            const real *g = sGeo + ve * 16;
            real rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
            real u[4], gxv[4], gyv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                u[c] = u_e[c * Np + vi];
                gxv[c] = rx * ur[c] + sx * us[c];
                gyv[c] = ry * ur[c] + sy * us[c];
                sGx[(ve * 4 + c) * Np + vi] = gxv[c];
                sGy[(ve * 4 + c) * Np + vi] = gyv[c];
            }
            double Ed = sp.K0in[((k0 + ve) * 4 + 3) * Np + vi];
            real p = pressure<real>(u, Ed, gm1d);
            sP[ve * Np + vi] = p;
            real cx[4], cy[4], vx[4], vy[4];
            adv_flux(u, p, ph, cx, cy);
            visc_flux(u, gxv, gyv, ph, vx, vy);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                real Fx = cx[c] - vx[c], Fy = cy[c] - vy[c];
                sFr[(ve * 4 + c) * Np + vi] = rx * Fx + ry * Fy;
                sFs[(ve * 4 + c) * Np + vi] = sx * Fx + sy * Fy;
            }
        }
        if constexpr (OI) {
            // flux at the cubature points from the state and broken gradient
            // interpolated there (the polynomial U_h itself, not nodal values)
            if (vol) {
                const real *u_e = sU + ve * 4 * Np;
                const real *g = sGeo + ve * 16;
                const real rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
                for (int q = vi; q < Nq; q += Np) {
                    real u[4] = {0, 0, 0, 0}, ur[4] = {0, 0, 0, 0}, us[4] = {0, 0, 0, 0};
                    for (int j = 0; j < Np; ++j) {
                        const real a = sVq[q * Np + j], b = sVqr[q * Np + j], d = sVqs[q * Np + j];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const real uj = u_e[c * Np + j];
                            u[c] += a * uj;
                            ur[c] += b * uj;
                            us[c] += d * uj;
                        }
                    }
                    real gxq[4], gyq[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        gxq[c] = rx * ur[c] + sx * us[c];
                        gyq[c] = ry * ur[c] + sy * us[c];
                    }
                    const real pq = pressure<real>(u, to_f64<real>(u[3]), gm1d);
                    real cx[4], cy[4], vx[4], vy[4];
                    adv_flux(u, pq, ph, cx, cy);
                    visc_flux(u, gxq, gyq, ph, vx, vy);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const real Fx = cx[c] - vx[c], Fy = cy[c] - vy[c];
                        sFq[((ve * 4 + c) * Nq + q) * 2] = rx * Fx + ry * Fy;
                        sFq[((ve * 4 + c) * Nq + q) * 2 + 1] = sx * Fx + sy * Fy;
                    }
                }
            }
        }
        const int fe = tid / NF, fm = tid - (tid / NF) * NF;
        const bool face = fe < ne;
        const int ff = fm / Nfp, fi = fm - (fm / Nfp) * Nfp;
        int btype = 0, f2 = 0, vm = 0, vp = 0;
        long long nbk = 0;
        if (face) {
            int4 cn = sp.conn[k0 + fe];
            nbk = (ff == 0) ? cn.x : (ff == 1 ? cn.y : cn.z);
            f2 = (cn.w >> (2 * ff)) & 3;
            btype = (cn.w >> (8 + 2 * ff)) & 3;
            vm = sFm[ff * Nfp + fi];
            vp = sFm[f2 * Nfp + (Nfp - 1 - fi)];
            const real *g = sGeo + fe * 16;
            real n1 = g[G_NX + ff], n2 = g[G_NY + ff];
            real u[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) u[c] = sU[(fe * 4 + c) * Np + vm];
            real ir = real(1) / u[0];
            real a = penalty_norm(u[0], u[1] * ir, u[2] * ir, u[3] * ir, n1, n2, ph);
            real b;
            if (btype == BCT_INTERIOR) {
                real w[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) w[c] = sN[((fe * 3 + ff) * 4 + c) * Np + vp];
                real iw = real(1) / w[0];
                b = penalty_norm(w[0], w[1] * iw, w[2] * iw, w[3] * iw, n1, n2, ph);
            } else if (btype == BCT_FARFIELD) {
                real iw = real(1) / ph.Uinf[0];
                b = penalty_norm(ph.Uinf[0], ph.Uinf[1] * iw, ph.Uinf[2] * iw, ph.Uinf[3] * iw, n1, n2, ph);
            } else {
                double Ed = sp.K0in[((k0 + fe) * 4 + 3) * Np + vm];
                real pw = pressure<real>(u, Ed, gm1d);
                real eb = (pw / ph.gm1 + real(0.5) * u[0] * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2)) * ir;
                b = penalty_norm(u[0], ph.vw1, ph.vw2, eb, n1, n2, ph);
            }
            sNorm[fe * NF + fm] = a > b ? a : b;
        }
        __syncthreads();

        // ---- P3: divergence (volume) and face flux (face nodes)
        real R[4] = {0, 0, 0, 0};
        if (vol && !OI) {
            const real *fr = sFr + ve * 4 * Np;
            const real *fs = sFs + ve * 4 * Np;
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                real dr = sDr[vi * Np + j], ds = sDs[vi * Np + j];
#pragma unroll
                for (int c = 0; c < 4; ++c) R[c] -= dr * fr[c * Np + j] + ds * fs[c * Np + j];
            }
        }
        if constexpr (OI) {
            // weak volume term: sum_q Sr_iq Fr_q + Ss_iq Fs_q (Sr = M^-1 Vqr^T W)
            if (vol) {
                const real *fq = sFq + ve * 4 * Nq * 2;
                for (int q = 0; q < Nq; ++q) {
                    const real a = sSr[vi * Nq + q], b = sSs[vi * Nq + q];
#pragma unroll
                    for (int c = 0; c < 4; ++c) R[c] += a * fq[(c * Nq + q) * 2] + b * fq[(c * Nq + q) * 2 + 1];
                }
            }
        }
        if (face) {
            const real *g = sGeo + fe * 16;
            real n1 = g[G_NX + ff], n2 = g[G_NY + ff], fsc = g[G_FS + ff];
            real gbar = real(0);
#pragma unroll
            for (int l = 0; l < Nfp; ++l) {
                real v = sNorm[fe * NF + ff * Nfp + l];
                gbar = v > gbar ? v : gbar;
            }
            real cinv = p1 * p2 * fsc * real(0.5);
            if (btype == BCT_INTERIOR) {
                real c2 = p1 * p2 * sNGeo[(fe * 3 + ff) * 8 + 4] * real(0.5);
                cinv = c2 > cinv ? c2 : cinv;
            }
            real sigma = sig_fac * gbar * cinv;
            real up[4], gxp[4], gyp[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                up[c] = sU[(fe * 4 + c) * Np + vm];
                gxp[c] = sGx[(fe * 4 + c) * Np + vm];
                gyp[c] = sGy[(fe * 4 + c) * Np + vm];
            }
            real pp = sP[fe * Np + vm];
            real Fnp[4], vxp[4], vyp[4];
            flux_n(up, pp, n1, n2, ph, Fnp);
            visc_flux(up, gxp, gyp, ph, vxp, vyp);
            real dH[4];
            // theta term inputs: jump U+ - U-, the state G is taken at, weight
            real jmp[4], gs[4], wth = real(1);
            {
                const real ir = real(1) / up[0];
                gs[0] = up[0]; gs[1] = up[1] * ir; gs[2] = up[2] * ir; gs[3] = up[3] * ir;
            }
            if (btype == BCT_INTERIOR) {
                const real *w = sN + (fe * 3 + ff) * 4 * Np;
                const real *ng = sNGeo + (fe * 3 + ff) * 8;
                real um[4], wr[4] = {0, 0, 0, 0}, ws[4] = {0, 0, 0, 0};
#pragma unroll
                for (int j = 0; j < Np; ++j) {
                    real dr = sDr[vp * Np + j], ds = sDs[vp * Np + j];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        real wj = w[c * Np + j];
                        wr[c] += dr * wj;
                        ws[c] += ds * wj;
                    }
                }
                real gxm[4], gym[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    um[c] = w[c * Np + vp];
                    gxm[c] = ng[0] * wr[c] + ng[2] * ws[c];
                    gym[c] = ng[1] * wr[c] + ng[3] * ws[c];
                }
                double Edm = sp.K0in[(nbk * 4 + 3) * Np + vp];
                real pm = pressure<real>(um, Edm, gm1d);
                real Fnm[4], vxm[4], vym[4], D[4];
                flux_n(um, pm, n1, n2, ph, Fnm);
                visc_flux(um, gxm, gym, ph, vxm, vym);
                roe_dissipation(up, pp, um, pm, n1, n2, ph, D);
                wth = real(0.5);
#pragma unroll
                for (int c = 0; c < 4; ++c) jmp[c] = up[c] - um[c];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    real vnp = vxp[c] * n1 + vyp[c] * n2, vnm = vxm[c] * n1 + vym[c] * n2;
                    dH[c] = real(0.5) * (Fnp[c] - Fnm[c]) - real(0.5) * D[c]
                          - real(0.5) * (vnp - vnm) - sigma * (up[c] - um[c]);
                }
            } else if (btype == BCT_FARFIELD) {
                real ub[4] = {ph.Uinf[0], ph.Uinf[1], ph.Uinf[2], ph.Uinf[3]};
                real Fnb[4], D[4];
                flux_n(ub, ph.pinf, n1, n2, ph, Fnb);
                roe_dissipation(up, pp, ub, ph.pinf, n1, n2, ph, D);
                // H = Roe - G(U+) grad U+ . n + sigma (U+ - Ub); F+.n - H:
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    dH[c] = real(0.5) * (Fnp[c] - Fnb[c]) - real(0.5) * D[c] - sigma * (up[c] - ub[c]);
                    jmp[c] = up[c] - ub[c];
                }
            } else {
                // wall: U^b from Q^b = (rho+, v_w, p+); H = n.(F_c - v_w U)(U^b)
                //       - G(U^b) grad U+ . n + sigma (U+ - U^b)
                real rb = up[0];
                real kw = real(0.5) * rb * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2);
                real ub[4] = {rb, rb * ph.vw1, rb * ph.vw2, pp / ph.gm1 + kw};
                real Fnb[4], vxb[4], vyb[4], qx, qy;
                flux_n(ub, pp, n1, n2, ph, Fnb);
                visc_flux_prim(rb, ph.vw1, ph.vw2, ub[3] / rb, gxp, gyp, ph, vxb, vyb, &qx, &qy);
                real vnb[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) vnb[c] = vxb[c] * n1 + vyb[c] * n2;
                if (ph.adiabatic) vnb[3] -= qx * n1 + qy * n2;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    real vnp = vxp[c] * n1 + vyp[c] * n2;
                    dH[c] = (Fnp[c] - vnp) - (Fnb[c] - vnb[c] + sigma * (up[c] - ub[c]));
                    jmp[c] = up[c] - ub[c];
                }
                gs[0] = rb; gs[1] = ph.vw1; gs[2] = ph.vw2; gs[3] = ub[3] / rb;
            }
            if constexpr (OI) {
                // weak form: the face term is -H itself, without the F+.n of the strong form
#pragma unroll
                for (int c = 0; c < 4; ++c) dH[c] -= Fnp[c] - (vxp[c] * n1 + vyp[c] * n2);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) sDH[(fe * NF + fm) * 4 + c] = fsc * dH[c];
            if constexpr (TH) {
                real tx[4], ty[4];
                theta_vec(gs[0], gs[1], gs[2], gs[3], jmp, n1, n2, ph, tx, ty);
                const real sc = theta * wth * fsc;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    sTH[(fe * NF + fm) * 8 + c] = sc * tx[c];
                    sTH[(fe * NF + fm) * 8 + 4 + c] = sc * ty[c];
                }
            }
        }
        __syncthreads();

        // ---- P4: lift, then the stage update (or the residual itself)
        if (vol) {
            const real *dh = sDH + ve * NF * 4;
#pragma unroll
            for (int m = 0; m < NF; ++m) {
                real l = sLIFT[vi * NF + m];
#pragma unroll
                for (int c = 0; c < 4; ++c) R[c] += l * dh[m * 4 + c];
            }
        }
        if constexpr (TH) {
            // lift the theta vectors, map to (r, s) and park them in the flux slots
            if (vol) {
                const real *th = sTH + ve * NF * 8;
                real Lx[4] = {0, 0, 0, 0}, Ly[4] = {0, 0, 0, 0};
#pragma unroll
                for (int m = 0; m < NF; ++m) {
                    const real l = sLIFT[vi * NF + m];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        Lx[c] += l * th[m * 8 + c];
                        Ly[c] += l * th[m * 8 + 4 + c];
                    }
                }
                const real *g = sGeo + ve * 16;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    sFr[(ve * 4 + c) * Np + vi] = g[G_RX] * Lx[c] + g[G_RY] * Ly[c];
                    sFs[(ve * 4 + c) * Np + vi] = g[G_SX] * Lx[c] + g[G_SY] * Ly[c];
                }
            }
            __syncthreads();
            if (vol) {
                const real *ar = sFr + ve * 4 * Np;
                const real *as = sFs + ve * 4 * Np;
#pragma unroll
                for (int j = 0; j < Np; ++j) {
                    const real wr = sWr[vi * Np + j], ws = sWs[vi * Np + j];
#pragma unroll
                    for (int c = 0; c < 4; ++c) R[c] += wr * ar[c * Np + j] + ws * as[c * Np + j];
                }
            }
        }
        if (vol) {
            const long long base = (k0 + ve) * 4 * Np + vi;
            if (sp.src) {
#pragma unroll
                for (int c = 0; c < 4; ++c) R[c] += to_real<real>(sp.src[base + c * Np]);
            }
            if (sp.mode == STAGE_RHS_ONLY) {
#pragma unroll
                for (int c = 0; c < 4; ++c) sp.Rout[base + c * Np] = to_f64<real>(R[c]);
            } else {
                const real dtr = to_real<real>(sp.dt);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long idx = base + c * Np;
                    double inc = to_f64<real>(dtr * R[c]);
                    double k1 = sp.first_stage ? inc : fma(sp.A, sp.K1[idx], inc);
                    sp.K1[idx] = k1;
                    sp.K0out[idx] = fma(sp.B, k1, sp.K0in[idx]);
                }
            }
        }
    }
}

}  // namespace dg
