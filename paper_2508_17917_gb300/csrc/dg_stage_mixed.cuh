// dg_stage_mixed.cuh -- fused residual + LSRK stage, mixed precision.
//
// Same method and phase structure as dg_stage.cuh (strong-form residual of
// Eq. dg_on_K and one stage of Algorithm 1), organised for GB300's FP32 and
// integer pipes:
//   * the state stays FP64 in HBM; a warp copies one 4*Np-double segment
//     (own element or one neighbour) with 16-byte loads and converts it to
//     FP32 by integer operations (cvt_d2f_trunc);
//   * shared memory holds node-major float4 records (rho, m1, m2, E), so one
//     LDS.128 feeds all four fields of a node; Dr and Ds are interleaved as
//     float2 so one LDS.64 feeds both derivative directions;
//   * the raw FP64 energies of the own element and of the neighbours stay in
//     shared memory for the FP64 pressure recovery, the raw own state for the
//     FP64 register update, and the tile's K1 block arrives by cp.async while
//     the other phases run;
//   * the volume phase keeps the total flux F = F_c - v_w U - G grad U of
//     every node, so a face node takes F+.n from it instead of re-evaluating
//     the own side's advective and viscous fluxes.
#pragma once
#include "dg_stage.cuh"

namespace dg {

// FP64 -> FP32 by truncation with integer operations (LOP3, IADD, SHF, ISETP,
// SEL, LOP3): magnitudes below 2^-126 flush to zero.  Finite states only (a
// non-finite state still shows up in the FP64 state after the update).
__device__ __forceinline__ float cvt_d2f_trunc(double d)
{
    unsigned hi = static_cast<unsigned>(__double2hiint(d));
    unsigned lo = static_cast<unsigned>(__double2loint(d));
    unsigned mag = hi & 0x7fffffffu;
    unsigned t = mag - 0x38000000u;              // exponent 1023 -> 127 bias
    unsigned f = __funnelshift_l(lo, t, 3);      // (t << 3) | (lo >> 29)
    f = (mag < 0x38100000u) ? 0u : f;
    return __uint_as_float(f | (hi & 0x80000000u));
}

// r[c] += d.x * u[c], s[c] += d.y * u[c] for the four fields of one node
__device__ __forceinline__ void acc_rs(float r[4], float s[4], const float2 d, const float4 u)
{
    r[0] = fmaf(d.x, u.x, r[0]); r[1] = fmaf(d.x, u.y, r[1]); r[2] = fmaf(d.x, u.z, r[2]); r[3] = fmaf(d.x, u.w, r[3]);
    s[0] = fmaf(d.y, u.x, s[0]); s[1] = fmaf(d.y, u.y, s[1]); s[2] = fmaf(d.y, u.z, s[2]); s[3] = fmaf(d.y, u.w, s[3]);
}

template <int P>
struct MixedLayout {
    using S = Shape<P>;
    static constexpr int Np = S::Np, NF = S::NF, E = S::E;
    static constexpr size_t al(size_t b) { return (b + 15) & ~size_t(15); }
    static constexpr size_t oD = 0;                                      // float2 Np*Np (Dr, Ds)
    static constexpr size_t oL = oD + al(sizeof(float2) * Np * Np);      // float Np*NF
    static constexpr size_t oFm = oL + al(sizeof(float) * Np * NF);      // int NF
    static constexpr size_t oConn = oFm + al(sizeof(int) * NF);          // int4 E
    static constexpr size_t oGeo = oConn + al(sizeof(int4) * E);         // float E*16
    static constexpr size_t oNGeo = oGeo + al(sizeof(float) * E * 16);   // float4 E*3*2
    static constexpr size_t oU = oNGeo + al(sizeof(float4) * E * 3 * 2); // float4 E*Np
    static constexpr size_t oN = oU + al(sizeof(float4) * E * Np);       // float4 E*3*Np
    static constexpr size_t oRaw = oN + al(sizeof(float4) * E * 3 * Np); // double E*4*Np
    static constexpr size_t oNEd = oRaw + al(sizeof(double) * E * 4 * Np);  // double E*3*Np
    static constexpr size_t oF = oNEd + al(sizeof(double) * E * 3 * Np);    // float4 E*Np*2
    static constexpr size_t oP = oF + al(sizeof(float4) * E * Np * 2);      // float E*Np
    static constexpr size_t oNorm = oP + al(sizeof(float) * E * Np);        // float E*NF
    static constexpr size_t oDH = oNorm + al(sizeof(float) * E * NF);       // float4 E*NF
    static constexpr size_t oK1 = oDH + al(sizeof(float4) * E * NF);        // double E*4*Np
    static constexpr size_t oFxy = oK1 + al(sizeof(double) * E * 4 * Np);   // float4 E*Np*2
    static constexpr size_t oNed = oFxy + al(sizeof(float4) * E * Np * 2);  // double scratch slot
    static constexpr size_t bytes = oNed + 16;
};

__device__ __forceinline__ void f4_to(const float4 &a, float o[4]) { o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; }
__device__ __forceinline__ float4 to_f4(const float o[4]) { return make_float4(o[0], o[1], o[2], o[3]); }

template <int P>
__global__ void __launch_bounds__(Shape<P>::NT, 3)
stage_mixed_kernel(StageParams sp, Phys<float> ph)
{
    using S = Shape<P>;
    using L = MixedLayout<P>;
    constexpr int Np = S::Np, Nfp = S::Nfp, NF = S::NF, E = S::E, NT = S::NT;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sD = reinterpret_cast<float2 *>(smem_raw + L::oD);
    float *sL = reinterpret_cast<float *>(smem_raw + L::oL);
    int *sFm = reinterpret_cast<int *>(smem_raw + L::oFm);
    int4 *sConn = reinterpret_cast<int4 *>(smem_raw + L::oConn);
    float *sGeo = reinterpret_cast<float *>(smem_raw + L::oGeo);
    float4 *sNGeo = reinterpret_cast<float4 *>(smem_raw + L::oNGeo);
    float4 *sU = reinterpret_cast<float4 *>(smem_raw + L::oU);
    float4 *sN = reinterpret_cast<float4 *>(smem_raw + L::oN);
    double *sRaw = reinterpret_cast<double *>(smem_raw + L::oRaw);
    double *sNEd = reinterpret_cast<double *>(smem_raw + L::oNEd);
    float4 *sF = reinterpret_cast<float4 *>(smem_raw + L::oF);
    float *sP = reinterpret_cast<float *>(smem_raw + L::oP);
    float *sNorm = reinterpret_cast<float *>(smem_raw + L::oNorm);
    float4 *sDH = reinterpret_cast<float4 *>(smem_raw + L::oDH);
    double *sK1 = reinterpret_cast<double *>(smem_raw + L::oK1);
    float4 *sFxy = reinterpret_cast<float4 *>(smem_raw + L::oFxy);
    double *sDummy = reinterpret_cast<double *>(smem_raw + L::oNed);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const float *ops = static_cast<const float *>(sp.ops);   // Dr | Ds | LIFT
        for (int i = tid; i < Np * Np; i += NT) sD[i] = make_float2(ops[i], ops[Np * Np + i]);
        for (int i = tid; i < Np * NF; i += NT) sL[i] = ops[2 * Np * Np + i];
        for (int i = tid; i < NF; i += NT) sFm[i] = sp.fmask[i];
    }
    const float *geo = static_cast<const float *>(sp.geo);
    const double *K0 = sp.K0in;
    const long long K = sp.K;
    const long long ntiles = (K + E - 1) / E;
    const double gm1d = sp.gm1;
    const float cinv_fac = 0.5f * float(P + 1) * float(P + 2);
    const float C1x3 = 3.0f * static_cast<float>(sp.C1);
    const float dtr = static_cast<float>(sp.dt);

    // per-lane chunk decomposition of a 4*Np segment: chunk ch holds doubles
    // 2ch, 2ch+1 of the [c][node] segment
    constexpr int NCH = 2 * Np;
    constexpr int NIT = (NCH + 31) / 32;
    int ch_c0[NIT], ch_j0[NIT], ch_c1[NIT], ch_j1[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        int ch = lane + 32 * it;
        int q = 2 * ch;
        ch_c0[it] = q / Np; ch_j0[it] = q - (q / Np) * Np;
        ch_c1[it] = (q + 1) / Np; ch_j1[it] = (q + 1) - ((q + 1) / Np) * Np;
    }
    __syncthreads();

    const int ve = tid / Np, vi = tid - (tid / Np) * Np;
    const int fe = tid / NF, fm = tid - (tid / NF) * NF;
    const int ff = fm / Nfp, fi = fm - (fm / Nfp) * Nfp;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long k0 = tile * E;
        const int ne = static_cast<int>((K - k0) < E ? (K - k0) : E);
        // ---- P1a: connectivity and own geometry of the tile
        if (tid < ne) sConn[tid] = sp.conn[k0 + tid];
        for (int idx = tid; idx < ne * 16; idx += NT) sGeo[idx] = geo[k0 * 16 + idx];
        __syncthreads();
        // ---- P1b: K1 block by asynchronous copies; own and neighbour state segments
        const bool need_k1 = (sp.mode == STAGE_UPDATE) && !sp.first_stage;
        if (need_k1) {
            const char *g = reinterpret_cast<const char *>(sp.K1 + k0 * 4 * Np);
            const unsigned s0 = static_cast<unsigned>(__cvta_generic_to_shared(sK1));
            for (int ch = tid; ch < ne * 2 * Np; ch += NT)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0 + 16u * ch),
                             "l"(g + 16 * ch));
            asm volatile("cp.async.commit_group;\n" ::);
        }
        for (int e = warp; e < ne; e += NW) {
            const double2 *g2 = reinterpret_cast<const double2 *>(K0 + (k0 + e) * (4 * Np));
            float *dstf = reinterpret_cast<float *>(sU + e * Np);
            double2 *raw = reinterpret_cast<double2 *>(sRaw + e * 4 * Np);
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int ch = lane + 32 * it;
                if (ch < NCH) {
                    const double2 v = __ldg(g2 + ch);
                    dstf[ch_j0[it] * 4 + ch_c0[it]] = cvt_d2f_trunc(v.x);
                    dstf[ch_j1[it] * 4 + ch_c1[it]] = cvt_d2f_trunc(v.y);
                    raw[ch] = v;
                }
            }
        }
        for (int seg = warp; seg < ne * 3; seg += NW) {
            const int e = seg / 3, f = seg - 3 * (seg / 3);
            const int4 cn = sConn[e];
            const long long src = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            const double2 *g2 = reinterpret_cast<const double2 *>(K0 + src * (4 * Np));
            float *dstf = reinterpret_cast<float *>(sN + seg * Np);
            double *ned = sNEd + seg * Np;
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int ch = lane + 32 * it;
                if (ch < NCH) {
                    const double2 v = __ldg(g2 + ch);
                    dstf[ch_j0[it] * 4 + ch_c0[it]] = cvt_d2f_trunc(v.x);
                    dstf[ch_j1[it] * 4 + ch_c1[it]] = cvt_d2f_trunc(v.y);
                    // raw energies for the FP64 pressure; other fields go to a dummy slot
                    *((ch_c0[it] == 3) ? ned + ch_j0[it] : sDummy) = v.x;
                    *((ch_c1[it] == 3) ? ned + ch_j1[it] : sDummy) = v.y;
                }
            }
        }
        if (tid < ne * 3) {
            const int e = tid / 3, f = tid - 3 * (tid / 3);
            const int4 cn = sConn[e];
            const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            const int f2 = (cn.w >> (2 * f)) & 3;
            const float4 m = *reinterpret_cast<const float4 *>(geo + nb * 16);
            sNGeo[tid * 2] = m;                                   // rx, ry, sx, sy
            sNGeo[tid * 2 + 1] = make_float4(geo[nb * 16 + G_FS + f2], 0.f, 0.f, 0.f);
        }
        __syncthreads();

        // ---- P2: volume gradient and fluxes; face-node penalty norms
        const bool vol = ve < ne;
        if (vol) {
            const float4 *ue = sU + ve * Np;
            float ur[4] = {0, 0, 0, 0}, us[4] = {0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < Np; ++j) acc_rs(ur, us, sD[vi * Np + j], ue[j]);
            const float *g = sGeo + ve * 16;
            const float rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
            float u[4], gx[4], gy[4];
            f4_to(ue[vi], u);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                gx[c] = rx * ur[c] + sx * us[c];
                gy[c] = ry * ur[c] + sy * us[c];
            }
            const float p = pressure<float>(u, sRaw[(ve * 4 + 3) * Np + vi], gm1d);
            sP[ve * Np + vi] = p;
            float cx[4], cy[4], vx[4], vy[4], fr[4], fs[4], Fx[4], Fy[4];
            adv_flux(u, p, ph, cx, cy);
            visc_flux(u, gx, gy, ph, vx, vy);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Fx[c] = cx[c] - vx[c];
                Fy[c] = cy[c] - vy[c];
                fr[c] = rx * Fx[c] + ry * Fy[c];
                fs[c] = sx * Fx[c] + sy * Fy[c];
            }
            sF[(ve * Np + vi) * 2] = to_f4(fr);
            sF[(ve * Np + vi) * 2 + 1] = to_f4(fs);
            sFxy[(ve * Np + vi) * 2] = to_f4(Fx);
            sFxy[(ve * Np + vi) * 2 + 1] = to_f4(Fy);
        }
        const bool face = fe < ne;
        int btype = 0, vm = 0, vp = 0;
        if (face) {
            const int4 cn = sConn[fe];
            const int f2 = (cn.w >> (2 * ff)) & 3;
            btype = (cn.w >> (8 + 2 * ff)) & 3;
            vm = sFm[ff * Nfp + fi];
            vp = sFm[f2 * Nfp + (Nfp - 1 - fi)];
            const float *g = sGeo + fe * 16;
            const float n1 = g[G_NX + ff], n2 = g[G_NY + ff];
            float u[4];
            f4_to(sU[fe * Np + vm], u);
            const float ir = 1.0f / u[0];
            const float a = penalty_norm(u[0], u[1] * ir, u[2] * ir, u[3] * ir, n1, n2, ph);
            float b;
            if (btype == BCT_INTERIOR) {
                float w[4];
                f4_to(sN[(fe * 3 + ff) * Np + vp], w);
                const float iw = 1.0f / w[0];
                b = penalty_norm(w[0], w[1] * iw, w[2] * iw, w[3] * iw, n1, n2, ph);
            } else if (btype == BCT_FARFIELD) {
                const float iw = 1.0f / ph.Uinf[0];
                b = penalty_norm(ph.Uinf[0], ph.Uinf[1] * iw, ph.Uinf[2] * iw, ph.Uinf[3] * iw, n1, n2, ph);
            } else {
                const float pw = pressure<float>(u, sRaw[(fe * 4 + 3) * Np + vm], gm1d);
                const float eb = (pw / ph.gm1 + 0.5f * u[0] * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2)) * ir;
                b = penalty_norm(u[0], ph.vw1, ph.vw2, eb, n1, n2, ph);
            }
            sNorm[fe * NF + fm] = fmaxf(a, b);
        }
        __syncthreads();

        // ---- P3: divergence (volume) and face fluxes (face nodes)
        float Dv[4] = {0, 0, 0, 0};       // divergence sum_j Dr_ij Fr_j + Ds_ij Fs_j
        if (vol) {
            const float4 *fe4 = sF + ve * Np * 2;
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                const float4 a = fe4[2 * j], b = fe4[2 * j + 1];
                const float2 d = sD[vi * Np + j];
                Dv[0] = fmaf(d.x, a.x, fmaf(d.y, b.x, Dv[0]));
                Dv[1] = fmaf(d.x, a.y, fmaf(d.y, b.y, Dv[1]));
                Dv[2] = fmaf(d.x, a.z, fmaf(d.y, b.z, Dv[2]));
                Dv[3] = fmaf(d.x, a.w, fmaf(d.y, b.w, Dv[3]));
            }
        }
        if (face) {
            const float *g = sGeo + fe * 16;
            const float n1 = g[G_NX + ff], n2 = g[G_NY + ff], fsc = g[G_FS + ff];
            float gbar = 0.f;
#pragma unroll
            for (int l = 0; l < Nfp; ++l) gbar = fmaxf(gbar, sNorm[fe * NF + ff * Nfp + l]);
            float cinv = cinv_fac * fsc;
            if (btype == BCT_INTERIOR) cinv = fmaxf(cinv, cinv_fac * sNGeo[(fe * 3 + ff) * 2 + 1].x);
            const float sigma = C1x3 * gbar * cinv;
            float up[4], dH[4], Ftp[4];
            f4_to(sU[fe * Np + vm], up);
            const float pp = sP[fe * Np + vm];
            {   // F+.n of the total flux F = F_c - v_w U - G grad U, from the volume phase
                const float4 a = sFxy[(fe * Np + vm) * 2], b = sFxy[(fe * Np + vm) * 2 + 1];
                Ftp[0] = a.x * n1 + b.x * n2; Ftp[1] = a.y * n1 + b.y * n2;
                Ftp[2] = a.z * n1 + b.z * n2; Ftp[3] = a.w * n1 + b.w * n2;
            }
            if (btype == BCT_INTERIOR) {
                const float4 *w = sN + (fe * 3 + ff) * Np;
                float wr[4] = {0, 0, 0, 0}, ws[4] = {0, 0, 0, 0};
#pragma unroll
                for (int j = 0; j < Np; ++j) acc_rs(wr, ws, sD[vp * Np + j], w[j]);
                const float4 nm0 = sNGeo[(fe * 3 + ff) * 2];
                float um[4], gxm[4], gym[4];
                f4_to(w[vp], um);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    gxm[c] = nm0.x * wr[c] + nm0.z * ws[c];
                    gym[c] = nm0.y * wr[c] + nm0.w * ws[c];
                }
                const float pm = pressure<float>(um, sNEd[(fe * 3 + ff) * Np + vp], gm1d);
                float Fnm[4], vxm[4], vym[4], D[4];
                flux_n(um, pm, n1, n2, ph, Fnm);
                visc_flux(um, gxm, gym, ph, vxm, vym);
                roe_dissipation(up, pp, um, pm, n1, n2, ph, D);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float Ftm = Fnm[c] - (vxm[c] * n1 + vym[c] * n2);
                    dH[c] = 0.5f * (Ftp[c] - Ftm) - 0.5f * D[c] - sigma * (up[c] - um[c]);
                }
            } else if (btype == BCT_FARFIELD) {
                const float ub[4] = {ph.Uinf[0], ph.Uinf[1], ph.Uinf[2], ph.Uinf[3]};
                float Fnp[4], Fnb[4], D[4];
                flux_n(up, pp, n1, n2, ph, Fnp);
                flux_n(ub, ph.pinf, n1, n2, ph, Fnb);
                roe_dissipation(up, pp, ub, ph.pinf, n1, n2, ph, D);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dH[c] = 0.5f * (Fnp[c] - Fnb[c]) - 0.5f * D[c] - sigma * (up[c] - ub[c]);
            } else {
                // own broken gradient at the wall node (wall faces only)
                float gxp[4], gyp[4];
                {
                    float ar[4] = {0, 0, 0, 0}, as[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < Np; ++j) acc_rs(ar, as, sD[vm * Np + j], sU[fe * Np + j]);
                    const float rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        gxp[c] = rx * ar[c] + sx * as[c];
                        gyp[c] = ry * ar[c] + sy * as[c];
                    }
                }
                const float rb = up[0];
                const float kw = 0.5f * rb * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2);
                const float ub[4] = {rb, rb * ph.vw1, rb * ph.vw2, pp / ph.gm1 + kw};
                float Fnb[4], vxb[4], vyb[4], qx, qy;
                flux_n(ub, pp, n1, n2, ph, Fnb);
                visc_flux_prim(rb, ph.vw1, ph.vw2, ub[3] / rb, gxp, gyp, ph, vxb, vyb, &qx, &qy);
                float vnb[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) vnb[c] = vxb[c] * n1 + vyb[c] * n2;
                if (ph.adiabatic) vnb[3] -= qx * n1 + qy * n2;
#pragma unroll
                for (int c = 0; c < 4; ++c) dH[c] = Ftp[c] - (Fnb[c] - vnb[c] + sigma * (up[c] - ub[c]));
            }
            sDH[fe * NF + fm] = make_float4(fsc * dH[0], fsc * dH[1], fsc * dH[2], fsc * dH[3]);
        }
        if (need_k1) asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();

        // ---- P4: lift and the stage update
        if (vol) {
            const float4 *dh = sDH + ve * NF;
            float R[4] = {-Dv[0], -Dv[1], -Dv[2], -Dv[3]};
#pragma unroll
            for (int m = 0; m < NF; ++m) {
                const float4 h = dh[m];
                const float l = sL[vi * NF + m];
                R[0] = fmaf(l, h.x, R[0]); R[1] = fmaf(l, h.y, R[1]); R[2] = fmaf(l, h.z, R[2]); R[3] = fmaf(l, h.w, R[3]);
            }
            const long long base = (k0 + ve) * 4 * Np + vi;
            if (sp.src) {
#pragma unroll
                for (int c = 0; c < 4; ++c) R[c] += cvt_d2f(sp.src[base + c * Np]);
            }
            if (sp.mode == STAGE_RHS_ONLY) {
#pragma unroll
                for (int c = 0; c < 4; ++c) sp.Rout[base + c * Np] = cvt_f2d(R[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double inc = cvt_f2d(dtr * R[c]);
                    const double k1 = sp.first_stage ? inc : fma(sp.A, sK1[(ve * 4 + c) * Np + vi], inc);
                    sp.K1[base + c * Np] = k1;
                    sp.K0out[base + c * Np] = fma(sp.B, k1, sRaw[(ve * 4 + c) * Np + vi]);
                }
            }
        }
    }
}

}  // namespace dg
