// dg_stage_mixed2.cuh -- the mixed-precision stage kernel with two nodes per
// thread.
//
// Same method, staging and phases as dg_stage_mixed.cuh (strong-form
// residual of Eq. dg_on_K, one stage of Algorithm 1, FP32 arithmetic with
// FP64 state, pressure recovery and registers).  The contractions there read
// one broadcast operand record (a node's four fields) per operator entry and
// feed one output node; shared-memory wavefronts, not FMAs, bound that
// kernel.  Here a thread owns volume nodes q and q + H of its element and two
// face nodes r and r + HF of one face, so every broadcast record feeds two
// outputs (and both face nodes share the neighbour's records), at 128
// threads per block with up to 128 registers per thread.
#pragma once
#include "dg_stage_mixed.cuh"

namespace dg {

template <int P>
struct Shape2 {
    static constexpr int Np = (P + 1) * (P + 2) / 2, Nfp = P + 1, NF = 3 * Nfp;
    static constexpr int H = (Np + 1) / 2;           // volume slot q: nodes q, q + H
    static constexpr int HF = (Nfp + 1) / 2;         // face slot (f, r): face nodes r, r + HF of face f
    static constexpr int SF = 3 * HF;
    static constexpr int W = H > SF ? H : SF;        // threads per element
    static constexpr int NT = 128;
    static constexpr int E = NT / W;
};

template <int P, bool BATCH, bool FUSE = false>
__global__ void __launch_bounds__(128, 4)
stage_mixed2_kernel(StageParams sp, Phys<float> ph)
{
    using S2 = Shape2<P>;
    constexpr int Np = S2::Np, Nfp = S2::Nfp, NF = S2::NF, E = S2::E, NT = S2::NT;
    constexpr int H = S2::H, HF = S2::HF, SF = S2::SF, W = S2::W;
    using L = MixedLayout<P, false, E>;
    constexpr int NpP = L::NpP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sD = reinterpret_cast<float2 *>(smem_raw + L::oD);
    float *sL = reinterpret_cast<float *>(smem_raw + L::oL);
    int *sFm = reinterpret_cast<int *>(smem_raw + L::oFm);
    int4 *sConn = reinterpret_cast<int4 *>(smem_raw + L::oConn);
    float *sGeo = reinterpret_cast<float *>(smem_raw + L::oGeo);
    float *sNGeo = reinterpret_cast<float *>(smem_raw + L::oNGeo);
    float4 *sU = reinterpret_cast<float4 *>(smem_raw + L::oU);
    float4 *sN = reinterpret_cast<float4 *>(smem_raw + L::oN);
    float *sPo = reinterpret_cast<float *>(smem_raw + L::oPo);
    float *sPn = reinterpret_cast<float *>(smem_raw + L::oPn);
    double *sRaw = reinterpret_cast<double *>(smem_raw + L::oRaw);
    double *sK1 = reinterpret_cast<double *>(smem_raw + L::oK1);
    float4 *sF = reinterpret_cast<float4 *>(smem_raw + L::oF);
    float4 *sFxy = reinterpret_cast<float4 *>(smem_raw + L::oFxy);
    float *sNorm = reinterpret_cast<float *>(smem_raw + L::oNorm);
    float4 *sDH = reinterpret_cast<float4 *>(smem_raw + L::oDH);
    const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(smem_raw));

    const int tid = threadIdx.x;
    {
        const float *ops = static_cast<const float *>(sp.ops);   // Dr | Ds | LIFT
        for (int i = tid; i < Np * Np; i += NT) sD[i] = make_float2(ops[i], ops[Np * Np + i]);
        for (int i = tid; i < Np * NF; i += NT) sL[i] = ops[2 * Np * Np + i];
        for (int i = tid; i < NF; i += NT) sFm[i] = sp.fmask[i];
    }
    const float *geo = static_cast<const float *>(sp.geo);
    const long long K = sp.K;
    const long long ntiles = BATCH ? sp.ntiles : (K + E - 1) / E;
    const double gm1d = sp.gm1;
    const float cinv_fac = 0.5f * float(P + 1) * float(P + 2);
    const float sig_fac = static_cast<float>(sp.sig_fac);
    float dtr = static_cast<float>(sp.dt);
    const bool update = sp.mode == STAGE_UPDATE;
    bool need_k1 = update && !sp.first_stage;
    __syncthreads();
    pdl_wait_then_release();

    const int el = tid / W, q = tid - (tid / W) * W;
    // volume slot: nodes i0, i1 (i1 = i0 when q + H is past the last node)
    const bool vslot = q < H;
    const int i0 = q, i1 = (q + H < Np) ? q + H : q;
    const bool v1 = vslot && (q + H < Np);
    // face slot: face ff, face nodes fi0, fi1 (fi1 = fi0 when past the face)
    const bool fslot = q < SF;
    const int ff = q / HF, rr = q - (q / HF) * HF;
    const int fi0 = rr, fi1 = (rr + HF < Nfp) ? rr + HF : rr;
    const bool f1 = fslot && (rr + HF < Nfp);

    for (int stg = 0; stg < (FUSE ? 5 : 1); ++stg) {
    if constexpr (FUSE) {
        if (stg > 0 && !grid_sync(sp.bar, sp.bar_err, gridDim.x, sp.bar_limit)) return;
        fused_stage(sp, stg);
        need_k1 = update && stg > 0;
    }
    // Software pipeline over the block's tiles.  Group A (FP32 state, pressure
    // and geometry of the tile and its neighbours) of tile t + 1 is copied
    // while tile t runs its update (P4), which reads none of those buffers;
    // group B (the FP64 registers K0, K1) of tile t is copied while tile t
    // runs P2 and P3.  The connectivity is double-buffered.
    auto tile_at = [&](long long t, long long &k0t, int &net) {
        if constexpr (BATCH) {
            const int4 td = sp.tiles[t];
            k0t = td.x;
            net = td.y;
        } else {
            k0t = t * E;
            net = static_cast<int>((K - k0t) < E ? (K - k0t) : E);
        }
    };
    auto issue_a = [&](long long k0t, int net, const int4 *cnt) {
        const char *gU = reinterpret_cast<const char *>(sp.Sin + k0t * Np);
        for (int c = tid; c < net * Np; c += NT) cp_async16(sbase + L::oU + 16u * c, gU + 16 * c);
        const char *gP = reinterpret_cast<const char *>(sp.Pin + k0t * NpP);
        for (int c = tid; c < net * (NpP / 4); c += NT) cp_async16(sbase + L::oPo + 16u * c, gP + 16 * c);
        const char *gG = reinterpret_cast<const char *>(geo + k0t * 16);
        for (int c = tid; c < net * 4; c += NT) cp_async16(sbase + L::oGeo + 16u * c, gG + 16 * c);
        for (int c = tid; c < net * 3 * Np; c += NT) {
            const int seg = c / Np, j = c - (c / Np) * Np;
            const int4 cn = cnt[seg / 3];
            const int f = seg - 3 * (seg / 3);
            const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            cp_async16(sbase + L::oN + 16u * c, sp.Sin + nb * Np + j);
        }
        for (int c = tid; c < net * 3 * (NpP / 4); c += NT) {
            const int seg = c / (NpP / 4), qq = c - (c / (NpP / 4)) * (NpP / 4);
            const int4 cn = cnt[seg / 3];
            const int f = seg - 3 * (seg / 3);
            const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            cp_async16(sbase + L::oPn + 16u * c, sp.Pin + nb * NpP + 4 * qq);
        }
        for (int c = tid; c < net * 3 * 4; c += NT) {
            const int seg = c >> 2, qq = c & 3;
            const int4 cn = cnt[seg / 3];
            const int f = seg - 3 * (seg / 3);
            const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
            cp_async16(sbase + L::oNGeo + 16u * c, geo + nb * 16 + 4 * qq);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    long long tile = blockIdx.x;
    int buf = 0;
    if (tile < ntiles) {
        long long k0f;
        int nef;
        tile_at(tile, k0f, nef);
        if (tid < nef) sConn[tid] = sp.conn[k0f + tid];
        __syncthreads();
        issue_a(k0f, nef, sConn);
    }
    for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
        long long k0;
        int ne;
        tile_at(tile, k0, ne);
        if constexpr (BATCH) {
            const BatchCase &cs = sp.cases[sp.tiles[tile].z];
            ph.mu = cvt_d2f(cs.mu);           // integer conversions: no FP64-pipe work per tile
            ph.vw2 = cvt_d2f(cs.vb);
            dtr = cvt_d2f(cs.dt);
        }
        const int4 *cnb = sConn + buf * E;
        int4 *cnx = sConn + (buf ^ 1) * E;
        const long long tn = tile + gridDim.x;
        const bool has_next = tn < ntiles;
        long long k0n = 0;
        int nen = 0;
        if (has_next) {
            tile_at(tn, k0n, nen);
            if (tid < nen) cnx[tid] = sp.conn[k0n + tid];
        }
        // ---- P1: group B of this tile; wait for group A
        {
            const char *gR = reinterpret_cast<const char *>(sp.K0in + k0 * 4 * Np);
            for (int c = tid; c < ne * 2 * Np; c += NT) cp_async16(sbase + L::oRaw + 16u * c, gR + 16 * c);
            if (need_k1) {
                const char *gK = reinterpret_cast<const char *>(sp.K1 + k0 * 4 * Np);
                for (int c = tid; c < ne * 2 * Np; c += NT) cp_async16(sbase + L::oK1 + 16u * c, gK + 16 * c);
            }
            asm volatile("cp.async.commit_group;\n" ::);
            asm volatile("cp.async.wait_group 1;\n" ::);
        }
        __syncthreads();

        const bool live = el < ne;
        // ---- P2: gradients and fluxes of two volume nodes; norms of two face nodes
        if (live && vslot) {
            const float4 *ue = sU + el * Np;
            float ur[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}}, us[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                const float4 uj = ue[j];
                acc_rs(ur[0], us[0], sD[i0 * Np + j], uj);
                acc_rs(ur[1], us[1], sD[i1 * Np + j], uj);
            }
            const float *g = sGeo + el * 16;
            const float rx = g[G_RX], ry = g[G_RY], sx = g[G_SX], sy = g[G_SY];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a == 1 && !v1) break;
                const int vi = a ? i1 : i0;
                float u[4], gx[4], gy[4];
                f4_to(ue[vi], u);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    gx[c] = rx * ur[a][c] + sx * us[a][c];
                    gy[c] = ry * ur[a][c] + sy * us[a][c];
                }
                const float p = sPo[el * NpP + vi];
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
                sF[(el * Np + vi) * 2] = to_f4(fr);
                sF[(el * Np + vi) * 2 + 1] = to_f4(fs);
                sFxy[(el * Np + vi) * 2] = to_f4(Fx);
                sFxy[(el * Np + vi) * 2 + 1] = to_f4(Fy);
            }
        }
        int btype = 0, f2 = 0;
        if (live && fslot) {
            const int4 cn = cnb[el];
            f2 = (cn.w >> (2 * ff)) & 3;
            btype = (cn.w >> (8 + 2 * ff)) & 3;
            const float *g = sGeo + el * 16;
            const float n1 = g[G_NX + ff], n2 = g[G_NY + ff];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (b == 1 && !f1) break;
                const int fi = b ? fi1 : fi0;
                const int vm = sFm[ff * Nfp + fi], vp = sFm[f2 * Nfp + (Nfp - 1 - fi)];
                float u[4];
                f4_to(sU[el * Np + vm], u);
                float w[4];
                if (btype == BCT_INTERIOR) f4_to(sN[(el * 3 + ff) * Np + vp], w);
                const float pw = (btype == BCT_WALL) ? sPo[el * NpP + vm] : 0.f;
                sNorm[el * NF + ff * Nfp + fi] = trace_norms_max(u, 1.0f / u[0], pw, btype, w, n1, n2, ph);
            }
        }
        __syncthreads();

        // ---- P3: divergence of two volume nodes; fluxes of two face nodes
        float Dv[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        if (live && vslot) {
            const float4 *fe4 = sF + el * Np * 2;
#pragma unroll
            for (int j = 0; j < Np; ++j) {
                const float4 a = fe4[2 * j], b = fe4[2 * j + 1];
                const float2 d0 = sD[i0 * Np + j], d1 = sD[i1 * Np + j];
                Dv[0][0] = fmaf(d0.x, a.x, fmaf(d0.y, b.x, Dv[0][0]));
                Dv[0][1] = fmaf(d0.x, a.y, fmaf(d0.y, b.y, Dv[0][1]));
                Dv[0][2] = fmaf(d0.x, a.z, fmaf(d0.y, b.z, Dv[0][2]));
                Dv[0][3] = fmaf(d0.x, a.w, fmaf(d0.y, b.w, Dv[0][3]));
                Dv[1][0] = fmaf(d1.x, a.x, fmaf(d1.y, b.x, Dv[1][0]));
                Dv[1][1] = fmaf(d1.x, a.y, fmaf(d1.y, b.y, Dv[1][1]));
                Dv[1][2] = fmaf(d1.x, a.z, fmaf(d1.y, b.z, Dv[1][2]));
                Dv[1][3] = fmaf(d1.x, a.w, fmaf(d1.y, b.w, Dv[1][3]));
            }
        }
        if (live && fslot) {
            const float *g = sGeo + el * 16;
            const float n1 = g[G_NX + ff], n2 = g[G_NY + ff], fsc = g[G_FS + ff];
            float gbar = 0.f;
#pragma unroll
            for (int l = 0; l < Nfp; ++l) gbar = fmaxf(gbar, sNorm[el * NF + ff * Nfp + l]);
            float cinv = cinv_fac * fsc;
            const float *ng = sNGeo + (el * 3 + ff) * 16;
            if (btype == BCT_INTERIOR) cinv = fmaxf(cinv, cinv_fac * ng[G_FS + f2]);
            const float sigma = sig_fac * gbar * cinv;
            const int vm0 = sFm[ff * Nfp + fi0], vm1 = sFm[ff * Nfp + fi1];
            const int vp0 = sFm[f2 * Nfp + (Nfp - 1 - fi0)], vp1 = sFm[f2 * Nfp + (Nfp - 1 - fi1)];
            // gradients needed at the two face nodes: the neighbour's (interior)
            // or the own one (wall), with the operator records shared
            float wr[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}}, ws[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
            if (btype != BCT_FARFIELD) {
                const bool inner = btype == BCT_INTERIOR;
                const float4 *src = inner ? sN + (el * 3 + ff) * Np : sU + el * Np;
                const int r0 = inner ? vp0 : vm0, r1 = inner ? vp1 : vm1;
#pragma unroll
                for (int j = 0; j < Np; ++j) {
                    const float4 wj = src[j];
                    acc_rs(wr[0], ws[0], sD[r0 * Np + j], wj);
                    acc_rs(wr[1], ws[1], sD[r1 * Np + j], wj);
                }
            }
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (b == 1 && !f1) break;
                const int fi = b ? fi1 : fi0, vm = b ? vm1 : vm0, vp = b ? vp1 : vp0;
                float up[4], dH[4], Ftp[4];
                f4_to(sU[el * Np + vm], up);
                const float pp = sPo[el * NpP + vm];
                {
                    const float4 a = sFxy[(el * Np + vm) * 2], c = sFxy[(el * Np + vm) * 2 + 1];
                    Ftp[0] = a.x * n1 + c.x * n2; Ftp[1] = a.y * n1 + c.y * n2;
                    Ftp[2] = a.z * n1 + c.z * n2; Ftp[3] = a.w * n1 + c.w * n2;
                }
                if (btype == BCT_INTERIOR) {
                    float um[4], gxm[4], gym[4];
                    f4_to(sN[(el * 3 + ff) * Np + vp], um);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        gxm[c] = ng[G_RX] * wr[b][c] + ng[G_SX] * ws[b][c];
                        gym[c] = ng[G_RY] * wr[b][c] + ng[G_SY] * ws[b][c];
                    }
                    const float pm = sPn[(el * 3 + ff) * NpP + vp];
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
                    float gxp[4], gyp[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        gxp[c] = g[G_RX] * wr[b][c] + g[G_SX] * ws[b][c];
                        gyp[c] = g[G_RY] * wr[b][c] + g[G_SY] * ws[b][c];
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
                sDH[el * NF + ff * Nfp + fi] = make_float4(fsc * dH[0], fsc * dH[1], fsc * dH[2], fsc * dH[3]);
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();
        if (has_next) issue_a(k0n, nen, cnx);

        // ---- P4: lift, the stage update and the FP32 copy of the new state
        if (live && vslot) {
            const float4 *dh = sDH + el * NF;
            float R[2][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                R[0][c] = -Dv[0][c];
                R[1][c] = -Dv[1][c];
            }
#pragma unroll
            for (int m = 0; m < NF; ++m) {
                const float4 h = dh[m];
                const float l0 = sL[i0 * NF + m], l1 = sL[i1 * NF + m];
                R[0][0] = fmaf(l0, h.x, R[0][0]); R[0][1] = fmaf(l0, h.y, R[0][1]);
                R[0][2] = fmaf(l0, h.z, R[0][2]); R[0][3] = fmaf(l0, h.w, R[0][3]);
                R[1][0] = fmaf(l1, h.x, R[1][0]); R[1][1] = fmaf(l1, h.y, R[1][1]);
                R[1][2] = fmaf(l1, h.z, R[1][2]); R[1][3] = fmaf(l1, h.w, R[1][3]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a == 1 && !v1) break;
                const int vi = a ? i1 : i0;
                const long long base = (k0 + el) * 4 * Np + vi;
                if (sp.src) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) R[a][c] += cvt_d2f(sp.src[base + c * Np]);
                }
                if (!update) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) sp.Rout[base + c * Np] = cvt_f2d(R[a][c]);
                } else {
                    double knew[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double inc = cvt_f2d(dtr * R[a][c]);
                        const double k1 = sp.first_stage ? inc : fma(sp.A, sK1[(el * 4 + c) * Np + vi], inc);
                        sp.K1[base + c * Np] = k1;
                        knew[c] = fma(sp.B, k1, sRaw[(el * 4 + c) * Np + vi]);
                        sp.K0out[base + c * Np] = knew[c];
                    }
                    const float un[4] = {cvt_d2f_trunc(knew[0]), cvt_d2f_trunc(knew[1]),
                                         cvt_d2f_trunc(knew[2]), cvt_d2f_trunc(knew[3])};
                    sp.Sout[(k0 + el) * Np + vi] = to_f4(un);
                    sp.Pout[(k0 + el) * NpP + vi] = pressure<float>(un, knew[3], gm1d);
                }
            }
        }
        __syncthreads();
    }
    }  // stages
}

}  // namespace dg
