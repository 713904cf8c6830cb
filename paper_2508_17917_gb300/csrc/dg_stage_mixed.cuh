// dg_stage_mixed.cuh -- fused residual + LSRK stage, mixed precision.
//
// Same method and phase structure as dg_stage.cuh (strong-form residual of
// Eq. dg_on_K and one stage of Algorithm 1), organised for GB300:
//   * the state and the Runge-Kutta register stay FP64 in HBM; every stage
//     also writes an FP32 copy of its output state (node-major float4 records
//     rho, m1, m2, E) and the node pressure, recovered in FP64 from the FP64
//     energy (p = (gamma-1)(E - rho|v|^2/2), Sec. 2.1) once per node;
//   * the next stage stages everything it reads -- own and neighbour FP32
//     records and pressures, the own FP64 state and K1 block, geometry --
//     with asynchronous 16-byte copies (cp.async), so no thread converts or
//     waits on a global load in the staging phase;
//   * node-major float4 records feed all four fields of a node with one
//     LDS.128; Dr and Ds are interleaved as 8-byte float2 records;
//   * the volume phase keeps the total flux F = F_c - v_w U - G grad U of
//     every node, so a face node reads F+.n instead of re-evaluating it;
//   * FP64 arithmetic is left to the pressure recovery and the register
//     update; FP64<->FP32 conversions are done with integer operations,
//     because GB300 executes conversion instructions on its FP64 pipe;
//   * the theta variant (SIP, NIPG) adds the face theta vectors, lifts them
//     and applies Wr, Ws to their (r, s) components in a second lift phase,
//     as in dg_stage.cuh.  Both the theta and the penalty term are linear in
//     the face jump U+ - U-, a small difference of large values, so this
//     variant forms the jump in FP64 from the FP64 states (the neighbour's
//     trace read from HBM/L2) instead of from the FP32 copies.
#pragma once
#include "dg_stage.cuh"
#include "pair2.cuh"

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

// r[c] += d.x * u[c], s[c] += d.y * u[c] for the four fields of one node,
// with paired FMAs over the field pairs (0, 1) and (2, 3)
__device__ __forceinline__ void acc_rs(float r[4], float s[4], const float2 d, const float4 u)
{
    const float2 dr = make_float2(d.x, d.x), ds = make_float2(d.y, d.y);
    const float2 u01 = make_float2(u.x, u.y), u23 = make_float2(u.z, u.w);
    const float2 r01 = __ffma2_rn(dr, u01, make_float2(r[0], r[1])), r23 = __ffma2_rn(dr, u23, make_float2(r[2], r[3]));
    const float2 s01 = __ffma2_rn(ds, u01, make_float2(s[0], s[1])), s23 = __ffma2_rn(ds, u23, make_float2(s[2], s[3]));
    r[0] = r01.x; r[1] = r01.y; r[2] = r23.x; r[3] = r23.y;
    s[0] = s01.x; s[1] = s01.y; s[2] = s23.x; s[3] = s23.y;
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

// Programmatic dependent launch: wait until the previous kernel of the
// stream has completed and its writes are visible (a no-op after an ordinary
// launch), then allow the next kernel's blocks to be scheduled as this
// kernel's blocks exit.  Called after the prologue that reads only constant
// operator tables, before the first read or write of the state.
__device__ __forceinline__ void pdl_wait_then_release()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Grid-wide barrier for the fused (cooperative) launch.  Thread 0 of every
// block makes the block's writes visible, counts the block in and waits for
// the generation to advance; the last block in resets the count and advances
// it.  Each wait gives up after `limit` sleeps of about 100 ns, sets *err and
// the kernel returns; blocks already waiting see *err and return too.  All
// blocks of a cooperative launch are resident, so a wait can only run out
// when the limit is (deliberately) too small.  Returns false on an error.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *err, unsigned nblocks, unsigned limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile int *verr = err;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned prev = atomicAdd(bar, 1u);
        int ok = 1;
        if (prev == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == gen) {
                if (*verr || it >= limit) {
                    ok = 0;
                    break;
                }
                ++it;
                __nanosleep(100);
            }
        }
        if (!ok) atomicExch(err, 1);
        __threadfence();
        s_ok = ok && !*verr;
    }
    __syncthreads();
    return s_ok != 0;
}

// Switch the stage-dependent fields of a fused launch to stage `stg`:
// ping-pong buffers, Runge-Kutta coefficients, first-stage flag.
__device__ __forceinline__ void fused_stage(StageParams &sp, int stg)
{
    if (stg > 0) {
        double *o = const_cast<double *>(sp.K0in);
        sp.K0in = sp.K0out;
        sp.K0out = o;
        float4 *so = const_cast<float4 *>(sp.Sin);
        sp.Sin = sp.Sout;
        sp.Sout = so;
        float *po = const_cast<float *>(sp.Pin);
        sp.Pin = sp.Pout;
        sp.Pout = po;
    }
    // constant indices only: a dynamically indexed parameter array would be
    // copied to local memory
    sp.A = stg == 0 ? sp.A5[0] : stg == 1 ? sp.A5[1] : stg == 2 ? sp.A5[2] : stg == 3 ? sp.A5[3] : sp.A5[4];
    sp.B = stg == 0 ? sp.B5[0] : stg == 1 ? sp.B5[1] : stg == 2 ? sp.B5[2] : stg == 3 ? sp.B5[3] : sp.B5[4];
    sp.first_stage = (stg == 0) ? 1 : 0;
}

template <int P, bool TH = false, int EE = Shape<P>::E>
struct MixedLayout {
    using S = Shape<P>;
    static constexpr int Np = S::Np, NF = S::NF, E = EE;
    static constexpr int NpP = (Np + 3) & ~3;                                 // padded pressure row
    static constexpr size_t al(size_t b) { return (b + 15) & ~size_t(15); }
    static constexpr size_t oD = 0;                                           // float2 Np*Np (Dr, Ds)
    static constexpr size_t oL = oD + al(sizeof(float2) * Np * Np);           // float Np*NF
    static constexpr size_t oFm = oL + al(sizeof(float) * Np * NF);           // int NF
    static constexpr size_t oConn = oFm + al(sizeof(int) * NF);               // int4 2E (two tiles)
    static constexpr size_t oGeo = oConn + al(sizeof(int4) * E * 2);          // float E*16
    static constexpr size_t oNGeo = oGeo + al(sizeof(float) * E * 16);        // float E*3*16
    static constexpr size_t oU = oNGeo + al(sizeof(float) * E * 3 * 16);      // float4 E*Np
    static constexpr size_t oN = oU + al(sizeof(float4) * E * Np);            // float4 E*3*Np
    static constexpr size_t oPo = oN + al(sizeof(float4) * E * 3 * Np);       // float E*NpP
    static constexpr size_t oPn = oPo + al(sizeof(float) * E * NpP);          // float E*3*NpP
    static constexpr size_t oRaw = oPn + al(sizeof(float) * E * 3 * NpP);     // double E*4*Np
    static constexpr size_t oK1 = oRaw + al(sizeof(double) * E * 4 * Np);     // double E*4*Np
    static constexpr size_t oF = oK1 + al(sizeof(double) * E * 4 * Np);       // float4 E*Np*2 (Fr, Fs)
    static constexpr size_t oFxy = oF + al(sizeof(float4) * E * Np * 2);      // float4 E*Np*2 (Fx, Fy)
    static constexpr size_t oNorm = oFxy + al(sizeof(float4) * E * Np * 2);   // float E*NF
    static constexpr size_t oDH = oNorm + al(sizeof(float) * E * NF);         // float4 E*NF
    static constexpr size_t oW = oDH + al(sizeof(float4) * E * NF);           // theta: float2 Np*Np (Wr, Ws)
    static constexpr size_t oTH = oW + (TH ? al(sizeof(float2) * Np * Np) : 0);  // theta: float4 E*NF*2
    static constexpr size_t bytes = oTH + (TH ? al(sizeof(float4) * E * NF * 2) : 0);
};

__device__ __forceinline__ void f4_to(const float4 &a, float o[4]) { o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; }
__device__ __forceinline__ float4 to_f4(const float o[4]) { return make_float4(o[0], o[1], o[2], o[3]); }

template <int P, bool TH, bool BATCH = false, bool FUSE = false>
__global__ void __launch_bounds__(Shape<P>::NT, TH ? 2 : 3)
stage_mixed_kernel(StageParams sp, Phys<float> ph)
{
    using S = Shape<P>;
    using L = MixedLayout<P, TH>;
    constexpr int Np = S::Np, Nfp = S::Nfp, NF = S::NF, E = S::E, NT = S::NT;
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
    float2 *sW = reinterpret_cast<float2 *>(smem_raw + L::oW);
    float4 *sTH = reinterpret_cast<float4 *>(smem_raw + L::oTH);
    const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(smem_raw));

    const int tid = threadIdx.x;
    {
        const float *ops = static_cast<const float *>(sp.ops);   // Dr | Ds | LIFT
        for (int i = tid; i < Np * Np; i += NT) sD[i] = make_float2(ops[i], ops[Np * Np + i]);
        for (int i = tid; i < Np * NF; i += NT) sL[i] = ops[2 * Np * Np + i];
        for (int i = tid; i < NF; i += NT) sFm[i] = sp.fmask[i];
        if constexpr (TH) {
            const float *w = ops + 2 * Np * Np + Np * NF;                 // Wr | Ws
            for (int i = tid; i < Np * Np; i += NT) sW[i] = make_float2(w[i], w[Np * Np + i]);
        }
    }
    const float *geo = static_cast<const float *>(sp.geo);
    const long long K = sp.K;
    const long long ntiles = BATCH ? sp.ntiles : (K + E - 1) / E;
    const double gm1d = sp.gm1;
    const float cinv_fac = 0.5f * float(P + 1) * float(P + 2);
    const float sig_fac = static_cast<float>(sp.sig_fac);
    const float theta = static_cast<float>(sp.theta);
    float dtr = static_cast<float>(sp.dt);
    const bool update = sp.mode == STAGE_UPDATE;
    bool need_k1 = update && !sp.first_stage;
    __syncthreads();
    pdl_wait_then_release();

    const int ve = tid / Np, vi = tid - (tid / Np) * Np;
    const int fe = tid / NF, fm = tid - (tid / NF) * NF;
    const int ff = fm / Nfp, fi = fm - (fm / Nfp) * Nfp;

    for (int stg = 0; stg < (FUSE ? 5 : 1); ++stg) {
    if constexpr (FUSE) {
        if (stg > 0 && !grid_sync(sp.bar, sp.bar_err, gridDim.x, sp.bar_limit)) return;
        fused_stage(sp, stg);
        need_k1 = update && stg > 0;
    }
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        long long k0 = tile * E;
        int ne = static_cast<int>((K - k0) < E ? (K - k0) : E);
        if constexpr (BATCH) {
            // tiles never straddle two cases: take the case's viscosity, mesh
            // velocity (transverse, from its Newmark step) and time step
            const int4 td = sp.tiles[tile];
            k0 = td.x;
            ne = td.y;
            const BatchCase &cs = sp.cases[td.z];
            ph.mu = cvt_d2f(cs.mu);           // integer conversions: no FP64-pipe work per tile
            ph.vw2 = cvt_d2f(cs.vb);
            dtr = cvt_d2f(cs.dt);
        }
        // ---- P1a: connectivity of the tile (needed to address the neighbours)
        if (tid < ne) sConn[tid] = sp.conn[k0 + tid];
        __syncthreads();
        // ---- P1b: asynchronous 16-byte copies of everything the tile reads
        {
            // own FP32 records, own pressures, own FP64 state, K1, own geometry
            const char *gU = reinterpret_cast<const char *>(sp.Sin + k0 * Np);
            for (int c = tid; c < ne * Np; c += NT) cp_async16(sbase + L::oU + 16u * c, gU + 16 * c);
            const char *gP = reinterpret_cast<const char *>(sp.Pin + k0 * NpP);
            for (int c = tid; c < ne * (NpP / 4); c += NT) cp_async16(sbase + L::oPo + 16u * c, gP + 16 * c);
            const char *gR = reinterpret_cast<const char *>(sp.K0in + k0 * 4 * Np);
            for (int c = tid; c < ne * 2 * Np; c += NT) cp_async16(sbase + L::oRaw + 16u * c, gR + 16 * c);
            if (need_k1) {
                const char *gK = reinterpret_cast<const char *>(sp.K1 + k0 * 4 * Np);
                for (int c = tid; c < ne * 2 * Np; c += NT) cp_async16(sbase + L::oK1 + 16u * c, gK + 16 * c);
            }
            const char *gG = reinterpret_cast<const char *>(geo + k0 * 16);
            for (int c = tid; c < ne * 4; c += NT) cp_async16(sbase + L::oGeo + 16u * c, gG + 16 * c);
            // neighbour FP32 records, pressures and geometry records
            for (int c = tid; c < ne * 3 * Np; c += NT) {
                const int seg = c / Np, j = c - (c / Np) * Np;
                const int4 cn = sConn[seg / 3];
                const int f = seg - 3 * (seg / 3);
                const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
                cp_async16(sbase + L::oN + 16u * c, sp.Sin + nb * Np + j);
            }
            for (int c = tid; c < ne * 3 * (NpP / 4); c += NT) {
                const int seg = c / (NpP / 4), q = c - (c / (NpP / 4)) * (NpP / 4);
                const int4 cn = sConn[seg / 3];
                const int f = seg - 3 * (seg / 3);
                const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
                cp_async16(sbase + L::oPn + 16u * c, sp.Pin + nb * NpP + 4 * q);
            }
            for (int c = tid; c < ne * 3 * 4; c += NT) {
                const int seg = c >> 2, q = c & 3;
                const int4 cn = sConn[seg / 3];
                const int f = seg - 3 * (seg / 3);
                const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
                cp_async16(sbase + L::oNGeo + 16u * c, geo + nb * 16 + 4 * q);
            }
            asm volatile("cp.async.commit_group;\n" ::);
            asm volatile("cp.async.wait_group 0;\n" ::);
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
            const float p = sPo[ve * NpP + vi];
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
            float w[4];
            if (btype == BCT_INTERIOR) f4_to(sN[(fe * 3 + ff) * Np + vp], w);
            const float pw = (btype == BCT_WALL) ? sPo[fe * NpP + vm] : 0.f;
            sNorm[fe * NF + fm] = trace_norms_max(u, 1.0f / u[0], pw, btype, w, n1, n2, ph);
        }
        __syncthreads();

        // ---- P3: divergence (volume) and face fluxes (face nodes)
        float Dv[4] = {0, 0, 0, 0};       // sum_j Dr_ij Fr_j + Ds_ij Fs_j
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
            const float *ng = sNGeo + (fe * 3 + ff) * 16;     // neighbour's geometry record
            if (btype == BCT_INTERIOR) {
                const int f2 = (sConn[fe].w >> (2 * ff)) & 3;
                cinv = fmaxf(cinv, cinv_fac * ng[G_FS + f2]);
            }
            const float sigma = sig_fac * gbar * cinv;
            float up[4], dH[4], Ftp[4];
            f4_to(sU[fe * Np + vm], up);
            float jmp[4], gs[4], wth = 1.0f;     // theta term: jump, state of G, weight
            {
                const float ir = 1.0f / up[0];
                gs[0] = up[0]; gs[1] = up[1] * ir; gs[2] = up[2] * ir; gs[3] = up[3] * ir;
            }
            const float pp = sPo[fe * NpP + vm];
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
                float um[4], gxm[4], gym[4];
                f4_to(w[vp], um);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    gxm[c] = ng[G_RX] * wr[c] + ng[G_SX] * ws[c];
                    gym[c] = ng[G_RY] * wr[c] + ng[G_SY] * ws[c];
                }
                const float pm = sPn[(fe * 3 + ff) * NpP + vp];
                if constexpr (TH) {
                    const int4 cn = sConn[fe];
                    const long long nb = (ff == 0) ? cn.x : (ff == 1 ? cn.y : cn.z);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        jmp[c] = cvt_d2f(sRaw[(fe * 4 + c) * Np + vm] - sp.K0in[(nb * 4 + c) * Np + vp]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) jmp[c] = up[c] - um[c];
                }
                float Fnm[4], vxm[4], vym[4], D[4];
                flux_n(um, pm, n1, n2, ph, Fnm);
                visc_flux(um, gxm, gym, ph, vxm, vym);
                roe_dissipation(up, pp, um, pm, n1, n2, ph, D);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float Ftm = Fnm[c] - (vxm[c] * n1 + vym[c] * n2);
                    dH[c] = 0.5f * (Ftp[c] - Ftm) - 0.5f * D[c] - sigma * jmp[c];
                }
                wth = 0.5f;
            } else if (btype == BCT_FARFIELD) {
                const float ub[4] = {ph.Uinf[0], ph.Uinf[1], ph.Uinf[2], ph.Uinf[3]};
                float Fnp[4], Fnb[4], D[4];
                flux_n(up, pp, n1, n2, ph, Fnp);
                flux_n(ub, ph.pinf, n1, n2, ph, Fnb);
                roe_dissipation(up, pp, ub, ph.pinf, n1, n2, ph, D);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    jmp[c] = TH ? cvt_d2f(sRaw[(fe * 4 + c) * Np + vm] - sp.uinf[c]) : up[c] - ub[c];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dH[c] = 0.5f * (Fnp[c] - Fnb[c]) - 0.5f * D[c] - sigma * jmp[c];
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
                for (int c = 0; c < 4; ++c) jmp[c] = up[c] - ub[c];
                // E+ - E^b = (|m+|^2 / rho - rho |v_w|^2) / 2 without the cancellation
                if constexpr (TH) jmp[3] = 0.5f * (up[1] * up[1] + up[2] * up[2]) / rb - kw;
#pragma unroll
                for (int c = 0; c < 4; ++c) dH[c] = Ftp[c] - (Fnb[c] - vnb[c] + sigma * jmp[c]);
                gs[0] = rb; gs[1] = ph.vw1; gs[2] = ph.vw2; gs[3] = ub[3] / rb;
            }
            sDH[fe * NF + fm] = make_float4(fsc * dH[0], fsc * dH[1], fsc * dH[2], fsc * dH[3]);
            if constexpr (TH) {
                float tx[4], ty[4];
                theta_vec(gs[0], gs[1], gs[2], gs[3], jmp, n1, n2, ph, tx, ty);
                const float sc = theta * wth * fsc;
                sTH[(fe * NF + fm) * 2] = make_float4(sc * tx[0], sc * tx[1], sc * tx[2], sc * tx[3]);
                sTH[(fe * NF + fm) * 2 + 1] = make_float4(sc * ty[0], sc * ty[1], sc * ty[2], sc * ty[3]);
            }
        }
        __syncthreads();

        // ---- P4: lift, the stage update and the FP32 copy of the new state
        float R[4] = {-Dv[0], -Dv[1], -Dv[2], -Dv[3]};
        if (vol) {
            const float4 *dh = sDH + ve * NF;
#pragma unroll
            for (int m = 0; m < NF; ++m) {
                const float4 h = dh[m];
                const float l = sL[vi * NF + m];
                R[0] = fmaf(l, h.x, R[0]); R[1] = fmaf(l, h.y, R[1]); R[2] = fmaf(l, h.z, R[2]); R[3] = fmaf(l, h.w, R[3]);
            }
        }
        if constexpr (TH) {
            // lift the theta vectors, map them to (r, s), park them in the flux slots
            if (vol) {
                const float4 *th = sTH + ve * NF * 2;
                float Lx[4] = {0, 0, 0, 0}, Ly[4] = {0, 0, 0, 0};
#pragma unroll
                for (int m = 0; m < NF; ++m) {
                    const float l = sL[vi * NF + m];
                    const float4 a = th[2 * m], b = th[2 * m + 1];
                    Lx[0] = fmaf(l, a.x, Lx[0]); Lx[1] = fmaf(l, a.y, Lx[1]); Lx[2] = fmaf(l, a.z, Lx[2]); Lx[3] = fmaf(l, a.w, Lx[3]);
                    Ly[0] = fmaf(l, b.x, Ly[0]); Ly[1] = fmaf(l, b.y, Ly[1]); Ly[2] = fmaf(l, b.z, Ly[2]); Ly[3] = fmaf(l, b.w, Ly[3]);
                }
                const float *g = sGeo + ve * 16;
                float ar[4], as[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ar[c] = g[G_RX] * Lx[c] + g[G_RY] * Ly[c];
                    as[c] = g[G_SX] * Lx[c] + g[G_SY] * Ly[c];
                }
                sF[(ve * Np + vi) * 2] = to_f4(ar);
                sF[(ve * Np + vi) * 2 + 1] = to_f4(as);
            }
            __syncthreads();
            if (vol) {
                const float4 *fe4 = sF + ve * Np * 2;
#pragma unroll
                for (int j = 0; j < Np; ++j) {
                    const float4 a = fe4[2 * j], b = fe4[2 * j + 1];
                    const float2 w = sW[vi * Np + j];
                    R[0] = fmaf(w.x, a.x, fmaf(w.y, b.x, R[0]));
                    R[1] = fmaf(w.x, a.y, fmaf(w.y, b.y, R[1]));
                    R[2] = fmaf(w.x, a.z, fmaf(w.y, b.z, R[2]));
                    R[3] = fmaf(w.x, a.w, fmaf(w.y, b.w, R[3]));
                }
            }
        }
        if (vol) {
            const long long base = (k0 + ve) * 4 * Np + vi;
            if (sp.src) {
#pragma unroll
                for (int c = 0; c < 4; ++c) R[c] += cvt_d2f(sp.src[base + c * Np]);
            }
            if (!update) {
#pragma unroll
                for (int c = 0; c < 4; ++c) sp.Rout[base + c * Np] = cvt_f2d(R[c]);
            } else {
                double knew[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double inc = cvt_f2d(dtr * R[c]);
                    const double k1 = sp.first_stage ? inc : fma(sp.A, sK1[(ve * 4 + c) * Np + vi], inc);
                    sp.K1[base + c * Np] = k1;
                    knew[c] = fma(sp.B, k1, sRaw[(ve * 4 + c) * Np + vi]);
                    sp.K0out[base + c * Np] = knew[c];
                }
                // FP32 copy of the new state and its pressure, recovered in FP64
                const float un[4] = {cvt_d2f_trunc(knew[0]), cvt_d2f_trunc(knew[1]),
                                     cvt_d2f_trunc(knew[2]), cvt_d2f_trunc(knew[3])};
                sp.Sout[(k0 + ve) * Np + vi] = to_f4(un);
                sp.Pout[(k0 + ve) * NpP + vi] = pressure<float>(un, knew[3], gm1d);
            }
        }
    }
    }  // stages
}

// Lambda_K of Eq. rayleigh_bound in FP32 from the FP32 state copy and the
// FP64-recovered pressures, one block per tile (same node / face-node thread
// map as the stage kernel).  Same readings as the FP64 time-step kernel:
// C_inv,2 = p^4 / rho_K^2 with rho_K = 2|K| / perimeter, G_K the largest
// diffusivity max(4/3, gamma/Pr) mu / rho over the face-node traces of both
// sides, sigma_K the largest penalty over the faces of K, C_inv,K the largest
// over its faces, beta_K the largest |b_ns|_2 over its nodes, beta'_K = 0.  Batch: the tile table gives
// the elements and the case (mu, v_b); otherwise tiles are E consecutive
// elements and ph holds mu and v_w.
template <int P>
__device__ __forceinline__ void dt_lambda_mixed_tile(const float4 *S, const float *Pr, const float *geo,
                                                     const int4 *conn, const int *fmask, const int4 *tiles,
                                                     const BatchCase *cases, long long K, Phys<float> ph,
                                                     float sig_fac, double *lam, long long blk)
{
    using Sh = Shape<P>;
    constexpr int Np = Sh::Np, Nfp = Sh::Nfp, NF = Sh::NF, E = Sh::E, NT = Sh::NT;
    constexpr int NpP = (Np + 3) & ~3;
    __shared__ float sNorm[E * NF];
    __shared__ float sRmin[E * NF];
    __shared__ float sBeta[E * Np];
    __shared__ int sFm[NF];
    const int tid = threadIdx.x;
    for (int i = tid; i < NF; i += NT) sFm[i] = fmask[i];
    long long k0 = blk * E;
    int ne = static_cast<int>((K - k0) < E ? (K - k0) : E);
    if (tiles) {
        const int4 td = tiles[blk];
        k0 = td.x;
        ne = td.y;
        ph.mu = static_cast<float>(cases[td.z].mu);
        ph.vw2 = static_cast<float>(cases[td.z].vb);
    }
    __syncthreads();
    const int fe = tid / NF, fm = tid - (tid / NF) * NF;
    if (fe < ne) {
        const long long k = k0 + fe;
        const int ff = fm / Nfp, fi = fm - ff * Nfp;
        const int4 cn = conn[k];
        const int f2 = (cn.w >> (2 * ff)) & 3, bt = (cn.w >> (8 + 2 * ff)) & 3;
        const int vm = sFm[ff * Nfp + fi], vp = sFm[f2 * Nfp + (Nfp - 1 - fi)];
        const float *g = geo + k * 16;
        const float n1 = g[G_NX + ff], n2 = g[G_NY + ff];
        const float4 u = S[k * Np + vm];
        const float uu[4] = {u.x, u.y, u.z, u.w};
        float w[4], rmin = u.x;
        if (bt == BCT_INTERIOR) {
            const long long nb = (ff == 0) ? cn.x : (ff == 1 ? cn.y : cn.z);
            f4_to(S[nb * Np + vp], w);
            rmin = fminf(rmin, w[0]);
        } else if (bt == BCT_FARFIELD) {
            rmin = fminf(rmin, ph.Uinf[0]);
        }
        const float pw = (bt == BCT_WALL) ? Pr[k * NpP + vm] : 0.f;
        sNorm[fe * NF + fm] = trace_norms_max(uu, 1.0f / u.x, pw, bt, w, n1, n2, ph);
        sRmin[fe * NF + fm] = rmin;
    }
    const int ve = tid / Np, vi = tid - (tid / Np) * Np;
    if (ve < ne) {
        const long long k = k0 + ve;
        const float4 u = S[k * Np + vi];
        const float ir = 1.0f / u.x;
        const float c = sqrtf(ph.gamma * Pr[k * NpP + vi] * ir);
        const float b1 = fabsf(u.y * ir - ph.vw1) + c, b2 = fabsf(u.z * ir - ph.vw2) + c;
        sBeta[ve * Np + vi] = sqrtf(b1 * b1 + b2 * b2);
    }
    __syncthreads();
    if (tid < ne) {
        const long long k = k0 + tid;
        const float *g = geo + k * 16;
        const int4 cn = conn[k];
        const float pp = float((P + 1) * (P + 2));
        float GK = 0.f, sigK = 0.f, ciK = 0.f, perim = 0.f, beta = 0.f;
        const float gdiff = fmaxf(4.0f / 3.0f, ph.gPr) * ph.mu;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            float gbar = 0.f, rmin = INFINITY;
            for (int i = 0; i < Nfp; ++i) {
                gbar = fmaxf(gbar, sNorm[tid * NF + f * Nfp + i]);
                rmin = fminf(rmin, sRmin[tid * NF + f * Nfp + i]);
            }
            const float fs = g[G_FS + f];
            const float ci = 0.5f * pp * fs;
            float cmax = ci;
            if (((cn.w >> (8 + 2 * f)) & 3) == BCT_INTERIOR) {
                const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
                const int f2 = (cn.w >> (2 * f)) & 3;
                cmax = fmaxf(ci, 0.5f * pp * geo[nb * 16 + G_FS + f2]);
            }
            GK = fmaxf(GK, gdiff / rmin);
            sigK = fmaxf(sigK, sig_fac * gbar * cmax);
            ciK = fmaxf(ciK, ci);
            perim += 2.0f * fs * g[G_J];
        }
        for (int i = 0; i < Np; ++i) beta = fmaxf(beta, sBeta[tid * Np + i]);
        const float rhoK = 2.0f * (2.0f * g[G_J]) / perim;
        const float p4 = float(P) * float(P) * float(P) * float(P);
        const float cinv2 = p4 / (rhoK * rhoK);
        lam[k] = cvt_f2d(1.5f * cinv2 * GK + 3.0f * ciK * (3.0f * sigK + beta));
    }
}

template <int P>
__global__ void __launch_bounds__(Shape<P>::NT)
dt_lambda_mixed_kernel(const float4 *S, const float *Pr, const float *geo, const int4 *conn, const int *fmask,
                       const int4 *tiles, const BatchCase *cases, long long K, Phys<float> ph, float sig_fac,
                       double *lam)
{
    dt_lambda_mixed_tile<P>(S, Pr, geo, conn, fmask, tiles, cases, K, ph, sig_fac, lam, blockIdx.x);
}

// The time-step bound of every degree group of a batch in one launch: block
// b works on tile b - first_block of the group whose block range holds b.
template <int... Ps>
__global__ void __launch_bounds__(256) dt_lambda_mixed_multi_kernel(DtGroups dgs, const BatchCase *cases,
                                                                   Phys<float> ph, float sig_fac)
{
    int gi = 0;
    while (gi + 1 < dgs.n && static_cast<long long>(blockIdx.x) >= dgs.g[gi + 1].first_block) ++gi;
    const DtGroup &G = dgs.g[gi];
    const long long blk = blockIdx.x - G.first_block;
    // exactly one case runs: the group's degree
    ((G.p == Ps ? dt_lambda_mixed_tile<Ps>(G.S, G.Pr, G.geo, G.conn, G.fmask, G.tiles, cases, G.K, ph, sig_fac,
                                           G.lam, blk)
                : void()), ...);
}

// FP32 copy and FP64-recovered pressure of a state (used when the state is
// set from outside the stage kernel).
template <int P>
__global__ void make_shadow_kernel(const double *K0, long long K, double gm1, float4 *S, float *Pr)
{
    constexpr int Np = (P + 1) * (P + 2) / 2, NpP = (Np + 3) & ~3;
    const long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (n >= K * Np) return;
    const long long k = n / Np;
    const int i = static_cast<int>(n - k * Np);
    double d[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = K0[(k * 4 + c) * Np + i];
    const float u[4] = {cvt_d2f_trunc(d[0]), cvt_d2f_trunc(d[1]), cvt_d2f_trunc(d[2]), cvt_d2f_trunc(d[3])};
    S[k * Np + i] = to_f4(u);
    Pr[k * NpP + i] = pressure<float>(u, d[3], gm1);
}

}  // namespace dg
