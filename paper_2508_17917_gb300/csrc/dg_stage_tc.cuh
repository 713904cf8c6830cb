// dg_stage_tc.cuh -- mixed-precision stage kernel with the operator products
// on the tensor cores.
//
// Same method as dg_stage_mixed.cuh: the strong-form residual of Eq. dg_on_K
// (IIP, and with the template flag TH the SIP / NIPG theta terms) and one
// stage of Algorithm 1, FP32 arithmetic with FP64 state, pressure recovery
// and registers.  What changes is how the work is laid out:
//
// * Every warp owns a tile of WE = 2 elements from load to store and
//   synchronises with __syncwarp only, so the warps of a block run
//   independently (no block barrier in the loop).  It gathers its elements'
//   neighbours with 16-byte cp.async by index; its own contiguous records
//   (FP32 state, pressure, geometry, FP64 registers) arrive by bulk copies
//   of the tensor memory accelerator on two per-warp mbarriers from p = 5 on
//   (cp.async below: measured).  The block's operator fragments (Dr, Ds,
//   LIFT) arrive by one bulk copy on an mbarrier in the prologue.  Every
//   mbarrier wait is bounded; one that gives up raises the barrier error
//   flag and the warp skips its remaining tiles.
// * The contractions -- broken gradient [Dr; Ds] U, divergence Dr Fr + Ds Fs
//   and lift LIFT (Fscale dH), all batched over the tile's elements as
//   (16 x 16)(16 x 8) products -- run as mma.sync m16n8k8 TF32 with FP32
//   accumulation.  Each FP32 operand x is split into x_hi (x with the low 13
//   mantissa bits rounded off) and x_lo = x - x_hi, and the product takes
//   A_hi B_hi + A_hi B_lo + A_lo B_hi, about 2^-21 relative to sum |A||B|.
//   The state and flux operands are taken relative to the element's first
//   node (perturbation form): Dr 1 = Ds 1 = 0 makes this exact in exact
//   arithmetic, and it keeps large means (the energy at low Mach) out of the
//   split.
// * The face-node gradients of the neighbours (Eq. ip_flux needs
//   {{G grad U}} on both sides) are the rows of [Dr; Ds] at the shared node
//   applied to the neighbour's staged state (FP32 FMAs: 5 of 16 rows are
//   needed, which costs fewer instructions than an MMA of all 16); a
//   boundary face names its own element, so a wall face gets the own
//   gradient the same way.
// * Theta variant: the face pass also forms the jumps in FP64 and the theta
//   vectors; the update pass lifts them (MMA), maps them to (r, s) per node
//   and applies the weak-form derivatives Wr, Ws (MMA, no reference node:
//   Wr 1 != 0).
//
// MMA fragment layout (m16n8k8, row.col, TF32; lane = 4 g + t):
//   A (16 x 8): a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4]
//   B (8 x 8):  b0 = B[t][g], b1 = B[t+4][g]
//   C (16 x 8): c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
// Rows are nodes, columns (element of the pair, field): column n = 4 e + c.
// After a shuffle with lane ^ 1 every lane holds all four fields of one node:
// node g + 8 (lane & 1) of element (lane >> 1) & 1 of the pair.  For p = 5
// and 6 (Np = 21, 28) the node rows span two 16-row tiles (MT = 2), so a lane
// holds one node per tile, and the contractions take up to four k-steps.
#pragma once
#include "dg_stage_mixed.cuh"
#include "pair2.cuh"

namespace dg {

template <int P>
struct ShapeTC {
    static constexpr int Np = (P + 1) * (P + 2) / 2, Nfp = P + 1, NF = 3 * Nfp;
    static_assert(Np <= 32 && NF <= 32, "at most two 16-row MMA tiles per operator: p <= 6");
    static constexpr int MT = (Np + 15) / 16;     // 16-row tiles of nodes
    static constexpr int KD = (Np + 7) / 8;       // k-steps over the nodes (Dr, Ds)
    static constexpr int KL = (NF + 7) / 8;       // k-steps over the face nodes (LIFT)
    static constexpr int WE = 2;                  // elements per warp tile
    static constexpr int EPP = (32 / NF < WE) ? 32 / NF : WE;   // elements per face-node pass
    static constexpr int NW = 4;                  // warps per block
    static constexpr int NT = 32 * NW;
    static constexpr int NpP = (Np + 3) & ~3;     // padded pressure row
    // float4 records per staged element / neighbour slot, and floats per
    // element of the flux and dH tables: sizes chosen so that the lanes of
    // a B-fragment load, and the face-node reads of the six slots, fall in
    // distinct shared-memory banks
    static constexpr int US = Np + ((12 - Np % 8) % 8);          // >= Np, = 4 mod 8
    static constexpr int UN = Np + ((13 - Np % 8) % 8);          // >= Np, = 5 mod 8
    static constexpr int FS = 128 * MT + 4;       // = 4 mod 32
    static constexpr int HS = 32 * KL + 16;       // = 16 mod 32
    // row stride (float2) of the (Dr, Ds) rows the face pass reads, one row
    // per lane: odd, so 16 consecutive rows start in distinct bank pairs
    static constexpr int DS = Np | 1;
    // operator fragments: Dr and Ds [MT][KD], LIFT [MT][KL], then (theta
    // variant) Wr and Ws [MT][KD], each [hi, lo][lane]
    static constexpr int NENT = 2 * MT * KD + MT * KL;           // entries of the IIP kernel
    static constexpr int NENT_ALL = NENT + 2 * MT * KD;          // with Wr, Ws
    static constexpr int NFRAG_ALL = NENT_ALL * 64;              // float4 in the table
    static constexpr bool FRAG_SMEM = MT == 1;    // staged in shared memory (else read through L1)
    // the warp's own element records by bulk copies (else cp.async per
    // lane): measured 3.5 % faster per step at p = 6 and 0.3 % at p = 5, 0.8 %
    // slower at p = 4 on 128^2 quads (neutral on 512^2), so from p = 5 on
    static constexpr bool TILE_BULK = MT > 1;
};

// operator table: the MMA fragments (ShapeTC<P>::NFRAG_ALL float4), then
// (Dr, Ds) in FP32 as float2 [Np][Np] for the face-node gradients of the
// neighbours
template <int P, bool TH = false>
struct TcLayout {
    using S = ShapeTC<P>;
    static constexpr int NFRAG = (TH ? S::NENT_ALL : S::NENT) * 64;    // fragments the kernel reads
    static constexpr int Np = S::Np, NF = S::NF, WE = S::WE, NpP = S::NpP;
    static constexpr size_t al(size_t b) { return (b + 15) & ~size_t(15); }
    // block header
    static constexpr size_t hFrag = 0;                                      // float4 [NFRAG] if FRAG_SMEM
    static constexpr size_t hFm = hFrag + (S::FRAG_SMEM ? sizeof(float4) * NFRAG : 0);      // int [NF]
    static constexpr size_t hD = hFm + al(sizeof(int) * NF);                // float2 [Np][DS]: (Dr, Ds)
    static constexpr size_t hBar = hD + al(sizeof(float2) * Np * S::DS);   // mbarrier of the operator copy
    static constexpr size_t header = hBar + 16;
    // one region per warp
    static constexpr size_t oConn = 0;                                      // int4 [WE]
    static constexpr size_t oGeo = oConn + al(16 * WE);                     // float [WE][16]
    static constexpr size_t oNGeo = oGeo + al(64 * WE);                     // float [3 WE][16]
    static constexpr size_t oU = oNGeo + al(64 * 3 * WE);                   // float4 [WE][US]
    static constexpr size_t oN = oU + al(16 * WE * S::US);                  // float4 [3 WE][UN]
    static constexpr size_t oPo = oN + al(16 * 3 * WE * S::UN);             // float [WE][NpP]
    static constexpr size_t oPn = oPo + al(4 * WE * NpP);                   // float [3 WE][NpP]
    static constexpr size_t oRaw = oPn + al(4 * 3 * WE * NpP);              // double [WE][4][Np]
    static constexpr size_t oK1 = oRaw + al(8 * WE * 4 * Np);               // double [WE][4][Np]
    static constexpr size_t oF = oK1 + al(8 * WE * 4 * Np);                 // float [WE][FS]: node j: Fr[4], Fs[4]
    static constexpr size_t oDH = oF + al(4 * WE * S::FS);                  // float [WE][HS]: slot r: Fscale dH[4]
    static constexpr size_t oTH = oDH + al(4 * WE * S::HS);                 // theta: float [2][WE][HS]: x, y vectors
    static constexpr size_t oBar = oTH + (TH ? al(4 * 2 * WE * S::HS) : 0);  // mbarriers: own tile, FP64 registers
    static constexpr size_t warp = oBar + 16;
    static constexpr size_t bytes = header + S::NW * warp;
};

// Bulk copies (the tensor memory accelerator's 1-D form) into shared memory,
// completing on an mbarrier: the warp's own tile and the operator table.
__device__ __forceinline__ void mbar_init1(unsigned bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// 16-byte aligned addresses, a multiple of 16 bytes
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// bounded wait for phase `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned limit)
{
    for (unsigned it = 0;; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it >= limit) return false;
        __nanosleep(100);
    }
}

__device__ __forceinline__ void mma_tf32(float c[4], const float4 &a, float b0, float b1)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)), "r"(__float_as_uint(a.w)),
          "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}

// x = hi + lo: hi is x rounded to TF32 (10 explicit mantissa bits, so
// |x - hi| <= 2^-11 |x|) and lo = x - hi, exact in FP32; the tensor core
// reads lo as TF32, dropping at most 2^-11 |lo| <= 2^-22 |x|
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo)
{
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    lo = x - hi;
}

// One k-step of C += A B with split operands, as three independent products:
// the large one into ch, the two corrections into cl (summed at the end), so
// consecutive MMAs of a contraction do not wait on each other
__device__ __forceinline__ void mma3(float ch[4], float cl[4], const float4 &ahi, const float4 &alo, float b0,
                                     float b1)
{
    float h0, l0, h1, l1;
    tf32_split(b0, h0, l0);
    tf32_split(b1, h1, l1);
    mma_tf32(ch, ahi, h0, h1);
    mma_tf32(cl, alo, h0, h1);
    mma_tf32(cl, ahi, l0, l1);
}

// C fragment -> the four fields of this lane's node (see the header comment)
__device__ __forceinline__ void frag_to_node(const float c[4], float v[4], int lane)
{
    const bool odd = lane & 1;
    const float x = odd ? c[0] : c[2], y = odd ? c[1] : c[3];
    const float rx = __shfl_xor_sync(0xffffffffu, x, 1), ry = __shfl_xor_sync(0xffffffffu, y, 1);
    v[0] = odd ? rx : c[0];
    v[1] = odd ? ry : c[1];
    v[2] = odd ? c[2] : rx;
    v[3] = odd ? c[3] : ry;
}

// Six blocks per SM (80 registers) for the stage-wise IIP kernel up to p = 4;
// four (128 registers) for the fused, theta and two-tile (p = 5, 6) kernels.
template <int P, bool BATCH = false, bool FUSE = false, bool TH = false>
__global__ void __launch_bounds__(128, (FUSE || TH || ShapeTC<P>::MT > 1) ? 4 : 6)
stage_tc_kernel(StageParams sp, Phys<float> ph)
{
    using S = ShapeTC<P>;
    using L = TcLayout<P, TH>;
    constexpr int Np = S::Np, Nfp = S::Nfp, NF = S::NF, WE = S::WE, NpP = S::NpP;
    constexpr int US = S::US, UN = S::UN, FS = S::FS, HS = S::HS;
    constexpr int MT = S::MT, KD = S::KD, KL = S::KL, EPP = S::EPP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const float4 *gFrag = static_cast<const float4 *>(sp.ops);
    const float4 *sFrag = reinterpret_cast<const float4 *>(smem_raw + L::hFrag);
    int *sFm = reinterpret_cast<int *>(smem_raw + L::hFm);
    const float2 *sD = reinterpret_cast<const float2 *>(smem_raw + L::hD);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(smem_raw));
    const unsigned barOps = sbase + unsigned(L::hBar);
    {
        // the mbarriers; the operator fragments (built on the host in
        // fragment order) by one bulk copy; (Dr, Ds) rows and the face node
        // table (strided rows) by the threads
        if (tid == 0) {
            mbar_init1(barOps);
            for (int w = 0; w < S::NW; ++w) {
                mbar_init1(sbase + unsigned(L::header + w * L::warp + L::oBar));
                mbar_init1(sbase + unsigned(L::header + w * L::warp + L::oBar + 8));
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if constexpr (S::FRAG_SMEM) {
                mbar_expect(barOps, unsigned(sizeof(float4) * L::NFRAG));
                bulk_g2s(sbase + unsigned(L::hFrag), gFrag, unsigned(sizeof(float4) * L::NFRAG), barOps);
            }
        }
        const float2 *dtab = reinterpret_cast<const float2 *>(gFrag + S::NFRAG_ALL);
        float2 *dD = reinterpret_cast<float2 *>(smem_raw + L::hD);
        for (int i = tid; i < Np * Np; i += S::NT) dD[(i / Np) * S::DS + i % Np] = dtab[i];
        for (int i = tid; i < NF; i += S::NT) sFm[i] = sp.fmask[i];
    }
    __syncthreads();
    // a copy wait that gives up marks the error flag; the warp (or, here,
    // the block) then skips its tiles but still meets every grid barrier
    bool failed = false;
    if constexpr (S::FRAG_SMEM) {
        failed = !__syncthreads_and(mbar_wait_bounded(barOps, 0u, sp.bar_limit));
        if (failed && tid == 0) {
            if (sp.bar_err) atomicExch(sp.bar_err, 1);
            mbar_wait_bounded(barOps, 0u, sp.bar_limit);      // the copy still lands in this block's memory
        }
    }
    pdl_wait_then_release();
    // fragment `h` (0 hi, 1 lo) of entry `ent` of the operator table
    auto frag = [&](int ent, int h) -> float4 {
        const int idx = (ent * 2 + h) * 32 + lane;
        if constexpr (S::FRAG_SMEM) return sFrag[idx];
        else return __ldg(gFrag + idx);
    };
    // entries: Dr [mt][ks], Ds [mt][ks], LIFT [mt][ks]
    auto ent_d = [&](int m, int mt, int ks) { return (m * MT + mt) * KD + ks; };
    auto ent_l = [&](int mt, int ks) { return 2 * MT * KD + mt * KL + ks; };
    auto ent_w = [&](int m, int mt, int ks) { return S::NENT + (m * MT + mt) * KD + ks; };   // Wr, Ws

    unsigned char *wb = smem_raw + L::header + wid * L::warp;
    const unsigned wsh = static_cast<unsigned>(__cvta_generic_to_shared(wb));
    const unsigned barA = wsh + unsigned(L::oBar), barB = barA + 8u;
    unsigned wit = 0;        // tiles this warp has started: the parity of its mbarriers' phases
    // a bounded copy wait gave up: raise the error flag, wait (bounded) for
    // the copies still landing in this warp's shared memory, skip the rest
    auto copy_wait_failed = [&](unsigned a, unsigned b, unsigned ph_) {
        failed = true;
        if (lane == 0) {
            if (sp.bar_err) atomicExch(sp.bar_err, 1);
            mbar_wait_bounded(a, ph_, sp.bar_limit);
            mbar_wait_bounded(b, ph_, sp.bar_limit);
        }
        __syncwarp();
    };
    int4 *sConn = reinterpret_cast<int4 *>(wb + L::oConn);
    const float *sGeo = reinterpret_cast<const float *>(wb + L::oGeo);
    const float *sNGeo = reinterpret_cast<const float *>(wb + L::oNGeo);
    const float4 *sU = reinterpret_cast<const float4 *>(wb + L::oU);
    const float4 *sN = reinterpret_cast<const float4 *>(wb + L::oN);
    const float *sPo = reinterpret_cast<const float *>(wb + L::oPo);
    const float *sPn = reinterpret_cast<const float *>(wb + L::oPn);
    const double *sRaw = reinterpret_cast<const double *>(wb + L::oRaw);
    const double *sK1 = reinterpret_cast<const double *>(wb + L::oK1);
    float *sF = reinterpret_cast<float *>(wb + L::oF);
    float *sDH = reinterpret_cast<float *>(wb + L::oDH);
    float *sTHx = reinterpret_cast<float *>(wb + L::oTH);        // theta variant only
    float *sTHy = sTHx + WE * HS;
    const float theta = static_cast<float>(sp.theta);

    const float *geo = static_cast<const float *>(sp.geo);
    const long long K = sp.K;
    const long long nwt = BATCH ? sp.ntiles : (K + WE - 1) / WE;
    const double gm1d = sp.gm1;
    const float cinv_fac = 0.5f * float(P + 1) * float(P + 2);
    const float sig_fac = static_cast<float>(sp.sig_fac);
    float dtr = static_cast<float>(sp.dt);
    const bool update = sp.mode == STAGE_UPDATE;
    bool need_k1 = update && !sp.first_stage;
    const int g = lane >> 2, t = lane & 3;
    const int jn = g + 8 * (lane & 1);       // node (within a 16-row tile) held after frag_to_node
    const int ep = (lane >> 1) & 1;          // element of the pair held after frag_to_node
    const int be = g >> 2, bc = g & 3;       // B column of this lane: element of the pair, field

    for (int stg = 0; stg < (FUSE ? 5 : 1); ++stg) {
    if constexpr (FUSE) {
        if (stg > 0 && !grid_sync(sp.bar, sp.bar_err, gridDim.x, sp.bar_limit)) return;
        fused_stage(sp, stg);
        need_k1 = update && stg > 0;
    }
    for (long long wt = static_cast<long long>(blockIdx.x) * S::NW + wid; wt < nwt;
         wt += static_cast<long long>(gridDim.x) * S::NW) {
        long long k0 = wt * WE;
        int ne = static_cast<int>((K - k0) < WE ? (K - k0) : WE);
        if constexpr (BATCH) {
            // warp tiles never straddle two cases: the case's viscosity, mesh
            // velocity and time step
            const int4 td = sp.tiles[wt];
            k0 = td.x;
            ne = td.y;
            const BatchCase &cs = sp.cases[td.z];
            ph.mu = cvt_d2f(cs.mu);           // integer conversions: no FP64-pipe work per tile
            ph.vw2 = cvt_d2f(cs.vb);
            dtr = cvt_d2f(cs.dt);
        }
        if (failed) continue;                    // a copy wait gave up: the flag is set
        if (lane < ne) sConn[lane] = sp.conn[k0 + lane];
        __syncwarp();
        // ---- the tile's own records, contiguous in memory -- A: FP32 state,
        // pressure and geometry; B: the FP64 registers, needed only by the
        // update.  TILE_BULK: bulk copies issued by lane 0 on the warp's two
        // mbarriers (one copy per element for the state: the staged rows are
        // padded); else 16-byte cp.async per lane in two commit groups.
        const unsigned par = wit & 1u;
        ++wit;
        if constexpr (S::TILE_BULK) {
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(barA, unsigned(ne) * (16u * Np + 4u * NpP + 64u));
                for (int e = 0; e < ne; ++e)
                    bulk_g2s(wsh + L::oU + 16u * (e * US), sp.Sin + (k0 + e) * Np, 16u * Np, barA);
                bulk_g2s(wsh + L::oPo, sp.Pin + k0 * NpP, 4u * NpP * ne, barA);
                bulk_g2s(wsh + L::oGeo, geo + k0 * 16, 64u * ne, barA);
                mbar_expect(barB, unsigned(ne) * 32u * Np * (need_k1 ? 2u : 1u));
                bulk_g2s(wsh + L::oRaw, sp.K0in + k0 * 4 * Np, 32u * Np * ne, barB);
                if (need_k1) bulk_g2s(wsh + L::oK1, sp.K1 + k0 * 4 * Np, 32u * Np * ne, barB);
            }
        } else {
            for (int c = lane; c < ne * Np; c += 32) {
                const int e = c / Np, j = c - (c / Np) * Np;
                cp_async16(wsh + L::oU + 16u * (e * US + j), sp.Sin + (k0 + e) * Np + j);
            }
            for (int c = lane; c < ne * (NpP / 4); c += 32)
                cp_async16(wsh + L::oPo + 16u * c, sp.Pin + k0 * NpP + 4 * c);
            for (int c = lane; c < ne * 4; c += 32) cp_async16(wsh + L::oGeo + 16u * c, geo + k0 * 16 + 4 * c);
        }
        // ---- the three face neighbours of every element (a boundary face
        // names its own element, so its slot holds the element itself):
        // gathers by index, 16-byte cp.async per lane
        {
            // LPS lanes per neighbour slot: one connectivity lookup per lane
            constexpr int LPS = 32 / (3 * WE);
            const int sl = lane / LPS, part = lane - (lane / LPS) * LPS;
            if (sl < 3 * ne) {
                const int4 cn = sConn[sl / 3];
                const int f = sl - 3 * (sl / 3);
                const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
                for (int j = part; j < Np; j += LPS)
                    cp_async16(wsh + L::oN + 16u * (sl * UN + j), sp.Sin + nb * Np + j);
                for (int qq = part; qq < NpP / 4; qq += LPS)
                    cp_async16(wsh + L::oPn + 16u * (sl * (NpP / 4) + qq), sp.Pin + nb * NpP + 4 * qq);
                for (int qq = part; qq < 4; qq += LPS)
                    cp_async16(wsh + L::oNGeo + 16u * (sl * 4 + qq), geo + nb * 16 + 4 * qq);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
        if constexpr (S::TILE_BULK) {
            asm volatile("cp.async.wait_group 0;\n" ::);
            bool ok = mbar_wait_bounded(barA, par, sp.bar_limit);
            if constexpr (TH) ok = ok && mbar_wait_bounded(barB, par, sp.bar_limit);   // FP64 jumps in the face pass
            if (!__all_sync(0xffffffffu, ok)) {
                copy_wait_failed(barA, barB, par);
                continue;
            }
        } else {
            for (int c = lane; c < ne * 2 * Np; c += 32)
                cp_async16(wsh + L::oRaw + 16u * c, sp.K0in + k0 * 4 * Np + 2 * c);
            if (need_k1)
                for (int c = lane; c < ne * 2 * Np; c += 32)
                    cp_async16(wsh + L::oK1 + 16u * c, sp.K1 + k0 * 4 * Np + 2 * c);
            asm volatile("cp.async.commit_group;\n" ::);
            if constexpr (TH)
                asm volatile("cp.async.wait_group 0;\n" ::);   // the face pass forms FP64 jumps
            else
                asm volatile("cp.async.wait_group 1;\n" ::);
        }
        __syncwarp();

        // ---- V: broken gradient (MMA) and total flux of every volume node
#pragma unroll
        for (int nt = 0; nt < WE / 2; ++nt) {
            // B: the element's state relative to its first node, rows k = 8 ks + t (+ 4)
            const float *ub = reinterpret_cast<const float *>(sU + (2 * nt + be) * US);
            const float ref = ub[bc];
            float b[2 * KD];
#pragma unroll
            for (int q = 0; q < 2 * KD; ++q) {
                const int k = t + 4 * q;
                b[q] = (k < Np) ? ub[4 * k + bc] - ref : 0.f;
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                float r0[4] = {0.f, 0.f, 0.f, 0.f}, r1[4] = {0.f, 0.f, 0.f, 0.f};
                float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < KD; ++ks) {
                    mma3(r0, r1, frag(ent_d(0, mt, ks), 0), frag(ent_d(0, mt, ks), 1), b[2 * ks], b[2 * ks + 1]);
                    mma3(s0, s1, frag(ent_d(1, mt, ks), 0), frag(ent_d(1, mt, ks), 1), b[2 * ks], b[2 * ks + 1]);
                }
                float cr[4], cs[4], ur[4], us[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    cr[c] = r0[c] + r1[c];
                    cs[c] = s0[c] + s1[c];
                }
                frag_to_node(cr, ur, lane);
                frag_to_node(cs, us, lane);
                const int e = 2 * nt + ep, j = 16 * mt + jn;
                if (e < ne && j < Np) {
                    const float *gg = sGeo + e * 16;
                    const float rx = gg[G_RX], ry = gg[G_RY], sx = gg[G_SX], sy = gg[G_SY];
                    float u[4], gx[4], gy[4];
                    f4_to(sU[e * US + j], u);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        gx[c] = rx * ur[c] + sx * us[c];
                        gy[c] = ry * ur[c] + sy * us[c];
                    }
                    const float p = sPo[e * NpP + j];
                    float cx[4], cy[4], vx[4], vy[4], fr[4], fs[4];
                    adv_flux(u, p, ph, cx, cy);
                    visc_flux(u, gx, gy, ph, vx, vy);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float Fx = cx[c] - vx[c], Fy = cy[c] - vy[c];
                        fr[c] = rx * Fx + ry * Fy;
                        fs[c] = sx * Fx + sy * Fy;
                    }
                    float4 *fo = reinterpret_cast<float4 *>(sF + e * FS + j * 8);
                    fo[0] = to_f4(fr);
                    fo[1] = to_f4(fs);
                }
            }
        }

        __syncwarp();   // the fluxes of V are read at the face nodes below

        // ---- F: at every face node (one per lane, the Nfp nodes of a face on
        // consecutive lanes): penalty norms of both traces, their maximum over
        // the face, and the numerical flux minus the own flux
        static_assert(EPP >= 1 && EPP * NF <= 32, "the face nodes of an element fit one pass");
#pragma unroll 1
        for (int pe = 0; pe < WE; pe += EPP) {
            if (pe >= ne) break;                 // warp-uniform: the tile has no element pe
            const bool act = lane < EPP * NF && pe + lane / NF < ne;
            const int q = act ? lane : 0;
            const int e = pe + q / NF, r = q - (q / NF) * NF, f = r / Nfp, i = r - (r / Nfp) * Nfp;
            const int4 cn = sConn[e];
            const int f2 = (cn.w >> (2 * f)) & 3, bt = (cn.w >> (8 + 2 * f)) & 3;
            const float *gg = sGeo + e * 16;
            const float n1 = gg[G_NX + f], n2 = gg[G_NY + f], fsc = gg[G_FS + f];
            const int vm = sFm[f * Nfp + i], vp = sFm[f2 * Nfp + (Nfp - 1 - i)];
            float up[4], dH[4], Ftp[4];
            f4_to(sU[e * US + vm], up);
            const float pp = sPo[e * NpP + vm];
            float nrm;
            {
                // the own trace and the other side's state (neighbour trace,
                // far field or wall ghost), both norms in paired arithmetic
                const float ir = 1.0f / up[0];
                float rb, vb1, vb2, eb;
                if (bt == BCT_INTERIOR) {
                    float w[4];
                    f4_to(sN[(e * 3 + f) * UN + vp], w);
                    const float iw = 1.0f / w[0];
                    rb = w[0]; vb1 = w[1] * iw; vb2 = w[2] * iw; eb = w[3] * iw;
                } else if (bt == BCT_FARFIELD) {
                    const float iw = 1.0f / ph.Uinf[0];
                    rb = ph.Uinf[0]; vb1 = ph.Uinf[1] * iw; vb2 = ph.Uinf[2] * iw; eb = ph.Uinf[3] * iw;
                } else {
                    rb = up[0]; vb1 = ph.vw1; vb2 = ph.vw2;
                    eb = (pp / ph.gm1 + 0.5f * up[0] * (ph.vw1 * ph.vw1 + ph.vw2 * ph.vw2)) * ir;
                }
                const pf2 nab = penalty_norm2(mk(up[0], rb), mk(up[1] * ir, vb1), mk(up[2] * ir, vb2),
                                              mk(up[3] * ir, eb), n1, n2, ph);
                nrm = fmaxf(nab.v.x, nab.v.y);
            }
            float gbar = 0.f;
#pragma unroll
            for (int l = 0; l < Nfp; ++l) gbar = fmaxf(gbar, __shfl_sync(0xffffffffu, nrm, lane - i + l));
            float cinv = cinv_fac * fsc;
            const float *ng = sNGeo + (e * 3 + f) * 16;
            if (bt == BCT_INTERIOR) cinv = fmaxf(cinv, cinv_fac * ng[G_FS + f2]);
            const float sigma = sig_fac * gbar * cinv;
            {
                // F+ . n from the contravariant fluxes: (Fx, Fy) = M^-1 (Fr, Fs)
                // with M = [[rx, ry], [sx, sy]]
                const float rx = gg[G_RX], ry = gg[G_RY], sx = gg[G_SX], sy = gg[G_SY];
                const float idet = 1.0f / (rx * sy - ry * sx);
                const float a = (n1 * sy - n2 * sx) * idet, b = (n2 * rx - n1 * ry) * idet;
                const float4 fr = *reinterpret_cast<const float4 *>(sF + e * FS + vm * 8);
                const float4 fs = *reinterpret_cast<const float4 *>(sF + e * FS + vm * 8 + 4);
                Ftp[0] = a * fr.x + b * fs.x;
                Ftp[1] = a * fr.y + b * fs.y;
                Ftp[2] = a * fr.z + b * fs.z;
                Ftp[3] = a * fr.w + b * fs.w;
            }
            // broken gradient of the other side at this face node: the
            // neighbour's at vp, or (wall) the element's own at vm; a boundary
            // face's slot holds the element itself
            float go_x[4] = {0.f, 0.f, 0.f, 0.f}, go_y[4] = {0.f, 0.f, 0.f, 0.f};
            if (bt != BCT_FARFIELD) {
                const float4 *src = sN + (e * 3 + f) * UN;
                const int row = (bt == BCT_INTERIOR) ? vp : vm;
                // fields in pairs (the two halves of a float4 record) with
                // paired FMAs: (r0, r1) += (Dr, Dr) (u0, u1), and so on
                float2 r01 = make_float2(0.f, 0.f), r23 = r01, s01 = r01, s23 = r01;
#pragma unroll
                for (int j = 0; j < Np; ++j) {
                    const float2 d = sD[row * S::DS + j];
                    const float4 u = src[j];
                    const float2 dr = make_float2(d.x, d.x), ds = make_float2(d.y, d.y);
                    const float2 u01 = make_float2(u.x, u.y), u23 = make_float2(u.z, u.w);
                    r01 = __ffma2_rn(dr, u01, r01);
                    r23 = __ffma2_rn(dr, u23, r23);
                    s01 = __ffma2_rn(ds, u01, s01);
                    s23 = __ffma2_rn(ds, u23, s23);
                }
                const float wr[4] = {r01.x, r01.y, r23.x, r23.y}, ws[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    go_x[c] = ng[G_RX] * wr[c] + ng[G_SX] * ws[c];
                    go_y[c] = ng[G_RY] * wr[c] + ng[G_SY] * ws[c];
                }
            }
            // the jump U+ - U- of the penalty (and theta) terms: a small
            // difference of large values, formed in FP64 in the theta variant;
            // the state G is evaluated at, and the theta weight (1/2 on an
            // interior face, where both sides add their share)
            float jmp[4], gs[4], wth = 1.0f;
            {
                const float ir = 1.0f / up[0];
                gs[0] = up[0]; gs[1] = up[1] * ir; gs[2] = up[2] * ir; gs[3] = up[3] * ir;
            }
            if (bt == BCT_INTERIOR) {
                float um[4];
                const float *gxm = go_x, *gym = go_y;
                f4_to(sN[(e * 3 + f) * UN + vp], um);
                const float pm = sPn[(e * 3 + f) * NpP + vp];
                if constexpr (TH) {
                    const long long nb = (f == 0) ? cn.x : (f == 1 ? cn.y : cn.z);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        jmp[c] = cvt_d2f(sRaw[(e * 4 + c) * Np + vm] - sp.K0in[(nb * 4 + c) * Np + vp]);
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
            } else if (bt == BCT_FARFIELD) {
                const float ub[4] = {ph.Uinf[0], ph.Uinf[1], ph.Uinf[2], ph.Uinf[3]};
                float Fnp[4], Fnb[4], D[4];
                flux_n(up, pp, n1, n2, ph, Fnp);
                flux_n(ub, ph.pinf, n1, n2, ph, Fnb);
                roe_dissipation(up, pp, ub, ph.pinf, n1, n2, ph, D);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    jmp[c] = TH ? cvt_d2f(sRaw[(e * 4 + c) * Np + vm] - sp.uinf[c]) : up[c] - ub[c];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dH[c] = 0.5f * (Fnp[c] - Fnb[c]) - 0.5f * D[c] - sigma * jmp[c];
            } else {
                const float *gxp = go_x, *gyp = go_y;
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
            if (act)
                *reinterpret_cast<float4 *>(sDH + e * HS + r * 4) =
                    make_float4(fsc * dH[0], fsc * dH[1], fsc * dH[2], fsc * dH[3]);
            if constexpr (TH) {
                float tx[4], ty[4];
                theta_vec(gs[0], gs[1], gs[2], gs[3], jmp, n1, n2, ph, tx, ty);
                const float sc = theta * wth * fsc;
                if (act) {
                    *reinterpret_cast<float4 *>(sTHx + e * HS + r * 4) =
                        make_float4(sc * tx[0], sc * tx[1], sc * tx[2], sc * tx[3]);
                    *reinterpret_cast<float4 *>(sTHy + e * HS + r * 4) =
                        make_float4(sc * ty[0], sc * ty[1], sc * ty[2], sc * ty[3]);
                }
            }
        }
        if constexpr (S::TILE_BULK && !TH) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(barB, par, sp.bar_limit))) {
                copy_wait_failed(barA, barB, par);
                continue;
            }
        } else if constexpr (!S::TILE_BULK) {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncwarp();

        // ---- U: R = -(Dr Fr + Ds Fs) + LIFT (Fscale dH) (MMA), then the stage
        // update and the FP32 copy of the new state, one node per lane and tile
#pragma unroll
        for (int nt = 0; nt < WE / 2; ++nt) {
            const float *fb = sF + (2 * nt + be) * FS;
            const float r0 = fb[bc], s0 = fb[4 + bc];
            const float *hb = sDH + (2 * nt + be) * HS;
            float br[2 * KD], bs[2 * KD], bh[2 * KL];
#pragma unroll
            for (int q = 0; q < 2 * KD; ++q) {
                const int k = t + 4 * q;
                br[q] = (k < Np) ? fb[8 * k + bc] - r0 : 0.f;
                bs[q] = (k < Np) ? fb[8 * k + 4 + bc] - s0 : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 2 * KL; ++q) {
                const int k = t + 4 * q;
                bh[q] = (k < NF) ? hb[4 * k + bc] : 0.f;
            }
            float cR[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                // divergence and lift, each with separate accumulators for
                // the large products and the corrections
                float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
                float l0[4] = {0.f, 0.f, 0.f, 0.f}, l1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < KD; ++ks) {
                    mma3(d0, d1, frag(ent_d(0, mt, ks), 0), frag(ent_d(0, mt, ks), 1), br[2 * ks], br[2 * ks + 1]);
                    mma3(d0, d1, frag(ent_d(1, mt, ks), 0), frag(ent_d(1, mt, ks), 1), bs[2 * ks], bs[2 * ks + 1]);
                }
#pragma unroll
                for (int ks = 0; ks < KL; ++ks)
                    mma3(l0, l1, frag(ent_l(mt, ks), 0), frag(ent_l(mt, ks), 1), bh[2 * ks], bh[2 * ks + 1]);
#pragma unroll
                for (int c = 0; c < 4; ++c) cR[mt][c] = (l0[c] + l1[c]) - (d0[c] + d1[c]);
            }
            if constexpr (TH) {
                // theta terms: lift the face vectors (x and y), map them to
                // (r, s) at every node, then apply Wr, Ws (weak-form
                // derivatives; Wr 1 != 0, so no reference is taken out)
                float bx[2 * KL], by[2 * KL];
                const float *xb = sTHx + (2 * nt + be) * HS, *yb = sTHy + (2 * nt + be) * HS;
#pragma unroll
                for (int q = 0; q < 2 * KL; ++q) {
                    const int k = t + 4 * q;
                    bx[q] = (k < NF) ? xb[4 * k + bc] : 0.f;
                    by[q] = (k < NF) ? yb[4 * k + bc] : 0.f;
                }
                __syncwarp();   // every lane holds its flux B values: sF is overwritten below
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    float x0[4] = {0.f, 0.f, 0.f, 0.f}, x1[4] = {0.f, 0.f, 0.f, 0.f};
                    float y0[4] = {0.f, 0.f, 0.f, 0.f}, y1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int ks = 0; ks < KL; ++ks) {
                        mma3(x0, x1, frag(ent_l(mt, ks), 0), frag(ent_l(mt, ks), 1), bx[2 * ks], bx[2 * ks + 1]);
                        mma3(y0, y1, frag(ent_l(mt, ks), 0), frag(ent_l(mt, ks), 1), by[2 * ks], by[2 * ks + 1]);
                    }
                    float cx[4], cy[4], Lx[4], Ly[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cx[c] = x0[c] + x1[c];
                        cy[c] = y0[c] + y1[c];
                    }
                    frag_to_node(cx, Lx, lane);
                    frag_to_node(cy, Ly, lane);
                    const int e = 2 * nt + ep, j = 16 * mt + jn;
                    if (e < ne && j < Np) {
                        const float *gg = sGeo + e * 16;
                        float ar[4], as[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            ar[c] = gg[G_RX] * Lx[c] + gg[G_RY] * Ly[c];
                            as[c] = gg[G_SX] * Lx[c] + gg[G_SY] * Ly[c];
                        }
                        float4 *fo = reinterpret_cast<float4 *>(sF + e * FS + j * 8);
                        fo[0] = to_f4(ar);
                        fo[1] = to_f4(as);
                    }
                }
                __syncwarp();
                float war[2 * KD], was[2 * KD];
#pragma unroll
                for (int q = 0; q < 2 * KD; ++q) {
                    const int k = t + 4 * q;
                    war[q] = (k < Np) ? fb[8 * k + bc] : 0.f;
                    was[q] = (k < Np) ? fb[8 * k + 4 + bc] : 0.f;
                }
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    float w0[4] = {0.f, 0.f, 0.f, 0.f}, w1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int ks = 0; ks < KD; ++ks) {
                        mma3(w0, w1, frag(ent_w(0, mt, ks), 0), frag(ent_w(0, mt, ks), 1), war[2 * ks], war[2 * ks + 1]);
                        mma3(w0, w1, frag(ent_w(1, mt, ks), 0), frag(ent_w(1, mt, ks), 1), was[2 * ks], was[2 * ks + 1]);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) cR[mt][c] += w0[c] + w1[c];
                }
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                float R[4];
                frag_to_node(cR[mt], R, lane);
                const int e = 2 * nt + ep, j = 16 * mt + jn;
                if (e < ne && j < Np) {
                    const long long base = (k0 + e) * 4 * Np + j;
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
                            const double k1 = sp.first_stage ? inc : fma(sp.A, sK1[(e * 4 + c) * Np + j], inc);
                            sp.K1[base + c * Np] = k1;
                            knew[c] = fma(sp.B, k1, sRaw[(e * 4 + c) * Np + j]);
                            sp.K0out[base + c * Np] = knew[c];
                        }
                        const float un[4] = {cvt_d2f_trunc(knew[0]), cvt_d2f_trunc(knew[1]),
                                             cvt_d2f_trunc(knew[2]), cvt_d2f_trunc(knew[3])};
                        sp.Sout[(k0 + e) * Np + j] = to_f4(un);
                        sp.Pout[(k0 + e) * NpP + j] = pressure<float>(un, knew[3], gm1d);
                    }
                }
            }
        }
        __syncwarp();
    }
    }  // stages
}

}  // namespace dg
