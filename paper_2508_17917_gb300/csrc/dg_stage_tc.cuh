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
#define TC_BID blockIdx.x
#define TC_NBLK gridDim.x
#include "dg_stage_tc_body.inc"
#undef TC_BID
#undef TC_NBLK
}

// The next chunk of warp tiles from a stage's counter: lane 0 takes
// kTileChunk tiles, every lane gets the first and (in `end`) one past the
// last; a first tile >= nwt means the stage has no tiles left.
constexpr unsigned kTileChunk = 8;
__device__ __forceinline__ long long tc_grab(unsigned *ctr, int lane, long long &end, long long nwt)
{
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(ctr, kTileChunk);
    c = __shfl_sync(0xffffffffu, c, 0);
    const long long first = static_cast<long long>(c);
    end = first + kTileChunk < nwt ? first + kTileChunk : nwt;
    return first;
}

// A degree group's share of the batch's single launch: the fused batch body
// (five stages, grid barriers among the group's own blocks) on blocks bid =
// 0..nblk-1 of the group.  Blocks of different groups share the SMs
// unevenly, so the group's warps take their tiles from a counter per stage
// (sp.bar[2 + stage], zeroed with the barrier words before the launch).
template <int P, bool BATCH, bool FUSE, bool TH>
__device__ __forceinline__ void stage_tc_group_body(StageParams sp, Phys<float> ph, unsigned tc_bid, unsigned tc_nblk)
{
#define TC_BID tc_bid
#define TC_NBLK tc_nblk
#define TC_DYNAMIC_TILES
#include "dg_stage_tc_body.inc"
#undef TC_DYNAMIC_TILES
#undef TC_BID
#undef TC_NBLK
}

}  // namespace dg
