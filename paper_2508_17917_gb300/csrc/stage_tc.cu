// stage_tc.cu -- the tensor-core stage kernel (mixed precision, IIP,
// p = 1..6): launch shape, launch, and the operator fragment table.
#include <cstring>

#include "dg_stage_tc.cuh"
#include "launch.h"

namespace dg {
namespace {

// persistent grid: SMs x resident blocks, capped by the warp tiles (units =
// K elements, or the tile count of a batch tile table); the fused variant
// must fit the grid on the GPU at once (cooperative launch)
template <int P, bool BATCH, bool FUSE, bool TH = false>
cudaError_t shape_tc_p(long long units, LaunchShape &ls)
{
    using S = ShapeTC<P>;
    using L = TcLayout<P, TH>;
    auto kern = stage_tc_kernel<P, BATCH, FUSE, TH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::NT, L::bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) {
        if (FUSE) return cudaErrorInvalidConfiguration;
        per_sm = 1;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long nwt = BATCH ? units : (units + S::WE - 1) / S::WE;
    const long long nblocks = (nwt + S::NW - 1) / S::NW;
    const long long grid = static_cast<long long>(sms) * per_sm;
    ls.grid = static_cast<int>(nblocks < grid ? nblocks : grid);
    if (ls.grid < 1) ls.grid = 1;
    ls.threads = S::NT;
    ls.smem = L::bytes;
    ls.elems_per_tile = S::WE;
    ls.theta = TH;
    ls.variant = 3;
    return cudaSuccess;
}

template <int P, bool BATCH, bool FUSE>
cudaError_t launch_tc_p(const LaunchShape &ls, const StageParams &sp, const Phys<float> &ph, cudaStream_t st)
{
    if (!FUSE && !BATCH) return launch_pdl(stage_tc_kernel<P, false, false>, ls, st, sp, ph);
    if (!FUSE) {
        stage_tc_kernel<P, true, false><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ls.grid);
    cfg.blockDim = dim3(ls.threads);
    cfg.dynamicSmemBytes = ls.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stage_tc_kernel<P, BATCH, true>, sp, ph);
}

template <int P>
cudaError_t shape_tc_any(long long units, bool batch, bool fused, bool theta, LaunchShape &ls)
{
    if (theta) {
        // the theta variant runs stage-wise on a single mesh
        if (batch || fused) return cudaErrorInvalidValue;
        return shape_tc_p<P, false, false, true>(units, ls);
    }
    if (batch) return fused ? shape_tc_p<P, true, true>(units, ls) : shape_tc_p<P, true, false>(units, ls);
    return fused ? shape_tc_p<P, false, true>(units, ls) : shape_tc_p<P, false, false>(units, ls);
}

template <int P>
cudaError_t launch_tc_any(bool batch, bool fused, const LaunchShape &ls, const StageParams &sp,
                          const Phys<float> &ph, cudaStream_t st)
{
    if (ls.theta) {
        if (batch || fused) return cudaErrorInvalidValue;
        return launch_pdl(stage_tc_kernel<P, false, false, true>, ls, st, sp, ph);
    }
    if (batch) return fused ? launch_tc_p<P, true, true>(ls, sp, ph, st) : launch_tc_p<P, true, false>(ls, sp, ph, st);
    return fused ? launch_tc_p<P, false, true>(ls, sp, ph, st) : launch_tc_p<P, false, false>(ls, sp, ph, st);
}

// The degree groups of a batch in one launch: group g owns blocks
// [first[g], first[g] + nblk[g]) and its own stage parameters (buffers, tile
// table, barrier words); the groups never wait on one another.
constexpr int kMaxMultiGroups = 8;
struct TcMulti {
    StageParams sp[kMaxMultiGroups];
    int p[kMaxMultiGroups];
    unsigned first[kMaxMultiGroups], nblk[kMaxMultiGroups];
    int ngroups;
};

// Four blocks per SM (128 registers): the p = 5, 6 bodies need them, and one
// kernel has one register budget.
__global__ void __launch_bounds__(128, 4) stage_tc_multi_kernel(const __grid_constant__ TcMulti m, Phys<float> ph)
{
    int g = 0;
    while (g + 1 < m.ngroups && blockIdx.x >= m.first[g + 1]) ++g;
    const unsigned bid = blockIdx.x - m.first[g], nb = m.nblk[g];
    switch (m.p[g]) {
    case 1: stage_tc_group_body<1, true, true, false>(m.sp[g], ph, bid, nb); break;
    case 2: stage_tc_group_body<2, true, true, false>(m.sp[g], ph, bid, nb); break;
    case 3: stage_tc_group_body<3, true, true, false>(m.sp[g], ph, bid, nb); break;
    case 4: stage_tc_group_body<4, true, true, false>(m.sp[g], ph, bid, nb); break;
    case 5: stage_tc_group_body<5, true, true, false>(m.sp[g], ph, bid, nb); break;
    case 6: stage_tc_group_body<6, true, true, false>(m.sp[g], ph, bid, nb); break;
    default: break;
    }
}

template <int P>
size_t tc_group_smem()
{
    return TcLayout<P, false>::bytes;
}

size_t tc_group_smem_any(int p)
{
    switch (p) {
    case 1: return tc_group_smem<1>();
    case 2: return tc_group_smem<2>();
    case 3: return tc_group_smem<3>();
    case 4: return tc_group_smem<4>();
    case 5: return tc_group_smem<5>();
    case 6: return tc_group_smem<6>();
    default: return 0;
    }
}

// x rounded to TF32 (10 explicit mantissa bits), ties away from zero; the
// operators are finite and far from the FP32 overflow threshold
float tf32_round(float x)
{
    unsigned u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

bool stage_tc_supported(int p) { return p >= 1 && p <= 6; }

int stage_tile_elems_tc() { return ShapeTC<1>::WE; }

cudaError_t stage_shape_tc(int p, long long units, bool batch, bool fused, LaunchShape &out, bool theta)
{
    switch (p) {
    case 1: return shape_tc_any<1>(units, batch, fused, theta, out);
    case 2: return shape_tc_any<2>(units, batch, fused, theta, out);
    case 3: return shape_tc_any<3>(units, batch, fused, theta, out);
    case 4: return shape_tc_any<4>(units, batch, fused, theta, out);
    case 5: return shape_tc_any<5>(units, batch, fused, theta, out);
    case 6: return shape_tc_any<6>(units, batch, fused, theta, out);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t stage_tc_multi_capacity(const int *ps, int ngroups, int &blocks, size_t &smem)
{
    if (ngroups < 1 || ngroups > kMaxMultiGroups) return cudaErrorInvalidValue;
    smem = 0;
    for (int g = 0; g < ngroups; ++g) {
        const size_t b = tc_group_smem_any(ps[g]);
        if (b == 0) return cudaErrorInvalidValue;
        smem = b > smem ? b : smem;
    }
    cudaError_t e = cudaFuncSetAttribute(stage_tc_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(stage_tc_multi_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_tc_multi_kernel, 128, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = per_sm * sms;
    return blocks >= ngroups ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_stage_tc_multi(int ngroups, const int *ps, const StageParams *sps, const unsigned *nblk,
                                  size_t smem, const Phys<float> &ph, cudaStream_t st)
{
    if (ngroups < 1 || ngroups > kMaxMultiGroups) return cudaErrorInvalidValue;
    TcMulti m{};
    m.ngroups = ngroups;
    unsigned total = 0;
    for (int g = 0; g < ngroups; ++g) {
        if (nblk[g] < 1) return cudaErrorInvalidValue;
        m.sp[g] = sps[g];
        m.p[g] = ps[g];
        m.first[g] = total;
        m.nblk[g] = nblk[g];
        total += nblk[g];
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stage_tc_multi_kernel, m, ph);
}

cudaError_t launch_stage_tc(int p, bool batch, bool fused, const LaunchShape &ls, const StageParams &sp,
                            const Phys<float> &ph, cudaStream_t st)
{
    switch (p) {
    case 1: return launch_tc_any<1>(batch, fused, ls, sp, ph, st);
    case 2: return launch_tc_any<2>(batch, fused, ls, sp, ph, st);
    case 3: return launch_tc_any<3>(batch, fused, ls, sp, ph, st);
    case 4: return launch_tc_any<4>(batch, fused, ls, sp, ph, st);
    case 5: return launch_tc_any<5>(batch, fused, ls, sp, ph, st);
    case 6: return launch_tc_any<6>(batch, fused, ls, sp, ph, st);
    default: return cudaErrorInvalidValue;
    }
}

// A operands of the three operators, zero-padded to 16 MT rows and 8 KD
// (Dr, Ds) or 8 KL (LIFT) columns, in the order the kernel reads them:
// entries Dr [MT][KD], Ds [MT][KD], LIFT [MT][KL], Wr [MT][KD], Ws [MT][KD]
// (the weak-form derivatives of the theta terms), each [hi, lo][lane][a0..a3]
// with lane = 4 g + t, a0 = A[16 mt + g][8 ks + t], a1 = A[16 mt + g + 8][8 ks + t],
// a2 = A[16 mt + g][8 ks + t + 4], a3 = A[16 mt + g + 8][8 ks + t + 4].  hi is
// the FP64 entry rounded to FP32 and then to TF32; lo is the remainder
// rounded the same way.  Followed by (Dr, Ds) in FP32 as interleaved pairs,
// row-major (the face-node rows).
void build_tc_fragments(int Np, int NF, const double *Dr, const double *Ds, const double *LIFT,
                        const double *Wr, const double *Ws, std::vector<float> &out)
{
    const int MT = (Np + 15) / 16, KD = (Np + 7) / 8, KL = (NF + 7) / 8;
    const int nent = 4 * MT * KD + MT * KL;
    const size_t nfrag = static_cast<size_t>(nent) * 64;            // float4
    out.assign(nfrag * 4 + 2 * static_cast<size_t>(Np) * Np, 0.0f);
    auto put = [&](int ent, const double *A, int ncols, int mt, int ks) {
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t = lane & 3;
            const int rows[4] = {16 * mt + g, 16 * mt + g + 8, 16 * mt + g, 16 * mt + g + 8};
            const int cols[4] = {8 * ks + t, 8 * ks + t, 8 * ks + t + 4, 8 * ks + t + 4};
            for (int a = 0; a < 4; ++a) {
                const double x = (rows[a] < Np && cols[a] < ncols) ? A[rows[a] * ncols + cols[a]] : 0.0;
                const float hi = tf32_round(static_cast<float>(x));
                const float lo = tf32_round(static_cast<float>(x - static_cast<double>(hi)));
                out[((static_cast<size_t>(ent) * 2 + 0) * 32 + lane) * 4 + a] = hi;
                out[((static_cast<size_t>(ent) * 2 + 1) * 32 + lane) * 4 + a] = lo;
            }
        }
    };
    for (int mt = 0; mt < MT; ++mt) {
        for (int ks = 0; ks < KD; ++ks) {
            put((0 * MT + mt) * KD + ks, Dr, Np, mt, ks);
            put((1 * MT + mt) * KD + ks, Ds, Np, mt, ks);
        }
        for (int ks = 0; ks < KL; ++ks) put(2 * MT * KD + mt * KL + ks, LIFT, NF, mt, ks);
        for (int ks = 0; ks < KD; ++ks) {
            put(2 * MT * KD + MT * KL + (0 * MT + mt) * KD + ks, Wr, Np, mt, ks);
            put(2 * MT * KD + MT * KL + (1 * MT + mt) * KD + ks, Ws, Np, mt, ks);
        }
    }
    float *d = out.data() + nfrag * 4;
    for (int i = 0; i < Np * Np; ++i) {
        d[2 * i] = static_cast<float>(Dr[i]);
        d[2 * i + 1] = static_cast<float>(Ds[i]);
    }
}

}  // namespace dg
