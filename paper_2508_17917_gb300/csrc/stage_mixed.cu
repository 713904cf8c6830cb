// stage_mixed.cu -- mixed-precision stage kernel instantiations (p = 1..6):
// FP32 arithmetic, FP64 state in HBM, FP64 pressure recovery and registers.
#include "dg_stage_mixed.cuh"
#include "dg_stage_mixed2.cuh"
#include "launch.h"

namespace dg {

namespace {

template <int P, bool TH>
cudaError_t shape_p(long long K, LaunchShape &ls)
{
    using L = MixedLayout<P, TH>;
    auto kern = stage_mixed_kernel<P, TH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Shape<P>::NT, L::bytes);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
    long long ntiles = (K + Shape<P>::E - 1) / Shape<P>::E;
    long long grid = static_cast<long long>(sms) * per_sm;
    ls.grid = static_cast<int>(ntiles < grid ? ntiles : grid);
    ls.threads = Shape<P>::NT;
    ls.smem = L::bytes;
    ls.elems_per_tile = Shape<P>::E;
    ls.theta = TH;
    return cudaSuccess;
}

template <int P>
cudaError_t launch_p(const LaunchShape &ls, const StageParams &sp, const Phys<float> &ph, cudaStream_t st)
{
    if (ls.theta) return launch_pdl(stage_mixed_kernel<P, true, false, false>, ls, st, sp, ph);
    return launch_pdl(stage_mixed_kernel<P, false, false, false>, ls, st, sp, ph);
}

template <int P>
cudaError_t shape_batch_p(long long ntiles, LaunchShape &ls)
{
    using L = MixedLayout<P, false>;
    auto kern = stage_mixed_kernel<P, false, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Shape<P>::NT, L::bytes);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
    long long grid = static_cast<long long>(sms) * per_sm;
    ls.grid = static_cast<int>(ntiles < grid ? ntiles : grid);
    ls.threads = Shape<P>::NT;
    ls.smem = L::bytes;
    ls.elems_per_tile = Shape<P>::E;
    ls.theta = false;
    return cudaSuccess;
}

template <int P>
cudaError_t launch_batch_p(const LaunchShape &ls, const StageParams &sp, const Phys<float> &ph, cudaStream_t st)
{
    // batch stage launches are graph-captured next to the batch's other
    // kernels: ordinary launches (overlapping launches measured slower there)
    stage_mixed_kernel<P, false, true><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
    return cudaGetLastError();
}

// two nodes per thread (IIP): shape for `ntiles` tiles (batch) or for K elements
template <int P, bool BATCH>
cudaError_t shape2_p(long long units, LaunchShape &ls)
{
    using S2 = Shape2<P>;
    using L = MixedLayout<P, false, S2::E>;
    auto kern = stage_mixed2_kernel<P, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::bytes));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S2::NT, L::bytes);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
    const long long ntiles = BATCH ? units : (units + S2::E - 1) / S2::E;
    long long grid = static_cast<long long>(sms) * per_sm;
    ls.grid = static_cast<int>(ntiles < grid ? ntiles : grid);
    ls.threads = S2::NT;
    ls.smem = L::bytes;
    ls.elems_per_tile = S2::E;
    ls.theta = false;
    ls.variant = 2;
    return cudaSuccess;
}

template <int P, bool BATCH>
cudaError_t launch2_p(const LaunchShape &ls, const StageParams &sp, const Phys<float> &ph, cudaStream_t st)
{
    if (BATCH) {
        stage_mixed2_kernel<P, true><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
        return cudaGetLastError();
    }
    return launch_pdl(stage_mixed2_kernel<P, false, false>, ls, st, sp, ph);
}

// fused variant: five stages per cooperative launch; the grid is the number
// of co-resident blocks of that instantiation (capped by the tile count)
template <int P, int V, bool BATCH>
cudaError_t fused_shape_p(long long units, LaunchShape &ls)
{
    const void *kern;
    int nt;
    size_t smem;
    long long ntiles;
    if (V == 2) {
        kern = reinterpret_cast<const void *>(stage_mixed2_kernel<P, BATCH, true>);
        nt = Shape2<P>::NT;
        smem = MixedLayout<P, false, Shape2<P>::E>::bytes;
        ntiles = BATCH ? units : (units + Shape2<P>::E - 1) / Shape2<P>::E;
        ls.elems_per_tile = Shape2<P>::E;
    } else {
        kern = reinterpret_cast<const void *>(stage_mixed_kernel<P, false, BATCH, true>);
        nt = Shape<P>::NT;
        smem = MixedLayout<P, false>::bytes;
        ntiles = BATCH ? units : (units + Shape<P>::E - 1) / Shape<P>::E;
        ls.elems_per_tile = Shape<P>::E;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = static_cast<long long>(sms) * per_sm;
    ls.grid = static_cast<int>(ntiles < grid ? ntiles : grid);
    ls.threads = nt;
    ls.smem = smem;
    ls.theta = false;
    ls.variant = V;
    return cudaSuccess;
}

template <int P, int V, bool BATCH>
cudaError_t fused_launch_p(const LaunchShape &ls, const StageParams &sp, const Phys<float> &ph, cudaStream_t st)
{
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
    if (V == 2) return cudaLaunchKernelEx(&cfg, stage_mixed2_kernel<P, BATCH, true>, sp, ph);
    return cudaLaunchKernelEx(&cfg, stage_mixed_kernel<P, false, BATCH, true>, sp, ph);
}

template <int P>
cudaError_t shadow_p(const double *K0, long long K, double gm1, float4 *S, float *Pr, cudaStream_t st)
{
    constexpr int Np = (P + 1) * (P + 2) / 2;
    const long long n = K * Np;
    const int threads = 256;
    make_shadow_kernel<P><<<static_cast<unsigned>((n + threads - 1) / threads), threads, 0, st>>>(K0, K, gm1, S, Pr);
    return cudaGetLastError();
}

}  // namespace

#define DG_SWITCH_P(p, CALL)                      \
    switch (p) {                                  \
    case 1: return CALL(1);                       \
    case 2: return CALL(2);                       \
    case 3: return CALL(3);                       \
    case 4: return CALL(4);                       \
    case 5: return CALL(5);                       \
    case 6: return CALL(6);                       \
    default: return cudaErrorInvalidValue;        \
    }

cudaError_t stage_shape_mixed(int p, long long K, bool theta, LaunchShape &out)
{
#define C_(P) (theta ? shape_p<P, true>(K, out) : shape_p<P, false>(K, out))
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t launch_stage_mixed(int p, const LaunchShape &ls, const StageParams &sp,
                               const Phys<float> &ph, cudaStream_t st)
{
#define C_(P) launch_p<P>(ls, sp, ph, st)
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t stage_shape_mixed_batch(int p, long long ntiles, LaunchShape &out)
{
#define C_(P) shape_batch_p<P>(ntiles, out)
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t launch_stage_mixed_batch(int p, const LaunchShape &ls, const StageParams &sp,
                                     const Phys<float> &ph, cudaStream_t st)
{
#define C_(P) launch_batch_p<P>(ls, sp, ph, st)
    DG_SWITCH_P(p, C_)
#undef C_
}

template <int P>
cudaError_t dt_mixed_p(const float4 *S, const float *Pr, const float *geo, const int4 *conn, const int *fmask,
                       const int4 *tiles, long long ntiles, const BatchCase *cases, long long K,
                       const Phys<float> &ph, float sig_fac, double *lam, cudaStream_t st)
{
    const long long nblk = tiles ? ntiles : (K + Shape<P>::E - 1) / Shape<P>::E;
    if (nblk < 1) return cudaSuccess;
    dt_lambda_mixed_kernel<P><<<static_cast<unsigned>(nblk), Shape<P>::NT, 0, st>>>(S, Pr, geo, conn, fmask, tiles,
                                                                                   cases, K, ph, sig_fac, lam);
    return cudaGetLastError();
}

cudaError_t launch_dt_lambda_mixed_multi(const DtGroups &dgs, const BatchCase *cases, const Phys<float> &ph,
                                         float sig_fac, cudaStream_t st)
{
    if (dgs.blocks < 1) return cudaSuccess;
    dt_lambda_mixed_multi_kernel<1, 2, 3, 4, 5, 6><<<static_cast<unsigned>(dgs.blocks), 256, 0, st>>>(
        dgs, cases, ph, sig_fac);
    return cudaGetLastError();
}

cudaError_t launch_dt_lambda_mixed(int p, const float4 *S, const float *Pr, const float *geo, const int4 *conn,
                                   const int *fmask, const int4 *tiles, long long ntiles, const BatchCase *cases,
                                   long long K, const Phys<float> &ph, float sig_fac, double *lam, cudaStream_t st)
{
#define C_(P) dt_mixed_p<P>(S, Pr, geo, conn, fmask, tiles, ntiles, cases, K, ph, sig_fac, lam, st)
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t stage_shape_mixed2(int p, long long units, bool batch, LaunchShape &out)
{
#define C_(P) (batch ? shape2_p<P, true>(units, out) : shape2_p<P, false>(units, out))
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t launch_stage_mixed2(int p, bool batch, const LaunchShape &ls, const StageParams &sp,
                                const Phys<float> &ph, cudaStream_t st)
{
#define C_(P) (batch ? launch2_p<P, true>(ls, sp, ph, st) : launch2_p<P, false>(ls, sp, ph, st))
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t stage_shape_mixed_fused(int p, int variant, bool batch, long long units, LaunchShape &out)
{
#define C_(P) (variant == 2 ? (batch ? fused_shape_p<P, 2, true>(units, out) : fused_shape_p<P, 2, false>(units, out)) \
                            : (batch ? fused_shape_p<P, 1, true>(units, out) : fused_shape_p<P, 1, false>(units, out)))
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t launch_stage_mixed_fused(int p, bool batch, const LaunchShape &ls, const StageParams &sp,
                                     const Phys<float> &ph, cudaStream_t st)
{
#define C_(P) (ls.variant == 2 ? (batch ? fused_launch_p<P, 2, true>(ls, sp, ph, st)                 \
                                        : fused_launch_p<P, 2, false>(ls, sp, ph, st))               \
                               : (batch ? fused_launch_p<P, 1, true>(ls, sp, ph, st)                 \
                                        : fused_launch_p<P, 1, false>(ls, sp, ph, st)))
    DG_SWITCH_P(p, C_)
#undef C_
}

int stage_tile_elems2(int p)
{
    switch (p) {
    case 1: return Shape2<1>::E;
    case 2: return Shape2<2>::E;
    case 3: return Shape2<3>::E;
    case 4: return Shape2<4>::E;
    case 5: return Shape2<5>::E;
    case 6: return Shape2<6>::E;
    default: return 0;
    }
}

int stage_tile_elems(int p)
{
    switch (p) {
    case 1: return Shape<1>::E;
    case 2: return Shape<2>::E;
    case 3: return Shape<3>::E;
    case 4: return Shape<4>::E;
    case 5: return Shape<5>::E;
    case 6: return Shape<6>::E;
    default: return 0;
    }
}

cudaError_t launch_make_shadow(int p, const double *K0, long long K, double gm1, float4 *S, float *Pr,
                               cudaStream_t st)
{
#define C_(P) shadow_p<P>(K0, K, gm1, S, Pr, st)
    DG_SWITCH_P(p, C_)
#undef C_
}

}  // namespace dg
