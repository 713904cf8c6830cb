// stage_fp64.cu -- FP64 instantiations of the fused stage kernel (p = 1..6).
#include "dg_stage.cuh"
#include "launch.h"

namespace dg {
namespace {

template <int P, typename real, bool TH, bool OI = false>
cudaError_t shape_p(long long K, LaunchShape &ls)
{
    using L = Smem<P, real, TH, OI>;
    auto kern = stage_kernel<P, real, TH, OI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L::bytes));
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
    ls.overint = OI;
    return cudaSuccess;
}

template <int P, typename real>
cudaError_t launch_p(const LaunchShape &ls, const StageParams &sp, const Phys<real> &ph, cudaStream_t st)
{
    if (ls.overint)
        stage_kernel<P, real, false, true><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
    else if (ls.theta)
        stage_kernel<P, real, true><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
    else
        stage_kernel<P, real, false><<<ls.grid, ls.threads, ls.smem, st>>>(sp, ph);
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

cudaError_t stage_shape_fp64(int p, long long K, bool theta, LaunchShape &out, bool overint)
{
#define C_(P) (overint ? shape_p<P, double, false, true>(K, out) \
                       : (theta ? shape_p<P, double, true>(K, out) : shape_p<P, double, false>(K, out)))
    DG_SWITCH_P(p, C_)
#undef C_
}

cudaError_t launch_stage_fp64(int p, const LaunchShape &ls, const StageParams &sp,
                              const Phys<double> &ph, cudaStream_t st)
{
#define C_(P) launch_p<P, double>(ls, sp, ph, st)
    DG_SWITCH_P(p, C_)
#undef C_
}

}  // namespace dg
