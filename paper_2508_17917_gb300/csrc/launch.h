// launch.h -- host-side launch wrappers for the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_device.cuh"

namespace dg {

struct StageParams;

struct LaunchShape {
    bool theta = false;      // kernel variant with the theta terms of the IP flux
    int grid = 0;
    int threads = 0;
    size_t smem = 0;
    int elems_per_tile = 0;
};

// Launch configuration of the fused stage kernel for degree p and K elements
// on the current device (persistent grid: SMs x resident CTAs, capped by tiles).
cudaError_t stage_shape_fp64(int p, long long K, bool theta, LaunchShape &out);
cudaError_t stage_shape_mixed(int p, long long K, bool theta, LaunchShape &out);
cudaError_t launch_stage_fp64(int p, const LaunchShape &ls, const StageParams &sp,
                              const Phys<double> &ph, cudaStream_t st);
cudaError_t launch_stage_mixed(int p, const LaunchShape &ls, const StageParams &sp,
                               const Phys<float> &ph, cudaStream_t st);
// FP32 copy [K][Np] float4 and FP64-recovered pressure [K][NpP] of a state
cudaError_t launch_make_shadow(int p, const double *K0, long long K, double gm1, float4 *S,
                               float *Pr, cudaStream_t st);
// padded pressure row length: Np rounded up to a multiple of 4
inline int pressure_row(int p) { return (((p + 1) * (p + 2) / 2) + 3) & ~3; }

struct AuxMesh {
    const double *U;          // [K][4][Np]
    const double *geo;        // double[16] per element
    const int4 *conn;
    const double *Dr, *Ds;    // Np*Np
    const int *fmask;         // 3*Nfp
    long long K;
    int p;
};

// Lambda_K of Eq. rayleigh_bound per element into lam[K] (FP64);
// sig_fac = C1 (1+theta)^2 (d+1) of Eq. penalty_final.
cudaError_t launch_dt_lambda(const AuxMesh &m, const Phys<double> &ph, double sig_fac,
                             double *lam, cudaStream_t st);
// max over lam[0..K) into *out (one block).
cudaError_t launch_max_reduce(const double *lam, long long K, double *out, cudaStream_t st);

// per-wall-face force/moment partials, then a deterministic sum into out[3]
cudaError_t launch_wall_force_faces(const AuxMesh &m, const Phys<double> &ph, const int2 *faces,
                                    const double *face_xy, const double *wface, int nwall,
                                    double xc, double yc, double *partial, cudaStream_t st);
cudaError_t launch_sum3(const double *partial, int n, double *out, cudaStream_t st);

// *flag = 1 if any of x[0..n) is not finite (flag must be zeroed first)
cudaError_t launch_nonfinite(const double *x, long long n, int *flag, cudaStream_t st);

}  // namespace dg
