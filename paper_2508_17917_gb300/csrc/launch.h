// launch.h -- host-side launch wrappers for the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dg_device.cuh"

namespace dg {

struct StageParams;
struct BatchCase;

struct LaunchShape {
    bool theta = false;      // kernel variant with the theta terms of the IP flux
    int variant = 1;         // mixed IIP kernel: 1 node per thread (1), 2 nodes per thread (2),
                             // tensor-core warp tiles (3)
    bool overint = false;    // FP64 kernel: volume flux integrated with a cubature rule
    int grid = 0;
    int threads = 0;
    size_t smem = 0;
    int elems_per_tile = 0;
};

// Launch `kern` with programmatic stream serialization: its blocks may be
// scheduled while the previous kernel of the stream drains; the kernel waits
// for that kernel (pdl_wait_then_release) before touching the state.
template <typename... Args>
inline cudaError_t launch_pdl(void (*kern)(Args...), const LaunchShape &ls, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ls.grid);
    cfg.blockDim = dim3(ls.threads);
    cfg.dynamicSmemBytes = ls.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}


// Launch configuration of the fused stage kernel for degree p and K elements
// on the current device (persistent grid: SMs x resident CTAs, capped by tiles).
cudaError_t stage_shape_fp64(int p, long long K, bool theta, LaunchShape &out, bool overint = false);
cudaError_t stage_shape_mixed(int p, long long K, bool theta, LaunchShape &out);
cudaError_t launch_stage_fp64(int p, const LaunchShape &ls, const StageParams &sp,
                              const Phys<double> &ph, cudaStream_t st);
cudaError_t launch_stage_mixed(int p, const LaunchShape &ls, const StageParams &sp,
                               const Phys<float> &ph, cudaStream_t st);
// batch variant of the mixed kernel (IIP): grid for `ntiles` tiles of a tile table
cudaError_t stage_shape_mixed_batch(int p, long long ntiles, LaunchShape &out);
cudaError_t launch_stage_mixed_batch(int p, const LaunchShape &ls, const StageParams &sp,
                                     const Phys<float> &ph, cudaStream_t st);
// Lambda_K in FP32 from the FP32 state copy (mixed path); tiles == nullptr:
// K elements in tiles of E, ph carries mu and v_w; otherwise the batch tile
// table and per-case mu, v_b
// Lambda_K of every degree group of a batch in one launch (one block per tile)
cudaError_t launch_dt_lambda_mixed_multi(const DtGroups &dgs, const BatchCase *cases, const Phys<float> &ph,
                                         float sig_fac, cudaStream_t st);
cudaError_t launch_dt_lambda_mixed(int p, const float4 *S, const float *Pr, const float *geo, const int4 *conn,
                                   const int *fmask, const int4 *tiles, long long ntiles, const BatchCase *cases,
                                   long long K, const Phys<float> &ph, float sig_fac, double *lam, cudaStream_t st);
// the mixed IIP kernel with two nodes per thread: units = K elements (single
// mesh) or the tile count of a tile table (batch); its tiles hold
// stage_tile_elems2(p) elements
cudaError_t stage_shape_mixed2(int p, long long units, bool batch, LaunchShape &out);
cudaError_t launch_stage_mixed2(int p, bool batch, const LaunchShape &ls, const StageParams &sp,
                                const Phys<float> &ph, cudaStream_t st);
int stage_tile_elems2(int p);
// five stages per cooperative launch (mixed IIP, shape `variant`): grid of
// co-resident blocks for `units` (K, or the tile count of a batch table)
cudaError_t stage_shape_mixed_fused(int p, int variant, bool batch, long long units, LaunchShape &out);
cudaError_t launch_stage_mixed_fused(int p, bool batch, const LaunchShape &ls, const StageParams &sp,
                                     const Phys<float> &ph, cudaStream_t st);
// elements per tile of the mixed kernel for degree p
int stage_tile_elems(int p);
// the tensor-core mixed IIP kernel (p = 1..6): warp tiles of 2 elements;
// its `ops` is the operator table of build_tc_fragments
bool stage_tc_supported(int p);
// elements per warp tile of the tensor-core kernel (any p)
int stage_tile_elems_tc();
// units = K elements (single mesh) or the tile count of a batch tile table;
// fused: five stages per cooperative launch with grid barriers
// theta: the SIP / NIPG variant (single mesh, stage-wise launches only)
cudaError_t stage_shape_tc(int p, long long units, bool batch, bool fused, LaunchShape &out, bool theta = false);
// the fused batch body of every degree group in one cooperative launch:
// blocks that fit the GPU at once and the shared memory per block (the
// largest group's layout), then the launch with nblk[g] blocks for group g
cudaError_t stage_tc_multi_capacity(const int *ps, int ngroups, int &blocks, size_t &smem);
cudaError_t launch_stage_tc_multi(int ngroups, const int *ps, const StageParams *sps, const unsigned *nblk,
                                  size_t smem, const Phys<float> &ph, cudaStream_t st);
cudaError_t launch_stage_tc(int p, bool batch, bool fused, const LaunchShape &ls, const StageParams &sp,
                            const Phys<float> &ph, cudaStream_t st);
// Dr, Ds [Np][Np], LIFT [Np][NF], Wr, Ws [Np][Np] (FP64, row-major) -> the kernel's
// operator table (TF32 hi / lo fragments of 16-row tiles, then (Dr, Ds) as
// FP32 pairs [Np][Np])
void build_tc_fragments(int Np, int NF, const double *Dr, const double *Ds, const double *LIFT,
                        const double *Wr, const double *Ws, std::vector<float> &out);
// FP32 copy [K][Np] float4 and FP64-recovered pressure [K][NpP] of a state
cudaError_t launch_make_shadow(int p, const double *K0, long long K, double gm1, float4 *S,
                               float *Pr, cudaStream_t st);
// padded pressure row length: Np rounded up to a multiple of 4
inline int pressure_row(int p) { return (((p + 1) * (p + 2) / 2) + 3) & ~3; }

struct BatchCase;

struct AuxMesh {
    const double *U;          // [K][4][Np]
    const int *elem_case = nullptr;         // batch: case of every element (mu, v_b)
    const BatchCase *cases = nullptr;
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

// batch: one block per case, max of lam over the case's element range
// [seg[2i], seg[2i+1]) -> cases[i].lam and dt = cfl / lam, or fixed[i] when
// fixed is not null (0 and bad = 1 if the bound is not finite); then the
// case's Newmark step with its lagged lift: sets v_b, advances t
cudaError_t launch_batch_dt_newmark(const double *lam, const long long *seg, BatchCase *cases, int ncases,
                                    double cfl, const double *fixed, cudaStream_t st);
// batch: the wall faces of every degree group in one launch (group g's faces
// numbered from g.base); partial[w] = (Fx, Fy, Mz) of face w, moment about 0
struct WallGroup {
    AuxMesh m;
    const int2 *faces;        // (element, face) of the group's wall faces
    const double *face_xy;    // their face nodes' coordinates, [nwall][Nfp][2]
    const double *wface;      // LGL weights [Nfp]
    int base, nwall;
};
struct WallGroups {
    WallGroup g[8];
    int n = 0, total = 0;
};
cudaError_t launch_batch_wall_forces(const WallGroups &wg, const Phys<double> &ph, double *partial,
                                     cudaStream_t st);
// batch: one block per case, sum of the wall-face partials [wseg[2i], wseg[2i+1]) -> Fx, Fy, Mz, and
// with hist: (t, dt, y, y', v_b, Fx, Fy, lam) of every case at row *counter, then ++*counter
// (ticket: a zeroed counter of finished blocks)
cudaError_t launch_batch_forces_record(const double *partial, const int *wseg, BatchCase *cases, int ncases,
                                       double *hist, int cap, int *counter, unsigned *ticket, cudaStream_t st);

// *flag = 1 if any of x[0..n) is not finite (flag must be zeroed first)
cudaError_t launch_nonfinite(const double *x, long long n, int *flag, cudaStream_t st);

// viscous source of the advected isentropic vortex (dg_set_source kind 2)
struct VortexSource {
    double beta, x0, y0, L, u0, v0;   // strength, centre at t = 0, period, advection velocity
    double mu, Pr;
    double invL, f0, c2, invPr;       // 1/L, beta/(2 pi), beta^2/(2 pi^2), 1/Pr
};
// broken gradient of every element (dg_broken_gradient): impl 0 FP64 on the
// CUDA cores, impl 1 split TF32 on tcgen05 with the tiles staged by TMA
struct GradTc05Args {
    const double *U;            // [K][4][Np] FP64 state (device)
    const double *Dr, *Ds;      // Np x Np operators (host, for the split image)
    const double *Dr_dev, *Ds_dev;   // the same on the device (impl 0)
    const double *geo;          // double[16] per element
    long long K;
    double *gx, *gy;            // [K][4][Np] outputs (device)
    float *bimg;                // device buffer of grad_tc05_bimg_floats(p) floats (impl 1)
    bool upload_ops;            // (re)write the split operator image into bimg first (impl 1)
    int *err;                   // set to 1 if a bounded wait gave up (impl 1)
    unsigned wait_limit;
};
size_t grad_tc05_bimg_floats(int p);
cudaError_t launch_broken_gradient(int p, int impl, const GradTc05Args &a, cudaStream_t st);

struct VortexCentres {
    double xc[5], yc[5];
    int ns;
};
// S[s][K][4][Np] at the times t[s], s < ns <= 5, from node coordinates
// xy = (x[K*Np], y[K*Np]) in one launch; fp64: double arithmetic, else float
// after the offsets
cudaError_t launch_vortex_source(bool fp64, const double *xy, long long nn, int Np, const VortexSource &v,
                                 const double *t, int ns, double *S, cudaStream_t st);

}  // namespace dg
