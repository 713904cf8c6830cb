// dg_api.cu -- implementation of the C ABI declared in include/dg.h.
//
// Host side of the library: parameter checks, mesh validation, the affine
// geometry of every element (Sec. 2.2, maps T_K), face matching, device
// buffers and the sequencing of the stage kernels into Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_stage.cuh"
#include "devbuf.h"
#include "launch.h"
#include "mesh.h"
#include "refops.h"
#include "rigid.h"
#include "rk.h"

namespace {

using dg::kRkA;
using dg::kRkB;
using dg::kRkC;

}  // namespace

struct dg_ctx {
    dg_params prm{};
    cudaStream_t stream = nullptr;
    dg::RefOps ops;
    std::string err;
    int64_t launches = 0;
    // mesh (host copies kept for coordinates)
    long long K = 0;
    std::vector<double> vx, vy;
    std::vector<int32_t> EToV;
    std::vector<double> geo64h;
    // device
    dg::DevBuf<double> K0a, K0b, K1, rtmp, geo64, ops64, Dr64, Ds64, src, lam, scal, fpart, fxy, wface;
    dg::DevBuf<float> geo32, ops32, P0a, P0b;     // mixed path: pressures of the two K0 buffers
    dg::DevBuf<float4> S0a, S0b;                  // mixed path: FP32 copies of the two K0 buffers
    dg::DevBuf<int4> conn;
    dg::DevBuf<int> fmask, flag;
    dg::DevBuf<int2> wall;
    int nwall = 0;
    bool cur_is_a = true;
    dg::LaunchShape shape;    // stage kernel in use
    dg::LaunchShape shape1, shape2;   // mixed IIP: one / two nodes per thread
    dg::LaunchShape shape3;           // mixed IIP, p <= 6: tensor-core warp tiles
    bool has_tc = false;              // shape3 is configured for the current mesh
    dg::DevBuf<float> tcfrag;         // operator fragments of the tensor-core kernel
    int variant_req = 0;      // 0: pick by timing on first use, 1, 2 or 3: forced
    bool tuned = false;
    // fused steps: five stages in one cooperative launch with grid barriers
    bool overint = false;     // FP64 path: over-integrated volume term
    bool fused = false;
    dg::LaunchShape fshape;
    int fshape_variant = 0;
    dg::DevBuf<unsigned> bar;
    dg::DevBuf<int> bar_err;
    unsigned bar_limit = 1u << 24;
    bool bar_used = false;
    bool copy_used = false;           // a stage kernel with bounded copy waits ran (reported where the API synchronises anyway)
    int source_kind = DG_SOURCE_NONE;
    dg::DevBuf<float> gimg;           // split [Dr; Ds] image of the tcgen05 gradient
    bool gimg_ready = false;          // gimg holds the image
    dg::DevBuf<double> gtmp;          // host-output staging of dg_broken_gradient
    dg::VortexSource vortex{};         // DG_SOURCE_VORTEX parameters
    dg::DevBuf<double> src_xy;        // node coordinates for the vortex source

    double *cur() { return cur_is_a ? K0a.ptr : K0b.ptr; }
    double *other() { return cur_is_a ? K0b.ptr : K0a.ptr; }
    float4 *scur() { return cur_is_a ? S0a.ptr : S0b.ptr; }
    float4 *sother() { return cur_is_a ? S0b.ptr : S0a.ptr; }
    float *pcur() { return cur_is_a ? P0a.ptr : P0b.ptr; }
    float *pother() { return cur_is_a ? P0b.ptr : P0a.ptr; }
    ~dg_ctx()
    {
        for (auto *b : {&K0a, &K0b, &K1, &rtmp, &geo64, &ops64, &Dr64, &Ds64, &src, &lam, &scal, &fpart, &fxy, &wface})
            b->release();
        geo32.release();
        ops32.release();
        tcfrag.release();
        P0a.release();
        P0b.release();
        S0a.release();
        S0b.release();
        conn.release();
        fmask.release();
        flag.release();
        wall.release();
    }
};

namespace {

const char *const kWaitGaveUp =
    "a bounded device wait gave up (a fused step's grid barrier or a stage kernel's copy wait: "
    "the state is not valid; or the tcgen05 gradient kernel: its output is not valid)";

dg_status fail(dg_ctx *c, dg_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

dg_status cuda_fail(dg_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, DG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DG_CUDA(ctx, expr)                                        \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);  \
    } while (0)

template <typename real>
dg::Phys<real> make_phys(const dg_params &p, const double vw[2])
{
    dg::Phys<real> ph;
    ph.gamma = real(p.gamma);
    ph.gm1 = real(p.gamma - 1.0);
    ph.mu = real(p.mu);
    ph.gPr = real(p.gamma / p.Pr);
    ph.vw1 = real(vw ? vw[0] : 0.0);
    ph.vw2 = real(vw ? vw[1] : 0.0);
    double E = p.p_inf / (p.gamma - 1.0) + 0.5 * p.rho_inf * (p.u_inf * p.u_inf + p.v_inf * p.v_inf);
    ph.Uinf[0] = real(p.rho_inf);
    ph.Uinf[1] = real(p.rho_inf * p.u_inf);
    ph.Uinf[2] = real(p.rho_inf * p.v_inf);
    ph.Uinf[3] = real(E);
    ph.pinf = real(p.p_inf);
    ph.adiabatic = p.adiabatic_zero_heatflux;
    return ph;
}

size_t ndof(const dg_ctx *c) { return static_cast<size_t>(c->K) * 4 * c->ops.Np; }

// Manufactured steady solution of Sec. 3.1: source S = div F_c - div F_v at
// (x, y) for U = (w, w, w, w^2), w = sin(kappa (x+y)) + C2 (velocity (1,1),
// p = (gamma-1)(w^2 - w), only the heat-flux row of F_v is non-zero).
void manufactured_source(double x, double y, double kappa, double C2, const dg_params &p, double S[4])
{
    const double phi = kappa * (x + y), g1 = p.gamma - 1.0;
    const double w = std::sin(phi) + C2, dw = kappa * std::cos(phi);
    const double dp = g1 * (2.0 * w - 1.0) * dw;           // d/dx p = d/dy p
    S[0] = 2.0 * dw;                                         // d(rho v1)/dx + d(rho v2)/dy
    S[1] = 2.0 * dw + dp;                                    // d(w + p)/dx + d(w)/dy
    S[2] = S[1];
    const double dEp = dp + 2.0 * w * dw;                    // d(p + eps)/dx
    const double heat = 2.0 * p.mu * p.gamma / p.Pr * kappa * kappa * std::sin(phi);
    S[3] = 2.0 * dEp + heat;                                 // minus div of heat flux -mu g/Pr kappa^2 sin
}

// C1 (1+theta)^2 (d+1) of Eq. penalty_final, d = 2
double sigma_factor(const dg_params &p) { return p.C1 * (1.0 + p.theta) * (1.0 + p.theta) * 3.0; }

dg_status run_stage(dg_ctx *c, int s, double t, double dt, const double vw[2], int mode,
                    const double *in, double *out, double *rout)
{
    dg::StageParams sp{};
    sp.K0in = in;
    sp.K0out = out;
    sp.K1 = c->K1.ptr;
    sp.Rout = rout;
    sp.conn = c->conn.ptr;
    sp.fmask = c->fmask.ptr;
    const double *src = (c->source_kind != DG_SOURCE_NONE) ? c->src.ptr : nullptr;
    if (c->source_kind == DG_SOURCE_VORTEX) {
        if (s < 0) {
            // a single residual: the time-dependent source at its time, into slot 0
            DG_CUDA(c, dg::launch_vortex_source(c->prm.precision == DG_PRECISION_FP64, c->src_xy.ptr,
                                                c->K * c->ops.Np, c->ops.Np, c->vortex, &t, 1, c->src.ptr,
                                                c->stream));
            c->launches += 1;
        } else {
            // the step's five stage times were evaluated by dg_lsrk_step
            src = c->src.ptr + static_cast<size_t>(s) * ndof(c);
        }
    }
    sp.src = src;
    sp.Sin = c->scur();
    sp.Pin = c->pcur();
    sp.Sout = c->sother();
    sp.Pout = c->pother();
    sp.K = c->K;
    sp.A = (s >= 0) ? kRkA[s] : 0.0;
    sp.B = (s >= 0) ? kRkB[s] : 0.0;
    sp.dt = dt;
    sp.gm1 = c->prm.gamma - 1.0;
    sp.sig_fac = sigma_factor(c->prm);
    sp.theta = c->prm.theta;
    {
        const dg_params &q = c->prm;
        sp.uinf[0] = q.rho_inf;
        sp.uinf[1] = q.rho_inf * q.u_inf;
        sp.uinf[2] = q.rho_inf * q.v_inf;
        sp.uinf[3] = q.p_inf / (q.gamma - 1.0) + 0.5 * q.rho_inf * (q.u_inf * q.u_inf + q.v_inf * q.v_inf);
    }
    sp.mode = mode;
    sp.first_stage = (s == 0) ? 1 : 0;
    (void)t;
    cudaError_t e;
    if (c->prm.precision == DG_PRECISION_FP64) {
        sp.geo = c->geo64.ptr;
        sp.ops = c->ops64.ptr;
        e = dg::launch_stage_fp64(c->prm.p, c->shape, sp, make_phys<double>(c->prm, vw), c->stream);
    } else {
        sp.geo = c->geo32.ptr;
        sp.ops = (c->shape.variant == 3) ? static_cast<const void *>(c->tcfrag.ptr) : c->ops32.ptr;
        if (c->shape.variant == 3) {
            // its bounded copy waits report through the barrier flag
            sp.bar_err = c->bar_err.ptr;
            sp.bar_limit = c->bar_limit;
            c->copy_used = true;
            e = dg::launch_stage_tc(c->prm.p, false, false, c->shape, sp, make_phys<float>(c->prm, vw), c->stream);
        }
        else if (c->shape.variant == 2)
            e = dg::launch_stage_mixed2(c->prm.p, false, c->shape, sp, make_phys<float>(c->prm, vw), c->stream);
        else
            e = dg::launch_stage_mixed(c->prm.p, c->shape, sp, make_phys<float>(c->prm, vw), c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
    c->launches += 1;
    return DG_OK;
}

dg::AuxMesh aux_mesh(dg_ctx *c)
{
    dg::AuxMesh m;
    m.U = c->cur();
    m.geo = c->geo64.ptr;
    m.conn = c->conn.ptr;
    m.Dr = c->Dr64.ptr;
    m.Ds = c->Ds64.ptr;
    m.fmask = c->fmask.ptr;
    m.K = c->K;
    m.p = c->prm.p;
    return m;
}

}  // namespace

extern "C" {

dg_status dg_reference_operators(int p, double *r, double *s, double *Dr, double *Ds, double *LIFT,
                                 int32_t *Fmask)
{
    dg::RefOps o;
    if (!dg::build_reference_operators(p, o)) return DG_EINVAL;
    if (r) std::copy(o.r.begin(), o.r.end(), r);
    if (s) std::copy(o.s.begin(), o.s.end(), s);
    if (Dr) std::copy(o.Dr.begin(), o.Dr.end(), Dr);
    if (Ds) std::copy(o.Ds.begin(), o.Ds.end(), Ds);
    if (LIFT) std::copy(o.LIFT.begin(), o.LIFT.end(), LIFT);
    if (Fmask)
        for (size_t i = 0; i < o.Fmask.size(); ++i) Fmask[i] = o.Fmask[i];
    return DG_OK;
}

dg_status dg_create(const dg_params *params, void *cuda_stream, dg_ctx **out)
{
    if (!out) return DG_EINVAL;
    *out = nullptr;
    if (!params) return DG_EINVAL;
    const dg_params &p = *params;
    if (p.p < 1 || p.p > 6 || !(p.gamma > 1.0) || !(p.Pr > 0.0) || !(p.mu >= 0.0) || !(p.C1 >= 0.0) ||
        !(p.rho_inf > 0.0) || !(p.p_inf > 0.0) ||
        (p.precision != DG_PRECISION_FP64 && p.precision != DG_PRECISION_MIXED))
        return DG_EINVAL;
    if (!(p.theta >= -1.0 && p.theta <= 1.0)) return DG_EINVAL;
    dg_ctx *c = new dg_ctx();
    c->prm = p;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!dg::build_reference_operators(p.p, c->ops)) {
        delete c;
        return DG_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        delete c;
        return DG_ECUDA;
    }
    const int Np = c->ops.Np, NF = 3 * c->ops.Nfp;
    std::vector<double> o64;
    o64.insert(o64.end(), c->ops.Dr.begin(), c->ops.Dr.end());
    o64.insert(o64.end(), c->ops.Ds.begin(), c->ops.Ds.end());
    o64.insert(o64.end(), c->ops.LIFT.begin(), c->ops.LIFT.end());
    o64.insert(o64.end(), c->ops.Wr.begin(), c->ops.Wr.end());
    o64.insert(o64.end(), c->ops.Ws.begin(), c->ops.Ws.end());
    {
        // over-integration operators, used by the FP64 kernel when enabled
        dg::OverintOps oi;
        if (!dg::build_overint_operators(c->ops, dg::overint_degree(p.p), oi)) {
            delete c;
            return DG_EINVAL;
        }
        for (const auto *v : {&oi.Vq, &oi.Vqr, &oi.Vqs, &oi.Sr, &oi.Ss}) o64.insert(o64.end(), v->begin(), v->end());
    }
    std::vector<float> o32(o64.begin(), o64.end());
    if (c->ops64.alloc(o64.size()) != cudaSuccess || c->ops32.alloc(o32.size()) != cudaSuccess ||
        c->Dr64.alloc(Np * Np) != cudaSuccess || c->Ds64.alloc(Np * Np) != cudaSuccess ||
        c->fmask.alloc(NF) != cudaSuccess || c->flag.alloc(1) != cudaSuccess || c->bar_err.alloc(1) != cudaSuccess ||
        c->scal.alloc(4) != cudaSuccess || c->wface.alloc(c->ops.Nfp) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DG_ECUDA;
    }
    cudaMemset(c->bar_err.ptr, 0, sizeof(int));
    cudaMemcpy(c->ops64.ptr, o64.data(), o64.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->ops32.ptr, o32.data(), o32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (dg::stage_tc_supported(p.p)) {
        std::vector<float> frag;
        dg::build_tc_fragments(Np, NF, c->ops.Dr.data(), c->ops.Ds.data(), c->ops.LIFT.data(), c->ops.Wr.data(),
                               c->ops.Ws.data(), frag);
        if (c->tcfrag.alloc(frag.size()) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return DG_ECUDA;
        }
        cudaMemcpy(c->tcfrag.ptr, frag.data(), frag.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    cudaMemcpy(c->Dr64.ptr, c->ops.Dr.data(), Np * Np * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->Ds64.ptr, c->ops.Ds.data(), Np * Np * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->fmask.ptr, c->ops.Fmask.data(), NF * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(c->wface.ptr, c->ops.wface.data(), c->ops.Nfp * sizeof(double), cudaMemcpyHostToDevice);
    if (cudaGetLastError() != cudaSuccess) {
        delete c;
        return DG_ECUDA;
    }
    *out = c;
    return DG_OK;
}

dg_status dg_destroy(dg_ctx *ctx)
{
    delete ctx;
    return DG_OK;
}

const char *dg_last_error(const dg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t dg_kernel_launches(const dg_ctx *ctx) { return ctx ? ctx->launches : 0; }

dg_status dg_set_overintegration(dg_ctx *c, int on)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (on && (c->prm.precision != DG_PRECISION_FP64 || c->prm.theta != 0.0))
        return fail(c, DG_EUNSUPPORTED, "over-integration is implemented in the FP64 IIP kernel");
    c->overint = on != 0;
    if (c->K > 0 && c->prm.precision == DG_PRECISION_FP64) {
        cudaError_t e = dg::stage_shape_fp64(c->prm.p, c->K, false, c->shape, c->overint);
        if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel configuration");
    }
    return DG_OK;
}

int dg_overint_degree(int p) { return (p >= 1 && p <= 6) ? dg::overint_degree(p) : 0; }

dg_status dg_set_fused_steps(dg_ctx *c, int on)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (on && (c->prm.precision != DG_PRECISION_MIXED || c->prm.theta != 0.0))
        return fail(c, DG_EUNSUPPORTED, "fused steps use the mixed-precision IIP kernels");
    if (on && !c->bar.ptr) {
        DG_CUDA(c, c->bar.alloc(2));
        DG_CUDA(c, cudaMemset(c->bar.ptr, 0, 2 * sizeof(unsigned)));
    }
    c->fused = on != 0;
    return DG_OK;
}

dg_status dg_set_barrier_limit(dg_ctx *c, uint32_t waits)
{
    if (!c) return DG_EINVAL;
    c->bar_limit = waits;
    return DG_OK;
}

dg_status dg_barrier_status(dg_ctx *c)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!c->bar_used && !c->copy_used) return DG_OK;
    int e = 0;
    DG_CUDA(c, cudaMemcpyAsync(&e, c->bar_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->bar_used = false;
    c->copy_used = false;
    if (e) {
        DG_CUDA(c, cudaMemset(c->bar_err.ptr, 0, sizeof(int)));
        return fail(c, DG_ETIMEOUT, kWaitGaveUp);
    }
    return DG_OK;
}

dg_status dg_set_stage_variant(dg_ctx *c, int variant)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (variant < 0 || variant > 3) return fail(c, DG_EINVAL, "variant must be 0, 1, 2 or 3");
    if (variant >= 2 && c->prm.precision != DG_PRECISION_MIXED)
        return fail(c, DG_EUNSUPPORTED, "the two-node and tensor-core kernels are mixed-precision kernels");
    if (variant == 2 && c->prm.theta != 0.0)
        return fail(c, DG_EUNSUPPORTED, "the two-node kernel is an IIP kernel");
    if (variant == 3 && !dg::stage_tc_supported(c->prm.p))
        return fail(c, DG_EUNSUPPORTED, "the tensor-core kernel covers p <= 6");
    c->variant_req = variant;
    c->tuned = (variant != 0);
    if (c->K > 0 && c->prm.precision == DG_PRECISION_MIXED)
        c->shape = (variant == 3) ? c->shape3 : (variant == 2) ? c->shape2 : c->shape1;
    return DG_OK;
}

int dg_stage_variant(const dg_ctx *c) { return c ? c->shape.variant : 0; }

dg_status dg_set_mesh(dg_ctx *c, int64_t Nv, const double *vx, const double *vy, int64_t K,
                      const int32_t *EToV, const int32_t *EToE, const int32_t *EToF, const int32_t *bc)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    dg::MeshArrays ma;
    std::string msg;
    const int mst = dg::build_mesh(c->ops, Nv, vx, vy, K, EToV, EToE, EToF, bc, ma, msg);
    if (mst == dg::MESH_EINVAL) return fail(c, DG_EINVAL, msg);
    if (mst != dg::MESH_OK) return fail(c, DG_EMESH, msg);
    const int Np = c->ops.Np;
    std::vector<double> &geo = ma.geo;
    std::vector<int4> &conn = ma.conn;
    std::vector<int2> &walls = ma.walls;
    std::vector<double> &wxy = ma.wxy;
    // --- device buffers
    c->K = K;
    const size_t nd = static_cast<size_t>(K) * 4 * Np;
    DG_CUDA(c, c->K0a.alloc(nd));
    DG_CUDA(c, c->K0b.alloc(nd));
    DG_CUDA(c, c->K1.alloc(nd));
    DG_CUDA(c, c->geo64.alloc(geo.size()));
    DG_CUDA(c, c->conn.alloc(K));
    DG_CUDA(c, c->lam.alloc(K));
    DG_CUDA(c, cudaMemcpy(c->geo64.ptr, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
    DG_CUDA(c, cudaMemcpy(c->conn.ptr, conn.data(), K * sizeof(int4), cudaMemcpyHostToDevice));
    if (c->prm.precision == DG_PRECISION_MIXED) {
        std::vector<float> g32(geo.begin(), geo.end());
        DG_CUDA(c, c->geo32.alloc(g32.size()));
        DG_CUDA(c, cudaMemcpy(c->geo32.ptr, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice));
        const size_t np = static_cast<size_t>(K) * Np, npp = static_cast<size_t>(K) * dg::pressure_row(c->prm.p);
        DG_CUDA(c, c->S0a.alloc(np));
        DG_CUDA(c, c->S0b.alloc(np));
        DG_CUDA(c, c->P0a.alloc(npp));
        DG_CUDA(c, c->P0b.alloc(npp));
        DG_CUDA(c, cudaMemsetAsync(c->S0a.ptr, 0, np * sizeof(float4), c->stream));
        DG_CUDA(c, cudaMemsetAsync(c->S0b.ptr, 0, np * sizeof(float4), c->stream));
        DG_CUDA(c, cudaMemsetAsync(c->P0a.ptr, 0, npp * sizeof(float), c->stream));
        DG_CUDA(c, cudaMemsetAsync(c->P0b.ptr, 0, npp * sizeof(float), c->stream));
    }
    c->nwall = static_cast<int>(walls.size());
    if (c->nwall > 0) {
        DG_CUDA(c, c->wall.alloc(walls.size()));
        DG_CUDA(c, c->fxy.alloc(wxy.size()));
        DG_CUDA(c, c->fpart.alloc(walls.size() * 3));
        DG_CUDA(c, cudaMemcpy(c->wall.ptr, walls.data(), walls.size() * sizeof(int2), cudaMemcpyHostToDevice));
        DG_CUDA(c, cudaMemcpy(c->fxy.ptr, wxy.data(), wxy.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    DG_CUDA(c, cudaMemsetAsync(c->K0a.ptr, 0, nd * sizeof(double), c->stream));
    DG_CUDA(c, cudaMemsetAsync(c->K1.ptr, 0, nd * sizeof(double), c->stream));
    c->cur_is_a = true;
    c->vx.assign(vx, vx + Nv);
    c->vy.assign(vy, vy + Nv);
    c->EToV.assign(EToV, EToV + K * 3);
    c->geo64h.swap(geo);
    c->source_kind = DG_SOURCE_NONE;
    const bool th = c->prm.theta != 0.0;
    cudaError_t e = (c->prm.precision == DG_PRECISION_FP64) ? dg::stage_shape_fp64(c->prm.p, K, th, c->shape, c->overint)
                                                             : dg::stage_shape_mixed(c->prm.p, K, th, c->shape);
    if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel configuration");
    c->shape1 = c->shape;
    c->tuned = false;
    c->fshape_variant = 0;           // the cooperative grid is sized per mesh
    c->has_tc = false;
    if (c->prm.precision == DG_PRECISION_MIXED) {
        if (!th) {
            e = dg::stage_shape_mixed2(c->prm.p, K, false, c->shape2);
            if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel configuration");
            if (c->variant_req == 2) c->shape = c->shape2;
        }
        if (dg::stage_tc_supported(c->prm.p)) {
            e = dg::stage_shape_tc(c->prm.p, K, false, false, c->shape3, th);
            if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel configuration");
            c->has_tc = true;
            if (c->variant_req == 3) c->shape = c->shape3;
        }
    }
    return DG_OK;
}

dg_status dg_node_coords(const dg_ctx *c, double *x, double *y)
{
    if (!c || !x || !y || c->K < 1) return DG_EINVAL;
    const int Np = c->ops.Np;
    for (long long k = 0; k < c->K; ++k) {
        int32_t v0 = c->EToV[k * 3], v1 = c->EToV[k * 3 + 1], v2 = c->EToV[k * 3 + 2];
        for (int i = 0; i < Np; ++i) {
            double r = c->ops.r[i], s = c->ops.s[i];
            x[k * Np + i] = 0.5 * (-(r + s) * c->vx[v0] + (1 + r) * c->vx[v1] + (1 + s) * c->vx[v2]);
            y[k * Np + i] = 0.5 * (-(r + s) * c->vy[v0] + (1 + r) * c->vy[v1] + (1 + s) * c->vy[v2]);
        }
    }
    return DG_OK;
}

dg_status dg_set_state(dg_ctx *c, const double *U, int on_device)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!U || c->K < 1) return fail(c, DG_EINVAL, "null state or no mesh");
    const size_t nd = ndof(c);
    c->cur_is_a = true;
    DG_CUDA(c, cudaMemcpyAsync(c->K0a.ptr, U, nd * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    DG_CUDA(c, cudaMemsetAsync(c->K1.ptr, 0, nd * sizeof(double), c->stream));
    if (c->prm.precision == DG_PRECISION_MIXED) {
        DG_CUDA(c, dg::launch_make_shadow(c->prm.p, c->K0a.ptr, c->K, c->prm.gamma - 1.0, c->S0a.ptr, c->P0a.ptr,
                                          c->stream));
        c->launches += 1;
    }
    if (!on_device) DG_CUDA(c, cudaStreamSynchronize(c->stream));
    return DG_OK;
}

dg_status dg_get_state(dg_ctx *c, double *U, int on_device)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (on_device && c->bar_used) {
        dg_status bs = dg_barrier_status(c);
        if (bs != DG_OK) return bs;
    }
    if (!U || c->K < 1) return fail(c, DG_EINVAL, "null state or no mesh");
    // host output: the error flag of the bounded device waits comes back with
    // the state, under the one synchronisation (device output stays
    // asynchronous after plain stage launches)
    const bool check = !on_device && (c->bar_used || c->copy_used);
    int e = 0;
    if (check) DG_CUDA(c, cudaMemcpyAsync(&e, c->bar_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaMemcpyAsync(U, c->cur(), ndof(c) * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) DG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (check) {
        c->bar_used = false;
        c->copy_used = false;
        if (e) {
            DG_CUDA(c, cudaMemset(c->bar_err.ptr, 0, sizeof(int)));
            return fail(c, DG_ETIMEOUT, kWaitGaveUp);
        }
    }
    return DG_OK;
}

dg_status dg_set_source(dg_ctx *c, int kind, const double *params)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (c->K < 1) return fail(c, DG_EINVAL, "no mesh");
    if (kind == DG_SOURCE_NONE) {
        c->source_kind = kind;
        return DG_OK;
    }
    if ((kind != DG_SOURCE_MANUFACTURED && kind != DG_SOURCE_VORTEX) || !params)
        return fail(c, DG_EINVAL, "unknown source kind");
    const int Np = c->ops.Np;
    std::vector<double> x(static_cast<size_t>(c->K) * Np), y(x.size());
    dg_node_coords(c, x.data(), y.data());
    if (kind == DG_SOURCE_VORTEX) {
        for (int q = 0; q < 6; ++q)
            if (!std::isfinite(params[q])) return fail(c, DG_EINVAL, "vortex source parameters must be finite");
        if (!(params[3] > 0.0)) return fail(c, DG_EINVAL, "vortex source period L must be > 0");
        const double pi = 3.14159265358979323846;
        c->vortex = dg::VortexSource{params[0], params[1], params[2], params[3], params[4], params[5],
                                     c->prm.mu, c->prm.Pr, 1.0 / params[3], params[0] / (2.0 * pi),
                                     params[0] * params[0] / (2.0 * pi * pi), 1.0 / c->prm.Pr};
        DG_CUDA(c, c->src_xy.alloc(2 * x.size()));
        DG_CUDA(c, cudaMemcpy(c->src_xy.ptr, x.data(), x.size() * sizeof(double), cudaMemcpyHostToDevice));
        DG_CUDA(c, cudaMemcpy(c->src_xy.ptr + x.size(), y.data(), y.size() * sizeof(double),
                              cudaMemcpyHostToDevice));
        DG_CUDA(c, c->src.alloc(5 * ndof(c)));         // one array per stage time of a step
        c->source_kind = kind;
        return DG_OK;
    }
    std::vector<double> S(ndof(c));
    for (long long k = 0; k < c->K; ++k)
        for (int i = 0; i < Np; ++i) {
            double s4[4];
            manufactured_source(x[k * Np + i], y[k * Np + i], params[0], params[1], c->prm, s4);
            for (int q = 0; q < 4; ++q) S[(k * 4 + q) * Np + i] = s4[q];
        }
    DG_CUDA(c, c->src.alloc(S.size()));
    DG_CUDA(c, cudaMemcpy(c->src.ptr, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice));
    c->source_kind = kind;
    return DG_OK;
}

// Mixed path, first use: time every available stage-kernel shape (one and
// two nodes per thread, tensor-core warp tiles; the two-node shape is IIP
// only) on the current state in residual-only mode and keep the fastest.
static dg_status tune_stage(dg_ctx *c, const double vw[2])
{
    if (c->tuned || c->prm.precision != DG_PRECISION_MIXED || c->variant_req != 0) {
        c->tuned = true;
        return DG_OK;
    }
    if (c->rtmp.n != ndof(c)) DG_CUDA(c, c->rtmp.alloc(ndof(c)));
    // events destroyed on every return path
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events()
        {
            for (auto &x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    DG_CUDA(c, cudaEventCreate(&ev.e[0]));
    DG_CUDA(c, cudaEventCreate(&ev.e[1]));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    float best = 0.f;
    dg::LaunchShape pick = c->shape1;
    for (const dg::LaunchShape *cand : {&c->shape1, &c->shape2, &c->shape3}) {
        if (cand == &c->shape3 && !c->has_tc) continue;
        if (cand == &c->shape2 && c->prm.theta != 0.0) continue;
        c->shape = *cand;
        float ms = 0.f;
        for (int rep = 0; rep < 5; ++rep) {
            if (rep == 2) DG_CUDA(c, cudaEventRecord(e0, c->stream));
            dg_status st = run_stage(c, -1, 0.0, 0.0, vw, dg::STAGE_RHS_ONLY, c->cur(), nullptr, c->rtmp.ptr);
            if (st != DG_OK) return st;
        }
        DG_CUDA(c, cudaEventRecord(e1, c->stream));
        DG_CUDA(c, cudaEventSynchronize(e1));
        DG_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (cand == &c->shape1 || ms < best) {
            best = ms;
            pick = *cand;
        }
    }
    c->shape = pick;
    c->tuned = true;
    return DG_OK;
}

dg_status dg_rhs(dg_ctx *c, double t, const double vw[2], double *dUdt, int on_device)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!dUdt || c->K < 1) return fail(c, DG_EINVAL, "null output or no mesh");
    double *out = dUdt;
    if (!on_device) {
        if (c->rtmp.n != ndof(c)) DG_CUDA(c, c->rtmp.alloc(ndof(c)));
        out = c->rtmp.ptr;
    }
    dg_status st = run_stage(c, -1, t, 0.0, vw, dg::STAGE_RHS_ONLY, c->cur(), nullptr, out);
    if (st != DG_OK) return st;
    if (!on_device) {
        DG_CUDA(c, cudaMemcpyAsync(dUdt, out, ndof(c) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        DG_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return DG_OK;
}

// One step as a single cooperative launch of the mixed IIP kernel (fused
// stages); the barrier counters are reset before every launch.
static dg_status run_fused_step(dg_ctx *c, double dt, const double vw[2])
{
    if (c->fshape_variant != c->shape.variant) {
        cudaError_t e = (c->shape.variant == 3)
                            ? dg::stage_shape_tc(c->prm.p, c->K, false, true, c->fshape)
                            : dg::stage_shape_mixed_fused(c->prm.p, c->shape.variant, false, c->K, c->fshape);
        if (e != cudaSuccess) return cuda_fail(c, e, "fused stage kernel configuration");
        c->fshape_variant = c->shape.variant;
    }
    dg::StageParams sp{};
    sp.K0in = c->cur();
    sp.K0out = c->other();
    sp.K1 = c->K1.ptr;
    sp.conn = c->conn.ptr;
    sp.fmask = c->fmask.ptr;
    sp.src = (c->source_kind != DG_SOURCE_NONE) ? c->src.ptr : nullptr;
    sp.Sin = c->scur();
    sp.Pin = c->pcur();
    sp.Sout = c->sother();
    sp.Pout = c->pother();
    sp.K = c->K;
    for (int i = 0; i < 5; ++i) {
        sp.A5[i] = kRkA[i];
        sp.B5[i] = kRkB[i];
    }
    sp.A = kRkA[0];
    sp.B = kRkB[0];
    sp.dt = dt;
    sp.gm1 = c->prm.gamma - 1.0;
    sp.sig_fac = sigma_factor(c->prm);
    sp.mode = dg::STAGE_UPDATE;
    sp.first_stage = 1;
    sp.geo = c->geo32.ptr;
    sp.ops = (c->fshape.variant == 3) ? static_cast<const void *>(c->tcfrag.ptr) : c->ops32.ptr;
    sp.bar = c->bar.ptr;
    sp.bar_err = c->bar_err.ptr;
    sp.bar_limit = c->bar_limit;
    DG_CUDA(c, cudaMemsetAsync(c->bar.ptr, 0, 2 * sizeof(unsigned), c->stream));
    if (c->fshape.variant == 3)
        DG_CUDA(c, dg::launch_stage_tc(c->prm.p, false, true, c->fshape, sp, make_phys<float>(c->prm, vw), c->stream));
    else
        DG_CUDA(c, dg::launch_stage_mixed_fused(c->prm.p, false, c->fshape, sp, make_phys<float>(c->prm, vw), c->stream));
    c->launches += 1;
    c->cur_is_a = !c->cur_is_a;   // five swaps
    c->bar_used = true;
    return DG_OK;
}

dg_status dg_lsrk_step(dg_ctx *c, double t, double dt, const double vw[2])
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (c->K < 1) return fail(c, DG_EINVAL, "no mesh");
    if (!std::isfinite(dt) || !std::isfinite(t)) return fail(c, DG_EINVAL, "t and dt must be finite");
    if (!c->tuned) {
        dg_status st = tune_stage(c, vw);
        if (st != DG_OK) return st;
    }
    // a time-dependent source is evaluated at the five stage times in one
    // launch before the stages, which then run as five launches
    if (c->fused && c->source_kind != DG_SOURCE_VORTEX) return run_fused_step(c, dt, vw);
    if (c->source_kind == DG_SOURCE_VORTEX) {
        double ts[5];
        for (int s = 0; s < 5; ++s) ts[s] = t + kRkC[s] * dt;
        DG_CUDA(c, dg::launch_vortex_source(c->prm.precision == DG_PRECISION_FP64, c->src_xy.ptr, c->K * c->ops.Np,
                                            c->ops.Np, c->vortex, ts, 5, c->src.ptr, c->stream));
        c->launches += 1;
    }
    for (int s = 0; s < 5; ++s) {
        dg_status st = run_stage(c, s, t + kRkC[s] * dt, dt, vw, dg::STAGE_UPDATE, c->cur(), c->other(), nullptr);
        if (st != DG_OK) return st;
        c->cur_is_a = !c->cur_is_a;
    }
    return DG_OK;
}

dg_status dg_lsrk_steps(dg_ctx *c, double t, double dt, const double vw[2], int nsteps)
{
    for (int n = 0; n < nsteps; ++n) {
        dg_status st = dg_lsrk_step(c, t + n * dt, dt, vw);
        if (st != DG_OK) return st;
    }
    return DG_OK;
}

dg_status dg_compute_dt(dg_ctx *c, double cfl, const double vw[2], double *dt)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!dt || c->K < 1 || !(cfl > 0.0)) return fail(c, DG_EINVAL, "need dt pointer, mesh and cfl > 0");
    dg::Phys<double> ph = make_phys<double>(c->prm, vw);
    DG_CUDA(c, dg::launch_dt_lambda(aux_mesh(c), ph, sigma_factor(c->prm), c->lam.ptr, c->stream));
    DG_CUDA(c, dg::launch_max_reduce(c->lam.ptr, c->K, c->scal.ptr, c->stream));
    c->launches += 2;
    double lam = 0.0;
    DG_CUDA(c, cudaMemcpyAsync(&lam, c->scal.ptr, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!std::isfinite(lam) || !(lam > 0.0)) return fail(c, DG_ENONFINITE, "time-step bound is not finite");
    *dt = cfl / lam;
    return DG_OK;
}

dg_status dg_wall_forces(dg_ctx *c, const double xc[2], double out[3])
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!out || c->K < 1) return fail(c, DG_EINVAL, "null output or no mesh");
    if (c->nwall == 0) {
        out[0] = out[1] = out[2] = 0.0;
        return DG_OK;
    }
    double x0 = xc ? xc[0] : 0.0, y0 = xc ? xc[1] : 0.0;
    dg::Phys<double> ph = make_phys<double>(c->prm, nullptr);
    DG_CUDA(c, dg::launch_wall_force_faces(aux_mesh(c), ph, c->wall.ptr, c->fxy.ptr, c->wface.ptr, c->nwall,
                                           x0, y0, c->fpart.ptr, c->stream));
    DG_CUDA(c, dg::launch_sum3(c->fpart.ptr, c->nwall, c->scal.ptr, c->stream));
    c->launches += 2;
    DG_CUDA(c, cudaMemcpyAsync(out, c->scal.ptr, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaStreamSynchronize(c->stream));
    return DG_OK;
}

dg_status dg_check_finite(dg_ctx *c, int *ok)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    {
        dg_status bs = dg_barrier_status(c);
        if (bs != DG_OK) return bs;
    }
    if (!ok || c->K < 1) return fail(c, DG_EINVAL, "null output or no mesh");
    DG_CUDA(c, cudaMemsetAsync(c->flag.ptr, 0, sizeof(int), c->stream));
    DG_CUDA(c, dg::launch_nonfinite(c->cur(), static_cast<long long>(ndof(c)), c->flag.ptr, c->stream));
    c->launches += 1;
    int f = 0;
    DG_CUDA(c, cudaMemcpyAsync(&f, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaStreamSynchronize(c->stream));
    *ok = f ? 0 : 1;
    return DG_OK;
}

dg_status dg_broken_gradient(dg_ctx *c, double *gx, double *gy, int on_device, int impl)
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!gx || !gy || c->K < 1) return fail(c, DG_EINVAL, "null output or no mesh");
    if (impl != 0 && impl != 1) return fail(c, DG_EINVAL, "impl must be 0 (FP64) or 1 (tcgen05)");
    const size_t n = ndof(c);
    double *ox = gx, *oy = gy;
    if (!on_device) {
        if (c->gtmp.n != 2 * n) DG_CUDA(c, c->gtmp.alloc(2 * n));
        ox = c->gtmp.ptr;
        oy = c->gtmp.ptr + n;
    }
    dg::GradTc05Args a{};
    a.U = c->cur();
    a.Dr = c->ops.Dr.data();
    a.Ds = c->ops.Ds.data();
    a.Dr_dev = c->Dr64.ptr;
    a.Ds_dev = c->Ds64.ptr;
    a.geo = c->geo64.ptr;
    a.K = c->K;
    a.gx = ox;
    a.gy = oy;
    a.wait_limit = 1u << 20;
    if (impl == 1) {
        const size_t nf = dg::grad_tc05_bimg_floats(c->prm.p);
        if (c->gimg.n != nf) {
            DG_CUDA(c, c->gimg.alloc(nf));
            c->gimg_ready = false;
        }
        if (!c->bar_err.ptr) {
            DG_CUDA(c, c->bar_err.alloc(1));
            DG_CUDA(c, cudaMemset(c->bar_err.ptr, 0, sizeof(int)));
        }
        a.bimg = c->gimg.ptr;
        a.upload_ops = !c->gimg_ready;   // the operators are fixed by p: one upload per context
        a.err = c->bar_err.ptr;        // reported by dg_barrier_status, as for fused steps
        c->bar_used = true;
    }
    DG_CUDA(c, dg::launch_broken_gradient(c->prm.p, impl, a, c->stream));
    if (impl == 1) c->gimg_ready = true;
    c->launches += 1;
    if (!on_device) {
        DG_CUDA(c, cudaMemcpyAsync(gx, ox, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        DG_CUDA(c, cudaMemcpyAsync(gy, oy, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        DG_CUDA(c, cudaStreamSynchronize(c->stream));
        return dg_barrier_status(c);
    }
    return DG_OK;
}

dg_status dg_rigid_step(const double coeff[3], double F, double dt, double state[3], double *v_b)
{
    if (!coeff || !state || !v_b || !(dt > 0.0)) return DG_EINVAL;
    double y = state[0], yd = state[1], ydd = state[2], vb = 0.0;
    if (!dg::newmark_step(coeff[0], coeff[1], coeff[2], F, dt, y, yd, ydd, vb)) return DG_EINVAL;
    *v_b = vb;
    state[0] = y;
    state[1] = yd;
    state[2] = ydd;
    return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Wall forces with library-resident scratch (no device allocation).
//
// dg_wall_forces sums per-face partials in a buffer that belongs to the mesh.
// This variant writes the partials and the summed triple into a fixed array
// compiled into the library instead, so the call itself never asks the CUDA
// allocator for memory.  The array is a host-side symbol: host code must not
// hand its name to a kernel; its device address is looked up once per device
// with cudaGetSymbolAddress and cached.
namespace {

constexpr int kNoallocMaxWallFaces = DG_NOALLOC_MAX_WALL_FACES;
constexpr int kNoallocMaxDevices = 64;

// nwall*3 partials followed by the 3-entry result; every call overwrites the
// entries it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_force_scratch[kNoallocMaxWallFaces * 3 + 4];

std::mutex g_noalloc_mutex;
double *g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device, with that device current).
dg_status noalloc_scratch(dg_ctx *c, double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(c, DG_EUNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_force_scratch);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_force_scratch)");
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return DG_OK;
}

}  // namespace

extern "C" dg_status dg_wall_forces_noalloc(dg_ctx *c, const double xc[2], double out[3])
{
    if (!c) return DG_EINVAL;
    c->err.clear();
    if (!out || c->K < 1) return fail(c, DG_EINVAL, "null output or no mesh");
    if (c->nwall > kNoallocMaxWallFaces)
        return fail(c, DG_EINVAL, "dg_wall_forces_noalloc: mesh has " + std::to_string(c->nwall) +
                                      " wall faces, more than the fixed scratch holds (" +
                                      std::to_string(kNoallocMaxWallFaces) + "); use dg_wall_forces");
    if (c->nwall == 0) {
        out[0] = out[1] = out[2] = 0.0;
        return DG_OK;
    }
    double *scratch = nullptr;
    dg_status st = noalloc_scratch(c, &scratch);
    if (st != DG_OK) return st;
    double *partial = scratch;
    double *result = scratch + static_cast<size_t>(kNoallocMaxWallFaces) * 3;
    double x0 = xc ? xc[0] : 0.0, y0 = xc ? xc[1] : 0.0;
    dg::Phys<double> ph = make_phys<double>(c->prm, nullptr);
    DG_CUDA(c, dg::launch_wall_force_faces(aux_mesh(c), ph, c->wall.ptr, c->fxy.ptr, c->wface.ptr, c->nwall,
                                           x0, y0, partial, c->stream));
    DG_CUDA(c, dg::launch_sum3(partial, c->nwall, result, c->stream));
    c->launches += 2;
    DG_CUDA(c, cudaMemcpyAsync(out, result, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(c, cudaStreamSynchronize(c->stream));
    return DG_OK;
}
