// batch.cu -- host side of the batch C ABI (include/dg_batch.h): many
// independent cylinder / VIV cases advanced together, Algorithm 3 per case
// on the device, optionally replayed from a CUDA graph.
//
// Layout: cases are grouped by polynomial degree.  A group stores the
// elements of its cases back to back ([K_g][4][Np] FP64 state, FP32 copies,
// geometry, connectivity with neighbour indices offset by the case's first
// element).  A tile table lists (first element, count, case) for every tile
// of the mixed stage kernel, so no tile straddles two cases and the kernel
// reads each case's dt, v_b and viscosity once per tile.  The time-step
// bound Lambda_K of every element of every group goes into one array with a
// contiguous range per case; wall-face partial forces likewise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dg_batch.h"
#include "devbuf.h"
#include "dg_stage.cuh"
#include "launch.h"
#include "mesh.h"
#include "refops.h"
#include "rk.h"

namespace {

using dg::DevBuf;

struct Group {
    int p = 0;
    dg::RefOps ops;
    long long K = 0;                 // elements of all cases of this degree
    long long lam_base = 0;          // first entry in the batch's Lambda_K array
    int wall_base = 0;               // first entry in the batch's wall partials
    int nwall = 0;
    long long ntiles = 0, ntiles2 = 0, ntiles3 = 0;
    dg::LaunchShape shape, shape2;   // one / two nodes per thread
    dg::LaunchShape shape3;          // tensor-core warp tiles (p <= 6)
    bool has_tc = false;
    int variant = 1;
    float t_tc = 0.f;                // the tuner's time of the tensor-core shape (ms, 3 launches), 0 if not timed
    dg::LaunchShape fshape;          // fused steps: cooperative launch of the chosen shape
    int fshape_variant = 0;
    DevBuf<unsigned> bar;            // fused steps: barrier words of this group (+ tile counters)
    DevBuf<double> K0a, K0b, K1, geo64, Dr64, Ds64, wface, fxy;
    DevBuf<float> geo32, ops32, P0a, P0b;
    DevBuf<float4> S0a, S0b;
    DevBuf<int4> conn, tiles, tiles2, tiles3;
    DevBuf<float> tcfrag;            // operator table of the tensor-core shape
    DevBuf<int> fmask, elem_case;
    DevBuf<int2> walls;
};

struct CaseHost {
    int group = 0;
    long long off = 0;               // first element within the group
    long long K = 0;
    int p = 0;
    std::vector<double> vx, vy;
    std::vector<int32_t> EToV;
};

}  // namespace

struct dg_batch {
    dg_params prm{};
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    std::vector<Group> groups;
    std::vector<CaseHost> cases;
    std::vector<dg::BatchCase> init;
    DevBuf<dg::BatchCase> dcases;
    DevBuf<double> lam, fpart;
    DevBuf<double> fixed_dt;         // per-case steps set by dg_batch_set_fixed_dt
    bool use_fixed = false;
    DevBuf<long long> seg;
    DevBuf<int> wseg, counter;
    DevBuf<unsigned> ticket;         // blocks done in the force-sum kernel (advances the history row)
    bool cur_is_a = true;
    bool forces_stale = true;
    int variant_req = 0;             // 0: tuned per degree group on the first run; 1, 2: forced
    bool tuned = false;
    bool fused = false;              // one cooperative launch per degree group and step
    bool fused_all = false;          // ... or one cooperative launch for all degree groups
    std::vector<unsigned> all_nblk;  // fused_all: blocks of each group (empty until sized)
    size_t all_smem = 0;
    DevBuf<int> bar_err;
    unsigned bar_limit = 1u << 24;
    // graphs: [0] starts from buffers a, [1] from buffers b
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_launches = 0;
    double graph_cfl = 0.0;
    double *graph_hist = nullptr;
    int graph_rows = 0;

    ~dg_batch()
    {
        drop_graphs();
        if (stream) cudaStreamDestroy(stream);
    }
    void drop_graphs()
    {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
};

namespace {

thread_local std::string g_create_err;     // message of the last failed dg_batch_create

dg_status bfail(dg_batch *b, dg_status st, const std::string &msg)
{
    if (b) b->err = msg;
    return st;
}

dg_status bcuda(dg_batch *b, cudaError_t e, const char *where)
{
    return bfail(b, DG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define B_CUDA(b, expr)                                          \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return bcuda(b, e_, #expr);       \
    } while (0)

template <typename real>
dg::Phys<real> phys_of(const dg_params &p)
{
    dg::Phys<real> ph;
    ph.gamma = real(p.gamma);
    ph.gm1 = real(p.gamma - 1.0);
    ph.mu = real(0);                 // per case, set in the kernels
    ph.gPr = real(p.gamma / p.Pr);
    ph.vw1 = real(0);
    ph.vw2 = real(0);                // per case
    const double E = p.p_inf / (p.gamma - 1.0) + 0.5 * p.rho_inf * (p.u_inf * p.u_inf + p.v_inf * p.v_inf);
    ph.Uinf[0] = real(p.rho_inf);
    ph.Uinf[1] = real(p.rho_inf * p.u_inf);
    ph.Uinf[2] = real(p.rho_inf * p.v_inf);
    ph.Uinf[3] = real(E);
    ph.pinf = real(p.p_inf);
    ph.adiabatic = p.adiabatic_zero_heatflux;
    return ph;
}

double sigma_factor(const dg_params &p) { return p.C1 * (1.0 + p.theta) * (1.0 + p.theta) * 3.0; }

dg::AuxMesh aux_of(const dg_batch *b, const Group &g)
{
    dg::AuxMesh m;
    m.U = b->cur_is_a ? g.K0a.ptr : g.K0b.ptr;
    m.elem_case = g.elem_case.ptr;
    m.cases = b->dcases.ptr;
    m.geo = g.geo64.ptr;
    m.conn = g.conn.ptr;
    m.Dr = g.Dr64.ptr;
    m.Ds = g.Ds64.ptr;
    m.fmask = g.fmask.ptr;
    m.K = g.K;
    m.p = g.p;
    return m;
}

// wall forces of every case into cases[].Fx, Fy, Mz (and, with a history,
// the step's record): one launch over the wall faces of every degree group,
// one block per case for the sums
dg_status enqueue_forces(dg_batch *b, double *hist = nullptr, int rows = 0)
{
    const dg::Phys<double> ph = phys_of<double>(b->prm);
    dg::WallGroups wg;
    for (auto &g : b->groups) {
        if (g.nwall == 0) continue;
        dg::WallGroup &w = wg.g[wg.n++];
        w.m = aux_of(b, g);
        w.faces = g.walls.ptr;
        w.face_xy = g.fxy.ptr;
        w.wface = g.wface.ptr;
        w.base = g.wall_base;
        w.nwall = g.nwall;
        wg.total = g.wall_base + g.nwall;
    }
    if (wg.total > 0) {
        B_CUDA(b, dg::launch_batch_wall_forces(wg, ph, b->fpart.ptr, b->stream));
        b->launches += 1;
    }
    B_CUDA(b, dg::launch_batch_forces_record(b->fpart.ptr, b->wseg.ptr, b->dcases.ptr,
                                             static_cast<int>(b->cases.size()), hist, rows, b->counter.ptr,
                                             b->ticket.ptr, b->stream));
    b->launches += 1;
    return DG_OK;
}

// The five stages of every degree group in one cooperative launch: each
// group runs the fused tensor-core body on its own share of the blocks, with
// grid barriers among those blocks only.  The first call sizes the shares in
// proportion to the tuner's time of each group's tensor-core shape (or, if
// the shapes were not timed, to its tiles times its nodes per element).
dg_status enqueue_stages_all(dg_batch *b, const dg::Phys<float> &ph32, double sf)
{
    const int ng = static_cast<int>(b->groups.size());
    std::vector<int> ps(ng);
    std::vector<dg::StageParams> sps(ng);
    for (int i = 0; i < ng; ++i) {
        Group &g = b->groups[i];
        if (!g.has_tc) return bfail(b, DG_EUNSUPPORTED, "one launch for all groups needs the tensor-core shape (p <= 6)");
        ps[i] = g.p;
        dg::StageParams &sp = sps[i];
        const bool a = b->cur_is_a;
        sp.K0in = a ? g.K0a.ptr : g.K0b.ptr;
        sp.K0out = a ? g.K0b.ptr : g.K0a.ptr;
        sp.K1 = g.K1.ptr;
        sp.geo = g.geo32.ptr;
        sp.conn = g.conn.ptr;
        sp.ops = g.tcfrag.ptr;
        sp.fmask = g.fmask.ptr;
        sp.Sin = a ? g.S0a.ptr : g.S0b.ptr;
        sp.Pin = a ? g.P0a.ptr : g.P0b.ptr;
        sp.Sout = a ? g.S0b.ptr : g.S0a.ptr;
        sp.Pout = a ? g.P0b.ptr : g.P0a.ptr;
        sp.K = g.K;
        sp.gm1 = b->prm.gamma - 1.0;
        sp.sig_fac = sf;
        sp.mode = dg::STAGE_UPDATE;
        sp.first_stage = 1;
        sp.cases = b->dcases.ptr;
        sp.bar_err = b->bar_err.ptr;
        sp.bar_limit = b->bar_limit;
        sp.tiles = g.tiles3.ptr;
        sp.ntiles = g.ntiles3;
        for (int s = 0; s < 5; ++s) {
            sp.A5[s] = dg::kRkA[s];
            sp.B5[s] = dg::kRkB[s];
        }
        sp.bar = g.bar.ptr;          // [0, 1] barrier, [2 .. 6] tile counters of the five stages
        B_CUDA(b, cudaMemsetAsync(g.bar.ptr, 0, 8 * sizeof(unsigned), b->stream));
    }
    if (b->all_nblk.size() != static_cast<size_t>(ng)) {
        int cap = 0;
        B_CUDA(b, dg::stage_tc_multi_capacity(ps.data(), ng, cap, b->all_smem));
        std::vector<double> w(ng);
        double wsum = 0.0;
        for (int i = 0; i < ng; ++i) {
            const Group &g = b->groups[i];
            w[i] = g.t_tc > 0.f ? static_cast<double>(g.t_tc) : static_cast<double>(g.ntiles3) * g.ops.Np;
            wsum += w[i];
        }
        b->all_nblk.assign(ng, 1u);
        int left = cap - ng;
        for (int i = 0; i < ng; ++i) {
            // at most one block per four warp tiles: a block runs four warps
            const long long most = (b->groups[i].ntiles3 + 3) / 4;
            long long extra = static_cast<long long>(w[i] / wsum * (cap - ng));
            if (extra > most - 1) extra = most - 1;
            if (extra > left) extra = left;
            if (extra < 0) extra = 0;
            b->all_nblk[i] += static_cast<unsigned>(extra);
            left -= static_cast<int>(extra);
        }
    }
    B_CUDA(b, dg::launch_stage_tc_multi(ng, ps.data(), sps.data(), b->all_nblk.data(), b->all_smem, ph32,
                                        b->stream));
    b->launches += 1;
    return DG_OK;
}

// one time step of every case (Algorithm 3), queued on the batch stream
dg_status enqueue_step(dg_batch *b, double cfl, double *hist, int rows)
{
    const int n = static_cast<int>(b->cases.size());
    const double sf = sigma_factor(b->prm);
    const dg::Phys<float> ph32 = phys_of<float>(b->prm);
    // FP32 bound from the FP32 state copy, a stability estimate recomputed
    // every step: one launch for all degree groups
    dg::DtGroups dgs{};
    for (auto &g : b->groups) {
        const bool a = b->cur_is_a;
        dg::DtGroup &d = dgs.g[dgs.n++];
        d.S = a ? g.S0a.ptr : g.S0b.ptr;
        d.Pr = a ? g.P0a.ptr : g.P0b.ptr;
        d.geo = g.geo32.ptr;
        d.conn = g.conn.ptr;
        d.fmask = g.fmask.ptr;
        d.tiles = g.tiles.ptr;
        d.K = g.K;
        d.ntiles = g.ntiles;
        d.first_block = dgs.blocks;
        d.lam = b->lam.ptr + g.lam_base;
        d.p = g.p;
        dgs.blocks += g.ntiles;
    }
    B_CUDA(b, dg::launch_dt_lambda_mixed_multi(dgs, b->dcases.ptr, ph32, static_cast<float>(sf), b->stream));
    b->launches += 1;
    B_CUDA(b, dg::launch_batch_dt_newmark(b->lam.ptr, b->seg.ptr, b->dcases.ptr, n, cfl,
                                          b->use_fixed ? b->fixed_dt.ptr : nullptr, b->stream));
    b->launches += 1;
    if (b->fused_all) {
        dg_status st = enqueue_stages_all(b, ph32, sf);
        if (st != DG_OK) return st;
        b->cur_is_a = !b->cur_is_a;
        return enqueue_forces(b, hist, rows);
    }
    for (int s = 0; s < (b->fused ? 1 : 5); ++s) {
        for (auto &g : b->groups) {
            dg::StageParams sp{};
            const bool a = b->cur_is_a;
            sp.K0in = a ? g.K0a.ptr : g.K0b.ptr;
            sp.K0out = a ? g.K0b.ptr : g.K0a.ptr;
            sp.K1 = g.K1.ptr;
            sp.geo = g.geo32.ptr;
            sp.conn = g.conn.ptr;
            sp.ops = g.ops32.ptr;
            sp.fmask = g.fmask.ptr;
            sp.Sin = a ? g.S0a.ptr : g.S0b.ptr;
            sp.Pin = a ? g.P0a.ptr : g.P0b.ptr;
            sp.Sout = a ? g.S0b.ptr : g.S0a.ptr;
            sp.Pout = a ? g.P0b.ptr : g.P0a.ptr;
            sp.K = g.K;
            sp.A = dg::kRkA[s];
            sp.B = dg::kRkB[s];
            sp.gm1 = b->prm.gamma - 1.0;
            sp.sig_fac = sf;
            sp.mode = dg::STAGE_UPDATE;
            sp.first_stage = (s == 0) ? 1 : 0;
            sp.cases = b->dcases.ptr;
            sp.bar_err = b->bar_err.ptr;          // grid barriers and copy waits report here
            sp.bar_limit = b->bar_limit;
            if (b->fused) {
                // the five stages in one cooperative launch (grid barriers between stages)
                sp.tiles = (g.variant == 3) ? g.tiles3.ptr : (g.variant == 2) ? g.tiles2.ptr : g.tiles.ptr;
                sp.ntiles = (g.variant == 3) ? g.ntiles3 : (g.variant == 2) ? g.ntiles2 : g.ntiles;
                if (g.variant == 3) sp.ops = g.tcfrag.ptr;
                if (g.fshape_variant != g.variant) {
                    if (g.variant == 3)
                        B_CUDA(b, dg::stage_shape_tc(g.p, sp.ntiles, true, true, g.fshape));
                    else
                        B_CUDA(b, dg::stage_shape_mixed_fused(g.p, g.variant, true, sp.ntiles, g.fshape));
                    g.fshape_variant = g.variant;
                }
                for (int i = 0; i < 5; ++i) {
                    sp.A5[i] = dg::kRkA[i];
                    sp.B5[i] = dg::kRkB[i];
                }
                sp.bar = g.bar.ptr;
                B_CUDA(b, cudaMemsetAsync(g.bar.ptr, 0, 2 * sizeof(unsigned), b->stream));
                if (g.variant == 3)
                    B_CUDA(b, dg::launch_stage_tc(g.p, true, true, g.fshape, sp, ph32, b->stream));
                else
                    B_CUDA(b, dg::launch_stage_mixed_fused(g.p, true, g.fshape, sp, ph32, b->stream));
            } else if (g.variant == 3) {
                sp.tiles = g.tiles3.ptr;
                sp.ntiles = g.ntiles3;
                sp.ops = g.tcfrag.ptr;
                B_CUDA(b, dg::launch_stage_tc(g.p, true, false, g.shape3, sp, ph32, b->stream));
            } else if (g.variant == 2) {
                sp.tiles = g.tiles2.ptr;
                sp.ntiles = g.ntiles2;
                B_CUDA(b, dg::launch_stage_mixed2(g.p, true, g.shape2, sp, ph32, b->stream));
            } else {
                sp.tiles = g.tiles.ptr;
                sp.ntiles = g.ntiles;
                B_CUDA(b, dg::launch_stage_mixed_batch(g.p, g.shape, sp, ph32, b->stream));
            }
            b->launches += 1;
        }
        b->cur_is_a = !b->cur_is_a;
    }
    return enqueue_forces(b, hist, rows);
}

// First run: per degree group, time every available stage-kernel shape on
// the current states in residual-only launches (into a scratch array) and
// keep the fastest.
dg_status tune_groups(dg_batch *b)
{
    if (b->tuned) return DG_OK;
    const dg::Phys<float> ph32 = phys_of<float>(b->prm);
    // events destroyed on every return path
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events()
        {
            for (auto &x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    B_CUDA(b, cudaEventCreate(&ev.e[0]));
    B_CUDA(b, cudaEventCreate(&ev.e[1]));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    for (auto &g : b->groups) {
        if (b->variant_req != 0) {
            // the tensor-core shape covers p <= 6; other groups would take the two-node shape
            g.variant = (b->variant_req == 3 && !g.has_tc) ? 2 : b->variant_req;
            continue;
        }
        DevBuf<double> scratch;
        B_CUDA(b, scratch.alloc(static_cast<size_t>(g.K) * 4 * g.ops.Np));
        float best = 0.f;
        for (int v = 1; v <= 3; ++v) {
            if (v == 3 && !g.has_tc) continue;
            dg::StageParams sp{};
            const bool a = b->cur_is_a;
            sp.K0in = a ? g.K0a.ptr : g.K0b.ptr;
            sp.K1 = g.K1.ptr;
            sp.Rout = scratch.ptr;
            sp.geo = g.geo32.ptr;
            sp.conn = g.conn.ptr;
            sp.ops = g.ops32.ptr;
            sp.fmask = g.fmask.ptr;
            sp.Sin = a ? g.S0a.ptr : g.S0b.ptr;
            sp.Pin = a ? g.P0a.ptr : g.P0b.ptr;
            sp.K = g.K;
            sp.gm1 = b->prm.gamma - 1.0;
            sp.sig_fac = sigma_factor(b->prm);
            sp.mode = dg::STAGE_RHS_ONLY;
            sp.first_stage = 1;
            sp.cases = b->dcases.ptr;
            sp.bar_err = b->bar_err.ptr;
            sp.bar_limit = b->bar_limit;
            float ms = 0.f;
            for (int rep = 0; rep < 5; ++rep) {
                if (rep == 2) B_CUDA(b, cudaEventRecord(e0, b->stream));
                if (v == 3) {
                    sp.tiles = g.tiles3.ptr;
                    sp.ntiles = g.ntiles3;
                    sp.ops = g.tcfrag.ptr;
                    B_CUDA(b, dg::launch_stage_tc(g.p, true, false, g.shape3, sp, ph32, b->stream));
                } else if (v == 2) {
                    sp.tiles = g.tiles2.ptr;
                    sp.ntiles = g.ntiles2;
                    B_CUDA(b, dg::launch_stage_mixed2(g.p, true, g.shape2, sp, ph32, b->stream));
                } else {
                    sp.tiles = g.tiles.ptr;
                    sp.ntiles = g.ntiles;
                    B_CUDA(b, dg::launch_stage_mixed_batch(g.p, g.shape, sp, ph32, b->stream));
                }
                b->launches += 1;
            }
            B_CUDA(b, cudaEventRecord(e1, b->stream));
            B_CUDA(b, cudaEventSynchronize(e1));
            B_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (v == 3) g.t_tc = ms;
            if (v == 1 || ms < best) {
                best = ms;
                g.variant = v;
            }
        }
    }
    b->tuned = true;
    return DG_OK;
}

bool valid_case(const dg_case &c)
{
    return c.p >= 1 && c.p <= 6 && c.vx && c.vy && c.EToV && c.EToE && c.EToF && c.bc && c.K >= 1 && c.Nv >= 3 &&
           c.mu >= 0.0 && std::isfinite(c.mu) && c.mass > 0.0 && std::isfinite(c.M_r) && std::isfinite(c.C_r) &&
           std::isfinite(c.K_r) && std::isfinite(c.y0) && std::isfinite(c.ydot0);
}

}  // namespace

extern "C" {

dg_status dg_batch_create(const dg_params *common, int ncases, const dg_case *cases, dg_batch **out)
{
    g_create_err.clear();
    auto cfail = [](dg_status st, const std::string &msg) {
        g_create_err = msg;
        return st;
    };
    if (!out) return cfail(DG_EINVAL, "null output");
    *out = nullptr;
    if (!common || !cases || ncases < 1) return cfail(DG_EINVAL, "need parameters and ncases >= 1");
    const dg_params &p = *common;
    if (!(p.gamma > 1.0) || !(p.Pr > 0.0) || !(p.C1 >= 0.0) || !(p.rho_inf > 0.0) || !(p.p_inf > 0.0))
        return cfail(DG_EINVAL, "bad common parameters");
    if (p.theta != 0.0 || p.precision != DG_PRECISION_MIXED)
        return cfail(DG_EUNSUPPORTED, "the batch runs the mixed-precision IIP kernel only");
    for (int i = 0; i < ncases; ++i)
        if (!valid_case(cases[i])) return cfail(DG_EINVAL, "case " + std::to_string(i) + ": bad description");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return cfail(DG_ECUDA, "no CUDA device");
    }
    dg_batch *b = new dg_batch();
    b->prm = p;
    auto bail = [&](dg_status st, const std::string &msg = "CUDA error while creating the batch") {
        *out = nullptr;
        cudaGetLastError();
        delete b;
        return cfail(st, msg);
    };
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(DG_ECUDA);
    // degree groups in increasing p
    std::vector<int> degrees;
    for (int i = 0; i < ncases; ++i) degrees.push_back(cases[i].p);
    std::sort(degrees.begin(), degrees.end());
    degrees.erase(std::unique(degrees.begin(), degrees.end()), degrees.end());
    b->groups.resize(degrees.size());
    b->cases.resize(ncases);
    b->init.resize(ncases);
    std::vector<long long> seg(2 * static_cast<size_t>(ncases));
    std::vector<int> wseg(2 * static_cast<size_t>(ncases));
    long long lam_total = 0;
    int wall_total = 0;
    for (size_t gi = 0; gi < degrees.size(); ++gi) {
        Group &g = b->groups[gi];
        g.p = degrees[gi];
        if (!dg::build_reference_operators(g.p, g.ops)) return bail(DG_EINVAL);
        const int Np = g.ops.Np, Nfp = g.ops.Nfp, NF = 3 * Nfp;
        const int E = dg::stage_tile_elems(g.p), E2 = dg::stage_tile_elems2(g.p), E3 = dg::stage_tile_elems_tc();
        std::vector<double> geo;
        std::vector<int4> conn;
        std::vector<int2> walls;
        std::vector<double> wxy;
        std::vector<int4> tiles, tiles2, tiles3;
        std::vector<int> ecase;
        g.lam_base = lam_total;
        g.wall_base = wall_total;
        for (int i = 0; i < ncases; ++i) {
            const dg_case &c = cases[i];
            if (c.p != g.p) continue;
            dg::MeshArrays ma;
            std::string msg;
            const int mst = dg::build_mesh(g.ops, c.Nv, c.vx, c.vy, c.K, c.EToV, c.EToE, c.EToF, c.bc, ma, msg);
            if (mst != dg::MESH_OK)
                return bail((mst == dg::MESH_EINVAL) ? DG_EINVAL : DG_EMESH, "case " + std::to_string(i) + ": " + msg);
            const long long off = g.K;
            if (off + c.K > (1LL << 30)) return bail(DG_EINVAL, "too many elements of one degree");
            CaseHost &ch = b->cases[i];
            ch.group = static_cast<int>(gi);
            ch.off = off;
            ch.K = c.K;
            ch.p = c.p;
            ch.vx.assign(c.vx, c.vx + c.Nv);
            ch.vy.assign(c.vy, c.vy + c.Nv);
            ch.EToV.assign(c.EToV, c.EToV + c.K * 3);
            for (auto &cn : ma.conn) {
                cn.x += static_cast<int>(off);
                cn.y += static_cast<int>(off);
                cn.z += static_cast<int>(off);
            }
            geo.insert(geo.end(), ma.geo.begin(), ma.geo.end());
            conn.insert(conn.end(), ma.conn.begin(), ma.conn.end());
            seg[2 * i] = lam_total + off;
            seg[2 * i + 1] = lam_total + off + c.K;
            wseg[2 * i] = wall_total + static_cast<int>(walls.size());
            for (auto w : ma.walls) walls.push_back(make_int2(w.x + static_cast<int>(off), w.y));
            wseg[2 * i + 1] = wall_total + static_cast<int>(walls.size());
            wxy.insert(wxy.end(), ma.wxy.begin(), ma.wxy.end());
            for (long long k0 = 0; k0 < c.K; k0 += E)
                tiles.push_back(make_int4(static_cast<int>(off + k0), static_cast<int>(std::min<long long>(E, c.K - k0)),
                                          i, 0));
            for (long long k0 = 0; k0 < c.K; k0 += E2)
                tiles2.push_back(make_int4(static_cast<int>(off + k0),
                                           static_cast<int>(std::min<long long>(E2, c.K - k0)), i, 0));
            for (long long k0 = 0; k0 < c.K; k0 += E3)
                tiles3.push_back(make_int4(static_cast<int>(off + k0),
                                           static_cast<int>(std::min<long long>(E3, c.K - k0)), i, 0));
            ecase.insert(ecase.end(), static_cast<size_t>(c.K), i);
            g.K += c.K;
            dg::BatchCase &bc = b->init[i];
            bc = dg::BatchCase{};
            bc.y = c.y0;
            bc.yd = c.ydot0;
            bc.Mr = c.M_r;
            bc.Cr = c.C_r;
            bc.Kr = c.K_r;
            bc.mass = c.mass;
            bc.mu = c.mu;
        }
        g.nwall = static_cast<int>(walls.size());
        g.ntiles = static_cast<long long>(tiles.size());
        g.ntiles2 = static_cast<long long>(tiles2.size());
        g.ntiles3 = static_cast<long long>(tiles3.size());
        g.has_tc = dg::stage_tc_supported(g.p);
        lam_total += g.K;
        wall_total += g.nwall;
        const size_t nd = static_cast<size_t>(g.K) * 4 * Np;
        const size_t npp = static_cast<size_t>(g.K) * dg::pressure_row(g.p);
        std::vector<double> o64;
        o64.insert(o64.end(), g.ops.Dr.begin(), g.ops.Dr.end());
        o64.insert(o64.end(), g.ops.Ds.begin(), g.ops.Ds.end());
        o64.insert(o64.end(), g.ops.LIFT.begin(), g.ops.LIFT.end());
        std::vector<float> o32(o64.begin(), o64.end());
        std::vector<float> g32(geo.begin(), geo.end());
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
        chk(g.K0a.alloc(nd));
        chk(g.K0b.alloc(nd));
        chk(g.K1.alloc(nd));
        chk(g.S0a.alloc(static_cast<size_t>(g.K) * Np));
        chk(g.S0b.alloc(static_cast<size_t>(g.K) * Np));
        chk(g.P0a.alloc(npp));
        chk(g.P0b.alloc(npp));
        chk(g.geo64.alloc(geo.size()));
        chk(g.geo32.alloc(g32.size()));
        chk(g.conn.alloc(conn.size()));
        chk(g.tiles.alloc(tiles.size()));
        chk(g.tiles2.alloc(tiles2.size()));
        chk(g.tiles3.alloc(tiles3.size()));
        std::vector<float> frag;
        if (g.has_tc) {
            dg::build_tc_fragments(Np, NF, g.ops.Dr.data(), g.ops.Ds.data(), g.ops.LIFT.data(), g.ops.Wr.data(),
                                   g.ops.Ws.data(), frag);
            chk(g.tcfrag.alloc(frag.size()));
        }
        chk(g.elem_case.alloc(ecase.size()));
        chk(g.ops32.alloc(o32.size()));
        chk(g.Dr64.alloc(static_cast<size_t>(Np) * Np));
        chk(g.Ds64.alloc(static_cast<size_t>(Np) * Np));
        chk(g.fmask.alloc(NF));
        chk(g.wface.alloc(Nfp));
        if (g.nwall > 0) {
            chk(g.walls.alloc(walls.size()));
            chk(g.fxy.alloc(wxy.size()));
        }
        if (e != cudaSuccess) return bail(DG_ECUDA);
        chk(cudaMemcpy(g.geo64.ptr, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.geo32.ptr, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.conn.ptr, conn.data(), conn.size() * sizeof(int4), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.tiles.ptr, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.tiles2.ptr, tiles2.data(), tiles2.size() * sizeof(int4), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.tiles3.ptr, tiles3.data(), tiles3.size() * sizeof(int4), cudaMemcpyHostToDevice));
        if (g.has_tc) chk(cudaMemcpy(g.tcfrag.ptr, frag.data(), frag.size() * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.elem_case.ptr, ecase.data(), ecase.size() * sizeof(int), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.ops32.ptr, o32.data(), o32.size() * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.Dr64.ptr, g.ops.Dr.data(), g.ops.Dr.size() * sizeof(double), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.Ds64.ptr, g.ops.Ds.data(), g.ops.Ds.size() * sizeof(double), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.fmask.ptr, g.ops.Fmask.data(), NF * sizeof(int), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(g.wface.ptr, g.ops.wface.data(), Nfp * sizeof(double), cudaMemcpyHostToDevice));
        if (g.nwall > 0) {
            chk(cudaMemcpy(g.walls.ptr, walls.data(), walls.size() * sizeof(int2), cudaMemcpyHostToDevice));
            chk(cudaMemcpy(g.fxy.ptr, wxy.data(), wxy.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        chk(cudaMemset(g.K0a.ptr, 0, nd * sizeof(double)));
        chk(cudaMemset(g.K0b.ptr, 0, nd * sizeof(double)));
        chk(cudaMemset(g.K1.ptr, 0, nd * sizeof(double)));
        chk(cudaMemset(g.S0a.ptr, 0, static_cast<size_t>(g.K) * Np * sizeof(float4)));
        chk(cudaMemset(g.S0b.ptr, 0, static_cast<size_t>(g.K) * Np * sizeof(float4)));
        chk(cudaMemset(g.P0a.ptr, 0, npp * sizeof(float)));
        chk(cudaMemset(g.P0b.ptr, 0, npp * sizeof(float)));
        chk(dg::stage_shape_mixed_batch(g.p, g.ntiles, g.shape));
        chk(dg::stage_shape_mixed2(g.p, g.ntiles2, true, g.shape2));
        if (g.has_tc) chk(dg::stage_shape_tc(g.p, g.ntiles3, true, false, g.shape3));
        if (e != cudaSuccess) return bail(DG_ECUDA);
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(b->dcases.alloc(ncases));
    chk(b->lam.alloc(static_cast<size_t>(lam_total)));
    chk(b->fpart.alloc(static_cast<size_t>(std::max(wall_total, 1)) * 3));
    chk(b->seg.alloc(seg.size()));
    chk(b->wseg.alloc(wseg.size()));
    chk(b->counter.alloc(1));
    chk(b->ticket.alloc(1));
    chk(b->bar_err.alloc(1));
    chk(cudaMemset(b->ticket.ptr, 0, sizeof(unsigned)));
    chk(cudaMemset(b->bar_err.ptr, 0, sizeof(int)));
    if (e != cudaSuccess) return bail(DG_ECUDA);
    chk(cudaMemcpy(b->dcases.ptr, b->init.data(), ncases * sizeof(dg::BatchCase), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(b->seg.ptr, seg.data(), seg.size() * sizeof(long long), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(b->wseg.ptr, wseg.data(), wseg.size() * sizeof(int), cudaMemcpyHostToDevice));
    chk(cudaMemset(b->counter.ptr, 0, sizeof(int)));
    chk(cudaMemset(b->fpart.ptr, 0, b->fpart.n * sizeof(double)));
    if (e != cudaSuccess) return bail(DG_ECUDA);
    *out = b;
    return DG_OK;
}

dg_status dg_batch_destroy(dg_batch *b)
{
    delete b;
    return DG_OK;
}

const char *dg_batch_last_error(const dg_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int64_t dg_batch_kernel_launches(const dg_batch *b) { return b ? b->launches : 0; }

dg_status dg_batch_set_stage_variant(dg_batch *b, int variant)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (variant < 0 || variant > 3) return bfail(b, DG_EINVAL, "variant must be 0, 1, 2 or 3");
    b->variant_req = variant;
    b->tuned = false;
    b->drop_graphs();
    b->graph_cfl = 0.0;
    return DG_OK;
}

dg_status dg_batch_set_fixed_dt(dg_batch *b, const double *dt)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    const size_t n = b->cases.size();
    if (!dt) {
        if (b->use_fixed) {
            b->use_fixed = false;
            b->drop_graphs();
            b->graph_cfl = 0.0;
        }
        return DG_OK;
    }
    for (size_t i = 0; i < n; ++i)
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i]))
            return bfail(b, DG_EINVAL, "fixed step of case " + std::to_string(i) + " must be finite and > 0");
    if (!b->fixed_dt.ptr) B_CUDA(b, b->fixed_dt.alloc(n));
    // the batch stream may still read the previous steps
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    B_CUDA(b, cudaMemcpy(b->fixed_dt.ptr, dt, n * sizeof(double), cudaMemcpyHostToDevice));
    if (!b->use_fixed) {
        b->use_fixed = true;
        b->drop_graphs();
        b->graph_cfl = 0.0;
    }
    return DG_OK;
}

dg_status dg_batch_set_fused_steps(dg_batch *b, int on)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (on < 0 || on > 2) return bfail(b, DG_EINVAL, "fused steps: 0 (off), 1 (per degree group) or 2 (all groups)");
    if (on) {
        for (auto &g : b->groups) {
            if (g.bar.ptr) continue;
            B_CUDA(b, g.bar.alloc(8));
            B_CUDA(b, cudaMemset(g.bar.ptr, 0, 8 * sizeof(unsigned)));
        }
    }
    b->fused = on != 0;
    b->fused_all = on == 2;
    b->all_nblk.clear();
    b->drop_graphs();
    b->graph_cfl = 0.0;
    return DG_OK;
}

int dg_batch_stage_variant(const dg_batch *b, int i)
{
    if (!b || i < 0 || i >= static_cast<int>(b->cases.size())) return 0;
    return b->groups[b->cases[i].group].variant;
}

void *dg_batch_stream(const dg_batch *b) { return b ? static_cast<void *>(b->stream) : nullptr; }

dg_status dg_batch_case_size(const dg_batch *b, int i, int64_t *K, int *p)
{
    if (!b || i < 0 || i >= static_cast<int>(b->cases.size())) return DG_EINVAL;
    if (K) *K = b->cases[i].K;
    if (p) *p = b->cases[i].p;
    return DG_OK;
}

dg_status dg_batch_node_coords(const dg_batch *b, int i, double *x, double *y)
{
    if (!b || !x || !y || i < 0 || i >= static_cast<int>(b->cases.size())) return DG_EINVAL;
    const CaseHost &c = b->cases[i];
    const dg::RefOps &o = b->groups[c.group].ops;
    for (long long k = 0; k < c.K; ++k) {
        const int32_t v0 = c.EToV[k * 3], v1 = c.EToV[k * 3 + 1], v2 = c.EToV[k * 3 + 2];
        for (int n = 0; n < o.Np; ++n) {
            const double r = o.r[n], s = o.s[n];
            x[k * o.Np + n] = 0.5 * (-(r + s) * c.vx[v0] + (1 + r) * c.vx[v1] + (1 + s) * c.vx[v2]);
            y[k * o.Np + n] = 0.5 * (-(r + s) * c.vy[v0] + (1 + r) * c.vy[v1] + (1 + s) * c.vy[v2]);
        }
    }
    return DG_OK;
}

dg_status dg_batch_set_state(dg_batch *b, int i, const double *U, int on_device)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (!U || i < 0 || i >= static_cast<int>(b->cases.size())) return bfail(b, DG_EINVAL, "bad case or null state");
    const CaseHost &c = b->cases[i];
    Group &g = b->groups[c.group];
    const int Np = g.ops.Np;
    const size_t off = static_cast<size_t>(c.off) * 4 * Np, n = static_cast<size_t>(c.K) * 4 * Np;
    double *cur = b->cur_is_a ? g.K0a.ptr : g.K0b.ptr;
    float4 *S = b->cur_is_a ? g.S0a.ptr : g.S0b.ptr;
    float *P = b->cur_is_a ? g.P0a.ptr : g.P0b.ptr;
    B_CUDA(b, cudaMemcpyAsync(cur + off, U, n * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    B_CUDA(b, cudaMemsetAsync(g.K1.ptr + off, 0, n * sizeof(double), b->stream));
    B_CUDA(b, dg::launch_make_shadow(g.p, cur + off, c.K, b->prm.gamma - 1.0, S + c.off * Np,
                                     P + c.off * dg::pressure_row(g.p), b->stream));
    b->launches += 1;
    b->forces_stale = true;
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return DG_OK;
}

dg_status dg_batch_get_state(dg_batch *b, int i, double *U, int on_device)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (!U || i < 0 || i >= static_cast<int>(b->cases.size())) return bfail(b, DG_EINVAL, "bad case or null state");
    const CaseHost &c = b->cases[i];
    Group &g = b->groups[c.group];
    const int Np = g.ops.Np;
    const size_t off = static_cast<size_t>(c.off) * 4 * Np, n = static_cast<size_t>(c.K) * 4 * Np;
    const double *cur = b->cur_is_a ? g.K0a.ptr : g.K0b.ptr;
    B_CUDA(b, cudaMemcpyAsync(U, cur + off, n * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return DG_OK;
}

dg_status dg_batch_reset_history(dg_batch *b)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    B_CUDA(b, cudaMemsetAsync(b->counter.ptr, 0, sizeof(int), b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return DG_OK;
}

dg_status dg_batch_run(dg_batch *b, double cfl, int nsteps, int use_graph, double *hist, int hist_rows)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (!(cfl > 0.0) || !std::isfinite(cfl) || nsteps < 0 || (hist && hist_rows < 0))
        return bfail(b, DG_EINVAL, "need cfl > 0, nsteps >= 0, hist_rows >= 0");
    if (b->forces_stale) {
        dg_status st = enqueue_forces(b);
        if (st != DG_OK) return st;
        b->forces_stale = false;
    }
    if (!b->tuned) {
        dg_status st = tune_groups(b);
        if (st != DG_OK) return st;
    }
    if (use_graph && nsteps > 0) {
        if (b->graph_cfl != cfl || b->graph_hist != hist || b->graph_rows != hist_rows) {
            b->drop_graphs();
            b->graph_cfl = cfl;
            b->graph_hist = hist;
            b->graph_rows = hist_rows;
        }
        for (int n = 0; n < nsteps; ++n) {
            const int which = b->cur_is_a ? 0 : 1;
            if (!b->graph[which]) {
                // capture one step starting from the current buffers; the step
                // flips the buffer parity (five stages), as a replay will
                const bool start_a = b->cur_is_a;
                const int64_t l0 = b->launches;
                B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                dg_status st = enqueue_step(b, cfl, hist, hist_rows);
                cudaGraph_t gr = nullptr;
                cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
                b->launches = l0;
                b->cur_is_a = start_a;
                if (st != DG_OK) {
                    if (gr) cudaGraphDestroy(gr);
                    return st;
                }
                if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&b->graph[which], gr, 0);
                cudaGraphDestroy(gr);
                if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
                // kernels per replay: dt per group, dt reduce, Newmark, 5 stages per group,
                // forces per group with walls, force sum, record
                // time-step bounds of all groups, dt + Newmark, the stage launches
                // per group, wall forces of all groups, force sums (+ history)
                bool walls = false;
                for (auto &g : b->groups) walls |= g.nwall > 0;
                const int64_t stages = b->fused_all ? 1 : static_cast<int64_t>(b->groups.size()) * (b->fused ? 1 : 5);
                int64_t per = 1 + 1 + stages + (walls ? 1 : 0) + 1;
                b->graph_launches = per;
            }
            B_CUDA(b, cudaGraphLaunch(b->graph[which], b->stream));
            b->launches += b->graph_launches;
            b->cur_is_a = !b->cur_is_a;
        }
    } else {
        for (int n = 0; n < nsteps; ++n) {
            dg_status st = enqueue_step(b, cfl, hist, hist_rows);
            if (st != DG_OK) return st;
        }
    }
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    {
        int e = 0;
        B_CUDA(b, cudaMemcpy(&e, b->bar_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            B_CUDA(b, cudaMemset(b->bar_err.ptr, 0, sizeof(int)));
            return bfail(b, DG_ETIMEOUT,
                         "a bounded device wait gave up (a fused step's grid barrier or a stage kernel's copy "
                         "wait); the states are not valid");
        }
    }
    std::vector<dg::BatchCase> h(b->cases.size());
    B_CUDA(b, cudaMemcpy(h.data(), b->dcases.ptr, h.size() * sizeof(dg::BatchCase), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); ++i)
        if (h[i].bad) return bfail(b, DG_ENONFINITE, "case " + std::to_string(i) + " met a non-finite time-step bound");
    return DG_OK;
}

dg_status dg_batch_rigid(dg_batch *b, double *out)
{
    if (!b) return DG_EINVAL;
    b->err.clear();
    if (!out) return bfail(b, DG_EINVAL, "null output");
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    std::vector<dg::BatchCase> h(b->cases.size());
    B_CUDA(b, cudaMemcpy(h.data(), b->dcases.ptr, h.size() * sizeof(dg::BatchCase), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); ++i) {
        double *o = out + i * 10;
        o[0] = h[i].t; o[1] = h[i].dt; o[2] = h[i].y; o[3] = h[i].yd; o[4] = h[i].ydd;
        o[5] = h[i].vb; o[6] = h[i].Fx; o[7] = h[i].Fy; o[8] = h[i].Mz; o[9] = h[i].bad;
    }
    return DG_OK;
}

}  // extern "C"
