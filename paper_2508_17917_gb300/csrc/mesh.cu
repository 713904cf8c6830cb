// mesh.cu -- host construction of the per-element geometry (Sec. 2.2, affine
// maps T_K), the packed connectivity and the wall-face lists, with the mesh
// checks the C ABI promises (index ranges, orientation, reciprocity, matching
// face nodes).  Shared by the single-mesh context and the batch.
#include "mesh.h"

#include <algorithm>
#include <cmath>

#include "dg_stage.cuh"

namespace dg {

int build_mesh(const RefOps &ops, int64_t Nv, const double *vx, const double *vy, int64_t K,
               const int32_t *EToV, const int32_t *EToE, const int32_t *EToF, const int32_t *bc,
               MeshArrays &out, std::string &msg)
{
    if (!vx || !vy || !EToV || !EToE || !EToF || !bc) { msg = "null mesh array"; return MESH_EINVAL; }
    if (K < 1 || Nv < 3) { msg = "need K >= 1 and Nv >= 3"; return MESH_EINVAL; }
    const int Np = ops.Np, Nfp = ops.Nfp;
    if (K * 4LL * Np > (1LL << 40)) { msg = "mesh too large"; return MESH_EINVAL; }
    // --- index checks and geometry
    std::vector<double> &geo = out.geo;
    geo.assign(static_cast<size_t>(K) * 16, 0.0);
    double scale = 0.0;
    for (int64_t i = 0; i < Nv; ++i) scale = std::max(scale, std::max(std::fabs(vx[i]), std::fabs(vy[i])));
    if (!(scale > 0.0) || !std::isfinite(scale)) { msg = "vertex coordinates not finite"; return MESH_EBAD; }
    for (int64_t k = 0; k < K; ++k) {
        int32_t v[3] = {EToV[k * 3], EToV[k * 3 + 1], EToV[k * 3 + 2]};
        for (int f = 0; f < 3; ++f) {
            if (v[f] < 0 || v[f] >= Nv) { msg = "EToV index out of range at element " + std::to_string(k); return MESH_EBAD; }
            int32_t e2 = EToE[k * 3 + f], f2 = EToF[k * 3 + f], b = bc[k * 3 + f];
            if (e2 < 0 || e2 >= K || f2 < 0 || f2 > 2 || b < 0 || b > 2)
                { msg = "EToE/EToF/bc out of range at element " + std::to_string(k); return MESH_EBAD; }
        }
        double x1 = vx[v[0]], y1 = vy[v[0]], x2 = vx[v[1]], y2 = vy[v[1]], x3 = vx[v[2]], y3 = vy[v[2]];
        double xr = 0.5 * (x2 - x1), xs = 0.5 * (x3 - x1), yr = 0.5 * (y2 - y1), ys = 0.5 * (y3 - y1);
        double J = xr * ys - xs * yr;
        if (!(J > 1e-14 * scale * scale))
            { msg = "element " + std::to_string(k) + " is clockwise or degenerate"; return MESH_EBAD; }
        double rx = ys / J, ry = -xs / J, sx = -yr / J, sy = xr / J;
        double *g = &geo[k * 16];
        g[G_RX] = rx; g[G_RY] = ry; g[G_SX] = sx; g[G_SY] = sy; g[G_J] = J;
        // outward normals from the metric: face 0 (s = -1): -grad s; face 1 (r+s = 0): grad(r+s);
        // face 2 (r = -1): -grad r; sJ = |grad| J
        double nn[3][2] = {{-sx, -sy}, {rx + sx, ry + sy}, {-rx, -ry}};
        for (int f = 0; f < 3; ++f) {
            double len = std::hypot(nn[f][0], nn[f][1]);
            g[G_NX + f] = nn[f][0] / len;
            g[G_NY + f] = nn[f][1] / len;
            g[G_FS + f] = len;          // Fscale = sJ / J = |grad| (since sJ = |grad| J)
        }
    }
    // --- reciprocity and face matching
    std::vector<int4> &conn = out.conn;
    conn.assign(K, make_int4(0, 0, 0, 0));
    for (int64_t k = 0; k < K; ++k) {
        int packed = 0;
        int nb[3];
        for (int f = 0; f < 3; ++f) {
            int32_t e2 = EToE[k * 3 + f], f2 = EToF[k * 3 + f], b = bc[k * 3 + f];
            nb[f] = e2;
            packed |= (f2 & 3) << (2 * f);
            packed |= (b & 3) << (8 + 2 * f);
            if (b != BCT_INTERIOR) {
                if (e2 != k || f2 != f) { msg = "boundary face must name itself at element " + std::to_string(k); return MESH_EBAD; }
                continue;
            }
            if (e2 == k) { msg = "interior face names its own element " + std::to_string(k); return MESH_EBAD; }
            if (EToE[e2 * 3 + f2] != k || EToF[e2 * 3 + f2] != f || bc[e2 * 3 + f2] != BCT_INTERIOR)
                { msg = "faces not reciprocal at element " + std::to_string(k); return MESH_EBAD; }
            // conforming, counter-clockwise: own (a, b) meets neighbour (b', a') up to one translation
            int32_t a = EToV[k * 3 + f], bb = EToV[k * 3 + (f + 1) % 3];
            int32_t a2 = EToV[e2 * 3 + f2], b2 = EToV[e2 * 3 + (f2 + 1) % 3];
            double tx1 = vx[a] - vx[b2], ty1 = vy[a] - vy[b2];
            double tx2 = vx[bb] - vx[a2], ty2 = vy[bb] - vy[a2];
            double tol = 1e-9 * scale;
            if (std::fabs(tx1 - tx2) > tol || std::fabs(ty1 - ty2) > tol)
                { msg = "face nodes do not match at element " + std::to_string(k); return MESH_EBAD; }
        }
        conn[k] = make_int4(nb[0], nb[1], nb[2], packed);
    }
    // --- wall faces and their node coordinates
    std::vector<int2> &walls = out.walls;
    std::vector<double> &wxy = out.wxy;
    walls.clear();
    wxy.clear();
    for (int64_t k = 0; k < K; ++k)
        for (int f = 0; f < 3; ++f)
            if (bc[k * 3 + f] == BCT_WALL) {
                walls.push_back(make_int2(static_cast<int>(k), f));
                int32_t v0 = EToV[k * 3], v1 = EToV[k * 3 + 1], v2 = EToV[k * 3 + 2];
                for (int i = 0; i < Nfp; ++i) {
                    int vm = ops.Fmask[f * Nfp + i];
                    double r = ops.r[vm], s = ops.s[vm];
                    wxy.push_back(0.5 * (-(r + s) * vx[v0] + (1 + r) * vx[v1] + (1 + s) * vx[v2]));
                    wxy.push_back(0.5 * (-(r + s) * vy[v0] + (1 + r) * vy[v1] + (1 + s) * vy[v2]));
                }
            }
    (void)Np;
    return MESH_OK;
}

}  // namespace dg
