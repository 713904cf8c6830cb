// mesh.h -- host construction of element geometry, connectivity and walls.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "refops.h"

namespace dg {

enum { MESH_OK = 0, MESH_EINVAL = 1, MESH_EBAD = 2 };

struct MeshArrays {
    std::vector<double> geo;     // K * 16: rx, ry, sx, sy, J, nx[3], ny[3], Fscale[3]
    std::vector<int4> conn;      // K: neighbours of faces 0..2, packed neighbour faces and bc
    std::vector<int2> walls;     // (element, face) of every wall face
    std::vector<double> wxy;     // 2 * Nfp node coordinates per wall face
};

// Validates the mesh and fills `out`; on failure returns MESH_EINVAL (null
// or too small) or MESH_EBAD (index out of range, clockwise or degenerate
// element, faces not reciprocal, face nodes that do not match) with `msg`.
int build_mesh(const RefOps &ops, int64_t Nv, const double *vx, const double *vy, int64_t K,
               const int32_t *EToV, const int32_t *EToE, const int32_t *EToF, const int32_t *bc,
               MeshArrays &out, std::string &msg);

}  // namespace dg
