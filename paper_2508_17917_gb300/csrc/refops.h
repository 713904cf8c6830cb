// refops.h -- host construction of the reference-triangle operators.
#pragma once
#include <vector>

namespace dg {

struct RefOps {
    int p = 0, Np = 0, Nfp = 0;
    std::vector<double> r, s;        // Np nodes
    std::vector<double> Dr, Ds;      // Np*Np row-major
    std::vector<double> LIFT;        // Np*(3*Nfp) row-major, face columns CCW
    std::vector<int> Fmask;          // 3*Nfp volume index, CCW along each face
    std::vector<double> M1D;         // 3*Nfp*Nfp face mass in CCW order
    std::vector<double> Mhat;        // Np*Np
    std::vector<double> wface;       // Nfp LGL weights (column sums of M1D)
    std::vector<double> Wr, Ws;      // Np*Np: M^-1 Dr^T M, M^-1 Ds^T M
};

// Builds every operator for degree p (1..6). Returns false on bad p.
bool build_reference_operators(int p, RefOps &out);

}  // namespace dg
