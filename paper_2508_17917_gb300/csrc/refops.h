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

// Over-integration of the volume term (Sec. 2.2, weak matrices): a
// collapsed-coordinate Gauss rule exact to total degree `deg` (N = floor(deg/2)
// + 1 Gauss-Legendre points in a times N Gauss-Jacobi (1, 0) points in b),
// the nodal basis and its (r, s) derivatives at its points, and the weak
// volume operators Sr = M^-1 Vqr^T W, Ss = M^-1 Vqs^T W.
struct OverintOps {
    int deg = 0, Nq = 0;
    std::vector<double> wq;              // Nq
    std::vector<double> Vq, Vqr, Vqs;    // Nq*Np
    std::vector<double> Sr, Ss;          // Np*Nq
};
bool build_overint_operators(const RefOps &o, int deg, OverintOps &out);

// The rule degree the library uses for degree p: min(3p, 15), at most 64 points.
int overint_degree(int p);

}  // namespace dg
