// refops.cpp -- reference-triangle operators for the nodal DG solver.
//
// Sec. 2.2 ("weak matrices and nodal formulation"): the nodal basis lives on
// the optimised warp-and-blend interpolation points, the modal basis is the
// orthonormal Dubiner-Proriol-Koornwinder (PKD) family on the collapsed
// coordinates a = 2(1+r)/(1-s) - 1, b = s:
//     psi_ij(r, s) = sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i,
// with P^(alpha,beta) the Jacobi polynomials normalised to unit weighted
// L2 norm.  From the Vandermonde matrix V_{n,m} = psi_m(r_n, s_n):
//     Dr = Vr V^-1, Ds = Vs V^-1, M^-1 = V V^T,
// and LIFT = M^-1 E M_e with M_e the 1D face mass matrix on the LGL points;
// Wr = M^-1 Dr^T M and Ws = M^-1 Ds^T M carry the theta terms of Eq. dg_on_K,
// which test a face quantity against the gradient of the basis.
//
// This builder is the library's own: Jacobi values by the three-term
// recurrence, LGL points by Newton iteration on P_p', matrix inverses by
// Gauss-Jordan elimination, derivatives of psi by the chain rule through
// (a, b).  Face nodes are stored counter-clockwise along each face so that
// the matching node on a conforming neighbour is the reversed index.
#include "refops.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace dg {
namespace {

// Orthonormal Jacobi polynomial P_n^(al,be)(x) / sqrt(h_n) by recurrence.
double jacobi(double x, double al, double be, int n)
{
    // h_0 = 2^(al+be+1) Gamma(al+1) Gamma(be+1) / Gamma(al+be+2)
    double h0 = std::pow(2.0, al + be + 1.0) * std::tgamma(al + 1.0) * std::tgamma(be + 1.0)
              / std::tgamma(al + be + 2.0);
    double p0 = 1.0 / std::sqrt(h0);
    if (n == 0) return p0;
    double h1 = (al + 1.0) * (be + 1.0) / (al + be + 3.0) * h0;
    double p1 = ((al + be + 2.0) * x / 2.0 + (al - be) / 2.0) / std::sqrt(h1);
    if (n == 1) return p1;
    // normalised recurrence x P_k = a_{k+1} P_{k+1} + b_k P_k + a_k P_{k-1}
    double a_prev = 2.0 / (2.0 + al + be) * std::sqrt((al + 1.0) * (be + 1.0) / (al + be + 3.0));
    double pm = p0, pc = p1;
    for (int k = 1; k < n; ++k) {
        double h = 2.0 * k + al + be;
        double a_next = 2.0 / (h + 2.0) *
                        std::sqrt((k + 1.0) * (k + 1.0 + al + be) * (k + 1.0 + al) * (k + 1.0 + be) /
                                  ((h + 1.0) * (h + 3.0)));
        double b = -(al * al - be * be) / (h * (h + 2.0));
        double pn = ((x - b) * pc - a_prev * pm) / a_next;
        pm = pc;
        pc = pn;
        a_prev = a_next;
    }
    return pc;
}

// d/dx of the orthonormal Jacobi polynomial: sqrt(n(n+al+be+1)) P_{n-1}^(al+1,be+1).
double jacobi_d(double x, double al, double be, int n)
{
    if (n == 0) return 0.0;
    return std::sqrt(n * (n + al + be + 1.0)) * jacobi(x, al + 1.0, be + 1.0, n - 1);
}

// Legendre P_n and P_n' at x.
void legendre(int n, double x, double &P, double &dP)
{
    double pm = 1.0, pc = x;
    if (n == 0) { P = 1.0; dP = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
        pm = pc;
        pc = pn;
    }
    P = pc;
    dP = n * (x * pc - pm) / (x * x - 1.0);
}

// LGL points on [-1, 1]: end points and the roots of P_n' (Newton, using the
// Legendre equation for P_n'').
std::vector<double> lgl(int n)
{
    std::vector<double> x(n + 1);
    x[0] = -1.0;
    x[n] = 1.0;
    for (int j = 1; j < n; ++j) {
        double t = -std::cos(M_PI * j / n);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(n, t, P, dP);
            double d2P = (2.0 * t * dP - n * (n + 1.0) * P) / (1.0 - t * t);
            double step = dP / d2P;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[j] = t;
    }
    std::sort(x.begin(), x.end());
    return x;
}

bool invert(std::vector<double> A, int n, std::vector<double> &X)
{
    X.assign(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) X[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[c * n + j], A[piv * n + j]);
                std::swap(X[c * n + j], X[piv * n + j]);
            }
        double d = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= d; X[c * n + j] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = A[r * n + c];
            if (m == 0.0) continue;
            for (int j = 0; j < n; ++j) { A[r * n + j] -= m * A[c * n + j]; X[r * n + j] -= m * X[c * n + j]; }
        }
    }
    return true;
}

std::vector<double> matmul(const std::vector<double> &A, const std::vector<double> &B, int n, int m, int k)
{
    // (n x m) * (m x k)
    std::vector<double> C(static_cast<size_t>(n) * k, 0.0);
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < m; ++l) {
            double a = A[i * m + l];
            for (int j = 0; j < k; ++j) C[i * k + j] += a * B[l * k + j];
        }
    return C;
}

// Scaled edge warp: interpolant on equispaced points of the LGL displacement,
// divided by (1 - t^2); zero at the edge ends.
double edge_warp(int p, const std::vector<double> &gl, double t)
{
    double w = 0.0;
    for (int i = 0; i <= p; ++i) {
        double ti = -1.0 + 2.0 * i / p;
        double l = 1.0;
        for (int j = 0; j <= p; ++j) {
            if (j == i) continue;
            double tj = -1.0 + 2.0 * j / p;
            l *= (t - tj) / (ti - tj);
        }
        w += (gl[i] - ti) * l;
    }
    if (std::fabs(t) < 1.0 - 1e-10) return w / (1.0 - t * t);
    return 0.0;
}

// Orthonormal PKD modes and their (r, s) derivatives at n points (r[k], s[k]),
// row-major [n][Np]: psi_ij = sqrt2 P_i(a) P_j^(2i+1,0)(b) (1-b)^i with the
// collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s.
void vandermonde(int p, const double *rr, const double *ss, int n, std::vector<double> &V,
                 std::vector<double> &Vr, std::vector<double> &Vs)
{
    const int Np = (p + 1) * (p + 2) / 2;
    V.assign(static_cast<size_t>(n) * Np, 0.0);
    Vr.assign(V.size(), 0.0);
    Vs.assign(V.size(), 0.0);
    for (int nd = 0; nd < n; ++nd) {
        double r = rr[nd], s = ss[nd];
        double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
        double b = s, om = 1.0 - b;
        int col = 0;
        for (int i = 0; i <= p; ++i)
            for (int j = 0; j <= p - i; ++j, ++col) {
                double fa = jacobi(a, 0, 0, i), dfa = jacobi_d(a, 0, 0, i);
                double gb = jacobi(b, 2.0 * i + 1.0, 0, j), dgb = jacobi_d(b, 2.0 * i + 1.0, 0, j);
                double omi = std::pow(om, i), omi1 = (i > 0) ? std::pow(om, i - 1) : 0.0;
                V[nd * Np + col] = std::sqrt(2.0) * fa * gb * omi;
                // d/dr: da/dr = 2/(1-b)
                Vr[nd * Np + col] = (i > 0) ? 2.0 * std::sqrt(2.0) * dfa * gb * omi1 : 0.0;
                // d/ds: da/ds = (1+a)/(1-b), plus the b-dependence of gb (1-b)^i
                double t1 = (i > 0) ? dfa * (1.0 + a) * gb * omi1 : 0.0;
                double t2 = fa * (dgb * omi - ((i > 0) ? i * gb * omi1 : 0.0));
                Vs[nd * Np + col] = std::sqrt(2.0) * (t1 + t2);
            }
    }
}

// n-point Gauss rule of the weight (1-x)^al (1+x)^be on [-1, 1]: the roots
// of the degree-n orthonormal Jacobi polynomial by Newton's method with
// deflation, weights 1 / sum_{m<n} P_m(x)^2 (Christoffel numbers).
void gauss_jacobi(int n, double al, double be, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double t = -std::cos(M_PI * (k + 0.5) / n);
        if (k > 0 && t <= x[k - 1]) t = x[k - 1] + 1e-3 * (1.0 - x[k - 1]);
        for (int it = 0; it < 200; ++it) {
            double P = jacobi(t, al, be, n), dP = jacobi_d(t, al, be, n);
            double sum = 0.0;
            for (int j = 0; j < k; ++j) sum += 1.0 / (t - x[j]);
            double step = P / (dP - P * sum);
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[k] = t;
    }
    std::sort(x.begin(), x.end());
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int m = 0; m < n; ++m) {
            double v = jacobi(x[k], al, be, m);
            s += v * v;
        }
        w[k] = 1.0 / s;
    }
}

}  // namespace

int overint_degree(int p) { return (3 * p < 15) ? 3 * p : 15; }

bool build_overint_operators(const RefOps &o, int deg, OverintOps &out)
{
    if (o.Np < 1 || deg < 1) return false;
    const int p = o.p, Np = o.Np, n = (deg + 2) / 2;
    std::vector<double> a, wa, b, wb;
    gauss_jacobi(n, 0.0, 0.0, a, wa);
    gauss_jacobi(n, 1.0, 0.0, b, wb);
    const int Nq = n * n;
    std::vector<double> rq(Nq), sq(Nq);
    out.deg = deg;
    out.Nq = Nq;
    out.wq.assign(Nq, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const int q = i * n + j;
            rq[q] = (1.0 + a[i]) * (1.0 - b[j]) / 2.0 - 1.0;
            sq[q] = b[j];
            out.wq[q] = wa[i] * wb[j] / 2.0;
        }
    std::vector<double> V, Vr, Vs, Q, Qr, Qs, Vinv;
    vandermonde(p, o.r.data(), o.s.data(), Np, V, Vr, Vs);
    if (!invert(V, Np, Vinv)) return false;
    vandermonde(p, rq.data(), sq.data(), Nq, Q, Qr, Qs);
    out.Vq = matmul(Q, Vinv, Nq, Np, Np);
    out.Vqr = matmul(Qr, Vinv, Nq, Np, Np);
    out.Vqs = matmul(Qs, Vinv, Nq, Np, Np);
    // Sr = M^-1 Vqr^T diag(w), Ss likewise (M^-1 = V V^T)
    std::vector<double> Vt(static_cast<size_t>(Np) * Np), TrW(static_cast<size_t>(Np) * Nq), TsW(TrW.size());
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) Vt[j * Np + i] = V[i * Np + j];
    std::vector<double> Minv = matmul(V, Vt, Np, Np, Np);
    for (int i = 0; i < Np; ++i)
        for (int q = 0; q < Nq; ++q) {
            TrW[i * Nq + q] = out.Vqr[q * Np + i] * out.wq[q];
            TsW[i * Nq + q] = out.Vqs[q * Np + i] * out.wq[q];
        }
    out.Sr = matmul(Minv, TrW, Np, Np, Nq);
    out.Ss = matmul(Minv, TsW, Np, Np, Nq);
    return true;
}

bool build_reference_operators(int p, RefOps &o)
{
    if (p < 1 || p > 6) return false;
    static const double kAlpha[6] = {0.0, 0.0, 1.4152, 0.1001, 0.2751, 0.9800};
    const double alpha = kAlpha[p - 1];
    o.p = p;
    o.Np = (p + 1) * (p + 2) / 2;
    o.Nfp = p + 1;
    const int Np = o.Np, Nfp = o.Nfp;
    std::vector<double> gl = lgl(p);

    // warp-and-blend nodes on the equilateral triangle, then to (r, s)
    o.r.resize(Np);
    o.s.resize(Np);
    const double sq3 = std::sqrt(3.0);
    int idx = 0;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= p - n; ++m, ++idx) {
            double Ltop = double(n) / p;          // weight of vertex (-1, 1)
            double Lright = double(m) / p;        // weight of vertex (1, -1)
            double Lleft = 1.0 - Ltop - Lright;   // weight of vertex (-1, -1)
            double x = Lright - Lleft;
            double y = (2.0 * Ltop - Lleft - Lright) / sq3;
            // bottom edge (opposite the top vertex), direction 0
            double d1 = 4.0 * Lleft * Lright * edge_warp(p, gl, Lright - Lleft) * (1.0 + alpha * alpha * Ltop * Ltop);
            // right edge (opposite the left vertex), direction 120 degrees
            double d2 = 4.0 * Ltop * Lright * edge_warp(p, gl, Ltop - Lright) * (1.0 + alpha * alpha * Lleft * Lleft);
            // left edge (opposite the right vertex), direction 240 degrees
            double d3 = 4.0 * Ltop * Lleft * edge_warp(p, gl, Lleft - Ltop) * (1.0 + alpha * alpha * Lright * Lright);
            x += d1 - 0.5 * d2 - 0.5 * d3;
            y += 0.5 * sq3 * d2 - 0.5 * sq3 * d3;
            double B1 = (sq3 * y + 1.0) / 3.0;
            double B2 = (-3.0 * x - sq3 * y + 2.0) / 6.0;
            double B3 = (3.0 * x - sq3 * y + 2.0) / 6.0;
            o.r[idx] = -B2 + B3 - B1;
            o.s[idx] = -B2 - B3 + B1;
        }

    // Vandermonde and its derivatives
    std::vector<double> V, Vr, Vs;
    vandermonde(p, o.r.data(), o.s.data(), Np, V, Vr, Vs);
    std::vector<double> Vinv;
    if (!invert(V, Np, Vinv)) return false;
    o.Dr = matmul(Vr, Vinv, Np, Np, Np);
    o.Ds = matmul(Vs, Vinv, Np, Np, Np);
    std::vector<double> Vt(Np * Np);
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) Vt[j * Np + i] = V[i * Np + j];
    std::vector<double> Minv = matmul(V, Vt, Np, Np, Np);
    if (!invert(Minv, Np, o.Mhat)) return false;

    // face nodes, counter-clockwise: (-1,-1)->(1,-1), (1,-1)->(-1,1), (-1,1)->(-1,-1)
    const double tol = 1e-10;
    o.Fmask.assign(3 * Nfp, -1);
    std::vector<double> tface(3 * Nfp);
    for (int f = 0; f < 3; ++f) {
        std::vector<std::pair<double, int>> list;
        for (int nd = 0; nd < Np; ++nd) {
            double r = o.r[nd], s = o.s[nd];
            if (f == 0 && std::fabs(s + 1.0) < tol) list.push_back({r, nd});
            if (f == 1 && std::fabs(r + s) < tol) list.push_back({s, nd});
            if (f == 2 && std::fabs(r + 1.0) < tol) list.push_back({-s, nd});
        }
        if (static_cast<int>(list.size()) != Nfp) return false;
        std::sort(list.begin(), list.end());
        for (int i = 0; i < Nfp; ++i) {
            o.Fmask[f * Nfp + i] = list[i].second;
            tface[f * Nfp + i] = list[i].first;
        }
    }
    // 1D face mass on each face: (V1 V1^T)^-1 with orthonormal Legendre V1
    o.M1D.assign(3 * Nfp * Nfp, 0.0);
    for (int f = 0; f < 3; ++f) {
        std::vector<double> V1(Nfp * Nfp), V1t(Nfp * Nfp), Mi, M;
        for (int i = 0; i < Nfp; ++i)
            for (int n = 0; n < Nfp; ++n) {
                V1[i * Nfp + n] = jacobi(tface[f * Nfp + i], 0, 0, n);
                V1t[n * Nfp + i] = V1[i * Nfp + n];
            }
        Mi = matmul(V1, V1t, Nfp, Nfp, Nfp);
        if (!invert(Mi, Nfp, M)) return false;
        std::copy(M.begin(), M.end(), o.M1D.begin() + f * Nfp * Nfp);
    }
    o.wface.assign(Nfp, 0.0);
    for (int i = 0; i < Nfp; ++i)
        for (int l = 0; l < Nfp; ++l) o.wface[l] += o.M1D[i * Nfp + l];
    // LIFT = M^-1 E M_e
    std::vector<double> Emat(Np * 3 * Nfp, 0.0);
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i < Nfp; ++i)
            for (int l = 0; l < Nfp; ++l)
                Emat[o.Fmask[f * Nfp + i] * (3 * Nfp) + f * Nfp + l] += o.M1D[f * Nfp * Nfp + i * Nfp + l];
    o.LIFT = matmul(Minv, Emat, Np, Np, 3 * Nfp);
    // Wr = M^-1 Dr^T M, Ws = M^-1 Ds^T M: nodal values of the function whose
    // L2 product with any l_i equals the product of the input with d l_i/dr
    std::vector<double> Drt(Np * Np), Dst(Np * Np);
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) {
            Drt[j * Np + i] = o.Dr[i * Np + j];
            Dst[j * Np + i] = o.Ds[i * Np + j];
        }
    o.Wr = matmul(matmul(Minv, Drt, Np, Np, Np), o.Mhat, Np, Np, Np);
    o.Ws = matmul(matmul(Minv, Dst, Np, Np, Np), o.Mhat, Np, Np, Np);
    return true;
}

}  // namespace dg
