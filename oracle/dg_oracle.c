/*
 * dg_oracle.c -- plain FP64 CPU oracle for the nodal interior-penalty DG
 * discretisation of the 2D compressible Navier-Stokes equations.
 *
 * Oracle header: test infrastructure only.  Tests, the smoke check and the
 * CPU-baseline leg of the benchmark may call this code; the CUDA library
 * never links or includes it, and it includes nothing from the library.
 *
 * It executes the method step by step in the paper's weak form, with plain
 * loops and no blocking or fusion:
 *   - conserved state U = (rho, rho v1, rho v2, eps), eps = total energy per
 *     volume (Sec. 2.1); pressure p = (gamma-1)(eps - rho|v|^2/2);
 *   - advective flux F_c minus the mesh-motion term v_w (x) U (Sec. 2.1);
 *   - viscous flux F_v = G(U) grad U with the four 4x4 blocks G11, G12, G21,
 *     G22 written out entry by entry as printed (Sec. 2.1);
 *   - broken gradient grad_h U = (rx Dr + sx Ds, ry Dr + sy Ds) U;
 *   - Roe flux with moving-wall eigenvalues, built as R |Lambda| R^-1 with an
 *     explicit eigenvector matrix and a Gauss-Jordan inverse (Eq. roe_flux);
 *   - interior-penalty diffusion flux for theta in [-1, 1] (Eq. ip_flux): the
 *     consistency and penalty terms through the face flux H_m, and the theta
 *     term H_theta of Eq. dg_on_K tested against grad l_i on the face, with
 *     weight 1/2 (the average) on interior faces and 1 on boundary faces,
 *     G taken at U+ (interior, far field) or at the wall state U^b;
 *   - penalty sigma_e = C1 (1+theta)^2 (d+1) Gbar_e max C_inv (Eq.
 *     penalty_final) with Gbar_e the largest spectral norm of
 *     N G N^T = n1^2 G11 + n1 n2 (G12+G21) + n2^2 G22 over the face nodes of
 *     both sides, the norm from a cyclic Jacobi eigen-solve of A^T A;
 *   - far-field and moving adiabatic wall terms (Sec. 2.2, boundary term);
 *   - residual R = M^-1 (S_x F_x + S_y F_y - sum_e E^e M_e H) (Eq. dg_on_K),
 *     with S = Dr^T M etc. written as the weak form;
 *   - 2N-storage five-stage Runge-Kutta step (Algorithm 1);
 *   - time step from the bound Lambda of Eq. rayleigh_bound (Appendix A);
 *   - wall force and moment, and the Newmark step of the 1-DOF oscillator
 *     (Eq. 1dof_oscillator, Algorithm 3).
 *
 * Readings where the paper is garbled or silent (pressure law, Roe factor
 * 1/2 and eigenvalue signs, boundary-face penalty, adiabatic heat flux, CFL
 * constants, which side's G the theta term uses on far-field faces) are
 * listed in the project's design notes and repeated next to the code that
 * takes them.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int p, Np, Nfp, K;
    const double *Dr, *Ds, *Mhat, *Minv;   /* Np*Np row-major */
    const long long *Fmask;                 /* 3*Nfp volume index of face node */
    const double *M1D;                      /* 3*Nfp*Nfp face mass per face */
    const double *rx, *ry, *sx, *sy, *J;    /* K */
    const double *nx, *ny, *sJ;             /* K*3 outward unit normal, |e|/2 */
    const long long *EToE, *EToF, *bc;      /* K*3 */
    const long long *mapP;                  /* K*3*Nfp neighbour volume node index */
    const double *x, *y;                    /* K*Np node coordinates */
    double gamma, Pr, mu, theta, C1;
    double rho_inf, u_inf, v_inf, p_inf;
    long long adiabatic_zero_heatflux;
    long long source_kind;                  /* 0 none, 1 manufactured solution of Sec. 3.1 */
    double src_kappa, src_C2;
    /* over-integration of the volume term (Sec. 2.2, weak matrices): Nq > 0
     * evaluates the flux at Nq cubature points, with the nodal basis values
     * Vq and derivatives Vqr, Vqs [Nq][Np] there and weights wq [Nq] */
    long long Nq;
    const double *Vq, *Vqr, *Vqs, *wq;
} oracle_problem;

enum { BC_INTERIOR = 0, BC_WALL = 1, BC_FARFIELD = 2 };

/* Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients. */
static const double RK_A[5] = {
    0.0,
    -567301805773.0 / 1357537059087.0,
    -2404267990393.0 / 2016746695238.0,
    -3550918686646.0 / 2091501179385.0,
    -1275806237668.0 / 842570457699.0};
static const double RK_B[5] = {
    1432997174477.0 / 9575080441755.0,
    5161836677717.0 / 13612068292357.0,
    1720146321549.0 / 2090206949498.0,
    3134564353537.0 / 4481467310338.0,
    2277821191437.0 / 14882151754819.0};
static const double RK_C[5] = {
    0.0,
    1432997174477.0 / 9575080441755.0,
    2526269341429.0 / 6820363962896.0,
    2006345519317.0 / 3224310063776.0,
    2802321613138.0 / 2924317926251.0};

void oracle_lsrk_coeffs(double *A, double *B, double *c)
{
    for (int i = 0; i < 5; ++i) { A[i] = RK_A[i]; B[i] = RK_B[i]; c[i] = RK_C[i]; }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- physics */

/* p = (gamma-1)(eps - rho |v|^2 / 2), eps = total energy per volume. */
static double pressure(const double U[4], double gamma)
{
    double v1 = U[1] / U[0], v2 = U[2] / U[0];
    return (gamma - 1.0) * (U[3] - 0.5 * U[0] * (v1 * v1 + v2 * v2));
}

/* F_c - v_w (x) U in both directions (Sec. 2.1). */
static void adv_flux(const double U[4], const double vw[2], double gamma,
                     double Fx[4], double Fy[4])
{
    double rho = U[0], v1 = U[1] / rho, v2 = U[2] / rho, p = pressure(U, gamma);
    Fx[0] = rho * v1;
    Fx[1] = rho * v1 * v1 + p;
    Fx[2] = rho * v1 * v2;
    Fx[3] = v1 * (p + U[3]);
    Fy[0] = rho * v2;
    Fy[1] = rho * v1 * v2;
    Fy[2] = rho * v2 * v2 + p;
    Fy[3] = v2 * (p + U[3]);
    for (int c = 0; c < 4; ++c) {
        Fx[c] -= vw[0] * U[c];
        Fy[c] -= vw[1] * U[c];
    }
}

/* n . (F_c - v_w (x) U) */
void oracle_flux_n(const double U[4], const double n[2], const double vw[2],
                   double gamma, double F[4])
{
    double Fx[4], Fy[4];
    adv_flux(U, vw, gamma, Fx, Fy);
    for (int c = 0; c < 4; ++c) F[c] = n[0] * Fx[c] + n[1] * Fy[c];
}

/* The four blocks of G(U), entry by entry (Sec. 2.1).  G[a][b] is G_{a+1,b+1};
 * stored row-major 4x4. */
void oracle_G_blocks(const double U[4], double gamma, double Pr, double mu,
                     double G[2][2][16])
{
    double rho = U[0], v1 = U[1] / rho, v2 = U[2] / rho, e = U[3] / rho;
    double vsq = v1 * v1 + v2 * v2, g = gamma / Pr, f = mu / rho;
    double g41_1 = -v1 * v1 / 3.0 - vsq - g * (e - vsq);
    double g41_2 = -v2 * v2 / 3.0 - vsq - g * (e - vsq);
    double G11[16] = {0, 0, 0, 0,
                      -4.0 / 3.0 * v1, 4.0 / 3.0, 0, 0,
                      -v2, 0, 1, 0,
                      g41_1, (4.0 / 3.0 - g) * v1, (1.0 - g) * v2, g};
    double G12[16] = {0, 0, 0, 0,
                      2.0 / 3.0 * v2, 0, -2.0 / 3.0, 0,
                      -v1, 1, 0, 0,
                      -v1 * v2 / 3.0, v2, -2.0 / 3.0 * v1, 0};
    double G21[16] = {0, 0, 0, 0,
                      -v2, 0, 1, 0,
                      2.0 / 3.0 * v1, -2.0 / 3.0, 0, 0,
                      -v1 * v2 / 3.0, -2.0 / 3.0 * v2, v1, 0};
    double G22[16] = {0, 0, 0, 0,
                      -v1, 1, 0, 0,
                      -4.0 / 3.0 * v2, 0, 4.0 / 3.0, 0,
                      g41_2, (1.0 - g) * v1, (4.0 / 3.0 - g) * v2, g};
    for (int i = 0; i < 16; ++i) {
        G[0][0][i] = f * G11[i];
        G[0][1][i] = f * G12[i];
        G[1][0][i] = f * G21[i];
        G[1][1][i] = f * G22[i];
    }
}

/* F_v = G(U) grad U: Fvx = G11 Ux + G12 Uy, Fvy = G21 Ux + G22 Uy. */
static void visc_flux(const double U[4], const double Ux[4], const double Uy[4],
                      double gamma, double Pr, double mu, double Fvx[4], double Fvy[4])
{
    double G[2][2][16];
    oracle_G_blocks(U, gamma, Pr, mu, G);
    for (int i = 0; i < 4; ++i) {
        double ax = 0, ay = 0;
        for (int j = 0; j < 4; ++j) {
            ax += G[0][0][4 * i + j] * Ux[j] + G[0][1][4 * i + j] * Uy[j];
            ay += G[1][0][4 * i + j] * Ux[j] + G[1][1][4 * i + j] * Uy[j];
        }
        Fvx[i] = ax;
        Fvy[i] = ay;
    }
}

/* Largest eigenvalue of a symmetric 4x4 matrix by cyclic Jacobi rotations. */
static double sym4_max_eig(double S[16])
{
    double a[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) a[i][j] = S[4 * i + j];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                tot += a[i][j] * a[i][j];
                if (i != j) off += a[i][j] * a[i][j];
            }
        if (off <= 1e-32 * tot || tot == 0.0) break;
        for (int pi = 0; pi < 3; ++pi)
            for (int q = pi + 1; q < 4; ++q) {
                if (a[pi][q] == 0.0) continue;
                double theta = (a[q][q] - a[pi][pi]) / (2.0 * a[pi][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) {           /* columns pi, q */
                    double akp = a[k][pi], akq = a[k][q];
                    a[k][pi] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {           /* rows pi, q */
                    double apk = a[pi][k], aqk = a[q][k];
                    a[pi][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
            }
    }
    double m = a[0][0];
    for (int i = 1; i < 4; ++i) if (a[i][i] > m) m = a[i][i];
    return m;
}

/* || n1^2 G11 + n1 n2 (G12 + G21) + n2^2 G22 ||_2 at state U (Sec. 2.2, penalty). */
double oracle_penalty_norm(const double U[4], const double n[2], double gamma,
                           double Pr, double mu)
{
    double G[2][2][16], A[16], S[16];
    oracle_G_blocks(U, gamma, Pr, mu, G);
    for (int i = 0; i < 16; ++i)
        A[i] = n[0] * n[0] * G[0][0][i] + n[0] * n[1] * (G[0][1][i] + G[1][0][i])
             + n[1] * n[1] * G[1][1][i];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0;
            for (int k = 0; k < 4; ++k) acc += A[4 * k + i] * A[4 * k + j];
            S[4 * i + j] = acc;
        }
    double lam = sym4_max_eig(S);
    return sqrt(lam > 0 ? lam : 0.0);
}

/* Inverse of a 4x4 matrix by Gauss-Jordan elimination with partial pivoting. */
static int inv4(const double A[16], double X[16])
{
    double a[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            a[i][j] = A[4 * i + j];
            a[i][4 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 8; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[col][col];
        for (int j = 0; j < 8; ++j) a[col][j] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int j = 0; j < 8; ++j) a[r][j] -= m * a[col][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) X[4 * i + j] = a[i][4 + j];
    return 0;
}

/* Roe flux at one face node (Eq. roe_flux, reading: 1/2 (F_n^+ + F_n^-) +
 * 1/2 |A| (U^+ - U^-), |A| = R |Lambda| R^-1 with eigenvalues
 * (v~ - v_w).n - c~, (v~ - v_w).n (twice), (v~ - v_w).n + c~ and Roe averages
 * weighted by sqrt(rho); H = (eps + p)/rho is the total enthalpy).
 * Optional outputs: Asigned = R Lambda R^-1, Aabs = R |Lambda| R^-1. */
int oracle_roe(const double Up[4], const double Um[4], const double n[2],
               const double vw[2], double gamma, double H[4],
               double *Asigned, double *Aabs)
{
    double wp = sqrt(Up[0]), wm = sqrt(Um[0]);
    double vp1 = Up[1] / Up[0], vp2 = Up[2] / Up[0];
    double vm1 = Um[1] / Um[0], vm2 = Um[2] / Um[0];
    double Hp = (Up[3] + pressure(Up, gamma)) / Up[0];
    double Hm = (Um[3] + pressure(Um, gamma)) / Um[0];
    double v1 = (wp * vp1 + wm * vm1) / (wp + wm);
    double v2 = (wp * vp2 + wm * vm2) / (wp + wm);
    double Ht = (wp * Hp + wm * Hm) / (wp + wm);
    double q2 = v1 * v1 + v2 * v2;
    double c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
    if (!(c2 > 0)) return -1;
    double c = sqrt(c2);
    double n1 = n[0], n2 = n[1], t1 = -n2, t2 = n1;
    double un = v1 * n1 + v2 * n2, ut = v1 * t1 + v2 * t2;
    double vwn = vw[0] * n1 + vw[1] * n2;
    /* right eigenvectors as columns */
    double R[16] = {
        1.0,             1.0,        0.0, 1.0,
        v1 - c * n1,     v1,         t1,  v1 + c * n1,
        v2 - c * n2,     v2,         t2,  v2 + c * n2,
        Ht - c * un,     0.5 * q2,   ut,  Ht + c * un};
    double lam[4] = {un - c - vwn, un - vwn, un - vwn, un + c - vwn};
    double Ri[16];
    if (inv4(R, Ri) != 0) return -1;
    double As[16], Aa[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0, a = 0;
            for (int k = 0; k < 4; ++k) {
                s += R[4 * i + k] * lam[k] * Ri[4 * k + j];
                a += R[4 * i + k] * fabs(lam[k]) * Ri[4 * k + j];
            }
            As[4 * i + j] = s;
            Aa[4 * i + j] = a;
        }
    if (Asigned) memcpy(Asigned, As, sizeof As);
    if (Aabs) memcpy(Aabs, Aa, sizeof Aa);
    if (H) {
        double Fp[4], Fm[4];
        oracle_flux_n(Up, n, vw, gamma, Fp);
        oracle_flux_n(Um, n, vw, gamma, Fm);
        for (int i = 0; i < 4; ++i) {
            double d = 0;
            for (int j = 0; j < 4; ++j) d += Aa[4 * i + j] * (Up[j] - Um[j]);
            H[i] = 0.5 * (Fp[i] + Fm[i]) + 0.5 * d;
        }
    }
    return 0;
}

/* Far-field ghost state U^b = (rho_inf, rho_inf v_inf, eps_inf). */
static void farfield_state(const oracle_problem *P, double Ub[4])
{
    double r = P->rho_inf, u = P->u_inf, v = P->v_inf;
    Ub[0] = r;
    Ub[1] = r * u;
    Ub[2] = r * v;
    Ub[3] = P->p_inf / (P->gamma - 1.0) + 0.5 * r * (u * u + v * v);
}

/* Wall ghost state from Q^b = (rho^+, v_w, p^+). */
static void wall_state(const double Up[4], const double vw[2], double gamma, double Ub[4])
{
    double r = Up[0], p = pressure(Up, gamma);
    Ub[0] = r;
    Ub[1] = r * vw[0];
    Ub[2] = r * vw[1];
    Ub[3] = p / (gamma - 1.0) + 0.5 * r * (vw[0] * vw[0] + vw[1] * vw[1]);
}

/* ---------------------------------------------------------------- helpers */

static void load_node(const double *U, int Np, long long k, long long i, double out[4])
{
    for (int c = 0; c < 4; ++c) out[c] = U[(k * 4 + c) * Np + i];
}

/* grad_h U at every node: Ux[k][c][i] = sum_j (rx Dr_ij + sx Ds_ij) U[k][c][j]. */
static void broken_gradient(const oracle_problem *P, const double *U, double *Ux, double *Uy)
{
    int Np = P->Np;
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < P->K; ++k) {
        for (int c = 0; c < 4; ++c) {
            const double *u = U + (k * 4 + c) * Np;
            for (int i = 0; i < Np; ++i) {
                double ur = 0, us = 0;
                for (int j = 0; j < Np; ++j) {
                    ur += P->Dr[i * Np + j] * u[j];
                    us += P->Ds[i * Np + j] * u[j];
                }
                Ux[(k * 4 + c) * Np + i] = P->rx[k] * ur + P->sx[k] * us;
                Uy[(k * 4 + c) * Np + i] = P->ry[k] * ur + P->sy[k] * us;
            }
        }
    }
}

/* C_inv(e, K, p) = (p+1)(p+d)|e| / (d |K|), d = 2, |e| = 2 sJ, |K| = 2 J. */
static double cinv(const oracle_problem *P, long long k, int f)
{
    double e = 2.0 * P->sJ[k * 3 + f], area = 2.0 * P->J[k];
    return (P->p + 1.0) * (P->p + 2.0) * e / (2.0 * area);
}

/* Penalty of face f of element k (Eq. penalty_final), given the other side's
 * states at the face nodes (neighbour trace or ghost state). */
static double face_sigma(const oracle_problem *P, long long k, int f,
                         const double (*Uplus)[4], const double (*Uother)[4])
{
    double n[2] = {P->nx[k * 3 + f], P->ny[k * 3 + f]};
    double Gbar = 0;
    for (int i = 0; i < P->Nfp; ++i) {
        double a = oracle_penalty_norm(Uplus[i], n, P->gamma, P->Pr, P->mu);
        double b = oracle_penalty_norm(Uother[i], n, P->gamma, P->Pr, P->mu);
        if (a > Gbar) Gbar = a;
        if (b > Gbar) Gbar = b;
    }
    double ci = cinv(P, k, f);
    if (P->bc[k * 3 + f] == BC_INTERIOR) {
        long long k2 = P->EToE[k * 3 + f];
        int f2 = (int)P->EToF[k * 3 + f];
        double c2 = cinv(P, k2, f2);
        if (c2 > ci) ci = c2;
    }
    double d = 2.0;
    return P->C1 * (1.0 + P->theta) * (1.0 + P->theta) * (d + 1.0) * Gbar * ci;
}

/* Gather, for face f of element k, the own trace, the other side's trace
 * (neighbour or ghost) and both gradients at the Nfp face nodes. */
static void face_traces(const oracle_problem *P, const double *U, const double *Ux,
                        const double *Uy, const double vw[2], long long k, int f,
                        double (*Up)[4], double (*Upx)[4], double (*Upy)[4],
                        double (*Uo)[4], double (*Uox)[4], double (*Uoy)[4])
{
    int Np = P->Np, Nfp = P->Nfp;
    long long btype = P->bc[k * 3 + f];
    for (int i = 0; i < Nfp; ++i) {
        long long vm = P->Fmask[f * Nfp + i];
        load_node(U, Np, k, vm, Up[i]);
        load_node(Ux, Np, k, vm, Upx[i]);
        load_node(Uy, Np, k, vm, Upy[i]);
        if (btype == BC_INTERIOR) {
            long long k2 = P->EToE[k * 3 + f];
            long long vp = P->mapP[(k * 3 + f) * Nfp + i];
            load_node(U, Np, k2, vp, Uo[i]);
            load_node(Ux, Np, k2, vp, Uox[i]);
            load_node(Uy, Np, k2, vp, Uoy[i]);
        } else if (btype == BC_FARFIELD) {
            farfield_state(P, Uo[i]);
            memcpy(Uox[i], Upx[i], sizeof(double) * 4);
            memcpy(Uoy[i], Upy[i], sizeof(double) * 4);
        } else {
            wall_state(Up[i], vw, P->gamma, Uo[i]);
            memcpy(Uox[i], Upx[i], sizeof(double) * 4);
            memcpy(Uoy[i], Upy[i], sizeof(double) * 4);
        }
    }
}

/* Numerical face flux H at one face node, oriented along the outward normal
 * of element k.  Interior and far field: Roe - {G grad U}.n + sigma [U];
 * wall: n.(F_c(U^b) - v_w (x) U^b) - G(U^b) grad U^+ . n + sigma (U^+ - U^b). */
static int face_flux(const oracle_problem *P, long long btype, const double n[2],
                     const double vw[2], double sigma,
                     const double Up[4], const double Upx[4], const double Upy[4],
                     const double Uo[4], const double Uox[4], const double Uoy[4],
                     double H[4])
{
    double g = P->gamma, Pr = P->Pr, mu = P->mu;
    double vx[4], vy[4];
    if (btype == BC_WALL) {
        double Fn[4];
        oracle_flux_n(Uo, n, vw, g, Fn);
        visc_flux(Uo, Upx, Upy, g, Pr, mu, vx, vy);
        double vn[4];
        for (int c = 0; c < 4; ++c) vn[c] = vx[c] * n[0] + vy[c] * n[1];
        if (P->adiabatic_zero_heatflux) {
            /* keep only the work of the viscous stress: v_w . (tau n) */
            vn[3] = vw[0] * vn[1] + vw[1] * vn[2];
        }
        for (int c = 0; c < 4; ++c) H[c] = Fn[c] - vn[c] + sigma * (Up[c] - Uo[c]);
        return 0;
    }
    double Hc[4];
    if (oracle_roe(Up, Uo, n, vw, g, Hc, NULL, NULL) != 0) return -1;
    double px[4], py[4];
    visc_flux(Up, Upx, Upy, g, Pr, mu, px, py);
    if (btype == BC_INTERIOR) {
        double ox[4], oy[4];
        visc_flux(Uo, Uox, Uoy, g, Pr, mu, ox, oy);
        for (int c = 0; c < 4; ++c) {
            double avg = 0.5 * ((px[c] + ox[c]) * n[0] + (py[c] + oy[c]) * n[1]);
            H[c] = Hc[c] - avg + sigma * (Up[c] - Uo[c]);
        }
    } else { /* far field: {G grad U} = G(U^+) grad U^+ on the boundary */
        for (int c = 0; c < 4; ++c)
            H[c] = Hc[c] - (px[c] * n[0] + py[c] * n[1]) + sigma * (Up[c] - Uo[c]);
    }
    return 0;
}

/* Source of the manufactured steady solution of Sec. 3.1:
 * U = (w, w, w, w^2), w = sin(phi) + C2, phi = kappa (x + y), so v = (1, 1),
 * eps/rho = w and p = (gamma-1)(w^2 - w).  S = div F_c(U) - div F_v(U),
 * derived here from U, the pressure law and the G blocks (the velocity is
 * constant, so only the heat-flux row of F_v survives):
 *   S_1 = 2 kappa cos(phi)
 *   S_2 = S_3 = kappa g1 sin(2 phi) + (2 kappa - kappa g1 + 2 kappa C2 g1) cos(phi)
 *   S_4 = 2 kappa gamma sin(2 phi) + (4 kappa gamma C2 - 2 kappa g1) cos(phi)
 *         + 2 gamma mu kappa^2 sin(phi) / Pr,          g1 = gamma - 1.
 * (The printed source carries 1/2 and 1 where this derivation gives 1 and 2
 * in front of the g1 cos terms.) */
void oracle_manufactured_source(double x, double y, double kappa, double C2, double gamma,
                                double Pr, double mu, double S[4])
{
    double phi = kappa * (x + y), g1 = gamma - 1.0;
    double sp = sin(phi), cp = cos(phi), s2 = sin(2.0 * phi);
    S[0] = 2.0 * kappa * cp;
    S[1] = kappa * g1 * s2 + (2.0 * kappa - kappa * g1 + 2.0 * kappa * C2 * g1) * cp;
    S[2] = S[1];
    S[3] = 2.0 * kappa * gamma * s2 + (4.0 * kappa * gamma * C2 - 2.0 * kappa * g1) * cp
         + 2.0 * gamma * mu * kappa * kappa * sp / Pr;
}

/* theta term of the IP flux (Eq. ip_flux, H_theta of Eq. dg_on_K) at one face
 * node: the 8-vector (U+ - U-)^T N G(U*) with N = n^T (x) I4, i.e.
 * t_x[k] = sum_c dU_c (n1 G11 + n2 G21)_{c,k},  t_y[k] = sum_c dU_c (n1 G12 + n2 G22)_{c,k},
 * G evaluated at Ustar (U+ on interior and far-field faces, U^b on walls). */
static void theta_vector(const double dU[4], const double Ustar[4], const double n[2], double gamma,
                         double Pr, double mu, double tx[4], double ty[4])
{
    double G[2][2][16];
    oracle_G_blocks(Ustar, gamma, Pr, mu, G);
    for (int k = 0; k < 4; ++k) {
        double ax = 0, ay = 0;
        for (int c = 0; c < 4; ++c) {
            ax += dU[c] * (n[0] * G[0][0][4 * c + k] + n[1] * G[1][0][4 * c + k]);
            ay += dU[c] * (n[0] * G[0][1][4 * c + k] + n[1] * G[1][1][4 * c + k]);
        }
        tx[k] = ax;
        ty[k] = ay;
    }
}

/* ---------------------------------------------------------------- residual */

/* R = M^-1 [ (S_x F_x + S_y F_y) - S_x H_theta,x - S_y H_theta,y - sum_e E^e M_e H_m ]
 * (Eq. dg_on_K); H_theta = -theta (U+ - U-)^T N G grad l_i, so its terms enter with +theta.
 * U, R: [K][4][Np]. */
int oracle_rhs(const oracle_problem *P, const double *U, double t, const double vw[2], double *R)
{
    (void)t;
    int Np = P->Np, Nfp = P->Nfp;
    long long K = P->K;
    size_t nd = (size_t)K * 4 * Np;
    double *Ux = malloc(nd * sizeof(double)), *Uy = malloc(nd * sizeof(double));
    if (!Ux || !Uy) { free(Ux); free(Uy); return -1; }
    broken_gradient(P, U, Ux, Uy);
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (long long k = 0; k < K; ++k) {
        double Fx[4][32], Fy[4][32];      /* total flux F = F_c - v_w U - F_v at nodes */
        for (int i = 0; i < Np; ++i) {
            double u[4], ux[4], uy[4], cx[4], cy[4], vx[4], vy[4];
            load_node(U, Np, k, i, u);
            load_node(Ux, Np, k, i, ux);
            load_node(Uy, Np, k, i, uy);
            adv_flux(u, vw, P->gamma, cx, cy);
            visc_flux(u, ux, uy, P->gamma, P->Pr, P->mu, vx, vy);
            for (int c = 0; c < 4; ++c) {
                Fx[c][i] = cx[c] - vx[c];
                Fy[c][i] = cy[c] - vy[c];
            }
        }
        /* face terms q_i = sum_e E^e (M_e H)_i, with M_e = sJ * M1D */
        double q[4][32];
        memset(q, 0, sizeof q);
        /* theta terms: th[c][i] = theta w int_e (dx l_i t_x[c] + dy l_i t_y[c]) ds */
        double th[4][32];
        memset(th, 0, sizeof th);
        for (int f = 0; f < 3; ++f) {
            double Up[8][4], Upx[8][4], Upy[8][4], Uo[8][4], Uox[8][4], Uoy[8][4], H[8][4];
            face_traces(P, U, Ux, Uy, vw, k, f, Up, Upx, Upy, Uo, Uox, Uoy);
            double sigma = face_sigma(P, k, f, (const double (*)[4])Up, (const double (*)[4])Uo);
            double n[2] = {P->nx[k * 3 + f], P->ny[k * 3 + f]};
            long long btype = P->bc[k * 3 + f];
            for (int i = 0; i < Nfp; ++i)
                err |= (face_flux(P, btype, n, vw, sigma, Up[i], Upx[i], Upy[i],
                                  Uo[i], Uox[i], Uoy[i], H[i]) != 0);
            const double *M1 = P->M1D + (size_t)f * Nfp * Nfp;
            double sJ = P->sJ[k * 3 + f];
            for (int i = 0; i < Nfp; ++i) {
                long long vm = P->Fmask[f * Nfp + i];
                for (int c = 0; c < 4; ++c) {
                    double acc = 0;
                    for (int l = 0; l < Nfp; ++l) acc += M1[i * Nfp + l] * H[l][c];
                    q[c][vm] += sJ * acc;
                }
            }
            if (P->theta != 0.0) {
                /* w = 1/2 from the average {{G grad Phi}} on interior faces, 1 on boundary
                 * faces; G at U+ (interior, far field) or at the wall state U^b */
                double w = (btype == BC_INTERIOR) ? 0.5 : 1.0;
                double tx[8][4], ty[8][4];
                for (int l = 0; l < Nfp; ++l) {
                    double dU[4];
                    for (int c = 0; c < 4; ++c) dU[c] = Up[l][c] - Uo[l][c];
                    const double *Ustar = (btype == BC_WALL) ? Uo[l] : Up[l];
                    theta_vector(dU, Ustar, n, P->gamma, P->Pr, P->mu, tx[l], ty[l]);
                }
                /* int_e f g ds = sJ f^T M1D g for face polynomials f, g; g = d l_i / dx at
                 * the face nodes, from the rows of Dr, Ds at those nodes */
                double rx = P->rx[k], ry = P->ry[k], sx = P->sx[k], sy = P->sy[k];
                for (int ii = 0; ii < Np; ++ii)
                    for (int m = 0; m < Nfp; ++m) {
                        long long vm = P->Fmask[f * Nfp + m];
                        double dxl = rx * P->Dr[vm * Np + ii] + sx * P->Ds[vm * Np + ii];
                        double dyl = ry * P->Dr[vm * Np + ii] + sy * P->Ds[vm * Np + ii];
                        for (int c = 0; c < 4; ++c) {
                            double fx = 0, fy = 0;
                            for (int l = 0; l < Nfp; ++l) {
                                fx += M1[m * Nfp + l] * tx[l][c];
                                fy += M1[m * Nfp + l] * ty[l][c];
                            }
                            th[c][ii] += P->theta * w * sJ * (dxl * fx + dyl * fy);
                        }
                    }
            }
        }
        /* weak volume term (Dr^T M F) scaled by the metric, then M^-1 */
        double rx = P->rx[k], ry = P->ry[k], sx = P->sx[k], sy = P->sy[k], J = P->J[k];
        /* over-integrated volume term: int F . grad l_m = sum_q w_q F(U_q, grad U_q) . grad l_m(x_q) */
        double oiv[4][32];
        if (P->Nq > 0) {
            memset(oiv, 0, sizeof oiv);
            for (long long qn = 0; qn < P->Nq; ++qn) {
                double u[4], ur[4], us[4], ux[4], uy[4], cx[4], cy[4], vx[4], vy[4];
                for (int c = 0; c < 4; ++c) {
                    double a = 0, b = 0, d = 0;
                    for (int j = 0; j < Np; ++j) {
                        double uj = U[(k * 4 + c) * Np + j];
                        a += P->Vq[qn * Np + j] * uj;
                        b += P->Vqr[qn * Np + j] * uj;
                        d += P->Vqs[qn * Np + j] * uj;
                    }
                    u[c] = a;
                    ur[c] = b;
                    us[c] = d;
                    ux[c] = rx * b + sx * d;
                    uy[c] = ry * b + sy * d;
                }
                (void)ur;
                (void)us;
                adv_flux(u, vw, P->gamma, cx, cy);
                visc_flux(u, ux, uy, P->gamma, P->Pr, P->mu, vx, vy);
                for (int m = 0; m < Np; ++m) {
                    double lx = rx * P->Vqr[qn * Np + m] + sx * P->Vqs[qn * Np + m];
                    double ly = ry * P->Vqr[qn * Np + m] + sy * P->Vqs[qn * Np + m];
                    for (int c = 0; c < 4; ++c)
                        oiv[c][m] += P->wq[qn] * (lx * (cx[c] - vx[c]) + ly * (cy[c] - vy[c]));
                }
            }
        }
        for (int c = 0; c < 4; ++c) {
            double a[32], b[32], vol[32];
            for (int j = 0; j < Np; ++j) {
                double sa = 0, sb = 0;
                for (int l = 0; l < Np; ++l) {
                    sa += P->Mhat[j * Np + l] * Fx[c][l];
                    sb += P->Mhat[j * Np + l] * Fy[c][l];
                }
                a[j] = sa;
                b[j] = sb;
            }
            for (int m = 0; m < Np; ++m) {
                double acc = 0;
                for (int j = 0; j < Np; ++j)
                    acc += (rx * P->Dr[j * Np + m] + sx * P->Ds[j * Np + m]) * a[j]
                         + (ry * P->Dr[j * Np + m] + sy * P->Ds[j * Np + m]) * b[j];
                if (P->Nq > 0) acc = oiv[c][m];
                /* (1/J) M^-1 of [ J * vol - face + theta terms ] */
                vol[m] = acc - q[c][m] / J + th[c][m] / J;
            }
            for (int i = 0; i < Np; ++i) {
                double acc = 0;
                for (int m = 0; m < Np; ++m) acc += P->Minv[i * Np + m] * vol[m];
                R[(k * 4 + c) * Np + i] = acc;
            }
        }
        if (P->source_kind == 1) {   /* nodal source (collocation) */
            for (int i = 0; i < Np; ++i) {
                double S[4];
                oracle_manufactured_source(P->x[k * Np + i], P->y[k * Np + i], P->src_kappa,
                                           P->src_C2, P->gamma, P->Pr, P->mu, S);
                for (int c = 0; c < 4; ++c) R[(k * 4 + c) * Np + i] += S[c];
            }
        }
    }
    free(Ux);
    free(Uy);
    return err ? -4 : 0;
}

/* Algorithm 1: K0 <- U; for each stage K1 <- A_i K1 + dt M^-1 R(t + c_i dt, K0);
 * K0 <- K0 + B_i K1; U <- K0.  The register K1 starts at zero. */
int oracle_lsrk_step(const oracle_problem *P, double *U, double t, double dt, const double vw[2])
{
    size_t nd = (size_t)P->K * 4 * P->Np;
    double *K1 = calloc(nd, sizeof(double)), *R = malloc(nd * sizeof(double));
    if (!K1 || !R) { free(K1); free(R); return -1; }
    int st = 0;
    for (int s = 0; s < 5 && st == 0; ++s) {
        st = oracle_rhs(P, U, t + RK_C[s] * dt, vw, R);
        for (size_t i = 0; i < nd; ++i) {
            K1[i] = RK_A[s] * K1[i] + dt * R[i];
            U[i] = U[i] + RK_B[s] * K1[i];
        }
    }
    free(K1);
    free(R);
    return st;
}

/* Broken gradient of U, Ux and Uy [K][4][Np] (for tests). */
int oracle_broken_gradient(const oracle_problem *P, const double *U, double *Ux, double *Uy)
{
    broken_gradient(P, U, Ux, Uy);
    return 0;
}

/* Penalty sigma_e of every face, [K][3] (for tests and the time step). */
int oracle_face_sigma(const oracle_problem *P, const double *U, const double vw[2], double *sigma)
{
    int Np = P->Np;
    size_t nd = (size_t)P->K * 4 * Np;
    double *Ux = malloc(nd * sizeof(double)), *Uy = malloc(nd * sizeof(double));
    if (!Ux || !Uy) { free(Ux); free(Uy); return -1; }
    broken_gradient(P, U, Ux, Uy);
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < P->K; ++k)
        for (int f = 0; f < 3; ++f) {
            double Up[8][4], Upx[8][4], Upy[8][4], Uo[8][4], Uox[8][4], Uoy[8][4];
            face_traces(P, U, Ux, Uy, vw, k, f, Up, Upx, Upy, Uo, Uox, Uoy);
            sigma[k * 3 + f] = face_sigma(P, k, f, (const double (*)[4])Up, (const double (*)[4])Uo);
        }
    free(Ux);
    free(Uy);
    return 0;
}

/* Largest diffusivity of the system on face f of element k: the largest
 * eigenvalue of N G N^T over the face nodes of both traces.  For a unit normal
 * N G N^T maps the normal derivative of U to the normal viscous flux; written
 * in (rho, rho v.n, rho v.t, eps) it is lower triangular with diagonal
 * (0, 4/3, 1, gamma/Pr) mu/rho, so the eigenvalue is max(4/3, gamma/Pr) mu/rho
 * whatever the normal (and whatever variables the system is written in). */
static double face_diffusivity(const oracle_problem *P, const double (*Uplus)[4],
                               const double (*Uother)[4])
{
    double gmax = P->gamma / P->Pr > 4.0 / 3.0 ? P->gamma / P->Pr : 4.0 / 3.0;
    double G = 0;
    for (int i = 0; i < P->Nfp; ++i) {
        double a = gmax * P->mu / Uplus[i][0];
        double b = gmax * P->mu / Uother[i][0];
        if (a > G) G = a;
        if (b > G) G = b;
    }
    return G;
}

/* Time step from Eq. rayleigh_bound: dt = CFL / max_K Lambda_K with
 * Lambda_K = 3/2 C_inv2(K) G_K + (d+1) C_inv,K (3 sigma_K + beta_K) + beta'_K.
 * Readings: C_inv2 = p^4 / rho_K^2 (C_grad = 1, rho_K the inradius);
 * G_K, the diffusion coefficient of the Appendix's scalar model problem, is the
 * largest diffusivity of the system, max(4/3, gamma/Pr) mu/rho, over the
 * face-node traces of both sides of every face of K (face_diffusivity);
 * sigma_K = max_e sigma_e, the penalty of Eq. penalty_final actually applied;
 * C_inv,K = max_e C_inv(e,K,p); beta_K = max over nodes of |b_ns|_2 with
 * (b_ns)_j = |v_j - v_w,j| + sqrt(gamma p / rho) (Eq. cfl_general); beta'_K = 0. */
int oracle_dt(const oracle_problem *P, const double *U, double cfl, const double vw[2],
              double *dt_out, double *lambda_K)
{
    int Np = P->Np;
    size_t nd = (size_t)P->K * 4 * Np;
    double *Ux = malloc(nd * sizeof(double)), *Uy = malloc(nd * sizeof(double));
    if (!Ux || !Uy) { free(Ux); free(Uy); return -1; }
    broken_gradient(P, U, Ux, Uy);
    double lam_max = 0;
    double d = 2.0, pp = P->p;
#pragma omp parallel for schedule(static) reduction(max : lam_max)
    for (long long k = 0; k < P->K; ++k) {
        double GK = 0, sigK = 0, ciK = 0, perim = 0;
        for (int f = 0; f < 3; ++f) {
            double Up[8][4], Upx[8][4], Upy[8][4], Uo[8][4], Uox[8][4], Uoy[8][4];
            face_traces(P, U, Ux, Uy, vw, k, f, Up, Upx, Upy, Uo, Uox, Uoy);
            double gb = face_diffusivity(P, (const double (*)[4])Up, (const double (*)[4])Uo);
            double sg = face_sigma(P, k, f, (const double (*)[4])Up, (const double (*)[4])Uo);
            double ci = cinv(P, k, f);
            if (gb > GK) GK = gb;
            if (sg > sigK) sigK = sg;
            if (ci > ciK) ciK = ci;
            perim += 2.0 * P->sJ[k * 3 + f];
        }
        double area = 2.0 * P->J[k];
        double rhoK = 2.0 * area / perim;
        double cinv2 = pp * pp * pp * pp / (rhoK * rhoK);
        double beta = 0;
        for (int i = 0; i < Np; ++i) {
            double u[4];
            load_node(U, Np, k, i, u);
            double pr = pressure(u, P->gamma);
            double c = sqrt(P->gamma * pr / u[0]);
            double b1 = fabs(u[1] / u[0] - vw[0]) + c, b2 = fabs(u[2] / u[0] - vw[1]) + c;
            double bn = sqrt(b1 * b1 + b2 * b2);
            if (bn > beta) beta = bn;
        }
        double lam = 1.5 * cinv2 * GK + (d + 1.0) * ciK * (3.0 * sigK + beta);
        if (lambda_K) lambda_K[k] = lam;
        if (lam > lam_max) lam_max = lam;
    }
    free(Ux);
    free(Uy);
    *dt_out = cfl / lam_max;
    return 0;
}

/* Force and moment of the fluid on the wall boundary: traction p n^+ - tau n^+
 * (n^+ the element's outward normal, i.e. into the body), integrated with the
 * face mass matrix; moment about xc.  out = (Fx, Fy, Mz). */
int oracle_wall_forces(const oracle_problem *P, const double *U, const double xc[2], double out[3])
{
    int Np = P->Np, Nfp = P->Nfp;
    double F0 = 0, F1 = 0, Mz = 0;
    for (long long k = 0; k < P->K; ++k)
        for (int f = 0; f < 3; ++f) {
            if (P->bc[k * 3 + f] != BC_WALL) continue;
            double n[2] = {P->nx[k * 3 + f], P->ny[k * 3 + f]};
            double tx[8], ty[8], mz[8];
            for (int i = 0; i < Nfp; ++i) {
                long long vm = P->Fmask[f * Nfp + i];
                double u[4], ux[4], uy[4], vx[4], vy[4];
                load_node(U, Np, k, vm, u);
                /* gradient at this node only */
                for (int c = 0; c < 4; ++c) {
                    double ur = 0, us = 0;
                    for (int j = 0; j < Np; ++j) {
                        ur += P->Dr[vm * Np + j] * U[(k * 4 + c) * Np + j];
                        us += P->Ds[vm * Np + j] * U[(k * 4 + c) * Np + j];
                    }
                    ux[c] = P->rx[k] * ur + P->sx[k] * us;
                    uy[c] = P->ry[k] * ur + P->sy[k] * us;
                }
                visc_flux(u, ux, uy, P->gamma, P->Pr, P->mu, vx, vy);
                double p = pressure(u, P->gamma);
                double tn1 = vx[1] * n[0] + vy[1] * n[1];
                double tn2 = vx[2] * n[0] + vy[2] * n[1];
                tx[i] = p * n[0] - tn1;
                ty[i] = p * n[1] - tn2;
                double xx = P->x[k * Np + vm] - xc[0], yy = P->y[k * Np + vm] - xc[1];
                mz[i] = xx * ty[i] - yy * tx[i];
            }
            const double *M1 = P->M1D + (size_t)f * Nfp * Nfp;
            double sJ = P->sJ[k * 3 + f];
            for (int i = 0; i < Nfp; ++i)
                for (int l = 0; l < Nfp; ++l) {
                    F0 += sJ * M1[i * Nfp + l] * tx[l];
                    F1 += sJ * M1[i * Nfp + l] * ty[l];
                    Mz += sJ * M1[i * Nfp + l] * mz[l];
                }
        }
    out[0] = F0;
    out[1] = F1;
    out[2] = Mz;
    return 0;
}

/* One Newmark step (beta = 1/4, gamma = 1/2) of M y'' + C y' + K y = F
 * (Eq. 1dof_oscillator), force taken at the new time level.
 * coeff = (M, C, K); state = (y, y', y'') in/out; vb = (y_new - y_old)/dt. */
int oracle_newmark_step(const double coeff[3], double F, double dt, double state[3], double *vb)
{
    const double beta = 0.25, gam = 0.5;
    double M = coeff[0], C = coeff[1], Kr = coeff[2];
    double y = state[0], yd = state[1], ydd = state[2];
    /* predictors */
    double yp = y + dt * yd + (0.5 - beta) * dt * dt * ydd;
    double ydp = yd + (1.0 - gam) * dt * ydd;
    double lhs = M + gam * dt * C + beta * dt * dt * Kr;
    if (lhs == 0.0) return -1;
    double ydd_new = (F - C * ydp - Kr * yp) / lhs;
    double y_new = yp + beta * dt * dt * ydd_new;
    double yd_new = ydp + gam * dt * ydd_new;
    if (vb) *vb = (y_new - y) / dt;
    state[0] = y_new;
    state[1] = yd_new;
    state[2] = ydd_new;
    return 0;
}
