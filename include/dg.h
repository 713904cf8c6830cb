/*
 * dg.h -- C ABI of the GB300 nodal interior-penalty DG solver for the 2D
 * compressible Navier-Stokes equations on triangles (arXiv 2508.17917).
 *
 * The library evaluates the semi-discrete right-hand side of the paper's
 * discretisation (Sec. 2.2, Eq. dg_on_K) fused with the five-stage 2N-storage
 * Runge-Kutta update (Sec. 2.3, Algorithm 1) in hand-written CUDA kernels
 * for sm_103a, plus the wall force integral, the CFL time step and the
 * rigid-body Newmark step of the coupled loop (Sec. 2.4, Algorithm 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - State layout (API and device): U[k][c][i], k = element, c = conserved
 *   field (rho, rho v1, rho v2, eps) with eps the total energy per volume
 *   (Sec. 2.1), i = element-local node; FP64, contiguous, K*4*Np doubles.
 * - Node numbering: the warp-and-blend nodes of degree p on the reference
 *   triangle {(-1,-1), (1,-1), (-1,1)}; node (n, m) has barycentric weight
 *   n/p on vertex (-1,1) and m/p on vertex (1,-1) before warping, numbered
 *   with n outer (row s = -1 first) and m inner (increasing r).
 *   Np = (p+1)(p+2)/2, 1 <= p <= 6.
 * - Mesh: EToV[k] lists the vertices of element k counter-clockwise; face f
 *   joins EToV[k][f] and EToV[k][(f+1)%3].  EToE/EToF give the neighbour
 *   element and its face; a boundary face names itself.  bc[k][f]: 0 interior
 *   or periodic, 1 moving adiabatic no-slip wall, 2 far field (Sec. 2.2,
 *   boundary term).  Periodic meshes repeat vertices on the wrapped edges so
 *   that each element is an ordinary affine triangle.
 * - Ownership: input arrays are copied before the call returns; the caller
 *   keeps device pointers passed with on_device = 1 alive until the work
 *   queued on the context's stream has finished.  The library owns all the
 *   device memory it allocates and frees it in dg_destroy.
 * - Streams: every device operation of a context is queued on the stream
 *   given to dg_create (a cudaStream_t, or NULL for the legacy default
 *   stream).  Calls that return host values (dg_get_state with host output,
 *   dg_compute_dt, dg_wall_forces, dg_check_finite) synchronise that stream.
 * - Errors: every call returns a dg_status; on failure the context keeps a
 *   message readable with dg_last_error.  No exception crosses the ABI.
 *   There is no CPU fallback: without a usable GB300 the device calls
 *   return DG_ECUDA.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum {
    DG_OK = 0,
    DG_EINVAL = -1,        /* bad argument: null pointer, size out of range   */
    DG_EMESH = -2,         /* mesh rejected: orientation, J <= 0, reciprocity */
    DG_ECUDA = -3,         /* CUDA runtime error (message has the details)    */
    DG_ENONFINITE = -4,    /* non-finite value found where finite is needed   */
    DG_ETIMEOUT = -5,      /* a bounded device wait gave up                   */
    DG_EUNSUPPORTED = -6   /* valid request the library does not implement    */
} dg_status;

enum { DG_PRECISION_FP64 = 0, DG_PRECISION_MIXED = 1 };
enum { DG_BC_INTERIOR = 0, DG_BC_WALL = 1, DG_BC_FARFIELD = 2 };
enum { DG_SOURCE_NONE = 0, DG_SOURCE_MANUFACTURED = 1, DG_SOURCE_VORTEX = 2 };

typedef struct {
    int p;                       /* polynomial degree, 1..6 (Sec. 2.2)                   */
    int precision;               /* DG_PRECISION_FP64 or DG_PRECISION_MIXED              */
    double gamma, Pr, mu;        /* adiabatic index, Prandtl number, viscosity (Sec. 2.1) */
    double theta;                /* IP variant (Eq. ip_flux), -1..1: 1 SIP, 0 IIP, -1 NIPG */
    double C1;                   /* penalty constant of Eq. penalty_final                */
    double rho_inf, u_inf, v_inf, p_inf;   /* far-field state (Sec. 2.2, boundary term) */
    int adiabatic_zero_heatflux; /* 1: wall energy flux keeps only v_w.(tau n)           */
} dg_params;

/* Create a context on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Builds the reference
 * operators of degree params->p (Sec. 2.2, weak matrices) and uploads them.
 * theta != 0 selects the kernel variant with the theta terms of Eq. dg_on_K
 * (weight 1/2 on interior faces, 1 on boundary faces; G at U+ on interior
 * and far-field faces, at the wall state on walls); the penalty is
 * C1 (1+theta)^2 (d+1) Gbar_e max C_inv (Eq. penalty_final), so theta = -1
 * has no penalty.
 * Errors: DG_EINVAL (null, p out of range, gamma <= 1, mu < 0, theta outside
 * [-1, 1], ...), DG_ECUDA.  *out is NULL on failure. */
dg_status dg_create(const dg_params *params, void *cuda_stream, dg_ctx **out);

/* Free the context and all its device memory.  NULL is accepted. */
dg_status dg_destroy(dg_ctx *ctx);

/* Upload a mesh (host arrays; Sec. 2.2 affine maps T_K, connectivity E^e).
 * vx, vy: Nv vertex coordinates.  EToV, EToE, EToF, bc: K*3 int32, layout as
 * above.  Computes the per-element metric (rx, ry, sx, sy, J), face normals
 * and face Jacobians, matches the face nodes of every interior face with the
 * reversed node order of its neighbour and checks that the matched nodes
 * differ by one constant translation (zero, or a period).  Allocates the
 * state buffers and sets the state to zero.
 * Errors: DG_EINVAL (null, K < 1, Nv < 3), DG_EMESH (index out of range,
 * clockwise or degenerate element, faces not reciprocal, face nodes that do
 * not match), DG_ECUDA. */
dg_status dg_set_mesh(dg_ctx *ctx, int64_t Nv, const double *vx, const double *vy,
                      int64_t K, const int32_t *EToV, const int32_t *EToE,
                      const int32_t *EToF, const int32_t *bc);

/* Tile shape of the mixed-precision stage kernel (no counterpart in the
 * paper): 1 = one volume node and one face node per thread (256 threads),
 * 2 = two volume nodes and two face nodes of one face per thread (128
 * threads; IIP only), 3 = one warp per tile of 2 elements with the Dr / Ds /
 * LIFT (and, for theta != 0, Wr / Ws) products on the tensor cores
 * (mma.sync TF32, three products of split operands, about 2^-21 relative;
 * p <= 6), 0 = time every available shape (residual-only launches on the
 * current state) at the first time step after a mesh upload and keep the
 * fastest (the default).  The FP64 path has one kernel and accepts 0 and 1.
 * The shapes round their FP32 arithmetic differently (all within the mixed
 * path's tolerance), and the tuner's choice depends on timings, so two runs
 * of the same input can differ in the last FP32 bits under variant 0: a
 * fixed variant (1, 2 or 3) is the bit-reproducible mode.
 * Errors: DG_EINVAL (variant outside 0..3), DG_EUNSUPPORTED (2 or 3 on the
 * FP64 path, 2 with theta != 0). */
dg_status dg_set_stage_variant(dg_ctx *ctx, int variant);

/* The tile shape in use: 1, 2 or 3 (the single-node kernel until tuned). */
int dg_stage_variant(const dg_ctx *ctx);

/* Over-integration of the volume term (Sec. 2.2, weak matrices: the paper
 * evaluates F(U_h) with a cubature rule to curb aliasing): on != 0 makes the
 * FP64 path integrate int_K F(U_h, grad U_h) . grad l_i with a collapsed
 * Gauss rule of total degree dg_overint_degree(p) = min(3p, 15) (at most 64
 * points) instead of through the nodal interpolant of F; the residual is
 * then R = M^-1 sum_q w_q grad l(x_q) . F_q - LIFT (Fscale H) (weak form).
 * Face fluxes stay at the LGL face nodes; the time-step bound is unchanged.
 * Errors: DG_EUNSUPPORTED (mixed precision or theta != 0), DG_ECUDA. */
dg_status dg_set_overintegration(dg_ctx *ctx, int on);

/* Degree of the over-integration rule for polynomial degree p (0 if p is
 * outside 1..6). */
int dg_overint_degree(int p);

/* Fused steps (mixed-precision IIP path; no counterpart in the paper): on != 0
 * runs each dg_lsrk_step as one cooperative launch whose blocks do all five
 * stages of Algorithm 1 with a grid-wide barrier between stages (the same
 * arithmetic as five launches; the fused kernel is compiled separately, so a
 * multiply-add may be contracted differently and results can differ in the
 * last FP32 bit of a residual).  Every barrier wait is bounded: after
 * dg_set_barrier_limit waits of about 100 ns it gives up, the launch ends
 * early, and the next dg_barrier_status, dg_get_state or dg_check_finite
 * returns DG_ETIMEOUT (the state is then not valid).
 * Errors: DG_EUNSUPPORTED (FP64 or theta != 0), DG_ECUDA. */
dg_status dg_set_fused_steps(dg_ctx *ctx, int on);

/* Waits of about 100 ns before a bounded device wait gives up: a fused
 * step's grid barrier, and the tensor-core stage kernel's waits for the bulk
 * copies of its operator table and of each warp's own element records
 * (default 2^24, about 1.7 s; 0 makes every wait give up unless its event
 * has already happened). */
dg_status dg_set_barrier_limit(dg_ctx *ctx, uint32_t waits);

/* DG_ETIMEOUT if a bounded device wait since the last check gave up -- a
 * grid barrier of a fused step, a copy wait of the tensor-core stage kernel,
 * or a wait of the tcgen05 gradient kernel of dg_broken_gradient -- (then
 * clears the flag), DG_OK otherwise.  Synchronises when such kernels ran.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_barrier_status(dg_ctx *ctx);

/* Copy the state in ([K][4][Np] FP64; host pointer if on_device == 0, device
 * pointer otherwise) and clear the Runge-Kutta register.
 * Errors: DG_EINVAL (null, no mesh yet), DG_ECUDA. */
dg_status dg_set_state(dg_ctx *ctx, const double *U, int on_device);

/* Copy the state out ([K][4][Np] FP64).  Host output synchronises the stream
 * and reports a bounded device wait that gave up since the last check
 * (DG_ETIMEOUT: the state is not valid); device output stays asynchronous
 * (after a fused step it checks the barrier flag first, which synchronises).
 * Errors: DG_EINVAL, DG_ETIMEOUT, DG_ECUDA. */
dg_status dg_get_state(dg_ctx *ctx, double *U, int on_device);

/* dU/dt = M^-1 R(t, U) of Eq. dg_on_K for the current state, with mesh
 * velocity vw (Sec. 2.1 term v_w (x) U), written to dUdt ([K][4][Np] FP64,
 * host or device).  Uses the context's precision.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_rhs(dg_ctx *ctx, double t, const double vw[2], double *dUdt, int on_device);

/* One time step of Algorithm 1 (five stages, Carpenter-Kennedy 2N-storage
 * coefficients) from t to t + dt with mesh velocity vw held fixed (Algorithm
 * 3).  Asynchronous: queued on the context's stream.
 * Errors: DG_EINVAL (no mesh, dt not finite), DG_ECUDA. */
dg_status dg_lsrk_step(dg_ctx *ctx, double t, double dt, const double vw[2]);

/* Several steps of dg_lsrk_step with a fixed dt, queued back to back. */
dg_status dg_lsrk_steps(dg_ctx *ctx, double t, double dt, const double vw[2], int nsteps);

/* dt = cfl / max_K Lambda_K with Lambda_K of Eq. rayleigh_bound (Appendix A)
 * evaluated in FP64 for the current state and mesh velocity vw.  Readings:
 * C_inv,2 = p^4 / rho_K^2 with rho_K the inradius, G_K the largest Gbar_e over
 * the faces of K, sigma_K and C_inv,K the largest over its faces, beta_K the
 * largest |b_ns|_2 over its nodes (Eq. cfl_general), beta'_K = 0.
 * Synchronises the stream.  Errors: DG_EINVAL, DG_ENONFINITE, DG_ECUDA. */
dg_status dg_compute_dt(dg_ctx *ctx, double cfl, const double vw[2], double *dt);

/* Force and moment of the fluid on all wall faces (bc == 1): traction
 * p n - tau n integrated with the face mass matrix, n the element's outward
 * normal; moment about xc.  out = (Fx, Fy, Mz) in FP64 (Sec. 2.4, Eq.
 * lift_drag).  Synchronises the stream.  Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_wall_forces(dg_ctx *ctx, const double xc[2], double out[3]);

/* One Newmark step (beta = 1/4, gamma = 1/2) of M y'' + C y' + K y = F
 * (Eq. 1dof_oscillator), host only, no context needed.  coeff = (M, C, K);
 * state = (y, y', y'') in/out; *v_b = (y_new - y_old)/dt, the mesh velocity
 * of Algorithm 3.  Errors: DG_EINVAL (null, dt <= 0, singular system). */
dg_status dg_rigid_step(const double coeff[3], double F, double dt, double state[3],
                        double *v_b);

/* *ok = 1 if every entry of the state is finite, else 0.  Synchronises.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_check_finite(dg_ctx *ctx, int *ok);

/* Add a nodal source to every residual evaluation (Sec. 3.1).  kind
 * DG_SOURCE_MANUFACTURED takes params = (kappa, C2) and adds the source of
 * the manufactured steady solution U = (w, w, w, w^2), w = sin(kappa(x+y)) + C2,
 * evaluated at the nodes.  kind DG_SOURCE_VORTEX takes params =
 * (beta, x0, y0, L, u0, v0) and adds S = -div F_v(U_v(x, t)), the viscous
 * source that makes the isentropic vortex U_v of strength beta, centred at
 * (x0, y0) at t = 0, carried at (u0, v0) on a periodic square of side L
 * (rho_inf = p_inf = 1), an exact Navier-Stokes solution (the source of the
 * advected-vortex workload; the paper's Sec. 3.1 builds its source the same
 * way from a manufactured solution); it is evaluated at the nodes at the
 * five stage times t + c_i dt of a step by one kernel launch before the
 * stages (FP64 arithmetic on the FP64 path, FP32 on the mixed path; the
 * library holds five state-sized arrays for it), and with it fused steps fall
 * back to five stage launches per step.  DG_SOURCE_NONE removes any source.
 * Errors: DG_EINVAL (no mesh, unknown kind, null params, L <= 0), DG_ECUDA. */
dg_status dg_set_source(dg_ctx *ctx, int kind, const double *params);

/* Node coordinates of the current mesh, x and y each [K][Np] FP64 host
 * arrays (affine map T_K of Sec. 2.2).  Errors: DG_EINVAL. */
dg_status dg_node_coords(const dg_ctx *ctx, double *x, double *y);

/* Reference operators of degree p built by the library (host only, no GPU
 * needed): nodes r, s [Np]; Dr, Ds [Np][Np] row-major; LIFT [Np][3*(p+1)]
 * with face-node columns in counter-clockwise order; Fmask [3][p+1] the
 * volume index of each face node, counter-clockwise along each face.  Any
 * output may be NULL.  Errors: DG_EINVAL (p out of range). */
dg_status dg_reference_operators(int p, double *r, double *s, double *Dr, double *Ds,
                                 double *LIFT, int32_t *Fmask);

/* Largest number of wall faces dg_wall_forces_noalloc accepts. */
#define DG_NOALLOC_MAX_WALL_FACES 16384

/* The wall force and moment of dg_wall_forces, computed without any device
 * allocation.  There is no counterpart of this call in the paper.
 *
 * Who needs it: code that may not call cudaMalloc/cudaFree at the point
 * where it asks for the forces -- for instance a structural solver embedded
 * in a larger application whose device memory is owned by that application's
 * own pool allocator, or a tight coupling loop that must not risk the device
 * synchronisation a cudaFree can cause.  dg_wall_forces keeps its per-face
 * partial sums in a buffer that belongs to the mesh; this call keeps them in
 * a fixed array of DG_NOALLOC_MAX_WALL_FACES * 3 + 4 doubles (about 384 KB)
 * that is part of the library image, so every GPU that loads the library
 * holds that array until the process exits.
 *
 * Behaviour: same inputs, result and synchronisation as dg_wall_forces
 * (out = (Fx, Fy, Mz), the context's stream is synchronised).  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  All calls in the
 * process share the one array, which keeps the last call's contents (every
 * call overwrites all the entries it reads, so nothing has to be cleared):
 * two calls whose work overlaps on the GPU -- different streams, or
 * different host threads -- race on it and must be serialised by the caller.
 * Errors: DG_EINVAL (null, no mesh, more than DG_NOALLOC_MAX_WALL_FACES wall
 * faces: the message says so and names dg_wall_forces as the alternative),
 * DG_EUNSUPPORTED (device index above 63), DG_ECUDA. */
dg_status dg_wall_forces_noalloc(dg_ctx *ctx, const double xc[2], double out[3]);

/* Broken gradient of the current state (Sec. 2.2: grad_h U =
 * (rx Dr + sx Ds, ry Dr + sy Ds) U on every element, the gradient the
 * residual's viscous fluxes use): gx, gy [K][4][Np] FP64, host pointers if
 * on_device == 0, device pointers (borrowed for the call) otherwise.
 * impl 0: FP64 arithmetic on the CUDA cores.  impl 1: the element products
 * batched 32 elements to a CTA as (128 x K)(K x 2 Np) products on the
 * fifth-generation tensor cores (tcgen05.mma kind::tf32, three products of
 * split operands, FP32 accumulation in tensor memory) with the FP64 state
 * tiles staged by the tensor memory accelerator; good to about 2^-21 of
 * sum |D||U| relative to the element's first node.  With device outputs the
 * call is asynchronous on the context's stream and a bounded wait of the
 * impl 1 kernel that gave up is reported by the next dg_barrier_status,
 * dg_get_state or dg_check_finite (DG_ETIMEOUT); with host outputs it
 * synchronises and reports it itself.  Errors: DG_EINVAL (null, no mesh,
 * bad impl), DG_ETIMEOUT, DG_ECUDA. */
dg_status dg_broken_gradient(dg_ctx *ctx, double *gx, double *gy, int on_device, int impl);

/* Number of the library's kernels launched by this context so far. */
int64_t dg_kernel_launches(const dg_ctx *ctx);

/* Message of the last failing call on ctx (empty string if none).  The
 * pointer stays valid until the next call on ctx. */
const char *dg_last_error(const dg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
