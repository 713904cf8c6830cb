/*
 * dg_batch.h -- C ABI for a batch of independent cylinder cases advanced
 * together: the weakly coupled fluid / rigid-body loop of Algorithm 3 run for
 * every case on the device.
 *
 * Every case has its own mesh, polynomial degree, viscosity and 1-DOF
 * oscillator (transverse motion, Eq. 1dof_oscillator); the far-field state,
 * gamma, Pr and the penalty constant are shared.  One time step of the batch
 * is, for every case i (Algorithm 3, Sec. 2.4):
 *   1. dt_i = cfl / max_K Lambda_K(U_i, v_w = (0, v_b,i))     (Eq. rayleigh_bound)
 *   2. Newmark step (beta = 1/4, gamma = 1/2) of M_r y'' + C_r y' + K_r y = F_r
 *      with F_r = (lift of the previous force evaluation) / mass_i, giving
 *      v_b,i = (y_new - y_old) / dt_i
 *   3. five-stage LSRK step (Algorithm 1) of U_i with mesh velocity (0, v_b,i)
 *   4. wall forces of U_i (drag Fx, lift Fy, moment Mz; Eq. lift_drag).
 * All of it is queued on the device with no host round trip: per step one
 * time-step kernel per degree group, a segmented reduction, the Newmark
 * kernel, five stage launches per degree group (mixed precision: FP32
 * arithmetic, FP64 state, pressure and Runge-Kutta registers), one
 * wall-force kernel per degree group and a segmented sum.  The step can be
 * captured once into a CUDA graph and replayed.
 *
 * Memory: the library owns all device memory (elements of cases with the same
 * degree are stored back to back; tiles of the stage kernel never straddle
 * two cases).  The batch runs on a stream it creates itself; every call that
 * returns data synchronises it.  Errors never throw.
 */
#ifndef DG_BATCH_H
#define DG_BATCH_H

#include <stdint.h>

#include "dg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_batch dg_batch;

/* One case of the batch.  Mesh arrays as for dg_set_mesh (copied; only read
 * during the call).  mu: viscosity of the case (Re = rho_inf |v_inf| D / mu).
 * Oscillator: M_r y'' + C_r y' + K_r y = lift / mass (Sec. 3.3: M_r = 1,
 * C_r = 4 pi f_n zeta, K_r = (1 + 1/m*)(2 pi f_n)^2, mass = m* rho pi D^2 / 4);
 * y0, ydot0: initial displacement and velocity (initial acceleration 0). */
typedef struct {
    int p;
    int64_t Nv;
    const double *vx, *vy;
    int64_t K;
    const int32_t *EToV, *EToE, *EToF, *bc;
    double mu;
    double M_r, C_r, K_r, mass;
    double y0, ydot0;
} dg_case;

/* Create a batch of ncases >= 1 cases on the current device.  common gives
 * gamma, Pr, theta (must be 0), C1, the far-field state and the wall flag;
 * its p and mu are ignored (per case); precision must be DG_PRECISION_MIXED.
 * Builds and validates every mesh (same checks as dg_set_mesh), groups cases
 * by degree and sets every state to zero.
 * Errors: DG_EINVAL (null, ncases < 1, p out of range, mu < 0, mass <= 0, ...),
 * DG_EUNSUPPORTED (theta != 0 or FP64 precision), DG_EMESH (the message,
 * from dg_batch_last_error(NULL), names the case), DG_ECUDA.  *out is NULL on
 * failure. */
dg_status dg_batch_create(const dg_params *common, int ncases, const dg_case *cases, dg_batch **out);

/* Free the batch and all its device memory.  NULL is accepted. */
dg_status dg_batch_destroy(dg_batch *b);

/* Message of the last failed call on this batch (empty after success); with
 * b == NULL, the message of this thread's last failed dg_batch_create. */
const char *dg_batch_last_error(const dg_batch *b);

/* Kernel launches queued by the batch so far (graph replays count the
 * kernels they contain). */
int64_t dg_batch_kernel_launches(const dg_batch *b);

/* Tile shape of the stage kernel per degree group (see dg_set_stage_variant):
 * 0 = time every available shape per group at the next dg_batch_run (the
 * default), 1, 2 or 3 = forced for every group (3: the tensor-core shape;
 * a forced shape is the bit-reproducible mode, as for a single context).
 * Drops captured graphs.  Errors: DG_EINVAL. */
dg_status dg_batch_set_stage_variant(dg_batch *b, int variant);

/* Fused steps for the batch (no counterpart in the paper, whose solver runs
 * one case per MPI job).  on = 1 replaces the five stage launches of each
 * degree group by one cooperative launch with grid barriers between the
 * stages (as dg_set_fused_steps); on = 2 runs the five stages of every
 * degree group in a single cooperative launch: each group takes a share of
 * the grid (sized on the first step in proportion to the tuner's time of its
 * tensor-core shape) and runs the tensor-core shape's fused body on it, with
 * grid barriers among its own blocks only, so one persistent launch per step
 * advances all cases through Algorithm 1's stages (Algorithm 3's force,
 * time-step and Newmark launches stay around it).  Every barrier wait is
 * bounded and a wait that gives up makes dg_batch_run return DG_ETIMEOUT.
 * 0 returns to five launches per group.  Drops captured graphs.
 * Errors: DG_EINVAL (on outside 0..2), DG_ECUDA. */
dg_status dg_batch_set_fused_steps(dg_batch *b, int on);

/* Fixed time steps: dt[ncases] (host, copied) replaces step 1's
 * dt_i = cfl / max_K Lambda_K by dt_i for every following dg_batch_run (the
 * cfl argument is then ignored); the bound is still evaluated every step,
 * recorded in the history and a case whose bound is not finite is still
 * frozen.  For runs over a stretch of physical time at a step the caller
 * chose (Sec. 3.2 runs at the largest stable step found by trial).
 * dt == NULL returns to the CFL bound.  Drops captured graphs when the mode
 * changes; synchronises the batch stream.
 * Errors: DG_EINVAL (a step not finite or <= 0), DG_ECUDA. */
dg_status dg_batch_set_fixed_dt(dg_batch *b, const double *dt);

/* The tile shape the group of case i uses (1, 2 or 3); 0 for a bad argument. */
int dg_batch_stage_variant(const dg_batch *b, int i);

/* The cudaStream_t the batch runs on (for events a caller records around
 * dg_batch_run); NULL for a NULL batch. */
void *dg_batch_stream(const dg_batch *b);

/* Elements K_i and degree p_i of case i.  Errors: DG_EINVAL. */
dg_status dg_batch_case_size(const dg_batch *b, int i, int64_t *K, int *p);

/* Nodal coordinates of case i, x and y [K_i][Np_i] (host).  Errors: DG_EINVAL. */
dg_status dg_batch_node_coords(const dg_batch *b, int i, double *x, double *y);

/* Copy the state of case i in or out ([K_i][4][Np_i] FP64, host pointer if
 * on_device == 0, device pointer otherwise).  set_state clears the case's
 * Runge-Kutta register and marks the forces stale (the next dg_batch_run
 * evaluates them before its first Newmark step).  Both synchronise.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_batch_set_state(dg_batch *b, int i, const double *U, int on_device);
dg_status dg_batch_get_state(dg_batch *b, int i, double *U, int on_device);

/* Advance every case by nsteps time steps of the loop above with CFL number
 * cfl > 0.  use_graph != 0 captures one step into a CUDA graph (two graphs,
 * one per parity of the state buffers; re-captured when cfl or hist change)
 * and replays it.  hist: optional device array of hist_rows x ncases x 8
 * doubles; after step n (counted from the last dg_batch_reset_history) row n
 * holds (t, dt, y, y', v_b, Fx, Fy, max Lambda_K) of every case; rows past
 * hist_rows are dropped; hist must be ready for writing on the batch's own
 * stream (synchronise the stream that allocated or cleared it first).
 * Synchronises at the end.
 * Errors: DG_EINVAL (cfl <= 0, nsteps < 0), DG_ENONFINITE (a case met a time
 * step bound that is not finite; that case is frozen, dt = 0), DG_ECUDA. */
dg_status dg_batch_run(dg_batch *b, double cfl, int nsteps, int use_graph, double *hist, int hist_rows);

/* Restart the history row counter at 0.  Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_batch_reset_history(dg_batch *b);

/* Per-case quantities after the last step, out[ncases][10]:
 * (t, dt, y, y', y'', v_b, Fx, Fy, Mz, frozen flag).  Synchronises.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_batch_rigid(dg_batch *b, double *out);

#ifdef __cplusplus
}
#endif

#endif /* DG_BATCH_H */
