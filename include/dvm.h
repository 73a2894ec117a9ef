/*
 * libdvm - GB300 (sm_103a) CUDA library for the Cartesian cut-cell
 * discrete-velocity method of Dechriste & Mieussens, "A Cartesian cut cell
 * method for rarefied flow simulations around moving obstacles"
 * (arXiv:1503.04544).
 *
 * One time step updates every (cell, discrete velocity) pair: the BGK
 * relaxation toward the local Maxwellian (Sec. 2.1, Eq. BGKDD), upwind or
 * limited fluxes across the Cartesian edges of each virtual cell and the
 * diffuse-reflection flux across its wall edge (Eq. FluxDD, Eq.
 * BoundaryDDv), the explicit update of each control volume (Eq. ExSchemeDD)
 * or the first-order semi-implicit one (Eq. ImpSchemeDD), and the wall
 * stress, force, torque and rigid rotation (Sec. 3.3.4).  2D
 * uses the reduced pair (f, g) (Sec. 2.2); 3D uses the full F (Sec. 5).
 *
 * Conventions
 *  - Every call returns a dvm_status.  Nothing aborts or throws across this
 *    boundary; dvm_last_error() gives a thread-local message.
 *  - The caller owns every pointer it passes.  Inputs are copied; the
 *    library never keeps a caller pointer.  The context owns its device
 *    buffers (allocated in dvm_create, freed in dvm_destroy).
 *  - Host arrays are plain C arrays; "on_device" pointers are CUDA device
 *    addresses valid on the context's device.
 *  - Work is enqueued on the context's stream.  Calls that return host data
 *    synchronise that stream.
 *  - Cell index: 2D k = j*nx + i; 3D k = (l*ny + j)*nx + i.
 *    Velocity index (Sec. 3.1): p = p2*nvx + p1, 3D p = (p3*nvy + p2)*nvx + p1,
 *    v = vmin + p*(vmax - vmin)/n per axis (vmax itself is not a grid point).
 *  - State layout in memory: [cell][component][p], 2 components (f, g) in 2D,
 *    1 (F) in 3D, FP32 or FP64 as chosen at creation.
 */
#ifndef DVM_H
#define DVM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DVM_OK = 0,
    DVM_ERR_ARG = 1,          /* invalid argument or size                       */
    DVM_ERR_CFL = 2,          /* time step violates the positivity condition    */
    DVM_ERR_GEOMETRY = 3,     /* saddle cell, merge walk out of bounds, ...      */
    DVM_ERR_NONPHYSICAL = 4,  /* non-positive density or temperature            */
    DVM_ERR_CUDA = 5,         /* a CUDA runtime call failed                      */
    DVM_ERR_OOM = 6,          /* device allocation failed                        */
    DVM_ERR_STATE = 7,        /* call out of order (e.g. step before a state)    */
    DVM_ERR_UNSUPPORTED = 8   /* valid but not implemented combination           */
} dvm_status;

enum { DVM_FP32 = 32, DVM_FP64 = 64 };
enum { DVM_UPWIND = 0, DVM_MUSCL = 1 };
enum { DVM_EXPLICIT = 0, DVM_IMEX = 1 };   /* time schemes, see dvm_set_time_scheme */
enum { DVM_BGK = 0, DVM_SHAKHOV = 1 };     /* collision models, see dvm_set_collision_model */
enum { DVM_EQ_DIRECT = 0, DVM_EQ_CONSERVATIVE = 1 };   /* equilibrium moments, see dvm_set_equilibrium */
enum { DVM_BC_PERIODIC = 0, DVM_BC_MAXWELLIAN = 1, DVM_BC_ZEROGRAD = 2 };
enum { DVM_SHAPE_NONE = 0, DVM_SHAPE_CIRCLE = 1, DVM_SHAPE_ELLIPSE = 2, DVM_SHAPE_SPHERE = 3,
       DVM_SHAPE_DISK_CONTAINER = 4, DVM_SHAPE_BOX_CONTAINER = 5 };
enum { DVM_GAS = 0, DVM_CUT = 1, DVM_SOLID = 2 };

/* Cartesian grid of Sec. 3.2.1: nx*ny (*nz) cells on the box. */
typedef struct {
    int dim;                  /* 2 or 3 */
    int nx, ny, nz;           /* nz ignored in 2D */
    double xmin, xmax, ymin, ymax, zmin, zmax;
} dvm_grid;

/* Discrete velocity grid of Sec. 3.1: n points per axis on [vmin, vmax). */
typedef struct {
    int nvx, nvy, nvz;
    double vxmin, vxmax, vymin, vymax, vzmin, vzmax;
} dvm_vgrid;

/* Physical and numerical parameters.  R = T0 = rho0 = 1.  The relaxation time
 * is tau = sqrt(pi)/2 * Kn * Lref / sqrt(2) / rho (Sec. 5).  The time step is
 * dt if dt > 0, else cfl / sum_d max_p |v_{p,d}| / dx_d. */
typedef struct {
    double Kn, Lref, cfl, dt;
} dvm_physics;

/* Obstacle (Sec. 3.3.4, Appendix A).  Level set: circle/sphere |x-c| - ra;
 * ellipse with semi-axes ra (along the body x axis) and rb, turned by theta,
 * first-order distance g/|grad g|.  Containers (2D; the gas is inside, the
 * cells outside are solid; not movable): disk ra - |x-c|; box with
 * half-widths ra along x and rb along y, min(x - (cx - ra), (cx + ra) - x,
 * y - (cy - rb), (cy + rb) - y).  movable = 1: free rotation about the
 * centre with moment of inertia `inertia` (Eq. motionDD_vit); the centre and
 * (vbx, vby) stay fixed.  Wall temperature Tw, or per angular sector when
 * nseg > 0: sector s spans from direction seg_dir[2s..2s+1] counter-
 * clockwise to the next one, with temperature Tw_seg[s]. */
typedef struct {
    int shape;
    double cx, cy, cz, ra, rb;
    double theta, omega;
    double vbx, vby;
    double mass, inertia;
    int movable;
    double Tw;
    int nseg;
    const double *Tw_seg;     /* host, [nseg]   */
    const double *seg_dir;    /* host, [2*nseg] */
} dvm_body;

typedef struct dvm_ctx dvm_ctx;

/* Create a solver for one problem on the current CUDA device: dim 2 (reduced
 * pair f, g; circle or ellipse, fixed or rotating) or dim 3 (full F; fixed
 * sphere), at least 4 cells and at most 64 velocities per axis.
 * precision: DVM_FP32 (state and transport in FP32; wall density, force,
 * torque, rigid-body ODE and mass diagnostic in FP64) or DVM_FP64.
 * scheme: DVM_UPWIND (Eq. FluxDD) or DVM_MUSCL (limited fluxes on full gas
 * stencils).  stream: a cudaStream_t, or NULL for a stream the context
 * creates.  All sides start periodic; no obstacle.
 * Errors: DVM_ERR_ARG (bad sizes), DVM_ERR_OOM, DVM_ERR_CUDA. */
int dvm_create(const dvm_grid *grid, const dvm_vgrid *vgrid, const dvm_physics *phys,
               int precision, int scheme, void *stream, dvm_ctx **out);

/* Release every device buffer of the context (NULL is a no-op). */
void dvm_destroy(dvm_ctx *ctx);

/* Domain boundary of one side (0..5 = x-, x+, y-, y+, z-, z+; Sec. 4 uses
 * periodic, Maxwellian and zero-gradient sides).  For DVM_BC_MAXWELLIAN,
 * `state` is a host array of (rho, ux, uy, uz, T) per boundary cell of the
 * side, ordered by the remaining cell index (2D: j for x sides, i for y
 * sides; 3D: row-major over the two remaining axes).  Opposite sides must
 * both be periodic or both not.  Errors: DVM_ERR_ARG. */
int dvm_set_bc(dvm_ctx *ctx, int side, int kind, const double *state);

/* Time scheme of dvm_step (Sec. 3.3): DVM_EXPLICIT, the first-order explicit
 * scheme (Eq. ExSchemeDD, the default; 3D Eq. eq-schema3D), or DVM_IMEX, the
 * first-order semi-implicit scheme (Eq. ImpSchemeDD): explicit transport,
 * then an implicit relaxation towards the Maxwellian of the moments at
 * t^{n+1} (the moments of the transported values), which lifts the dt < tau
 * limit of the explicit scheme at small Knudsen numbers.  The drag adjoint
 * differentiates the explicit scheme only.  Errors: DVM_ERR_ARG. */
int dvm_set_time_scheme(dvm_ctx *ctx, int scheme);

/* Collision model (Sec. 2.1-2.2): DVM_BGK (Eq. BGKDD, the default) or
 * DVM_SHAKHOV with Prandtl number Pr >= 0 (Eq. ShakhovDD): the explicit
 * scheme relaxes towards
 *   f_S = M [1 + (1 - Pr) c.q (|c|^2/T - 4) / (5 P T)],
 *   g_S = T/2 M [1 + (1 - Pr) c.q (|c|^2/T - 2) / (5 P T)],
 * c = v - u, P = rho T (R = 1), with the heat flux
 * q = sum c (|c|^2/2 f + g) dv of the control volume at t^n (Eq.
 * MacroscopicDDv); in 3D F_S = M [1 + (1 - Pr) c.q (|c|^2/T - 5) / (5 P T)]
 * with q = sum c |c|^2/2 F dv (Sec. 2.1).  Pr = 1 is the BGK model.  The
 * Shakhov model runs with a fixed, rotating (2D) or no obstacle and with
 * both time schemes (the semi-implicit one relaxes towards the Shakhov
 * equilibrium with the heat flux q_T / (1 + nu Pr) of the transported
 * values, nu = dt/tau); the conservative equilibrium and the velocity split
 * are BGK only (DVM_ERR_UNSUPPORTED here or there), and so is the drag
 * adjoint.  The 2D explicit step takes q from moments that the previous
 * step's kernels summed (raw third moments of the new state, shifted to each
 * cell's velocity), so a step right after the state is set, and every FP64
 * step, first reads F^n once for q; the 3D explicit step reads F^n once for
 * q before the step in FP32, and adds the Shakhov term after the BGK step in
 * FP64.  Errors: DVM_ERR_ARG (model or Pr), DVM_ERR_UNSUPPORTED,
 * DVM_ERR_OOM. */
int dvm_set_collision_model(dvm_ctx *ctx, int model, double Pr);

/* Moments that set the BGK equilibrium of each control volume (Sec. 3.1).
 * DVM_EQ_DIRECT (the default): the direct discrete moments rho, u, T of the
 * state (Eq. MacroscopicDDv).  DVM_EQ_CONSERVATIVE: the (rho, u, T) whose
 * discrete equilibrium on the velocity grid (f_eq = M, 2D g_eq = T/2 M) has
 * the discrete mass, momentum and energy of the state, found every step by
 * Newton's method from the direct moments (one kernel, one thread per cell;
 * FP32 or FP64 as the state), so that the collision term conserves them
 * exactly on coarse velocity grids too.  The relaxation time stays
 * tau0 / rho with the direct density.  Both time schemes (the semi-implicit
 * one takes the parameters of the transported state); BGK only: with the
 * Shakhov model, here or in dvm_set_collision_model, DVM_ERR_UNSUPPORTED,
 * and the drag adjoint refuses the conservative mode.  A Newton iteration
 * that does not converge (10 steps) or leaves rho or T non-positive makes the
 * step fail with DVM_ERR_NONPHYSICAL.  Errors: DVM_ERR_ARG (mode),
 * DVM_ERR_UNSUPPORTED, DVM_ERR_OOM. */
int dvm_set_equilibrium(dvm_ctx *ctx, int mode);

/* Place the obstacle and build the Appendix A geometry on the device (level
 * set, cell types, edge lengths, wall edges, areas, control volumes).  2D:
 * circle, ellipse, disk or box container; 3D: sphere.  Errors:
 * DVM_ERR_GEOMETRY, DVM_ERR_ARG (sizes, a movable container, a movable body
 * without inertia), DVM_ERR_UNSUPPORTED (a shape of the other dimension),
 * DVM_ERR_STATE (between the calls of a velocity-split step). */
int dvm_set_body(dvm_ctx *ctx, const dvm_body *body);

/* Maxwellian initial state from host arrays of per-cell (rho, ux, uy, uz, T);
 * a NULL array means 0 for velocities, 1 for rho and T.  Solid cells get 0.
 * Errors: DVM_ERR_STATE (no geometry yet). */
int dvm_init_maxwellian(dvm_ctx *ctx, const double *rho, const double *ux,
                        const double *uy, const double *uz, const double *T);

/* Copy a full state in or out.  bytes must equal ncell*ncomp*nv*elem.
 * on_device = 0: host pointer; 1: device pointer.  Errors: DVM_ERR_ARG. */
int dvm_set_state(dvm_ctx *ctx, const void *f, size_t bytes, int on_device);
int dvm_get_state(dvm_ctx *ctx, void *f, size_t bytes, int on_device);

/* Checkpoint and restart of the time iteration (Sec. 3.3.5; the paper runs
 * long simulations but defines no file format, this one is the library's).
 * dvm_save writes to the file `path` (created or truncated, caller-owned name)
 * a header (grid and velocity grid sizes, precision, space and time schemes,
 * velocity splits, body kind, dt, tau0, steps done), the state in the public
 * layout of dvm_get_state, the partial moment sums of the current state and
 * the rigid-body record (angle, angular velocity, the cos/sin of the angle as
 * the device computed them, last force and torque).  dvm_load reads such a
 * file into a context made with the same grid, velocity grid, precision,
 * schemes and body: the state, the sums, the body (a moving body's geometry
 * is rebuilt at the saved angle), the step count and the time scheme are
 * restored, so that stepping continues bit for bit as the saved context
 * would have.  The force history restarts empty.  Both synchronise the
 * context's stream.  Errors: DVM_ERR_STATE (dvm_save before any state),
 * DVM_ERR_ARG (file not writable or readable, not a checkpoint, or one of
 * another problem), DVM_ERR_CUDA. */
int dvm_save(dvm_ctx *ctx, const char *path);
int dvm_load(dvm_ctx *ctx, const char *path);

/* Advance nsteps steps (the 7 steps of Sec. 3.3.5; the time scheme of
 * dvm_set_time_scheme), enqueued on the context's stream in chunks of up to
 * 1024 steps without host synchronisation inside a chunk.  Before a chunk the
 * call copies the stepping state on the device (state, moment sums, rigid
 * body: one more state-sized device buffer, allocated at the first call);
 * after it, it reads the device error flags and checks the moments of the
 * chunk's last state.  On a failure it steps the chunk again one step at a
 * time from the copy and leaves the state, the body and the step count at the
 * last good step, the input of the first step that failed: no geometry
 * error, and rho > 0 and T > 0 in every gas cell of its output.
 * Errors: DVM_ERR_NONPHYSICAL, DVM_ERR_GEOMETRY, DVM_ERR_OOM (no memory for
 * the copy), DVM_ERR_CUDA. */
int dvm_step(dvm_ctx *ctx, int nsteps);

/* dvm_step with (enable != 0, the default) or without the copy and the
 * rollback above; without it a failing call leaves the state after its last
 * step.  Errors: DVM_ERR_ARG for a null ctx. */
int dvm_rollback(dvm_ctx *ctx, int enable);

/* Same as dvm_step but without the final synchronisation and flag check
 * (for timing and graph capture); dvm_check() reads the flags later.
 * From 8 steps on, with per-launch timing (dvm_timing) off, the steps after
 * the first of the call (and the first after a state change) go to the
 * device as replays of a CUDA graph of two steps captured on the context's
 * stream: the same kernels in the same order, so the state is bitwise that
 * of launch-by-launch stepping.  If the stream cannot be captured (the legacy
 * default stream, or a capture already in progress) the call steps launch by
 * launch.  The graphs are released at the next dvm_check / dvm_step; a call
 * that finds 64 of them unreleased waits for the stream once to release them. */
int dvm_step_async(dvm_ctx *ctx, int nsteps);
int dvm_check(dvm_ctx *ctx);

/* Switch the two-step graph replays of dvm_step / dvm_step_async on
 * (enable != 0, the default) or off.  Errors: DVM_ERR_ARG for a null ctx. */
int dvm_graphs(dvm_ctx *ctx, int enable);

/* Per-cell moments of the current state (Eq. MacroscopicDDv): density,
 * velocity and temperature into arrays of ncell entries (any pointer may be
 * NULL; uz is 0 in 2D).  on_device = 0: host arrays; 1: device arrays on the
 * context's device (written on the context's stream, which the call
 * synchronises).  The velocity sums are compensated in the state precision
 * and the moments formed from them in FP64.  Solid cells give 0.
 * Errors: DVM_ERR_STATE on a velocity-split context (its moments need the
 * sums over every rank), DVM_ERR_CUDA. */
int dvm_moments(dvm_ctx *ctx, double *rho, double *ux, double *uy, double *uz, double *T, int on_device);

/* Velocity split (Sec. 5.2, "velocity parallelization"): each rank holds
 * every cell for a slab of the velocity grid, transports and relaxes its own
 * velocities, and the ranks exchange one sum per step (two with the
 * semi-implicit scheme).  2D and 3D, explicit or semi-implicit scheme, BGK
 * (direct or conservative equilibrium), fixed or (2D) rotating obstacle.
 *
 * dvm_set_velocity_split declares that this context's velocity grid (given
 * to dvm_create) is the rows [k0, k0 + n) of the last axis (v_y in 2D, v_z in
 * 3D) of the whole grid `global` (the other axes and the step equal; k0 an
 * integer).  Call it right after dvm_create, before dvm_set_body and any
 * state.  Unless dvm_physics gave dt, the time step becomes the CFL step of
 * the whole grid, so every rank steps with the same dt.  The context then
 * steps only through the two calls below; dvm_step and dvm_moments return
 * DVM_ERR_STATE, and dvm_mass gives the mass of this rank's velocities (sum
 * it over the ranks).
 *
 * One step:
 *   dvm_split_begin(ctx, xbuf)   enqueues the fusion of merged control
 *       volumes and writes this rank's contributions to xbuf, a device buffer
 *       of dvm_split_size FP64 elements (in both state precisions):
 *       the moment sums of every cell, [D + 2][ncell] (2D: sum f, vx f,
 *       vy f, |v|^2/2 f + g; 3D: sum F, vx F, vy F, vz F, |v|^2/2 F, over
 *       this rank's velocities, Eq. MacroscopicDDv), then the wall sums of
 *       every wall cell (2D [wall slot][8], 3D [wall slot][14]: outgoing
 *       c f, incoming c M[1, u_w, T_w] and the stress products, Eqs.
 *       BoundaryDDv, StressTensorDD);
 *   the caller sums xbuf element-wise over the ranks, in place, on the
 *       context's stream (an all-reduce: the only exchange of the step);
 *   dvm_split_finish(ctx, xbuf)  finishes the step from the summed xbuf:
 *       wall density, force, torque and rotation (identical on every rank),
 *       fluxes, relaxation and the control volumes of this rank's velocities.
 * With the semi-implicit scheme (Eq. ImpSchemeDD) the relaxation needs the
 * moments of the transported values over every velocity, so the step has a
 * second exchange:
 *   dvm_split_finish(ctx, xbuf)  transports (fluxes and control volumes, no
 *       relaxation) and writes this rank's moment sums of the transported
 *       values to xbuf ([D + 2][ncell], as in dvm_split_begin);
 *   the caller sums xbuf over the ranks again;
 *   dvm_split_relax(ctx, xbuf)  relaxes this rank's velocities towards the
 *       equilibrium of the summed moments (conservative parameters included)
 *       and ends the step.
 * The calls are asynchronous; dvm_check reads the error flags.  The ranks
 * must hold the same problem (grid, body, boundaries, time scheme) and step
 * in lockstep.  Between the calls of one step, dvm_set_state,
 * dvm_init_maxwellian, dvm_load, dvm_set_body, dvm_set_time_scheme and
 * dvm_set_equilibrium return DVM_ERR_STATE.  Errors: DVM_ERR_ARG (not a slab,
 * null buffer), DVM_ERR_STATE (order), DVM_ERR_UNSUPPORTED (Shakhov),
 * DVM_ERR_CUDA. */
int dvm_set_velocity_split(dvm_ctx *ctx, const dvm_vgrid *global);
int dvm_split_size(dvm_ctx *ctx, size_t *count);
int dvm_split_begin(dvm_ctx *ctx, void *xbuf);
int dvm_split_finish(dvm_ctx *ctx, void *xbuf);
int dvm_split_relax(dvm_ctx *ctx, void *xbuf);

/* Force (F[0..2]) and torque about the z axis exerted by the gas on the body
 * at the start of the last step (Eqs. eq-force, eq-torque), FP64. */
int dvm_wall_force(dvm_ctx *ctx, double *F, double *torque);

/* Per-step history of the last min(n, steps taken) steps, oldest first:
 * Fx, Fy, Fz, torque at t^n and theta, omega after the step (any pointer may
 * be NULL).  Returns the number of entries written through *count. */
int dvm_history(dvm_ctx *ctx, double *Fx, double *Fy, double *Fz, double *torque,
                double *theta, double *omega, int n, int *count);

/* Body angle and angular velocity after the last step. */
int dvm_body_state(dvm_ctx *ctx, double *theta, double *omega);

/* Total mass sum_cells sbar * sum_p f dv (Eq. def-masse), FP64. */
int dvm_mass(dvm_ctx *ctx, double *mass);

/* Time step, relaxation scale tau0 (tau = tau0/rho), and sizes. */
int dvm_info(dvm_ctx *ctx, double *dt, double *tau0, long long *ncell, int *nv,
             int *ncomp, int *elem_bytes);

/* 2D geometry of the current time level, copied to host arrays (any may be
 * NULL): type/cgas [ncell], lx [(nx+1)*ny], ly [nx*(ny+1)], lw, nwx, nwy,
 * rwx, rwy, sbar [ncell], master [ncell] (-1 for cells in no control
 * volume).  Layouts as in Appendix A: vertical edge a of row j at
 * j*(nx+1)+a, horizontal edge b of column i at b*nx+i. */
int dvm_geometry2d(dvm_ctx *ctx, int8_t *type, int8_t *cgas, double *lx, double *ly,
                   double *lw, double *nwx, double *nwy, double *rwx, double *rwy,
                   double *sbar, int32_t *master);

/* 3D geometry (Sec. 5; faces from the Appendix A construction, the wall face
 * closing the polyhedron), copied to host arrays (any may be NULL):
 * type/cgas [ncell]; face areas ax [(nx+1)*ny*nz] (face a of row (j, k) at
 * (k*ny + j)*(nx+1) + a), ay [nx*(ny+1)*nz] (face b of (i, k) at
 * (k*(ny+1) + b)*nx + i), az [nx*ny*(nz+1)] (face c of (i, j) at
 * (c*ny + j)*nx + i); wall area sw, unit normal (nwx, nwy, nwz) pointing into
 * the solid, wall centre (rwx, rwy, rwz), virtual-cell volume vol and master
 * [ncell].  Errors: DVM_ERR_ARG on a 2D context. */
int dvm_geometry3d(dvm_ctx *ctx, int8_t *type, int8_t *cgas, double *ax, double *ay, double *az,
                   double *sw, double *nwx, double *nwy, double *nwz, double *rwx, double *rwy,
                   double *rwz, double *vol, int32_t *master);

/* Rebuild the 2D geometry for an explicit (cos theta, sin theta) pair, for
 * bit-exact comparisons with an independent implementation. */
int dvm_geometry2d_at(dvm_ctx *ctx, double cos_t, double sin_t);

/* Drag gradient by the discrete adjoint (the paper has no adjoint: the step of
 * Sec. 3.3.5 is differentiated as it stands; 2D, fixed obstacle).  Runs
 * nsteps forward steps from the current state, checkpointing it every
 * checkpoint_every steps on the device, and returns
 *   J       F_x of the state after nsteps steps (Eqs. StressTensorDD, eq-force)
 *   gTw     dJ/dT_w per wall sector [nseg], or [1] for a uniform wall
 *   gbc_s   dJ/d(rho, ux, uy, uz, T) of every cell of Maxwellian side s
 *           [5 * side cells] (nullable; zeros for other sides)
 *   gprim0  dJ/d(rho, ux, uy, uz, T) of each cell of the initial Maxwellian
 *           [5 * ncell] (nullable; needs a state set by dvm_init_maxwellian)
 *   ms_forward, ms_reverse  device time of the checkpointed forward run and of
 *           the reverse sweep (recomputation included), nullable.
 * The reverse sweep recomputes each segment from its checkpoint onto a device
 * tape of checkpoint_every states and applies the transposed step (limiter
 * derivative of the branch the forward takes).  The context is left at the
 * state after nsteps steps.  Device memory: ceil(nsteps/K) + K + 3 states.
 * Errors: DVM_ERR_UNSUPPORTED (3D, no or moving obstacle), DVM_ERR_ARG,
 * DVM_ERR_STATE, DVM_ERR_OOM, DVM_ERR_NONPHYSICAL. */
int dvm_drag_adjoint(dvm_ctx *ctx, int nsteps, int checkpoint_every, double *J, double *gTw,
                     double *gbc0, double *gbc1, double *gbc2, double *gbc3, double *gprim0,
                     double *ms_forward, double *ms_reverse);

/* Device memory the adjoint calls may use to keep the forward run's tape
 * (default 0).  The reverse sweep needs, for every step, the state it
 * linearises around and the limiter branches that step took; by default it
 * recomputes each checkpoint segment from its checkpoint.  With a budget,
 * the forward run writes whole segments (the last ones of the run, as many
 * as fit: (checkpoint_every - 1) states, partial sums and branch words each)
 * straight into device buffers and records every step's branches, and the
 * reverse sweep reads them without recomputing.  The budget is capped by the
 * free device memory less 4 GiB; buffers that cannot be allocated keep
 * fewer segments.  Results are those of the recomputing sweep (a step that
 * records its branches computes the same values as a plain step).  The
 * buffers stay allocated for later calls; a smaller budget frees what it no
 * longer allows at once, and dvm_destroy frees the rest.  Errors:
 * DVM_ERR_ARG (null context). */
int dvm_set_adjoint_tape(dvm_ctx *ctx, size_t max_bytes);

/* Discrete adjoint of nsteps steps for a general objective (the paper has
 * no adjoint; the step of Sec. 3.3.5 is differentiated as it stands, with
 * the same restrictions as dvm_drag_adjoint: 2D, fixed obstacle, explicit
 * scheme, BGK with the direct moments):
 *   J = [with_drag] F_x(F^N) + <seed, F^N>,
 * F^N the state after nsteps steps as dvm_get_state returns it.
 *   seed     dJ/dF^N of the linear part, public layout [cell][comp][p] in
 *            the state precision, host or device (seed_on_device); nullable
 *            if with_drag
 *   lambda0  receives dJ/dF^0, public layout and state precision, host or
 *            device (lambda0_on_device); nullable
 *   J        receives F_x(F^N) when with_drag, else 0
 *   gTw, gbc0..3, gprim0  as in dvm_drag_adjoint, for this J
 * The context is left at F^N.  Errors as dvm_drag_adjoint, and DVM_ERR_ARG
 * for no objective. */
int dvm_adjoint(dvm_ctx *ctx, int nsteps, int checkpoint_every, int with_drag, const void *seed,
                int seed_on_device, void *lambda0, int lambda0_on_device, double *J, double *gTw,
                double *gbc0, double *gbc1, double *gbc2, double *gbc3, double *gprim0);

/* One transposed step (vector-Jacobian product of the step of Sec. 3.3.5):
 * lambda_n = (dF^{n+1}/dF^n)^T lambda_np1 around the current state F^n, and
 * gTw[nseg] (or [1]) = <lambda_np1, dF^{n+1}/dT_w>.  Both buffers in the
 * public layout and state precision, host (on_device = 0) or device (1).
 * The context advances one step, to F^{n+1}.  dvm_adjoint with nsteps = 1,
 * no drag and the seed lambda_np1. */
int dvm_step_vjp(dvm_ctx *ctx, const void *lambda_np1, void *lambda_n, int on_device, double *gTw);

/* Live timing of one kernel: enable = 1 the fused bulk stream-and-relax
 * kernel, 2 the Shakhov model's own kernel (dvm_set_collision_model: the
 * heat-flux pass where it runs, the FP64 3D Shakhov term), 0 off.  Every step
 * records a CUDA event pair around that kernel's launch on the context's
 * stream.  dvm_kernel_time synchronises the stream, returns the summed
 * duration in milliseconds and the number of timed launches, and clears the
 * record. */
int dvm_timing(dvm_ctx *ctx, int enable);
int dvm_kernel_time(dvm_ctx *ctx, double *bulk_ms, long long *launches);

/* FP64 fused multiply-add throughput of the current device in GFLOP/s
 * (instrumentation; the paper has no counterpart): the ceiling of the FP64
 * step, which on this part is bound by the FP64 pipe rather than by HBM.  A
 * kernel of 16 independent FMA chains per thread on 4 blocks of 256 threads
 * per SM, timed with CUDA events on `stream` (a cudaStream_t or NULL), best
 * of three launches after one untimed; 2 flop per FMA.  Allocates and frees
 * a small output buffer.  Errors: DVM_ERR_ARG, DVM_ERR_CUDA. */
int dvm_fp64_peak(void *stream, double *gflops);

/* Number of kernels this context has launched since creation. */
int dvm_launches(dvm_ctx *ctx, long long *count);

/* Cells by role at the current time level: non-solid cells, cells updated by
 * the bulk kernel, control volumes handled by the cut-cell kernel, wall
 * cells. */
int dvm_cell_counts(dvm_ctx *ctx, long long *nonsolid, long long *bulk, long long *cvs,
                    long long *walls);

/* Total mass of a state, allocating no device memory.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc,
 * such as a hook inside a framework whose allocator owns all device memory
 * and forbids allocation while the hook runs, or a loop with a fixed memory
 * budget that must not grow once it runs.
 *   f      device pointer, state in the public layout [cell][comp][p],
 *          FP32 or FP64 as `precision` says; only component 0 is summed
 *   sbar   device pointer, ncell cell areas (2D) or volumes (3D)
 *   dv     velocity cell measure (product of the grid steps)
 *   mass   device pointer, receives sum_cells sbar * sum_p f dv (FP64)
 *   stream cudaStream_t or NULL (legacy default stream); asynchronous
 * The scratch (one FP64 value per cell) is a static device array of 2^20
 * cells (8 MiB) held by every GPU that loads the library until exit; larger
 * states are rejected with DVM_ERR_ARG.  The first call on a device (and the
 * first in a new context of it, e.g. after cudaDeviceReset) looks up the
 * array's address with that device current: make that call before any
 * stream capture.  Every entry the call reads from the array it writes
 * first, so no clearing is needed.  All calls share the array, so calls
 * whose work overlaps on the GPU (different streams, no ordering) race;
 * order them.
 * Errors: DVM_ERR_ARG, DVM_ERR_CUDA. */
int dvm_mass_noalloc(const void *f, int precision, long long ncell, int ncomp, int nv,
                     const double *sbar, double dv, double *mass, void *stream);

/* Thread-local description of the last error. */
const char *dvm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
