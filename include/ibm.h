/*
 * ibm.h - C ABI of the GB300 discrete-forcing immersed boundary library.
 *
 * The library advances the compressible Navier-Stokes equations with heat
 * exchange (Riahi, Goncalves da Silva, Meldi, arXiv 2301.09349, Sec. 2.1) on
 * a uniform Cartesian grid, with an immersed body represented by Lagrangian
 * markers (Sec. 2.2).  One time step is:
 *   1. an SSP-RK2 finite-volume predictor without sources (App. B, step 1):
 *      MUSCL/van Leer reconstruction of (rho, u, p), Rusanov convective flux,
 *      central viscous stress and heat flux (Sec. 2.2.2 schemes);
 *   2. interpolation of rho, rho u and rho e to the markers with the
 *      regularised 3-point delta (Eq. interp) and the direct-forcing terms
 *      F = a_s((rho_L U)^d - I[rho u]) (Eq. forceMomentum) and
 *      Q = a_e c_v((rho_L Theta)^d - (rho_L Theta)^l) (Eq. corr3.8), a = 1/dt;
 *   3. spreading of F and Q to the grid (Eq. force2, weights eps from the
 *      quadrature system A eps = 1 of Sec. 2.2) and the forced update of
 *      momentum and internal energy (App. B, Eqs. u_centralF2, e_centralF2),
 *      the f.u work being dropped (Sec. 2.2.1).
 *
 * Conventions
 *  - Every call returns an ibm_status (IBM_OK = 0).  No C++ exception and no
 *    process exit crosses this boundary.  ibm_last_error() gives a message.
 *  - Memory ownership: the caller owns all device memory.  The library carves
 *    its device buffers out of one caller-provided workspace (size from
 *    ibm_workspace_bytes) and never allocates device memory itself.  The
 *    handle owns only host metadata.  Host arrays passed in are copied before
 *    the call returns.
 *  - Streams: every device operation is ordered on the stream given at
 *    creation (a cudaStream_t passed as void*; NULL = legacy default stream).
 *    ibm_step does not synchronize; asynchronous errors (non-finite state,
 *    quadrature not converged, a moving marker leaving the admissible region)
 *    are recorded on the device and reported by the next synchronizing call:
 *    ibm_sync, ibm_get_state, ibm_forces_and_nusselt and the ibm_get_* calls.
 *  - State layout: component-major, (dim+2) planes of nx*ny*nz cells, cell
 *    (i,j,k) at i + nx*(j + ny*k); components (rho, rho u, rho v, [rho w],
 *    rho E) in units rho_inf = U_inf = T_inf = D = 1 (gas constant
 *    r = 1/(gamma Ma^2)).  Element type float (fp_bytes 4) or double (8).
 *  - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef IBM_GB300_H
#define IBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ibm_status;

#define IBM_OK 0
#define IBM_ERR_ARG 1         /* invalid argument (null pointer, bad size, marker too close to an edge) */
#define IBM_ERR_CUDA 2        /* a CUDA runtime call or kernel launch failed */
#define IBM_ERR_NONFINITE 3   /* the state became non-finite or non-positive */
#define IBM_ERR_NOCONV 4      /* the quadrature solve did not reach its tolerance */
#define IBM_ERR_WORKSPACE 5   /* workspace too small, or marker capacity exceeded */
#define IBM_ERR_TIMEOUT 6     /* a bounded device wait gave up */
#define IBM_ERR_STATE 7       /* call out of order (e.g. step before set_state) */
#define IBM_ERR_UNSUPPORTED 8 /* declared but not provided by this build */
#define IBM_ERR_BOUNDS 9      /* (bounds-checked build only) a kernel met an index outside
                                 its array; the access was skipped */

/* boundary conditions per domain face */
#define IBM_BC_FREESTREAM 0   /* Dirichlet: ghost cells hold the free stream (inlet, Sec. 3.1) */
#define IBM_BC_ZEROGRAD 1     /* ghost cells copy the adjacent cell (outlet / supersonic side) */
#define IBM_BC_SLIP 2         /* mirror with the normal momentum negated (subsonic side, Sec. 3.1) */
#define IBM_BC_PERIODIC 3

typedef struct ibm_grid ibm_grid; /* opaque handle */

typedef struct {
    int dim;               /* 2 or 3 */
    int n[3];              /* cells per axis, each >= 4 (n[2] = 1 when dim == 2) */
    double lo[3];          /* lower domain corner */
    double h;              /* uniform spacing (Delta x = Delta y = Delta z) */
    int fp_bytes;          /* 4: float fields; 8: double fields */
    double gamma, Pr, Re, Mach;  /* Re <= 0: inviscid */
    double sutherland_S;   /* Sutherland constant / T_inf */
    double cfl;            /* CFL number for the adaptive step */
    int bc[6];             /* IBM_BC_* for x-, x+, y-, y+, z-, z+ */
    int tile[3];           /* marker-binning tile in cells per axis (tile[2] = 1 in 2D) */
    double D;              /* reference length for Cd, Cl, Nu */
    int energy_reading;    /* 0: heat source on internal energy (Eq. e_centralF2); 1: on total energy */
    int forcing_per_stage; /* 0: forcing once after the SSP-RK2 predictor (App. B, default);
                              1: after each stage; the step's reported sources are then
                              G1/2 + G2, the first stage's reaching U^{n+1} with weight 1/2 */
} ibm_grid_desc;

/* Prescribed rigid motion of all markers (Sec. 5):
 * X(t) = X(0) + amp sin(2 pi freq t) e_axis, body velocity dX/dt. */
typedef struct {
    double amp;
    double freq;
    int axis;
} ibm_motion;

/* Bytes of device workspace needed for a grid and a marker capacity.
 * Returns 0 when the description is invalid.  Host-only, no CUDA call. */
size_t ibm_workspace_bytes(const ibm_grid_desc *desc, int max_markers);

/* Create a handle over a caller-owned device workspace of `bytes` bytes
 * (256-byte aligned, at least ibm_workspace_bytes).  `stream` is a
 * cudaStream_t.  Errors: IBM_ERR_ARG (bad description / pointers),
 * IBM_ERR_WORKSPACE (too small), IBM_ERR_CUDA. */
ibm_status ibm_create_grid(const ibm_grid_desc *desc, int max_markers, void *dev_workspace,
                           size_t bytes, void *stream, ibm_grid **out);

/* Release the handle (host metadata only; the workspace stays the caller's). */
ibm_status ibm_destroy(ibm_grid *g);

/* Copy a conserved state from device memory `U` ((dim+2)*N elements of the
 * grid's type) into the handle's state; resets the simulated time to 0. */
ibm_status ibm_set_state(ibm_grid *g, const void *U);

/* Copy the current state to device memory `U`; synchronizes the stream and
 * reports any recorded asynchronous error. */
ibm_status ibm_get_state(ibm_grid *g, void *U);

/* Host-memory variants of set/get (the copy runs on the handle's stream;
 * page-locked buffers give asynchronous transfers). */
ibm_status ibm_set_state_host(ibm_grid *g, const void *U_host);
ibm_status ibm_get_state_host(ibm_grid *g, void *U_host);

/* Define the immersed body by n markers (Sec. 2.2).  X0: n*dim host doubles
 * (marker k at X0[k*dim ..]); Ub: n*dim body velocities or NULL (= 0);
 * Tw: n wall temperatures / T_inf; motion: NULL for a body at rest.
 * dedup != 0 keeps, per mesh cell, only the marker closest to the cell
 * centre (Sec. 3.1; ties keep the lowest index); kept markers retain their
 * input order.  Every marker's owner cell floor((X - lo)/h) must be at least
 * two cells from each domain edge (IBM_ERR_ARG otherwise).  Builds the
 * marker-to-cell bins and solves A eps = 1 (blocking).  n = 0 removes the
 * body.  *n_kept (may be NULL) receives the number of kept markers. */
ibm_status ibm_set_markers(ibm_grid *g, int n, const double *X0, const double *Ub,
                           const double *Tw, const ibm_motion *motion, int dedup, int *n_kept);

/* Replace the wall temperatures of the kept markers (n_kept host doubles,
 * in kept order).  The copy is queued on the handle's stream and takes
 * effect from the next step; with a page-locked buffer it is asynchronous,
 * so the caller keeps the buffer unchanged until the next synchronizing
 * call (pageable memory is copied before the call returns). */
ibm_status ibm_set_wall_temperature(ibm_grid *g, const double *Tw);

/* Stopping rule of the quadrature solve A~ eps~ = 1 (Sec. 2.2): the
 * iterative solver (more than 160 markers) stops when
 * max_k |1 - (A~ eps~)_k| <= tol, after at most maxit iterations
 * (IBM_ERR_NOCONV otherwise); the direct solver (up to 160 markers) refines
 * to its rounding floor and checks the same bound.  Defaults 1e-12 and 4000.
 * Takes effect from the next ibm_set_markers (and every step of a moving
 * body).  Errors: IBM_ERR_ARG (tol outside (0, 1) or maxit < 1). */
ibm_status ibm_set_quadrature(ibm_grid *g, double tol, int maxit);

/* Advance nsteps IBM steps.  dt_fixed > 0 imposes the step size; otherwise
 * dt = cfl / max_j s_j is computed on the device from the state at the start
 * of each step (formed at the end of the previous step, or when the state is
 * set).  Asynchronous; no host synchronization. */
ibm_status ibm_step(ibm_grid *g, int nsteps, double dt_fixed);

/* steps_per_graph > 0 (even): ibm_step replays whole chunks of that many
 * steps from CUDA graphs captured on first use (one per starting buffer and
 * dt_fixed; recaptured after ibm_set_markers), the remainder launched
 * directly.  Cuts the per-launch host cost of small grids.  Graphs are not
 * used while profiling or recording.  0 (default) = direct launches. */
ibm_status ibm_step_graphs(ibm_grid *g, int steps_per_graph);

/* Force on the body and heat rate into the fluid from the last step's
 * marker forcing (Sec. 3.1, Eq. Bulk): force = -h^d sum_k eps~_k F_k,
 * heat = h^d sum_k eps~_k Q_k; Cd = 2 force_x / (rho U^2 Lref),
 * Cl = 2 force_y / (rho U^2 Lref), Lref = D (2D) or pi D^2/4 (3D);
 * Nu = heat D / (lambda_inf A_s (mean T_w - 1)), A_s = pi D (2D) or pi D^2
 * (3D) (NaN when mean T_w = 1 or inviscid).  Any output may be NULL.
 * Synchronizes the stream. */
ibm_status ibm_forces_and_nusselt(ibm_grid *g, double force[3], double *heat_rate, double *Cd,
                                  double *Cl, double *Nu);

/* ---- discrete adjoint ----------------------------------------------------
 * Gradient of J = dJ_dCd * Cd + dJ_dNu * Nu, with Cd and Nu those of the
 * LAST recorded step (as ibm_forces_and_nusselt reports them), with respect
 * to the kept markers' positions and wall temperatures: the exact derivative
 * of the discrete map that the recorded ibm_step calls computed (Sec. 2.1-2.2,
 * App. B), under these conventions: the step sizes of the recorded run are
 * held fixed; bins, kept markers and the band do not move; the limiter and
 * the max/abs of the Rusanov flux take the branch of the forward run; the
 * weights eps~ = A~^{-1} 1 are differentiated exactly (one extra solve with A~).
 * Static markers only.  The forward states are recomputed from checkpoints
 * taken every `every` steps. */

/* Bytes of the adjoint workspace for max_steps recorded steps with a
 * checkpoint every `every` steps: ceil(max_steps/every) + 3 every + 6
 * states (a replayed segment keeps each step's state, U1 and U*),
 * (dim+2) x N doubles and a few doubles per marker and segment step (0 if
 * invalid). */
size_t ibm_adjoint_workspace_bytes(const ibm_grid_desc *desc, int max_markers, int max_steps,
                                   int every);

/* Start recording into a 256-byte aligned device workspace of at least
 * ibm_adjoint_workspace_bytes bytes (caller-owned): every following ibm_step
 * stores its step size and, every `every` steps, its starting state.  A new
 * state or new markers restart the recording.  More than max_steps steps
 * give IBM_ERR_WORKSPACE (before any work); moving markers
 * IBM_ERR_UNSUPPORTED. */
ibm_status ibm_record(ibm_grid *g, int max_steps, int every, void *dev_workspace, size_t bytes);

/* The reverse sweep over all recorded steps.  dJ_dX: n_kept*dim doubles,
 * dJ_dTw: n_kept doubles (host, kept-marker order; either may be NULL).
 * The handle's state, time and last marker forcing are left unchanged.
 * Synchronizes.  Errors: IBM_ERR_STATE (nothing recorded), IBM_ERR_ARG (Nu
 * weighted but undefined), IBM_ERR_NOCONV (the weights' adjoint solve). */
ibm_status ibm_backward(ibm_grid *g, double dJ_dCd, double dJ_dNu, double *dJ_dX, double *dJ_dTw);

/* out = J_L(U)^T V: the transpose of the Jacobian of the flux operator
 * L(U) of ibm_rhs applied to V (all (dim+2) x N device arrays of the grid's
 * type).  Needs ibm_record's workspace (FP64 scratch).  Asynchronous. */
ibm_status ibm_rhs_vjp(ibm_grid *g, const void *U, const void *V, void *out);

/* Surface pressure coefficient at every kept marker from the current state:
 * C_p,k = (I[p]_k - p_inf) / (rho_inf U_inf^2 / 2), with p = (gamma - 1)
 * (rho E - |rho u|^2/(2 rho)) interpolated by the weights of Eq. interp
 * (the paper plots C_p around the body, Sec. 3).  cp: n_kept host doubles.
 * Synchronizes. */
ibm_status ibm_surface_pressure(ibm_grid *g, double *cp);

/* Wait for the handle's stream and report any recorded device error. */
ibm_status ibm_sync(ibm_grid *g);

/* Message of the last error on this handle ("" if none); g may be NULL for
 * errors of ibm_create_grid. */
const char *ibm_last_error(const ibm_grid *g);

/* ---- inspection (synchronizing; host outputs, any may be NULL) ---------- */

/* Kept markers: positions at the current time (n_kept*dim), quadrature
 * weights eps~ (n_kept; eps = h^d eps~), and their input indices. */
ibm_status ibm_get_markers(ibm_grid *g, double *X, double *eps_t, int *input_index);

/* Last step's forcing per kept marker: rho_L (n_kept), F (n_kept*dim) and
 * Q (n_kept), with F = a_s((rho_L U)^d - I[rho u]), Q = a_e(rho_L c_v T_w -
 * I[rho e]), a_s = a_e = 1/dt. */
ibm_status ibm_get_marker_forcing(ibm_grid *g, double *rhoL, double *F, double *Q);

/* Marker-to-cell bins: tile_off (n_tiles+1), perm (n_kept) and the sorted
 * keys (n_kept), key = tile_id * cells_per_tile + cell_in_tile, tile ids and
 * cells within a tile x-fastest.  *n_tiles receives the tile count. */
ibm_status ibm_get_bins(ibm_grid *g, int *tile_off, int *perm, unsigned *keys, int *n_tiles);

/* Size of the last step taken (0 before any step), simulated time and
 * steps taken. */
ibm_status ibm_get_time(ibm_grid *g, double *dt, double *t, long long *steps);

/* ---- operators on caller device buffers (stream-ordered) --------------- */

/* L(U) of the unforced finite-volume scheme: the rate of change of the
 * conserved state, both (dim+2)*N of the grid's type in device memory. */
ibm_status ibm_rhs(ibm_grid *g, const void *U, void *L);

/* Interpolation I (Eq. interp) of nc device fields (nc*N, grid type) to the
 * kept markers: out is n_kept*nc doubles in device memory, marker-major. */
ibm_status ibm_interpolate(ibm_grid *g, const void *field, int nc, double *out);

/* Spreading S (Eq. force2): r_j = sum_k R_k Phi_k(j) eps~_k for nc marker
 * quantities R (n_kept*nc device doubles, marker-major) into out (nc*N of
 * the grid's type, device); cells outside every support are set to 0. */
ibm_status ibm_spread(ibm_grid *g, const double *R, int nc, void *out);

/* ---- kernel timing (CUDA events on the handle's stream) ------------------ */

#define IBM_PROF_STAGE1 0   /* fluid stage 1: L(U^n) and the step size */
#define IBM_PROF_STAGE2 1   /* fluid stage 2: the SSP-RK2 predictor U* */
#define IBM_PROF_MARKERS 2  /* moving markers: motion, bins, quadrature */
#define IBM_PROF_INTERP 3   /* interpolation and direct forcing */
#define IBM_PROF_SPREAD 4   /* spreading and the forced update */
#define IBM_PROF_FINISH 5   /* force/heat sums and the time update */
#define IBM_PROF_GROUPS 6

/* enable != 0 starts recording an event pair around each kernel group of
 * every subsequent ibm_step (and resets the totals); 0 stops recording. */
ibm_status ibm_profile(ibm_grid *g, int enable);

/* Synchronize, then return per group the summed device milliseconds and the
 * number of kernel launches since the last ibm_profile(g, 1) or read; both
 * arrays hold IBM_PROF_GROUPS entries (either may be NULL).  Resets. */
ibm_status ibm_profile_read(ibm_grid *g, double *ms, long long *launches);

/* ---- allocation-free stage 1 ------------------------------------------- */

/* Largest step-size reduction (thread blocks of 2048 cells) that
 * ibm_rhs_dt_noalloc serves: grids of up to 2^27 cells. */
#define IBM_NOALLOC_MAX_CTAS 65536

/* Fluid stage 1 for callers that cannot allocate device memory: writes
 * L = L(U) (as ibm_rhs) and the stable step size *dt = cfl / max_j s_j(U)
 * (as ibm_step computes it), with no handle and no workspace.  There is no
 * counterpart in the paper: this is a packaging of the scheme for hosts that
 * own all device memory (a plug-in that may not call cudaMalloc) or loops
 * that cannot afford an allocation.
 *  - desc: grid description (host); U, L: (dim+2)*N device elements of the
 *    grid's type; dt: one device double; stream: a cudaStream_t.
 *  - Scratch (block maxima, a ticket counter, an error word) lives in one
 *    static device array of 65536 doubles + 256 bytes (about 512 KiB) that
 *    every GPU loading the library holds until the process exits.  The first
 *    call on a device resolves that array's device address (once per device,
 *    with that device current); make that first call before any stream
 *    capture.
 *  - Every call shares the array: calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 *  - A non-finite or non-positive state gives *dt = 0.  No device memory is
 *    allocated or freed.  Errors: IBM_ERR_ARG (invalid description, null
 *    buffer, or a grid of more than 2^27 cells (IBM_NOALLOC_MAX_CTAS blocks); the
 *    message is ibm_last_error(NULL)), IBM_ERR_CUDA.  Asynchronous. */
ibm_status ibm_rhs_dt_noalloc(const ibm_grid_desc *desc, const void *U, void *L, double *dt,
                              void *stream);

/* ---- batches of independent 2D grids ----------------------------------- */

/* A batch advances many independent 2D cases (their own grid size, flow
 * parameters, markers and step size) together: each stage of the step is one
 * persistent kernel launch over a list of (case, tile) work items, so small
 * grids do not each pay a launch and leave most of the GPU idle.  The method
 * per case is exactly that of ibm_step (Sec. 2.1-2.2, App. B); a batch step
 * gives bitwise the same states, step sizes and force sums as calling
 * ibm_step on every case, for every tuning.  Static markers only.
 *
 * Each case is an ordinary ibm_grid owned by the batch (ibm_batch_case):
 * set its state and markers, read its state, forces and time with the usual
 * calls.  ibm_step on one case alone is allowed (the batch notices and
 * rebuilds its tables); ibm_destroy on it is refused. */
typedef struct ibm_batch ibm_batch;

typedef struct {
    int tile_shape;        /* fluid-stage tile: 0 = 16x16, 1 = 32x8, 2 = 64x4, 3 = 8x32 cells */
    int markers_per_block; /* interpolation: warps (one marker each) per CTA, 1..16 */
    int use_graph;         /* != 0: replay each step from a captured CUDA graph */
} ibm_batch_tuning;

/* Bytes of device workspace for ncases grids (descs[ncases], host) with the
 * given marker capacities (max_markers[ncases], host; NULL = 0 each).  All
 * cases must be 2D with the same fp_bytes.  0 if any argument is invalid. */
size_t ibm_batch_workspace_bytes(int ncases, const ibm_grid_desc *descs, const int *max_markers);

/* Create the batch and its ncases grids in one 256-byte aligned device
 * workspace of at least ibm_batch_workspace_bytes bytes (caller-owned).
 * All device work is ordered on `stream`.  Default tuning: shape 0, 4 warps,
 * graphs on.  Errors: IBM_ERR_ARG, IBM_ERR_UNSUPPORTED (a 3D case or mixed
 * fp_bytes), IBM_ERR_WORKSPACE, IBM_ERR_CUDA (message: ibm_batch_last_error(NULL)). */
ibm_status ibm_create_batch(int ncases, const ibm_grid_desc *descs, const int *max_markers,
                            void *dev_workspace, size_t bytes, void *stream, ibm_batch **out);
ibm_status ibm_batch_destroy(ibm_batch *b);

/* The grid of case c (owned by the batch; NULL if out of range). */
ibm_grid *ibm_batch_case(ibm_batch *b, int c);

/* nsteps steps of every case (dt_fixed as in ibm_step).  Every case needs a
 * state; a case with moving markers gives IBM_ERR_UNSUPPORTED.  The first
 * step after a marker change reads the cases' tile counts (synchronizes);
 * otherwise asynchronous, five kernel launches (or one graph) per step. */
ibm_status ibm_batch_step(ibm_batch *b, int nsteps, double dt_fixed);

/* Synchronize and check every case's error word; on error *bad_case (may be
 * NULL) is the first failing case and the status is that case's. */
ibm_status ibm_batch_sync(ibm_batch *b, int *bad_case);

/* Wall temperatures of every case in one upload: Tw holds the kept markers of
 * case 0, then case 1, ... (host, ibm_batch_case(b, c)'s n_kept values per
 * case, in each case's kept order), the batch counterpart of
 * ibm_set_wall_temperature (T_w of Eq. corr3.8's target rho_L c_v T_w).
 * Every value must be finite and positive (IBM_ERR_ARG otherwise, nothing
 * changed).  Tw is read before the call returns if it is pageable and by the
 * stream's copy otherwise, so page-locked buffers must stay unchanged until
 * the next synchronizing call. */
ibm_status ibm_batch_set_wall_temperature(ibm_batch *b, const double *Tw);

/* Forces of all cases from one gathered device read: out[c*8 + i] for
 * i = 0..7 holds Fx, Fy, Q, Cd, Cl, Nu, dt, t of case c (as
 * ibm_forces_and_nusselt and ibm_get_time).  Synchronizes. */
ibm_status ibm_batch_forces(ibm_batch *b, double *out);

ibm_status ibm_batch_get_tuning(const ibm_batch *b, ibm_batch_tuning *t);
ibm_status ibm_batch_set_tuning(ibm_batch *b, const ibm_batch_tuning *t);

/* Time every tile shape (stage 1 + stage 2, reps passes each) and every
 * markers-per-block choice (1, 2, 4, 8, 16 warps; reps interpolation passes)
 * on the current states, keep the fastest of each, and return the measured
 * milliseconds per pass in stage_ms[4] and interp_ms[5] (either may be NULL).
 * The states, step sizes and last marker forcing are left unchanged; the
 * tuning only changes speed, never results.  Synchronizes. */
ibm_status ibm_batch_autotune(ibm_batch *b, int reps, double *stage_ms, double *interp_ms);

/* Kernel timing of batch steps, as ibm_profile / ibm_profile_read (groups
 * IBM_PROF_STAGE1, _STAGE2, _INTERP, _SPREAD, _FINISH; each counts one
 * launch per step).  While it is enabled, steps are launched directly
 * rather than replayed from graphs. */
ibm_status ibm_batch_profile(ibm_batch *b, int enable);
ibm_status ibm_batch_profile_read(ibm_batch *b, double *ms, long long *launches);

const char *ibm_batch_last_error(const ibm_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* IBM_GB300_H */
