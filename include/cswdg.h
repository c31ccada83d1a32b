/*
 * cswdg.h -- C interface of the GB300 (sm_103a) RKDG + compact subcell WENO
 * (CSWENO) solver for 2D Burgers and 2D Euler on unstructured triangles,
 * after Kochi & Ramakrishna, arXiv 2106.06280.
 *
 * Conventions for every entry point:
 *  - Every function returns a cswdg_status; nothing throws or aborts across
 *    the interface.  On failure cswdg_last_error() gives a one-line reason.
 *  - Pointers named *_host are host memory owned by the caller, read or
 *    written only during the call.  Pointers named *_dev are device memory
 *    owned by the caller.  The library owns every other device buffer.
 *  - Cell-indexed arrays are in the caller's cell order (the order of `tri`
 *    in cswdg_mesh_upload); the library reorders cells internally for
 *    locality and undoes it on every read.
 *  - Modal arrays are double, laid out modes[(c*nvar + v)*np + m] for cell c,
 *    variable v (Burgers: u; Euler: rho, rho u, rho v, E) and mode m < np =
 *    (k+1)(k+2)/2, as coefficients of the physically orthonormal basis
 *    psi^K_m(x) = sqrt(2/|K|) psi_m(r(x)), where psi_m is the orthonormal
 *    Dubiner basis on the reference triangle {r,s >= -1, r+s <= 0}
 *    (Sec. 2, Eq. triangleBasis; mode order of the index m there) and r(x)
 *    the affine map taking the triangle's vertices tri[3c], tri[3c+1],
 *    tri[3c+2] to (-1,-1), (1,-1), (-1,1).  The local mass matrix
 *    (Eq. massMatrix2D) is then the identity and the cell mean is
 *    modes[.., 0] / sqrt(|K|).
 *  - Work is issued on cswdg_config.stream (NULL: the legacy default
 *    stream).  Calls that return host data synchronise that stream.
 *  - A solver is not thread-safe; distinct solvers are independent.
 */
#ifndef CSWDG_H
#define CSWDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cswdg_solver cswdg_solver;

typedef enum {
    CSWDG_OK = 0,
    CSWDG_EINVAL = 1,    /* bad argument or call order */
    CSWDG_ECUDA = 2,     /* CUDA runtime error */
    CSWDG_EMESH = 3,     /* non-conforming mesh, unpaired periodic face, missing tag */
    CSWDG_ENONPHYS = 4,  /* Euler cell mean with rho <= 0 or p <= 0, or a NaN */
    CSWDG_ELSQ = 5,      /* rank-deficient stencil least squares at set-up */
    CSWDG_ETIMEOUT = 6,  /* a bounded device wait expired (asynchronous copy into shared memory) */
    CSWDG_ENOMEM = 7     /* device allocation failed */
} cswdg_status;

enum { CSWDG_BURGERS = 0, CSWDG_EULER = 1 };
enum { CSWDG_FP64 = 0, CSWDG_FP32_BULK = 1, CSWDG_FP32 = 2 };
enum { CSWDG_LIMITER_OFF = 0, CSWDG_LIMITER_KXRCF = 1, CSWDG_LIMITER_ALL = 2 };
/* Boundary kinds, cswdg_set_boundary. */
enum {
    CSWDG_BC_PERIODIC = 0,     /* paired by translation (mesh_upload `period`) */
    CSWDG_BC_DIRICHLET = 1,    /* params: nvar constant conserved values */
    CSWDG_BC_TRANSMISSIVE = 2, /* flux: the cell mean as the outside state; detection and stencil: interior trace */
    CSWDG_BC_WALL = 3,         /* Euler: interior trace with the normal momentum reversed */
    CSWDG_BC_SHOCKLINE = 4     /* params: x0, cot, speed, A[nvar], B[nvar];
                                  ghost = A where x < x0 + y*cot + speed*t, else B */
};

typedef struct {
    int32_t equation;  /* CSWDG_BURGERS (Eq. 2dBurgers) or CSWDG_EULER (Eq. 2dEulerEquations) */
    int32_t degree;    /* k in {1, 2}: P^k DG, np = (k+1)(k+2)/2 (Sec. 2) */
    int32_t precision; /* CSWDG_FP64: every step in double.  CSWDG_FP32_BULK: state,
                          operator, RK update and reconstruction polynomials in
                          float with float accumulation; the smoothness-indicator
                          sums, beta_1, tau and the nonlinear weights in double; the
                          troubled-cell and positivity decisions screened in float
                          and recomputed in double when within a relative 1e-3 of
                          the threshold.  CSWDG_FP32: as FP32_BULK with the
                          smoothness indicators and weights in float too (quotient
                          forms that stay inside the float range) */
    int32_t limiter;   /* CSWDG_LIMITER_*: off, troubled cells (Sec. 3.1 KXRCF with ||U_j|| the cell's L2
                          norm over its normalised measure; Euler cells whose polynomial has a
                          non-positive density or pressure at a quadrature point), every cell */
    double c_k;        /* KXRCF threshold C_K (Sec. 3.1 takes 1) */
    double cfl;        /* time-step factor of the CFL rule used when dt <= 0 */
    double gamma;      /* ratio of specific heats (1.4) */
    void *stream;      /* cudaStream_t, or NULL */
} cswdg_config;

/* Create a solver.  Allocates nothing on the device until mesh upload.
 * Errors: EINVAL (unsupported equation/degree/precision/limiter). */
cswdg_status cswdg_create(const cswdg_config *cfg, cswdg_solver **out);

/* Free every device and host resource of the solver (NULL is a no-op). */
void cswdg_destroy(cswdg_solver *s);

/* One-line description of the last error of this solver (never NULL). */
const char *cswdg_last_error(const cswdg_solver *s);

/* Boundary kind and parameters of a face tag (0 <= tag < 16).  Must precede
 * cswdg_mesh_upload for every tag the mesh uses.  Errors: EINVAL. */
cswdg_status cswdg_set_boundary(cswdg_solver *s, int32_t tag, int32_t kind,
                                const double *params_host, int32_t nparams);

/* Upload a conforming straight-sided triangulation (Sec. 2, Eq. triangulation).
 *   xy_host[2*nv]        vertex coordinates
 *   tri_host[3*nc]       counter-clockwise vertex indices per triangle
 *   bface_host[3*nbf]    every boundary edge as (v0, v1, tag)
 *   period_host[2]       (Lx, Ly) translations pairing CSWDG_BC_PERIODIC faces, or NULL
 * Builds faces, neighbours, periodic pairs, a Morton locality order, per-cell
 * geometry, and (limiter on) the per-cell stencil operators of the CSWENO
 * reconstruction on the device.  Sets t = 0 and a zero state.
 * Errors: EINVAL, EMESH, ELSQ, ENOMEM, ECUDA. */
cswdg_status cswdg_mesh_upload(cswdg_solver *s, int64_t nv, const double *xy_host,
                               int64_t nc, const int32_t *tri_host,
                               int64_t nbf, const int32_t *bface_host,
                               const double *period_host);

/* Number of volume-quadrature points per cell (3 for k=1, 7 for k=2). */
int32_t cswdg_num_ic_points(const cswdg_solver *s);

/* Physical coordinates of the volume-quadrature points:
 * xy_host[(c*Q + q)*2 + {0,1}], Q = cswdg_num_ic_points. */
cswdg_status cswdg_ic_points(cswdg_solver *s, double *xy_host);

/* L2 projection of initial values given at those points,
 * values_host[(c*Q + q)*nvar + v], onto the modes.  apply_limiter: 0 none;
 * 1 one pass of the configured limiter at t = 0; 2 one pass reconstructing
 * every cell (for discontinuous data, whose projection can leave negative
 * density or pressure inside cells the detector does not flag).  The
 * limiter runs only when the solver was created with a limiter.
 * Errors: EINVAL, ENONPHYS, ECUDA. */
cswdg_status cswdg_project_ic(cswdg_solver *s, const double *values_host, int32_t apply_limiter);

/* Advance nsteps SSP-RK3 steps (Sec. 3.2, Eq. timeIntegrate, Table tvd: third
 * order), the limiter after every stage.  dt > 0: fixed step; dt <= 0: the
 * CFL rule dt = cfl * min_K r_K / max_K lambda_K (r_K the inradius, lambda_K
 * the largest wave speed of the cell mean).  Steps are clipped so that t never
 * passes t_end; once t == t_end further steps do nothing.  The steps run as a
 * CUDA graph on the solver's stream; the call waits for them once, at the end
 * (to read the time and the error bits).  With a finite t_end (< 1e299) and
 * more than 256 steps, the steps are launched 256 at a time and the call also
 * reads the time after each batch, returning once t_end is reached or an error
 * bit is set, so a large nsteps may stand for "until t_end".  t_out_host
 * (nullable) receives the time reached.
 * Errors: EINVAL, ENONPHYS, ECUDA. */
cswdg_status cswdg_step(cswdg_solver *s, double dt, int64_t nsteps, double t_end, double *t_out_host);

/* The same steps launched one kernel at a time (no graph) with a CUDA event
 * after every launch; ms_host[5] receives the summed device time of each
 * kernel class: [0] CFL reduction + step begin, [1] operator + RK stage,
 * [2] KXRCF detection, [3] CSWENO reconstruction, [4] write-back of the
 * reconstructed modes.  launches_host (nullable): kernels launched.
 * Advances the state like cswdg_step.  Errors: EINVAL, ENONPHYS, ECUDA. */
cswdg_status cswdg_profile_step(cswdg_solver *s, double dt, int64_t nsteps, double t_end,
                                double *ms_host, int64_t *launches_host);

/* Adjoint of the spatial operator (Sec. 2 weak form with the quadrature,
 * local Lax-Friedrichs flux and boundary ghosts of cswdg_eval_rhs):
 * grad = (dL_h/du)^T lambda at state modes_in and time t, all host arrays of
 * nc*nvar*np doubles in the user basis and cell order (as cswdg_eval_rhs), so
 * that  sum(lambda * (L_h(u + e d) - L_h(u)))/e -> sum(grad * d).  At the
 * maximum inside the Lax-Friedrichs speed the derivative follows the branch the
 * forward flux takes.  The limiter is not part of L_h.  Overwrites the
 * solver's state (as cswdg_eval_rhs).  Errors: EINVAL, ECUDA. */
cswdg_status cswdg_rhs_adjoint(cswdg_solver *s, double t, const double *modes_in, const double *lambda_in, double *grad_out);

/* Adjoint of one limiter pass (Sec. 3.1 detection, Sec. 3.2 reconstruction)
 * at state modes_in and time t, with the troubled-cell flags frozen as the
 * forward pass sets them: grad = (d Lim/du)^T lambda, where Lim keeps the
 * unflagged cells and the cell means and replaces the other modes of flagged
 * cells by the reconstruction; the derivative runs through the least-squares
 * fits, smoothness indicators, nonlinear weights and (Euler) the
 * characteristic transforms.  A cell whose reconstruction the positivity
 * fallback replaced contributes nothing.  flags_out (nullable, nc bytes): the
 * flags.  Host arrays as cswdg_rhs_adjoint.  Overwrites the solver's state.
 * Errors: EINVAL (limiter off), ECUDA. */
cswdg_status cswdg_limit_adjoint(cswdg_solver *s, double t, const double *modes_in, const double *lambda_in, double *grad_out,
                                 uint8_t *flags_out);

/* Hand-written adjoint of nsteps SSP-RK3 steps (Sec. 4, Table tvd) with the
 * limiter after every stage (Sec. 3): runs the steps forward from
 * u0_user, keeping the state every checkpoint_every steps, then sweeps back:
 * each segment is recomputed stage by stage from its checkpoint (keeping the
 * unlimited stage outputs and the troubled-cell lists), and the transposed
 * stage updates are applied with the operator adjoint of cswdg_rhs_adjoint
 * and the limiter adjoint of cswdg_limit_adjoint (flags frozen as the forward
 * run set them, derivatives through the WENO weights).  Returns in g0_user
 * the gradient (du_N/du_0)^T gT_user, and in uT_user (nullable) the final
 * state u_N.  dt > 0: every step has size dt; dt <= 0: the forward sweep
 * takes the CFL rule of cswdg_step at every step and the reverse sweep holds
 * the sizes it chose fixed (the dependence of dt on the state is not
 * differentiated); dt_host (nullable, nsteps doubles) receives the sizes.
 * The every-cell limiter is treated like KXRCF with every cell flagged.  Host
 * arrays: nc*nvar*np doubles, user basis and cell order.  Device work
 * memory: about (nsteps/checkpoint_every + 6 checkpoint_every + 5) state
 * arrays and 3 checkpoint_every cell lists, allocated and freed inside the
 * call.  Leaves the solver at u_N and t plus the sum of the step sizes.
 * Errors: EINVAL, ENONPHYS (also a CFL step of no positive size), ENOMEM,
 * ECUDA. */
cswdg_status cswdg_adjoint_steps(cswdg_solver *s, double dt, int64_t nsteps, int32_t checkpoint_every, const double *u0_user,
                                 const double *gT_user, double *uT_user, double *g0_user, double *dt_host);

/* Launch-shape autotuner for the stage kernel (operator + RK update; no
 * counterpart in the paper).  Times CSWDG_TUNE_CANDIDATES shapes -- cells per
 * block 64/128/256, one block per tile of cells or a persistent grid of
 * (SMs x resident blocks), every cell computing its three faces or each face
 * computed once per tile (tile_faces, see cswdg_set_stage_shape) -- on the
 * current state and keeps the fastest for later steps.  Call after the
 * initial condition is set.  ms_host (nullable, CSWDG_TUNE_CANDIDATES
 * doubles): mean kernel time of each candidate in the order 64, 128, 256 (one
 * block per tile), 64 x 8, 128 x 4, 256 x 2, 128 x 8 blocks per SM, then with
 * tile_faces 128, 256 (one block per tile), 128 x 4, 256 x 2 blocks per SM.
 * chosen_host (nullable, 3 int32): cells per block, grid (0 = one block per
 * tile), tile_faces (0/1).  The state is not changed.
 * Errors: EINVAL (no mesh), ECUDA. */
#define CSWDG_TUNE_CANDIDATES 11
cswdg_status cswdg_autotune(cswdg_solver *s, double *ms_host, int32_t *chosen_host);

/* Set the stage kernel's launch shape directly: cells per block (64, 128 or
 * 256), the number of blocks (0: one block per tile of cells; > 0: that
 * many blocks, each looping over tiles) and tile_faces (0: every cell
 * evaluates its three face integrals, forming its neighbours' traces from
 * their modes; 1: a block first writes its cells' traces at the face points to
 * shared memory, then computes the flux of each face between two of its cells
 * once (and of each face to another tile or the boundary from the traces and
 * ghosts as before), 128 or 256 cells per block).  Results do not depend on
 * the shape: the two variants agree bit for bit.  Errors: EINVAL. */
cswdg_status cswdg_set_stage_shape(cswdg_solver *s, int32_t cells_per_block, int32_t grid, int32_t tile_faces);

/* Self-test of the device error path (no counterpart in the paper): launches
 * one warp that waits, with the wait primitive of the reconstruction kernel's
 * bounded waits and at most `polls` polls (1 .. 4,194,304, the kernel's own
 * limit), on a shared-memory barrier phase that never completes, so the wait
 * runs out and sets the timeout error bit; no copy or other work is pending
 * on the barrier, nothing faults or hangs.  Returns CSWDG_ETIMEOUT (the status
 * any bounded wait that ran out produces) and clears the bit, so the solver
 * stays usable; the state is not touched.
 * Errors: EINVAL (no mesh, polls out of range), ECUDA. */
cswdg_status cswdg_selftest_timeout(cswdg_solver *s, int32_t polls);

/* Kernels one cswdg_step step launches (use_cfl: dt <= 0). */
int32_t cswdg_launches_per_step(const cswdg_solver *s, int32_t use_cfl);

/* Current time; set the time (e.g. after restoring a checkpoint). */
cswdg_status cswdg_get_time(cswdg_solver *s, double *t_host);
cswdg_status cswdg_set_time(cswdg_solver *s, double t);

/* Read / write the modal state (layout above, nc*nvar*np doubles).
 * Together with cswdg_set_time this is a full checkpoint. */
cswdg_status cswdg_read_modes(cswdg_solver *s, double *modes_host);
cswdg_status cswdg_write_modes(cswdg_solver *s, const double *modes_host);

/* cswdg_read_modes / cswdg_write_modes with single-precision host arrays (same
 * layout: modes_host[(c*nvar + v)*np + m], physically orthonormal basis, user
 * cell order; caller-owned, nc*nvar*np floats).  In the FP32 and FP32-bulk modes
 * the state itself is float, so only the basis scaling is rounded to float on
 * the way; half the bytes of the double pair cross the bus.  Both wait for
 * their copy.  Errors: EINVAL, ECUDA. */
cswdg_status cswdg_read_modes_f32(cswdg_solver *s, float *modes_host);
cswdg_status cswdg_write_modes_f32(cswdg_solver *s, const float *modes_host);

/* Troubled-cell flags of the last limiter pass (1 byte per cell, 0 or 1);
 * with the limiter off all zero. */
cswdg_status cswdg_read_flags(cswdg_solver *s, uint8_t *flags_host);

/* Number of cells flagged by the last limiter pass. */
cswdg_status cswdg_num_flagged(cswdg_solver *s, int64_t *n_host);

/* sum_K |K| * mean_K per variable (nvar doubles). */
cswdg_status cswdg_conservation(cswdg_solver *s, double *sums_host);

/* The semi-discrete operator alone (Sec. 2, Eq. weakFormScheme2D with the
 * local Lax-Friedrichs flux of Sec. 2 and M = I): rhs = L_h(u) at time t for
 * the given modes.  Replaces the solver state by modes_in.
 * Errors: EINVAL, ECUDA. */
cswdg_status cswdg_eval_rhs(cswdg_solver *s, double t, const double *modes_in_host, double *rhs_host);

/* One limiter pass alone (Sec. 3.1 detection, or every cell, then Sec. 3.2
 * reconstruction of the flagged cells) at time t: the solver state becomes
 * the limited modes_in; modes_out_host and flags_host (both nullable) receive
 * the result.  Errors: EINVAL, ENONPHYS, ECUDA. */
cswdg_status cswdg_limit(cswdg_solver *s, double t, const double *modes_in_host,
                         double *modes_out_host, uint8_t *flags_host);

/* Time step the CFL rule gives for the current state (no clipping). */
cswdg_status cswdg_cfl_dt(cswdg_solver *s, double *dt_host);

/* Device-pointer variant of one SSP-RK3 stage for callers that manage their
 * own buffers: out = a*un + b*(uprev + dt*L_h(uprev)) at time t_rhs, in the
 * library's internal layout (see cswdg_internal_layout) and precision.
 * un_dev may be NULL when a == 0.  The kernels move cells in 16-byte vectors:
 * every pointer must be 16-byte aligned (cudaMalloc's are), else EINVAL.
 * out_dev must not overlap uprev_dev (other cells read it during the stage);
 * it may equal un_dev.  No limiter.  Errors: EINVAL, ECUDA. */
cswdg_status cswdg_stage_dev(cswdg_solver *s, const void *un_dev, const void *uprev_dev, void *out_dev,
                             double a, double b, double dt, double t_rhs);

/* Internal layout of device state arrays: cell-major, element (v, m) of
 * internal cell i at [(i*nvar + v)*np + m] of the precision's type (double in
 * FP64, float in FP32_BULK and FP32), internal cell i = perm_host[user cell].
 * Coefficients are sqrt(2/|K|) times the user modes (the reference-orthonormal
 * basis).  ldc_host (nullable) receives the padded cell count of the
 * per-cell geometry arrays (>= nc; state arrays need nc*nvar*np values).
 * perm_host (nullable) receives nc int32 user->internal indices. */
cswdg_status cswdg_internal_layout(cswdg_solver *s, int64_t *ldc_host, int32_t *perm_host);

/* Diagnostic: the per-cell CSWENO operator block of a user cell as built at
 * mesh upload (subcell-mean weights, least-squares pseudo-inverses,
 * smoothness-indicator factor, gradient maps, projection, mean side length;
 * layout of Ops<K> in csrc/kernels.h).  *n receives its length (0 with the
 * limiter off); out (nullable) receives the values as doubles. */
cswdg_status cswdg_stencil_operator(cswdg_solver *s, int64_t cell, double *out_host, int32_t *n_host);

/* Allocation-free variant of cswdg_conservation for callers that cannot
 * allocate device memory at the time of the call -- for example code that
 * runs while a CUDA graph is being captured with allocations not allowed,
 * real-time loops with a fixed memory budget, or host applications that own
 * every device allocation themselves.  (The paper has no counterpart; this is
 * an interface service.)
 *   modes_dev  device state of nc cells in the library's internal layout and
 *              precision (cswdg_internal_layout), caller-owned
 *   sums_dev   device output, nvar doubles: sum_K |K| * mean_K per variable
 * Work is queued on the solver's stream; nothing is synchronised.  The
 * reduction's scratch is one fixed device array inside the library (2 MiB on
 * every GPU that loads it, held until the process exits), so the call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library call.  Limit: at most
 * 16,777,216 cells (larger meshes get CSWDG_EINVAL).  The work runs on the
 * solver's device (the one current when its mesh was uploaded), whichever
 * device is current at the call; the call makes it current for its duration
 * and restores the caller's device.  The first call for a device looks up the
 * array's device address there (cudaGetSymbolAddress, once per device, safe
 * from several host threads); make that first call before any stream capture.
 * All calls share the array: two calls whose
 * work overlaps on the GPU (different streams, or different solvers on the
 * same device at the same time) race; calls queued on one stream do not.
 * Every call rewrites the part of the scratch it reads, so no clearing is
 * needed.  Errors: EINVAL, ECUDA. */
cswdg_status cswdg_conservation_noalloc(cswdg_solver *s, const void *modes_dev, double *sums_dev);

/* FP64 FMA throughput of the current device, measured (no counterpart in the
 * paper; the ceiling for the FP64-pipe-bound parts of the path): 5 launches of
 * 8 x SMs blocks of 256 threads, each thread running 8 independent chains of
 * 4,096 fused multiply-adds, timed with CUDA events on `stream` (a
 * cudaStream_t, 0 for the default stream).  *gflops_out receives 2 x FMAs / s
 * in GFLOP/s.  Allocates one 8-byte device word for the duration of the call.
 * Errors: EINVAL (null output), ENOMEM, ECUDA. */
cswdg_status cswdg_probe_fp64_fma(void *stream, double *gflops_out);

/* Host-side mesh processing alone, without a solver or a device (no
 * counterpart in the paper; for tests and inspection): the connectivity,
 * periodic pairing, locality order and geometry that cswdg_mesh_upload builds.
 * degree 1 or 2; bc_kind_host: CSWDG_BC_* kind of each of the 16 face tags
 * (as set by cswdg_set_boundary); the mesh arguments as cswdg_mesh_upload.
 * Outputs (each nullable), in the internal cell order:
 *   geo_host  14 x nc doubles, array-major: 2 dr/dx, 2 dr/dy, 2 ds/dx, 2 ds/dy,
 *             then for local faces f = 0, 1, 2 the outward unit normal (x, y)
 *             and |n~| = 2 |edge| / |cell|, then the KXRCF scale kappa;
 *   nbr_host  3 x nc: the internal index of the neighbour across face f, or
 *             -(boundary record + 1) for a boundary face;
 *   nbf_host  nc: the neighbour's local face index of each face, 2 bits per face;
 *   perm_host nc: the caller's index of each internal cell.
 * Errors: EINVAL, EMESH (the status only; there is no solver to hold a message). */
cswdg_status cswdg_host_mesh(int32_t degree, const int32_t *bc_kind_host, int64_t nv, const double *xy_host, int64_t nc,
                             const int32_t *tri_host, int64_t nbf, const int32_t *bface_host, const double *period_host,
                             double *geo_host, int32_t *nbr_host, uint8_t *nbf_host, int32_t *perm_host);

#ifdef __cplusplus
}
#endif
#endif /* CSWDG_H */
