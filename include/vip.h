/*
 * vip.h -- C ABI of libvip, the GPU (sm_103a) path of the virtual interpolation
 * point (VIP) fractional-step solver of Park, Jo and Choe, "Virtual
 * Interpolation Point Method for Viscous Flows in Complex Geometries".
 *
 * The calls follow the paper's statement of the problem: a node set and its
 * geometry (Sec. 3: the node set Lambda), the moving least-squares fit (Sec. 3:
 * quadratic basis, weight function Phi, dilation rho), the flow parameters
 * (Sec. 2: Re, dt) and then the fractional step, Eqs. (12)-(15), per time step.
 *
 * Conventions for every call
 *   - Every call returns vip_status; none aborts, traps or exits.  After an
 *     error vip_last_error() gives a one-line diagnostic.
 *   - Array arguments are plain pointers.  Unless stated otherwise a pointer
 *     may be host memory (pageable or pinned) or device memory of the
 *     context's device; the library copies from / into it (cudaMemcpyDefault).
 *     Inputs are copied, so the caller keeps ownership and may reuse them as
 *     soon as the call returns.  Outputs go into caller-owned buffers.
 *   - Node arrays are in the caller's order, geometries concatenated in the
 *     order they were added ("global node order").
 *   - Work is issued on the stream passed to vip_create.  Calls that return
 *     host data synchronise that stream; vip_step does not.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef VIP_H
#define VIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vip_ctx vip_ctx; /* opaque, owned by the library */

typedef enum {
    VIP_OK = 0,
    VIP_ERR_ARG = 1,              /* invalid argument or call order */
    VIP_ERR_CUDA = 2,             /* a CUDA runtime call failed */
    VIP_ERR_SINGULAR_STENCIL = 3, /* a moment matrix failed its Cholesky test */
    VIP_ERR_NOT_CONVERGED = 4,    /* a Krylov solve hit its iteration limit */
    VIP_ERR_BREAKDOWN = 5,        /* BiCGSTAB could not continue (no progress) */
    VIP_ERR_NONFINITE = 6,        /* NaN/Inf in an input or a residual */
    VIP_ERR_TIMEOUT = 7,          /* a device-side wait ran out its spin limit */
    VIP_ERR_OOM = 8               /* device allocation failed */
} vip_status;

/* Node kinds (one byte per node), Sec. 5 boundary conditions:
 *   INTERIOR  momentum and Poisson equations collocated at the node;
 *   WALL      velocity Dirichlet (value from vip_set_state, held fixed),
 *             pressure-increment zero normal derivative (walls, lid, inflow);
 *   SLIP      u zero normal derivative, v Dirichlet, pressure increment zero
 *             normal derivative (channel top/bottom, "v = 0, t_x = 0");
 *   OUTLET    velocity zero normal derivative, pressure increment = 0
 *             (traction-free outflow). */
enum { VIP_NODE_INTERIOR = 0, VIP_NODE_WALL = 1, VIP_NODE_SLIP = 2, VIP_NODE_OUTLET = 3 };

/* Weight function Phi of Sec. 3, in r = |x_i - xbar| / rho:
 *   CUBIC_SPLINE  2/3-4r^2+4r^3 (r<=1/2), 4/3-4r+4r^2-4r^3/3 (1/2<r<1), 0 else;
 *   PAPER         (1 - r^((1-r)^2))^4 for r < 1, 0 else (the printed form). */
enum { VIP_W_CUBIC_SPLINE = 0, VIP_W_PAPER = 1 };

/* Precision of the Krylov solves (Eqs. 12-13).  Every form stops on the same
 * test, the FP64 relative residual ||b - A x|| / ||b|| <= rtol of the FP64
 * operator, so they differ in cost and in the rounding of the solution only.
 *   FP64   BiCGSTAB in FP64 on FP64 operators; the Poisson solve's multigrid
 *          preconditioner in FP64;
 *   MIXED  iterative refinement: FP64 residual b - A x on FP64 operators; the
 *          correction equation A d = r solved by BiCGSTAB in FP32 arithmetic
 *          on FP32 vectors and FP32 copies of the operators (stencil rows
 *          applied in differenced form, sum_k a_ik (d_k - d_i) + rowsum_i d_i
 *          with the FP64 row sum rounded to FP32), preconditioned by an FP32
 *          V-cycle, to a relative tolerance set by vip_set_refinement; the
 *          correction is accumulated without rounding loss (an FP32 pair per
 *          row, error-free sums and products); repeated until the FP64
 *          residual meets rtol;
 *   MG32   BiCGSTAB in FP64 (operator applications, vectors, dot products)
 *          whose multigrid preconditioner runs in FP32 (FP32 copies of every
 *          level's operator, FP32 vectors); only the Poisson solve has a
 *          preconditioner, so the Helmholtz solves run as FP64. */
enum { VIP_PREC_FP64 = 0, VIP_PREC_MIXED = 1, VIP_PREC_MG32 = 2 };

/* Identity operator wherever the paper writes I in Eq. (12):
 *   EXACT  the identity; MLS  the MLS approximant D^[0,0] (Eq. vip:1). */
enum { VIP_IDENTITY_EXACT = 0, VIP_IDENTITY_MLS = 1 };

/* Pressure of Eqs. (12) and (15) (the paper prints r^n of Eq. 12 without a
 * pressure term but Eq. 15 with p^n; these forms are readings of the pair):
 *   INCREMENTAL           r^n carries -G p^n, so phi is the pressure increment,
 *                         and p^{n+1} = p^n + phi - (dt/2Re) L phi at every node;
 *                         the wall pressures are carried from step to step, and
 *                         on some node sets the linearised step then has an
 *                         eigenvalue slightly above 1 (the circle of radius 0.55
 *                         at h = 1/128, Re 40, dt = 0.15 h: 1.0088, neutral at
 *                         h = 1/64), so a long run there grows without bound;
 *   KIM_MOIN              r^n as printed (no pressure term), so phi is the whole
 *                         pseudo-pressure of Kim and Moin, and
 *                         p^{n+1} = phi - (dt/2Re) L phi (Eq. 15 without p^n); the
 *                         steady state carries a splitting error of order dt;
 *   INCREMENTAL_INTERIOR  INCREMENTAL with the term -(dt/2Re) L phi of Eq. 15 at
 *                         interior nodes only (boundary nodes: p^n + phi).  At a
 *                         boundary node L is a one-sided MLS fit; on the 28.072
 *                         degree wedge of Sec. 5 the term there feeds a growing
 *                         wall-pressure mode (an eigenvalue of the linearised
 *                         step above 1), which this form does not have (on the
 *                         circle at h = 1/128 it has one too, 1.0024; KIM_MOIN,
 *                         which carries no pressure, has none there). */
enum { VIP_PRESSURE_INCREMENTAL = 0, VIP_PRESSURE_KIM_MOIN = 1, VIP_PRESSURE_INCREMENTAL_INTERIOR = 2 };

/* Tables and operators that can be exported (vip_get_stencil) or applied
 * (vip_apply).  Rows are global nodes; columns are global nodes, except the
 * column index N (total node count) of the POISSON operator, which is the
 * extra unknown mu of a closed domain (see VIP_OP_POISSON).
 *   NBR          neighbour lists of the nodes, value = 1           (Sec. 3)
 *   D00..D02     node derivative approximants D^[a,b]      (Eq. fmlsrk:2)
 *   LAPLACE      D^[2,0] + D^[0,2]                             (Eq. vip:1)
 *   VIP_E..VIP_S MLS interpolation Psi^[0,0](x_vip) to the east, west,
 *                north and south VIPs of interior nodes (empty rows for
 *                boundary nodes)                                (Sec. 4.1)
 *   GX, GY       merged VIP differences (u(x_e)-u(x_w))/|x_e-x_w| and
 *                (u(x_n)-u(x_s))/|x_n-x_s| (Sec. 4.1 items 2 and 3)
 *   HELM_U/V     Helmholtz operator of Eq. (12) times dt for u and v with
 *                the boundary rows
 *   POISSON      operator of Eq. (13) with boundary rows; for a geometry
 *                with no OUTLET node it is bordered by one extra unknown mu
 *                (column and row N + k for the k-th such geometry): interior
 *                rows i carry + mu, the first interior node k0 of the geometry
 *                gets the row (-4/h^2) phi_k0 = 0, and row N + k holds node k0's
 *                own equation plus mu. */
enum {
    VIP_OP_NBR = 0, VIP_OP_D00 = 1, VIP_OP_D10 = 2, VIP_OP_D01 = 3, VIP_OP_D20 = 4,
    VIP_OP_D11 = 5, VIP_OP_D02 = 6, VIP_OP_LAPLACE = 7, VIP_OP_VIP_E = 8,
    VIP_OP_VIP_W = 9, VIP_OP_VIP_N = 10, VIP_OP_VIP_S = 11, VIP_OP_GX = 12,
    VIP_OP_GY = 13, VIP_OP_HELM_U = 14, VIP_OP_HELM_V = 15, VIP_OP_POISSON = 16,
    VIP_OP_COUNT = 17
};

typedef struct {
    int64_t steps;            /* time steps taken since vip_set_state */
    int32_t helm_iters;       /* last step: BiCGSTAB iterations, Helmholtz (max over systems) */
    int32_t poisson_iters;    /* last step: inner BiCGSTAB iterations, Poisson (max) */
    int32_t poisson_outer;    /* last step: FP64 refinement passes, Poisson (max) */
    int32_t status;           /* first vip_status raised on the device, VIP_OK if none */
    double helm_relres;       /* last step: final FP64 relative residual (max) */
    double poisson_relres;    /* last step: final FP64 relative residual (max) */
    int64_t total_poisson_iters; /* inner Poisson iterations summed over all steps */
    int64_t total_poisson_outer; /* FP64 refinement passes of the Poisson solves, summed */
    int64_t total_helm_iters;    /* Helmholtz iterations (max over systems), summed */
} vip_step_stats;

/* Phases of one fractional step, timed with CUDA events recorded on the
 * context's stream inside each step (see vip_set_profiling). */
enum { VIP_PHASE_RHS = 0, VIP_PHASE_HELMHOLTZ = 1, VIP_PHASE_DIVERGENCE = 2,
       VIP_PHASE_POISSON = 3, VIP_PHASE_PROJECT = 4, VIP_PHASE_COUNT = 5 };

/* Create a context on CUDA device `device`; work is issued on `cuda_stream`
 * (a cudaStream_t, NULL = the legacy default stream). */
vip_status vip_create(vip_ctx** out, int device, void* cuda_stream);
void vip_destroy(vip_ctx* ctx);
const char* vip_last_error(const vip_ctx* ctx);

/* Add one geometry (node set Lambda of Sec. 3) to the context's batch.
 * n nodes; x, y coordinates; kind per node (VIP_NODE_*); nx, ny unit outward
 * normal of the fluid domain at boundary nodes (ignored at interior nodes);
 * h_local > 0, the local node spacing (rho = support * h_local, VIPs at
 * +-h_local/2, normal auxiliary points at h_local and 2 h_local, see
 * vip_set_probes); Lx, Ly > 0
 * make the geometry periodic with that period (0 = not periodic).  All arrays
 * are copied.  *geom_out receives the geometry index (0, 1, ...).
 * Must precede vip_build. */
vip_status vip_add_nodes(vip_ctx* ctx, int64_t n, const double* x, const double* y,
                         const uint8_t* kind, const double* nx, const double* ny,
                         const double* h_local, double Lx, double Ly, int32_t* geom_out);

/* MLS fit of Sec. 3: basis_order must be 2 (the six-term quadratic basis);
 * weight is VIP_W_*; support is the ratio rho / h_local (> 1).  Defaults:
 * 2, VIP_W_CUBIC_SPLINE, 2.2.  Must precede vip_build. */
vip_status vip_set_mls(vip_ctx* ctx, int basis_order, int weight, double support);

/* Placement of the two auxiliary points on the inward normal of a boundary node
 * (the zero-normal-derivative rows of the pressure increment, q_i - 4/3 q(x_b1)
 * + 1/3 q(x_b2) = 0; the paper states no boundary condition for phi, so these
 * rows are a reading of Sec. 2 and 4):
 *   NORMAL  x_b1 = x_i - h_local n_i, x_b2 = x_i - 2 h_local n_i;
 *   INSIDE  the same with h_local replaced by a step s_i that starts at h_local
 *           and is multiplied by 0.7 (at most 12 times) while x_b2 lies less
 *           than 0.05 h_j inside the tangent at the boundary node j nearest to
 *           x_b2, i.e. while (x_b2 - x_j) . n_j > -0.05 h_j.  Where two walls
 *           meet at a narrow angle (the 28.072 degree apex of the triangular
 *           cavity of Sec. 5) the plain points pass through the opposite wall.
 * Nearest: smallest Euclidean distance (periodic minimum image) among the
 * geometry's non-interior nodes.  INSIDE needs a support ratio above 2 (the
 * search radius is the support radius of the boundary node, which contains
 * x_b2); vip_build returns VIP_ERR_ARG otherwise. */
enum { VIP_PROBES_NORMAL = 0, VIP_PROBES_INSIDE = 1 };

/* Normal-point placement VIP_PROBES_* of geometry `geom` (-1 = every
 * geometry); default NORMAL.  Must precede vip_build.  VIP_ERR_ARG for a bad
 * mode or geometry index, or after vip_build. */
vip_status vip_set_probes(vip_ctx* ctx, int32_t geom, int mode);

/* Flow parameters of geometry `geom` (-1 = every geometry): Reynolds number
 * and time step of Sec. 2.  Must precede vip_build (the operators depend on
 * dt/Re). */
vip_status vip_set_flow(vip_ctx* ctx, int32_t geom, double Re, double dt);

/* Krylov settings: precision VIP_PREC_*, relative residual tolerance
 * ||b - A x||_2 <= rtol ||b||_2 for both solves, iteration limit per solve,
 * identity VIP_IDENTITY_*.  Defaults FP64, 1e-8, 20000, EXACT.
 * The identity mode must be set before vip_build. */
vip_status vip_set_solver(vip_ctx* ctx, int precision, double rtol, int32_t max_iters,
                          int identity);

/* Pressure form VIP_PRESSURE_* of the fractional step (default INCREMENTAL).
 * May be called at any time; the next step uses it.  VIP_ERR_ARG for a bad
 * form. */
vip_status vip_set_pressure(vip_ctx* ctx, int form);

/* Inner tolerance of the MIXED form's refinement loop (not in the paper; the
 * solves of Eqs. 12-13 stop at the same FP64 residual whatever it is): each FP32
 * BiCGSTAB pass stops when its recursive residual has fallen to inner_rtol times
 * the FP64 residual it started from (or to rtol ||b|| / 2).  `which` =
 * VIP_OP_POISSON (the pressure-increment solve; default 1e-4) or VIP_OP_HELM_U (both
 * Helmholtz solves; default 1e-6: near the identity, their FP32 inner solve reaches
 * the FP64 tolerance in one pass).  inner_rtol in (0, 1).  VIP_ERR_ARG otherwise.
 * May be called at any time. */
vip_status vip_set_inner_tolerance(vip_ctx* ctx, int which, double inner_rtol);

/* vip_set_inner_tolerance for both solves at once. */
vip_status vip_set_refinement(vip_ctx* ctx, double inner_rtol);

/* Build everything that depends only on the geometry and flow parameters:
 * neighbour search (nodes, VIPs, normal auxiliary points), MLS moment
 * matrices and weights (Eq. fmlsrk:2), merged operators (Eqs. 12-15,
 * Sec. 4.1).  Returns VIP_ERR_SINGULAR_STENCIL if some moment matrix fails
 * its Cholesky test (the message names the point). Synchronous. */
vip_status vip_build(vip_ctx* ctx);

/* Set u^n, v^n, p^n (N doubles each, global node order; NULL p = zero) and
 * reset phi, the convection history and the step counter.  Velocity Dirichlet
 * values are taken from u, v at Dirichlet nodes and held fixed. */
vip_status vip_set_state(vip_ctx* ctx, const double* u, const double* v, const double* p);

/* Overwrite u^n, v^n, p^n (N doubles each, global node order) and continue:
 * unlike vip_set_state, phi, the convection history, the step counter and
 * the Dirichlet values are kept.  For callers that change the fields between
 * steps.  Asynchronous for device pointers and pinned host memory. */
vip_status vip_load_state(vip_ctx* ctx, const double* u, const double* v, const double* p);

/* Advance nsteps fractional steps, Eqs. (12)-(15), for every geometry.
 * Asynchronous on the context's stream (one CUDA graph launch per step when
 * graphs are enabled).  Device-side failures are reported by vip_get_stats. */
vip_status vip_step(vip_ctx* ctx, int32_t nsteps);

/* Copy the state out (N doubles each; any pointer may be NULL).  phi is the
 * last pressure increment.  Synchronises the stream. */
vip_status vip_get_state(vip_ctx* ctx, double* u, double* v, double* p, double* phi);

/* ---- checkpoint and resume (not in the paper) --------------------------------
 * A checkpoint holds everything the next fractional step depends on: u^n, v^n,
 * p^n, the last pressure increment phi (the Poisson solve's initial guess), the
 * convection term N^{n-1} of the Adams-Bashforth extrapolation (Eq. 12), the held
 * Dirichlet values, the learned warm start's history (the increment before phi)
 * and the step counter (which selects the first step's Euler start).  The
 * network's parameters and the extrapolation coefficient are not part of it.  Restoring it makes the following vip_step calls repeat, bit for bit,
 * the steps that followed the save (the kernels' reductions are deterministic).
 * Statistics counters (vip_get_stats totals, vip_get_geometry_iters) are not part
 * of it.  Layout: a 64-byte header (magic, node/row/geometry counts, host step
 * count, checksum = the sum modulo 2^64 of the body's 64-bit words), then nine
 * arrays of R doubles in the padded row space, then the step counter; R is an
 * internal size, so buffers are sized by vip_checkpoint_size.
 *
 * vip_checkpoint_size: *bytes = the buffer size for this context.  After vip_build.
 * vip_checkpoint: save != 0 writes a checkpoint to buf (host or device memory of
 * `bytes` bytes, caller-owned); save == 0 restores one, returning VIP_ERR_ARG
 * (state unchanged) if buf holds no checkpoint of a context of the same sizes or
 * its checksum does not match.  Synchronous; uses a device scratch buffer of the
 * checkpoint's size when buf is host memory, freed before it returns. */
vip_status vip_checkpoint_size(vip_ctx* ctx, int64_t* bytes);
vip_status vip_checkpoint(vip_ctx* ctx, int save, void* buf);

/* enable != 0: vip_step waits for each step and adds the CUDA-event time of
 * every phase (VIP_PHASE_*) to a running total; 0 stops it.  Enabling resets
 * the totals. */
vip_status vip_set_profiling(vip_ctx* ctx, int enable);

/* Phase times summed over the profiled steps (ms, VIP_PHASE_COUNT doubles)
 * and the number of profiled steps. */
vip_status vip_get_profile(vip_ctx* ctx, double* phase_ms, int64_t* nsteps);

/* Statistics of the last step (synchronises).  Returns the device status. */
vip_status vip_get_stats(vip_ctx* ctx, vip_step_stats* out);

/* Poisson BiCGSTAB iterations of each geometry (int64 per geometry, in the order
 * the geometries were added), summed over the steps since vip_set_state.  In a
 * context with several geometries all systems are solved by one launch and a
 * system that has converged stops iterating, so these are the per-geometry work
 * counts (vip_get_stats reports the maximum).  Synchronises. */
vip_status vip_get_geometry_iters(vip_ctx* ctx, int64_t* poisson_iters);

/* Total node count N and the number of geometries. */
vip_status vip_get_sizes(vip_ctx* ctx, int64_t* n_nodes, int32_t* n_geoms);

/* Size of an exported table: rows (N, or N + number of bordered geometries
 * for VIP_OP_POISSON) and stored entries.  After vip_build. */
vip_status vip_stencil_info(vip_ctx* ctx, int which, int64_t* nrows, int64_t* nnz);

/* Device storage of a Krylov operator (the Helmholtz operator of Eq. 12,
 * `which` = VIP_OP_HELM_U or VIP_OP_HELM_V, which share one table, or the Poisson
 * operator of Eq. 13, VIP_OP_POISSON; the storage itself is not in the paper), as
 * each operator application reads it: `slices` slices of 32 rows;
 * `uniform_slices` of them hold the same stencil in all 32 rows (the same value,
 * bit for bit, at each entry, and columns at the same offsets from the row or at
 * the same column) and read it from a table of distinct stencils (uniform slices
 * with equal stencils share one copy) of `uniform_entries` entries in total; the
 * other slices are read as
 * `other_entries` stored entries (8-byte value + 4-byte column each, padding
 * included).  Any output pointer may be NULL.  After vip_build. */
vip_status vip_operator_layout(vip_ctx* ctx, int which, int64_t* slices, int64_t* uniform_slices,
                               int64_t* uniform_entries, int64_t* other_entries);

/* Size of the Poisson preconditioner's hierarchy (not in the paper; see
 * vip_set_multigrid): `levels` coarse levels, the last solved exactly by a dense
 * inverse per geometry; `coarsest_entries` = sum over geometries of m_g^2, m_g the
 * geometry's cells on that level (each V-cycle reads these FP64 entries once).
 * Zeros without a multigrid.  Any output pointer may be NULL.  After vip_build. */
vip_status vip_multigrid_info(vip_ctx* ctx, int32_t* levels, int64_t* coarsest_entries);

/* Export table `which` as CSR: row_ptr[nrows+1], col[nnz], val[nnz], columns
 * ascending within a row.  Host or device pointers.  Synchronises. */
vip_status vip_get_stencil(vip_ctx* ctx, int which, int64_t* row_ptr, int32_t* col,
                           double* val);

/* y = Op x for a table `which` in FP64 (x of length = columns, y = rows).
 * Synchronises. */
vip_status vip_apply(vip_ctx* ctx, int which, const double* x, double* y);

/* Convection term of Sec. 4.1 item 1 at every node (zero at boundary nodes)
 * for the velocity field (u, v).  Synchronises. */
vip_status vip_convection(vip_ctx* ctx, const double* u, const double* v, double* Nu,
                          double* Nv);

/* Solve system `which` (VIP_OP_HELM_U, VIP_OP_HELM_V or VIP_OP_POISSON) for
 * every geometry at once with the step's Krylov solver: b and x have the
 * operator's row count; x holds the initial guess on entry and the solution
 * on return.  iters (may be NULL) gets the iteration count, relres (may be
 * NULL) the largest final FP64 relative residual over geometries. */
vip_status vip_solve(vip_ctx* ctx, int which, const double* b, double* x, int precision,
                     double rtol, int32_t max_iters, int32_t* iters, double* relres);

/* ---- multigrid parameters and their autotuner --------------------------------
 * Not part of the paper's method: the Poisson solve of Eq. (13) is preconditioned
 * by an aggregation multigrid V-cycle (l1-Jacobi smoothing with damping omega,
 * coarse-grid correction scaled by corr; defaults 1.0 and 1.5).  Both change the
 * iteration count only, never the residual the solve stops at. */
vip_status vip_set_multigrid(vip_ctx* ctx, float omega, float corr);

/* Parity of the multigrid's first cell grid for geometry geom (-1: every geometry):
 * level 1 aggregates the nodes of 2h x 2h cells of the geometry's background
 * lattice; shift_x = 1 (shift_y = 1) moves the cell boundaries by one lattice
 * spacing in x (y).  Not part of the paper's method; like omega and corr it changes
 * the iteration count of the Eq. (13) solve, never the residual it stops at.
 * Default 0, 0.  Shifts are 0 or 1, a periodic axis keeps 0.  Before vip_build
 * (VIP_ERR_ARG after it, for a bad index or value). */
vip_status vip_set_mg_shift(vip_ctx* ctx, int32_t geom, int32_t shift_x, int32_t shift_y);

#define VIP_TUNE_MAX 16
typedef struct {
    int32_t ncand;                 /* candidates tried (nomega x ncorr) */
    int32_t best;                  /* index of the chosen candidate */
    float omega[VIP_TUNE_MAX];     /* candidate k: omega[k], corr[k] */
    float corr[VIP_TUNE_MAX];
    int32_t iters[VIP_TUNE_MAX];   /* Poisson BiCGSTAB iterations (max over geometries) */
    double ms[VIP_TUNE_MAX];       /* device time of the solve, -1 if it failed */
} vip_tune_result;

/* Time the pressure-increment solve of the last step (its right-hand side, from a
 * zero initial guess, to the context's tolerance) for every pair of omegas[0..nomega)
 * and corrs[0..ncorr) (at most VIP_TUNE_MAX pairs; omega in (0, 1.5], corr in (0, 3]),
 * apply the fastest pair that converged (as vip_set_multigrid) and report all of them.
 * Needs vip_build, the multigrid and at least one vip_step since vip_set_state; the
 * state is not changed.  Uses one R-double device scratch vector, freed before it
 * returns.  Synchronous. */
vip_status vip_autotune(vip_ctx* ctx, const float* omegas, int32_t nomega, const float* corrs,
                        int32_t ncorr, vip_tune_result* out);

/* ---- learned warm start of the pressure-increment solve ------------------
 * Not part of the paper's method: the Poisson solve of Eq. (13) starts from
 *   phi^n + a (phi^n - phi^{n-1}) + S * prediction
 * and runs to the same tolerance (Eq. 13 unchanged).  a is a temporal
 * extrapolation coefficient fitted by least squares on the collected solves;
 * the prediction is a 6-layer 3x3 convolutional network (BF16 tensor-core
 * kernels, FP32 accumulation) on each geometry's regular background lattice,
 * from u*, v*, the divergence right-hand side, phi^n, phi^n - phi^{n-1} and node
 * masks, trained on what the extrapolation leaves of phi^{n+1} - phi^n, in units
 * of S D: S the RMS of phi^n and D the RMS of (phi^n - phi^{n-1}) / S, per
 * geometry.  Untrained (a = 0, last layer zero) the guess is phi^n, the
 * previous-increment guess. */
typedef struct {
    int32_t epochs;     /* passes over the collected samples */
    double lr;          /* Adam step size */
    uint64_t seed;      /* sample order */
    double first_loss;  /* out: mean loss of the first epoch */
    double final_loss;  /* out: mean loss of the trained network over the samples */
    double extrap;      /* out: the fitted extrapolation coefficient a */
    double base_loss;   /* out: mean loss of the extrapolation alone (output zero) */
    int32_t net_kept;   /* out: 1 if final_loss < base_loss; 0: the network's last
                           layer was zeroed, the guess is the extrapolation alone */
} vip_train_cfg;

/* enable != 0: from the next step on, store (network input, solved increment
 * change) of every step, up to max_samples (device memory, owned by the context);
 * steps run without the CUDA graph while collecting.  0 stops collecting. */
vip_status vip_ws_collect(vip_ctx* ctx, int enable, int32_t max_samples);

/* Fit the extrapolation coefficient a on the collected samples (least squares
 * over interior lattice nodes, clamped to [-1, 2]), then train the network on
 * what a (phi^n - phi^{n-1}) leaves of phi^{n+1} - phi^n (Adam, one sample per
 * update, the loss of vip_ws_set_loss over interior lattice nodes); the network is
 * kept only if it lowers the mean loss over the samples below that of the
 * extrapolation alone, else its last layer is zeroed.  Synchronous. */
vip_status vip_ws_train(vip_ctx* ctx, vip_train_cfg* cfg);

/* The Poisson solve's initial guess in vip_step: enable 0: phi^n (the previous
 * increment); 1: the learned guess, extrapolation plus network; 2: the fitted
 * extrapolation alone, phi^n + a (phi^n - phi^{n-1}) (no network evaluation).
 * Other values: VIP_ERR_ARG. */
vip_status vip_ws_enable(vip_ctx* ctx, int enable);

/* direction 0: copy the FP32 parameters out to buf; 1: load them from buf.
 * *count receives the parameter count (buf may be NULL to query it).  Layout:
 * for each layer, weights [3][3][cin][cout] then bias [cout]; widths
 * 16 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1. */
vip_status vip_ws_params(vip_ctx* ctx, int direction, float* buf, int64_t* count);

/* Evaluate the network on one H x W lattice image x[H][W][16] (FP32, converted
 * to BF16); y[H][W] (may be NULL) receives the output.  With target, mask and
 * grads non-NULL also the loss set by vip_ws_set_loss over mask != 0 (*loss) and
 * its parameter gradients (grads, parameter layout).  Synchronous. */
vip_status vip_ws_eval(vip_ctx* ctx, int32_t H, int32_t W, const float* x, float* y, float* grads,
                       const float* target, const float* mask, double* loss);

/* Loss of the network's training (vip_ws_train) and of vip_ws_eval, over the
 * interior lattice nodes, with e = prediction - target:
 *   kind 0: mean squared error, mean of e^2;
 *   kind 1 (default): residual proxy, mean of (Delta e)^2 + lam e^2, Delta the
 *           5-point lattice Laplacian (lattice units, zero outside the image):
 *           the solve starts from the residual the guess leaves, the Poisson
 *           operator applied to its error, so rough errors weigh more than smooth
 *           ones.  lam >= 0 (default 0.01).
 * VIP_ERR_ARG for another kind or a negative weight. */
vip_status vip_ws_set_loss(vip_ctx* ctx, int kind, double lam);

/* Samples of the extrapolation coefficient's least-squares fit in vip_ws_train:
 * window 0 (default) every collected sample, window >= 1 the last `window` of
 * them.  A collection that starts at an impulsive start is dominated by its first
 * large increments; a window fits the coefficient to the recent flow (h = 1/32
 * cylinder, 2,000 samples: a = 0.990 over all, 0.999 over the last 40, and 440
 * against 335 Poisson iterations over 40 held-out steps).  Errors: VIP_ERR_ARG
 * (before vip_build, window < 0). */
vip_status vip_ws_set_fit_window(vip_ctx* ctx, int32_t window);

/* set != 0: set the extrapolation coefficient to *a (in [-1, 2], else
 * VIP_ERR_ARG); 0: read it into *a.  With vip_ws_params it moves a trained warm
 * start from one context to another. */
vip_status vip_ws_extrapolation(vip_ctx* ctx, int set, double* a);

/* One Adam update of the network parameters (the optimiser of vip_ws_train:
 * beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, FP32) with step size lr > 0,
 * applied to the gradients of the last vip_ws_eval call that computed gradients
 * (or of the last training sample); the step count runs from the last load of the
 * parameters by vip_ws_params (direction 1), which also zeroes the moments.
 * Synchronous.  With vip_ws_eval it lets a caller train on samples of its own. */
vip_status vip_ws_adam(vip_ctx* ctx, double lr);

/* ---- BiCGSTAB without device allocation -----------------------------------
 * An addition of this library; the paper has no counterpart.  For callers that
 * must not allocate device memory while they run: a process whose device memory
 * belongs to another framework's caching allocator (a cudaMalloc behind its back
 * can fail or fragment its pool), a real-time loop, or code under a fixed memory
 * budget.  vip_solve needs a context (vip_create/vip_build allocate); this call
 * needs none.
 *
 * Solves A x = b in FP64 with unpreconditioned BiCGSTAB for a general square
 * sparse A given as CSR (row_ptr[n+1], col[nnz] in [0, n), val[nnz]); all five
 * arrays are DEVICE pointers owned by the caller, on `device`.  x holds the
 * initial guess on entry and the solution on return.  Stops when
 * ||b - A x|| <= rtol ||b|| (the recursive residual) or after max_iters
 * iterations (VIP_ERR_NOT_CONVERGED, x = last iterate).  iters (may be NULL)
 * gets the iteration count, relres (may be NULL) the true relative residual of
 * the returned x.  The call runs on cuda_stream (NULL = the legacy default
 * stream) of `device`, synchronises with it, and leaves the caller's current
 * device as it was.
 *
 * Workspace: file-scope static device memory, at most VIP_STATIC_MAX_ROWS rows;
 * larger n returns VIP_ERR_ARG before any device work.  Each call clears the
 * barrier words and result record it uses (on cuda_stream); nothing needs to be
 * zero beforehand.  The call is synchronous (it waits for cuda_stream and reads
 * its result back), so it cannot be recorded into a CUDA graph: on a stream that
 * is capturing it returns VIP_ERR_ARG before any work, leaving the capture
 * intact.  The first call on a device looks up the workspace's device address
 * (and loads the module there) and keeps it for the life of the process; after
 * a cudaDeviceReset of that device the kept address is stale, so a process that
 * resets a device must not call this entry point on it again.  All calls on one
 * device share the one workspace, so calls that overlap in time on that device
 * (other streams, other host threads) race and must be serialised by the caller.
 * Errors: VIP_ERR_ARG (bad size or tolerance; a NULL pointer, a host pointer or
 * memory of another device; a capturing stream), VIP_ERR_CUDA,
 * VIP_ERR_BREAKDOWN, VIP_ERR_NOT_CONVERGED, VIP_ERR_TIMEOUT (a grid-barrier wait
 * ran out; the result is not valid). */
#define VIP_STATIC_MAX_ROWS 131072
vip_status vip_bicgstab_static(int device, void* cuda_stream, int64_t n, const int64_t* row_ptr,
                               const int32_t* col, const double* val, const double* b, double* x,
                               double rtol, int32_t max_iters, int32_t* iters, double* relres);

/* ---- three-dimensional operator build --------------------------------------
 * The paper's introduction and Sec. 3 state that the method carries over to
 * three dimensions with the quadratic basis of ten monomials
 * [1, xi, eta, zeta, xi^2, xi eta, xi zeta, eta^2, eta zeta, zeta^2]; it shows no
 * 3D flow.  These calls build the 3D counterparts of the 2D tables (neighbour
 * search and MLS weights of Sec. 3, Eq. fmlsrk:2; the operators of Eq. vip:1 and
 * Sec. 4.1) on the GPU, with the readings of the 2D build: strict support
 * |x_i - xbar| < rho, rho = support * h of the point's own node; VIPs at half the
 * node's spacing along each axis (six: east/west along x, north/south along y,
 * top/bottom along z); at boundary nodes the zero-normal-derivative row
 * q_i - (4/3) q(x_i - h n_i) + (1/3) q(x_i - 2 h n_i) with MLS values at the two
 * normal points.  The 3D fractional step (vip_3d_step below) runs on node sets
 * of interior and wall nodes, periodic or not.
 * A vip_3d handle has the conventions of vip_ctx (status returns, copied
 * inputs, caller-owned outputs, host or device pointers, its own stream). */
typedef struct vip_3d vip_3d; /* opaque, owned by the library */

/* Tables of the 3D build, exported as CSR (rows = nodes, columns = nodes):
 *   NBR               neighbour lists of the nodes, value = 1
 *   D000 .. D002      node derivative approximants D^[a,b,c] for (0,0,0),
 *                     (1,0,0), (0,1,0), (0,0,1), (2,0,0), (0,2,0), (0,0,2)
 *   LAPLACE           D^[2,0,0] + D^[0,2,0] + D^[0,0,2]
 *   VIP_E .. VIP_B    interpolation Psi^[0,0,0](x_vip) to the six VIPs of the
 *                     interior nodes (empty rows for boundary nodes)
 *   GX, GY, GZ        (q(x_e) - q(x_w)) / |x_e - x_w| and its y and z
 *                     counterparts (interior rows)
 *   NEUMANN           q_i - (4/3) q(x_i - h n_i) + (1/3) q(x_i - 2 h n_i)
 *                     (boundary rows) */
enum {
    VIP3_OP_NBR = 0, VIP3_OP_D000 = 1, VIP3_OP_D100 = 2, VIP3_OP_D010 = 3, VIP3_OP_D001 = 4,
    VIP3_OP_D200 = 5, VIP3_OP_D020 = 6, VIP3_OP_D002 = 7, VIP3_OP_LAPLACE = 8,
    VIP3_OP_VIP_E = 9, VIP3_OP_VIP_W = 10, VIP3_OP_VIP_N = 11, VIP3_OP_VIP_S = 12,
    VIP3_OP_VIP_T = 13, VIP3_OP_VIP_B = 14, VIP3_OP_GX = 15, VIP3_OP_GY = 16, VIP3_OP_GZ = 17,
    VIP3_OP_NEUMANN = 18, VIP3_OP_COUNT = 19
};

/* Create a handle on `device` (work issued on cuda_stream, NULL = legacy default
 * stream).  Errors: VIP_ERR_ARG, VIP_ERR_CUDA. */
vip_status vip_3d_create(vip_3d** out, int device, void* cuda_stream);

/* Node set: n nodes (1 <= n < 2^31 - 1) with coordinates x, y, z, kinds (the
 * VIP_NODE_* codes; every non-interior kind gets a NEUMANN row), unit outward
 * normals (nx, ny, nz; read at non-interior nodes only) and local spacing h > 0.
 * Lx, Ly, Lz: periods, all three > 0 (periodic; coordinates in [0, L)) or all
 * three 0.  Replaces an earlier node set and its tables.  Errors: VIP_ERR_ARG
 * (sizes, non-finite or non-positive values, mixed periodicity, periodic
 * coordinates outside [0, L), a non-interior node in a periodic set),
 * VIP_ERR_CUDA, VIP_ERR_OOM. */
vip_status vip_3d_set_nodes(vip_3d* b, int64_t n, const double* x, const double* y,
                            const double* z, const uint8_t* kind, const double* nx,
                            const double* ny, const double* nz, const double* h, double Lx,
                            double Ly, double Lz);

/* Weight function (VIP_W_*) and support ratio rho / h (> 1; default cubic
 * spline, 2.2).  Errors: VIP_ERR_ARG. */
vip_status vip_3d_set_mls(vip_3d* b, int weight, double support);

/* Neighbour lists (at most 160 per point) and MLS weights of every node, VIP and
 * normal point.  Synchronises.  Errors: VIP_ERR_ARG (no node set; a point with
 * more than 160 neighbours), VIP_ERR_SINGULAR_STENCIL (a
 * moment matrix failed its Cholesky test; vip_3d_last_error names the point),
 * VIP_ERR_CUDA, VIP_ERR_OOM. */
vip_status vip_3d_build(vip_3d* b);

/* Row count (the node count) and entry count of table `which`.  Assembles the
 * table on the device on first use.  Errors: VIP_ERR_ARG (not built, bad
 * which), VIP_ERR_CUDA, VIP_ERR_OOM. */
vip_status vip_3d_stencil_size(vip_3d* b, int which, int64_t* nrows, int64_t* nnz);

/* Export table `which` as CSR: row_ptr[nrows+1], col[nnz] (ascending within a
 * row), val[nnz]; host or device pointers.  Synchronises.  Errors as
 * vip_3d_stencil_size. */
vip_status vip_3d_get_stencil(vip_3d* b, int which, int64_t* row_ptr, int32_t* col, double* val);

/* y = Op x in FP64 on the device for table `which` (x and y of the node count;
 * host or device pointers).  Synchronises.  Errors as vip_3d_stencil_size. */
vip_status vip_3d_apply(vip_3d* b, int which, const double* x, double* y);

/* ---- the fractional step in 3D (Sec. 2, Eqs. 12-15) ------------------------
 * The step of the 2D library in three coordinates on a built node set of
 * interior and wall nodes (VIP_NODE_WALL: velocity Dirichlet, holding the value
 * of the last vip_3d_set_state; pressure increment with zero normal derivative
 * through the NEUMANN rows, scaled by -6/h^2): convection through the six VIPs
 * of each interior node (Sec. 4.1 item 1), Adams-Bashforth 2 (N^{-1} = N^0 on the
 * first step), Crank-Nicolson viscous term with the exact identity, the
 * incremental pressure reading (r^n carries -G p^n; p^{n+1} = p^n + phi -
 * (dt/2Re) L phi at every node), the MLS Laplacian in the Poisson equation.  No
 * node fixes phi, so the Poisson system is bordered by one unknown mu added to
 * the interior rows, the first interior node k0's own equation moved to an extra
 * row and its row replaced by (-6/h_k0^2) phi_k0 = 0.  Every solve is
 * unpreconditioned FP64 BiCGSTAB to ||b - A x|| <= rtol ||b|| on the true
 * residual, the Helmholtz solves starting from u^n, the Poisson solve from
 * (phi^n, mu^n).  The 2D library's multigrid has no 3D counterpart, so the
 * Poisson iterations grow with the node count.
 *
 * vip_3d_set_flow: Re > 0, dt > 0, rtol in (0, 1), max_iters >= 1 per solve.
 * vip_3d_set_state: u, v, w, p of every node (host or device); phi, mu and the
 *   Adams-Bashforth history are reset.
 * vip_3d_step: nsteps steps; synchronous.  After an error other than
 *   VIP_ERR_ARG the fields and the Adams-Bashforth history are partly updated:
 *   set the state again before stepping on.  Errors: VIP_ERR_ARG (not built, no
 *   flow or state, SLIP or OUTLET nodes, no interior node), VIP_ERR_NOT_CONVERGED,
 *   VIP_ERR_BREAKDOWN,
 *   VIP_ERR_NONFINITE, VIP_ERR_CUDA, VIP_ERR_OOM.
 * vip_3d_get_state: u, v, w, p, phi of every node into caller buffers (any may
 *   be NULL).
 * vip_3d_get_iters: steps taken since vip_3d_set_state, and of the last step the
 *   Helmholtz iterations (three solves together), the Poisson iterations and
 *   the Poisson solve's true relative residual (any pointer may be NULL). */
vip_status vip_3d_set_flow(vip_3d* b, double Re, double dt, double rtol, int32_t max_iters);
vip_status vip_3d_set_state(vip_3d* b, const double* u, const double* v, const double* w,
                            const double* p);
vip_status vip_3d_step(vip_3d* b, int32_t nsteps);
vip_status vip_3d_get_state(vip_3d* b, double* u, double* v, double* w, double* p, double* phi);
vip_status vip_3d_get_iters(vip_3d* b, int64_t* steps, int32_t* helm_iters, int32_t* poisson_iters,
                            double* poisson_relres);

/* One-line diagnostic of the last error on this handle ("" if none). */
const char* vip_3d_last_error(const vip_3d* b);

/* Free the handle and its device memory.  NULL is allowed. */
void vip_3d_destroy(vip_3d* b);

#ifdef __cplusplus
}
#endif
#endif /* VIP_H */
