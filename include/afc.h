/*
 * afc.h - C ABI of libafc, a GB300 (sm_103a) library for algebraic flux
 * correction (AFC) of P1/Q1 finite element discretisations of 3D
 * convection-diffusion-reaction (CDR) equations.
 *
 * Method: Jha, Partl, Ahmed, Kuzmin, "An assessment of solvers for algebraically
 * stabilized discretizations of convection-diffusion-reaction equations"
 * (arXiv 2110.15676).  Section / equation names below refer to that paper.
 *
 * Conventions shared by every call
 *  - Every call returns an int status (afc_status).  No C++ exception crosses
 *    this boundary.  afc_status_str() gives a message; afc_last_error() gives
 *    the detail of the last failure on the calling thread.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Pointers
 *    documented as "device" must point to memory on the problem's device.
 *  - The library owns every device buffer it allocates, until afc_destroy().
 *  - All device work is enqueued on the stream given at creation (NULL = the
 *    legacy default stream).  Calls that return values to host memory
 *    synchronise that stream before returning.
 *  - A problem handle is used by one host thread at a time.
 *  - Structured meshes number nodes ix + nx*(iy + ny*iz) (x fastest).
 *  - All floating point data is IEEE double unless stated otherwise.
 */
#ifndef AFC_H
#define AFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afc_problem_s* afc_problem;

typedef enum {
  AFC_OK = 0,
  AFC_NOT_CONVERGED = 1,  /* result valid (last iterate), tolerance not met   */
  AFC_E_INVALID = -1,     /* bad argument or size                             */
  AFC_E_OOM = -2,         /* device allocation failed                         */
  AFC_E_CUDA = -3,        /* CUDA runtime error (detail in afc_last_error)    */
  AFC_E_NAN = -4,         /* NaN or Inf met in a residual or solver scalar    */
  AFC_E_TIMEOUT = -5,     /* a bounded device wait expired                    */
  AFC_E_STATE = -6        /* call out of order (e.g. step before assemble)    */
} afc_status;

typedef enum { AFC_P1 = 0, AFC_Q1 = 1 } afc_elem;     /* tetrahedra / trilinear hexahedra */

/* Which matrix family afc_assemble builds.
 * FCT: A = eps*S + K + c*M_C (Sec. 2), D from A, AA = A + D.
 * MC : flux correction of the eps = 0, c = 0 operator (Remark rem:assembling_mc):
 *      D from the convective matrix K, AA = K + D + eps*S + c*M_L (lumped reaction). */
typedef enum { AFC_FAMILY_FCT = 0, AFC_FAMILY_MC = 1 } afc_family;

typedef enum { AFC_SSP2 = 0, AFC_SSP3 = 1, AFC_CN_NONLINEAR = 2, AFC_CN_LINEAR = 3 } afc_scheme;
/* Limiters: alpha = 0 (NONE), alpha = 1 (GALERKIN), Zalesak's (Sec. 2.1.3, FCT
 * schemes), monolithic convex (Eq. MClimiter) and monolithic upwind (Sec. 3, MU
 * limiter; stationary problems, MC family). */
typedef enum {
  AFC_LIM_NONE = 0, AFC_LIM_GALERKIN = 1, AFC_LIM_ZALESAK = 2, AFC_LIM_MC = 3, AFC_LIM_MU = 4
} afc_limiter;
typedef enum { AFC_KSP_BICGSTAB = 0, AFC_KSP_GMRES = 1 } afc_ksp;
typedef enum { AFC_FP64 = 0, AFC_MIXED = 1 } afc_precision;

/* Matrices afc_export_csr can return. */
typedef enum {
  AFC_MAT_MC = 0,      /* consistent mass m_ij                                     */
  AFC_MAT_A = 1,       /* matrix whose off-diagonals define D (FCT: A, MC: K)       */
  AFC_MAT_D = 2,       /* discrete upwinding d_ij                                   */
  AFC_MAT_LOW = 3,     /* low-order operator AA = A + D (no Dirichlet rows applied) */
  AFC_MAT_K = 4,       /* convection (b . grad phi_j, phi_i)                        */
  AFC_MAT_S = 5        /* stiffness (grad phi_j, grad phi_i)                        */
} afc_matrix;

typedef struct {
  int64_t n_nodes;        /* N                                                     */
  int64_t nnz;            /* stored pattern entries (pairs with m_ij != 0, and i=i) */
  int64_t n_edges;        /* pairs i < j in the pattern                            */
  int32_t n_offsets;      /* K: distinct column offsets j - i (odd, contains 0)    */
  int32_t max_offset;     /* largest |j - i|                                       */
  int64_t device_bytes;   /* device memory held by the problem                     */
  int32_t assembled;      /* 1 after afc_assemble                                  */
  int32_t family;         /* afc_family of the assembly                            */
} afc_info;

/* Options of afc_step / afc_solve_stationary (see afc_default_opts). */
typedef struct {
  int32_t scheme;         /* afc_scheme (afc_step only)                                   */
  int32_t limiter;        /* afc_limiter                                                  */
  double dt;              /* time step (afc_step); see afc_cfl_timestep                   */
  double fp_tol;          /* nonlinear stop: ||res||_2 < sqrt(N) * fp_tol (Eq. tol_formula)*/
  int32_t fp_maxit;       /* max fixed-point iterations                                   */
  int32_t fp_fixed_its;   /* > 0: run exactly this many fixed-point corrections           */
  double omega;           /* damping of the fixed point (Sec. 4)                          */
  int32_t ksp;            /* afc_ksp                                                      */
  int32_t ksp_maxit;      /* max inner iterations (per solve)                             */
  double ksp_atol;        /* inner stop: ||r||_2 < max(ksp_atol, ksp_rtol * ||r_0||_2)    */
  double ksp_rtol;
  int32_t gmres_restart;  /* GMRES(m) restart length, 1..32                               */
  int32_t precision;      /* afc_precision: AFC_MIXED runs the inner solve (CN, stationary)*/
                          /* or the raw fluxes r_ij (SSP) in FP32; limiter sums, alpha    */
                          /* and the lumped-mass update stay FP64; the stationary MC      */
                          /* residual and clip run in float pairs (see                    */
                          /* afc_mc_residual_sweep)                                       */
  int32_t prelimit;       /* CN: apply Eq. prelimiting (L = 2)                            */
  int32_t graph;          /* 1: run the whole step / solve as one CUDA graph with the     */
                          /* loop control on the device (default); 0: host-driven loop    */
} afc_opts;

typedef struct {
  int32_t outer_its;      /* fixed-point corrections (linear solves) performed            */
  int32_t inner_its;      /* Krylov iterations summed over the solves                     */
  int32_t stages;         /* explicit FE stages performed                                 */
  int32_t status;         /* same as the call's return value                              */
  double res0;            /* first nonlinear residual norm                                */
  double res_final;       /* last nonlinear residual norm                                 */
  double umin, umax;      /* extremes of the returned solution                            */
  double dmp_violation;   /* max(0, lo - umin, umax - hi): how far the returned solution  */
                          /* lies outside [lo, hi], the range of the call's input state   */
                          /* and of the Dirichlet values.  The discrete maximum principle */
                          /* of the limited schemes (Sec. 2.1.3, Eq. MClimiter) keeps it  */
                          /* at rounding level for f = 0, c = 0 (the stationary solve: at */
                          /* the level of its tolerance); a source can raise u above hi   */
  double t_ms;            /* host wall time of the call (per-kernel device times: see     */
                          /* afc_profile)                                                 */
} afc_stats;

/* ---- lifetime -------------------------------------------------------------- */

/* Uniform box grid [lo, hi] with nx*ny*nz nodes (each >= 2).  P1 cuts every
 * cell into the six Kuhn tetrahedra sharing the cell diagonal from its corner
 * (0,0,0) to (1,1,1); Q1 uses one trilinear hexahedron per cell.  `stream` is a
 * cudaStream_t (or NULL).  On success *out owns the problem. */
int afc_create_structured(int elem, int nx, int ny, int nz, const double lo[3], const double hi[3],
                          int device, void* stream, afc_problem* out);

/* Mesh from an element list (host arrays): xyz[3*n_nodes] (x, y, z per node),
 * conn[4*n_cells] (P1) or conn[8*n_cells] (Q1, local vertex k = dx + 2dy + 4dz
 * of a box-shaped cell).  The pattern may use at most 63 distinct column
 * offsets j - i (always true for meshes of up to 32 nodes and for structured
 * grids); AFC_E_INVALID otherwise. */
int afc_create_from_elements(int elem, int64_t n_nodes, const double* xyz, int64_t n_cells,
                             const int32_t* conn, int device, void* stream, afc_problem* out);

int afc_destroy(afc_problem p);

/* ---- data --------------------------------------------------------------------- */

/* Coefficients of Eq. tcdr / Eq. cdr (host arrays):
 *  eps       diffusion, >= 0;
 *  b_nodal   velocity at the nodes, b_nodal[3*i + d] (interpolated with the element
 *            basis), or NULL to use the constant b_const[3] at every node;
 *  c_nodal   reaction at the nodes (N values >= 0, interpolated with the element
 *            basis: the Galerkin matrix (c_h phi_j, phi_i), lumped to its row sums in
 *            the MC family), or NULL for the constant c_const >= 0 (c_const M_C, and
 *            c_const M_L in the MC family);
 *  f_nodal   source at the nodes (NULL = 0); the load vector is M_L f_nodal.
 * AFC_E_INVALID for a negative or non-finite eps or reaction, or neither b_nodal
 * nor b_const.  The next afc_assemble uses them. */
int afc_set_coefficients(afc_problem p, double eps, const double* b_nodal, const double b_const[3],
                         const double* c_nodal, double c_const, const double* f_nodal);

/* Dirichlet set: mask[N] (nonzero = Dirichlet node), values[N] (used where mask). */
int afc_set_dirichlet(afc_problem p, const uint8_t* mask, const double* values);

/* Assemble on the device: M_C, M_L, S, K, A, D and AA (Sec. 2, Eq. low_order_disc)
 * for the given family; with precision AFC_MIXED also FP32 copies of the system
 * matrices.  Needs coefficients; Dirichlet data may be set before or after. */
int afc_assemble(afc_problem p, int family, int precision);

int afc_get_info(afc_problem p, afc_info* out);

/* Copy one matrix out as CSR with sorted columns (host arrays of n_nodes + 1,
 * nnz, nnz entries; see afc_get_info).  For tests and inspection. */
int afc_export_csr(afc_problem p, int which, int32_t* rowptr, int32_t* col, double* val);

/* Lumped mass m_i = sum_j m_ij (host array of N). */
int afc_export_lumped_mass(afc_problem p, double* mL);

/* Solution vector u (N doubles); is_device selects a device or a host pointer. */
int afc_set_solution(afc_problem p, const double* u, int is_device);
int afc_get_solution(afc_problem p, double* u, int is_device);

/* Reading of a CFL number: dt = cfl * min over non-Dirichlet i of m_i / AA_ii. */
int afc_cfl_timestep(afc_problem p, double cfl, double* dt);

void afc_default_opts(afc_opts* o);

/* ---- the hot path ---------------------------------------------------------- */

/* One time step of the stored solution.
 *  AFC_SSP2 / AFC_SSP3: explicit FE-SSP stages (Eq. FE-SSP) with the predictor
 *    u~ = u + dt M_L^{-1}(f - AA u) and Zalesak's limiter (Sec. 2.1.2, 2.1.3),
 *    combined as Heun (SSP2, Sec. 2.1.2) or three-stage Shu-Osher (SSP3).
 *  AFC_CN_NONLINEAR: Eq. CNZal solved by the damped fixed point of Sec. 4 with
 *    fluxes Eq. flux_002 (+ Eq. prelimiting if opts->prelimit), the predictor
 *    Eq. forward_euler and a Jacobi-preconditioned Krylov solve per iteration.
 *    With limiter AFC_LIM_MC (MC family, FP64) each stage is the transient MC
 *    update of Sec. 2.2: the fluxes Eq. defn_r_ij_SSP clipped by Eq. MClimiter
 *    with the bounds and bar states of the stage input.
 *    With AFC_LIM_MC (MC family) the CN step uses F* = (F*(u^n) + F*(u^{n-1})) / 2
 *    with F*(u) = sum_j r*_ij(u), the fluxes of Eq. defn_r_ij_SSP clipped by
 *    Eq. MClimiter (Sec. 2.2).
 *  AFC_CN_LINEAR: linear Zal+CN (Sec. 2.1.1): u^n in Eq. flux_002 is replaced by
 *    2 u~ - u^{n-1}, so F* is known before the step and Eq. CNZal is one linear
 *    system, solved by one Krylov solve (fp_tol, fp_maxit, omega are not used).
 * Returns AFC_NOT_CONVERGED (solution updated with the last iterate) if the
 * fixed point did not reach fp_tol within fp_maxit. */
int afc_step(afc_problem p, const afc_opts* o, afc_stats* st);

/* Stationary AFC system AA u = f + F*(u) (Sec. 3, Sec. 3.1) with the MC limiter
 * (Eq. MClimiter), the MU limiter (Sec. 3, MU limiter) or alpha = 1 / alpha = 0,
 * by the damped fixed point of Sec. 4 in defect form, starting from the stored
 * solution.  Needs the MC family assembly for any limiter but NONE. */
int afc_solve_stationary(afc_problem p, const afc_opts* o, afc_stats* st);

/* ---- single passes, for parity checks and diagnostics (host arrays) -------- */

/* One forward-Euler FCT stage from the stored solution, without changing it:
 * predictor u_tilde, Zalesak factors R+ / R-, limited sum F* and the new state
 * (Eq. FE-SSP).  Any output pointer may be NULL. */
int afc_fe_stage(afc_problem p, double dt, int limiter, double* u_tilde, double* Rp, double* Rm,
                 double* Fstar, double* u_new);

/* Limited antidiffusive sum of the CN scheme for given u_new, u_old (host, N):
 * F*(u_new, u_old) of Eq. CNZal with Zalesak factors built from the CN predictor
 * of u_old.  Also returns the predictor and R+ / R- (may be NULL). */
int afc_cn_limited_sum(afc_problem p, double dt, int limiter, int prelimit, const double* u_new,
                       const double* u_old, double* u_tilde, double* Rp, double* Rm, double* Fstar);

/* Limited sum F*_i = sum_j alpha_ij r_ij of the stationary fluxes r_ij = d_ij (u_j - u_i)
 * for a given u (host, N): MC (Eq. MClimiter, with the bounds u_max / u_min of
 * Eq. u_max_min), MU (Sec. 3, MU limiter; u_max / u_min not written), GALERKIN or
 * NONE (outputs may be NULL). */
int afc_mc_limited_sum(afc_problem p, int limiter, const double* u, double* umax, double* umin,
                       double* Fstar);

/* Same limited sum as afc_mc_limited_sum, for callers that cannot allocate
 * device memory (for example code running while a stream is being captured, or
 * an embedding runtime that forbids cudaMalloc after start-up).  The paper has
 * no counterpart; this is a deployment variant.
 *  u      device array of N doubles (no halo needed), input state;
 *  Fstar  device array of N doubles, output F*_i (0 at Dirichlet rows).
 * The bounds u_max / u_min it needs live in a fixed 4 MiB device array that
 * every GPU loading the library holds until exit, so N may be at most 262144
 * (AFC_E_INVALID otherwise).  Like afc_mc_limited_sum it needs the MC family
 * assembly for any limiter but NONE (AFC_E_STATE otherwise).  The calling
 * thread's current device is the same after the call as before it.  No
 * cudaMalloc, cudaFree or allocating library call is made.  Work is enqueued on the problem's stream and the call returns
 * without synchronising.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (other
 * streams or other problems on the same device) race. */
int afc_mc_limited_sum_noalloc(afc_problem p, int limiter, const double* u, double* Fstar);

/* One limiter + residual sweep of the stationary problem on the stored solution:
 * bounds (Eq. u_max_min), limited fluxes (Eq. MClimiter, or alpha = 1 / 0 per
 * `limiter`) and res = f + F*(u) - AA u into internal buffers.  Only enqueued on
 * the problem's stream (no synchronisation, no host copy): for timing the sweep.
 * On a mixed-precision assembly the MC and Galerkin sweeps run as the stationary
 * solve with AFC_MIXED runs them: in float-pair arithmetic on the FP32 pipe (values
 * carried as two floats, 48 significand bits), which agrees with the FP64 sweep to
 * ~1e-14 of the magnitudes summed.  Values must stay below 2^127 in magnitude. */
int afc_mc_residual_sweep(afc_problem p, int limiter);

/* Copy out (host array of N) the nonlinear residual res = f + F*(u) - AA u of the
 * stationary problem (Sec. 4; 0 at Dirichlet rows) that the last
 * afc_mc_residual_sweep left in its internal buffer.  Synchronises the stream. */
int afc_get_residual(afc_problem p, double* res);

/* y = AA x (which = AFC_MAT_LOW) or y = M x (AFC_MAT_MC), host arrays of N. */
int afc_apply(afc_problem p, int which, const double* x, double* y);

/* Solve the system matrix of the stationary problem (system = 0: AA with
 * identity Dirichlet rows) or of the CN step (system = 1: M_L/dt + AA/2 with
 * identity Dirichlet rows) for host rhs / x (x in: ignored, out: solution),
 * Jacobi-preconditioned BiCGStab or GMRES per the options. */
int afc_linear_solve(afc_problem p, int system, double dt, const afc_opts* o, const double* rhs,
                     double* x, int* its, double* res);

/* ---- batches of independent problems ------------------------------------------
 *
 * A batch runs the explicit FE-SSP step (as afc_step with AFC_SSP2 / AFC_SSP3)
 * of many independent problems together: every pass of a stage (rate, edges,
 * factors, correct; see afc_step) covers the rows of all instances in one
 * launch, so small instances do not leave the GPU idle, and each time step is
 * one CUDA graph.  Each instance keeps its own arrays and its own stored
 * solution (afc_set_solution / afc_get_solution still apply), and gives the same
 * result bit for bit as afc_step on it alone with the same options. */
typedef struct afc_batch_s* afc_batch;

/* Launch shapes of a batched step. */
typedef enum {
  AFC_BATCH_AUTO = 0,       /* the tuned shape for this batch's size class, else PER_STAGE  */
  AFC_BATCH_PER_PASS = 1,   /* one launch per pass (4 per stage), each over all instances    */
  AFC_BATCH_PER_STAGE = 2,  /* one persistent cooperative launch per stage; the passes are   */
                            /* separated by grid-wide barriers with a bounded wait          */
  AFC_BATCH_PER_STEP = 3    /* one persistent cooperative launch per time step              */
} afc_batch_mode;

typedef struct {
  int32_t mode;           /* afc_batch_mode                                               */
  int32_t block;          /* threads per block = rows per tile: 128, 256 or 512           */
  int32_t blocks_per_sm;  /* persistent modes: resident blocks per SM, 0 = most that fit  */
  double ms_per_step;     /* afc_batch_tune: measured device time of one step (output)    */
} afc_batch_tuning;

/* Batch of `count` assembled problems on one device (at most 65536).  The batch
 * keeps the handles (not copies): the problems must outlive it and must not be
 * used by other calls while a batch call runs.  Work is enqueued on the stream
 * of list[0]. */
int afc_batch_create(const afc_problem* list, int count, afc_batch* out);
int afc_batch_destroy(afc_batch b);

/* `nsteps` explicit SSP steps of every instance.  opts->scheme is AFC_SSP2 or
 * AFC_SSP3, opts->limiter NONE / GALERKIN / ZALESAK, opts->precision FP64 or
 * MIXED (see afc_opts); opts->graph is ignored (the step is always a graph).
 * dt: host array of `count` time steps, or NULL to use opts->dt for all.
 * stats: host array of `count` results (umin, umax, stages) or NULL.
 * Returns AFC_E_TIMEOUT if a grid barrier of a persistent launch gave up waiting
 * (the instances' solutions are then undefined).  Synchronises the stream. */
int afc_batch_step(afc_batch b, const afc_opts* o, const double* dt, int nsteps, afc_stats* stats);

/* Fix the launch shape (mode AFC_BATCH_AUTO returns to the tuned / default one). */
int afc_batch_set_tuning(afc_batch b, const afc_batch_tuning* t);
int afc_batch_get_tuning(afc_batch b, afc_batch_tuning* t);

/* Time every launch shape (modes x block sizes x residency) on this batch with
 * these options, keep the fastest for the batch and for its size class (element
 * types present, log2 of the total and of the mean node count, precision,
 * limiter, scheme) for later batches of the process, and return it in *best.
 * The instances' solutions are saved before and restored after the trials. */
int afc_batch_tune(afc_batch b, const afc_opts* o, const double* dt, afc_batch_tuning* best);

/* Total nodes of the batch's instances and the number of kernel launches its
 * calls have issued (either pointer may be NULL). */
int afc_batch_info(afc_batch b, int64_t* total_nodes, int64_t* launches);

/* ---- a request server ------------------------------------------------------------
 *
 * A server solves requests (a transient SSP run or a stationary solve of one CDR
 * problem on a box grid) submitted from any thread, with the problems' data
 * resident on the device while they run:
 *  - AFC_SERVE_BATCHED: admission threads admit requests in arrival order
 *    while their estimated device memory fits the budget and the slot count
 *    allows, and build their problems, `builders` at once; all admitted transient
 *    requests advance
 *    together in batched SSP steps (afc_batch_step), in chunks of at most
 *    max_chunk steps, and requests admitted meanwhile join at the next chunk;
 *    stationary requests run concurrently, each on its own stream, on
 *    `stationary_workers` threads.
 *  - AFC_SERVE_SERIAL: one request at a time in arrival order (afc_step per
 *    step, afc_solve_stationary), nothing overlapped: the plain baseline.
 * A request's result does not depend on the other requests (a batched step
 * gives an instance the same bits as afc_step). */
typedef struct afc_server_s* afc_server;

typedef enum { AFC_REQ_TRANSIENT = 0, AFC_REQ_STATIONARY = 1 } afc_request_kind;
typedef enum { AFC_SERVE_BATCHED = 0, AFC_SERVE_SERIAL = 1 } afc_serve_mode;
typedef enum {
  AFC_REQ_PENDING = 0,    /* submitted, not admitted                                     */
  AFC_REQ_RUNNING = 1,    /* admitted: problem resident on the device                    */
  AFC_REQ_DONE = 2,       /* finished; status may be AFC_NOT_CONVERGED                    */
  AFC_REQ_FAILED = 3,     /* a library call failed; status holds its code                 */
  AFC_REQ_CANCELLED = 4
} afc_request_state;

typedef struct {
  int32_t kind;           /* afc_request_kind                                              */
  int32_t elem;           /* afc_elem                                                      */
  int32_t n[3];           /* nodes per side of the box grid                                */
  double lo[3], hi[3];    /* the box                                                       */
  double eps, c;          /* diffusion, reaction                                           */
  const double* b;        /* 3N nodal velocity (copied at submission)                      */
  const double* f;        /* N nodal source, or NULL                                       */
  const uint8_t* dir_mask;/* N                                                             */
  const double* u_dir;    /* N Dirichlet values                                            */
  const double* u0;       /* N initial data (transient) or initial guess (stationary)     */
  int32_t family;         /* afc_family to assemble                                        */
  int32_t steps;          /* transient: number of steps                                    */
  double cfl;             /* transient: dt = cfl * min m_i / AA_ii unless opts.dt > 0      */
  afc_opts opts;          /* scheme (SSP2 / SSP3), limiter, precision, solver settings     */
} afc_request;

typedef struct {
  int32_t state;          /* afc_request_state                                             */
  int32_t status;         /* afc_status of the solve                                       */
  afc_stats stats;        /* transient: stages, umin, umax, the largest dmp_violation of its    */
                          /* steps; stationary: as afc_solve_stationary                    */
  int64_t n_nodes;
  double t_submit, t_admit, t_done;   /* seconds on the server's clock                     */
  char message[160];      /* FAILED: the library's error detail                            */
} afc_result;

typedef struct {
  int32_t mode;               /* afc_serve_mode                                            */
  int32_t max_active;         /* requests admitted at once                                 */
  int64_t hbm_budget;         /* device bytes admitted requests may hold (estimated)       */
  int32_t stationary_workers; /* concurrent stationary solves (1..64)                      */
  int32_t max_chunk;          /* transient steps per batched call                          */
  int32_t builders;           /* AFC_SERVE_BATCHED: requests whose problems are built at   */
                              /* once (1..64; admission stays in arrival order)            */
} afc_serve_config;

typedef struct {
  int64_t pending, active, bytes_in_use, completed, failed;
  int64_t chunks;             /* batched calls issued                                      */
  int64_t batched_steps;      /* steps advanced by those calls                             */
  int64_t max_batch;          /* most transient requests in one batch                      */
  int64_t instance_steps;     /* steps times instances of those calls: instance_steps /    */
                              /* batched_steps is the mean batch size over steps           */
  double clock;               /* seconds since the server started                          */
} afc_serve_info;

void afc_serve_default_config(afc_serve_config* c);
/* Device bytes the server reserves for a request while it runs (host only). */
int64_t afc_serve_estimate_bytes(const afc_request* r);
int afc_serve_create(int device, const afc_serve_config* cfg, afc_server* out);
/* Copies the request's arrays; returns at once with its id.  AFC_E_INVALID if the
 * request is malformed or alone exceeds the budget. */
int afc_serve_submit(afc_server s, const afc_request* r, int64_t* id);
/* Current state of a request; if it is done, u_out (n_nodes host doubles, may be
 * NULL) receives the solution. */
int afc_serve_poll(afc_server s, int64_t id, afc_result* res, double* u_out);
/* As poll, after waiting until the request has finished (timeout_s < 0: no
 * limit); AFC_E_TIMEOUT if it has not finished in time. */
int afc_serve_wait(afc_server s, int64_t id, double timeout_s, afc_result* res, double* u_out);
/* Pending requests are dropped; running transient requests leave at the next
 * chunk; a running stationary solve finishes first.  The state becomes CANCELLED. */
int afc_serve_cancel(afc_server s, int64_t id);
/* Forget a finished request (its result). */
int afc_serve_release(afc_server s, int64_t id);
int afc_serve_get_info(afc_server s, afc_serve_info* out);
/* Stops the threads (running solves finish), cancels pending requests, frees all. */
int afc_serve_destroy(afc_server s);

/* ---- diagnostics -------------------------------------------------------------- */

/* Per-kernel device time of the library's launches on this problem.
 * mode != 0 clears earlier records and starts recording; 0 stops.  While on,
 * every launch is bracketed by two events on the problem's stream. */
int afc_profile(afc_problem p, int mode);

/* Recorded totals, one entry per kernel name (at most cap): names[48*k] holds a
 * NUL-terminated name, total_ms[k] the summed device time, launches[k] the
 * count; *n receives the number of entries.  *all_launches (may be NULL)
 * receives the number of kernel launches issued on this problem since its
 * creation, recorded or not.  Synchronises the stream. */
int afc_profile_read(afc_problem p, int cap, char* names, double* total_ms, int64_t* launches, int* n,
                     int64_t* all_launches);

/* Self-test of the bounded grid waits of the persistent kernels (their failure
 * detection, exercised without a fault).  One launch of two blocks on `device`
 * in which block 1 never arrives at a grid barrier, so block 0's wait runs out
 * after limit_ms milliseconds of the device's global timer (0 < limit_ms <=
 * 4000), records the error in the barrier state and returns, as a barrier of a
 * solver launch does after its 4 s limit.  *observed receives the status the
 * host derives from that state (AFC_E_TIMEOUT when the wait ran out, AFC_OK if
 * it did not), *waited_ms (may be NULL) the host-measured duration of the launch.
 * Returns AFC_OK when a launch after the expired wait ran and returned its
 * result (the context stays usable), AFC_E_INVALID for a bad limit or a NULL
 * `observed`, AFC_E_CUDA on a CUDA error.  Allocates and frees 20 bytes of
 * device memory. */
int afc_selftest_grid_wait(int device, double limit_ms, int* observed, double* waited_ms);

/* Self-test of the float-pair arithmetic of the mixed MC sweep (the split of a double
 * into the pair hi = RN(x), lo = RN(x - hi) on the integer pipe, and the exact widening
 * of a float to double): on `device`, for the n doubles of the host array x, writes
 * hi[i], lo[i] and hi_widened[i] = hi[i] as a double (host arrays of n values, owned by
 * the caller).  0 <= n <= 2^26.  Returns AFC_OK, AFC_E_INVALID for a bad n or a NULL
 * array, AFC_E_CUDA on a CUDA error.  Allocates and frees 24 n bytes of device memory. */
int afc_selftest_split(int device, const double* x, int64_t n, float* hi, float* lo, double* hi_widened);

/* Limit of the bounded waits at the grid barriers of this problem's persistent
 * BiCGStab launches (default 4000 ms, the largest allowed; 0 <= limit_ms <= 4000).
 * A wait that reaches it records the error and every later barrier of the launch
 * passes at once, so the launch ends; afc_step / afc_solve_stationary then return
 * AFC_E_TIMEOUT (the solution is not a valid iterate: restore it with
 * afc_set_solution) and clear the barrier state for the next call.  With 0 the
 * first wait that finds a barrier still closed gives up at once, which lets a test
 * take the timeout path without any fault.  Failure detection of the solver
 * (bounded device waits), not part of the method. */
int afc_set_grid_wait_limit(afc_problem p, double limit_ms);

const char* afc_status_str(int status);
const char* afc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AFC_H */
