/*
 * fnpf.h -- C ABI of the GB300 (sm_103a) FNPF-SEM hot path.
 *
 * Method: fully nonlinear potential flow on a free-surface-following mesh,
 * arXiv 2506.09435.  Per explicit RK4 stage (paper Sec. 3.2, Sec. 3.4 Steps
 * 4.1-4.6): move the mesh with eta, solve the Laplace problem for the velocity
 * potential phi with phi = phi_eta on the free surface (Sec. 2, Eq.
 * Laplace_strong; weak form Sec. 3.1.1, Eq. Laplace_weak), recover the
 * vertical surface velocity w, and evaluate the Zakharov free-surface
 * conditions (Sec. 2, Eqs. kinematic/dynamic_free_surface_strong).
 *
 * Discretisation (readings of the paper, which uses P_p prisms):
 *   Q_p GLL tensor-product hexahedra (2D: quadrilaterals in the (x, z) slice)
 *   on an Nx x Ny surface grid extruded into Nz layers; z = -h + sigma (eta + h)
 *   with uniform layers; GLL quadrature at the nodes; lumped GLL surface mass.
 *
 * Data layout ("plane-major"): a volume field has N = Nv * Ns entries,
 * index = k * Ns + col, k = 0 (bottom) .. Nv - 1 = p Nz (free surface),
 * col = iy * ncx + ix (ix fastest), ncx = p Nx (+1 if walled in x),
 * ncy = p Ny (+1 if walled in y; 1 in 2D), Ns = ncx * ncy.  The surface plane is
 * the last Ns entries; the first N_I = (Nv - 1) Ns entries are the unknowns of
 * the Laplace solve.  A surface field has Ns entries in column order.
 *
 * Conventions for every call below:
 *   - double / float pointers to field data are DEVICE pointers owned by the
 *     caller; the library never frees or retains them beyond the call;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); work is
 *     enqueued on it.  A solve keeps its convergence test on the device and
 *     the host reads the flag every check_every iterations, so solve, DtN and
 *     RK4 calls wait for the stream at those points; apply, diagonal and
 *     right-hand-side calls only enqueue;
 *   - no exception crosses the ABI; failures return a status and leave a
 *     message for fnpf_last_error(); FNPF_EINVAL is returned before any
 *     work is enqueued.
 */
#ifndef FNPF_H
#define FNPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FNPF_OK = 0,
  FNPF_EINVAL = 1,        /* bad argument: NULL pointer, size, order, depth   */
  FNPF_ENOMEM = 2,        /* device allocation failed                         */
  FNPF_ECUDA = 3,         /* a CUDA runtime call failed                       */
  FNPF_ENOCONV = 4,       /* iteration cap reached before the tolerance       */
  FNPF_EBREAKDOWN = 5,    /* CG breakdown: p^T A p <= 0 or not finite         */
  FNPF_EDIVERGED = 6,     /* non-finite state, or eta + h <= 0 (mesh folded)  */
  FNPF_EUNSUPPORTED = 7   /* valid but not implemented combination            */
} fnpf_status;

enum { FNPF_BOX = 0, FNPF_ISOPARAMETRIC = 1 };
/* FNPF_FP64: everything in FP64.  FNPF_MIXED: FP64 defect correction around
 * an FP32 PCG with FP32 operator and FP32 p-multigrid.  FNPF_FP64_PC32: FP64
 * PCG (FP64 operator, vectors, dot products) whose p-multigrid preconditioner
 * runs in FP32 on the rounded residual (FNPF_PMG only; with FNPF_JACOBI it is
 * FNPF_FP64). */
enum { FNPF_FP64 = 0, FNPF_MIXED = 1, FNPF_FP64_PC32 = 2 };
enum { FNPF_JACOBI = 0, FNPF_PMG = 1 };
/* Coarsest multigrid level (p = 1): FNPF_COARSE_CLUSTER assembles its 27-point
 * (9-point in 2D) stencil once per solve and runs the whole coarse Chebyshev
 * sweep in one kernel on one thread-block cluster of 8 CTAs (levels of at most
 * 32768 unknowns; larger ones fall back to FNPF_COARSE_LAUNCHES, one operator
 * launch per Chebyshev step).  Both apply the same polynomial. */
enum { FNPF_COARSE_LAUNCHES = 0, FNPF_COARSE_CLUSTER = 1 };
/* Chebyshev smoothers of FNPF_PMG: FNPF_CHEB_FIRST = first-kind Chebyshev
 * acceleration of Jacobi on [lmax/cheb_range, lmax] (Saad, Iterative Methods, Alg.
 * 12.1); FNPF_CHEB_FOURTH = fourth-kind Chebyshev smoother on [0, lmax]
 * (Lottes, Numer. Linear Algebra Appl. 2023).  lmax of D^-1 A is estimated per
 * level on the device. */
enum { FNPF_CHEB_FIRST = 1, FNPF_CHEB_FOURTH = 4 };
/* Free-surface model.  FNPF_NONLINEAR: fully nonlinear potential flow, the
 * mesh follows eta (Sec. 3.1.2) and the Zakharov conditions give the
 * right-hand side (Sec. 2).  FNPF_LINEAR: linear potential flow (the paper's
 * LPF, Sec. 1 and 2): the Laplace problem is solved on the still-water domain
 * (the geometry takes eta = 0 wherever it would take eta) and the surface
 * conditions are d eta/dt = w, d phi/dt = -g eta. */
enum { FNPF_NONLINEAR = 0, FNPF_LINEAR = 1 };
/* Order sequence of the p-multigrid levels: FNPF_MG_HALVE p -> p/2 -> ... -> 1,
 * FNPF_MG_TWO_LEVEL p -> 1, FNPF_MG_STEP2 p -> p-2 -> ... -> 1. */
enum { FNPF_MG_HALVE = 0, FNPF_MG_TWO_LEVEL = 1, FNPF_MG_STEP2 = 2 };

/* Mesh descriptor.  All arrays are HOST pointers, copied at creation. */
typedef struct {
  int dim;                 /* 2: (x, z) vertical slice; 3: (x, y, z)              */
  int nx, ny, nz;          /* elements per direction (ny ignored in 2D), >= 1      */
  int p;                   /* GLL order, 1..8                                      */
  int periodic_x, periodic_y; /* 1: periodic (>= 2 elements that way); 0: walls     */
  int horiz_kind;          /* FNPF_BOX (Lx, Ly) or FNPF_ISOPARAMETRIC (X, Y)        */
  double Lx, Ly;           /* box lengths (FNPF_BOX)                               */
  const double* X;         /* [Ns] surface-node x (FNPF_ISOPARAMETRIC), else NULL  */
  const double* Y;         /* [Ns] surface-node y (FNPF_ISOPARAMETRIC), else NULL  */
  const double* h;         /* [Ns] still-water depth at surface nodes, all > 0     */
  double g;                /* gravitational acceleration (> 0)                     */
} fnpf_mesh_desc;

/* Solver options (fnpf_default_opts fills every field). */
typedef struct {
  int precision;           /* FNPF_FP64, FNPF_MIXED or FNPF_FP64_PC32              */
  int precond;             /* FNPF_JACOBI or FNPF_PMG                              */
  double rtol;             /* stop when ||r||_2 <= max(rtol ||b||_2, atol)         */
  double atol;
  int max_iter;            /* CG iteration cap per solve (ENOCONV beyond)          */
  int check_every;         /* host reads the convergence flag every k iterations  */
  int cheb_degree;         /* degree of the pre- and post-smoothing Chebyshev
                              sweeps on every level but the coarsest (FNPF_PMG)   */
  int coarse_iters;        /* degree of the coarsest level's Chebyshev sweep
                              (FNPF_PMG)                                          */
  double inner_rtol;       /* inner FP32 solve tolerance (FNPF_MIXED)              */
  int max_outer;           /* defect-correction cap (FNPF_MIXED)                   */
  int use_graphs;          /* 1: replay CG iterations as CUDA graphs (not while
                              instrumentation is enabled); 0: plain launches      */
  int store_metric;        /* FP64 operator (of every precision form; in FNPF_MIXED
                              the lift, projection and outer residuals):
                              1 = rebuild the metric G from eta
                              once per solve into device memory (6 doubles per
                              point, allocated at the first solve) and read it in
                              every application; 0 = rebuild it per application */
  int coarse_solver;       /* FNPF_COARSE_CLUSTER or FNPF_COARSE_LAUNCHES (FNPF_PMG) */
  int cheb_kind;           /* FNPF_CHEB_FIRST or FNPF_CHEB_FOURTH (FNPF_PMG)        */
  double cheb_range;       /* FNPF_CHEB_FIRST smooths [lmax / cheb_range, lmax] (> 1) */
  int model;               /* FNPF_NONLINEAR or FNPF_LINEAR                        */
  int mg_schedule;         /* FNPF_MG_HALVE, FNPF_MG_TWO_LEVEL or FNPF_MG_STEP2     */
  int projection;          /* 0..8: initial guess of a Laplace solve = the Galerkin
                              projection of the solution onto the span of the last
                              `projection` solutions of this mesh (and of the
                              caller's guess), in the current operator (Fischer's
                              projection for successive right-hand sides); 0 keeps
                              the caller's guess.  Costs `projection` operator
                              applications and 2 x projection x N_I doubles
                              per mesh (allocated at the first solve); the
                              adjoint solves of fnpf_step_adjoint project onto
                              their own history (as much memory again). */
} fnpf_opts;

typedef struct {
  int iters;               /* CG iterations (inner iterations for FNPF_MIXED)     */
  int outer_iters;         /* defect-correction steps (0 unless FNPF_MIXED)        */
  double rel_res;          /* final ||r|| / ||b|| (FP64 residual)                  */
  int status;              /* fnpf_status of this solve                            */
  float ms;                /* device time of the solve                             */
} fnpf_solve_info;

typedef struct fnpf_mesh fnpf_mesh;

/* Node counts of a descriptor without creating anything (host arithmetic only):
 * n_vol = (p Nz + 1) Ns, n_surf = Ns.  Returns FNPF_EINVAL on a bad descriptor. */
fnpf_status fnpf_count_dofs(const fnpf_mesh_desc* desc, int64_t* n_vol, int64_t* n_surf);

/* Fills *opts with the defaults: FP64, Jacobi, rtol 1e-10, atol 0,
 * max_iter 20000, check_every 16, cheb_degree 3, coarse_iters 6,
 * inner_rtol 1e-5, max_outer 20, use_graphs 1, store_metric 1,
 * coarse_solver FNPF_COARSE_CLUSTER, cheb_kind FNPF_CHEB_FIRST, cheb_range 160,
 * model FNPF_NONLINEAR, mg_schedule FNPF_MG_HALVE, projection 8. */
void fnpf_default_opts(fnpf_opts* opts);

/* Creates a mesh on the current CUDA device: GLL tables, horizontal metric,
 * lumped surface mass, depth, and all solver workspaces (device memory, owned
 * by the mesh).  opts may be NULL (defaults).  Sec. 3.1.2, Sec. 3.4 Step 1.
 * Errors: EINVAL (descriptor), ENOMEM, ECUDA. */
fnpf_status fnpf_create_mesh(const fnpf_mesh_desc* desc, const fnpf_opts* opts, fnpf_mesh** out);
void fnpf_destroy_mesh(fnpf_mesh* mesh);
fnpf_status fnpf_set_opts(fnpf_mesh* mesh, const fnpf_opts* opts);
fnpf_status fnpf_mesh_sizes(const fnpf_mesh* mesh, int64_t* n_vol, int64_t* n_surf);

/* Physical (x, y) of every surface column into HOST arrays [Ns] (y = 0 in 2D;
 * a periodic seam column reports its first copy, x = 0 / y = 0). */
fnpf_status fnpf_surface_coords(const fnpf_mesh* mesh, double* x, double* y);

/* y = A(eta) x: the assembled stiffness matrix of the weak Laplace form
 * (Eq. Laplace_weak, all N rows, no Dirichlet masking) applied to x [N];
 * eta [Ns].  Matrix-free, sum-factorised, geometric factors rebuilt from eta.
 * x and y must not overlap. */
fnpf_status fnpf_apply(fnpf_mesh* mesh, const double* eta, const double* x, double* y, void* stream);

/* The FP32 operator of the FNPF_MIXED inner solves (FP32 tables, geometry and
 * contractions): y = A32(eta) x with eta [Ns], x, y [N] float. */
fnpf_status fnpf_apply_f32(fnpf_mesh* mesh, const float* eta, const float* x, float* y, void* stream);

/* d = diag(A(eta)) [N] (Jacobi preconditioner of the Laplace solve). */
fnpf_status fnpf_diagonal(fnpf_mesh* mesh, const double* eta, double* d, void* stream);

/* z = M r: one application of the FP64 preconditioner of the Laplace solve
 * (the paper preconditions its CG with algebraic multigrid, Sec. 4 solver
 * settings; this is the p-multigrid V-cycle of FNPF_PMG, or the Jacobi
 * preconditioner z = diag(A_II)^-1 r of FNPF_JACOBI) for the geometry of eta
 * [Ns]: the set-up (level geometry, diagonals, Chebyshev intervals from a
 * deterministic Lanczos run) is done from eta on every call.  r, z [N_I] device
 * doubles in the interior layout of the unknowns (planes 0 .. nv-2), not
 * overlapping.  M is a fixed symmetric positive definite operator for a given
 * eta and options.  Ignores opts.precision (always FP64).  Synchronous on
 * `stream` only through stream order.  Errors: EINVAL (NULL), ENOMEM, ECUDA. */
fnpf_status fnpf_precond_apply(fnpf_mesh* mesh, const double* eta, const double* r, double* z, void* stream);

/* Laplace solve (Sec. 3.4 Steps 4.1-4.3): A_II phi_I = -A_IS phi_eta.
 * eta, phis [Ns]; phi [N]: on entry its first N_I entries are the initial
 * guess, on return phi holds the solution with phi = phis on the surface
 * plane.  info may be NULL.  The failure statuses ENOCONV, EBREAKDOWN and
 * EDIVERGED are returned by the call itself. */
fnpf_status fnpf_laplace_solve(fnpf_mesh* mesh, const double* eta, const double* phis, double* phi,
                               fnpf_solve_info* info, void* stream);

/* Dirichlet-to-Neumann map (Steps 4.1-4.5): w = d phi / dz on the surface,
 * w [Ns].  The volume potential is kept inside the mesh and warm-starts the
 * next solve. */
fnpf_status fnpf_dtn(fnpf_mesh* mesh, const double* eta, const double* phis, double* w,
                     fnpf_solve_info* info, void* stream);

/* Zakharov right-hand side (Step 4.6, lumped GLL mass): given eta, phis, w [Ns]
 * returns d eta/dt and d phi_eta/dt [Ns]. */
fnpf_status fnpf_zakharov_rhs(fnpf_mesh* mesh, const double* eta, const double* phis, const double* w,
                              double* deta, double* dphis, void* stream);

/* One classical RK4 step (Sec. 3.2) of the state (eta, phis) [Ns], in place:
 * four DtN solves and right-hand sides, then the relaxation zones (if set)
 * with the targets at time t + dt.  info may be NULL or point to 4 structs
 * (one per stage).  The first call runs host-driven solves; later calls (with
 * use_graphs and instrumentation off) replay one captured CUDA graph per step
 * whose CG loops are conditional WHILE nodes evaluated on the device, and wait
 * for the stream once (re-captured when eta, phis or dt change). */
fnpf_status fnpf_rk4_step(fnpf_mesh* mesh, double* eta, double* phis, double t, double dt,
                          fnpf_solve_info* info, void* stream);

/* Operator application without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as a
 * plug-in inside a host application that owns all device memory through its
 * own pool, or a loop with a fixed, pre-reserved memory budget where an
 * allocation could fail or stall.  Computes y = A(eta) x exactly as
 * fnpf_apply does, for an FNPF_BOX mesh described by desc (host struct; its
 * h, X, Y pointers are ignored) with the depth h [Ns], eta [Ns], x [N] and
 * y [N] given as caller-owned DEVICE arrays.  The lengths are not passed and
 * cannot be checked: the caller guarantees them.  Every h and eta + h must be
 * positive and finite (the vertical Jacobian (eta + h) / (2 Nz) is divided
 * by); unlike fnpf_create_mesh, this call does not check the depth, and a
 * zero or negative value gives inf or NaN in y.
 * The GLL tables, the box metric and the operator's scratch live in one
 * file-scope device array of 16 MiB (2,097,152 doubles) that every GPU
 * loading the library holds until exit; a mesh needs
 * n^2 + 2n + 5 n_ecol L + Nv n_ecol R doubles of it (L = (p+1)^2, R = 4p in
 * 3D; L = p+1, R = 2 in 2D; n_ecol = Nx Ny; each part rounded up to 32), and
 * a larger mesh is rejected with FNPF_EINVAL before any work is enqueued.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (each call rewrites what it reads); calls that overlap on
 * the GPU race on it.  Errors: EINVAL, EUNSUPPORTED (not FNPF_BOX), ECUDA;
 * the message is available from fnpf_last_error(NULL). */
fnpf_status fnpf_apply_noalloc(const fnpf_mesh_desc* desc, const double* h, const double* eta, const double* x,
                               double* y, void* stream);

/* Autotuner: times every elements-per-CTA shape of the FP64 and of the FP32
 * operator kernel on this mesh (eta [Ns]) and keeps the fastest of each (3D:
 * shapes 0-3 run one thread per vertical GLL line, shapes 4-7 the
 * line-decomposed kernel whose contractions use the even-odd symmetry of the
 * GLL derivative matrix, shapes 8-11 one thread per vertical line with two
 * element layers in flight); the
 * chosen shape indices are returned when the pointers are non-NULL.  Runs
 * automatically before the first solve of a mesh; waits for the stream. */
fnpf_status fnpf_autotune(fnpf_mesh* mesh, const double* eta, int* variant64, int* variant32, void* stream);

/* Sets the elements-per-CTA shapes (0..11 in 3D, 0 in 2D; the same indices
 * fnpf_autotune returns) of the FP64 and FP32 operator kernels by hand and
 * marks the mesh as tuned, so that no later solve re-tunes it.  Host-only.
 * Errors: EINVAL (index out of range). */
fnpf_status fnpf_set_shapes(fnpf_mesh* mesh, int variant64, int variant32);

/* The current shape indices and the element columns per CTA they stand for
 * (any pointer may be NULL).  Host-only.  Errors: EINVAL (mesh NULL). */
fnpf_status fnpf_get_shapes(const fnpf_mesh* mesh, int* variant64, int* variant32, int* columns64, int* columns32);

/* Instrumentation (tracing): when enabled, every operator application issued
 * by a solve is bracketed by CUDA events on the solve's stream, and the
 * elapsed device time and count are accumulated.  The launch counter counts
 * every kernel the library enqueues for this mesh, enabled or not.
 * fnpf_profile_read returns the totals and, if reset != 0, clears them. */
fnpf_status fnpf_profile_enable(fnpf_mesh* mesh, int on);
fnpf_status fnpf_profile_read(fnpf_mesh* mesh, double* apply_ms, int64_t* apply_count, int64_t* kernel_launches,
                              int reset);
/* The same totals for the FP32 operator applications of FNPF_MIXED solves
 * (fnpf_profile_read above reports the FP64 ones; its reset clears both). */
fnpf_status fnpf_profile_read_fp32(fnpf_mesh* mesh, double* apply_ms, int64_t* apply_count);

/* Relaxation zones (Sec. 3.3; Step 4.7 of Sec. 3.4): after every RK4 step,
 * f <- (1 - C_r) f + C_r f_true for f in {eta, phi_eta}.  In generation nodes
 * (gen = 1) the target is the linear incident wave
 *   eta_I = a cos(kx x + ky y - omega t + phase),
 *   phi_I = (g a / omega) cosh(k (eta_I + h)) / cosh(k h) sin(kx x + ky y - omega t + phase),
 * k = |(kx, ky)|, h the node's depth, multiplied by the ramp min(1, t / ramp_time)
 * (the paper activates generation over five wave periods); in absorption nodes
 * (gen = 0) the target is 0.  C_r = 0 leaves a node untouched.  cr and gen
 * are HOST arrays [Ns], copied; a NULL cr removes the relaxation. */
typedef struct {
  const double* cr;        /* [Ns] relaxation weight in [0, 1]                  */
  const double* gen;       /* [Ns] 1: generation target, 0: absorption target   */
  double amp, kx, ky, omega, phase;
  double ramp_time;        /* > 0 */
} fnpf_relaxation;
fnpf_status fnpf_set_relaxation(fnpf_mesh* mesh, const fnpf_relaxation* relax);

/* Modal filter of free-surface fields (Sec. 3.2, modal filtering; applied in
 * Step 4.7).  On every surface element the nodal values are mapped to the
 * coefficients of the tensor-product orthonormal Legendre basis (Vandermonde
 * matrix at the GLL nodes), mode (a, b) is scaled by sigma_a sigma_b with
 *   sigma_k = 1 (k <= cutoff),  exp(-alpha ((k - cutoff) / (p - cutoff))^order) (k > cutoff),
 * and the result is mapped back; the element-interior nodes take the filtered
 * values, nodes shared between elements keep theirs.  Once set, every RK4 step
 * filters eta and phi after the relaxation.  alpha = 0 (or a NULL filter)
 * turns it off.  Errors: EINVAL (alpha < 0 or not finite, order < 1,
 * cutoff outside 0..p-1). */
typedef struct {
  double alpha;            /* damping of the highest mode: sigma_p = exp(-alpha) */
  int order;               /* s >= 1 */
  int cutoff;              /* N_c in 0..p-1: modes up to N_c are kept */
} fnpf_filter;
fnpf_status fnpf_set_filter(fnpf_mesh* mesh, const fnpf_filter* filter);

/* Over-integration of the nonlinear free-surface terms (Sec. 3.2, with the
 * modal filter; reading: collocation is replaced on each surface element by
 * an exactly integrated projection).  With points = M > 0, every Zakharov
 * right-hand side of FNPF_NONLINEAR (fnpf_rk4_step stages, fnpf_zakharov_rhs)
 * is evaluated as follows: eta, phi_eta and w are interpolated from the GLL
 * nodes to the M x M (2D: M) Gauss-Legendre points of each surface element,
 * with the horizontal gradients of the interpolants; f_eta and f_phi are
 * evaluated there and replaced by their L2 projection onto the degree-p
 * polynomials of the element's reference coordinates (exact Gauss sums of the
 * Legendre coefficients), evaluated at the GLL nodes; shared nodes combine the
 * element values with the lumped-mass weights w_i w_j |det H|.  Polynomial
 * right-hand sides of degree <= p per direction are unchanged; modes above p
 * are dropped instead of aliased.  Quadratic terms are integrated exactly
 * from M >= (3p + 1) / 2 + 1, cubic ones from M >= 2p + 1 on affine elements.
 * points = 0 turns it off.  Tables and the Gauss-point metric are built on the
 * host and copied (synchronous); the adjoint step returns EUNSUPPORTED while
 * it is on.  Errors: EINVAL (points outside 0 or p+1..17, singular
 * horizontal Jacobian), ENOMEM, ECUDA. */
fnpf_status fnpf_set_dealias(fnpf_mesh* mesh, int points);

/* Applies the filter set by fnpf_set_filter to one surface field f [Ns]
 * (device, in place), on `stream`.  Errors: EINVAL (no filter set). */
fnpf_status fnpf_filter_apply(fnpf_mesh* mesh, double* f, void* stream);

/* Ensembles of independent tanks (batched form; Sec. 3.4's RK4 step, Steps
 * 4.1-4.7, for many tanks at once).  An ensemble groups existing, distinct
 * meshes (not owned; they must outlive it; the same mesh twice is EINVAL).
 * fnpf_ensemble_rk4_step advances tank i by one RK4 step of size dts[i] from
 * time ts[i], state etas[i], phiss[i] (device arrays, in place), exactly as
 * fnpf_rk4_step would.  The first call steps each
 * tank on its own (set-up, autotuning); from the second call on, all tanks'
 * steps run as one launch of a captured CUDA graph with one host
 * synchronisation per ensemble step.  In that graph, tanks whose steps are the
 * same sequence of kernels (same order, dimension and options) form batched
 * groups: every kernel of the step is ONE launch over all tanks of the group
 * (the grids concatenated, each block working on its own tank), every CG or
 * defect-correction loop one device-side loop that runs while any tank's loop
 * runs, a tank whose loop has finished skipping its work; the tanks of an order
 * are given the kernel shapes the autotuner chose for the largest of them
 * (fnpf_set_shapes).  Groups (fnpf_ensemble_set_batching) and the tanks that
 * are not batched (tape on, over-integration) run as concurrent branches.  The graph is
 * re-captured when a state pointer or step size changes.  info may be NULL or
 * point to 4 n structs (tank-major).  Returns the first failing tank's status;
 * fnpf_ensemble_last_error names it. */
typedef struct fnpf_ensemble fnpf_ensemble;
fnpf_status fnpf_ensemble_create(fnpf_mesh* const* meshes, int n, fnpf_ensemble** out);
void fnpf_ensemble_destroy(fnpf_ensemble* ens);
fnpf_status fnpf_ensemble_rk4_step(fnpf_ensemble* ens, double* const* etas, double* const* phiss, const double* ts,
                                   const double* dts, fnpf_solve_info* info, void* stream);
const char* fnpf_ensemble_last_error(const fnpf_ensemble* ens);
/* Batched groups on (1, the default) or off (0: every tank its own branch of
 * per-tank kernels), and the size of a group: at most max_tanks tanks (1..32;
 * 0: 32) and at most max_dof degrees of freedom (<= 0: no limit; a tank larger
 * than the limit runs on its own).  Tanks of a class fill groups in
 * increasing size; a group of one tank runs as its own branch.  Takes effect
 * at the next step.  Errors: EINVAL (max_tanks out of range). */
fnpf_status fnpf_ensemble_set_batching(fnpf_ensemble* ens, int on, int max_tanks, int64_t max_dof);
/* Batched groups and the tanks in them of the current graph, and the kernels
 * the last ensemble step launched (any pointer may be NULL).  Errors: EINVAL. */
fnpf_status fnpf_ensemble_stats(const fnpf_ensemble* ens, int* groups, int* batched_tanks, int64_t* kernels);

/* Adjoint of one RK4 step (reverse mode; the differentiation form built around
 * the paper's method, Sec. 3.2 and Sec. 3.4 Steps 4.1-4.7).  Given the step's
 * input state eta_n, phis_n [Ns] and lam = dJ/d(eta, phis) at the step's output
 * (lam_eta, lam_phis [Ns]), writes dJ/d(eta, phis) at its input into
 * lam_eta_out, lam_phis_out (may alias the inputs) and ADDS dJ/dh into lam_h
 * [Ns] when it is not NULL.  The step is recomputed (four forward solves,
 * storing the stage states and potentials), then each stage costs one adjoint
 * Laplace solve with the same PCG (the operator is symmetric), the
 * vector-Jacobian products of the Zakharov right-hand side and of the
 * vertical-velocity recovery, and the product with the eta- and h-derivative
 * of the operator.  Relaxation zones enter through (1 - C_r).  FP64 only
 * (the mesh's precond, rtol and max_iter apply to every solve).  Waits for the
 * stream at every solve.  Workspace (4 N_I + ~30 Ns doubles) is allocated at
 * the first call. */
fnpf_status fnpf_step_adjoint(fnpf_mesh* mesh, const double* eta_n, const double* phis_n, const double* lam_eta,
                              const double* lam_phis, double* lam_eta_out, double* lam_phis_out, double* lam_h,
                              double t, double dt, void* stream);

/* Conserved quantities of the state (eta, phis) [Ns] (the diagnostics of the
 * paper's conservation checks): mass M = sum_c W_c eta_c and energy
 * E = 1/2 phi^T A(eta) phi + 1/2 g sum_c W_c eta_c^2 (unit density), with W_c
 * the lumped GLL surface mass (Sec. 3.1.1, Eq. free_surface_weak), phi the
 * Laplace solution with phi = phis on the surface (Sec. 2, Eq. Laplace_strong;
 * the mesh's solver and options, into the mesh-owned potential) and A(eta)
 * the stiffness matrix of Eq. Laplace_weak in the geometry of the mesh's
 * model.  Writes the two HOST doubles *mass and *energy; waits for the
 * stream.  An N-double workspace is allocated at the first call.  info may be
 * NULL (the solve's report otherwise).  Errors: EINVAL (NULL), ENOMEM, ECUDA,
 * the solve's ENOCONV / EBREAKDOWN / EDIVERGED. */
fnpf_status fnpf_invariants(fnpf_mesh* mesh, const double* eta, const double* phis, double* mass, double* energy,
                            fnpf_solve_info* info, void* stream);

/* Measurement utility (no counterpart in the paper): enqueues `blocks` CTAs of
 * 256 threads that each run 8 independent FMA chains for iters x 16 steps in
 * FP64 (precision FNPF_FP64) or FP32 (FNPF_MIXED), and reports in *flops (host,
 * may be NULL) the floating-point operations that launch performs (2 per FMA).
 * The caller times the launch on `stream`; flops / time is the FMA pipe's
 * throughput, the denominator of an ALU roofline.  out is a device scratch
 * element of that precision (never written for the inputs used).
 * Errors: EINVAL (blocks or iters < 1, out NULL, other precision), ECUDA. */
fnpf_status fnpf_fma_probe(int precision, int blocks, int iters, void* out, double* flops, void* stream);

/* Vector-Jacobian product of the Laplace solve (the differentiation form
 * around Sec. 3.4 Steps 4.1-4.3): for phi [N] = fnpf_laplace_solve(eta, phis)
 * (passed in: the forward solution, interior and surface plane) and a
 * cotangent gbar [N] of phi, ADDS
 *   lam_phis += gbar_S - A_SI psi,   lam_eta (, lam_h) -= d(psi^T A(eta, h) phi)/d(eta, h),
 * with psi the solution of the adjoint problem A_II psi = gbar_I (the mesh's
 * PCG; A is symmetric).  This is what a user-defined functional of the
 * volume potential (e.g. a force on a structure) needs to be differentiated
 * with respect to the state and the depth.  lam_h may be NULL.  FP64, nonlinear
 * model only (EUNSUPPORTED as fnpf_step_adjoint).  Waits for the stream.
 * Errors: EINVAL (NULL), ENOMEM, ECUDA, the solve's statuses. */
fnpf_status fnpf_laplace_solve_vjp(fnpf_mesh* mesh, const double* eta, const double* phis, const double* phi,
                                   const double* gbar, double* lam_eta, double* lam_phis, double* lam_h,
                                   void* stream);

/* Tape of forward steps for the adjoint (the checkpointed reverse sweep of the
 * differentiation form built around the paper's RK4 step, Sec. 3.2).  After
 * fnpf_tape_begin(mesh, capacity), every successful fnpf_rk4_step records the
 * four stage states and stage potentials of the step into the next slot
 * (0, 1, ...; capacity slots of 4 N_I + 8 Ns doubles, allocated here; a step
 * beyond the capacity fails with EINVAL) until fnpf_tape_end.  Both invalidate
 * the captured step graph once (recording is part of the capture).
 * fnpf_step_adjoint_taped then runs the reverse sweep of fnpf_step_adjoint for
 * the step recorded in `slot` without recomputing its forward solves: the same
 * result up to the solver tolerance, at the cost of the four adjoint solves and
 * the vector-Jacobian products.  The tape holds the slots until the next
 * fnpf_tape_begin.  Errors: EINVAL (NULL, capacity < 1, slot not recorded
 * since the last fnpf_tape_begin), ENOMEM, EUNSUPPORTED (as
 * fnpf_step_adjoint), ECUDA. */
fnpf_status fnpf_tape_begin(fnpf_mesh* mesh, int capacity);
fnpf_status fnpf_tape_end(fnpf_mesh* mesh);
fnpf_status fnpf_step_adjoint_taped(fnpf_mesh* mesh, int slot, const double* lam_eta, const double* lam_phis,
                                    double* lam_eta_out, double* lam_phis_out, double* lam_h, double dt,
                                    void* stream);

/* Prism elements over an unstructured triangular surface mesh (the paper's
 * own mesh, Sec. 3.1.2: a triangular free-surface mesh extruded into N_z
 * layers of prisms whose columns follow the free surface).  Element: degree-p
 * polynomials on the triangle times the degree-p GLL basis in the vertical;
 * triangle nodes of Blyth & Pozrikidis built from the 1D GLL points;
 * straight-sided triangles; z = -h + sigma (eta + h); quadrature: the
 * (p+2)^2-point collapsed Gauss-Legendre rule on the triangle times GLL
 * collocation in the vertical.  Surface numbering: the vertices, then p - 1
 * nodes per edge (edges in order of first appearance over the triangles'
 * edges (A,B), (B,C), (A,C); nodes from the lower to the higher vertex
 * number), then each triangle's interior nodes, local order (i, j) with j
 * outer; volume node (plane k, surface node c) = k * Ns + c.  Walls (zero
 * normal derivative) on the boundary and the bottom.
 *
 * fnpf_prism_numbering (host only): verts [2 nverts] (x, y), tris [3 ntris]
 * (vertex numbers, counter-clockwise), order p (1..8) -> the surface node of
 * every local triangle node tnodes [ntris][(p+1)(p+2)/2], the surface node
 * coordinates x, y [Ns] (any of the three may be NULL) and *ns = Ns.
 * fnpf_prism_tables (host only): values and r, s-derivatives of the nodal
 * basis at the quadrature points L, Lr, Ls [nq][(p+1)(p+2)/2] and weights
 * wq [nq] (any may be NULL), *nq = (p+2)^2.
 * fnpf_prism_create copies the mesh (host arrays) to the device;
 * fnpf_prism_apply computes y = A(eta, h) x (all device arrays: eta, h [Ns],
 * x, y [N], N = (N_z p + 1) Ns; the full operator, surface rows included;
 * eta + h > 0 assumed), deterministic (element results summed per node in a
 * fixed order), asynchronous on stream.  Errors: EINVAL (NULL, sizes, a
 * vertex out of range, a repeated vertex, a triangle of zero or negative
 * area), ENOMEM, ECUDA; the message from fnpf_prism_last_error(mesh or NULL). */
typedef struct fnpf_prism fnpf_prism;
fnpf_status fnpf_prism_numbering(const double* verts, int nverts, const int* tris, int ntris, int p, int* tnodes,
                                 double* x, double* y, int* ns);
fnpf_status fnpf_prism_tables(int p, double* L, double* Lr, double* Ls, double* wq, int* nq);
fnpf_status fnpf_prism_create(const double* verts, int nverts, const int* tris, int ntris, int p, int nz,
                              fnpf_prism** out);
void fnpf_prism_destroy(fnpf_prism* mesh);
fnpf_status fnpf_prism_sizes(const fnpf_prism* mesh, int64_t* n_vol, int64_t* n_surf);
fnpf_status fnpf_prism_apply(fnpf_prism* mesh, const double* eta, const double* h, const double* x, double* y,
                             void* stream);
const char* fnpf_prism_last_error(const fnpf_prism* mesh);

/* The Laplace solve, the Dirichlet-to-Neumann map and the RK4 step on the prism
 * mesh (Sec. 3.1.2 mesh; Sec. 3.4 Steps 4.1-4.6; ERK4, Sec. 3.2).
 *   geometry: G = w |det J| J^-1 J^-T at every quadrature point of every prism
 *     from eta and h (z = -h + sigma (eta + h)), stored once per solve (the
 *     operator of fnpf_prism_apply, Eq. Laplace_weak, with that stored metric);
 *   solve: A_II phi_I = -A_IS phis (Eq. Laplace_strong: phi = phis on the
 *     surface plane, zero normal derivative on the bottom and the walls) by
 *     preconditioned CG to ||r|| <= rtol ||b|| with its scalars on the
 *     device, the host reading the convergence state every iteration
 *     (FNPF_PMG) or every 8 iterations (Jacobi, and the surface-mass solves);
 *   w = d phi / dz at the surface nodes: phi_t / z_t on the top layer's
 *     vertical GLL line (the extrusion is vertical, so every prism sharing the
 *     line gives the same value);
 *   right-hand side: the kinematic and dynamic free-surface conditions (Sec. 2)
 *     f_eta = -grad eta . grad phis + w (1 + |grad eta|^2),
 *     f_phi = -g eta - |grad phis|^2 / 2 + w^2 (1 + |grad eta|^2) / 2
 *     (FNPF_LINEAR: f_eta = w, f_phi = -g eta with the solve and w on the
 *     still-water geometry eta = 0), evaluated at the triangle quadrature
 *     points and projected onto the nodal surface space with the consistent
 *     mass, M k = int f l_i dA (Eq. free_surface_weak; the mass solve by
 *     Jacobi-PCG to mass_rtol on the matrix assembled at the first call);
 *   RK4: the classical four stages and combination, (eta, phis) updated in
 *     place only when all four stages succeed;
 *   FNPF_PMG: the CG preconditioner is one p-multigrid V-cycle over the orders
 *     p, p/2, ..., 1 of the same prisms (rediscretised on the geometry of eta
 *     and h interpolated to each order; the spaces are nested, so prolongation
 *     is exact interpolation and restriction its transpose), first-kind
 *     Chebyshev acceleration of Jacobi on [lmax / cheb_range, lmax] of every
 *     level as smoother (Saad, Iterative Methods, Alg. 12.1; lmax = 1.1 x the
 *     largest Ritz value of 12 Jacobi-PCG steps, per solve and once per
 *     RK4 step), Chebyshev of
 *     degree coarse_iters on the coarsest level: a fixed symmetric positive
 *     definite preconditioner, so plain PCG converges to the same solution.
 * Arrays are DEVICE pointers owned by the caller: eta, h, phis, w, k_eta,
 * k_phis [Ns]; phi, diag, x, y [N] (layout of fnpf_prism_apply: plane-major,
 * surface plane last).  fnpf_prism_laplace_solve reads phi's interior entries
 * as the initial guess and writes the whole of phi (phis on the surface
 * plane).  fnpf_prism_dtn, _rhs and _rk4_step solve into the mesh's own
 * potential, which warm-starts the next solve.  fnpf_prism_diagonal writes the
 * diagonal of A(eta, h) (the Jacobi preconditioner), fnpf_prism_apply_stored
 * y = A(eta, h) x through the stored metric, fnpf_prism_precond_apply z [N] =
 * the preconditioner of opts (Jacobi or one V-cycle) applied to the interior
 * entries of r [N] (z zero on the surface plane).  opts may be NULL (defaults).
 * info: NULL, one struct, or 4 (fnpf_prism_rk4_step, one per stage): iters =
 * Laplace CG iterations (FNPF_MIXED: inner iterations), outer_iters = defect-
 * correction steps (0 unless FNPF_MIXED), rel_res = ||r|| / ||b|| (FP64),
 * status; ms = 0.  The first call on a mesh allocates its workspace (about
 * 28 N + 9 nprisms (p + 1) (p + 2)^2 doubles, the projection basis included;
 * synchronising the device) and builds the surface tables, the first FNPF_PMG
 * call the hierarchy (per level about the same in FP64 and half of it in
 * FP32); later calls allocate nothing.  Calls on one mesh must not overlap;
 * each returns after its stream has finished its work (the CG loops read
 * their state from the device every few iterations).  eta + h > 0 is assumed (not checked).
 * Errors: EINVAL (NULL, non-finite dt, bad options), ENOMEM, ECUDA, ENOCONV
 * (an iteration cap reached), EBREAKDOWN (p.Ap <= 0), EDIVERGED (non-finite
 * residual); the message from fnpf_prism_last_error(mesh). */
typedef struct {
  double rtol;             /* Laplace CG: ||r|| <= rtol ||b|| (default 1e-10)     */
  int max_iter;            /* its iteration cap (default 20000)                   */
  double mass_rtol;        /* surface-mass CG tolerance (default 1e-13)           */
  int mass_max_iter;       /* its cap (default 5000)                              */
  double g;                /* gravitational acceleration (default 9.81)           */
  int model;               /* FNPF_NONLINEAR (default) or FNPF_LINEAR             */
  int precond;             /* FNPF_JACOBI (default) or FNPF_PMG                   */
  int cheb_degree;         /* FNPF_PMG: Chebyshev degree of pre/post smoothing (3) */
  int coarse_iters;        /* FNPF_PMG: Chebyshev degree on the coarsest level (6) */
  double cheb_range;       /* FNPF_PMG: smoothers act on [lmax / range, lmax] (40) */
  int precision;           /* FNPF_FP64 (default); FNPF_FP64_PC32: FP64 PCG with
                              the V-cycle in FP32 (FP32 tables, metric, vectors);
                              FNPF_MIXED: FP64 defect correction around an FP32
                              PCG (FP32 operator and V-cycle, dot products
                              accumulated in FP64) solved to inner_rtol times
                              the current FP64 residual; both FNPF_PMG only
                              (FNPF_FP64 with Jacobi)                         */
  int projection;          /* 0..8: initial guess of a solve = the A-orthogonal
                              projection of the solution onto the span of the
                              last `projection` solutions of this mesh and the
                              caller's guess (Fischer's projection for
                              successive right-hand sides; `projection`
                              operator applications more per solve); 0 (the
                              default) starts from the caller's guess     */
  double inner_rtol;       /* FNPF_MIXED: inner tolerance (default 1e-5)          */
  int max_outer;           /* FNPF_MIXED: defect-correction steps (default 20)    */
} fnpf_prism_opts;
void fnpf_prism_default_opts(fnpf_prism_opts* opts);
fnpf_status fnpf_prism_diagonal(fnpf_prism* mesh, const double* eta, const double* h, double* diag, void* stream);
fnpf_status fnpf_prism_apply_stored(fnpf_prism* mesh, const double* eta, const double* h, const double* x, double* y,
                                    void* stream);
fnpf_status fnpf_prism_precond_apply(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta,
                                     const double* h, const double* r, double* z, void* stream);
fnpf_status fnpf_prism_laplace_solve(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta,
                                     const double* h, const double* phis, double* phi, fnpf_solve_info* info,
                                     void* stream);
/* Vector-Jacobian product of the prism Laplace solve (the differentiation form
 * around Steps 4.1-4.3 of Sec. 3.4): for phi [N] = fnpf_prism_laplace_solve
 * (eta, h, phis) and a cotangent lam_phi = dJ/dphi [N], writes dJ/deta,
 * dJ/dphis and (lam_h non-NULL) dJ/dh [Ns]: one adjoint solve A_II psi =
 * lam_phi,I with the solver of opts (A is symmetric; no projection), then
 * dJ/dphis = lam_phi,S - (A psi)_S and dJ/d(eta, h) = -d(psi^T A(eta, h) phi)
 * /d(eta, h), the metric's derivative at every quadrature point from
 * d J^-1 = -J^-1 dJ J^-1 and d|det J| = |det J| tr(J^-1 dJ) through the
 * vertical row (z_r, z_s, z_t) of J, chained to the nodal eta and h.  phi
 * must be the solution for these eta, h (surface plane = phis).  Device
 * arrays; errors as fnpf_prism_laplace_solve. */
fnpf_status fnpf_prism_laplace_solve_vjp(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta,
                                         const double* h, const double* phi, const double* lam_phi, double* lam_eta,
                                         double* lam_phis, double* lam_h, fnpf_solve_info* info, void* stream);
/* Adjoint of one prism RK4 step (the differentiation form around Sec. 3.2's
 * ERK4 step, Sec. 3.4 Steps 4.1-4.6): for the step from (eta_n, phis_n) [Ns]
 * and the cotangents (lam_eta, lam_phis) = dJ/d(eta, phis)_(n+1), writes
 * dJ/d(eta, phis)_n into (lam_eta_out, lam_phis_out) and, if lam_h is not
 * NULL, dJ/dh [Ns].  The forward stages are recomputed with opts (their
 * states, potentials and w kept in the mesh's workspace), then each stage in
 * reverse: two surface-mass solves for the cotangents of the projected
 * conditions (M is symmetric), the conditions' and w's products at the
 * triangle points and nodes, and fnpf_prism_laplace_solve_vjp's adjoint solve
 * and geometric term; with relaxation zones the blend's product comes first
 * (the cotangents scaled by 1 - C_r, and the target potential's dependence
 * on h into dJ/dh; t is the step's start time), and with a modal filter its
 * transpose before that; errors as fnpf_prism_rk4_step.  Device arrays; the outputs
 * may not alias the inputs. */
fnpf_status fnpf_prism_step_adjoint(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* h,
                                    const double* eta_n, const double* phis_n, const double* lam_eta,
                                    const double* lam_phis, double* lam_eta_out, double* lam_phis_out, double* lam_h,
                                    double t, double dt, void* stream);
fnpf_status fnpf_prism_dtn(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta, const double* h,
                           const double* phis, double* w, fnpf_solve_info* info, void* stream);
fnpf_status fnpf_prism_rhs(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta, const double* h,
                           const double* phis, double* k_eta, double* k_phis, fnpf_solve_info* info, void* stream);
fnpf_status fnpf_prism_rk4_step(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* h, double* eta,
                                double* phis, double t, double dt, fnpf_solve_info* info, void* stream);

/* Mass and energy of a prism state (eta, phis) [Ns] (device): M = int eta dA
 * = 1^T M_s eta with the consistent surface mass M_s, and E = 1/2 phi^T A phi
 * + 1/2 g eta^T M_s eta (unit density), phi the Laplace solution with
 * phi = phis on the surface (into the mesh's potential) and A the stiffness
 * matrix of the model's geometry (eta, or still water for FNPF_LINEAR).
 * Writes the HOST doubles *mass and *energy; waits for the stream.  Errors:
 * EINVAL (NULL, bad options), ENOMEM, ECUDA, the solve's statuses. */
fnpf_status fnpf_prism_invariants(fnpf_prism* mesh, const fnpf_prism_opts* opts, const double* eta, const double* h,
                                  const double* phis, double* mass, double* energy, fnpf_solve_info* info,
                                  void* stream);

/* Relaxation zones on the prism mesh (Sec. 3.3; Step 4.7): after every
 * fnpf_prism_rk4_step from t to t + dt, f <- (1 - C_r) f + C_r f_true at every
 * surface node, the targets of fnpf_set_relaxation (the linear incident wave
 * with the ramp in generation nodes, zero in absorption nodes) at t + dt with
 * the node's depth h; then the modal filter, when set.  cr and gen are HOST
 * arrays [Ns] in the numbering of fnpf_prism_numbering, copied (synchronous);
 * a NULL relax or cr removes the zones.  Errors: EINVAL (cr outside [0, 1],
 * a non-finite gen, ramp_time <= 0, non-finite wave parameters, omega <= 0
 * with generation nodes), ENOMEM, ECUDA. */
fnpf_status fnpf_prism_set_relaxation(fnpf_prism* mesh, const fnpf_relaxation* relax);

/* Modal filter on the prism mesh's triangular surface elements (Sec. 3.2,
 * modal filtering; applied in Step 4.7).  On every triangle the nodal values
 * are mapped to the coefficients of the orthonormal Dubiner basis on the
 * reference triangle (V[r][c] = psi_c(node r)), mode (i, j) is scaled by
 * sigma_(i+j) with the weights of fnpf_filter (by total degree), and mapped
 * back; the triangle-interior nodes (p >= 3) take the filtered values, nodes on
 * edges and vertices keep theirs.  Once set, every fnpf_prism_rk4_step filters
 * eta and phi_eta after the RK4 combination.  alpha = 0 (or NULL) turns it off.
 * fnpf_prism_set_filter builds the matrix on the host and copies it
 * (synchronous); fnpf_prism_filter_apply filters one field f [Ns] (device, in
 * place) on `stream`.  Errors: EINVAL (alpha < 0 or not finite, order < 1,
 * cutoff outside 0..p-1; apply without a filter), ENOMEM, ECUDA. */
fnpf_status fnpf_prism_set_filter(fnpf_prism* mesh, const fnpf_filter* filter);
fnpf_status fnpf_prism_filter_apply(fnpf_prism* mesh, double* f, void* stream);

/* Message of the last failure on this mesh (or of the last create failure
 * when mesh is NULL).  Valid until the next call on the same mesh. */
const char* fnpf_last_error(const fnpf_mesh* mesh);
const char* fnpf_status_string(fnpf_status s);

#ifdef __cplusplus
}
#endif
#endif /* FNPF_H */
