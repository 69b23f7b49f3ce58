/*
 * jfnk.h -- C ABI of the GB300 (sm_103a) Jacobian-free Newton-GMRES solver
 * with the DG->FV subgrid multigrid preconditioner of Birken, Dedner and
 * Kloefkorn, "A Jacobian-free multigrid preconditioner for discontinuous
 * Galerkin methods applied to numerical weather prediction" (arXiv 2505.24504).
 *
 * Conventions shared by every call
 * --------------------------------
 * Unknowns.  A state is the perturbation U' = U - Ubar of the nodal values of
 *   U = (rho, rho u, rho w, rho theta) on the tensor Gauss-Legendre nodes of a
 *   Q_k element (Sec. 2.1; eq. perturbed-euler of Sec. 4).  Ubar is the
 *   environmental atmosphere chosen in jfnk_physics.
 * Layout.  A DG vector holds N = 4 * nx * nz * (k+1)^2 doubles, ordered
 *   [variable][ez][ex][b][a]: variable slowest, then element row ez (z index),
 *   element column ex, node index b along z, node index a along x (fastest).
 *   Nodes within an element ascend in x and z.
 * Memory.  Arguments named *_dev are device pointers (cudaMalloc'd or any
 *   device allocation such as a torch CUDA tensor) owned by the caller; the
 *   library never frees or retains them past the call.  *_host arguments are
 *   host pointers.  The context owns all tables and workspace.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Every
 *   call is ordered on that stream.  Calls that return results to the host
 *   (implicit_step's stats, norms) synchronise the stream before returning.
 * Errors.  0 on success, else a negative JFNK_E* code; jfnk_strerror() names
 *   it.  There is no CPU fallback: without a usable CUDA device, jfnk_create
 *   returns JFNK_ECUDA.
 * Threads.  A context is not thread safe; use one context per host thread.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JFNK_OK 0
#define JFNK_EINVAL (-1)    /* bad argument: k outside [1,4], sizes, NULL, bad mg key */
#define JFNK_ENOMEM (-2)    /* device allocation failed (nothing leaked) */
#define JFNK_ECUDA (-3)     /* a CUDA call failed */
#define JFNK_ENOTCONV (-4)  /* Newton or GMRES hit its iteration cap; state restored */
#define JFNK_ETIMEOUT (-5)  /* the step's time budget (opts.time_budget_ms) ran out; state restored */
#define JFNK_ENAN (-6)      /* a norm became non-finite; state restored */

typedef struct jfnk_ctx jfnk_ctx;

/* Cartesian grid of nx x nz quadrilaterals over [x0,x1] x [z0,z1].
 * Slip walls on all sides unless periodic_x = 1 (then periodic in x, slip
 * walls at bottom and top), as in the test cases of Sec. 4. */
typedef struct {
    int nx, nz;
    double x0, x1, z0, z1;
    int periodic_x;
} jfnk_grid;

/* Model of Sec. 4, eq. (compressible-euler): c_p, c_v [J/(kg K)], gravity g
 * [m/s^2], reference pressure p0 [Pa], kinematic viscosity mu [m^2/s]
 * (mu = 0: Euler).  background 0: isentropic atmosphere theta = theta0,
 * T = theta0 - g z / c_p, p = p0 (T/theta0)^(c_p/R) (Sec. 4.2, 4.3);
 * background 1: uniform state rho = p0/(R theta0), theta = theta0, wind
 * (ubg, wbg) (meant for g = 0); background 2: constant Brunt-Vaisala
 * frequency N_bv with surface temperature theta0 and mean flow ubg (Sec. 4.1):
 * theta = theta0 exp(z/H), T = theta0 (alpha - (alpha-1) exp(z/H)),
 * p = p0 exp(c_p/R (ln(T/theta0) - z/H)), H = g/N^2, alpha = g H/(c_p theta0). */
typedef struct {
    double cp, cv, g, p0, theta0, mu;
    int background;
    double ubg, wbg;
    double N_bv;
} jfnk_physics;

/* Solver options.  Defaults (jfnk_default_opts) follow Sec. 3.1 and Sec. 4:
 * Newton TOL 1e-8 (the paper's runs use 1e-3), Eisenstat-Walker choice 2 with
 * gamma = 0.1, alpha = 1, GMRES restart 30, preconditioner key "mg111111V".
 *  mg_key       "mg a b c d e f G" of Sec. 4: DG pre/post, finest FV
 *               pre/post, intermediate and coarsest FV pre/post smoothing
 *               steps, cycle V or W.  "" disables the preconditioner.
 *  fv_levels    number of FV levels (subgrid first, then agglomeration).
 *  massfix      1: transfer with the mass fix of eq. (transfer-mass-fix).
 *  transfer_l2  1: transfer by L2 projection onto the subcells (subcell averages
 *               of the DG polynomial, mass conservative, no mass fix) and its
 *               inverse, instead of interpolation at the subcell centres.
 *  precond_prec 64: preconditioner in FP64 with finite-difference products
 *               exactly as the paper; 32: preconditioner (DG smoothing,
 *               transfers, all FV levels) in FP32 with exact tangent-linear
 *               products; 16: as 32 with every vector written on the coarsest
 *               FV level (state, iterate, right-hand side) rounded to bfloat16
 *               (the numerics of bf16 storage; arithmetic stays FP32).
 *               The Newton residual, the outer FD Jv, the background
 *               subtraction and GMRES stay FP64 in every mode.
 *  sigma_fv, sigma_dg  pseudo-time CFL factors of the smoothers (Sec. 3.5).
 *  c_ip         interior-penalty constant of the viscous flux.
 *  use_graphs   1 (default): capture one preconditioner application in a CUDA
 *               graph on first use (and again when alpha_dt changes) and replay
 *               it; 0: launch the kernels one by one.  Same results either way.
 *  tile_*, fv_split_cells  launch shapes (results do not depend on them, except
 *               fv_split_cells, which changes the summation order of the FV
 *               operator at rounding level); jfnk_autotune picks them by timing.
 *  precond_fd_eps  numerator c of the step eps = c / |x| of the finite-difference
 *               products inside the FP64 preconditioner (FV levels and DG
 *               smoothing); 0 (default): c = sqrt(eps_mach) as in Sec. 3.1.  A
 *               larger c keeps eps x_i many ulps above the state's rounding, so
 *               that two implementations of Q^-1 can be compared tightly.  The
 *               outer Jacobian-free product of GMRES always uses Sec. 3.1's eps.
 *  time_budget_ms  wall-clock budget of one implicit_step in milliseconds, checked
 *               on the host after every Arnoldi step and Newton iteration; when it
 *               runs out the step returns JFNK_ETIMEOUT with U restored to U^n.
 *               0 (default): no budget. */
typedef struct {
    double newton_tol;
    int newton_max;
    int gmres_restart, gmres_max;
    double ew_gamma, ew_alpha, ew_eta0, ew_eta_max;
    char mg_key[16];
    int fv_levels;
    int massfix;
    int transfer_l2;
    int precond_prec;
    double sigma_fv, sigma_dg, c_ip;
    int use_graphs;
    int tile_faces;      /* threads per block of the DG face kernel: 64, 128, 256 (0: 128) */
    int tile_volume;     /* elements per DG volume block: 1 = ~64 threads, 2 = ~128 (0: 2) */
    int tile_fv;         /* threads per block of the FV cell kernels: 64, 128, 256 (0: 128); the
                            face-once kernel of large levels takes 32 x 8 cells at 256, 32 x 4 else */
    int fv_split_cells;  /* FV levels with fewer cells than this run four lanes per cell (one
                            per face), larger levels the face-once tile kernel (0: 65536) */
    int profile;         /* 1: time the phases of implicit_step with CUDA events (jfnk_stats) */
    double precond_fd_eps;
    double time_budget_ms;
    int dg_fused;        /* FP32 tangent DG products of the preconditioner: 0 or 1 one fused
                            launch per product (faces, volume and epilogue per element strip),
                            2 a face launch and a volume launch */
    int rk_stages;       /* stages s of the pseudo-time smoother (Sec. 3.5), 1..4 (0: 1) */
    double rk_alpha[4];  /* its low-storage coefficients: one smoothing step is
                            w_k = w_0 + rk_alpha[k-1] dtau (b - g'w_{k-1}), k = 1..s; the
                            default s = 1, rk_alpha[0] = 1 is the paper's explicit Euler;
                            e.g. s = 4, (1/4, 1/3, 1/2, 1) is Jameson, Schmidt and Turkel's
                            four-stage scheme (AIAA 81-1259, 1981) */
} jfnk_opts;

/* Counters of one implicit_step (Sec. 4.2 counts linear iterations and
 * operator calls). */
typedef struct {
    int status;          /* JFNK_OK or the error of the step */
    int stages;
    int newton_its;      /* summed over stages */
    int gmres_its;       /* summed over Newton iterations */
    int dg_calls;        /* DG operator evaluations (residuals and products) */
    int fv_calls;        /* FV operator evaluations on all levels */
    double res0;         /* |G(U^0)| of the last stage */
    double res_final;    /* |G| at exit of the last stage */
    /* device time by phase (ms), filled when opts.profile = 1, else 0:
     * preconditioner applications, FD products, Gram-Schmidt + norms,
     * Newton residuals + linearisations */
    double t_precond_ms, t_jv_ms, t_orth_ms, t_newton_ms;
    int reorth;          /* Arnoldi steps that needed the second Gram-Schmidt pass */
} jfnk_stats;

void jfnk_default_opts(jfnk_opts *opts);

/* Create a context for one grid / order / model.  opts may be NULL
 * (defaults).  Allocates tables, background, Krylov basis (restart+1 DG
 * vectors in FP64 plus restart preconditioned vectors), FV levels and
 * reduction scratch on the current CUDA device.  Returns JFNK_EINVAL for
 * k outside [1,4], nx or nz < 1, non-positive extents or a bad key. */
int jfnk_create(const jfnk_grid *grid, int k, const jfnk_physics *phys,
                const jfnk_opts *opts, jfnk_ctx **out);
void jfnk_destroy(jfnk_ctx *ctx);

/* N = 4 nx nz (k+1)^2. */
size_t jfnk_num_unknowns(const jfnk_ctx *ctx);

/* Device bytes jfnk_create would allocate for these arguments (HBM
 * admission); 0 on invalid arguments. */
size_t jfnk_workspace_bytes(const jfnk_grid *grid, int k, const jfnk_opts *opts);

/* Node coordinates in the DG layout without the variable index:
 * nx nz (k+1)^2 doubles each, written to host memory. */
int jfnk_node_coords(const jfnk_ctx *ctx, double *x_host, double *z_host);

/* Initial perturbation state from a potential-temperature perturbation theta'
 * given at the nodes (nx nz (k+1)^2 doubles, device), by the pressure-
 * preserving insertion of eq. (add-perturbation): p and v of the background
 * are kept, theta = theta~ + theta', rho = p0^(R/c_p) p~^(1/gamma) / (R theta).
 * Writes U' = U - Ubar (N doubles, device).  Nodal interpolation equals the
 * L2 projection of Sec. 2.2 under the collocated GL quadrature. */
int jfnk_init_state(jfnk_ctx *ctx, const double *theta_pert_dev, double *U_dev, void *stream);

/* f = M^-1 L_h(U') (eq. convDiscr with eqs. elementint and surfaceint, in the
 * well-balanced perturbation form of Sec. 4): HLLC convective flux, symmetric
 * interior-penalty viscous flux, gravity source -g rho', slip walls by a
 * mirrored ghost state.  U' and f are N doubles on the device; they must not
 * overlap.  U' = 0 gives f = 0 exactly. */
int dg_residual(jfnk_ctx *ctx, const double *U_dev, double *f_dev, void *stream);

/* Jacobian-free product of Sec. 3.1 for G(U) = U - alpha_dt f(U) - Ubar_s:
 *   G'(U) y ~ y - alpha_dt (f(U + eps y) - f(U)) / eps,
 * eps = sqrt(eps_mach)/|y|_2 (eps_mach = 2^-52) when eps <= 0, else the given
 * eps.  fU_dev = f(U) may be NULL (then computed here).  y = 0 gives Jy = 0.
 * All vectors are N doubles on the device; Jy must not alias U, fU or y. */
int jv_product(jfnk_ctx *ctx, const double *U_dev, const double *fU_dev, const double *y_dev,
               double alpha_dt, double eps, double *Jy_dev, void *stream);

/* z = Q^-1 r with Q^-1 = T^-1 q^-1 T (eq. preconditioner): DG pre-smoothing,
 * transfer of the DG residual to the FV subgrid with mass fix
 * (eq. transfer-mass-fix), one FV multigrid cycle from zero linearised at
 * T U' (Sec. 3.4), transfer back, DG post-smoothing; smoothing by explicit
 * Euler pseudo-time steps (Sec. 3.5).  U', r, z are N doubles on the device;
 * z must not alias U or r. */
int mg_precondition(jfnk_ctx *ctx, const double *U_dev, double alpha_dt, const double *r_dev,
                    double *z_dev, void *stream);

/* One implicit step U^n -> U^{n+1} in place (U' on the device):
 * scheme 0 backward Euler, 1 SDIRK2 of Ellsiepen (Sec. 2.2, alpha = 1 -
 * sqrt(2)/2).  Each stage solves eq. (newton) by inexact Newton from
 * U_s^0 = Ubar_s with right-preconditioned flexible GMRES and Eisenstat-
 * Walker tolerances (Sec. 3.1).  On JFNK_ENOTCONV, JFNK_ENAN or JFNK_ETIMEOUT
 * the state is restored to U^n.  stats may be NULL.  Synchronises the stream. */
int implicit_step(jfnk_ctx *ctx, double *U_dev, double dt, int scheme, jfnk_stats *stats,
                  void *stream);

/* Euclidean norm |x|_2 of n doubles (device) written to *out_dev (device):
 * the unweighted l2 norm of Sec. 3.1 (Newton stop test |G(U^k)| < TOL |G(U^0)|
 * and eps = sqrt(eps_mach)/|y|).  Deterministic: per-block partial sums in the
 * context's scratch, then one fixed-order final sum.  n = 0 gives 0. */
int jfnk_norm2(jfnk_ctx *ctx, const double *x_dev, size_t n, double *out_dev, void *stream);

/* The norm of jfnk_norm2 without a context and without allocating anything,
 * for callers that must not allocate device memory: code running while a CUDA
 * graph is being captured, allocator or memory-pool callbacks, and services
 * with a device-memory budget fixed at start-up (these cannot create a
 * context either, since jfnk_create allocates).  The paper has no counterpart.
 * x: n doubles (device); *out_dev (device) receives |x|_2.
 * Scratch: a fixed 4096-double device array inside the library (32 KiB on
 * every GPU that loads it, held until the process exits), so
 * n <= JFNK_NORM2_NOALLOC_MAX_N = 4096 * 8192 = 33,554,432; larger n returns
 * JFNK_EINVAL before anything is launched.
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current): make that first call before
 * capturing a stream.  The address stays cached for the life of the process,
 * so a device that is reset (cudaDeviceReset) afterwards must not be given to
 * this call again in that process.  Every call uses the same array, so calls that overlap on
 * the GPU (on different streams, or from several host threads) race; order
 * them on one stream.  Each call overwrites every partial it later reads, so
 * nothing needs clearing between calls. */
#define JFNK_NORM2_NOALLOC_MAX_N ((size_t)4096 * 8192)
int jfnk_norm2_noalloc(const double *x_dev, size_t n, double *out_dev, void *stream);

/* ---- batched ensembles ------------------------------------------------ */

/* A batch of n member contexts (any grids, orders, models and options; each
 * context belongs to at most one batch at a time).  The batch owns one CUDA
 * stream per member and a pool of min(max_threads, n) host threads
 * (max_threads <= 0: min(n, 16)).  The contexts stay owned by the caller. */
typedef struct jfnk_batch jfnk_batch;
int jfnk_batch_create(jfnk_ctx *const *ctxs, int n, int max_threads, jfnk_batch **out);
void jfnk_batch_destroy(jfnk_batch *batch);

/* One implicit step of every member: U[i] (device, in/out) of member i with
 * step dt[i] and scheme[i] (0 BE, 1 SDIRK2).  Members run concurrently on
 * their own streams, largest first; each member's result is bit-identical to
 * implicit_step on that member alone.  status[i] / stats[i] (may be NULL)
 * receive each member's outcome; returns JFNK_OK or the first member error.
 * Returns when every member has finished. */
int jfnk_batch_step(jfnk_batch *batch, double *const *U_dev, const double *dt, const int *scheme,
                    int *status, jfnk_stats *stats);

/* How jfnk_batch_step runs the members (the result of every member is the same
 * in both, bit for bit):
 *  JFNK_BATCH_STREAMS (default): concurrently on their own streams from the host
 *    thread pool, each member with its own launches and graphs.
 *  JFNK_BATCH_LOCKSTEP: members of the same order k form a class.  One host
 *    thread per member runs the member's solver with its kernel launches and
 *    stream operations recorded; whenever every unfinished member of a class waits
 *    for a value from the device (a norm, a Hessenberg column), the recorded work
 *    of the class is replayed on the stream of its first member, and members whose
 *    next launch is the same operator kernel (same precision and mode, same block
 *    shape) share ONE launch whose blocks are dealt out to them.  The classes run
 *    concurrently.  No graphs in this mode.  Needs 64 MiB of device memory and
 *    64 MiB of pinned host memory for the replay's argument tables (JFNK_ENOMEM if
 *    they cannot be had; the mode is then unchanged).
 * JFNK_EINVAL for another mode or a null batch. */
#define JFNK_BATCH_STREAMS 0
#define JFNK_BATCH_LOCKSTEP 1
#define JFNK_BATCH_LOCKSTEP_UNGROUPED 2   /* lock-step rounds, every launch replayed alone (for comparison) */
int jfnk_batch_set_mode(jfnk_batch *batch, int mode);

/* Launch counts of the last lock-step jfnk_batch_step: kernel launches issued,
 * how many of them were grouped over two or more members, the launches the
 * members would have issued alone (all summed over the classes), and the replay
 * rounds (synchronisation points) of the class with the most.  Any pointer may be
 * NULL.  JFNK_EINVAL for a null batch. */
int jfnk_batch_last_launches(const jfnk_batch *batch, unsigned long long *launches, unsigned long long *grouped,
                             unsigned long long *member_launches, unsigned long long *rounds);

/* Host wall-clock milliseconds of the last lock-step jfnk_batch_step, summed
 * over the rounds of a class (the largest over the classes): ms3[0] waiting for
 * the members to reach their next synchronisation point (host solver work and
 * recording), ms3[1] issuing the replay, ms3[2] waiting for the device to finish
 * it.  JFNK_EINVAL for null arguments. */
int jfnk_batch_last_times(const jfnk_batch *batch, double *ms3);

/* f_m = M^-1 L_h(U'_m) (the residual of dg_residual, Sec. 2.1 and Sec. 4) for every
 * member m at once, on `stream`: members are grouped by (order k, viscous or
 * not), and each group takes ONE face launch and ONE volume launch whose blocks
 * are dealt out to the members in turn (a member's blocks see that member's
 * grid, order, physics and buffers).  U_dev[m], f_dev[m]: device arrays of
 * member m's jfnk_num_unknowns doubles in its layout, U_dev[m] != f_dev[m]
 * (host arrays of n device pointers).  Results are bit-identical to
 * dg_residual on each member.  Uses the members' face scratch, so no member may
 * run other work concurrently.  JFNK_EINVAL for null or aliased arguments. */
int jfnk_batch_dg_residual(jfnk_batch *batch, const double *const *U_dev, double *const *f_dev, void *stream);

/* ---- diagnostics (pieces of mg_precondition, for parity tests) -------- */

/* Number of FV levels and the size of level l (0 = finest subgrid). */
int jfnk_fv_levels(const jfnk_ctx *ctx);
int jfnk_fv_level_size(const jfnk_ctx *ctx, int level, int *NX, int *NZ);

/* v = T^mf u (DG -> finest FV, layout [variable][J][I], J = ez(k+1)+j,
 * I = ex(k+1)+i; 4 NX NZ doubles).  Mass fix if the context's massfix = 1. */
int jfnk_transfer_to_fv(jfnk_ctx *ctx, const double *u_dev, double *v_dev, void *stream);

/* u = T^-1 v (finest FV -> DG) with the mass fix applied back. */
int jfnk_transfer_to_dg(jfnk_ctx *ctx, const double *v_dev, double *u_dev, void *stream);

/* f = f_low(u') on FV level l (k = 0 scheme in perturbation form, FP64). */
int jfnk_fv_residual(jfnk_ctx *ctx, int level, const double *u_dev, double *f_dev, void *stream);

/* p = p0 (R E / p0)^gamma for n values E = rho theta (device arrays): the EOS
 * every kernel evaluates, with the table-driven power.  Exposed so that its
 * accuracy can be checked against CUDA's pow. */
int jfnk_eos_pressure(jfnk_ctx *ctx, const double *E_dev, size_t n, double *p_dev, void *stream);

/* out = y - alpha_dt J(U) y, the FP32 DG product of the preconditioner's
 * smoothing steps (Sec. 3.5) at state U' (contexts with precond_prec < 64):
 * tangent-linear FP32 fluxes in the launch form dg_fused selects, widened to
 * FP64.
 * U, y, out: device arrays of N doubles in the state layout.  J is the
 * derivative of f = M^-1 L_h (eq. convDiscr) at U along y.  Overwrites the
 * preconditioner's FP32 linearisation and workspace (the next implicit_step
 * or mg_precondition linearises again).  Errors: JFNK_EINVAL for a null
 * pointer or an FP64-preconditioner context. */
int jfnk_tangent_product(jfnk_ctx *ctx, const double *U_dev, const double *y_dev, double alpha_dt,
                         double *out_dev, void *stream);

/* Times the two kernels of one DG operator evaluation with CUDA events
 * recorded on `stream` around each launch: which 0 = FP64 residual,
 * 1 = FP64 finite-difference product with direction y (in the form the
 * solver's Arnoldi steps use: face traces of U stored by the residual at U,
 * plus eps times the traces of y), 2 = FP32 tangent product (contexts with
 * precond_prec < 64).  Runs `reps` evaluations;
 * ms[0], ms[1] receive the mean duration of the face and the volume kernel.
 * which 3 (FP32 contexts with a preconditioner): the finest FV level's two
 * FP32 kernels linearised at U with alpha dt = 1 and x = b = y, ms[0] one
 * pseudo-time smoothing step, ms[1] the defect fused with the restriction;
 * which 4: the three Gram-Schmidt launches against 8 basis vectors (y unused),
 * ms[0] the FP32 first pass, ms[1] the second and third passes.  Modes 3 and 4
 * overwrite the context's preconditioner and Krylov workspace. */
int jfnk_time_operator(jfnk_ctx *ctx, int which, const double *U_dev, const double *y_dev, int reps,
                       double *ms_host, void *stream);

/* Autotuner of the launch shapes: times every (tile_faces, tile_volume)
 * pair on `reps` FP64 FD products at state U with direction y (CUDA events on
 * `stream`), and every (tile_fv, fv_split_cells) pair on `reps` preconditioner
 * applications linearised at U (contexts with a preconditioner), keeps the
 * fastest in the context and writes them to best[0..3] = tile_faces,
 * tile_volume, tile_fv, fv_split_cells (host) and their times in ms to
 * ms[0..1] (host; ms[1] = 0 without a preconditioner).  Results of every
 * call are independent of the shapes; only speed changes. */
int jfnk_autotune(jfnk_ctx *ctx, const double *U_dev, const double *y_dev, int reps, int *best_host,
                  double *ms_host, void *stream);

/* Number of kernels this library has launched in this process. */
unsigned long long jfnk_launch_count(void);

const char *jfnk_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* JFNK_H */
