/*
 * dg.h - C ABI of a GB300 (sm_103a) implementation of the implicit
 * spectral/hp discontinuous Galerkin compressible Navier-Stokes solver hot
 * path: the DG residual, the Jacobian-free Newton-Krylov product, restarted
 * GMRES, the block relaxed Jacobi (BRJ) preconditioner, Newton and SDIRK
 * time stepping (arXiv 2002.04222, Sec. 3-4).
 *
 * Conventions for every entry point
 *  - Vectors are caller-owned DEVICE buffers of doubles in the layout
 *    u[e][v][m]: element e (0..n_elem-1), conservative variable
 *    v = (rho, rho u_1..rho u_d, E) (n_var = dim+2), modal coefficient m of the
 *    tensor-product modified basis (n_mode = (P+1)^dim, first direction
 *    fastest; 1-D mode 0 = (1-x)/2, mode P = (1+x)/2, 0<p<P the bubble
 *    (1-x)(1+x)/4 P_{p-1}^{(1,1)}(x)).  Length n_dof = n_elem*n_var*n_mode.
 *  - Descriptors (dg_mesh_desc, dg_physics, configs) are HOST memory and are
 *    copied; the library never frees caller memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    stream-ordered; dg_gmres and sdirk_step synchronise the stream before
 *    returning (their statistics are host values).
 *  - Errors: a dg_status is returned, nothing is thrown across the ABI.
 *    DG_ERR_ARG for invalid arguments, DG_ERR_UNSUPPORTED for a
 *    (dim, P, Q) or feature the compiled library does not provide, DG_ERR_CUDA for a
 *    CUDA failure (sticky errors included), DG_ERR_OOM when device memory
 *    runs out, DG_ERR_NONFINITE when a norm is not finite,
 *    DG_ERR_NOT_CONVERGED when an iteration cap is hit (stats are filled and
 *    the output holds the last iterate).
 *  - Handles are not thread-safe; one handle may be used by one host thread
 *    at a time.  All work of one handle must be on one stream at a time.
 */
#ifndef DG_JFNK_H
#define DG_JFNK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,
  DG_ERR_CUDA = -2,
  DG_ERR_OOM = -3,
  DG_ERR_NONFINITE = -4,
  DG_ERR_NOT_CONVERGED = -5,
  DG_ERR_UNSUPPORTED = -6,
  DG_ERR_TIMEOUT = -7
} dg_status;

typedef struct dg_mesh_s* dg_mesh_t;       /* geometry, tables, workspaces */
typedef struct dg_precond_s* dg_precond_t; /* BRJ blocks + trace Jacobians */

/* Mesh of quadrilaterals (dim 2) or hexahedra (dim 3), Sec. 3.1.
 * nodes[e][a][x]: geometry nodes of element e, a = tensor index of the
 *   (geom_order+1)^dim equispaced reference nodes (first direction fastest).
 *   geom_order = 1 (straight-sided) or 2 (quadratic: 9 / 27 nodes).  Meshes
 *   whose elements are all axis-aligned boxes take kernels with a diagonal
 *   metric and the tensor-product inverse mass matrix; any other mesh
 *   (curved, rotated or sheared elements) takes the general-geometry kernels:
 *   per-point metrics d xi/d x and w|J| at the volume and face points,
 *   owner-side unit normals and surface weights by Nanson's formula, and a
 *   dense inverse element mass matrix (Sec. 3.1: M = B^T Lambda(wJ) B), all
 *   computed once on the device; (dim, P, Q) without general-geometry kernels
 *   and elements with non-positive |J| give DG_ERR_UNSUPPORTED / DG_ERR_ARG.
 * faces[f][6] = (eL, fL, eR, fR, orient, bc): local face 2r is xi_r = -1,
 *   2r+1 is xi_r = +1; interior and periodic faces have eR >= 0 and bc = -1,
 *   physical boundary faces eR = fR = -1 and bc = index into dg_physics.bc.
 *   orient must be 0 (face points of both sides coincide in order).
 * Q: Gauss-Legendre points per direction (volume and faces). */
typedef struct {
  int dim, P, Q, n_elem, geom_order, n_faces;
  const double* nodes;  /* host, n_elem*(geom_order+1)^dim*dim */
  const int32_t* faces; /* host, n_faces*6 */
} dg_mesh_desc;

/* Numerical advection fluxes (Sec. 4.3 lists them among the solvers'
 * options): Roe without entropy fix; HLLC and HLL with Einfeldt
 * (Roe-averaged) wave-speed estimates; local Lax-Friedrichs (Rusanov,
 * penalty = the larger |u_n| + c of the two sides); AUSM of Liou and Steffen
 * with the van Leer Mach-number and pressure splittings. */
enum { DG_RIEMANN_ROE = 0, DG_RIEMANN_HLLC = 1, DG_RIEMANN_HLL = 2, DG_RIEMANN_LF = 3,
       DG_RIEMANN_AUSM = 4 };
enum { DG_BC_DIRICHLET = 1, DG_BC_ISO_WALL = 2, DG_BC_ADIA_WALL = 3, DG_BC_FARFIELD = 4 };
enum { DG_FIELD_UNIFORM = 0, DG_FIELD_VORTEX = 1, DG_FIELD_POISEUILLE = 2, DG_FIELD_TGV = 3,
       DG_FIELD_CYLINDER = 4, DG_FIELD_SHOCK = 5 };
enum { DG_FORCING_NONE = 0, DG_FORCING_POISEUILLE = 1 };

/* Physical model, Sec. 2.1: p = rho T / (gamma Ma^2), constant mu = 1/Re
 * (mu_law 0) or Sutherland's law with T_inf_K kelvin (mu_law 1), heat flux
 * -mu/(Ma^2 Pr (gamma-1)) grad T.  viscous = 0 gives the Euler equations.
 * field / fpar select the analytic field used by dg_project, by Dirichlet
 * and far-field boundaries and by the wall temperature (vortex: u0, v0, phi,
 * xc, yc, scale; Poiseuille: theta, L, dp/dx; uniform: rho, u, v, w, T, or
 * the stream (1, 1, 0, 0, 1) when fpar[0] = 0; cylinder: that stream,
 * brought to rest at the wall radius fpar[0] by the factor
 * 1 - exp(-(r - fpar[0]) / fpar[1]) when fpar[1] > 0; shock: an oblique
 * shock at fpar[0] degrees to the x axis meeting y = 0 at x = fpar[1], the
 * stream (1, 0) at T = 1 below the line and the Rankine-Hugoniot state
 * behind it above).
 * bc[i] is the type of boundary i:
 *   DG_BC_DIRICHLET  exterior and viscous state = the analytic field
 *   DG_BC_ISO_WALL   no-slip wall at the analytic wall temperature
 *   DG_BC_ADIA_WALL  no-slip adiabatic wall: Riemann flux against the
 *                    interior state with reversed normal momentum, viscous
 *                    state (rho_L, 0, p_L/(gamma-1)), zero energy component
 *                    of the viscous normal flux and of S_j
 *   DG_BC_FARFIELD   characteristic state from the Riemann invariants
 *                    u_n +- 2c/(gamma-1) (outgoing from the interior,
 *                    incoming from the analytic field), entropy and
 *                    tangential velocity from the upwind side
 * (Sec. 4.3 lists the adiabatic no-slip wall and the Riemann-invariant far
 * field without formulas, Sec. 6.4 applies the latter on the outer boundary
 * of the cylinder; these are the textbook one-dimensional characteristic and
 * reflection forms.) */
typedef struct {
  double gamma, Pr, Ma, Re, T_inf_K, beta_s;
  int viscous, mu_law, riemann /* DG_RIEMANN_* */, forcing, field;
  double fpar[8];
  int n_bc;
  int bc[8];
  /* Shock capturing by artificial viscosity (Sec. 3.1.2; av = 1, viscous
   * only).  Per element, the modal sensor of the density
   *   s_e = log10(|rho - Pi rho|^2 / |rho|^2),
   * Pi the L2 projection onto degree <= P-1 in each reference direction and
   * both norms on the reference element, gives S_e = 0 below s0 - av_kappa,
   * 1 above s0 + av_kappa and (1 + sin(pi (s_e - s0) / (2 av_kappa))) / 2
   * between, s0 = log10(1/P^4).  The viscosity mu + mu_av and conductivity
   * (mu + mu_av) C_p / Pr use mu_av = av_mu0 S_e (h_e / P) rho (c + |u|) at
   * each volume point, h_e = |element|^(1/dim); on a face the mean of the
   * two sides' values from their traces (the interior side's on a boundary).
   * The residual recomputes S_e from its argument on every call; the BRJ
   * preconditioner holds mu_av at its linearisation state.  av = 2 also
   * multiplies mu_av at each point by Ducros' sensor
   * (div u)^2 / ((div u)^2 + |curl u|^2 + 1e-6) of the point's velocity
   * gradient (on a face: the face-average gradient at the mean trace state,
   * the interior trace on a boundary), which keeps the viscosity out of
   * vortical regions; dg_precond_build refuses full_jacobian with it.  av = 0
   * leaves the model unchanged. */
  int av;
  double av_mu0, av_kappa;
} dg_physics;

typedef struct {
  int dim, P, Q, n_elem, n_var, n_mode, n_quad, n_faces;
  long long n_dof;
} dg_mesh_info_t;

/* Create a mesh handle: uploads geometry and connectivity, builds the 1-D
 * tables, element metrics and the forcing vector on `stream`.  *out owns all
 * device workspaces of the residual; free it with dg_mesh_destroy. */
dg_status dg_mesh_create(const dg_mesh_desc* mesh, const dg_physics* phys, void* stream,
                         dg_mesh_t* out);
dg_status dg_mesh_destroy(dg_mesh_t m);
dg_status dg_mesh_info(dg_mesh_t m, dg_mesh_info_t* info);

/* Autotuning of the sum-factorisation kernels (no counterpart in the paper,
 * whose kernels ran on CPUs): dg_autotune times every launch shape (elements
 * per CTA, threads per CTA) of the volume and lift kernels that fits one CTA's
 * shared memory, reps launches each, on the projected analytic field, and keeps
 * the fastest for this mesh; result receives the choice and its times (ms per
 * launch; *_default: the shape in effect before the call, the built-in one on
 * a fresh mesh, timed also when it is not a candidate).  dg_set_tune applies a shape taken
 * from a stored tuning table (DG_ERR_ARG if it is not a candidate for this
 * (dim, P, Q)).  Results do not depend on the shape. */
typedef struct {
  int vol_epb, vol_threads, lift_epb, lift_threads;
  double vol_ms, lift_ms, vol_ms_default, lift_ms_default;
} dg_tune_result;
dg_status dg_autotune(dg_mesh_t m, int reps, dg_tune_result* result, void* stream);
dg_status dg_set_tune(dg_mesh_t m, const dg_tune_result* t);

/* u = L2 projection of the workload's analytic field at time t (Sec. 3.1,
 * Eq. coeff: M u = B^T Lambda(wJ) U(x_q)). */
dg_status dg_project(dg_mesh_t m, double t, double* u, void* stream);

/* r = R(u, t) = M^-1 L(u, t), the right-hand side of M du/dt = L
 * (Sec. 3.1, Eq. matrix-form-equations; Sec. 3.2, Eq. ode).  u and r must
 * not alias. */
dg_status dg_residual(dg_mesh_t m, const double* u, double t, double* r, void* stream);

/* Shock capturing (Sec. 3.1.2): fac[e] = av_mu0 S_e h_e / P for every
 * element at the state u (device, [n_elem]), the factor that multiplies
 * rho (c + |u|) in the artificial viscosity; S_e = fac[e] P / (av_mu0 h_e) is
 * the modal sensor.  The same kernel runs at the start of every residual
 * evaluation.  DG_ERR_UNSUPPORTED when the mesh was created with av = 0. */
dg_status dg_av_factor(dg_mesh_t m, const double* u, double* fac, void* stream);

/* Jacobian-free product (Sec. 4.2.2, Eq. Jacobian-free-matrix, eps-JF):
 *   out = alpha*v + beta*(R(u + eps v, t) - r_u)/eps,
 *   eps = sqrt(2^-52) * ||u||_2 / ||v||_2  (sqrt(2^-52)/||v|| if u = 0),
 * where r_u = R(u, t) was computed by the caller.  Newton use:
 * alpha = 1, beta = -dt*a_mm gives dN/du . v; alpha = 0, beta = 1 gives
 * dR/du . v.  If v = 0, out = 0.  out must not alias u, r_u or v. */
dg_status dg_jvp(dg_mesh_t m, const double* u, const double* r_u, double t, const double* v,
                 double alpha, double beta, double* out, void* stream);

enum { DG_PREC_FP64 = 0, DG_PREC_FP32 = 1, DG_PREC_BF16 = 2 };
/* BRJ(J) settings (Sec. 4.2.2, Eq. precond-Jacobi): J sweeps (>= 1),
 * relaxation omega, storage/arithmetic precision of the blocks.  graphs != 0
 * replays the 2J-1 launches of one apply as a CUDA graph, captured once per
 * (q, out) pointer pair on the handle's own stream and fenced to the caller's
 * stream with events (same arithmetic, fewer launches from the host); the
 * graphs are dropped on every rebuild and bypassed while dg_profile_enable is
 * on.  An apply with graphs on must not itself run inside a stream capture. */
typedef struct {
  int J;
  int precision;
  double omega;
  int graphs;
  int tc_invert; /* FP32 / BF16 modes: run the rank-32 trailing updates of the
                    block inversion on the tensor cores (TF32 head + tail
                    products, FP32 accumulation; same result to FP32 rounding;
                    slower than the default SIMT kernel at P = 3, 4) */
  int fused;     /* != 0: each sweep after the first as one kernel that forms
                    q - (L+U) q^(j-1) of an element in shared memory and
                    multiplies it by the element's block in the same launch
                    (J-1 fewer launches and no HBM round trip of the sweep's
                    right-hand side; bitwise the same result; one more
                    n_dof-vector of device memory) */
  int full_jacobian; /* != 0: keep terms 4 and 5 of Eq. Jacobian-matrix-form2,
                    which the paper neglects: the numerical flux's dependence
                    on the face gradients (dH^n/d grad_j Q = -c n . dG/d grad_j Q,
                    c = 1/2 inside and 1 on a boundary, exact since G is linear
                    in the gradient) and the symmetric-flux lift with dS/dQ by
                    the one-sided difference of Eq. numerical-Jac-on-traces, in
                    the diagonal blocks and in the neighbour coupling (L+U);
                    viscous flows on meshes of axis-aligned elements, not with
                    fused (DG_ERR_UNSUPPORTED otherwise); 3 (NV D NV) values per
                    face point and side are stored */
} dg_prec_cfg;

/* Build (or rebuild in place, when *inout is not NULL and was built for the
 * same mesh) the BRJ preconditioner of dN/du = I - dt_a M^-1 dL/du at (u, t)
 * (Sec. 4.2.2, Eq. Jacobian-matrix-form/-form2, numerical-Jac-on-traces):
 * element-volume Jacobians from the exact flux derivatives, trace flux
 * Jacobians by one-sided differences with chi_k = sqrt(2^-52)*||u_k||_2,
 * the trace-gradient and symmetric-flux terms neglected (kept with
 * cfg->full_jacobian); the diagonal blocks are inverted in place (Gauss-
 * Jordan with partial pivoting, in the blocks' precision; BF16 blocks are
 * inverted in FP32 and rounded) and stored, the trace Jacobians kept for the
 * off-diagonal product.  Returns DG_ERR_NONFINITE when the elimination of
 * a block finds no non-zero pivot (a singular block). */
dg_status dg_precond_build(dg_mesh_t m, const double* u, double t, double dt_a,
                           const dg_prec_cfg* cfg, dg_precond_t* inout, void* stream);
/* FP64 blocks need 2 nm^2 doubles of shared memory per CTA (up to P = 3 in
 * 3-D) and, on general-geometry meshes, P <= 2; otherwise DG_ERR_UNSUPPORTED.
 * out = P^-1 q by the BRJ(J) iteration from q^0 = 0 (Eq. precond-Jacobi).
 * out must not alias q. */
dg_status dg_precond_apply(dg_precond_t p, const double* q, double* out, void* stream);
dg_status dg_precond_destroy(dg_precond_t p);

/* Restarted right-preconditioned GMRES (Sec. 3.2; Saad & Schultz) for
 * (I - dt_a dR/du(u)) x = b with the Jacobian-free product at (u, r_u):
 * x0 = 0, Arnoldi by classical Gram-Schmidt applied twice with fixed-order
 * FP64 reductions, Givens rotations, stop when the residual estimate is
 * <= rtol*||b||, at most max_cycles restarts of length restart
 * (1 <= restart <= 64).  p may be NULL (no preconditioner).
 * graphs != 0 launches each Arnoldi step (preconditioner apply, Jacobian-free
 * product, both Gram-Schmidt passes, the norm and the normalisation) as one
 * CUDA graph, captured the first time a (step index, restart, u, r_u,
 * preconditioner) set is seen and replayed afterwards; the results are bitwise
 * those of graphs = 0.  The mesh handle keeps up to 128 such graphs (the
 * oldest is dropped), and drops them all when its launch tuning changes or
 * its Krylov basis is reallocated.  Per-kernel profiling launches plainly.
 * dg_gmres_noalloc ignores graphs (it launches plainly). */
typedef struct {
  int restart;
  int max_cycles;
  double rtol;
  int graphs;
} dg_gmres_cfg;
typedef struct {
  int iters, cycles, converged;
  double res0, res;
} dg_gmres_stats;
dg_status dg_gmres(dg_mesh_t m, dg_precond_t p, const double* u, const double* r_u, double t,
                   double dt_a, const double* b, double* x, const dg_gmres_cfg* cfg,
                   dg_gmres_stats* stats, void* stream);

/* GMRES for callers that cannot allocate device memory (the paper has no
 * counterpart; this is an interface for such callers).  dg_gmres allocates its
 * Krylov basis with cudaMalloc on its first call; an application whose memory
 * pool has reserved the whole device up front, or a loop that forbids
 * allocator calls once it runs, cannot do that.  dg_gmres_noalloc solves the
 * same system with the same algorithm and arguments as dg_gmres, but keeps the
 * basis (restart+1 vectors, plus restart preconditioned vectors when p is not
 * NULL) in one static device array of DG_GMRES_NOALLOC_MAX_DOUBLES doubles
 * (16 MiB) that every GPU loading the library holds until exit; it calls no
 * cudaMalloc, cudaFree or allocating routine.  It ignores cfg->graphs, and it
 * runs the preconditioner's sweeps as plain kernel launches even when p was
 * built with graphs != 0 (capturing and instantiating a graph allocates; the
 * result is the same).  Like dg_gmres, it reads each Hessenberg column back to
 * the host and synchronises the stream after every Arnoldi step.  It returns
 * DG_ERR_ARG when n_dof * (restart + 1 + (p ? restart : 0)) exceeds the
 * array.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) as its set-up, so make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  The mesh and
 * preconditioner handles must already exist (they are created with
 * allocation, once, at set-up).  Per-kernel profiling (dg_profile_enable)
 * creates CUDA events; leave it off around this call. */
#define DG_GMRES_NOALLOC_MAX_DOUBLES 2097152
dg_status dg_gmres_noalloc(dg_mesh_t m, dg_precond_t p, const double* u, const double* r_u,
                           double t, double dt_a, const double* b, double* x,
                           const dg_gmres_cfg* cfg, dg_gmres_stats* stats, void* stream);

/* One implicit Runge-Kutta step (Sec. 3.2, Eq. rk-stage, rk-final; App. A
 * tableaus): each implicit stage solves
 *   N(u) = u - S_m - dt a_mm R(u, t + c_m dt) = 0,  S_m = u^n + sum_{j<m} a_mj E^j,
 * by Newton (Eq. Newton-Iteration) from u = S_m, stopping when
 * ||N|| < alpha ||N(S_m)|| (Eq. nonlinear-critria) or, if abs_tol > 0, when
 * ||N|| < abs_tol; E^m = dt R(u^m) from the converged iterate, and
 * u^{n+1} = u^n + sum_m b_m E^m.  Tableaus: DG_BE backward Euler (one stage,
 * a = b = c = 1), DG_SDIRK2 (lambda = 1 - sqrt(2)/2), DG_SDIRK3
 * (lambda = 0.4358665215), DG_ESDIRK4 the six-stage fourth-order table of
 * App. A (explicit first stage, diagonal 1/4, stiffly accurate; its first
 * column, printed as symbols, is read as a_i0 = a_i1, and its nodes are the
 * row sums).  The preconditioner in *p_inout is built at (u^n, t) for
 * dt a_mm (the diagonal all implicit stages share) when *p_inout is NULL or
 * rebuild != 0, and reused otherwise (freezing, Sec. 4.2.2); it is left in
 * *p_inout for the next step.  A learned guess (cfg.guess) needs a tableau
 * without an explicit stage and at most as many stages as the guess was
 * created with (DG_ERR_UNSUPPORTED otherwise).  DG_ERR_ARG for an unknown
 * tableau. */
enum { DG_BE = 1, DG_SDIRK2 = 2, DG_SDIRK3 = 3, DG_ESDIRK4 = 4 };
#define DG_MAX_STAGES 6
typedef struct {
  int tableau;
  double alpha;
  double abs_tol;
  int max_newton;
  int rebuild;
  int use_precond;
  dg_gmres_cfg gmres;
  dg_prec_cfg prec;
  struct dg_guess_s* guess; /* optional learned initial guess (NULL: S_m) */
  int guess_train_iters;    /* Adam steps per converged stage */
} dg_sdirk_cfg;
/* Per-step statistics; the stage arrays hold the first DG_MAX_STAGES stages
 * (an explicit stage reports 0 iterations and residuals). */
typedef struct {
  int newton_iters, gmres_iters, stages, precond_built;
  int stage_newton[DG_MAX_STAGES], stage_gmres[DG_MAX_STAGES];
  double stage_res0[DG_MAX_STAGES], stage_res[DG_MAX_STAGES];
  int guess_used; /* stages that started from the learned guess */
} dg_step_stats;
dg_status sdirk_step(dg_mesh_t m, const dg_sdirk_cfg* cfg, double* u_inout, double t, double dt,
                     dg_precond_t* p_inout, dg_step_stats* stats, void* stream);

/* One step of the second-order backward differentiation formula (Sec. 4.3
 * lists BDF2 among the implicit schemes) at a constant step size dt:
 *   3 u^{n+1} - 4 u^n + u^{n-1} = 2 dt R(u^{n+1}, t + dt),
 * solved as one Newton stage N(u) = u - S - (2 dt/3) R(u, t + dt) with
 * S = (4 u^n - u^{n-1})/3, from u = S, with the criteria, GMRES and
 * preconditioner settings of cfg (tableau ignored; the preconditioner is
 * built for dt_a = 2 dt/3).  u_inout holds u^n on entry and u^{n+1} on return;
 * u_prev_inout holds u^{n-1} on entry and u^n on return (they must differ).
 * The first step of a run needs u^{-1}: take it with sdirk_step.  cfg.guess
 * must be NULL (DG_ERR_UNSUPPORTED).  stats->stages = 1. */
dg_status bdf2_step(dg_mesh_t m, const dg_sdirk_cfg* cfg, double* u_inout, double* u_prev_inout,
                    double t, double dt, dg_precond_t* p_inout, dg_step_stats* stats,
                    void* stream);

/* Learned Newton initial guess.  The paper's guess for stage m is S_m
 * (Eq. Newton-initial-guess); this optional extension starts Newton from
 *   S_m + d_prev + y (x) tau_m,
 * where d_prev is the converged increment u^m - S_m of the same stage in the
 * previous step (an extrapolation in time) and y a per-element MLP per stage,
 *   x_e = [u^n/s0, (u^n-u^{n-1})/s1, d_prev/s2]   (s_k[v]: per-variable RMS),
 *   a1 = tanh(x W1 + b1), a2 = tanh(a1 W2 + b2), y = a2 W3 + b3,
 * trained online with Adam on the remainder (u^m - S_m - d_prev)/tau_m
 * (tau_m[v]: its per-variable RMS), BF16 operands and FP32 accumulation in
 * every product, FP32 master parameters.  mlp = 0 keeps only the
 * extrapolation.  The guess only seeds Newton: sdirk_step keeps S_m when the
 * guess's ||N|| is not smaller, and stops Newton at the absolute tolerance
 * alpha ||N(S_m)|| (the plain method's criterion) in both cases.  Training
 * data are the converged stages of the steps taken (dg_guess_train, called by
 * sdirk_step when cfg.guess is set). */
typedef struct dg_guess_s* dg_guess_t;
typedef struct {
  int stages, hidden, mlp;
  float lr, beta1, beta2, eps;
  float gate; /* use the MLP correction of a stage once its training loss is
                 below gate x that of a zero correction (<= 0: 0.2) */
} dg_guess_cfg;
/* params (ignored when mlp = 0): host FP32 arrays, for each stage s the six arrays
 * params[6s+0..5] = W1 [3 N_v N_m][hidden], b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], W3 [hidden][N_v N_m], b3 [N_v N_m] (row-major), copied. */
dg_status dg_guess_create(dg_mesh_t m, const dg_guess_cfg* cfg, const float* const* params,
                          dg_guess_t* out);
dg_status dg_guess_destroy(dg_guess_t g);
/* Append a step solution u (device) to the two-entry history (u^n, u^{n-1}). */
dg_status dg_guess_push(dg_guess_t g, const double* u, void* stream);
/* *ready = 1 when the history is full and stage `stage` has a previous increment. */
dg_status dg_guess_ready(dg_guess_t g, int stage, int* ready);
/* out = S + d_prev (+ MLP correction) for stage `stage` (device vectors). */
dg_status dg_guess_predict(dg_guess_t g, int stage, const double* S, double* out, void* stream);
/* Record the converged stage: iters Adam steps on the target
 * (u - S - d_prev)/tau of stage `stage` (all elements one batch; skipped until
 * a previous increment exists), then d_prev = u - S.  loss_first/last (host,
 * may be NULL): loss before the first and after the last step (-1 when no
 * training happened); grads_host (may be NULL, entries may be NULL): the six
 * FP32 gradients at the entry parameters.  iters = 0 evaluates without
 * updating the parameters. */
dg_status dg_guess_train(dg_guess_t g, int stage, const double* S, const double* u, int iters,
                         double* loss_first, double* loss_last, float* const* grads_host,
                         void* stream);
/* Copy the six FP32 master parameters of a stage to host arrays. */
dg_status dg_guess_params(dg_guess_t g, int stage, float* const* host_out);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all handles, all streams); a diagnostic counter for benchmarks. */
long long dg_kernel_launches(void);

/* Per-kernel timing (diagnostics, not part of the method): while enabled,
 * the library brackets each of its kernel launches with CUDA events on the
 * launch stream.  dg_profile_read synchronises the device and returns, per
 * kernel family, the launch count and summed device time since the previous
 * read (at most cap entries in out, *n set to the number written). */
typedef struct {
  char name[24];
  long long launches;
  double ms;
} dg_kernel_time;
dg_status dg_profile_enable(int on);
dg_status dg_profile_read(dg_kernel_time* out, int cap, int* n);

/* Measured FP64 FMA throughput of this GPU in TFLOP/s (diagnostic, no
 * counterpart in the paper): reps timed launches of a kernel whose threads run
 * eight independent fused multiply-add chains at full occupancy, timed with
 * CUDA events on `stream` after one warm-up launch (2 flops per FMA).  The
 * residual kernels are bound by this pipe; the benchmark divides their
 * algorithmic flop rate by this figure. */
dg_status dg_peak_fp64(int reps, double* tflops, void* stream);

/* Static description of a status code. */
const char* dg_status_string(dg_status s);

#ifdef __cplusplus
}
#endif
#endif /* DG_JFNK_H */
