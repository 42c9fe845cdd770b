// Internal definitions shared by the CUDA translation units of the DG library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include "../../include/dg.h"

namespace dg {

constexpr int QMAX = 8;   // largest Gauss point count per direction
constexpr int NMAX = 7;   // largest (P+1)
constexpr int MAX_RESTART = 64;  // largest GMRES restart length

// 1-D tables of one (P, Q) pair, passed by value to the kernels.
struct Tables {
  double B[QMAX * NMAX];      // B[q*n + k] = psi_k(x_q)
  double Dq[QMAX * QMAX];     // Dq[q*Q + k] = l_k'(x_q): collocation derivative on the Gauss points
  double w[QMAX];             // Gauss weights
  double x[QMAX];             // Gauss points
  double lm[QMAX], lp[QMAX];  // Lagrange extrapolation weights to xi = -1 and xi = +1
  double Minv[NMAX * NMAX];   // inverse of the 1-D mass matrix B^T diag(w) B
  double dpm[NMAX], dpp[NMAX];// psi_k'(-1), psi_k'(+1)
  int n, q;
};

// Physical model on the device (copy of dg_physics with derived constants).
struct Phys {
  double gamma, gm1, Pr, Ma, Re, mu, kappa_fac, T_inf_K, beta_s, gMa2;
  int viscous, mu_law, riemann, forcing, field;
  double fpar[8];
  int bc[8];
  // shock capturing (Sec. 3.1.2): mu_0 and the ramp half-width of the modal
  // sensor; avf = the per-element factor mu_0 S_e h_e / P of the state last
  // passed to the residual (device, [E]; nullptr without shock capturing)
  double av_mu0, av_kappa;
  const double* avf;
  int av_mode;  // 1: modal sensor; 2: modal sensor times Ducros' sensor at each point
};

// Modified-basis-to-Legendre transform of one direction for the modal sensor:
// T[a*n + k] = Legendre coefficient a of psi_k, nrm[a] = |L_a|^2 = 2/(2a+1).
// lo, hi: the ramp's ends as energy ratios, 10^(s0 -+ kappa) with s0 = log10(P^-4).
struct SensorTab {
  double T[NMAX * NMAX];
  double nrm[NMAX];
  double lo, hi;
};

// Element geometry of an axis-aligned affine element: origin and edge lengths.
struct ElemGeo {
  double x0[3];
  double h[3];
  double rh[3];       // 2/h: reference-to-physical derivative factors
  double detJ, idet;  // |J| = prod h/2 and its inverse
};

// device pointers of the general-geometry data, passed by value to kernels
struct GenGeo {
  const double* vgeo;   // [E][DIM*DIM+1][NQ]
  const double* vx;     // [E][DIM][NQ]
  const double* fgeo;   // [E][2DIM][DIM*DIM][NF]
  const double* fdat;   // [F][2DIM+1][NF]
  const double* fbeta;  // [F]
  const double* minv;   // [E][NM][NM]
};

}  // namespace dg

struct dg_precond_s;

namespace dg {
// launch shape of the sum-factorisation kernels (elements and threads per CTA)
struct Tune {
  int vol_epb, vol_threads, lift_epb, lift_threads;
};
}  // namespace dg

struct dg_mesh_s {
  int dim, P, Q, E, nv, nm, nq, nf, F;
  long long ndof;
  dg::Tables tab;
  dg::Phys phys;
  dg::Tune tune;
  // device buffers
  dg::ElemGeo* geo = nullptr;   // [E] axis-aligned affine elements (curved = 0)
  // general elements (curved = 1: quadratic, or straight-sided but not
  // axis-aligned): per-point metrics, face data and dense inverse mass matrices
  int curved = 0;
  double* vgeo = nullptr;       // [E][dim*dim+1][nq]: d xi_r/d x_j (r-major), then w|J|
  double* vx = nullptr;         // [E][dim][nq] coordinates of the volume points
  double* fgeo = nullptr;       // [E][2dim][dim*dim][nf] d xi_r/d x_j at the face points
  double* fdat = nullptr;       // [F][2dim+1][nf] owner normal n, w^G J^G, coordinates x
  double* fbeta = nullptr;      // [F] interior-penalty factor (P+1)^2 / h
  double* minv = nullptr;       // [E][nm][nm] inverse element mass matrices
  int32_t* faces = nullptr;     // [F][6]
  double* hbuf = nullptr;       // [E][dim][nv][nq]   weighted volume fluxes
  double* tbuf = nullptr;       // [E][2dim][(1+dim)nv][nf] face traces
  double* fbuf = nullptr;       // [E][2dim][(1+dim)nv][nf] face fluxes to lift
  double* force = nullptr;      // [ndof] M^-1 B^T wJ f (nullptr when no forcing)
  double* avf = nullptr;        // [E] artificial-viscosity factor (shock capturing only)
  dg::SensorTab stab;
  double* scratch = nullptr;    // [64]: [0,4) JFNK eps, 1/eps, norms; [8,13) BRJ chi;
                                //   [16] inversion failure flag; [24,26) GMRES {t, -dt_a}
  double* red = nullptr;        // reduction partials
  double* w1 = nullptr;         // work vectors of ndof
  double* w2 = nullptr;
  // GMRES workspace (lazily sized)
  double* krylov = nullptr;     // V[(m+1)][ndof] then Z[m][ndof]
  int krylov_m = 0;
  double* hdev = nullptr;       // [2*(mmax+2)] Hessenberg column on device
  double* hhost = nullptr;      // pinned host mirror
  // SDIRK workspace
  double* stage = nullptr;      // [DG_MAX_STAGES + 7][ndof]: E^0..E^5, S, U, R, N, U2, R2, N2
  std::vector<std::vector<int>> elem_faces;  // host: face id of (e, lf)
  // graph replay of GMRES Arnoldi steps (one instantiated graph per step index
  // and operand set; see gmres_impl)
  struct ArnoldiGraph {
    int k, mr;
    const double *u, *r_u;
    double* V;
    const void* p;
    unsigned long long pgen;
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<ArnoldiGraph> agraphs;
  cudaStream_t gs = nullptr;  // capture stream
};

namespace dg {

// error plumbing
dg_status cuda_status(cudaError_t e);
#define DG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return ::dg::cuda_status(_e); \
  } while (0)
// count of kernels launched by the library (diagnostics: dg_kernel_launches)
extern long long g_launches;
#define DG_LAUNCHED(n)                                     \
  do {                                                     \
    __atomic_fetch_add(&::dg::g_launches, (long long)(n), __ATOMIC_RELAXED); \
    cudaError_t _e = cudaGetLastError();                   \
    if (_e != cudaSuccess) return ::dg::cuda_status(_e);   \
  } while (0)
// optional per-kernel timing with CUDA events on the launch stream
enum KernelId {
  K_VOL, K_FACE, K_LIFT, K_PROJECT, K_DOT, K_MULTIDOT, K_MULTIAXPY, K_VEC,
  K_BRJ_WEIGHTS, K_BRJ_TRACEJAC, K_BRJ_BLOCK, K_BRJ_INVERT, K_BRJ_DIAG,
  K_BRJ_OFFDIAG, K_MLP, K_BRJ_SWEEP, K_SENSOR, K_COUNT
};
int prof_begin(int id, cudaStream_t s);
void prof_end(int handle, cudaStream_t s);
bool profiling_on();
#define DG_PROF(id, stream, ...)                    \
  do {                                              \
    const int _ph = ::dg::prof_begin(id, stream);   \
    __VA_ARGS__;                                    \
    ::dg::prof_end(_ph, stream);                    \
  } while (0)
#define DG_TRY(call)                 \
  do {                               \
    dg_status _s = (call);           \
    if (_s != DG_OK) return _s;      \
  } while (0)

// residual pipeline (dg_residual.cu)
enum EvalMode { EVAL_RESIDUAL = 0, EVAL_JVP = 1 };
struct EvalArgs {
  const double* u;     // base state
  const double* v;     // JVP direction (nullptr for a plain residual)
  const double* r_u;   // R(u) (JVP only)
  const double* eps;   // device scalars {eps, 1/eps} (JVP only)
  double alpha, beta;  // JVP combination
  double t;
  double* out;
  // optional device scalars {t, beta} read by the kernels in place of t and
  // beta, so that a captured graph serves every time level and step size
  const double* dscal = nullptr;
  bool skip_vol = false, skip_lift = false;  // autotuning times the kernels separately
};
dg_status launch_residual(dg_mesh_s* m, const EvalArgs& a, cudaStream_t s);
dg_status build_general_geometry(dg_mesh_s* m, const double* nodes_host, int g, cudaStream_t s);
dg_status launch_project(dg_mesh_s* m, int what, double t, double* out, cudaStream_t s);
// artificial-viscosity factor mu_0 S_e h_e / P of every element at u into out [E]
dg_status launch_sensor(dg_mesh_s* m, const double* u, double* out, cudaStream_t s);
bool supported(int dim, int P, int Q);
bool supported_curved(int dim, int P, int Q);  // general-geometry instances
inline GenGeo gen_geo(const dg_mesh_s* m) {
  return GenGeo{m->vgeo, m->vx, m->fgeo, m->fdat, m->fbeta, m->minv};
}
void init_tune(dg_mesh_s* m);
dg_status autotune(dg_mesh_s* m, int reps, dg_tune_result* res, cudaStream_t s);
bool tune_valid(dg_mesh_s* m, const dg_tune_result* t);

// learned initial guess (dg_learned.cu)
bool guess_history_empty(const dg_guess_s* g);
bool guess_history_full(const dg_guess_s* g);
int guess_stage_count(const dg_guess_s* g);

// dense vector kernels (dg_blas.cu)
constexpr int RED_BLOCKS = 296;   // 2 per SM: fixed, so reductions repeat bitwise
dg_status dot(const double* a, const double* b, long long n, double* partial, double* out,
              cudaStream_t s);
dg_status finish_sum(const double* partial, int np, double* out, cudaStream_t s);
dg_status multi_dot(const double* V, int k, const double* w, long long n, double* partial,
                    double* out, cudaStream_t s);
dg_status multi_axpy(double* w, const double* V, int k, const double* h, long long n,
                     cudaStream_t s);  // w -= sum_i h_i V_i
dg_status axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s);
dg_status lincomb(double* y, const double* x, double a, const double* z, double b, long long n,
                  cudaStream_t s);  // y = a x + b z
dg_status scale_dev(double* y, const double* x, const double* sdev, int inv, long long n,
                    cudaStream_t s);
dg_status jvp_eps(const double* u, const double* v, long long n, double* partial, double* eps,
                  cudaStream_t s);
dg_status newton_resid(double* N, const double* u, const double* S, const double* R, double dta,
                       long long n, cudaStream_t s);
dg_status set_scalars(double* d, double a, double b, cudaStream_t s);  // d[0] = a, d[1] = b
// w = w / sqrt(*hsq) when sqrt(*hsq) > 0 (the same arithmetic as axpby(w, 1/h, w, 0))
dg_status normalize_dev(double* w, const double* hsq, long long n, cudaStream_t s);
void drop_arnoldi_graphs(dg_mesh_s* m);

}  // namespace dg
