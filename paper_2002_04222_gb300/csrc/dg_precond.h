// Internal interface of the block relaxed Jacobi preconditioner.
#pragma once
#include "dg_internal.h"

struct dg_precond_s {
  dg_mesh_s* mesh = nullptr;
  int J = 7;
  int precision = DG_PREC_FP64;
  double omega = 1.0;
  double dt_a = 0.0;
  int nb = 0;             // block size n_var * n_mode
  // identity of the apply's launch sequence (handle, J, omega, dt_a): new
  // whenever one changes, so graphs that captured the sweeps re-capture
  unsigned long long gen = 0;
  void* blocks = nullptr; // [E][nb][nb] inverse diagonal blocks (double, float or bf16)
  void* jd = nullptr;     // [E][2d][nf][nv][nv] own-side trace Jacobians (double or float)
  void* jo = nullptr;     // [E][2d][nv][nv][nf] neighbour trace Jacobians (point fastest)
  int32_t* nbr = nullptr; // [E][2d] neighbour (element * 2d + local face) or -1
  double* tr = nullptr;   // [E][2d][nv][nf] face values of the current iterate
  double* qh = nullptr;   // [ndof] iterate
  double* y = nullptr;    // [ndof] right-hand side of a sweep
  void* work = nullptr;   // build workspace
  size_t work_bytes = 0;
  int wchunk = 1;          // elements per pass of the weights workspace
  // graph replay of the apply (one instantiated graph per (q, out) pair)
  struct Graph {
    const double* q;
    double* out;
    cudaGraphExec_t exec;
    long long kernels;     // kernel launches the graph holds
  };
  int use_graphs = 0;
  int tc_invert = 0;      // FP32 blocks: trailing updates of the inversion on the tensor cores
  int fused = 0;          // sweeps j >= 2 as one off-diagonal + block kernel
  double* qh2 = nullptr;  // [ndof] second iterate buffer of the fused sweeps (lazily allocated)
  // terms 4-5 of the element Jacobian (full_jacobian): per element face and
  // point, K = s wJ dH/d grad Q [k][j][l], S_own / S_nbr = c wJ dS/dQ [i][k][l]
  int full = 0;
  void* jk = nullptr;
  void* jsd = nullptr;
  void* jso = nullptr;
  std::vector<Graph> graphs;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace dg {
dg_status precond_apply_impl(dg_precond_s* p, const double* q, double* out, cudaStream_t s);
// one fused sweep: out = omega D^-1 (q - (L+U) qprev) + (1-omega) qprev (dg_sweep.cu)
dg_status dispatch_sweep(dg_precond_s* p, const double* qprev, const double* q, double* out,
                         cudaStream_t s);
// the apply as plain kernel launches on s (for capture inside a larger graph)
dg_status precond_sweeps(dg_precond_s* p, const double* q, double* out, cudaStream_t s);
void precond_drop_graphs(dg_precond_s* p);
// in-place inversion of E blocks nb x nb (row stride ld), panel in registers
// (dg_invert.cu); supported for nb up to 640 (FP32) / 384 (FP64)
bool invert_rows_supported(int nb, bool fp64);
// terms 4-5 (dg_brj_visc.cu): supported (dim, P, Q), values per face point
// and side of each of the three arrays, build (after the block assembly,
// before the inversion) and the off-diagonal addition y += dt_a M^-1 (...) qh
bool visc_supported(int dim, int P, int Q);
size_t visc_values_per_face_point(int dim);
dg_status visc_build(dg_mesh_s* m, dg_precond_s* pc, double t, double dta, void* blk, int ld,
                     bool fp64, cudaStream_t s);
dg_status visc_offdiag(dg_precond_s* pc, const double* qh, double* y, cudaStream_t s);
dg_status launch_invert_rows(void* blocks, bool fp64, int E, int nb, int ld, int* fail,
                             cudaStream_t s);
inline dg_mesh_s* precond_mesh(dg_precond_s* p) { return p->mesh; }
}  // namespace dg
