// GMRES entry point for callers that must not allocate device memory.
//
// dg_gmres sizes its Krylov basis on its first call with cudaMalloc.  Some
// callers cannot allocate while they solve: applications whose memory pool
// has reserved the whole device up front, or loops that forbid allocator
// calls once they run (real-time or latency-bound drivers).  For them
// dg_gmres_noalloc runs the same algorithm with its Krylov basis in one
// file-scope static device array of fixed size, so the call performs no
// cudaMalloc, cudaFree or other allocating routine (host side included: its
// small Hessenberg arrays live on the stack).  The preconditioner's sweeps
// run as plain kernel launches whatever its graph setting, because
// capturing and instantiating a graph allocates.  Like dg_gmres, the call
// reads the Hessenberg column back to the host and synchronises the stream
// after every Arnoldi step.
#include <cmath>
#include <cuda_runtime.h>
#include "dg_internal.h"
#include "dg_precond.h"

namespace dg {

// Krylov scratch shared by every dg_gmres_noalloc call on a device; it holds
// the last call's contents.  Calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_krylov[DG_GMRES_NOALLOC_MAX_DOUBLES];

constexpr int MAX_DEVICES = 64;
static double* g_noalloc_ptr[MAX_DEVICES] = {nullptr};

// Device address of the static array for the current device (looked up once
// per device; in host code the array's name is only a host-side stand-in).
static dg_status noalloc_scratch(double** out) {
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return DG_ERR_UNSUPPORTED;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    DG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_krylov));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return DG_OK;
}

static dg_status noalloc_norm(dg_mesh_s* m, const double* a, double* out, cudaStream_t s) {
  DG_TRY(dot(a, a, m->ndof, m->red, m->hdev, s));
  DG_CUDA(cudaMemcpyAsync(m->hhost, m->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  *out = std::sqrt(m->hhost[0]);
  return std::isfinite(*out) ? DG_OK : DG_ERR_NONFINITE;
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_gmres_noalloc(dg_mesh_t m, dg_precond_t p, const double* u,
                                      const double* r_u, double t, double dt_a, const double* b,
                                      double* x, const dg_gmres_cfg* cfg, dg_gmres_stats* st,
                                      void* stream) {
  if (!m || !u || !r_u || !b || !x || !cfg) return DG_ERR_ARG;
  if (cfg->restart < 1 || cfg->restart > MAX_RESTART || cfg->max_cycles < 1 || !(cfg->rtol > 0.0))
    return DG_ERR_ARG;
  if (p && precond_mesh(p) != m) return DG_ERR_ARG;
  const int mr = cfg->restart;
  const long long n = m->ndof;
  const long long nvec = (long long)(mr + 1) + (p ? mr : 0);
  if (n * nvec > (long long)DG_GMRES_NOALLOC_MAX_DOUBLES) return DG_ERR_ARG;  // basis too large
  cudaStream_t s = (cudaStream_t)stream;
  double* V = nullptr;
  DG_TRY(noalloc_scratch(&V));
  double* Z = p ? V + (size_t)(mr + 1) * n : nullptr;
  dg_gmres_stats S{};
  double bn;
  DG_TRY(noalloc_norm(m, b, &bn, s));
  S.res0 = bn;
  DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  if (bn == 0.0) {
    S.converged = 1;
    if (st) *st = S;
    return DG_OK;
  }
  const double tol = cfg->rtol * bn;
  double H[(MAX_RESTART + 1) * MAX_RESTART], cs[MAX_RESTART], sn[MAX_RESTART];
  double g[MAX_RESTART + 1], y[MAX_RESTART];
  double* hd = m->hdev;
  double* hh = m->hhost;
  for (int cyc = 0; cyc < cfg->max_cycles; ++cyc) {
    double beta;
    if (cyc == 0) {
      DG_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      beta = bn;
    } else {
      DG_TRY(dg_jvp(m, u, r_u, t, x, 1.0, -dt_a, m->w2, s));
      DG_TRY(lincomb(V, b, 1.0, m->w2, -1.0, n, s));
      DG_TRY(noalloc_norm(m, V, &beta, s));
    }
    S.res = beta;
    if (beta <= tol) {
      S.converged = 1;
      break;
    }
    S.cycles++;
    DG_TRY(axpby(V, 1.0 / beta, V, 0.0, n, s));
    for (int i = 0; i <= mr; ++i) g[i] = 0.0;
    g[0] = beta;
    int kused = 0;
    bool done = false;
    for (int k = 0; k < mr; ++k) {
      const double* vk = V + (size_t)k * n;
      const double* zk = vk;
      if (p) {
        double* zz = Z + (size_t)k * n;
        // plain launches, never the graph replay: capturing and instantiating
        // a graph allocates (precond_sweeps is what the replay runs)
        DG_TRY(precond_sweeps(p, vk, zz, s));
        zk = zz;
      }
      double* w = V + (size_t)(k + 1) * n;
      DG_TRY(dg_jvp(m, u, r_u, t, zk, 1.0, -dt_a, w, s));
      S.iters++;
      DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd, s));
      DG_TRY(multi_axpy(w, V, k + 1, hd, n, s));
      DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd + (mr + 2), s));
      DG_TRY(multi_axpy(w, V, k + 1, hd + (mr + 2), n, s));
      DG_TRY(dot(w, w, n, m->red, hd + 2 * (mr + 2), s));
      DG_CUDA(cudaMemcpyAsync(hh, hd, sizeof(double) * 3 * (mr + 2), cudaMemcpyDeviceToHost, s));
      DG_CUDA(cudaStreamSynchronize(s));
      const double hn = std::sqrt(hh[2 * (mr + 2)]);
      if (!std::isfinite(hn)) return DG_ERR_NONFINITE;
      for (int i = 0; i <= k; ++i) H[(size_t)i * mr + k] = hh[i] + hh[(mr + 2) + i];
      H[(size_t)(k + 1) * mr + k] = hn;
      if (hn > 0.0) DG_TRY(axpby(w, 1.0 / hn, w, 0.0, n, s));
      for (int i = 0; i < k; ++i) {
        const double t0 = cs[i] * H[(size_t)i * mr + k] + sn[i] * H[(size_t)(i + 1) * mr + k];
        H[(size_t)(i + 1) * mr + k] = -sn[i] * H[(size_t)i * mr + k] + cs[i] * H[(size_t)(i + 1) * mr + k];
        H[(size_t)i * mr + k] = t0;
      }
      const double den = std::hypot(H[(size_t)k * mr + k], H[(size_t)(k + 1) * mr + k]);
      cs[k] = H[(size_t)k * mr + k] / den;
      sn[k] = H[(size_t)(k + 1) * mr + k] / den;
      H[(size_t)k * mr + k] = den;
      H[(size_t)(k + 1) * mr + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      kused = k + 1;
      S.res = std::fabs(g[k + 1]);
      if (S.res <= tol || hn == 0.0) {
        done = S.res <= tol;
        break;
      }
    }
    for (int i = kused - 1; i >= 0; --i) {
      double acc = g[i];
      for (int j = i + 1; j < kused; ++j) acc -= H[(size_t)i * mr + j] * y[j];
      y[i] = acc / H[(size_t)i * mr + i];
    }
    for (int i = 0; i < kused; ++i) hh[i] = -y[i];
    DG_CUDA(cudaMemcpyAsync(hd, hh, sizeof(double) * kused, cudaMemcpyHostToDevice, s));
    DG_TRY(multi_axpy(x, p ? Z : V, kused, hd, n, s));
    DG_CUDA(cudaStreamSynchronize(s));
    if (done) {
      S.converged = 1;
      break;
    }
  }
  if (st) *st = S;
  return S.converged ? DG_OK : DG_ERR_NOT_CONVERGED;
}
