// C ABI entry points: mesh set-up (1-D tables, metrics, connectivity checks),
// residual, Jacobian-free product, GMRES, Newton and SDIRK orchestration.
// The host drives the Krylov/Newton/SDIRK loops; every vector operation,
// reduction and residual evaluation runs in the library's CUDA kernels.
#include <cmath>
#include <cstring>
#include <cstdio>
#include <new>
#include <vector>
#include "dg_internal.h"
#include "dg_precond.h"

namespace dg {

long long g_launches = 0;

// ---------------------------------------------------------------- profiling
static const char* kernel_names[K_COUNT] = {
    "dg_vol", "dg_face", "dg_lift", "dg_project", "dot", "multi_dot", "multi_axpy", "vector",
    "brj_weights", "brj_tracejac", "brj_block", "brj_invert", "brj_diag",
    "brj_offdiag", "mlp_gemm", "brj_sweep", "dg_sensor"};
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool profiling_on() { return g_prof; }

int prof_begin(int id, cudaStream_t s) {
  if (!g_prof) return -1;
  ProfRec r{id, take_event(), take_event()};
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int h, cudaStream_t s) {
  if (h < 0) return;
  cudaEventRecord(g_recs[h].b, s);
}

dg_status cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DG_ERR_OOM;
  }
  return DG_ERR_CUDA;
}

// ---------------------------------------------------------------- 1-D tables
static void gauss_legendre(int Q, double* x, double* w) {
  for (int i = 0; i < Q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (Q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= Q; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pq = Q == 0 ? 1.0 : p1, pm = p0;
      if (Q == 1) {
        pq = z;
        pm = 1.0;
      }
      double dp = Q * (z * pq - pm) / (z * z - 1.0);
      double dz = pq / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        it = 100;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= Q; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pq = Q == 1 ? z : p1, pm = Q == 1 ? 1.0 : p0;
    double dp = Q * (z * pq - pm) / (z * z - 1.0);
    x[Q - 1 - i] = z;
    w[Q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Jacobi P_n^(1,1)(x) and derivative
static void jacobi11(int n, double x, double* p, double* dp) {
  auto val = [](int n, double a, double b, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((a - b) + (a + b + 2.0) * x);
    for (int k = 1; k < n; ++k) {
      double c = 2.0 * k + a + b;
      double a1 = 2.0 * (k + 1) * (k + a + b + 1) * c;
      double a2 = (c + 1) * (a * a - b * b);
      double a3 = c * (c + 1) * (c + 2);
      double a4 = 2.0 * (k + a) * (k + b) * (c + 2);
      double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  *p = val(n, 1.0, 1.0, x);
  *dp = n == 0 ? 0.0 : 0.5 * (n + 3) * val(n - 1, 2.0, 2.0, x);
}

// modified basis psi_k(x) and derivative, k = 0..P
static void modified_basis(int P, double x, double* phi, double* dphi) {
  phi[0] = 0.5 * (1 - x);
  dphi[0] = -0.5;
  phi[P] = 0.5 * (1 + x);
  dphi[P] = 0.5;
  for (int p = 1; p < P; ++p) {
    double j, dj;
    jacobi11(p - 1, x, &j, &dj);
    double b = 0.25 * (1 - x) * (1 + x);
    phi[p] = b * j;
    dphi[p] = -0.5 * x * j + b * dj;
  }
}

static bool invert_small(int n, const double* A, double* Ainv) {
  std::vector<double> M(A, A + n * n), I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > std::fabs(M[piv * n + c])) piv = r;
    if (M[piv * n + c] == 0.0) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(M[c * n + k], M[piv * n + k]);
      std::swap(I[c * n + k], I[piv * n + k]);
    }
    double d = 1.0 / M[c * n + c];
    for (int k = 0; k < n; ++k) {
      M[c * n + k] *= d;
      I[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        M[r * n + k] -= f * M[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  std::memcpy(Ainv, I.data(), sizeof(double) * n * n);
  return true;
}

static void build_tables(int P, int Q, Tables& t) {
  std::memset(&t, 0, sizeof(t));
  const int n = P + 1;
  t.n = n;
  t.q = Q;
  gauss_legendre(Q, t.x, t.w);
  double phi[NMAX], dphi[NMAX];
  for (int q = 0; q < Q; ++q) {
    modified_basis(P, t.x[q], phi, dphi);
    for (int k = 0; k < n; ++k) t.B[q * n + k] = phi[k];
  }
  // barycentric weights of the Gauss points
  double bw[QMAX];
  for (int k = 0; k < Q; ++k) {
    double p = 1.0;
    for (int j = 0; j < Q; ++j)
      if (j != k) p *= (t.x[k] - t.x[j]);
    bw[k] = 1.0 / p;
  }
  for (int i = 0; i < Q; ++i) {
    double diag = 0.0;
    for (int k = 0; k < Q; ++k) {
      if (k == i) continue;
      double d = (bw[k] / bw[i]) / (t.x[i] - t.x[k]);
      t.Dq[i * Q + k] = d;
      diag -= d;
    }
    t.Dq[i * Q + i] = diag;
  }
  for (int k = 0; k < Q; ++k) {
    double am = 1.0, ap = 1.0;
    for (int j = 0; j < Q; ++j) {
      if (j == k) continue;
      am *= (-1.0 - t.x[j]) / (t.x[k] - t.x[j]);
      ap *= (1.0 - t.x[j]) / (t.x[k] - t.x[j]);
    }
    t.lm[k] = am;
    t.lp[k] = ap;
  }
  double M1[NMAX * NMAX];
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double s = 0.0;
      for (int q = 0; q < Q; ++q) s += t.B[q * n + a] * t.w[q] * t.B[q * n + b];
      M1[a * n + b] = s;
    }
  invert_small(n, M1, t.Minv);
  modified_basis(P, -1.0, phi, dphi);
  for (int k = 0; k < n; ++k) t.dpm[k] = dphi[k];
  modified_basis(P, 1.0, phi, dphi);
  for (int k = 0; k < n; ++k) t.dpp[k] = dphi[k];
}

// Modal sensor table: the Legendre coefficients of the modified basis,
// T[a][k] = (2a+1)/2 sum_q w_q L_a(x_q) psi_k(x_q) (the Gauss rule is exact,
// the product has degree <= 2P <= 2Q-1), and |L_a|^2 = 2/(2a+1).
static void build_sensor_table(int P, double kappa, const Tables& t, SensorTab& st) {
  std::memset(&st, 0, sizeof(st));
  const int n = P + 1;
  for (int q = 0; q < t.q; ++q) {
    double L[NMAX];
    L[0] = 1.0;
    if (n > 1) L[1] = t.x[q];
    for (int a = 2; a < n; ++a) L[a] = ((2 * a - 1) * t.x[q] * L[a - 1] - (a - 1) * L[a - 2]) / a;
    for (int a = 0; a < n; ++a)
      for (int k = 0; k < n; ++k) st.T[a * n + k] += 0.5 * (2 * a + 1) * t.w[q] * L[a] * t.B[q * n + k];
  }
  for (int a = 0; a < n; ++a) st.nrm[a] = 2.0 / (2 * a + 1);
  const double p4 = 1.0 / ((double)P * P * P * P);
  st.lo = p4 * std::pow(10.0, -kappa);
  st.hi = p4 * std::pow(10.0, kappa);
}

void drop_arnoldi_graphs(dg_mesh_s* m) {
  for (auto& g : m->agraphs) cudaGraphExecDestroy(g.exec);
  m->agraphs.clear();
}

}  // namespace dg

using namespace dg;

extern "C" {

long long dg_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

dg_status dg_profile_enable(int on) {
  g_prof = on != 0;
  return DG_OK;
}

dg_status dg_profile_read(dg_kernel_time* out, int cap, int* n) {
  if (!out || !n || cap < 0) return DG_ERR_ARG;
  DG_CUDA(cudaDeviceSynchronize());
  double ms[K_COUNT] = {0};
  long long cnt[K_COUNT] = {0};
  for (const ProfRec& r : g_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.id] += t;
    cnt[r.id]++;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_recs.clear();
  int k = 0;
  for (int i = 0; i < K_COUNT; ++i) {
    if (cnt[i] == 0) continue;
    if (k < cap) {
      std::memset(out[k].name, 0, sizeof(out[k].name));
      std::strncpy(out[k].name, kernel_names[i], sizeof(out[k].name) - 1);
      out[k].launches = cnt[i];
      out[k].ms = ms[i];
    }
    ++k;
  }
  *n = k < cap ? k : cap;
  return DG_OK;
}

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_OOM: return "out of device memory";
    case DG_ERR_NONFINITE: return "non-finite norm";
    case DG_ERR_NOT_CONVERGED: return "iteration cap reached without convergence";
    case DG_ERR_UNSUPPORTED: return "unsupported configuration";
    case DG_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

static void free_mesh(dg_mesh_s* m) {
  if (!m) return;
  cudaFree(m->geo);
  cudaFree(m->faces);
  cudaFree(m->hbuf);
  cudaFree(m->tbuf);
  cudaFree(m->fbuf);
  cudaFree(m->vgeo);
  cudaFree(m->vx);
  cudaFree(m->fgeo);
  cudaFree(m->fdat);
  cudaFree(m->fbeta);
  cudaFree(m->minv);
  cudaFree(m->force);
  cudaFree(m->avf);
  cudaFree(m->scratch);
  cudaFree(m->red);
  cudaFree(m->w1);
  cudaFree(m->w2);
  cudaFree(m->krylov);
  cudaFree(m->hdev);
  cudaFree(m->stage);
  if (m->hhost) cudaFreeHost(m->hhost);
  drop_arnoldi_graphs(m);
  if (m->gs) cudaStreamDestroy(m->gs);
  delete m;
}

dg_status dg_mesh_create(const dg_mesh_desc* md, const dg_physics* ph, void* stream,
                         dg_mesh_t* out) {
  if (!md || !ph || !out || !md->nodes || !md->faces) return DG_ERR_ARG;
  *out = nullptr;
  const int d = md->dim;
  if (d != 2 && d != 3) return DG_ERR_ARG;
  if (md->P < 1 || md->Q < 1 || md->n_elem < 1 || md->n_faces < 1) return DG_ERR_ARG;
  if (md->P + 1 > NMAX || md->Q > QMAX) return DG_ERR_UNSUPPORTED;
  if (md->geom_order != 1 && md->geom_order != 2) return DG_ERR_UNSUPPORTED;
  if (!supported(d, md->P, md->Q)) return DG_ERR_UNSUPPORTED;
  if (ph->n_bc < 0 || ph->n_bc > 8) return DG_ERR_ARG;
  if (ph->riemann < DG_RIEMANN_ROE || ph->riemann > DG_RIEMANN_AUSM) return DG_ERR_ARG;
  if (ph->av < 0 || ph->av > 2) return DG_ERR_ARG;
  if (ph->av && (!ph->viscous || !(ph->av_mu0 >= 0.0) || !(ph->av_kappa > 0.0)))
    return DG_ERR_ARG;  // artificial viscosity enters through the diffusion flux
  cudaStream_t s = (cudaStream_t)stream;
  const int E = md->n_elem, F = md->n_faces;
  // axis-aligned affine boxes take the diagonal-metric kernels; any other
  // element (quadratic, rotated, sheared) the general-geometry kernels
  std::vector<ElemGeo> geo(E);
  bool boxes = md->geom_order == 1;
  const int nn = 1 << d;
  for (int e = 0; e < E && boxes; ++e) {
    const double* X = md->nodes + (size_t)e * nn * d;
    ElemGeo g{};
    for (int r = 0; r < d; ++r) {
      g.x0[r] = X[r];
      g.h[r] = X[(1 << r) * d + r] - X[r];
      if (!(g.h[r] > 0.0)) boxes = false;
    }
    for (int a = 0; a < nn && boxes; ++a)
      for (int r = 0; r < d; ++r) {
        double expect = g.x0[r] + (((a >> r) & 1) ? g.h[r] : 0.0);
        if (std::fabs(X[a * d + r] - expect) > 1e-12 * (1.0 + std::fabs(expect))) boxes = false;
      }
    g.detJ = 1.0;
    for (int r = 0; r < 3; ++r) {
      g.rh[r] = r < d ? 2.0 / g.h[r] : 0.0;
      if (r < d) g.detJ *= 0.5 * g.h[r];
    }
    g.idet = 1.0 / g.detJ;
    geo[e] = g;
  }
  if (!boxes) std::fill(geo.begin(), geo.end(), ElemGeo{});
  if (!boxes && !supported_curved(d, md->P, md->Q)) return DG_ERR_UNSUPPORTED;
  // connectivity: every (element, local face) exactly once, aligned sides
  std::vector<int> seen((size_t)E * 2 * d, 0);
  for (int f = 0; f < F; ++f) {
    const int32_t* fc = md->faces + (size_t)f * 6;
    int eL = fc[0], fL = fc[1], eR = fc[2], fR = fc[3], orient = fc[4], bc = fc[5];
    if (eL < 0 || eL >= E || fL < 0 || fL >= 2 * d) return DG_ERR_ARG;
    if (orient != 0) return DG_ERR_UNSUPPORTED;
    seen[(size_t)eL * 2 * d + fL]++;
    if (eR >= 0) {
      if (eR >= E || fR < 0 || fR >= 2 * d) return DG_ERR_ARG;
      if ((fR >> 1) != (fL >> 1) || (fR & 1) == (fL & 1)) return DG_ERR_UNSUPPORTED;
      seen[(size_t)eR * 2 * d + fR]++;
    } else {
      if (bc < 0 || bc >= ph->n_bc) return DG_ERR_ARG;
      int t = ph->bc[bc];
      if (t != DG_BC_DIRICHLET && t != DG_BC_ISO_WALL && t != DG_BC_ADIA_WALL &&
          t != DG_BC_FARFIELD)
        return DG_ERR_UNSUPPORTED;
    }
  }
  for (size_t i = 0; i < seen.size(); ++i)
    if (seen[i] != 1) return DG_ERR_ARG;

  dg_mesh_s* m = new (std::nothrow) dg_mesh_s();
  if (!m) return DG_ERR_OOM;
  m->dim = d;
  m->P = md->P;
  m->Q = md->Q;
  m->E = E;
  m->F = F;
  m->nv = d + 2;
  const int n = md->P + 1;
  m->nm = d == 2 ? n * n : n * n * n;
  m->nq = d == 2 ? md->Q * md->Q : md->Q * md->Q * md->Q;
  m->nf = d == 2 ? md->Q : md->Q * md->Q;
  m->ndof = (long long)E * m->nv * m->nm;
  build_tables(md->P, md->Q, m->tab);
  init_tune(m);
  Phys& p = m->phys;
  std::memset(&p, 0, sizeof(p));
  p.gamma = ph->gamma;
  p.gm1 = ph->gamma - 1.0;
  p.Pr = ph->Pr;
  p.Ma = ph->Ma;
  p.Re = ph->Re;
  p.mu = 1.0 / ph->Re;
  p.kappa_fac = 1.0 / (ph->Ma * ph->Ma * ph->Pr * (ph->gamma - 1.0));
  p.T_inf_K = ph->T_inf_K;
  p.beta_s = ph->beta_s;
  p.gMa2 = ph->gamma * ph->Ma * ph->Ma;
  p.viscous = ph->viscous;
  p.mu_law = ph->mu_law;
  p.riemann = ph->riemann;
  p.forcing = ph->forcing;
  p.field = ph->field;
  for (int i = 0; i < 8; ++i) {
    p.fpar[i] = ph->fpar[i];
    p.bc[i] = ph->bc[i];
  }
  const size_t nd = (size_t)m->ndof;
  const size_t ntr = (size_t)E * 2 * d * (1 + d) * m->nv * m->nf;
  cudaError_t err = cudaSuccess;
  // every workspace starts zeroed: no kernel result may depend on what an
  // earlier allocation left in the memory
  auto alloc = [&](void** ptr, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc(ptr, bytes);
    if (err == cudaSuccess) err = cudaMemsetAsync(*ptr, 0, bytes, s);
  };
  alloc((void**)&m->geo, sizeof(ElemGeo) * E);
  alloc((void**)&m->faces, sizeof(int32_t) * 6 * F);
  alloc((void**)&m->hbuf, sizeof(double) * (size_t)E * d * m->nv * m->nq);
  alloc((void**)&m->tbuf, sizeof(double) * ntr);
  alloc((void**)&m->fbuf, sizeof(double) * ntr);
  alloc((void**)&m->scratch, sizeof(double) * 64);
  alloc((void**)&m->red, sizeof(double) * RED_BLOCKS * (MAX_RESTART + 8));
  alloc((void**)&m->hdev, sizeof(double) * 4 * (MAX_RESTART + 2));
  if (err == cudaSuccess) err = cudaMallocHost((void**)&m->hhost, sizeof(double) * 4 * (MAX_RESTART + 2));
  alloc((void**)&m->w1, sizeof(double) * nd);
  alloc((void**)&m->w2, sizeof(double) * nd);
  if (ph->forcing) alloc((void**)&m->force, sizeof(double) * nd);
  if (ph->av) {
    alloc((void**)&m->avf, sizeof(double) * E);
    p.avf = m->avf;
    p.av_mu0 = ph->av_mu0;
    p.av_kappa = ph->av_kappa;
    p.av_mode = ph->av;
    build_sensor_table(md->P, ph->av_kappa, m->tab, m->stab);
  }
  if (err != cudaSuccess) {
    free_mesh(m);
    return cuda_status(err);
  }
  err = cudaMemcpyAsync(m->geo, geo.data(), sizeof(ElemGeo) * E, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(m->faces, md->faces, sizeof(int32_t) * 6 * F, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    free_mesh(m);
    return cuda_status(err);
  }
  if (!boxes) {
    m->curved = 1;
    dg_status st = build_general_geometry(m, md->nodes, md->geom_order, s);
    if (st != DG_OK) {
      free_mesh(m);
      return st;
    }
  }
  if (ph->forcing) {
    dg_status st = launch_project(m, 1, 0.0, m->force, s);
    if (st != DG_OK) {
      free_mesh(m);
      return st;
    }
  }
  *out = m;
  return DG_OK;
}

dg_status dg_mesh_destroy(dg_mesh_t m) {
  if (!m) return DG_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  free_mesh(m);
  return e == cudaSuccess ? DG_OK : cuda_status(e);
}

dg_status dg_mesh_info(dg_mesh_t m, dg_mesh_info_t* info) {
  if (!m || !info) return DG_ERR_ARG;
  info->dim = m->dim;
  info->P = m->P;
  info->Q = m->Q;
  info->n_elem = m->E;
  info->n_var = m->nv;
  info->n_mode = m->nm;
  info->n_quad = m->nq;
  info->n_faces = m->F;
  info->n_dof = m->ndof;
  return DG_OK;
}

dg_status dg_autotune(dg_mesh_t m, int reps, dg_tune_result* result, void* stream) {
  if (!m || !result || reps < 1) return DG_ERR_ARG;
  dg_tune_result r{};
  DG_TRY(autotune(m, reps, &r, (cudaStream_t)stream));
  drop_arnoldi_graphs(m);  // captured with the previous launch shapes
  *result = r;
  return DG_OK;
}

dg_status dg_set_tune(dg_mesh_t m, const dg_tune_result* t) {
  if (!m || !t) return DG_ERR_ARG;
  if (!tune_valid(m, t)) return DG_ERR_ARG;
  m->tune.vol_epb = t->vol_epb;
  m->tune.vol_threads = t->vol_threads;
  m->tune.lift_epb = t->lift_epb;
  m->tune.lift_threads = t->lift_threads;
  drop_arnoldi_graphs(m);
  return DG_OK;
}

dg_status dg_project(dg_mesh_t m, double t, double* u, void* stream) {
  if (!m || !u) return DG_ERR_ARG;
  return launch_project(m, 0, t, u, (cudaStream_t)stream);
}

dg_status dg_av_factor(dg_mesh_t m, const double* u, double* fac, void* stream) {
  if (!m || !u || !fac) return DG_ERR_ARG;
  if (!m->phys.avf) return DG_ERR_UNSUPPORTED;
  return launch_sensor(m, u, fac, (cudaStream_t)stream);
}

dg_status dg_residual(dg_mesh_t m, const double* u, double t, double* r, void* stream) {
  if (!m || !u || !r || u == r) return DG_ERR_ARG;
  EvalArgs a{};
  a.u = u;
  a.t = t;
  a.out = r;
  return launch_residual(m, a, (cudaStream_t)stream);
}

dg_status dg_jvp(dg_mesh_t m, const double* u, const double* r_u, double t, const double* v,
                 double alpha, double beta, double* out, void* stream) {
  if (!m || !u || !r_u || !v || !out) return DG_ERR_ARG;
  if (out == u || out == r_u || out == v) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DG_TRY(jvp_eps(u, v, m->ndof, m->red, m->scratch, s));
  EvalArgs a{};
  a.u = u;
  a.v = v;
  a.r_u = r_u;
  a.eps = m->scratch;
  a.alpha = alpha;
  a.beta = beta;
  a.t = t;
  a.out = out;
  return launch_residual(m, a, s);
}

// ---------------------------------------------------------------- GMRES
static dg_status ensure_krylov(dg_mesh_s* m, int restart) {
  if (m->krylov && m->krylov_m >= restart) return DG_OK;
  drop_arnoldi_graphs(m);  // they hold the old basis
  cudaFree(m->krylov);  // implicitly synchronises the device
  m->krylov = nullptr;
  const size_t nd = (size_t)m->ndof;
  DG_CUDA(cudaMalloc(&m->krylov, sizeof(double) * nd * (2 * (size_t)restart + 1)));
  DG_CUDA(cudaMemset(m->krylov, 0, sizeof(double) * nd * (2 * (size_t)restart + 1)));
  m->krylov_m = restart;
  return DG_OK;
}

static dg_status host_norm(dg_mesh_s* m, const double* a, double* out, cudaStream_t s) {
  DG_TRY(dot(a, a, m->ndof, m->red, m->hdev, s));
  DG_CUDA(cudaMemcpyAsync(m->hhost, m->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  *out = std::sqrt(m->hhost[0]);
  if (!std::isfinite(*out)) return DG_ERR_NONFINITE;
  return DG_OK;
}

// A z = z - dt_a (R(u + eps z) - r_u)/eps
static dg_status apply_A(dg_mesh_s* m, const double* u, const double* r_u, double t, double dta,
                         const double* z, double* out, cudaStream_t s) {
  return dg_jvp(m, u, r_u, t, z, 1.0, -dta, out, s);
}

// The device work of Arnoldi step k: z_k = P^-1 v_k, w = A z_k by the
// Jacobian-free product, two classical Gram-Schmidt passes, ||w||^2, the
// Hessenberg column copied to the pinned host mirror and w normalised with
// the norm read on the device.  t and -dt_a come from the device scalars
// dscal, so one captured sequence serves every stage and step.
static dg_status arnoldi_step_ops(dg_mesh_s* m, dg_precond_s* p, const double* u,
                                  const double* r_u, const double* dscal, double* V, int k,
                                  int mr, cudaStream_t s) {
  const long long n = m->ndof;
  double* hd = m->hdev;
  const double* vk = V + (size_t)k * n;
  const double* zk = vk;
  if (p) {
    double* zz = V + (size_t)(mr + 1) * n + (size_t)k * n;
    DG_TRY(precond_sweeps(p, vk, zz, s));
    zk = zz;
  }
  double* w = V + (size_t)(k + 1) * n;
  DG_TRY(jvp_eps(u, zk, n, m->red, m->scratch, s));
  EvalArgs a{};
  a.u = u;
  a.v = zk;
  a.r_u = r_u;
  a.eps = m->scratch;
  a.alpha = 1.0;
  a.dscal = dscal;
  a.out = w;
  DG_TRY(launch_residual(m, a, s));
  DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd, s));
  DG_TRY(multi_axpy(w, V, k + 1, hd, n, s));
  DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd + (mr + 2), s));
  DG_TRY(multi_axpy(w, V, k + 1, hd + (mr + 2), n, s));
  DG_TRY(dot(w, w, n, m->red, hd + 2 * (mr + 2), s));
  DG_CUDA(cudaMemcpyAsync(m->hhost, hd, sizeof(double) * 3 * (mr + 2), cudaMemcpyDeviceToHost, s));
  return normalize_dev(w, hd + 2 * (mr + 2), n, s);
}

static constexpr size_t kMaxArnoldiGraphs = 2 * MAX_RESTART;

// Launch Arnoldi step k as one graph on s: captured on the mesh's own stream
// the first time its (k, restart, u, r_u, basis, preconditioner) set is seen,
// then replayed.  The graph bakes in pointers and launch shapes, which is why
// they form the key and why a new preconditioner sequence or launch tuning
// leads to a new capture.
static dg_status arnoldi_step_graph(dg_mesh_s* m, dg_precond_s* p, const double* u,
                                    const double* r_u, const double* dscal, double* V, int k,
                                    int mr, cudaStream_t s) {
  const unsigned long long pgen = p ? p->gen : 0;
  for (auto& g : m->agraphs)
    if (g.k == k && g.mr == mr && g.u == u && g.r_u == r_u && g.V == V && g.p == p && g.pgen == pgen) {
      __atomic_fetch_add(&g_launches, g.kernels, __ATOMIC_RELAXED);
      DG_CUDA(cudaGraphLaunch(g.exec, s));
      return DG_OK;
    }
  if (!m->gs) DG_CUDA(cudaStreamCreateWithFlags(&m->gs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  const long long before = dg_kernel_launches();
  DG_CUDA(cudaStreamBeginCapture(m->gs, cudaStreamCaptureModeThreadLocal));
  const dg_status st = arnoldi_step_ops(m, p, u, r_u, dscal, V, k, mr, m->gs);
  const long long kernels = dg_kernel_launches() - before;  // counted once, by the capture
  const cudaError_t ce = cudaStreamEndCapture(m->gs, &graph);
  if (st != DG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  DG_CUDA(ce);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  DG_CUDA(ie);
  if (m->agraphs.size() >= kMaxArnoldiGraphs) {
    cudaGraphExecDestroy(m->agraphs.front().exec);
    m->agraphs.erase(m->agraphs.begin());
  }
  m->agraphs.push_back({k, mr, u, r_u, V, p, pgen, exec, kernels});
  DG_CUDA(cudaGraphLaunch(exec, s));
  return DG_OK;
}

static dg_status gmres_impl(dg_mesh_s* m, dg_precond_s* p, const double* u, const double* r_u,
                            double t, double dta, const double* b, double* x,
                            const dg_gmres_cfg* cfg, dg_gmres_stats* st, cudaStream_t s) {
  const int mr = cfg->restart;
  const long long n = m->ndof;
  DG_TRY(ensure_krylov(m, mr));
  double* V = m->krylov;                       // (mr+1) vectors
  double* Z = p ? V + (size_t)(mr + 1) * n : nullptr;  // mr vectors
  dg_gmres_stats S{};
  double bn;
  DG_TRY(host_norm(m, b, &bn, s));
  S.res0 = bn;
  DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  if (bn == 0.0) {
    S.converged = 1;
    if (st) *st = S;
    return DG_OK;
  }
  const double tol = cfg->rtol * bn;
  std::vector<double> H((size_t)(mr + 1) * mr), cs(mr), sn(mr), g(mr + 1), y(mr);
  double* hd = m->hdev;
  double* hh = m->hhost;
  // graph replay of the Arnoldi steps; per-kernel profiling launches plainly
  const bool use_graph = cfg->graphs && !profiling_on();
  double* dscal = m->scratch + 24;
  if (use_graph) DG_TRY(set_scalars(dscal, t, -dta, s));
  for (int cyc = 0; cyc < cfg->max_cycles; ++cyc) {
    double beta;
    if (cyc == 0) {
      DG_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      beta = bn;
    } else {
      DG_TRY(apply_A(m, u, r_u, t, dta, x, m->w2, s));
      DG_TRY(lincomb(V, b, 1.0, m->w2, -1.0, n, s));
      DG_TRY(host_norm(m, V, &beta, s));
    }
    S.res = beta;
    if (beta <= tol) {
      S.converged = 1;
      break;
    }
    S.cycles++;
    DG_TRY(axpby(V, 1.0 / beta, V, 0.0, n, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kused = 0;
    bool done = false;
    for (int k = 0; k < mr; ++k) {
      double* w = V + (size_t)(k + 1) * n;
      if (use_graph) {
        DG_TRY(arnoldi_step_graph(m, p, u, r_u, dscal, V, k, mr, s));
      } else {
        const double* vk = V + (size_t)k * n;
        const double* zk = vk;
        if (p) {
          double* zz = Z + (size_t)k * n;
          DG_TRY(precond_apply_impl(p, vk, zz, s));
          zk = zz;
        }
        DG_TRY(apply_A(m, u, r_u, t, dta, zk, w, s));
        // classical Gram-Schmidt, applied twice
        DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd, s));
        DG_TRY(multi_axpy(w, V, k + 1, hd, n, s));
        DG_TRY(multi_dot(V, k + 1, w, n, m->red, hd + (mr + 2), s));
        DG_TRY(multi_axpy(w, V, k + 1, hd + (mr + 2), n, s));
        DG_TRY(dot(w, w, n, m->red, hd + 2 * (mr + 2), s));
        DG_CUDA(cudaMemcpyAsync(hh, hd, sizeof(double) * 3 * (mr + 2), cudaMemcpyDeviceToHost, s));
      }
      S.iters++;
      DG_CUDA(cudaStreamSynchronize(s));
      const double hn = std::sqrt(hh[2 * (mr + 2)]);
      if (!std::isfinite(hn)) return DG_ERR_NONFINITE;
      for (int i = 0; i <= k; ++i) H[(size_t)i * mr + k] = hh[i] + hh[(mr + 2) + i];
      H[(size_t)(k + 1) * mr + k] = hn;
      // (the graph normalised w on the device)
      if (!use_graph && hn > 0.0) DG_TRY(axpby(w, 1.0 / hn, w, 0.0, n, s));
      for (int i = 0; i < k; ++i) {
        double t0 = cs[i] * H[(size_t)i * mr + k] + sn[i] * H[(size_t)(i + 1) * mr + k];
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
    // x += sum_i y_i z_i  (multi_axpy subtracts: pass -y)
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

dg_status dg_gmres(dg_mesh_t m, dg_precond_t p, const double* u, const double* r_u, double t,
                   double dt_a, const double* b, double* x, const dg_gmres_cfg* cfg,
                   dg_gmres_stats* stats, void* stream) {
  if (!m || !u || !r_u || !b || !x || !cfg) return DG_ERR_ARG;
  if (cfg->restart < 1 || cfg->restart > MAX_RESTART || cfg->max_cycles < 1 || !(cfg->rtol > 0.0))
    return DG_ERR_ARG;
  if (p && precond_mesh(p) != m) return DG_ERR_ARG;
  return gmres_impl(m, p, u, r_u, t, dt_a, b, x, cfg, stats, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- SDIRK, BDF2
struct Tableau {
  int M;
  double A[DG_MAX_STAGES][DG_MAX_STAGES], b[DG_MAX_STAGES], c[DG_MAX_STAGES];
  double gdiag;  // the diagonal shared by the implicit stages
};

// Butcher tables of App. A (and backward Euler).  The six-stage fourth-order
// table is printed with symbols in its first column; each names the entry
// beside it (a_i0 = a_i1), the nodes are the row sums and the weights the
// last row (stiffly accurate).
static bool make_tableau(int which, Tableau& T) {
  std::memset(&T, 0, sizeof(T));
  if (which == DG_BE) {
    T.M = 1;
    T.A[0][0] = 1.0;
    T.b[0] = 1.0;
  } else if (which == DG_SDIRK2) {
    const double l = 1.0 - std::sqrt(2.0) / 2.0;
    T.M = 2;
    T.A[0][0] = l;
    T.A[1][0] = 1 - l;
    T.A[1][1] = l;
    T.b[0] = 1 - l;
    T.b[1] = l;
  } else if (which == DG_SDIRK3) {
    const double l = 0.4358665215;
    const double b1 = (-6 * l * l + 16 * l - 1) / 4, b2 = (6 * l * l - 20 * l + 5) / 4;
    T.M = 3;
    T.A[0][0] = l;
    T.A[1][0] = (1 - l) / 2;
    T.A[1][1] = l;
    T.A[2][0] = b1;
    T.A[2][1] = b2;
    T.A[2][2] = l;
    T.b[0] = b1;
    T.b[1] = b2;
    T.b[2] = l;
  } else if (which == DG_ESDIRK4) {
    const double r = std::sqrt(2.0);
    T.M = 6;
    T.A[1][1] = 0.25;
    T.A[2][1] = (1 - r) / 8;
    T.A[2][2] = 0.25;
    T.A[3][1] = (5 - 7 * r) / 64;
    T.A[3][2] = 7 * (1 + r) / 32;
    T.A[3][3] = 0.25;
    T.A[4][1] = (-13796 - 54539 * r) / 125000;
    T.A[4][2] = (506605 + 132109 * r) / 437500;
    T.A[4][3] = 166 * (-97 + 376 * r) / 109375;
    T.A[4][4] = 0.25;
    T.A[5][1] = (1181 - 987 * r) / 13782;
    T.A[5][2] = 47 * (-267 + 1783 * r) / 273343;
    T.A[5][3] = -16 * (-22922 + 3525 * r) / 571953;
    T.A[5][4] = -15625 * (97 + 376 * r) / 90749876;
    T.A[5][5] = 0.25;
    for (int i = 1; i < 6; ++i) T.A[i][0] = T.A[i][1];
    for (int j = 0; j < 6; ++j) T.b[j] = T.A[5][j];
  } else {
    return false;
  }
  for (int i = 0; i < T.M; ++i) {
    T.c[i] = 0;
    for (int j = 0; j <= i; ++j) T.c[i] += T.A[i][j];
    if (T.gdiag == 0.0) T.gdiag = T.A[i][i];
  }
  return true;
}

static dg_status check_step_cfg(const dg_sdirk_cfg* cfg) {
  if (cfg->gmres.restart < 1 || cfg->gmres.restart > MAX_RESTART || cfg->gmres.max_cycles < 1 ||
      !(cfg->gmres.rtol > 0.0) || cfg->max_newton < 0)
    return DG_ERR_ARG;
  return DG_OK;
}

// the step's device vectors: E^0..E^5, S, U, R, N and the learned guess's
// candidate U2, R2, N2
static dg_status step_buffers(dg_mesh_s* m, double** Ev, double** rest) {
  const size_t n = (size_t)m->ndof;
  if (!m->stage) {
    DG_CUDA(cudaMalloc(&m->stage, sizeof(double) * n * (DG_MAX_STAGES + 7)));
    DG_CUDA(cudaMemset(m->stage, 0, sizeof(double) * n * (DG_MAX_STAGES + 7)));
  }
  for (int i = 0; i < DG_MAX_STAGES; ++i) Ev[i] = m->stage + i * n;
  for (int i = 0; i < 7; ++i) rest[i] = m->stage + (DG_MAX_STAGES + i) * n;
  return DG_OK;
}

struct StageResult {
  int it = 0, gits = 0;
  double res0 = 0.0, res = 0.0;
  bool conv = false;
  int guess_used = 0;
};

// Newton (Eq. Newton-Iteration) on N(u) = u - S - dta R(u, ti) from u = S, or
// from the learned guess of stage gstage when it lowers ||N||; stops at
// ||N|| < alpha ||N(S)|| (abs_tol instead when > 0; an absolute number in
// every case once a guess is in use).  On return U holds the iterate, R its
// residual R(U, ti) and N = N(U) (the candidate buffers may have been swapped
// in).
static dg_status newton_stage(dg_mesh_s* m, const dg_sdirk_cfg* cfg, dg_precond_s* P,
                              dg_guess_s* G, int gstage, const double* Sv, double ti, double dta,
                              double*& U, double*& R, double*& Nn, double*& U2, double*& R2,
                              double*& N2, StageResult* out, cudaStream_t s) {
  const long long n = m->ndof;
  double* dx = m->w1;
  StageResult o;
  DG_CUDA(cudaMemcpyAsync(U, Sv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_TRY(dg_residual(m, U, ti, R, s));
  DG_TRY(newton_resid(Nn, U, Sv, R, dta, n, s));
  double res;
  DG_TRY(host_norm(m, Nn, &res, s));
  o.res0 = res;
  const double tol = cfg->abs_tol > 0.0 ? cfg->abs_tol : cfg->alpha * o.res0;
  // with a learned guess the criterion stays alpha ||N(S)||, as an absolute tolerance
  const bool abs_mode = cfg->abs_tol > 0.0 || G != nullptr;
  if (G) {
    int ready = 0;
    DG_TRY(dg_guess_ready(G, gstage, &ready));
    if (ready) {
      DG_TRY(dg_guess_predict(G, gstage, Sv, U2, s));
      DG_TRY(dg_residual(m, U2, ti, R2, s));
      DG_TRY(newton_resid(N2, U2, Sv, R2, dta, n, s));
      double resc;
      const dg_status ns = host_norm(m, N2, &resc, s);
      if (ns != DG_OK && ns != DG_ERR_NONFINITE) return ns;
      // a non-finite candidate (e.g. a predicted state without positive
      // density) is rejected like any guess that does not lower ||N||
      if (ns == DG_OK && resc < o.res0) {
        std::swap(U, U2);
        std::swap(R, R2);
        std::swap(Nn, N2);
        res = resc;
        o.guess_used = 1;
      }
    }
  }
  while (true) {
    if (res <= 0.0 || ((o.it > 0 || abs_mode) && res < tol)) {
      o.conv = true;
      break;
    }
    if (o.it >= cfg->max_newton) break;
    dg_gmres_stats gs{};
    dg_status g = gmres_impl(m, P, U, R, ti, dta, Nn, dx, &cfg->gmres, &gs, s);
    if (g != DG_OK && g != DG_ERR_NOT_CONVERGED) return g;
    o.gits += gs.iters;
    DG_TRY(axpby(U, 1.0, dx, 1.0, n, s));
    ++o.it;
    DG_TRY(dg_residual(m, U, ti, R, s));
    DG_TRY(newton_resid(Nn, U, Sv, R, dta, n, s));
    DG_TRY(host_norm(m, Nn, &res, s));
  }
  o.res = res;
  *out = o;
  return DG_OK;
}

static void record_stage(dg_step_stats& st, int i, const StageResult& o) {
  st.newton_iters += o.it;
  st.gmres_iters += o.gits;
  st.guess_used += o.guess_used;
  if (i < DG_MAX_STAGES) {
    st.stage_newton[i] = o.it;
    st.stage_gmres[i] = o.gits;
    st.stage_res0[i] = o.res0;
    st.stage_res[i] = o.res;
  }
}

dg_status sdirk_step(dg_mesh_t m, const dg_sdirk_cfg* cfg, double* u_n, double t, double dt,
                     dg_precond_t* p_inout, dg_step_stats* stats, void* stream) {
  if (!m || !cfg || !u_n || !(dt > 0.0)) return DG_ERR_ARG;
  Tableau T;
  if (!make_tableau(cfg->tableau, T)) return DG_ERR_ARG;
  if (cfg->use_precond && !p_inout) return DG_ERR_ARG;
  DG_TRY(check_step_cfg(cfg));
  dg_guess_s* G = cfg->guess;
  // the learned guess keeps one network per stage, at most four; the explicit
  // first stage of the fourth-order scheme would shift the stage indices
  if (G && (T.M > guess_stage_count(G) || T.A[0][0] == 0.0)) return DG_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = m->ndof;
  double *Ev[DG_MAX_STAGES], *B[7];
  DG_TRY(step_buffers(m, Ev, B));
  double *Sv = B[0], *U = B[1], *R = B[2], *Nn = B[3], *U2 = B[4], *R2 = B[5], *N2 = B[6];
  dg_step_stats st{};
  st.stages = T.M;
  dg_precond_s* P = nullptr;
  if (cfg->use_precond) {
    // every implicit stage shares the diagonal a_mm, hence one preconditioner
    if (!*p_inout || cfg->rebuild) {
      DG_TRY(dg_precond_build(m, u_n, t, dt * T.gdiag, &cfg->prec, p_inout, s));
      st.precond_built = 1;
    }
    P = *p_inout;
  }
  dg_status result = DG_OK;
  if (G && guess_history_empty(G)) DG_TRY(dg_guess_push(G, u_n, s));
  for (int i = 0; i < T.M; ++i) {
    // S_i = u^n + sum_{j<i} a_ij E^j
    DG_CUDA(cudaMemcpyAsync(Sv, u_n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < i; ++j) DG_TRY(axpby(Sv, T.A[i][j], Ev[j], 1.0, n, s));
    const double ti = t + T.c[i] * dt, dta = dt * T.A[i][i];
    StageResult o;
    if (dta == 0.0) {
      // explicit stage: u^i = S_i
      DG_TRY(dg_residual(m, Sv, ti, R, s));
      o.conv = true;
    } else {
      DG_TRY(newton_stage(m, cfg, P, G, i, Sv, ti, dta, U, R, Nn, U2, R2, N2, &o, s));
    }
    if (!o.conv) result = DG_ERR_NOT_CONVERGED;
    record_stage(st, i, o);
    // E^i = dt R(u^i) from the residual of the converged iterate
    DG_TRY(axpby(Ev[i], dt, R, 0.0, n, s));
    // the converged stage trains the stage's network (needs a full history)
    // (and its increment becomes the extrapolation base of the next step)
    if (G && o.conv)
      DG_TRY(dg_guess_train(G, i, Sv, U, cfg->guess_train_iters, nullptr, nullptr, nullptr, s));
  }
  for (int i = 0; i < T.M; ++i) DG_TRY(axpby(u_n, T.b[i], Ev[i], 1.0, n, s));
  if (G) DG_TRY(dg_guess_push(G, u_n, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (stats) *stats = st;
  return result;
}

dg_status bdf2_step(dg_mesh_t m, const dg_sdirk_cfg* cfg, double* u_n, double* u_prev, double t,
                    double dt, dg_precond_t* p_inout, dg_step_stats* stats, void* stream) {
  if (!m || !cfg || !u_n || !u_prev || u_n == u_prev || !(dt > 0.0)) return DG_ERR_ARG;
  if (cfg->use_precond && !p_inout) return DG_ERR_ARG;
  if (cfg->guess) return DG_ERR_UNSUPPORTED;
  DG_TRY(check_step_cfg(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = m->ndof;
  double *Ev[DG_MAX_STAGES], *B[7];
  DG_TRY(step_buffers(m, Ev, B));
  double *Sv = B[0], *U = B[1], *R = B[2], *Nn = B[3], *U2 = B[4], *R2 = B[5], *N2 = B[6];
  const double dta = 2.0 * dt / 3.0;
  dg_step_stats st{};
  st.stages = 1;
  dg_precond_s* P = nullptr;
  if (cfg->use_precond) {
    if (!*p_inout || cfg->rebuild) {
      DG_TRY(dg_precond_build(m, u_n, t, dta, &cfg->prec, p_inout, s));
      st.precond_built = 1;
    }
    P = *p_inout;
  }
  // S = (4 u^n - u^{n-1}) / 3
  DG_TRY(lincomb(Sv, u_n, 4.0 / 3.0, u_prev, -1.0 / 3.0, n, s));
  StageResult o;
  DG_TRY(newton_stage(m, cfg, P, nullptr, 0, Sv, t + dt, dta, U, R, Nn, U2, R2, N2, &o, s));
  record_stage(st, 0, o);
  DG_CUDA(cudaMemcpyAsync(u_prev, u_n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaMemcpyAsync(u_n, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (stats) *stats = st;
  return o.conv ? DG_OK : DG_ERR_NOT_CONVERGED;
}

}  // extern "C"
