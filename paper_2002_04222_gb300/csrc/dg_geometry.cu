// Geometry of general (curved or non-axis-aligned) elements, Sec. 3.1: the
// isoparametric map of each element from its (g+1)^d equispaced nodes (g = 1
// straight-sided, g = 2 quadratic), evaluated once per mesh on the device:
//   vgeo  d xi_r / d x_j and w_q |J| at every volume Gauss point,
//   vx    the physical coordinates of those points,
//   fgeo  d xi_r / d x_j at every face point of every element face,
//   fdat  per face (owner side): outward unit normal n, w^G J^G and x,
//   fbeta the penalty (P+1)^2 / h with h = min over the two sides of
//         |Omega_e| / |Gamma_f|,
//   minv  the inverse of the dense element mass matrix B^T diag(w|J|) B.
// Normals and surface Jacobians follow Nanson's formula n dA = |J| grad xi_r dA_ref.
#include <cmath>
#include <vector>
#include "dg_internal.h"

namespace dg {

// 1-D Lagrange shape functions of order G on the equispaced nodes of [-1, 1]
template <int G>
__device__ __forceinline__ void shape1d(double x, double* N, double* dN) {
  if (G == 1) {
    N[0] = 0.5 * (1.0 - x);
    N[1] = 0.5 * (1.0 + x);
    dN[0] = -0.5;
    dN[1] = 0.5;
  } else {
    N[0] = 0.5 * x * (x - 1.0);
    N[1] = 1.0 - x * x;
    N[2] = 0.5 * x * (x + 1.0);
    dN[0] = x - 0.5;
    dN[1] = -2.0 * x;
    dN[2] = x + 0.5;
  }
}

// x(xi) and J[i][r] = d x_i / d xi_r of element nodes X[a][i]
template <int D, int G>
__device__ void map_point(const double* __restrict__ X, const double* xi, double* x,
                          double J[D][D]) {
  constexpr int NA = G + 1;
  double N[D][NA], dN[D][NA];
#pragma unroll
  for (int r = 0; r < D; ++r) shape1d<G>(xi[r], N[r], dN[r]);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    x[i] = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) J[i][r] = 0.0;
  }
  constexpr int NN = D == 2 ? NA * NA : NA * NA * NA;
  for (int a = 0; a < NN; ++a) {
    const int a0 = a % NA, a1 = (a / NA) % NA, a2 = D == 3 ? a / (NA * NA) : 0;
    const int ai[3] = {a0, a1, a2};
    double v = 1.0, dv[D];
#pragma unroll
    for (int r = 0; r < D; ++r) v *= N[r][ai[r]];
#pragma unroll
    for (int s = 0; s < D; ++s) {
      double p = dN[s][ai[s]];
#pragma unroll
      for (int r = 0; r < D; ++r)
        if (r != s) p *= N[r][ai[r]];
      dv[s] = p;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double xa = X[a * D + i];
      x[i] = fma(v, xa, x[i]);
#pragma unroll
      for (int s = 0; s < D; ++s) J[i][s] = fma(dv[s], xa, J[i][s]);
    }
  }
}

// det J and the inverse metric ginv[r][j] = d xi_r / d x_j
template <int D>
__device__ double invert_jacobian(const double J[D][D], double ginv[D][D]) {
  if (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double id = 1.0 / det;
    ginv[0][0] = J[1][1] * id;
    ginv[0][1] = -J[0][1] * id;
    ginv[1][0] = -J[1][0] * id;
    ginv[1][1] = J[0][0] * id;
    return det;
  }
  // cofactors: ginv = adj(J) / det
  double c[3][3];
  c[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  c[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  c[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  c[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  c[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  c[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  c[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  c[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  c[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * c[0][0] + J[0][1] * c[1][0] + J[0][2] * c[2][0];
  const double id = 1.0 / det;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int j = 0; j < 3; ++j) ginv[r][j] = c[r][j] * id;
  return det;
}

// reference coordinates of face point p of local face lf (the tangential
// Gauss indices in the order of the trace buffers)
template <int D>
__device__ __forceinline__ void face_xi(const Tables& tab, int Q, int lf, int p, double* xi,
                                        double* wf) {
  const int r = lf >> 1;
  int c[3] = {0, 0, 0};
  if (D == 2) {
    c[1 - r] = p;
  } else {
    const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
    c[t0] = p % Q;
    c[t1] = p / Q;
  }
  double w = 1.0;
#pragma unroll
  for (int s = 0; s < D; ++s) {
    if (s == r) {
      xi[s] = (lf & 1) ? 1.0 : -1.0;
    } else {
      xi[s] = tab.x[c[s]];
      w *= tab.w[c[s]];
    }
  }
  *wf = w;
}

template <int D, int G>
__global__ void geo_volume_kernel(const __grid_constant__ Tables tab, int Q, int E,
                                  const double* __restrict__ nodes, double* __restrict__ vgeo,
                                  double* __restrict__ vx, int* __restrict__ fail) {
  constexpr int NN = D == 2 ? (G + 1) * (G + 1) : (G + 1) * (G + 1) * (G + 1);
  const int NQ = D == 2 ? Q * Q : Q * Q * Q;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)E * NQ) return;
  const int e = (int)(idx / NQ), q = (int)(idx - (long long)e * NQ);
  const int c[3] = {q % Q, (q / Q) % Q, D == 3 ? q / (Q * Q) : 0};
  double xi[D], x[D], J[D][D], gi[D][D];
  double w = 1.0;
#pragma unroll
  for (int r = 0; r < D; ++r) {
    xi[r] = tab.x[c[r]];
    w *= tab.w[c[r]];
  }
  map_point<D, G>(nodes + (long long)e * NN * D, xi, x, J);
  const double det = invert_jacobian<D>(J, gi);
  if (!(det > 0.0)) atomicOr(fail, 1);
  double* g = vgeo + (long long)e * (D * D + 1) * NQ + q;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int j = 0; j < D; ++j) g[(r * D + j) * NQ] = gi[r][j];
  g[D * D * NQ] = w * det;
#pragma unroll
  for (int i = 0; i < D; ++i) vx[((long long)e * D + i) * NQ + q] = x[i];
}

template <int D, int G>
__global__ void geo_face_points_kernel(const __grid_constant__ Tables tab, int Q, int E,
                                       const double* __restrict__ nodes,
                                       double* __restrict__ fgeo, int* __restrict__ fail) {
  constexpr int NN = D == 2 ? (G + 1) * (G + 1) : (G + 1) * (G + 1) * (G + 1);
  const int NF = D == 2 ? Q : Q * Q;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)E * 2 * D * NF) return;
  const int p = (int)(idx % NF);
  const int lf = (int)((idx / NF) % (2 * D));
  const int e = (int)(idx / ((long long)NF * 2 * D));
  double xi[D], x[D], J[D][D], gi[D][D], wf;
  face_xi<D>(tab, Q, lf, p, xi, &wf);
  map_point<D, G>(nodes + (long long)e * NN * D, xi, x, J);
  const double det = invert_jacobian<D>(J, gi);
  if (!(det > 0.0)) atomicOr(fail, 1);
  double* g = fgeo + ((long long)e * 2 * D + lf) * D * D * NF + p;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int j = 0; j < D; ++j) g[(r * D + j) * NF] = gi[r][j];
}

// owner-side normal, surface weight and coordinates of every face point
template <int D, int G>
__global__ void geo_face_data_kernel(const __grid_constant__ Tables tab, int Q, int F,
                                     const int32_t* __restrict__ faces,
                                     const double* __restrict__ nodes,
                                     double* __restrict__ fdat) {
  constexpr int NN = D == 2 ? (G + 1) * (G + 1) : (G + 1) * (G + 1) * (G + 1);
  const int NF = D == 2 ? Q : Q * Q;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)F * NF) return;
  const int f = (int)(idx / NF), p = (int)(idx - (long long)f * NF);
  const int eL = faces[f * 6 + 0], fL = faces[f * 6 + 1];
  const int r = fL >> 1;
  double xi[D], x[D], J[D][D], gi[D][D], wf;
  face_xi<D>(tab, Q, fL, p, xi, &wf);
  map_point<D, G>(nodes + (long long)eL * NN * D, xi, x, J);
  const double det = invert_jacobian<D>(J, gi);
  double mag = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) mag += gi[r][j] * gi[r][j];
  mag = sqrt(mag);
  const double sgn = (fL & 1) ? 1.0 : -1.0;
  double* o = fdat + (long long)f * (2 * D + 1) * NF + p;
#pragma unroll
  for (int j = 0; j < D; ++j) o[j * NF] = sgn * gi[r][j] / mag;
  o[D * NF] = wf * fabs(det) * mag;
#pragma unroll
  for (int j = 0; j < D; ++j) o[(D + 1 + j) * NF] = x[j];
}

// |Omega_e| = sum_q w|J|
__global__ void elem_volume_kernel(const double* __restrict__ vgeo, int E, int D, int NQ,
                                   double* __restrict__ vol) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double* w = vgeo + (long long)e * (D * D + 1) * NQ + (long long)D * D * NQ;
  double s = 0.0;
  for (int q = 0; q < NQ; ++q) s += w[q];
  vol[e] = s;
}

// beta_p = (P+1)^2 / min(|Omega_L|, |Omega_R|) |Gamma_f|
__global__ void face_beta_kernel(const int32_t* __restrict__ faces, int F, int D, int NF, int P,
                                 const double* __restrict__ vol, const double* __restrict__ fdat,
                                 double* __restrict__ beta) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double* w = fdat + (long long)f * (2 * D + 1) * NF + (long long)D * NF;
  double area = 0.0;
  for (int p = 0; p < NF; ++p) area += w[p];
  const int eL = faces[f * 6 + 0], eR = faces[f * 6 + 2];
  double h = vol[eL] / area;
  if (eR >= 0) h = fmin(h, vol[eR] / area);
  beta[f] = (double)((P + 1) * (P + 1)) / h;
}

// M_e = B^T diag(w|J|) B assembled and inverted (Gauss-Jordan, SPD: no
// pivoting needed) in shared memory, one block per element
__global__ void __launch_bounds__(256) mass_inverse_kernel(const __grid_constant__ Tables tab,
                                                           int D, int Q, int E,
                                                           const double* __restrict__ vgeo,
                                                           double* __restrict__ minv,
                                                           int* __restrict__ fail) {
  extern __shared__ double sm[];
  const int n = tab.n;
  const int NM = D == 2 ? n * n : n * n * n;
  const int NQ = D == 2 ? Q * Q : Q * Q * Q;
  double* A = sm;              // [NM][NM]
  double* wq = A + NM * NM;    // [NQ]
  double* col = wq + NQ;       // [NM]
  __shared__ double piv;
  const int e = blockIdx.x;
  const double* wJ = vgeo + (long long)e * (D * D + 1) * NQ + (long long)D * D * NQ;
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) wq[q] = wJ[q];
  __syncthreads();
  for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
    const int a = i / NM, b = i % NM;
    const int am[3] = {a % n, (a / n) % n, D == 3 ? a / (n * n) : 0};
    const int bm[3] = {b % n, (b / n) % n, D == 3 ? b / (n * n) : 0};
    double s = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const int c[3] = {q % Q, (q / Q) % Q, D == 3 ? q / (Q * Q) : 0};
      double v = wq[q];
      for (int r = 0; r < D; ++r) v *= tab.B[c[r] * n + am[r]] * tab.B[c[r] * n + bm[r]];
      s += v;
    }
    A[i] = s;
  }
  __syncthreads();
  for (int k = 0; k < NM; ++k) {
    if (threadIdx.x == 0) {
      piv = A[k * NM + k];
      if (!(piv > 0.0)) atomicOr(fail, 2);
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int j = threadIdx.x; j < NM; j += blockDim.x) {
      A[k * NM + j] = (j == k ? 1.0 : A[k * NM + j]) * ip;
      col[j] = A[j * NM + k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
      const int a = i / NM, b = i % NM;
      if (a == k) continue;
      const double f = col[a];
      A[i] = (b == k ? 0.0 : A[i]) - f * A[k * NM + b];
    }
    __syncthreads();
  }
  double* out = minv + (long long)e * NM * NM;
  for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) out[i] = A[i];
}

template <int D, int G>
static void launch_geometry(dg_mesh_s* m, const double* nodes, int* fail, cudaStream_t s) {
  const int Q = m->Q;
  const long long nv = (long long)m->E * m->nq, nf = (long long)m->E * 2 * D * m->nf;
  geo_volume_kernel<D, G><<<(unsigned)((nv + 127) / 128), 128, 0, s>>>(m->tab, Q, m->E, nodes,
                                                                         m->vgeo, m->vx, fail);
  geo_face_points_kernel<D, G><<<(unsigned)((nf + 127) / 128), 128, 0, s>>>(m->tab, Q, m->E,
                                                                              nodes, m->fgeo, fail);
  const long long nff = (long long)m->F * m->nf;
  geo_face_data_kernel<D, G><<<(unsigned)((nff + 127) / 128), 128, 0, s>>>(m->tab, Q, m->F,
                                                                             m->faces, nodes, m->fdat);
}

dg_status build_general_geometry(dg_mesh_s* m, const double* nodes_host, int g, cudaStream_t s) {
  const int D = m->dim, E = m->E, F = m->F;
  const int na = g == 1 ? (1 << D) : (D == 2 ? 9 : 27);
  const size_t nn = (size_t)E * na * D;
  double* nodes = nullptr;
  double* vol = nullptr;
  int* fail = nullptr;
  cudaError_t err = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc(ptr, bytes);
    if (err == cudaSuccess) err = cudaMemsetAsync(*ptr, 0, bytes, s);
  };
  alloc((void**)&m->vgeo, sizeof(double) * (size_t)E * (D * D + 1) * m->nq);
  alloc((void**)&m->vx, sizeof(double) * (size_t)E * D * m->nq);
  alloc((void**)&m->fgeo, sizeof(double) * (size_t)E * 2 * D * D * D * m->nf);
  alloc((void**)&m->fdat, sizeof(double) * (size_t)F * (2 * D + 1) * m->nf);
  alloc((void**)&m->fbeta, sizeof(double) * (size_t)F);
  alloc((void**)&m->minv, sizeof(double) * (size_t)E * m->nm * m->nm);
  alloc((void**)&nodes, sizeof(double) * nn);
  alloc((void**)&vol, sizeof(double) * (size_t)E);
  alloc((void**)&fail, sizeof(int));
  if (err == cudaSuccess) err = cudaMemcpyAsync(nodes, nodes_host, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(fail, 0, sizeof(int), s);
  dg_status st = err == cudaSuccess ? DG_OK : cuda_status(err);
  int hfail = 0;
  if (st == DG_OK) {
    if (D == 2 && g == 1) launch_geometry<2, 1>(m, nodes, fail, s);
    if (D == 2 && g == 2) launch_geometry<2, 2>(m, nodes, fail, s);
    if (D == 3 && g == 1) launch_geometry<3, 1>(m, nodes, fail, s);
    if (D == 3 && g == 2) launch_geometry<3, 2>(m, nodes, fail, s);
    elem_volume_kernel<<<(E + 127) / 128, 128, 0, s>>>(m->vgeo, E, D, m->nq, vol);
    face_beta_kernel<<<(F + 127) / 128, 128, 0, s>>>(m->faces, F, D, m->nf, m->P, vol, m->fdat,
                                                     m->fbeta);
    const size_t sm = sizeof(double) * ((size_t)m->nm * m->nm + m->nq + m->nm);
    err = cudaFuncSetAttribute(mass_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
    if (err == cudaSuccess) {
      mass_inverse_kernel<<<E, 256, sm, s>>>(m->tab, D, m->Q, E, m->vgeo, m->minv, fail);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) st = cuda_status(err);
  }
  cudaFree(nodes);
  cudaFree(vol);
  cudaFree(fail);
  if (st == DG_OK && hfail) st = DG_ERR_ARG;  // inverted element or singular mass matrix
  return st;
}

}  // namespace dg
