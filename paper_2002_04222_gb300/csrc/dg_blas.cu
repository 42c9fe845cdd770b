// Dense FP64 vector kernels of the Krylov/Newton layer.  Reductions use a
// fixed grid (RED_BLOCKS blocks, fixed per-block chunks, fixed-shape trees)
// so that every norm and dot product repeats bitwise from run to run.
#include "dg_internal.h"

namespace dg {

constexpr int RT = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// partial[b] = sum over chunk b of a*b  (nvec independent pairs at stride)
__global__ void __launch_bounds__(RT) dot_partial_kernel(const double* __restrict__ a,
                                                         const double* __restrict__ b,
                                                         long long n, double* __restrict__ partial) {
  __shared__ double sh[RT];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += RT) s = fma(a[i], b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RT) finish_kernel(const double* __restrict__ partial, int np,
                                                    int nsum, double* __restrict__ out) {
  // out[j] = sum_b partial[j*np + b] for j < nsum (one block per j)
  __shared__ double sh[RT];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += RT) s += partial[(long long)j * np + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0 && j < nsum) out[j] = s;
}

dg_status dot(const double* a, const double* b, long long n, double* partial, double* out,
              cudaStream_t s) {
  DG_PROF(K_DOT, s, dot_partial_kernel<<<RED_BLOCKS, RT, 0, s>>>(a, b, n, partial));
  DG_PROF(K_DOT, s, finish_kernel<<<1, RT, 0, s>>>(partial, RED_BLOCKS, 1, out));
  DG_LAUNCHED(2);
  return DG_OK;
}

dg_status finish_sum(const double* partial, int np, double* out, cudaStream_t s) {
  finish_kernel<<<1, RT, 0, s>>>(partial, np, 1, out);
  DG_LAUNCHED(1);
  return DG_OK;
}

// partial[i*RED_BLOCKS + b] = chunk-b part of V_i . w for i in [8*blockIdx.y, +8)
__global__ void __launch_bounds__(RT) multi_dot_kernel(const double* __restrict__ V, int k,
                                                       const double* __restrict__ w, long long n,
                                                       double* __restrict__ partial) {
  __shared__ double sh[RT];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  const int i0 = blockIdx.y * 8;
  double acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0;
  for (long long x = lo + threadIdx.x; x < hi; x += RT) {
    const double wx = w[x];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i0 + j < k) acc[j] = fma(V[(long long)(i0 + j) * n + x], wx, acc[j]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const double s = block_sum(acc[j], sh);
    if (threadIdx.x == 0 && i0 + j < k) partial[(long long)(i0 + j) * gridDim.x + blockIdx.x] = s;
  }
}

dg_status multi_dot(const double* V, int k, const double* w, long long n, double* partial,
                    double* out, cudaStream_t s) {
  dim3 grid(RED_BLOCKS, (k + 7) / 8);
  DG_PROF(K_MULTIDOT, s, multi_dot_kernel<<<grid, RT, 0, s>>>(V, k, w, n, partial));
  DG_PROF(K_MULTIDOT, s, finish_kernel<<<k, RT, 0, s>>>(partial, RED_BLOCKS, k, out));
  DG_LAUNCHED(2);
  return DG_OK;
}

// w -= sum_i h_i V_i
__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, int k,
                                  const double* __restrict__ h, long long n) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    double acc = w[x];
    for (int i = 0; i < k; ++i) acc = fma(-h[i], V[(long long)i * n + x], acc);
    w[x] = acc;
  }
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

dg_status multi_axpy(double* w, const double* V, int k, const double* h, long long n,
                     cudaStream_t s) {
  DG_PROF(K_MULTIAXPY, s, multi_axpy_kernel<<<grid_for(n), 256, 0, s>>>(w, V, k, h, n));
  DG_LAUNCHED(1);
  return DG_OK;
}

// y = a x + b y; with b = 0, y is output only and is not read (a fresh
// buffer may hold anything, and 0 * NaN is NaN).  x may be y (scaling in
// place), hence no __restrict__.
__global__ void axpby_kernel(double* y, double a, const double* x, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);
}
dg_status axpby(double* y, double a, const double* x, double b, long long n, cudaStream_t s) {
  DG_PROF(K_VEC, s, axpby_kernel<<<grid_for(n), 256, 0, s>>>(y, a, x, b, n));
  DG_LAUNCHED(1);
  return DG_OK;
}

__global__ void lincomb_kernel(double* __restrict__ y, const double* __restrict__ x, double a,
                               const double* __restrict__ z, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * z[i]);
}
dg_status lincomb(double* y, const double* x, double a, const double* z, double b, long long n,
                  cudaStream_t s) {
  DG_PROF(K_VEC, s, lincomb_kernel<<<grid_for(n), 256, 0, s>>>(y, x, a, z, b, n));
  DG_LAUNCHED(1);
  return DG_OK;
}

// y = x * s or x / s with s a device scalar (the reciprocal formed once per
// block: an FP64 division per thread would cost more than the stream)
__global__ void scale_dev_kernel(double* __restrict__ y, const double* __restrict__ x,
                                 const double* __restrict__ sdev, int inv, long long n) {
  __shared__ double ss;
  if (threadIdx.x == 0) ss = inv ? 1.0 / sdev[0] : sdev[0];
  __syncthreads();
  const double s = ss;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}
dg_status scale_dev(double* y, const double* x, const double* sdev, int inv, long long n,
                    cudaStream_t s) {
  scale_dev_kernel<<<grid_for(n), 256, 0, s>>>(y, x, sdev, inv, n);
  DG_LAUNCHED(1);
  return DG_OK;
}

// eps = sqrt(2^-52) ||u|| / ||v|| (sqrt(2^-52)/||v|| when u = 0); eps = 0 when v = 0
__global__ void eps_finish_kernel(const double* __restrict__ partial, double* __restrict__ eps) {
  __shared__ double sh[RT];
  double su = 0.0, sv = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += RT) {
    su += partial[i];
    sv += partial[RED_BLOCKS + i];
  }
  su = block_sum(su, sh);
  sv = block_sum(sv, sh);
  if (threadIdx.x == 0) {
    const double nu = sqrt(su), nv = sqrt(sv);
    const double e = nv > 0.0 ? 1.4901161193847656e-08 * (nu > 0.0 ? nu : 1.0) / nv : 0.0;
    eps[0] = e;
    eps[1] = e > 0.0 ? 1.0 / e : 0.0;
    eps[2] = nu;
    eps[3] = nv;
  }
}

dg_status jvp_eps(const double* u, const double* v, long long n, double* partial, double* eps,
                  cudaStream_t s) {
  DG_PROF(K_DOT, s, dot_partial_kernel<<<RED_BLOCKS, RT, 0, s>>>(u, u, n, partial));
  DG_PROF(K_DOT, s, dot_partial_kernel<<<RED_BLOCKS, RT, 0, s>>>(v, v, n, partial + RED_BLOCKS));
  DG_PROF(K_DOT, s, eps_finish_kernel<<<1, RT, 0, s>>>(partial, eps));
  DG_LAUNCHED(3);
  return DG_OK;
}

// Nneg = S + dta R - u  (= -N(u) of Eq. nonlinear-equation-system)
__global__ void newton_resid_kernel(double* __restrict__ Nn, const double* __restrict__ u,
                                    const double* __restrict__ S, const double* __restrict__ R,
                                    double dta, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    Nn[i] = fma(dta, R[i], S[i]) - u[i];
}
dg_status newton_resid(double* N, const double* u, const double* S, const double* R, double dta,
                       long long n, cudaStream_t s) {
  DG_PROF(K_VEC, s, newton_resid_kernel<<<grid_for(n), 256, 0, s>>>(N, u, S, R, dta, n));
  DG_LAUNCHED(1);
  return DG_OK;
}

__global__ void set_scalars_kernel(double* __restrict__ d, double a, double b) {
  d[0] = a;
  d[1] = b;
}
dg_status set_scalars(double* d, double a, double b, cudaStream_t s) {
  DG_PROF(K_VEC, s, set_scalars_kernel<<<1, 1, 0, s>>>(d, a, b));
  DG_LAUNCHED(1);
  return DG_OK;
}

// the Arnoldi normalisation with the norm read on the device: h = sqrt(*hsq),
// w = (1/h) w + 0 w as axpby_kernel forms it, skipped when h is 0 or not finite
__global__ void normalize_dev_kernel(double* __restrict__ w, const double* __restrict__ hsq,
                                     long long n) {
  __shared__ double sa;  // 1/h once per block (FP64 sqrt and division are long sequences)
  if (threadIdx.x == 0) {
    const double h = sqrt(hsq[0]);
    sa = (h > 0.0 && isfinite(h)) ? 1.0 / h : 0.0;
  }
  __syncthreads();
  const double a = sa;
  if (a == 0.0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = fma(a, w[i], 0.0 * w[i]);
}
dg_status normalize_dev(double* w, const double* hsq, long long n, cudaStream_t s) {
  DG_PROF(K_VEC, s, normalize_dev_kernel<<<grid_for(n), 256, 0, s>>>(w, hsq, n));
  DG_LAUNCHED(1);
  return DG_OK;
}

}  // namespace dg
