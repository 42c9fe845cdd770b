// Learned Newton initial guess (the plain guess of Sec. 3.2,
// Eq. Newton-initial-guess, is S_m): the stage increment u^m - S_m is
// extrapolated from the same stage of the previous step, d_prev, and a
// per-element MLP per stage, trained online on the converged stages with Adam,
// predicts the remaining correction.
//
//   features  x_e = [u^n/s0, (u^n-u^{n-1})/s1, d_prev/s2]  (BF16)
//   network   a1 = tanh(x W1 + b1), a2 = tanh(a1 W2 + b2), y = a2 W3 + b3
//   guess     S_m + d_prev + y (x) tau_m   (mlp = 0: S_m + d_prev)
// Every product takes BF16 operands and accumulates in FP32 (gemm_kernel);
// master parameters and Adam moments are FP32; weight gradients use a
// deterministic split-K reduction.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include <cuda_bf16.h>
#include "dg_internal.h"

namespace dg {

typedef __nv_bfloat16 bf16;

enum { EPI_NONE = 0, EPI_TANH = 1, EPI_DTANH = 2 };

// C = op(A) op(B) (+ bias) with epilogue; row-major storage.
//   A: TA ? [K][lda] (use its transpose) : [M][lda];  B: TB ? [N][ldb] : [K][ldb]
// gridDim.z > 1: split-K, block z covers k in [z*kc, (z+1)*kc) and writes the
// partial product to C + z*M*ldc (no epilogue).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const bf16* __restrict__ A,
                                                   int lda, const bf16* __restrict__ B, int ldb,
                                                   const float* __restrict__ bias,
                                                   const float* __restrict__ aux,
                                                   float* __restrict__ C, bf16* __restrict__ Cb,
                                                   int ldc, int kc) {
  constexpr int BM = 64, BN = 64, BK = 32;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kc, kend = min(K, kbeg + kc);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int i = threadIdx.x; i < BM * BK; i += 256) {
      int mm, kk;
      if (TA) {  // consecutive threads along m (contiguous in memory)
        mm = i % BM;
        kk = i / BM;
      } else {
        kk = i % BK;
        mm = i / BK;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = __bfloat162float(TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]);
      As[kk][mm] = v;
    }
    for (int i = threadIdx.x; i < BN * BK; i += 256) {
      int nn, kk;
      if (TB) {
        kk = i % BK;
        nn = i / BK;
      } else {
        nn = i % BN;
        kk = i / BN;
      }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < kend) v = __bfloat162float(TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* Cz = C + (long long)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (gridDim.z == 1) {
        if (bias) v += bias[n];
        if (EPI == EPI_TANH) v = tanhf(v);
        if (EPI == EPI_DTANH) {
          const float a = aux[(long long)m * ldc + n];
          v *= 1.f - a * a;
        }
        if (Cb) Cb[(long long)m * ldc + n] = __float2bfloat16_rn(v);
      }
      Cz[(long long)m * ldc + n] = v;
    }
  }
}

// out[i] = sum_z part[z][i] in order (deterministic split-K reduction)
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int nz, long long n,
                                     float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[(long long)z * n + i];
    out[i] = s;
  }
}

// column sums of a [M][N] matrix (bias gradients), one block per column group
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ X, int M, int N,
                                                     float* __restrict__ out) {
  __shared__ float sh[256];
  const int n = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += 256) s += X[(long long)m * N + n];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = sh[0];
}

// per-variable sums of squares over [E][nv][nm] of x = a (mode 0), a - b (mode 1)
// or a - b - c (mode 2); one block per variable, deterministic
__global__ void __launch_bounds__(256) var_sumsq_kernel(const double* __restrict__ a,
                                                        const double* __restrict__ b,
                                                        const double* __restrict__ c, int mode,
                                                        int E, int nv, int nm,
                                                        double* __restrict__ out) {
  __shared__ double sh[256];
  const int v = blockIdx.x;
  double s = 0.0;
  for (long long i = threadIdx.x; i < (long long)E * nm; i += 256) {
    const long long e = i / nm, m = i % nm;
    const long long g = (e * nv + v) * nm + m;
    double x = a[g];
    if (mode >= 1) x -= b[g];
    if (mode == 2) x -= c[g];
    s = fma(x, x, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = sh[0];
}

// inv[k] = 1/RMS, rms[k] = RMS (RMS := 1 where it is 0), k < n
__global__ void inv_rms_kernel(const double* __restrict__ sumsq, int n, long long count,
                               double* __restrict__ inv, double* __restrict__ rms) {
  const int k = threadIdx.x;
  if (k >= n) return;
  double r = sqrt(sumsq[k] / (double)count);
  if (!(r > 0.0)) r = 1.0;
  inv[k] = 1.0 / r;
  if (rms) rms[k] = r;
}

// X[e][blk*nb + v*nm + m] = bf16(F_blk / s_blk[v]), F = (u^n, u^n - u^{n-1}, d_prev)
__global__ void features_kernel(const double* __restrict__ h0, const double* __restrict__ h1,
                                const double* __restrict__ dp, const double* __restrict__ inv,
                                int E, int nv, int nm, bf16* __restrict__ X) {
  const int nb = nv * nm;
  const long long n = (long long)E * 3 * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / (3 * nb);
    const int r = (int)(i % (3 * nb));
    const int blk = r / nb, j = r % nb, v = j / nm;
    const long long g = e * nb + j;
    const double x = blk == 0 ? h0[g] : (blk == 1 ? h0[g] - h1[g] : dp[g]);
    X[i] = __float2bfloat16_rn((float)(x * inv[blk * nv + v]));
  }
}

// T = (u - S - d_prev) / tau[v]
__global__ void target_kernel(const double* __restrict__ u, const double* __restrict__ S,
                              const double* __restrict__ dp, const double* __restrict__ inv_tau,
                              long long n, int nm, int nv, float* __restrict__ T) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)((i / nm) % nv);
    T[i] = (float)((u[i] - S[i] - dp[i]) * inv_tau[v]);
  }
}

// dY = (Y - T)/n (FP32 and BF16), partial loss sums (sum (Y-T)^2 / 2n) per block
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ Y,
                                                   const float* __restrict__ T, long long n,
                                                   float* __restrict__ dY, bf16* __restrict__ dYb,
                                                   double* __restrict__ partial) {
  __shared__ double sh[256];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  const float inv = 1.0f / (float)n;
  const double dinv = 1.0 / (double)n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) {
    const float d = Y[i] - T[i];
    s += 0.5 * (double)d * (double)d * dinv;
    const float g = d * inv;
    dY[i] = g;
    dYb[i] = __float2bfloat16_rn(g);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out = S + d_prev (+ Y tau[v])
__global__ void predict_kernel(const double* __restrict__ S, const double* __restrict__ dp,
                               const float* __restrict__ Y, const double* __restrict__ tau,
                               long long n, int nm, int nv, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v = S[i] + dp[i];
    if (Y) v += (double)Y[i] * tau[(i / nm) % nv];
    out[i] = v;
  }
}

// d = u - S
__global__ void increment_kernel(const double* __restrict__ u, const double* __restrict__ S,
                                 long long n, double* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = u[i] - S[i];
}

// Adam on FP32 master parameters; refresh the BF16 copy (if any)
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, bf16* __restrict__ pb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float pn = p[i] - upd;
    p[i] = pn;
    if (pb) pb[i] = __float2bfloat16_rn(pn);
  }
}

__global__ void to_bf16_f32_kernel(const float* __restrict__ src, bf16* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

static int grid1(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

template <bool TA, bool TB, int EPI>
static dg_status gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                      const float* bias, const float* aux, float* C, bf16* Cb, int ldc,
                      cudaStream_t s, int splits = 1, float* part = nullptr) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  if (splits == 1) {
    gemm_kernel<TA, TB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, aux, C, Cb, ldc, K);
    DG_LAUNCHED(1);
    return DG_OK;
  }
  const int kc = ((K + splits - 1) / splits + 31) / 32 * 32;
  grid.z = (K + kc - 1) / kc;
  gemm_kernel<TA, TB, EPI_NONE><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, nullptr, nullptr, part,
                                                     nullptr, ldc, kc);
  splitk_reduce_kernel<<<grid1((long long)M * ldc), 256, 0, s>>>(part, grid.z, (long long)M * ldc, C);
  DG_LAUNCHED(2);
  return DG_OK;
}

}  // namespace dg

using namespace dg;

// ---------------------------------------------------------------- handle
struct dg_guess_s {
  dg_mesh_s* mesh = nullptr;
  int M = 0, H = 0, din = 0, dout = 0, E = 0, nv = 0, nm = 0, mlp = 1;
  float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  // the MLP correction is used once the stage's training loss (after its last
  // update, on its own batch) is below gate x the loss of the zero correction
  float gate = 0.2f;
  double loss[4] = {1e300, 1e300, 1e300, 1e300};
  float* p[4][6] = {};   // FP32 master parameters per stage
  float* am[4][6] = {};  // Adam moments
  float* av[4][6] = {};
  bf16* wb[4][3] = {};   // BF16 weight copies
  int t[4] = {0, 0, 0, 0};
  double* tau = nullptr;     // [4][nv] target RMS, [4..8)[nv] its inverse
  double* hist[2] = {};      // u^n (hist[head]) and u^{n-1}
  int nhist = 0, head = -1;
  double* dprev[4] = {};     // converged increment u^m - S_m of the previous step, per stage
  int dvalid[4] = {0, 0, 0, 0};
  int feat_stage = -1;       // stage whose features are in X (-1: none)
  bf16* X = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *T = nullptr, *dY = nullptr, *D2 = nullptr,
        *D1 = nullptr;
  bf16 *A1b = nullptr, *A2b = nullptr, *dYb = nullptr, *D2b = nullptr, *D1b = nullptr;
  float* g[6] = {};
  float* part = nullptr;
  double* red = nullptr;     // [0, RED_BLOCKS): loss partials; RB: loss; RB+8: feature sums; RB+32: target sums
  double* inv = nullptr;     // feature scales [3][nv]
  double* host = nullptr;    // pinned
};

static size_t param_size(const dg_guess_s* g, int i) {
  switch (i) {
    case 0: return (size_t)g->din * g->H;
    case 1: return g->H;
    case 2: return (size_t)g->H * g->H;
    case 3: return g->H;
    case 4: return (size_t)g->H * g->dout;
    default: return g->dout;
  }
}

static void free_guess(dg_guess_s* g) {
  if (!g) return;
  for (int m = 0; m < 4; ++m) {
    for (int i = 0; i < 6; ++i) {
      cudaFree(g->p[m][i]);
      cudaFree(g->am[m][i]);
      cudaFree(g->av[m][i]);
    }
    for (int i = 0; i < 3; ++i) cudaFree(g->wb[m][i]);
    cudaFree(g->dprev[m]);
  }
  for (int i = 0; i < 2; ++i) cudaFree(g->hist[i]);
  for (int i = 0; i < 6; ++i) cudaFree(g->g[i]);
  void* bufs[] = {g->tau, g->X, g->Z1, g->Z2, g->Y, g->T, g->dY, g->D2, g->D1, g->A1b, g->A2b,
                  g->dYb, g->D2b, g->D1b, g->part, g->red, g->inv};
  for (void* b : bufs) cudaFree(b);
  if (g->host) cudaFreeHost(g->host);
  delete g;
}

namespace dg {

bool guess_history_empty(const dg_guess_s* g) { return g->nhist == 0; }
bool guess_history_full(const dg_guess_s* g) { return g->nhist >= 2; }

static dg_status guess_features(dg_guess_s* g, int st, cudaStream_t s) {
  const double* h0 = g->hist[g->head];
  const double* h1 = g->hist[(g->head + 1) % 2];
  double* fs = g->red + RED_BLOCKS + 8;
  var_sumsq_kernel<<<g->nv, 256, 0, s>>>(h0, nullptr, nullptr, 0, g->E, g->nv, g->nm, fs);
  var_sumsq_kernel<<<g->nv, 256, 0, s>>>(h0, h1, nullptr, 1, g->E, g->nv, g->nm, fs + g->nv);
  var_sumsq_kernel<<<g->nv, 256, 0, s>>>(g->dprev[st], nullptr, nullptr, 0, g->E, g->nv, g->nm,
                                         fs + 2 * g->nv);
  inv_rms_kernel<<<1, 32, 0, s>>>(fs, 3 * g->nv, (long long)g->E * g->nm, g->inv, nullptr);
  features_kernel<<<grid1((long long)g->E * g->din), 256, 0, s>>>(h0, h1, g->dprev[st], g->inv,
                                                                  g->E, g->nv, g->nm, g->X);
  DG_LAUNCHED(5);
  g->feat_stage = st;
  return DG_OK;
}

static dg_status guess_forward(dg_guess_s* g, int st, cudaStream_t s) {
  const int E = g->E, H = g->H;
  DG_TRY((gemm<false, false, EPI_TANH>(E, H, g->din, g->X, g->din, g->wb[st][0], H, g->p[st][1],
                                       nullptr, g->Z1, g->A1b, H, s)));
  DG_TRY((gemm<false, false, EPI_TANH>(E, H, H, g->A1b, H, g->wb[st][1], H, g->p[st][3], nullptr,
                                       g->Z2, g->A2b, H, s)));
  DG_TRY((gemm<false, false, EPI_NONE>(E, g->dout, H, g->A2b, H, g->wb[st][2], g->dout,
                                       g->p[st][5], nullptr, g->Y, nullptr, g->dout, s)));
  return DG_OK;
}

// loss (to loss_dev) and gradients of stage st for the target in g->T
static dg_status guess_backward(dg_guess_s* g, int st, double* loss_dev, cudaStream_t s) {
  const int E = g->E, H = g->H, dout = g->dout, din = g->din;
  const long long n = (long long)E * dout;
  DG_TRY(guess_forward(g, st, s));
  loss_kernel<<<RED_BLOCKS, 256, 0, s>>>(g->Y, g->T, n, g->dY, g->dYb, g->red);
  DG_LAUNCHED(1);
  const int splits = 32;
  DG_TRY((gemm<true, false, EPI_NONE>(H, dout, E, g->A2b, H, g->dYb, dout, nullptr, nullptr,
                                      g->g[4], nullptr, dout, s, splits, g->part)));
  colsum_kernel<<<dout, 256, 0, s>>>(g->dY, E, dout, g->g[5]);
  DG_LAUNCHED(1);
  DG_TRY((gemm<false, true, EPI_DTANH>(E, H, dout, g->dYb, dout, g->wb[st][2], dout, nullptr,
                                       g->Z2, g->D2, g->D2b, H, s)));
  DG_TRY((gemm<true, false, EPI_NONE>(H, H, E, g->A1b, H, g->D2b, H, nullptr, nullptr, g->g[2],
                                      nullptr, H, s, splits, g->part)));
  colsum_kernel<<<H, 256, 0, s>>>(g->D2, E, H, g->g[3]);
  DG_LAUNCHED(1);
  DG_TRY((gemm<false, true, EPI_DTANH>(E, H, H, g->D2b, H, g->wb[st][1], H, nullptr, g->Z1, g->D1,
                                       g->D1b, H, s)));
  DG_TRY((gemm<true, false, EPI_NONE>(din, H, E, g->X, din, g->D1b, H, nullptr, nullptr, g->g[0],
                                      nullptr, H, s, splits, g->part)));
  colsum_kernel<<<H, 256, 0, s>>>(g->D1, E, H, g->g[1]);
  DG_LAUNCHED(1);
  DG_TRY(finish_sum(g->red, RED_BLOCKS, loss_dev, s));
  return DG_OK;
}

}  // namespace dg

extern "C" {

dg_status dg_guess_create(dg_mesh_t m, const dg_guess_cfg* cfg, const float* const* params,
                          dg_guess_t* out) {
  if (!m || !cfg || !out) return DG_ERR_ARG;
  if (cfg->stages < 1 || cfg->stages > 4) return DG_ERR_ARG;
  if (cfg->mlp && (!params || cfg->hidden < 1 || cfg->hidden > 4096)) return DG_ERR_ARG;
  dg_guess_s* g = new (std::nothrow) dg_guess_s();
  if (!g) return DG_ERR_OOM;
  g->mesh = m;
  g->M = cfg->stages;
  g->H = cfg->mlp ? cfg->hidden : 0;
  g->mlp = cfg->mlp != 0;
  g->nv = m->nv;
  g->nm = m->nm;
  g->E = m->E;
  g->dout = m->nv * m->nm;
  g->din = 3 * g->dout;
  g->lr = cfg->lr;
  g->b1 = cfg->beta1;
  g->b2 = cfg->beta2;
  g->eps = cfg->eps;
  if (cfg->gate > 0.f) g->gate = cfg->gate;
  cudaError_t err = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc(p, bytes);
    if (err == cudaSuccess) err = cudaMemset(*p, 0, bytes);
  };
  const size_t E = g->E, H = g->H, nd = (size_t)m->ndof;
  for (int st = 0; st < g->M; ++st) alloc((void**)&g->dprev[st], 8 * nd);
  for (int i = 0; i < 2; ++i) alloc((void**)&g->hist[i], 8 * nd);
  alloc((void**)&g->tau, 8 * 8 * g->nv);
  alloc((void**)&g->red, 8 * (RED_BLOCKS + 64));
  alloc((void**)&g->inv, 8 * 3 * g->nv);
  if (err == cudaSuccess) err = cudaMallocHost((void**)&g->host, 64);
  if (g->mlp) {
    for (int st = 0; st < g->M; ++st) {
      for (int i = 0; i < 6; ++i) {
        const size_t n = param_size(g, i);
        alloc((void**)&g->p[st][i], 4 * n);
        alloc((void**)&g->am[st][i], 4 * n);
        alloc((void**)&g->av[st][i], 4 * n);
        if (err == cudaSuccess)
          err = cudaMemcpy(g->p[st][i], params[st * 6 + i], 4 * n, cudaMemcpyHostToDevice);
        if (i % 2 == 0) alloc((void**)&g->wb[st][i / 2], 2 * n);
      }
    }
    for (int i = 0; i < 6; ++i) alloc((void**)&g->g[i], 4 * param_size(g, i));
    alloc((void**)&g->X, 2 * E * g->din);
    alloc((void**)&g->Z1, 4 * E * H);
    alloc((void**)&g->Z2, 4 * E * H);
    alloc((void**)&g->D1, 4 * E * H);
    alloc((void**)&g->D2, 4 * E * H);
    alloc((void**)&g->Y, 4 * E * g->dout);
    alloc((void**)&g->T, 4 * E * g->dout);
    alloc((void**)&g->dY, 4 * E * g->dout);
    alloc((void**)&g->A1b, 2 * E * H);
    alloc((void**)&g->A2b, 2 * E * H);
    alloc((void**)&g->D1b, 2 * E * H);
    alloc((void**)&g->D2b, 2 * E * H);
    alloc((void**)&g->dYb, 2 * E * g->dout);
    size_t pmax = 0;
    for (int i = 0; i < 6; i += 2) pmax = param_size(g, i) > pmax ? param_size(g, i) : pmax;
    alloc((void**)&g->part, 4 * 32 * pmax);
  }
  if (err != cudaSuccess) {
    free_guess(g);
    return cuda_status(err);
  }
  std::vector<double> ones(8 * g->nv, 1.0);
  cudaMemcpy(g->tau, ones.data(), 8 * ones.size(), cudaMemcpyHostToDevice);
  if (g->mlp)
    for (int st = 0; st < g->M; ++st)
      for (int i = 0; i < 3; ++i) {
        const long long n = (long long)param_size(g, 2 * i);
        to_bf16_f32_kernel<<<grid1(n), 256>>>(g->p[st][2 * i], g->wb[st][i], n);
      }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_guess(g);
    return DG_ERR_CUDA;
  }
  *out = g;
  return DG_OK;
}

dg_status dg_guess_destroy(dg_guess_t g) {
  if (!g) return DG_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  free_guess(g);
  return e == cudaSuccess ? DG_OK : cuda_status(e);
}

dg_status dg_guess_push(dg_guess_t g, const double* u, void* stream) {
  if (!g || !u) return DG_ERR_ARG;
  g->head = (g->head + 1) % 2;
  DG_CUDA(cudaMemcpyAsync(g->hist[g->head], u, 8 * (size_t)g->mesh->ndof,
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  if (g->nhist < 2) g->nhist++;
  g->feat_stage = -1;
  return DG_OK;
}

dg_status dg_guess_ready(dg_guess_t g, int stage, int* ready) {
  if (!g || !ready || stage < 0 || stage >= g->M) return DG_ERR_ARG;
  *ready = g->nhist >= 2 && g->dvalid[stage];
  return DG_OK;
}

dg_status dg_guess_predict(dg_guess_t g, int stage, const double* S, double* out, void* stream) {
  if (!g || !S || !out || stage < 0 || stage >= g->M) return DG_ERR_ARG;
  if (g->nhist < 2 || !g->dvalid[stage]) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // loss of the zero correction on unit-RMS targets is 1/2
  const bool use_mlp = g->mlp && g->loss[stage] < 0.5 * g->gate;
  if (use_mlp) {
    if (g->feat_stage != stage) DG_TRY(guess_features(g, stage, s));
    DG_TRY(guess_forward(g, stage, s));
  }
  predict_kernel<<<grid1(g->mesh->ndof), 256, 0, s>>>(S, g->dprev[stage], use_mlp ? g->Y : nullptr,
                                                      g->tau + stage * g->nv, g->mesh->ndof,
                                                      g->nm, g->nv, out);
  DG_LAUNCHED(1);
  return DG_OK;
}

dg_status dg_guess_train(dg_guess_t g, int stage, const double* S, const double* u, int iters,
                         double* loss_first, double* loss_last, float* const* grads_host,
                         void* stream) {
  if (!g || !S || !u || stage < 0 || stage >= g->M || iters < 0) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = g->mesh->ndof;
  double* host = g->host;
  host[0] = host[1] = -1.0;
  const bool learn = g->mlp && g->nhist >= 2 && g->dvalid[stage];
  if (learn) {
    if (g->feat_stage != stage) DG_TRY(guess_features(g, stage, s));
    // target scale tau_m[v] = per-variable RMS of u - S - d_prev
    double* ts = g->red + RED_BLOCKS + 32;
    var_sumsq_kernel<<<g->nv, 256, 0, s>>>(u, S, g->dprev[stage], 2, g->E, g->nv, g->nm, ts);
    inv_rms_kernel<<<1, 32, 0, s>>>(ts, g->nv, (long long)g->E * g->nm,
                                    g->tau + (4 + stage) * g->nv, g->tau + stage * g->nv);
    target_kernel<<<grid1(n), 256, 0, s>>>(u, S, g->dprev[stage], g->tau + (4 + stage) * g->nv, n,
                                           g->nm, g->nv, g->T);
    DG_LAUNCHED(3);
    double* ld = g->red + RED_BLOCKS;
    for (int it = 0; it < (iters > 0 ? iters : 1); ++it) {
      DG_TRY(guess_backward(g, stage, ld, s));
      if (it == 0) {
        DG_CUDA(cudaMemcpyAsync(host, ld, 8, cudaMemcpyDeviceToHost, s));
        if (grads_host)
          for (int i = 0; i < 6; ++i)
            if (grads_host[i])
              DG_CUDA(cudaMemcpyAsync(grads_host[i], g->g[i], 4 * param_size(g, i),
                                      cudaMemcpyDeviceToHost, s));
      }
      if (iters == 0) break;
      g->t[stage]++;
      const float c1 = 1.f - powf(g->b1, (float)g->t[stage]);
      const float c2 = 1.f - powf(g->b2, (float)g->t[stage]);
      for (int i = 0; i < 6; ++i) {
        const long long np = (long long)param_size(g, i);
        adam_kernel<<<grid1(np), 256, 0, s>>>(g->p[stage][i], g->am[stage][i], g->av[stage][i],
                                             g->g[i], np, g->lr, g->b1, g->b2, g->eps, c1, c2,
                                             i % 2 == 0 ? g->wb[stage][i / 2] : nullptr);
      }
      DG_LAUNCHED(6);
    }
    if (iters > 0) {
      DG_TRY(guess_backward(g, stage, ld, s));
      DG_CUDA(cudaMemcpyAsync(host + 1, ld, 8, cudaMemcpyDeviceToHost, s));
    }
  }
  // the converged increment becomes the extrapolation base of the next step
  increment_kernel<<<grid1(n), 256, 0, s>>>(u, S, n, g->dprev[stage]);
  DG_LAUNCHED(1);
  g->dvalid[stage] = 1;
  if (g->feat_stage == stage) g->feat_stage = -1;
  DG_CUDA(cudaStreamSynchronize(s));
  if (loss_first) *loss_first = host[0];
  if (loss_last) *loss_last = iters > 0 ? host[1] : host[0];
  if (learn && iters > 0) g->loss[stage] = host[1];
  return DG_OK;
}

dg_status dg_guess_params(dg_guess_t g, int stage, float* const* host_out) {
  if (!g || !host_out || stage < 0 || stage >= g->M || !g->mlp) return DG_ERR_ARG;
  DG_CUDA(cudaDeviceSynchronize());
  for (int i = 0; i < 6; ++i)
    if (host_out[i])
      DG_CUDA(cudaMemcpy(host_out[i], g->p[stage][i], 4 * param_size(g, i), cudaMemcpyDeviceToHost));
  return DG_OK;
}

}  // extern "C"
