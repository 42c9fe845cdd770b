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
#include "dg_tc.cuh"

namespace dg {

typedef __nv_bfloat16 bf16;

enum { EPI_NONE = 0, EPI_TANH = 1, EPI_DTANH = 2 };

// C = A B^T (+ bias) with epilogue on the fifth-generation tensor cores:
// A [M][lda] and B [N][ldb] BF16 with K contiguous (ld a multiple of 8),
// copied by cp.async into a ring of TC_NS shared-memory stages in the K-major
// core-matrix layout (zero-filled outside the matrix), one thread issuing
// tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into an FP32
// accumulator in tensor memory, the four warps reading it back (one row per
// thread) for the epilogue: bias, tanh or tanh' (times 1 - aux^2), FP32 C,
// BF16 Cb and the BF16 transpose CbT (coalesced: consecutive rows are
// consecutive threads).  gridDim.z > 1: split-K, block z covers
// k in [z kc, (z+1) kc) and writes its FP32 partial to C + z M N (dense).
constexpr int TC_BM = 128, TC_BK = 64, TC_NS = 4;
constexpr int TC_WAIT = 1 << 20;  // mbarrier polls before a wait gives up

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_wait_stages() { asm volatile("cp.async.wait_group %0;" ::"n"(TC_NS - 2)); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;"); }

// rows [row0, row0 + ROWS) x k in [k0, k0 + TC_BK) of X into a K-major tile
template <int ROWS>
__device__ __forceinline__ void issue_tile(uint8_t* dst, const bf16* __restrict__ X, int ld,
                                           int row0, int nrows, int k0, int kend) {
  constexpr int SBO = (TC_BK / 8) * 128;
  const uint32_t base = tc::smem_addr(dst);
  for (int i = threadIdx.x; i < ROWS * (TC_BK / 8); i += blockDim.x) {
    const int r = i / (TC_BK / 8), kv = (i % (TC_BK / 8)) * 8;
    const int gr = row0 + r, gk = k0 + kv;
    int bytes = 0;
    const bf16* src = X;
    if (gr < nrows && gk < kend) {
      bytes = min(16, 2 * (kend - gk));
      src = X + (long long)gr * ld + gk;
    }
    cp_async16(base + (r >> 3) * SBO + (kv >> 3) * 128 + (r & 7) * 16, src, bytes);
  }
}

template <int EPI>
__device__ __forceinline__ float epilogue(float x, int m, int n, const float* bias,
                                          const float* aux, int ldaux) {
  if (bias) x += bias[n];
  if (EPI == EPI_TANH) x = tanhf(x);
  if (EPI == EPI_DTANH) {
    const float a = aux[(long long)m * ldaux + n];
    x *= 1.f - a * a;
  }
  return x;
}

template <int EPI, int BN>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, const bf16* __restrict__ A,
                                                   int lda, const bf16* __restrict__ B, int ldb,
                                                   const float* __restrict__ bias,
                                                   const float* __restrict__ aux, int ldaux,
                                                   float* __restrict__ C, int ldc,
                                                   bf16* __restrict__ Cb, int ldcb,
                                                   bf16* __restrict__ CbT, int ldct, int kc,
                                                   int* __restrict__ err) {
  constexpr int ATILE = TC_BM * TC_BK * 2, BTILE = BN * TC_BK * 2, STAGE = ATILE + BTILE;
  constexpr int SBO = (TC_BK / 8) * 128;
  extern __shared__ __align__(1024) uint8_t smraw[];
  __shared__ __align__(8) uint64_t mbar[TC_NS];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kc, kend = min(K, kbeg + kc);
  const int nch = kend > kbeg ? (kend - kbeg + TC_BK - 1) / TC_BK : 0;
  if (warp == 0) tc::tmem_alloc(&tmem_slot, BN);
  if (tid == 0)
    for (int i = 0; i < TC_NS; ++i) tc::mbar_init(&mbar[i], 1);
  for (int c = 0; c < TC_NS - 1; ++c) {  // prologue: chunks 0 .. TC_NS - 2
    if (c < nch) {
      uint8_t* sA = smraw + c * STAGE;
      issue_tile<TC_BM>(sA, A, lda, m0, M, kbeg + c * TC_BK, kend);
      issue_tile<BN>(sA + ATILE, B, ldb, n0, N, kbeg + c * TC_BK, kend);
    }
    cp_commit();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  int issued = 0;
  for (int c = 0; c < nch; ++c) {
    cp_wait_stages();  // this thread's copies of chunk c have landed ...
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();   // ... and every thread's
    tc::fence_after();
    uint8_t* sA = smraw + (c % TC_NS) * STAGE;
    if (tid == 0) {
      constexpr uint32_t id = tc::idesc(1, TC_BM, BN);
#pragma unroll
      for (int ks = 0; ks < TC_BK / 16; ++ks) {
        const uint64_t da = tc::desc(tc::smem_addr(sA) + ks * 256, 128, SBO);
        const uint64_t db = tc::desc(tc::smem_addr(sA + ATILE) + ks * 256, 128, SBO);
        tc::mma_bf16(tmem, da, db, id, (c > 0 || ks > 0) ? 1u : 0u);
      }
      tc::commit(&mbar[c % TC_NS]);
    }
    issued = c + 1;
    // chunk c + TC_NS - 1 goes into the stage of chunk c - 1 once its MMAs are done
    const int nc = c + TC_NS - 1;
    if (nc < nch) {
      if (c >= 1) {
        const int pc = c - 1;
        const bool w = tc::mbar_wait(&mbar[pc % TC_NS], (pc / TC_NS) & 1, TC_WAIT);
        if (!__syncthreads_and(w)) {
          ok = false;
          break;
        }
      }
      uint8_t* dA = smraw + (nc % TC_NS) * STAGE;
      issue_tile<TC_BM>(dA, A, lda, m0, M, kbeg + nc * TC_BK, kend);
      issue_tile<BN>(dA + ATILE, B, ldb, n0, N, kbeg + nc * TC_BK, kend);
    }
    cp_commit();
  }
  cp_wait_all();
  // the last commit arrives once every MMA of this CTA is done
  if (issued > 0) {
    const int c = issued - 1;
    const bool w = tc::mbar_wait(&mbar[c % TC_NS], (c / TC_NS) & 1, TC_WAIT);
    ok = __syncthreads_and(w && ok);
  }
  tc::fence_after();
  if (ok) {
    const int m = m0 + warp * 32 + (tid & 31);
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    const bool split = gridDim.z > 1;
    for (int cc = 0; cc < BN && n0 + cc < N; cc += 16) {
      float v[16];
      if (nch > 0) {
        tc::ld16(tmem + lanes + cc, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + cc + j;
          if (n >= N) break;
          if (split) {
            C[((long long)blockIdx.z * M + m) * N + n] = v[j];
          } else {
            const float x = epilogue<EPI>(v[j], m, n, bias, aux, ldaux);
            if (C) C[(long long)m * ldc + n] = x;
            if (Cb) Cb[(long long)m * ldcb + n] = __float2bfloat16_rn(x);
            if (CbT) CbT[(long long)n * ldct + m] = __float2bfloat16_rn(x);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

// sum of the split-K partials in order (deterministic), then the epilogue
template <int EPI>
__global__ void splitk_epilogue_kernel(const float* __restrict__ part, int nz, int M, int N,
                                       const float* __restrict__ bias,
                                       const float* __restrict__ aux, int ldaux,
                                       float* __restrict__ C, int ldc, bf16* __restrict__ Cb,
                                       int ldcb, bf16* __restrict__ CbT, int ldct) {
  const long long n_all = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_all;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / N), n = (int)(i % N);
    float x = 0.f;
    for (int z = 0; z < nz; ++z) x += part[(long long)z * n_all + i];
    x = epilogue<EPI>(x, m, n, bias, aux, ldaux);
    if (C) C[(long long)m * ldc + n] = x;
    if (Cb) Cb[(long long)m * ldcb + n] = __float2bfloat16_rn(x);
    if (CbT) CbT[(long long)n * ldct + m] = __float2bfloat16_rn(x);
  }
}

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
// or a - b - c (mode 2): block (b, v) sums a contiguous range of elements of
// variable v into out[v * VB + b] (fixed partition and order: deterministic)
constexpr int VB = 64;
__global__ void __launch_bounds__(256) var_sumsq_kernel(const double* __restrict__ a,
                                                        const double* __restrict__ b,
                                                        const double* __restrict__ c, int mode,
                                                        int E, int nv, int nm,
                                                        double* __restrict__ out) {
  __shared__ double sh[256];
  const int v = blockIdx.y;
  const int per = (E + VB - 1) / VB;
  const int e0 = blockIdx.x * per, e1 = min(E, e0 + per);
  double s = 0.0;
  for (long long i = threadIdx.x; i < (long long)max(e1 - e0, 0) * nm; i += 256) {
    const long long e = e0 + i / nm, m = i % nm;
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
  if (threadIdx.x == 0) out[v * VB + blockIdx.x] = sh[0];
}

// inv[k] = 1/RMS, rms[k] = RMS of the VB partial sums of k (RMS := 1 where it is 0), k < n
__global__ void inv_rms_kernel(const double* __restrict__ part, int n, long long count,
                               double* __restrict__ inv, double* __restrict__ rms) {
  const int k = threadIdx.x;
  if (k >= n) return;
  double t = 0.0;
  for (int b = 0; b < VB; ++b) t += part[k * VB + b];
  double r = sqrt(t / (double)count);
  if (!(r > 0.0)) r = 1.0;
  inv[k] = 1.0 / r;
  if (rms) rms[k] = r;
}

// X[e][blk*nb + v*nm + m] = bf16(F_blk / s_blk[v]), F = (u^n, u^n - u^{n-1}, d_prev),
// row stride ldx, and its transpose XT[blk*nb + v*nm + m][e] (row stride ldt)
__global__ void features_kernel(const double* __restrict__ h0, const double* __restrict__ h1,
                                const double* __restrict__ dp, const double* __restrict__ inv,
                                int E, int nv, int nm, bf16* __restrict__ X, int ldx,
                                bf16* __restrict__ XT, int ldt) {
  const int nb = nv * nm;
  const long long n = (long long)E * 3 * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    // e fastest: the transposed writes are coalesced, the direct ones strided
    const long long e = i % E;
    const int r = (int)(i / E);
    const int blk = r / nb, j = r % nb, v = j / nm;
    const long long g = e * nb + j;
    const double x = blk == 0 ? h0[g] : (blk == 1 ? h0[g] - h1[g] : dp[g]);
    const bf16 b = __float2bfloat16_rn((float)(x * inv[blk * nv + v]));
    X[e * ldx + r] = b;
    XT[(long long)r * ldt + e] = b;
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

// dY = (Y - T)/n (FP32 [E][nb], BF16 [E][ldb] and its BF16 transpose [nb][ldt]),
// partial loss sums (sum (Y-T)^2 / 2n) per block
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ Y,
                                                   const float* __restrict__ T, int E, int nb,
                                                   float* __restrict__ dY, bf16* __restrict__ dYb,
                                                   int ldb, bf16* __restrict__ dYbT, int ldt,
                                                   double* __restrict__ partial) {
  __shared__ double sh[256];
  const long long n = (long long)E * nb;
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  const float inv = 1.0f / (float)n;
  const double dinv = 1.0 / (double)n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) {
    const float d = Y[i] - T[i];
    s += 0.5 * (double)d * (double)d * dinv;
    const float g = d * inv;
    const long long e = i / nb;
    const int j = (int)(i % nb);
    dY[i] = g;
    const bf16 b = __float2bfloat16_rn(g);
    dYb[e * ldb + j] = b;
    if (dYbT) dYbT[(long long)j * ldt + e] = b;
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
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = p[i] - upd;
  }
}

// BF16 operand copies of a weight matrix W [rows][cols] (FP32 master):
// wT [cols][ldT] = W^T and, when wP is given, wP [rows][ldP] = W
__global__ void weight_copies_kernel(const float* __restrict__ W, int rows, int cols,
                                     bf16* __restrict__ wT, int ldT, bf16* __restrict__ wP,
                                     int ldP) {
  const long long n = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    const bf16 b = __float2bfloat16_rn(W[i]);
    wT[(long long)c * ldT + r] = b;
    if (wP) wP[(long long)r * ldP + c] = b;
  }
}

static int grid1(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

// output operands of one GEMM (null pointers are skipped)
struct GemmOut {
  float* C;
  int ldc;
  bf16* Cb;
  int ldcb;
  bf16* CbT;
  int ldct;
};

template <int EPI, int BN>
static dg_status gemm_bn(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                         const float* bias, const float* aux, int ldaux, const GemmOut& o,
                         int splits, float* part, int* err, cudaStream_t s) {
  constexpr size_t smem = (size_t)TC_NS * (TC_BM * TC_BK * 2 + BN * TC_BK * 2);
  static bool attr = false;  // per instantiation
  if (!attr) {
    DG_CUDA(cudaFuncSetAttribute(gemm_kernel<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  dim3 grid((N + BN - 1) / BN, (M + TC_BM - 1) / TC_BM, 1);
  if (splits <= 1) {
    DG_PROF(K_MLP, s, gemm_kernel<EPI, BN><<<grid, 128, smem, s>>>(
        M, N, K, A, lda, B, ldb, bias, aux, ldaux, o.C, o.ldc, o.Cb, o.ldcb, o.CbT, o.ldct, K, err));
    DG_LAUNCHED(1);
    return DG_OK;
  }
  const int nch = (K + TC_BK - 1) / TC_BK;
  const int kc = (nch + splits - 1) / splits * TC_BK;
  grid.z = (K + kc - 1) / kc;
  DG_PROF(K_MLP, s, gemm_kernel<EPI, BN><<<grid, 128, smem, s>>>(
      M, N, K, A, lda, B, ldb, nullptr, nullptr, 0, part, N, nullptr, 0, nullptr, 0, kc, err));
  splitk_epilogue_kernel<EPI><<<grid1((long long)M * N), 256, 0, s>>>(
      part, grid.z, M, N, bias, aux, ldaux, o.C, o.ldc, o.Cb, o.ldcb, o.CbT, o.ldct);
  DG_LAUNCHED(2);
  return DG_OK;
}

// C = A B^T: tile width and split-K chosen so that at least ~150 CTAs run
template <int EPI>
static dg_status gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                      const float* bias, const float* aux, int ldaux, const GemmOut& o,
                      float* part, size_t part_cap, int* err, cudaStream_t s) {
  if (lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return DG_ERR_ARG;
  const int mt = (M + TC_BM - 1) / TC_BM;
  const bool wide = N > 64 && (long long)mt * ((N + 127) / 128) >= 150;
  const int nt = wide ? (N + 127) / 128 : (N + 63) / 64;
  const int nch = (K + TC_BK - 1) / TC_BK;
  int splits = 1;
  if ((long long)mt * nt < 150 && part) {
    splits = (150 + mt * nt - 1) / (mt * nt);
    splits = splits < nch ? splits : nch;
    splits = splits < 32 ? splits : 32;
    while (splits > 1 && (size_t)splits * M * N > part_cap) --splits;
  }
  if (wide) return gemm_bn<EPI, 128>(M, N, K, A, lda, B, ldb, bias, aux, ldaux, o, splits, part, err, s);
  return gemm_bn<EPI, 64>(M, N, K, A, lda, B, ldb, bias, aux, ldaux, o, splits, part, err, s);
}

}  // namespace dg

using namespace dg;

// ---------------------------------------------------------------- handle
struct dg_guess_s {
  dg_mesh_s* mesh = nullptr;
  int M = 0, H = 0, din = 0, dout = 0, E = 0, nv = 0, nm = 0, mlp = 1;
  int ldi = 0, ldo = 0, ldh = 0, lde = 0;  // din, dout, H, E rounded up to 8 (16-byte rows)
  float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  // the MLP correction is used once the stage's training loss (after its last
  // update, on its own batch) is below gate x the loss of the zero correction
  float gate = 0.2f;
  double loss[4] = {1e300, 1e300, 1e300, 1e300};
  float* p[4][6] = {};   // FP32 master parameters per stage
  float* am[4][6] = {};  // Adam moments
  float* av[4][6] = {};
  // BF16 operand copies, K contiguous: W1^T [H][ldi], W2^T [H][ldh], W3^T [dout][ldh]
  // (forward) and W2 [H][ldh], W3 [H][ldo] (backward)
  bf16* wT[4][3] = {};
  bf16* wP[4][3] = {};
  int t[4] = {0, 0, 0, 0};
  double* tau = nullptr;     // [4][nv] target RMS, [4..8)[nv] its inverse
  double* hist[2] = {};      // u^n (hist[head]) and u^{n-1}
  int nhist = 0, head = -1;
  double* dprev[4] = {};     // converged increment u^m - S_m of the previous step, per stage
  int dvalid[4] = {0, 0, 0, 0};
  int feat_stage = -1;       // stage whose features are in X (-1: none)
  // BF16 activations [E][ld*] and their transposes [*][lde] (operands of the
  // weight-gradient products, whose contraction runs over the elements)
  bf16 *X = nullptr, *XT = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *T = nullptr, *dY = nullptr, *D2 = nullptr,
        *D1 = nullptr;
  bf16 *A1b = nullptr, *A2b = nullptr, *dYb = nullptr, *D2b = nullptr;
  bf16 *A1bT = nullptr, *A2bT = nullptr, *dYbT = nullptr, *D2bT = nullptr, *D1bT = nullptr;
  float* g[6] = {};
  float* part = nullptr;     // split-K partial sums
  size_t part_cap = 0;
  double* red = nullptr;     // [0, RED_BLOCKS): loss partials; RB: loss
  double* inv = nullptr;     // feature scales [3][nv]
  double* vs = nullptr;      // per-variable partial sums of squares [4][nv][VB]
  double* host = nullptr;    // pinned
  int* tcerr = nullptr;      // set by a tensor-core GEMM whose wait gave up
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
    for (int i = 0; i < 3; ++i) {
      cudaFree(g->wT[m][i]);
      cudaFree(g->wP[m][i]);
    }
    cudaFree(g->dprev[m]);
  }
  for (int i = 0; i < 2; ++i) cudaFree(g->hist[i]);
  for (int i = 0; i < 6; ++i) cudaFree(g->g[i]);
  void* bufs[] = {g->tau,  g->X,    g->XT,   g->Z1,   g->Z2,   g->Y,    g->T,    g->dY,
                  g->D2,   g->D1,   g->A1b,  g->A2b,  g->dYb,  g->D2b,  g->A1bT, g->A2bT,
                  g->dYbT, g->D2bT, g->D1bT, g->part, g->red,  g->inv,  g->tcerr, g->vs};
  for (void* b : bufs) cudaFree(b);
  if (g->host) cudaFreeHost(g->host);
  delete g;
}

namespace dg {

bool guess_history_empty(const dg_guess_s* g) { return g->nhist == 0; }
bool guess_history_full(const dg_guess_s* g) { return g->nhist >= 2; }
int guess_stage_count(const dg_guess_s* g) { return g->M; }

static dg_status guess_features(dg_guess_s* g, int st, cudaStream_t s) {
  const double* h0 = g->hist[g->head];
  const double* h1 = g->hist[(g->head + 1) % 2];
  double* fs = g->vs;
  const dim3 vg(VB, g->nv);
  var_sumsq_kernel<<<vg, 256, 0, s>>>(h0, nullptr, nullptr, 0, g->E, g->nv, g->nm, fs);
  var_sumsq_kernel<<<vg, 256, 0, s>>>(h0, h1, nullptr, 1, g->E, g->nv, g->nm, fs + g->nv * VB);
  var_sumsq_kernel<<<vg, 256, 0, s>>>(g->dprev[st], nullptr, nullptr, 0, g->E, g->nv, g->nm,
                                      fs + 2 * g->nv * VB);
  inv_rms_kernel<<<1, 32, 0, s>>>(fs, 3 * g->nv, (long long)g->E * g->nm, g->inv, nullptr);
  features_kernel<<<grid1((long long)g->E * g->din), 256, 0, s>>>(
      h0, h1, g->dprev[st], g->inv, g->E, g->nv, g->nm, g->X, g->ldi, g->XT, g->lde);
  DG_LAUNCHED(5);
  g->feat_stage = st;
  return DG_OK;
}

// forward pass of stage st on the features in X (train: also the transposed
// activations the weight gradients need)
static dg_status guess_forward(dg_guess_s* g, int st, bool train, cudaStream_t s) {
  const int E = g->E, H = g->H;
  const GemmOut o1{g->Z1, H, g->A1b, g->ldh, train ? g->A1bT : nullptr, g->lde};
  DG_TRY(gemm<EPI_TANH>(E, H, g->din, g->X, g->ldi, g->wT[st][0], g->ldi, g->p[st][1], nullptr, 0,
                        o1, g->part, g->part_cap, g->tcerr, s));
  const GemmOut o2{g->Z2, H, g->A2b, g->ldh, train ? g->A2bT : nullptr, g->lde};
  DG_TRY(gemm<EPI_TANH>(E, H, H, g->A1b, g->ldh, g->wT[st][1], g->ldh, g->p[st][3], nullptr, 0, o2,
                        g->part, g->part_cap, g->tcerr, s));
  const GemmOut o3{g->Y, g->dout, nullptr, 0, nullptr, 0};
  DG_TRY(gemm<EPI_NONE>(E, g->dout, H, g->A2b, g->ldh, g->wT[st][2], g->ldh, g->p[st][5], nullptr,
                        0, o3, g->part, g->part_cap, g->tcerr, s));
  return DG_OK;
}

// loss (to loss_dev) of stage st for the target in g->T
static dg_status guess_loss(dg_guess_s* g, int st, double* loss_dev, cudaStream_t s) {
  DG_TRY(guess_forward(g, st, false, s));
  loss_kernel<<<RED_BLOCKS, 256, 0, s>>>(g->Y, g->T, g->E, g->dout, g->dY, g->dYb, g->ldo,
                                         nullptr, 0, g->red);
  DG_LAUNCHED(1);
  return finish_sum(g->red, RED_BLOCKS, loss_dev, s);
}

// loss (to loss_dev) and gradients of stage st for the target in g->T
static dg_status guess_backward(dg_guess_s* g, int st, double* loss_dev, cudaStream_t s) {
  const int E = g->E, H = g->H, dout = g->dout, din = g->din;
  DG_TRY(guess_forward(g, st, true, s));
  loss_kernel<<<RED_BLOCKS, 256, 0, s>>>(g->Y, g->T, E, dout, g->dY, g->dYb, g->ldo, g->dYbT,
                                         g->lde, g->red);
  DG_LAUNCHED(1);
  // dW3 = A2^T dY, db3 = column sums of dY
  DG_TRY(gemm<EPI_NONE>(H, dout, E, g->A2bT, g->lde, g->dYbT, g->lde, nullptr, nullptr, 0,
                        GemmOut{g->g[4], dout, nullptr, 0, nullptr, 0}, g->part, g->part_cap,
                        g->tcerr, s));
  colsum_kernel<<<dout, 256, 0, s>>>(g->dY, E, dout, g->g[5]);
  DG_LAUNCHED(1);
  // dZ2 = (dY W3^T) (1 - A2^2)
  DG_TRY(gemm<EPI_DTANH>(E, H, dout, g->dYb, g->ldo, g->wP[st][2], g->ldo, nullptr, g->Z2, H,
                         GemmOut{g->D2, H, g->D2b, g->ldh, g->D2bT, g->lde}, g->part, g->part_cap,
                         g->tcerr, s));
  DG_TRY(gemm<EPI_NONE>(H, H, E, g->A1bT, g->lde, g->D2bT, g->lde, nullptr, nullptr, 0,
                        GemmOut{g->g[2], H, nullptr, 0, nullptr, 0}, g->part, g->part_cap, g->tcerr,
                        s));
  colsum_kernel<<<H, 256, 0, s>>>(g->D2, E, H, g->g[3]);
  DG_LAUNCHED(1);
  // dZ1 = (dZ2 W2^T) (1 - A1^2)
  DG_TRY(gemm<EPI_DTANH>(E, H, H, g->D2b, g->ldh, g->wP[st][1], g->ldh, nullptr, g->Z1, H,
                         GemmOut{g->D1, H, nullptr, 0, g->D1bT, g->lde}, g->part, g->part_cap,
                         g->tcerr, s));
  DG_TRY(gemm<EPI_NONE>(din, H, E, g->XT, g->lde, g->D1bT, g->lde, nullptr, nullptr, 0,
                        GemmOut{g->g[0], H, nullptr, 0, nullptr, 0}, g->part, g->part_cap, g->tcerr,
                        s));
  colsum_kernel<<<H, 256, 0, s>>>(g->D1, E, H, g->g[1]);
  DG_LAUNCHED(1);
  DG_TRY(finish_sum(g->red, RED_BLOCKS, loss_dev, s));
  return DG_OK;
}

// the BF16 operand copies of stage st's weights
static void weight_copies(dg_guess_s* g, int st, cudaStream_t s) {
  const int H = g->H;
  weight_copies_kernel<<<grid1((long long)g->din * H), 256, 0, s>>>(g->p[st][0], g->din, H,
                                                                    g->wT[st][0], g->ldi, nullptr, 0);
  weight_copies_kernel<<<grid1((long long)H * H), 256, 0, s>>>(g->p[st][2], H, H, g->wT[st][1],
                                                               g->ldh, g->wP[st][1], g->ldh);
  weight_copies_kernel<<<grid1((long long)H * g->dout), 256, 0, s>>>(
      g->p[st][4], H, g->dout, g->wT[st][2], g->ldh, g->wP[st][2], g->ldo);
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
  g->ldi = (g->din + 7) / 8 * 8;
  g->ldo = (g->dout + 7) / 8 * 8;
  g->ldh = (g->H + 7) / 8 * 8;
  g->lde = (g->E + 7) / 8 * 8;
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
  alloc((void**)&g->tcerr, sizeof(int) * 4);
  alloc((void**)&g->vs, sizeof(double) * 4 * g->nv * VB);
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
      }
      const size_t ldi = g->ldi, ldo = g->ldo, ldh = g->ldh;
      alloc((void**)&g->wT[st][0], 2 * H * ldi);
      alloc((void**)&g->wT[st][1], 2 * H * ldh);
      alloc((void**)&g->wT[st][2], 2 * g->dout * ldh);
      alloc((void**)&g->wP[st][1], 2 * H * ldh);
      alloc((void**)&g->wP[st][2], 2 * H * ldo);
    }
    const size_t lde = g->lde;
    for (int i = 0; i < 6; ++i) alloc((void**)&g->g[i], 4 * param_size(g, i));
    alloc((void**)&g->X, 2 * E * g->ldi);
    alloc((void**)&g->XT, 2 * g->din * lde);
    alloc((void**)&g->Z1, 4 * E * H);
    alloc((void**)&g->Z2, 4 * E * H);
    alloc((void**)&g->D1, 4 * E * H);
    alloc((void**)&g->D2, 4 * E * H);
    alloc((void**)&g->Y, 4 * E * g->dout);
    alloc((void**)&g->T, 4 * E * g->dout);
    alloc((void**)&g->dY, 4 * E * g->dout);
    alloc((void**)&g->A1b, 2 * E * g->ldh);
    alloc((void**)&g->A2b, 2 * E * g->ldh);
    alloc((void**)&g->D2b, 2 * E * g->ldh);
    alloc((void**)&g->dYb, 2 * E * g->ldo);
    alloc((void**)&g->A1bT, 2 * H * lde);
    alloc((void**)&g->A2bT, 2 * H * lde);
    alloc((void**)&g->D2bT, 2 * H * lde);
    alloc((void**)&g->D1bT, 2 * H * lde);
    alloc((void**)&g->dYbT, 2 * g->dout * lde);
    // split-K partials: up to 32 slices of the largest weight gradient
    size_t pmax = 0;
    for (int i = 0; i < 6; i += 2) pmax = param_size(g, i) > pmax ? param_size(g, i) : pmax;
    g->part_cap = 32 * pmax;
    alloc((void**)&g->part, 4 * g->part_cap);
  }
  if (err != cudaSuccess) {
    free_guess(g);
    return cuda_status(err);
  }
  std::vector<double> ones(8 * g->nv, 1.0);
  cudaMemcpy(g->tau, ones.data(), 8 * ones.size(), cudaMemcpyHostToDevice);
  if (g->mlp)
    for (int st = 0; st < g->M; ++st) weight_copies(g, st, 0);
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
    DG_TRY(guess_forward(g, stage, false, s));
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
  host[2] = 0.0;
  const bool learn = g->mlp && g->nhist >= 2 && g->dvalid[stage];
  if (learn) {
    if (g->feat_stage != stage) DG_TRY(guess_features(g, stage, s));
    // target scale tau_m[v] = per-variable RMS of u - S - d_prev
    double* ts = g->vs + 3 * g->nv * VB;
    var_sumsq_kernel<<<dim3(VB, g->nv), 256, 0, s>>>(u, S, g->dprev[stage], 2, g->E, g->nv, g->nm,
                                                     ts);
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
                                             g->g[i], np, g->lr, g->b1, g->b2, g->eps, c1, c2);
      }
      weight_copies(g, stage, s);
      DG_LAUNCHED(9);
    }
    if (iters > 0) {
      DG_TRY(guess_loss(g, stage, ld, s));
      DG_CUDA(cudaMemcpyAsync(host + 1, ld, 8, cudaMemcpyDeviceToHost, s));
    }
    DG_CUDA(cudaMemcpyAsync(host + 2, g->tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  // the converged increment becomes the extrapolation base of the next step
  increment_kernel<<<grid1(n), 256, 0, s>>>(u, S, n, g->dprev[stage]);
  DG_LAUNCHED(1);
  g->dvalid[stage] = 1;
  if (g->feat_stage == stage) g->feat_stage = -1;
  DG_CUDA(cudaStreamSynchronize(s));
  if (learn && *reinterpret_cast<const int*>(host + 2) != 0) return DG_ERR_TIMEOUT;
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
