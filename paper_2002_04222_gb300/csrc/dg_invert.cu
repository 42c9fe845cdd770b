// In-place inversion of the BRJ diagonal blocks (Eq. precond-Jacobi needs
// D^-1; the paper factors and inverts each block, Sec. 4.2.2): blocked
// Gauss-Jordan elimination with partial pivoting, one CTA per element.
//
// Each panel of B = 32 pivot columns is factorised with the panel held in
// registers, one row per thread: a pivot step is a block-wide argmax, the
// exchange of two register rows through shared memory and a rank-1 update of
// every thread's own row, two barriers per pivot and no global memory access.
// The panel's row interchanges reach the other columns once per panel: each
// column's thread gathers the permuted pivot rows and the displaced rows
// from global memory in one batch of independent loads, into registers.  The
// other columns then take the rank-32 update A[:, c] += (T_K - E_K) A[K, c]
// with T_K the panel's transformation (shared memory, broadcast reads) and
// A[K, c] in those registers.  The inverse's columns are un-permuted at the end by a gather of
// 32-row tiles staged in shared memory.
#include <cuda_bf16.h>
#include "dg_internal.h"
#include "dg_precond.h"

namespace dg {

constexpr int IR_B = 32;   // panel width

template <typename T>
struct Vec4T;
template <>
struct Vec4T<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct Vec4T<double> {
  using V = double2;
  static constexpr int W = 2;
};

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) brj_invert_rows_kernel(T* __restrict__ blocks, int nb,
                                                               int ld, int* __restrict__ fail) {
  constexpr int B = IR_B;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);              // [nb][B] panel (T_K columns), later tiles
  T* S1 = P + (size_t)nb * B;                      // [B] pivot row exchange
  T* S2 = S1 + B;                                  // [B]
  int* perm = reinterpret_cast<int*>(S2 + B);      // [nb] pivot row of each step
  int* srcK = perm + nb;                           // [B] source row of each K row
  int* outRow = srcK + B;                          // [B] displaced rows outside K
  int* srcO = outRow + B;                          // [B] their source rows
  int* track = srcO + B;                           // [B] pivot rows of the panel
  int* sg = track + B;                             // [nb] final column permutation
  __shared__ T redv[32];
  __shared__ int redi[32];
  __shared__ int nout_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  T* A = blocks + (long long)blockIdx.x * nb * ld;
  for (int k0 = 0; k0 < nb; k0 += B) {
    const int bw = nb - k0 < B ? nb - k0 : B;
    // ---- panel rows into registers (row tid)
    T row[B];
#pragma unroll
    for (int j = 0; j < B; ++j) row[j] = (T)0;
    if (tid < nb) {
      const T* src = A + (long long)tid * ld + k0;
      if (bw == B) {
        using V = typename Vec4T<T>::V;
        constexpr int W = Vec4T<T>::W;
#pragma unroll
        for (int q = 0; q < B / W; ++q) {
          const V v = *reinterpret_cast<const V*>(src + q * W);
          const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int w = 0; w < W; ++w) row[q * W + w] = pv[w];
        }
      } else {
#pragma unroll
        for (int j = 0; j < B; ++j)
          if (j < bw) row[j] = src[j];
      }
    }
    // ---- factorise the panel (unrolled: the register row is indexed statically)
    bool ok = true;
#pragma unroll
    for (int j = 0; j < B; ++j) {
      if (j >= bw) break;
      const int k = k0 + j;
      // pivot: largest |row[j]| over rows >= k, lowest index on ties
      T best = (T)-1;
      int bi = nb;
      if (tid >= k && tid < nb) {
        best = fabs(row[j]);
        bi = tid;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        redv[warp] = best;
        redi[warp] = bi;
      }
      __syncthreads();
      T pmag = redv[0];
      int pr = redi[0];
      for (int w = 1; w < nwarp; ++w) {
        const T ov = redv[w];
        const int oi = redi[w];
        if (ov > pmag || (ov == pmag && oi < pr)) {
          pmag = ov;
          pr = oi;
        }
      }
      if (!(pmag > (T)0) || pr >= nb) {  // singular (or non-finite) block: leave uniformly
        ok = false;
        break;
      }
      // exchange rows k and pr through shared memory; the pivot row is pr's
      if (tid == pr) {
#pragma unroll
        for (int jj = 0; jj < B; ++jj) S1[jj] = row[jj];
      }
      if (tid == k && pr != k) {
#pragma unroll
        for (int jj = 0; jj < B; ++jj) S2[jj] = row[jj];
      }
      if (tid == 0) {
        perm[k] = pr;
        track[j] = pr;
      }
      __syncthreads();
      const T ipiv = (T)1 / S1[j];
      if (tid == k) {
#pragma unroll
        for (int jj = 0; jj < B; ++jj) row[jj] = jj == j ? ipiv : S1[jj] * ipiv;
      } else if (tid < nb) {
        if (tid == pr) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) row[jj] = S2[jj];
        }
        // rank-1 update with the scaled pivot row, whose pivot entry is ipiv
        // (the pivot column becomes the transformation's column)
        const T f = row[j];
#pragma unroll
        for (int jj = 0; jj < B; ++jj)
          row[jj] = jj == j ? -f * ipiv : row[jj] - f * (S1[jj] * ipiv);
      }
      // (the next step's first barrier orders these reads of S1/S2 before
      // their next writes)
    }
    if (!ok) {
      if (tid == 0) atomicExch(fail, 1);
      return;
    }
    // ---- panel to shared memory and to its columns of A (T_K)
    if (tid < nb) {
      T* dst = A + (long long)tid * ld + k0;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        P[tid * B + jj] = row[jj];
        if (jj < bw) dst[jj] = row[jj];
      }
    }
    // source rows of the panel's permutation: simulate the swaps on the
    // affected rows (K and the rows exchanged with them)
    if (tid == 0) {
      int nout = 0;
      // K rows start as themselves; displaced rows are recorded as they appear
      for (int j = 0; j < B; ++j) srcK[j] = k0 + j;
      for (int j = 0; j < bw; ++j) {
        const int pr = track[j];
        if (pr == k0 + j) continue;
        if (pr < k0 + bw) {   // swap inside K
          const int a = srcK[j];
          srcK[j] = srcK[pr - k0];
          srcK[pr - k0] = a;
        } else {
          int o = 0;
          while (o < nout && outRow[o] != pr) ++o;
          if (o == nout) {
            outRow[nout] = pr;
            srcO[nout] = pr;
            ++nout;
          }
          const int a = srcK[j];
          srcK[j] = srcO[o];
          srcO[o] = a;
        }
      }
      nout_s = nout;
    }
    __syncthreads();
    const int nout = nout_s;
    // ---- other columns: apply the interchanges, then the rank-B update
    if (tid < nb && (tid < k0 || tid >= k0 + bw)) {
      const int c = tid;
      T ak[B], ov[B];
#pragma unroll
      for (int j = 0; j < B; ++j) ak[j] = j < bw ? A[(long long)srcK[j] * ld + c] : (T)0;
#pragma unroll
      for (int o = 0; o < B; ++o) ov[o] = o < nout ? A[(long long)srcO[o] * ld + c] : (T)0;
#pragma unroll
      for (int o = 0; o < B; ++o)
        if (o < nout) A[(long long)outRow[o] * ld + c] = ov[o];
      // rows outside K: A[i][c] + sum_j T[i][j] ak[j]; rows in K: sum_j T[i][j] ak[j];
      // eight rows per batch, the next batch's loads issued before this
      // batch's products (different rows of the column: no overlap)
      auto load8 = [&](int i0, T* v) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int i = i0 + t;
          v[t] = (i < nb && (i < k0 || i >= k0 + bw)) ? A[(long long)i * ld + c] : (T)0;
        }
      };
      T cur[8], nxt[8];
      load8(0, cur);
      for (int i0 = 0; i0 < nb; i0 += 8) {
        if (i0 + 8 < nb) load8(i0 + 8, nxt);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int i = i0 + t;
          if (i >= nb) break;
          const T* u = P + i * B;
          T a = cur[t];
#pragma unroll
          for (int j = 0; j < B; ++j) a += u[j] * ak[j];
          cur[t] = a;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (i0 + t < nb) A[(long long)(i0 + t) * ld + c] = cur[t];
#pragma unroll
        for (int t = 0; t < 8; ++t) cur[t] = nxt[t];
      }
    }
    __syncthreads();
  }
  // ---- un-permute the inverse's columns: out[:, c] = A[:, sigma(c)], sigma
  // the composition of the column exchanges taken in reverse order
  if (tid == 0) {
    for (int c = 0; c < nb; ++c) sg[c] = c;
    for (int k = nb - 1; k >= 0; --k) {
      const int pr = perm[k];
      if (pr != k) {
        const int a = sg[k];
        sg[k] = sg[pr];
        sg[pr] = a;
      }
    }
  }
  __syncthreads();
  // 32-row tiles through shared memory
  for (int r0 = 0; r0 < nb; r0 += B) {
    const int rows = nb - r0 < B ? nb - r0 : B;
    for (int i = tid; i < rows * nb; i += blockDim.x) {
      const int r = i / nb, c = i - r * nb;
      P[r * nb + c] = A[(long long)(r0 + r) * ld + c];
    }
    __syncthreads();
    for (int i = tid; i < rows * nb; i += blockDim.x) {
      const int r = i / nb, c = i - r * nb;
      A[(long long)(r0 + r) * ld + c] = P[r * nb + sg[c]];
    }
    __syncthreads();
  }
}

size_t invert_rows_smem(int nb, size_t elem) {
  return elem * ((size_t)nb * IR_B + 2 * IR_B) + sizeof(int) * ((size_t)2 * nb + 4 * IR_B);
}

// thread bounds: one thread per row (and per column), registers for the
// panel row, the 32 pivot-row values and the displaced rows of a column
constexpr int IR_MAXT_F32 = 640, IR_MAXT_F64 = 384;

bool invert_rows_supported(int nb, bool fp64) {
  return nb <= (fp64 ? IR_MAXT_F64 : IR_MAXT_F32) &&
         invert_rows_smem(nb, fp64 ? 8 : 4) <= 227 * 1024;
}

dg_status launch_invert_rows(void* blocks, bool fp64, int E, int nb, int ld, int* fail,
                             cudaStream_t s) {
  if (!invert_rows_supported(nb, fp64)) return DG_ERR_UNSUPPORTED;
  const int threads = (nb + 31) / 32 * 32;
  const size_t sm = invert_rows_smem(nb, fp64 ? 8 : 4);
  if (fp64) {
    auto kern = brj_invert_rows_kernel<double, IR_MAXT_F64>;
    DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    DG_PROF(K_BRJ_INVERT, s, kern<<<E, threads, sm, s>>>((double*)blocks, nb, ld, fail));
  } else {
    auto kern = brj_invert_rows_kernel<float, IR_MAXT_F32>;
    DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    DG_PROF(K_BRJ_INVERT, s, kern<<<E, threads, sm, s>>>((float*)blocks, nb, ld, fail));
  }
  return DG_OK;  // (the caller counts the launch and checks it)
}

}  // namespace dg
