// In-place inversion of the BRJ diagonal blocks (Eq. precond-Jacobi needs
// D^-1; the paper factors and inverts each block, Sec. 4.2.2): blocked
// Gauss-Jordan elimination with partial pivoting, one CTA per element.
//
// Each panel of B = 32 pivot columns is factorised with the panel held in
// registers, one row per thread.  The pivot loop is not unrolled: after each
// pivot the register row is rotated left by one place, so the current pivot
// column is always row[0] and the loop body (a few hundred instructions)
// stays in the instruction cache; after the panel the row is back in column
// order.  A pivot step has one barrier: every warp's best candidate row and
// the current row k are written to double-buffered shared slots before it,
// and every thread picks the winner after it (FP32: one 64-bit key, the
// magnitude's bits above the complemented row index, reduced by shuffles
// within and across warps; lowest row on ties).  The panel's row
// interchanges reach the other columns once per panel: a row map built from
// the panel's pivots gives each column's thread the pivot rows and the
// displaced rows to gather from global memory in one batch of independent
// loads.  The other columns then take the rank-32 update
// A[:, c] += (T_K - E_K) A[K, c] with T_K the panel's transformation (shared
// memory, broadcast reads) and A[K, c] in registers, LA rows of loads in
// flight per thread.  The inverse's columns are un-permuted at the end by a
// gather of 32-row tiles staged in shared memory.  The arithmetic (each
// product, sum and its order) is that of the plain Gauss-Jordan sweep with
// partial pivoting, so the result does not depend on the launch shape.
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

// largest (value, lowest index) over the warp
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    k = ok > k ? ok : k;
  }
  return k;
}

// shared memory: T_K panel [nb][B], candidate rows [2][MAXT/32][B], row k
// [2][B] (T); pivots [nb], panel pivots [B], displaced rows and their
// sources [B] each, row/column map [nb] (int)
template <typename T>
__host__ __device__ constexpr size_t invert_rows_smem_t(int nb, int maxt) {
  return sizeof(T) * ((size_t)nb * IR_B + 2 * (size_t)(maxt / 32) * IR_B + 2 * IR_B) +
         sizeof(int) * ((size_t)2 * nb + 3 * IR_B);
}

template <typename T, int MAXT, int MINB, int LA>
__global__ void __launch_bounds__(MAXT, MINB) brj_invert_rows_kernel(T* __restrict__ blocks, int nb,
                                                                     int ld, int* __restrict__ fail) {
  constexpr int B = IR_B;
  constexpr int MW = MAXT / 32;
  constexpr bool KEY = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);                 // [nb][B] panel (T_K), later tiles
  T* cand = P + (size_t)nb * B;                       // [2][MW][B] best row of each warp
  T* rowk = cand + 2 * MW * B;                        // [2][B] row k before the exchange
  int* perm = reinterpret_cast<int*>(rowk + 2 * B);   // [nb] pivot row of each step
  int* track = perm + nb;                             // [B] pivot rows of the panel
  int* outRow = track + B;                            // [B] displaced rows outside K
  int* srcO = outRow + B;                             // [B] their source rows
  int* sg = srcO + B;                                 // [nb] row map, then column map
  __shared__ unsigned long long keys[2][32];
  __shared__ T redv[2][32];
  __shared__ int redi[2][32];
  __shared__ int nout_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  T* A = blocks + (long long)blockIdx.x * nb * ld;
  int buf = 0;
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
    // ---- factorise the panel: pivot column j is row[0] at step j
    bool ok = true;
#pragma unroll 1
    for (int j = 0; j < bw; ++j) {
      const int k = k0 + j;
      T* cw = cand + (buf * MW + warp) * B;
      int pr;
      bool good;
      if constexpr (KEY) {
        // |a| >= 0 orders as its bits; NaN maps above every number and fails
        unsigned long long key = 0;
        if (tid >= k && tid < nb) {
          const float m = fabsf((float)row[0]);
          const unsigned mb = m >= 0.0f ? __float_as_uint(m) : 0xFFFFFFFFu;
          key = ((unsigned long long)mb << 32) | (unsigned)(0xFFFFFFFFu - tid);
        }
        key = warp_max_u64(key);
        const int bi = key ? (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFu)) : -1;
        if (tid == bi) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) cw[jj] = row[jj];
        }
        if (tid == k) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) rowk[buf * B + jj] = row[jj];
        }
        if (lane == 0) keys[buf][warp] = key;
        __syncthreads();
        const unsigned long long g = warp_max_u64(lane < nwarp ? keys[buf][lane] : 0ull);
        const unsigned hi = (unsigned)(g >> 32);
        good = hi != 0u && hi <= 0x7F800000u;
        pr = good ? (int)(0xFFFFFFFFu - (unsigned)(g & 0xFFFFFFFFu)) : nb;
      } else {
        T best = (T)-1;
        int bi = nb;
        if (tid >= k && tid < nb) {
          best = fabs(row[0]);
          bi = tid;
        }
        warp_argmax(best, bi);
        if (tid == bi) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) cw[jj] = row[jj];
        }
        if (tid == k) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) rowk[buf * B + jj] = row[jj];
        }
        if (lane == 0) {
          redv[buf][warp] = best;
          redi[buf][warp] = bi;
        }
        __syncthreads();
        T pmag = lane < nwarp ? redv[buf][lane] : (T)-1;
        pr = lane < nwarp ? redi[buf][lane] : nb;
        warp_argmax(pmag, pr);
        good = pmag > (T)0 && pr < nb;
      }
      if (!good) {  // singular (or non-finite) block: leave uniformly
        ok = false;
        break;
      }
      // the pivot row is the winning warp's candidate; row k's old values
      // go to row pr
      const T* S1 = cand + (buf * MW + (pr >> 5)) * B;
      const T* S2 = rowk + buf * B;
      if (tid == 0) {
        perm[k] = pr;
        track[j] = pr;
      }
      const T ipiv = (T)1 / S1[0];
      T r0;
      if (tid == k) {
        r0 = ipiv;
#pragma unroll
        for (int jj = 1; jj < B; ++jj) row[jj] = S1[jj] * ipiv;
      } else {
        if (tid == pr) {
#pragma unroll
          for (int jj = 0; jj < B; ++jj) row[jj] = S2[jj];
        }
        // rank-1 update with the scaled pivot row, whose pivot entry is ipiv
        // (the pivot column becomes the transformation's column)
        const T f = row[0];
        r0 = -f * ipiv;
#pragma unroll
        for (int jj = 1; jj < B; ++jj) row[jj] = row[jj] - f * (S1[jj] * ipiv);
      }
#pragma unroll
      for (int jj = 0; jj < B - 1; ++jj) row[jj] = row[jj + 1];
      row[B - 1] = r0;
      // (slots of buffer buf are written again two steps later, after the
      // next step's barrier, which every thread reaches after these reads)
      buf ^= 1;
    }
    if (!ok) {
      if (tid == 0) atomicExch(fail, 1);
      return;
    }
    // a ragged last panel: finish the rotation to column order
#pragma unroll 1
    for (int r = bw; r < B; ++r) {
      const T r0 = row[0];
#pragma unroll
      for (int jj = 0; jj < B - 1; ++jj) row[jj] = row[jj + 1];
      row[B - 1] = r0;
    }
    // ---- panel to shared memory and to its columns of A (T_K)
    if (tid < nb) {
      T* dst = A + (long long)tid * ld + k0;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) P[tid * B + jj] = row[jj];
      if (bw == B) {
        using V = typename Vec4T<T>::V;
        constexpr int W = Vec4T<T>::W;
#pragma unroll
        for (int q = 0; q < B / W; ++q) {
          V v;
          T* pv = reinterpret_cast<T*>(&v);
#pragma unroll
          for (int w = 0; w < W; ++w) pv[w] = row[q * W + w];
          *reinterpret_cast<V*>(dst + q * W) = v;
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < B; ++jj)
          if (jj < bw) dst[jj] = row[jj];
      }
      sg[tid] = tid;
    }
    __syncthreads();
    // row map of the panel's interchanges: sg[r] = the row whose old values
    // row r now holds (in order: a later exchange may move a row an earlier
    // one moved; each exchanges k0 + j with a row >= k0 + j)
    if (tid == 0) {
      for (int j = 0; j < bw; ++j) {
        const int pr = track[j];
        const int a = sg[k0 + j], b = sg[pr];
        sg[k0 + j] = b;
        sg[pr] = a;
      }
    }
    __syncthreads();
    // rows outside the panel that an exchange displaced, each listed once
    if (warp == 0) {
      const int r = lane < bw ? track[lane] : -1;
      const bool outside = r >= k0 + bw;
      const unsigned same = __match_any_sync(0xffffffffu, outside ? r : -1 - lane);
      const bool first = outside && (__ffs(same) - 1) == lane;
      const unsigned fm = __ballot_sync(0xffffffffu, first);
      if (first) {
        const int pos = __popc(fm & ((1u << lane) - 1u));
        outRow[pos] = r;
        srcO[pos] = sg[r];
      }
      if (lane == 0) nout_s = __popc(fm);
    }
    __syncthreads();
    const int nout = nout_s;
    // ---- other columns: apply the interchanges, then the rank-B update
    if (tid < nb && (tid < k0 || tid >= k0 + bw)) {
      const int c = tid;
      T ak[B];
      {
        T ov[B];
#pragma unroll
        for (int j = 0; j < B; ++j) ak[j] = j < bw ? A[(long long)sg[k0 + j] * ld + c] : (T)0;
#pragma unroll
        for (int o = 0; o < B; ++o) ov[o] = o < nout ? A[(long long)srcO[o] * ld + c] : (T)0;
#pragma unroll
        for (int o = 0; o < B; ++o)
          if (o < nout) A[(long long)outRow[o] * ld + c] = ov[o];
      }
      // rows outside K: A[i][c] + sum_j T[i][j] ak[j]; rows in K: sum_j T[i][j] ak[j];
      // LA rows per batch, the next batch's loads issued before this
      // batch's products (different rows of the column: no overlap)
      auto load_rows = [&](int i0, T* v) {
#pragma unroll
        for (int t = 0; t < LA; ++t) {
          const int i = i0 + t;
          v[t] = (i < nb && (i < k0 || i >= k0 + bw)) ? A[(long long)i * ld + c] : (T)0;
        }
      };
      T cur[LA], nxt[LA];
      load_rows(0, cur);
      for (int i0 = 0; i0 < nb; i0 += LA) {
        if (i0 + LA < nb) load_rows(i0 + LA, nxt);
#pragma unroll
        for (int t = 0; t < LA; ++t) {
          const int i = i0 + t;
          if (i >= nb) break;
          const T* u = P + i * B;
          T a = cur[t];
#pragma unroll
          for (int j = 0; j < B; ++j) a += u[j] * ak[j];
          cur[t] = a;
        }
#pragma unroll
        for (int t = 0; t < LA; ++t)
          if (i0 + t < nb) A[(long long)(i0 + t) * ld + c] = cur[t];
#pragma unroll
        for (int t = 0; t < LA; ++t) cur[t] = nxt[t];
      }
    }
    __syncthreads();
  }
  // ---- un-permute the inverse's columns: out[:, c] = A[:, sigma(c)], sigma
  // the composition of the column exchanges taken in reverse order
  for (int c = tid; c < nb; c += blockDim.x) sg[c] = c;
  __syncthreads();
  if (tid == 0) {
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
  // 32-row tiles through shared memory, eight loads in flight per thread
  for (int r0 = 0; r0 < nb; r0 += B) {
    const int rows = nb - r0 < B ? nb - r0 : B;
    const int n = rows * nb;
    for (int i = tid; i < n; i += 8 * blockDim.x) {
      T v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int ii = i + t * blockDim.x;
        if (ii < n) {
          const int r = ii / nb, c = ii - r * nb;
          v[t] = A[(long long)(r0 + r) * ld + c];
        }
      }
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (i + t * blockDim.x < n) P[i + t * blockDim.x] = v[t];
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      const int r = i / nb, c = i - r * nb;
      A[(long long)(r0 + r) * ld + c] = P[r * nb + sg[c]];
    }
    __syncthreads();
  }
}

// launch shapes: one thread per row (and per column); FP32 blocks of up to
// 320 rows (P = 3) at two CTAs per SM with 16 rows of loads in flight, up
// to 640 rows (P = 4) at one; FP64 blocks of up to 384 rows
constexpr int IR_MAXT_F32S = 320, IR_MAXT_F32 = 640, IR_MAXT_F64 = 384;

bool invert_rows_supported(int nb, bool fp64) {
  return fp64 ? nb <= IR_MAXT_F64 && invert_rows_smem_t<double>(nb, IR_MAXT_F64) <= 227 * 1024
              : nb <= IR_MAXT_F32 && invert_rows_smem_t<float>(nb, IR_MAXT_F32) <= 227 * 1024;
}

template <typename T, int MAXT, int MINB, int LA>
static dg_status launch_rows(T* blocks, int E, int nb, int ld, int* fail, cudaStream_t s) {
  auto kern = brj_invert_rows_kernel<T, MAXT, MINB, LA>;
  const int threads = (nb + 31) / 32 * 32;
  const size_t sm = invert_rows_smem_t<T>(nb, MAXT);
  DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  DG_PROF(K_BRJ_INVERT, s, kern<<<E, threads, sm, s>>>(blocks, nb, ld, fail));
  return DG_OK;
}

dg_status launch_invert_rows(void* blocks, bool fp64, int E, int nb, int ld, int* fail,
                             cudaStream_t s) {
  if (!invert_rows_supported(nb, fp64)) return DG_ERR_UNSUPPORTED;
  if (fp64) return launch_rows<double, IR_MAXT_F64, 1, 8>((double*)blocks, E, nb, ld, fail, s);
  if (nb <= IR_MAXT_F32S)
    return launch_rows<float, IR_MAXT_F32S, 2, 16>((float*)blocks, E, nb, ld, fail, s);
  return launch_rows<float, IR_MAXT_F32, 1, 8>((float*)blocks, E, nb, ld, fail, s);
  // (the caller counts the launch and checks it)
}

}  // namespace dg
