// Device building blocks of the BRJ apply (Eq. precond-Jacobi), shared by the
// separate off-diagonal and block kernels (dg_precond.cu) and the fused
// one-kernel sweep (dg_sweep.cu): the per-element off-diagonal product, the
// per-element product with a transposed inverse block, and the instance list
// of (dimension, P, Q) the preconditioner is built for.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>
#include "dg_internal.h"
#include "dg_sumfact.cuh"

namespace dg {

__host__ __device__ constexpr int round_up8(int x) { return (x + 7) & ~7; }

// tensor index (m_0, m_1, m_2) of mode m (m_0 fastest)
template <int DIM, int N>
__device__ __forceinline__ void mode_coords(int m, int* mc) {
  mc[0] = m % N;
  mc[1] = (m / N) % N;
  mc[2] = DIM == 3 ? m / (N * N) : 0;
}

#define DG_PREC_INSTANCES(X)                                                                  \
  X(2, 1, 3) X(2, 2, 3) X(2, 2, 4) X(2, 3, 5) X(2, 4, 6) X(2, 5, 7) X(2, 6, 8) X(3, 1, 3) \
  X(3, 2, 4) X(3, 2, 5) X(3, 3, 5) X(3, 3, 6) X(3, 4, 6) X(3, 4, 8)

// Hint that brings the 16-byte-aligned interior of [p, p + bytes) of global
// memory toward L2 (bulk prefetch: no registers, no shared memory, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const size_t g = __cvta_generic_to_global(p);
  const size_t a = (g + 15) & ~(size_t)15, b = (g + bytes) & ~(size_t)15;
  if (b > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                 : "memory");
}

// The off-diagonal product of element e by one block of NTH threads: the
// neighbour face values are evaluated from the neighbour's face-mode
// coefficients (2-D sum factorisation), multiplied by the stored neighbour
// trace Jacobians, lifted onto the face modes and multiplied by the inverse
// mass matrix, all in the apply precision TA; emit(i, y_i) receives
// y_e = q_e + dt_a M^-1 (...) entry by entry (i = v N_m + m).
template <int DIM, int P, int Q, typename TA, typename TJ, bool CV, int NTH, class Emit>
__device__ __forceinline__ void offdiag_element(const Tables& tab, const ElemGeo* __restrict__ geo,
                                                const double* __restrict__ minv,
                                                const TJ* __restrict__ Jo,
                                                const int32_t* __restrict__ nbr,
                                                const double* __restrict__ qh,
                                                const double* __restrict__ q, double dta, int e,
                                                Emit emit) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NF = C::NF;
  constexpr int NS = DIM == 2 ? N : N * N;        // face-slice modes
  constexpr int NT = DIM == 2 ? 1 : Q * N;        // half-transformed slice per variable
  __shared__ TA sB[Q * N], sMi[N * N];
  __shared__ TA cs[2 * DIM * NV * NS];            // neighbour face-slice coefficients
  __shared__ TA ct[2 * DIM * NV * NT];
  __shared__ TA tr[2 * DIM * NV * NF];            // neighbour face values, then Jo . values
  __shared__ TA L0[NV * NM], L1[NV * NM];
  // the element's neighbour trace Jacobians (one face per thread) and q are
  // read late; start their way from DRAM now
  if (threadIdx.x < 2 * DIM)
    prefetch_l2(Jo + ((long long)e * 2 * DIM + threadIdx.x) * NV * NV * NF, sizeof(TJ) * NV * NV * NF);
  else if (threadIdx.x == 2 * DIM)
    prefetch_l2(q + (long long)e * NV * NM, sizeof(double) * NV * NM);
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) sB[i] = (TA)tab.B[i];
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sMi[i] = (TA)tab.Minv[i];
  // gather the neighbour's face slice (modes with m_r = vertex of its face)
  for (int i = threadIdx.x; i < 2 * DIM * NV * NS; i += blockDim.x) {
    const int a = i % NS, v = (i / NS) % NV, lf = i / (NS * NV);
    const int nb = nbr[e * 2 * DIM + lf];
    TA val = (TA)0;
    if (nb >= 0) {
      const int en = nb / (2 * DIM), fn = nb % (2 * DIM);
      const int r = fn >> 1, vert = (fn & 1) ? P : 0;
      int mc[3] = {0, 0, 0};
      mc[r] = vert;
      if (DIM == 2) {
        mc[1 - r] = a;
      } else {
        const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
        mc[t0] = a % N;
        mc[t1] = a / N;
      }
      val = (TA)qh[((long long)en * NV + v) * NM + mc[0] + N * (mc[1] + N * mc[2])];
    }
    cs[i] = val;
  }
  __syncthreads();
  // face values: contract the first tangential mode index, then the second
  if (DIM == 2) {
    for (int i = threadIdx.x; i < 2 * DIM * NV * NF; i += blockDim.x) {
      const int p = i % NF, fv = i / NF;
      TA acc = (TA)0;
#pragma unroll
      for (int a = 0; a < N; ++a) acc += sB[p * N + a] * cs[fv * NS + a];
      tr[i] = acc;
    }
  } else {
    for (int i = threadIdx.x; i < 2 * DIM * NV * NT; i += blockDim.x) {
      const int p0 = i % Q, b = (i / Q) % N, fv = i / NT;
      TA acc = (TA)0;
#pragma unroll
      for (int a = 0; a < N; ++a) acc += sB[p0 * N + a] * cs[fv * NS + a + N * b];
      ct[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * DIM * NV * NF; i += blockDim.x) {
      const int p = i % NF, fv = i / NF;
      const int p0 = p % Q, p1 = p / Q;
      TA acc = (TA)0;
#pragma unroll
      for (int b = 0; b < N; ++b) acc += sB[p1 * N + b] * ct[fv * NT + p0 + Q * b];
      tr[i] = acc;
    }
  }
  __syncthreads();
  // Jo . values (in registers, then back to tr)
  TA prod[(2 * DIM * NV * NF + NTH - 1) / NTH];
#pragma unroll
  for (int t = 0; t < (2 * DIM * NV * NF + NTH - 1) / NTH; ++t) {
    const int i = threadIdx.x + NTH * t;
    TA s2 = (TA)0;
    if (i < 2 * DIM * NV * NF) {
      const int p = i % NF, k = (i / NF) % NV, lf = i / (NF * NV);
      if (nbr[e * 2 * DIM + lf] >= 0) {
        const TJ* j = Jo + (((long long)e * 2 * DIM + lf) * NV + k) * NV * NF + p;
        const TA* t0 = tr + lf * NV * NF + p;
#pragma unroll
        for (int l = 0; l < NV; ++l) s2 += (TA)j[l * NF] * t0[l * NF];
      }
    }
    prod[t] = s2;
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < (2 * DIM * NV * NF + NTH - 1) / NTH; ++t) {
    const int i = threadIdx.x + NTH * t;
    if (i < 2 * DIM * NV * NF) tr[i] = prod[t];
  }
  __syncthreads();
  if (DIM == 3) {
    // lift, first tangential direction: ct[lf][v][a][p1] = sum_p0 B[p0][a] tr[lf][v][p0 + Q p1]
    for (int i = threadIdx.x; i < 2 * DIM * NV * NT; i += blockDim.x) {
      const int p1 = i % Q, a = (i / Q) % N, fv = i / NT;
      const TA* c = tr + fv * NF + Q * p1;
      TA acc = (TA)0;
#pragma unroll
      for (int p0 = 0; p0 < Q; ++p0) acc += sB[p0 * N + a] * c[p0];
      ct[i] = acc;
    }
    __syncthreads();
  }
  // lift onto the face modes of this element (second tangential direction in 3-D)
  for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) {
    const int v = i / NM, m = i % NM;
    int mc[3];
    mode_coords<DIM, N>(m, mc);
    TA s2 = (TA)0;
#pragma unroll
    for (int lf = 0; lf < 2 * DIM; ++lf) {
      const int r = lf >> 1, vert = (lf & 1) ? P : 0;
      if (mc[r] != vert) continue;
      if (DIM == 2) {
        const TA* c = tr + (lf * NV + v) * NF;
        const int a = mc[1 - r];
#pragma unroll
        for (int p = 0; p < Q; ++p) s2 += sB[p * N + a] * c[p];
      } else {
        const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
        const int a = mc[t0], b = mc[t1];
        const TA* c = ct + (lf * NV + v) * NT + a * Q;
#pragma unroll
        for (int p1 = 0; p1 < Q; ++p1) s2 += sB[p1 * N + b] * c[p1];
      }
    }
    L0[i] = s2;
  }
  __syncthreads();
  if constexpr (CV) {
    // dense inverse mass matrix of the element (symmetric)
    // (one thread per mode m: each entry of M^-1 is read once for all variables)
    const double* Me = minv + (long long)e * NM * NM;
    for (int m = threadIdx.x; m < NM; m += blockDim.x) {
      TA s2[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) s2[v] = (TA)0;
      for (int kk = 0; kk < NM; ++kk) {
        const TA mk = (TA)Me[kk * NM + m];
#pragma unroll
        for (int v = 0; v < NV; ++v) s2[v] += mk * L0[v * NM + kk];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const long long gi = ((long long)e * NV + v) * NM + m;
        emit(v * NM + m, q[gi] + dta * (double)s2[v]);
      }
    }
    return;
  }
  // inverse mass matrix, axis by axis
  TA* src = L0;
  TA* dst = L1;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) {
      const int m = i % NM;
      int mc[3];
      mode_coords<DIM, N>(m, mc);
      const int str = ax == 0 ? 1 : (ax == 1 ? N : N * N);
      const int base = i - mc[ax] * str;
      TA s2 = (TA)0;
#pragma unroll
      for (int kk = 0; kk < N; ++kk) s2 += sMi[mc[ax] * N + kk] * src[base + kk * str];
      dst[i] = s2;
    }
    __syncthreads();
    TA* t = src;
    src = dst;
    dst = t;
  }
  const double idet = geo[e].idet;
  const double sc = dta * idet;
  for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) {
    const long long gi = (long long)e * NV * NM + i;
    emit(i, q[gi] + sc * (double)src[i]);
  }
}

// out = omega D^-1 y + (1-omega) qprev with the block stored transposed
// (At[c][r] = (D^-1)[r][c], rows padded to ld): each thread owns VW
// consecutive rows and streams the columns with one 16-byte load per column,
// so a warp reads 512 contiguous bytes per column and needs no reduction;
// SPLIT thread groups share the columns and add their partial sums in shared
// memory.  Arithmetic in TA (FP64 for FP64 blocks, FP32 otherwise).
template <typename TB>
struct Vec16;
template <>
struct Vec16<double> {
  static constexpr int W = 2;
  using TA = double;
  using R = double2;  // one 16-byte load
  __device__ static R ld(const double* p) { return __ldcs(reinterpret_cast<const double2*>(p)); }
  __device__ static void cvt(const R& v, double* o) {
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct Vec16<float> {
  static constexpr int W = 4;
  using TA = float;
  using R = float4;
  __device__ static R ld(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
  __device__ static void cvt(const R& v, float* o) {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};
template <>
struct Vec16<__nv_bfloat16> {
  static constexpr int W = 8;
  using TA = float;
  using R = uint4;
  __device__ static R ld(const __nv_bfloat16* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
  __device__ static void cvt(const R& v, float* o) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __bfloat1622float2(h[t]);
      o[2 * t] = f.x;
      o[2 * t + 1] = f.y;
    }
  }
};

// The block product of element e: out_e = omega D_e^-1 y_e + (1-omega) qprev_e
// with y_e already in shared memory (sy, nb entries); part holds split x ld
// partial sums.
template <typename TB>
__device__ __forceinline__ void diag_element(const TB* __restrict__ blocks, int nb, int ld,
                                             int split, const typename Vec16<TB>::TA* sy,
                                             typename Vec16<TB>::TA* part,
                                             const double* __restrict__ qprev, double omega,
                                             double* __restrict__ out, int e) {
  using V = Vec16<TB>;
  using TA = typename V::TA;
  constexpr int W = V::W;
  const int nrq = ld / W;                                // row groups
  const int rq = threadIdx.x % nrq, sp = threadIdx.x / nrq;
  const int chunk = (nb + split - 1) / split;
  const int c0 = sp * chunk, c1 = min(nb, c0 + chunk);
  TA acc[W];
#pragma unroll
  for (int t = 0; t < W; ++t) acc[t] = (TA)0;
  if (sp < split) {
    const TB* A = blocks + (long long)e * nb * ld + rq * W;
    // U columns per step, their loads issued together; the ragged last step
    // predicates its loads instead of running a one-load-at-a-time remainder
    constexpr int U = sizeof(TB) == 2 ? 8 : 4;
    for (int c = c0; c < c1; c += U) {
      typename V::R r[U];  // raw 16-byte loads, widened when used
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c + u < c1) r[u] = V::ld(A + (long long)(c + u) * ld);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c + u < c1) {
          TA a[W];
          V::cvt(r[u], a);
          const TA yc = sy[c + u];
#pragma unroll
          for (int t = 0; t < W; ++t) acc[t] += a[t] * yc;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < W; ++t) part[sp * ld + rq * W + t] = acc[t];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    TA s2 = (TA)0;
    for (int k = 0; k < split; ++k) s2 += part[k * ld + r];
    const long long gi = (long long)e * nb + r;
    out[gi] = omega == 1.0 ? (double)s2 : omega * (double)s2 + (1.0 - omega) * qprev[gi];
  }
}

// FP32/FP64 blocks launch at most 256 threads, BF16 blocks up to 512 (twice the
// column groups, half the bytes each); registers capped so that 6 and 2 CTAs
// fit an SM
#define DG_DIAG_BOUNDS(TB) __launch_bounds__(sizeof(TB) == 2 ? 512 : 256, sizeof(TB) == 2 ? 2 : 6)

}  // namespace dg
