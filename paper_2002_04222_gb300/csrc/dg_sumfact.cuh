// Sum-factorisation helpers shared by the residual and preconditioner
// kernels: compile-time sizes of one (dim, P, Q) instance, the generic
// one-axis tensor contraction, table staging and Gauss-grid indexing.
#pragma once
#include "dg_internal.h"

namespace dg {

template <int DIM, int P, int Q>
struct Cfg {
  static constexpr int N = P + 1;
  static constexpr int NV = DIM + 2;
  static constexpr int NM = DIM == 2 ? N * N : N * N * N;
  static constexpr int NQ = DIM == 2 ? Q * Q : Q * Q * Q;
  static constexpr int NF = DIM == 2 ? Q : Q * Q;
  static constexpr int NFACE = 2 * DIM;
  static constexpr int NFLD = 1 + DIM;
  static constexpr int NT = 256;
  static constexpr int EPB = DIM == 2 ? (NT / NQ > 0 ? NT / NQ : 1) : 1;
  static constexpr int Q2 = DIM == 2 ? 1 : Q;  // extent of axis 2 on the Gauss grid
  static constexpr int N2 = DIM == 2 ? 1 : N;
  static constexpr int TAB = Q * N + Q * Q + 2 * Q + N * N + Q;  // doubles of staged tables
  // shared memory (doubles) per block
  static constexpr int VOL_SM = TAB + EPB * (NV * NM + (1 + DIM) * NV * NQ + (DIM == 2 ? NV * NQ : 0));
  static constexpr int LIFT_SM = TAB + EPB * ((DIM + 1) * NV * NQ + 2 * NV * NQ);
  // shared memory (doubles) for a runtime number of elements per block
  static constexpr int vol_sm(int e) {
    return TAB + e * (NV * NM + (1 + DIM) * NV * NQ + (DIM == 2 ? NV * NQ : 0));
  }
  static constexpr int lift_sm(int e) { return TAB + e * ((DIM + 1) * NV * NQ + 2 * NV * NQ); }
};

// (dim, P, Q) instances with general-geometry (curved / rotated) kernels
#define DG_CURVED_INSTANCES(X) X(2, 2, 4) X(2, 3, 5) X(3, 1, 3) X(3, 2, 5) X(3, 3, 6) X(3, 4, 8)
template <int D, int P, int Q>
constexpr bool has_curved() {
#define DG_HC(D_, P_, Q_) \
  if (D == D_ && P == P_ && Q == Q_) return true;
  DG_CURVED_INSTANCES(DG_HC)
#undef DG_HC
  return false;
}

// Y[r][o] = sum_k M[o_ax*MS0 + k*MS1] X[r][i(o, k)] for every replica r
// (element x variable) and output index o; axis AX changes extent NIN -> NOUT.
template <int I0, int I1, int I2, int AX, int NOUT, int MS0, int MS1, bool ACC>
__device__ __forceinline__ void contract(const double* __restrict__ X, double* __restrict__ Y,
                                         const double* __restrict__ M, int nrep) {
  constexpr int O0 = AX == 0 ? NOUT : I0;
  constexpr int O1 = AX == 1 ? NOUT : I1;
  constexpr int O2 = AX == 2 ? NOUT : I2;
  constexpr int NIN = AX == 0 ? I0 : (AX == 1 ? I1 : I2);
  constexpr int ISTR = AX == 0 ? 1 : (AX == 1 ? I0 : I0 * I1);
  constexpr int OSZ = O0 * O1 * O2, ISZ = I0 * I1 * I2;
  for (int idx = threadIdx.x; idx < nrep * OSZ; idx += blockDim.x) {
    const int r = idx / OSZ, o = idx - r * OSZ;
    const int o0 = o % O0, o1 = (o / O0) % O1, o2 = o / (O0 * O1);
    const int oa = AX == 0 ? o0 : (AX == 1 ? o1 : o2);
    const double* xp = X + r * ISZ + (AX == 0 ? 0 : o0) + (AX == 1 ? 0 : o1 * I0) +
                       (AX == 2 ? 0 : o2 * I0 * I1);
    double acc = ACC ? Y[idx] : 0.0;
#pragma unroll
    for (int k = 0; k < NIN; ++k) acc = fma(M[oa * MS0 + k * MS1], xp[k * ISTR], acc);
    Y[idx] = acc;
  }
}

template <int DIM, int P, int Q>
__device__ __forceinline__ void stage_tables(const Tables& tab, double* s) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N;
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) s[i] = tab.B[i];
  for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) s[Q * N + i] = tab.Dq[i];
  for (int i = threadIdx.x; i < Q; i += blockDim.x) {
    s[Q * N + Q * Q + i] = tab.lm[i];
    s[Q * N + Q * Q + Q + i] = tab.lp[i];
    s[Q * N + Q * Q + 2 * Q + N * N + i] = tab.w[i];
  }
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) s[Q * N + Q * Q + 2 * Q + i] = tab.Minv[i];
}

// Coordinates (q0, q1, q2) of Gauss-grid point q and face-point index of the
// face normal to direction r.
template <int DIM, int Q>
__device__ __forceinline__ void grid_coords(int q, int* c) {
  c[0] = q % Q;
  c[1] = (q / Q) % Q;
  c[2] = DIM == 3 ? q / (Q * Q) : 0;
}
template <int DIM, int Q>
__device__ __forceinline__ int face_point(const int* c, int r) {
  if (DIM == 2) return c[1 - r];
  const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
  return c[t0] + Q * c[t1];
}

}  // namespace dg
