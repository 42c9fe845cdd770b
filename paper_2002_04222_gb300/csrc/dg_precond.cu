// Block relaxed Jacobi preconditioner BRJ(J) of Sec. 4.2.2.
//
// Build (Eq. Jacobian-matrix-form, -form2, numerical-Jac-on-traces):
//   brj_weights_kernel  state and gradient at the Gauss points (sum
//                       factorisation), exact flux Jacobians dH_j/dQ (dual
//                       numbers) and dH_j/d(grad_i Q) (G is linear in grad Q),
//                       times w|J| and the reference metric;
//   brj_tracejac_kernel one thread per face point: one-sided differences of
//                       the numerical flux in each trace variable (boundary
//                       states re-evaluated), chi_k = sqrt(eps)||u_k||;
//   brj_block_kernel    one block per (element, variable pair): the volume
//                       terms sum_q (D_j B)^T W (B; D_i B) by sum factorisation
//                       plus the own-side trace term B_f^T J B_f, then
//                       D = I - dt_a M^-1 X, stored transposed;
//   brj_invert_blocked_kernel  blocked in-place Gauss-Jordan inversion with
//                       partial pivoting of every diagonal block.
// Apply (Eq. precond-Jacobi): q^1 = D^-1 q; q^j = D^-1 (q - (L+U) q^(j-1)), the
// off-diagonal product formed on the fly from the neighbour traces and the
// stored neighbour trace Jacobians (brj_offdiag_kernel, which also evaluates the
// neighbour traces), the block product by brj_diag_cm_kernel (HBM-bound batched
// GEMV streaming the transposed blocks column by column); both on the
// per-element device functions of dg_brj_apply.cuh, which the fused form of a
// sweep (brj_sweep_kernel, dg_sweep.cu) runs back to back in one kernel.
#include <cmath>
#include <cstring>
#include <cuda_bf16.h>
#include <new>
#include <type_traits>
#include <vector>
#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_precond.h"
#include "dg_sumfact.cuh"
#include "dg_tc.cuh"
#include "dg_brj_apply.cuh"

namespace dg {

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static constexpr int code = DG_PREC_FP64;
};
template <>
struct Prec<float> {
  static constexpr int code = DG_PREC_FP32;
};


// ------------------------------------------------------------ weights
// W[e][k][l][j][a][q] (q fastest: one contiguous slice per variable pair),
//                       a = 0: w|J| (2/h_j) dH_jk/dQ_l;
//                       a = 1+i: w|J| (2/h_j)(2/h_i) dH_jk/d(d_i Q_l)
// General elements (CV): with G[r][j] = d xi_r / d x_j at the point,
//   a = 0:   w|J| sum_j G[r][j] dH_jk/dQ_l                      (row index r)
//   a = 1+s: w|J| sum_{j,i} G[r][j] dH_jk/d(d_i Q_l) G[s][i]
template <int DIM, int P, int Q, typename TW, bool CV>
__global__ void __launch_bounds__(256) brj_weights_kernel(const __grid_constant__ Tables tab,
                                                          const __grid_constant__ Phys ph,
                                                          const ElemGeo* __restrict__ geo,
                                                          const __grid_constant__ GenGeo gg,
                                                          int e_begin, int ne,
                                                          const double* __restrict__ u,
                                                          TW* __restrict__ W) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NQ = C::NQ, Q2 = C::Q2, N2 = C::N2;
  constexpr int NW = DIM * (DIM + 1) * NV * NV;
  constexpr int JA = DIM * (DIM + 1);
  extern __shared__ double sm[];
  double* sB = sm;
  double* sD = sB + Q * N;
  double* sw = sD + Q * Q + 2 * Q + N * N;
  double* sU = sm + C::TAB;
  double* sQ = sU + NV * NM;
  double* sG = sQ + NV * NQ;  // DIM arrays
  double* sT = sG + DIM * NV * NQ;
  const int el = blockIdx.x;
  const int e = e_begin + el;
  stage_tables<DIM, P, Q>(tab, sm);
  for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) sU[i] = u[(long long)e * NV * NM + i];
  __syncthreads();
  if (DIM == 2) {
    contract<N, N, 1, 0, Q, N, 1, false>(sU, sT, sB, NV);
    __syncthreads();
    contract<Q, N, 1, 1, Q, N, 1, false>(sT, sQ, sB, NV);
  } else {
    contract<N, N, N2, 0, Q, N, 1, false>(sU, sG + NV * NQ, sB, NV);
    __syncthreads();
    contract<Q, N, N2, 1, Q, N, 1, false>(sG + NV * NQ, sG + 2 * NV * NQ, sB, NV);
    __syncthreads();
    contract<Q, Q, N2, 2, Q, N, 1, false>(sG + 2 * NV * NQ, sQ, sB, NV);
  }
  __syncthreads();
  contract<Q, Q, Q2, 0, Q, Q, 1, false>(sQ, sG, sD, NV);
  contract<Q, Q, Q2, 1, Q, Q, 1, false>(sQ, sG + NV * NQ, sD, NV);
  if (DIM == 3) contract<Q, Q, Q2, 2, Q, Q, 1, false>(sQ, sG + 2 * NV * NQ, sD, NV);
  __syncthreads();
  if constexpr (CV) {
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
      const double* gp = gg.vgeo + (long long)e * (DIM * DIM + 1) * NQ + q;
      double gi[DIM][DIM];
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int j = 0; j < DIM; ++j) gi[r][j] = gp[(r * DIM + j) * NQ];
      const double wJ = gp[DIM * DIM * NQ];
      double U[NV], dU[DIM][NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        U[v] = sQ[v * NQ + q];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          double a = 0.0;
#pragma unroll
          for (int r = 0; r < DIM; ++r) a = fma(gi[r][j], sG[(r * NV + v) * NQ + q], a);
          dU[j][v] = a;
        }
      }
      // artificial viscosity held at the linearisation state (not differentiated)
      const double mua = ph.avf ? av_point<DIM>(U, ph, ph.avf[e]) *
                                     (ph.av_mode == 2 ? ducros<DIM>(U, dU) : 1.0)
                             : 0.0;
      TW* Wq = W + (long long)el * NQ * NW + q;  // [(k NV + l) JA + ja][NQ]
      for (int l = 0; l < NV; ++l) {
        Dual Ud[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Ud[v] = Dual(U[v], v == l ? 1.0 : 0.0);
        Dual F[DIM][NV];
        euler_flux<DIM>(Ud, ph, F);
        if (ph.viscous) {
          Dual G[DIM][NV];
          viscous_flux<DIM, Dual, double>(Ud, dU, ph, G, mua);
#pragma unroll
          for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int k = 0; k < NV; ++k) F[j][k] = F[j][k] - G[j][k];
        }
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            double a = 0.0;
#pragma unroll
            for (int j = 0; j < DIM; ++j) a = fma(gi[r][j], F[j][k].d, a);
            Wq[((k * NV + l) * JA + r * (DIM + 1) + 0) * NQ] = (TW)(wJ * a);
          }
        double acc[DIM][DIM][NV];
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int s2 = 0; s2 < DIM; ++s2)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[r][s2][k] = 0.0;
        if (ph.viscous) {
          for (int i = 0; i < DIM; ++i) {
            double gu[DIM][NV], G[DIM][NV];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
              for (int v = 0; v < NV; ++v) gu[a][v] = (a == i && v == l) ? 1.0 : 0.0;
            viscous_flux<DIM>(U, gu, ph, G, mua);
#pragma unroll
            for (int r = 0; r < DIM; ++r)
#pragma unroll
              for (int k = 0; k < NV; ++k) {
                double tr = 0.0;
#pragma unroll
                for (int j = 0; j < DIM; ++j) tr = fma(gi[r][j], -G[j][k], tr);
#pragma unroll
                for (int s2 = 0; s2 < DIM; ++s2) acc[r][s2][k] = fma(tr, gi[s2][i], acc[r][s2][k]);
              }
          }
        }
#pragma unroll
        for (int r = 0; r < DIM; ++r)
#pragma unroll
          for (int s2 = 0; s2 < DIM; ++s2)
#pragma unroll
            for (int k = 0; k < NV; ++k)
              Wq[((k * NV + l) * JA + r * (DIM + 1) + 1 + s2) * NQ] = (TW)(wJ * acc[r][s2][k]);
      }
    }
    return;
  }
  const ElemGeo g = geo[e];
  double rh[DIM], detJ = 1.0;
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
    rh[r] = 2.0 / g.h[r];
    detJ *= 0.5 * g.h[r];
  }
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
    int c[3];
    grid_coords<DIM, Q>(q, c);
    const double wJ = sw[c[0]] * sw[c[1]] * (DIM == 3 ? sw[c[2]] : 1.0) * detJ;
    double U[NV], dU[DIM][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      U[v] = sQ[v * NQ + q];
#pragma unroll
      for (int r = 0; r < DIM; ++r) dU[r][v] = sG[(r * NV + v) * NQ + q] * rh[r];
    }
    const double mua = ph.avf ? av_point<DIM>(U, ph, ph.avf[e]) *
                                     (ph.av_mode == 2 ? ducros<DIM>(U, dU) : 1.0)
                             : 0.0;
    TW* Wq = W + (long long)el * NQ * NW + q;  // [(k NV + l) JA + ja][NQ]
    for (int l = 0; l < NV; ++l) {
      Dual Ud[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Ud[v] = Dual(U[v], v == l ? 1.0 : 0.0);
      Dual F[DIM][NV];
      euler_flux<DIM>(Ud, ph, F);
      if (ph.viscous) {
        Dual G[DIM][NV];
        viscous_flux<DIM, Dual, double>(Ud, dU, ph, G, mua);
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int k = 0; k < NV; ++k) F[j][k] = F[j][k] - G[j][k];
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < NV; ++k)
          Wq[((k * NV + l) * JA + j * (DIM + 1) + 0) * NQ] = (TW)(wJ * rh[j] * F[j][k].d);
    }
    for (int i = 0; i < DIM; ++i)
      for (int l = 0; l < NV; ++l) {
        double G[DIM][NV];
        if (ph.viscous) {
          double gu[DIM][NV];
#pragma unroll
          for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int v = 0; v < NV; ++v) gu[a][v] = (a == i && v == l) ? 1.0 : 0.0;
          viscous_flux<DIM>(U, gu, ph, G, mua);
        } else {
#pragma unroll
          for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int v = 0; v < NV; ++v) G[a][v] = 0.0;
        }
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int k = 0; k < NV; ++k)
            Wq[((k * NV + l) * JA + j * (DIM + 1) + 1 + i) * NQ] = (TW)(-wJ * rh[j] * rh[i] * G[j][k]);
      }
  }
}

// ------------------------------------------------------------ trace Jacobians
// Jd[e][lf][p][k][l] = s wJf dH_k/dQ_own,l ; Jo[e][lf][k][l][p] = s wJf dH_k/dQ_nbr,l
// with s = -1 on the owner (left) side and +1 on the right side (Jo with the
// face point fastest, so that the apply's product reads it coalesced).
template <int DIM, int P, int Q, typename TJ>
__global__ void __launch_bounds__(128) brj_tracejac_kernel(
    const __grid_constant__ Tables tab, const __grid_constant__ Phys ph,
    const ElemGeo* __restrict__ geo, const int32_t* __restrict__ faces, int F, double t,
    const double* __restrict__ tbuf, const double* __restrict__ chi, TJ* __restrict__ Jd,
    TJ* __restrict__ Jo) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NF = C::NF;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  const int f = idx / NF, p = idx - f * NF;
  const int eL = faces[f * 6 + 0], fL = faces[f * 6 + 1];
  const int eR = faces[f * 6 + 2], fR = faces[f * 6 + 3], bc = faces[f * 6 + 5];
  const int r = fL >> 1;
  const double sgn = (fL & 1) ? 1.0 : -1.0;
  const ElemGeo gL = geo[eL];
  int pt[2] = {p % Q, DIM == 3 ? p / Q : 0};
  double x[3] = {0, 0, 0};
  double wJf = 1.0;
  {
    int a = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      if (k == r) {
        x[k] = gL.x0[k] + ((fL & 1) ? gL.h[k] : 0.0);
      } else {
        x[k] = gL.x0[k] + 0.5 * (tab.x[pt[a]] + 1.0) * gL.h[k];
        wJf *= tab.w[pt[a]] * 0.5 * gL.h[k];
        ++a;
      }
    }
  }
  double QL[NV], QR[NV], dQa[DIM][NV];
  const double* tl = tbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
  double hmin = gL.h[r];
  int bctype = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    QL[v] = tl[v * NF];
#pragma unroll
    for (int j = 0; j < DIM; ++j) dQa[j][v] = tl[((1 + j) * NV + v) * NF];
  }
  if (eR >= 0) {
    hmin = fmin(hmin, geo[eR].h[r]);
    const double* tr = tbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      QR[v] = tr[v * NF];
#pragma unroll
      for (int j = 0; j < DIM; ++j) dQa[j][v] = 0.5 * (dQa[j][v] + tr[((1 + j) * NV + v) * NF]);
    }
  } else {
    bctype = ph.bc[bc];
#pragma unroll
    for (int v = 0; v < NV; ++v) QR[v] = 0.0;
  }
  const double beta = (double)((P + 1) * (P + 1)) / hmin;
  double H0[NV], H1[NV], S[DIM][NV];
  // artificial viscosity held at the linearisation state's traces
  const double mua = av_face<DIM>(ph, eL, eR, QL, QR, dQa);
  numerical_flux<DIM>(QL, QR, bctype, x, t, dQa, r, sgn, beta, ph, H0, S, mua);
  TJ* jdl = Jd + (((long long)eL * 2 * DIM + fL) * NF + p) * NV * NV;
  TJ* jol = Jo + ((long long)eL * 2 * DIM + fL) * NV * NV * NF + p;
  TJ* jdr = eR >= 0 ? Jd + (((long long)eR * 2 * DIM + fR) * NF + p) * NV * NV : nullptr;
  TJ* jor = eR >= 0 ? Jo + ((long long)eR * 2 * DIM + fR) * NV * NV * NF + p : nullptr;
  for (int l = 0; l < NV; ++l) {
    const double h = chi[l];
    const double ih = 1.0 / h;
    double Qp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Qp[v] = QL[v] + (v == l ? h : 0.0);
    numerical_flux<DIM>(Qp, QR, bctype, x, t, dQa, r, sgn, beta, ph, H1, S, mua);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double dHdL = (H1[k] - H0[k]) * ih;
      jdl[k * NV + l] = (TJ)(-wJf * dHdL);
      if (eR >= 0) jor[(k * NV + l) * NF] = (TJ)(wJf * dHdL);
    }
    if (eR >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Qp[v] = QR[v] + (v == l ? h : 0.0);
      numerical_flux<DIM>(QL, Qp, bctype, x, t, dQa, r, sgn, beta, ph, H1, S, mua);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const double dHdR = (H1[k] - H0[k]) * ih;
        jol[(k * NV + l) * NF] = (TJ)(-wJf * dHdR);
        jdr[k * NV + l] = (TJ)(wJf * dHdR);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) jol[(k * NV + l) * NF] = (TJ)0;
    }
  }
}

// the same on general elements: owner normal, surface weight and point from
// the face data, the face's penalty factor
template <int DIM, int P, int Q, typename TJ>
__global__ void __launch_bounds__(128) brj_tracejac_gen_kernel(
    const __grid_constant__ Phys ph, const __grid_constant__ GenGeo gg,
    const int32_t* __restrict__ faces, int F, double t, const double* __restrict__ tbuf,
    const double* __restrict__ chi, TJ* __restrict__ Jd, TJ* __restrict__ Jo) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NF = C::NF;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  const int f = idx / NF, p = idx - f * NF;
  const int eL = faces[f * 6 + 0], fL = faces[f * 6 + 1];
  const int eR = faces[f * 6 + 2], fR = faces[f * 6 + 3], bc = faces[f * 6 + 5];
  const double* fd = gg.fdat + (long long)f * (2 * DIM + 1) * NF + p;
  double n[DIM], x[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    n[j] = fd[j * NF];
    x[j] = fd[(DIM + 1 + j) * NF];
  }
  const double wJf = fd[DIM * NF];
  const double beta = gg.fbeta[f];
  double QL[NV], QR[NV], dQa[DIM][NV];
  const double* tl = tbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
  int bctype = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    QL[v] = tl[v * NF];
#pragma unroll
    for (int j = 0; j < DIM; ++j) dQa[j][v] = tl[((1 + j) * NV + v) * NF];
  }
  if (eR >= 0) {
    const double* tr = tbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      QR[v] = tr[v * NF];
#pragma unroll
      for (int j = 0; j < DIM; ++j) dQa[j][v] = 0.5 * (dQa[j][v] + tr[((1 + j) * NV + v) * NF]);
    }
  } else {
    bctype = ph.bc[bc];
#pragma unroll
    for (int v = 0; v < NV; ++v) QR[v] = 0.0;
  }
  double H0[NV], H1[NV], S[DIM][NV];
  const double mua = av_face<DIM>(ph, eL, eR, QL, QR, dQa);
  numerical_flux_n<DIM>(QL, QR, bctype, x, t, dQa, n, beta, ph, H0, S, mua);
  TJ* jdl = Jd + (((long long)eL * 2 * DIM + fL) * NF + p) * NV * NV;
  TJ* jol = Jo + ((long long)eL * 2 * DIM + fL) * NV * NV * NF + p;
  TJ* jdr = eR >= 0 ? Jd + (((long long)eR * 2 * DIM + fR) * NF + p) * NV * NV : nullptr;
  TJ* jor = eR >= 0 ? Jo + ((long long)eR * 2 * DIM + fR) * NV * NV * NF + p : nullptr;
  for (int l = 0; l < NV; ++l) {
    const double h = chi[l];
    const double ih = 1.0 / h;
    double Qp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Qp[v] = QL[v] + (v == l ? h : 0.0);
    numerical_flux_n<DIM>(Qp, QR, bctype, x, t, dQa, n, beta, ph, H1, S, mua);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double dHdL = (H1[k] - H0[k]) * ih;
      jdl[k * NV + l] = (TJ)(-wJf * dHdL);
      if (eR >= 0) jor[(k * NV + l) * NF] = (TJ)(wJf * dHdL);
    }
    if (eR >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Qp[v] = QR[v] + (v == l ? h : 0.0);
      numerical_flux_n<DIM>(QL, Qp, bctype, x, t, dQa, n, beta, ph, H1, S, mua);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const double dHdR = (H1[k] - H0[k]) * ih;
        jol[(k * NV + l) * NF] = (TJ)(-wJf * dHdR);
        jdr[k * NV + l] = (TJ)(wJf * dHdR);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) jol[(k * NV + l) * NF] = (TJ)0;
    }
  }
}

// ------------------------------------------------------------ block assembly

// Element block of (k, l) by sum factorisation.  With the per-point weights
// W_ja(q) (test derivative direction j, trial slot a: value or derivative a-1)
// and the 1-D tables b (value) and d (derivative) of the modified basis,
//   X[n][m] = sum_{j,a} sum_q W_ja(q) prod_r f_r(q_r, m_r) g_r(q_r, n_r),
//   f_r = d if r = j else b,  g_r = d if r = a-1 else b,
// contracted one Gauss direction at a time: 3-D: q0 (per (j,a)), q1 (per (j,a),
// accumulated by the factor types of direction 2), q2 (once per type); 2-D:
// q0 per (j,a) accumulated by the types of direction 1, then q1.  The own-side
// trace term adds, on each face, the face-slice modes (vertex mode across the
// face) contracted over the two (one) tangential face-point directions.
template <int DIM, int P, int Q, typename T, bool CV>
__global__ void __launch_bounds__(256) brj_block_kernel(
    const __grid_constant__ Tables tab, const ElemGeo* __restrict__ geo,
    const double* __restrict__ minv, int e_begin, const T* __restrict__ W,
    const T* __restrict__ Jd, double dta, T* __restrict__ blocks, int ld) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NQ = C::NQ, NF = C::NF;
  constexpr int NW = DIM * (DIM + 1) * NV * NV;
  constexpr int JA = DIM * (DIM + 1);
  constexpr int N2 = N * N;
  // 3-D: T1 [N2][Q*Q] per (j,a), T2 [N2*N2][Q] per type; 2-D: T1 [4][N2][Q]
  constexpr int T1SZ = DIM == 3 ? N2 * Q * Q : 4 * N2 * Q;
  constexpr int T2SZ = DIM == 3 ? N2 * N2 * Q : 0;
  __shared__ T sB1[Q * N], sD1[Q * N];
  __shared__ double sMi[N * N];
  extern __shared__ unsigned char smraw[];
  T* X = reinterpret_cast<T*>(smraw);           // [NM (col n)][NM (row m)]
  T* Y = X + NM * NM;
  T* sW = Y + NM * NM;                          // [JA][NQ]; later the dense M^-1
  T* T1 = sW + (CV && NM * NM > JA * NQ ? NM * NM : JA * NQ);
  T* T2 = T1 + T1SZ;
  const int el = blockIdx.x, e = e_begin + el;
  const int k = blockIdx.y / NV, l = blockIdx.y % NV;
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) {
    sB1[i] = (T)tab.B[i];
    const int q = i / N, m = i % N;
    double d = 0.0;  // psi_m'(x_q) by collocation (exact)
    for (int j = 0; j < Q; ++j) d += tab.Dq[q * Q + j] * tab.B[j * N + m];
    sD1[i] = (T)d;
  }
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sMi[i] = tab.Minv[i];
  const T* We = W + (long long)el * NQ * NW;
  for (int i = threadIdx.x; i < NQ * JA; i += blockDim.x)
    sW[i] = We[(long long)(k * NV + l) * JA * NQ + i];  // contiguous slice of (k, l)
  for (int i = threadIdx.x; i < T1SZ + T2SZ; i += blockDim.x) T1[i] = (T)0;
  __syncthreads();
  // factor of direction r for test (F) / trial (G) side of combination (j, a)
  auto ftab = [&](int j, int r) -> const T* { return r == j ? sD1 : sB1; };
  auto gtab = [&](int a, int r) -> const T* { return r == a - 1 ? sD1 : sB1; };
  if constexpr (DIM == 3) {
    // products of the test and trial factors of one direction,
    // FG[c][q][m + N n] = f(q, m) g(q, n) with f = d if c & 2 else b and
    // g = d if c & 1 else b: each contraction below is then one FMA per term,
    // and a thread keeps N outputs in registers per operand it loads
    T* FG = Y;  // Y is free until the mass-matrix step
    for (int i = threadIdx.x; i < 4 * Q * N2; i += blockDim.x) {
      const int c = i / (Q * N2), rem = i % (Q * N2);
      const int q = rem / N2, mn = rem % N2;
      const T* f = (c & 2) ? sD1 : sB1;
      const T* g = (c & 1) ? sD1 : sB1;
      FG[i] = f[q * N + mn % N] * g[q * N + mn / N];
    }
    // one pass per factor type of direction 2 (f2, g2 in {b, d}): the (j, a)
    // of that type are contracted over q0 and q1 into T2, then q2 into X
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) X[i] = (T)0;
    for (int type = 0; type < 4; ++type) {
      for (int i = threadIdx.x; i < N2 * N2 * Q; i += blockDim.x) T2[i] = (T)0;
      __syncthreads();
      for (int ja = 0; ja < JA; ++ja) {
        const int j = ja / (DIM + 1), a = ja % (DIM + 1);
        if ((j == 2 ? 2 : 0) + (a == 3 ? 1 : 0) != type) continue;
        const T* fg0 = FG + ((j == 0 ? 2 : 0) + (a == 1 ? 1 : 0)) * Q * N2;
        const T* fg1 = FG + ((j == 1 ? 2 : 0) + (a == 2 ? 1 : 0)) * Q * N2;
        const T* w = sW + ja * NQ;
        // contract q0: T1[(m0 + N n0)][q1 + Q q2], a thread per (q1 q2, n0), m0 in registers
        for (int i = threadIdx.x; i < Q * Q * N; i += blockDim.x) {
          const int qq = i % (Q * Q), n0 = i / (Q * Q);
          T acc[N];
#pragma unroll
          for (int m0 = 0; m0 < N; ++m0) acc[m0] = (T)0;
#pragma unroll
          for (int q0 = 0; q0 < Q; ++q0) {
            const T wv = w[q0 + Q * qq];
            const T* fr = fg0 + q0 * N2 + N * n0;
#pragma unroll
            for (int m0 = 0; m0 < N; ++m0) acc[m0] += fr[m0] * wv;
          }
#pragma unroll
          for (int m0 = 0; m0 < N; ++m0) T1[(m0 + N * n0) * Q * Q + qq] = acc[m0];
        }
        __syncthreads();
        // contract q1: T2[((m0 + N n0) N2 + m1 + N n1) Q + q2] +=, a thread per
        // (mn0, q2, n1), m1 in registers
        for (int i = threadIdx.x; i < N2 * Q * N; i += blockDim.x) {
          const int q2 = i % Q, r = i / Q;
          const int n1 = r % N, mn0 = r / N;
          T acc[N];
#pragma unroll
          for (int m1 = 0; m1 < N; ++m1) acc[m1] = (T)0;
#pragma unroll
          for (int q1 = 0; q1 < Q; ++q1) {
            const T tv = T1[mn0 * Q * Q + q1 + Q * q2];
            const T* fr = fg1 + q1 * N2 + N * n1;
#pragma unroll
            for (int m1 = 0; m1 < N; ++m1) acc[m1] += fr[m1] * tv;
          }
#pragma unroll
          for (int m1 = 0; m1 < N; ++m1) T2[(mn0 * N2 + m1 + N * n1) * Q + q2] += acc[m1];
        }
        __syncthreads();
      }
      // contract q2 into X[n][m], a thread per (m0, m1, n0, n1, n2) (m0, m1
      // fastest: neighbouring threads touch neighbouring rows of X), m2 in
      // registers
      const T* fg2 = FG + type * Q * N2;
      for (int i = threadIdx.x; i < N2 * N2 * N; i += blockDim.x) {
        const int m0 = i % N, m1 = (i / N) % N, n0 = (i / N2) % N, n1 = (i / (N2 * N)) % N;
        const int n2 = i / (N2 * N2);
        const int mn0 = m0 + N * n0, mn1 = m1 + N * n1;
        const T* t2 = T2 + (mn0 * N2 + mn1) * Q;
        T acc[N];
#pragma unroll
        for (int m2 = 0; m2 < N; ++m2) acc[m2] = (T)0;
#pragma unroll
        for (int q2 = 0; q2 < Q; ++q2) {
          const T tv = t2[q2];
          const T* fr = fg2 + q2 * N2 + N * n2;
#pragma unroll
          for (int m2 = 0; m2 < N; ++m2) acc[m2] += fr[m2] * tv;
        }
        const int n = n0 + N * (n1 + N * n2);
#pragma unroll
        for (int m2 = 0; m2 < N; ++m2) X[n * NM + m0 + N * (m1 + N * m2)] += acc[m2];
      }
      __syncthreads();
    }
  } else {
    for (int ja = 0; ja < JA; ++ja) {
      const int j = ja / (DIM + 1), a = ja % (DIM + 1);
      const T* f0 = ftab(j, 0); const T* g0 = gtab(a, 0);
      const int type = (j == 1 ? 2 : 0) + (a == 2 ? 1 : 0);
      const T* w = sW + ja * NQ;
      // contract q0: T1[type][(m0 + N n0)][q1] +=
      T* t1 = T1 + type * N2 * Q;
      for (int i = threadIdx.x; i < N2 * Q; i += blockDim.x) {
        const int mn = i / Q, q1 = i % Q;
        const int m0 = mn % N, n0 = mn / N;
        T acc = (T)0;
#pragma unroll
        for (int q0 = 0; q0 < Q; ++q0) acc += f0[q0 * N + m0] * g0[q0 * N + n0] * w[q0 + Q * q1];
        t1[i] += acc;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
      const int n = i / NM, m = i % NM;
      const int m0 = m % N, m1 = m / N, n0 = n % N, n1 = n / N;
      T acc = (T)0;
#pragma unroll
      for (int type = 0; type < 4; ++type) {
        const T* f1 = (type & 2) ? sD1 : sB1;
        const T* g1 = (type & 1) ? sD1 : sB1;
        const T* t1 = T1 + type * N2 * Q + (m0 + N * n0) * Q;
#pragma unroll
        for (int q1 = 0; q1 < Q; ++q1) acc += f1[q1 * N + m1] * g1[q1 * N + n1] * t1[q1];
      }
      X[i] = acc;
    }
  }
  __syncthreads();
  // own-side trace term, face by face (face-slice modes only)
  for (int lf = 0; lf < 2 * DIM; ++lf) {
    const int r = lf >> 1;
    const int vert = (lf & 1) ? P : 0;
    const T* jd = Jd + (((long long)e * 2 * DIM + lf) * NF) * NV * NV + k * NV + l;
    T* sJ = T1;  // [NF] face values, then [N2][Q] partial contraction
    T* S1 = T1 + NF;
    for (int p = threadIdx.x; p < NF; p += blockDim.x) sJ[p] = jd[(long long)p * NV * NV];
    __syncthreads();
    if constexpr (DIM == 3) {
      const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
      // S1[(a0 + N b0)][p1] = sum_p0 b(p0, a0) b(p0, b0) J(p0 + Q p1)
      for (int i = threadIdx.x; i < N2 * Q; i += blockDim.x) {
        const int ab = i / Q, p1 = i % Q;
        const int a0 = ab % N, b0 = ab / N;
        T acc = (T)0;
#pragma unroll
        for (int p0 = 0; p0 < Q; ++p0) acc += sB1[p0 * N + a0] * sB1[p0 * N + b0] * sJ[p0 + Q * p1];
        S1[i] = acc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N2 * N2; i += blockDim.x) {
        const int a0 = i % N, b0 = (i / N) % N, a1 = (i / N2) % N, b1 = i / (N2 * N);
        T acc = (T)0;
#pragma unroll
        for (int p1 = 0; p1 < Q; ++p1)
          acc += sB1[p1 * N + a1] * sB1[p1 * N + b1] * S1[(a0 + N * b0) * Q + p1];
        int mc[3], nc[3];
        mc[r] = vert;
        nc[r] = vert;
        mc[t0] = a0;
        mc[t1] = a1;
        nc[t0] = b0;
        nc[t1] = b1;
        const int m = mc[0] + N * (mc[1] + N * mc[2]), n = nc[0] + N * (nc[1] + N * nc[2]);
        X[n * NM + m] += acc;
      }
    } else {
      const int t0 = 1 - r;
      for (int i = threadIdx.x; i < N2; i += blockDim.x) {
        const int a0 = i % N, b0 = i / N;
        T acc = (T)0;
#pragma unroll
        for (int p = 0; p < Q; ++p) acc += sB1[p * N + a0] * sB1[p * N + b0] * sJ[p];
        int mc[2], nc[2];
        mc[r] = vert;
        nc[r] = vert;
        mc[t0] = a0;
        nc[t0] = b0;
        X[(nc[0] + N * nc[1]) * NM + mc[0] + N * mc[1]] += acc;
      }
    }
    __syncthreads();
  }
  T* src = X;
  T* dst = Y;
  if constexpr (CV) {
    // dense M_e^-1 (symmetric) on the row index, staged in the W slot
    T* sMd = sW;
    const double* Me = minv + (long long)e * NM * NM;
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) sMd[i] = (T)Me[i];
    __syncthreads();
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
      const int col = i / NM, m = i % NM;
      T a = (T)0;
      for (int kk = 0; kk < NM; ++kk) a += sMd[kk * NM + m] * src[col * NM + kk];
      dst[i] = a;
    }
    __syncthreads();
    T* out = blocks + (long long)e * (NV * NM) * ld;
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
      const int m = i / NM, n = i % NM;
      double val = -dta * (double)dst[n * NM + m];
      if (k == l && m == n) val += 1.0;
      out[(long long)(l * NM + n) * ld + k * NM + m] = (T)val;
    }
    return;
  }
  // M^-1 on the row (test) index: |J|^-1 (M1^-1)^(x)DIM, axis by axis
  const double idet = geo[e].idet;
  for (int ax = 0; ax < DIM; ++ax) {
    for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
      const int col = i / NM, m = i % NM;
      int mc[3];
      mode_coords<DIM, N>(m, mc);
      const int str = ax == 0 ? 1 : (ax == 1 ? N : N * N);
      const int base = m - mc[ax] * str;
      double s = 0.0;
#pragma unroll
      for (int kk = 0; kk < N; ++kk)
        s += sMi[mc[ax] * N + kk] * (double)src[col * NM + base + kk * str];
      dst[i] = (T)s;
    }
    __syncthreads();
    T* tmp = src;
    src = dst;
    dst = tmp;
  }
  // D = I - dt_a M^-1 X into rows k*NM + m, columns l*NM + n
  T* out = blocks + (long long)e * (NV * NM) * ld;
  for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
    const int m = i / NM, n = i % NM;
    double val = -dta * idet * (double)src[n * NM + m];
    if (k == l && m == n) val += 1.0;
    // stored transposed: the inverse of the transpose is the transpose of the
    // inverse, which the column-streaming block GEMV reads
    out[(long long)(l * NM + n) * ld + k * NM + m] = (T)val;
  }
}

// ------------------------------------------------------------ inversion
// Blocked in-place Gauss-Jordan inversion with partial pivoting, one block per
// element.  Pivot columns K = [k0, k0+B) are processed as a panel held in
// shared memory (row interchanges applied to whole rows at once); afterwards
// the panel holds the columns K of the composite transformation T_K, and every
// other column c is updated in one pass, A[:, c] += (T_K - E_K) A[K, c], a
// rank-B update, so the block is read and written once per panel instead of
// once per pivot.  The inverse's columns are un-permuted at the end.
template <typename T, int B>
__global__ void __launch_bounds__(512) brj_invert_blocked_kernel(T* __restrict__ blocks, int nb,
                                                                 int ld, int* __restrict__ fail) {
  extern __shared__ unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);     // [nb][B] panel
  T* Ak = P + (size_t)nb * B;             // [B][nb] old pivot rows
  T* prow = Ak + (size_t)B * nb;          // [B] scaled pivot row of the panel
  T* fcol = prow + B;                     // [nb] multipliers
  int* perm = reinterpret_cast<int*>(fcol + nb);
  __shared__ T redv[32];
  __shared__ int redi[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  T* A = blocks + (long long)blockIdx.x * nb * ld;
  for (int k0 = 0; k0 < nb; k0 += B) {
    const int bw = nb - k0 < B ? nb - k0 : B;
    for (int i = threadIdx.x; i < nb * B; i += blockDim.x) {
      const int r = i / B, j = i % B;
      P[i] = j < bw ? A[(long long)r * ld + k0 + j] : (T)0;
    }
    __syncthreads();
    for (int j = 0; j < bw; ++j) {
      const int k = k0 + j;
      // pivot: largest |P[i][j]|, i >= k (lowest index on ties): warp shuffles,
      // then one exchange through shared memory
      T best = (T)-1;
      int bi = k;
      for (int i = k + threadIdx.x; i < nb; i += blockDim.x) {
        const T v = fabs(P[i * B + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
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
      if (!(pmag > (T)0)) {
        if (threadIdx.x == 0) atomicExch(fail, 1);
        return;
      }
      if (threadIdx.x == 0) perm[k] = pr;
      if (pr != k) {
        for (int jj = threadIdx.x; jj < B; jj += blockDim.x) {
          const T a = P[k * B + jj];
          P[k * B + jj] = P[pr * B + jj];
          P[pr * B + jj] = a;
        }
        for (int c = threadIdx.x; c < nb; c += blockDim.x) {
          if (c >= k0 && c < k0 + bw) continue;
          const T a = A[(long long)k * ld + c];
          A[(long long)k * ld + c] = A[(long long)pr * ld + c];
          A[(long long)pr * ld + c] = a;
        }
      }
      __syncthreads();
      const T ipiv = (T)1 / P[k * B + j];
      for (int jj = threadIdx.x; jj < B; jj += blockDim.x)
        prow[jj] = jj == j ? ipiv : P[k * B + jj] * ipiv;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) fcol[i] = P[i * B + j];
      __syncthreads();
      for (int i2 = threadIdx.x; i2 < nb * B; i2 += blockDim.x) {
        const int i = i2 / B, jj = i2 % B;
        if (i == k) {
          P[i2] = prow[jj];
        } else {
          const T a = jj == j ? (T)0 : P[i2];
          P[i2] = a - fcol[i] * prow[jj];
        }
      }
      __syncthreads();
    }
    // old rows K of the columns outside the panel (after the interchanges)
    for (int i = threadIdx.x; i < B * nb; i += blockDim.x) {
      const int j = i / nb, c = i % nb;
      Ak[i] = (j < bw && (c < k0 || c >= k0 + bw)) ? A[(long long)(k0 + j) * ld + c] : (T)0;
    }
    __syncthreads();
    // A[:, c] += (T_K - E_K) A[K, c] for c outside the panel, eight rows per
    // batch of independent loads: the T_K A[K, c] product in the inner loop,
    // the E_K A[K, c] term (row K_j loses A[K_j, c]) once per row of the
    // panel's rows; panel columns <- T_K
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
      if (c >= k0 && c < k0 + bw) continue;
      T ak[B];
#pragma unroll
      for (int j = 0; j < B; ++j) ak[j] = Ak[j * nb + c];
      for (int i0 = 0; i0 < nb; i0 += 8) {
        T acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = i0 + t < nb ? A[(long long)(i0 + t) * ld + c] : (T)0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int i = i0 + t;
          if (i >= nb) break;
          const T* u = P + i * B;
          T a = acc[t];
#pragma unroll
          for (int j = 0; j < B; ++j) a += u[j] * ak[j];
          const int dj = i - k0;
          if (dj >= 0 && dj < B) a -= Ak[dj * nb + c];
          acc[t] = a;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (i0 + t < nb) A[(long long)(i0 + t) * ld + c] = acc[t];
      }
    }
    for (int i = threadIdx.x; i < nb * B; i += blockDim.x) {
      const int r = i / B, j = i % B;
      if (j < bw) A[(long long)r * ld + k0 + j] = P[i];
    }
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {
    const int pr = perm[k];
    if (pr != k)
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const T a = A[(long long)i * ld + k];
        A[(long long)i * ld + k] = A[(long long)i * ld + pr];
        A[(long long)i * ld + pr] = a;
      }
    __syncthreads();
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// chi_k = sqrt(2^-52) ||u_k||_2 (sqrt(2^-52) when the variable vanishes)
__global__ void __launch_bounds__(256) var_norm_kernel(const double* __restrict__ u, int E,
                                                       int nv, int nm, double* __restrict__ chi) {
  __shared__ double sh[256];
  const int k = blockIdx.x;
  double s = 0.0;
  for (long long i = threadIdx.x; i < (long long)E * nm; i += 256) {
    const long long e = i / nm, m = i % nm;
    const double v = u[(e * nv + k) * nm + m];
    s = fma(v, v, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nk = sqrt(sh[0]);
    chi[k] = 1.4901161193847656e-08 * (nk > 0.0 ? nk : 1.0);
  }
}

// The same blocked Gauss-Jordan inversion (FP32 blocks) with the trailing
// rank-32 update A[:, c] += (T_K - E_K) A[K, c] on the tensor cores: tcgen05
// kind::tf32 products with FP32 accumulation in tensor memory, each operand
// split into a TF32 head and a TF32 tail (x = hi + lo, hi = x with its 13 low
// mantissa bits cleared) and the three products hi*hi + hi*lo + lo*hi summed,
// which keeps the update to FP32 accuracy.  Row tiles of 128 (M) by column
// chunks of up to 256 (N), K = the 32 panel columns; operands staged by the
// CTA's threads in the K-major core-matrix layout; the accumulator is read
// back one row per thread (warps w and w + 4 share the rows of lane quarter
// w and split the columns) and added to A in global memory.  The panel
// factorisation is the SIMT code of brj_invert_blocked_kernel.
constexpr int TCI_B = 32, TCI_N = 256, TCI_WAIT = 1 << 20;

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__global__ void __launch_bounds__(256) brj_invert_tc_kernel(float* __restrict__ blocks, int nb,
                                                            int ld, int* __restrict__ fail) {
  constexpr int B = TCI_B;
  constexpr int SBO = (B / 4) * 128;              // TF32 tiles: 8 core matrices along K
  constexpr int UT = 128 * B * 4, VT = TCI_N * B * 4;
  extern __shared__ __align__(1024) unsigned char smraw[];
  uint8_t* Uh = smraw;
  uint8_t* Ul = Uh + UT;
  uint8_t* Vh = Ul + UT;
  uint8_t* Vl = Vh + VT;
  float* P = reinterpret_cast<float*>(Vl + VT);   // [nb][B] panel
  float* prow = P + (size_t)nb * B;               // [B]
  float* fcol = prow + B;                         // [nb]
  int* perm = reinterpret_cast<int*>(fcol + nb);
  __shared__ float redv[32];
  __shared__ int redi[32];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (warp == 0) tc::tmem_alloc(&tmem_slot, TCI_N);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  float* A = blocks + (long long)blockIdx.x * nb * ld;
  for (int k0 = 0; k0 < nb && ok; k0 += B) {
    const int bw = nb - k0 < B ? nb - k0 : B;
    for (int i = tid; i < nb * B; i += blockDim.x) {
      const int r = i / B, j = i % B;
      P[i] = j < bw ? A[(long long)r * ld + k0 + j] : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < bw; ++j) {
      const int k = k0 + j;
      float best = -1.f;
      int bi = k;
      for (int i = k + tid; i < nb; i += blockDim.x) {
        const float v = fabsf(P[i * B + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
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
      float pmag = redv[0];
      int pr = redi[0];
      for (int w = 1; w < nwarp; ++w) {
        const float ov = redv[w];
        const int oi = redi[w];
        if (ov > pmag || (ov == pmag && oi < pr)) {
          pmag = ov;
          pr = oi;
        }
      }
      if (!(pmag > 0.f)) {  // singular block: leave (uniformly) through the common exit
        if (tid == 0) atomicExch(fail, 1);
        ok = false;
        break;
      }
      if (tid == 0) perm[k] = pr;
      if (pr != k) {
        for (int jj = tid; jj < B; jj += blockDim.x) {
          const float a = P[k * B + jj];
          P[k * B + jj] = P[pr * B + jj];
          P[pr * B + jj] = a;
        }
        for (int c = tid; c < nb; c += blockDim.x) {
          if (c >= k0 && c < k0 + bw) continue;
          const float a = A[(long long)k * ld + c];
          A[(long long)k * ld + c] = A[(long long)pr * ld + c];
          A[(long long)pr * ld + c] = a;
        }
      }
      __syncthreads();
      const float ipiv = 1.f / P[k * B + j];
      for (int jj = tid; jj < B; jj += blockDim.x) prow[jj] = jj == j ? ipiv : P[k * B + jj] * ipiv;
      for (int i = tid; i < nb; i += blockDim.x) fcol[i] = P[i * B + j];
      __syncthreads();
      for (int i2 = tid; i2 < nb * B; i2 += blockDim.x) {
        const int i = i2 / B, jj = i2 % B;
        if (i == k) {
          P[i2] = prow[jj];
        } else {
          const float a = jj == j ? 0.f : P[i2];
          P[i2] = a - fcol[i] * prow[jj];
        }
      }
      __syncthreads();
    }
    if (!ok) break;
    // trailing update on the tensor cores, column chunk by row tile
    for (int nc0 = 0; nc0 < nb && ok; nc0 += TCI_N) {
      const int ncols = nb - nc0 < TCI_N ? nb - nc0 : TCI_N;
      const int nmma = (ncols + 15) / 16 * 16;
      // V: rows c (outside the panel) x K = old pivot rows A[k0 + j][c]
      for (int i = tid; i < nmma * B; i += blockDim.x) {
        const int r = i / B, j = i % B, c = nc0 + r;
        float x = 0.f;
        if (c < nb && j < bw && (c < k0 || c >= k0 + bw)) x = A[(long long)(k0 + j) * ld + c];
        float hi, lo;
        tf32_split(x, hi, lo);
        const int off = (r >> 3) * SBO + (j >> 2) * 128 + (r & 7) * 16 + (j & 3) * 4;
        *reinterpret_cast<float*>(Vh + off) = hi;
        *reinterpret_cast<float*>(Vl + off) = lo;
      }
      for (int rt = 0; rt < nb && ok; rt += 128) {
        // U: rows i x K = (T_K - E_K)[i][j]
        for (int i2 = tid; i2 < 128 * B; i2 += blockDim.x) {
          const int r = i2 / B, j = i2 % B, i = rt + r;
          float x = 0.f;
          if (i < nb && j < bw) x = P[i * B + j] - (i == k0 + j ? 1.f : 0.f);
          float hi, lo;
          tf32_split(x, hi, lo);
          const int off = (r >> 3) * SBO + (j >> 2) * 128 + (r & 7) * 16 + (j & 3) * 4;
          *reinterpret_cast<float*>(Uh + off) = hi;
          *reinterpret_cast<float*>(Ul + off) = lo;
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
          const uint32_t id = tc::idesc(2, 128, nmma);
#pragma unroll
          for (int ks = 0; ks < B / 8; ++ks) {
            const uint64_t uh = tc::desc(tc::smem_addr(Uh) + ks * 256, 128, SBO);
            const uint64_t ul = tc::desc(tc::smem_addr(Ul) + ks * 256, 128, SBO);
            const uint64_t vh = tc::desc(tc::smem_addr(Vh) + ks * 256, 128, SBO);
            const uint64_t vl = tc::desc(tc::smem_addr(Vl) + ks * 256, 128, SBO);
            tc::mma_tf32(tmem, uh, vh, id, ks > 0 ? 1u : 0u);
            tc::mma_tf32(tmem, uh, vl, id, 1u);
            tc::mma_tf32(tmem, ul, vh, id, 1u);
          }
          tc::commit(&mbar);
        }
        const bool w = tc::mbar_wait(&mbar, phase, TCI_WAIT);
        phase ^= 1u;
        if (!__syncthreads_and(w)) {
          if (tid == 0) atomicExch(fail, 2);
          ok = false;
          break;
        }
        tc::fence_after();
        // A[i][c] += accumulator, one row per thread; the two warp groups
        // split the 16-column chunks
        const int q = warp & 3, grp = warp >> 2, ngrp = nwarp >> 2;
        const int i = rt + q * 32 + lane;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        for (int cc = grp * 16; cc < nmma; cc += 16 * ngrp) {
          float v[16];
          tc::ld16(tmem + lanes + cc, v);
          if (i < nb) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int c = nc0 + cc + t;
              if (c < nb && (c < k0 || c >= k0 + bw)) A[(long long)i * ld + c] += v[t];
            }
          }
        }
        tc::fence_before();
        __syncthreads();  // tiles and accumulator are reused by the next product
      }
    }
    if (!ok) break;
    for (int i = tid; i < nb * B; i += blockDim.x) {
      const int r = i / B, j = i % B;
      if (j < bw) A[(long long)r * ld + k0 + j] = P[i];
    }
    __syncthreads();
  }
  if (ok) {
    for (int k = nb - 1; k >= 0; --k) {
      const int pr = perm[k];
      if (pr != k)
        for (int i = tid; i < nb; i += blockDim.x) {
          const float a = A[(long long)i * ld + k];
          A[(long long)i * ld + k] = A[(long long)i * ld + pr];
          A[(long long)i * ld + pr] = a;
        }
      __syncthreads();
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TCI_N);
}

// ------------------------------------------------------------ apply
// y = q - (L+U) qh = q + dt_a M^-1 sum_faces B_f^T (Jo . trace of the neighbour's qh)
// y = q - (L+U) qh, one block of 128 threads per element
template <int DIM, int P, int Q, typename TA, typename TJ, bool CV>
__global__ void __launch_bounds__(128) brj_offdiag_kernel(
    const __grid_constant__ Tables tab, const ElemGeo* __restrict__ geo,
    const double* __restrict__ minv, int E, const TJ* __restrict__ Jo,
    const int32_t* __restrict__ nbr, const double* __restrict__ qh,
    const double* __restrict__ q, double dta, double* __restrict__ y) {
  constexpr int NB = Cfg<DIM, P, Q>::NV * Cfg<DIM, P, Q>::NM;
  const int e = blockIdx.x;
  offdiag_element<DIM, P, Q, TA, TJ, CV, 128>(tab, geo, minv, Jo, nbr, qh, q, dta, e,
                                              [&](int i, double v) { y[(long long)e * NB + i] = v; });
}

// ------------------------------------------------------------ drivers
template <int DIM, int P, int Q>
struct BRJImpl {
  using C = Cfg<DIM, P, Q>;

  template <typename T, bool CV>
  static dg_status build(dg_mesh_s* m, dg_precond_s* pc, const double* u, double t, double dta,
                         cudaStream_t s) {
    constexpr int NV = C::NV, NM = C::NM, NQ = C::NQ, NF = C::NF;
    const int E = m->E, nb = pc->nb, ld = round_up8(nb);
    // traces of Q and grad Q at u (residual pass fills the trace buffer)
    EvalArgs a{};
    a.u = u;
    a.t = t;
    a.out = m->w2;
    DG_TRY(launch_residual(m, a, s));
    double* chi = m->scratch + 8;
    var_norm_kernel<<<NV, 256, 0, s>>>(u, E, NV, NM, chi);
    DG_LAUNCHED(1);
    T* Jd = (T*)pc->jd;
    T* Jo = (T*)pc->jo;
    const GenGeo gg = gen_geo(m);
    if constexpr (CV) {
      DG_PROF(K_BRJ_TRACEJAC, s, brj_tracejac_gen_kernel<DIM, P, Q, T><<<(m->F * NF + 127) / 128, 128, 0, s>>>(
          m->phys, gg, m->faces, m->F, t, m->tbuf, chi, Jd, Jo));
    } else {
      DG_PROF(K_BRJ_TRACEJAC, s, brj_tracejac_kernel<DIM, P, Q, T><<<(m->F * NF + 127) / 128, 128, 0, s>>>(
          m->tab, m->phys, m->geo, m->faces, m->F, t, m->tbuf, chi, Jd, Jo));
    }
    DG_LAUNCHED(1);
    // blocks: FP64 mode stores double, FP32/BF16 modes assemble in float
    T* blk = (T*)(pc->precision == DG_PREC_BF16 ? pc->work : pc->blocks);
    T* Wbuf = (T*)((char*)pc->work +
                   (pc->precision == DG_PREC_BF16 ? sizeof(float) * (size_t)E * nb * ld : 0));
    const size_t wsm = sizeof(double) * (C::TAB + NV * NM + (1 + DIM) * NV * NQ + (DIM == 2 ? NV * NQ : 0));
    DG_CUDA(cudaFuncSetAttribute(brj_weights_kernel<DIM, P, Q, T, CV>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
    // general elements stage the dense M^-1 beside the weights
    const int wsz = NQ * DIM * (DIM + 1);
    constexpr int N2 = C::N * C::N;
    constexpr int TSZ = DIM == 3 ? N2 * Q * Q + N2 * N2 * Q : 4 * N2 * Q;
    const size_t bsm = sizeof(T) * (2 * NM * NM + (CV && NM * NM > wsz ? NM * NM : wsz) + TSZ);
    DG_CUDA(cudaFuncSetAttribute(brj_block_kernel<DIM, P, Q, T, CV>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
    const int CH = pc->wchunk;
    for (int e0 = 0; e0 < E; e0 += CH) {
      const int ne = E - e0 < CH ? E - e0 : CH;
      DG_PROF(K_BRJ_WEIGHTS, s, brj_weights_kernel<DIM, P, Q, T, CV><<<ne, 256, wsm, s>>>(
          m->tab, m->phys, m->geo, gg, e0, ne, u, Wbuf));
      DG_LAUNCHED(1);
      DG_PROF(K_BRJ_BLOCK, s, brj_block_kernel<DIM, P, Q, T, CV><<<dim3(ne, NV * NV), 256, bsm, s>>>(
          m->tab, m->geo, m->minv, e0, Wbuf, Jd, dta, blk, ld));
      DG_LAUNCHED(1);
    }
    if (pc->full)  // terms 4-5 of the element with itself, before the inversion
      DG_TRY(visc_build(m, pc, t, dta, blk, ld, std::is_same<T, double>::value, s));
    int* fail = (int*)(m->scratch + 16);
    DG_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), s));
    constexpr int IB = 32;  // panel width of the blocked inversion
    bool tc_done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (pc->tc_invert) {
      // FP32 blocks (FP32 and BF16 modes): trailing updates on the tensor cores
      const size_t ism = 2 * (size_t)(128 + TCI_N) * TCI_B * 4 +
                         sizeof(float) * ((size_t)nb * TCI_B + TCI_B + nb) + sizeof(int) * nb;
      DG_CUDA(cudaFuncSetAttribute(brj_invert_tc_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
      DG_PROF(K_BRJ_INVERT, s, brj_invert_tc_kernel<<<E, 256, ism, s>>>(blk, nb, ld, fail));
      tc_done = true;
      }
    }
    if (!tc_done && invert_rows_supported(nb, std::is_same<T, double>::value)) {
      // panel in registers, deferred row interchanges (dg_invert.cu)
      DG_TRY(launch_invert_rows(blk, std::is_same<T, double>::value, E, nb, ld, fail, s));
      tc_done = true;
    }
    if (!tc_done) {
      const size_t ism = sizeof(T) * ((size_t)2 * nb * IB + IB + nb) + sizeof(int) * nb;
      DG_CUDA(cudaFuncSetAttribute(brj_invert_blocked_kernel<T, IB>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
      // one thread per column of the block (the trailing update's unit of work)
      const int ith = nb <= 512 ? (nb + 31) / 32 * 32 : 512;
      DG_PROF(K_BRJ_INVERT, s, brj_invert_blocked_kernel<T, IB><<<E, ith, ism, s>>>(blk, nb, ld, fail));
    }
    DG_LAUNCHED(1);
    if (pc->precision == DG_PREC_BF16) {
      const long long n = (long long)E * nb * ld;
      to_bf16_kernel<<<152 * 16, 256, 0, s>>>((const float*)blk, (__nv_bfloat16*)pc->blocks, n);
      DG_LAUNCHED(1);
    }
    int hfail = 0;
    DG_CUDA(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    return hfail ? DG_ERR_NONFINITE : DG_OK;
  }

  template <typename TA, typename TJ, bool CV>
  static dg_status offdiag(dg_mesh_s* m, dg_precond_s* pc, const double* qh, const double* q,
                           double* y, cudaStream_t s) {
    DG_PROF(K_BRJ_OFFDIAG, s, brj_offdiag_kernel<DIM, P, Q, TA, TJ, CV><<<m->E, 128, 0, s>>>(
        m->tab, m->geo, m->minv, m->E, (const TJ*)pc->jo, pc->nbr, qh, q, pc->dt_a, y));
    DG_LAUNCHED(1);
    return DG_OK;
  }
};

template <typename TB>
__global__ void DG_DIAG_BOUNDS(TB)
    brj_diag_cm_kernel(const TB* __restrict__ blocks, int nb, int ld, int split,
                       const double* __restrict__ y, const double* __restrict__ qprev,
                       double omega, double* __restrict__ out) {
  using TA = typename Vec16<TB>::TA;
  extern __shared__ unsigned char smraw[];
  TA* sy = reinterpret_cast<TA*>(smraw);                 // [nb]
  TA* part = sy + nb;                                    // [split][ld]
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sy[i] = (TA)y[(long long)e * nb + i];
  __syncthreads();
  diag_element<TB>(blocks, nb, ld, split, sy, part, qprev, omega, out, e);
}

template <typename TB>
static dg_status diag_launch(const void* blocks, int E, int nb, int ld, const double* y,
                             const double* qprev, double omega, double* out, cudaStream_t s) {
  using V = Vec16<TB>;
  const int nrq = ld / V::W;
  // BF16 columns carry half the bytes of FP32 ones: twice the column groups
  // keep the same number of loads in flight
  const int budget = sizeof(TB) == 2 ? 512 : 256;
  int split = budget / nrq;
  if (split < 1) split = 1;
  const int threads = ((nrq * split + 31) / 32) * 32;
  if (threads > budget) return DG_ERR_UNSUPPORTED;  // ld > budget W: not built
  const size_t sm = sizeof(typename V::TA) * ((size_t)nb + (size_t)split * ld);
  DG_PROF(K_BRJ_DIAG, s, brj_diag_cm_kernel<TB><<<E, threads, sm, s>>>(
      (const TB*)blocks, nb, ld, split, y, qprev, omega, out));
  DG_LAUNCHED(1);
  return DG_OK;
}

static dg_status diag_apply(dg_precond_s* pc, double omega, const double* y, const double* qprev,
                            double* out, cudaStream_t s) {
  const int E = pc->mesh->E, nb = pc->nb, ld = round_up8(nb);
  if (pc->precision == DG_PREC_FP64)
    return diag_launch<double>(pc->blocks, E, nb, ld, y, qprev, omega, out, s);
  if (pc->precision == DG_PREC_FP32)
    return diag_launch<float>(pc->blocks, E, nb, ld, y, qprev, omega, out, s);
  return diag_launch<__nv_bfloat16>(pc->blocks, E, nb, ld, y, qprev, omega, out, s);
}



// geometry kind at run time; general-geometry kernels only where instantiated
template <int D, int P, int Q, typename T>
static dg_status build_dispatch(dg_mesh_s* m, dg_precond_s* pc, const double* u, double t,
                                double dta, cudaStream_t s) {
  if (!m->curved) return BRJImpl<D, P, Q>::template build<T, false>(m, pc, u, t, dta, s);
  if constexpr (has_curved<D, P, Q>())
    return BRJImpl<D, P, Q>::template build<T, true>(m, pc, u, t, dta, s);
  return DG_ERR_UNSUPPORTED;
}

template <int D, int P, int Q, typename TA>
static dg_status offdiag_dispatch(dg_mesh_s* m, dg_precond_s* pc, const double* qh,
                                  const double* q, double* y, cudaStream_t s) {
  if (!m->curved) return BRJImpl<D, P, Q>::template offdiag<TA, TA, false>(m, pc, qh, q, y, s);
  if constexpr (has_curved<D, P, Q>())
    return BRJImpl<D, P, Q>::template offdiag<TA, TA, true>(m, pc, qh, q, y, s);
  return DG_ERR_UNSUPPORTED;
}

static dg_status dispatch_build(dg_mesh_s* m, dg_precond_s* pc, const double* u, double t,
                                double dta, cudaStream_t s) {
#define DG_B(D_, P_, Q_)                                                     \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                            \
    if (pc->precision == DG_PREC_FP64)                                       \
      return build_dispatch<D_, P_, Q_, double>(m, pc, u, t, dta, s);        \
    return build_dispatch<D_, P_, Q_, float>(m, pc, u, t, dta, s);           \
  }
  DG_PREC_INSTANCES(DG_B)
#undef DG_B
  return DG_ERR_UNSUPPORTED;
}

static dg_status dispatch_offdiag(dg_precond_s* pc, const double* qh, const double* q, double* y,
                                  cudaStream_t s) {
  dg_mesh_s* m = pc->mesh;
#define DG_O(D_, P_, Q_)                                                     \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                            \
    if (pc->precision == DG_PREC_FP64)                                       \
      return offdiag_dispatch<D_, P_, Q_, double>(m, pc, qh, q, y, s);       \
    return offdiag_dispatch<D_, P_, Q_, float>(m, pc, qh, q, y, s);          \
  }
  DG_PREC_INSTANCES(DG_O)
#undef DG_O
  return DG_ERR_UNSUPPORTED;
}

// the fused form of the sweeps: sweep 1 as before, then each later sweep one
// launch reading the previous iterate from one buffer and writing the next
// into the other (the neighbours read the previous iterate while it is
// replaced, so the two cannot share a buffer)
static dg_status precond_sweeps_fused(dg_precond_s* pc, const double* q, double* out,
                                      cudaStream_t s) {
  double* cur = pc->J == 1 ? out : pc->qh;
  DG_TRY(diag_apply(pc, 1.0, q, nullptr, cur, s));
  if (pc->omega != 1.0) DG_TRY(axpby(cur, 0.0, cur, pc->omega, pc->mesh->ndof, s));
  for (int j = 1; j < pc->J; ++j) {
    double* nxt = j == pc->J - 1 ? out : (cur == pc->qh ? pc->qh2 : pc->qh);
    DG_TRY(dispatch_sweep(pc, cur, q, nxt, s));
    cur = nxt;
  }
  return DG_OK;
}

// the J sweeps of Eq. precond-Jacobi as kernel launches on stream s
dg_status precond_sweeps(dg_precond_s* pc, const double* q, double* out, cudaStream_t s) {
  if (pc->fused) return precond_sweeps_fused(pc, q, out, s);
  // sweep 1 from qh = 0: D^-1 q (the relaxation term vanishes)
  double* cur = pc->J == 1 ? out : pc->qh;
  DG_TRY(diag_apply(pc, 1.0, q, nullptr, cur, s));
  if (pc->omega != 1.0) DG_TRY(axpby(cur, 0.0, cur, pc->omega, pc->mesh->ndof, s));
  for (int j = 1; j < pc->J; ++j) {
    DG_TRY(dispatch_offdiag(pc, cur, q, pc->y, s));
    if (pc->full) DG_TRY(visc_offdiag(pc, cur, pc->y, s));  // terms 4-5 of (L+U)
    double* nxt = j == pc->J - 1 ? out : pc->qh;
    if (nxt != cur && pc->omega != 1.0)
      DG_CUDA(cudaMemcpyAsync(nxt, cur, sizeof(double) * pc->mesh->ndof, cudaMemcpyDeviceToDevice, s));
    DG_TRY(diag_apply(pc, pc->omega, pc->y, nxt, nxt, s));
    cur = nxt;
  }
  return DG_OK;
}

static constexpr size_t kMaxGraphs = 128;

void precond_drop_graphs(dg_precond_s* pc) {
  for (auto& g : pc->graphs) cudaGraphExecDestroy(g.exec);
  pc->graphs.clear();
}

// With graphs enabled, the sweeps for each (q, out) pair are captured once on
// the handle's own stream and replayed as one graph launch, fenced to the
// caller's stream with events (the captured kernels see fixed pointers, so
// the Krylov slots of GMRES each get one graph, reused for the handle's life;
// a rebuild drops them).  Per-kernel profiling bypasses the graphs.
dg_status precond_apply_impl(dg_precond_s* pc, const double* q, double* out, cudaStream_t s) {
  if (!pc->use_graphs || profiling_on()) return precond_sweeps(pc, q, out, s);
  if (!pc->cs) {
    DG_CUDA(cudaStreamCreateWithFlags(&pc->cs, cudaStreamNonBlocking));
    DG_CUDA(cudaEventCreateWithFlags(&pc->ev_in, cudaEventDisableTiming));
    DG_CUDA(cudaEventCreateWithFlags(&pc->ev_out, cudaEventDisableTiming));
  }
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  for (auto& g : pc->graphs)
    if (g.q == q && g.out == out) {
      exec = g.exec;
      kernels = g.kernels;
    }
  if (!exec) {
    cudaGraph_t graph = nullptr;
    const long long before = dg_kernel_launches();
    DG_CUDA(cudaStreamBeginCapture(pc->cs, cudaStreamCaptureModeThreadLocal));
    const dg_status st = precond_sweeps(pc, q, out, pc->cs);
    kernels = dg_kernel_launches() - before;
    const cudaError_t ce = cudaStreamEndCapture(pc->cs, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    DG_CUDA(ce);
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    DG_CUDA(ie);
    if (pc->graphs.size() >= kMaxGraphs) {  // callers cycling through many buffers
      cudaGraphExecDestroy(pc->graphs.front().exec);
      pc->graphs.erase(pc->graphs.begin());
    }
    pc->graphs.push_back({q, out, exec, kernels});
  }
  // the capture counted the graph's kernels once; each replay launches them again
  else
    __atomic_fetch_add(&g_launches, kernels, __ATOMIC_RELAXED);
  DG_CUDA(cudaEventRecord(pc->ev_in, s));
  DG_CUDA(cudaStreamWaitEvent(pc->cs, pc->ev_in, 0));
  DG_CUDA(cudaGraphLaunch(exec, pc->cs));
  DG_CUDA(cudaEventRecord(pc->ev_out, pc->cs));
  DG_CUDA(cudaStreamWaitEvent(s, pc->ev_out, 0));
  return DG_OK;
}

}  // namespace dg

using namespace dg;

static void free_precond(dg_precond_s* p) {
  if (!p) return;
  cudaFree(p->blocks);
  cudaFree(p->jd);
  cudaFree(p->jo);
  cudaFree(p->nbr);
  cudaFree(p->tr);
  cudaFree(p->qh);
  cudaFree(p->qh2);
  cudaFree(p->y);
  cudaFree(p->work);
  cudaFree(p->jk);
  cudaFree(p->jsd);
  cudaFree(p->jso);
  precond_drop_graphs(p);
  if (p->cs) cudaStreamDestroy(p->cs);
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->ev_out) cudaEventDestroy(p->ev_out);
  delete p;
}

extern "C" {

dg_status dg_precond_build(dg_mesh_t m, const double* u, double t, double dt_a,
                           const dg_prec_cfg* cfg, dg_precond_t* inout, void* stream) {
  if (!m || !u || !cfg || !inout) return DG_ERR_ARG;
  if (cfg->J < 1 || !(cfg->omega > 0.0)) return DG_ERR_ARG;
  if (cfg->precision < DG_PREC_FP64 || cfg->precision > DG_PREC_BF16) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = m->dim, E = m->E, NV = m->nv;
  const int nb = NV * m->nm, ld = round_up8(nb);
  if (cfg->precision == DG_PREC_FP64 && 2 * (size_t)m->nm * m->nm * 8 > 200 * 1024)
    return DG_ERR_UNSUPPORTED;
  // FP64 blocks on general elements only up to P = 2: the one FP64 P = 3 build
  // on a curved mesh that ran ended in a device fault whose cause reading the
  // kernels has not found, so that configuration is not offered (FP32 and
  // BF16 blocks cover the curved workloads at every P)
  if (cfg->precision == DG_PREC_FP64 && m->curved && m->P > 2) return DG_ERR_UNSUPPORTED;
  // terms 4-5: viscous flows on axis-aligned elements, the two-kernel sweeps
  const int full = cfg->full_jacobian && m->phys.viscous;
  if (full && (m->curved || cfg->fused || !visc_supported(d, m->P, m->Q) ||
               (m->phys.avf && m->phys.av_mode == 2)))
    return DG_ERR_UNSUPPORTED;
  dg_precond_s* p = *inout;
  if (p && (p->mesh != m || p->precision != cfg->precision || p->full != full)) {
    free_precond(p);
    *inout = nullptr;
    p = nullptr;
  }
  const size_t vb = cfg->precision == DG_PREC_FP64 ? 8 : 4;  // build / trace-Jacobian value size
  const size_t nwq = (size_t)d * (d + 1) * NV * NV * m->nq;  // weights per element
  if (!p) {
    p = new (std::nothrow) dg_precond_s();
    if (!p) return DG_ERR_OOM;
    p->mesh = m;
    p->precision = cfg->precision;
    p->nb = nb;
    const size_t bsz = cfg->precision == DG_PREC_FP64 ? 8 : (cfg->precision == DG_PREC_FP32 ? 4 : 2);
    const size_t njac = (size_t)E * 2 * d * m->nf * NV * NV;
    // weights workspace: bounded to ~1 GiB by processing elements in chunks
    size_t per = nwq * vb;
    int ch = (int)((size_t(1) << 30) / per);
    if (ch < 1) ch = 1;
    if (ch > E) ch = E;
    p->wchunk = ch;
    const size_t stage = cfg->precision == DG_PREC_BF16 ? sizeof(float) * (size_t)E * nb * ld : 0;
    p->work_bytes = stage + per * ch;
    cudaError_t err = cudaSuccess;
    // zeroed workspaces (the blocks' padding columns included)
    auto alloc = [&](void** ptr, size_t bytes) {
      if (err == cudaSuccess) err = cudaMalloc(ptr, bytes);
      if (err == cudaSuccess) err = cudaMemset(*ptr, 0, bytes);
    };
    alloc(&p->blocks, bsz * (size_t)E * nb * ld);
    alloc(&p->jd, vb * njac);
    alloc(&p->jo, vb * njac);
    alloc((void**)&p->nbr, sizeof(int32_t) * E * 2 * d);
    alloc((void**)&p->qh, sizeof(double) * (size_t)m->ndof);
    alloc((void**)&p->y, sizeof(double) * (size_t)m->ndof);
    alloc(&p->work, p->work_bytes);
    if (full) {
      p->full = 1;
      const size_t nv3 = (size_t)E * 2 * d * m->nf * visc_values_per_face_point(d) * vb;
      alloc(&p->jk, nv3);
      alloc(&p->jsd, nv3);
      alloc(&p->jso, nv3);
    }
    // zero padding columns once: the block kernels never write them
    if (err == cudaSuccess) err = cudaMemset(p->blocks, 0, bsz * (size_t)E * nb * ld);
    if (err == cudaSuccess) err = cudaMemset(p->work, 0, p->work_bytes);
    if (err != cudaSuccess) {
      free_precond(p);
      return cuda_status(err);
    }
    // neighbour map (element * 2d + local face of the other side) per element face
    std::vector<int32_t> faces((size_t)m->F * 6), nbr((size_t)E * 2 * d, -1);
    if (cudaMemcpy(faces.data(), m->faces, sizeof(int32_t) * 6 * m->F, cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      free_precond(p);
      return DG_ERR_CUDA;
    }
    for (int f = 0; f < m->F; ++f) {
      const int eL = faces[f * 6], fL = faces[f * 6 + 1], eR = faces[f * 6 + 2], fR = faces[f * 6 + 3];
      if (eR >= 0) {
        nbr[(size_t)eL * 2 * d + fL] = eR * 2 * d + fR;
        nbr[(size_t)eR * 2 * d + fR] = eL * 2 * d + fL;
      }
    }
    if (cudaMemcpy(p->nbr, nbr.data(), sizeof(int32_t) * nbr.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      free_precond(p);
      return DG_ERR_CUDA;
    }
    *inout = p;
  }
  // the captured sweeps hold J, omega and the launch shapes: a rebuild re-captures
  precond_drop_graphs(p);
  static unsigned long long g_gen = 0;
  // (the sweeps take J, omega, dt_a and their form by value; everything else by pointer
  // into buffers that a rebuild refills in place)
  if (p->gen == 0 || p->J != cfg->J || p->omega != cfg->omega || p->dt_a != dt_a ||
      p->fused != (cfg->fused != 0))
    p->gen = __atomic_add_fetch(&g_gen, 1ULL, __ATOMIC_RELAXED);
  if (cfg->fused && !p->qh2) {
    DG_CUDA(cudaMalloc((void**)&p->qh2, sizeof(double) * (size_t)m->ndof));
    DG_CUDA(cudaMemset(p->qh2, 0, sizeof(double) * (size_t)m->ndof));
  }
  p->fused = cfg->fused != 0;
  p->use_graphs = cfg->graphs;
  p->tc_invert = cfg->tc_invert;
  p->J = cfg->J;
  p->omega = cfg->omega;
  p->dt_a = dt_a;
  return dispatch_build(m, p, u, t, dt_a, s);
}

dg_status dg_precond_apply(dg_precond_t p, const double* q, double* out, void* stream) {
  if (!p || !q || !out || q == out) return DG_ERR_ARG;
  return precond_apply_impl(p, q, out, (cudaStream_t)stream);
}

dg_status dg_precond_destroy(dg_precond_t p) {
  if (!p) return DG_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  free_precond(p);
  return e == cudaSuccess ? DG_OK : cuda_status(e);
}

}  // extern "C"
