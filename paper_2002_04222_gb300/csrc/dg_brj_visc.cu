// Terms 4 and 5 of Eq. Jacobian-matrix-form2 (Sec. 4.2.2), which the paper
// neglects: the trace-gradient term (the numerical flux's dependence on the
// face gradients, through n . G({Q}, {grad Q})) and the symmetric-flux term
// (the lift sum_i integral d_i phi S_i with S_i = G_i({Q}, n (x) [Q])).  An
// option of the BRJ preconditioner (dg_prec_cfg.full_jacobian), on meshes of
// axis-aligned elements:
//   brj_visc_trace_kernel  one thread per face point: dH^n_k/d(grad_j Q_l)
//                          = -c sum_i n_i G_ik({Q}, e_j (x) e_l) (G is linear in
//                          the gradient; c = 1/2 inside, 1 on a boundary) and
//                          dS_i/dQ of both sides by the one-sided difference of
//                          Eq. numerical-Jac-on-traces (boundary states
//                          re-evaluated), stored per element face with the
//                          side's sign and the surface weight;
//   brj_block_visc_kernel  adds -dt_a M^-1 (terms 4 + 5 of the element with
//                          itself) to each diagonal block before inversion;
//   brj_offdiag_visc_kernel  adds dt_a M^-1 (terms 4 + 5 of the neighbours) . qh
//                          to the sweep's right-hand side y after the term-3
//                          off-diagonal product.
#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_precond.h"
#include "dg_sumfact.cuh"
#include "dg_brj_apply.cuh"

namespace dg {

// S_i = G_i({Q}, n (x) [Q]) at a face point from the two traces (boundary:
// the boundary state from QL; the energy component vanishes on an adiabatic
// wall), and the state {Q} it is evaluated at
template <int D>
__device__ inline void symmetric_flux(const double* QL, const double* QRin, int bctype,
                                      const double* x, double t, const double* n, const Phys& ph,
                                      double S[D][D + 2], double* Qa_out, double mu_add) {
  constexpr int NV = D + 2;
  double QR[NV], Qa[NV], jump[NV];
  bool adiabatic = false;
  if (bctype > 0) {
    adiabatic = boundary_states<D>(bctype, ph, x, t, QL, n, QR, Qa);
#pragma unroll
    for (int v = 0; v < NV; ++v) jump[v] = QL[v] - Qa[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Qa[v] = 0.5 * (QL[v] + QRin[v]);
      jump[v] = QL[v] - QRin[v];
    }
  }
  double gS[D][NV];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int v = 0; v < NV; ++v) gS[j][v] = n[j] * jump[v];
  viscous_flux<D>(Qa, gS, ph, S, mu_add);
  if (adiabatic)
#pragma unroll
    for (int j = 0; j < D; ++j) S[j][NV - 1] = 0.0;
  if (Qa_out)
#pragma unroll
    for (int v = 0; v < NV; ++v) Qa_out[v] = Qa[v];
}

// per face point and side: K [k][j][l] (NV D NV), S_own and S_nbr [i][k][l] (D NV NV)
template <int DIM>
struct ViscSizes {
  static constexpr int NV = DIM + 2;
  static constexpr int NK = NV * DIM * NV;
  static constexpr int NS = DIM * NV * NV;
};

template <int DIM, int P, int Q, typename TJ>
__global__ void __launch_bounds__(128) brj_visc_trace_kernel(
    const __grid_constant__ Tables tab, const __grid_constant__ Phys ph,
    const ElemGeo* __restrict__ geo, const int32_t* __restrict__ faces, int F, double t,
    const double* __restrict__ tbuf, const double* __restrict__ chi, TJ* __restrict__ Kd,
    TJ* __restrict__ Sd, TJ* __restrict__ So) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NF = C::NF;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  constexpr int NK = ViscSizes<DIM>::NK, NS = ViscSizes<DIM>::NS;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  const int f = idx / NF, p = idx - f * NF;
  const int eL = faces[f * 6 + 0], fL = faces[f * 6 + 1];
  const int eR = faces[f * 6 + 2], fR = faces[f * 6 + 3], bc = faces[f * 6 + 5];
  const int r = fL >> 1;
  const double sgn = (fL & 1) ? 1.0 : -1.0;
  const ElemGeo gL = geo[eL];
  int pt[2] = {p % Q, DIM == 3 ? p / Q : 0};
  double x[3] = {0, 0, 0}, n[DIM];
  double wJf = 1.0;
  {
    int a = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      n[k] = k == r ? sgn : 0.0;
      if (k == r) {
        x[k] = gL.x0[k] + ((fL & 1) ? gL.h[k] : 0.0);
      } else {
        x[k] = gL.x0[k] + 0.5 * (tab.x[pt[a]] + 1.0) * gL.h[k];
        wJf *= tab.w[pt[a]] * 0.5 * gL.h[k];
        ++a;
      }
    }
  }
  double QL[NV], QR[NV];
  const double* tl = tbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
#pragma unroll
  for (int v = 0; v < NV; ++v) QL[v] = tl[v * NF];
  int bctype = 0;
  if (eR >= 0) {
    const double* tr = tbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int v = 0; v < NV; ++v) QR[v] = tr[v * NF];
  } else {
    bctype = ph.bc[bc];
#pragma unroll
    for (int v = 0; v < NV; ++v) QR[v] = 0.0;
  }
  const bool interior = eR >= 0;
  const double cg = interior ? 0.5 : 1.0;
  const double cs = cg * ph.beta_s;
  double S0[DIM][NV], S1[DIM][NV], Qa[NV];
  // artificial viscosity held at the linearisation state's traces
  // (the face-average gradient enters only with Ducros' sensor, which the
  // build refuses together with these terms)
  const double zgrad[DIM][DIM + 2] = {};
  const double mua = av_face<DIM>(ph, eL, eR, QL, QR, zgrad);
  symmetric_flux<DIM>(QL, QR, bctype, x, t, n, ph, S0, Qa, mua);
  const bool adiabatic = bctype == DG_BC_ADIA_WALL;
  TJ* kl = Kd + (((long long)eL * 2 * DIM + fL) * NF + p) * NK;
  TJ* kr = interior ? Kd + (((long long)eR * 2 * DIM + fR) * NF + p) * NK : nullptr;
  // term 4: K[k][j][l] = s wJ dH_k/d(grad_j Q_l) = -s wJ c sgn G_rk(Qa, e_j (x) e_l)
  for (int j = 0; j < DIM; ++j)
    for (int l = 0; l < NV; ++l) {
      double gu[DIM][NV], G[DIM][NV];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int v = 0; v < NV; ++v) gu[a][v] = (a == j && v == l) ? 1.0 : 0.0;
      viscous_flux<DIM>(Qa, gu, ph, G, mua);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const double dh = (adiabatic && k == NV - 1) ? 0.0 : -cg * sgn * G[r][k];
        kl[(k * DIM + j) * NV + l] = (TJ)(-wJf * dh);
        if (interior) kr[(k * DIM + j) * NV + l] = (TJ)(wJf * dh);
      }
    }
  // term 5: dS_i/dQ of each side, one-sided differences with chi_l
  TJ* sdl = Sd + (((long long)eL * 2 * DIM + fL) * NF + p) * NS;
  TJ* sol = So + (((long long)eL * 2 * DIM + fL) * NF + p) * NS;
  TJ* sdr = interior ? Sd + (((long long)eR * 2 * DIM + fR) * NF + p) * NS : nullptr;
  TJ* sor = interior ? So + (((long long)eR * 2 * DIM + fR) * NF + p) * NS : nullptr;
  for (int l = 0; l < NV; ++l) {
    const double h = chi[l], ih = 1.0 / h;
    double Qp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Qp[v] = QL[v] + (v == l ? h : 0.0);
    symmetric_flux<DIM>(Qp, QR, bctype, x, t, n, ph, S1, nullptr, mua);
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const double d = cs * wJf * (S1[i][k] - S0[i][k]) * ih;
        sdl[(i * NV + k) * NV + l] = (TJ)d;
        if (interior) sor[(i * NV + k) * NV + l] = (TJ)d;
      }
    if (interior) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Qp[v] = QR[v] + (v == l ? h : 0.0);
      symmetric_flux<DIM>(QL, Qp, bctype, x, t, n, ph, S1, nullptr, mua);
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const double d = cs * wJf * (S1[i][k] - S0[i][k]) * ih;
          sol[(i * NV + k) * NV + l] = (TJ)d;
          sdr[(i * NV + k) * NV + l] = (TJ)d;
        }
    } else {
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int k = 0; k < NV; ++k) sol[(i * NV + k) * NV + l] = (TJ)0;
    }
  }
}

// Value (j < 0) or physical derivative d/dx_j of mode m of an axis-aligned
// element at face point p of its local face lf (1-D tables: B and the
// collocation derivative sD at the Gauss points, psi and psi' at -1 and +1).
template <int DIM, int P, int Q>
struct FaceBasis {
  static constexpr int N = P + 1;
  const double* sB;   // [Q][N]
  const double* sD;   // [Q][N]
  const double* dend; // [2][N] psi'(-1), psi'(+1)
  __device__ double operator()(int lf, int p, int m, int j, const double* rh) const {
    const int r = lf >> 1, side = lf & 1;
    int mc[3];
    mc[0] = m % N;
    mc[1] = (m / N) % N;
    mc[2] = DIM == 3 ? m / (N * N) : 0;
    int pc[3] = {0, 0, 0};
    if (DIM == 2) {
      pc[1 - r] = p;
    } else {
      const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
      pc[t0] = p % Q;
      pc[t1] = p / Q;
    }
    double v = 1.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      if (d == r) {
        const double val = (mc[d] == (side ? P : 0)) ? 1.0 : 0.0;
        v *= (j == d) ? dend[side * N + mc[d]] : val;
      } else {
        v *= (j == d) ? sD[pc[d] * N + mc[d]] : sB[pc[d] * N + mc[d]];
      }
    }
    return j >= 0 ? v * rh[j] : v;
  }
};

template <int DIM, int P, int Q>
__device__ inline void stage_face_tables(const Tables& tab, double* sB, double* sD, double* dend) {
  constexpr int N = P + 1;
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) {
    sB[i] = tab.B[i];
    const int q = i / N, m = i % N;
    double d = 0.0;  // psi_m'(x_q) by collocation (exact)
    for (int j = 0; j < Q; ++j) d += tab.Dq[q * Q + j] * tab.B[j * N + m];
    sD[i] = d;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    dend[i] = tab.dpm[i];
    dend[N + i] = tab.dpp[i];
  }
}

// M^-1 = |J|^-1 (M1^-1)^(x)DIM applied in place to nrep vectors of NM modes
// (src, dst ping-pong in shared memory); returns the buffer holding the result
template <int DIM, int N, typename T>
__device__ inline T* apply_minv_tensor(const double* sMi, double idet, T* src, T* dst, int nrep) {
  constexpr int NM = DIM == 2 ? N * N : N * N * N;
  for (int ax = 0; ax < DIM; ++ax) {
    for (int i = threadIdx.x; i < nrep * NM; i += blockDim.x) {
      const int rep = i / NM, m = i % NM;
      int mc[3];
      mode_coords<DIM, N>(m, mc);
      const int str = ax == 0 ? 1 : (ax == 1 ? N : N * N);
      const int base = rep * NM + m - mc[ax] * str;
      double s = 0.0;
#pragma unroll
      for (int kk = 0; kk < N; ++kk) s += sMi[mc[ax] * N + kk] * (double)src[base + kk * str];
      dst[i] = (T)(ax == DIM - 1 ? s * idet : s);
    }
    __syncthreads();
    T* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// the element's own terms 4-5 for variable pair (k, l), added as
// -dt_a M^-1 X to the (transposed) diagonal block
template <int DIM, int P, int Q, typename T>
__global__ void __launch_bounds__(256) brj_block_visc_kernel(
    const __grid_constant__ Tables tab, const ElemGeo* __restrict__ geo, const T* __restrict__ Kd,
    const T* __restrict__ Sd, double dta, T* __restrict__ blocks, int ld) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NF = C::NF;
  constexpr int NK = ViscSizes<DIM>::NK, NS = ViscSizes<DIM>::NS;
  constexpr int NSL = DIM == 2 ? N : N * N;  // face-slice modes
  __shared__ double sB[Q * N], sD[Q * N], dend[2 * N], sMi[N * N];
  __shared__ double sK[NF * DIM], sS[NF * DIM];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* X = reinterpret_cast<T*>(smraw);  // [NM][NM]: X[n][m], trial n, test m
  T* Y = X + NM * NM;
  const int e = blockIdx.x;
  const int k = blockIdx.y / NV, l = blockIdx.y % NV;
  stage_face_tables<DIM, P, Q>(tab, sB, sD, dend);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sMi[i] = tab.Minv[i];
  for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) X[i] = (T)0;
  const ElemGeo g = geo[e];
  double rh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) rh[d] = g.rh[d];
  __syncthreads();
  FaceBasis<DIM, P, Q> fb{sB, sD, dend};
  for (int lf = 0; lf < 2 * DIM; ++lf) {
    const int r = lf >> 1, vert = (lf & 1) ? P : 0;
    const T* kp = Kd + ((long long)e * 2 * DIM + lf) * NF * NK;
    const T* sp = Sd + ((long long)e * 2 * DIM + lf) * NF * NS;
    for (int i = threadIdx.x; i < NF * DIM; i += blockDim.x) {
      const int p = i / DIM, j = i % DIM;
      sK[i] = (double)kp[(long long)p * NK + (k * DIM + j) * NV + l];
      sS[i] = (double)sp[(long long)p * NS + (j * NV + k) * NV + l];
    }
    __syncthreads();
    // term 4: X[n][m] += sum_p B_f(p, m) sum_j K_pj G_j(p, n), m on the face slice
    for (int i = threadIdx.x; i < NSL * NM; i += blockDim.x) {
      const int a = i / NM, n = i % NM;
      int mc[3] = {0, 0, 0};
      mc[r] = vert;
      if (DIM == 2) {
        mc[1 - r] = a;
      } else {
        const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
        mc[t0] = a % N;
        mc[t1] = a / N;
      }
      const int m = mc[0] + N * (mc[1] + N * mc[2]);
      double acc = 0.0;
      for (int p = 0; p < NF; ++p) {
        const double bm = fb(lf, p, m, -1, rh);
        double gk = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) gk += sK[p * DIM + j] * fb(lf, p, n, j, rh);
        acc += bm * gk;
      }
      X[n * NM + m] += (T)acc;
    }
    __syncthreads();
    // term 5: X[n][m] += sum_p sum_i G_i(p, m) S_pi B_f(p, n), n on the face slice
    for (int i = threadIdx.x; i < NSL * NM; i += blockDim.x) {
      const int a = i / NM, m = i % NM;
      int nc[3] = {0, 0, 0};
      nc[r] = vert;
      if (DIM == 2) {
        nc[1 - r] = a;
      } else {
        const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
        nc[t0] = a % N;
        nc[t1] = a / N;
      }
      const int n = nc[0] + N * (nc[1] + N * nc[2]);
      double acc = 0.0;
      for (int p = 0; p < NF; ++p) {
        double gs = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) gs += fb(lf, p, m, j, rh) * sS[p * DIM + j];
        acc += gs * fb(lf, p, n, -1, rh);
      }
      X[n * NM + m] += (T)acc;
    }
    __syncthreads();
  }
  // M^-1 on the test index m (rows of each trial column n), then D -= dt_a M^-1 X
  const T* res = apply_minv_tensor<DIM, N, T>(sMi, g.idet, X, Y, NM);
  T* out = blocks + (long long)e * (NV * NM) * ld;
  for (int i = threadIdx.x; i < NM * NM; i += blockDim.x) {
    const int n = i / NM, m = i % NM;
    T* o = out + (long long)(l * NM + n) * ld + k * NM + m;
    *o = (T)((double)*o - dta * (double)res[n * NM + m]);
  }
}

// y_e += dt_a M^-1 (terms 4-5 of the neighbours) . qh, one block per element
template <int DIM, int P, int Q, typename TJ>
__global__ void __launch_bounds__(128) brj_offdiag_visc_kernel(
    const __grid_constant__ Tables tab, const ElemGeo* __restrict__ geo,
    const TJ* __restrict__ Kd, const TJ* __restrict__ So, const int32_t* __restrict__ nbr,
    const double* __restrict__ qh, double dta, double* __restrict__ y) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NF = C::NF;
  constexpr int NK = ViscSizes<DIM>::NK, NS = ViscSizes<DIM>::NS;
  __shared__ double sB[Q * N], sD[Q * N], dend[2 * N], sMi[N * N];
  __shared__ double qn[NV * NM];                 // neighbour coefficients
  __shared__ double tv[NV * NF], tg[DIM * NV * NF];  // its face values and gradients
  __shared__ double z4[NV * NF], z5[DIM * NV * NF];
  __shared__ double L0[NV * NM], L1[NV * NM];
  const int e = blockIdx.x;
  stage_face_tables<DIM, P, Q>(tab, sB, sD, dend);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sMi[i] = tab.Minv[i];
  for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) L0[i] = 0.0;
  const ElemGeo g = geo[e];
  double rh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) rh[d] = g.rh[d];
  FaceBasis<DIM, P, Q> fb{sB, sD, dend};
  __syncthreads();
  for (int lf = 0; lf < 2 * DIM; ++lf) {
    const int nb = nbr[e * 2 * DIM + lf];
    if (nb < 0) continue;  // (uniform over the block)
    const int en = nb / (2 * DIM), fn = nb % (2 * DIM);
    const ElemGeo gn = geo[en];
    double rhn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) rhn[d] = gn.rh[d];
    for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) qn[i] = qh[(long long)en * NV * NM + i];
    __syncthreads();
    // the neighbour's values and physical gradients at the shared face points
    for (int i = threadIdx.x; i < (1 + DIM) * NV * NF; i += blockDim.x) {
      const int p = i % NF, v = (i / NF) % NV, fld = i / (NV * NF);
      double acc = 0.0;
      for (int mm = 0; mm < NM; ++mm) acc += fb(fn, p, mm, fld - 1, rhn) * qn[v * NM + mm];
      if (fld == 0)
        tv[v * NF + p] = acc;
      else
        tg[((fld - 1) * NV + v) * NF + p] = acc;
    }
    __syncthreads();
    const TJ* kp = Kd + ((long long)e * 2 * DIM + lf) * NF * NK;
    const TJ* sp = So + ((long long)e * 2 * DIM + lf) * NF * NS;
    // z4[k][p] = sum_{j,l} K[p][k][j][l] grad_j q_l ; z5[i][k][p] = sum_l So[p][i][k][l] q_l
    for (int i = threadIdx.x; i < NV * NF; i += blockDim.x) {
      const int p = i % NF, kk = i / NF;
      double a = 0.0;
      for (int j = 0; j < DIM; ++j)
        for (int l = 0; l < NV; ++l)
          a += (double)kp[(long long)p * NK + (kk * DIM + j) * NV + l] * tg[(j * NV + l) * NF + p];
      z4[kk * NF + p] = a;
      for (int j = 0; j < DIM; ++j) {
        double b = 0.0;
        for (int l = 0; l < NV; ++l)
          b += (double)sp[(long long)p * NS + (j * NV + kk) * NV + l] * tv[l * NF + p];
        z5[(j * NV + kk) * NF + p] = b;
      }
    }
    __syncthreads();
    // lift: L[k][m] += sum_p B_f(p, m) z4[k][p] + sum_p sum_i G_i(p, m) z5[i][k][p]
    for (int i = threadIdx.x; i < NV * NM; i += blockDim.x) {
      const int kk = i / NM, m = i % NM;
      double a = 0.0;
      for (int p = 0; p < NF; ++p) {
        a += fb(lf, p, m, -1, rh) * z4[kk * NF + p];
#pragma unroll
        for (int j = 0; j < DIM; ++j) a += fb(lf, p, m, j, rh) * z5[(j * NV + kk) * NF + p];
      }
      L0[i] += a;
    }
    __syncthreads();
  }
  const double* res = apply_minv_tensor<DIM, N, double>(sMi, g.idet, L0, L1, NV);
  for (int i = threadIdx.x; i < NV * NM; i += blockDim.x)
    y[(long long)e * NV * NM + i] += dta * res[i];
}

// ---------------------------------------------------------------- drivers
#define DG_VISC_INSTANCES(X) \
  X(2, 1, 3) X(2, 2, 3) X(2, 2, 4) X(2, 3, 5) X(2, 4, 6) X(2, 5, 7) X(2, 6, 8) X(3, 1, 3) \
  X(3, 2, 4) X(3, 3, 6)

bool visc_supported(int dim, int P, int Q) {
#define DG_VS(D_, P_, Q_) \
  if (dim == D_ && P == P_ && Q == Q_) return true;
  DG_VISC_INSTANCES(DG_VS)
#undef DG_VS
  return false;
}

size_t visc_values_per_face_point(int dim) {
  return dim == 2 ? ViscSizes<2>::NK : ViscSizes<3>::NK;  // NK = NS
}

template <int D, int P, int Q, typename T>
static dg_status visc_build_t(dg_mesh_s* m, dg_precond_s* pc, double t, double dta,
                              void* blk, int ld, cudaStream_t s) {
  using C = Cfg<D, P, Q>;
  const double* chi = m->scratch + 8;  // set by the term-3 build
  T* K = (T*)pc->jk;
  T* Sd = (T*)pc->jsd;
  T* So = (T*)pc->jso;
  DG_PROF(K_BRJ_TRACEJAC, s, brj_visc_trace_kernel<D, P, Q, T><<<(m->F * C::NF + 127) / 128, 128, 0, s>>>(
      m->tab, m->phys, m->geo, m->faces, m->F, t, m->tbuf, chi, K, Sd, So));
  DG_LAUNCHED(1);
  const size_t sm = sizeof(T) * 2 * C::NM * C::NM;
  DG_CUDA(cudaFuncSetAttribute(brj_block_visc_kernel<D, P, Q, T>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  DG_PROF(K_BRJ_BLOCK, s, brj_block_visc_kernel<D, P, Q, T><<<dim3(m->E, C::NV * C::NV), 256, sm, s>>>(
      m->tab, m->geo, K, Sd, dta, (T*)blk, ld));
  DG_LAUNCHED(1);
  return DG_OK;
}

dg_status visc_build(dg_mesh_s* m, dg_precond_s* pc, double t, double dta, void* blk, int ld,
                     bool fp64, cudaStream_t s) {
#define DG_VB(D_, P_, Q_)                                                        \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                                \
    if (fp64) return visc_build_t<D_, P_, Q_, double>(m, pc, t, dta, blk, ld, s); \
    return visc_build_t<D_, P_, Q_, float>(m, pc, t, dta, blk, ld, s);           \
  }
  DG_VISC_INSTANCES(DG_VB)
#undef DG_VB
  return DG_ERR_UNSUPPORTED;
}

dg_status visc_offdiag(dg_precond_s* pc, const double* qh, double* y, cudaStream_t s) {
  dg_mesh_s* m = pc->mesh;
  const bool fp64 = pc->precision == DG_PREC_FP64;
#define DG_VO(D_, P_, Q_)                                                                    \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                                            \
    if (fp64) {                                                                              \
      DG_PROF(K_BRJ_OFFDIAG, s, brj_offdiag_visc_kernel<D_, P_, Q_, double><<<m->E, 128, 0, s>>>( \
          m->tab, m->geo, (const double*)pc->jk, (const double*)pc->jso, pc->nbr, qh, pc->dt_a, y)); \
    } else {                                                                                 \
      DG_PROF(K_BRJ_OFFDIAG, s, brj_offdiag_visc_kernel<D_, P_, Q_, float><<<m->E, 128, 0, s>>>( \
          m->tab, m->geo, (const float*)pc->jk, (const float*)pc->jso, pc->nbr, qh, pc->dt_a, y)); \
    }                                                                                        \
    DG_LAUNCHED(1);                                                                          \
    return DG_OK;                                                                            \
  }
  DG_VISC_INSTANCES(DG_VO)
#undef DG_VO
  return DG_ERR_UNSUPPORTED;
}

}  // namespace dg
