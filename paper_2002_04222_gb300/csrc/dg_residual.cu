// DG residual R(u) = M^-1 L(u, t) of Sec. 3.1 (Eq. matrix-form-equations) in
// three FP64 kernels, each in two geometry variants: axis-aligned affine
// quads/hexes (diagonal metric, tensor-product inverse mass) and general
// elements (curved or rotated: per-point metrics, dense inverse mass):
//   vol_kernel   sum-factorised BwdTrans (B), collocation derivatives on the
//                Gauss grid (D_j), fused Euler + viscous volume flux H_j
//                weighted by w|J| and the reference metric, and the face
//                traces of Q and grad Q (interpolation J to the faces);
//   face_kernel  one thread per face point: Riemann flux (Roe/HLLC), the
//                interior-penalty viscous flux and the symmetric flux S_i;
//   lift_kernel  spreads the face fluxes back onto the Gauss grid (J^T),
//                applies sum_j D_j^T, B^T and the inverse mass matrix
//                |J|^-1 (M1^-1)^(x)d, adds the forcing and (for the
//                Jacobian-free product) the finite-difference combination.
// FP64 throughout: on GB300 this path is bound by the FP64 pipe, so every
// stage is written to issue as few FP64 instructions as possible.
#include <cstdio>
#include <vector>
#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_sumfact.cuh"

namespace dg {

// ---------------------------------------------------------------- shock sensor
// Artificial-viscosity factor f_e = mu_0 S_e h_e / P of element e (Sec. 3.1.2),
// by one warp: the density's modified-basis coefficients (in A, overwritten;
// B is scratch of the same size) go to Legendre coefficients c by the 1-D
// transform along each direction; the reference-element L2 norms are then
// sums of c^2 times the Legendre norms, and the part removed by the
// projection onto degree <= P-1 per direction is the set of modes with some
// index equal to P.  Lane 0 writes avf[e].
template <int DIM, int P, int Q, bool CV>
__device__ void sensor_element(const SensorTab& st, const Phys& ph,
                               const ElemGeo* __restrict__ geo, const GenGeo& gg, int e,
                               double* A, double* B, int lane, double* __restrict__ avf) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NM = C::NM, NQ = C::NQ;
  double* src = A;
  double* dst = B;
  int stride = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    for (int mm = lane; mm < NM; mm += 32) {
      const int id = (mm / stride) % N;
      const int m0 = mm - id * stride;
      double a = 0.0;
#pragma unroll
      for (int k = 0; k < N; ++k) a = fma(st.T[id * N + k], src[m0 + k * stride], a);
      dst[mm] = a;
    }
    __syncwarp();
    double* tmp = src;
    src = dst;
    dst = tmp;
    stride *= N;
  }
  double num = 0.0, den = 0.0, vol = 0.0;
  for (int mm = lane; mm < NM; mm += 32) {
    int r = mm;
    double wgt = 1.0;
    bool top = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int id = r % N;
      r /= N;
      wgt *= st.nrm[id];
      top = top || id == P;
    }
    const double c2 = src[mm] * src[mm] * wgt;
    den += c2;
    if (top) num += c2;
  }
  if constexpr (CV) {
    const double* wj = gg.vgeo + (long long)e * (DIM * DIM + 1) * NQ + DIM * DIM * NQ;
    for (int q = lane; q < NQ; q += 32) vol += wj[q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
    vol += __shfl_xor_sync(0xffffffffu, vol, o);
  }
  if (lane != 0) return;
  // below the ramp (the common case) no logarithm, sine or root is taken
  double S = 0.0;
  if (num > 0.0 && den > 0.0 && num >= st.lo * den) {
    if (num > st.hi * den) {
      S = 1.0;
    } else {
      const double se = log10(num / den), s0 = -4.0 * log10((double)P), kap = ph.av_kappa;
      S = 0.5 * (1.0 + sin(3.14159265358979323846 * (se - s0) / (2.0 * kap)));
    }
  }
  if (S == 0.0) {
    avf[e] = 0.0;
    return;
  }
  if constexpr (!CV) vol = geo[e].detJ * (double)(1 << DIM);
  const double h = DIM == 2 ? sqrt(vol) : cbrt(vol);
  avf[e] = ph.av_mu0 * S * h / (double)P;
}

// The factor of every element at u alone (dg_av_factor); the residual
// computes it inside the volume kernel.  One warp per element.
constexpr int SENSOR_WARPS = 8;
template <int DIM, int P, int Q, bool CV>
__global__ void __launch_bounds__(32 * SENSOR_WARPS) sensor_kernel(
    const __grid_constant__ SensorTab st, const __grid_constant__ Phys ph,
    const ElemGeo* __restrict__ geo, const __grid_constant__ GenGeo gg, int E,
    const double* __restrict__ u, double* __restrict__ avf) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NM = C::NM;
  __shared__ double sA[SENSOR_WARPS][NM], sC[SENSOR_WARPS][NM];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * SENSOR_WARPS + w;
  if (e >= E) return;  // warp-uniform; the kernel has no block-wide barrier
  const long long base = (long long)e * NV * NM;  // variable 0: density
  for (int k = lane; k < NM; k += 32) sA[w][k] = u[base + k];
  __syncwarp();
  sensor_element<DIM, P, Q, CV>(st, ph, geo, gg, e, sA[w], sC[w], lane, avf);
}

// ---------------------------------------------------------------- kernel 1
template <int DIM, int P, int Q, bool CV>
__global__ void __launch_bounds__(256) vol_kernel(const __grid_constant__ Tables tab,
                                                  const __grid_constant__ Phys ph,
                                                  const ElemGeo* __restrict__ geo,
                                                  const __grid_constant__ GenGeo gg, int E,
                                                  const double* __restrict__ u,
                                                  const double* __restrict__ v,
                                                  const double* __restrict__ epsp,
                                                  double* __restrict__ hbuf,
                                                  double* __restrict__ tbuf, const int EPB,
                                                  const __grid_constant__ SensorTab st,
                                                  double* __restrict__ avf_out) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NQ = C::NQ, NF = C::NF;
  constexpr int Q2 = C::Q2, N2 = C::N2;
  extern __shared__ double sm[];
  double* sB = sm;
  double* sD = sB + Q * N;
  double* sl = sD + Q * Q;  // lm, lp
  double* sw = sl + 2 * Q + N * N;
  double* sU = sm + C::TAB;            // [EPB][NV][NM]
  double* sQ = sU + EPB * NV * NM;     // [EPB][NV][NQ]
  double* sG = sQ + EPB * NV * NQ;     // DIM arrays [EPB][NV][NQ]
  double* sT = sG + EPB * DIM * NV * NQ;  // 2-D only: scratch
  const int e0 = blockIdx.x * EPB;
  const int nrep = EPB * NV;

  stage_tables<DIM, P, Q>(tab, sm);
  const double eps = v ? epsp[0] : 0.0;
  for (int i = threadIdx.x; i < EPB * NV * NM; i += blockDim.x) {
    const int eb = i / (NV * NM);
    const long long g = (long long)(e0 + eb) * NV * NM + (i - eb * NV * NM);
    double val = 0.0;
    if (e0 + eb < E) {
      val = u[g];
      if (v) val = fma(eps, v[g], val);
    }
    sU[i] = val;
  }
  __syncthreads();
  if (avf_out) {
    // shock capturing: the factor of each element at the evaluated state, one
    // warp per element, the density coefficients copied to scratch in sQ
    // (free until BwdTrans); the volume flux below and the face kernel read it
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int eb = wp; eb < EPB; eb += nw) {
      if (e0 + eb >= E) continue;  // warp-uniform
      double* A = sQ + (long long)eb * NV * NQ;
      double* Bs = A + NM;
      for (int k = lane; k < NM; k += 32) A[k] = sU[eb * NV * NM + k];
      __syncwarp();
      sensor_element<DIM, P, Q, CV>(st, ph, geo, gg, e0 + eb, A, Bs, lane, avf_out);
      __syncwarp();
    }
    __syncthreads();
  }
  // BwdTrans: contract direction 0, 1 (, 2) with B
  if (DIM == 2) {
    contract<N, N, 1, 0, Q, N, 1, false>(sU, sT, sB, nrep);
    __syncthreads();
    contract<Q, N, 1, 1, Q, N, 1, false>(sT, sQ, sB, nrep);
  } else {
    double* t1 = sG + EPB * NV * NQ;       // reuse gradient slots 1 and 2
    double* t2 = sG + 2 * EPB * NV * NQ;
    contract<N, N, N2, 0, Q, N, 1, false>(sU, t1, sB, nrep);
    __syncthreads();
    contract<Q, N, N2, 1, Q, N, 1, false>(t1, t2, sB, nrep);
    __syncthreads();
    contract<Q, Q, N2, 2, Q, N, 1, false>(t2, sQ, sB, nrep);
  }
  __syncthreads();
  // reference derivatives on the Gauss grid (exact for the degree-P expansion)
  contract<Q, Q, Q2, 0, Q, Q, 1, false>(sQ, sG, sD, nrep);
  contract<Q, Q, Q2, 1, Q, Q, 1, false>(sQ, sG + EPB * NV * NQ, sD, nrep);
  if (DIM == 3) contract<Q, Q, Q2, 2, Q, Q, 1, false>(sQ, sG + 2 * EPB * NV * NQ, sD, nrep);
  __syncthreads();
  // volume flux at the Gauss points
  for (int idx = threadIdx.x; idx < EPB * NQ; idx += blockDim.x) {
    const int eb = idx / NQ, q = idx - eb * NQ;
    const int e = e0 + eb;
    if (e >= E) continue;
    if constexpr (CV) {
      // general element: grad = sum_r (d xi_r/dx) d_r, contravariant flux
      // w|J| sum_j (d xi_r/d x_j) H_j
      const double* gp = gg.vgeo + (long long)e * (DIM * DIM + 1) * NQ + q;
      double gi[DIM][DIM];
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int j = 0; j < DIM; ++j) gi[r][j] = gp[(r * DIM + j) * NQ];
      const double wJ = gp[DIM * DIM * NQ];
      double U[NV], dU[DIM][NV], H[DIM][NV];
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) {
        U[vv] = sQ[(eb * NV + vv) * NQ + q];
        double dr[DIM];
#pragma unroll
        for (int r = 0; r < DIM; ++r) dr[r] = sG[((r * EPB + eb) * NV + vv) * NQ + q];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          double a = 0.0;
#pragma unroll
          for (int r = 0; r < DIM; ++r) a = fma(gi[r][j], dr[r], a);
          dU[j][vv] = a;
        }
      }
      ns_volume_flux<DIM>(U, dU, ph, H, ph.avf ? ph.avf[e] : 0.0);
      double* hb = hbuf + (long long)e * DIM * NV * NQ + q;
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) {
          double a = 0.0;
#pragma unroll
          for (int j = 0; j < DIM; ++j) a = fma(gi[r][j], H[j][vv], a);
          hb[(r * NV + vv) * NQ] = wJ * a;
        }
      continue;
    }
    const ElemGeo g = geo[e];
    int c[3];
    grid_coords<DIM, Q>(q, c);
    double U[NV], dU[DIM][NV], H[DIM][NV];
    double rh[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) rh[r] = g.rh[r];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      U[vv] = sQ[(eb * NV + vv) * NQ + q];
#pragma unroll
      for (int r = 0; r < DIM; ++r) dU[r][vv] = sG[((r * EPB + eb) * NV + vv) * NQ + q] * rh[r];
    }
    ns_volume_flux<DIM>(U, dU, ph, H, ph.avf ? ph.avf[e] : 0.0);
    double wJ = sw[c[0]] * sw[c[1]] * (DIM == 3 ? sw[c[2]] : 1.0);
    wJ *= g.detJ;
    double* hb = hbuf + (long long)e * DIM * NV * NQ + q;
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      const double s = wJ * rh[r];
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) hb[(r * NV + vv) * NQ] = s * H[r][vv];
    }
  }
  // face traces of Q and grad Q by Lagrange extrapolation along the normal
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  if constexpr (CV) {
    // general element: extrapolate the value and the DIM reference
    // derivatives (polynomials along the line), then map the derivatives with
    // the metric of the face point
    constexpr int NTV = 2 * DIM * NV * NF;
    for (int idx = threadIdx.x; idx < EPB * NTV; idx += blockDim.x) {
      const int eb = idx / NTV;
      int rem = idx - eb * NTV;
      const int e = e0 + eb;
      if (e >= E) continue;
      const int p = rem % NF;
      rem /= NF;
      const int vv = rem % NV;
      const int lf = rem / NV;
      const int r = lf >> 1;
      const double* lw = sl + (lf & 1) * Q;
      int c[3] = {0, 0, 0};
      if (DIM == 2) {
        c[1 - r] = p;
      } else {
        const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
        c[t0] = p % Q;
        c[t1] = p / Q;
      }
      const int base = c[0] + Q * c[1] + Q * Q * c[2];
      const int str = r == 0 ? 1 : (r == 1 ? Q : Q * Q);
      double ext[1 + DIM];
#pragma unroll
      for (int fld = 0; fld <= DIM; ++fld) {
        const double* src = fld == 0 ? sQ + (eb * NV + vv) * NQ
                                     : sG + (((fld - 1) * EPB + eb) * NV + vv) * NQ;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < Q; ++k) acc = fma(lw[k], src[base + k * str], acc);
        ext[fld] = acc;
      }
      const double* gp = gg.fgeo + ((long long)e * 2 * DIM + lf) * DIM * DIM * NF + p;
      double* tb = tbuf + (long long)e * NTR + (lf * (1 + DIM) * NV + vv) * NF + p;
      tb[0] = ext[0];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double a = 0.0;
#pragma unroll
        for (int rr = 0; rr < DIM; ++rr) a = fma(gp[(rr * DIM + j) * NF], ext[1 + rr], a);
        tb[(1 + j) * NV * NF] = a;
      }
    }
    return;
  }
  for (int idx = threadIdx.x; idx < EPB * NTR; idx += blockDim.x) {
    const int eb = idx / NTR;
    int rem = idx - eb * NTR;
    const int e = e0 + eb;
    if (e >= E) continue;
    const int p = rem % NF;
    rem /= NF;
    const int vv = rem % NV;
    rem /= NV;
    const int fld = rem % (1 + DIM);
    const int lf = rem / (1 + DIM);
    const int r = lf >> 1;
    const double* lw = sl + (lf & 1) * Q;
    const double* src = fld == 0 ? sQ + (eb * NV + vv) * NQ
                                 : sG + (((fld - 1) * EPB + eb) * NV + vv) * NQ;
    // grid offset of the face point and stride along direction r
    int c[3] = {0, 0, 0};
    if (DIM == 2) {
      c[1 - r] = p;
    } else {
      const int t0 = r == 0 ? 1 : 0, t1 = r == 2 ? 1 : 2;
      c[t0] = p % Q;
      c[t1] = p / Q;
    }
    const int base = c[0] + Q * c[1] + Q * Q * c[2];
    const int str = r == 0 ? 1 : (r == 1 ? Q : Q * Q);
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k) acc = fma(lw[k], src[base + k * str], acc);
    if (fld > 0) acc *= geo[e].rh[fld - 1];
    tbuf[(long long)e * NTR + ((lf * (1 + DIM) + fld) * NV + vv) * NF + p] = acc;
  }
}

// ---------------------------------------------------------------- kernel 2
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(128) face_kernel(const __grid_constant__ Tables tab,
                                                   const __grid_constant__ Phys ph,
                                                   const ElemGeo* __restrict__ geo,
                                                   const int32_t* __restrict__ faces, int F,
                                                   double t, const double* __restrict__ dscal,
                                                   const double* __restrict__ tbuf,
                                                   double* __restrict__ fbuf) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NF = C::NF;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  if (dscal) t = dscal[0];
  const int f = idx / NF, p = idx - f * NF;
  const int eL = faces[f * 6 + 0], fL = faces[f * 6 + 1];
  const int eR = faces[f * 6 + 2], fR = faces[f * 6 + 3], bc = faces[f * 6 + 5];
  const int r = fL >> 1;
  const double sgn = (fL & 1) ? 1.0 : -1.0;
  const ElemGeo gL = geo[eL];
  // tangential Gauss indices of the face point
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
  double QL[NV], dQL[DIM][NV], QR[NV], dQa[DIM][NV];
  const double* tl = tbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) {
    QL[vv] = tl[vv * NF];
#pragma unroll
    for (int j = 0; j < DIM; ++j) dQL[j][vv] = tl[((1 + j) * NV + vv) * NF];
  }
  double rmax = gL.rh[r], cfac;  // 2 / min(h_L, h_R)
  double rhR[DIM];
  int bctype = 0;
  if (eR >= 0) {
    const ElemGeo gR = geo[eR];
    rmax = fmax(rmax, gR.rh[r]);
#pragma unroll
    for (int k = 0; k < DIM; ++k) rhR[k] = gR.rh[k];
    const double* tr = tbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      QR[vv] = tr[vv * NF];
#pragma unroll
      for (int j = 0; j < DIM; ++j) dQa[j][vv] = 0.5 * (dQL[j][vv] + tr[((1 + j) * NV + vv) * NF]);
    }
    cfac = 0.5;
  } else {
    bctype = ph.bc[bc];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      QR[vv] = 0.0;
#pragma unroll
      for (int j = 0; j < DIM; ++j) dQa[j][vv] = dQL[j][vv];
    }
    cfac = 1.0;
  }
  double Hn[NV], S[DIM][NV];
  const double beta = (double)((P + 1) * (P + 1)) * 0.5 * rmax;  // (P+1)^2 / h
  const double mua = av_face<DIM>(ph, eL, eR, QL, QR, dQa);
  if (r == 0)
    numerical_flux_axis<DIM, 0>(QL, QR, bctype, x, t, dQa, sgn, beta, ph, Hn, S, mua);
  else if (r == 1)
    numerical_flux_axis<DIM, 1>(QL, QR, bctype, x, t, dQa, sgn, beta, ph, Hn, S, mua);
  else
    numerical_flux_axis<DIM, DIM - 1>(QL, QR, bctype, x, t, dQa, sgn, beta, ph, Hn, S, mua);
  double* fl = fbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
  const double cs = ph.viscous ? cfac * ph.beta_s * wJf : 0.0;
  double csL[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) csL[j] = cs * gL.rh[j];
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) {
    fl[vv * NF] = -Hn[vv] * wJf;
#pragma unroll
    for (int j = 0; j < DIM; ++j) fl[((1 + j) * NV + vv) * NF] = csL[j] * S[j][vv];
  }
  if (eR >= 0) {
    double* fr = fbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int j = 0; j < DIM; ++j) csL[j] = cs * rhR[j];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      fr[vv * NF] = Hn[vv] * wJf;
#pragma unroll
      for (int j = 0; j < DIM; ++j) fr[((1 + j) * NV + vv) * NF] = csL[j] * S[j][vv];
    }
  }
}

// general elements: one thread per face point with the owner-side normal,
// surface weight and coordinates of the point, the face's penalty factor, and
// each side's metric at the point for the symmetric-flux lift
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(128) face_kernel_gen(const __grid_constant__ Phys ph,
                                                       const __grid_constant__ GenGeo gg,
                                                       const int32_t* __restrict__ faces, int F,
                                                       double t, const double* __restrict__ dscal,
                                                       const double* __restrict__ tbuf,
                                                       double* __restrict__ fbuf) {
  using C = Cfg<DIM, P, Q>;
  constexpr int NV = C::NV, NF = C::NF;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  if (dscal) t = dscal[0];
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
  double QL[NV], QR[NV], dQa[DIM][NV];
  const double* tl = tbuf + (long long)eL * NTR + (fL * (1 + DIM)) * NV * NF + p;
#pragma unroll
  for (int vv = 0; vv < NV; ++vv) {
    QL[vv] = tl[vv * NF];
#pragma unroll
    for (int j = 0; j < DIM; ++j) dQa[j][vv] = tl[((1 + j) * NV + vv) * NF];
  }
  int bctype = 0;
  double cfac = 1.0;
  if (eR >= 0) {
    const double* tr = tbuf + (long long)eR * NTR + (fR * (1 + DIM)) * NV * NF + p;
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      QR[vv] = tr[vv * NF];
#pragma unroll
      for (int j = 0; j < DIM; ++j) dQa[j][vv] = 0.5 * (dQa[j][vv] + tr[((1 + j) * NV + vv) * NF]);
    }
    cfac = 0.5;
  } else {
    bctype = ph.bc[bc];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) QR[vv] = 0.0;
  }
  double Hn[NV], S[DIM][NV];
  numerical_flux_n<DIM>(QL, QR, bctype, x, t, dQa, n, gg.fbeta[f], ph, Hn, S,
                        av_face<DIM>(ph, eL, eR, QL, QR, dQa));
  const double cs = ph.viscous ? cfac * ph.beta_s * wJf : 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int e = side == 0 ? eL : eR, lf = side == 0 ? fL : fR;
    if (e < 0) break;
    const double* gp = gg.fgeo + ((long long)e * 2 * DIM + lf) * DIM * DIM * NF + p;
    double* fo = fbuf + (long long)e * NTR + (lf * (1 + DIM)) * NV * NF + p;
    const double sg = side == 0 ? -wJf : wJf;
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) fo[vv * NF] = sg * Hn[vv];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      double gr[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) gr[j] = cs * gp[(r * DIM + j) * NF];
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) {
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) a = fma(gr[j], S[j][vv], a);
        fo[((1 + r) * NV + vv) * NF] = a;
      }
    }
  }
}

// B^T on G [EPB][NV][NQ] -> result in R [EPB][NV][NM] (general elements: the
// dense inverse mass matrix is applied by the caller)
template <int DIM, int P, int Q>
__device__ __forceinline__ void bt_only(double* sG, double* t1, double* t2, double* sR,
                                        const double* sB, int nrep) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, Q2 = C::Q2, N2 = C::N2;
  if (DIM == 2) {
    contract<Q, Q, 1, 1, N, 1, N, false>(sG, t1, sB, nrep);
    __syncthreads();
    contract<Q, N, 1, 0, N, 1, N, false>(t1, sR, sB, nrep);
  } else {
    contract<Q, Q, Q2, 2, N, 1, N, false>(sG, t1, sB, nrep);
    __syncthreads();
    contract<Q, Q, N2, 1, N, 1, N, false>(t1, t2, sB, nrep);
    __syncthreads();
    contract<Q, N, N2, 0, N, 1, N, false>(t2, sR, sB, nrep);
  }
  __syncthreads();
}

// out = M_e^-1 x for the coefficient vector x (NM values in shared memory)
template <int NM>
__device__ __forceinline__ double dense_minv_row(const double* __restrict__ Mi, int m,
                                                 const double* x) {
  double a = 0.0;
#pragma unroll 8
  for (int k = 0; k < NM; ++k) a = fma(Mi[(long long)k * NM + m], x[k], a);  // M^-1 symmetric
  return a;
}

// B^T then |J|^-1 (M1^-1)^(x)d on G [EPB][NV][NQ] -> result in R [EPB][NV][NM]
template <int DIM, int P, int Q>
__device__ __forceinline__ void bt_minv(double* sG, double* t1, double* t2, double* sR,
                                        const double* sB, const double* sMi, int nrep) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, Q2 = C::Q2, N2 = C::N2;
  if (DIM == 2) {
    contract<Q, Q, 1, 1, N, 1, N, false>(sG, t1, sB, nrep);
    __syncthreads();
    contract<Q, N, 1, 0, N, 1, N, false>(t1, t2, sB, nrep);
    __syncthreads();
    contract<N, N, 1, 0, N, N, 1, false>(t2, t1, sMi, nrep);
    __syncthreads();
    contract<N, N, 1, 1, N, N, 1, false>(t1, sR, sMi, nrep);
  } else {
    contract<Q, Q, Q2, 2, N, 1, N, false>(sG, t1, sB, nrep);
    __syncthreads();
    contract<Q, Q, N2, 1, N, 1, N, false>(t1, t2, sB, nrep);
    __syncthreads();
    contract<Q, N, N2, 0, N, 1, N, false>(t2, t1, sB, nrep);
    __syncthreads();
    contract<N, N, N2, 0, N, N, 1, false>(t1, t2, sMi, nrep);
    __syncthreads();
    contract<N, N, N2, 1, N, N, 1, false>(t2, t1, sMi, nrep);
    __syncthreads();
    contract<N, N, N2, 2, N, N, 1, false>(t1, sR, sMi, nrep);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- kernel 3
template <int DIM, int P, int Q, bool CV>
__global__ void __launch_bounds__(256) lift_kernel(const __grid_constant__ Tables tab,
                                                   const ElemGeo* __restrict__ geo,
                                                   const __grid_constant__ GenGeo gg, int E,
                                                   const double* __restrict__ hbuf,
                                                   const double* __restrict__ fbuf,
                                                   const double* __restrict__ force,
                                                   const double* __restrict__ v,
                                                   const double* __restrict__ r_u,
                                                   const double* __restrict__ epsp, double alpha,
                                                   double beta, const double* __restrict__ dscal,
                                                   double* __restrict__ out, const int EPB) {
  if (dscal) beta = dscal[1];
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NQ = C::NQ, NF = C::NF;
  constexpr int Q2 = C::Q2;
  constexpr int NTR = 2 * DIM * (1 + DIM) * NV * NF;
  extern __shared__ double sm[];
  double* sB = sm;
  double* sD = sB + Q * N;
  double* sl = sD + Q * Q;
  double* sMi = sl + 2 * Q;
  double* sH = sm + C::TAB;             // DIM arrays [EPB][NV][NQ]
  double* sG = sH + DIM * EPB * NV * NQ;  // [EPB][NV][NQ]
  double* t1 = sG + EPB * NV * NQ;
  double* t2 = t1 + EPB * NV * NQ;
  const int e0 = blockIdx.x * EPB;
  const int nrep = EPB * NV;
  stage_tables<DIM, P, Q>(tab, sm);
  for (int i = threadIdx.x; i < EPB * DIM * NV * NQ; i += blockDim.x) {
    const int eb = i / (DIM * NV * NQ), rem = i - eb * DIM * NV * NQ;
    const int r = rem / (NV * NQ), o = rem - r * NV * NQ;
    sH[(r * EPB + eb) * NV * NQ + o] =
        e0 + eb < E ? hbuf[(long long)(e0 + eb) * DIM * NV * NQ + rem] : 0.0;
  }
  __syncthreads();
  // J^T: spread the face fluxes of the 2*DIM faces onto the Gauss grid
  for (int idx = threadIdx.x; idx < EPB * NV * NQ; idx += blockDim.x) {
    const int eb = idx / (NV * NQ), rem = idx - eb * NV * NQ;
    const int vv = rem / NQ, q = rem - vv * NQ;
    const int e = e0 + eb;
    double gsum = 0.0;
    double hs[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) hs[j] = 0.0;
    if (e < E) {
      int c[3];
      grid_coords<DIM, Q>(q, c);
      const double* fb = fbuf + (long long)e * NTR;
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        const int p = face_point<DIM, Q>(c, r);
        const double am = sl[c[r]], ap = sl[Q + c[r]];
        const double* fm = fb + ((2 * r) * (1 + DIM) * NV + vv) * NF + p;
        const double* fp = fb + ((2 * r + 1) * (1 + DIM) * NV + vv) * NF + p;
        gsum = fma(am, fm[0], fma(ap, fp[0], gsum));
#pragma unroll
        for (int j = 0; j < DIM; ++j)
          hs[j] = fma(am, fm[(1 + j) * NV * NF], fma(ap, fp[(1 + j) * NV * NF], hs[j]));
      }
    }
    sG[idx] = gsum;
#pragma unroll
    for (int j = 0; j < DIM; ++j) sH[j * EPB * NV * NQ + idx] += hs[j];
  }
  __syncthreads();
  // G += sum_j D_j^T H_j
  contract<Q, Q, Q2, 0, Q, 1, Q, true>(sH, sG, sD, nrep);
  __syncthreads();
  contract<Q, Q, Q2, 1, Q, 1, Q, true>(sH + EPB * NV * NQ, sG, sD, nrep);
  __syncthreads();
  if (DIM == 3) {
    contract<Q, Q, Q2, 2, Q, 1, Q, true>(sH + 2 * EPB * NV * NQ, sG, sD, nrep);
    __syncthreads();
  }
  double* sR = sH;  // reuse
  if constexpr (CV)
    bt_only<DIM, P, Q>(sG, t1, t2, sR, sB, nrep);
  else
    bt_minv<DIM, P, Q>(sG, t1, t2, sR, sB, sMi, nrep);
  for (int i = threadIdx.x; i < EPB * NV * NM; i += blockDim.x) {
    const int eb = i / (NV * NM);
    const int e = e0 + eb;
    if (e >= E) continue;
    const long long gi = (long long)e * NV * NM + (i - eb * NV * NM);
    double R;
    if constexpr (CV) {
      const int m = i % NM;
      R = dense_minv_row<NM>(gg.minv + (long long)e * NM * NM, m, sR + (i - m));
    } else {
      R = sR[i] * geo[e].idet;
    }
    if (force) R += force[gi];
    if (r_u) {
      const double ie = epsp[1];
      R = (R - r_u[gi]) * ie * beta;
      if (alpha != 0.0) R = fma(alpha, v[gi], R);
    }
    out[gi] = R;
  }
}

// L2 projection of the analytic field (what = 0) or of the forcing (what = 1)
template <int DIM, int P, int Q, bool CV>
__global__ void __launch_bounds__(256) project_kernel(const __grid_constant__ Tables tab,
                                                      const __grid_constant__ Phys ph,
                                                      const ElemGeo* __restrict__ geo,
                                                      const __grid_constant__ GenGeo gg, int E,
                                                      int what, double t,
                                                      double* __restrict__ out) {
  using C = Cfg<DIM, P, Q>;
  constexpr int N = C::N, NV = C::NV, NM = C::NM, NQ = C::NQ, EPB = C::EPB;
  extern __shared__ double sm[];
  double* sB = sm;
  double* sl = sB + Q * N + Q * Q;
  double* sMi = sl + 2 * Q;
  double* sw = sMi + N * N;
  double* sH = sm + C::TAB;
  double* sG = sH + DIM * EPB * NV * NQ;
  double* t1 = sG + EPB * NV * NQ;
  double* t2 = t1 + EPB * NV * NQ;
  const int e0 = blockIdx.x * EPB;
  stage_tables<DIM, P, Q>(tab, sm);
  __syncthreads();
  for (int idx = threadIdx.x; idx < EPB * NQ; idx += blockDim.x) {
    const int eb = idx / NQ, q = idx - eb * NQ;
    const int e = e0 + eb;
    double U[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) U[vv] = 0.0;
    if (e < E) {
      double x[3] = {0, 0, 0};
      double wJ = 1.0;
      if constexpr (CV) {
        for (int r = 0; r < DIM; ++r) x[r] = gg.vx[((long long)e * DIM + r) * NQ + q];
        wJ = gg.vgeo[((long long)e * (DIM * DIM + 1) + DIM * DIM) * NQ + q];
      } else {
        const ElemGeo g = geo[e];
        int c[3];
        grid_coords<DIM, Q>(q, c);
        for (int r = 0; r < DIM; ++r) {
          x[r] = g.x0[r] + 0.5 * (tab.x[c[r]] + 1.0) * g.h[r];
          wJ *= sw[c[r]] * 0.5 * g.h[r];
        }
      }
      if (what == 0)
        exact_state(DIM, ph, x, t, U);
      else
        forcing(DIM, ph, x, U);
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) U[vv] *= wJ;
    }
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) sG[(eb * NV + vv) * NQ + q] = U[vv];
  }
  __syncthreads();
  if constexpr (CV)
    bt_only<DIM, P, Q>(sG, t1, t2, sH, sB, EPB * NV);
  else
    bt_minv<DIM, P, Q>(sG, t1, t2, sH, sB, sMi, EPB * NV);
  for (int i = threadIdx.x; i < EPB * NV * NM; i += blockDim.x) {
    const int eb = i / (NV * NM);
    const int e = e0 + eb;
    if (e >= E) continue;
    double val;
    if constexpr (CV) {
      const int m = i % NM;
      val = dense_minv_row<NM>(gg.minv + (long long)e * NM * NM, m, sH + (i - m));
    } else {
      val = sH[i] * geo[e].idet;
    }
    out[(long long)e * NV * NM + (i - eb * NV * NM)] = val;
  }
}

// ---------------------------------------------------------------- launchers
template <int DIM, int P, int Q, bool CV>
static dg_status run_residual_g(dg_mesh_s* m, const EvalArgs& a, cudaStream_t s) {
  using C = Cfg<DIM, P, Q>;
  const int vepb = m->tune.vol_epb, vnt = m->tune.vol_threads;
  const int lepb = m->tune.lift_epb, lnt = m->tune.lift_threads;
  const size_t vsm = sizeof(double) * C::vol_sm(vepb), lsm = sizeof(double) * C::lift_sm(lepb);
  const GenGeo gg = gen_geo(m);
  DG_CUDA(cudaFuncSetAttribute(vol_kernel<DIM, P, Q, CV>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
  DG_CUDA(cudaFuncSetAttribute(lift_kernel<DIM, P, Q, CV>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
  if (!a.skip_vol) {
    // (with shock capturing the volume kernel also writes the elements'
    // artificial-viscosity factors, which the face kernel reads)
    DG_PROF(K_VOL, s, vol_kernel<DIM, P, Q, CV><<<(m->E + vepb - 1) / vepb, vnt, vsm, s>>>(
        m->tab, m->phys, m->geo, gg, m->E, a.u, a.v, a.eps, m->hbuf, m->tbuf, vepb, m->stab,
        m->phys.avf ? m->avf : nullptr));
    DG_LAUNCHED(1);
    const int nfp = m->F * C::NF;
    if constexpr (CV) {
      DG_PROF(K_FACE, s, face_kernel_gen<DIM, P, Q><<<(nfp + 127) / 128, 128, 0, s>>>(
          m->phys, gg, m->faces, m->F, a.t, a.dscal, m->tbuf, m->fbuf));
    } else {
      DG_PROF(K_FACE, s, face_kernel<DIM, P, Q><<<(nfp + 127) / 128, 128, 0, s>>>(
          m->tab, m->phys, m->geo, m->faces, m->F, a.t, a.dscal, m->tbuf, m->fbuf));
    }
    DG_LAUNCHED(1);
  }
  if (!a.skip_lift) {
    DG_PROF(K_LIFT, s, lift_kernel<DIM, P, Q, CV><<<(m->E + lepb - 1) / lepb, lnt, lsm, s>>>(
        m->tab, m->geo, gg, m->E, m->hbuf, m->fbuf, m->force, a.v, a.r_u, a.eps, a.alpha, a.beta,
        a.dscal, a.out, lepb));
    DG_LAUNCHED(1);
  }
  return DG_OK;
}

template <int DIM, int P, int Q>
static dg_status run_residual(dg_mesh_s* m, const EvalArgs& a, cudaStream_t s) {
  if (m->curved) {
    if constexpr (has_curved<DIM, P, Q>()) return run_residual_g<DIM, P, Q, true>(m, a, s);
    return DG_ERR_UNSUPPORTED;
  }
  return run_residual_g<DIM, P, Q, false>(m, a, s);
}

template <int DIM, int P, int Q>
static void default_tune(dg_mesh_s* m) {
  using C = Cfg<DIM, P, Q>;
  m->tune.vol_epb = m->tune.lift_epb = C::EPB;
  m->tune.vol_threads = m->tune.lift_threads = C::NT;
}

// candidate (elements per CTA, threads per CTA) launch shapes of the
// sum-factorisation kernels that fit the shared memory of one CTA
template <int DIM, int P, int Q>
static void tune_candidates(std::vector<int2>& vol, std::vector<int2>& lift) {
  using C = Cfg<DIM, P, Q>;
  const int epbs3[] = {1, 2, 3, 4};
  const int epbs2[] = {1, 2, 4, 8, 16, 32};
  // every warp multiple up to the kernels' bound: a count just above the
  // Gauss points of one or more elements (224 for 216 at Q = 6) gives the
  // per-point flux stage one pass without idle lanes
  const int nts[] = {64, 96, 128, 160, 192, 224, 256};
  const size_t cap = 200 * 1024;
  for (int e : (DIM == 3 ? std::vector<int>(epbs3, epbs3 + 4) : std::vector<int>(epbs2, epbs2 + 6)))
    for (int t : nts) {
      if (DIM == 3 && t < 128) continue;
      if (sizeof(double) * C::vol_sm(e) <= cap) vol.push_back(make_int2(e, t));
      if (sizeof(double) * C::lift_sm(e) <= cap) lift.push_back(make_int2(e, t));
    }
}

template <int DIM, int P, int Q, bool CV>
static dg_status run_project_g(dg_mesh_s* m, int what, double t, double* out, cudaStream_t s) {
  using C = Cfg<DIM, P, Q>;
  const int nb = (m->E + C::EPB - 1) / C::EPB;
  const size_t lsm = sizeof(double) * C::LIFT_SM;
  DG_CUDA(cudaFuncSetAttribute(project_kernel<DIM, P, Q, CV>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
  DG_PROF(K_PROJECT, s, project_kernel<DIM, P, Q, CV><<<nb, C::NT, lsm, s>>>(
      m->tab, m->phys, m->geo, gen_geo(m), m->E, what, t, out));
  DG_LAUNCHED(1);
  return DG_OK;
}

template <int DIM, int P, int Q>
static dg_status run_project(dg_mesh_s* m, int what, double t, double* out, cudaStream_t s) {
  if (m->curved) {
    if constexpr (has_curved<DIM, P, Q>()) return run_project_g<DIM, P, Q, true>(m, what, t, out, s);
    return DG_ERR_UNSUPPORTED;
  }
  return run_project_g<DIM, P, Q, false>(m, what, t, out, s);
}

// (dim, P, Q) instances built into the library
#define DG_INSTANCES(X)                                                                       \
  X(2, 1, 3) X(2, 2, 3) X(2, 2, 4) X(2, 3, 5) X(2, 4, 6) X(2, 5, 7) X(2, 6, 8) X(3, 1, 3) \
  X(3, 2, 4) X(3, 2, 5) X(3, 3, 5) X(3, 3, 6) X(3, 4, 6) X(3, 4, 8)

bool supported_curved(int dim, int P, int Q) {
#define DG_SUP(D_, P_, Q_) \
  if (dim == D_ && P == P_ && Q == Q_) return true;
  DG_CURVED_INSTANCES(DG_SUP)
#undef DG_SUP
  return false;
}

bool supported(int dim, int P, int Q) {
#define DG_SUP(D_, P_, Q_) \
  if (dim == D_ && P == P_ && Q == Q_) return true;
  DG_INSTANCES(DG_SUP)
#undef DG_SUP
  return false;
}

dg_status launch_residual(dg_mesh_s* m, const EvalArgs& a, cudaStream_t s) {
#define DG_RUN(D_, P_, Q_) \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) return run_residual<D_, P_, Q_>(m, a, s);
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
  return DG_ERR_UNSUPPORTED;
}

template <int DIM, int P, int Q>
static dg_status run_sensor(dg_mesh_s* m, const double* u, double* out, cudaStream_t s) {
  const GenGeo gg = gen_geo(m);
  const int nb = (m->E + SENSOR_WARPS - 1) / SENSOR_WARPS;
  if (m->curved) {
    if constexpr (has_curved<DIM, P, Q>()) {
      DG_PROF(K_SENSOR, s, sensor_kernel<DIM, P, Q, true><<<nb, 32 * SENSOR_WARPS, 0, s>>>(
          m->stab, m->phys, m->geo, gg, m->E, u, out));
      DG_LAUNCHED(1);
      return DG_OK;
    }
    return DG_ERR_UNSUPPORTED;
  }
  DG_PROF(K_SENSOR, s, sensor_kernel<DIM, P, Q, false><<<nb, 32 * SENSOR_WARPS, 0, s>>>(
      m->stab, m->phys, m->geo, gg, m->E, u, out));
  DG_LAUNCHED(1);
  return DG_OK;
}

dg_status launch_sensor(dg_mesh_s* m, const double* u, double* out, cudaStream_t s) {
#define DG_RUN(D_, P_, Q_) \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) return run_sensor<D_, P_, Q_>(m, u, out, s);
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
  return DG_ERR_UNSUPPORTED;
}

dg_status launch_project(dg_mesh_s* m, int what, double t, double* out, cudaStream_t s) {
#define DG_RUN(D_, P_, Q_) \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) return run_project<D_, P_, Q_>(m, what, t, out, s);
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
  return DG_ERR_UNSUPPORTED;
}

template <int DIM, int P, int Q>
static dg_status run_autotune(dg_mesh_s* m, int reps, dg_tune_result* res, cudaStream_t s) {
  std::vector<int2> vc, lc;
  tune_candidates<DIM, P, Q>(vc, lc);
  // a valid state to time on: the projected analytic field
  DG_TRY(launch_project(m, 0, 0.0, m->w1, s));
  EvalArgs a{};
  a.u = m->w1;
  a.out = m->w2;
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  const Tune keep = m->tune;
  auto time_it = [&](bool vol) -> double {
    EvalArgs b = a;
    b.skip_vol = !vol;
    b.skip_lift = vol;
    run_residual<DIM, P, Q>(m, b, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) run_residual<DIM, P, Q>(m, b, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  // volume + face kernels (the face kernel's launch is fixed and adds the same time to each);
  // the shape in effect before tuning is timed too when it is not a candidate
  double best = 1e30, dflt = -1.0;
  Tune t = keep;
  for (const int2& c : vc) {
    m->tune.vol_epb = c.x;
    m->tune.vol_threads = c.y;
    const double ms = time_it(true);
    if (c.x == keep.vol_epb && c.y == keep.vol_threads) dflt = ms;
    if (ms < best) {
      best = ms;
      t.vol_epb = c.x;
      t.vol_threads = c.y;
    }
  }
  if (dflt < 0.0) {
    m->tune.vol_epb = keep.vol_epb;
    m->tune.vol_threads = keep.vol_threads;
    dflt = time_it(true);
  }
  res->vol_ms = best;
  res->vol_ms_default = dflt;
  m->tune.vol_epb = t.vol_epb;
  m->tune.vol_threads = t.vol_threads;
  run_residual<DIM, P, Q>(m, a, s);  // traces and fluxes for the lift timing
  best = 1e30;
  dflt = -1.0;
  for (const int2& c : lc) {
    m->tune.lift_epb = c.x;
    m->tune.lift_threads = c.y;
    const double ms = time_it(false);
    if (c.x == keep.lift_epb && c.y == keep.lift_threads) dflt = ms;
    if (ms < best) {
      best = ms;
      t.lift_epb = c.x;
      t.lift_threads = c.y;
    }
  }
  if (dflt < 0.0) {
    m->tune.lift_epb = keep.lift_epb;
    m->tune.lift_threads = keep.lift_threads;
    dflt = time_it(false);
  }
  res->lift_ms = best;
  res->lift_ms_default = dflt;
  m->tune = t;
  res->vol_epb = t.vol_epb;
  res->vol_threads = t.vol_threads;
  res->lift_epb = t.lift_epb;
  res->lift_threads = t.lift_threads;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

void init_tune(dg_mesh_s* m) {
#define DG_RUN(D_, P_, Q_) \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) default_tune<D_, P_, Q_>(m);
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
}

dg_status autotune(dg_mesh_s* m, int reps, dg_tune_result* res, cudaStream_t s) {
#define DG_RUN(D_, P_, Q_) \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) return run_autotune<D_, P_, Q_>(m, reps, res, s);
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
  return DG_ERR_UNSUPPORTED;
}

bool tune_valid(dg_mesh_s* m, const dg_tune_result* t) {
  bool ok = false;
#define DG_RUN(D_, P_, Q_)                                                            \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                                     \
    std::vector<int2> vc, lc;                                                         \
    tune_candidates<D_, P_, Q_>(vc, lc);                                              \
    bool v = false, l = false;                                                        \
    for (const int2& c : vc) v |= c.x == t->vol_epb && c.y == t->vol_threads;         \
    for (const int2& c : lc) l |= c.x == t->lift_epb && c.y == t->lift_threads;       \
    ok = v && l;                                                                      \
  }
  DG_INSTANCES(DG_RUN)
#undef DG_RUN
  return ok;
}

}  // namespace dg
