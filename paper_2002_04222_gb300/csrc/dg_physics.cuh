// Device-side physics of the compressible Navier-Stokes equations (Sec. 2.1)
// and the numerical fluxes of Sec. 3.1, templated on the scalar type so that
// the volume flux can also be differentiated exactly with dual numbers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include "dg_internal.h"

namespace dg {

// ------------------------------------------------------------ dual numbers
// Forward-mode derivative carrier: v + d*e with e^2 = 0.
struct Dual {
  double v, d;
  __host__ __device__ Dual() : v(0), d(0) {}
  __host__ __device__ Dual(double a) : v(a), d(0) {}
  __host__ __device__ Dual(double a, double b) : v(a), d(b) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__host__ __device__ inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
__host__ __device__ inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
__device__ inline Dual dsqrt(Dual a) {
  double s = sqrt(a.v);
  return Dual(s, 0.5 * a.d / s);
}
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline double val(double a) { return a; }
__device__ inline double val(Dual a) { return a.v; }

// ------------------------------------------------------------ state helpers
template <int D, typename T>
__device__ inline void primitives(const T* U, const Phys& ph, T& irho, T* vel, T& p, T& temp) {
  irho = T(1.0) / U[0];
  T ke = T(0.0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vel[k] = U[1 + k] * irho;
    ke += U[1 + k] * vel[k];
  }
  p = T(ph.gm1) * (U[D + 1] - T(0.5) * ke);
  temp = T(ph.gMa2) * p * irho;
}

template <typename T>
__device__ inline T viscosity(const T& temp, const Phys& ph) {
  if (ph.mu_law == 0) return T(ph.mu);
  double s = 110.0 / ph.T_inf_K;
  return temp * dsqrt(temp) * T(ph.mu * (1.0 + s)) / (temp + T(s));
}

// Advection flux F[i][v] of Eq. (conserved fluxes).
template <int D, typename T>
__device__ inline void euler_flux(const T* U, const Phys& ph, T F[D][D + 2]) {
  T irho, vel[D], p, temp;
  primitives<D>(U, ph, irho, vel, p, temp);
  T Ep = U[D + 1] + p;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    F[i][0] = U[1 + i];
#pragma unroll
    for (int k = 0; k < D; ++k) F[i][1 + k] = U[1 + i] * vel[k];
    F[i][1 + i] += p;
    F[i][D + 1] = vel[i] * Ep;
  }
}

// Diffusion flux G[i][v] of Eq. (conserved fluxes) from the physical gradient
// dU[j][v] of the conservative variables (linear in dU at fixed U).  mu_add:
// artificial viscosity added to mu (and, through kappa_fac, its conductivity
// mu_add C_p / Pr); a constant here, so a dual-number U does not carry its
// derivative.
template <int D, typename T, typename TG>
__device__ inline void viscous_flux(const T* U, const TG dU[D][D + 2], const Phys& ph,
                                    T G[D][D + 2], double mu_add = 0.0) {
  T irho, vel[D], p, temp;
  primitives<D>(U, ph, irho, vel, p, temp);
  T mu = viscosity(temp, ph);
  if (mu_add != 0.0) mu += T(mu_add);
  T e = U[D + 1] * irho;
  T dvel[D][D], dT[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T de = (T(dU[j][D + 1]) - e * T(dU[j][0])) * irho;
    T s = de;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      dvel[j][k] = (T(dU[j][1 + k]) - vel[k] * T(dU[j][0])) * irho;
      s -= dvel[j][k] * vel[k];
    }
    dT[j] = T(ph.gMa2 * ph.gm1) * s;
  }
  T div = T(0.0);
#pragma unroll
  for (int k = 0; k < D; ++k) div += dvel[k][k];
  T kap = mu * T(ph.kappa_fac);
  T twothird = T(2.0 / 3.0) * mu * div;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    G[i][0] = T(0.0);
    T en = kap * dT[i];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      T tau = mu * (dvel[k][i] + dvel[i][k]);
      if (i == k) tau -= twothird;
      G[i][1 + k] = tau;
      en += vel[k] * tau;
    }
    G[i][D + 1] = en;
  }
}

// ------------------------------------------------------------ shock capturing
// Ducros' sensor (div u)^2 / ((div u)^2 + |curl u|^2 + eps) from the velocity
// gradient dv[j][k] = d u_k / d x_j (Sec. 3.1.2 lists it beside the modal
// sensor; with av = 2 it multiplies the artificial viscosity at each point)
constexpr double DUCROS_EPS = 1e-6;  // squared velocity-gradient floor (1e-3)
template <int D>
__device__ inline double ducros_ratio(const double dv[D][D]) {
  double div = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) div += dv[k][k];
  double c2;
  if constexpr (D == 2) {
    const double w = dv[0][1] - dv[1][0];
    c2 = w * w;
  } else {
    const double wx = dv[1][D - 1] - dv[D - 1][1], wy = dv[D - 1][0] - dv[0][D - 1];
    const double wz = dv[0][1] - dv[1][0];
    c2 = wx * wx + wy * wy + wz * wz;
  }
  return div * div / (div * div + c2 + DUCROS_EPS);
}

// the same from a state U and the gradient dU[j][v] of the conservative variables
template <int D>
__device__ inline double ducros(const double* U, const double dU[D][D + 2]) {
  const double irho = 1.0 / U[0];
  double dv[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) dv[j][k] = (dU[j][1 + k] - U[1 + k] * irho * dU[j][0]) * irho;
  return ducros_ratio<D>(dv);
}

// Artificial viscosity at a point (Sec. 3.1.2): mu_av = f_e rho (c + |u|),
// f_e = mu_0 S_e h_e / P the element factor of the modal sensor.
template <int D>
__device__ inline double av_point(const double* U, const Phys& ph, double fe) {
  if (fe == 0.0) return 0.0;
  const double irho = 1.0 / U[0];
  double ke = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) ke = fma(U[1 + k], U[1 + k], ke);
  ke *= irho;  // rho |u|^2
  const double p = ph.gm1 * (U[D + 1] - 0.5 * ke);
  return fe * U[0] * (sqrt(ph.gamma * p * irho) + sqrt(ke * irho));
}

// Artificial viscosity on a face point: the mean of the two sides' values,
// each from its own trace and element factor; the interior side's alone on a
// boundary face (eR < 0); dQa is the face-average gradient (av = 2).
template <int D>
__device__ inline double av_face(const Phys& ph, int eL, int eR, const double* QL,
                                 const double* QR, const double dQa[D][D + 2]) {
  if (!ph.avf) return 0.0;
  double a = av_point<D>(QL, ph, ph.avf[eL]);
  if (eR >= 0) a = 0.5 * (a + av_point<D>(QR, ph, ph.avf[eR]));
  if (ph.av_mode == 2 && a != 0.0) {
    // Ducros' sensor of the face-average gradient at the mean trace state
    // (a boundary face: the interior trace)
    double Qm[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Qm[v] = eR >= 0 ? 0.5 * (QL[v] + QR[v]) : QL[v];
    a *= ducros<D>(Qm, dQa);
  }
  return a;
}

// Normal Euler flux F(U).n
template <int D>
__device__ inline void euler_flux_n(const double* U, const double* n, const Phys& ph,
                                    double* Fn, double& p_out, double* vel_out) {
  double irho, vel[D], p, temp;
  primitives<D>(U, ph, irho, vel, p, temp);
  double un = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) un += vel[k] * n[k];
  Fn[0] = U[0] * un;
#pragma unroll
  for (int k = 0; k < D; ++k) Fn[1 + k] = U[1 + k] * un + p * n[k];
  Fn[D + 1] = (U[D + 1] + p) * un;
  p_out = p;
#pragma unroll
  for (int k = 0; k < D; ++k) vel_out[k] = vel[k];
}

// Roe's approximate Riemann flux without entropy fix (Toro, Ch. 11).
template <int D>
__device__ inline void roe_flux(const double* UL, const double* UR, const double* n,
                                const Phys& ph, double* Fh) {
  double FL[D + 2], FR[D + 2], vL[D], vR[D], pL, pR;
  euler_flux_n<D>(UL, n, ph, FL, pL, vL);
  euler_flux_n<D>(UR, n, ph, FR, pR, vR);
  double rL = UL[0], rR = UR[0];
  double HL = (UL[D + 1] + pL) / rL, HR = (UR[D + 1] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double rt = sL * sR;
  double isum = 1.0 / (sL + sR);
  double ut[D], du[D], q2 = 0, unt = 0, dun = 0, udu = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ut[k] = (sL * vL[k] + sR * vR[k]) * isum;
    du[k] = vR[k] - vL[k];
    q2 += ut[k] * ut[k];
    unt += ut[k] * n[k];
    dun += du[k] * n[k];
    udu += ut[k] * du[k];
  }
  double Ht = (sL * HL + sR * HR) * isum;
  double c2 = ph.gm1 * (Ht - 0.5 * q2);
  double c = sqrt(c2);
  double ic2 = 1.0 / c2;
  double dr = rR - rL, dp = pR - pL;
  double a1 = (dp - rt * c * dun) * 0.5 * ic2;
  double a5 = (dp + rt * c * dun) * 0.5 * ic2;
  double a2 = dr - dp * ic2;
  double l1 = fabs(unt - c), l2 = fabs(unt), l5 = fabs(unt + c);
  double w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2, ws = l2 * rt;
  Fh[0] = 0.5 * (FL[0] + FR[0]) - 0.5 * (w1 + w2 + w5);
#pragma unroll
  for (int k = 0; k < D; ++k)
    Fh[1 + k] = 0.5 * (FL[1 + k] + FR[1 + k]) -
                0.5 * (w1 * (ut[k] - c * n[k]) + w5 * (ut[k] + c * n[k]) + w2 * ut[k] +
                       ws * (du[k] - dun * n[k]));
  Fh[D + 1] = 0.5 * (FL[D + 1] + FR[D + 1]) -
              0.5 * (w1 * (Ht - unt * c) + w5 * (Ht + unt * c) + w2 * 0.5 * q2 +
                     ws * (udu - unt * dun));
}

// HLLC flux (Toro, Ch. 10) with Einfeldt (Roe-averaged) wave speeds.
template <int D>
__device__ inline void hllc_flux(const double* UL, const double* UR, const double* n,
                                 const Phys& ph, double* Fh) {
  double FL[D + 2], FR[D + 2], vL[D], vR[D], pL, pR;
  euler_flux_n<D>(UL, n, ph, FL, pL, vL);
  euler_flux_n<D>(UR, n, ph, FR, pR, vR);
  double rL = UL[0], rR = UR[0];
  double cL = sqrt(ph.gamma * pL / rL), cR = sqrt(ph.gamma * pR / rR);
  double HL = (UL[D + 1] + pL) / rL, HR = (UR[D + 1] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double isum = 1.0 / (sL + sR);
  double q2 = 0, unt = 0, unL = 0, unR = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double u = (sL * vL[k] + sR * vR[k]) * isum;
    q2 += u * u;
    unt += u * n[k];
    unL += vL[k] * n[k];
    unR += vR[k] * n[k];
  }
  double Ht = (sL * HL + sR * HR) * isum;
  double ct = sqrt(ph.gm1 * (Ht - 0.5 * q2));
  double SL = fmin(unL - cL, unt - ct);
  double SR = fmax(unR + cR, unt + ct);
  double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) /
              (rL * (SL - unL) - rR * (SR - unR));
  if (SL >= 0.0) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = FL[v];
  } else if (Ss < 0.0 && SR <= 0.0) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = FR[v];
  } else {
    const bool left = Ss >= 0.0;
    const double* U = left ? UL : UR;
    const double* F = left ? FL : FR;
    const double* vv = left ? vL : vR;
    double r = left ? rL : rR, p = left ? pL : pR, un = left ? unL : unR, S = left ? SL : SR;
    double f = r * (S - un) / (S - Ss);
    double st[D + 2];
    st[0] = f;
#pragma unroll
    for (int k = 0; k < D; ++k) st[1 + k] = f * (vv[k] + (Ss - un) * n[k]);
    st[D + 1] = f * (U[D + 1] / r + (Ss - un) * (Ss + p / (r * (S - un))));
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = F[v] + S * (st[v] - U[v]);
  }
}

// HLL flux (one intermediate state between the fastest waves; Toro, Ch. 10)
// with the same Einfeldt speed estimates as hllc_flux.
template <int D>
__device__ inline void hll_flux(const double* UL, const double* UR, const double* n,
                                const Phys& ph, double* Fh) {
  double FL[D + 2], FR[D + 2], vL[D], vR[D], pL, pR;
  euler_flux_n<D>(UL, n, ph, FL, pL, vL);
  euler_flux_n<D>(UR, n, ph, FR, pR, vR);
  double rL = UL[0], rR = UR[0];
  double cL = sqrt(ph.gamma * pL / rL), cR = sqrt(ph.gamma * pR / rR);
  double HL = (UL[D + 1] + pL) / rL, HR = (UR[D + 1] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double isum = 1.0 / (sL + sR);
  double q2 = 0, unt = 0, unL = 0, unR = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double u = (sL * vL[k] + sR * vR[k]) * isum;
    q2 += u * u;
    unt += u * n[k];
    unL += vL[k] * n[k];
    unR += vR[k] * n[k];
  }
  double Ht = (sL * HL + sR * HR) * isum;
  double ct = sqrt(ph.gm1 * (Ht - 0.5 * q2));
  double SL = fmin(unL - cL, unt - ct);
  double SR = fmax(unR + cR, unt + ct);
  if (SL >= 0.0) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = FL[v];
  } else if (SR <= 0.0) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = FR[v];
  } else {
    const double idS = 1.0 / (SR - SL);
#pragma unroll
    for (int v = 0; v < D + 2; ++v) Fh[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * idS;
  }
}

// Local Lax-Friedrichs (Rusanov): mean normal flux minus the jump times half
// the larger spectral radius |u_n| + c of the two sides.
template <int D>
__device__ inline void lf_flux(const double* UL, const double* UR, const double* n,
                               const Phys& ph, double* Fh) {
  double FL[D + 2], FR[D + 2], vL[D], vR[D], pL, pR;
  euler_flux_n<D>(UL, n, ph, FL, pL, vL);
  euler_flux_n<D>(UR, n, ph, FR, pR, vR);
  double unL = 0, unR = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    unL += vL[k] * n[k];
    unR += vR[k] * n[k];
  }
  const double lam = fmax(fabs(unL) + sqrt(ph.gamma * pL / UL[0]),
                          fabs(unR) + sqrt(ph.gamma * pR / UR[0]));
#pragma unroll
  for (int v = 0; v < D + 2; ++v) Fh[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
}

// AUSM (Liou and Steffen 1993): interface Mach number from the van Leer
// splittings M+(M_L) + M-(M_R) carries the upwinded c (rho, rho u, rho H); the
// pressure splittings p+(M_L) p_L + p-(M_R) p_R act on the momentum.
template <int D>
__device__ inline void ausm_flux(const double* UL, const double* UR, const double* n,
                                 const Phys& ph, double* Fh) {
  double irL, vL[D], pL, TL, irR, vR[D], pR, TR;
  primitives<D>(UL, ph, irL, vL, pL, TL);
  primitives<D>(UR, ph, irR, vR, pR, TR);
  const double cL = sqrt(ph.gamma * pL * irL), cR = sqrt(ph.gamma * pR * irR);
  double unL = 0, unR = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    unL += vL[k] * n[k];
    unR += vR[k] * n[k];
  }
  const double ML = unL / cL, MR = unR / cR;
  double Mp, Mm, Pp, Pm;
  if (fabs(ML) <= 1.0) {
    Mp = 0.25 * (ML + 1.0) * (ML + 1.0);
    Pp = Mp * (2.0 - ML);
  } else {
    Mp = 0.5 * (ML + fabs(ML));
    Pp = ML > 0.0 ? 1.0 : 0.0;
  }
  if (fabs(MR) <= 1.0) {
    Mm = -0.25 * (MR - 1.0) * (MR - 1.0);
    Pm = -Mm * (2.0 + MR);
  } else {
    Mm = 0.5 * (MR - fabs(MR));
    Pm = MR < 0.0 ? 1.0 : 0.0;
  }
  const double mh = Mp + Mm, ph2 = Pp * pL + Pm * pR;
  const double a = 0.5 * (mh + fabs(mh)), b = 0.5 * (mh - fabs(mh));  // upwind weights
  // c (rho, rho u, rho H) of each side
  Fh[0] = a * cL * UL[0] + b * cR * UR[0];
#pragma unroll
  for (int k = 0; k < D; ++k) Fh[1 + k] = a * cL * UL[1 + k] + b * cR * UR[1 + k] + ph2 * n[k];
  Fh[D + 1] = a * cL * (UL[D + 1] + pL) + b * cR * (UR[D + 1] + pR);
}

template <int D>
__device__ inline void riemann_flux(const double* UL, const double* UR, const double* n,
                                    const Phys& ph, double* Fh) {
  switch (ph.riemann) {
    case DG_RIEMANN_HLLC: hllc_flux<D>(UL, UR, n, ph, Fh); break;
    case DG_RIEMANN_HLL: hll_flux<D>(UL, UR, n, ph, Fh); break;
    case DG_RIEMANN_LF: lf_flux<D>(UL, UR, n, ph, Fh); break;
    case DG_RIEMANN_AUSM: ausm_flux<D>(UL, UR, n, ph, Fh); break;
    default: roe_flux<D>(UL, UR, n, ph, Fh);
  }
}

// ------------------------------------------------------------ analytic fields
__device__ inline void conservative_from(int D, double rho, const double* vel, double temp,
                                         const Phys& ph, double* U) {
  double p = rho * temp / ph.gMa2;
  double ke = 0;
  U[0] = rho;
  for (int k = 0; k < D; ++k) {
    U[1 + k] = rho * vel[k];
    ke += vel[k] * vel[k];
  }
  U[D + 1] = p / ph.gm1 + 0.5 * rho * ke;
}

// State of the workload's analytic field at x (Sec. 6.1 vortex with the
// sign of the u perturbation that makes it a vortex; manufactured
// Poiseuille; Taylor-Green vortex; uniform stream).
__device__ inline void exact_state(int D, const Phys& ph, const double* x, double t, double* U) {
  double rho = 1.0, temp = 1.0, vel[3] = {0.0, 0.0, 0.0};
  const double PI = 3.14159265358979323846;
  if (ph.field == DG_FIELD_VORTEX) {
    double u0 = ph.fpar[0], v0 = ph.fpar[1], phi = ph.fpar[2], xc = ph.fpar[3], yc = ph.fpar[4],
           s = ph.fpar[5];
    double dx = x[0] - (xc + u0 * t), dy = x[1] - (yc + v0 * t);
    dx -= rint(dx);
    dy -= rint(dy);
    double X = s * dx, Y = s * dy;
    double ex = exp(1.0 - X * X - Y * Y);
    vel[0] = u0 - phi / (2 * PI) * Y * ex;
    vel[1] = v0 + phi / (2 * PI) * X * ex;
    temp = 1.0 - ph.gm1 * ph.Ma * ph.Ma * phi * phi / (16 * PI * PI) * ex * ex;
    rho = pow(temp, 1.0 / ph.gm1);
  } else if (ph.field == DG_FIELD_POISEUILLE) {
    double theta = ph.fpar[0], L = ph.fpar[1], dpdx = ph.fpar[2];
    double y = x[1];
    vel[0] = -dpdx / (2 * ph.mu) * (y * (L - y) + theta * y * y * (L - y) * (L - y));
    double p = 1.0 / ph.gMa2 + dpdx * x[0];
    rho = 1.0;
    temp = ph.gMa2 * p / rho;
  } else if (ph.field == DG_FIELD_TGV) {
    double X = x[0], Y = x[1], Z = x[2];
    vel[0] = sin(X) * cos(Y) * cos(Z);
    vel[1] = -cos(X) * sin(Y) * cos(Z);
    double pinf = 1.0 / ph.gMa2;
    double p = pinf + (cos(2 * X) + cos(2 * Y)) * (cos(2 * Z) + 2.0) / 16.0;
    rho = p / pinf;
    temp = 1.0;
  } else if (ph.field == DG_FIELD_UNIFORM && ph.fpar[0] > 0.0) {  // (rho, u, v, w, T)
    rho = ph.fpar[0];
    for (int k = 0; k < D; ++k) vel[k] = ph.fpar[1 + k];
    temp = ph.fpar[4];
  } else if (ph.field == DG_FIELD_SHOCK) {
    // oblique shock at beta = fpar[0] degrees to the x axis, meeting y = 0 at
    // x = fpar[1]: the stream (1, 0) below the line, above it the state the
    // Rankine-Hugoniot jump conditions give for the normal Mach number
    // Ma sin(beta) (tangential velocity unchanged)
    // fpar[2] > 0: a smooth passage between the two states over the width
    // fpar[2] (fraction (1 + tanh(s / w)) / 2 of the signed distance s to the
    // line, on the primitive variables); fpar[3] > 0: the velocity brought to
    // rest at y = 0 by 1 - exp(-y / fpar[3])
    const double beta = ph.fpar[0] * (PI / 180.0);
    const double sb = sin(beta), cb = cos(beta);
    double post;
    if (ph.fpar[2] > 0.0)
      post = 0.5 * (1.0 + tanh((x[1] * cb - (ph.fpar[1] - x[0]) * sb) / ph.fpar[2]));
    else
      post = x[1] > (ph.fpar[1] - x[0]) * (sb / cb) ? 1.0 : 0.0;
    const double mn2 = ph.Ma * ph.Ma * sb * sb;
    const double rr = (ph.gamma + 1.0) * mn2 / (ph.gm1 * mn2 + 2.0);   // rho2 / rho1
    const double pr = 1.0 + 2.0 * ph.gamma / (ph.gamma + 1.0) * (mn2 - 1.0);  // p2 / p1
    const double un = sb / rr, ut = cb;  // normal and tangential speeds behind
    rho = 1.0 + post * (rr - 1.0);
    vel[0] = 1.0 + post * (un * sb + ut * cb - 1.0);
    vel[1] = post * (un * cb - ut * sb);
    if (ph.fpar[3] > 0.0) {
      const double f = 1.0 - exp(-x[1] / ph.fpar[3]);
      vel[0] *= f;
      vel[1] *= f;
    }
    temp = (1.0 + post * (pr - 1.0)) / rho;  // gamma Ma^2 p / rho with p1 = 1/(gamma Ma^2)
  } else if (ph.field == DG_FIELD_CYLINDER && ph.fpar[1] > 0.0) {
    // stream brought to rest at the wall r = fpar[0] over the length fpar[1]
    const double r = sqrt(x[0] * x[0] + x[1] * x[1]);
    vel[0] = 1.0 - exp(-fmax(r - ph.fpar[0], 0.0) / ph.fpar[1]);
  } else {  // uniform / cylinder free stream
    vel[0] = 1.0;
  }
  conservative_from(D, rho, vel, temp, ph, U);
}

// Manufactured source of the compressible Poiseuille case (App. B) with the
// energy component built on h(y) = y(L-y) + theta y^2 (L-y)^2.
__device__ inline void forcing(int D, const Phys& ph, const double* x, double* f) {
  for (int v = 0; v < D + 2; ++v) f[v] = 0.0;
  if (ph.forcing != DG_FORCING_POISEUILLE) return;
  double theta = ph.fpar[0], L = ph.fpar[1], dpdx = ph.fpar[2], mu = ph.mu;
  double y = x[1];
  double c = L * L - 6 * y * L + 6 * y * y;
  double h = y * (L - y) + theta * y * y * (L - y) * (L - y);
  double q = 2 * theta * y * L - 2 * theta * y * y + 1;
  f[1] = dpdx * theta * c;
  f[D + 1] = dpdx * dpdx / (2 * mu) * h * (1 - theta * c - ph.gamma / ph.gm1) -
             dpdx * dpdx / (4 * mu) * (L - 2 * y) * (L - 2 * y) * q * q;
}

__device__ inline double wall_temperature(const Phys& ph, const double* x) {
  if (ph.field == DG_FIELD_POISEUILLE) return 1.0 + ph.gMa2 * ph.fpar[2] * x[0];
  return 1.0;
}

// Characteristic far-field state from the interior state UL and the free
// stream Ui along the outward unit normal n: outgoing invariant
// u_n + 2c/(gamma-1) from UL, incoming u_n - 2c/(gamma-1) from Ui, entropy and
// tangential velocity from the upwind side; supersonic normal flow takes the
// upwind state whole.
template <int D>
__device__ inline void farfield_state(const Phys& ph, const double* UL, const double* Ui,
                                      const double* n, double* UB) {
  double irL, vL[D], pL, TL, iri, vi[D], pi, Ti;
  primitives<D>(UL, ph, irL, vL, pL, TL);
  primitives<D>(Ui, ph, iri, vi, pi, Ti);
  const double g = ph.gamma;
  const double cL = sqrt(g * pL * irL), ci = sqrt(g * pi * iri);
  double un = 0.0, uni = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    un += vL[k] * n[k];
    uni += vi[k] * n[k];
  }
  if (un >= cL) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) UB[v] = UL[v];
    return;
  }
  if (un <= -cL) {
#pragma unroll
    for (int v = 0; v < D + 2; ++v) UB[v] = Ui[v];
    return;
  }
  const double Rp = un + 2.0 * cL / ph.gm1, Rm = uni - 2.0 * ci / ph.gm1;
  const double unb = 0.5 * (Rp + Rm), cb = 0.25 * ph.gm1 * (Rp - Rm);
  const bool out = unb > 0.0;
  const double sup = out ? pL / pow(UL[0], g) : pi / pow(Ui[0], g);
  const double* vu = out ? vL : vi;
  double vun = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) vun += vu[k] * n[k];
  const double rb = pow(cb * cb / (g * sup), 1.0 / ph.gm1);
  const double pb = rb * cb * cb / g;
  double ke = 0.0;
  UB[0] = rb;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double vb = vu[k] - vun * n[k] + unb * n[k];
    UB[1 + k] = rb * vb;
    ke += vb * vb;
  }
  UB[D + 1] = pb / ph.gm1 + 0.5 * rb * ke;
}

// Weakly imposed boundary data (the boundary types of dg.h): QR the exterior
// state of the Riemann flux, QB the state of the viscous flux and of the
// penalty jump Q_L - Q_B.  Returns true on an adiabatic wall, where the
// energy components of G^n and S_j vanish.
template <int D>
__device__ inline bool boundary_states(int bctype, const Phys& ph, const double* x, double t,
                                       const double* UL, const double* n, double* QR,
                                       double* QB) {
  constexpr int NV = D + 2;
  if (bctype == DG_BC_ISO_WALL) {
    const double Tw = wall_temperature(ph, x);
    QB[0] = UL[0];
#pragma unroll
    for (int k = 0; k < D; ++k) QB[1 + k] = 0.0;
    QB[D + 1] = UL[0] * Tw / (ph.gamma * ph.gm1 * ph.Ma * ph.Ma);
  } else if (bctype == DG_BC_ADIA_WALL) {
    double ir, vel[D], p, T;
    primitives<D>(UL, ph, ir, vel, p, T);
    double mn = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) mn += UL[1 + k] * n[k];
    QR[0] = UL[0];
#pragma unroll
    for (int k = 0; k < D; ++k) QR[1 + k] = UL[1 + k] - 2.0 * mn * n[k];
    QR[D + 1] = UL[D + 1];
    QB[0] = UL[0];
#pragma unroll
    for (int k = 0; k < D; ++k) QB[1 + k] = 0.0;
    QB[D + 1] = p / ph.gm1;
    return true;
  } else if (bctype == DG_BC_FARFIELD) {
    double Ui[NV];
    exact_state(D, ph, x, t, Ui);
    farfield_state<D>(ph, UL, Ui, n, QB);
  } else {  // DG_BC_DIRICHLET
    exact_state(D, ph, x, t, QB);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) QR[v] = QB[v];
  return false;
}

// Numerical normal flux H^n = F^n - G^n on a face with owner-side unit
// normal n (Sec. 3.1, with the adjoint-consistent interior penalty):
//   S_i  = G_i({Q}, n (x) [Q]),  [Q] = Q_L - Q_R  (Q_L - Q_B on a boundary),
//   G^n  = n . (G({Q}, {grad Q}) - beta_p S),
// where on a boundary face the Riemann flux takes the exterior state Q_R and
// {Q} = Q_B (boundary_states) with the interior gradient.  dQa is the
// face-average gradient.
template <int D>
__device__ inline void numerical_flux_n(const double* QL, const double* QRin, int bctype,
                                        const double* x, double t, const double dQa[D][D + 2],
                                        const double* n, double beta, const Phys& ph,
                                        double* Hn, double S[D][D + 2], double mu_add = 0.0) {
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
      QR[v] = QRin[v];
      Qa[v] = 0.5 * (QL[v] + QR[v]);
      jump[v] = QL[v] - QR[v];
    }
  }
  riemann_flux<D>(QL, QR, n, ph, Hn);
  if (ph.viscous) {
    double gS[D][NV];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) gS[j][v] = n[j] * jump[v];
    viscous_flux<D>(Qa, gS, ph, S, mu_add);
    double Gv[D][NV];
    viscous_flux<D>(Qa, dQa, ph, Gv, mu_add);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (adiabatic && v == NV - 1) continue;
      double gn = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) gn += n[j] * (Gv[j][v] - beta * S[j][v]);
      Hn[v] -= gn;
    }
    if (adiabatic)
#pragma unroll
      for (int j = 0; j < D; ++j) S[j][NV - 1] = 0.0;
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) S[j][v] = 0.0;
  }
}

// the same for the axis normal n = sgn e_r
template <int D>
__device__ inline void numerical_flux(const double* QL, const double* QRin, int bctype,
                                      const double* x, double t, const double dQa[D][D + 2],
                                      int r, double sgn, double beta, const Phys& ph,
                                      double* Hn, double S[D][D + 2], double mu_add = 0.0) {
  double n[D];
#pragma unroll
  for (int k = 0; k < D; ++k) n[k] = k == r ? sgn : 0.0;
  numerical_flux_n<D>(QL, QRin, bctype, x, t, dQa, n, beta, ph, Hn, S, mu_add);
}

// ------------------------------------------------------------ fused / axis-specialised forms
// The same fluxes with the work that is identically zero removed: one
// evaluation of the primitive variables shared by F and G, and, on a face with
// normal n = sgn e_R (R known at compile time), only row R of G for the
// average gradient and the rank-1 gradient n (x) [Q] for S.  Equal to the
// generic forms above up to rounding order.

// H = F - G at a volume point with shared primitive variables
template <int D>
__device__ inline void ns_volume_flux(const double* U, const double dU[D][D + 2], const Phys& ph,
                                      double H[D][D + 2], double fe = 0.0) {
  constexpr int NV = D + 2;
  const double irho = 1.0 / U[0];
  double vel[D], ke = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vel[k] = U[1 + k] * irho;
    ke = fma(U[1 + k], vel[k], ke);
  }
  const double p = ph.gm1 * (U[D + 1] - 0.5 * ke);
  const double Ep = U[D + 1] + p;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    H[i][0] = U[1 + i];
#pragma unroll
    for (int k = 0; k < D; ++k) H[i][1 + k] = U[1 + i] * vel[k];
    H[i][1 + i] += p;
    H[i][D + 1] = vel[i] * Ep;
  }
  if (!ph.viscous) return;
  const double temp = ph.gMa2 * p * irho;
  double mu = viscosity(temp, ph);
  const double e = U[D + 1] * irho;
  double dvel[D][D], dT[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = (dU[j][D + 1] - e * dU[j][0]) * irho;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      dvel[j][k] = (dU[j][1 + k] - vel[k] * dU[j][0]) * irho;
      s = fma(-dvel[j][k], vel[k], s);
    }
    dT[j] = ph.gMa2 * ph.gm1 * s;
  }
  double div = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) div += dvel[k][k];
  if (fe != 0.0) {
    double a = fe * U[0] * (sqrt(ph.gamma * p * irho) + sqrt(ke * irho));
    if (ph.av_mode == 2) a *= ducros_ratio<D>(dvel);
    mu += a;
  }
  const double kap = mu * ph.kappa_fac;
  const double tt = (2.0 / 3.0) * mu * div;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double en = kap * dT[i];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double tau = mu * (dvel[k][i] + dvel[i][k]);
      if (i == k) tau -= tt;
      H[i][1 + k] -= tau;
      en = fma(vel[k], tau, en);
    }
    H[i][D + 1] -= en;
  }
}

// Roe flux for n = sgn e_R
template <int D, int R>
__device__ inline void roe_flux_axis(const double* UL, const double* UR, double sgn,
                                     const Phys& ph, double* Fh) {
  constexpr int NV = D + 2;
  // 1/rho and sqrt(rho) of both sides from one reciprocal square root each
  const double rsL = rsqrt(UL[0]), rsR = rsqrt(UR[0]);
  const double iL = rsL * rsL, iR = rsR * rsR;
  double vL[D], vR[D], keL = 0.0, keR = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vL[k] = UL[1 + k] * iL;
    vR[k] = UR[1 + k] * iR;
    keL = fma(UL[1 + k], vL[k], keL);
    keR = fma(UR[1 + k], vR[k], keR);
  }
  const double pL = ph.gm1 * (UL[D + 1] - 0.5 * keL), pR = ph.gm1 * (UR[D + 1] - 0.5 * keR);
  const double unL = sgn * vL[R], unR = sgn * vR[R];
  double FL[NV], FR[NV];
  FL[0] = UL[0] * unL;
  FR[0] = UR[0] * unR;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    FL[1 + k] = UL[1 + k] * unL;
    FR[1 + k] = UR[1 + k] * unR;
  }
  FL[1 + R] += sgn * pL;
  FR[1 + R] += sgn * pR;
  FL[D + 1] = (UL[D + 1] + pL) * unL;
  FR[D + 1] = (UR[D + 1] + pR) * unR;
  const double HL = (UL[D + 1] + pL) * iL, HR = (UR[D + 1] + pR) * iR;
  const double sL = UL[0] * rsL, sR = UR[0] * rsR;
  const double rt = sL * sR;
  const double isum = 1.0 / (sL + sR);
  double ut[D], du[D], q2 = 0.0, udu = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ut[k] = (sL * vL[k] + sR * vR[k]) * isum;
    du[k] = vR[k] - vL[k];
    q2 = fma(ut[k], ut[k], q2);
    if (k != R) udu = fma(ut[k], du[k], udu);
  }
  const double unt = sgn * ut[R], dun = sgn * du[R];
  const double Ht = (sL * HL + sR * HR) * isum;
  const double c2 = ph.gm1 * (Ht - 0.5 * q2);
  const double rc = rsqrt(c2);
  const double c = c2 * rc, ic2 = rc * rc;
  const double dp = pR - pL;
  const double a1 = (dp - rt * c * dun) * 0.5 * ic2;
  const double a5 = (dp + rt * c * dun) * 0.5 * ic2;
  const double a2 = (UR[0] - UL[0]) - dp * ic2;
  const double l2 = fabs(unt);
  const double w1 = fabs(unt - c) * a1, w5 = fabs(unt + c) * a5, w2 = l2 * a2, ws = l2 * rt;
  Fh[0] = 0.5 * (FL[0] + FR[0] - (w1 + w2 + w5));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double d = (w1 + w5 + w2) * ut[k];
    if (k == R)
      d += (w5 - w1) * c * sgn;
    else
      d += ws * du[k];
    Fh[1 + k] = 0.5 * (FL[1 + k] + FR[1 + k] - d);
  }
  Fh[D + 1] = 0.5 * (FL[D + 1] + FR[D + 1] -
                     ((w1 + w5) * Ht + (w5 - w1) * unt * c + w2 * 0.5 * q2 + ws * udu));
}

// primitive data shared by the viscous fluxes of one state
template <int D>
struct ViscPrim {
  double irho, vel[D], e, mu, kap;
};
template <int D>
__device__ inline void visc_prim(const double* U, const Phys& ph, ViscPrim<D>& s,
                                 double mu_add = 0.0) {
  s.irho = 1.0 / U[0];
  double ke = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s.vel[k] = U[1 + k] * s.irho;
    ke = fma(U[1 + k], s.vel[k], ke);
  }
  const double p = ph.gm1 * (U[D + 1] - 0.5 * ke);
  s.e = U[D + 1] * s.irho;
  s.mu = viscosity(ph.gMa2 * p * s.irho, ph);
  if (mu_add != 0.0) s.mu += mu_add;
  s.kap = s.mu * ph.kappa_fac;
}

// row R of G(U, dU)
template <int D, int R>
__device__ inline void viscous_row(const ViscPrim<D>& s, const double dU[D][D + 2],
                                   const Phys& ph, double* G) {
  double dv[D][D];  // dv[j][k] = d u_k / d x_j, only the entries row R needs
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (j == R || k == R || j == k) dv[j][k] = (dU[j][1 + k] - s.vel[k] * dU[j][0]) * s.irho;
  double div = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) div += dv[k][k];
  double st = (dU[R][D + 1] - s.e * dU[R][0]) * s.irho;
#pragma unroll
  for (int k = 0; k < D; ++k) st = fma(-dv[R][k], s.vel[k], st);
  double en = s.kap * (ph.gMa2 * ph.gm1 * st);
  G[0] = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double tau = s.mu * (dv[k][R] + dv[R][k]);
    if (k == R) tau -= (2.0 / 3.0) * s.mu * div;
    G[1 + k] = tau;
    en = fma(s.vel[k], tau, en);
  }
  G[D + 1] = en;
}

// G(U, g) for a gradient whose only non-zero row is R (= g)
template <int D, int R>
__device__ inline void viscous_rank1(const ViscPrim<D>& s, const double* g, const Phys& ph,
                                     double S[D][D + 2]) {
  double a[D];  // d u_k / d x_R
#pragma unroll
  for (int k = 0; k < D; ++k) a[k] = (g[1 + k] - s.vel[k] * g[0]) * s.irho;
  double st = (g[D + 1] - s.e * g[0]) * s.irho;
#pragma unroll
  for (int k = 0; k < D; ++k) st = fma(-a[k], s.vel[k], st);
  const double dTR = ph.gMa2 * ph.gm1 * st;
  const double tt = (2.0 / 3.0) * s.mu * a[R];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    S[i][0] = 0.0;
    if (i == R) {
      double en = s.kap * dTR;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double tau = k == R ? 2.0 * s.mu * a[R] - tt : s.mu * a[k];
        S[i][1 + k] = tau;
        en = fma(s.vel[k], tau, en);
      }
      S[i][D + 1] = en;
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) S[i][1 + k] = k == R ? s.mu * a[i] : (k == i ? -tt : 0.0);
      S[i][D + 1] = s.vel[R] * s.mu * a[i] - s.vel[i] * tt;
    }
  }
}

// numerical_flux for the normal sgn e_R
template <int D, int R>
__device__ inline void numerical_flux_axis(const double* QL, const double* QRin, int bctype,
                                           const double* x, double t,
                                           const double dQa[D][D + 2], double sgn, double beta,
                                           const Phys& ph, double* Hn, double S[D][D + 2],
                                           double mu_add = 0.0) {
  constexpr int NV = D + 2;
  double QR[NV], Qa[NV], Qj[NV];
  bool adiabatic = false;
  if (bctype > 0) {
    double n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = k == R ? sgn : 0.0;
    adiabatic = boundary_states<D>(bctype, ph, x, t, QL, n, QR, Qa);
#pragma unroll
    for (int v = 0; v < NV; ++v) Qj[v] = Qa[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      QR[v] = QRin[v];
      Qa[v] = 0.5 * (QL[v] + QR[v]);
      Qj[v] = QR[v];
    }
  }
  if (ph.riemann != DG_RIEMANN_ROE) {
    double n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = k == R ? sgn : 0.0;
    riemann_flux<D>(QL, QR, n, ph, Hn);
  } else {
    roe_flux_axis<D, R>(QL, QR, sgn, ph, Hn);
  }
  if (ph.viscous) {
    ViscPrim<D> pa;
    visc_prim<D>(Qa, ph, pa, mu_add);
    double g[NV], Gr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) g[v] = sgn * (QL[v] - Qj[v]);
    viscous_rank1<D, R>(pa, g, ph, S);
    viscous_row<D, R>(pa, dQa, ph, Gr);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (!(adiabatic && v == NV - 1)) Hn[v] -= sgn * (Gr[v] - beta * S[R][v]);
    if (adiabatic)
#pragma unroll
      for (int j = 0; j < D; ++j) S[j][NV - 1] = 0.0;
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) S[j][v] = 0.0;
  }
}

}  // namespace dg
