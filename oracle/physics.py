"""Governing equations (Sec. 2.1), numerical fluxes (Sec. 3.1), analytic
fields of the verification cases (Sec. 6.1, App. B) and boundary states.

State layout: U[..., v] with v = (rho, rho u_1..rho u_d, E); fluxes
F[..., i, v] with i the flux direction.  All functions are vectorised over
leading axes.  euler_flux and viscous_flux use no abs/max/sqrt of the state,
so they accept complex arrays (complex-step differentiation).
"""
import numpy as np

# identifiers shared with the workloads package (plain integers)
BC_DIRICHLET, BC_ISO_WALL, BC_ADIA_WALL, BC_FARFIELD = 1, 2, 3, 4
FIELD_UNIFORM, FIELD_VORTEX, FIELD_POISEUILLE, FIELD_TGV, FIELD_CYLINDER, FIELD_SHOCK = 0, 1, 2, 3, 4, 5
RIEMANN_ROE, RIEMANN_HLLC, RIEMANN_HLL, RIEMANN_LF, RIEMANN_AUSM = 0, 1, 2, 3, 4
FORCING_NONE, FORCING_POISEUILLE = 0, 1


def primitives(U, ph):
    """rho, velocity [..., d], pressure p = (gamma-1)(E - rho|u|^2/2) and
    temperature T = gamma Ma^2 p / rho (equation of state, Sec. 2.1)."""
    d = U.shape[-1] - 2
    rho = U[..., 0]
    vel = U[..., 1:1 + d] / rho[..., None]
    E = U[..., -1]
    p = (ph.gamma - 1.0) * (E - 0.5 * np.sum(U[..., 1:1 + d] * vel, axis=-1))
    T = ph.gamma * ph.Ma ** 2 * p / rho
    return rho, vel, p, T


def conservative(rho, vel, p, ph):
    E = p / (ph.gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return np.concatenate([rho[..., None], rho[..., None] * vel, E[..., None]], axis=-1)


def euler_flux(U, ph):
    """Advection flux F_i = (rho u_i, rho u_i u + p e_i, u_i (E + p))."""
    d = U.shape[-1] - 2
    rho, vel, p, _ = primitives(U, ph)
    F = np.zeros(U.shape[:-1] + (d, d + 2), dtype=U.dtype)
    for i in range(d):
        F[..., i, 0] = U[..., 1 + i]
        for k in range(d):
            F[..., i, 1 + k] = U[..., 1 + i] * vel[..., k]
        F[..., i, 1 + i] += p
        F[..., i, -1] = vel[..., i] * (U[..., -1] + p)
    return F


def viscosity(T, ph):
    """Constant mu = 1/Re, or Sutherland's law with T_inf in kelvin (Sec. 2.1)."""
    if ph.mu_law == 0:
        return np.full_like(T, 1.0 / ph.Re)
    s = 110.0 / ph.T_inf_K
    return T ** 1.5 / ph.Re * (1.0 + s) / (T + s)


def artificial_viscosity(U, factor, ph):
    """mu_av = mu_0 rho (h/P) (c + |u|) S (Sec. 3.1.2) at each point, with the
    element factor mu_0 S h / P given (factor, broadcast over the points)."""
    rho, vel, p, _ = primitives(U, ph)
    c = np.sqrt(ph.gamma * p / rho)
    return factor * rho * (c + np.sqrt(np.sum(vel * vel, axis=-1)))


DUCROS_EPS = 1e-6    # squared velocity-gradient floor: below 1e-3 the flow counts as uniform


def ducros(U, dU, ph):
    """Ducros' sensor (Sec. 3.1.2 lists it beside the modal sensor):
    (div u)^2 / ((div u)^2 + |curl u|^2 + eps) at each point, from the state U
    and the gradient dU[..., j, v] of the conservative variables: 1 in a pure
    compression or expansion, 0 in a rigid rotation or a shear layer."""
    d = U.shape[-1] - 2
    rho = U[..., 0]
    vel = U[..., 1:1 + d] / rho[..., None]
    # dv[..., j, k] = d u_k / d x_j
    dv = (dU[..., 1:1 + d] - vel[..., None, :] * dU[..., :, 0:1]) / rho[..., None, None]
    div = np.einsum("...jj->...", dv)
    if d == 2:
        curl2 = (dv[..., 0, 1] - dv[..., 1, 0]) ** 2
    else:
        curl2 = ((dv[..., 1, 2] - dv[..., 2, 1]) ** 2 + (dv[..., 2, 0] - dv[..., 0, 2]) ** 2
                 + (dv[..., 0, 1] - dv[..., 1, 0]) ** 2)
    return div * div / (div * div + curl2 + DUCROS_EPS)


def viscous_flux(U, dU, ph, mu_av=None):
    """Diffusion flux G_i = (0, tau_i1..tau_id, u_j tau_ij - q_i) with the
    Stokes stress tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu div(u) delta_ij and
    Fourier heat flux q_i = -mu / (Ma^2 Pr (gamma-1)) dT/dx_i.  dU[..., j, v]
    is the gradient of the conservative variables; G is linear in dU.  mu_av
    (optional, per point): artificial viscosity added to mu; its conductivity
    mu_av C_p / Pr (Sec. 3.1.2) has the physical factor 1/(Ma^2 Pr (gamma-1))
    because C_p = 1/((gamma-1) Ma^2) in these units."""
    d = U.shape[-1] - 2
    g, Ma = ph.gamma, ph.Ma
    rho, vel, p, T = primitives(U, ph)
    mu = viscosity(T, ph)
    if mu_av is not None:
        mu = mu + mu_av
    drho = dU[..., 0]                                  # [..., j]
    dvel = (dU[..., 1:1 + d] - vel[..., None, :] * drho[..., :, None]) / rho[..., None, None]
    # dvel[..., j, k] = d u_k / d x_j
    e = U[..., -1] / rho
    de = (dU[..., -1] - e[..., None] * drho) / rho[..., None]
    dT = g * Ma ** 2 * (g - 1.0) * (de - np.einsum("...jk,...k->...j", dvel, vel))
    div = np.einsum("...jj->...", dvel)
    kappa = mu / (Ma ** 2 * ph.Pr * (g - 1.0))
    G = np.zeros(U.shape[:-1] + (d, d + 2), dtype=np.result_type(U, dU))
    for i in range(d):
        for k in range(d):
            tau = mu * (dvel[..., k, i] + dvel[..., i, k])
            if i == k:
                tau = tau - 2.0 / 3.0 * mu * div
            G[..., i, 1 + k] = tau
            G[..., i, -1] += vel[..., k] * tau
        G[..., i, -1] += kappa * dT[..., i]
    return G


def roe_flux(UL, UR, n, ph):
    """Roe's approximate Riemann flux without entropy fix (Toro, Ch. 11),
    normal n pointing from L to R."""
    g = ph.gamma
    rL, vL, pL, _ = primitives(UL, ph)
    rR, vR, pR, _ = primitives(UR, ph)
    HL = (UL[..., -1] + pL) / rL
    HR = (UR[..., -1] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    rt = sL * sR
    ut = (sL[..., None] * vL + sR[..., None] * vR) / (sL + sR)[..., None]
    Ht = (sL * HL + sR * HR) / (sL + sR)
    q2 = np.sum(ut * ut, axis=-1)
    c2 = (g - 1.0) * (Ht - 0.5 * q2)
    c = np.sqrt(c2)
    unt = np.sum(ut * n, axis=-1)
    dr, dp = rR - rL, pR - pL
    du = vR - vL
    dun = np.sum(du * n, axis=-1)
    a1 = (dp - rt * c * dun) / (2 * c2)
    a5 = (dp + rt * c * dun) / (2 * c2)
    a2 = dr - dp / c2
    l1, l2, l5 = np.abs(unt - c), np.abs(unt), np.abs(unt + c)
    one = np.ones_like(unt)

    def vec(s, m, e):
        return np.concatenate([s[..., None], m, e[..., None]], axis=-1)

    w1 = (l1 * a1)[..., None] * vec(one, ut - c[..., None] * n, Ht - unt * c)
    w5 = (l5 * a5)[..., None] * vec(one, ut + c[..., None] * n, Ht + unt * c)
    w2 = l2[..., None] * (a2[..., None] * vec(one, ut, 0.5 * q2)
                          + rt[..., None] * vec(0 * one, du - dun[..., None] * n,
                                                np.sum(ut * du, axis=-1) - unt * dun))
    FL = np.einsum("...iv,...i->...v", euler_flux(UL, ph), n)
    FR = np.einsum("...iv,...i->...v", euler_flux(UR, ph), n)
    return 0.5 * (FL + FR) - 0.5 * (w1 + w2 + w5)


def hllc_flux(UL, UR, n, ph):
    """HLLC flux (Toro, Ch. 10) with Einfeldt (Roe-averaged) wave-speed
    estimates S_L = min(u_nL - c_L, u~_n - c~), S_R = max(u_nR + c_R, u~_n + c~)."""
    g = ph.gamma
    rL, vL, pL, _ = primitives(UL, ph)
    rR, vR, pR, _ = primitives(UR, ph)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    HL = (UL[..., -1] + pL) / rL
    HR = (UR[..., -1] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    ut = (sL[..., None] * vL + sR[..., None] * vR) / (sL + sR)[..., None]
    Ht = (sL * HL + sR * HR) / (sL + sR)
    ct = np.sqrt((g - 1.0) * (Ht - 0.5 * np.sum(ut * ut, axis=-1)))
    unL, unR = np.sum(vL * n, -1), np.sum(vR * n, -1)
    unt = np.sum(ut * n, -1)
    SL = np.minimum(unL - cL, unt - ct)
    SR = np.maximum(unR + cR, unt + ct)
    Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR))
    FL = np.einsum("...iv,...i->...v", euler_flux(UL, ph), n)
    FR = np.einsum("...iv,...i->...v", euler_flux(UR, ph), n)

    def star(U, r, v, p, un, S):
        f = r * (S - un) / (S - Ss)
        m = f[..., None] * (v + (Ss - un)[..., None] * n)
        e = f * (U[..., -1] / r + (Ss - un) * (Ss + p / (r * (S - un))))
        return np.concatenate([f[..., None], m, e[..., None]], axis=-1)

    FsL = FL + SL[..., None] * (star(UL, rL, vL, pL, unL, SL) - UL)
    FsR = FR + SR[..., None] * (star(UR, rR, vR, pR, unR, SR) - UR)
    out = np.where((SL >= 0)[..., None], FL,
                   np.where((Ss >= 0)[..., None], FsL,
                            np.where((SR > 0)[..., None], FsR, FR)))
    return out


def hll_flux(UL, UR, n, ph):
    """HLL flux (Harten, Lax and van Leer; Toro, Ch. 10): one intermediate
    state between the fastest left- and right-going waves, with the Einfeldt
    (Roe-averaged) speed estimates of hllc_flux:
    F = F_L if S_L >= 0, F_R if S_R <= 0, else
    (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)."""
    g = ph.gamma
    rL, vL, pL, _ = primitives(UL, ph)
    rR, vR, pR, _ = primitives(UR, ph)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    HL = (UL[..., -1] + pL) / rL
    HR = (UR[..., -1] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    ut = (sL[..., None] * vL + sR[..., None] * vR) / (sL + sR)[..., None]
    Ht = (sL * HL + sR * HR) / (sL + sR)
    ct = np.sqrt((g - 1.0) * (Ht - 0.5 * np.sum(ut * ut, axis=-1)))
    unL, unR, unt = np.sum(vL * n, -1), np.sum(vR * n, -1), np.sum(ut * n, -1)
    SL = np.minimum(unL - cL, unt - ct)
    SR = np.maximum(unR + cR, unt + ct)
    FL = np.einsum("...iv,...i->...v", euler_flux(UL, ph), n)
    FR = np.einsum("...iv,...i->...v", euler_flux(UR, ph), n)
    Fm = (SR[..., None] * FL - SL[..., None] * FR + (SL * SR)[..., None] * (UR - UL)) \
        / (SR - SL)[..., None]
    return np.where((SL >= 0)[..., None], FL, np.where((SR <= 0)[..., None], FR, Fm))


def lax_friedrichs_flux(UL, UR, n, ph):
    """Local Lax-Friedrichs (Rusanov) flux: the mean of the two normal fluxes
    minus a jump penalty at the larger of the two sides' spectral radii
    |u_n| + c (Toro, Ch. 10)."""
    g = ph.gamma
    rL, vL, pL, _ = primitives(UL, ph)
    rR, vR, pR, _ = primitives(UR, ph)
    lam = np.maximum(np.abs(np.sum(vL * n, -1)) + np.sqrt(g * pL / rL),
                     np.abs(np.sum(vR * n, -1)) + np.sqrt(g * pR / rR))
    FL = np.einsum("...iv,...i->...v", euler_flux(UL, ph), n)
    FR = np.einsum("...iv,...i->...v", euler_flux(UR, ph), n)
    return 0.5 * (FL + FR) - 0.5 * lam[..., None] * (UR - UL)


def ausm_flux(UL, UR, n, ph):
    """AUSM flux of Liou and Steffen (1993): the convective part is the
    interface Mach number m = M+(M_L) + M-(M_R) times the upwinded
    c (rho, rho u, rho H), the pressure part p+(M_L) p_L + p-(M_R) p_R on the
    momentum, with the van Leer polynomial splittings
      M+- = +-(M +- 1)^2 / 4,  p+- = (M +- 1)^2 (2 -+ M) / 4    for |M| <= 1,
      M+- = (M +- |M|) / 2,    p+- = (1 +- sign M) / 2           otherwise,
    M = u_n / c on each side (normal velocity along n)."""
    g = ph.gamma
    d = UL.shape[-1] - 2
    rL, vL, pL, _ = primitives(UL, ph)
    rR, vR, pR, _ = primitives(UR, ph)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ML, MR = np.sum(vL * n, -1) / cL, np.sum(vR * n, -1) / cR
    sub_L, sub_R = np.abs(ML) <= 1.0, np.abs(MR) <= 1.0
    Mp = np.where(sub_L, 0.25 * (ML + 1.0) ** 2, 0.5 * (ML + np.abs(ML)))
    Mm = np.where(sub_R, -0.25 * (MR - 1.0) ** 2, 0.5 * (MR - np.abs(MR)))
    Pp = np.where(sub_L, 0.25 * (ML + 1.0) ** 2 * (2.0 - ML), 0.5 * (1.0 + np.sign(ML)))
    Pm = np.where(sub_R, 0.25 * (MR - 1.0) ** 2 * (2.0 + MR), 0.5 * (1.0 - np.sign(MR)))
    m = Mp + Mm
    p = Pp * pL + Pm * pR

    def phi(U, r, c, pp):     # c (rho, rho u, rho H)
        return c[..., None] * np.concatenate([r[..., None], U[..., 1:1 + d],
                                              (U[..., -1] + pp)[..., None]], axis=-1)

    fL, fR = phi(UL, rL, cL, pL), phi(UR, rR, cR, pR)
    F = 0.5 * m[..., None] * (fL + fR) - 0.5 * np.abs(m)[..., None] * (fR - fL)
    F[..., 1:1 + d] += p[..., None] * n
    return F


def riemann_flux(UL, UR, n, ph):
    """The numerical advection flux selected by ph.riemann (Sec. 4.3 lists
    Roe, HLL, HLLC, AUSM and Lax-Friedrichs among the solvers' fluxes)."""
    return {RIEMANN_ROE: roe_flux, RIEMANN_HLLC: hllc_flux, RIEMANN_HLL: hll_flux,
            RIEMANN_LF: lax_friedrichs_flux, RIEMANN_AUSM: ausm_flux}[ph.riemann](UL, UR, n, ph)


# ---------------------------------------------------------------- analytic fields

def exact_state(ph, x, t):
    """Conservative state of the workload's analytic field at points x[..., d]."""
    d = x.shape[-1]
    g, Ma = ph.gamma, ph.Ma
    shp = x.shape[:-1]
    if ph.fid in (FIELD_UNIFORM, FIELD_CYLINDER):
        rho = np.ones(shp)
        vel = np.zeros(shp + (d,))
        vel[..., 0] = 1.0
        T = np.ones(shp)
        if ph.fid == FIELD_UNIFORM and len(ph.fpar) >= 5 and ph.fpar[0] > 0:
            rho = rho * ph.fpar[0]
            vel = np.broadcast_to(np.asarray(ph.fpar[1:1 + d], float), shp + (d,)).copy()
            T = T * ph.fpar[4]
        if ph.fid == FIELD_CYLINDER and len(ph.fpar) >= 2 and ph.fpar[1] > 0:
            # stream brought to rest at the wall r = fpar[0] over the length fpar[1]
            r = np.sqrt(x[..., 0] ** 2 + x[..., 1] ** 2)
            vel = vel * (1.0 - np.exp(-np.maximum(r - ph.fpar[0], 0.0) / ph.fpar[1]))[..., None]
    elif ph.fid == FIELD_VORTEX:
        # isentropic vortex (Sec. 6.1) on [0,1]^2 = [0,10]^2 scaled by 1/s, with the
        # sign of the u perturbation that makes it a vortex, and T from the radial
        # momentum balance in the p = rho T/(gamma Ma^2) non-dimensionalisation
        u0, v0, phi, xc, yc, s = ph.fpar
        cx = xc + u0 * t
        cy = yc + v0 * t
        dx = x[..., 0] - cx
        dy = x[..., 1] - cy
        dx = dx - np.round(dx)        # nearest periodic image (period 1)
        dy = dy - np.round(dy)
        X, Y = s * dx, s * dy
        ex = np.exp(1.0 - X * X - Y * Y)
        vel = np.stack([u0 - phi / (2 * np.pi) * Y * ex, v0 + phi / (2 * np.pi) * X * ex], -1)
        T = 1.0 - (g - 1.0) * Ma ** 2 * phi ** 2 / (16 * np.pi ** 2) * ex * ex
        rho = T ** (1.0 / (g - 1.0))
    elif ph.fid == FIELD_POISEUILLE:
        theta, L, dpdx = ph.fpar
        mu = 1.0 / ph.Re
        y = x[..., 1]
        rho = np.ones(shp)
        vel = np.zeros(shp + (d,))
        vel[..., 0] = -dpdx / (2 * mu) * (y * (L - y) + theta * y * y * (L - y) ** 2)
        p = 1.0 / (g * Ma ** 2) + dpdx * x[..., 0]
        T = g * Ma ** 2 * p / rho
    elif ph.fid == FIELD_SHOCK:
        # oblique shock of angle beta (to the x axis) reaching the line y = 0
        # at x = x_sh: the uniform stream (1, 0) at T = 1 below the shock
        # line y = (x_sh - x) tan(beta), the Rankine-Hugoniot state above it.
        # fpar[2] = w > 0: the primitive variables pass from one state to the
        # other by the fraction (1 + tanh(s / w)) / 2 of the signed distance
        # s = y cos(beta) - (x_sh - x) sin(beta) to the line; fpar[3] = l > 0:
        # the velocity is brought to rest at the wall y = 0 by 1 - exp(-y / l)
        beta, xsh = np.radians(ph.fpar[0]), ph.fpar[1]
        width = ph.fpar[2] if len(ph.fpar) > 2 else 0.0
        layer = ph.fpar[3] if len(ph.fpar) > 3 else 0.0
        r2, v2, p2 = oblique_shock_state(beta, ph)
        if width > 0.0:
            dist = x[..., 1] * np.cos(beta) - (xsh - x[..., 0]) * np.sin(beta)
            post = 0.5 * (1.0 + np.tanh(dist / width))
        else:
            post = (x[..., 1] > (xsh - x[..., 0]) * np.tan(beta)).astype(float)
        p1 = 1.0 / (g * Ma ** 2)
        rho = 1.0 + post * (r2 - 1.0)
        vel = np.zeros(shp + (d,))
        vel[..., 0] = 1.0 + post * (v2[0] - 1.0)
        vel[..., 1] = post * v2[1]
        if layer > 0.0:
            vel *= (1.0 - np.exp(-x[..., 1] / layer))[..., None]
        p = p1 + post * (p2 - p1)
        T = g * Ma ** 2 * p / rho
    elif ph.fid == FIELD_TGV:
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        vel = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z),
                        np.zeros(shp)], -1)
        pinf = 1.0 / (g * Ma ** 2)
        p = pinf + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
        rho = p / pinf
        T = np.ones(shp)
    else:
        raise ValueError(ph.fid)
    p = rho * T / (g * Ma ** 2)
    return conservative(rho, vel, p, ph)


def oblique_shock_state(beta, ph):
    """State behind an oblique shock of angle beta met by the stream (1, 0),
    rho = 1, p = 1/(gamma Ma^2) (Rankine-Hugoniot relations for the normal
    Mach number Ma sin(beta); the tangential velocity is continuous; the shock
    normal n = (sin beta, cos beta) points from the upstream side).  Returns
    (rho2, velocity2, p2)."""
    g, Ma = ph.gamma, ph.Ma
    n = np.array([np.sin(beta), np.cos(beta)])
    t = np.array([np.cos(beta), -np.sin(beta)])
    u1 = np.array([1.0, 0.0])
    m1n2 = (Ma * np.sin(beta)) ** 2
    r2 = (g + 1) * m1n2 / ((g - 1) * m1n2 + 2)
    p2 = (1 + 2 * g / (g + 1) * (m1n2 - 1)) / (g * Ma ** 2)
    v2 = (u1 @ n) / r2 * n + (u1 @ t) * t
    return r2, v2, p2


def forcing(ph, x, t):
    """Manufactured source of the compressible Poiseuille case (App. B), with
    f_4 built on h(y) = y(L-y) + theta y^2 (L-y)^2 (the printed f_4 has y(L-y)
    and an unmatched parenthesis; this form makes the steady residual of the
    exact solution vanish identically with constant mu)."""
    f = np.zeros(x.shape[:-1] + (x.shape[-1] + 2,))
    if ph.forcing == FORCING_NONE:
        return f
    theta, L, dpdx = ph.fpar
    mu = 1.0 / ph.Re
    g = ph.gamma
    y = x[..., 1]
    c = L * L - 6 * y * L + 6 * y * y
    h = y * (L - y) + theta * y * y * (L - y) ** 2
    f[..., 1] = dpdx * theta * c
    f[..., -1] = (dpdx ** 2 / (2 * mu) * h * (1 - theta * c - g / (g - 1))
                  - dpdx ** 2 / (4 * mu) * (L - 2 * y) ** 2 * (2 * theta * y * L - 2 * theta * y * y + 1) ** 2)
    return f


def wall_temperature(ph, x):
    if ph.fid == FIELD_POISEUILLE:
        _, _, dpdx = ph.fpar
        return 1.0 + ph.gamma * ph.Ma ** 2 * dpdx * x[..., 0]
    return np.ones(x.shape[:-1])


def farfield_state(ph, UL, Uinf, n):
    """Characteristic far-field state (Sec. 4.3 lists a Riemann-invariant
    condition, used on the outer boundary of the cylinder of Sec. 6.4, without
    its formulas; this is the textbook one-dimensional reading along the
    outward normal n).  With c the speed of sound, the outgoing invariant
    R+ = u_n + 2c/(gamma-1) is taken from the interior state UL and the
    incoming R- = u_n - 2c/(gamma-1) from the free stream Uinf; their half sum
    and quarter difference give u_n and c on the boundary.  Entropy p/rho^gamma
    and the tangential velocity come from the upwind side (interior where the
    boundary normal velocity leaves the domain).  Supersonic normal flow
    (|u_n| >= c in the interior) takes the whole state from the upwind side."""
    g = ph.gamma
    rho, vel, p, _ = primitives(UL, ph)
    ri, vi, pi, _ = primitives(Uinf, ph)
    c = np.sqrt(g * p / rho)
    ci = np.sqrt(g * pi / ri)
    un = np.sum(vel * n, axis=-1)
    uni = np.sum(vi * n, axis=-1)
    Rp = un + 2.0 * c / (g - 1.0)
    Rm = uni - 2.0 * ci / (g - 1.0)
    unb = 0.5 * (Rp + Rm)
    cb = 0.25 * (g - 1.0) * (Rp - Rm)
    out = (unb > 0.0)[..., None]
    s_up = np.where(unb > 0.0, p / rho ** g, pi / ri ** g)
    v_up = np.where(out, vel, vi)
    vt = v_up - np.sum(v_up * n, axis=-1)[..., None] * n
    rb = (cb * cb / (g * s_up)) ** (1.0 / (g - 1.0))
    pb = rb * cb * cb / g
    Ub = conservative(rb, vt + unb[..., None] * n, pb, ph)
    Ub = np.where((un >= c)[..., None], UL, Ub)
    Ub = np.where((un <= -c)[..., None], Uinf, Ub)
    return Ub


def boundary_states(ph, bctype, x, t, UL, n):
    """Weakly imposed boundary data on the face points of a physical boundary:
    (U_r, U_b, adiabatic).  U_r is the exterior state of the Riemann flux, U_b
    the state of the viscous flux and of the interior-penalty jump Q_L - U_b
    (the interior gradient is used on the boundary).  On an adiabatic wall the
    energy components of the viscous normal flux G^n and of S_j vanish (zero
    heat flux through the wall; the wall state has zero velocity, so the
    viscous work is zero too).
      Dirichlet:      U_r = U_b = the workload's analytic state
      isothermal wall U_r = U_b = (rho_L, 0, rho_L T_w / (gamma (gamma-1) Ma^2))
      adiabatic wall  U_r = interior state with the normal momentum reversed,
                      U_b = (rho_L, 0, p_L / (gamma-1))  (wall temperature = T_L)
      far field       U_r = U_b = farfield_state(UL, analytic state)"""
    g, Ma = ph.gamma, ph.Ma
    if bctype == BC_DIRICHLET:
        Ue = exact_state(ph, x, t)
        return Ue, Ue, False
    if bctype == BC_ISO_WALL:
        Tw = wall_temperature(ph, x)
        rho = UL[..., 0]
        Ub = np.zeros_like(UL)
        Ub[..., 0] = rho
        Ub[..., -1] = rho * Tw / (g * (g - 1.0) * Ma ** 2)
        return Ub, Ub, False
    if bctype == BC_ADIA_WALL:
        rho, vel, p, _ = primitives(UL, ph)
        vm = vel - 2.0 * np.sum(vel * n, axis=-1)[..., None] * n
        Ur = conservative(rho, vm, p, ph)
        Ub = conservative(rho, np.zeros_like(vel), p, ph)
        return Ur, Ub, True
    if bctype == BC_FARFIELD:
        Ub = farfield_state(ph, UL, exact_state(ph, x, t), n)
        return Ub, Ub, False
    raise NotImplementedError(f"boundary type {bctype}")
