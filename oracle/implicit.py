"""Implicit machinery of Sec. 3.2 and Sec. 4.2.2: the Jacobian-free product,
restarted right-preconditioned GMRES, the block relaxed Jacobi preconditioner
BRJ(J), Newton's method and SDIRK time stepping (App. A).

Norms are the Euclidean norm of the full coefficient vector.
"""
from dataclasses import dataclass, field
import numpy as np
from . import physics as phy

EPS_HAT = 2.0 ** -52          # machine epsilon of IEEE double (2.22e-16)


def norm(x):
    return float(np.sqrt(np.sum(x * x)))


# ------------------------------------------------------------------- JFNK (Eq. 24-25)

def jfnk_eps(u, v):
    """epsilon = sqrt(eps_hat) ||u|| / ||v||  (Eq. eps-JF scaled by ||v||, so
    that it equals the paper's value for unit-norm v; sqrt(eps_hat)/||v|| when
    u = 0)."""
    nu, nv = norm(u), norm(v)
    return np.sqrt(EPS_HAT) * (nu if nu > 0 else 1.0) / nv


def jvp(dg, u, r_u, t, v, alpha, beta):
    """alpha v + beta (R(u + eps v) - R(u)) / eps  (Eq. Jacobian-free-matrix).
    With alpha = 1, beta = -dt a_mm this is dN/du . v of Eq. Newton-Iteration."""
    nv = norm(v)
    if nv == 0.0:
        return alpha * v
    eps = jfnk_eps(u, v)
    return alpha * v + beta * (dg.residual(u + eps * v, t) - r_u) / eps


# ------------------------------------------------------------------- GMRES

@dataclass
class GmresConfig:
    restart: int = 30
    rtol: float = 5e-2
    max_cycles: int = 10
    ortho: str = "cgs2"       # or "mgs"


@dataclass
class GmresStats:
    iters: int = 0
    cycles: int = 0
    converged: bool = False
    res: float = 0.0
    res0: float = 0.0


def gmres(apply_A, b, precond=None, cfg=None):
    """Restarted GMRES (Saad & Schultz) with right preconditioning
    (Eq. preconditioning): solves A x = b from x0 = 0, stopping when the
    residual estimate drops below rtol * ||b||; Arnoldi by classical
    Gram-Schmidt applied twice (cgs2) or modified Gram-Schmidt (mgs); the
    least-squares problem is reduced by Givens rotations."""
    cfg = cfg if cfg is not None else GmresConfig()
    Pinv = precond if precond is not None else (lambda z: z)
    x = np.zeros_like(b)
    st = GmresStats()
    bn = norm(b)
    st.res0 = bn
    if bn == 0.0:
        st.converged = True
        return x, st
    m = cfg.restart
    for cyc in range(cfg.max_cycles):
        r = b if cyc == 0 else b - apply_A(x)
        beta = norm(r)
        st.res = beta
        if beta <= cfg.rtol * bn:
            st.converged = True
            break
        st.cycles += 1
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        k_used = 0
        for k in range(m):
            w = apply_A(Pinv(V[k]))
            st.iters += 1
            if cfg.ortho == "cgs2":
                Vm = np.stack([v.ravel() for v in V])
                h = Vm @ w.ravel()
                w = w - (Vm.T @ h).reshape(w.shape)
                h2 = Vm @ w.ravel()
                w = w - (Vm.T @ h2).reshape(w.shape)
                h = h + h2
            else:
                h = np.zeros(k + 1)
                for i in range(k + 1):
                    h[i] = np.sum(V[i] * w)
                    w = w - h[i] * V[i]
            hn = norm(w)
            H[:k + 1, k] = h
            H[k + 1, k] = hn
            V.append(w / hn if hn > 0 else w)
            for i in range(k):
                t0 = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t0
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            gvec[k + 1] = -sn[k] * gvec[k]
            gvec[k] = cs[k] * gvec[k]
            k_used = k + 1
            st.res = abs(gvec[k + 1])
            if st.res <= cfg.rtol * bn or hn == 0.0:
                break
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (gvec[i] - H[i, i + 1:k_used] @ y[i + 1:k_used]) / H[i, i]
        x = x + Pinv(sum(y[i] * V[i] for i in range(k_used)))
        if st.res <= cfg.rtol * bn:
            st.converged = True
            break
    return x, st



# ------------------------------------------------------------------- BRJ (Sec. 4.2.2)

def trace_fd_steps(u):
    """chi_k = sqrt(eps_hat) * ||u_k|| with ||u_k|| the coefficient norm of
    variable k over the mesh (sqrt(eps_hat) when that norm is zero)."""
    nk = np.sqrt(np.sum(u * u, axis=(0, 2)))
    nk[nk == 0] = 1.0
    return np.sqrt(EPS_HAT) * nk


class BRJ:
    """Block relaxed Jacobi preconditioner for dN/du = I - dt_a M^-1 dL/du
    (Eq. Jacobian-matrix-form), split into element blocks L + D + U
    (Eq. L+D+U) and applied by the iteration of Eq. precond-Jacobi.

    Kept terms of Eq. Jacobian-matrix-form2: the two element-volume terms
    (exact flux Jacobians, by complex-step differentiation of F and linearity
    of G in grad Q) and the trace term with the numerical flux Jacobians
    dH^n/dQ^+- taken by the one-sided finite difference of
    Eq. numerical-Jac-on-traces (boundary states re-evaluated).  The two
    terms with the trace-gradient and symmetric-flux Jacobians are neglected
    (the paper's choice), unless full=True:
      term 4  (B^G)^T wJ (dH^n/d grad_j Q^+-) (d grad_j Q^+-/d u_e2): H^n
              depends on the face gradients only through n . G({Q}, {grad Q})
              (interior face: {grad Q} = the mean of the two sides; boundary:
              the interior gradient), and G is linear in the gradient, so
              dH^n_k/d(grad_j Q_l) = -c sum_i n_i G_ik({Q}, e_j (x) e_l),
              c = 1/2 on interior and 1 on boundary faces;
      term 5  the symmetric-flux lift sum_i integral d_i phi S_i with
              dS/dQ^+- by the same one-sided difference as term 3;
    both enter the diagonal blocks and, on interior faces, the neighbour
    coupling (L + U), stored then as dense element-pair blocks per face.
    """

    assembly_dtype = np.float64

    def __init__(self, dg, u, t, dt_a, J=7, omega=1.0, assembly_dtype=np.float64, full=False):
        """assembly_dtype: precision of the two volume-term contractions (float32
        measures the rounding floor of a single-precision block assembly);
        full: keep terms 4 and 5 of Eq. Jacobian-matrix-form2."""
        self.dg, self.J, self.omega, self.dt_a = dg, J, omega, dt_a
        self.assembly_dtype = assembly_dtype
        self.full = full and dg.ph.viscous
        d, nv, nm, E = dg.dim, dg.nv, dg.nm, dg.E
        self.nb = nv * nm
        # artificial viscosity frozen at u (Sec. 4.2.2: its derivatives are neglected)
        self.av = getattr(dg.ph, "av", 0) and dg.ph.viscous
        self.fac = dg.av_factor(u) if self.av else None
        dLdu = self._volume_jacobian(u)                            # [E][v m][l n]
        self.off = []
        self.off_full = []
        chi = trace_fd_steps(u)
        for g in dg.groups:
            JL, JR = self._trace_jacobians(g, u, t, chi)           # [f][p][k][l]
            wJ = g["wJ"]
            BL = dg.Bf[g["fL"]]
            blk = -np.einsum("pm,fp,fpkl,pn->fkmln", BL, wJ, JL, BL, optimize=True)
            np.add.at(dLdu, g["eL"], blk.reshape(-1, self.nb, self.nb))
            if g["bctype"] is None:
                BR = dg.Bf[g["fR"]]
                blk = np.einsum("pm,fp,fpkl,pn->fkmln", BR, wJ, JR, BR, optimize=True)
                np.add.at(dLdu, g["eR"], blk.reshape(-1, self.nb, self.nb))
                self.off.append((g, JL, JR))
            if self.full:
                LL, LR, RL, RR = self._viscous_trace_blocks(g, u, t, chi)
                np.add.at(dLdu, g["eL"], LL)
                if g["bctype"] is None:
                    np.add.at(dLdu, g["eR"], RR)
                    self.off_full.append((g, LR, RL))
        # D = I - dt_a M^-1 dL/du (diagonal blocks), then invert
        Minv = dg.Minv
        MdL = np.einsum("emn,eknlo->ekmlo", Minv, dLdu.reshape(E, nv, nm, nv, nm))
        D = np.eye(self.nb)[None] - dt_a * MdL.reshape(E, self.nb, self.nb)
        self.D = D
        self.Dinv = np.linalg.inv(D)

    def _volume_jacobian(self, u):
        dg, ph = self.dg, self.dg.ph
        d, nv, nm, E = dg.dim, dg.nv, dg.nm, dg.E
        Qv = dg.values(u, dg.B)
        dQ = dg.gradients(u, dg.D, dg.ginv)
        mu_q = dg.volume_av(self.fac, Qv, dQ) if getattr(self, "av", 0) else None
        h = 1e-30
        # A0[e,q,j,k,l] = dH_jk/dQ_l at fixed grad Q (complex step)
        A0 = np.zeros(Qv.shape[:2] + (d, nv, nv))
        for l in range(nv):
            Qc = Qv.astype(complex)
            Qc[..., l] += 1j * h
            Hc = phy.euler_flux(Qc, ph)
            if ph.viscous:
                Hc = Hc - phy.viscous_flux(Qc, dQ.astype(complex), ph, mu_q)
            A0[..., l] = Hc.imag / h
        # A1[e,q,j,i,k,l] = dH_jk / d(grad_i Q_l) = -G_jk(Q, e_i (x) e_l)
        A1 = np.zeros(Qv.shape[:2] + (d, d, nv, nv))
        if ph.viscous:
            for i in range(d):
                for l in range(nv):
                    gu = np.zeros(dQ.shape)
                    gu[..., i, l] = 1.0
                    A1[..., :, i, :, l] = -phy.viscous_flux(Qv, gu, ph, mu_q)
        # physical derivative tables DB[e,j,q,m] = sum_r ginv[e,q,r,j] D_r[q,m]
        DB = np.einsum("eqrj,rqm->ejqm", dg.ginv, dg.D)
        wJ = dg.wJ
        # volume terms 1 and 2 of Eq. Jacobian-matrix-form2
        c = lambda a: np.asarray(a, dtype=self.assembly_dtype)
        T = np.einsum("eq,ejqm,eqjkl,qn->ekmln", c(wJ), c(DB), c(A0), c(dg.B), optimize=True)
        T += np.einsum("eq,ejqm,eqjikl,eiqn->ekmln", c(wJ), c(DB), c(A1), c(DB), optimize=True)
        return T.astype(np.float64).reshape(E, nv * nm, nv * nm)

    def _flux_only(self, g, QL, QR, dQa, t, mu_f=None):
        """H^n on group g as a function of the two traces at fixed gradients;
        on boundary faces QR is recomputed from QL by the boundary condition."""
        dg = self.dg
        if g["bctype"] is None:
            Qa = 0.5 * (QL + QR)
        else:
            QR, Qa, _ = phy.boundary_states(dg.ph, g["bctype"], g["x"], t, QL, g["n"])
        Hh, _ = dg.face_flux(g, QL, QR, Qa, dQa, t, mu_f)
        return Hh

    def _symmetric_flux(self, g, QL, QR, t, mu_f=None):
        """S_i on group g as a function of the two traces (boundary: QR from
        QL by the boundary condition), [f][p][i][v]."""
        dg = self.dg
        if g["bctype"] is None:
            Qa = 0.5 * (QL + QR)
            jump = QL - QR
        else:
            _, Qa, _ = phy.boundary_states(dg.ph, g["bctype"], g["x"], t, QL, g["n"])
            jump = QL - Qa
        S = phy.viscous_flux(Qa, g["n"][..., :, None] * jump[..., None, :], dg.ph, mu_f)
        if g["bctype"] == phy.BC_ADIA_WALL:
            S[..., -1] = 0.0
        return S

    def _viscous_trace_blocks(self, g, u, t, chi):
        """Terms 4 and 5 of Eq. Jacobian-matrix-form2 on group g as dense
        blocks [f][v m][l n]: (dL_eL/du_eL, dL_eL/du_eR, dL_eR/du_eL,
        dL_eR/du_eR); the last three are None on boundary faces."""
        dg, ph = self.dg, self.dg.ph
        d, nv, nb = dg.dim, dg.nv, self.nb
        QL, QR, Qa, dQa, _, _ = dg.face_states(g, u, t)
        mu_f = dg.face_av(g, self.fac, QL, QR, dQa) if self.av else None
        n, wJ = g["n"], g["wJ"]
        interior = g["bctype"] is None
        c_grad = 0.5 if interior else 1.0
        # physical derivative of each mode at the face points, [f][p][j][m]
        GL = np.einsum("fprj,rpm->fpjm", g["ginvL"], np.asarray(dg.Df[g["fL"]]))
        BL = dg.Bf[g["fL"]]
        # term 4: dH^n_k / d(grad_j Q_l) (same on both sides of an interior face)
        KG = np.zeros(QL.shape[:2] + (nv, d, nv))
        for j in range(d):
            for l in range(nv):
                gu = np.zeros(QL.shape[:2] + (d, nv))
                gu[..., j, l] = 1.0
                Gu = phy.viscous_flux(Qa, gu, ph, mu_f)             # [f][p][i][k]
                KG[..., j, l] = -c_grad * np.einsum("fpi,fpik->fpk", n, Gu)
        if g["bctype"] == phy.BC_ADIA_WALL:
            KG[..., -1, :, :] = 0.0
        # term 5: dS_i / dQ^side by the one-sided difference of term 3
        S0 = self._symmetric_flux(g, QL, QR, t, mu_f)
        SL = np.zeros(S0.shape + (nv,))
        SR = np.zeros(S0.shape + (nv,))
        for l in range(nv):
            Qp = QL.copy()
            Qp[..., l] += chi[l]
            SL[..., l] = (self._symmetric_flux(g, Qp, QR, t, mu_f) - S0) / chi[l]
            if interior:
                Qp = QR.copy()
                Qp[..., l] += chi[l]
                SR[..., l] = (self._symmetric_flux(g, QL, Qp, t, mu_f) - S0) / chi[l]
        c_sym = (0.5 if interior else 1.0) * ph.beta_s

        def t4(Brow, G_col, sign):
            # sign * sum_p Brow[p,m] wJ KG[p,k,j,l] G_col[p,j,n]
            return sign * np.einsum("pm,fp,fpkjl,fpjn->fkmln", Brow, wJ, KG, G_col,
                                    optimize=True).reshape(-1, nb, nb)

        def t5(G_row, Sd, Bcol):
            # c sum_p sum_i G_row[p,i,m] wJ dS_i,k/dQ_l B_col[p,n]
            return c_sym * np.einsum("fpim,fp,fpikl,pn->fkmln", G_row, wJ, Sd, Bcol,
                                     optimize=True).reshape(-1, nb, nb)

        LL = t4(BL, GL, -1.0) + t5(GL, SL, BL)
        if not interior:
            return LL, None, None, None
        GR = np.einsum("fprj,rpm->fpjm", g["ginvR"], np.asarray(dg.Df[g["fR"]]))
        BR = dg.Bf[g["fR"]]
        LR = t4(BL, GR, -1.0) + t5(GL, SR, BR)
        RL = t4(BR, GL, +1.0) + t5(GR, SL, BL)
        RR = t4(BR, GR, +1.0) + t5(GR, SR, BR)
        return LL, LR, RL, RR

    def _trace_jacobians(self, g, u, t, chi):
        dg = self.dg
        nv = dg.nv
        QL, QR, Qa, dQa, _, _ = dg.face_states(g, u, t)
        mu_f = dg.face_av(g, self.fac, QL, QR, dQa) if self.av else None
        H0 = self._flux_only(g, QL, QR, dQa, t, mu_f)
        JL = np.zeros(QL.shape + (nv,))
        JR = np.zeros(QL.shape + (nv,))
        for l in range(nv):
            Qp = QL.copy()
            Qp[..., l] += chi[l]
            JL[..., l] = (self._flux_only(g, Qp, QR, dQa, t, mu_f) - H0) / chi[l]
            if g["bctype"] is None:
                Qp = QR.copy()
                Qp[..., l] += chi[l]
                JR[..., l] = (self._flux_only(g, QL, Qp, dQa, t, mu_f) - H0) / chi[l]
        return JL, JR

    def offdiag(self, q):
        """(L + U) q: the neighbour coupling of the trace term, times
        -dt_a M^-1."""
        dg = self.dg
        out = np.zeros_like(q)
        for g, JL, JR in self.off:
            wJ = g["wJ"]
            qL = dg.values(q, dg.Bf[g["fL"]], g["eL"])
            qR = dg.values(q, dg.Bf[g["fR"]], g["eR"])
            # dL_L/du_R q_R = -B_L^T wJ JR qR ; dL_R/du_L q_L = +B_R^T wJ JL qL
            out[g["eL"]] -= np.einsum("pm,fp,fpkl,fpl->fkm", dg.Bf[g["fL"]], wJ, JR, qR)
            out[g["eR"]] += np.einsum("pm,fp,fpkl,fpl->fkm", dg.Bf[g["fR"]], wJ, JL, qL)
        shp = out.shape[1:]
        for g, LR, RL in self.off_full:
            # terms 4-5: dense neighbour blocks dL_eL/du_eR and dL_eR/du_eL
            qR = q[g["eR"]].reshape(len(g["eR"]), -1)
            qL = q[g["eL"]].reshape(len(g["eL"]), -1)
            out[g["eL"]] += np.einsum("fab,fb->fa", LR, qR).reshape((-1,) + shp)
            out[g["eR"]] += np.einsum("fab,fb->fa", RL, qL).reshape((-1,) + shp)
        return -self.dt_a * dg.apply_minv(out)

    def diag_solve(self, y):
        E = self.dg.E
        return np.einsum("eab,eb->ea", self.Dinv, y.reshape(E, -1)).reshape(y.shape)

    def apply(self, q):
        """q^J of Eq. precond-Jacobi from q^0 = 0."""
        qh = np.zeros_like(q)
        for j in range(self.J):
            y = q if j == 0 else q - self.offdiag(qh)
            qh = self.omega * self.diag_solve(y) + (1.0 - self.omega) * qh
        return qh

    def memory_bytes_paper_layout(self, value_bytes=4):
        """Per-element storage in the paper's accounting (Tab. BRJ memory):
        the diagonal inverse block (N_v N_m)^2 and, for each of the 2d faces of
        the element, the two N_v x N_v trace Jacobians at each face point."""
        dg = self.dg
        diag = self.nb ** 2 * value_bytes
        off = 2 * dg.dim * 2 * dg.nf * dg.nv * dg.nv * value_bytes
        return diag, off


# ------------------------------------------------------------------- Newton + SDIRK

@dataclass
class NewtonConfig:
    alpha: float = 1e-3          # relative tolerance of Eq. nonlinear-critria
    abs_tol: float = 0.0         # > 0: absolute tolerance instead
    max_iters: int = 20
    gmres: GmresConfig = field(default_factory=GmresConfig)


@dataclass
class NewtonStats:
    iters: int = 0
    gmres_iters: int = 0
    res0: float = 0.0
    res: float = 0.0
    converged: bool = False


def newton(dg, S, t, dt_a, u0, precond=None, cfg=None):
    """Newton's method (Eq. Newton-initial-guess, Newton-Iteration) on
    N(u) = u - S - dt_a R(u, t) (Eq. nonlinear-equation-system), each linear
    step solved by JFNK GMRES.  Returns (u, R(u), stats)."""
    cfg = cfg if cfg is not None else NewtonConfig()
    u = u0.copy()
    R = dg.residual(u, t)
    N = u - S - dt_a * R
    st = NewtonStats()
    st.res0 = st.res = norm(N)
    tol = cfg.abs_tol if cfg.abs_tol > 0 else cfg.alpha * st.res0
    while True:
        if st.res <= 0.0 or (st.iters > 0 or cfg.abs_tol > 0) and st.res < tol:
            st.converged = True
            break
        if st.iters >= cfg.max_iters:
            break
        Ru = R

        def A(v, u=u, Ru=Ru):
            return jvp(dg, u, Ru, t, v, 1.0, -dt_a)

        dx, gs = gmres(A, -N, precond, cfg.gmres)
        st.gmres_iters += gs.iters
        u = u + dx
        st.iters += 1
        R = dg.residual(u, t)
        N = u - S - dt_a * R
        st.res = norm(N)
    return u, R, st


def sdirk_tableau(name):
    """Butcher tableaus of App. A (Tab. RK-coeff): SDIRK2 with
    lambda = 1 - sqrt(2)/2, SDIRK3 with lambda = 0.4358665215, and the
    six-stage fourth-order scheme with an explicit first stage and diagonal
    1/4 ("esdirk4"); plus backward Euler ("be", one stage with a = b = c = 1),
    which Sec. 4.3 lists among the implicit schemes.

    The fourth-order table is printed with symbols a^{i1} in its first
    column: each names the entry beside it in the second column (a^{i0} =
    a^{i1}, as in the Kennedy-Carpenter scheme the paper cites).  The nodes c
    are then the row sums; the printed third node (2 - sqrt 2)/2 is read as
    (2 - sqrt 2)/4, the row sum of (1 - sqrt 2)/8, (1 - sqrt 2)/8, 1/4 (with
    the printed node the row-sum reading of the first column violates the
    order conditions).  The weights are the last row (stiffly accurate)."""
    if name == "be":
        return np.array([[1.0]]), np.array([1.0]), np.array([1.0])
    if name == "esdirk4":
        r2 = np.sqrt(2.0)
        A = np.zeros((6, 6))
        A[1, 1] = 0.25
        A[2, 1], A[2, 2] = (1 - r2) / 8, 0.25
        A[3, 1], A[3, 2], A[3, 3] = (5 - 7 * r2) / 64, 7 * (1 + r2) / 32, 0.25
        A[4, 1] = (-13796 - 54539 * r2) / 125000
        A[4, 2] = (506605 + 132109 * r2) / 437500
        A[4, 3] = 166 * (-97 + 376 * r2) / 109375
        A[4, 4] = 0.25
        A[5, 1] = (1181 - 987 * r2) / 13782
        A[5, 2] = 47 * (-267 + 1783 * r2) / 273343
        A[5, 3] = -16 * (-22922 + 3525 * r2) / 571953
        A[5, 4] = -15625 * (97 + 376 * r2) / 90749876
        A[5, 5] = 0.25
        A[1:, 0] = A[1:, 1]
        return A, A[5].copy(), A.sum(axis=1)
    if name == "sdirk2":
        lam = 1.0 - np.sqrt(2.0) / 2.0
        A = np.array([[lam, 0.0], [1.0 - lam, lam]])
        b = np.array([1.0 - lam, lam])
    elif name == "sdirk3":
        lam = 0.4358665215
        b1 = (-6 * lam ** 2 + 16 * lam - 1) / 4
        b2 = (6 * lam ** 2 - 20 * lam + 5) / 4
        A = np.array([[lam, 0, 0], [(1 - lam) / 2, lam, 0], [b1, b2, lam]])
        b = np.array([b1, b2, lam])
    else:
        raise ValueError(name)
    return A, b, A.sum(axis=1)


@dataclass
class StepStats:
    newton_iters: int = 0
    gmres_iters: int = 0
    stages: list = None


def sdirk_step(dg, u_n, t, dt, tableau="sdirk2", precond=None, cfg=None,
               guess=None):
    """One step of Eq. rk-stage / rk-final: each stage solves
    N(u^m) = u^m - S_m - dt a_mm R(u^m, t + c_m dt) = 0 by Newton from
    S_m (or guess(m, S_m)); E^m = dt R(u^m) is taken from the residual of the
    converged iterate; u^{n+1} = u^n + sum_i b_i E^i."""
    A, b, c = sdirk_tableau(tableau)
    M = len(b)
    E = []
    st = StepStats(stages=[])
    for m in range(M):
        S = u_n + sum(A[m, i] * E[i] for i in range(m))
        if A[m, m] == 0.0:
            # explicit stage (the first stage of esdirk4): u^m = S_m, no solve
            um, Rm, ns = S, dg.residual(S, t + c[m] * dt), NewtonStats(converged=True)
        else:
            u0 = S if guess is None else guess(m, S)
            um, Rm, ns = newton(dg, S, t + c[m] * dt, dt * A[m, m], u0, precond, cfg)
        st.newton_iters += ns.iters
        st.gmres_iters += ns.gmres_iters
        st.stages.append(ns)
        E.append(dt * Rm)
    return u_n + sum(b[i] * E[i] for i in range(M)), st


def bdf2_step(dg, u_n, u_prev, t, dt, precond=None, cfg=None):
    """One step of the second-order backward differentiation formula (Sec. 4.3
    lists it among the implicit schemes) at a constant step size:
    3 u^{n+1} - 4 u^n + u^{n-1} = 2 dt R(u^{n+1}, t + dt), i.e. Newton on
    N(u) = u - S - (2 dt / 3) R(u) with S = (4 u^n - u^{n-1}) / 3, from u = S."""
    S = (4.0 * u_n - u_prev) / 3.0
    u, _, ns = newton(dg, S, t + dt, 2.0 * dt / 3.0, S, precond, cfg)
    return u, StepStats(newton_iters=ns.iters, gmres_iters=ns.gmres_iters, stages=[ns])
