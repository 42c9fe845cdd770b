"""The DG residual R(u) = M^-1 L(u, t) of the matrix form (Sec. 3.1,
Eq. matrix-form-equations), written per element with dense operators.

  M du/dt = sum_j B^T D_j^T Lambda(wJ) H_j(Q)                     volume
            - (B^G M_c)^T Lambda(w^G J^G) H^n                     Riemann + IP flux
            + sum_j (symmetric-flux lift of S_j)                  IP symmetric term
            + B^T Lambda(wJ) f                                    forcing (App. B)

Readings of the interior-penalty terms (Eq. IP-final is printed with signs that
do not agree with the matrix form): the standard symmetric interior penalty
method is used, i.e. on a face with owner-side normal n and jump
[Q] = Q_int - Q_ext,
  S_i = G_i({Q}, n (x) [Q]) = sum_{j,l} K({Q})_ijkl n_j [Q_l]
  G^n = n . G({Q}, {grad Q}) - beta_p n . S            (dissipative penalty)
and each side adds  +c * integral( sum_i d_i phi * S_i )  with c = 1/2 on
interior faces and c = 1 on boundary faces (where {Q} is the boundary state
and {grad Q} the interior gradient).  This is the adjoint-consistent
symmetric term (the jump enters K through its gradient slot, the test
function through its flux slot); contracting the jump with the flux slot
instead, as the printed index order suggests, makes the operator
non-symmetric when K lacks the minor symmetry K_ijkl = K_ijlk, which the
symmetry test at rest detects.  beta_p = (P+1)^2 / h, h = min over the two
sides of |Omega_e| / |Gamma_f|.
Face values and gradients are evaluated from the modal expansion directly at
the face points, which equals interpolating the volume-point values with J
(exact for the polynomial expansion on affine elements).
"""
import numpy as np
from . import basis as bs
from . import geometry as geo
from . import physics as phy


class DG:
    def __init__(self, mesh, P, Q, ph, kind="modal"):
        self.mesh, self.P, self.Q, self.ph = mesh, P, Q, ph
        d = self.dim = mesh.dim
        self.nv = d + 2
        self.n = P + 1
        self.nm = self.n ** d
        self.nq = Q ** d
        self.nf = Q ** (d - 1)
        E = self.E = mesh.n_elem
        xq, wq = bs.gauss_legendre(Q)
        phi1, dphi1 = bs.basis_1d(P, xq, kind)
        self.B, self.D = bs.tensor_tables(phi1, dphi1, d)
        self.D = np.array(self.D)                                   # [r][q][m]
        qidx = np.indices((Q,) * d).reshape(d, -1)[::-1]
        self.xi = np.stack([xq[qidx[r]] for r in range(d)], -1)     # [q][d]
        self.w = np.prod([wq[qidx[r]] for r in range(d)], axis=0)   # [q]
        # volume geometry
        self.x, jac = geo.map_points(mesh.nodes, mesh.geom_order, self.xi)
        det, self.ginv = geo.metrics(jac)
        if np.any(det <= 0):
            raise ValueError("element with non-positive Jacobian")
        self.wJ = self.w[None, :] * det                             # [E][q]
        self.vol = self.wJ.sum(axis=1)
        M = np.einsum("qm,eq,qn->emn", self.B, self.wJ, self.B)
        self.Minv = np.linalg.inv(M)                                # [E][m][m]
        # faces
        self.xi_f, self.Bf, self.Df = bs.face_tables(P, Q, d, kind)
        if d > 1:
            fidx = np.indices((Q,) * (d - 1)).reshape(d - 1, -1)[::-1]
            self.wf = np.prod([wq[fidx[a]] for a in range(d - 1)], axis=0)
        else:
            self.wf = np.ones(1)
        self._build_faces()
        # shock-capturing sensor (Sec. 3.1.2): L2 projection onto polynomials of
        # degree <= P-1 per direction at the Gauss points (reference element)
        L = np.stack([bs.jacobi(k, 0.0, 0.0, xq)[0] for k in range(P)], axis=1)  # [Q][P]
        W1 = np.diag(wq)
        pi1 = L @ np.linalg.solve(L.T @ W1 @ L, L.T @ W1)
        Pi = np.ones((1, 1))
        for _ in range(d):
            Pi = np.kron(pi1, Pi)          # first direction fastest
        self.sensor_proj = Pi
        self.h_elem = self.vol ** (1.0 / d)

    # ------------------------------------------------------------------ faces
    def _side_geometry(self, elems, lf):
        x, jac = geo.map_points(self.mesh.nodes[elems], self.mesh.geom_order, self.xi_f[lf])
        det, ginv = geo.metrics(jac)
        n, jf = geo.face_normal(ginv, det, lf)
        return x, ginv, n, jf

    def _build_faces(self):
        F = self.mesh.faces
        groups = {}
        for f in range(F.shape[0]):
            eL, fL, eR, fR, orient, bc = (int(v) for v in F[f])
            if orient != 0:
                raise NotImplementedError("only aligned face orientations")
            groups.setdefault((fL, fR, bc if eR < 0 else -1), []).append(f)
        self.groups = []
        for (fL, fR, bc), fl in sorted(groups.items()):
            fl = np.asarray(fl)
            g = {"fL": fL, "fR": fR, "faces": fl, "eL": F[fl, 0].astype(np.int64)}
            x, ginvL, n, jf = self._side_geometry(g["eL"], fL)
            g["x"], g["ginvL"], g["n"] = x, ginvL, n
            g["wJ"] = self.wf[None, :] * jf
            area = g["wJ"].sum(axis=1)
            hL = self.vol[g["eL"]] / area
            if fR >= 0:
                g["eR"] = F[fl, 2].astype(np.int64)
                _, ginvR, _, _ = self._side_geometry(g["eR"], fR)
                g["ginvR"] = ginvR
                h = np.minimum(hL, self.vol[g["eR"]] / area)
                g["bctype"] = None
            else:
                h = hL
                g["bctype"] = self.ph.bc[bc]
            g["beta"] = (self.P + 1) ** 2 / h
            self.groups.append(g)

    # --------------------------------------------------------------- helpers
    def values(self, u, Bmat, elems=None):
        uu = u if elems is None else u[elems]
        return np.einsum("qm,evm->eqv", Bmat, uu)

    def gradients(self, u, Dmat, ginv, elems=None):
        """Physical gradients [e][p][j][v] from reference derivatives and the
        inverse metric."""
        uu = u if elems is None else u[elems]
        dxi = np.stack([np.einsum("qm,evm->eqv", Dmat[r], uu) for r in range(self.dim)], axis=2)
        return np.einsum("eprj,eprv->epjv", ginv, dxi)

    def face_states(self, g, u, t):
        """Interior/exterior traces, averages and jump on one face group."""
        QL = self.values(u, self.Bf[g["fL"]], g["eL"])
        dQL = self.gradients(u, self.Df[g["fL"]], g["ginvL"], g["eL"])
        if g["bctype"] is None:
            QR = self.values(u, self.Bf[g["fR"]], g["eR"])
            dQR = self.gradients(u, self.Df[g["fR"]], g["ginvR"], g["eR"])
            return QL, QR, 0.5 * (QL + QR), 0.5 * (dQL + dQR), dQL, dQR
        Qr, Qb, _ = phy.boundary_states(self.ph, g["bctype"], g["x"], t, QL, g["n"])
        return QL, Qr, Qb, dQL, dQL, None

    # ------------------------------------------------------ shock capturing
    def sensor(self, u):
        """Persson-Peraire modal-decay sensor (Sec. 3.1.2 cites it) per element:
        s_e = log10(|rho - Pi rho|^2 / |rho|^2), Pi the L2 projection of the
        density onto polynomials of degree <= P-1 per direction, both norms in
        the reference element (Gauss rule, exact for these degrees); S_e = 0 for
        s_e < s0 - kappa, 1 for s_e > s0 + kappa and (1 + sin(pi (s_e - s0) /
        (2 kappa))) / 2 between, s0 = log10(1/P^4)."""
        ph = self.ph
        rq = self.values(u[:, :1], self.B)[..., 0]                     # [E][q]
        dr = rq - rq @ self.sensor_proj.T
        num = np.einsum("q,eq->e", self.w, dr * dr)
        den = np.einsum("q,eq->e", self.w, rq * rq)
        with np.errstate(divide="ignore"):
            se = np.log10(num / den)
        s0, kap = np.log10(1.0 / self.P ** 4), ph.av_kappa
        ramp = 0.5 * (1.0 + np.sin(np.pi * np.clip(se - s0, -kap, kap) / (2.0 * kap)))
        return np.where(se < s0 - kap, 0.0, np.where(se > s0 + kap, 1.0, ramp))

    def av_factor(self, u):
        """mu_0 S_e h_e / P per element (h_e = |Omega_e|^(1/d)); zeros without
        shock capturing."""
        if not getattr(self.ph, "av", 0):
            return np.zeros(self.E)
        return self.ph.av_mu0 * self.sensor(u) * self.h_elem / self.P

    def face_av(self, g, fac, QL, QR, dQa):
        """Artificial viscosity at the face points: the mean of the two sides'
        values from their own traces (a boundary face: the interior side's);
        with av = 2 times Ducros' sensor of the face-average gradient dQa at the
        mean trace state (a boundary face: the interior trace)."""
        aL = phy.artificial_viscosity(QL, fac[g["eL"]][:, None], self.ph)
        if g["bctype"] is None:
            a = 0.5 * (aL + phy.artificial_viscosity(QR, fac[g["eR"]][:, None], self.ph))
            Qm = 0.5 * (QL + QR)
        else:
            a, Qm = aL, QL
        if getattr(self.ph, "av", 0) == 2:
            a = a * phy.ducros(Qm, dQa, self.ph)
        return a

    def volume_av(self, fac, Qv, dQ):
        """Artificial viscosity at the volume points (av = 2: times Ducros'
        sensor of the point's gradient)."""
        a = phy.artificial_viscosity(Qv, fac[:, None], self.ph)
        if getattr(self.ph, "av", 0) == 2:
            a = a * phy.ducros(Qv, dQ, self.ph)
        return a

    def face_flux(self, g, QL, QR, Qa, dQa, t, mu_av=None):
        """Numerical normal flux H^n = F^n - G^n and symmetric fluxes S_j on the
        face points of group g (owner-side normal).  QR is the exterior state
        of the Riemann flux and Qa the state of the viscous flux; the jump is
        Q_L - Q_R on interior faces and Q_L - Q_b on boundary faces.  mu_av:
        artificial viscosity at the face points (None: none)."""
        n = g["n"]
        Fh = phy.riemann_flux(QL, QR, n, self.ph)
        if not self.ph.viscous:
            return Fh, None
        jump = QL - (QR if g["bctype"] is None else Qa)
        S = phy.viscous_flux(Qa, n[..., :, None] * jump[..., None, :], self.ph, mu_av)   # [f][p][i][v]
        Gv = phy.viscous_flux(Qa, dQa, self.ph, mu_av) - g["beta"][:, None, None, None] * S
        Gh = np.einsum("fpi,fpiv->fpv", n, Gv)
        if g["bctype"] == phy.BC_ADIA_WALL:
            Gh[..., -1] = 0.0
            S[..., -1] = 0.0
        return Fh - Gh, S

    def lift_S(self, S, wJ, Dmat, ginv):
        """sum_i integral d_i phi * S_i over face points -> [f][v][m]."""
        T = np.einsum("fprj,fpjv->fprv", ginv, S * wJ[..., None, None])
        return sum(np.einsum("pm,fpv->fvm", Dmat[r], T[:, :, r]) for r in range(self.dim))

    # --------------------------------------------------------------- operator
    def rhs(self, u, t=0.0, faces=True):
        """L(u, t) of Eq. ode, [E][v][m] (faces=False: the volume term only)."""
        ph = self.ph
        Qv = self.values(u, self.B)
        dQ = self.gradients(u, self.D, self.ginv)
        av = getattr(ph, "av", 0)
        fac = self.av_factor(u) if av else None
        H = phy.euler_flux(Qv, ph)
        if ph.viscous:
            mu_q = self.volume_av(fac, Qv, dQ) if av else None
            H = H - phy.viscous_flux(Qv, dQ, ph, mu_q)
        Ht = np.einsum("eqrj,eqjv->eqrv", self.ginv, H) * self.wJ[:, :, None, None]
        L = sum(np.einsum("qm,eqv->evm", self.D[r], Ht[:, :, r]) for r in range(self.dim))
        for g in (self.groups if faces else []):
            QL, QR, Qa, dQa, _, _ = self.face_states(g, u, t)
            mu_f = self.face_av(g, fac, QL, QR, dQa) if av else None
            Hh, S = self.face_flux(g, QL, QR, Qa, dQa, t, mu_f)
            wJ = g["wJ"]
            L[g["eL"]] -= np.einsum("pm,fpv->fvm", self.Bf[g["fL"]], Hh * wJ[..., None])
            c = (0.5 if g["bctype"] is None else 1.0) * ph.beta_s
            if S is not None:
                L[g["eL"]] += c * self.lift_S(S, wJ, self.Df[g["fL"]], g["ginvL"])
            if g["bctype"] is None:
                L[g["eR"]] += np.einsum("pm,fpv->fvm", self.Bf[g["fR"]], Hh * wJ[..., None])
                if S is not None:
                    L[g["eR"]] += c * self.lift_S(S, wJ, self.Df[g["fR"]], g["ginvR"])
        if ph.forcing and faces:
            f = phy.forcing(ph, self.x, t)
            L += np.einsum("qm,eqv->evm", self.B, f * self.wJ[..., None])
        return L

    def apply_minv(self, L):
        return np.einsum("emn,evn->evm", self.Minv, L)

    def residual(self, u, t=0.0):
        """R(u, t) = M^-1 L(u, t): the right-hand side of M du/dt = L."""
        return self.apply_minv(self.rhs(u, t))

    # ------------------------------------------------------------- utilities
    def project(self, fn, t=0.0):
        """L2 projection of a pointwise field fn(x) -> [..., nv] onto V^P."""
        U = fn(self.x)
        b = np.einsum("qm,eqv->evm", self.B, U * self.wJ[..., None])
        return self.apply_minv(b)

    def project_exact(self, t=0.0):
        return self.project(lambda x: phy.exact_state(self.ph, x, t))

    def l2_error(self, u, fn):
        """Per-variable L2 norm of (u_h - fn) over the mesh."""
        diff = self.values(u, self.B) - fn(self.x)
        return np.sqrt(np.einsum("eq,eqv->v", self.wJ, diff * diff))

    def integral(self, L):
        """Integral of the function whose weak right-hand side is L: sum over
        elements of 1^T L (the test function phi = 1 is the sum of the vertex
        modes for the modified basis and of all modes for the nodal basis)."""
        return np.einsum("evm,m->v", L, self.one_coeffs())

    def one_coeffs(self):
        """Coefficients of the constant function 1 in the basis."""
        c = np.linalg.lstsq(self.B, np.ones(self.nq), rcond=None)[0]
        return c
