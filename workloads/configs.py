"""Physical parameters and meshes of the synthetic workloads.

Every workload is defined by a mesh, a Physics record and an analytic field
id; the analytic formulas themselves (initial fields, exact solutions,
forcing) are implemented separately by the oracle and by the CUDA library.
"""
from dataclasses import dataclass, field as dc_field
import numpy as np
from .mesh import box_mesh, clustered_spacing, mapped_box_mesh, ogrid_mesh

# boundary-condition types (entry of the per-boundary table)
BC_PERIODIC = 0      # never in the table: periodic faces are interior faces
BC_DIRICHLET = 1     # weak Dirichlet state from the workload's exact solution
BC_ISO_WALL = 2      # isothermal no-slip wall, T from the exact solution
BC_ADIA_WALL = 3     # adiabatic no-slip wall
BC_FARFIELD = 4      # characteristic (Riemann-invariant) far field

# analytic fields
FIELD_UNIFORM = 0
FIELD_VORTEX = 1
FIELD_POISEUILLE = 2
FIELD_TGV = 3
FIELD_CYLINDER = 4   # uniform stream (1, 0, 0) at T = 1, rho = 1
FIELD_SHOCK = 5      # oblique shock: stream (1, 0) below the shock line, post-shock state above
# FIELD_UNIFORM is the uniform state fpar = (rho, u, v, w, T), or the stream
# (1, 1, 0, 0, 1) when fpar is empty

RIEMANN_ROE = 0
RIEMANN_HLLC = 1
RIEMANN_HLL = 2
RIEMANN_LF = 3       # local Lax-Friedrichs (Rusanov)
RIEMANN_AUSM = 4
FORCING_NONE = 0
FORCING_POISEUILLE = 1


@dataclass
class Physics:
    gamma: float = 1.4
    Pr: float = 0.72
    Ma: float = 0.1
    Re: float = 100.0
    viscous: bool = True
    mu_law: int = 0            # 0 constant mu = 1/Re, 1 Sutherland
    T_inf_K: float = 288.15    # reference temperature for Sutherland's law
    riemann: int = RIEMANN_ROE
    beta_s: float = 1.0
    forcing: int = FORCING_NONE
    fid: int = FIELD_UNIFORM   # analytic field id
    # field parameters (vortex: u0, v0, phi, xc, yc, scale;
    # Poiseuille: theta, L, dpdx; uniform: rho, u, v, w, T)
    fpar: tuple = ()
    bc: list = dc_field(default_factory=list)   # bc[id] = type
    av: int = 0                # shock capturing: 1 modal sensor, 2 modal sensor x Ducros
    av_mu0: float = 0.25       # mu_0 of Sec. 3.1.2
    av_kappa: float = 1.0      # half-width of the sensor's ramp (decades)

    @property
    def mu(self):
        return 1.0 / self.Re


@dataclass
class Case:
    name: str
    mesh: object
    P: int
    Q: int
    phys: Physics


def vortex_case(n=8, P=2, Q=None, Ma=0.1, Re=100.0, viscous=True, riemann=RIEMANN_ROE):
    """Isentropic vortex on the periodic unit square, n x n quads."""
    Q = P + 2 if Q is None else Q
    lines = [np.linspace(0.0, 1.0, n + 1)] * 2
    m = box_mesh(lines, (True, True))
    ph = Physics(Ma=Ma, Re=Re, viscous=viscous, riemann=riemann, fid=FIELD_VORTEX,
                 fpar=(1.0, 0.5, 5.0, 0.5, 0.5, 10.0))
    return Case(f"vortex{n}x{n}_P{P}", m, P, Q, ph)


def poiseuille_case(P, nx=16, ny=8, ratio=1.1, Q=None, Ma=0.2, Re=100.0, theta=0.01,
                    x_bc=BC_DIRICHLET, y_bc=BC_ISO_WALL):
    """Manufactured compressible Poiseuille channel [0,2]x[0,1], wall-clustered
    in y (geometric ratio from each wall), Dirichlet at x = 0, 2 and
    isothermal walls at y = 0, 1."""
    Q = P + 2 if Q is None else Q
    xl = np.linspace(0.0, 2.0, nx + 1)
    yl = clustered_spacing(ny // 2, ratio, 1.0)
    m = box_mesh([xl, yl], (False, False), side_bc=[0, 0, 1, 1])
    mu = 1.0 / Re
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_POISEUILLE, forcing=FORCING_POISEUILLE,
                 fpar=(theta, 1.0, -8.0 * mu), bc=[x_bc, y_bc])
    return Case(f"poiseuille{nx}x{ny}_P{P}", m, P, Q, ph)


def tgv_case(n=16, P=3, Q=None, Re=1600.0, Ma=0.1, riemann=RIEMANN_ROE):
    """Taylor-Green vortex on the periodic box [-pi, pi]^3, n^3 hexes."""
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    lines = [np.linspace(-np.pi, np.pi, n + 1)] * 3
    m = box_mesh(lines, (True, True, True))
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_TGV, riemann=riemann)
    return Case(f"tgv{n}^3_P{P}", m, P, Q, ph)


def tgv_dt(n, P, Ma, cfl=0.10, factor=10.0):
    """Time step of the Taylor-Green workloads: factor x the explicit step of
    Eq. CFL (c_lambda = 0.2, d_RK = 2) at the given CFL on n^3 elements of the
    periodic box [-pi, pi]^3, with c + |u| = 1/Ma + 1 (T = 1, |u| <= 1)."""
    dx = 2 * np.pi / n
    return factor * cfl * 2.0 * dx / (0.2 * (1.0 / Ma + 1.0) * P * P)


def small_tgv_case(shape=(4, 3, 2), P=2, Q=None, Re=1600.0, Ma=0.1, riemann=RIEMANN_ROE,
                   stretch=False):
    """A small periodic 3-D box with an anisotropic element count (and
    optionally non-uniform spacing), used for parity cases."""
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    lines = []
    for r, n in enumerate(shape):
        l = np.linspace(-np.pi, np.pi, n + 1)
        if stretch:
            s = np.linspace(0, 1, n + 1)
            l = -np.pi + 2 * np.pi * (s + 0.08 * np.sin(2 * np.pi * s) * (r + 1) / 3)
        lines.append(l)
    m = box_mesh(lines, (True, True, True))
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_TGV, riemann=riemann)
    return Case(f"box{shape}_P{P}", m, P, Q, ph)


def cylinder_case(n_r=64, n_theta=96, n_z=12, P=3, Q=None, Re=3900.0, Ma=0.2, wall_layer=0.0):
    """Curved O-grid around a unit-diameter cylinder (radius 0.5), outer
    radius 20, radial growth 1.08, span pi: adiabatic wall and far field.
    wall_layer > 0 brings the initial stream to rest at the wall over that
    length (the far-field state is the undisturbed stream)."""
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    m = ogrid_mesh(n_r, n_theta, n_z, 0.5, 20.0, 1.08, np.pi)
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_CYLINDER, bc=[BC_ADIA_WALL, BC_FARFIELD],
                 fpar=(0.5, wall_layer))
    return Case(f"cylinder{n_r}x{n_theta}x{n_z}_P{P}", m, P, Q, ph)


def wavy_box_case(shape=(3, 3, 2), P=2, Q=None, amp=0.12, Re=1600.0, Ma=0.1,
                  riemann=RIEMANN_ROE):
    """Periodic box [-pi, pi]^3 on quadratic hexes whose nodes are displaced by
    a smooth periodic field (every element curved, faces conforming), with the
    Taylor-Green field."""
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    lines = [np.linspace(-np.pi, np.pi, n + 1) for n in shape]

    def wave(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return np.stack([x + amp * np.sin(y) * np.sin(z),
                         y + amp * np.sin(z + 0.5) * np.sin(x),
                         z + amp * np.sin(x) * np.sin(y + 0.3)], -1)

    m = mapped_box_mesh(lines, (True, True, True), wave, order=2)
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_TGV, riemann=riemann)
    return Case(f"wavy{shape}_P{P}", m, P, Q, ph)


def rotation_matrix(dim, angles=(0.5, -0.3, 0.8)):
    """A proper rotation: about z in 2-D; z-y-x Euler angles in 3-D."""
    a, b, c = angles
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    if dim == 2:
        return Rz[:2, :2]
    Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, np.cos(c), -np.sin(c)], [0, np.sin(c), np.cos(c)]])
    return Rz @ Ry @ Rx


def rotated_box_case(shape=(3, 2, 2), P=2, Q=None, order=1, Re=1600.0, Ma=0.1,
                     riemann=RIEMANN_ROE):
    """The periodic box of small_tgv_case rigidly rotated (straight-sided
    elements with non-diagonal metrics; order 2 writes the same elements with
    27 nodes)."""
    dim = len(shape)
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    lines = [np.linspace(-np.pi, np.pi, n + 1) for n in shape]
    R = rotation_matrix(dim)
    m = mapped_box_mesh(lines, (True,) * dim, lambda X: X @ R.T, order=order)
    m.meta["rotation"] = R
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_TGV if dim == 3 else FIELD_UNIFORM, riemann=riemann)
    return Case(f"rotated{shape}_P{P}_g{order}", m, P, Q, ph)


def small_cylinder_case(n_r=3, n_theta=8, n_z=2, P=2, Q=None, Re=3900.0, Ma=0.2,
                        r_out=3.0, bc=(BC_ADIA_WALL, BC_FARFIELD), wall_layer=0.0):
    """A coarse O-grid (radius 0.5 to r_out) with the cylinder workload's
    boundary conditions, for parity cases."""
    Q = int(np.ceil(3 * (P + 1) / 2)) if Q is None else Q
    m = ogrid_mesh(n_r, n_theta, n_z, 0.5, r_out, 1.08, np.pi)
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_CYLINDER, bc=list(bc), fpar=(0.5, wall_layer))
    return Case(f"cylinder{n_r}x{n_theta}x{n_z}_P{P}", m, P, Q, ph)


def wall_spacing(n, ratio, length=1.0):
    """Grid lines on [0, length] with n cells growing geometrically by `ratio`
    away from 0 (one wall)."""
    h = ratio ** np.arange(n)
    return np.concatenate([[0.0], np.cumsum(h)]) / h.sum() * length


def swbli_case(nx=119, ny=39, P=3, Q=None, Ma=2.15, Re=1.0e5, beta_deg=30.8, x0=0.3, x1=2.0,
               height=1.0, ratio=1.1, av=1, riemann=RIEMANN_ROE, shock_width=0.02,
               wall_layer=0.01):
    """Shock-wave / boundary-layer interaction of the kind of Sec. 6.5: an
    oblique shock of angle beta_deg (to the stream) generated above the plate
    reaches the adiabatic no-slip wall y = 0 at x = 1 (the unit length, on
    which Re is based); the domain [x0, x1] x [0, height] (nx x ny quads,
    spacing growing by `ratio` away from the wall), the uniform stream at Ma
    below the shock line and the Rankine-Hugoniot state above it imposed on
    the inflow (x = x0) and top sides, a characteristic far-field outflow,
    the artificial-viscosity shock capturing of Sec. 3.1.2 (av = 1).  The field
    (initial state and boundary data) passes through the shock over
    `shock_width` and has the velocity brought to rest at the wall over
    `wall_layer` (0: a sharp jump, a uniform stream down to the wall)."""
    Q = P + 2 if Q is None else Q
    xl = np.linspace(x0, x1, nx + 1)
    yl = wall_spacing(ny, ratio, height)
    m = box_mesh([xl, yl], (False, False), side_bc=[0, 1, 2, 0])
    ph = Physics(Ma=Ma, Re=Re, fid=FIELD_SHOCK, fpar=(beta_deg, 1.0, shock_width, wall_layer),
                 bc=[BC_DIRICHLET, BC_FARFIELD, BC_ADIA_WALL], av=av, riemann=riemann)
    return Case(f"swbli{nx}x{ny}_P{P}", m, P, Q, ph)

