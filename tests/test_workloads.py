"""The seeded synthetic workloads have the shapes of the configurations they
stand for: element counts, domains, periodicity, boundary tags, spacing laws
and quadrature counts (Gauss points ceil(3(P+1)/2) for the 3-D cases, P+2
for the 2-D ones)."""
import numpy as np
import pytest

import workloads as w


def boundary_tags(mesh):
    F = mesh.faces
    tags, counts = np.unique(F[F[:, 2] < 0, 5], return_counts=True)
    return dict(zip(tags.tolist(), counts.tolist()))


def test_vortex_unit_square_periodic():
    c = w.vortex_case(n=8, P=2)
    m = c.mesh
    assert (m.dim, m.n_elem, c.P, c.Q) == (2, 64, 2, 4)
    assert np.all(m.faces[:, 2] >= 0)                  # no boundary: periodic both ways
    assert m.n_faces == 2 * 64
    assert m.nodes.min() == 0.0 and m.nodes.max() == 1.0
    assert (c.phys.Ma, c.phys.Re) == (0.1, 100.0)


@pytest.mark.parametrize("P", [1, 3, 6])
def test_poiseuille_channel_wall_clustered(P):
    c = w.poiseuille_case(P)
    m = c.mesh
    assert (m.dim, m.n_elem, c.Q) == (2, 128, P + 2)
    x = np.unique(np.round(m.nodes[..., 0], 12))
    y = np.unique(np.round(m.nodes[..., 1], 12))
    assert len(x) == 17 and x[0] == 0.0 and x[-1] == 2.0
    assert len(y) == 9 and y[0] == 0.0 and y[-1] == 1.0
    h = np.diff(y)
    np.testing.assert_allclose(h[1:4] / h[:3], 1.1, rtol=1e-9)         # growth away from y = 0
    np.testing.assert_allclose(h[::-1], h, rtol=1e-9)                  # symmetric about y = 1/2
    tags = boundary_tags(m)
    assert tags == {0: 16, 1: 32}                                      # x ends (Dirichlet), walls
    assert c.phys.bc[0] == w.BC_DIRICHLET and c.phys.bc[1] == w.BC_ISO_WALL
    assert (c.phys.Ma, c.phys.Re) == (0.2, 100.0)


@pytest.mark.parametrize("n,P,Q,E", [(16, 3, 6, 4096), (24, 4, 8, 13_824)])
def test_taylor_green_boxes(n, P, Q, E):
    c = w.tgv_case(n, P)
    m = c.mesh
    assert (m.dim, m.n_elem, c.P, c.Q) == (3, E, P, Q)
    assert np.all(m.faces[:, 2] >= 0) and m.n_faces == 3 * E
    np.testing.assert_allclose([m.nodes.min(), m.nodes.max()], [-np.pi, np.pi], rtol=0, atol=1e-15)
    assert (c.phys.Ma, c.phys.Re) == (0.1, 1600.0)
    # degrees of freedom of the configuration
    assert E * 5 * (P + 1) ** 3 == {3: 1_310_720, 4: 8_640_000}[P]


def test_cylinder_ogrid():
    c = w.cylinder_case()
    m = c.mesh
    assert (m.dim, m.geom_order, m.n_elem, c.P, c.Q) == (3, 2, 64 * 96 * 12, 3, 6)
    assert m.nodes.shape == (73_728, 27, 3)
    assert m.n_elem * 5 * 64 == 23_592_960
    r = np.hypot(m.nodes[..., 0], m.nodes[..., 1])
    np.testing.assert_allclose([r.min(), r.max()], [0.5, 20.0], rtol=1e-14)
    z = m.nodes[..., 2]
    np.testing.assert_allclose([z.min(), z.max()], [0.0, np.pi], rtol=0, atol=1e-15)
    # vertex radii: 65 lines growing by 1.08 (quadratic nodes add the midpoints)
    radii = np.unique(np.round(r, 10))
    assert len(radii) == 2 * 64 + 1
    rv = radii[::2]
    np.testing.assert_allclose(np.diff(rv)[1:] / np.diff(rv)[:-1], 1.08, rtol=1e-8)
    np.testing.assert_allclose(radii[1::2], 0.5 * (rv[1:] + rv[:-1]), rtol=1e-9)
    # one wall face and one far-field face per (azimuthal, spanwise) cell
    assert boundary_tags(m) == {0: 96 * 12, 1: 96 * 12}
    assert c.phys.bc[0] == w.BC_ADIA_WALL and c.phys.bc[1] == w.BC_FARFIELD
    assert (c.phys.Ma, c.phys.Re) == (0.2, 3900.0)
