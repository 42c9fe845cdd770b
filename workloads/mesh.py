"""Structured quad/hex meshes described as element nodes plus a face table.

Layout (shared with the C ABI `dg_mesh_desc`):
  nodes[e][a][x]   geometry nodes of element e, a = tensor index of the
                   (g+1)^d equispaced reference nodes (first direction fastest),
                   x = physical coordinate; g = 1 (affine) or 2 (quadratic).
  faces[f] = (eL, fL, eR, fR, orient, bc)
                   local face 2r is xi_r = -1, 2r+1 is xi_r = +1; eR = fR = -1
                   and bc >= 0 (index into the boundary table) on a physical
                   boundary, bc = -1 on interior and periodic faces; the face
                   points of both sides coincide point by point (orient = 0).
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class Mesh:
    dim: int
    geom_order: int
    nodes: np.ndarray           # float64 [E][(g+1)^d][dim]
    faces: np.ndarray           # int32   [F][6]
    shape: tuple = ()           # elements per direction (structured generators)
    periodic: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def n_elem(self):
        return int(self.nodes.shape[0])

    @property
    def n_faces(self):
        return int(self.faces.shape[0])


def clustered_spacing(n_half, ratio, length=1.0):
    """Grid lines on [0, length] with 2*n_half cells, geometric growth `ratio`
    away from both ends (wall clustering), symmetric about the centre."""
    h = ratio ** np.arange(n_half)
    half = np.concatenate([[0.0], np.cumsum(h)])
    half = half / half[-1] * (0.5 * length)
    return np.concatenate([half, length - half[::-1][1:]])


def _faces_structured(shape, periodic, side_bc):
    dim = len(shape)
    idx = np.arange(int(np.prod(shape))).reshape(shape[::-1])  # [k][j][i]
    faces = []
    for r in range(dim):
        ax = dim - 1 - r  # numpy axis of direction r
        n = shape[r]
        for e in idx.flat:
            pos = np.unravel_index(e, idx.shape)
            c = pos[ax]
            # face on the +r side of e
            if c + 1 < n or periodic[r]:
                nb = list(pos)
                nb[ax] = (c + 1) % n
                faces.append((e, 2 * r + 1, int(idx[tuple(nb)]), 2 * r, 0, -1))
            else:
                faces.append((e, 2 * r + 1, -1, -1, 0, side_bc[2 * r + 1]))
            if c == 0 and not periodic[r]:
                faces.append((e, 2 * r, -1, -1, 0, side_bc[2 * r]))
    return np.asarray(faces, dtype=np.int32)


def box_mesh(lines, periodic, side_bc=None):
    """Axis-aligned affine quads (2-D) / hexes (3-D) on the tensor grid given by
    `lines` (one coordinate array per direction)."""
    dim = len(lines)
    shape = tuple(len(l) - 1 for l in lines)
    if side_bc is None:
        side_bc = [-1] * (2 * dim)
    E = int(np.prod(shape))
    nodes = np.zeros((E, 2 ** dim, dim))
    for e in range(E):
        c = np.unravel_index(e, shape[::-1])[::-1]  # (i, j[, k])
        for a in range(2 ** dim):
            bits = [(a >> r) & 1 for r in range(dim)]
            for r in range(dim):
                nodes[e, a, r] = lines[r][c[r] + bits[r]]
    faces = _faces_structured(shape, periodic, side_bc)
    return Mesh(dim, 1, nodes, faces, shape, tuple(periodic))


def mapped_box_mesh(lines, periodic, fn, order=2, side_bc=None):
    """The tensor grid of `lines` with every element's (order+1)^d equispaced
    reference nodes sent through the point map `fn` (x[..., d] -> x[..., d]).
    Neighbours evaluate fn at the same points of a shared face, so the faces
    stay conforming; with a map whose displacement is periodic the periodic
    faces match too.  order = 1 with a linear fn gives straight-sided
    (possibly rotated or sheared) elements."""
    dim = len(lines)
    shape = tuple(len(l) - 1 for l in lines)
    if side_bc is None:
        side_bc = [-1] * (2 * dim)
    E = int(np.prod(shape))
    na = (order + 1) ** dim
    cell = np.stack(np.unravel_index(np.arange(E), shape[::-1])[::-1], -1)      # [E][d] (i, j[, k])
    a = np.stack(np.unravel_index(np.arange(na), (order + 1,) * dim)[::-1], -1)  # [na][d]
    X = np.zeros((E, na, dim))
    for r in range(dim):
        lo = lines[r][cell[:, r]]
        hi = lines[r][cell[:, r] + 1]
        X[:, :, r] = lo[:, None] + (hi - lo)[:, None] * a[None, :, r] / order
    nodes = fn(X)
    faces = _faces_structured(shape, periodic, side_bc)
    return Mesh(dim, order, nodes, faces, shape, tuple(periodic))


def ogrid_mesh(n_r, n_theta, n_z, r_in, r_out, ratio, span):
    """Quadratic (27-node) hexes of an O-grid around a cylinder of radius r_in:
    direction 0 = radial (geometric growth `ratio`), 1 = azimuthal (periodic),
    2 = spanwise (periodic).  Side 0 (r = r_in) is boundary 0 (wall), side 1
    (r = r_out) is boundary 1 (far field)."""
    h = ratio ** np.arange(n_r)
    rl = r_in + (r_out - r_in) * np.concatenate([[0.0], np.cumsum(h)]) / h.sum()
    tl = np.linspace(0.0, 2 * np.pi, n_theta + 1)
    zl = np.linspace(0.0, span, n_z + 1)

    def polar(X):
        r, th, z = X[..., 0], X[..., 1], X[..., 2]
        return np.stack([r * np.cos(th), r * np.sin(th), z], -1)

    m = mapped_box_mesh([rl, tl, zl], (False, True, True), polar, order=2,
                        side_bc=[0, 1, -1, -1, -1, -1])
    return m
