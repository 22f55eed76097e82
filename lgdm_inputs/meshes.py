"""Structured meshes in the layout the LGDM library takes.

Conventions (shared by both sides, so that fields indexed by element, node or
Gauss point line up):

* Nodes carry ``d`` displacement dofs and one micro-equivalent-strain dof,
  interleaved per node: dof ``nd*a + i`` with ``nd = d + 1``; ``i < d`` are
  displacements, ``i == d`` is the micro-equivalent strain.
* Coordinates are SoA float64 arrays ``x, y, z`` in mm (unused ones are None).
* ``conn`` is int32 ``[nel, nen]``, element-major.  Local node order: 2-node
  bar left→right; 4-node quad counter-clockwise from the (-1,-1) corner;
  8-node hex the bottom face (zeta=-1) counter-clockwise, then the top face;
  3-node bar: the two ends, then the middle; 9-node quad: the four corners
  as the 4-node quad, the mid-side nodes of the edges xi2=-1, xi1=+1, xi2=+1,
  xi1=-1, then the centre.  The vertex nodes come first in every element.
* ``e_scale[e]`` multiplies the elasticity tensor only (a notch is 1e-6);
  ``vol_scale[e]`` multiplies the integration measure (bar cross-section,
  plate thickness).
"""
from dataclasses import dataclass
from typing import Optional

import numpy as np

L2, Q4, H8, L3, Q9 = 1, 2, 3, 4, 5   # element type codes, same values as the C ABI
NEN = {L2: 2, Q4: 4, H8: 8, L3: 3, Q9: 9}
DIM = {L2: 1, Q4: 2, H8: 3, L3: 1, Q9: 2}


@dataclass
class Mesh:
    elem: int
    x: np.ndarray
    y: Optional[np.ndarray]
    z: Optional[np.ndarray]
    conn: np.ndarray
    e_scale: np.ndarray
    vol_scale: np.ndarray
    shape: tuple = ()           # element counts per axis, for reporting only

    @property
    def dim(self) -> int:
        return DIM[self.elem]

    @property
    def nen(self) -> int:
        return NEN[self.elem]

    @property
    def ngp(self) -> int:
        return NEN[self.elem]   # 2, 2x2, 2x2x2 (linear), 3, 3x3 (quadratic) Gauss points

    @property
    def nd(self) -> int:
        return self.dim + 1

    @property
    def nnode(self) -> int:
        return int(self.x.shape[0])

    @property
    def nel(self) -> int:
        return int(self.conn.shape[0])

    @property
    def ndof(self) -> int:
        return self.nd * self.nnode

    def coords(self) -> np.ndarray:
        cols = [self.x] + [c for c in (self.y, self.z) if c is not None]
        return np.stack(cols[: self.dim], axis=1)


def node_dofs(mesh: Mesh, nodes: np.ndarray, comp: int) -> np.ndarray:
    """Global dof numbers of component ``comp`` at ``nodes`` (interleaved)."""
    return (mesh.nd * np.asarray(nodes, dtype=np.int64) + comp).astype(np.int32)


def bar_l2(n: int, length: float, area: float) -> Mesh:
    x = np.linspace(0.0, length, n + 1)
    conn = np.stack([np.arange(n), np.arange(1, n + 1)], axis=1).astype(np.int32)
    return Mesh(L2, x, None, None, conn, np.ones(n), np.full(n, float(area)), (n,))


def bar_l3(n: int, length: float, area: float) -> Mesh:
    """n 3-node elements; node 2e is the left end of element e, 2e+1 its middle."""
    x = np.linspace(0.0, length, 2 * n + 1)
    e = np.arange(n)
    conn = np.stack([2 * e, 2 * e + 2, 2 * e + 1], axis=1).astype(np.int32)
    return Mesh(L3, x, None, None, conn, np.ones(n), np.full(n, float(area)), (n,))


def plate_q9(nx: int, ny: int, lx: float, ly: float, thickness: float = 1.0) -> Mesh:
    """nx x ny 9-node elements on a (2nx+1) x (2ny+1) node grid (node id =
    J*(2nx+1) + I); element j*nx + i has its corners at grid (2i, 2j) .. (2i+2, 2j+2)."""
    gx, gy = 2 * nx + 1, 2 * ny + 1
    xs = np.linspace(0.0, lx, gx)
    ys = np.linspace(0.0, ly, gy)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    I, J = (2 * i).ravel(), (2 * j).ravel()

    def nid(di, dj):
        return (J + dj) * gx + I + di

    conn = np.stack([nid(0, 0), nid(2, 0), nid(2, 2), nid(0, 2),
                     nid(1, 0), nid(2, 1), nid(1, 2), nid(0, 1), nid(1, 1)], axis=1).astype(np.int32)
    nel = nx * ny
    return Mesh(Q9, X.ravel().copy(), Y.ravel().copy(), None, conn,
                np.ones(nel), np.full(nel, float(thickness)), (nx, ny))


def plate_q4(nx: int, ny: int, lx: float, ly: float, thickness: float = 1.0) -> Mesh:
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")        # node id = j*(nx+1) + i
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    n0 = (j * (nx + 1) + i).ravel()                  # element id = j*nx + i
    conn = np.stack([n0, n0 + 1, n0 + nx + 2, n0 + nx + 1], axis=1).astype(np.int32)
    nel = nx * ny
    return Mesh(Q4, X.ravel().copy(), Y.ravel().copy(), None, conn,
                np.ones(nel), np.full(nel, float(thickness)), (nx, ny))


def beam_h8(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float) -> Mesh:
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")  # node id = (k*(ny+1)+j)*(nx+1)+i
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sxy = 1, (nx + 1)
    sz = (nx + 1) * (ny + 1)
    n0 = ((k * (ny + 1) + j) * (nx + 1) + i).ravel()  # element id = (k*ny+j)*nx+i
    bottom = [n0, n0 + sx, n0 + sx + sxy, n0 + sxy]
    top = [b + sz for b in bottom]
    conn = np.stack(bottom + top, axis=1).astype(np.int32)
    nel = nx * ny * nz
    return Mesh(H8, X.ravel().copy(), Y.ravel().copy(), Z.ravel().copy(), conn,
                np.ones(nel), np.ones(nel), (nx, ny, nz))
