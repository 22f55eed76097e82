"""Problem definitions: material, Dirichlet lists, load schedules, random states.

The three single-simulation workloads mirror the paper's 1D bar, 2D notched
plate and 3D notched specimen (Sec. 3.1-3.3) at the sizes and parameters of the
benchmark configurations; the batch and serving draws add the seeded variety
those configurations ask for.  Readings applied here (boundary lines, notch
placement, weak element, h = 1e-9 E) are listed with the design notes.
"""
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .meshes import Mesh, bar_l2, bar_l3, plate_q4, plate_q9, beam_h8, node_dofs


@dataclass
class Material:
    E: float = 20000.0          # MPa
    nu: float = 0.2
    k: float = 10.0             # compressive/tensile strength ratio (Eq. A.3)
    kappa0: float = 1e-4        # damage threshold (Eq. A.1)
    alpha: float = 0.99
    beta: float = 300.0
    R: float = 0.005            # residual interaction (Eq. A.4)
    eta: float = 5.0            # interaction exponent "n" (Eq. A.4)
    c: float = 4.0              # gradient parameter, mm^2
    h: Optional[float] = None   # coupling modulus; None -> 1e-9 * E
    evm_variant: int = 0        # 0: de Vree coefficients, 1: literal print
    h_stress: int = 0           # 0: stress without the h-term, 1: Eq. 2 literal (with it)

    def __post_init__(self):
        if self.h is None:
            self.h = 1e-9 * self.E


@dataclass
class BCs:
    """Displacement control: u[dir_dof[i]] = dir_scale[i] * load_param.

    The reaction is sum_i dir_scale[i] * r_u[dir_dof[i]], the generalized force
    conjugate to the load parameter (supports have scale 0 and drop out).
    """
    dir_dof: np.ndarray
    dir_scale: np.ndarray


@dataclass
class Problem:
    name: str
    mesh: Mesh
    material: Material
    bcs: BCs
    u_max: float
    n_steps: int
    newton_tol: float = 1e-8
    max_newton: int = 50
    max_halvings: int = 6

    def load(self, step: int) -> float:
        return self.u_max * step / self.n_steps


def _bcs(pairs):
    dofs = np.concatenate([p[0] for p in pairs]).astype(np.int32)
    scale = np.concatenate([np.full(len(p[0]), float(p[1])) for p in pairs])
    return BCs(dofs, scale)


def bar_problem(n: int = 100, length: float = 100.0, area: float = 10.0,
                weak_factor: float = 0.9, u_max: float = 0.02, n_steps: int = 200,
                material: Optional[Material] = None, order: int = 1,
                weak_span: Optional[tuple] = None) -> Problem:
    """1D bar in tension.  The middle element (0-based n//2) has a weaker
    section, or, with ``weak_span`` = (x0, x1), every element whose centre
    lies in it.  order 1: 2-node elements for both fields; order 2: 3-node
    quadratic u with linear micro-equivalent strain."""
    mesh = bar_l2(n, length, area) if order == 1 else bar_l3(n, length, area)
    if weak_span is None:
        mesh.vol_scale[n // 2] *= weak_factor
    else:
        xc = (np.arange(n) + 0.5) * length / n
        mesh.vol_scale[(xc > weak_span[0]) & (xc < weak_span[1])] *= weak_factor
    mat = material or Material(E=20000.0, nu=0.0, k=1.0, c=4.0)
    right = n if order == 1 else 2 * n
    bcs = _bcs([(node_dofs(mesh, [0], 0), 0.0), (node_dofs(mesh, [right], 0), 1.0)])
    return Problem("bar1d" if order == 1 else "bar1d_l3", mesh, mat, bcs, u_max, n_steps)


def sen_plate_problem(nx: int = 200, ny: int = 200, lx: float = 100.0, ly: float = 100.0,
                      notch_frac: float = 0.5, u_max: float = 0.1, n_steps: int = 500,
                      material: Optional[Material] = None, order: int = 1) -> Problem:
    """Plane-strain single-edge-notched plate pulled at the top edge.

    Notch: element row ny//2, the first round(notch_frac*nx) elements from the
    left edge, elasticity scaled by 1e-6.  Bottom edge fixed in x and y; top
    edge u_y = load, u_x free; the micro-equivalent strain is free everywhere.
    order 1: 4-node elements for both fields; order 2: 9-node biquadratic u
    with bilinear micro-equivalent strain.
    """
    mesh = plate_q4(nx, ny, lx, ly) if order == 1 else plate_q9(nx, ny, lx, ly)
    jn = ny // 2
    nnotch = int(round(notch_frac * nx))
    mesh.e_scale[jn * nx + np.arange(nnotch)] = 1e-6
    row = order * nx + 1                          # nodes per grid row
    bottom = np.arange(row)
    top = order * ny * row + np.arange(row)
    mat = material or Material(c=1.0)
    bcs = _bcs([(node_dofs(mesh, bottom, 0), 0.0), (node_dofs(mesh, bottom, 1), 0.0),
                (node_dofs(mesh, top, 1), 1.0)])
    return Problem("sen_plate_q4" if order == 1 else "sen_plate_q9", mesh, mat, bcs, u_max, n_steps)


def paper_bar_problem(n: int = 1000, n_steps: int = 1000) -> Problem:
    """The paper's 1D bar (Sec. 3.1, Fig. 10): 3-node quadratic u, linear
    micro-equivalent strain, E = 1 GPa, h = 1e-9 E, kappa0 = 1e-4,
    c = 10 mm^2, alpha = 0.99, beta = 25, R = 0.005, n = 5; 0.02 mm in 1000
    steps on 500, 800 or 1000 elements.  Length, section and defect are not
    printed: 100 mm, 10 mm^2, and the section 0.9x over x in [49, 51] mm (a
    fixed physical defect, so the meshes converge)."""
    mat = Material(E=1000.0, nu=0.0, k=1.0, kappa0=1e-4, alpha=0.99, beta=25.0, R=0.005,
                   eta=5.0, c=10.0)
    p = bar_problem(n, 100.0, 10.0, 0.9, u_max=0.02, n_steps=n_steps, material=mat, order=2,
                    weak_span=(49.0, 51.0))
    p.name = "paper_bar_l3"
    return p


def paper_sen_plate_problem(n: int = 100, n_steps: int = 80) -> Problem:
    """The paper's 2D side-edge-notched specimen (Sec. 3.2): 9-node
    biquadratic u with bilinear micro-equivalent strain on n x n elements
    (50, 100 or 120), 80 equal load steps.  Fig. 15 (geometry and parameters)
    is not in the text: the plate of the notched-plate workload (100 mm
    square, half-width notch at mid-height, its material), pulled to 0.02 mm
    -- the printed 0.8 mm would put that plate's peak inside the first step."""
    p = sen_plate_problem(n, n, u_max=0.02 * n_steps / 80, n_steps=n_steps, order=2)
    p.name = "paper_sen_plate_q9"
    return p


def paper_sen_slab_problem(n: int = 50, nz: int = 5, thickness: float = 10.0, n_steps: int = 80) -> Problem:
    """The paper's 3D side-edge-notched specimen (Sec. 3.3): the 2D specimen
    extruded to 10 mm, trilinear 8-node elements for both fields, n x n x nz
    elements (50x50x5, 80x80x5, 100x100x5), 80 equal load steps.  Geometry,
    parameters and load (0.02 mm) as the 2D reading; the bottom face is fixed
    in x, y, z, the top face pulled in y; the notch runs through the thickness."""
    mesh = beam_h8(n, n, nz, 100.0, 100.0, thickness)
    nxp = n + 1
    k, j, i = np.meshgrid(np.arange(nz + 1), [0], np.arange(nxp), indexing="ij")
    bottom = ((k * nxp + j) * nxp + i).ravel()
    top = bottom + n * nxp
    kk, ii = np.meshgrid(np.arange(nz), np.arange(int(round(0.5 * n))), indexing="ij")
    notch = ((kk * n + n // 2) * n + ii).ravel()
    mesh.e_scale[notch] = 1e-6
    bcs = _bcs([(node_dofs(mesh, bottom, 0), 0.0), (node_dofs(mesh, bottom, 1), 0.0),
                (node_dofs(mesh, bottom, 2), 0.0), (node_dofs(mesh, top, 1), 1.0)])
    return Problem("paper_sen_slab_h8", mesh, Material(c=1.0), bcs, 0.02 * n_steps / 80, n_steps)


def tpb_beam_problem(nx: int = 200, ny: int = 40, nz: int = 40, lx: float = 200.0,
                     ly: float = 40.0, lz: float = 40.0, u_max: float = 0.5,
                     n_steps: int = 300, material: Optional[Material] = None) -> Problem:
    """Notched beam in three-point bending (x span, y width, z height).

    Supports: bottom lines (z=0) at x=0 and x=lx have u_z=0; the x=0 line also
    u_x=0; node (0,0,0) u_y=0.  Load: u_z = -load on the top line (z=lz) at
    node column nx//2.  Notch: element column nx//2, layers k < nz//2, all j.
    """
    mesh = beam_h8(nx, ny, nz, lx, ly, lz)
    nxp, nyp = nx + 1, ny + 1
    jj = np.arange(nyp)
    left = jj * nxp                             # k = 0, i = 0
    right = jj * nxp + nx                       # k = 0, i = nx
    load = nz * nxp * nyp + jj * nxp + nx // 2  # k = nz, i = nx//2
    k, j = np.meshgrid(np.arange(nz // 2), np.arange(ny), indexing="ij")
    notch = ((k * ny + j) * nx + nx // 2).ravel()
    mesh.e_scale[notch] = 1e-6
    mat = material or Material(c=4.0)
    bcs = _bcs([(node_dofs(mesh, left, 2), 0.0), (node_dofs(mesh, right, 2), 0.0),
                (node_dofs(mesh, left, 0), 0.0), (node_dofs(mesh, [0], 1), 0.0),
                (node_dofs(mesh, load, 2), -1.0)])
    return Problem("tpb_beam_h8", mesh, mat, bcs, u_max, n_steps)


def _plate_draw(rng: np.random.Generator, n_steps: int) -> Problem:
    n = int(round(np.exp(rng.uniform(np.log(20.0), np.log(300.0)))))
    frac = rng.uniform(0.2, 0.6)
    mat = Material(kappa0=rng.uniform(0.8e-4, 1.5e-4), beta=rng.uniform(200.0, 500.0),
                   eta=rng.uniform(3.0, 8.0), c=rng.uniform(0.5, 4.0))
    return sen_plate_problem(n, n, notch_frac=frac, u_max=0.1, n_steps=n_steps, material=mat)


def batch_plate_problems(seed: int = 3, count: int = 256, n_steps: int = 300) -> List[Problem]:
    """Uneven batch of notched plates: edge count log-uniform in [20, 300]."""
    rng = np.random.default_rng(seed)
    return [_plate_draw(rng, n_steps) for _ in range(count)]


@dataclass
class Request:
    arrival: float               # seconds from trace start
    problem: Problem
    seed_index: int


def serving_trace(seed: int = 4, count: int = 400, rate: float = 20.0,
                  n_steps: int = 300, plate_share: float = 0.7) -> List[Request]:
    """Poisson arrivals of mixed plate and beam simulations."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        if rng.uniform() < plate_share:
            prob = _plate_draw(rng, n_steps)
        else:
            s = float(np.exp(rng.uniform(0.0, np.log(4.0))))
            mat = Material(c=rng.uniform(0.5, 4.0))
            prob = tpb_beam_problem(int(round(40 * s)), int(round(8 * s)), int(round(8 * s)),
                                    u_max=0.5, n_steps=n_steps, material=mat)
        out.append(Request(t, prob, i))
    return out


def random_state(mesh: Mesh, seed: int, kappa0: float = 1e-4, strain: float = 2e-4):
    """A random admissible state: (u [ndof], kappa_hist [nel*ngp]).

    Displacements follow a random homogeneous strain of size ``strain`` plus
    nodal noise; micro-equivalent strains are uniform in [0, 3 kappa0]; 60 % of
    the Gauss points carry a history above kappa0, the rest sit at kappa0.
    This gives loading, unloading, damaged and undamaged points together.
    """
    rng = np.random.default_rng(seed)
    X = mesh.coords()
    d = mesh.dim
    G = rng.normal(size=(d, d)) * strain
    span = np.ptp(X, axis=0).max() if X.shape[0] > 1 else 1.0
    h = span / max(mesh.shape) if mesh.shape else 1.0
    U = X @ G.T + rng.normal(size=X.shape) * 0.3 * strain * h
    u = np.zeros((mesh.nnode, mesh.nd))
    u[:, :d] = U
    u[:, d] = rng.uniform(0.0, 3.0 * kappa0, size=mesh.nnode)
    kh = np.full(mesh.nel * mesh.ngp, kappa0)
    m = rng.uniform(size=kh.shape) < 0.6
    kh[m] += rng.uniform(0.0, 2.0 * kappa0, size=int(m.sum()))
    return u.ravel(), kh
