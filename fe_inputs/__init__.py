"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module defines the *problem*, never the eigensolver: it assembles the
pencil ``S v = omega^2 M v`` of Sec. 2 (eq. def:basisMatrixEVP) for first-order
(P1) finite elements on voxel domains split into Kuhn simplices, with the mass
matrix lumped to its row sums (Remark 2.1), and it draws seeded
N(0,1) start vectors. No filter weight, time step, orthogonalisation or
Rayleigh-Ritz arithmetic lives here.

Layout of every problem returned:
  * ``row_ptr`` int64[n+1], ``col`` int32[nnz], ``val`` float64[nnz]: CSR of S,
    columns ascending inside a row, every structural FE coupling kept (also the
    ones whose element sums cancel to an exact 0.0);
  * ``m`` float64[n]: the lumped mass diagonal (all entries > 0);
  * dofs numbered lexicographically over the node grid, x fastest, after
    Dirichlet nodes are eliminated.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "kuhn_simplices", "cell_matrices", "assemble_voxels",
    "square_grid", "box_grid", "flared_tube", "start_vectors", "WORKLOADS",
]


@dataclass
class Problem:
    """A sparse generalized eigenproblem S v = omega^2 M v with diagonal M."""
    name: str
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    m: np.ndarray
    # grid description (cells per axis, spacing per axis) for tensor grids
    cells: tuple = ()
    h: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col.astype(np.int64), self.row_ptr),
                             shape=(self.n, self.n))


# --------------------------------------------------------------------------
# reference cell: Kuhn simplices and P1 element matrices
# --------------------------------------------------------------------------

def kuhn_simplices(dim: int) -> list[np.ndarray]:
    """Kuhn (Freudenthal) split of the unit cell in ``dim`` dimensions.

    One simplex per permutation of the axes: walk from corner 0 to corner
    (1,..,1) adding one unit vector at a time. Returns a list of
    (dim+1, dim) integer corner coordinates.
    """
    out = []
    for perm in itertools.permutations(range(dim)):
        pts = [np.zeros(dim, dtype=np.int64)]
        for a in perm:
            nxt = pts[-1].copy()
            nxt[a] = 1
            pts.append(nxt)
        out.append(np.array(pts))
    return out


def corner_index(c) -> int:
    """Corner of the unit cell -> index sum_a c_a 2^a (axis 0 = x fastest)."""
    return int(sum(int(v) << a for a, v in enumerate(c)))


def cell_matrices(h: tuple[float, ...]):
    """P1 stiffness (2^d x 2^d), lumped mass (2^d) and structural pattern of one cell.

    Each Kuhn simplex contributes vol * grad(phi_i) . grad(phi_j) to the
    stiffness and vol/(d+1) to the lumped mass of each of its vertices. The
    structural pattern marks vertex pairs that share a simplex (an FE coupling
    exists even when its value cancels to zero).
    """
    dim = len(h)
    nc = 1 << dim
    K = np.zeros((nc, nc))
    mass = np.zeros(nc)
    struct = np.zeros((nc, nc), dtype=bool)
    scale = np.asarray(h, dtype=np.float64)
    for simplex in kuhn_simplices(dim):
        x = simplex * scale                       # (d+1, d) physical vertices
        D = (x[1:] - x[0]).T                      # columns x_i - x_0
        vol = abs(np.linalg.det(D)) / math.factorial(dim)
        Dinv = np.linalg.inv(D)                   # row i-1 = grad phi_i
        grads = np.vstack([-Dinv.sum(axis=0), Dinv])
        Kloc = vol * grads @ grads.T
        idx = [corner_index(c) for c in simplex]
        for a in range(dim + 1):
            mass[idx[a]] += vol / (dim + 1)
            for b in range(dim + 1):
                K[idx[a], idx[b]] += Kloc[a, b]
                struct[idx[a], idx[b]] = True
    return K, mass, struct


# --------------------------------------------------------------------------
# assembly on a voxel domain
# --------------------------------------------------------------------------

def _offsets(dim: int) -> np.ndarray:
    """Neighbour offsets that can carry a Kuhn coupling: all nonzero
    components of one sign (plus the zero offset)."""
    offs = []
    for o in itertools.product((-1, 0, 1), repeat=dim):
        nz = [v for v in o if v != 0]
        if all(v > 0 for v in nz) or all(v < 0 for v in nz):
            offs.append(o)
    return np.array(offs, dtype=np.int64)


def assemble_voxels(present: np.ndarray, h: tuple[float, ...],
                    dirichlet: np.ndarray, name: str = "voxels") -> Problem:
    """Assemble lumped P1 on the cells marked in ``present``.

    present:   bool array of cells, numpy shape (n_{d-1}, ..., n_0) (x last).
    h:         spacing per axis, (h_x, h_y[, h_z]).
    dirichlet: bool array of nodes, shape (n_{d-1}+1, ..., n_0+1); those nodes
               are eliminated (homogeneous Dirichlet). All other nodes touching
               a present cell are dofs (natural Neumann condition elsewhere).
    """
    dim = present.ndim
    assert len(h) == dim
    K, cmass, cstruct = cell_matrices(tuple(h))
    nc = 1 << dim
    node_shape = tuple(s + 1 for s in present.shape)

    # node mask: bit j set if the cell at (node - 1 + s_j) is present, where
    # corner index j encodes s_j; the node is corner (1 - s_j) of that cell.
    pad = np.pad(present, 1, mode="constant", constant_values=False)
    mask = np.zeros(node_shape, dtype=np.int64)
    for j in range(nc):
        s = [(j >> a) & 1 for a in range(dim)]            # per axis, x = axis 0
        # numpy axis order is reversed (x last)
        sl = tuple(slice(s[a], s[a] + node_shape[dim - 1 - a])
                   for a in reversed(range(dim)))
        mask |= pad[sl].astype(np.int64) << j

    offs = _offsets(dim)                                    # (n_off, dim), x first
    n_off = len(offs)
    nmask = 1 << nc
    table_val = np.zeros((nmask, n_off))
    table_str = np.zeros((nmask, n_off), dtype=bool)
    table_mass = np.zeros(nmask)
    for mk in range(nmask):
        for j in range(nc):
            if not (mk >> j) & 1:
                continue
            me = [1 - ((j >> a) & 1) for a in range(dim)]   # node's corner in cell j
            ci = corner_index(me)
            table_mass[mk] += cmass[ci]
            for oi, o in enumerate(offs):
                nb = [me[a] + o[a] for a in range(dim)]
                if all(0 <= v <= 1 for v in nb):
                    cj = corner_index(nb)
                    if cstruct[ci, cj]:
                        table_val[mk, oi] += K[ci, cj]
                        table_str[mk, oi] = True

    free = (mask != 0) & ~dirichlet
    flat_free = free.ravel()
    lin = np.flatnonzero(flat_free)                         # linear node ids of dofs
    n = lin.size
    cidx = np.full(flat_free.size, -1, dtype=np.int64)
    cidx[lin] = np.arange(n, dtype=np.int64)
    fmask = mask.ravel()[lin]

    # linear offset of each stencil offset, sorted ascending -> columns ascend
    strides = [1]
    for a in range(1, dim):
        strides.append(strides[-1] * node_shape[dim - a])
    lin_off = np.array([sum(o[a] * strides[a] for a in range(dim)) for o in offs])
    order = np.argsort(lin_off)
    offs, lin_off = offs[order], lin_off[order]
    table_val, table_str = table_val[:, order], table_str[:, order]

    coords = np.unravel_index(lin, node_shape)              # numpy axis order
    coords = [coords[dim - 1 - a] for a in range(dim)]      # x first
    cols = np.empty((n, n_off), dtype=np.int64)
    keep = np.empty((n, n_off), dtype=bool)
    for oi in range(n_off):
        ok = table_str[fmask, oi].copy()
        for a in range(dim):
            c = coords[a] + offs[oi, a]
            ok &= (c >= 0) & (c < node_shape[dim - 1 - a])
        q = lin + lin_off[oi]
        q = np.where(ok, q, 0)
        cq = cidx[q]
        ok &= cq >= 0
        cols[:, oi] = cq
        keep[:, oi] = ok
    vals = table_val[fmask]                                  # (n, n_off)
    counts = keep.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[keep].astype(np.int32)
    val = np.ascontiguousarray(vals[keep])
    m = table_mass[fmask].copy()
    return Problem(name=name, n=n, row_ptr=row_ptr, col=col, val=val, m=m,
                   cells=tuple(reversed(present.shape)), h=tuple(h))


def box_grid(cells: tuple[int, ...], extent: tuple[float, ...] | None = None,
             name: str | None = None) -> Problem:
    """Tensor grid of ``cells`` (x first) over a box, Dirichlet on every face.

    With ``extent`` None each axis has length 1 (h_a = 1 / n_a).
    """
    dim = len(cells)
    if extent is None:
        extent = (1.0,) * dim
    h = tuple(float(e) / c for e, c in zip(extent, cells))
    shape = tuple(reversed(cells))
    present = np.ones(shape, dtype=bool)
    node_shape = tuple(s + 1 for s in shape)
    dirichlet = np.zeros(node_shape, dtype=bool)
    for ax in range(dim):
        idx = [slice(None)] * dim
        idx[ax] = 0
        dirichlet[tuple(idx)] = True
        idx[ax] = node_shape[ax] - 1
        dirichlet[tuple(idx)] = True
    p = assemble_voxels(present, h, dirichlet,
                        name=name or "box_" + "x".join(map(str, cells)))
    p.meta["extent"] = tuple(extent)
    return p


def square_grid(n: int) -> Problem:
    """Unit square, P1 right triangles on an n x n grid, Dirichlet boundary."""
    return box_grid((n, n), name=f"square{n}")


def flared_tube(h: float, length: float = 1.0, r0: float = 0.02,
                growth: float = 3.0, name: str | None = None) -> Problem:
    """Voxelised flared tube: radius r0*exp(growth*x) for x in [0, length].

    A cell is present when its centre lies inside the tube. Homogeneous
    Dirichlet on the mouth plane x = 0, natural (Neumann) condition on every
    other wall.
    """
    rmax = r0 * math.exp(growth * length)
    nx = int(round(length / h))
    ny = int(math.ceil(2 * rmax / h))
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h - ny * h / 2
    r = r0 * np.exp(growth * xc)
    present = (yc[:, None, None] ** 2 + yc[None, :, None] ** 2
               <= r[None, None, :] ** 2)                     # shape (nz, ny, nx)
    dirichlet = np.zeros((ny + 1, ny + 1, nx + 1), dtype=bool)
    dirichlet[:, :, 0] = True
    p = assemble_voxels(present, (h, h, h), dirichlet,
                        name=name or f"flared_tube_h{h:g}")
    p.meta.update(dict(length=length, r0=r0, growth=growth))
    return p


# --------------------------------------------------------------------------
# start vectors
# --------------------------------------------------------------------------

def start_vectors(n: int, b: int = 1, seed: int = 0) -> np.ndarray:
    """b independent N(0,1) vectors of length n from numpy's PCG64 stream
    ``default_rng(seed)``; shape (b, n), C-contiguous (= n x b column-major)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((b, n)))


# --------------------------------------------------------------------------
# workloads (the sizes and filter parameters the library is measured on)
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    """A measured configuration: the problem(s), the filter and the solver sizes.

    ``build`` returns one Problem or a list of them (a batch of meshes solved in one
    context). ``intervals(problem)`` gives the F filter intervals [(wmin, wmax), ...]
    of a mesh; the solver uses the first one."""
    name: str
    build: object                 # () -> Problem | list[Problem]
    omega_min: float
    omega_max: float
    L: int
    kmax: int
    precision: str = "fp64"       # "fp64" | "fp32"
    b: int = 1                    # block size (start vectors per mesh)
    cfl: float = 0.9              # tau = cfl * 2 / omega_max(S, M)
    power_iters: int = 300
    seed: int = 0
    intervals: object = None      # (Problem) -> list of (wmin, wmax); None: [(omega_min, omega_max)]
    check_every: int = 5
    tol: float = 0.0              # acceptance; 0: 1e-8 (fp64) / 1e-5 (fp32)
    tts_kmax: int = 0             # Krylov dimension at which the FP64 solve accepts every distinct
                                  # eigenvalue of the interval at 1e-8, and so does the next
                                  # larger one in steps of 10 (0: not measured)

    def mesh_intervals(self, p: Problem):
        return self.intervals(p) if self.intervals else [(self.omega_min, self.omega_max)]

    def acceptance(self) -> float:
        return self.tol or (1e-8 if self.precision == "fp64" else 1e-5)


# 12 boxes of uneven size, uniform spacing h = 1/64 (extent = cells / 64): 29,791 ..
# 857,375 dofs, 3.13 M in total
BATCH12_CELLS = [(32, 32, 32), (40, 40, 40), (48, 40, 32), (48, 48, 48), (56, 48, 40), (64, 48, 48),
                 (64, 64, 64), (72, 64, 56), (80, 64, 64), (80, 80, 80), (88, 80, 72), (96, 96, 96)]


def batch12():
    return [box_grid(c, extent=tuple(x / 64.0 for x in c), name="box_" + "x".join(map(str, c)))
            for c in BATCH12_CELLS]


def weyl_intervals(p: Problem, counts=(100, 200, 300, 400), width: int = 15):
    """Four disjoint intervals in the lower spectrum of a box, each expected to hold
    ~``width`` eigenvalues by Weyl's law N(omega) ~ V omega^3 / (6 pi^2)."""
    V = float(np.prod(p.meta.get("extent", (1.0,) * len(p.cells))))
    w = lambda N: (6.0 * math.pi ** 2 * N / V) ** (1.0 / 3.0)
    return [(w(c), w(c + width)) for c in counts]


WORKLOADS = {
    # 2D unit square, P1 triangles, 64x64 cells (3969 dofs)
    "square64_fp64": Workload("square64_fp64", lambda: square_grid(64),
                              20.0, 30.0, L=300, kmax=40),
    # a box of the cube's size with incommensurate edges (2,005,965 dofs): every
    # eigenvalue is simple; [24, 28] holds 81 of them (smallest relative gap 1.9e-5)
    "box2m_fp64": Workload("box2m_fp64", lambda: box_grid((136, 128, 118), extent=(1.0, 0.91, 0.83)),
                           24.0, 28.0, L=600, kmax=60, tts_kmax=210),
    # 3D unit cube, Kuhn tets, 128^3 cells (2,048,383 dofs)
    "cube128_fp64": Workload("cube128_fp64", lambda: box_grid((128, 128, 128)),
                             40.0, 45.0, L=600, kmax=60, tts_kmax=260),
    "cube128_fp32": Workload("cube128_fp32", lambda: box_grid((128, 128, 128)),
                             40.0, 45.0, L=600, kmax=60, precision="fp32"),
    # 12 uneven boxes in one context, blocks of 8 start vectors, 4 intervals per mesh
    "batch12_fp32": Workload("batch12_fp32", batch12, 0.0, 0.0, L=600, kmax=64, precision="fp32",
                             b=8, intervals=weyl_intervals, check_every=16),
    # voxelised flared tube r = 0.02 exp(3x), x in [0, 1], h = 1.74e-3 (~16 M dofs)
    "horn16m_fp32": Workload("horn16m_fp32", lambda: flared_tube(1.74e-3), 60.0, 66.0, L=1000,
                             kmax=200, precision="fp32", b=8, check_every=40),
}
