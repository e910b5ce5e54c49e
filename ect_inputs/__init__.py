"""Seeded synthetic inputs for the eddy-current probe-in-tube problem.

This module produces the *inputs* of the method and nothing else: the
tetrahedral mesh (structured Kuhn subdivision of a box, optionally jittered),
its partition into subdomain blocks, the boundary-condition mask, the per-tet
material coefficients of the two configurations (the "vacuum" background and
the configuration with a defect, deposit or support plate), the coil
descriptions and the probe positions.  It holds none of the method's
arithmetic (no element integrals, no right-hand side, no solve, no impedance):
both the CUDA library and the CPU oracle consume what it returns, and each of
them computes the method on its own.

Geometry follows the paper's setting (Sec. 1 and Sec. 4): a tube inside a
convex box-shaped domain, an annular probe coil pair inside the tube, a tube
support plate (TSP) with a quatrefoil hole, and a defect region Omega_d.
Where the paper leaves geometry open, the values used here are stated in the
config table below (all lengths in metres, conductivities in S/m).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MU0 = 4.0e-7 * math.pi
NU0 = 1.0 / MU0

# Boundary-condition mask bits: component of A fixed to zero on the box faces
# (A.n = 0 on the boundary of a box means A_x = 0 on x-faces, etc.).
BC_AX, BC_AY, BC_AZ = 1, 2, 4


@dataclasses.dataclass
class Coil:
    """Annular coil carrying an azimuthal current density of magnitude J_e.

    The coil occupies r_in <= r <= r_out (r measured from the tube axis, the
    z axis through the box centre) and |z - (z_probe + z_offset)| <= length/2.
    """
    r_in: float = 6.0e-3
    r_out: float = 7.5e-3
    length: float = 2.0e-3
    z_offset: float = 0.0
    J_e: float = 1.0e6

    @property
    def current(self) -> float:
        """Nominal ampere-turn current I = J_e * (r_out - r_in) * length."""
        return self.J_e * (self.r_out - self.r_in) * self.length

    def as_tuple(self):
        return (self.r_in, self.r_out, self.length, self.z_offset, self.J_e)


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray            # (N,3) float64 node coordinates [m]
    tets: np.ndarray           # (T,4) int32, positively oriented
    block_of_node: np.ndarray  # (N,) int32, non-decreasing, contiguous blocks
    bc_mask: np.ndarray        # (N,) uint8, BC_AX|BC_AY|BC_AZ bits
    shape: tuple               # (nx, ny, nz) nodes
    block_shape: tuple         # (sx, sy, sz) nodes per subdomain block
    lengths: tuple             # (Lx, Ly, Lz) box size [m]

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_blocks(self) -> int:
        return int(self.block_of_node[-1]) + 1 if self.n_nodes else 0


@dataclasses.dataclass
class Problem:
    mesh: Mesh
    sigma: np.ndarray     # (T,) background ("vacuum") conductivity
    nu: np.ndarray        # (T,) background reluctivity 1/mu
    sigma_d: np.ndarray   # (T,) defect conductivity, NaN = same as background
    nu_d: np.ndarray      # (T,) defect reluctivity, NaN = same as background
    coils: list           # two Coil objects (the probe's coil pair)
    z_pos: np.ndarray     # (n_pos,) probe positions along the axis [m]
    freq: float = 1.0e5
    nu_tilde: float = NU0
    delta: float = 1.0    # V-gauge penalty factor [1/m^2]
    name: str = ""

    @property
    def omega(self) -> float:
        return 2.0 * math.pi * self.freq


# ----------------------------------------------------------------------------
# Structured Kuhn mesh
# ----------------------------------------------------------------------------

# The six Kuhn tetrahedra of the unit cube: monotone lattice paths from corner
# (0,0,0) to (1,1,1), one per permutation of the three axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _perm_sign(p):
    s = 1
    p = list(p)
    for i in range(3):
        for j in range(i + 1, 3):
            if p[i] > p[j]:
                s = -s
    return s


def _kuhn_corner_paths():
    """Return (6,4,3) integer corner offsets, each tet positively oriented."""
    out = []
    for p in _PERMS:
        c = [np.zeros(3, dtype=np.int64)]
        for ax in p:
            nxt = c[-1].copy()
            nxt[ax] += 1
            c.append(nxt)
        if _perm_sign(p) < 0:
            c[2], c[3] = c[3], c[2]
        out.append(np.stack(c))
    return np.stack(out)


def node_order(shape, block_shape):
    """Map grid index g = i + nx*(j + ny*k) to the subdomain-major node id.

    Nodes are grouped into boxes of block_shape nodes (ragged at the far
    faces); blocks are ordered x-fastest, and nodes within a block x-fastest.
    Returns (new_id_of_grid (G,), block_of_node (N,)).
    """
    nx, ny, nz = shape
    sx, sy, sz = block_shape
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    I = I.ravel(); J = J.ravel(); K = K.ravel()
    nbx = -(-nx // sx); nby = -(-ny // sy)
    blk = (I // sx) + nbx * ((J // sy) + nby * (K // sz))
    loc = (I % sx) + sx * ((J % sy) + sy * (K % sz))
    key = blk.astype(np.int64) * (sx * sy * sz) + loc
    order = np.argsort(key, kind="stable")          # new id -> grid index
    new_id = np.empty_like(order)
    new_id[order] = np.arange(order.size)
    blk_sorted = blk[order]
    # relabel block ids densely (every block is non-empty on a full grid)
    _, dense = np.unique(blk_sorted, return_inverse=True)
    return new_id.astype(np.int64), dense.astype(np.int32)


def box_mesh(shape, lengths, block_shape=(2, 2, 4), jitter=0.0, seed=0):
    """Structured Kuhn tetrahedral mesh of a box centred on the z axis.

    shape = (nx, ny, nz) nodes, lengths = (Lx, Ly, Lz) metres; x, y in
    [-L/2, L/2], z in [-Lz/2, Lz/2].  jitter > 0 moves interior nodes by
    U[-jitter*h, jitter*h] per axis, face nodes only within their face, and
    keeps edge and corner nodes fixed so that the box faces stay planar.
    """
    nx, ny, nz = shape
    Lx, Ly, Lz = lengths
    hx, hy, hz = Lx / (nx - 1), Ly / (ny - 1), Lz / (nz - 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel(); j = j.ravel(); k = k.ravel()
    x = -0.5 * Lx + i * hx
    y = -0.5 * Ly + j * hy
    z = -0.5 * Lz + k * hz
    onx = (i == 0) | (i == nx - 1)
    ony = (j == 0) | (j == ny - 1)
    onz = (k == 0) | (k == nz - 1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=(x.size, 3))
        nfaces = onx.astype(int) + ony.astype(int) + onz.astype(int)
        mx = (nfaces == 0) | ((nfaces == 1) & ~onx)
        my = (nfaces == 0) | ((nfaces == 1) & ~ony)
        mz = (nfaces == 0) | ((nfaces == 1) & ~onz)
        x = x + np.where(mx, d[:, 0] * hx, 0.0)
        y = y + np.where(my, d[:, 1] * hy, 0.0)
        z = z + np.where(mz, d[:, 2] * hz, 0.0)
    bc = (onx * BC_AX + ony * BC_AY + onz * BC_AZ).astype(np.uint8)

    new_id, block_of_node = node_order(shape, block_shape)
    n = nx * ny * nz
    xyz = np.empty((n, 3))
    xyz[new_id, 0] = x
    xyz[new_id, 1] = y
    xyz[new_id, 2] = z
    bc_mask = np.empty(n, dtype=np.uint8)
    bc_mask[new_id] = bc

    # cells and their 6 Kuhn tets
    ck, cj, ci = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1),
                             indexing="ij")
    ci = ci.ravel(); cj = cj.ravel(); ck = ck.ravel()
    paths = _kuhn_corner_paths()                     # (6,4,3)
    gi = ci[:, None, None] + paths[None, :, :, 0]
    gj = cj[:, None, None] + paths[None, :, :, 1]
    gk = ck[:, None, None] + paths[None, :, :, 2]
    g = gi + nx * (gj + ny * gk)                     # (C,6,4) grid ids
    tets = new_id[g].reshape(-1, 4).astype(np.int32)
    return Mesh(xyz=xyz, tets=tets, block_of_node=block_of_node, bc_mask=bc_mask,
                shape=tuple(shape), block_shape=tuple(block_shape),
                lengths=tuple(lengths))


def unstructured_box_mesh(shape, lengths, jitter=0.12, seed=0, block_nodes=8):
    """Unstructured tetrahedral mesh of the box, not a Kuhn mesh.

    Nodes: the nx x ny x nz grid plus one node at the centre of every cell.
    Every quadrilateral cell face is cut along one of its two diagonals,
    chosen at random per face (shared by the two cells of an interior face,
    so the mesh is conforming), and every cell is filled by the 12 tets that
    join its centre node to the 12 face triangles.  Then all nodes move by
    U[-jitter*h, jitter*h] per axis (interior grid nodes and centres freely,
    face nodes within their face, edge nodes along their edge, corners
    fixed, so the box faces stay planar), and tets are oriented positively.
    Valences vary from node to node (grid nodes touch 24 to 56 tets of
    different shapes, centres 12), and every tet keeps a volume of order h^3.

    The nodes are numbered grid first (lexicographic), then centres, and
    block_of_node is a placeholder (consecutive runs of block_nodes nodes);
    a partitioner assigns the real subdomains and node order (permute_mesh)."""
    nx, ny, nz = shape
    L = np.array(lengths, dtype=np.float64)
    h = L / (np.array(shape) - 1)
    rng = np.random.default_rng(seed)
    gid = lambda i, j, k: i + nx * (j + ny * k)  # noqa: E731
    k3, j3, i3 = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    gx = np.stack([i3.ravel(), j3.ravel(), k3.ravel()], axis=1).astype(np.float64)
    ng = nx * ny * nz
    ck, cj, ci = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    nc = cells.shape[0]
    xyz = np.concatenate([gx, cells + 0.5]) * h[None, :] - 0.5 * L[None, :]
    # diagonal choice per face: faces normal to axis a at grid plane index, keyed by the lower corner
    diag = [rng.integers(0, 2, size=(nx, ny, nz)) for _ in range(3)]
    tets = []
    for c in range(nc):
        i, j, k = cells[c]
        centre = ng + c
        for a in range(3):                       # the two faces normal to axis a
            b1, b2 = [(1, 2), (0, 2), (0, 1)][a]
            for side in (0, 1):
                base = [i, j, k]
                base[a] += side
                def corner(u, v):
                    q = list(base)
                    q[b1] += u
                    q[b2] += v
                    return gid(*q)
                q00, q10, q01, q11 = corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)
                if diag[a][tuple(base)]:
                    tris = ((q00, q10, q11), (q00, q11, q01))
                else:
                    tris = ((q00, q10, q01), (q10, q11, q01))
                for tri in tris:
                    tets.append((tri[0], tri[1], tri[2], centre))
    tets = np.array(tets, dtype=np.int64)
    vol = tet_volumes(xyz, tets)
    flip = vol < 0.0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    # jitter (grid part keeps its face/edge/corner classes)
    on = [np.concatenate([(gx[:, a] == 0) | (gx[:, a] == shape[a] - 1), np.zeros(nc, dtype=bool)])
          for a in range(3)]
    nfaces = on[0].astype(int) + on[1].astype(int) + on[2].astype(int)
    d = rng.uniform(-jitter, jitter, size=xyz.shape) * h[None, :]
    for a in range(3):
        movable = (nfaces == 0) | ((nfaces >= 1) & (nfaces <= 2) & ~on[a])
        xyz[:, a] += np.where(movable, d[:, a], 0.0)
    vol = tet_volumes(xyz, tets)
    if vol.min() <= 0.02 * float(np.prod(h)) / 12.0:
        raise ValueError("jitter too large: a tetrahedron lost most of its volume")
    bc = (on[0] * BC_AX + on[1] * BC_AY + on[2] * BC_AZ).astype(np.uint8)
    n = xyz.shape[0]
    block = (np.arange(n) // block_nodes).astype(np.int32)
    return Mesh(xyz=xyz, tets=tets.astype(np.int32), block_of_node=block, bc_mask=bc,
                shape=tuple(shape), block_shape=(block_nodes,), lengths=tuple(lengths))


def permute_mesh(mesh, new_id, block_of_new):
    """The same mesh with node i renamed new_id[i]; block_of_new gives the
    subdomain of each renamed node (non-decreasing).  Tets keep their order."""
    new_id = np.asarray(new_id, dtype=np.int64)
    n = mesh.n_nodes
    if np.sort(new_id).tolist() != list(range(n)):
        raise ValueError("new_id is not a permutation")
    xyz = np.empty_like(mesh.xyz)
    xyz[new_id] = mesh.xyz
    bc = np.empty_like(mesh.bc_mask)
    bc[new_id] = mesh.bc_mask
    return Mesh(xyz=xyz, tets=new_id[mesh.tets].astype(np.int32),
                block_of_node=np.asarray(block_of_new, dtype=np.int32), bc_mask=bc, shape=mesh.shape,
                block_shape=mesh.block_shape, lengths=mesh.lengths)


def write_tetgen(prefix, mesh, region=None):
    """Write the mesh in TetGen's documented text format: prefix.node (index,
    x, y, z, boundary marker = the A.n = 0 bit mask) and prefix.ele (index,
    four node indices, optional region attribute), indices from 0."""
    n, t = mesh.n_nodes, mesh.n_tets
    with open(prefix + ".node", "w") as f:
        f.write(f"{n} 3 0 1\n")
        for i in range(n):
            x, y, z = (float(v) for v in mesh.xyz[i])
            f.write(f"{i} {x!r} {y!r} {z!r} {int(mesh.bc_mask[i])}\n")
    with open(prefix + ".ele", "w") as f:
        f.write(f"{t} 4 {0 if region is None else 1}\n")
        for k in range(t):
            a, b, c, d = (int(v) for v in mesh.tets[k])
            tail = "" if region is None else f" {int(region[k])}"
            f.write(f"{k} {a} {b} {c} {d}{tail}\n")


def read_tetgen(prefix):
    """Read prefix.node / prefix.ele (TetGen text format; '#' comments, first
    index 0 or 1, optional point attributes and boundary marker, optional
    tet region attribute).  Returns (xyz (N,3), tets (T,4) 0-based, bc marker
    (N,) or None, region (T,) or None)."""
    def rows(path):
        out = []
        with open(path) as f:
            for line in f:
                line = line.split("#", 1)[0].split()
                if line:
                    out.append(line)
        return out

    nrows = rows(prefix + ".node")
    n, dim, nattr, nbm = (int(v) for v in nrows[0][:4])
    if dim != 3:
        raise ValueError("3-D points expected")
    pts = nrows[1:1 + n]
    first = int(pts[0][0])
    xyz = np.array([[float(v) for v in r[1:4]] for r in pts])
    bc = np.array([int(r[4 + nattr]) for r in pts], dtype=np.int64) if nbm else None
    erows = rows(prefix + ".ele")
    t, npt, nreg = (int(v) for v in erows[0][:3])
    if npt != 4:
        raise ValueError("linear tetrahedra (4 nodes) expected")
    ele = erows[1:1 + t]
    tets = np.array([[int(v) - first for v in r[1:5]] for r in ele], dtype=np.int64)
    region = np.array([float(r[5]) for r in ele]) if nreg else None
    return xyz, tets, bc, region


def tet_volumes(xyz, tets):
    """Signed volumes (used only to validate generated meshes)."""
    p = xyz[tets]
    a = p[:, 1] - p[:, 0]
    b = p[:, 2] - p[:, 0]
    c = p[:, 3] - p[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def centroids(mesh):
    return mesh.xyz[mesh.tets].mean(axis=1)


# Interior sample lattice for volume fractions: the 35 points of the degree-4
# barycentric lattice (n_a >= 0, sum n_a = 4) shrunk by 4/5 about the
# centroid, i.e. barycentric weights (4 n_a + 1)/20.  No point lies on a face,
# so a point is never shared by two tets.
LATTICE = np.array([(4 * a + 1, 4 * b + 1, 4 * c + 1, 4 * (4 - a - b - c) + 1)
                    for a in range(5) for b in range(5 - a) for c in range(5 - a - b)],
                   dtype=np.float64)
assert LATTICE.shape == (35, 4)


def lattice_fraction(mesh, inside_fn, tet_subset=None, chunk=1 << 18):
    """Fraction of the 35 lattice points of each tet for which inside_fn holds.

    Points are formed as (((m0*x0 + m1*x1) + m2*x2) + m3*x3) * 0.05 in float64
    with m_a = 4 n_a + 1.
    inside_fn(x, y, z) -> bool array.  Returns (T,) float64 (0 outside subset).
    """
    T = mesh.n_tets
    f = np.zeros(T)
    idx = np.arange(T) if tet_subset is None else np.asarray(tet_subset)
    for s in range(0, idx.size, chunk):
        sl = idx[s:s + chunk]
        p = mesh.xyz[mesh.tets[sl]]                  # (c,4,3)
        acc = None
        for a in range(4):
            term = LATTICE[None, :, a, None] * p[:, None, a, :]
            acc = term if acc is None else acc + term
        pts = acc * 0.05                             # (c,35,3)
        ins = inside_fn(pts[..., 0], pts[..., 1], pts[..., 2])
        f[sl] = ins.sum(axis=1) / 35.0
    return f


# ----------------------------------------------------------------------------
# Materials
# ----------------------------------------------------------------------------

TUBE_R_IN = 8.5e-3
TUBE_R_OUT = 9.6e-3
SIGMA_TUBE = 1.0e6
SIGMA_TSP = 1.4e6
TSP_HALF_THICK = 10.0e-3
TSP_HOLE_R = 10.0e-3
TSP_LOBE_R = 3.0e-3
TSP_LOBE_CENTER = 11.5e-3


def tube_tets(c):
    r = np.hypot(c[:, 0], c[:, 1])
    return (r >= TUBE_R_IN) & (r < TUBE_R_OUT)


def tsp_tets(c):
    """Support plate: |z| <= 10 mm outside a quatrefoil hole (Sec. 1)."""
    r = np.hypot(c[:, 0], c[:, 1])
    hole = r < TSP_HOLE_R
    for q in range(4):
        th = math.radians(45.0 + 90.0 * q)
        cx, cy = TSP_LOBE_CENTER * math.cos(th), TSP_LOBE_CENTER * math.sin(th)
        hole |= np.hypot(c[:, 0] - cx, c[:, 1] - cy) < TSP_LOBE_R
    return (np.abs(c[:, 2]) <= TSP_HALF_THICK) & ~hole


def probe_coils(gap=2.0e-3, length=2.0e-3):
    """The probe's coil pair: two identical coils, their facing ends `gap` apart."""
    off = 0.5 * (gap + length)
    return [Coil(z_offset=-off, length=length), Coil(z_offset=+off, length=length)]


# ----------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------

CONFIGS = {
    # name: (shape, lengths, jitter)
    "c1": ((16, 16, 32), (20e-3, 20e-3, 40e-3), 0.0),
    "c2": ((53, 53, 356), (30e-3, 30e-3, 200e-3), 0.15),
    "c3": ((63, 63, 126), (20e-3, 20e-3, 40e-3), 0.0),
    "c4": ((84, 84, 567), (30e-3, 30e-3, 200e-3), 0.0),
    "c5": ((50, 50, 100), (20e-3, 20e-3, 40e-3), 0.0),
}


def wall_loss_problem(shape, lengths, block_shape=(2, 2, 4), jitter=0.0, seed=0,
                      z_pos=(0.0,), sigma_d=0.5e6, name="", mesh=None):
    """Tube in water with a wall-loss patch as the defect (configs 1 and 3).

    Omega_d = tube-wall tets with centroid z in [-2, 2] mm and polar angle in
    [0, pi/2]; there the conductivity drops from 1e6 to sigma_d.  `mesh`
    replaces the structured mesh (e.g. unstructured_box_mesh of the same box).
    """
    m = mesh if mesh is not None else box_mesh(shape, lengths, block_shape, jitter, seed)
    c = centroids(m)
    tube = tube_tets(c)
    sigma = np.where(tube, SIGMA_TUBE, 0.0)
    nu = np.full(m.n_tets, NU0)
    th = np.arctan2(c[:, 1], c[:, 0])
    patch = tube & (np.abs(c[:, 2]) <= 2.0e-3) & (th >= 0.0) & (th <= 0.5 * math.pi)
    sig_d = np.where(patch, sigma_d, np.nan)
    nu_d = np.full(m.n_tets, np.nan)
    return Problem(mesh=m, sigma=sigma, nu=nu, sigma_d=sig_d, nu_d=nu_d,
                   coils=probe_coils(), z_pos=np.asarray(z_pos, dtype=np.float64), name=name)


def tsp_problem(shape, lengths, block_shape=(2, 2, 4), jitter=0.0, seed=0,
                z_pos=(10.0e-3,), name=""):
    """Tube through a support plate (configs 2 and 4).

    The background treats the TSP region as vacuum (the paper's M0 system) and
    the defect configuration gives it sigma = 1.4e6 (the M1 system): Omega_d is
    the TSP, as in the paper's two experiment tables.
    """
    m = box_mesh(shape, lengths, block_shape, jitter, seed)
    c = centroids(m)
    tube = tube_tets(c)
    tsp = tsp_tets(c) & ~tube
    sigma = np.where(tube, SIGMA_TUBE, 0.0)
    nu = np.full(m.n_tets, NU0)
    sig_d = np.where(tsp, SIGMA_TSP, np.nan)
    nu_d = np.full(m.n_tets, np.nan)
    return Problem(mesh=m, sigma=sigma, nu=nu, sigma_d=sig_d, nu_d=nu_d,
                   coils=probe_coils(), z_pos=np.asarray(z_pos, dtype=np.float64), name=name)


def deposit_params(seed):
    """Deposit parameters drawn for surrogate sample `seed`.

    Returns (thickness [m], axial length [m], sigma [S/m], mu_r,
    azimuthal coverage [rad], axial centre [m]).
    """
    rng = np.random.default_rng(1_000_003 + int(seed))
    t = rng.uniform(0.0, 0.5e-3)
    ell = rng.uniform(2.0e-3, 20.0e-3)
    sig = rng.uniform(1.0e4, 1.0e6)
    mur = rng.uniform(1.0, 5.0)
    cov = rng.uniform(0.0, 2.0 * math.pi)
    zc = rng.uniform(-10.0e-3, 10.0e-3)
    return np.array([t, ell, sig, mur, cov, zc])


def deposit_problem(shape, lengths, params, block_shape=(2, 2, 4), z_pos=None, mesh=None,
                    name=""):
    """Tube with an annular-sector deposit on its outer wall (config 5).

    The deposit occupies r in [9.6, 9.6 + t] mm, |z - z_c| <= l/2 and polar
    angle in [0, coverage]; each tet takes the volume fraction f of its 35
    lattice points inside it and blends sigma and nu linearly with f.
    """
    m = mesh if mesh is not None else box_mesh(shape, lengths, block_shape)
    c = centroids(m)
    tube = tube_tets(c)
    sigma = np.where(tube, SIGMA_TUBE, 0.0)
    nu = np.full(m.n_tets, NU0)
    t, ell, sd, mur, cov, zc = [float(v) for v in params]

    def inside(x, y, z):
        r2 = x * x + y * y
        th = np.mod(np.arctan2(y, x), 2.0 * math.pi)
        return ((r2 >= TUBE_R_OUT ** 2) & (r2 <= (TUBE_R_OUT + t) ** 2)
                & (np.abs(z - zc) <= 0.5 * ell) & (th <= cov))

    r = np.hypot(c[:, 0], c[:, 1])
    near = np.nonzero((r > TUBE_R_OUT - 2e-3) & (r < TUBE_R_OUT + t + 2e-3)
                      & (np.abs(c[:, 2] - zc) < 0.5 * ell + 2e-3))[0]
    f = lattice_fraction(m, inside, near)
    hit = f > 0.0
    sig_d = np.where(hit, sigma + f * (sd - sigma), np.nan)
    nu_d = np.where(hit, nu + f * (NU0 / mur - nu), np.nan)
    if z_pos is None:
        z_pos = -15.875e-3 + 0.25e-3 * np.arange(128)
    return Problem(mesh=m, sigma=sigma, nu=nu, sigma_d=sig_d, nu_d=nu_d,
                   coils=probe_coils(), z_pos=np.asarray(z_pos, dtype=np.float64), name=name)


def make_config(name, block_shape=(2, 2, 4), seed=0):
    """Build one of the five workloads by name ('c1' .. 'c5')."""
    shape, lengths, jitter = CONFIGS[name]
    if name == "c1":
        return wall_loss_problem(shape, lengths, block_shape, jitter, seed, z_pos=(0.0,),
                                 name=name)
    if name == "c3":
        zp = -15.75e-3 + 0.5e-3 * np.arange(64)
        return wall_loss_problem(shape, lengths, block_shape, jitter, seed, z_pos=zp, name=name)
    if name in ("c2", "c4"):
        return tsp_problem(shape, lengths, block_shape, jitter, seed, z_pos=(10.0e-3,), name=name)
    if name == "c5":
        return deposit_problem(shape, lengths, deposit_params(seed), block_shape, name=name)
    raise KeyError(name)
