"""Oracle: the impedance boundary condition on the support-plate surface.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 (Eq. IBC) replaces the volume of a good conductor (the tube support
plate, TSP) by a condition on its surface Gamma_p, valid up to O(delta^2):

    n x (1/mu) curl A = -(1/Z) (i omega A_tau + grad_tau V),   Z = (1 - i)/(delta sigma_p),
    delta = sqrt(2/(omega mu_p sigma_p)),   A_tau = n x (A x n).

Readings (the paper states the condition and its two surface integrals,
Eqs. ibcROTA / ibcNORM, but does not use them in its experiments):
  * n is the normal of the computational domain pointing into the plate
    (out of the domain), the orientation for which the condition is the
    exact surface impedance of a conducting half-space under the e^{-i omega t}
    convention of E = i omega A + grad V;
  * the plate region is removed from the domain: its tets contribute no
    volume form, and every dof of a node that touches only plate tets is
    fixed to zero (identity row and column), the field having decayed
    inside the plate;
  * V is not carried on Gamma_p when the plate is the only conductor there
    (V lives on the conducting nodes of the remaining domain), so Eq. ibcNORM
    has nothing to couple and Eq. ibcROTA adds to the A-A block the surface form
        -(i omega / Z) int_Gamma A_tau . Phi_tau ds,
    i.e. for a surface triangle F with unit normal n and nodes a, b:
        -(i omega / Z) |F| (1 + d_ab)/12 (d_ij - n_i n_j),
    which is symmetric, so the matrix stays complex symmetric;
  * Delta Z of a configuration with the IBC is the coil-EMF difference
    (Eq. impedkl's volume form needs the plate's volume fields, which the
    IBC does not compute).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import fem

MU0 = 4.0e-7 * math.pi

# the four faces of a tet (local node triples) and the node opposite each
_FACES = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


def surface_impedance(omega, sigma_p, mu_p):
    """Z = (1 - i)/(delta sigma_p) with the skin depth delta = sqrt(2/(omega mu_p sigma_p))."""
    delta = math.sqrt(2.0 / (omega * mu_p * sigma_p))
    return (1.0 - 1.0j) / (delta * sigma_p)


def plate_surface(xyz, tets, plate):
    """Faces of Gamma_p: faces shared by a plate tet and a non-plate tet.

    Returns (faces (F,3) node indices, normals (F,3) unit, pointing into the
    plate tet)."""
    tets = np.asarray(tets, dtype=np.int64)
    plate = np.asarray(plate, dtype=bool)
    keys = {}
    for t in range(tets.shape[0]):
        for f in range(4):
            key = tuple(sorted(tets[t, _FACES[f]]))
            keys.setdefault(key, []).append((t, f))
    faces, normals = [], []
    xyz = np.asarray(xyz, dtype=np.float64)
    for key, owners in keys.items():
        if len(owners) != 2:
            continue
        (t0, f0), (t1, f1) = owners
        if plate[t0] == plate[t1]:
            continue
        tp, fp = (t0, f0) if plate[t0] else (t1, f1)
        tri = tets[tp, _FACES[fp]]
        opp = tets[tp, fp]                                # the plate tet's node off this face
        p0, p1, p2 = xyz[tri]
        n = np.cross(p1 - p0, p2 - p0)
        n /= np.linalg.norm(n)
        if np.dot(xyz[opp] - p0, n) < 0.0:                # point into the plate tet
            n = -n
        faces.append(tri)
        normals.append(n)
    return np.array(faces, dtype=np.int64).reshape(-1, 3), np.array(normals).reshape(-1, 3)


def surface_matrix(xyz, faces, normals, n_nodes, coef):
    """Scalar CSR of coef * int_Gamma A_tau . Phi_tau over the triangles (4 dofs per node;
    only the A-A components are touched)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    rows, cols, vals = [], [], []
    for tri, n in zip(faces, normals):
        p0, p1, p2 = xyz[tri]
        area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0))
        P = np.eye(3) - np.outer(n, n)                   # tangential projector
        for a in range(3):
            for b in range(3):
                m = area * (2.0 if a == b else 1.0) / 12.0   # int_F l_a l_b
                for i in range(3):
                    for j in range(3):
                        if P[i, j] != 0.0:
                            rows.append(4 * tri[a] + i)
                            cols.append(4 * tri[b] + j)
                            vals.append(coef * m * P[i, j])
    N = 4 * n_nodes
    M = sp.coo_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(N, N)).tocsr()
    M.sum_duplicates()
    return M


def system_matrix_ibc(problem, plate, sigma_p, mu_p=MU0, which="vacuum"):
    """The constrained matrix of configuration `which` with the plate tets removed and the
    impedance condition on their surface (the coefficients of the other tets are those
    of `which`)."""
    m = problem.mesh
    plate = np.asarray(plate, dtype=bool)
    s, nu = fem.effective_coefficients(problem.sigma, problem.nu, problem.sigma_d, problem.nu_d, which)
    keep = ~plate
    M = fem.assemble_raw(m.xyz, m.tets[keep], s[keep], nu[keep], problem.nu_tilde, problem.omega, problem.delta)
    faces, normals = plate_surface(m.xyz, m.tets, plate)
    Z = surface_impedance(problem.omega, sigma_p, mu_p)
    M = M + surface_matrix(m.xyz, faces, normals, m.n_nodes, -1j * problem.omega / Z)
    cond = fem.conducting_nodes(m.n_nodes, m.tets[keep], s[keep])
    d, v = fem.fixed_dofs(m.bc_mask, cond)
    inside = np.ones(m.n_nodes, dtype=bool)
    inside[np.asarray(m.tets)[keep].ravel()] = False      # nodes touching only plate tets
    void = (4 * np.nonzero(inside)[0][:, None] + np.arange(3)[None]).ravel()
    d = np.union1d(d, void)                               # their V dofs are already in v
    return fem.apply_constraints(M, d, np.setdiff1d(v, d)), (d, v)


def constrain_rhs_ibc(b, fixed):
    """Zero the load at the fixed dofs of an IBC configuration."""
    d, v = fixed
    b = np.array(b, dtype=np.complex128, copy=True)
    b[..., d] = 0.0
    b[..., v] = 0.0
    return b
