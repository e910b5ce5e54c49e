"""Oracle: the coil source term and its load vector.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4 gives the source as a divergence-free azimuthal current on the coil,
J = J_e (-y, x, 0)/sqrt(x^2 + y^2), and Sec. 3 says the discrete source is
"the mass matrix times the interpolation of J".  Reading: the mass matrix is
assembled over the coil tets only, each weighted by the fraction f_K of 35
interior sample points (barycentric weights (4 n_a + 1)/20, sum n_a = 4)
that lie inside the coil annulus, and J is
interpolated at that tet's nodes:

    b_(a,i) = sum_{K containing a} f_K |K|/20 (J_i(x_a) + sum_{b in K} J_i(x_b)),

which is sum_b f_K int_K l_a l_b J_i(x_b).  V rows carry no load.
"""
from __future__ import annotations

import numpy as np

from .fem import tet_geometry

# the 35 sample points: barycentric weights (4 n_a + 1)/20 with n_a >= 0,
# n0+n1+n2+n3 = 4 (the degree-4 lattice shrunk by 4/5 about the centroid)
_LAT = np.array([(4 * a + 1, 4 * b + 1, 4 * c + 1, 4 * (4 - a - b - c) + 1)
                 for a in range(5) for b in range(5 - a) for c in range(5 - a - b)],
                dtype=np.float64)


def coil_fraction(xyz, tets, coil, z_probe):
    """f_K for every tet: share of lattice points inside the coil.

    Sample point = (((m0 x0 + m1 x1) + m2 x2) + m3 x3) * 0.05 with m_a the
    integer weights 4 n_a + 1 (every operation rounded separately in
    float64); it is inside when
    r_in^2 <= x^2 + y^2 <= r_out^2 and |z - (z_probe + z_offset)| <= length/2
    """
    r_in, r_out, length, z_off, _ = coil
    p = np.asarray(xyz, dtype=np.float64)[np.asarray(tets)]    # (T,4,3)
    acc = None
    for a in range(4):
        term = _LAT[None, :, a, None] * p[:, None, a, :]
        acc = term if acc is None else acc + term
    pts = acc * 0.05
    x, y, z = pts[..., 0], pts[..., 1], pts[..., 2]
    r2 = x * x + y * y
    zc = z_probe + z_off
    inside = ((r2 >= r_in * r_in) & (r2 <= r_out * r_out)
              & (np.abs(z - zc) <= 0.5 * length))
    return inside.sum(axis=1) / 35.0


def source_at_nodes(xyz, J_e):
    """J at the nodes: J_e (-y, x, 0)/r, zero on the axis (r < 1e-12)."""
    x = xyz[:, 0]
    y = xyz[:, 1]
    r = np.sqrt(x * x + y * y)
    on_axis = r < 1e-12
    rs = np.where(on_axis, 1.0, r)
    J = np.zeros((xyz.shape[0], 3))
    J[:, 0] = np.where(on_axis, 0.0, -J_e * y / rs)
    J[:, 1] = np.where(on_axis, 0.0, J_e * x / rs)
    return J


def coil_rhs(xyz, tets, coil, z_probe):
    """Load vector b (4N,) complex for one coil at one probe position."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    f = coil_fraction(xyz, tets, coil, z_probe)
    sel = np.nonzero(f > 0.0)[0]
    N = xyz.shape[0]
    b = np.zeros((N, 4), dtype=np.complex128)
    if sel.size == 0:
        return b.ravel()
    t = tets[sel]
    vol, _ = tet_geometry(xyz, t)
    J = source_at_nodes(xyz, coil[4])
    Jt = J[t]                                        # (S,4,3)
    w = (f[sel] * vol / 20.0)[:, None, None]
    contrib = w * (Jt + Jt.sum(axis=1, keepdims=True))
    for a in range(4):
        np.add.at(b, (t[:, a], slice(0, 3)), contrib[:, a, :])
    return b.ravel()
