"""Pins for the oracle's impedance boundary condition (Sec. 2, Eq. IBC and
ibcROTA): the plate volume replaced by -(i omega/Z) int A_tau . Phi_tau on
its surface, Z = (1 - i)/(delta sigma_p).

  * half-space: for a conducting half-space the condition is exact, and the
    field above it is linear in z, A_x = C (1 + (1 - i) z / delta); P1
    reproduces linear fields, so the discrete solution must equal it at every
    node (to rounding).  A wrong sign of the term, Z for 1/Z, a missing
    tangential projector or 1/6 for 1/12 in the surface mass all fail;
  * the surface form is complex symmetric and acts on tangential components
    only (normal components of A see nothing);
  * surface extraction: on a structured mesh with a box-shaped plate, the
    faces found are exactly the plate's exposed faces, their total area is
    the plate's exposed area and every normal points into the plate;
  * skin-depth agreement: the air field above a volume-meshed conducting
    slab converges to the IBC field as the slab mesh is refined below the
    skin depth;
  * the support-plate problem: Delta Z with the IBC has the sign and the
    magnitude of the volume model's on a coarse mesh (agreement within tens
    of percent there, not to rounding: the volume model is under-resolved).
"""
import math

import numpy as np
import pytest

import ect_inputs as E
from oracle import fem, ibc, impedance, rhs, solve
from tests.helpers import dirichlet_solve


def _column(nz, L, w):
    m = E.box_mesh((3, 3, nz), (w, w, L), (1, 1, 1), jitter=0.0)
    xyz = m.xyz.copy()
    xyz[:, 2] += 0.5 * L                          # z in [0, L]
    return m, xyz


@pytest.mark.parametrize("nz", [5, 12])
def test_half_space_field_is_reproduced_exactly(nz):
    freq, sig_p = 1.0e5, 1.4e6
    om = 2 * math.pi * freq
    delta = math.sqrt(2.0 / (om * E.MU0 * sig_p))
    L, w = 4.0 * delta, 1.0 * delta
    m, xyz = _column(nz, L, w)
    N = m.n_nodes
    M = fem.assemble_raw(xyz, m.tets, np.zeros(m.n_tets), np.full(m.n_tets, E.NU0), E.NU0, om, 0.0)
    z = xyz[:, 2]
    bottom = np.isclose(z, 0.0)
    tri = []
    for t in m.tets:
        on = [a for a in t if bottom[a]]
        if len(on) == 3:
            tri.append(on)
    tri = np.array(tri)
    normals = np.tile([0.0, 0.0, -1.0], (len(tri), 1))       # out of the air column, into the conductor
    Z = ibc.surface_impedance(om, sig_p, E.MU0)
    M = M + ibc.surface_matrix(xyz, tri, normals, N, -1j * om / Z)
    onx = np.isclose(np.abs(xyz[:, 0]), 0.5 * w)
    ony = np.isclose(np.abs(xyz[:, 1]), 0.5 * w)
    top = np.isclose(z, L)
    fixed, vals = [], []
    for a in range(N):
        fixed.append(4 * a + 3); vals.append(0.0)               # no V (no conductor in the column)
        if onx[a] or bottom[a] or top[a]:
            fixed.append(4 * a + 2); vals.append(0.0)           # A_z = 0
        if ony[a] or bottom[a] or top[a]:
            fixed.append(4 * a + 1); vals.append(0.0)           # A_y = 0
        if top[a]:
            fixed.append(4 * a + 0); vals.append(1.0)           # drive A_x = 1 at the top
    fixed = np.array(fixed); vals = np.array(vals, dtype=np.complex128)
    order = np.argsort(fixed)
    u = dirichlet_solve(M, np.zeros(4 * N, dtype=np.complex128), fixed[order], vals[order])
    C = 1.0 / (1.0 + (1.0 - 1.0j) * L / delta)
    exact = C * (1.0 + (1.0 - 1.0j) * z / delta)
    assert np.abs(u[0::4] - exact).max() <= 1e-12
    assert np.abs(u[1::4]).max() <= 1e-12 and np.abs(u[2::4]).max() <= 1e-12


def test_surface_form_symmetric_and_tangential():
    rng = np.random.default_rng(3)
    xyz = rng.normal(size=(6, 3))
    tri = np.array([[0, 1, 2], [2, 3, 4], [1, 4, 5]])
    normals = []
    for t in tri:
        n = np.cross(xyz[t[1]] - xyz[t[0]], xyz[t[2]] - xyz[t[0]])
        normals.append(n / np.linalg.norm(n))
    normals = np.array(normals)
    S = ibc.surface_matrix(xyz, tri, normals, 6, 2.0 - 3.0j).toarray()
    assert np.abs(S - S.T).max() <= 1e-15 * np.abs(S).max()
    assert np.abs(S[3::4]).max() == 0.0 and np.abs(S[:, 3::4]).max() == 0.0   # V untouched
    # a field normal to one triangle everywhere on it sees nothing from that triangle
    one = ibc.surface_matrix(xyz, tri[:1], normals[:1], 6, 1.0).toarray()
    A = np.zeros(24)
    for a in tri[0]:
        A[4 * a:4 * a + 3] = normals[0]
    assert np.abs(one @ A).max() <= 1e-15
    # total surface mass of a tangential constant field = coef * area
    t0 = np.cross(normals[0], [1.0, 0.0, 0.0]); t0 /= np.linalg.norm(t0)
    B = np.zeros(24)
    for a in tri[0]:
        B[4 * a:4 * a + 3] = t0
    area = 0.5 * np.linalg.norm(np.cross(xyz[1] - xyz[0], xyz[2] - xyz[0]))
    assert abs(B @ one @ B - area) <= 1e-14 * area


def test_plate_surface_of_a_box_plate():
    m = E.box_mesh((6, 6, 8), (5.0, 5.0, 7.0), (1, 1, 1))
    c = E.centroids(m)
    plate = (np.abs(c[:, 0]) < 1.5) & (np.abs(c[:, 1]) < 1.5) & (c[:, 2] > -1.5) & (c[:, 2] < 1.5)
    faces, normals = ibc.plate_surface(m.xyz, m.tets, plate)
    # the plate is the 3 x 3 x 3 block of cells in the middle: 6 sides of 9 unit squares, 2 triangles each
    assert len(faces) == 6 * 9 * 2
    area = sum(0.5 * np.linalg.norm(np.cross(m.xyz[f[1]] - m.xyz[f[0]], m.xyz[f[2]] - m.xyz[f[0]])) for f in faces)
    assert abs(area - 54.0) < 1e-12
    cen = m.xyz[faces].mean(axis=1)
    assert np.all(np.einsum("fi,fi->f", normals, -cen) > 0)        # into the plate (centred at the origin)


def _air_over_conductor(nz_air, nz_cond, L, D, w, sig_p, om):
    """Column: conductor slab z in [-D, 0] (volume-meshed), air z in [0, L], A_x = 1 at the
    top, A = 0 at the bottom of the slab; returns (z of the air nodes, A_x there)."""
    nz = nz_air + nz_cond - 1
    m = E.box_mesh((3, 3, nz), (w, w, L + D), (1, 1, 1), jitter=0.0)
    xyz = m.xyz.copy()
    # grade: nz_cond layers over [-D, 0], nz_air layers over [0, L]
    k = np.round((xyz[:, 2] + 0.5 * (L + D)) / (L + D) * (nz - 1)).astype(int)
    zc = np.where(k < nz_cond, -D + D * k / (nz_cond - 1), L * (k - (nz_cond - 1)) / (nz_air - 1))
    xyz[:, 2] = zc
    c = xyz[m.tets].mean(axis=1)
    sig = np.where(c[:, 2] < 0.0, sig_p, 0.0)
    M = fem.assemble_raw(xyz, m.tets, sig, np.full(m.n_tets, E.NU0), E.NU0, om, 0.0)
    N = m.n_nodes
    onx = np.isclose(np.abs(xyz[:, 0]), 0.5 * w)
    ony = np.isclose(np.abs(xyz[:, 1]), 0.5 * w)
    top, bot = np.isclose(xyz[:, 2], L), np.isclose(xyz[:, 2], -D)
    fixed, vals = [], []
    for a in range(N):
        fixed.append(4 * a + 3); vals.append(0.0)
        if onx[a] or top[a] or bot[a]:
            fixed.append(4 * a + 2); vals.append(0.0)
        if ony[a] or top[a] or bot[a]:
            fixed.append(4 * a + 1); vals.append(0.0)
        if top[a] or bot[a]:
            fixed.append(4 * a + 0); vals.append(1.0 if top[a] else 0.0)
    fixed = np.array(fixed); vals = np.array(vals, dtype=np.complex128)
    order = np.argsort(fixed)
    u = dirichlet_solve(M, np.zeros(4 * N, dtype=np.complex128), fixed[order], vals[order])
    air = xyz[:, 2] >= 0.0
    return xyz[air, 2], u[0::4][air]


def test_volume_conductor_approaches_the_ibc_field_as_h_shrinks():
    """Skin-depth agreement: the air field above a volume-meshed conducting slab (thickness
    8 delta) converges, as the mesh inside the slab is refined, to the field the IBC gives,
    which is exact for a half-space (previous test)."""
    freq, sig_p = 1.0e5, 1.4e6
    om = 2 * math.pi * freq
    delta = math.sqrt(2.0 / (om * E.MU0 * sig_p))
    L, D, w = 4.0 * delta, 8.0 * delta, 0.5 * delta
    C = 1.0 / (1.0 + (1.0 - 1.0j) * L / delta)
    errs = []
    for nzc in (9, 17, 33, 65):                        # h = delta, delta/2, delta/4, delta/8 in the slab
        z, ax = _air_over_conductor(5, nzc, L, D, w, sig_p, om)
        ibc_field = C * (1.0 + (1.0 - 1.0j) * z / delta)
        errs.append(np.abs(ax - ibc_field).max())
    assert errs[-1] < 1e-3
    # measured ratios 3.0, 2.5, 2.3 per halving: at least first order (the tet mass couples a
    # node to its lateral neighbours unevenly, so the 3-D solution of this 1-D field carries a
    # small O(h) lateral ripple on top of the second-order error)
    assert all(errs[i] / errs[i + 1] > 1.8 for i in range(len(errs) - 1)), errs


def test_ibc_delta_z_on_the_support_plate_problem():
    """Support plate with the IBC against the volume-meshed plate on the same coarse mesh
    (h ~ 1.7 delta inside the plate, so the volume model itself is under-resolved there):
    the same sign and magnitude, reciprocity exact."""
    p = E.tsp_problem((14, 14, 36), (30e-3, 30e-3, 60e-3), (2, 2, 4), 0.0, 0, z_pos=(10e-3,))
    plate = np.isfinite(p.sigma_d)
    M0 = fem.system_matrix(p, "vacuum")
    Mv = fem.system_matrix(p, "defect")
    Mi, fixed = ibc.system_matrix_ibc(p, plate, E.SIGMA_TSP, which="vacuum")
    assert abs(Mi - Mi.T).max() <= 1e-14 * abs(Mi).max()
    b = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), 10e-3), p, "vacuum")
         for c in p.coils]
    bi = [ibc.constrain_rhs_ibc(bk, fixed) for bk in b]
    assert all(np.array_equal(x, y) for x, y in zip(b, bi))            # the coil is outside the plate
    u0 = [solve.superlu_solve(M0, bk)[0] for bk in b]
    uv = [solve.superlu_solve(Mv, bk)[0] for bk in b]
    ui = [solve.superlu_solve(Mi, bk)[0] for bk in b]
    I = [c.current for c in p.coils]
    dzv = impedance.delta_z_emf_matrix(b, u0, uv, I, p.omega)
    dzi = impedance.delta_z_emf_matrix(b, u0, ui, I, p.omega)
    rel = np.abs(dzi - dzv).max() / np.abs(dzv).max()
    assert rel < 0.6, (rel, dzv[0, 0], dzi[0, 0])
    assert np.all(np.sign(dzi.real) == np.sign(dzv.real)) and np.all(np.sign(dzi.imag) == np.sign(dzv.imag))
    assert abs(dzi[0, 1] - dzi[1, 0]) <= 1e-8 * np.abs(dzi).max()     # reciprocity
