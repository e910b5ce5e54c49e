"""Pins for the oracle's element matrices and assembly (CPU only).

Each test checks the oracle against something the mathematics fixes, not
against a retyped copy of its own formulas:
  * barycentric gradients reproduce linear functions;
  * the P1 mass formula against a degree-2 quadrature rule;
  * element matrices are complex symmetric;
  * K_P1 * 1 = 0 and sum of the mass matrix = |Omega|;
  * curl-curl + div-div with nu = nu_tilde equals the vector Laplacian
    nu (I_3 x K_P1) after A.n = 0 elimination (null-Lagrangian identity);
  * a Dirichlet solve reproduces a linear (A, V) field exactly (P1 patch test);
  * manufactured smooth solution: second-order nodal convergence;
  * skin-effect decay exp(-(1-i) z / delta) with delta = sqrt(2/(omega mu sigma))
    from the skin depth formula of Sec. 2 (Eq. IBC text).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import ect_inputs as E
from oracle import fem
from tests.helpers import QUAD4, dirichlet_solve, hat_gradients_4x4, quad_load


def small_mesh(shape=(4, 4, 5), lengths=(1.0, 1.2, 1.5), jitter=0.15, seed=3):
    return E.box_mesh(shape, lengths, (2, 2, 2), jitter=jitter, seed=seed)


def test_gradients_reproduce_linear_functions():
    m = small_mesh()
    vol, g = fem.tet_geometry(m.xyz, m.tets)
    assert np.all(vol > 0)
    p = m.xyz[m.tets]
    # sum_a g_a = 0 and sum_a x_a (x) g_a = I
    assert np.abs(g.sum(axis=1)).max() < 1e-12 * np.abs(g).max()
    I = np.einsum("kai,kaj->kij", p, g)
    assert np.abs(I - np.eye(3)).max() < 1e-12
    # independent route: inverse of the 4x4 vertex matrix
    for k in range(0, m.n_tets, 7):
        np.testing.assert_allclose(g[k], hat_gradients_4x4(p[k]), rtol=0, atol=1e-10 * np.abs(g[k]).max())
    # volumes: sum = box volume
    assert abs(vol.sum() - np.prod(m.lengths)) < 1e-12


def test_mass_formula_matches_quadrature():
    m = small_mesh()
    vol, g = fem.tet_geometry(m.xyz, m.tets)
    E0 = fem.element_matrices(vol, g, np.ones(m.n_tets), np.zeros(m.n_tets), 0.0, 1.0, 0.0)
    # with nu = nu_t = 0, sigma = omega = 1: AA_ii = -i * int l_a l_b
    mass = -E0[:, :, :, 0, 0].imag
    quad = np.einsum("qa,qb->ab", QUAD4, QUAD4)[None] * (vol / 4.0)[:, None, None]
    np.testing.assert_allclose(mass, quad, rtol=1e-13, atol=0)
    assert abs(mass.sum() - vol.sum()) < 1e-13


def test_element_matrices_complex_symmetric():
    m = small_mesh()
    vol, g = fem.tet_geometry(m.xyz, m.tets)
    rng = np.random.default_rng(0)
    E0 = fem.element_matrices(vol, g, rng.uniform(0, 2e6, m.n_tets), rng.uniform(1e5, 1e6, m.n_tets),
                              7e5, 2 * math.pi * 1e5, 3.0)
    Et = np.transpose(E0, (0, 2, 1, 4, 3))
    assert np.abs(E0 - Et).max() <= 1e-15 * np.abs(E0).max()


def test_scalar_laplacian_kernel_and_mass_total():
    m = small_mesh()
    vol, g = fem.tet_geometry(m.xyz, m.tets)
    E0 = fem.element_matrices(vol, g, np.zeros(m.n_tets), np.ones(m.n_tets), 0.0, 1.0, 0.0)
    # with sigma = 0, nu = 1, nu_t = 0: AA_00 = |K| g_a.g_b + |K|(0 - g_a0 g_b0)
    # the x-x entry of curl-curl is |K|(g_a.g_b - g_a0 g_b0); its row sums vanish
    rows = E0[:, :, :, 0, 0].real.sum(axis=2)
    assert np.abs(rows).max() < 1e-12 * np.abs(E0).max()
    M = fem.assemble_raw(m.xyz, m.tets, np.ones(m.n_tets), np.zeros(m.n_tets), 0.0, 1.0, 0.0)
    # global mass (imag of -M on A_x dofs) sums to |Omega|
    Ax = np.arange(m.n_nodes) * 4
    assert abs(-M[Ax][:, Ax].sum().imag - np.prod(m.lengths)) < 1e-12


def _scalar_p1_stiffness(xyz, tets):
    """K_P1 assembled from hat gradients of the 4x4 vertex matrix."""
    N = xyz.shape[0]
    rows, cols, vals = [], [], []
    for t in tets:
        p = xyz[t]
        G = hat_gradients_4x4(p)
        v = abs(np.linalg.det(p[1:] - p[0])) / 6.0
        K = v * G @ G.T
        for a in range(4):
            for b in range(4):
                rows.append(t[a]); cols.append(t[b]); vals.append(K[a, b])
    return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


def test_vector_laplacian_identity():
    """curl-curl + div-div (nu = nu_t) = nu (I3 x K_P1) after A.n = 0 elimination."""
    m = small_mesh(shape=(4, 5, 4), jitter=0.15)
    nu = 2.5
    M = fem.assemble_raw(m.xyz, m.tets, np.zeros(m.n_tets), np.full(m.n_tets, nu), nu, 1.0, 0.0)
    cond = np.zeros(m.n_nodes, dtype=bool)
    d, v = fem.fixed_dofs(m.bc_mask, cond)
    M = fem.apply_constraints(M, d, v).toarray()
    K = _scalar_p1_stiffness(m.xyz, m.tets).toarray()
    N = m.n_nodes
    expect = np.zeros((4 * N, 4 * N), dtype=np.complex128)
    for c in range(3):
        expect[c::4, c::4] = nu * K
    keep = np.ones(4 * N)
    keep[np.concatenate([d, v])] = 0
    expect = expect * keep[:, None] * keep[None, :]
    expect[np.concatenate([d, v]), np.concatenate([d, v])] = 1.0
    assert np.abs(M - expect).max() < 1e-12 * np.abs(expect).max()


def test_assembled_matrix_symmetric():
    p = E.wall_loss_problem((5, 5, 8), (20e-3, 20e-3, 40e-3), (2, 2, 2), 0.15, 1)
    M = fem.system_matrix(p, "defect")
    D = abs(M - M.T)
    assert D.max() <= 1e-14 * abs(M).max()


def test_linear_patch_reproduced_exactly():
    """P1 reproduces a linear divergence-free A and linear V (delta = 0)."""
    m = small_mesh(shape=(5, 5, 5), lengths=(1.0, 1.0, 1.0), jitter=0.15, seed=7)
    sig, nu, nut, om = 3.0, 1.7, 0.9, 2.0
    rng = np.random.default_rng(5)
    G = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    G[2, 2] = -(G[0, 0] + G[1, 1])               # div A = 0
    A0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    vg = rng.normal(size=3) + 1j * rng.normal(size=3)
    V0 = 0.3 - 0.2j

    def field(x):
        A = A0[None] + x @ G.T
        V = V0 + x @ vg
        return A, V

    def source(x):                                # J = -sigma (i omega A + grad V)
        A, _ = field(x)
        out = np.zeros((x.shape[0], 4), dtype=np.complex128)
        out[:, :3] = -sig * (1j * om * A + vg[None])
        return out

    M = fem.assemble_raw(m.xyz, m.tets, np.full(m.n_tets, sig), np.full(m.n_tets, nu), nut, om, 0.0)
    f = quad_load(m.xyz, m.tets, source)
    A, V = field(m.xyz)
    exact = np.concatenate([A, V[:, None]], axis=1).ravel()
    bnd = np.nonzero(m.bc_mask > 0)[0]
    fixed = (4 * bnd[:, None] + np.arange(4)[None]).ravel()
    u = dirichlet_solve(M, f, fixed, exact[fixed])
    assert np.abs(u - exact).max() <= 1e-12 * np.abs(exact).max()


def test_manufactured_solution_second_order():
    """Smooth (A, V) with all-Dirichlet data: nodal error falls ~4x per halving of h."""
    sig, nu, nut, om = 2.0, 1.0, 1.5, 3.0
    pi = math.pi

    def exact(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        A = np.stack([np.sin(pi * Y) * np.cos(Z), np.sin(X) * Z * Z, np.cos(pi * X * Y)], axis=1)
        V = np.exp(X) * np.sin(Y + Z)
        return A.astype(np.complex128), V.astype(np.complex128)

    def source(x):
        # J = nu curl curl A - nu_t grad div A - sigma E, f_V = (sigma/(i omega)) div E,
        # E = i omega A + grad V  (derivatives worked out by hand below)
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        A, V = exact(x)
        # vector Laplacian and grad div of A
        lapA = np.stack([-pi * pi * np.sin(pi * Y) * np.cos(Z) - np.sin(pi * Y) * np.cos(Z),
                         -np.sin(X) * Z * Z + 2.0 * np.sin(X),
                         -pi * pi * (X * X + Y * Y) * np.cos(pi * X * Y)], axis=1)
        # div A = 0 + 0 + 0 (A_x indep. of x, A_y indep. of y, A_z indep. of z)
        graddiv = np.zeros_like(lapA)
        curlcurl = graddiv - lapA
        gradV = np.stack([np.exp(X) * np.sin(Y + Z), np.exp(X) * np.cos(Y + Z),
                          np.exp(X) * np.cos(Y + Z)], axis=1)
        Ef = 1j * om * A + gradV
        lapV = np.exp(X) * np.sin(Y + Z) - 2.0 * np.exp(X) * np.sin(Y + Z)
        divE = 1j * om * 0.0 + lapV
        out = np.zeros((x.shape[0], 4), dtype=np.complex128)
        out[:, :3] = nu * curlcurl - nut * graddiv - sig * Ef
        out[:, 3] = (sig / (1j * om)) * divE
        return out

    errs = []
    for n in (5, 9, 17):
        m = E.box_mesh((n, n, n), (1.0, 1.0, 1.0), (2, 2, 2), jitter=0.0)
        xyz = m.xyz + 0.5                          # box [0,1]^3
        M = fem.assemble_raw(xyz, m.tets, np.full(m.n_tets, sig), np.full(m.n_tets, nu), nut, om, 0.0)
        f = quad_load(xyz, m.tets, source)
        A, V = exact(xyz)
        ex = np.concatenate([A, V[:, None]], axis=1).ravel()
        bnd = np.nonzero(m.bc_mask > 0)[0]
        fixed = (4 * bnd[:, None] + np.arange(4)[None]).ravel()
        u = dirichlet_solve(M, f, fixed, ex[fixed])
        errs.append(np.abs(u - ex).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[2] < 1e-2
    assert r1 > 3.0 and r2 > 3.3, errs


def _skin_solution(nz, L, sigma, freq):
    """Ax(z) driven at z = 0 in a uniform conductor column (V fixed to 0)."""
    w = 2.0 * L / (nz - 1)                          # cubic cells: lateral h = h_z
    m = E.box_mesh((3, 3, nz), (w, w, L), (1, 1, 1), jitter=0.0)
    xyz = m.xyz.copy()
    xyz[:, 2] += 0.5 * L                            # z in [0, L]
    om = 2 * math.pi * freq
    M = fem.assemble_raw(xyz, m.tets, np.full(m.n_tets, sigma), np.full(m.n_tets, E.NU0), E.NU0, om, 0.0)
    N = m.n_nodes
    z = xyz[:, 2]
    onx = np.isclose(np.abs(xyz[:, 0]), 0.5 * w)
    ony = np.isclose(np.abs(xyz[:, 1]), 0.5 * w)
    z0 = np.isclose(z, 0.0)
    zL = np.isclose(z, L)
    fixed, vals = [], []
    for a in range(N):
        fixed.append(4 * a + 3); vals.append(0.0)               # V = 0
        if onx[a] or z0[a] or zL[a]:
            fixed.append(4 * a + 2); vals.append(0.0)           # A_z = 0
        if ony[a] or z0[a] or zL[a]:
            fixed.append(4 * a + 1); vals.append(0.0)           # A_y = 0
        if z0[a]:
            fixed.append(4 * a + 0); vals.append(1.0)           # drive A_x = 1
        elif zL[a]:
            fixed.append(4 * a + 0); vals.append(0.0)
    fixed = np.array(fixed); vals = np.array(vals, dtype=np.complex128)
    order = np.argsort(fixed)
    u = dirichlet_solve(M, np.zeros(4 * N, dtype=np.complex128), fixed[order], vals[order])
    return z, u[0::4]


def test_skin_depth_decay():
    freq, sigma = 1.0e5, 1.0e6
    delta = math.sqrt(2.0 / (2 * math.pi * freq * E.MU0 * sigma))
    assert abs(delta - 1.5915e-3) < 1e-6            # 1.59 mm at 100 kHz, 1 MS/m
    L = 12 * delta
    errs = []
    for nz in (25, 49, 97):
        z, ax = _skin_solution(nz, L, sigma, freq)
        exact = np.exp(-(1 - 1j) * z / delta)
        sel = z < 4 * delta
        errs.append(np.abs(ax[sel] - exact[sel]).max())
    assert errs[-1] < 5e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5, errs


def _scalar_p1_mass_quadrature(xyz, tets, weight):
    """sum_K weight_K int_K l_a l_b by the 4-point rule (hat values = barycentric weights)."""
    N = xyz.shape[0]
    p = xyz[tets]
    vol = np.abs(np.linalg.det(p[:, 1:] - p[:, :1])) / 6.0
    loc = np.einsum("qa,qb->ab", QUAD4, QUAD4) / 4.0            # int l_a l_b / |K|
    vals = (weight * vol)[:, None, None] * loc[None]
    r = np.repeat(tets, 4, axis=1).ravel()
    c = np.tile(tets, (1, 4)).ravel()
    return sp.coo_matrix((vals.ravel(), (r, c)), shape=(N, N)).tocsr()


def _weighted_p1_stiffness(xyz, tets, weight):
    """sum_K weight_K |K| grad l_a . grad l_b with gradients from the 4x4 vertex matrix."""
    N = xyz.shape[0]
    rows, cols, vals = [], [], []
    for t, wk in zip(tets, weight):
        p = xyz[t]
        G = hat_gradients_4x4(p)
        v = abs(np.linalg.det(p[1:] - p[0])) / 6.0
        K = wk * v * G @ G.T
        for a in range(4):
            for b in range(4):
                rows.append(t[a]); cols.append(t[b]); vals.append(K[a, b])
    return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


@pytest.mark.parametrize("delta", [0.0, 1.0, 7.3e3])
def test_gauge_penalty_block_closed_form(delta):
    """V-V block of the coupled form with the gauge penalty of Sec. 4:
    -(1/(i omega)) [K_sigma + delta M_sigma], where K_sigma and M_sigma are the
    sigma-weighted P1 stiffness and mass matrices built here by independent
    routes (4x4 vertex-matrix gradients, 4-point quadrature).  A dropped sigma,
    a wrong mass weight (1/12 for 1/20) or delta on the stiffness fails it."""
    m = small_mesh(shape=(4, 5, 4), jitter=0.15, seed=11)
    rng = np.random.default_rng(4)
    sig = rng.uniform(0.5e6, 2.0e6, m.n_tets)                    # tet-wise conductivity
    om = 2 * math.pi * 1.0e5
    M = fem.assemble_raw(m.xyz, m.tets, sig, np.zeros(m.n_tets), 0.0, om, delta)
    V = 4 * np.arange(m.n_nodes) + 3
    MVV = M[V][:, V].toarray()
    K = _weighted_p1_stiffness(m.xyz, m.tets, sig).toarray()
    Ms = _scalar_p1_mass_quadrature(m.xyz, m.tets, sig).toarray()
    expect = -(1.0 / (1j * om)) * (K + delta * Ms)
    assert np.abs(MVV - expect).max() <= 1e-13 * np.abs(expect).max()
    # the penalty touches nothing but the V-V block
    M0 = fem.assemble_raw(m.xyz, m.tets, sig, np.zeros(m.n_tets), 0.0, om, 0.0)
    D = (M - M0).tocoo()
    assert np.all(D.row % 4 == 3) and np.all(D.col % 4 == 3)


def test_gauge_penalty_on_constant_potential():
    """K 1 = 0, so a constant V is seen only through the penalty:
    (M_VV 1)_a = -(delta/(i omega)) sum_{K ni a} sigma_K |K| / 4, and the total is
    -(delta/(i omega)) int sigma (the lumped P1 mass, int l_a = |K|/4 per tet)."""
    m = small_mesh(shape=(5, 4, 4), jitter=0.15, seed=12)
    rng = np.random.default_rng(6)
    sig = rng.uniform(0.5e6, 2.0e6, m.n_tets)
    om, delta = 2 * math.pi * 3.0e4, 42.0
    M = fem.assemble_raw(m.xyz, m.tets, sig, np.zeros(m.n_tets), 0.0, om, delta)
    V = 4 * np.arange(m.n_nodes) + 3
    y = M[V][:, V] @ np.ones(m.n_nodes)
    p = m.xyz[m.tets]
    vol = np.abs(np.linalg.det(p[:, 1:] - p[:, :1])) / 6.0
    lumped = np.zeros(m.n_nodes)
    np.add.at(lumped, m.tets.ravel(), np.repeat(sig * vol / 4.0, 4))
    expect = -(delta / (1j * om)) * lumped
    assert np.abs(y - expect).max() <= 1e-12 * np.abs(expect).max()
    assert abs(y.sum() - (-(delta / (1j * om)) * (sig * vol).sum())) <= 1e-12 * abs(y.sum())
