"""Pins for the oracle's coil load, linear solvers and impedance (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import ect_inputs as E
from oracle import fem, impedance, rhs, solve
from tests.helpers import QUAD4


# ---------------------------------------------------------------- coil load

def test_sample_points_interior_and_symmetric():
    lat = rhs._LAT / 20.0
    assert lat.shape == (35, 4)
    np.testing.assert_allclose(lat.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert np.all(lat > 0)                                # strictly interior
    assert len({tuple(r) for r in lat}) == 35
    np.testing.assert_allclose(lat.mean(axis=0), 0.25, rtol=1e-14)   # centred


def test_coil_volume_and_moment_converge():
    """Sum f_K |K| -> coil volume; sum_a (x_a x b_a)_z -> J_e int r dV."""
    coil = E.Coil()
    vol_exact = math.pi * (coil.r_out ** 2 - coil.r_in ** 2) * coil.length
    mom_exact = coil.J_e * 2 * math.pi * coil.length * (coil.r_out ** 3 - coil.r_in ** 3) / 3
    errs = []
    for n in (21, 41):
        m = E.box_mesh((n, n, n // 4 + 1), (20e-3, 20e-3, 5e-3), (2, 2, 2))
        f = rhs.coil_fraction(m.xyz, m.tets, coil.as_tuple(), 0.0)
        vol, _ = fem.tet_geometry(m.xyz, m.tets)
        b = rhs.coil_rhs(m.xyz, m.tets, coil.as_tuple(), 0.0).reshape(-1, 4)
        mom = np.sum(m.xyz[:, 0] * b[:, 1] - m.xyz[:, 1] * b[:, 0]).real
        errs.append((abs((f * vol).sum() / vol_exact - 1), abs(mom / mom_exact - 1)))
        assert np.all(b[:, 3] == 0) and np.all(b.imag == 0)
    assert errs[-1][0] < 0.03 and errs[-1][1] < 0.03, errs
    assert errs[-1][0] < errs[0][0] and errs[-1][1] < errs[0][1], errs


def test_coil_load_equals_quadrature_of_interpolated_source():
    """b_a = sum_K f_K int_K (P1 interpolant of J) l_a, with the 4-point rule."""
    p = E.wall_loss_problem((12, 12, 10), (20e-3, 20e-3, 10e-3), (2, 2, 2), 0.15, 2)
    m = p.mesh
    coil = p.coils[0].as_tuple()
    b = rhs.coil_rhs(m.xyz, m.tets, coil, 0.0).reshape(-1, 4)
    f = rhs.coil_fraction(m.xyz, m.tets, coil, 0.0)
    Jn = rhs.source_at_nodes(m.xyz, coil[4])
    expect = np.zeros((m.n_nodes, 4))
    for k in np.nonzero(f > 0)[0]:
        t = m.tets[k]
        P = m.xyz[t]
        vol = abs(np.linalg.det(P[1:] - P[0])) / 6.0
        for q in range(4):
            Jq = QUAD4[q] @ Jn[t]
            for a in range(4):
                expect[t[a], :3] += f[k] * 0.25 * vol * QUAD4[q, a] * Jq
    assert np.abs(b.real - expect).max() <= 1e-12 * np.abs(expect).max()
    assert (f > 0).sum() > 10


def test_source_is_azimuthal_unit():
    xyz = np.random.default_rng(1).normal(size=(50, 3))
    xyz[0, :2] = 0.0
    J = rhs.source_at_nodes(xyz, 2.0)
    assert np.all(J[0] == 0.0)
    np.testing.assert_allclose(np.linalg.norm(J[1:], axis=1), 2.0, rtol=1e-14)
    np.testing.assert_allclose(np.einsum("ij,ij->i", J[1:, :2], xyz[1:, :2]), 0.0, atol=1e-14)


# ---------------------------------------------------------------- solvers

def tiny_problem(shape=(5, 5, 6), seed=0):
    return E.wall_loss_problem(shape, (20e-3, 20e-3, 40e-3), (2, 2, 3), 0.15, seed)


def test_givens_rotation():
    rng = np.random.default_rng(2)
    for _ in range(20):
        a, b = rng.normal(size=2) + 1j * rng.normal(size=2)
        c, s, r = solve.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-14 * abs(r) and abs(out[0] - r) < 1e-14 * abs(r)
        np.testing.assert_allclose(G @ G.conj().T, np.eye(2), atol=1e-14)


def test_cgs2_orthogonality():
    rng = np.random.default_rng(3)
    n, k = 400, 12
    V, _ = np.linalg.qr(rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k)))
    w = rng.normal(size=n) + 1j * rng.normal(size=n)
    h, w2, beta = solve.cgs2(V, w)
    assert np.abs(V.conj().T @ w2).max() < 1e-13 * np.linalg.norm(w)
    np.testing.assert_allclose(V @ h + w2, w, atol=1e-13 * np.linalg.norm(w))
    assert abs(beta - np.linalg.norm(w2)) < 1e-14 * beta


def test_fgmres_matches_dense_on_random_system():
    rng = np.random.default_rng(4)
    n = 80
    A = np.eye(n) * 4 + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / math.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    x, info = solve.fgmres(A, b, tol=1e-13, restart=15)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11 * np.abs(x).max())
    assert info["relres"] <= 1e-13


def test_direct_and_krylov_solves_agree_on_tiny_mesh():
    p = tiny_problem()
    M = fem.system_matrix(p, "defect")
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "defect")
    assert np.linalg.norm(b) > 0
    xd = solve.dense_solve(M, b)
    xs, _ = solve.superlu_solve(M, b)
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    P = solve.block_jacobi(S, p.mesh.block_of_node)
    y, info = solve.fgmres(S, t * b, lambda r: solve.block_jacobi_apply(P, r), tol=1e-13, restart=300,
                           maxiter=5000)
    xk = t * y
    # every solver leaves a small scaled residual (backward error) ...
    for x, tol in ((xd, 1e-10), (xs, 1e-10), (xk, 1e-12)):
        assert np.linalg.norm(t * (b - M @ x)) <= tol * np.linalg.norm(t * b)
    # ... and the solutions agree to within kappa(M) times it
    kappa = np.linalg.cond(M.toarray())
    scale = np.linalg.norm(xd)
    assert np.linalg.norm(xs - xd) < kappa * 1e-15 * scale
    assert np.linalg.norm(xk - xd) < kappa * 1e-12 * scale
    assert np.linalg.norm(t * (b - M @ xk)) <= 1e-12 * np.linalg.norm(t * b)


def test_single_block_preconditioner_is_exact():
    p = tiny_problem((4, 4, 4))
    M = fem.system_matrix(p, "defect")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    P = solve.block_jacobi(S, np.zeros(p.mesh.n_nodes, dtype=np.int32))
    b = np.random.default_rng(5).normal(size=S.shape[0]) + 0j
    # the dense inverse is exact up to kappa * eps ~ 1e-10 here
    y, info = solve.fgmres(S, b, lambda r: solve.block_jacobi_apply(P, r), tol=1e-8)
    assert info["iters"] == 1


def test_block_jacobi_blocks_are_inverses():
    p = tiny_problem()
    M = fem.system_matrix(p, "vacuum")
    t = fem.scaling(M)
    S = fem.scaled(M, t).toarray()
    starts, stops, inv = solve.block_jacobi(S, p.mesh.block_of_node)
    assert starts[0] == 0 and stops[-1] == S.shape[0]
    for s, e, B in zip(starts, stops, inv):
        np.testing.assert_allclose(B @ S[s:e, s:e], np.eye(e - s), atol=1e-10)


# ---------------------------------------------------------------- impedance

def _solve_all(p):
    M0 = fem.system_matrix(p, "vacuum")
    Md = fem.system_matrix(p, "defect")
    b = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), p.z_pos[0]), p, "vacuum")
         for c in p.coils]
    u0 = [solve.dense_solve(M0, bk) for bk in b]
    ud = [solve.dense_solve(Md, bk) for bk in b]
    I = [c.current for c in p.coils]
    return M0, Md, b, u0, ud, I


def imp_problem(sigma_d=0.5e6, seed=0):
    p = E.wall_loss_problem((9, 9, 11), (20e-3, 20e-3, 20e-3), (3, 3, 3), 0.1, seed,
                            z_pos=(0.0,), sigma_d=sigma_d)
    return p


def test_reciprocity_equals_emf_difference_and_symmetry():
    p = imp_problem()
    M0, Md, b, u0, ud, I = _solve_all(p)
    dz = impedance.delta_z_matrix(M0, Md, u0, ud, I, p.omega)
    dze = impedance.delta_z_emf_matrix(b, u0, ud, I, p.omega)
    assert np.abs(dz).max() > 0
    assert np.abs(dz - dze).max() <= 1e-9 * np.abs(dz).max()
    assert abs(dz[0, 1] - dz[1, 0]) <= 1e-9 * np.abs(dz).max()


def test_zero_contrast_gives_zero():
    p = imp_problem(sigma_d=1.0e6)                 # same as the tube
    M0, Md, b, u0, ud, I = _solve_all(p)
    dz = impedance.delta_z_matrix(M0, Md, u0, ud, I, p.omega)
    assert np.all(dz == 0)


def test_born_limit_linear_in_contrast():
    r = []
    for eps in (1e-3, 5e-4):
        p = imp_problem(sigma_d=1.0e6 * (1 - eps))
        M0, Md, b, u0, ud, I = _solve_all(p)
        r.append(impedance.delta_z_matrix(M0, Md, u0, ud, I, p.omega)[0, 0] / eps)
    assert abs(r[0] - r[1]) <= 2e-3 * abs(r[1])


def test_insulator_impedance_is_inductive_and_conductor_passive():
    p = imp_problem()
    M0, Md, b, u0, ud, I = _solve_all(p)
    Z = np.array([[impedance.z_emf(b[k], u0[l], I[k], I[l], p.omega) for l in range(2)] for k in range(2)])
    assert Z[0, 0].real > 0 and Z[1, 1].real > 0            # passive: Re Z >= 0
    assert Z[0, 0].imag < 0                                 # inductive, exp(-i omega t)
    p.sigma = np.zeros_like(p.sigma)
    p.sigma_d = np.full_like(p.sigma_d, np.nan)
    M0 = fem.system_matrix(p, "vacuum")
    u = solve.dense_solve(M0, b[0])
    z = impedance.z_emf(b[0], u, I[0], I[0], p.omega)
    assert abs(z.real) <= 1e-12 * abs(z) and z.imag < 0


def test_signal_modes_as_printed():
    dz = np.array([[1 + 2j, 3 - 1j], [3 - 1j, -2 + 0.5j]])
    fa, f3 = impedance.signal_modes(dz)
    assert fa == 0.5j * (4 + 1j) and f3 == 0.5j * (3 + 1.5j)


# ---------------------------------------------------------------- conductor-V coarse space

def test_coarse_matrix_is_sum_of_unscaled_vv_couplings():
    """E_cd = sum over conducting nodes i in group c, j in group d of M[V_i, V_j] (brute force)."""
    p = tiny_problem((6, 6, 8), seed=4)
    M = fem.system_matrix(p, "defect")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "defect")
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    Z, E, Ei = solve.coarse_v(S, t, p.mesh.block_of_node, cond, 2)
    groups = sorted({int(b) // 2 for b in p.mesh.block_of_node[cond]})
    Md = M.toarray()
    ref = np.zeros((len(groups), len(groups)), dtype=complex)
    for i in np.nonzero(cond)[0]:
        for j in np.nonzero(cond)[0]:
            ci = groups.index(int(p.mesh.block_of_node[i]) // 2)
            cj = groups.index(int(p.mesh.block_of_node[j]) // 2)
            ref[ci, cj] += Md[4 * i + 3, 4 * j + 3]
    assert np.abs(E - ref).max() <= 1e-12 * np.abs(ref).max()
    np.testing.assert_allclose(Ei @ E, np.eye(len(groups)), atol=1e-9)


def test_coarse_correction_is_exact_on_the_coarse_space():
    p = tiny_problem((6, 6, 8), seed=5)
    M = fem.system_matrix(p, "vacuum")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "vacuum")
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    Z, E, Ei = solve.coarse_v(S, t, p.mesh.block_of_node, cond, 1)
    c = np.random.default_rng(0).normal(size=Z.shape[1]) + 0j
    r = S @ (Z @ c)
    np.testing.assert_allclose(Z @ (Ei @ (Z.T @ r)), Z @ c, atol=1e-9 * np.abs(Z @ c).max())


def test_two_level_removes_restart_stagnation():
    """One-level FGMRES(30) stalls near 1e-7 on this mesh; the coarse V space converges."""
    p = E.wall_loss_problem((9, 9, 12), (20e-3, 20e-3, 30e-3), (2, 2, 3), 0.1, 3, z_pos=(0.0,))
    M = fem.system_matrix(p, "vacuum")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    P = solve.block_jacobi(S, p.mesh.block_of_node)
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, p.sigma)
    C = solve.coarse_v(S, t, p.mesh.block_of_node, cond, 1)
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "vacuum")
    _, i1 = solve.fgmres(S, t * b, lambda r: solve.block_jacobi_apply(P, r), tol=1e-10, restart=30, maxiter=1500)
    _, i2 = solve.fgmres(S, t * b, lambda r: solve.two_level_apply(P, C, r), tol=1e-10, restart=30, maxiter=1500)
    assert i1["relres"] > 1e-9
    assert i2["relres"] <= 1e-10 and i2["iters"] < 400


def test_selective_reorthogonalisation():
    rng = np.random.default_rng(8)
    n, k = 300, 6
    V, _ = np.linalg.qr(rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k)))
    w = rng.normal(size=n) + 1j * rng.normal(size=n)          # mostly outside span(V): one pass
    h, w2, _ = solve.cgs2(V, w, selective=True)
    np.testing.assert_allclose(h, V.conj().T @ w, rtol=1e-13)
    w = V @ (rng.normal(size=k) + 0j) + 1e-6 * (rng.normal(size=n) + 0j)   # nearly inside: two passes
    h, w2, beta = solve.cgs2(V, w, selective=True)
    assert np.abs(V.conj().T @ w2).max() < 1e-13 * np.linalg.norm(w)
    p = tiny_problem()
    M = fem.system_matrix(p, "defect")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    P = solve.block_jacobi(S, p.mesh.block_of_node)
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "defect")
    y, info = solve.fgmres(S, t * b, lambda r: solve.block_jacobi_apply(P, r), tol=1e-11, restart=300,
                           selective=True)
    assert info["relres"] <= 1e-11


def test_one_pass_gram_schmidt():
    """One classical pass: h = V^H w exactly, w_new = w - V h, and the loss of orthogonality
    is bounded by the cancellation (visible for a vector nearly inside span(V), removed by a
    second pass); FGMRES with it still reaches the dense solution."""
    rng = np.random.default_rng(9)
    n, k = 300, 6
    V, _ = np.linalg.qr(rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k)))
    w = V @ (rng.normal(size=k) + 0j) + 1e-6 * (rng.normal(size=n) + 0j)
    h, w1, beta = solve.cgs2(V, w, one_pass=True)
    np.testing.assert_allclose(h, V.conj().T @ w, rtol=1e-13)
    np.testing.assert_allclose(w1, w - V @ h, rtol=0, atol=1e-15 * np.linalg.norm(w))
    assert beta == pytest.approx(np.linalg.norm(w1), rel=1e-14)
    _, w2, _ = solve.cgs2(V, w)                                  # two passes: orthogonal to eps
    assert np.abs(V.conj().T @ w2).max() <= np.abs(V.conj().T @ w1).max() + 1e-300
    A = np.eye(40) * 4 + rng.normal(size=(40, 40)) + 1j * rng.normal(size=(40, 40))
    b = rng.normal(size=40) + 1j * rng.normal(size=40)
    x, info = solve.fgmres(A, b, tol=1e-12, restart=40, one_pass=True)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    assert info["relres"] <= 1e-12


# ---------------------------------------------------------------- aggregation multigrid

def _amg_case(shape=(7, 7, 9), which="vacuum"):
    p = E.wall_loss_problem(shape, (20e-3, 20e-3, 30e-3), (2, 2, 2), 0.1, 6, z_pos=(0.0,))
    M = fem.system_matrix(p, which)
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, which)
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    d, v = fem.fixed_dofs(p.mesh.bc_mask, cond)
    w = solve.near_null_weights(t, np.concatenate([d, v]))
    G = solve.node_graph_from_tets(p.mesh.n_nodes, p.mesh.tets)
    return p, M, t, S, w, G, cond


def test_greedy_aggregates_rule():
    # path graph 0-1-2-3-4-5-6: seeds 0 (takes 1), 2 (takes 3), 4 (takes 5), 6
    n = 7
    r = np.r_[np.arange(n), np.arange(n - 1), np.arange(1, n)]
    c = np.r_[np.arange(n), np.arange(1, n), np.arange(n - 1)]
    G = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    np.testing.assert_array_equal(solve.greedy_aggregates(G, 8), [0, 0, 1, 1, 2, 2, 3])
    np.testing.assert_array_equal(solve.greedy_aggregates(G, 1), np.arange(n))


def test_amg_coarse_operator_is_galerkin_and_preserves_constants():
    p, M, t, S, w, G, cond = _amg_case()
    lv = solve.amg_setup(S, w, p.mesh.block_of_node, G, max_coarse_dofs=64, agg_size=4)
    assert len(lv) >= 3
    L0 = lv[0]
    # level-1 operator = P^T S P (+ identity on empty coarse dofs)
    A1 = lv[1]["A"]
    E1 = (L0["P"].T @ S @ L0["P"]).toarray()
    empty = np.asarray(abs(L0["P"]).sum(axis=0)).ravel() == 0
    np.testing.assert_allclose(A1.toarray(), E1 + np.diag(empty.astype(float)), atol=1e-12 * abs(E1).max())
    # the unscaled constant A_x field is in the range of P0 (near-null preservation)
    x = np.zeros(S.shape[0])
    x[0::4] = 1.0
    x[np.asarray(w) == 0] = 0.0
    y = x / t
    c = np.zeros(L0["P"].shape[1])
    nz = ~empty
    c[nz] = 0.0
    c[np.arange(0, c.size, 4)[nz[0::4]]] = 1.0
    np.testing.assert_allclose(L0["P"] @ c, y * (np.asarray(w) != 0), rtol=1e-13)


def test_amg_w_cycle_converges_fast():
    p, M, t, S, w, G, cond = _amg_case((11, 11, 15))
    lv = solve.amg_setup(S, w, p.mesh.block_of_node, G, max_coarse_dofs=256, agg_size=8)
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "vacuum")
    P = solve.block_jacobi(S, p.mesh.block_of_node)
    _, i1 = solve.fgmres(S, t * b, lambda r: solve.block_jacobi_apply(P, r), tol=1e-10, restart=30, maxiter=600)
    _, i2 = solve.fgmres(S, t * b, lambda r: solve.amg_apply(lv, r), tol=1e-10, restart=30, maxiter=600)
    assert i2["relres"] <= 1e-10
    assert i2["iters"] < 0.5 * i1["iters"]
