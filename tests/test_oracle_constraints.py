"""Pins of the oracle's coefficient selection and constraint handling by brute force.

Each check restates what the function must do element by element (loops over tets, nodes and
dofs) on a tiny mesh and compares; a dropped condition, a swapped component bit or a constraint
applied to the wrong dof fails one of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import ect_inputs as E
from oracle import fem, solve


@pytest.fixture(scope="module")
def tiny():
    return E.wall_loss_problem((5, 5, 7), (20e-3, 20e-3, 30e-3), (2, 2, 2), 0.1, 3, z_pos=(0.0,))


def test_effective_coefficients_select_background_or_defect(tiny):
    p = tiny
    s0, n0 = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "vacuum")
    assert np.array_equal(s0, p.sigma) and np.array_equal(n0, p.nu)
    s1, n1 = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "defect")
    for t in range(p.mesh.n_tets):
        want_s = p.sigma[t] if np.isnan(p.sigma_d[t]) else p.sigma_d[t]
        want_n = p.nu[t] if np.isnan(p.nu_d[t]) else p.nu_d[t]
        assert s1[t] == want_s and n1[t] == want_n
    assert np.any(~np.isnan(p.sigma_d))                  # the case has a defect region at all
    with pytest.raises(ValueError):
        fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "other")


def test_conducting_nodes_by_brute_force(tiny):
    p = tiny
    m = p.mesh
    got = fem.conducting_nodes(m.n_nodes, m.tets, p.sigma)
    want = np.zeros(m.n_nodes, dtype=bool)
    for t in range(m.n_tets):
        if p.sigma[t] > 0.0:
            for a in range(4):
                want[m.tets[t, a]] = True
    assert np.array_equal(got, want)
    assert 0 < want.sum() < m.n_nodes


def test_fixed_dofs_by_brute_force(tiny):
    p = tiny
    m = p.mesh
    cond = fem.conducting_nodes(m.n_nodes, m.tets, p.sigma)
    d, v = fem.fixed_dofs(m.bc_mask, cond)
    want_d, want_v = [], []
    for i in range(m.n_nodes):
        for c in range(3):
            if (int(m.bc_mask[i]) >> c) & 1:
                want_d.append(4 * i + c)
        if not cond[i]:
            want_v.append(4 * i + 3)
    assert sorted(d.tolist()) == sorted(want_d)
    assert sorted(v.tolist()) == sorted(want_v)
    assert len(want_d) > 0


def test_apply_constraints_rows_columns_and_free_block(tiny):
    p = tiny
    m = p.mesh
    s, nu = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "vacuum")
    raw = fem.assemble_raw(m.xyz, m.tets, s, nu, p.nu_tilde, p.omega, p.delta).tocsr()
    cond = fem.conducting_nodes(m.n_nodes, m.tets, s)
    d, v = fem.fixed_dofs(m.bc_mask, cond)
    M = fem.apply_constraints(raw, d, v).toarray()
    R = raw.toarray()
    fixed = np.zeros(R.shape[0], dtype=bool)
    fixed[d] = True
    fixed[v] = True
    for i in np.nonzero(fixed)[0]:
        e = np.zeros(R.shape[0])
        e[i] = 1.0
        assert np.array_equal(M[i], e) and np.array_equal(M[:, i], e)
    free = ~fixed
    assert np.array_equal(M[np.ix_(free, free)], R[np.ix_(free, free)])
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()  # complex symmetric (not Hermitian)


def test_near_null_weights_and_scaling(tiny):
    p = tiny
    M = fem.system_matrix(p, "vacuum")
    t = fem.scaling(M)
    dg = np.abs(M.diagonal())
    assert np.allclose(t, 1.0 / np.sqrt(dg), rtol=1e-15, atol=0.0)
    S = fem.scaled(M, t)
    assert np.allclose(np.abs(S.diagonal()), 1.0, rtol=1e-14)   # unit-modulus diagonal
    D = sp.diags(t)
    assert abs(S - D @ M @ D).max() <= 1e-15 * abs(S).max()
    fixed = np.array([0, 5, 9])
    w = solve.near_null_weights(t, fixed)
    for i in range(t.size):
        assert w[i] == (0.0 if i in fixed else 1.0 / t[i])
