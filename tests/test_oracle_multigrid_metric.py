"""The metric of the multigrid-cycle parity test, pinned on the CPU.

The W-cycle's output z = C r is dominated by the coarse correction of the
near-null (gauge) modes, so its plain 2-norm hides errors elsewhere: a
swapped pair of aggregates on a coarse level moves z by ~1e-6 relative,
below the rounding noise of an FP32 cycle.  The parity test therefore
measures e_S = ||S (z - z_ref)|| / ||S z_ref|| (S the scaled finest matrix):
S damps the near-null modes by their small eigenvalues and leaves the rest.

Pins, on the oracle's own hierarchy (three levels):
  * an FP32 (complex64) execution of the oracle's cycle stays below a tenth
    of the FP32 bound of the GPU test (rounding alone: <= 8.4e-4 here; the
    GPU's FP32 cycle measured <= 3.9e-3 on the parity meshes, its kernels sum
    in other orders, so the bound is 1e-2);
  * indexing errors planted in the hierarchy (two aggregates exchanged in a
    prolongator, all aggregates shifted by one, a smoothing block dropped, a
    block inverse with its rows reversed) exceed the bound for every right-
    hand side, and the smallest of them stays below the old 2-norm bound,
    i.e. the new metric sees what the old one could not.
"""
import numpy as np
import pytest

import ect_inputs as E
from oracle import fem, solve

E_S_F32 = 1e-2     # FP32 bound of the GPU cycle parity test (e_S per right-hand side)
E_2_OLD = 3e-2     # the former 2-norm bound


def _levels(shape):
    p = E.wall_loss_problem(shape, (20e-3, 20e-3, 30e-3), (2, 2, 2), 0.15, 4, z_pos=(0.0,))
    M = fem.system_matrix(p, "defect")
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "defect")
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    d, v = fem.fixed_dofs(p.mesh.bc_mask, cond)
    w = solve.near_null_weights(t, np.concatenate([d, v]))
    G = solve.node_graph_from_tets(p.mesh.n_nodes, p.mesh.tets)
    return S, solve.amg_setup(S, w, p.mesh.block_of_node, G)


def _complex64(levels):
    out = []
    for L in levels:
        if "inv" in L:
            out.append(dict(A=L["A"].astype(np.complex64), inv=L["inv"].astype(np.complex64)))
        else:
            st, sp_, inv = L["BJ"]
            out.append(dict(A=L["A"].astype(np.complex64), P=L["P"].astype(np.float32),
                            BJ=(st, sp_, [B.astype(np.complex64) for B in inv])))
    return out


def _swap_aggregates(levels, l, a, b):
    """Copy of the hierarchy whose level-l prolongator has the columns of
    aggregates a and b exchanged (a coarse-level indexing error)."""
    out = [dict(L) for L in levels]
    P = out[l]["P"].tocsc()
    cols = np.arange(P.shape[1])
    ia, ib = 4 * a + np.arange(4), 4 * b + np.arange(4)
    cols[ia], cols[ib] = cols[ib].copy(), cols[ia].copy()
    out[l]["P"] = P[:, cols].tocsr()
    return out


def e_s(S, z, ref):
    return np.linalg.norm(S @ (z - ref)) / np.linalg.norm(S @ ref)


@pytest.fixture(scope="module")
def three_level():
    S, lv = _levels((17, 16, 21))
    assert len(lv) == 3
    return S, lv


def test_fp32_cycle_within_bound(three_level):
    S, lv = three_level
    lv32 = _complex64(lv)
    rng = np.random.default_rng(11)
    for _ in range(4):
        r = rng.normal(size=S.shape[0]) + 1j * rng.normal(size=S.shape[0])
        z = solve.amg_apply(lv, r)
        z32 = solve.amg_apply(lv32, r.astype(np.complex64)).astype(np.complex128)
        assert e_s(S, z32, z) <= E_S_F32 / 10


def _shift_aggregates(levels, l):
    out = [dict(L) for L in levels]
    P = out[l]["P"].tocsc()
    out[l]["P"] = P[:, np.roll(np.arange(P.shape[1]), 4)].tocsr()
    return out


def _edit_block(levels, l, b, fn):
    out = [dict(L) for L in levels]
    st, sp_, inv = out[l]["BJ"]
    inv = list(inv)
    inv[b] = fn(inv[b])
    out[l]["BJ"] = (st, sp_, inv)
    return out


PLANTED = {
    "swap L0 aggregates 2,3": lambda lv: _swap_aggregates(lv, 0, 2, 3),
    "swap L1 aggregates 5,9": lambda lv: _swap_aggregates(lv, 1, 5, 9),
    "shift L1 aggregates": lambda lv: _shift_aggregates(lv, 1),
    "drop L0 block 7": lambda lv: _edit_block(lv, 0, 7, lambda B: 0.0 * B),
    "drop L1 block 3": lambda lv: _edit_block(lv, 1, 3, lambda B: 0.0 * B),
    "reverse rows of L1 block 3": lambda lv: _edit_block(lv, 1, 3, lambda B: B[::-1].copy()),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_coarse_indexing_error_is_caught(three_level, name):
    S, lv = three_level
    bad = PLANTED[name](lv)
    rng = np.random.default_rng(12)
    for _ in range(3):
        r = rng.normal(size=S.shape[0]) + 1j * rng.normal(size=S.shape[0])
        z = solve.amg_apply(lv, r)
        zb = solve.amg_apply(bad, r)
        assert e_s(S, zb, z) > E_S_F32, name                        # the S-weighted metric fails it


def test_old_two_norm_metric_missed_a_planted_error(three_level):
    S, lv = three_level
    bad = PLANTED["drop L1 block 3"](lv)
    rng = np.random.default_rng(13)
    r = rng.normal(size=S.shape[0]) + 1j * rng.normal(size=S.shape[0])
    z = solve.amg_apply(lv, r)
    zb = solve.amg_apply(bad, r)
    assert np.linalg.norm(zb - z) / np.linalg.norm(z) < E_2_OLD      # 2-norm: within the old bound
    assert e_s(S, zb, z) > E_S_F32                                  # S-weighted: caught
