"""Frequency as a batch dimension (Eq. impedmod's signals over a sweep): one
assembly pass writes both configurations at several frequencies, one
lockstep solve covers every frequency, and Delta Z per frequency matches the
oracle assembled at that frequency.  Tolerances as in test_gpu_parity."""
import dataclasses

import numpy as np
import pytest

import ect_inputs as E
from oracle import fem, ibc, impedance, rhs, solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
FREQS = (3.0e4, 1.0e5, 2.5e5)


@pytest.fixture(scope="module")
def ect():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect as ect_mod
    build.build()
    ect_mod.load_library()
    return ect_mod


@pytest.fixture(scope="module")
def case(ect):
    p = E.wall_loss_problem((10, 11, 13), (20e-3, 20e-3, 30e-3), (2, 3, 2), 0.15, 5, z_pos=(0.0, 1.5e-3))
    ctx = ect.Context()
    ctx.load_problem(p)
    mask = ect.ECT_F64 | ect.ECT_F32
    ctx.assemble_sweep(FREQS, mask)
    for f in range(len(FREQS)):
        for cfg in (0, 1):
            ctx.precond_setup(ect.sweep_matrix(f, cfg), mask, -1)
    return ctx, p


def _check_matrix(ctx, which, O):
    from tests.test_gpu_parity import bsr_to_csr
    rp, col, val = ctx.matrix_copy(which)
    G = bsr_to_csr(rp, col, val)
    d = np.sqrt(np.abs(O.diagonal()))
    D = (G - O).tocoo()
    assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300), which


def test_sweep_assembly_matches_oracle_at_each_frequency(ect, case):
    ctx, p = case
    for f, fr in enumerate(FREQS):
        pf = dataclasses.replace(p, freq=fr)
        for cfg, w in ((0, "vacuum"), (1, "defect")):
            _check_matrix(ctx, ect.sweep_matrix(f, cfg), fem.system_matrix(pf, w))


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_sweep_solve_residual_and_delta_z(ect, case, mode):
    ctx, p = case
    opts = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED,
                               restart=30 if mode == "f64" else 16, inner_iters=16)
    n = 4 * p.mesh.n_nodes
    F = len(FREQS)
    B = np.stack([fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), 0.0), p, "vacuum")
                  for c in p.coils])
    b = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(B, (F, 2, n)))).cuda()
    x = torch.empty_like(b)
    st = ctx.solve_sweep(ect.ECT_DEFECT, b, x, 2, opts)
    assert st["converged"] == 2 * F
    X = x.cpu().numpy()
    for f, fr in enumerate(FREQS):
        M = fem.system_matrix(dataclasses.replace(p, freq=fr), "defect")
        t = fem.scaling(M)
        for c in range(2):
            res = np.linalg.norm(t * (B[c] - M @ X[f, c])) / np.linalg.norm(t * B[c])
            assert res <= 1e-10 * 1.0001, (fr, c, res)
    dz, st = ctx.impedance_sweep(p.coils, p.z_pos, opts)
    assert dz.shape == (F, len(p.z_pos), 2, 2)
    I = [c.current for c in p.coils]
    for f, fr in enumerate(FREQS):
        pf = dataclasses.replace(p, freq=fr)
        M0, Md = fem.system_matrix(pf, "vacuum"), fem.system_matrix(pf, "defect")
        _, lu0 = solve.superlu_solve(M0, B[0])
        _, lud = solve.superlu_solve(Md, B[0])
        for q, z in enumerate(p.z_pos):
            bz = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), z), p, "vacuum")
                  for c in p.coils]
            ref = impedance.delta_z_matrix(M0, Md, [lu0.solve(bk) for bk in bz], [lud.solve(bk) for bk in bz],
                                           I, pf.omega)
            assert np.abs(dz[f, q] - ref).max() <= 1e-6 * np.abs(ref).max(), (fr, q)
    # the signal changes with frequency (the sweep is not one frequency repeated)
    assert np.abs(dz[0, 0] - dz[2, 0]).max() > 1e-2 * np.abs(dz[2, 0]).max()


def test_sweep_equals_single_frequency_solves(ect, case):
    ctx, p = case
    opts = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_MIXED, restart=16, inner_iters=16)
    dz_sweep, _ = ctx.impedance_sweep(p.coils, p.z_pos, opts)
    single = ect.Context()
    for f, fr in enumerate(FREQS):
        single.load_problem(dataclasses.replace(p, freq=fr))
        for w in (0, 1):
            single.assemble(w, ect.ECT_F64 | ect.ECT_F32)
            single.precond_setup(w, ect.ECT_F64 | ect.ECT_F32, -1)
        dz1, _ = single.impedance(p.coils, p.z_pos, opts)
        assert np.abs(dz1 - dz_sweep[f]).max() <= 1e-7 * np.abs(dz1).max(), fr
    single.close()


def test_sweep_with_impedance_boundary_condition(ect):
    p = E.tsp_problem((12, 12, 30), (30e-3, 30e-3, 60e-3), (2, 2, 4), 0.15, 2, z_pos=(10e-3,))
    plate = np.isfinite(p.sigma_d)
    ctx = ect.Context()
    ctx.load_problem(p)
    ctx.set_ibc(ect.ECT_DEFECT, plate, E.SIGMA_TSP, E.NU0)
    freqs = (5.0e4, 2.0e5)
    ctx.assemble_sweep(freqs, ect.ECT_F64)
    for f, fr in enumerate(freqs):
        pf = dataclasses.replace(p, freq=fr)
        _check_matrix(ctx, ect.sweep_matrix(f, 0), fem.system_matrix(pf, "vacuum"))
        Mi, _ = ibc.system_matrix_ibc(pf, plate, E.SIGMA_TSP, E.MU0, which="defect")
        _check_matrix(ctx, ect.sweep_matrix(f, 1), Mi)
    ctx.close()
