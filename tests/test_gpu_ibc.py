"""GPU path with the impedance boundary condition on the support plate (Sec. 2,
Eq. IBC / ibcROTA): the plate tets removed, the surface term on their
boundary, against the oracle (oracle/ibc.py).  Assembly entrywise, solves by
the true residual with the oracle's matrix, Delta Z (coil-EMF form, the
IBC computes no plate volume fields) against SuperLU: 1e-6 relative."""
import numpy as np
import pytest

import ect_inputs as E
from oracle import fem, ibc, impedance, rhs, solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect
    build.build()
    ect.load_library()
    p = E.tsp_problem((12, 12, 30), (30e-3, 30e-3, 60e-3), (2, 2, 4), 0.15, 2, z_pos=(10e-3,))
    plate = np.isfinite(p.sigma_d)
    ctx = ect.Context()
    ctx.load_problem(p)
    ctx.set_ibc(ect.ECT_DEFECT, plate, E.SIGMA_TSP, E.NU0)
    mask = ect.ECT_F64 | ect.ECT_F32
    for w in (ect.ECT_VACUUM, ect.ECT_DEFECT):
        ctx.assemble(w, mask)
        ctx.precond_setup(w, mask, -1)
    M0 = fem.system_matrix(p, "vacuum")
    Mi, fixed = ibc.system_matrix_ibc(p, plate, E.SIGMA_TSP, E.MU0, which="defect")
    return ect, ctx, p, plate, M0, Mi, fixed


def test_ibc_assembly_matches_oracle(case):
    ect, ctx, p, plate, M0, Mi, fixed = case
    from tests.test_gpu_parity import bsr_to_csr
    rp, col, val = ctx.matrix_copy(ect.ECT_DEFECT)
    G = bsr_to_csr(rp, col, val)
    d = np.sqrt(np.abs(Mi.diagonal()))
    D = (G - Mi).tocoo()
    assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300)
    assert abs(G - G.T).max() <= 1e-13 * abs(G).max()
    # the background matrix is untouched by the condition on the defect configuration
    rp, col, val = ctx.matrix_copy(ect.ECT_VACUUM)
    G0 = bsr_to_csr(rp, col, val)
    d0 = np.sqrt(np.abs(M0.diagonal()))
    D0 = (G0 - M0).tocoo()
    assert np.all(np.abs(D0.data) <= 1e-12 * d0[D0.row] * d0[D0.col] + 1e-300)


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_ibc_solve_and_delta_z(case, mode):
    ect, ctx, p, plate, M0, Mi, fixed = case
    z = p.z_pos[0]
    B = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), z), p, "vacuum") for c in p.coils]
    assert all(np.abs(ibc.constrain_rhs_ibc(b, fixed) - b).max() == 0.0 for b in B)
    opts = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED,
                               restart=30 if mode == "f64" else 16, inner_iters=16)
    b = torch.from_numpy(np.stack(B)).cuda()
    x = torch.empty_like(b)
    ctx.solve(ect.ECT_DEFECT, b, x, 2, opts)
    X = x.cpu().numpy()
    t = fem.scaling(Mi)
    for c in range(2):
        res = np.linalg.norm(t * (B[c] - Mi @ X[c])) / np.linalg.norm(t * B[c])
        assert res <= 1e-10 * 1.0001, (c, res)
    I = [c.current for c in p.coils]
    _, lu0 = solve.superlu_solve(M0, B[0])
    _, lui = solve.superlu_solve(Mi, B[0])
    u0 = [lu0.solve(bk) for bk in B]
    ui = [lui.solve(bk) for bk in B]
    ref = impedance.delta_z_emf_matrix(B, u0, ui, I, p.omega)
    dz, _ = ctx.impedance(p.coils, np.array([z]), opts)
    assert np.abs(dz[0] - ref).max() <= 1e-6 * np.abs(ref).max()
    # the kernel-level call needs the sources with the condition set
    with pytest.raises(ect.EctError):
        ctx.delta_z(x, x, None, I)
    with pytest.raises(ect.EctError):
        ctx.delta_z_static(x.unsqueeze(0), x.unsqueeze(0), None, I, 1)


def test_ibc_cleared_restores_the_volume_model(case):
    ect, ctx, p, plate, M0, Mi, fixed = case
    from tests.test_gpu_parity import bsr_to_csr
    ctx.set_ibc(ect.ECT_DEFECT, None, 0.0, 0.0)
    ctx.assemble(ect.ECT_DEFECT, ect.ECT_F64)
    rp, col, val = ctx.matrix_copy(ect.ECT_DEFECT)
    G = bsr_to_csr(rp, col, val)
    Md = fem.system_matrix(p, "defect")
    d = np.sqrt(np.abs(Md.diagonal()))
    D = (G - Md).tocoo()
    assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300)
