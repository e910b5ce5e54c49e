"""GPU path on an unstructured mesh (Sec. 3, Steps 1-2 with a body of
tetrahedra that is not a structured grid): grid nodes and cell centres,
cells cut along randomly chosen face diagonals, all nodes jittered
(ect_inputs.unstructured_box_mesh), partitioned by the library's own
recursive coordinate bisection (ect_partition) and renumbered; then
assembly, mixed and FP64 solves and Delta Z against the CPU oracle.

The oracle works on the mesh in its original numbering (it never sees the
library's partition); GPU results are mapped back through the permutation
before they are compared.  Tolerances as in test_gpu_parity: assembly
1e-12 sqrt(|M_ii||M_jj|), true residual <= tol with the oracle's matrix,
Delta Z <= 1e-6 relative to the oracle's SuperLU value."""
import numpy as np
import pytest
import scipy.sparse as sp

import ect_inputs as E
from oracle import fem, impedance, rhs, solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOX = (20e-3, 20e-3, 40e-3)


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect
    build.build()
    ect.load_library()
    m0 = E.unstructured_box_mesh((12, 12, 18), BOX, seed=4)
    p0 = E.wall_loss_problem(None, BOX, z_pos=(0.5e-3,), mesh=m0)
    new_id, blk = ect.partition(m0.xyz, 16)
    p1 = E.wall_loss_problem(None, BOX, z_pos=(0.5e-3,), mesh=E.permute_mesh(m0, new_id, blk))
    ctx = ect.Context()
    ctx.load_problem(p1)
    mask = ect.ECT_F64 | ect.ECT_F32
    for w in (ect.ECT_VACUUM, ect.ECT_DEFECT):
        ctx.assemble(w, mask)
        ctx.precond_setup(w, mask, -1)
    dof = (4 * np.asarray(new_id, dtype=np.int64)[:, None] + np.arange(4)[None]).ravel()  # old dof -> new dof
    M = {w: fem.system_matrix(p0, w) for w in ("vacuum", "defect")}
    return ect, ctx, p0, p1, dof, M


def test_partition_sizes(case):
    ect, ctx, p0, p1, dof, M = case
    sizes = np.bincount(p1.mesh.block_of_node)
    assert sizes.max() <= 16 and sizes.size <= 2 * (-(-p0.mesh.n_nodes // 16))


def test_unstructured_assembly_matches_oracle(case):
    ect, ctx, p0, p1, dof, M = case
    from tests.test_gpu_parity import bsr_to_csr
    for w, wi in (("vacuum", 0), ("defect", 1)):
        rp, col, val = ctx.matrix_copy(wi)
        G = bsr_to_csr(rp, col, val)[dof][:, dof]              # back to the original numbering
        O = M[w]
        d = np.sqrt(np.abs(O.diagonal()))
        D = (G - O).tocoo()
        assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300), w


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_unstructured_solve_and_delta_z(case, mode):
    ect, ctx, p0, p1, dof, M = case
    z = p0.z_pos[0]
    B0 = [fem.constrain_rhs(rhs.coil_rhs(p0.mesh.xyz, p0.mesh.tets, c.as_tuple(), z), p0, "vacuum") for c in p0.coils]
    opts = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED,
                               restart=30 if mode == "f64" else 16, inner_iters=16)
    n = 4 * p1.mesh.n_nodes
    b = torch.empty(2, n, dtype=torch.complex128, device="cuda")
    for c in range(2):
        ctx.coil_rhs(p1.coils[c], np.array([z]), b[c:c + 1])
    Bg = b.cpu().numpy()
    for c in range(2):                                           # same source in both numberings
        assert np.abs(Bg[c][dof] - B0[c]).max() <= 1e-13 * np.abs(B0[c]).max()
    sol = {}
    for w, wi in (("vacuum", 0), ("defect", 1)):
        x = torch.empty_like(b)
        try:
            st = ctx.solve(wi, b, x, 2, opts)
        except ect.EctError as e:
            raise AssertionError((w, mode, str(e), e.stats))
        X = x.cpu().numpy()[:, dof]
        t = fem.scaling(M[w])
        for c in range(2):
            res = np.linalg.norm(t * (B0[c] - M[w] @ X[c])) / np.linalg.norm(t * B0[c])
            assert res <= 1e-10 * 1.0001, (w, c, res, st)
        sol[w] = X
    cur = [c.current for c in p0.coils]
    back = np.argsort(dof)                                       # original numbering -> renumbered
    u0g = torch.from_numpy(np.ascontiguousarray(sol["vacuum"][:, back])).cuda()
    udg = torch.from_numpy(np.ascontiguousarray(sol["defect"][:, back])).cuda()
    dz_gpu, _ = ctx.delta_z(u0g, udg, None, cur)
    _, lu0 = solve.superlu_solve(M["vacuum"], B0[0])
    _, lud = solve.superlu_solve(M["defect"], B0[0])
    u0 = [lu0.solve(bk) for bk in B0]
    ud = [lud.solve(bk) for bk in B0]
    ref = impedance.delta_z_matrix(M["vacuum"], M["defect"], u0, ud, cur, p0.omega)
    assert np.abs(ref).max() > 0
    assert np.abs(dz_gpu - ref).max() <= 1e-6 * np.abs(ref).max()
    # the public scan call on the renumbered mesh gives the same Delta Z
    dz_scan, _ = ctx.impedance(p1.coils, np.array([z]), opts)
    assert np.abs(dz_scan[0] - ref).max() <= 1e-6 * np.abs(ref).max()
