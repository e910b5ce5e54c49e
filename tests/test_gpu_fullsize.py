"""Full-size parity (config 2: 1,000,004 nodes, 4,000,016 complex unknowns).

At this size the oracle cannot assemble or solve the whole system in test
time, so it checks sampled outputs it can compute one by one, in the launch
configuration the benchmark times (mixed precision, batched coil sources,
multigrid preconditioner):
  * 256 sampled block rows of both assembled matrices, recomputed by the
    oracle from the tets around each sampled node (same tolerance as the small
    parity test);
  * the residual of the GPU solution on those rows, computed on the CPU with
    the oracle's rows: |t_i (b - M x)_i| <= tol ||T b|| must hold for every row
    when the global scaled residual is <= tol;
  * Delta Z: the reciprocity reduction against the independent coil-EMF
    difference (agreement to the solve tolerance) and the symmetry dZ_12 = dZ_21.
"""
import numpy as np
import pytest

import ect_inputs as E
from oracle import fem, rhs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def oracle_rows(p, which, nodes, n_nodes):
    """Constrained rows 4*node + c of the system matrix, from the tets around each node."""
    m = p.mesh
    s, nu = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, which)
    cond = fem.conducting_nodes(n_nodes, m.tets, s)
    d, v = fem.fixed_dofs(m.bc_mask, cond)
    fixed = np.zeros(4 * n_nodes, dtype=bool)
    fixed[d] = True
    fixed[v] = True
    out = {}
    mask = np.isin(m.tets, nodes).any(axis=1)
    sel = np.nonzero(mask)[0]
    vol, g = fem.tet_geometry(m.xyz, m.tets[sel])
    Em = fem.element_matrices(vol, g, s[sel], nu[sel], p.nu_tilde, p.omega, p.delta)
    for node in nodes:
        row = {}
        for q, t in enumerate(sel):
            tet = m.tets[t]
            hit = np.nonzero(tet == node)[0]
            if hit.size == 0:
                continue
            a = hit[0]
            for bb in range(4):
                j = int(tet[bb])
                blk = row.setdefault(j, np.zeros((4, 4), dtype=np.complex128))
                blk += Em[q, a, bb]
        for j, blk in row.items():
            for r in range(4):
                for c in range(4):
                    if fixed[4 * node + r] or fixed[4 * j + c]:
                        blk[r, c] = 1.0 if (j == node and r == c and fixed[4 * node + r]) else 0.0
        out[int(node)] = row
    return out, fixed


@pytest.fixture(scope="module")
def c2():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect
    build.build()
    p = E.make_config("c2")
    ctx = ect.Context()
    ctx.load_problem(p)
    for w in (0, 1):
        ctx.assemble(w, ect.ECT_F64 | ect.ECT_F32)
        ctx.precond_setup(w, ect.ECT_F64 | ect.ECT_F32, -1)
    rng = np.random.default_rng(2)
    N = p.mesh.n_nodes
    # sample nodes: random ones plus nodes inside the conductor and the plate
    c = E.centroids(p.mesh)
    sig_t = np.nonzero(np.isfinite(p.sigma_d))[0][:2000]
    nodes = np.unique(np.concatenate([rng.choice(N, 200, replace=False),
                                      p.mesh.tets[rng.choice(sig_t, 28, replace=False)].ravel()[:56]]))
    return ect, ctx, p, nodes


def test_fullsize_assembly_sampled_rows(c2):
    ect, ctx, p, nodes = c2
    N = p.mesh.n_nodes
    for w, name in ((0, "vacuum"), (1, "defect")):
        rp, col, val = ctx.matrix_copy(w)
        rows, _ = oracle_rows(p, name, nodes, N)
        for node, row in rows.items():
            s0, s1 = rp[node], rp[node + 1]
            gcols = col[s0:s1]
            assert sorted(row) == sorted(gcols.tolist()), node
            for q, j in enumerate(gcols):
                ref = row[int(j)]
                got = val[s0 + q]
                scale = np.abs(ref).max() + np.abs(np.diag(row[node])).max()
                assert np.abs(got - ref).max() <= 1e-12 * scale, (name, node, j)


def test_fullsize_mixed_solve_residual_and_delta_z(c2):
    ect, ctx, p, nodes = c2
    N = p.mesh.n_nodes
    n = 4 * N
    B = torch.empty(1, 2, n, dtype=torch.complex128, device="cuda")
    for ci in range(2):
        t = torch.empty(1, n, dtype=torch.complex128, device="cuda")
        ctx.coil_rhs(p.coils[ci], p.z_pos[:1], t)
        B[:, ci] = t
    opts = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_MIXED, restart=16, inner_iters=12, max_iters=300)
    U = {}
    for w, name in ((0, "vacuum"), (1, "defect")):
        X = torch.empty_like(B)
        st = ctx.solve(w, B, X, 2, opts)
        assert st["converged"] == 2 and st["relres_max"] <= 1e-10
        U[w] = X
        # sampled residual rows with the oracle's rows and scaling
        rows, _ = oracle_rows(p, name, nodes, N)
        tvec = ctx.scaling_copy(w)
        x = X[0].cpu().numpy()
        b = B[0].cpu().numpy()
        for ci in range(2):
            bnorm = np.linalg.norm(tvec * b[ci])
            xr = x[ci].reshape(N, 4)
            for node, row in rows.items():
                r = b[ci][4 * node:4 * node + 4].copy()
                for j, blk in row.items():
                    r -= blk @ xr[j]
                assert np.abs(tvec[4 * node:4 * node + 4] * r).max() <= 1e-10 * bnorm * 1.0001, (name, node)
    cur = [c.current for c in p.coils]
    dz, dze = ctx.delta_z(U[0][0], U[1][0], B[0], cur)
    scale = np.abs(dz).max()
    assert scale > 0
    assert np.abs(dz - dze).max() <= 1e-6 * scale
    assert abs(dz[0, 1] - dz[1, 0]) <= 1e-6 * scale
