"""Parity at the other full-size configurations, checked through sampled rows and invariants.

* 500,094 nodes (2,000,376 complex unknowns), wall-loss patch, 64 probe positions: one batched
  solve of 64 right-hand sides per matrix (mixed precision, multigrid, graphs) with the Krylov
  lengths and tile the autotuner picks on one tile of the batch, tolerance 1e-10.
* 4,000,752 nodes (16,003,008 complex unknowns), TSP support plate, one position and two coils:
  mixed precision to 1e-8.

At these sizes the oracle cannot solve the system, so each case checks what it can compute one
row at a time and what holds at any size:
  * the residual of the GPU solution on sampled block rows recomputed by the oracle from the tets
    around each node (|t_i (b - M x)_i| <= tol ||T b|| for every row when the global scaled
    residual is <= tol);
  * Delta Z by reciprocity against the independent coil-EMF difference, per position.
"""
import gc

import numpy as np
import pytest

import ect_inputs as E
from test_gpu_fullsize import oracle_rows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _context(p):
    from paper_1602_03207_gb300 import build, ect
    build.build()
    gc.collect()
    torch.cuda.empty_cache()
    ctx = ect.Context()
    ctx.load_problem(p)
    for w in (0, 1):
        ctx.assemble(w, ect.ECT_F64 | ect.ECT_F32)
        ctx.precond_setup(w, ect.ECT_F64 | ect.ECT_F32, -1)
    return ect, ctx


def _sample_nodes(p, rng, n_random=120):
    N = p.mesh.n_nodes
    cond = np.nonzero(np.isfinite(p.sigma_d))[0]
    picked = p.mesh.tets[rng.choice(cond, 12, replace=False)].ravel()
    return np.unique(np.concatenate([rng.choice(N, n_random, replace=False), picked]))


def _check_rows(ctx, p, name, w, nodes, B, X, tol):
    N = p.mesh.n_nodes
    rows, _ = oracle_rows(p, name, nodes, N)
    tvec = ctx.scaling_copy(w)
    for q in range(B.shape[0]):
        b = B[q].cpu().numpy()
        x = X[q].cpu().numpy().reshape(N, 4)
        bnorm = np.linalg.norm(tvec * b)
        for node, row in rows.items():
            r = b[4 * node:4 * node + 4].copy()
            for j, blk in row.items():
                r -= blk @ x[j]
            assert np.abs(tvec[4 * node:4 * node + 4] * r).max() <= tol * bnorm * 1.0001, (name, q, node)


def test_c3_batched_64_positions_autotuned():
    p = E.make_config("c3")
    ect, ctx = _context(p)
    try:
        N = p.mesh.n_nodes
        n = 4 * N
        k = len(p.z_pos)
        assert k == 64
        B = torch.empty(k, n, dtype=torch.complex128, device="cuda")
        ctx.coil_rhs(p.coils[0], p.z_pos, B)
        # tune on one tile of the batch at a looser tolerance (each candidate is a full solve),
        # then solve all 64 right-hand sides to 1e-10 with the winner
        work = torch.empty_like(B[:8])
        base = ect.default_options(tol=1e-8, mode=ect.ECT_MODE_MIXED, max_iters=600)
        best, _ = ctx.autotune(1, B[:8].contiguous(), work, 8, base)
        del work
        assert best.mode == ect.ECT_MODE_MIXED
        best.tol = 1e-10
        best.max_iters = 3000
        rng = np.random.default_rng(3)
        nodes = _sample_nodes(p, rng)
        U = {}
        for w, name in ((0, "vacuum"), (1, "defect")):
            X = torch.empty_like(B)
            st = ctx.solve(w, B, X, k, best)
            print(name, "rhs_tile", best.rhs_tile, "restart", best.restart, "inner", best.inner_iters, st)
            assert st["converged"] == k and st["relres_max"] <= 1e-10, st
            assert st["launches"] > 0
            _check_rows(ctx, p, name, w, nodes, B[::9], X[::9], 1e-10)
            U[w] = X
        cur = [p.coils[0].current] * 2
        worst = 0.0
        for q in range(0, k, 7):
            u0 = U[0][q].unsqueeze(0).expand(2, -1).contiguous()
            ud = U[1][q].unsqueeze(0).expand(2, -1).contiguous()
            b = B[q].unsqueeze(0).expand(2, -1).contiguous()
            dz, dze = ctx.delta_z(u0, ud, b, cur)
            assert abs(dz[0, 0]) > 0
            worst = max(worst, abs(dz[0, 0] - dze[0, 0]) / abs(dz[0, 0]))
        # the EMF form is a difference of two whole impedances, |Z| >> |dZ| for a small wall loss:
        # its error is the solve tolerance amplified by |Z| / |dZ|
        assert worst <= 1e-4, worst
    finally:
        ctx.close()


def test_c4_mixed_16m_unknowns():
    p = E.make_config("c4")
    ect, ctx = _context(p)
    try:
        N = p.mesh.n_nodes
        n = 4 * N
        assert n == 16003008
        B = torch.empty(2, n, dtype=torch.complex128, device="cuda")
        for ci in range(2):
            t = torch.empty(1, n, dtype=torch.complex128, device="cuda")
            ctx.coil_rhs(p.coils[ci], p.z_pos[:1], t)
            B[ci] = t[0]
        opts = ect.default_options(tol=1e-8, mode=ect.ECT_MODE_MIXED, restart=16, inner_iters=12, max_iters=400)
        rng = np.random.default_rng(4)
        nodes = _sample_nodes(p, rng, n_random=80)
        U = {}
        for w, name in ((0, "vacuum"), (1, "defect")):
            X = torch.empty_like(B)
            st = ctx.solve(w, B, X, 2, opts)
            print(name, st)
            assert st["converged"] == 2 and st["relres_max"] <= 1e-8, st
            _check_rows(ctx, p, name, w, nodes, B, X, 1e-8)
            U[w] = X
        dz, dze = ctx.delta_z(U[0], U[1], B, [c.current for c in p.coils])
        scale = np.abs(dz).max()
        assert scale > 0
        # reciprocity and EMF forms agree to the solve tolerance amplified by |Z| / |dZ|
        assert np.abs(dz - dze).max() <= 1e-4 * scale
        assert abs(dz[0, 1] - dz[1, 0]) <= 1e-4 * scale
    finally:
        ctx.close()
