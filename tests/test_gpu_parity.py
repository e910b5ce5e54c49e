"""GPU parity: every step of the CUDA path against the FP64 CPU oracle.

All GPU work goes through the C ABI (libect.so via the ctypes binding).
Tolerances (derived from the arithmetic of each step):
  assembly / FP64 SpMV   |diff_ij| <= 1e-12 sqrt(|M_ii| |M_jj|)   (sum of ~24
                          tet terms, each ~10 roundings of 1.1e-16)
  FP32 scaled SpMV       <= 2e-6 relative (unit-scaled entries, 15 blocks/row)
  block inverse apply    <= 1e-9 (FP64) / 1e-3 (FP32) relative: kappa(S_ss) eps
  coil load              <= 1e-13 relative (point-in-coil decisions are exact)
  solve                  ||T(b - M_oracle x)|| <= tol ||T b|| with the oracle's matrix
  Delta Z                <= 1e-6 relative to the oracle (SuperLU) value
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ect_inputs as E
from oracle import fem, impedance, rhs, solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ect():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1602_03207_gb300 import build, ect as ect_mod
    build.build()
    ect_mod.load_library()
    return ect_mod


def small_problem(seed=1):
    # 10 x 11 x 13 nodes, ragged 2x3x2 subdomains, jittered: several SpMV tiles and a ragged tail
    return E.wall_loss_problem((10, 11, 13), (20e-3, 20e-3, 30e-3), (2, 3, 2), 0.15, seed, z_pos=(0.0,))


def make_ctx(ect, p, f32=True, group=1):
    ctx = ect.Context()
    ctx.load_problem(p)
    mask = ect.ECT_F64 | (ect.ECT_F32 if f32 else 0)
    for w in (ect.ECT_VACUUM, ect.ECT_DEFECT):
        ctx.assemble(w, mask)
        ctx.precond_setup(w, mask, group)
    return ctx


def bsr_to_csr(rp, col, val):
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    R = (4 * rows[:, None, None] + np.arange(4)[None, :, None]).repeat(4, axis=2)
    Cc = (4 * col[:, None, None] + np.arange(4)[None, None, :]).repeat(4, axis=1)
    return sp.csr_matrix((val.ravel(), (R.ravel(), Cc.ravel())), shape=(4 * n, 4 * n))


def crand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


WHICH = {"vacuum": 0, "defect": 1}


@pytest.fixture(scope="module")
def small(ect):
    p = small_problem()
    ctx = make_ctx(ect, p)
    M = {w: fem.system_matrix(p, w) for w in WHICH}
    return p, ctx, M


def test_assembly_matches_oracle(ect, small):
    p, ctx, M = small
    for w, wi in WHICH.items():
        rp, col, val = ctx.matrix_copy(wi)
        G = bsr_to_csr(rp, col, val)
        O = M[w]
        d = np.sqrt(np.abs(O.diagonal()))
        D = (G - O).tocoo()
        bound = 1e-12 * d[D.row] * d[D.col]
        assert np.all(np.abs(D.data) <= bound + 1e-300), w
        # every oracle entry is inside the BSR pattern, and the GPU matrix is symmetric
        assert abs(G - G.T).max() <= 1e-13 * abs(G).max()


def test_assembly_matches_oracle_large_gauge_penalty(ect):
    """The V-gauge penalty (Sec. 4) at delta = 10 m^-2 instead of 1: the V-V
    blocks of the conducting nodes change, the bound stays the same."""
    import dataclasses
    p = dataclasses.replace(small_problem(seed=2), delta=10.0)
    ctx = ect.Context()
    ctx.load_problem(p)
    for w, wi in WHICH.items():
        ctx.assemble(wi, ect.ECT_F64)
        rp, col, val = ctx.matrix_copy(wi)
        G = bsr_to_csr(rp, col, val)
        O = fem.system_matrix(p, w)
        d = np.sqrt(np.abs(O.diagonal()))
        D = (G - O).tocoo()
        assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300), w
    ctx.close()


def test_scaling_matches_oracle(ect, small):
    p, ctx, M = small
    for w, wi in WHICH.items():
        t = ctx.scaling_copy(wi)
        np.testing.assert_allclose(t, fem.scaling(M[w]), rtol=1e-13)


def test_spmv_f64_batch(ect, small):
    p, ctx, M = small
    rng = np.random.default_rng(0)
    n = 4 * p.mesh.n_nodes
    for k in (1, 3, 9, 19):                      # 19 = two full tiles of 8, then 2 and 1
        X = crand(rng, k, n)
        x = dev(X)
        y = torch.empty_like(x)
        ctx.spmv(WHICH["defect"], x, y, k)
        Y = y.cpu().numpy()
        ref = (M["defect"] @ X.T).T
        scale = np.abs(M["defect"]).max() * np.abs(X).max()
        assert np.abs(Y - ref).max() <= 1e-13 * scale, k


@pytest.mark.parametrize("rows", [0, 8, 64, -1, -2])      # staged tilings (auto = 16), thread- and warp-per-row
def test_spmv_f32_scaled(ect, small, rows):
    p, ctx, M = small
    rng = np.random.default_rng(1)
    n = 4 * p.mesh.n_nodes
    t = fem.scaling(M["vacuum"])
    S = fem.scaled(M["vacuum"], t)
    ctx.set_spmm_rows(rows)
    for k in (1, 2, 8, 11, 19):                             # full and partial right-hand-side tiles
        X = crand(rng, k, n)
        x = dev(X, torch.complex64)
        y = torch.empty_like(x)
        ctx.spmv(WHICH["vacuum"], x, y, k, precision=ect.ECT_F32)
        ref = (S @ X.T).T
        err = np.linalg.norm(y.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 2e-6, (rows, k)
    ctx.set_spmm_rows(0)


def test_spmv_f32_staged_many_tiles(ect):
    """Staged SpMM on a mesh of ~1000 tiles of 16 rows (ragged last tile, 14-15
    blocks per row), elementwise against the oracle's scaled matrix."""
    p = E.wall_loss_problem((27, 25, 26), (20e-3, 20e-3, 30e-3), (2, 2, 4), 0.15, 3, z_pos=(0.0,))
    ctx = ect.Context()
    ctx.load_problem(p)
    ctx.assemble(ect.ECT_DEFECT, ect.ECT_F64 | ect.ECT_F32)
    S = fem.scaled(fem.system_matrix(p, "defect"), ctx.scaling_copy(ect.ECT_DEFECT))
    rng = np.random.default_rng(7)
    X = crand(rng, 9, S.shape[0]).astype(np.complex64)
    ref = (S @ X.T.astype(np.complex128)).T
    for rows in (16, 0, -2):
        ctx.set_spmm_rows(rows)
        x = dev(X, torch.complex64)
        y = torch.empty_like(x)
        ctx.spmv(ect.ECT_DEFECT, x, y, 9, precision=ect.ECT_F32)
        Y = y.cpu().numpy()
        scale = np.abs(S).max() * np.abs(X).max()
        assert np.abs(Y - ref).max() <= 1e-5 * scale, rows
        err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 2e-6, rows
    ctx.close()


def _oracle_amg(p, M, which, blocks=None):
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, which)
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    d, v = fem.fixed_dofs(p.mesh.bc_mask, cond)
    w = solve.near_null_weights(t, np.concatenate([d, v]))
    G = solve.node_graph_from_tets(p.mesh.n_nodes, p.mesh.tets)
    return solve.amg_setup(S, w, p.mesh.block_of_node if blocks is None else blocks, G)


def split_blocks(block_of_node, parts):
    """The smoothing blocks of ect_set_block_split(parts): each subdomain (a contiguous node range)
    cut into min(parts, n) contiguous pieces at n q / parts."""
    b = np.asarray(block_of_node)
    starts = np.flatnonzero(np.r_[True, b[1:] != b[:-1]])
    ends = np.r_[starts[1:], b.size]
    out = np.empty(b.size, dtype=np.int64)
    nb = 0
    for s0, e0 in zip(starts, ends):
        n = e0 - s0
        m = min(parts, n)
        for q in range(m):
            out[s0 + n * q // m:s0 + n * (q + 1) // m] = nb
            nb += 1
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("parts", [2, 4])
def test_precond_apply_split_blocks(ect, prec, parts):
    """Block-Jacobi over subdomains cut into 2 or 4 smoothing blocks (the FP32 apply then packs
    several blocks into each CTA) against the oracle's block-Jacobi over the same blocks, and one
    W-cycle whose first aggregates are those blocks against the oracle's."""
    p = E.wall_loss_problem((17, 16, 21), (20e-3, 20e-3, 30e-3), (2, 2, 4), 0.15, 4, z_pos=(0.0,))
    blocks = split_blocks(p.mesh.block_of_node, parts)
    M = fem.system_matrix(p, "defect")
    S = fem.scaled(M, fem.scaling(M))
    rng = np.random.default_rng(5)
    n = 4 * p.mesh.n_nodes
    k = 11                                       # one full tile of 8 and a partial one
    R = crand(rng, k, n)
    dt, pr = (torch.complex128, ect.ECT_F64) if prec == "f64" else (torch.complex64, ect.ECT_F32)
    r = dev(R, dt)
    mask = ect.ECT_F64 | ect.ECT_F32
    for group, tol in ((0, 1e-9 if prec == "f64" else 1e-3), (-1, 1e-7 if prec == "f64" else 1e-2)):
        ctx = ect.Context()
        ctx.load_problem(p)
        ctx.set_block_split(parts)
        ctx.assemble(ect.ECT_DEFECT, mask)
        ctx.precond_setup(ect.ECT_DEFECT, mask, group)
        z = torch.empty_like(r)
        ctx.precond_apply(ect.ECT_DEFECT, r, z, k, precision=pr)
        Z = z.cpu().numpy()
        if group == 0:
            P = solve.block_jacobi(S, blocks)
            for q in range(k):
                ref = solve.two_level_apply(P, None, R[q])
                assert np.linalg.norm(Z[q] - ref) <= tol * np.linalg.norm(ref), (group, q)
        else:
            lv = _oracle_amg(p, M, "defect", blocks)
            for q in range(k):
                ref = solve.amg_apply(lv, R[q])
                es = np.linalg.norm(S @ (Z[q] - ref)) / np.linalg.norm(S @ ref)
                assert es <= tol, (group, q, es)
        ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(10, 11, 13), (17, 16, 21), (30, 30, 24)])
def test_multigrid_apply_matches_oracle(ect, prec, shape):
    """One W-cycle (2 and 3 levels) against the oracle's, same hierarchy rules.

    Metric e_S = ||S (z - z_ref)|| / ||S z_ref|| per right-hand side (S the
    scaled finest matrix): z is dominated by the coarse correction of the
    near-null gauge modes, which S damps, so e_S sees errors on every level
    (pinned in test_oracle_multigrid_metric: an FP32 execution of the
    oracle's cycle stays below a tenth of the FP32 bound, indexing errors
    planted on a coarse level exceed it).  Bounds: FP32 1e-2 (the GPU's FP32
    cycles measured <= 3.9e-3, median ~2e-3, here); FP64
    1e-7: the GPU inverts the coarsest operator (condition ~1e8) by Gauss-Jordan,
    the oracle by LAPACK, so the two coarse corrections differ by ~kappa eps64
    ~1e-8 relative (measured 2-3e-9 in e_S).  The 30 x 30 x 24 mesh (21,600 nodes) has the residual updates
    t -= AP e and the shared-memory-staged SpMM on its finest level; it runs
    the FP32 cycle with the staged kernels and with the unstaged ones."""
    p = E.wall_loss_problem(shape, (20e-3, 20e-3, 30e-3), (2, 2, 2), 0.15, 4, z_pos=(0.0,))
    ctx = make_ctx(ect, p, group=-1)
    M = fem.system_matrix(p, "defect")
    lv = _oracle_amg(p, M, "defect")
    S = fem.scaled(M, fem.scaling(M))
    assert len(lv) >= (3 if shape[0] > 10 else 2)
    rng = np.random.default_rng(11)
    n = 4 * p.mesh.n_nodes
    k = 19 if shape[0] < 30 else 11              # full tiles of 8, then partial ones
    R = crand(rng, k, n)
    refs = [solve.amg_apply(lv, R[q]) for q in range(k)]
    dt, pr, tol = ((torch.complex128, ect.ECT_F64, 1e-7) if prec == "f64" else (torch.complex64, ect.ECT_F32, 1e-2))
    r = dev(R, dt)
    for rows in ((0, -1, -2) if prec == "f32" else (0,)):
        ctx.set_spmm_rows(rows)
        z = torch.empty_like(r)
        ctx.precond_apply(1, r, z, k, precision=pr)
        Z = z.cpu().numpy()
        es = [np.linalg.norm(S @ (Z[q] - refs[q])) / np.linalg.norm(S @ refs[q]) for q in range(k)]
        assert max(es) <= tol, (rows, int(np.argmax(es)), max(es), float(np.median(es)))
    ctx.set_spmm_rows(0)
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_multigrid_solve(ect, mode):
    p = E.wall_loss_problem((17, 16, 21), (20e-3, 20e-3, 30e-3), (2, 2, 2), 0.15, 4, z_pos=(0.0,))
    M = {w: fem.system_matrix(p, w) for w in WHICH}
    ctx = make_ctx(ect, p, group=-1)
    opts = ect.default_options(tol=1e-10, restart=30, mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED,
                               inner_iters=10, max_iters=2000 if mode == "f64" else 200)
    for w in WHICH:
        X, st = _solve_check(ect, p, ctx, M, w, opts)
        assert st["converged"] == 2 and st["iters"] < 400, st


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("group", [0, 1, 3])
def test_precond_apply(ect, small, prec, group):
    """Block-Jacobi (group 0) and the two-level conductor-V coarse space (groups 1, 3)."""
    p, ctx1, M = small
    ctx = ctx1 if group == 1 else make_ctx(ect, p, group=group)
    rng = np.random.default_rng(2)
    n = 4 * p.mesh.n_nodes
    t = fem.scaling(M["defect"])
    S = fem.scaled(M["defect"], t)
    P = solve.block_jacobi(S, p.mesh.block_of_node)
    s, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "defect")
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s)
    C = solve.coarse_v(S, t, p.mesh.block_of_node, cond, group) if group else None
    k = 11                                       # one full tile of 8 and a partial one
    R = crand(rng, k, n)
    dt, pr, tol = ((torch.complex128, ect.ECT_F64, 1e-9) if prec == "f64" else (torch.complex64, ect.ECT_F32, 1e-3))
    r = dev(R, dt)
    z = torch.empty_like(r)
    ctx.precond_apply(WHICH["defect"], r, z, k, precision=pr)
    Z = z.cpu().numpy()
    for q in range(k):
        ref = solve.two_level_apply(P, C, R[q])
        assert np.linalg.norm(Z[q] - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,j", [(1000, 1), (70001, 7), (5003, 33)])
def test_cgs2_matches_oracle(ect, prec, n, j):
    rng = np.random.default_rng(n + j)
    Vq, _ = np.linalg.qr(crand(rng, n, j))
    w = crand(rng, n)
    h_ref, w_ref, beta_ref = solve.cgs2(Vq, w)
    dt, pr, tol = ((torch.complex128, ect.ECT_F64, 1e-12) if prec == "f64" else (torch.complex64, ect.ECT_F32, 2e-5))
    ctx = ect.Context()
    V = dev(Vq.T, dt)
    wd = dev(w, dt)
    h, beta = ctx.cgs2(V, wd, precision=pr)
    nw = np.linalg.norm(w)
    assert np.abs(h - h_ref).max() <= tol * nw
    assert abs(beta - beta_ref) <= tol * nw
    assert np.linalg.norm(wd.cpu().numpy() - w_ref) <= tol * nw
    ctx.close()


def test_coil_rhs_matches_oracle(ect, small):
    p, ctx, M = small
    n = 4 * p.mesh.n_nodes
    zs = np.array([0.0, 3.3e-3, -7.1e-3])
    for c in p.coils:
        out = torch.empty(3, n, dtype=torch.complex128, device="cuda")
        ctx.coil_rhs(c, zs, out)
        B = out.cpu().numpy()
        for q, z in enumerate(zs):
            ref = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), z), p, "vacuum")
            assert np.abs(ref).max() > 0
            assert np.abs(B[q] - ref).max() <= 1e-13 * np.abs(ref).max()


def _solve_check(ect, p, ctx, M, which, opts, k=2, x_init=None):
    n = 4 * p.mesh.n_nodes
    B = np.stack([fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), p.z_pos[0]), p, which)
                  for c in p.coils][:k])
    b = dev(B)
    x = torch.empty_like(b) if x_init is None else dev(x_init)
    st = ctx.solve(WHICH[which], b, x, k, opts)
    X = x.cpu().numpy()
    t = fem.scaling(M[which])
    for q in range(k):
        res = np.linalg.norm(t * (B[q] - M[which] @ X[q])) / np.linalg.norm(t * B[q])
        assert res <= opts.tol * 1.0001, (q, res, st)
    return X, st


@pytest.mark.parametrize("mode", ["f64", "mixed"])
@pytest.mark.parametrize("graph", [0, 1])
def test_solve_residual_with_oracle_matrix(ect, small, mode, graph):
    p, ctx, M = small
    opts = ect.default_options(tol=1e-10, restart=30, use_graph=graph,
                               mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED, inner_iters=20)
    for w in WHICH:
        X, st = _solve_check(ect, p, ctx, M, w, opts)
        assert st["converged"] == 2


@pytest.mark.parametrize("rows", [8, 16, -1, -2])
def test_mixed_solve_spmm_tilings(ect, small, rows):
    """Mixed mode with the staged FP32 SpMM at other row tilings and with the unstaged kernels."""
    p, ctx, M = small
    opts = ect.default_options(tol=1e-10, restart=16, mode=ect.ECT_MODE_MIXED, inner_iters=16, spmm_rows=rows)
    for w in WHICH:
        X, st = _solve_check(ect, p, ctx, M, w, opts)
        assert st["converged"] == 2


@pytest.mark.parametrize("reorth", [0, 2, 3])
def test_mixed_solve_gram_schmidt_variants(ect, small, reorth):
    """Mixed mode with two passes always (0), one inner pass (2), one pass in both loops (3)."""
    p, ctx, M = small
    opts = ect.default_options(tol=1e-10, restart=16, mode=ect.ECT_MODE_MIXED, inner_iters=16, reorth=reorth)
    for w in WHICH:
        X, st = _solve_check(ect, p, ctx, M, w, opts)
        assert st["converged"] == 2


def test_solve_batch_equals_single(ect, small):
    p, ctx, M = small
    opts = ect.default_options(tol=1e-11)
    X2, _ = _solve_check(ect, p, ctx, M, "defect", opts, k=2)
    X1, _ = _solve_check(ect, p, ctx, M, "defect", opts, k=1)
    assert np.linalg.norm(X2[0] - X1[0]) <= 1e-6 * np.linalg.norm(X1[0])


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_initial_guess(ect, small, mode):
    """x0 = 1: the vacuum solutions as the defect system's initial guess (the warm start of a
    deposit scan) meet the same tolerance against the oracle's matrix in fewer iterations, and a
    guess already far inside the tolerance needs no iteration."""
    p, ctx, M = small
    kw = dict(restart=16, mode=ect.ECT_MODE_F64 if mode == "f64" else ect.ECT_MODE_MIXED, inner_iters=16)
    cold = ect.default_options(tol=1e-10, **kw)
    X0, _ = _solve_check(ect, p, ctx, M, "vacuum", cold)
    Xd, st_cold = _solve_check(ect, p, ctx, M, "defect", cold)
    warm = ect.default_options(tol=1e-10, x0=1, **kw)
    Xw, st_warm = _solve_check(ect, p, ctx, M, "defect", warm, x_init=X0)
    assert st_warm["converged"] == 2 and 0 < st_warm["iters"] <= st_cold["iters"], (st_warm, st_cold)
    Xt, _ = _solve_check(ect, p, ctx, M, "defect", ect.default_options(tol=1e-12, **kw))
    Xe, st_e = _solve_check(ect, p, ctx, M, "defect", warm, x_init=Xt)
    assert st_e["iters"] == 0 and st_e["converged"] == 2, st_e
    assert np.array_equal(Xe, Xt) or np.abs(Xe - Xt).max() <= 1e-14 * np.abs(Xt).max()


def test_delta_z_kernel_on_oracle_solutions(ect, small):
    """Kernel (e) alone: oracle solutions in, Delta Z out, against the oracle's global formula."""
    p, ctx, M = small
    b = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), 0.0), p, "vacuum") for c in p.coils]
    u0 = [solve.dense_solve(M["vacuum"], bk) for bk in b]
    ud = [solve.dense_solve(M["defect"], bk) for bk in b]
    I = [c.current for c in p.coils]
    ref = impedance.delta_z_matrix(M["vacuum"], M["defect"], u0, ud, I, p.omega)
    ref_emf = impedance.delta_z_emf_matrix(b, u0, ud, I, p.omega)
    dz, dze = ctx.delta_z(dev(np.stack(u0)), dev(np.stack(ud)), dev(np.stack(b)), I)
    assert np.abs(dz - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(dze - ref_emf).max() <= 1e-11 * np.abs(ref_emf).max()


def test_impedance_c1_against_oracle_golden(ect):
    g = json.load(open(os.path.join(HERE, "golden", "c1_oracle.json")))
    ref = np.array([[complex(*g["dz"][k][l]) for l in range(2)] for k in range(2)])
    p = E.make_config("c1")
    ctx = make_ctx(ect, p)
    for mode in (ect.ECT_MODE_F64, ect.ECT_MODE_MIXED):
        opts = ect.default_options(tol=1e-10, mode=mode, inner_iters=20)
        dz, st = ctx.impedance(p.coils, p.z_pos, opts)
        err = np.abs(dz[0] - ref).max() / np.abs(ref).max()
        assert err <= 1e-6, (mode, err, st)
        assert st["converged"] == 4
        assert abs(dz[0, 0, 1] - dz[0, 1, 0]) <= 1e-6 * np.abs(ref).max()


# ------------------------------------------------------------------ edge cases

def test_zero_contrast_gives_exact_zero(ect):
    p = small_problem()
    p.sigma_d = np.full_like(p.sigma_d, np.nan)
    ctx = make_ctx(ect, p, f32=False)
    dz, st = ctx.impedance(p.coils, p.z_pos, ect.default_options(tol=1e-10))
    assert np.all(dz == 0)


def test_coil_outside_mesh_gives_zero_solution(ect, small):
    p, ctx, M = small
    n = 4 * p.mesh.n_nodes
    b = torch.empty(1, n, dtype=torch.complex128, device="cuda")
    ctx.coil_rhs(p.coils[0], [1.0], b)                  # 1 m away along the axis
    assert torch.count_nonzero(b).item() == 0
    x = torch.full_like(b, 1.0)
    st = ctx.solve(0, b, x, 1)
    assert st["converged"] == 1 and torch.count_nonzero(x).item() == 0


def test_not_converged_and_timeout_report(ect, small):
    p, ctx, M = small
    n = 4 * p.mesh.n_nodes
    b = torch.empty(1, n, dtype=torch.complex128, device="cuda")
    ctx.coil_rhs(p.coils[0], [0.0], b)
    x = torch.empty_like(b)
    with pytest.raises(ect.EctError) as e:
        ctx.solve(0, b, x, 1, ect.default_options(restart=5, max_iters=5))
    assert e.value.code == ect.ECT_ERR_NOT_CONVERGED and e.value.stats["iters"] == 5
    assert 0 < e.value.stats["relres_max"] < 1
    with pytest.raises(ect.EctError) as e:
        ctx.solve(0, b, x, 1, ect.default_options(timeout_s=1e-12))
    assert e.value.code == ect.ECT_ERR_TIMEOUT


def test_bad_meshes_rejected(ect):
    p = small_problem()
    m = p.mesh
    ctx = ect.Context()
    bad = m.tets.copy()
    bad[5, [1, 2]] = bad[5, [2, 1]]                         # inverted tet
    with pytest.raises(ect.EctError) as e:
        ctx.set_mesh(m.xyz, bad, p.sigma, p.nu, None, None, m.block_of_node, m.bc_mask)
    assert e.value.code == ect.ECT_ERR_MESH
    bad = m.tets.copy()
    bad[0, 0] = m.n_nodes                                   # index out of range
    with pytest.raises(ect.EctError) as e:
        ctx.set_mesh(m.xyz, bad, p.sigma, p.nu, None, None, m.block_of_node, m.bc_mask)
    assert e.value.code == ect.ECT_ERR_MESH
    with pytest.raises(ect.EctError) as e:                  # one block of all nodes (> 16)
        ctx.set_mesh(m.xyz, m.tets, p.sigma, p.nu, None, None, np.zeros(m.n_nodes, np.int32), m.bc_mask)
    assert e.value.code == ect.ECT_ERR_ARG
    with pytest.raises(ect.EctError) as e:                  # solve before assembly
        ctx.set_mesh(m.xyz, m.tets, p.sigma, p.nu, None, None, m.block_of_node, m.bc_mask)
        b = torch.zeros(1, 4 * m.n_nodes, dtype=torch.complex128, device="cuda")
        ctx.solve(0, b, torch.empty_like(b), 1)
    assert e.value.code == ect.ECT_ERR_STATE


def test_empty_and_oversized_batches_rejected(ect, small):
    """k = 0 and k beyond the documented limits are argument errors, reported before any work."""
    p, ctx, M = small
    n = 4 * p.mesh.n_nodes
    b = torch.zeros(1, n, dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    for k in (0, 4097):
        with pytest.raises(ect.EctError) as e:
            ctx.solve(0, b, x, k)
        assert e.value.code == ect.ECT_ERR_ARG, k
    with pytest.raises(ect.EctError) as e:
        ctx.spmv(0, b, x, 0)
    assert e.value.code == ect.ECT_ERR_ARG
    with pytest.raises(ect.EctError) as e:
        ctx.coil_rhs(p.coils[0], np.zeros(0), b)
    assert e.value.code == ect.ECT_ERR_ARG
    for batch in (0, 100, 65536 + 256):
        with pytest.raises(ect.EctError):
            ect.Surrogate(batch=batch)


def test_autotune_returns_converging_options(ect, small):
    p, ctx, M = small
    n = 4 * p.mesh.n_nodes
    B = np.stack([fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), 0.0), p, "defect")
                  for c in p.coils])
    b = dev(B)
    work = torch.empty_like(b)
    for mode in (ect.ECT_MODE_F64, ect.ECT_MODE_MIXED):
        best, st = ctx.autotune(1, b, work, 2, ect.default_options(tol=1e-10, mode=mode))
        assert best.rhs_tile in (-1, 1, 2, 4, 8) and st["converged"] == 2
        assert best.mode == mode and 1 <= best.restart <= 64
        assert best.spmm_rows in ((0, 24, 16, -1, -2) if mode == ect.ECT_MODE_MIXED else (0,))
        assert ctx.block_split() in (1, 2)                 # the subdomain split the tuner applied
        for w in ("defect", "vacuum"):                     # both preconditioners rebuilt for it
            X, st2 = _solve_check(ect, p, ctx, M, w, best)
            assert st2["converged"] == 2


def test_set_defect_reassembles_only_the_defect_matrix(ect):
    p = small_problem(seed=2)
    ctx = make_ctx(ect, p, f32=False)
    p2 = small_problem(seed=2)
    p2.sigma_d = np.where(np.isnan(p.sigma_d), np.nan, 0.2e6)
    ctx.set_defect(p2.sigma_d, p2.nu_d)
    with pytest.raises(ect.EctError) as e:                 # defect matrix must be rebuilt first
        ctx.matrix_copy(1)
    assert e.value.code == ect.ECT_ERR_STATE
    ctx.assemble(1, ect.ECT_F64)
    G = bsr_to_csr(*ctx.matrix_copy(1))
    O = fem.system_matrix(p2, "defect")
    d = np.sqrt(np.abs(O.diagonal()))
    D = (G - O).tocoo()
    assert np.all(np.abs(D.data) <= 1e-12 * d[D.row] * d[D.col] + 1e-300)
    G0 = bsr_to_csr(*ctx.matrix_copy(0))                    # vacuum untouched
    assert abs(G0 - fem.system_matrix(p2, "vacuum")).max() <= 1e-12 * abs(G0).max()
