"""Oracle: linear solves of the constrained system.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper factorises the global matrix once with SuperLU and then solves one
right-hand side per probe position (Sec. 3, Steps 5-6).  The oracle offers:
  * dense_solve    numpy.linalg.solve (LAPACK LU) for tiny meshes;
  * superlu_solve  scipy's SuperLU, the paper's own solver family;
  * block_jacobi   the inverses of the diagonal blocks of the scaled matrix
                   over the node subdomains (the subdomain-block
                   preconditioner: z = blockdiag(S_ss)^-1 r);
  * coarse_v       the conductor-V coarse space: one coarse unknown per
                   group of `group` consecutive subdomains that touches the
                   conductor, constant (=1 in the unscaled V) on that group's
                   conducting nodes; E = Z^T S Z and the additive two-level
                   preconditioner z = blockdiag(S_ss)^-1 r + Z E^-1 Z^T r;
  * fgmres         restarted flexible GMRES (Saad's algorithm) with
                   classical Gram-Schmidt applied twice, complex Givens
                   rotations for the Hessenberg least-squares problem, and a
                   right preconditioner (plain GMRES when it is None).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def dense_solve(M, b):
    """LAPACK LU solve on the dense matrix (tiny meshes; the direct solve of Sec. 3, Step 5)."""
    return np.linalg.solve(M.toarray() if sp.issparse(M) else M, b)


def superlu_solve(M, b):
    """SuperLU solve, the paper's own solver family (Sec. 3, Step 5)."""
    lu = spla.splu(sp.csc_matrix(M))
    return lu.solve(np.asarray(b)), lu


def block_ranges(block_of_node):
    """Dof ranges [start, stop) of each subdomain block (4 dofs per node)."""
    bon = np.asarray(block_of_node)
    starts = np.flatnonzero(np.r_[True, bon[1:] != bon[:-1]])
    stops = np.r_[starts[1:], bon.size]
    return 4 * starts, 4 * stops


def block_jacobi(S, block_of_node):
    """Dense inverses of the diagonal blocks S[s:e, s:e]."""
    S = sp.csr_matrix(S)
    starts, stops = block_ranges(block_of_node)
    inv = []
    for s, e in zip(starts, stops):
        inv.append(np.linalg.inv(S[s:e, s:e].toarray()))
    return starts, stops, inv


def block_jacobi_apply(P, r):
    """z = blockdiag(S_ss)^-1 r over the subdomain blocks (the partition of Sec. 3, Step 2,
    used as a preconditioner)."""
    starts, stops, inv = P
    z = np.empty_like(r, dtype=np.complex128)
    for s, e, B in zip(starts, stops, inv):
        z[s:e] = B @ r[s:e]
    return z


def coarse_v(S, t, block_of_node, conducting, group):
    """Coarse space Z (n x nc, real), its Galerkin matrix E = Z^T S Z and E^-1.

    Column c of Z is 1/t_d on the V dof d of every conducting node whose
    subdomain id // group equals the c-th such group (in increasing order),
    i.e. the unscaled field V = 1 on those nodes and 0 elsewhere.  The idea
    follows the per-component gauge condition of Sec. 4 (V is fixed only up to
    a constant on each conducting component); here the constants are taken
    per group of subdomains of the partition (Sec. 3), which also captures
    the smooth V modes along the conductor that block-Jacobi leaves slow."""
    bon = np.asarray(block_of_node)
    cond = np.asarray(conducting, dtype=bool)
    nodes = np.nonzero(cond)[0]
    n = S.shape[0]
    if nodes.size == 0:
        return None
    grp = bon[nodes] // group
    _, cid = np.unique(grp, return_inverse=True)
    dofs = 4 * nodes + 3
    Z = sp.csr_matrix((1.0 / np.asarray(t)[dofs], (dofs, cid)), shape=(n, int(cid.max()) + 1))
    E = (Z.T @ (sp.csr_matrix(S) @ Z)).toarray()
    return Z, E, np.linalg.inv(E)


def two_level_apply(P, C, r):
    """z = blockdiag(S_ss)^-1 r + Z E^-1 Z^T r (C = coarse_v(...), may be None)."""
    z = block_jacobi_apply(P, r)
    if C is not None:
        Z, _, Ei = C
        z = z + Z @ (Ei @ (Z.T @ r))
    return z


def givens(a, b):
    """Complex Givens rotation (c real, s complex) with [c s; -conj(s) c][a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0.0:
        return 0.0, 1.0 + 0.0j, b
    rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    ph = a / abs(a)
    return abs(a) / rho, ph * np.conj(b) / rho, ph * rho


def cgs2(V, w, selective=False, one_pass=False):
    """Orthogonalise w against the orthonormal columns of V twice (CGS2).

    Returns (h, w_new, beta) with h = coefficients accumulated over both
    passes (Hermitian inner product) and beta = ||w_new||.  With
    selective=True the second pass runs only when the first one removed more
    than half of ||w||^2 (||w_1||^2 < ||w_0||^2 / 2, the Daniel-Gragg-Kaufman-
    Stewart test with eta = 1/sqrt(2)); with one_pass=True it never runs
    (classical Gram-Schmidt, the usual GMRES default).  The paper names GMRES but
    not its Gram-Schmidt variant, so all three are offered."""
    n0 = np.vdot(w, w).real
    h1 = V.conj().T @ w
    w = w - V @ h1
    if one_pass or (selective and np.vdot(w, w).real >= 0.5 * n0):
        return h1, w, np.linalg.norm(w)
    h2 = V.conj().T @ w
    w = w - V @ h2
    return h1 + h2, w, np.linalg.norm(w)


def fgmres(A, b, precond=None, x0=None, tol=1e-10, restart=30, maxiter=10000, selective=False,
           one_pass=False):
    """Restarted right-preconditioned flexible GMRES (Saad).

    A and precond are callables (or matrices).  Stops when the true residual
    ||b - A x|| / ||b|| <= tol at a restart, or after maxiter iterations.
    `selective` / `one_pass` choose the Gram-Schmidt variant (see cgs2).
    Returns (x, info) with info = dict(iters, relres, history)."""
    mv = A if callable(A) else (lambda v: A @ v)
    pc = (lambda v: v) if precond is None else (precond if callable(precond) else (lambda v: precond @ v))
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), dict(iters=0, relres=0.0, history=hist)
    total = 0
    r = b - mv(x)
    beta = np.linalg.norm(r)
    while True:
        relres = beta / bnorm
        hist.append(relres)
        if relres <= tol or total >= maxiter:
            break
        m = min(restart, maxiter - total)
        V = np.zeros((n, m + 1), dtype=np.complex128)
        Z = np.zeros((n, m), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Z[:, j] = pc(V[:, j])
            w = mv(Z[:, j])
            h, w, hn = cgs2(V[:, :j + 1], w, selective, one_pass)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):                      # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s, rr = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            k = j + 1
            total += 1
            if hn == 0.0 or abs(g[j + 1]) / bnorm <= tol:
                break
            V[:, j + 1] = w / hn
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:, :k] @ y
        r = b - mv(x)
        beta = np.linalg.norm(r)
    return x, dict(iters=total, relres=beta / bnorm, history=hist)


# ---------------------------------------------------------------- aggregation multigrid
#
# Multilevel version of the subdomain idea: the subdomains of the partition
# (Sec. 3, Step 2) are the aggregates of the first coarsening, and they are
# also the smoothing blocks of the finest level.  Definitions:
#   * near-null weights w: 1/t on free dofs of the finest level (the unscaled
#     field equal to 1 in one component), 0 on constrained dofs; on coarser
#     levels 1 on non-empty coarse dofs, 0 on empty ones;
#   * tentative prolongator P (no smoothing): column (I, c) holds w on the
#     component-c dofs of the nodes of aggregate I; E = P^T A P, plus the
#     identity on coarse dofs whose column is empty;
#   * coarse node graph: I ~ J when some node of I shares a stored block with
#     some node of J (the finest graph is "nodes share a tet");
#   * aggregates of a coarse level: greedy in increasing node order, a seed
#     takes its not yet aggregated neighbours (increasing order) up to
#     `agg_size` nodes; coarse nodes are renumbered so that aggregates are
#     contiguous (stable by aggregate);
#   * cycle: z = B^-1 r; gamma times { z += P mg(P^T (r - A z)) }; z += B^-1 (r - A z),
#     with B the block diagonal over the level's aggregates, gamma = 2 (W-cycle)
#     and 1 when the next level is the coarsest, which is solved densely.


def node_graph_from_tets(n_nodes, tets):
    """Node adjacency of the mesh (nodes sharing a tet), as sorted neighbour lists."""
    tets = np.asarray(tets, dtype=np.int64)
    r = np.repeat(tets, 4, axis=1).ravel()
    c = np.tile(tets, (1, 4)).ravel()
    G = sp.csr_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(n_nodes, n_nodes))
    G.sum_duplicates()
    G.sort_indices()
    return G


def greedy_aggregates(G, agg_size):
    """Greedy aggregation: each unaggregated seed takes its unaggregated neighbours in
    increasing order, at most agg_size nodes.  The paper has no multigrid: this is the
    coarse space built on its partition (Sec. 3, Step 2), as in the notes above."""
    G = sp.csr_matrix(G)
    G.sort_indices()
    n = G.shape[0]
    agg = -np.ones(n, dtype=np.int64)
    na = 0
    for i in range(n):
        if agg[i] >= 0:
            continue
        members = [i]
        for j in G.indices[G.indptr[i]:G.indptr[i + 1]]:
            if len(members) >= agg_size:
                break
            if j != i and agg[j] < 0:
                members.append(j)
        agg[members] = na
        na += 1
    return agg


def amg_setup(S, w0, node_agg0, G0, max_coarse_dofs=2048, agg_size=8):
    """Levels of the aggregation hierarchy (see the notes above).

    S: scaled matrix, w0: finest near-null weights (4n), node_agg0: aggregate of
    each finest node (non-decreasing, the subdomain blocks), G0: finest node graph."""
    levels = []
    A = sp.csr_matrix(S)
    w = np.asarray(w0, dtype=np.float64)
    agg = np.asarray(node_agg0, dtype=np.int64)
    G = sp.csr_matrix(G0)
    while True:
        n = A.shape[0] // 4
        na = int(agg.max()) + 1
        BJ = block_jacobi(A, agg)
        rows = np.arange(4 * n)
        cols = 4 * np.repeat(agg, 4) + np.tile(np.arange(4), n)
        P = sp.csr_matrix((w, (rows, cols)), shape=(4 * n, 4 * na))
        empty = np.asarray(abs(P).sum(axis=0)).ravel() == 0
        Ac = (P.T @ A @ P).tocsr() + sp.diags(empty.astype(np.float64))
        wc = np.where(empty, 0.0, 1.0)
        Ag = sp.csr_matrix((np.ones(n, dtype=np.int8), (agg, np.arange(n))), shape=(na, n))
        Gc = (Ag @ G @ Ag.T).tocsr()
        Gc.sort_indices()
        if 4 * na <= max_coarse_dofs:
            levels.append(dict(A=A, P=P, BJ=BJ))
            Acd = Ac.toarray()
            levels.append(dict(A=Ac, inv=np.linalg.inv(Acd)))
            return levels
        cagg = greedy_aggregates(Gc, agg_size)
        order = np.argsort(cagg, kind="stable")
        perm = (4 * order[:, None] + np.arange(4)[None]).ravel()
        P = P[:, perm].tocsr()
        levels.append(dict(A=A, P=P, BJ=BJ))
        A = Ac[perm][:, perm].tocsr()
        w = wc[perm]
        G = Gc[order][:, order].tocsr()
        G.sort_indices()
        agg = cagg[order]


def amg_apply(levels, r, l=0, gamma=2):
    """One W-cycle (gamma = 2, 1 above the coarsest level): block-Jacobi pre-smoothing,
    coarse corrections, block-Jacobi post-smoothing (the cycle defined in the notes above)."""
    L = levels[l]
    if "inv" in L:
        return L["inv"] @ r
    A, P, BJ = L["A"], L["P"], L["BJ"]
    z = block_jacobi_apply(BJ, r)
    g = 1 if "inv" in levels[l + 1] else gamma
    for _ in range(g):
        z = z + P @ amg_apply(levels, P.T @ (r - A @ z), l + 1, gamma)
    z = z + block_jacobi_apply(BJ, r - A @ z)
    return z


def near_null_weights(t, fixed_dofs):
    """Tentative-prolongator weights: 1/t on free dofs (a constant unscaled field per
    component), 0 on constrained ones."""
    w = 1.0 / np.asarray(t, dtype=np.float64)
    w[np.asarray(fixed_dofs)] = 0.0
    return w
