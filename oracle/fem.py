"""Oracle: P1 nodal A-V element matrices, assembly and boundary conditions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The discrete system is the Galerkin matrix of the paper's coupled form
(Sec. 2, the form L = L11 + L12 + L21 + L22 after the V equation is scaled by
-1/(i omega)):

  L((A,V),(Phi,phi)) = int nu curl A . curl Phi + int nu_t div A div Phi
                       - (1/(i omega)) int sigma (i omega A + grad V) . (i omega Phi + grad phi)
                       - (1/(i omega)) int delta sigma V phi          (gauge penalty, Sec. 4)

with nu = 1/mu and nu_t = 1/mu_tilde.  Unknowns are ordered per node as
(A_x, A_y, A_z, V); global dof index = 4*node + component.

Readings (paper silent or garbled there):
  * the weak form is authoritative: E = i omega A + grad V everywhere (the
    strong form's sign is garbled);
  * L11 includes the -i omega sigma mass term, as the expansion of the coupled
    form and the Freefem listing both have it (the printed L11 omits it);
  * no extra mu factors (the listing's mu*sigma scalings are not used);
  * test functions are real P1 hat functions, so the matrix is the bilinear
    (complex symmetric, M^T = M) one;
  * mu_tilde = mu_0 (nu_tilde is a parameter);
  * A.n = 0 on the box faces by strong elimination: zero row and column,
    unit diagonal, zero load;
  * V exists only on conducting nodes; at every node that touches no
    sigma > 0 tet its row/column is the identity (zero load);
  * the V gauge is the penalty delta*sigma*V added inside L22.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tet_geometry(xyz, tets):
    """Volumes |K| (T,) and barycentric gradients g (T,4,3) of each tet (the P1 hat
    functions of Sec. 3, Step 3).

    With J the 3x3 matrix whose rows are x_a - x_0 (a = 1..3), the
    barycentric coordinates satisfy x - x_0 = sum_a lambda_a (x_a - x_0), so
    (lambda_1, lambda_2, lambda_3) = (x - x_0) J^{-1}: grad lambda_a is the
    a-th column of J^{-1}, and grad lambda_0 = -sum of the others.
    """
    p = np.asarray(xyz, dtype=np.float64)[np.asarray(tets)]
    J = p[:, 1:, :] - p[:, :1, :]                 # (T,3,3) rows x_a - x_0
    vol = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)                        # columns = grad lambda_1..3
    g = np.empty((p.shape[0], 4, 3))
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    return vol, g


def element_matrices(vol, g, sigma, nu, nu_tilde, omega, delta):
    """Element matrices E[K, a, b, r, c] for tets K (complex128, (T,4,4,4,4)): the blocks
    L11, L12, L21, L22 of the coupled form of Sec. 2 with the gauge penalty of Sec. 4.

    a, b are local nodes (test, trial), r, c components (row = test
    component, col = trial component), component 3 = V.  Blocks:
      AA_ij = |K| [nu (d_ij g_a.g_b - g_aj g_bi) + nu_t g_ai g_bj]
              - i omega sigma |K| (1 + d_ab)/20 d_ij
      AV_i  = -sigma |K| g_bi / 4          (row A_i at a, col V at b)
      VA_j  = -sigma |K| g_aj / 4          (row V at a, col A_j at b)
      VV    = -(sigma/(i omega)) |K| [g_a.g_b + delta (1 + d_ab)/20]
    The P1 integrals used: int_K grad l_a . grad l_b = |K| g_a.g_b,
    int_K l_a l_b = |K| (1 + d_ab)/20, int_K l_a = |K|/4.
    """
    T = vol.shape[0]
    vol = vol[:, None, None]
    sig = np.asarray(sigma, dtype=np.float64)[:, None, None]
    nu = np.asarray(nu, dtype=np.float64)[:, None, None]
    gg = np.einsum("kai,kbi->kab", g, g)              # g_a . g_b
    mass = (1.0 + np.eye(4))[None] / 20.0             # (1 + d_ab)/20
    E = np.zeros((T, 4, 4, 4, 4), dtype=np.complex128)
    eye3 = np.eye(3)
    # curl-curl: (grad l_b x e_j) . (grad l_a x e_i) = d_ij g_a.g_b - g_aj g_bi
    curl = (gg[:, :, :, None, None] * eye3[None, None, None]
            - np.einsum("kaj,kbi->kabij", g, g))
    div = np.einsum("kai,kbj->kabij", g, g)           # g_ai g_bj
    AA = (vol[..., None, None] * (nu[..., None, None] * curl + nu_tilde * div)
          - 1j * omega * (sig * vol * mass)[..., None, None] * eye3[None, None, None])
    E[:, :, :, :3, :3] = AA
    E[:, :, :, :3, 3] = -(sig * vol)[..., None] * g[:, None, :, :] / 4.0    # g_bi
    E[:, :, :, 3, :3] = -(sig * vol)[..., None] * g[:, :, None, :] / 4.0    # g_aj
    E[:, :, :, 3, 3] = -(sig / (1j * omega)) * vol * (gg + delta * mass)
    return E


def effective_coefficients(sigma, nu, sigma_d, nu_d, which):
    """Per-tet (sigma, nu) of the background ('vacuum') or 'defect' matrix (the M_0 / M_d
    pair of Eq. impedkl).

    The defect arrays use NaN for "same as background"."""
    sigma = np.asarray(sigma, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    if which == "vacuum":
        return sigma, nu
    if which != "defect":
        raise ValueError(which)
    s = np.where(np.isnan(sigma_d), sigma, sigma_d)
    n = np.where(np.isnan(nu_d), nu, nu_d)
    return s, n


def conducting_nodes(n_nodes, tets, sigma):
    """Boolean (N,): node touches at least one tet with sigma > 0 (V lives on the conductor,
    Sec. 2; reading in the module notes)."""
    c = np.zeros(n_nodes, dtype=bool)
    c[np.asarray(tets)[np.asarray(sigma) > 0.0].ravel()] = True
    return c


def assemble_raw(xyz, tets, sigma, nu, nu_tilde, omega, delta, chunk=1 << 16):
    """Scalar CSR sum of the element matrices (before boundary conditions): the assembly of
    Sec. 3, Steps 3-4, done serially."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    n = 4 * xyz.shape[0]
    M = sp.csr_matrix((n, n), dtype=np.complex128)
    comp = np.arange(4)
    for s in range(0, tets.shape[0], chunk):
        t = tets[s:s + chunk]
        vol, g = tet_geometry(xyz, t)
        E = element_matrices(vol, g, sigma[s:s + chunk], nu[s:s + chunk], nu_tilde, omega, delta)
        ra = 4 * t[:, :, None, None, None] + comp[None, None, None, :, None]
        cb = 4 * t[:, None, :, None, None] + comp[None, None, None, None, :]
        rows = np.broadcast_to(ra, E.shape).ravel()
        cols = np.broadcast_to(cb, E.shape).ravel()
        M = M + sp.coo_matrix((E.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    return M


def fixed_dofs(bc_mask, conducting):
    """Dof indices eliminated by A.n = 0 on the box faces (Sec. 2 boundary conditions), and
    V dofs of non-conducting nodes."""
    bc = np.asarray(bc_mask, dtype=np.int64)
    N = bc.shape[0]
    node = np.arange(N)
    dir_ = [4 * node[(bc >> c) & 1 == 1] + c for c in range(3)]
    dirichlet = np.sort(np.concatenate(dir_))
    v_identity = 4 * node[~np.asarray(conducting)] + 3
    return dirichlet, v_identity


def apply_constraints(M, dirichlet, v_identity):
    """Zero the rows and columns of the constrained dofs and put 1 on the diagonal."""
    n = M.shape[0]
    keep = np.ones(n)
    fixed = np.concatenate([dirichlet, v_identity])
    keep[fixed] = 0.0
    Dk = sp.diags(keep)
    M = (Dk @ M @ Dk).tocsr()
    one = np.zeros(n)
    one[fixed] = 1.0
    M = (M + sp.diags(one)).tocsr()
    M.eliminate_zeros()
    return M


def system_matrix(problem, which):
    """The constrained system matrix of the 'vacuum' or 'defect' configuration."""
    m = problem.mesh
    s, n = effective_coefficients(problem.sigma, problem.nu, problem.sigma_d, problem.nu_d, which)
    M = assemble_raw(m.xyz, m.tets, s, n, problem.nu_tilde, problem.omega, problem.delta)
    cond = conducting_nodes(m.n_nodes, m.tets, s)
    d, v = fixed_dofs(m.bc_mask, cond)
    return apply_constraints(M, d, v)


def constrain_rhs(b, problem, which):
    """Zero the load at the constrained dofs (matching apply_constraints)."""
    m = problem.mesh
    s, _ = effective_coefficients(problem.sigma, problem.nu, problem.sigma_d, problem.nu_d, which)
    cond = conducting_nodes(m.n_nodes, m.tets, s)
    d, v = fixed_dofs(m.bc_mask, cond)
    b = np.array(b, dtype=np.complex128, copy=True)
    b[..., d] = 0.0
    b[..., v] = 0.0
    return b


def scaling(M):
    """Symmetric diagonal scaling t_i = 1/sqrt(|M_ii|); S = diag(t) M diag(t)."""
    d = np.abs(M.diagonal())
    return 1.0 / np.sqrt(d)


def scaled(M, t):
    """S = diag(t) M diag(t).  The paper does not say how residuals are measured; the
    solver's gate is the relative residual of this symmetrically scaled system, because the
    diagonal magnitudes of the A and V rows differ by ~1e5 and the unscaled norm hides the V
    equations."""
    D = sp.diags(t)
    return (D @ M @ D).tocsr()
