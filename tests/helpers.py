"""Shared helpers for the test suite (no method arithmetic of its own
beyond textbook quadrature and Dirichlet lifting)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Degree-2 exact 4-point rule on a tetrahedron (barycentric a, b, b, b with
# a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights 1/4 of the volume).
QA = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
QB = (5.0 - np.sqrt(5.0)) / 20.0
QUAD4 = np.array([[QA, QB, QB, QB], [QB, QA, QB, QB], [QB, QB, QA, QB], [QB, QB, QB, QA]])


def hat_gradients_4x4(p):
    """Gradients of the P1 hat functions on one tet via the 4x4 vertex matrix.

    The hat function l_a = c0 + c.x with l_a(x_b) = delta_ab, so the
    coefficient columns are the columns of inv([1 x y z]); an independent
    route from the oracle's Jacobian-inverse formula."""
    A = np.hstack([np.ones((4, 1)), p])
    C = np.linalg.inv(A)
    return C[1:, :].T                       # (4,3): row a = grad l_a


def dirichlet_solve(M, f, fixed, values):
    """Solve M u = f with u[fixed] = values (lifting), returns u."""
    n = M.shape[0]
    free = np.setdiff1d(np.arange(n), fixed)
    u = np.zeros(n, dtype=np.complex128)
    u[fixed] = values
    M = sp.csr_matrix(M)
    rhs = f[free] - M[free][:, fixed] @ values
    u[free] = spla.spsolve(sp.csc_matrix(M[free][:, free]), rhs)
    return u


def quad_load(xyz, tets, F):
    """Load vector int F . l_a over the mesh with the 4-point rule.

    F maps (n,3) points to (n,4) complex values (one per component), and
    the result is (N*4,) with dof = 4*node + component."""
    p = xyz[tets]                                    # (T,4,3)
    J = p[:, 1:, :] - p[:, :1, :]
    vol = np.abs(np.linalg.det(J)) / 6.0
    N = xyz.shape[0]
    b = np.zeros((N, 4), dtype=np.complex128)
    for q in range(4):
        lam = QUAD4[q]
        x = np.einsum("a,tac->tc", lam, p)
        Fq = F(x)                                    # (T,4)
        for a in range(4):
            np.add.at(b, tets[:, a], (0.25 * vol * lam[a])[:, None] * Fq)
    return b.ravel()
