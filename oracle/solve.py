"""Global assembly and linear solves of K u = f (Eq. 1) for the oracle (test infrastructure only).

K = sum_e P_e^T K_e P_e, with P_e the element prolongation of ``mesh.DPMesh`` (identity gather on
conforming nodes, minimum-rule interpolation on constrained edge nodes).  Supports are homogeneous
Dirichlet conditions: fixed rows and columns are removed and u = 0 there.  The paper does not name
its solver; the oracle solves exactly (dense Cholesky, sparse LU) where that fits, and otherwise by a
plain FP64 Jacobi-preconditioned CG to a stated tolerance.
"""
import functools

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .element import element_stiffness, simp, subcell_stiffness


@functools.lru_cache(maxsize=None)
def K0_table(p, d, nu, hx=1.0, hy=1.0):
    """Cached subcell stiffness table K0[s] for class (p, d) (App. B composite integration)."""
    t = subcell_stiffness(p, d, nu, hx, hy)
    t.setflags(write=False)
    return t


def element_matrices(mesh, rho, E0, Emin, nu, q):
    """Dense K_e for every element: K_e = sum_s E(rho_s) K0[s] (Eqs. 2-3, composite rule)."""
    Ke = []
    for e in range(mesh.nel):
        p, d = int(mesh.p[e]), int(mesh.d[e])
        r = rho[mesh.design_off[e]:mesh.design_off[e + 1]]
        Ke.append(element_stiffness(K0_table(p, d, nu, mesh.hx, mesh.hy), simp(r, E0, Emin, q)))
    return Ke


def assemble(mesh, Ke):
    """Global sparse K = sum_e P_e^T K_e P_e (CSR, ndof x ndof, all DOFs incl. supported ones)."""
    rows, cols, vals = [], [], []
    for e in range(mesh.nel):
        P, G = mesh.prolongation(e)
        Kg = P.T @ Ke[e] @ P
        rows.append(np.repeat(G, len(G)))
        cols.append(np.tile(G, len(G)))
        vals.append(Kg.ravel())
    K = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(mesh.ndof, mesh.ndof)).tocsr()
    K.sum_duplicates()
    return K


def free_dofs(ndof, fixed):
    mask = np.ones(ndof, dtype=bool)
    mask[np.asarray(fixed, dtype=np.int64)] = False
    return np.nonzero(mask)[0]


def solve_direct(K, f, fixed, refine=3):
    """Exact solve of the supported system: dense Cholesky for small systems (library primitive),
    sparse LU (SuperLU, library primitive) otherwise.  The system is first equilibrated with the
    symmetric diagonal scaling S = diag(A)^-1/2 (A -> S A S, b -> S b, u = S y), which removes the
    1e9 row-scale spread that Emin = 1e-9 E0 creates, then ``refine`` steps of FP64 iterative
    refinement y += Ahat^-1 (bhat - Ahat y) follow.  Returns the full-length u (0 on supports)."""
    free = free_dofs(K.shape[0], fixed)
    Kff = K[free][:, free].tocsr()
    s = 1.0 / np.sqrt(Kff.diagonal())
    Ahat = (scipy.sparse.diags(s) @ Kff @ scipy.sparse.diags(s)).tocsr()
    b = s * f[free]
    if len(free) <= 4000:
        c = scipy.linalg.cho_factor(Ahat.toarray(), lower=True)
        solve1 = lambda r: scipy.linalg.cho_solve(c, r)
    else:
        lu = scipy.sparse.linalg.splu(Ahat.tocsc(), permc_spec="MMD_AT_PLUS_A")
        solve1 = lu.solve
    y = solve1(b)
    for _ in range(refine):
        y = y + solve1(b - Ahat @ y)
    u = np.zeros(K.shape[0])
    u[free] = s * y
    return u


def pcg(K, f, fixed, rtol=1e-12, maxiter=200000, x0=None, scaled=False):
    """Plain FP64 Jacobi-preconditioned conjugate gradients on the supported system.

    Textbook PCG (Hestenes-Stiefel with z = D^-1 r), stopped when ||r|| <= rtol ||f|| in the l2
    norm, or in the D^-1 norm (||r||^2 = r^T D^-1 r) when ``scaled``.
    Returns (u, iterations, final relative residual in that norm).
    """
    free = free_dofs(K.shape[0], fixed)
    A = K[free][:, free].tocsr()
    b = f[free]
    dinv = 1.0 / A.diagonal()
    x = np.zeros(len(free)) if x0 is None else x0[free].copy()
    r = b - A @ x
    z = dinv * r
    pdir = z.copy()
    rz = r @ z
    norm = (lambda v: np.sqrt(v @ (dinv * v))) if scaled else np.linalg.norm
    nb = norm(b)
    it = 0
    while norm(r) > rtol * nb and it < maxiter:
        qv = A @ pdir
        alpha = rz / (pdir @ qv)
        x += alpha * pdir
        r -= alpha * qv
        z = dinv * r
        rz_new = r @ z
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        it += 1
    u = np.zeros(K.shape[0])
    u[free] = x
    return u, it, norm(r) / nb


def solve(mesh, rho, fixed, f, E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    """Build, assemble and solve exactly.  Returns (u, K, Ke list)."""
    Ke = element_matrices(mesh, rho, E0, Emin, nu, q)
    K = assemble(mesh, Ke)
    return solve_direct(K, f, fixed), K, Ke
