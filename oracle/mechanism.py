"""A general objective J = z^T u and its adjoint sensitivities, for the compliant-mechanism
(force inverter) problem of Sec. 4.1, Fig. 6b (test infrastructure only).

Eq. 1 states the objective as J = z^T u with K u = f; for the force inverter z is the unit vector
of the output DOF, and springs of stiffness k_in and k_out tie the input and output DOFs to
ground (k_in = 1, k_out = 0.001, f_in = 1; Sec. 4.1).  The problem is not self-adjoint: with the
adjoint field v solving K v = z (K symmetric, springs included),

    dJ/drho_s = z^T du/drho_s = -v^T (dK/drho_s) u = -E'(rho_s) v_e^T K0[s] u_e.

For compliance (z = f) v = u and this reduces to the compliance sensitivity.  Each bilinear form
is evaluated naively with a dense K0[s] matrix-vector product after the rigid-motion removal of
both element fields (K0[s] annihilates rigid motions on either side).

Reading of Fig. 6b (its picture is not in the text; labels only): a full 2L x L domain; the input
DOF is u_x at the mid-height vertex of the left edge, loaded by f_in (+x) and held by the spring
k_in; the output DOF is u_x at the mid-height vertex of the right edge, held by k_out; both
displacement components are clamped along the left edge within 0.01 L of the top and bottom
corners (at least the corner vertices).  The inverter minimises J = u_out (the output moves
against the input).
"""
import numpy as np
import scipy.sparse

from .element import remove_rigid_motion, simp_deriv
from .solve import K0_table


def inverter_problem(mesh, k_in=1.0, k_out=1e-3, f_in=1.0, clamp=0.01):
    """(fixed DOFs, f, z, spring DOFs, spring stiffnesses) of the force inverter (reading above).
    Needs an even nely (mid-height vertices)."""
    if mesh.nely % 2:
        raise ValueError("the input and output sit at mid-height vertices: nely must be even")
    L = mesh.nely * mesh.hy
    xy = mesh.node_xy()
    left = mesh.side_nodes(0)
    y = xy[left, 1]
    held = left[(y <= clamp * L + 1e-12) | (y >= L - clamp * L - 1e-12)]
    fixed = np.sort(np.concatenate([2 * held, 2 * held + 1]))
    din = 2 * mesh.vertex(0, mesh.nely // 2)
    dout = 2 * mesh.vertex(mesh.nelx, mesh.nely // 2)
    f = np.zeros(mesh.ndof)
    f[din] = f_in
    z = np.zeros(mesh.ndof)
    z[dout] = 1.0
    return fixed, f, z, np.array([din, dout], dtype=np.int64), np.array([k_in, k_out])


def add_springs(K, dofs, k):
    """K + sum_i k_i e_{d_i} e_{d_i}^T (springs to ground)."""
    n = K.shape[0]
    return (K + scipy.sparse.coo_matrix((np.asarray(k, dtype=np.float64), (dofs, dofs)), shape=(n, n))).tocsr()


def adjoint_sensitivity(mesh, u, v, rho, E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    """dJ/drho_s = -E'(rho_s) v_e^T K0[s] u_e, packed like rho (v solves K v = z)."""
    w = np.zeros(mesh.design_len)
    for e in range(mesh.nel):
        p, d = int(mesh.p[e]), int(mesh.d[e])
        ue = remove_rigid_motion(p, mesh.gather(e, u), mesh.hx, mesh.hy)
        ve = remove_rigid_motion(p, mesh.gather(e, v), mesh.hx, mesh.hy)
        K0 = K0_table(p, d, nu, mesh.hx, mesh.hy)
        off = mesh.design_off[e]
        for s in range(d * d):
            w[off + s] = ve @ (K0[s] @ ue)
    return -simp_deriv(rho, E0, Emin, q) * w
