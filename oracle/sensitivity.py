"""Compliance and its design sensitivities (test infrastructure only).

Compliance C = f^T u is the objective of Eq. 1 with z = f (Sec. 4.1).  The paper uses design
sensitivities (Sec. 2.1) but does not print their formula.  For compliance the problem is
self-adjoint (adjoint lambda = -u), and with the composite stiffness K_e = sum_s E(rho_s) K0[s]
(Eqs. 2-3, App. B) differentiating C = f^T u gives

    dC/drho_s = -E'(rho_s) u_e^T K0[s] u_e,      E'(rho) = q rho^(q-1) (E0 - Emin).

The oracle evaluates each quadratic form naively with a dense K0[s] matrix-vector product, after
removing the element's rigid motion (which every K0[s] annihilates) so that no digits are lost to
cancellation.
"""
import numpy as np

from .element import remove_rigid_motion, simp, simp_deriv
from .solve import K0_table


def compliance(f, u):
    """C = f^T u (Eq. 1 with z = f)."""
    return float(np.dot(f, u))


def subcell_energies(mesh, u, nu):
    """w_s = u_e^T K0[s] u_e for every subcell of every element, packed like rho."""
    w = np.zeros(mesh.design_len)
    for e in range(mesh.nel):
        p, d = int(mesh.p[e]), int(mesh.d[e])
        ue = remove_rigid_motion(p, mesh.gather(e, u), mesh.hx, mesh.hy)
        K0 = K0_table(p, d, nu, mesh.hx, mesh.hy)
        off = mesh.design_off[e]
        for s in range(d * d):
            w[off + s] = ue @ (K0[s] @ ue)
    return w


def sensitivity(mesh, u, rho, E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    """dC/drho_s = -E'(rho_s) u_e^T K0[s] u_e, packed like rho (self-adjoint, lambda = -u)."""
    return -simp_deriv(rho, E0, Emin, q) * subcell_energies(mesh, u, nu)


def energy_split(mesh, u, rho, E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    """sum_e sum_s E(rho_s) w_s, which must equal u^T K u = C (energy identity)."""
    return float(np.sum(simp(rho, E0, Emin, q) * subcell_energies(mesh, u, nu)))
