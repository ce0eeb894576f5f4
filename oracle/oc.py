"""Optimality-criteria design update (test infrastructure only).

The paper does not name its optimizer (Sec. 4).  This is the textbook OC update for compliance
with a volume constraint (fixed-point update with move limit and damping exponent eta, the
Lagrange multiplier found by bisection):

    rho_new = clip(rho * (-dc / (lambda * dv))^eta, max(0, rho - m), min(1, rho + m)),
    lambda such that sum(rho_new * dv) = V0 * total area.
"""
import numpy as np


def oc_update(rho, dc, dv, vol_target, move=0.2, eta=0.5, l1=0.0, l2=1e9, tol=1e-10):
    """One OC step.  ``dv`` is each subcell's area, ``vol_target`` the allowed material area.

    Bisection on lambda in [l1, l2] until (l2 - l1) / (l1 + l2) <= tol; the returned design is the
    one at the final midpoint.  Returns (rho_new, lambda).
    """
    rho = np.asarray(rho, dtype=np.float64)
    B = np.maximum(-np.asarray(dc, dtype=np.float64), 0.0) / dv
    lo = np.maximum(0.0, rho - move)
    hi = np.minimum(1.0, rho + move)
    while (l2 - l1) / (l1 + l2) > tol:
        lmid = 0.5 * (l1 + l2)
        rnew = np.clip(rho * (B / lmid) ** eta, lo, hi)
        if np.dot(rnew, dv) > vol_target:
            l1 = lmid
        else:
            l2 = lmid
    lmid = 0.5 * (l1 + l2)
    return np.clip(rho * (B / lmid) ** eta, lo, hi), lmid


def subcell_areas(mesh):
    """dv_s = hx * hy / d_e^2 for every subcell, packed like rho."""
    return np.repeat(mesh.hx * mesh.hy / mesh.d.astype(np.float64) ** 2, mesh.d ** 2)
