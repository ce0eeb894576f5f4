"""The composite refinement indicator and the dp map update (test infrastructure only).

* Kelly analysis indicator Gamma^a (Sec. 3.2.1, Eq. 9);
* density indicator Gamma^d (Sec. 3.2.2, Eqs. 10-13 and the case list before them);
* QR-error indicator eps^QR (Sec. 3.2.3, Eq. 14);
* the dp-adaptivity map update (Sec. 3.3, steps 2-4) with alpha^d_r = alpha^d_c = 1 (Sec. 5).

Readings where the paper is silent or garbled are stated in each docstring.
"""
import functools
import math

import numpy as np
import scipy.linalg

from .basis import gauss_legendre
from .element import (interpolation_matrix, remove_rigid_motion, scalar_mass, shape_grad, simp, vector_dofs)
from .solve import K0_table


# ----------------------------------------------------------------------------- Kelly (Eq. 9)
def _edge_dn(p, side, t, hx, hy):
    """Normal-direction shape derivatives on one element side at edge parameters t.

    side 0: x = 0 (left), 1: x = hx (right), 2: y = 0 (bottom), 3: y = hy (top).  Returns the
    derivative along +x for sides 0/1 and along +y for sides 2/3 (a fixed global normal per edge)."""
    t = np.asarray(t, dtype=np.float64)
    one = np.ones_like(t)
    if side in (0, 1):
        _, Nx, _ = shape_grad(p, (-1.0 if side == 0 else 1.0) * one, t, hx, hy)
        return Nx
    _, _, Ny = shape_grad(p, t, (-1.0 if side == 2 else 1.0) * one, hx, hy)
    return Ny


@functools.lru_cache(maxsize=None)
def _edge_dn_rule(p, side, pF, hx, hy):
    """``_edge_dn`` at the (pF+1)-point Gauss nodes of an edge, with the weights (a pure function of
    its small integer arguments, kept once per combination)."""
    g, w = gauss_legendre(pF + 1)
    dn = _edge_dn(p, side, g, hx, hy)
    dn.setflags(write=False)
    return dn, w


def kelly(mesh, u):
    """Gamma^a_i = sum over faces F of element i of c_F * integral_F [du/dn]^2 ds (Eq. 9).

    [du/dn] is the jump of the normal derivative of both displacement components across an
    interior edge; c_F = h_F / (2 p_F) with h_F the element diagonal and p_F the larger order of
    the two elements (Sec. 3.2.1).  The edge integral uses a (p_F+1)-point Gauss rule, exact for the
    squared jump (degree <= 2 p_F).  Boundary edges contribute nothing (no jump is defined there).
    Each interior edge adds its term to both of its elements.  No square root is taken: Eq. 9 has
    none and the ranking does not depend on it.
    """
    nx, ny = mesh.nelx, mesh.nely
    hF = math.sqrt(mesh.hx ** 2 + mesh.hy ** 2)
    ue = [mesh.gather(e, u) for e in range(mesh.nel)]
    gam = np.zeros(mesh.nel)

    def jump_integral(eA, sideA, eB, sideB, length):
        pA, pB = int(mesh.p[eA]), int(mesh.p[eB])
        pF = max(pA, pB)
        dA, w = _edge_dn_rule(pA, sideA, pF, mesh.hx, mesh.hy)
        dB, _ = _edge_dn_rule(pB, sideB, pF, mesh.hx, mesh.hy)
        val = 0.0
        for c in range(2):
            jmp = dA.T @ ue[eA][c::2] - dB.T @ ue[eB][c::2]
            val += np.sum(w * jmp * jmp) * 0.5 * length
        return hF / (2.0 * pF) * val

    for iy in range(ny):
        for ix in range(1, nx):
            L, R = iy * nx + ix - 1, iy * nx + ix
            c = jump_integral(L, 1, R, 0, mesh.hy)
            gam[L] += c
            gam[R] += c
    for iy in range(1, ny):
        for ix in range(nx):
            B, T = (iy - 1) * nx + ix, iy * nx + ix
            c = jump_integral(B, 3, T, 2, mesh.hx)
            gam[B] += c
            gam[T] += c
    return gam


# ----------------------------------------------------------------------------- density indicator
def density_bands(rho_min, rho_max, cycle, alpha=0.2, beta=0.8):
    """(rho_avg, r_l, r_u, c_l, c_u) of Eqs. 10-13 with rho_avg = (rho_max + rho_min)/2."""
    ravg = 0.5 * (rho_max + rho_min)
    fac = ravg * math.exp(-beta * (cycle - 1))
    return (ravg, rho_min + (1.0 - alpha) * fac, rho_max - (1.0 - alpha) * fac,
            rho_min + alpha * fac, rho_max - alpha * fac)


def gamma_d(mesh, rho, cycle=1, alpha=0.2, beta=0.8):
    """Density indicator Gamma^d_k (Sec. 3.2.2).

    For each density cell j of element k (here: the d_k^2 subcells), the first matching case of
    the paper's list adds its contribution, in cell order:
      r_l <= rho <= rho_avg : + (rho - r_l) / n
      rho_avg < rho <= r_u  : + (r_u - rho) / n
      rho <= c_l            : - (c_l - rho) / n
      rho >= c_u            : - (rho - c_u) / n
    with n = n_{d,k} the element's cell count.  Garbled symbols read as: "r_avg" -> rho_avg and
    "rho_u" -> r_u.  rho_min / rho_max are global over all cells; cycle is k~ (from 1).
    """
    ravg, rl, ru, cl, cu = density_bands(float(rho.min()), float(rho.max()), cycle, alpha, beta)
    out = np.zeros(mesh.nel)
    for k in range(mesh.nel):
        cells = rho[mesh.design_off[k]:mesh.design_off[k + 1]]
        n = float(len(cells))
        g = 0.0
        for r in cells:
            r = float(r)
            if rl <= r <= ravg:
                g += (r - rl) / n
            elif ravg < r <= ru:
                g += (ru - r) / n
            elif r <= cl:
                g -= (cl - r) / n
            elif r >= cu:
                g -= (r - cu) / n
        out[k] = g
    return out


# ----------------------------------------------------------------------------- QR error (Eq. 14)
def qr_fixed_local_dofs(p):
    """The 3 DOFs pinned in the order-p element problem: u_x, u_y at the bottom-left vertex and
    u_y at the bottom-right vertex (local node p)."""
    return np.array([0, 1, 2 * p + 1])


@functools.lru_cache(maxsize=None)
def qr_load_transfer(p):
    """Matrix R with f^(p+1) = R f^(p) (reading of Sec. 3.2.3's load transfer).

    The paper forms f^(p+1) "by integrating the product of the interpolated original load field
    and the refined shape functions".  Reading: the load field is the order-p field g whose
    consistent nodal loads are f^(p) (M^(p) c = f^(p), g = sum_k c_k N_k^(p)); then
    f^(p+1)_j = integral N_j^(p+1) g = (M^(p+1,p) M^(p)^-1 f^(p))_j.  This transfer is work-consistent
    (f^(p+1) . T v = f^(p) . v for every order-p field v), so 0 <= eps < 1.
    """
    Mp = vector_dofs(scalar_mass(p, p))
    M1p = vector_dofs(scalar_mass(p + 1, p))
    R = M1p @ np.linalg.inv(Mp)
    R.setflags(write=False)
    return R


@functools.lru_cache(maxsize=None)
def _prolong_vec(p):
    """Vector-DOF nodal interpolation from order p to p + 1 (kept once per order)."""
    T = vector_dofs(interpolation_matrix(p, p + 1))
    T.setflags(write=False)
    return T


def qr_error_element(p, d, rho_e, ue, E0, Emin, nu, q, hx=1.0, hy=1.0, fixed=None):
    """eps^QR = 1 - J^(p) / J^(p+1) for one element (Eq. 14).

    K^(p), K^(p+1): composite stiffness of the same subcells at orders p and p+1.
    f^(p) = K^(p) u^(p) (element internal load); f^(p+1) by ``qr_load_transfer``.
    u^(p+1): 3 DOFs copied from the interpolant T u^(p) (bottom-left u_x, u_y; bottom-right u_y),
    the rest from K^(p+1) u = f^(p+1) by dense Cholesky.  J = 1/2 u^T K u for both orders.
    When J^(p+1) = 0 (rigid or zero u) eps is 0.  ``fixed`` overrides the three pinned local DOFs of
    the order-(p+1) problem (any set that removes the rigid modes gives the same eps).  eps does not
    change when a rigid motion is added to u^(p) (f^(p), both energies and the relative solution are
    unchanged), so the element's rigid motion is removed first to keep the energies free of
    cancellation.
    """
    ue = remove_rigid_motion(p, np.asarray(ue, dtype=np.float64), hx, hy)
    E = simp(rho_e, E0, Emin, q)
    Kp = np.tensordot(E, K0_table(p, d, nu, hx, hy), axes=(0, 0))
    K1 = np.tensordot(E, K0_table(p + 1, d, nu, hx, hy), axes=(0, 0))
    fp = Kp @ ue
    f1 = qr_load_transfer(p) @ fp
    T = _prolong_vec(p)
    fx = qr_fixed_local_dofs(p + 1) if fixed is None else np.asarray(fixed)
    fr = np.setdiff1d(np.arange(K1.shape[0]), fx)
    u1 = np.zeros(K1.shape[0])
    u1[fx] = (T @ ue)[fx]
    rhs = f1[fr] - K1[np.ix_(fr, fx)] @ u1[fx]
    u1[fr] = scipy.linalg.cho_solve(scipy.linalg.cho_factor(K1[np.ix_(fr, fr)], lower=True), rhs)
    Jp = 0.5 * ue @ (Kp @ ue)
    J1 = 0.5 * u1 @ (K1 @ u1)
    return 0.0 if J1 == 0.0 else 1.0 - Jp / J1


def qr_error(mesh, u, rho, E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    """eps^QR for every element (Sec. 3.2.3)."""
    out = np.zeros(mesh.nel)
    for e in range(mesh.nel):
        r = rho[mesh.design_off[e]:mesh.design_off[e + 1]]
        out[e] = qr_error_element(int(mesh.p[e]), int(mesh.d[e]), r, mesh.gather(e, u),
                                  E0, Emin, nu, q, mesh.hx, mesh.hy)
    return out


# ----------------------------------------------------------------------------- map update
def smooth_p(p, nelx, nely, max_jump=2):
    """Raise lower orders until edge-neighbour orders differ by at most ``max_jump``
    (Sec. 3.3 step 3(c)iv).  Repeated sweeps p_k <- max(p_k, max_j p_j - max_jump) to the fixed
    point: the least fixed point above p, independent of sweep order, reached within the paper's
    (p_max - p_min - 2) sweeps."""
    P = np.asarray(p, dtype=np.int64).reshape(nely, nelx).copy()
    while True:
        nb = np.full_like(P, -(1 << 40))      # no neighbour
        nb[:, 1:] = np.maximum(nb[:, 1:], P[:, :-1])
        nb[:, :-1] = np.maximum(nb[:, :-1], P[:, 1:])
        nb[1:, :] = np.maximum(nb[1:, :], P[:-1, :])
        nb[:-1, :] = np.maximum(nb[:-1, :], P[1:, :])
        Pn = np.maximum(P, nb - max_jump)
        if np.array_equal(Pn, P):
            return P.ravel()
        P = Pn


def design_count_for_order(p, d_max=64):
    """Per-axis design count after the d update (Sec. 3.3 step 3(c)v, B): the element-level
    bound N_d = n_e - 3 = 2(p+1)^2 - 3 (rigid modes removed), capped at d_max (= 64, Table 1),
    realised as the largest square grid d x d with d^2 <= min(N_d, d_max)."""
    nd = min(2 * (p + 1) ** 2 - 3, d_max)
    return math.isqrt(nd)


def map_update(nelx, nely, p, gamma_a, gamma_d_vals, eps_qr, frac_a_refine=0.10, frac_a_coarsen=0.05,
               alpha_d_refine=1.0, alpha_d_coarsen=1.0, alpha_qr=0.9, p_max=5, d_max=64):
    """dp map update of Sec. 3.3, steps 2-4.  Returns (p_new, d_new, theta).

    Step 2 (analysis): sort Gamma^a ascending (ties by element index); the first
    floor(frac_a_coarsen * nel) get theta = -1 and p - 1 (not below 1), the last
    floor(frac_a_refine * nel) get theta = +1 and p + 1.  (The paper's alpha^d_c in this step is
    read as alpha^a_c.)
    Step 3 (density): alpha^d fractions are taken of the elements with Gamma^d < 0 (coarsening,
    most negative first) and Gamma^d > 0 (refining, most positive first), so alpha = 1 coarsens
    every element with Gamma^d < 0 and refines every one with Gamma^d > 0 (Sec. 5).  Coarsening:
    p = 1 -> theta = -2; p > 1 and theta = 0 -> p - 1.  Refining: theta in {0, -1} -> p + 1.
    Then the p-jump smoothing and the d update (theta = -2 -> d = 1, else ``design_count_for_order``).
    Step 4 (QR): p + 1 where eps^QR > alpha_QR; eps is that of the solved (input) orders.
    Every increase is capped at p_max.
    """
    nel = nelx * nely
    p = np.asarray(p, dtype=np.int64).copy()
    theta = np.zeros(nel, dtype=np.int64)
    order = np.argsort(np.asarray(gamma_a), kind="stable")
    nc = int(math.floor(frac_a_coarsen * nel))
    nr = int(math.floor(frac_a_refine * nel))
    for k in order[:nc]:
        theta[k] = -1
        p[k] = max(p[k] - 1, 1)
    for k in order[nel - nr:]:
        theta[k] = 1
        p[k] = min(p[k] + 1, p_max)

    gd = np.asarray(gamma_d_vals)
    order = np.argsort(gd, kind="stable")
    neg = [k for k in order if gd[k] < 0]
    pos = [k for k in order if gd[k] > 0]
    coarsen = set(neg[:int(math.floor(alpha_d_coarsen * len(neg)))])
    refine = set(pos[len(pos) - int(math.floor(alpha_d_refine * len(pos))):])
    for k in range(nel):
        if k in coarsen:
            if p[k] == 1:
                theta[k] = -2
            elif theta[k] == 0:
                p[k] -= 1
        if k in refine and theta[k] in (0, -1):
            p[k] = min(p[k] + 1, p_max)

    p = smooth_p(p, nelx, nely)
    d = np.array([1 if theta[k] == -2 else design_count_for_order(int(p[k]), d_max) for k in range(nel)],
                 dtype=np.int64)
    eps = np.asarray(eps_qr)
    for k in range(nel):
        if eps[k] > alpha_qr:
            p[k] = min(p[k] + 1, p_max)
    return p, d, theta
