"""Element-level matrices of the MTO element (test infrastructure only).

Local numbering of a Q_p element: node (a, b), a the x-index and b the y-index in 0..p on the GLL
grid, node id n = b*(p+1) + a; local DOF 2n + c with c = 0 (u_x) or 1 (u_y).  Reference square
[-1, 1]^2 maps affinely onto [0, hx] x [0, hy].  A d x d element carries d^2 constant-density
subcells (the density cells of Sec. 2.1), subcell s = j*d + i covering
[i/d, (i+1)/d] x [j/d, (j+1)/d] of the element.
"""
import numpy as np

from .basis import gauss_legendre, gll_nodes, lagrange, lagrange_deriv


def D0(nu):
    """Plane-stress constitutive matrix normalised by Young's modulus (D_0 of Eq. 3).

    The paper states isotropic linear elasticity with nu = 0.3 (Sec. 4.1); plane stress is the
    reading for these 2D problems.  Voigt order (eps_xx, eps_yy, gamma_xy).
    """
    return np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]]) / (1.0 - nu * nu)


def simp(rho, E0, Emin, q):
    """SIMP modulus E(rho) = Emin + rho^q (E0 - Emin) (Eq. 3)."""
    rho = np.asarray(rho, dtype=np.float64)
    return Emin + rho ** q * (E0 - Emin)


def simp_deriv(rho, E0, Emin, q):
    """dE/drho = q rho^(q-1) (E0 - Emin), the derivative of Eq. 3."""
    rho = np.asarray(rho, dtype=np.float64)
    return q * rho ** (q - 1.0) * (E0 - Emin)


def shape_grad(p, xi, eta, hx=1.0, hy=1.0):
    """Shape values N[n, m] and physical gradients dNdx, dNdy [n, m] at reference points (xi_m, eta_m)."""
    z = gll_nodes(p)
    Lx, Ly = lagrange(z, xi), lagrange(z, eta)
    Dx, Dy = lagrange_deriv(z, xi), lagrange_deriv(z, eta)
    n1 = p + 1
    N = np.zeros((n1 * n1, len(xi)))
    Nx = np.zeros_like(N)
    Ny = np.zeros_like(N)
    for b in range(n1):
        for a in range(n1):
            n = b * n1 + a
            N[n] = Lx[a] * Ly[b]
            Nx[n] = Dx[a] * Ly[b] * (2.0 / hx)
            Ny[n] = Lx[a] * Dy[b] * (2.0 / hy)
    return N, Nx, Ny


def B_matrix(Nx, Ny, m):
    """Strain-displacement matrix B (3 x n_e) at point m (the B of Eq. 2)."""
    nn = Nx.shape[0]
    B = np.zeros((3, 2 * nn))
    B[0, 0::2] = Nx[:, m]
    B[1, 1::2] = Ny[:, m]
    B[2, 0::2] = Ny[:, m]
    B[2, 1::2] = Nx[:, m]
    return B


def _rule_on_box(nq, x0, x1, y0, y1):
    """Tensor Gauss rule with nq points per axis on the reference box [x0, x1] x [y0, y1]."""
    g, w = gauss_legendre(nq)
    xs = 0.5 * (x0 + x1) + 0.5 * (x1 - x0) * g
    ys = 0.5 * (y0 + y1) + 0.5 * (y1 - y0) * g
    XI, ETA = np.meshgrid(xs, ys, indexing="xy")
    W = np.outer(w, w) * 0.25 * (x1 - x0) * (y1 - y0)
    return XI.ravel(), ETA.ravel(), W.ravel()


def subcell_stiffness(p, d, nu, hx=1.0, hy=1.0):
    """K0[s] = integral over subcell s of B^T D0 B (unit modulus), shape (d*d, n_e, n_e).

    Composite integration (App. B): density is constant per subcell, so the element stiffness is
    the modulus-weighted sum of these subcell matrices.  On an affine square the integrand is a
    polynomial of degree <= 2p per axis, so the (p+1) x (p+1) Gauss rule mapped to the subcell is
    exact (Table B gives 2x2 for p = 1, d = 1).
    """
    D = D0(nu)
    n_e = 2 * (p + 1) ** 2
    K0 = np.zeros((d * d, n_e, n_e))
    jac = 0.25 * hx * hy
    for j in range(d):
        for i in range(d):
            s = j * d + i
            xi, eta, w = _rule_on_box(p + 1, -1 + 2.0 * i / d, -1 + 2.0 * (i + 1) / d,
                                      -1 + 2.0 * j / d, -1 + 2.0 * (j + 1) / d)
            _, Nx, Ny = shape_grad(p, xi, eta, hx, hy)
            for m in range(len(w)):
                B = B_matrix(Nx, Ny, m)
                K0[s] += B.T @ D @ B * (w[m] * jac)
    return K0


def homogeneous_stiffness(p, nu, hx=1.0, hy=1.0, nq=None):
    """Whole-element stiffness with unit modulus from one (p+1)^2 (or nq^2) Gauss rule.

    Independent of the subcell split: used to check sum_s K0[s] == K_hom.
    """
    nq = p + 1 if nq is None else nq
    D = D0(nu)
    xi, eta, w = _rule_on_box(nq, -1.0, 1.0, -1.0, 1.0)
    _, Nx, Ny = shape_grad(p, xi, eta, hx, hy)
    n_e = 2 * (p + 1) ** 2
    K = np.zeros((n_e, n_e))
    for m in range(len(w)):
        B = B_matrix(Nx, Ny, m)
        K += B.T @ D @ B * (w[m] * 0.25 * hx * hy)
    return K


def element_stiffness(K0, E):
    """K_e = sum_s E_s K0[s] (Eq. 2 with Eq. 3 under composite integration, App. B)."""
    return np.tensordot(np.asarray(E, dtype=np.float64), K0, axes=(0, 0))


def scalar_mass(p_row, p_col, hx=1.0, hy=1.0):
    """M[j, k] = integral over the element of N_j^(p_row) N_k^(p_col) (one displacement component).

    Integrand degree p_row + p_col per axis; a (max(p_row, p_col) + 1)-point Gauss rule is exact.
    """
    nq = max(p_row, p_col) + 1
    xi, eta, w = _rule_on_box(nq, -1.0, 1.0, -1.0, 1.0)
    Nr, _, _ = shape_grad(p_row, xi, eta, hx, hy)
    Nc, _, _ = shape_grad(p_col, xi, eta, hx, hy)
    return (Nr * (w * 0.25 * hx * hy)) @ Nc.T


def interpolation_matrix(p_from, p_to):
    """T[j, k] = N_k^(p_from)(x_j^(p_to)): nodal interpolation of an order-p_from field onto the
    GLL nodes of order p_to, per displacement component (scalar, (p_to+1)^2 x (p_from+1)^2).

    For p_to >= p_from this is exact prolongation: Q_p_from is contained in Q_p_to.
    """
    zt = gll_nodes(p_to)
    zf = gll_nodes(p_from)
    L = lagrange(zf, zt)  # L[k, j] = l_k(zt_j)
    nt, nf = p_to + 1, p_from + 1
    T = np.zeros((nt * nt, nf * nf))
    for bj in range(nt):
        for aj in range(nt):
            for bk in range(nf):
                for ak in range(nf):
                    T[bj * nt + aj, bk * nf + ak] = L[ak, aj] * L[bk, bj]
    return T


def vector_dofs(S):
    """Expand a scalar (per-node) operator to the interleaved 2-component DOF layout."""
    r, c = S.shape
    V = np.zeros((2 * r, 2 * c))
    V[0::2, 0::2] = S
    V[1::2, 1::2] = S
    return V


def remove_rigid_motion(p, ue, hx=1.0, hy=1.0):
    """u_e minus its least-squares rigid motion (translation and infinitesimal rotation).

    Every K0_s annihilates rigid motions, so u^T K0_s u, K_e u and the QR energies are unchanged
    in exact arithmetic; removing the (often dominant) rigid part first avoids the cancellation
    that otherwise costs digits when an element moves far but strains little."""
    xy = node_coords(p, hx, hy)
    xc = xy[:, 0] - xy[:, 0].mean()
    yc = xy[:, 1] - xy[:, 1].mean()
    ux, uy = ue[0::2], ue[1::2]
    om = np.sum(xc * uy - yc * ux) / np.sum(xc * xc + yc * yc)
    out = np.empty_like(ue)
    out[0::2] = ux - ux.mean() + om * yc
    out[1::2] = uy - uy.mean() - om * xc
    return out


def node_coords(p, hx=1.0, hy=1.0):
    """Physical coordinates (x, y) of the (p+1)^2 local nodes, in local node order."""
    z = gll_nodes(p)
    n1 = p + 1
    xy = np.zeros((n1 * n1, 2))
    for b in range(n1):
        for a in range(n1):
            xy[b * n1 + a] = ((z[a] + 1) * 0.5 * hx, (z[b] + 1) * 0.5 * hy)
    return xy
