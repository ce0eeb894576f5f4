"""The P2 density filter of Sec. 2.1 (Eqs. 4-5) and its adjoint (test infrastructure only).

Eq. 4: rho~_i = sum_j H_ij rho^_j / sum_j H_ij over the density cells j whose centres lie within R
of point i, with H_ij = R - dist(i, j) (Eq. 5).  Reading for the composite integration used here
(each element's d x d subcells are both its density cells and its constant-density integration
cells): the filter is evaluated at the subcell centres, from the design values of all subcells of
the mesh (across element edges) whose centres lie within R, without volume weights (as printed);
R = 0.3 h (Sec. 4.1).  The physical densities rho~ then enter K_e = sum_s E(rho~_s) K0[s].

The adjoint (chain rule of the sensitivities): dJ/drho_t = sum_s H_st / W_s dJ/drho~_s with
W_s = sum_k H_sk.  The neighbour search is scipy's k-d tree (a library primitive); the weights
and sums follow Eqs. 4-5 directly.
"""
import numpy as np
import scipy.sparse
import scipy.spatial


def subcell_centres(mesh):
    """Centres (x, y) of every subcell, packed like rho (element e, subcell s = j d + i)."""
    xy = np.zeros((mesh.design_len, 2))
    for e in range(mesh.nel):
        ex, ey, d = e % mesh.nelx, e // mesh.nelx, int(mesh.d[e])
        off = mesh.design_off[e]
        for j in range(d):
            for i in range(d):
                xy[off + j * d + i] = ((ex + (i + 0.5) / d) * mesh.hx, (ey + (j + 0.5) / d) * mesh.hy)
    return xy


def filter_matrix(mesh, R):
    """Sparse H with H_st = R - dist(s, t) for subcell centres closer than R (Eq. 5), s = t included."""
    c = subcell_centres(mesh)
    pairs = scipy.spatial.cKDTree(c).query_pairs(R, output_type="ndarray")
    dist = np.linalg.norm(c[pairs[:, 0]] - c[pairs[:, 1]], axis=1)
    keep = dist < R
    a, b, w = pairs[keep, 0], pairs[keep, 1], R - dist[keep]
    n = mesh.design_len
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([w, w, np.full(n, R)])
    return scipy.sparse.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def density_filter(mesh, rho, R):
    """rho~ = (H rho) / (H 1) (Eq. 4 at the subcell centres)."""
    H = filter_matrix(mesh, R)
    return (H @ rho) / np.asarray(H.sum(axis=1)).ravel()


def density_filter_adjoint(mesh, g, R):
    """H^T (g / W): the gradient with respect to the design values of a function whose gradient
    with respect to the filtered densities is g."""
    H = filter_matrix(mesh, R)
    W = np.asarray(H.sum(axis=1)).ravel()
    return H.T @ (g / W)
