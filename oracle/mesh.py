"""Structured dp-adaptive mesh: minimum-rule conformity and the canonical DOF numbering
(test infrastructure only).

The analysis mesh is a structured grid of nelx x nely quadrilaterals (Sec. 2.1) with a per-element
shape-function order p_e (Sec. 3.3, p_max = 5) and a per-element design resolution, here d_e x d_e
constant-density subcells.  The paper does not say how continuity is kept across an edge whose
two elements have different p; its implementation is deal.II hp (Acknowledgements), whose default
for FE_Q is the *minimum rule*, and the p-jump cap of 2 (Sec. 3.3, step 3(c)iv) limits the jumps.
Reading used here:

* an edge carries the trace space of order p_E = min(p_left, p_right) (boundary edge: its one
  element's p); its own unknowns are the p_E - 1 interior GLL nodes of that order;
* a higher-order element's nodes on that edge are constrained to interpolate the edge's trace;
* vertices are shared, cell-interior nodes are private.

Canonical global node numbering (an integer map, required bit-exact on both sides):
  1. vertices, row-major: node = iy*(nelx+1) + ix;
  2. interior nodes of horizontal edges, edge id iy*nelx + ix (iy = 0..nely), nodes left -> right;
  3. interior nodes of vertical edges, edge id iy*(nelx+1) + ix (iy = 0..nely-1), bottom -> top;
  4. cell-interior nodes, elements row-major, local (a, b) row-major with a fastest;
and DOF = 2*node + component.
"""
import numpy as np

from .basis import gauss_legendre, gll_nodes, lagrange


class DPMesh:
    """nelx x nely structured mesh with per-element order ``p`` and per-axis design count ``d``.

    Element e = ey*nelx + ex covers [ex*hx, (ex+1)*hx] x [ey*hy, (ey+1)*hy].
    """

    def __init__(self, nelx, nely, p, d, hx=1.0, hy=1.0):
        self.nelx, self.nely = int(nelx), int(nely)
        self.nel = self.nelx * self.nely
        self.hx, self.hy = float(hx), float(hy)
        self.p = np.asarray(p, dtype=np.int64).reshape(self.nel)
        self.d = np.asarray(d, dtype=np.int64).reshape(self.nel)
        if self.p.min() < 1 or self.d.min() < 1:
            raise ValueError("p >= 1 and d >= 1 required")
        nx, ny = self.nelx, self.nely
        P = self.p.reshape(ny, nx)
        # edge orders by the minimum rule
        pH = np.zeros((ny + 1, nx), dtype=np.int64)
        pH[0, :] = P[0, :]
        pH[ny, :] = P[ny - 1, :]
        pH[1:ny, :] = np.minimum(P[:-1, :], P[1:, :])
        pV = np.zeros((ny, nx + 1), dtype=np.int64)
        pV[:, 0] = P[:, 0]
        pV[:, nx] = P[:, nx - 1]
        pV[:, 1:nx] = np.minimum(P[:, :-1], P[:, 1:])
        self.pH, self.pV = pH.ravel(), pV.ravel()
        self.n_vert = (nx + 1) * (ny + 1)
        nH = self.pH - 1
        nV = self.pV - 1
        nI = (self.p - 1) ** 2
        self.h_base = self.n_vert + np.concatenate([[0], np.cumsum(nH)[:-1]])
        self.v_base = self.n_vert + nH.sum() + np.concatenate([[0], np.cumsum(nV)[:-1]])
        self.i_base = self.n_vert + nH.sum() + nV.sum() + np.concatenate([[0], np.cumsum(nI)[:-1]])
        self.n_nodes = int(self.n_vert + nH.sum() + nV.sum() + nI.sum())
        self.ndof = 2 * self.n_nodes
        S = self.d ** 2
        self.design_off = np.concatenate([[0], np.cumsum(S)])
        self.design_len = int(self.design_off[-1])

    # ---------------------------------------------------------------- nodes
    def vertex(self, ix, iy):
        return iy * (self.nelx + 1) + ix

    def _edge_nodes_h(self, ix, iy):
        """Global nodes of horizontal edge (ix, iy) in parameter order and their GLL positions."""
        hid = iy * self.nelx + ix
        pE = int(self.pH[hid])
        nodes = [self.vertex(ix, iy)] + [int(self.h_base[hid]) + k for k in range(pE - 1)] + [self.vertex(ix + 1, iy)]
        return nodes, pE

    def _edge_nodes_v(self, ix, iy):
        vid = iy * (self.nelx + 1) + ix
        pE = int(self.pV[vid])
        nodes = [self.vertex(ix, iy)] + [int(self.v_base[vid]) + k for k in range(pE - 1)] + [self.vertex(ix, iy + 1)]
        return nodes, pE

    def element_node_map(self, e):
        """For each local node of element e: a list of (global node, weight) pairs.

        A node on an edge of lower order p_E interpolates that edge's order-p_E trace:
        weight_k = l_k^(p_E)(t) at the node's GLL position t (minimum rule).
        """
        ex, ey = e % self.nelx, e // self.nelx
        p = int(self.p[e])
        z = gll_nodes(p)
        out = []
        for b in range(p + 1):
            for a in range(p + 1):
                if a in (0, p) and b in (0, p):
                    out.append([(self.vertex(ex + a // p, ey + b // p), 1.0)])
                elif b in (0, p):
                    nodes, pE = self._edge_nodes_h(ex, ey + b // p)
                    out.append(self._edge_weights(nodes, pE, p, a, z[a]))
                elif a in (0, p):
                    nodes, pE = self._edge_nodes_v(ex + a // p, ey)
                    out.append(self._edge_weights(nodes, pE, p, b, z[b]))
                else:
                    out.append([(int(self.i_base[e]) + (b - 1) * (p - 1) + (a - 1), 1.0)])
        return out

    @staticmethod
    def _edge_weights(nodes, pE, p, k, t):
        if pE == p:
            return [(nodes[k], 1.0)]
        w = lagrange(gll_nodes(pE), [t])[:, 0]
        return [(nodes[j], float(w[j])) for j in range(pE + 1)]

    def prolongation(self, e):
        """Dense P_e (n_e x m) and the m global DOFs it maps from: u_e = P_e u[G_e]."""
        nm = self.element_node_map(e)
        gnodes = sorted({g for lst in nm for g, _ in lst})
        col = {g: i for i, g in enumerate(gnodes)}
        n_e = 2 * len(nm)
        P = np.zeros((n_e, 2 * len(gnodes)))
        for ln, lst in enumerate(nm):
            for g, w in lst:
                P[2 * ln, 2 * col[g]] += w
                P[2 * ln + 1, 2 * col[g] + 1] += w
        G = np.empty(2 * len(gnodes), dtype=np.int64)
        G[0::2] = 2 * np.asarray(gnodes)
        G[1::2] = 2 * np.asarray(gnodes) + 1
        return P, G

    def is_conforming_simple(self, e):
        """True when every node of e maps to exactly one global node with weight 1."""
        return all(len(lst) == 1 for lst in self.element_node_map(e))

    def gather_index(self, e):
        """Global DOF index per local DOF for an element without constrained nodes."""
        nm = self.element_node_map(e)
        g = np.empty(2 * len(nm), dtype=np.int64)
        for ln, lst in enumerate(nm):
            assert len(lst) == 1 and lst[0][1] == 1.0
            g[2 * ln] = 2 * lst[0][0]
            g[2 * ln + 1] = 2 * lst[0][0] + 1
        return g

    def gather(self, e, u):
        P, G = self.prolongation(e)
        return P @ u[G]

    # ---------------------------------------------------------------- boundary sets
    def side_nodes(self, side):
        """Global nodes on one side of the domain: 0 = left (x=0), 1 = right, 2 = bottom (y=0), 3 = top."""
        nx, ny = self.nelx, self.nely
        nodes = []
        if side in (0, 1):
            ix = 0 if side == 0 else nx
            for iy in range(ny):
                en, _ = self._edge_nodes_v(ix, iy)
                nodes.extend(en[:-1])
            nodes.append(self.vertex(ix, ny))
        else:
            iy = 0 if side == 2 else ny
            for ix in range(nx):
                en, _ = self._edge_nodes_h(ix, iy)
                nodes.extend(en[:-1])
            nodes.append(self.vertex(nx, iy))
        return np.array(sorted(set(nodes)), dtype=np.int64)

    def node_xy(self):
        """Physical coordinates of every global node (vertices, edge nodes, interiors)."""
        xy = np.zeros((self.n_nodes, 2))
        for e in range(self.nel):
            ex, ey = e % self.nelx, e // self.nelx
            p = int(self.p[e])
            z = gll_nodes(p)
            nm = self.element_node_map(e)
            for b in range(p + 1):
                for a in range(p + 1):
                    lst = nm[b * (p + 1) + a]
                    if len(lst) == 1:
                        xy[lst[0][0]] = ((ex + (z[a] + 1) / 2) * self.hx, (ey + (z[b] + 1) / 2) * self.hy)
        return xy


def cantilever_bc(mesh):
    """Cantilever of Sec. 4.1 (Fig. 3a): left edge clamped, unit downward point load at the
    mid-height node of the right edge.  Returns (fixed DOFs, load vector)."""
    if mesh.nely % 2:
        raise ValueError("mid-right load needs an even nely (vertex node)")
    left = mesh.side_nodes(0)
    fixed = np.sort(np.concatenate([2 * left, 2 * left + 1]))
    f = np.zeros(mesh.ndof)
    f[2 * mesh.vertex(mesh.nelx, mesh.nely // 2) + 1] = -1.0
    return fixed, f


def mbb_bc(mesh):
    """MBB half-beam (textbook; not in the paper): u_x = 0 on the left edge (symmetry line),
    u_y = 0 at the bottom-right vertex, unit downward load at the top-left vertex."""
    left = mesh.side_nodes(0)
    fixed = np.sort(np.concatenate([2 * left, [2 * mesh.vertex(mesh.nelx, 0) + 1]]))
    f = np.zeros(mesh.ndof)
    f[2 * mesh.vertex(0, mesh.nely) + 1] = -1.0
    return fixed, f


def side_edges(mesh, side):
    """The boundary edges of one side in order (0 = left, 1 = right, 2 = bottom, 3 = top): a list of
    (global nodes in parameter order, edge order p_E, edge length)."""
    nx, ny = mesh.nelx, mesh.nely
    if side in (0, 1):
        ix = 0 if side == 0 else nx
        return [mesh._edge_nodes_v(ix, iy) + (mesh.hy,) for iy in range(ny)]
    iy = 0 if side == 2 else ny
    return [mesh._edge_nodes_h(ix, iy) + (mesh.hx,) for ix in range(nx)]


def side_load(mesh, side, comp, traction):
    """Consistent nodal loads of a uniform traction (force per unit length, component ``comp``)
    on one side of the domain: f_k = traction * integral over the side of N_k ds, summed over the
    boundary edges.  On an edge of order p_E the trace of N_k is the Lagrange polynomial l_k of
    the edge's GLL nodes; its integral is taken with a (p_E + 1)-point Gauss-Legendre rule (exact
    for degree p_E).  Returns the load vector [ndof]."""
    f = np.zeros(mesh.ndof)
    for nodes, pE, length in side_edges(mesh, side):
        g, w = gauss_legendre(pE + 1)
        L = lagrange(gll_nodes(pE), g)          # L[k, j] = l_k(g_j)
        for k, node in enumerate(nodes):
            f[2 * node + comp] += traction * 0.5 * length * float(L[k] @ w)
    return f


def distributed_cantilever_bc(mesh, total=1.0):
    """Cantilever with a distributed load (Sec. 4.1, Fig. 6a): left edge clamped, a uniform
    downward traction on the top edge.  The paper's F = 0.5 N/L on a 2L-wide top edge is a total
    load of 1 N; here the traction is -total / (nelx hx), so the total load is ``total``.
    Returns (fixed DOFs, load vector)."""
    left = mesh.side_nodes(0)
    fixed = np.sort(np.concatenate([2 * left, 2 * left + 1]))
    f = side_load(mesh, 3, 1, -total / (mesh.nelx * mesh.hx))
    return fixed, f
