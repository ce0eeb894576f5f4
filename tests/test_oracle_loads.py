"""Pins for the oracle's consistent edge loads (the distributed-load cantilever of Sec. 4.1,
Fig. 6a): closed-form totals and moments, the textbook nodal values of linear (h/2, h) and quadratic
(Simpson h/6, 4h/6) edges, and work consistency with polynomial fields on mixed-order sides."""
import numpy as np
import pytest

from oracle.mesh import DPMesh, distributed_cantilever_bc, side_load, side_edges


def mesh(p, nelx=6, nely=3):
    return DPMesh(nelx, nely, np.asarray(p).ravel() if np.ndim(p) else np.full(nelx * nely, p),
                  np.full(nelx * nely, 2))


def test_linear_edges_textbook_values():
    m = mesh(1)
    f = side_load(m, 3, 1, -2.0)
    top = [m.vertex(ix, m.nely) for ix in range(m.nelx + 1)]
    want = np.full(m.nelx + 1, -2.0)
    want[0] = want[-1] = -1.0
    np.testing.assert_allclose(f[2 * np.array(top) + 1], want, rtol=0, atol=1e-15)
    assert np.count_nonzero(f) == m.nelx + 1


def test_quadratic_edges_simpson_values():
    m = mesh(2)
    f = side_load(m, 3, 0, 6.0)
    for nodes, pE, length in side_edges(m, 3):
        assert pE == 2
        # the mid-edge node belongs to this edge only: 4/6 of t h
        assert abs(f[2 * nodes[1]] - 4.0) < 1e-14
    # an interior vertex takes 1/6 from each neighbouring edge
    assert abs(f[2 * m.vertex(2, m.nely)] - 2.0) < 1e-14
    assert abs(f[2 * m.vertex(0, m.nely)] - 1.0) < 1e-14


# orders along the top row with jumps of 1 and 2; the rest of the mesh is arbitrary
P_MIXED = np.array([[2, 3, 1, 3, 5, 4],
                    [1, 2, 3, 3, 4, 5],
                    [3, 1, 2, 4, 5, 3]])


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_totals_and_work_consistency_mixed_orders(side):
    m = DPMesh(6, 3, P_MIXED.ravel(), np.full(18, 2))
    t = -0.75
    f = side_load(m, side, 1, t)
    xy = m.node_xy()
    length = m.nely * m.hy if side in (0, 1) else m.nelx * m.hx
    s = xy[:, 1] if side in (0, 1) else xy[:, 0]            # coordinate along the side
    uy = lambda g: np.repeat(g, 2) * np.tile([0.0, 1.0], m.n_nodes)
    # total load: t * length; first moment: t * length^2 / 2 (linear fields are in every order)
    assert abs(f @ uy(np.ones(m.n_nodes)) - t * length) < 1e-13
    assert abs(f @ uy(s) - t * length ** 2 / 2) < 1e-12
    # a quadratic field lies in the trace space of edges of order >= 2: checked on the sides
    # whose edges all have order >= 2 (the right side here)
    orders = [pE for _, pE, _ in side_edges(m, side)]
    if min(orders) >= 2:
        assert abs(f @ uy(s ** 2) - t * length ** 3 / 3) < 1e-11


def test_distributed_cantilever_total_load():
    m = DPMesh(40, 20, np.full(800, 2), np.full(800, 4))
    fixed, f = distributed_cantilever_bc(m)
    assert abs(f.sum() + 1.0) < 1e-13                      # total downward load 1 (0.5 N/L over 2L)
    assert np.all(f[0::2] == 0.0)
    # 2 * 40 + 1 top nodes carry load
    assert np.count_nonzero(f) == 2 * 40 + 1
