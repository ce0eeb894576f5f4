"""Pins for oracle/mesh.py and oracle/solve.py: the paper's DOF counts, the patch test across
p-jumps, rigid modes of the assembled operator, solver agreement, and an independent assembly of
the bilinear cantilever in the published 88-line numbering."""
import json
import os

import numpy as np
import pytest
import scipy.sparse

from oracle.element import homogeneous_stiffness
from oracle.mesh import DPMesh, cantilever_bc, mbb_bc
from oracle.solve import assemble, element_matrices, pcg, solve_direct, free_dofs
from oracle.sensitivity import compliance

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_dof_counts():
    pins = json.load(open(os.path.join(GOLD, "paper_pins.json")))
    for key, p, d in (("dp_cycle1_40x20_q2_d16", 2, 4), ("uniform_mto_40x20_q5_d64", 5, 8)):
        m = DPMesh(40, 20, np.full(800, p), np.full(800, d))
        fixed, _ = cantilever_bc(m)
        assert m.ndof - len(fixed) == pins[key]["free_dofs"]
        assert m.design_len == pins[key]["design_points"]
    r = pins["reference_mesh_design_resolution"]
    assert r["mto_nelx"] * r["d_axis"] == r["nelx"] and r["mto_nely"] * r["d_axis"] == r["nely"]


def test_large_mbb_dof_count():
    m = DPMesh(1024, 512, np.full(1024 * 512, 3, dtype=np.int64), np.full(1024 * 512, 8, dtype=np.int64))
    assert m.ndof == 9_446_402
    assert m.design_len == 33_554_432


def mixed_mesh():
    # orders with jumps of 1 and 2 across edges
    p = np.array([[1, 2, 3, 3],
                  [2, 3, 1, 2],
                  [3, 3, 2, 1]]).ravel()
    return DPMesh(4, 3, p, np.full(12, 2))


def test_numbering_is_consistent():
    m = mixed_mesh()
    xy = m.node_xy()
    # every global node is referenced by some element with weight 1 (owned) and positions are distinct
    seen = np.zeros(m.n_nodes, bool)
    for e in range(m.nel):
        for lst in m.element_node_map(e):
            if len(lst) == 1:
                seen[lst[0][0]] = True
    assert seen.all()
    assert len(np.unique(np.round(xy, 12), axis=0)) == m.n_nodes
    # vertices row-major
    for iy in range(m.nely + 1):
        for ix in range(m.nelx + 1):
            np.testing.assert_allclose(xy[m.vertex(ix, iy)], (ix, iy), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_uniform_node_count(p):
    m = DPMesh(5, 3, np.full(15, p), np.ones(15))
    assert m.n_nodes == (5 * p + 1) * (3 * p + 1)


def test_patch_test_mixed_orders():
    """Uniform modulus, linear displacement on the boundary: the interior reproduces it exactly,
    across p-jumps of 1 and 2 (minimum-rule constraints)."""
    m = mixed_mesh()
    rho = np.ones(m.design_len)
    K = assemble(m, element_matrices(m, rho, 1.0, 1e-9, 0.3, 3.0))
    xy = m.node_xy()
    ulin = np.zeros(m.ndof)
    ulin[0::2] = 1e-3 * xy[:, 0] - 2e-4 * xy[:, 1] + 0.3
    ulin[1::2] = 5e-4 * xy[:, 0] + 7e-4 * xy[:, 1] - 0.1
    bnodes = np.unique(np.concatenate([m.side_nodes(s) for s in range(4)]))
    bd = np.sort(np.concatenate([2 * bnodes, 2 * bnodes + 1]))
    fr = free_dofs(m.ndof, bd)
    Kd = K.toarray()
    u = ulin.copy()
    u[fr] = np.linalg.solve(Kd[np.ix_(fr, fr)], -Kd[np.ix_(fr, bd)] @ ulin[bd])
    np.testing.assert_allclose(u, ulin, atol=1e-13)
    # interior equilibrium of the linear field: K u vanishes at free DOFs
    assert np.abs((K @ ulin)[fr]).max() < 1e-13


def test_unsupported_operator_has_three_zero_modes():
    m = mixed_mesh()
    rng = np.random.default_rng(0)
    K = assemble(m, element_matrices(m, rng.uniform(0.2, 1, m.design_len), 1.0, 1e-9, 0.3, 3.0)).toarray()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 3


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_solvers_agree_tiny(p):
    m = DPMesh(4, 2, np.full(8, p), np.full(8, 2))
    rng = np.random.default_rng(p)
    rho = rng.uniform(0.01, 1, m.design_len)
    fixed, f = cantilever_bc(m)
    K = assemble(m, element_matrices(m, rho, 1.0, 1e-9, 0.3, 3.0))
    u = solve_direct(K, f, fixed)
    fr = free_dofs(m.ndof, fixed)
    ub = np.zeros(m.ndof)
    ub[fr] = np.linalg.solve(K.toarray()[np.ix_(fr, fr)], f[fr])     # brute-force LU
    np.testing.assert_allclose(u, ub, rtol=0, atol=1e-10 * np.abs(ub).max())   # kappa ~ 1e6 here
    up, it, rr = pcg(K, f, fixed, rtol=1e-13)
    np.testing.assert_allclose(up, ub, rtol=0, atol=1e-9 * np.abs(ub).max())
    C = compliance(f, u)
    assert abs(C - u @ (K @ u)) < 1e-10 * abs(C)


def test_splu_branch_matches_pcg():
    m = DPMesh(40, 20, np.full(800, 2), np.full(800, 2))          # > 4000 free DOFs: sparse LU branch
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.1, 1, m.design_len)
    fixed, f = mbb_bc(m)
    K = assemble(m, element_matrices(m, rho, 1.0, 1e-9, 0.3, 3.0))
    assert m.ndof - len(fixed) > 4000
    u = solve_direct(K, f, fixed)
    up, _, _ = pcg(K, f, fixed, rtol=1e-13)
    np.testing.assert_allclose(up, u, atol=1e-9 * np.abs(u).max())


def test_compliance_scales_inversely_with_modulus():
    m = DPMesh(6, 4, np.full(24, 2), np.full(24, 2))
    rho = np.full(m.design_len, 0.6)
    fixed, f = cantilever_bc(m)
    C1 = compliance(f, solve_direct(assemble(m, element_matrices(m, rho, 1.0, 1e-9, 0.3, 3.0)), f, fixed))
    C2 = compliance(f, solve_direct(assemble(m, element_matrices(m, rho, 4.0, 4e-9, 0.3, 3.0)), f, fixed))
    assert abs(C1 / C2 - 4.0) < 1e-12


def test_bilinear_cantilever_independent_assembly():
    """p = 1, one density per element: the compliance equals that of an independent assembly with
    the published closed-form element in the 88-line code's column-major, top-down numbering."""
    nelx, nely, nu = 12, 6, 0.3
    rng = np.random.default_rng(11)
    x = rng.uniform(0.1, 1, nelx * nely)
    m = DPMesh(nelx, nely, np.ones(nelx * nely), np.ones(nelx * nely))
    fixed, f = cantilever_bc(m)
    u = solve_direct(assemble(m, element_matrices(m, x, 1.0, 1e-9, nu, 3.0)), f, fixed)
    C = compliance(f, u)

    from tests.test_oracle_element import top88_KE
    KE = top88_KE(nu)
    nn = (nelx + 1) * (nely + 1)
    rows, cols, vals = [], [], []
    for ey in range(nely):
        for ex in range(nelx):
            # column-major node ids counted from the top: n(ix, iy_up) = ix*(nely+1) + (nely - iy_up)
            node = lambda ix, iy: ix * (nely + 1) + (nely - iy)
            ns = [node(ex, ey), node(ex + 1, ey), node(ex + 1, ey + 1), node(ex, ey + 1)]
            ed = np.array([[2 * n, 2 * n + 1] for n in ns]).ravel()
            Ee = 1e-9 + x[ey * nelx + ex] ** 3 * (1 - 1e-9)
            rows.append(np.repeat(ed, 8)); cols.append(np.tile(ed, 8)); vals.append((Ee * KE).ravel())
    K = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(2 * nn, 2 * nn)).tocsr()
    fx = np.array([[2 * (0 * (nely + 1) + r), 2 * r + 1] for r in range(nely + 1)]).ravel()
    F = np.zeros(2 * nn)
    F[2 * (nelx * (nely + 1) + nely // 2) + 1] = -1.0
    fr = np.setdiff1d(np.arange(2 * nn), fx)
    U = np.zeros(2 * nn)
    U[fr] = scipy.sparse.linalg.spsolve(K[fr][:, fr].tocsc(), F[fr])
    assert abs(F @ U - C) < 1e-11 * abs(C)
