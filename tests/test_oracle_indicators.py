"""Pins for oracle/indicators.py and oracle/oc.py."""
import json
import math
import os

import numpy as np
import pytest

from oracle.element import interpolation_matrix, node_coords, subcell_stiffness, vector_dofs, simp
from oracle.indicators import (density_bands, design_count_for_order, gamma_d, kelly, map_update,
                               qr_error, qr_error_element, qr_load_transfer, smooth_p)
from oracle.mesh import DPMesh, cantilever_bc
from oracle.oc import oc_update, subcell_areas
from oracle.solve import solve

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Kelly
def field_on_nodes(m, fx, fy):
    xy = m.node_xy()
    u = np.zeros(m.ndof)
    u[0::2] = fx(xy[:, 0], xy[:, 1])
    u[1::2] = fy(xy[:, 0], xy[:, 1])
    return u


def test_kelly_zero_for_linear_field():
    m = DPMesh(4, 3, np.array([1, 2, 3, 3, 2, 3, 1, 2, 3, 3, 2, 1]), np.full(12, 2))
    u = field_on_nodes(m, lambda x, y: 0.3 * x - 0.2 * y + 1, lambda x, y: 0.1 * x + 0.5 * y)
    assert np.abs(kelly(m, u)).max() < 1e-25


def test_kelly_zero_for_smooth_polynomial_within_order():
    # a global quadratic has continuous gradient: zero jumps on a uniform p = 2 mesh
    m = DPMesh(3, 2, np.full(6, 2), np.ones(6))
    u = field_on_nodes(m, lambda x, y: x * x - x * y, lambda x, y: y * y + 0.5 * x)
    assert np.abs(kelly(m, u)).max() < 1e-24


def test_kelly_hand_value_two_elements():
    """2 x 1 bilinear mesh, u_x = x on [0,1] and 2 - x on [1,2]: the x-derivative jumps by 2 across
    the shared edge of length 1, integral = 4, c_F = sqrt(2)/2, so each element gets 2 sqrt(2)."""
    m = DPMesh(2, 1, np.ones(2), np.ones(2))
    u = field_on_nodes(m, lambda x, y: np.where(x <= 1, x, 2 - x), lambda x, y: 0 * x)
    np.testing.assert_allclose(kelly(m, u), [2 * math.sqrt(2), 2 * math.sqrt(2)], rtol=1e-14)


def test_kelly_hand_value_mixed_orders():
    """Left element p = 1, right element p = 3 (edge order 1).  u_y = 0, u_x = x on the left and
    x + (x-1)^2 (x-2)... chosen as a field of the right element's order that vanishes to first
    order at the edge: u_x = x + a (x-1)^2 on [1,2].  Normal-derivative jump is 0 -> Gamma = 0; with
    u_x = x + b (x-1) on [1,2] the jump is b, integral b^2, c_F = sqrt(2)/(2*3)."""
    m = DPMesh(2, 1, np.array([1, 3]), np.ones(2))
    u = field_on_nodes(m, lambda x, y: np.where(x <= 1, x, x + 0.7 * (x - 1) ** 2), lambda x, y: 0 * x)
    assert np.abs(kelly(m, u)).max() < 1e-25
    b = 0.4
    u = field_on_nodes(m, lambda x, y: np.where(x <= 1, x, x + b * (x - 1)), lambda x, y: 0 * x)
    np.testing.assert_allclose(kelly(m, u), [b * b * math.sqrt(2) / 6] * 2, rtol=1e-13)


# ------------------------------------------------------------------ density indicator
def test_gamma_d_hand_cases():
    gold = json.load(open(os.path.join(GOLD, "gamma_d_hand_cases.json")))
    cases = gold["cases"]
    # element 0 holds the global extremes (rho_min = 0, rho_max = 1); the tested cells follow
    rows = [[0.0, 1.0, 0.0, 1.0]] + [c["cells"] for c in cases]
    m = DPMesh(len(rows), 1, np.ones(len(rows)), np.full(len(rows), 2))
    rho = np.concatenate(rows)
    g = gamma_d(m, rho, cycle=1)
    for k, c in enumerate(cases):
        assert abs(g[k + 1] - c["gamma_d"]) < 1e-15, c["why"]


def test_density_bands_cycle_dependence():
    ravg, rl, ru, cl, cu = density_bands(0.0, 1.0, 1)
    np.testing.assert_allclose([ravg, rl, ru, cl, cu], [0.5, 0.4, 0.6, 0.1, 0.9], atol=1e-16)
    ravg, rl, ru, cl, cu = density_bands(0.0, 1.0, 3)
    s = 0.5 * math.exp(-1.6)
    np.testing.assert_allclose([rl, ru, cl, cu], [0.8 * s, 1 - 0.8 * s, 0.2 * s, 1 - 0.2 * s], atol=1e-16)
    # the refinement band widens with the cycle index
    assert rl < 0.4 and ru > 0.6


# ------------------------------------------------------------------ QR error
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_qr_load_transfer_is_work_consistent(p):
    R = qr_load_transfer(p)
    T = vector_dofs(interpolation_matrix(p, p + 1))
    np.testing.assert_allclose(T.T @ R, np.eye(2 * (p + 1) ** 2), atol=1e-12)


@pytest.mark.parametrize("p,d", [(1, 2), (2, 4), (3, 8), (2, 3)])
def test_composite_stiffness_restricts_across_orders(p, d):
    """T^T K^(p+1) T = K^(p): both orders integrate the same energy exactly on the same subcells."""
    T = vector_dofs(interpolation_matrix(p, p + 1))
    K0p, K01 = subcell_stiffness(p, d, 0.3), subcell_stiffness(p + 1, d, 0.3)
    for s in range(d * d):
        np.testing.assert_allclose(T.T @ K01[s] @ T, K0p[s], atol=1e-13)


def test_qr_error_range_and_fixed_dof_independence():
    rng = np.random.default_rng(9)
    for p, d in [(1, 2), (2, 4), (3, 8), (4, 2)]:
        for trial in range(3):
            rho_e = rng.uniform(0, 1, d * d) if trial else (rng.uniform(size=d * d) > 0.5).astype(float)
            ue = rng.standard_normal(2 * (p + 1) ** 2)
            e1 = qr_error_element(p, d, rho_e, ue, 1.0, 1e-9, 0.3, 3.0)
            assert 0.0 <= e1 < 1.0
            # another set of 3 rigid-mode-removing DOFs of the (p+1) element: top-right vertex
            # (both components) and u_y of the top-left vertex
            n1 = p + 2
            tr, tl = n1 * n1 - 1, n1 * (n1 - 1)
            e2 = qr_error_element(p, d, rho_e, ue, 1.0, 1e-9, 0.3, 3.0, fixed=[2 * tr, 2 * tr + 1, 2 * tl + 1])
            assert abs(e1 - e2) < 1e-10
            # invariance to scaling of u and of the moduli
            e3 = qr_error_element(p, d, rho_e, 7.5 * ue, 3.0, 3e-9, 0.3, 3.0)
            assert abs(e1 - e3) < 1e-10


def test_qr_error_invariant_to_rigid_motion():
    """eps is unchanged by adding a rigid motion to u^(p) (checked at a magnitude where the
    unremoved computation is still accurate)."""
    from oracle.element import remove_rigid_motion
    rng = np.random.default_rng(5)
    for p in (1, 2, 3):
        xy = node_coords(p)
        ue = 1e-3 * rng.standard_normal(2 * len(xy))
        r = np.zeros_like(ue)
        r[0::2] = 0.3 - 0.02 * xy[:, 1]
        r[1::2] = -0.1 + 0.02 * xy[:, 0]
        e1 = qr_error_element(p, 2, rng.uniform(0.1, 1, 4), ue, 1.0, 1e-9, 0.3, 3.0)
        e2 = qr_error_element(p, 2, rng.uniform(0.1, 1, 4) * 0 + 1, ue + r, 1.0, 1e-9, 0.3, 3.0)
        e3 = qr_error_element(p, 2, np.ones(4), ue, 1.0, 1e-9, 0.3, 3.0)
        assert abs(e2 - e3) < 1e-10
        # the removed part is exactly rigid: K annihilates the difference
        Kh = subcell_stiffness(p, 1, 0.3)[0]
        dlt = (ue + r) - remove_rigid_motion(p, ue + r)
        assert np.abs(Kh @ dlt).max() < 1e-14


def test_qr_error_zero_displacement():
    assert qr_error_element(2, 4, np.ones(16), np.zeros(18), 1.0, 1e-9, 0.3, 3.0) == 0.0


def test_qr_error_is_energy_ratio_of_nested_spaces():
    """J^(p+1) >= J^(p) with equality when the order-p solution already solves the (p+1) problem:
    for p -> p+1 on a field in Q_p whose internal load is reproduced, e.g. a single element whose
    u^(p) is the exact order-(p+1) solution restricted... checked here as the monotone bound over
    random fields and orders (eps >= 0) and eps < 1 for fields with strain."""
    rng = np.random.default_rng(1)
    for p in (1, 2, 3):
        xy = node_coords(p)
        ue = np.zeros(2 * len(xy))
        ue[0::2] = 1e-3 * xy[:, 0] ** 2
        ue[1::2] = -1e-3 * xy[:, 0] * xy[:, 1]
        e = qr_error_element(p, 2, rng.uniform(0.1, 1, 4), ue, 1.0, 1e-9, 0.3, 3.0)
        assert 0 <= e < 1


# ------------------------------------------------------------------ map update
def test_smoothing_matches_distance_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        nx, ny = rng.integers(1, 7, size=2)
        p = rng.integers(1, 6, size=nx * ny)
        got = smooth_p(p, nx, ny)
        X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
        X, Y = X.ravel(), Y.ravel()
        want = np.array([max(p[j] - 2 * (abs(X[j] - X[k]) + abs(Y[j] - Y[k])) for j in range(nx * ny))
                         for k in range(nx * ny)])
        np.testing.assert_array_equal(got, want)


def test_design_count_rule():
    # N_d = 2(p+1)^2 - 3 capped at 64, largest square grid below it
    assert [design_count_for_order(p) for p in (1, 2, 3, 4, 5)] == [2, 3, 5, 6, 8]
    assert design_count_for_order(10) == 8


def test_map_update_hand_case():
    """10 x 2 mesh, 20 elements: floor(0.05*20) = 1 coarsened and floor(0.10*20) = 2 refined by
    Gamma^a; Gamma^d signs drive the density step; eps > 0.9 adds one order last."""
    nelx, nely = 10, 2
    p = np.full(20, 2)
    p[0] = 1
    ga = np.arange(20, dtype=float)          # element 0 lowest, 18 and 19 highest
    gd = np.zeros(20)
    gd[0] = -0.05                            # p = 1 already (theta -1 from Kelly): theta -> -2
    gd[5] = -0.01                            # p 2 -> 1 (theta 0)
    gd[19] = 0.02                            # theta = +1 from Kelly: no density refinement
    gd[7] = 0.03                             # p 2 -> 3
    eps = np.zeros(20)
    eps[12] = 0.95
    pn, dn, th = map_update(nelx, nely, p, ga, gd, eps)
    want_p = np.full(20, 2)
    want_p[0] = 1
    want_p[5] = 1
    want_p[7] = 3
    want_p[18] = 3
    want_p[19] = 3
    want_p[12] = 3                           # QR
    np.testing.assert_array_equal(pn, want_p)
    assert th[0] == -2 and th[18] == 1 and th[19] == 1 and th[5] == 0
    assert dn[0] == 1 and dn[5] == 2 and dn[7] == 5 and dn[1] == 3
    assert dn[12] == 3                       # d follows the pre-QR order


def test_map_update_counts_and_caps():
    rng = np.random.default_rng(8)
    nelx, nely = 17, 9
    nel = nelx * nely
    p = rng.integers(1, 6, nel)
    p = smooth_p(p, nelx, nely)
    ga = rng.uniform(size=nel)
    pn, dn, th = map_update(nelx, nely, p, ga, np.zeros(nel), np.zeros(nel))
    assert np.sum(th == 1) == math.floor(0.10 * nel) and np.sum(th == -1) == math.floor(0.05 * nel)
    assert pn.max() <= 5 and pn.min() >= 1
    P = pn.reshape(nely, nelx)
    assert np.abs(np.diff(P, axis=0)).max() <= 2 and np.abs(np.diff(P, axis=1)).max() <= 2


# ------------------------------------------------------------------ OC
def test_oc_volume_bounds_and_move():
    m = DPMesh(6, 4, np.full(24, 2), np.array([2, 4] * 12))
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.1, 0.9, m.design_len)
    dc = -rng.uniform(0.0, 5.0, m.design_len)
    dv = subcell_areas(m)
    V = 0.4 * m.nel
    rn, lam = oc_update(rho, dc, dv, V)
    assert abs(rn @ dv - V) < 1e-8 * V
    assert (rn >= 0).all() and (rn <= 1).all()
    assert (np.abs(rn - rho) <= 0.2 + 1e-15).all()
    assert lam > 0


def test_qr_load_transfer_uniform_body_force_hand_values():
    """A uniform x body force b = 1 on the unit square: its Q1 consistent loads are 1/4 per node;
    the transferred Q2 loads are the integrals of the Q2 shape functions, i.e. products of the
    Simpson weights (1/6, 2/3, 1/6): corners 1/36, edge mid-nodes 1/9, centre 4/9."""
    f1 = np.zeros(8)
    f1[0::2] = 0.25
    f2 = qr_load_transfer(1) @ f1
    w = np.array([1 / 6, 2 / 3, 1 / 6])
    want = np.zeros(18)
    want[0::2] = np.outer(w, w).ravel()
    np.testing.assert_allclose(f2, want, atol=1e-15)


def test_qr_energy_by_pseudo_inverse():
    """J^(p+1) = 1/2 f'^T K'^+ f' for a self-equilibrated load: the pinned-DOF Cholesky route and an
    eigen-decomposition pseudo-inverse give the same eps."""
    from oracle.element import subcell_stiffness
    from oracle.solve import K0_table
    rng = np.random.default_rng(12)
    for p, d in [(1, 2), (2, 3), (3, 4)]:
        rho_e = rng.uniform(0.05, 1, d * d)
        ue = rng.standard_normal(2 * (p + 1) ** 2)
        E = simp(rho_e, 1.0, 1e-9, 3.0)
        Kp = np.tensordot(E, K0_table(p, d, 0.3), axes=(0, 0))
        K1 = np.tensordot(E, K0_table(p + 1, d, 0.3), axes=(0, 0))
        f1 = qr_load_transfer(p) @ (Kp @ ue)
        w, V = np.linalg.eigh(K1)
        keep = w > 1e-10 * w.max()
        J1 = 0.5 * np.sum((V[:, keep].T @ f1) ** 2 / w[keep])
        Jp = 0.5 * ue @ Kp @ ue
        assert abs((1 - Jp / J1) - qr_error_element(p, d, rho_e, ue, 1.0, 1e-9, 0.3, 3.0)) < 1e-9


def test_oc_uniform_closed_form():
    """Equal densities and sensitivities: the update is uniform, so it lands on V0 / area exactly
    (within the move limit)."""
    m = DPMesh(4, 2, np.full(8, 1), np.full(8, 2))
    dv = subcell_areas(m)
    rho = np.full(m.design_len, 0.5)
    rn, lam = oc_update(rho, np.full(m.design_len, -2.0), dv, 0.6 * m.nel)
    np.testing.assert_allclose(rn, 0.6, atol=1e-9)
    # lambda: 0.5 * sqrt(2 / (lambda * 0.25)) = 0.6  ->  lambda = 8 * (0.5/0.6)^2
    assert abs(lam - 8 * (0.5 / 0.6) ** 2) < 1e-7 * lam
