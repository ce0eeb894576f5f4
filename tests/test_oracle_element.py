"""Pins for oracle/element.py: symmetry, rigid modes, the homogeneous element, the published
bilinear plane-stress element, linearity in the moduli."""
import json
import os

import numpy as np
import pytest

from oracle.element import (D0, element_stiffness, homogeneous_stiffness, interpolation_matrix,
                            node_coords, scalar_mass, simp, simp_deriv, subcell_stiffness)

NU = 0.3
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def top88_KE(nu):
    """Closed-form unit-modulus bilinear plane-stress element on a unit square (Andreassen et al.,
    'Efficient topology optimization in MATLAB using 88 lines of code', 2011), nodes ordered
    counter-clockwise from the lower-left corner."""
    A11 = np.array([[12, 3, -6, -3], [3, 12, 3, 0], [-6, 3, 12, -3], [-3, 0, -3, 12]], float)
    A12 = np.array([[-6, -3, 0, 3], [-3, -6, -3, -6], [0, -3, -6, 3], [3, -6, 3, -6]], float)
    B11 = np.array([[-4, 3, -2, 9], [3, -4, -9, 4], [-2, -9, -4, -3], [9, 4, -3, -4]], float)
    B12 = np.array([[2, -3, 4, -9], [-3, 2, 9, -2], [4, 9, 2, 3], [-9, -2, 3, 2]], float)
    return 1 / (1 - nu ** 2) / 24 * (np.block([[A11, A12], [A12.T, A11]]) + nu * np.block([[B11, B12], [B12.T, B11]]))


def test_bilinear_matches_published_closed_form():
    K = homogeneous_stiffness(1, NU)
    # oracle local nodes: (0,0),(1,0),(0,1),(1,1); published order: LL, LR, UR, UL
    perm_nodes = [0, 1, 3, 2]
    perm = np.array([[2 * n, 2 * n + 1] for n in perm_nodes]).ravel()
    np.testing.assert_allclose(K[np.ix_(perm, perm)], top88_KE(NU), atol=1e-15)


def rigid_modes(p, hx=1.0, hy=1.0):
    xy = node_coords(p, hx, hy)
    n = len(xy)
    R = np.zeros((2 * n, 3))
    R[0::2, 0] = 1
    R[1::2, 1] = 1
    R[0::2, 2] = -xy[:, 1]
    R[1::2, 2] = xy[:, 0]
    return R


@pytest.mark.parametrize("p,d", [(1, 1), (1, 2), (2, 4), (3, 8), (4, 3), (5, 2)])
def test_subcells_sum_to_homogeneous(p, d):
    K0 = subcell_stiffness(p, d, NU)
    assert K0.shape == (d * d, 2 * (p + 1) ** 2, 2 * (p + 1) ** 2)
    np.testing.assert_allclose(K0, K0.transpose(0, 2, 1), atol=1e-15)
    # independent whole-element rule, and an over-integrated one (exactness of (p+1)^2)
    Kh = homogeneous_stiffness(p, NU)
    np.testing.assert_allclose(K0.sum(axis=0), Kh, atol=1e-13 * np.abs(Kh).max())
    np.testing.assert_allclose(homogeneous_stiffness(p, NU, nq=p + 3), Kh, atol=1e-13 * np.abs(Kh).max())


@pytest.mark.parametrize("p,d", [(1, 2), (2, 4), (3, 8), (4, 2)])
def test_rigid_modes_and_rank(p, d):
    rng = np.random.default_rng(7)
    K0 = subcell_stiffness(p, d, NU)
    E = simp(rng.uniform(0.05, 1, d * d), 1.0, 1e-9, 3.0)
    Ke = element_stiffness(K0, E)
    R = rigid_modes(p)
    assert np.abs(Ke @ R).max() < 1e-13 * np.abs(Ke).max()
    ev = np.linalg.eigvalsh(Ke)
    tol = 1e-11 * ev.max()
    assert np.sum(np.abs(ev) < tol) == 3
    assert ev.min() > -tol


def test_q10_has_239_deformation_modes():
    pins = json.load(open(os.path.join(GOLD, "paper_pins.json")))["q10_deformation_modes"]
    K = homogeneous_stiffness(pins["p"], NU)
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev > 1e-10 * ev.max()) == pins["modes"]


def test_table_b_support_points():
    pins = json.load(open(os.path.join(GOLD, "paper_pins.json")))["table_b_support_points"]
    for p, n in zip(pins["p"], pins["n_sup"]):
        assert len(node_coords(p)) == n


def test_linearity_and_uniform_density():
    p, d = 3, 4
    K0 = subcell_stiffness(p, d, NU)
    rng = np.random.default_rng(3)
    a, b = rng.uniform(size=d * d), rng.uniform(size=d * d)
    np.testing.assert_allclose(element_stiffness(K0, 2 * a + 3 * b),
                               2 * element_stiffness(K0, a) + 3 * element_stiffness(K0, b), atol=1e-13)
    np.testing.assert_allclose(element_stiffness(K0, np.full(d * d, 0.7)), 0.7 * homogeneous_stiffness(p, NU),
                               atol=1e-13)


def test_constant_strain_energy():
    """u = eps0 applied as a linear field: u^T K u = area * eps^T D0 eps (closed form)."""
    for p in (1, 2, 3, 4):
        xy = node_coords(p)
        ex, ey, g = 1e-3, -4e-4, 2.5e-4
        u = np.zeros(2 * len(xy))
        u[0::2] = ex * xy[:, 0] + 0.5 * g * xy[:, 1]
        u[1::2] = ey * xy[:, 1] + 0.5 * g * xy[:, 0]
        eps = np.array([ex, ey, g])
        K = homogeneous_stiffness(p, NU)
        assert abs(u @ K @ u - eps @ D0(NU) @ eps) < 1e-15


def test_simp_and_derivative():
    r = np.linspace(0, 1, 11)
    np.testing.assert_allclose(simp(r, 1, 1e-9, 3), 1e-9 + r ** 3 * (1 - 1e-9))
    h = 1e-6
    rr = np.linspace(0.1, 0.9, 9)
    np.testing.assert_allclose(simp_deriv(rr, 1, 1e-9, 3), (simp(rr + h, 1, 1e-9, 3) - simp(rr - h, 1, 1e-9, 3)) / (2 * h),
                               rtol=1e-8)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_and_interpolation(p):
    M = scalar_mass(p, p)
    assert abs(M.sum() - 1.0) < 1e-14        # integral of 1 over the unit square
    T = interpolation_matrix(p, p + 1)
    M1 = scalar_mass(p + 1, p + 1)
    np.testing.assert_allclose(T.T @ M1 @ T, M, atol=1e-15)
    np.testing.assert_allclose(scalar_mass(p + 1, p), M1 @ T, atol=1e-15)
    np.testing.assert_allclose(T.sum(axis=1), 1.0, atol=1e-14)
