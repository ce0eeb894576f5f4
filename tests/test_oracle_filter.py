"""Pins for oracle/filter.py (P2 density filter, Sec. 2.1 Eqs. 4-5): hand values of a spike on a
uniform grid, partition of unity, the identity below the cell spacing, exact reproduction of linear
fields where the stencil is symmetric, the adjoint's dot-product identity, and finite differences
of a functional through the filter."""
import numpy as np
import pytest

from oracle.filter import density_filter, density_filter_adjoint, filter_matrix, subcell_centres
from oracle.mesh import DPMesh


def uniform(d=4, nelx=5, nely=4):
    return DPMesh(nelx, nely, np.full(nelx * nely, 1), np.full(nelx * nely, d))


def test_spike_hand_values():
    # uniform spacing a = 1/4; R = 1.1 a reaches only the 4 edge neighbours (distance a, weight
    # 0.1 a) besides the cell itself (weight 1.1 a); the diagonal neighbours sit at 1.414 a
    m = uniform(4)
    a = 0.25
    R = 1.1 * a
    c = subcell_centres(m)
    s = int(np.argmin(np.linalg.norm(c - [2.375, 1.875], axis=1)))     # an interior subcell
    rho = np.zeros(m.design_len)
    rho[s] = 1.0
    rt = density_filter(m, rho, R)
    assert abs(rt[s] - 1.1 / 1.5) < 1e-15
    nb = np.flatnonzero(np.isclose(np.linalg.norm(c - c[s], axis=1), a))
    assert len(nb) == 4
    np.testing.assert_allclose(rt[nb], 0.1 / 1.5, rtol=1e-14)
    assert np.count_nonzero(rt) == 5


def test_constant_and_identity():
    m = DPMesh(4, 3, np.full(12, 2), np.array([1, 2, 4, 2, 1, 4, 4, 2, 1, 2, 4, 1]))
    rho = np.full(m.design_len, 0.37)
    np.testing.assert_allclose(density_filter(m, rho, 0.3), rho, rtol=1e-15)
    r = np.random.default_rng(0).uniform(size=m.design_len)
    # below the smallest centre spacing (1/4) only the cell itself is within R
    np.testing.assert_allclose(density_filter(m, r, 0.2), r, rtol=1e-15)


def test_linear_field_interior():
    m = uniform(4, 8, 6)
    c = subcell_centres(m)
    rho = 0.3 * c[:, 0] - 0.2 * c[:, 1] + 0.5
    R = 0.3
    rt = density_filter(m, rho, R)
    inner = (c[:, 0] > R) & (c[:, 0] < 8 - R) & (c[:, 1] > R) & (c[:, 1] < 6 - R)
    np.testing.assert_allclose(rt[inner], rho[inner], rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_and_finite_differences(seed):
    rng = np.random.default_rng(seed)
    m = DPMesh(5, 4, np.full(20, 2), rng.choice([1, 2, 4], 20))
    R = 0.3
    x = rng.uniform(size=m.design_len)
    y = rng.uniform(size=m.design_len)
    assert abs(density_filter(m, x, R) @ y - x @ density_filter_adjoint(m, y, R)) < 1e-13
    # J(rho) = sum_s c_s rho~_s^2: dJ/drho = adjoint(2 c rho~)
    cw = rng.uniform(size=m.design_len)
    J = lambda r: float(cw @ density_filter(m, r, R) ** 2)
    g = density_filter_adjoint(m, 2 * cw * density_filter(m, x, R), R)
    h = 1e-6
    for s in rng.choice(m.design_len, 6, replace=False):
        e = np.zeros(m.design_len)
        e[s] = h
        fd = (J(x + e) - J(x - e)) / (2 * h)
        assert abs(fd - g[s]) < 1e-8


def test_symmetric_weights():
    m = DPMesh(3, 3, np.full(9, 1), np.array([1, 2, 4, 8, 4, 2, 1, 2, 4]))
    H = filter_matrix(m, 0.3)
    assert abs(H - H.T).max() == 0.0
    assert H.min() >= 0.0
