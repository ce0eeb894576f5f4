"""Pins for oracle/sensitivity.py: central finite differences with exact solves, the energy split,
rigid-mode invariance."""
import numpy as np
import pytest

from oracle.element import simp
from oracle.mesh import DPMesh, cantilever_bc, mbb_bc
from oracle.sensitivity import compliance, energy_split, sensitivity, subcell_energies
from oracle.solve import solve


@pytest.mark.parametrize("bc", ["cantilever", "mbb"])
def test_sensitivity_matches_central_differences(bc):
    p = np.array([1, 2, 3, 2, 3, 3, 2, 1, 2, 2, 3, 2])
    d = np.array([2, 1, 3, 2, 2, 4, 1, 2, 3, 2, 1, 2])
    m = DPMesh(4, 3 if bc == "mbb" else 3, p, d) if bc == "mbb" else DPMesh(6, 2, p, d)
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.2, 1.0, m.design_len)
    fixed, f = (cantilever_bc if bc == "cantilever" else mbb_bc)(m)
    u, K, _ = solve(m, rho, fixed, f)
    dc = sensitivity(m, u, rho)
    h = 1e-6
    for s in rng.choice(m.design_len, 12, replace=False):
        rp, rm = rho.copy(), rho.copy()
        rp[s] += h
        rm[s] -= h
        Cp = compliance(f, solve(m, rp, fixed, f)[0])
        Cm = compliance(f, solve(m, rm, fixed, f)[0])
        fd = (Cp - Cm) / (2 * h)
        assert abs(fd - dc[s]) <= 1e-6 * np.abs(dc).max() + 1e-6 * abs(dc[s])


def test_energy_split_equals_compliance():
    m = DPMesh(8, 4, np.full(32, 2), np.full(32, 4))
    rng = np.random.default_rng(2)
    rho = 0.5 + rng.uniform(-0.1, 0.1, m.design_len)
    fixed, f = cantilever_bc(m)
    u, K, _ = solve(m, rho, fixed, f)
    C = compliance(f, u)
    assert abs(energy_split(m, u, rho) - C) < 1e-11 * C
    # sensitivities of a compliance problem are non-positive
    assert (sensitivity(m, u, rho) <= 0).all()


def test_quadratic_forms_ignore_rigid_motion():
    m = DPMesh(3, 2, np.array([1, 2, 3, 2, 3, 1]), np.array([1, 2, 3, 4, 2, 3]))
    rng = np.random.default_rng(4)
    u = rng.standard_normal(m.ndof)
    xy = m.node_xy()
    r = np.zeros(m.ndof)
    r[0::2] = 3.0 - 0.7 * xy[:, 1]
    r[1::2] = -2.0 + 0.7 * xy[:, 0]
    w0 = subcell_energies(m, u, 0.3)
    w1 = subcell_energies(m, u + 1e3 * r, 0.3)
    np.testing.assert_allclose(w1, w0, rtol=1e-7, atol=1e-9 * np.abs(w0).max())
