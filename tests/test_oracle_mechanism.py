"""Pins for oracle/mechanism.py (general objective J = z^T u with springs, Sec. 4.1 force inverter):
a one-DOF closed form of the spring addition, reciprocity z^T u = f^T v of the adjoint solve, the
compliance special case z = f, and central finite differences of J with exact solves."""
import numpy as np
import pytest

from oracle.element import homogeneous_stiffness, simp
from oracle.mechanism import add_springs, adjoint_sensitivity, inverter_problem
from oracle.mesh import DPMesh, cantilever_bc
from oracle.sensitivity import sensitivity
from oracle.solve import assemble, element_matrices, solve_direct


def test_spring_one_dof_closed_form():
    # one Q1 element, every DOF held but u_x of the top-right vertex (local DOF 6 in the
    # interleaved (a, b) order: vertex 3 = (1, 1)); load 1 there and a spring k: u = 1 / (K_44 + k)
    m = DPMesh(1, 1, [1], [1])
    Ke = homogeneous_stiffness(1, 0.3)
    K = assemble(m, [Ke * 0.7])
    dof = 2 * m.vertex(1, 1)
    fixed = np.setdiff1d(np.arange(m.ndof), [dof])
    f = np.zeros(m.ndof)
    f[dof] = 1.0
    k = 0.25
    u = solve_direct(add_springs(K, np.array([dof]), [k]), f, fixed)
    assert abs(u[dof] - 1.0 / (0.7 * Ke[6, 6] + k)) < 1e-15


def small(seed, p=(1, 2, 3)):
    rng = np.random.default_rng(seed)
    nelx, nely = 6, 4
    P = rng.choice(p, nelx * nely)
    D = rng.choice([1, 2], nelx * nely)
    m = DPMesh(nelx, nely, P, D)
    rho = rng.uniform(0.2, 1.0, m.design_len)
    return m, rho


@pytest.mark.parametrize("seed", [0, 1])
def test_reciprocity_and_compliance_case(seed):
    m, rho = small(seed)
    fixed, f, z, sd, sk = inverter_problem(m)
    K = add_springs(assemble(m, element_matrices(m, rho, 1.0, 1e-9, 0.3, 3.0)), sd, sk)
    u = solve_direct(K, f, fixed)
    v = solve_direct(K, z, fixed)
    assert abs(z @ u - f @ v) <= 1e-12 * abs(z @ u)
    # z = f: v = u and the adjoint sensitivity is the compliance sensitivity
    dJ = adjoint_sensitivity(m, u, u, rho)
    dC = sensitivity(m, u, rho)
    np.testing.assert_allclose(dJ, dC, rtol=1e-12, atol=1e-14 * np.abs(dC).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_central_differences(seed):
    m, rho = small(seed)
    fixed, f, z, sd, sk = inverter_problem(m)

    def J(r):
        K = add_springs(assemble(m, element_matrices(m, r, 1.0, 1e-9, 0.3, 3.0)), sd, sk)
        return z @ solve_direct(K, f, fixed), K

    J0, K = J(rho)
    u = solve_direct(K, f, fixed)
    v = solve_direct(K, z, fixed)
    g = adjoint_sensitivity(m, u, v, rho)
    rng = np.random.default_rng(seed + 10)
    h = 1e-6
    for s in rng.choice(m.design_len, 8, replace=False):
        rp, rm = rho.copy(), rho.copy()
        rp[s] += h
        rm[s] -= h
        fd = (J(rp)[0] - J(rm)[0]) / (2 * h)
        assert abs(fd - g[s]) <= 1e-6 * np.abs(g).max() + 1e-5 * abs(g[s]), (s, fd, g[s])


def test_inverter_geometry():
    m = DPMesh(8, 4, np.full(32, 2), np.full(32, 2))
    fixed, f, z, sd, sk = inverter_problem(m)
    assert f.sum() == 1.0 and z.sum() == 1.0
    assert sd[0] == 2 * m.vertex(0, 2) and sd[1] == 2 * m.vertex(8, 2)
    # corners held (both components), nothing else at this resolution
    held = {2 * m.vertex(0, 0), 2 * m.vertex(0, 0) + 1, 2 * m.vertex(0, 4), 2 * m.vertex(0, 4) + 1}
    assert set(fixed.tolist()) == held
