"""The force inverter (Sec. 4.1, Fig. 6b) on the GPU path against the oracle: springs in the
operator, the adjoint solve K v = z, J = z^T u and dJ/drho = -E' v_e^T K0 u_e, plus the compliance
special case of the adjoint kernel (v = u gives the compliance sensitivities)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import mechanism as omc
from oracle import mesh as om
from oracle import solve as osv


@pytest.fixture(scope="module")
def mto():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_09821_gb300 as m
    from paper_1811_09821_gb300 import _build
    _build.build()
    m.load_library()
    return m


@pytest.mark.parametrize("name,path", [("cantilever_20x10_p2_d4", "fp64"), ("dp_cantilever_40x20", "mixed"),
                                       ("dp_cantilever_40x20", "fp64")])
def test_inverter_objective_and_adjoint_sensitivity(mto, name, path):
    pr = W.named(name)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f, z, sd, sk = omc.inverter_problem(m)
    K = omc.add_springs(osv.assemble(m, osv.element_matrices(m, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)), sd, sk)
    u_o = osv.solve_direct(K, f, fixed)
    v_o = osv.solve_direct(K, z, fixed)
    J_o = z @ u_o
    g_o = omc.adjoint_sensitivity(m, u_o, v_o, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)

    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    gfixed, gf, gz = mto.inverter_case(h)
    np.testing.assert_array_equal(gfixed, fixed)
    np.testing.assert_array_equal(gf.cpu().numpy(), f)
    np.testing.assert_array_equal(gz.cpu().numpy(), z)
    h.set_supports(gfixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    rho = torch.tensor(pr.rho, dtype=torch.float64, device="cuda")
    prec = mto.MTO_MIXED if path == "mixed" else mto.MTO_FP64
    h.build_elements(rho, mat, prec)
    # the operator with springs against the oracle's K + S
    x = np.random.default_rng(1).standard_normal(h.ndof)
    y = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.apply(torch.tensor(x, device="cuda"), y)
    want = K @ x
    assert np.abs(y.cpu().numpy() - want).max() < 1e-13 * np.abs(want).max()
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    for rhs, out in ((gf, u), (gz, v)):
        h.solve(rhs, out, precision=prec, rtol=1e-12, norm=mto.NORM_L2, max_iter=40000, precond=mto.PREC_MG,
                raise_on_noconv=False)
    # the soft output spring (k_out = 1e-3) and the thin members make this problem worse conditioned
    # than the compliance cases: an l2 solve at 1e-12 pins u to ~2e-8 here
    for got, ref in ((u, u_o), (v, v_o)):
        err = np.linalg.norm(got.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 1e-7, err
    J = float(gz @ u)
    assert abs(J - J_o) < 1e-8 * abs(J_o)
    assert abs(J - float(gf @ v)) < 1e-8 * abs(J)          # reciprocity on the GPU solves
    g = torch.zeros(h.design_len, dtype=torch.float64, device="cuda")
    h.sensitivity_adjoint(u, v, rho, mat, g)
    gn = g.cpu().numpy()
    assert np.abs(gn - g_o).max() < 1e-6 * np.abs(g_o).max()
    assert np.linalg.norm(gn - g_o) < 1e-6 * np.linalg.norm(g_o)
    # the bilinear kernel with v = u is the compliance sensitivity
    dc = torch.zeros_like(g)
    h.sensitivity(u, gf, rho, mat, dc)
    h.sensitivity_adjoint(u, u, rho, mat, g)
    np.testing.assert_allclose(g.cpu().numpy(), dc.cpu().numpy(), rtol=1e-12,
                               atol=1e-14 * float(dc.abs().max()))
    h.set_springs([], [])
    h.close()
