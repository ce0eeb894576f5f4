"""The P2 density filter (Sec. 2.1, Eqs. 4-5) and its adjoint on the GPU against the oracle, on
uniform and mixed design resolutions, including the full-size dp-adaptive cantilever (1.3M
subcells) on sampled subcells, and the chain rule through the differentiable compliance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import filter as ofl
from oracle import mesh as om
from oracle import sensitivity as ose
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


@pytest.mark.parametrize("name,R", [("cantilever_20x10_p2_d4", 0.3), ("dp_cantilever_40x20", 0.3),
                                    ("dp_cantilever_40x20", 1.7), ("mbb_40x20_p3_d8", 0.3)])
def test_filter_and_adjoint_match_oracle(mto, name, R):
    pr = W.named(name)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    rng = np.random.default_rng(4)
    x = rng.uniform(size=m.design_len)
    g = rng.standard_normal(m.design_len)
    xt = torch.tensor(x, device="cuda")
    out = torch.empty_like(xt)
    h.filter(xt, out, R)
    np.testing.assert_allclose(out.cpu().numpy(), ofl.density_filter(m, x, R), rtol=1e-13, atol=0)
    h.filter_adjoint(torch.tensor(g, device="cuda"), out, R)
    want = ofl.density_filter_adjoint(m, g, R)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-13 * np.abs(want).max())
    h.close()


def test_filter_fullsize_sampled(mto):
    """1.3M subcells of the dp-adaptive cantilever: every output against the oracle's Eq. 4 on a
    random sample of 20,000 subcells (the oracle's sparse filter matrix rows)."""
    pr = W.named("dp_cantilever_320x160")
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    rho = torch.tensor(pr.rho, device="cuda")
    out = torch.empty_like(rho)
    h.filter(rho, out, 0.3)
    H = ofl.filter_matrix(m, 0.3)
    rng = np.random.default_rng(9)
    s = rng.choice(m.design_len, 20000, replace=False)
    Hs = H[s]
    want = (Hs @ pr.rho) / np.asarray(Hs.sum(axis=1)).ravel()
    np.testing.assert_allclose(out.cpu().numpy()[s], want, rtol=1e-13, atol=0)
    h.close()


def test_filtered_compliance_gradient(mto):
    """dC/drho through the filter (torch autograd: FilterFn then ComplianceFn) against the oracle's
    dC/drho~ pulled back by its adjoint filter."""
    pr = W.named("dp_cantilever_40x20")
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    R = 0.3
    rt = ofl.density_filter(m, pr.rho, R)
    fixed, f = om.cantilever_bc(m)
    K = osv.assemble(m, osv.element_matrices(m, rt, pr.E0, pr.Emin, pr.nu, pr.q))
    u = osv.solve_direct(K, f, fixed)
    C_o = ose.compliance(f, u)
    g_o = ofl.density_filter_adjoint(m, ose.sensitivity(m, u, rt, pr.E0, pr.Emin, pr.nu, pr.q), R)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    gfixed, gf = mto.load_case(h, pr.load)
    h.set_supports(gfixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    r = torch.tensor(pr.rho, device="cuda").requires_grad_(True)
    C = mto.compliance(h, mto.density_filter(h, r, R), gf, mat, precision=mto.MTO_MIXED, rtol=1e-10,
                       norm=mto.NORM_JACOBI, max_iter=40000, precond=mto.PREC_MG)
    C.backward()
    assert abs(float(C.detach()) - C_o) < 1e-8 * abs(C_o)
    g = r.grad.cpu().numpy()
    assert np.abs(g - g_o).max() < 1e-6 * np.abs(g_o).max()
    h.close()
