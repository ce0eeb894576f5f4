"""Distributed load (Sec. 4.1, Fig. 6a) and node lookup on the GPU path against the oracle:
consistent side loads on mixed-order sides bit-for-bit in the DOFs they touch and to rounding in
value, edge DOF lookup identical to the oracle's numbering, and the distributed-load cantilever
solved, its compliance and sensitivities matched to the stated tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
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


def test_side_loads_and_edge_dofs(mto):
    pr = W.named("dp_cantilever_40x20")
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    for side in range(4):
        for comp in (0, 1):
            f = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
            h.side_load(side, comp, -0.37, f)
            want = om.side_load(m, side, comp, -0.37)
            got = f.cpu().numpy()
            np.testing.assert_array_equal(np.flatnonzero(got), np.flatnonzero(want))
            np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-16)
    rng = np.random.default_rng(7)
    for _ in range(40):
        ix, iy = int(rng.integers(0, pr.nelx)), int(rng.integers(0, pr.nely + 1))
        nodes, _ = m._edge_nodes_h(ix, iy)
        np.testing.assert_array_equal(h.edge_dofs(0, ix, iy, 1), 2 * np.array(nodes) + 1)
        ix, iy = int(rng.integers(0, pr.nelx + 1)), int(rng.integers(0, pr.nely))
        nodes, _ = m._edge_nodes_v(ix, iy)
        np.testing.assert_array_equal(h.edge_dofs(1, ix, iy, 0), 2 * np.array(nodes))
    with pytest.raises(mto.MTOError):
        h.edge_dofs(0, pr.nelx, 0, 0)
    h.close()


@pytest.mark.parametrize("name", ["cantilever_20x10_p2_d4", "dp_cantilever_40x20"])
def test_distributed_cantilever_parity(mto, name):
    pr = W.named(name)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f = om.distributed_cantilever_bc(m)
    K = osv.assemble(m, osv.element_matrices(m, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q))
    u_o = osv.solve_direct(K, f, fixed)
    C_o = ose.compliance(f, u_o)
    dc_o = ose.sensitivity(m, u_o, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    gfixed, gf = mto.load_case(h, W.CANTILEVER_DISTRIBUTED)
    np.testing.assert_array_equal(gfixed, fixed)
    np.testing.assert_allclose(gf.cpu().numpy(), f, rtol=1e-14, atol=1e-17)
    h.set_supports(gfixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    rho = torch.tensor(pr.rho, dtype=torch.float64, device="cuda")
    h.build_elements(rho, mat, mto.MTO_MIXED)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(gf, u, precision=mto.MTO_MIXED, rtol=1e-10, norm=mto.NORM_JACOBI, max_iter=40000, precond=mto.PREC_MG)
    uerr = np.linalg.norm(u.cpu().numpy() - u_o) / np.linalg.norm(u_o)
    assert uerr < 1e-8, uerr
    dc = torch.zeros(h.design_len, dtype=torch.float64, device="cuda")
    C = h.sensitivity(u, gf, rho, mat, dc, precision=mto.MTO_FP64)
    assert abs(C - C_o) < 1e-8 * abs(C_o)
    assert np.abs(dc.cpu().numpy() - dc_o).max() < 1e-6 * np.abs(dc_o).max()
    h.close()
