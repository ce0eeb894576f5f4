"""The dp-adaptive cycle (Sec. 3.3, Sec. 4.1) on the GPU path: the paper's initial mesh (40 x 20,
Q2, 4 x 4 design points, point-load cantilever, V0 = 0.45, R = 0.3 h), three cycles.  Checked
against the oracle at every cycle: the Table 2 counts of cycle 1 (6560 free DOFs, 12800 design
points), the maps of each cycle's update (the oracle's indicators and map update on the GPU's
final solved state, bit-exact outside a guard band), the design transfer to the next cycle's
layout, the stopping rule on the returned objective values, and the design transfer kernel on
its own for every pair of counts; plus the compliance and the displacement of each final state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import adaptive as oad
from oracle import indicators as oi
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


def test_transfer_design_kernel(mto):
    rng = np.random.default_rng(3)
    nelx, nely = 7, 5
    nel = nelx * nely
    d_old = rng.integers(1, 9, nel).astype(np.int32)
    d_new = rng.integers(1, 9, nel).astype(np.int32)
    d_new[:5] = d_old[:5]
    rho = rng.uniform(size=int((d_old.astype(np.int64) ** 2).sum()))
    h = mto.Handle(0)
    h.setup(nelx, nely, np.full(nel, 2, np.int32), d_new)
    out = torch.empty(h.design_len, dtype=torch.float64, device="cuda")
    h.transfer_design(d_old, torch.tensor(rho, device="cuda"), out)
    want = oad.transfer_design(d_old, rho, d_new)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-14, atol=1e-16)
    n5 = int((d_old[:5].astype(np.int64) ** 2).sum())
    np.testing.assert_array_equal(out.cpu().numpy()[:n5], rho[:n5])
    h.close()


def test_adaptive_cycles_against_oracle(mto):
    from paper_1811_09821_gb300 import adaptive
    nelx, nely = 40, 20
    nel = nelx * nely
    p0 = np.full(nel, 2, np.int32)
    d0 = np.full(nel, 4, np.int32)
    vol = 0.45
    rho0 = np.full(nel * 16, vol)
    R = 0.3
    recs = adaptive.run(nelx, nely, p0, d0, rho0, W.CANTILEVER, vol, cycles=3, max_iters=25, radius=R, keep=True)
    assert len(recs) == 3
    assert recs[0].free_dofs == 6560 and recs[0].design_points == 12800
    for i, rc in enumerate(recs):
        # stopping rule on the returned objective values (or the iteration cap)
        J = rc.J
        stops = [oad.cycle_converged(J[t - 1], J[t], rc.cycle) for t in range(1, len(J))]
        assert not any(stops[:-1])
        assert stops[-1] or rc.iterations == 25
        # the final state against the oracle: the solves stop at a relative compliance accuracy of
        # 1e-9, so J (the energy form) is within 1e-8 of the exact compliance and u within
        # ||u - u*||_K^2 <= 1e-8 C of the exact displacement
        m = om.DPMesh(nelx, nely, rc.p, rc.d)
        fixed, f = om.cantilever_bc(m)
        rf = rc.state["rho_f"].cpu().numpy()
        K = osv.assemble(m, osv.element_matrices(m, rf, 1.0, 1e-9, 0.3, 3.0))
        u_o = osv.solve_direct(K, f, fixed)
        C_o = ose.compliance(f, u_o)
        u = rc.state["u"].cpu().numpy()
        e = u - u_o
        assert e @ (K @ e) <= 1e-8 * C_o
        assert abs(J[-1] - C_o) <= 1e-8 * C_o
        # indicators and maps of the update, on the GPU's own state
        ga = oi.kelly(m, u)
        gd = oi.gamma_d(m, rf, cycle=rc.cycle)
        eq = oi.qr_error(m, u, rf, 1.0, 1e-9, 0.3, 3.0)
        ind = rc.state["indicators"]
        np.testing.assert_allclose(ind["gamma_a"].cpu().numpy(), ga, rtol=1e-9, atol=1e-12 * np.abs(ga).max())
        np.testing.assert_allclose(ind["gamma_d"].cpu().numpy(), gd, rtol=0, atol=1e-15)
        np.testing.assert_allclose(ind["eps_qr"].cpu().numpy(), eq, rtol=0, atol=1e-6)
        srt = np.sort(ga, kind="stable")
        nc, nr = int(np.floor(0.05 * nel)), int(np.floor(0.10 * nel))
        ties = sum(int(srt[k] - srt[k - 1] <= 1e-12 * abs(srt[k])) for k in (nc, nel - nr))
        ties += int(((gd != 0) & (np.abs(gd) <= 1e-12 * np.abs(gd).max())).sum())
        ties += int((np.abs(eq - 0.9) <= 1e-6).sum())
        pn, dn, th = oi.map_update(nelx, nely, rc.p, ga, gd, eq)
        np.testing.assert_array_equal(rc.p_new, pn)
        np.testing.assert_array_equal(rc.d_new, dn)
        assert ties == 0
        # the design carried to the next cycle
        if i + 1 < len(recs):
            np.testing.assert_array_equal(recs[i + 1].p, pn)
            np.testing.assert_array_equal(recs[i + 1].d, dn)
            want = oad.transfer_design(rc.d, rc.state["rho"].cpu().numpy(), dn)
            np.testing.assert_allclose(rc.state["rho_next"].cpu().numpy(), want, rtol=1e-14, atol=1e-16)
    print("cycles:", [(r.cycle, r.free_dofs, r.design_points, r.iterations, round(r.J[-1], 4)) for r in recs])
