"""Full-size checks in the bench's launch configuration, where the oracle cannot solve the whole
problem in seconds: sampled outputs the oracle computes one by one (element matrices, numbering,
density indicator) and properties that hold at any size (residual evaluated with the oracle's own
assembled operator, the energy identity, the energy split of the sensitivities, and central
finite differences of the compliance for the adjoint gradient)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import element as oe
from oracle import indicators as oi
from oracle import mesh as om
from oracle import solve as osv

BENCH_RTOL = 1e-8


@pytest.fixture(scope="module")
def mto():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_09821_gb300 as m
    from paper_1811_09821_gb300 import _build
    _build.build()
    m.load_library()
    return m


_CACHE = {}


def full_case(mto, name):
    if name in _CACHE:
        return _CACHE[name]
    pr = W.named(name)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f = (om.mbb_bc if pr.load == W.MBB else om.cantilever_bc)(m)
    K = osv.assemble(m, osv.element_matrices(m, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q))
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    gfixed, gf = mto.load_case(h, pr.load)
    h.set_supports(gfixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    rho = torch.tensor(pr.rho, dtype=torch.float64, device="cuda")
    out = dict(pr=pr, m=m, fixed=fixed, f=f, K=K, h=h, gfixed=gfixed, gf=gf, mat=mat, rho=rho)
    _CACHE[name] = out
    return out


@pytest.mark.parametrize("name", ["mbb_160x80_p3_d8", "dp_cantilever_320x160"])
def test_fullsize_numbering_and_build(mto, name):
    c = full_case(mto, name)
    pr, m, h = c["pr"], c["m"], c["h"]
    assert h.ndof == m.ndof and h.design_len == m.design_len
    np.testing.assert_array_equal(c["gfixed"], c["fixed"])
    rng = np.random.default_rng(17)
    sample = rng.choice(m.nel, 64, replace=False)
    for build, tol in ((mto.MTO_FP64, 1e-14), (mto.MTO_MIXED, 1e-13)):
        h.build_elements(c["rho"], c["mat"], build)
        for e in sample:
            p, d = int(m.p[e]), int(m.d[e])
            want_full = oe.element_stiffness(osv.K0_table(p, d, pr.nu), oe.simp(
                pr.rho[m.design_off[e]:m.design_off[e + 1]], pr.E0, pr.Emin, pr.q))
            iu = np.triu_indices(want_full.shape[0])
            want = want_full[iu]
            got = h.element_matrix(int(e), p)
            assert np.abs(got - want).max() <= tol * np.abs(want).max(), (e, build)
            got_nodes = h.element_nodes(int(e))
            want_nodes = m.element_node_map(int(e))
            assert [[g for g, _ in a] for a in got_nodes] == [[g for g, _ in a] for a in want_nodes]


@pytest.mark.parametrize("name", ["mbb_160x80_p3_d8", "dp_cantilever_320x160"])
def test_fullsize_solve_properties(mto, name):
    """The bench's solves (mixed: FP64 refinement around the split-precision operator; plain FP64;
    multigrid-preconditioned, l2 rtol 1e-8) meet their residual when it is recomputed with the
    oracle's assembled FP64 operator; energy identity; the two paths agree on C."""
    c = full_case(mto, name)
    h, K, f = c["h"], c["K"], c["f"]
    Cs = {}
    for build, prec in ((mto.MTO_MIXED, mto.MTO_MIXED), (mto.MTO_FP64, mto.MTO_FP64)):
        h.build_elements(c["rho"], c["mat"], build)
        u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
        it, rr = h.solve(c["gf"], u, precision=prec, rtol=BENCH_RTOL, max_iter=400000, precond=mto.PREC_MG)
        ug = u.cpu().numpy()
        r = f - K @ ug
        r[c["fixed"]] = 0.0
        assert np.all(ug[c["fixed"]] == 0.0)
        rel = np.linalg.norm(r) / np.linalg.norm(f)
        assert rel <= 2 * BENCH_RTOL, (build, rel, rr, it)
        C = float(f @ ug)
        # energy identity f^T u - u^T K u = u^T r, bounded by ||u|| ||r||
        assert abs(C - ug @ (K @ ug)) <= 1.01 * np.linalg.norm(ug) * np.linalg.norm(r) + 1e-12 * abs(C)
        Cs[build] = C
    assert abs(Cs[mto.MTO_MIXED] - Cs[mto.MTO_FP64]) <= 1e-7 * abs(Cs[mto.MTO_FP64])


@pytest.mark.parametrize("name", ["mbb_160x80_p3_d8", "dp_cantilever_320x160"])
def test_fullsize_density_indicator_sampled(mto, name):
    c = full_case(mto, name)
    pr, m, h = c["pr"], c["m"], c["h"]
    h.build_elements(c["rho"], c["mat"], mto.MTO_MIXED)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(c["gf"], u, precision=mto.MTO_MIXED, rtol=BENCH_RTOL, max_iter=400000, precond=mto.PREC_MG)
    ind = h.indicator(u, c["rho"], c["mat"])
    gd = oi.gamma_d(m, pr.rho)
    np.testing.assert_allclose(ind["gamma_d"].cpu().numpy(), gd, rtol=0, atol=1e-15)
    eq = ind["eps_qr"].cpu().numpy()
    assert np.all(eq >= -1e-9) and np.all(eq < 1.0)
    assert np.all(ind["gamma_a"].cpu().numpy() >= 0.0)
    pn = ind["p_new"].cpu().numpy()
    assert pn.min() >= 1 and pn.max() <= 5


def element_energy(mto, h, u, f, rho, mat, dc, pr):
    """u^T K(rho) u as sum_s E(rho_s) w_s with w_s = -dc_s / E'(rho_s) from the sensitivity kernel
    (element-wise, after the rigid-motion removal: free of the cancellation that a global
    u^T (K u) suffers on compliant designs)."""
    h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64, want_C=False)
    r = rho.cpu().numpy()
    E = oe.simp(r, pr.E0, pr.Emin, pr.q)
    dE = oe.simp_deriv(r, pr.E0, pr.Emin, pr.q)
    return float(np.sum(E * (-dc.cpu().numpy() / dE)))


def test_fullsize_energy_split_and_fd_gradient(mto):
    """dp-adaptive cantilever (smooth densities, all E' > 0).  (1) sum_s E_s w_s, w_s =
    -dc_s / E'(rho_s), equals u^T K u from the operator (to 1e-6: the global product loses ~1e-8 to
    cancellation on this compliant design).  (2) The adjoint gradient against central finite
    differences of the compliance along 5 seeded random directions over all 1.3M design values
    (v_s = sign(dc_s) U(0.5, 1.5)): (C(rho + h v) - C(rho - h v)) / 2h = dc . v within 1e-5, each C
    the energy functional 2 f^T u - u^T K u of a re-solved u (exact at the solution, second order
    in the solve error), h = 1e-5.  A single design value moved by 1e-6 changes C by ~1e-11 of C,
    below what any FP64 solve of this size resolves, so the check moves all values along a
    direction (the oracle's own tests check single-value differences with exact solves on small
    meshes); the directions follow the sign of dc so that dc . v does not cancel."""
    c = full_case(mto, "dp_cantilever_320x160")
    pr, h = c["pr"], c["h"]
    f, rho, mat = c["gf"], c["rho"], c["mat"]
    h.build_elements(rho, mat, mto.MTO_FP64)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(f, u, precision=mto.MTO_FP64, rtol=1e-8, max_iter=40000, precond=mto.PREC_MG)
    dc = torch.zeros(h.design_len, dtype=torch.float64, device="cuda")
    h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64)
    dcn = dc.cpu().numpy().copy()
    scratch = torch.zeros_like(u)
    h.apply(u, scratch)
    uKu = float(u @ scratch)
    dE = oe.simp_deriv(pr.rho, pr.E0, pr.Emin, pr.q)
    assert np.all(dE > 0)
    eK = element_energy(mto, h, u, f, rho, mat, dc, pr)
    assert abs(eK - uKu) <= 1e-6 * abs(uKu), (eK, uKu)
    rng = np.random.default_rng(181109821 + 3)
    hstep = 1e-5
    u0 = u.clone()
    work = torch.zeros_like(dc)
    errs = []
    for _ in range(5):
        v = np.sign(dcn) * rng.uniform(0.5, 1.5, size=len(dcn))
        vals = []
        for sign in (1.0, -1.0):
            r2 = rho + sign * hstep * torch.tensor(v, device="cuda")
            h.build_elements(r2, mat, mto.MTO_FP64)
            u.copy_(u0)
            h.solve(f, u, precision=mto.MTO_FP64, rtol=1e-8, max_iter=40000, warm_start=True, precond=mto.PREC_MG)
            vals.append(2.0 * float(f @ u) - element_energy(mto, h, u, f, r2, mat, work, pr))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        want = float(dcn @ v)
        errs.append(abs(fd - want) / abs(want))
    assert max(errs) < 1e-5, errs
