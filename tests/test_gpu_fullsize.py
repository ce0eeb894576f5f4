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


def _ties(values, cuts, band):
    """Elements whose value lies within ``band`` of any cut-off (ambiguous decisions)."""
    v = np.asarray(values)
    out = np.zeros(v.shape, dtype=bool)
    for c in cuts:
        out |= np.abs(v - c) <= band
    return out


@pytest.mark.parametrize("name", ["mbb_160x80_p3_d8", "dp_cantilever_320x160"])
def test_fullsize_indicators_and_maps(mto, name):
    """Step (d) at full size on the GPU's own solved u (the bench's mixed solve): the oracle
    evaluates Kelly, the density indicator and the QR error on the same u for every element, and
    its map update on its own indicator values.  Gamma^a within 1e-9 relative, Gamma^d within
    1e-15, eps^QR within 1e-6 (its element problems reach condition numbers of ~1e10); p_new,
    d_new and theta bit-exact.  Guard band: an element whose
    indicator lies within the comparison tolerance of a decision cut-off (the Gamma^a values at the
    two rank boundaries, Gamma^d = 0, eps = alpha_QR = 0.9) could be decided either way by two
    correct FP64 evaluations; the count of such elements is reported and must be 0 on these seeded
    workloads (it is)."""
    c = full_case(mto, name)
    pr, m, h = c["pr"], c["m"], c["h"]
    h.build_elements(c["rho"], c["mat"], mto.MTO_MIXED)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(c["gf"], u, precision=mto.MTO_MIXED, rtol=BENCH_RTOL, max_iter=400000, precond=mto.PREC_MG)
    ind = h.indicator(u, c["rho"], c["mat"])
    un = u.cpu().numpy()
    ga = oi.kelly(m, un)
    gd = oi.gamma_d(m, pr.rho)
    eq = oi.qr_error(m, un, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)
    np.testing.assert_allclose(ind["gamma_a"].cpu().numpy(), ga, rtol=1e-9, atol=1e-12 * np.abs(ga).max())
    np.testing.assert_allclose(ind["gamma_d"].cpu().numpy(), gd, rtol=0, atol=1e-15)
    # eps = 1 - J^p / J^(p+1) of element problems whose condition reaches ~1e10 (solid/void
    # elements): two FP64 evaluations agree to ~1e-16 x 1e10 = 1e-6
    np.testing.assert_allclose(ind["eps_qr"].cpu().numpy(), eq, rtol=0, atol=1e-6)
    # guard band (1e-12 relative): the decisions are the two rank boundaries of Gamma^a, the sign
    # of Gamma^d and eps > 0.9; an element within the band of a cut-off is a tie, reported with
    # its neighbour across the boundary, and expected nowhere on these seeded workloads
    nel = m.nel
    order = np.argsort(ga, kind="stable")
    srt = ga[order]
    nc, nr = int(np.floor(0.05 * nel)), int(np.floor(0.10 * nel))
    ties = []
    for k in (nc, nel - nr):
        if srt[k] - srt[k - 1] <= 1e-12 * abs(srt[k]):
            ties.append(("Gamma^a rank", int(order[k - 1]), int(order[k]), srt[k - 1], srt[k]))
    ties += [("Gamma^d sign", int(e), gd[e]) for e in np.flatnonzero((gd != 0) & (np.abs(gd) <= 1e-12 * np.abs(gd).max()))]
    ties += [("eps 0.9", int(e), eq[e]) for e in np.flatnonzero(np.abs(eq - 0.9) <= 1e-6)]
    print(f"{name}: ties {ties}")
    pn, dn, th = oi.map_update(pr.nelx, pr.nely, pr.p, ga, gd, eq)
    np.testing.assert_array_equal(ind["p_new"].cpu().numpy(), pn)
    np.testing.assert_array_equal(ind["d_new"].cpu().numpy(), dn)
    np.testing.assert_array_equal(ind["theta"].cpu().numpy(), th)
    assert not ties, ties


def element_energy(mto, h, u, f, rho, mat, dc, pr):
    """u^T K(rho) u as sum_s E(rho_s) w_s with w_s = -dc_s / E'(rho_s) from the sensitivity kernel
    (element-wise, after the rigid-motion removal: free of the cancellation that a global
    u^T (K u) suffers on compliant designs)."""
    h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64, want_C=False)
    r = rho.cpu().numpy()
    E = oe.simp(r, pr.E0, pr.Emin, pr.q)
    dE = oe.simp_deriv(r, pr.E0, pr.Emin, pr.q)
    return float(np.sum(E * (-dc.cpu().numpy() / dE)))


def abs_energy(m, pr, un):
    """sum_e |u_e|^T |K_e| |u_e| (oracle element matrices): the scale of the rounding errors of any
    evaluation of u^T K u as a sum of element terms."""
    tot = 0.0
    for e in range(m.nel):
        p, d = int(m.p[e]), int(m.d[e])
        Ke = oe.element_stiffness(osv.K0_table(p, d, pr.nu), oe.simp(
            pr.rho[m.design_off[e]:m.design_off[e + 1]], pr.E0, pr.Emin, pr.q))
        ue = np.abs(m.gather(e, un))
        tot += ue @ (np.abs(Ke) @ ue)
    return tot


# rounding of an FP64 evaluation of u^T K u as element sums: each element term sums n_e^2 <= 72^2
# products, the element terms are added in blocks; 256 eps bounds the accumulated relative error
# of those sums with room to spare (n_e + log2 of the term count is below 100 here)
ENERGY_EPS = 256 * np.finfo(np.float64).eps


def test_fullsize_energy_split(mto):
    """dp-adaptive cantilever (smooth densities, all E' > 0): sum_s E_s w_s with
    w_s = -dc_s / E'(rho_s) from the sensitivity kernel equals u^T K u from the operator, within
    the rounding bound of the two evaluations: 256 eps sum_e |u_e|^T |K_e| |u_e|."""
    c = full_case(mto, "dp_cantilever_320x160")
    pr, h, m = c["pr"], c["h"], c["m"]
    f, rho, mat = c["gf"], c["rho"], c["mat"]
    h.build_elements(rho, mat, mto.MTO_FP64)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(f, u, precision=mto.MTO_FP64, rtol=1e-8, max_iter=40000, precond=mto.PREC_MG)
    dc = torch.zeros(h.design_len, dtype=torch.float64, device="cuda")
    scratch = torch.zeros_like(u)
    h.apply(u, scratch)
    uKu = float(u @ scratch)
    assert np.all(oe.simp_deriv(pr.rho, pr.E0, pr.Emin, pr.q) > 0)
    eK = element_energy(mto, h, u, f, rho, mat, dc, pr)
    bound = ENERGY_EPS * abs_energy(m, pr, u.cpu().numpy())
    assert abs(eK - uKu) <= bound, (eK, uKu, bound)


def test_fullsize_autograd_fd_50_points(mto):
    """The adjoint gradient of the differentiable compliance (``compliance(...).backward()``) on the
    dp-adaptive cantilever against central finite differences at h = 1e-6 on 50 seeded design
    values drawn with probability proportional to |dC/drho| (so that h |dc| stands far above the
    rounding of C).  Each perturbed compliance is the energy functional 2 f^T u - u^T K u of an
    FP64 solve warm-started from the unperturbed u (exact at the solution, second order in the
    solve error).  Tolerance per point: the rounding bound of the two energy evaluations divided
    by 2h (2 x 256 eps sum_e |u_e|^T |K_e| |u_e| / 2h) plus the stated 1e-6 relative accuracy of
    dC/drho."""
    c = full_case(mto, "dp_cantilever_320x160")
    pr, h, m = c["pr"], c["h"], c["m"]
    f, rho, mat = c["gf"], c["rho"], c["mat"]
    r = rho.clone().requires_grad_(True)
    C = mto.compliance(h, r, f, mat, precision=mto.MTO_MIXED, rtol=1e-12, norm=mto.NORM_ENERGY,
                       max_iter=200000, precond=mto.PREC_MG)
    C.backward()
    g = r.grad.cpu().numpy()
    h.build_elements(rho, mat, mto.MTO_FP64)
    u0 = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(f, u0, precision=mto.MTO_FP64, rtol=1e-13, norm=mto.NORM_ENERGY, max_iter=200000,
            precond=mto.PREC_MG)
    rng = np.random.default_rng(181109821 + 3)
    w = np.abs(g) / np.abs(g).sum()
    pts = rng.choice(len(g), 50, replace=False, p=w)
    hstep = 1e-6
    round_C = ENERGY_EPS * abs_energy(m, pr, u0.cpu().numpy())
    u = torch.zeros_like(u0)
    work = torch.zeros_like(rho)
    worst = 0.0
    for s in pts:
        vals = []
        for sign in (1.0, -1.0):
            r2 = rho.clone()
            r2[int(s)] += sign * hstep
            h.build_elements(r2, mat, mto.MTO_FP64)
            u.copy_(u0)
            h.solve(f, u, precision=mto.MTO_FP64, rtol=1e-14, norm=mto.NORM_ENERGY, max_iter=20000,
                    warm_start=True, precond=mto.PREC_MG, raise_on_noconv=False)
            vals.append(2.0 * float(f @ u) - element_energy(mto, h, u, f, r2, mat, work, pr))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        tol = 2 * round_C / (2 * hstep) + 1e-6 * abs(g[s])
        assert abs(fd - g[s]) <= tol, (int(s), fd, g[s], tol)
        worst = max(worst, abs(fd - g[s]) / abs(g[s]))
    print(f"worst relative FD deviation over 50 points: {worst:.2e}")
