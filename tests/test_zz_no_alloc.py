"""mto_compliance_noalloc (an entry point with no counterpart in the paper): the compliance
C = f^T u with block partials in a fixed device array instead of allocated workspace.  Checked
against the compliance mto_sensitivity reports for the same solved displacement, on two calls in a
row (bit-identical to each other), plus its size limit and the empty case."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W

MAX_N = 8192 * 2048


@pytest.fixture(scope="module")
def mto():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_09821_gb300 as m
    from paper_1811_09821_gb300 import _build
    _build.build()
    m.load_library()
    return m


def call(mto, f, u, n, out):
    return mto.compliance_noalloc(f, u, out, n=n)


@pytest.mark.parametrize("name", ["cantilever_20x10_p2_d4", "mbb_160x80_p3_d8"])
def test_noalloc_compliance_matches_sensitivity(mto, name):
    pr = W.named(name)
    h = mto.Handle(0)
    h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f = mto.load_case(h, pr.load)
    h.set_supports(fixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    rho = torch.tensor(pr.rho, dtype=torch.float64, device="cuda")
    h.build_elements(rho, mat, mto.MTO_FP64)
    u = torch.zeros(h.ndof, dtype=torch.float64, device="cuda")
    h.solve(f, u, rtol=1e-8, max_iter=400000, precond=mto.PREC_MG)
    dc = torch.zeros(h.design_len, dtype=torch.float64, device="cuda")
    C_ref = h.sensitivity(u, f, rho, mat, dc)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert call(mto, f, u, h.ndof, out[0:]) == 0
    assert call(mto, f, u, h.ndof, out[1:]) == 0
    torch.cuda.synchronize()
    c1, c2 = out.cpu().tolist()
    assert c1 == c2                       # same n: same partition and summation order
    assert abs(c1 - C_ref) <= 1e-13 * abs(C_ref), (c1, C_ref)
    assert abs(c1 - float(f.cpu().numpy() @ u.cpu().numpy())) <= 1e-13 * abs(C_ref)
    h.close()


def test_noalloc_limits(mto):
    f = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert call(mto, f, f, 0, out) == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
    assert call(mto, f, f, 4, out) == 0
    torch.cuda.synchronize()
    assert out.item() == 4.0
    # beyond the scratch: refused by the library before any launch (the pointers are never read);
    # the binding's own checks refuse n beyond the tensors first
    L = mto.load_library()
    import ctypes
    st = torch.cuda.current_stream(0).cuda_stream
    for n in (MAX_N + 1, -1):
        assert L.mto_compliance_noalloc(0, f.data_ptr(), f.data_ptr(), n, ctypes.c_void_p(st), out.data_ptr()) == 1
    with pytest.raises(ValueError):
        call(mto, f, f, 5, out)
    with pytest.raises(ValueError):
        call(mto, f.float(), f, 4, out)
