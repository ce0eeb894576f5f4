"""GB300 (sm_103a) hot path of dp-adaptive multi-resolution topology optimization
(Gupta, van Keulen, Langelaar, arXiv:1811.09821): element build, matrix-free PCG solve,
compliance sensitivities and the composite refinement indicator, as CUDA kernels behind the C ABI
of ``include/mto.h`` (``libmto.so``).

This module is the thin Python binding: it marshals arguments (torch CUDA tensors for device
memory, numpy arrays for host maps) into the C calls of the same names.  Every step of the path
runs in the library's kernels; there is no CPU fallback, and importing this package raises when
``libmto.so`` cannot be loaded.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmto.so")

MTO_FP64, MTO_MIXED, MTO_MIXED32 = 0, 1, 2
NORM_L2, NORM_JACOBI, NORM_ENERGY = 0, 1, 2
BUILD_TENSOR, BUILD_SIMT = 0, 1
OP_FP64, OP_SPLIT, OP_LEAD = 0, 1, 2
OPK_AUTO, OPK_PIPE, OPK_STAGED, OPK_GENERIC = -1, 0, 1, 2
PREC_JACOBI, PREC_SCHWARZ, PREC_MG = 0, 1, 2
SMOOTH_JACOBI, SMOOTH_BLOCK = 0, 1
MG_OP_AUTO, MG_OP_SPLIT, MG_OP_LEAD = 0, 1, 2
STATUS = {0: "MTO_OK", 1: "MTO_EINVAL", 2: "MTO_ENOMEM", 3: "MTO_ECUDA", 4: "MTO_ENOCONV", 5: "MTO_ENAN",
          6: "MTO_ETIMEOUT"}
P_MAX, D_MAX = 6, 16
MTO_P_MAX_NODES = P_MAX + 2


class MTOError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(ctypes.Structure):
    """Material of Eq. 3 / Sec. 4.1 (plane stress)."""
    _fields_ = [("E0", ctypes.c_double), ("Emin", ctypes.c_double), ("nu", ctypes.c_double), ("q", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rtol", ctypes.c_double), ("inner_rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("norm", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("inner_max", ctypes.c_int32), ("mg_degree", ctypes.c_int32), ("mg_smoother", ctypes.c_int32),
                ("mg_operator", ctypes.c_int32)]


class IndicatorOpts(ctypes.Structure):
    """Sec. 3.2 / 3.3 parameters; defaults are the paper's values."""
    _fields_ = [("cycle", ctypes.c_int32), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("frac_a_refine", ctypes.c_double), ("frac_a_coarsen", ctypes.c_double),
                ("alpha_d_refine", ctypes.c_double), ("alpha_d_coarsen", ctypes.c_double),
                ("alpha_qr", ctypes.c_double), ("p_max", ctypes.c_int32), ("d_max", ctypes.c_int32)]

    @classmethod
    def paper(cls, cycle=1):
        return cls(cycle, 0.2, 0.8, 0.10, 0.05, 1.0, 1.0, 0.9, 5, 64)


# every symbol declared in include/mto.h
SYMBOLS = ["mto_create", "mto_destroy", "mto_last_error", "mto_set_stream", "mto_setup", "mto_set_supports",
           "mto_vertex_dof", "mto_side_dofs", "mto_element_nodes", "mto_element_matrix", "mto_build_elements", "mto_solve", "mto_apply",
           "mto_sensitivity", "mto_indicator", "mto_map_update", "mto_oc_update", "mto_timing_enable", "mto_timing_read",
           "mto_set_build_path",
           "mto_memory", "mto_launch_count", "mto_compliance_noalloc", "mto_compliance", "mto_apply_operator",
           "mto_set_operator_kernel", "mto_element_matrix_split", "mto_edge_dofs", "mto_side_load",
           "mto_set_springs", "mto_sensitivity_adjoint", "mto_side_dofs_in",
           "mto_filter", "mto_filter_adjoint", "mto_transfer_design", "mto_compliance_energy",
           "mto_autotune", "mto_build_elements_batched", "mto_solve_batched", "mto_sensitivity_batched"]
TIME_FAMILIES = {"apply32": 0, "apply64": 1, "build": 2, "sens": 3, "indicator": 4, "vector": 5, "applydf64": 6,
                 "precond": 7, "oc": 8, "applylead": 9}

_lib = None


def load_library(path=LIB_PATH):
    """Load libmto.so and declare its signatures.  Raises OSError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "mto_create": ([P(vp), ctypes.c_int, vp], ctypes.c_int),
        "mto_destroy": ([vp], ctypes.c_int),
        "mto_last_error": ([vp], ctypes.c_char_p),
        "mto_set_stream": ([vp, vp], ctypes.c_int),
        "mto_setup": ([vp, i32, i32, dbl, dbl, P(i32), P(i32), P(i64), P(i64)], ctypes.c_int),
        "mto_set_supports": ([vp, P(i64), i64], ctypes.c_int),
        "mto_vertex_dof": ([vp, i32, i32, i32, P(i64)], ctypes.c_int),
        "mto_side_dofs": ([vp, i32, i32, P(i64), i64, P(i64)], ctypes.c_int),
        "mto_element_nodes": ([vp, i64, P(i64), P(dbl), P(i32)], ctypes.c_int),
        "mto_element_matrix": ([vp, i64, P(dbl)], ctypes.c_int),
        "mto_build_elements": ([vp, vp, P(Material), i32], ctypes.c_int),
        "mto_solve": ([vp, vp, vp, P(SolveOpts), P(i32), P(dbl)], ctypes.c_int),
        "mto_apply": ([vp, vp, vp], ctypes.c_int),
        "mto_sensitivity": ([vp, vp, vp, vp, P(Material), i32, vp, P(dbl)], ctypes.c_int),
        "mto_indicator": ([vp, vp, vp, P(Material), P(IndicatorOpts), vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "mto_map_update": ([vp, vp, vp, vp, P(IndicatorOpts), vp, vp, vp], ctypes.c_int),
        "mto_oc_update": ([vp, vp, vp, dbl, dbl, dbl, vp, P(dbl)], ctypes.c_int),
        "mto_timing_enable": ([vp, i32], ctypes.c_int),
        "mto_set_build_path": ([vp, i32], ctypes.c_int),
        "mto_timing_read": ([vp, i32, P(i64), P(dbl)], ctypes.c_int),
        "mto_memory": ([vp, P(i64)], ctypes.c_int),
        "mto_launch_count": ([vp, P(i64)], ctypes.c_int),
        "mto_compliance_noalloc": ([i32, vp, vp, i64, vp, vp], ctypes.c_int),
        "mto_compliance": ([vp, vp, vp, vp, P(dbl)], ctypes.c_int),
        "mto_edge_dofs": ([vp, i32, i32, i32, i32, P(i64), i64, P(i64)], ctypes.c_int),
        "mto_side_load": ([vp, i32, i32, dbl, vp], ctypes.c_int),
        "mto_set_springs": ([vp, P(i64), P(dbl), i64], ctypes.c_int),
        "mto_side_dofs_in": ([vp, i32, i32, dbl, dbl, P(i64), i64, P(i64)], ctypes.c_int),
        "mto_filter": ([vp, dbl, vp, vp], ctypes.c_int),
        "mto_transfer_design": ([vp, P(i32), vp, vp], ctypes.c_int),
        "mto_compliance_energy": ([vp, vp, vp, vp, P(Material), P(dbl)], ctypes.c_int),
        "mto_autotune": ([vp, P(i32), P(dbl)], ctypes.c_int),
        "mto_build_elements_batched": ([P(vp), i32, P(vp), P(Material), i32], ctypes.c_int),
        "mto_solve_batched": ([P(vp), i32, P(vp), P(vp), P(SolveOpts), P(i32), P(dbl), P(i32)], ctypes.c_int),
        "mto_sensitivity_batched": ([P(vp), i32, P(vp), P(vp), P(vp), P(Material), P(vp), P(dbl)], ctypes.c_int),
        "mto_filter_adjoint": ([vp, dbl, vp, vp], ctypes.c_int),
        "mto_sensitivity_adjoint": ([vp, vp, vp, vp, P(Material), vp], ctypes.c_int),
        "mto_apply_operator": ([vp, i32, vp, vp, P(dbl)], ctypes.c_int),
        "mto_set_operator_kernel": ([vp, i32], ctypes.c_int),
        "mto_element_matrix_split": ([vp, i64, P(ctypes.c_float), P(ctypes.c_float)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """One problem instance on one CUDA device: owns the numbering, element matrices and workspace."""

    def __init__(self, device=0, stream=None):
        self.L = load_library()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._check(self.L.mto_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self.ndof = self.design_len = None

    def _check(self, status):
        if status != 0:
            msg = self.L.mto_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise MTOError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.mto_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- mesh and supports
    def setup(self, nelx, nely, p, d, hx=1.0, hy=1.0):
        self.hx, self.hy = hx, hy
        p = np.ascontiguousarray(p, dtype=np.int32)
        d = np.ascontiguousarray(d, dtype=np.int32)
        nd, dl = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.L.mto_setup(self.h, nelx, nely, hx, hy, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(nd),
                                     ctypes.byref(dl)))
        self.nelx, self.nely, self.nel = nelx, nely, nelx * nely
        self.ndof, self.design_len = nd.value, dl.value
        return self.ndof, self.design_len

    def set_supports(self, fixed):
        fixed = np.ascontiguousarray(fixed, dtype=np.int64)
        self._check(self.L.mto_set_supports(self.h, fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            len(fixed)))

    def set_springs(self, dofs, k):
        """Springs to ground k_i at global DOFs dofs_i (operator K + sum k_i e e^T)."""
        dofs = np.ascontiguousarray(dofs, dtype=np.int64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        self._check(self.L.mto_set_springs(self.h, dofs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(dofs)))

    def vertex_dof(self, ix, iy, comp):
        out = ctypes.c_int64()
        self._check(self.L.mto_vertex_dof(self.h, ix, iy, comp, ctypes.byref(out)))
        return out.value

    def side_dofs(self, side, comp=-1):
        n = ctypes.c_int64()
        self._check(self.L.mto_side_dofs(self.h, side, comp, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self.L.mto_side_dofs(self.h, side, comp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         n.value, ctypes.byref(n)))
        return out

    def side_dofs_in(self, side, comp, s0, s1):
        """side_dofs restricted to nodes whose coordinate along the side lies in [s0, s1]."""
        n = ctypes.c_int64()
        self._check(self.L.mto_side_dofs_in(self.h, side, comp, s0, s1, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self.L.mto_side_dofs_in(self.h, side, comp, s0, s1,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n.value,
                                            ctypes.byref(n)))
        return out

    def edge_dofs(self, direction, ix, iy, comp):
        """DOFs (component comp) of the nodes of mesh edge (direction 0: horizontal from vertex
        (ix, iy); 1: vertical), in parameter order."""
        n = ctypes.c_int64()
        out = np.zeros(MTO_P_MAX_NODES, dtype=np.int64)
        self._check(self.L.mto_edge_dofs(self.h, direction, ix, iy, comp,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(out),
                                         ctypes.byref(n)))
        return out[:n.value].copy()

    def side_load(self, side, comp, traction, f):
        """f += consistent nodal loads of a uniform traction on one side (device float64 [ndof])."""
        self._check(self.L.mto_side_load(self.h, side, comp, traction, _ptr(f, torch.float64)))
        return f

    def element_nodes(self, e):
        """Per local node of element e: list of (global node, weight) (minimum-rule map)."""
        m = (P_MAX + 1) ** 2
        nodes = np.zeros(m * 8, dtype=np.int64)
        w = np.zeros(m * 8)
        c = np.zeros(m, dtype=np.int32)
        self._check(self.L.mto_element_nodes(self.h, e, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                             w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        out = []
        for ln in range(m):
            if c[ln] == 0:
                break
            out.append([(int(nodes[ln * 8 + k]), float(w[ln * 8 + k])) for k in range(c[ln])])
        return out

    def element_matrix(self, e, p):
        """Packed upper triangle of element e's current matrix (numpy, n_e (n_e + 1) / 2)."""
        ne = 2 * (p + 1) ** 2
        out = np.zeros(ne * (ne + 1) // 2)
        self._check(self.L.mto_element_matrix(self.h, e, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    # ---------------------------------------------------------------- the four steps
    def build_elements(self, rho, mat, precision=MTO_FP64):
        self._check(self.L.mto_build_elements(self.h, _ptr(rho, torch.float64), ctypes.byref(mat), precision))

    def solve(self, f, u, precision=MTO_FP64, rtol=1e-8, inner_rtol=0.0, max_iter=200000, max_outer=50,
              warm_start=False, check_every=64, norm=NORM_L2, precond=PREC_SCHWARZ, inner_max=0,
              mg_degree=0, mg_smoother=SMOOTH_JACOBI, mg_operator=MG_OP_AUTO, raise_on_noconv=True):
        o = SolveOpts(precision, rtol, inner_rtol, max_iter, max_outer, int(bool(warm_start)), check_every, norm,
                      precond, inner_max, mg_degree, mg_smoother, mg_operator)
        it, rr = ctypes.c_int32(), ctypes.c_double()
        st = self.L.mto_solve(self.h, _ptr(f, torch.float64), _ptr(u, torch.float64), ctypes.byref(o),
                              ctypes.byref(it), ctypes.byref(rr))
        if st != 0 and not (st == 4 and not raise_on_noconv):
            self._check(st)
        return it.value, rr.value

    def apply(self, x, y):
        self._check(self.L.mto_apply(self.h, _ptr(x, torch.float64), _ptr(y, torch.float64)))

    def apply_operator(self, x, y, op=OP_FP64, want_xKx=True):
        """y = K x with the FP64 matrices (OP_FP64), the split-precision pair (OP_SPLIT, the inner
        PCG's kernels) or the pair's FP32 leading part (OP_LEAD, the multigrid cycle's copy); returns
        x^T K x as the launches reduce it (or None)."""
        v = ctypes.c_double()
        self._check(self.L.mto_apply_operator(self.h, op, _ptr(x, torch.float64), _ptr(y, torch.float64),
                                              ctypes.byref(v) if want_xKx else None))
        return v.value if want_xKx else None

    def autotune(self):
        """Time the split operator's kernels per order class and keep the fastest; returns
        {p: (chosen kernel, [us pipe, us staged, us generic])} for the tuned classes."""
        ch = np.zeros(P_MAX + 1, np.int32)
        us = np.zeros(3 * (P_MAX + 1))
        self._check(self.L.mto_autotune(self.h, ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        us.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return {p: (int(ch[p]), us[3 * p:3 * p + 3].tolist()) for p in range(1, P_MAX + 1) if ch[p] >= -1}

    def set_operator_kernel(self, kernel):
        self._check(self.L.mto_set_operator_kernel(self.h, kernel))

    def element_matrix_split(self, e, p):
        """(hi, lo) packed upper triangles (float32) of element e's split-precision pair."""
        ne = 2 * (p + 1) ** 2
        P = ne * (ne + 1) // 2
        hi, lo = np.zeros(P, np.float32), np.zeros(P, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self.L.mto_element_matrix_split(self.h, e, hi.ctypes.data_as(fp), lo.ctypes.data_as(fp)))
        return hi, lo

    def compliance_energy(self, u, f, rho, mat):
        """C(u) = 2 f^T u - u^T K(rho) u from element energies (second-order accurate in u's error)."""
        C = ctypes.c_double()
        self._check(self.L.mto_compliance_energy(self.h, _ptr(u, torch.float64), _ptr(f, torch.float64),
                                                 _ptr(rho, torch.float64), ctypes.byref(mat), ctypes.byref(C)))
        return C.value

    def compliance(self, f, u, out=None):
        """C = f^T u in the handle's workspace: into the device scalar ``out`` (asynchronous) when
        given, else returned as a float."""
        if out is not None:
            self._check(self.L.mto_compliance(self.h, _ptr(f, torch.float64), _ptr(u, torch.float64),
                                              _ptr(out, torch.float64), None))
            return out
        C = ctypes.c_double()
        self._check(self.L.mto_compliance(self.h, _ptr(f, torch.float64), _ptr(u, torch.float64), None,
                                          ctypes.byref(C)))
        return C.value

    def sensitivity(self, u, f, rho, mat, dc, precision=MTO_FP64, want_C=True):
        C = ctypes.c_double()
        self._check(self.L.mto_sensitivity(self.h, _ptr(u, torch.float64), _ptr(f, torch.float64),
                                           _ptr(rho, torch.float64), ctypes.byref(mat), precision,
                                           _ptr(dc, torch.float64), ctypes.byref(C) if want_C else None))
        return C.value if want_C else None

    def transfer_design(self, d_old, rho_old, rho_new):
        """rho_new (packed for the current maps) from rho_old packed for the per-element counts d_old."""
        d_old = np.ascontiguousarray(d_old, dtype=np.int32)
        self._check(self.L.mto_transfer_design(self.h, d_old.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                               _ptr(rho_old, torch.float64), _ptr(rho_new, torch.float64)))
        return rho_new

    def filter(self, rho, out, radius):
        """out = P2-filtered densities of rho (Eqs. 4-5 at the subcell centres)."""
        self._check(self.L.mto_filter(self.h, radius, _ptr(rho, torch.float64), _ptr(out, torch.float64)))
        return out

    def filter_adjoint(self, g_f, out, radius):
        """out = dJ/drho from g_f = dJ/drho_f (the filter's transpose with its weight sums)."""
        self._check(self.L.mto_filter_adjoint(self.h, radius, _ptr(g_f, torch.float64), _ptr(out, torch.float64)))
        return out

    def sensitivity_adjoint(self, u, v, rho, mat, dc):
        """dJ/drho for J = z^T u with the adjoint v (K v = z): dc = -E' v_e^T K0 u_e."""
        self._check(self.L.mto_sensitivity_adjoint(self.h, _ptr(u, torch.float64), _ptr(v, torch.float64),
                                                   _ptr(rho, torch.float64), ctypes.byref(mat),
                                                   _ptr(dc, torch.float64)))
        return dc

    def indicator(self, u, rho, mat, opts=None, maps=True):
        opts = opts or IndicatorOpts.paper()
        dev = self.device
        ga = torch.empty(self.nel, dtype=torch.float64, device=dev)
        gd = torch.empty_like(ga)
        eq = torch.empty_like(ga)
        pn = torch.empty(self.nel, dtype=torch.int32, device=dev) if maps else None
        dn = torch.empty_like(pn) if maps else None
        th = torch.empty(self.nel, dtype=torch.int8, device=dev) if maps else None
        self._check(self.L.mto_indicator(self.h, _ptr(u, torch.float64), _ptr(rho, torch.float64), ctypes.byref(mat),
                                         ctypes.byref(opts), _ptr(ga), _ptr(gd), _ptr(eq), _ptr(pn), _ptr(dn),
                                         _ptr(th)))
        return dict(gamma_a=ga, gamma_d=gd, eps_qr=eq, p_new=pn, d_new=dn, theta=th)

    def map_update(self, gamma_a, gamma_d, eps_qr, opts=None):
        opts = opts or IndicatorOpts.paper()
        pn = torch.empty(self.nel, dtype=torch.int32, device=self.device)
        dn = torch.empty_like(pn)
        th = torch.empty(self.nel, dtype=torch.int8, device=self.device)
        self._check(self.L.mto_map_update(self.h, _ptr(gamma_a, torch.float64), _ptr(gamma_d, torch.float64),
                                          _ptr(eps_qr, torch.float64), ctypes.byref(opts), _ptr(pn), _ptr(dn),
                                          _ptr(th)))
        return pn, dn, th

    def oc_update(self, rho, dc, volfrac, rho_new, move=0.2, eta=0.5, want_lambda=True):
        lam = ctypes.c_double()
        self._check(self.L.mto_oc_update(self.h, _ptr(rho, torch.float64), _ptr(dc, torch.float64), volfrac, move, eta,
                                         _ptr(rho_new, torch.float64), ctypes.byref(lam) if want_lambda else None))
        return lam.value if want_lambda else None

    def set_build_path(self, path):
        self._check(self.L.mto_set_build_path(self.h, path))

    def timing_enable(self, on=True):
        """on: True (every kernel family), "sampled" (the first operator launch of each chunk of
        PCG iterations only: low overhead) or False."""
        self._check(self.L.mto_timing_enable(self.h, 2 if on == "sampled" else int(bool(on))))

    def timing_read(self):
        """{family: (kernel launches, device ms)} since the last timing_enable."""
        out = {}
        for name, fam in TIME_FAMILIES.items():
            n, ms = ctypes.c_int64(), ctypes.c_double()
            self._check(self.L.mto_timing_read(self.h, fam, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (n.value, ms.value)
        return out

    def memory(self):
        b = ctypes.c_int64()
        self._check(self.L.mto_memory(self.h, ctypes.byref(b)))
        return b.value

    def launch_count(self):
        c = ctypes.c_int64()
        self._check(self.L.mto_launch_count(self.h, ctypes.byref(c)))
        return c.value


def compliance_noalloc(f, u, out, n=None, device=0, stream=None):
    """C = f^T u over the first n entries into out[0] (device float64) through
    mto_compliance_noalloc, which allocates nothing (see include/mto.h: its fixed scratch is
    shared by every caller on a device, so overlapping calls race).  f, u and out must be
    contiguous float64 tensors on CUDA device ``device`` with n <= f.numel(), u.numel(); else
    ValueError before any library call.  Returns the library's status code."""
    n = int(f.numel() if n is None else n)
    for name, t in (("f", f), ("u", u), ("out", out)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"compliance_noalloc: {name} must be a contiguous float64 tensor")
        if not t.is_cuda or t.device.index != device:
            raise ValueError(f"compliance_noalloc: {name} must live on cuda:{device}")
    if out.numel() < 1 or n > f.numel() or n > u.numel():
        raise ValueError("compliance_noalloc: n exceeds the length of f or u, or out is empty")
    L = load_library()
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream(device).cuda_stream
    return L.mto_compliance_noalloc(device, f.data_ptr(), u.data_ptr(), n, ctypes.c_void_p(st), out.data_ptr())


def _ptrs(ts, dtype=torch.float64):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t, dtype).value
    return arr


def _handles(hs):
    arr = (ctypes.c_void_p * len(hs))()
    for i, h in enumerate(hs):
        arr[i] = h.h.value
    return arr


def _check_batch(L, hs, st):
    if st != 0:
        msgs = [h.L.mto_last_error(h.h).decode() for h in hs]
        raise MTOError(st, "; ".join(m for m in msgs if m) or "batched call failed")


def build_elements_batched(handles, rhos, mat, precision=MTO_MIXED):
    """Step (a) of every instance (asynchronous, each on its handle's stream)."""
    L = load_library()
    _check_batch(L, handles, L.mto_build_elements_batched(_handles(handles), len(handles), _ptrs(rhos),
                                                          ctypes.byref(mat), precision))


def solve_batched(handles, fs, us, precision=MTO_MIXED, rtol=1e-8, inner_rtol=0.0, max_iter=200000, max_outer=50,
                  warm_start=False, check_every=32, norm=NORM_ENERGY, precond=PREC_MG, inner_max=0, mg_degree=0,
                  mg_smoother=SMOOTH_JACOBI, mg_operator=MG_OP_AUTO, raise_on_error=True):
    """Step (b) of every instance, advanced together (mto_solve_batched).  Returns (iterations,
    relative residuals, statuses) as numpy arrays."""
    L = load_library()
    n = len(handles)
    o = SolveOpts(precision, rtol, inner_rtol, max_iter, max_outer, int(bool(warm_start)), check_every, norm,
                  precond, inner_max, mg_degree, mg_smoother, mg_operator)
    it = np.zeros(n, np.int32)
    rr = np.zeros(n)
    stt = np.zeros(n, np.int32)
    st = L.mto_solve_batched(_handles(handles), n, _ptrs(fs), _ptrs(us), ctypes.byref(o),
                             it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if raise_on_error:
        _check_batch(L, handles, st)
    return it, rr, stt


def sensitivity_batched(handles, us, fs, rhos, mat, dcs, want_C=True):
    """Step (c) of every instance; returns the compliances f^T u (numpy) when want_C."""
    L = load_library()
    n = len(handles)
    C = np.zeros(n)
    _check_batch(L, handles, L.mto_sensitivity_batched(_handles(handles), n, _ptrs(us), _ptrs(fs), _ptrs(rhos),
                                                       ctypes.byref(mat), _ptrs(dcs),
                                                       C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                       if want_C else None))
    return C if want_C else None


def load_case(handle, load):
    """Supports and load vector of a named load case, placed with the library's own numbering.

    cantilever: left edge clamped, F = -1 (y) at vertex (nelx, nely/2) (Sec. 4.1, Fig. 3a);
    cantilever_distributed: left edge clamped, a uniform downward traction of total 1 on the top
    edge (Sec. 4.1, Fig. 6a);
    mbb: u_x = 0 on the left edge, u_y = 0 at vertex (nelx, 0), F = -1 (y) at vertex (0, nely).
    Returns (fixed DOFs as numpy int64, f as a CUDA float64 tensor)."""
    nx, ny = handle.nelx, handle.nely
    f = torch.zeros(handle.ndof, dtype=torch.float64, device=handle.device)
    if load == "cantilever":
        fixed = handle.side_dofs(0, -1)
        f[handle.vertex_dof(nx, ny // 2, 1)] = -1.0
    elif load == "cantilever_distributed":
        # Sec. 4.1, Fig. 6a: F = 0.5 N/L on the 2L top edge = a total downward load of 1
        fixed = handle.side_dofs(0, -1)
        handle.side_load(3, 1, -1.0 / (nx * handle.hx), f)
    elif load == "mbb":
        fixed = np.concatenate([handle.side_dofs(0, 0), [handle.vertex_dof(nx, 0, 1)]]).astype(np.int64)
        f[handle.vertex_dof(0, ny, 1)] = -1.0
    else:
        raise ValueError(load)
    return np.sort(fixed), f


def inverter_case(handle, k_in=1.0, k_out=1e-3, f_in=1.0, clamp=0.01):
    """The force inverter of Sec. 4.1 (Fig. 6b) placed with the library's numbering: both components
    held along the left edge within clamp * L of its two corners, f_in (+x) at the mid-height vertex
    of the left edge with a spring k_in, the output u_x at the mid-height vertex of the right edge
    with a spring k_out (set on the handle).  Returns (fixed DOFs, f, z) with J = z^T u."""
    nx, ny = handle.nelx, handle.nely
    L = ny * handle.hy
    fixed = np.union1d(handle.side_dofs_in(0, -1, -1.0, clamp * L + 1e-12),
                       handle.side_dofs_in(0, -1, L - clamp * L - 1e-12, L + 1.0)).astype(np.int64)
    din, dout = handle.vertex_dof(0, ny // 2, 0), handle.vertex_dof(nx, ny // 2, 0)
    f = torch.zeros(handle.ndof, dtype=torch.float64, device=handle.device)
    z = torch.zeros_like(f)
    f[din] = f_in
    z[dout] = 1.0
    handle.set_springs([din, dout], [k_in, k_out])
    return fixed, f, z


def material(E0=1.0, Emin=1e-9, nu=0.3, q=3.0):
    return Material(E0, Emin, nu, q)


class ComplianceFn(torch.autograd.Function):
    """Compliance C(rho) = f^T u(rho) as a differentiable torch function.

    forward: mto_build_elements + mto_solve, C = f^T u by mto_compliance (a reduction in the
    handle's own workspace, on the handle's stream); keeps u.  backward: the adjoint of
    the self-adjoint compliance problem is lambda = -u, so dC/drho_s = -E'(rho_s) u_e^T K0_s u_e is
    one mto_sensitivity launch on the stored u (no per-subcell products are kept).
    Use through ``compliance(handle, rho, f, mat, ...)``."""

    @staticmethod
    def forward(ctx, rho, handle, f, mat, precision, solve_opts):
        handle.build_elements(rho, mat, precision)
        u = torch.zeros(handle.ndof, dtype=torch.float64, device=rho.device)
        handle.solve(f, u, precision=precision, **solve_opts)
        ctx.handle, ctx.mat = handle, mat
        ctx.save_for_backward(rho, f, u)
        c = torch.empty((), dtype=torch.float64, device=rho.device)
        handle.compliance(f, u, out=c)
        return c

    @staticmethod
    def backward(ctx, grad_c):
        rho, f, u = ctx.saved_tensors
        dc = torch.empty_like(rho)
        ctx.handle.sensitivity(u, f, rho, ctx.mat, dc, precision=MTO_FP64, want_C=False)
        return grad_c * dc, None, None, None, None, None


class FilterFn(torch.autograd.Function):
    """The P2 density filter (Sec. 2.1, Eqs. 4-5) as a differentiable torch function: forward
    mto_filter, backward mto_filter_adjoint (the chain rule of the sensitivities)."""

    @staticmethod
    def forward(ctx, rho, handle, radius):
        ctx.handle, ctx.radius = handle, radius
        return handle.filter(rho, torch.empty_like(rho), radius)

    @staticmethod
    def backward(ctx, g):
        return ctx.handle.filter_adjoint(g.contiguous(), torch.empty_like(g), ctx.radius), None, None


def density_filter(handle, rho, radius):
    """Differentiable P2-filtered densities of the design rho (device float64, packed)."""
    return FilterFn.apply(rho, handle, radius)


def compliance(handle, rho, f, mat, precision=MTO_MIXED, **solve_opts):
    """Differentiable compliance of the design rho (device float64, packed) on a set-up handle with
    supports: C = f^T u with K(rho) u = f; ``C.backward()`` fills ``rho.grad`` with dC/drho."""
    return ComplianceFn.apply(rho, handle, f, mat, precision, solve_opts)
