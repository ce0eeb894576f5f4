"""The dp-adaptive TO cycle (Sec. 3.3, Sec. 4.1) as a sequence of the library's calls.

Each cycle k = 1, 2, ... runs optimality-criteria iterations on the current (p, d) maps until the
objective changes by less than Delta J_1 gamma^(k-1) between two consecutive iterations (Sec. 4.1:
Delta J_1 = 0.04, gamma = 0.6; read as the absolute change), then evaluates the composite indicator
and the map update (mto_indicator) on the last solved state, sets the handle up on the new maps and
moves the design to the new design points (mto_transfer_design).  Every numerical step runs in the
library's kernels; this module only sequences the calls and compares the objective values the
library returns.

With a filter radius the build takes the P2-filtered densities (mto_filter, Sec. 2.1), the
sensitivities pass back through mto_filter_adjoint, and the indicators see the filtered (physical)
densities that the solved displacement belongs to.
"""
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (MTO_FP64, MTO_MIXED, NORM_ENERGY, PREC_MG, Handle, IndicatorOpts, load_case, material)


@dataclass
class Cycle:
    cycle: int
    ndof: int
    free_dofs: int
    design_points: int
    iterations: int
    J: list                      # objective after each solve of the cycle
    pcg_iterations: int
    p: np.ndarray                # maps the cycle ran on
    d: np.ndarray
    p_new: np.ndarray = None     # maps for the next cycle
    d_new: np.ndarray = None
    state: dict = field(default_factory=dict)   # device tensors of the last solved state (keep=True)


def converged(J_prev, J_cur, cycle, dJ1=0.04, gamma=0.6):
    """The cycle's stopping rule: |J_cur - J_prev| < dJ1 gamma^(cycle - 1)."""
    return abs(J_cur - J_prev) < dJ1 * gamma ** (cycle - 1)


def run(nelx, nely, p, d, rho, load, volfrac, cycles=4, max_iters=60, radius=0.0, precision=MTO_MIXED,
        rtol=1e-9, dJ1=0.04, gamma=0.6, move=0.2, eta=0.5, mat=None, device=0, keep=False, p_max=5, d_max=64):
    """dp-adaptive compliance minimisation.  rho: initial packed design (numpy) for the maps p, d.
    Each solve is warm-started and stops at the relative compliance accuracy rtol
    (MTO_NORM_ENERGY); J is the compliance in its energy form (mto_compliance_energy).
    Returns the list of Cycle records; with keep=True each record holds the cycle's last state
    (u, rho, filtered rho, f) as device tensors."""
    mat = mat or material()
    dev = torch.device("cuda", device)
    h = Handle(device)
    p = np.asarray(p, dtype=np.int32).copy()
    d = np.asarray(d, dtype=np.int32).copy()
    rho_t = torch.tensor(np.asarray(rho, dtype=np.float64), device=dev)
    out = []
    for k in range(1, cycles + 1):
        ndof, dlen = h.setup(nelx, nely, p, d)
        fixed, f = load_case(h, load)
        h.set_supports(fixed)
        u = torch.zeros(ndof, dtype=torch.float64, device=dev)
        dc_f = torch.zeros(dlen, dtype=torch.float64, device=dev)
        dc = torch.zeros(dlen, dtype=torch.float64, device=dev)
        rho_f = torch.empty_like(rho_t) if radius > 0 else rho_t
        rho_new = torch.empty_like(rho_t)
        J, its, pcg = [], 0, 0
        while True:
            if radius > 0:
                h.filter(rho_t, rho_f, radius)
            h.build_elements(rho_f, mat, precision)
            it, _ = h.solve(f, u, precision=precision, rtol=rtol, norm=NORM_ENERGY, max_iter=400000,
                            check_every=16, precond=PREC_MG, warm_start=its > 0)
            pcg += it
            h.sensitivity(u, f, rho_f, mat, dc_f, precision=MTO_FP64, want_C=False)
            J.append(h.compliance_energy(u, f, rho_f, mat))
            if len(J) > 1 and converged(J[-2], J[-1], k, dJ1, gamma):
                break
            if its >= max_iters:
                break
            if radius > 0:
                h.filter_adjoint(dc_f, dc, radius)
            else:
                dc.copy_(dc_f)
            h.oc_update(rho_t, dc, volfrac, rho_new, move=move, eta=eta, want_lambda=False)
            rho_t, rho_new = rho_new, rho_t
            if radius == 0:
                rho_f = rho_t
            its += 1
        ind = h.indicator(u, rho_f, mat, IndicatorOpts.paper(k) if (p_max, d_max) == (5, 64) else
                          _opts(k, p_max, d_max))
        rec = Cycle(k, ndof, ndof - len(fixed), dlen, its, J, pcg, p.copy(), d.copy(),
                    ind["p_new"].cpu().numpy(), ind["d_new"].cpu().numpy())
        if keep:
            rec.state = dict(u=u.clone(), rho=rho_t.clone(), rho_f=rho_f.clone(), f=f.clone(),
                             indicators={kk: (v.clone() if v is not None else None) for kk, v in ind.items()})
        out.append(rec)
        if k == cycles:
            break
        d_old = d
        p, d = rec.p_new.astype(np.int32), rec.d_new.astype(np.int32)
        rho_old = rho_t
        ndof, dlen = h.setup(nelx, nely, p, d)
        rho_t = torch.empty(dlen, dtype=torch.float64, device=dev)
        h.transfer_design(d_old, rho_old, rho_t)
        if keep:
            rec.state["rho_next"] = rho_t.clone()
    h.close()
    return out


def _opts(k, p_max, d_max):
    o = IndicatorOpts.paper(k)
    o.p_max, o.d_max = p_max, d_max
    return o
