"""Pieces of the dp-adaptive TO cycle around the hot path (Sec. 3.3, Sec. 4.1) that the paper
leaves to the reader (test infrastructure only).

* Design transfer when an element's design count changes (the paper does not say how the design
  variables move to the new design points).  Reading: each new subcell takes the area-weighted
  mean of the old subcells it overlaps (both are constant-density squares of the same element),
  which keeps every element's material volume and reproduces unchanged and nested layouts exactly.
* The cycle's stopping rule (Sec. 4.1): the k-th cycle stops when the change of the objective
  between two consecutive iterations falls below Delta J_1 gamma^(k - 1), Delta J_1 = 0.04,
  gamma = 0.6.  Reading: the absolute change |J_i - J_{i-1}| (the paper speaks of a change in
  objective value).
"""
import numpy as np


def overlap_1d(n_new, n_old):
    """O[i, k] = length of [i/n_new, (i+1)/n_new] intersected with [k/n_old, (k+1)/n_old]."""
    O = np.zeros((n_new, n_old))
    for i in range(n_new):
        a0, a1 = i / n_new, (i + 1) / n_new
        for k in range(n_old):
            b0, b1 = k / n_old, (k + 1) / n_old
            O[i, k] = max(0.0, min(a1, b1) - max(a0, b0))
    return O


def transfer_design(d_old, rho_old, d_new):
    """Packed design values for the per-element design counts d_new from those for d_old:
    new subcell (i, j) = sum over old (k, l) of overlap_x(i, k) overlap_y(j, l) rho_old(k, l),
    divided by the new subcell's area (1 / d_new^2 of the element); an element whose count is
    unchanged keeps its values as they are."""
    d_old = np.asarray(d_old)
    d_new = np.asarray(d_new)
    off_old = np.concatenate([[0], np.cumsum(d_old.astype(np.int64) ** 2)])
    out = []
    for e in range(len(d_old)):
        do, dn = int(d_old[e]), int(d_new[e])
        old = np.asarray(rho_old[off_old[e]:off_old[e + 1]]).reshape(do, do)   # [l (y), k (x)]
        if dn == do:   # unchanged layout: the values themselves (no rounding of the weights)
            out.append(old.ravel().copy())
            continue
        O = overlap_1d(dn, do)
        new = np.zeros((dn, dn))
        for j in range(dn):
            for i in range(dn):
                acc = 0.0
                for l in range(do):
                    for k in range(do):
                        acc += O[i, k] * O[j, l] * old[l, k]
                new[j, i] = acc * dn * dn
        out.append(new.ravel())
    return np.concatenate(out)


def cycle_converged(J_prev, J_cur, cycle, dJ1=0.04, gamma=0.6):
    """Stopping rule of cycle `cycle` (from 1): |J_cur - J_prev| < dJ1 * gamma^(cycle - 1)."""
    return abs(J_cur - J_prev) < dJ1 * gamma ** (cycle - 1)
