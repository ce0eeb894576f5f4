"""Pins for oracle/adaptive.py: the design transfer is the identity for unchanged counts, copies a
parent into its children and averages children into their parent for nested counts, keeps each
element's volume for any pair of counts (overlaps of 3 and 2, 5 and 8), and keeps constants; the
stopping thresholds of the first cycles are the paper's (0.04 and 0.024, Sec. 4.1)."""
import numpy as np
import pytest

from oracle.adaptive import cycle_converged, overlap_1d, transfer_design


def test_overlap_rows_and_columns():
    O = overlap_1d(3, 2)
    np.testing.assert_allclose(O.sum(axis=1), 1 / 3)
    np.testing.assert_allclose(O.sum(axis=0), 1 / 2)
    assert abs(O[1, 0] - 1 / 6) < 1e-16 and abs(O[1, 1] - 1 / 6) < 1e-16


def test_identity_nested_and_volume():
    rng = np.random.default_rng(0)
    d_old = np.array([1, 2, 4, 3, 8, 5])
    rho = rng.uniform(size=int((d_old ** 2).sum()))
    np.testing.assert_array_equal(transfer_design(d_old, rho, d_old), rho)
    # 2 -> 4: every child equals its parent; 4 -> 2: the parent is the mean of its children
    r2 = np.array([0.1, 0.2, 0.3, 0.4])
    r4 = transfer_design([2], r2, [4]).reshape(4, 4)
    np.testing.assert_allclose(r4, np.kron(r2.reshape(2, 2), np.ones((2, 2))), rtol=1e-15)
    back = transfer_design([4], r4.ravel(), [2])
    np.testing.assert_allclose(back, r2, rtol=1e-15)
    d_new = np.array([2, 1, 8, 2, 5, 8])
    out = transfer_design(d_old, rho, d_new)
    off_o = np.concatenate([[0], np.cumsum(d_old ** 2)])
    off_n = np.concatenate([[0], np.cumsum(d_new ** 2)])
    for e in range(len(d_old)):
        vo = rho[off_o[e]:off_o[e + 1]].sum() / d_old[e] ** 2
        vn = out[off_n[e]:off_n[e + 1]].sum() / d_new[e] ** 2
        assert abs(vo - vn) < 1e-15
    const = transfer_design(d_old, np.full(len(rho), 0.42), d_new)
    np.testing.assert_allclose(const, 0.42, rtol=1e-15)


def test_stopping_thresholds():
    assert cycle_converged(10.0, 10.039, 1) and not cycle_converged(10.0, 10.041, 1)
    assert cycle_converged(10.0, 10.0239, 2) and not cycle_converged(10.0, 10.0241, 2)
