"""Identities the GPU kernels rely on, checked on CPU with the oracle's own quantities (they pin the
kernels' reformulations, not the oracle):

* QR error (Eq. 14): the kernel takes J^(p+1) = 1/2 u1^T K u1 from the right-hand side of the
  pinned element problem, 1/2 (u1_f^T f1_f + v^T (K u1)_pinned), with the pinned rows saved before
  the modification; on the oracle's element problems both forms agree to rounding.
* OC update: the kernel clips non-negative doubles by signed 64-bit compares of their bit patterns
  (exact: non-negative doubles order like their bits), and sums the area-scaled clip
  sum_j clip(dv_j t_j c, dv_j lo_j, dv_j hi_j) in place of sum_j dv_j clip(t_j c, lo_j, hi_j)
  (equal to rounding for dv > 0: scaling commutes with the clip, only the product order differs).
"""
import numpy as np

from oracle.element import simp
from oracle.indicators import qr_fixed_local_dofs, qr_load_transfer, _prolong_vec, remove_rigid_motion
from oracle.solve import K0_table


def test_qr_energy_from_right_hand_side():
    rng = np.random.default_rng(7)
    for p, d in ((1, 2), (2, 4), (3, 8)):
        for trial in range(3):
            rho = rng.uniform(0.0, 1.0, d * d) ** 3
            rho[rng.uniform(size=d * d) < 0.3] = 0.0
            ue = remove_rigid_motion(p, rng.standard_normal(2 * (p + 1) ** 2), 1.0, 1.0)
            E = simp(rho, 1.0, 1e-9, 3.0)
            Kp = np.tensordot(E, K0_table(p, d, 0.3), axes=(0, 0))
            K1 = np.tensordot(E, K0_table(p + 1, d, 0.3), axes=(0, 0))
            f1 = qr_load_transfer(p) @ (Kp @ ue)
            fx = qr_fixed_local_dofs(p + 1)
            fr = np.setdiff1d(np.arange(K1.shape[0]), fx)
            u1 = np.zeros(K1.shape[0])
            u1[fx] = (_prolong_vec(p) @ ue)[fx]
            u1[fr] = np.linalg.solve(K1[np.ix_(fr, fr)], f1[fr] - K1[np.ix_(fr, fx)] @ u1[fx])
            direct = 0.5 * u1 @ (K1 @ u1)
            from_rhs = 0.5 * (u1[fr] @ f1[fr] + u1[fx] @ (K1[fx, :] @ u1))
            scale = 0.5 * np.abs(u1) @ (np.abs(K1) @ np.abs(u1))
            assert abs(direct - from_rhs) <= 1e-9 * scale, (p, d, direct, from_rhs)


def clip_by_bits(x, lo, hi):
    xi, li, hi_ = (np.asarray(v, dtype=np.float64).view(np.int64) for v in (x, lo, hi))
    return np.minimum(np.maximum(xi, li), hi_).view(np.float64)


def test_nonnegative_clip_by_integer_compares():
    rng = np.random.default_rng(11)
    n = 200000
    lo = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-300, 300, n)
    hi = lo + np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-300, 300, n)
    x = np.abs(rng.standard_normal(n)) * 10.0 ** rng.integers(-310, 308, n)     # subnormals too
    x[:1000] = 0.0
    x[1000:2000] = -0.0
    lo[2000:3000] = 0.0
    got = clip_by_bits(x, lo, hi)
    want = np.minimum(np.maximum(x, lo), hi)
    assert np.array_equal(got, want)          # -0.0 == 0.0: a signed zero may come back as +0.0


def test_area_scaled_clip_sum():
    rng = np.random.default_rng(5)
    n = 4096
    rho = rng.uniform(0.0, 1.0, n)
    t = rng.uniform(0.0, 2.0, n)
    dv = np.repeat(1.0 / np.array([4.0, 9.0, 64.0, 16.0]), n // 4)     # subcell areas 1/d^2
    lo, hi = np.maximum(0.0, rho - 0.2), np.minimum(1.0, rho + 0.2)
    for c in (0.1, 0.7, 1.3, 5.0):
        per = dv * np.minimum(np.maximum(t * c, lo), hi)
        scaled = np.minimum(np.maximum((dv * t) * c, dv * lo), dv * hi)
        assert np.allclose(per, scaled, rtol=4e-16, atol=0.0)


def triangle_pair(t):
    """The QR kernel's decode of a packed-triangle index (trailing-block pairs of the L D L^T
    update, and the packed lower storage itself), as in the kernel: t = s (s + 1) / 2 + r with
    0 <= r <= s, s first estimated in FP32 and then corrected."""
    s = int((np.sqrt(np.float32(8.0) * np.float32(t) + np.float32(1.0)) - np.float32(1.0)) * np.float32(0.5))
    while s * (s + 1) // 2 > t:
        s -= 1
    while (s + 1) * (s + 2) // 2 <= t:
        s += 1
    return s, t - s * (s + 1) // 2


def test_packed_lower_index_round_trip():
    """Row-major packed lower storage: index i (i + 1) / 2 + j decodes back to (i, j) for every entry
    of the largest order-(p+1) matrix (n1 = 128, 8256 entries)."""
    for i in range(128):
        for j in range(i + 1):
            assert triangle_pair(i * (i + 1) // 2 + j) == (i, j)


def test_trailing_pairs_cover_the_block_once():
    """Every pair (i, j), c < j <= i < n1, of the trailing block of pivot c comes from exactly one
    t < m (m + 1) / 2 (m = n1 - 1 - c), for the element sizes of orders 2..7 (n1 = 2 (p+1)^2)."""
    for n1 in (18, 32, 50, 72, 98, 128):
        for c in range(n1):
            m = n1 - 1 - c
            seen = set()
            for t in range(m * (m + 1) // 2):
                s, r = triangle_pair(t)
                assert 0 <= r <= s < m
                i, j = n1 - 1 - r, n1 - 1 - s
                assert c < j <= i < n1
                seen.add((i, j))
            assert len(seen) == m * (m + 1) // 2
