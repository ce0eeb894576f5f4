"""Seeded input generators (host logic, no GPU): packing round trips, exact volume fractions,
connectivity of the binary designs, order-jump caps of the dp maps, and the tiled beam."""
import numpy as np

import workloads as W


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(0)
    f = rng.random((3 * 4, 5 * 4))
    packed = W.pack_uniform(f, 5, 3, 4)
    assert packed.shape == (5 * 3 * 16,)
    # element e = ey * nelx + ex owns its 4 x 4 block, x fastest inside
    assert np.array_equal(packed[:16].reshape(4, 4), f[:4, :4])
    assert np.array_equal(W.unpack_uniform(packed, 5, 3, 4), f)


def test_binary_beam_volume_and_connectivity():
    pr = W.mbb_binary(40, 20, sigma=4.0, seed_index=12)
    fine = W.unpack_uniform(pr.rho, 40, 20, 8)
    assert set(np.unique(fine)) <= {0.0, 1.0}
    assert int(fine.sum()) == int(round(0.3 * fine.size))
    # every solid cell reaches the frame through 4-connected solid cells
    import scipy.ndimage as ndi
    lab, n = ndi.label(fine > 0.5)
    assert n == 1


def test_dp_cantilever_maps():
    pr = W.named("dp_cantilever_40x20")
    P = pr.p.reshape(pr.nely, pr.nelx)
    assert max(np.abs(np.diff(P, axis=0)).max(), np.abs(np.diff(P, axis=1)).max()) <= 2
    assert set(np.unique(pr.p)) <= {1, 2, 3, 4, 5}
    assert set(np.unique(pr.d)) <= {1, 2, 4, 8}
    assert len(pr.rho) == int(np.sum(pr.d.astype(np.int64) ** 2))
    assert pr.rho.min() >= 1e-3 - 1e-15 and pr.rho.max() <= 1.0


def test_tiled_beam_repeats_the_base_design():
    base = W.mbb_binary()
    big = W.mbb_tiled(2, 2)
    fb = W.unpack_uniform(base.rho, base.nelx, base.nely, 8)
    ft = W.unpack_uniform(big.rho, big.nelx, big.nely, 8)
    ny, nx = fb.shape
    for ty in range(2):
        for tx in range(2):
            assert np.array_equal(ft[ty * ny:(ty + 1) * ny, tx * nx:(tx + 1) * nx], fb)


def test_generators_are_seeded():
    a = W.named("mbb_40x20_p3_d8").rho
    b = W.named("mbb_40x20_p3_d8").rho
    assert np.array_equal(a, b)
