"""Seeded synthetic inputs for the dp-adaptive MTO hot path.

This module holds input generation only (meshes, order / design maps, density fields, load cases)
and none of the method's arithmetic.  It is the one module that both the CPU oracle (``oracle/``)
and the CUDA path (``paper_1811_09821_gb300``) use, so that they see identical inputs.

The paper's test problems are synthetic (Sec. 4.1: cantilever with a point load on a 40 x 20 mesh,
Q2 elements with 4 x 4 design points, E0 = 1, nu = 0.3, q = 3, Emin = 1e-9 E0).  The workloads below
stand in for them at several scales; the MBB half-beam is a textbook addition.  Random numbers come
from numpy's PCG64 with seed 181109821 + workload index.

Packed design layout: element e = ey*nelx + ex owns d_e^2 consecutive values starting at
design_off[e] (exclusive prefix sum of d^2); subcell s = j*d_e + i covers
[i/d_e, (i+1)/d_e] x [j/d_e, (j+1)/d_e] of the element (i along x).
"""
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 181109821

# load cases: how the supports and the point load are placed (the DOF numbering is each side's own)
CANTILEVER = "cantilever"   # left edge clamped (u_x = u_y = 0); F = -1 in y at vertex (nelx, nely/2)
MBB = "mbb"                 # u_x = 0 on the left edge; u_y = 0 at vertex (nelx, 0); F = -1 in y at (0, nely)
CANTILEVER_DISTRIBUTED = "cantilever_distributed"   # left edge clamped; uniform downward traction on
                                                    # the top edge, total 1 (Sec. 4.1, Fig. 6a)


@dataclass
class Problem:
    name: str
    nelx: int
    nely: int
    p: np.ndarray            # int32 [nel] shape-function order per element
    d: np.ndarray            # int32 [nel] per-axis design count per element
    rho: np.ndarray          # float64 [design_len] packed densities
    load: str                # CANTILEVER or MBB
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    q: float = 3.0
    extra: dict = field(default_factory=dict)

    @property
    def nel(self):
        return self.nelx * self.nely

    @property
    def design_off(self):
        return np.concatenate([[0], np.cumsum(self.d.astype(np.int64) ** 2)])


def _smooth_noise(rng, ny, nx, sigma):
    """White noise smoothed by a periodic Gaussian of std ``sigma`` cells (FFT), zero mean, unit std."""
    w = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2))
    s = np.real(np.fft.ifft2(np.fft.fft2(w) * g))
    s -= s.mean()
    return s / s.std()


def pack_uniform(field_2d, nelx, nely, d):
    """Packed layout of a (nely*d) x (nelx*d) fine field for a uniform per-axis design count d."""
    f = field_2d.reshape(nely, d, nelx, d)          # [ey, j, ex, i]
    return np.ascontiguousarray(f.transpose(0, 2, 1, 3)).reshape(-1).astype(np.float64)


def unpack_uniform(packed, nelx, nely, d):
    """The (nely*d) x (nelx*d) fine field of a packed uniform layout (inverse of pack_uniform)."""
    f = np.asarray(packed).reshape(nely, nelx, d, d)   # [ey, ex, j, i]
    return np.ascontiguousarray(f.transpose(0, 2, 1, 3)).reshape(nely * d, nelx * d)


def pack_mixed(fine, nelx, nely, d_map, r):
    """Packed layout for per-element design counts from a fine field with r x r cells per element.

    Subcell (i, j) of an element with count d takes the mean of the fine cells whose centres fall
    inside it (d must divide r) or, otherwise, the fine cell under its centre."""
    out = []
    F = fine.reshape(nely, r, nelx, r)
    for e in range(nelx * nely):
        ex, ey = e % nelx, e // nelx
        blk = F[ey, :, ex, :]                         # [j_fine, i_fine]
        d = int(d_map[e])
        if r % d == 0:
            k = r // d
            out.append(blk.reshape(d, k, d, k).mean(axis=(1, 3)).reshape(-1))
        else:
            c = ((np.arange(d) + 0.5) * r / d).astype(int)
            out.append(blk[np.ix_(c, c)].reshape(-1))
    return np.concatenate(out).astype(np.float64)


def _frame_bias(ny, nx, width):
    """1 on a band of ``width`` cells along all four sides of an ny x nx grid, else 0: a load-carrying
    frame, so that loads and supports always sit in material."""
    b = np.zeros((ny, nx))
    b[:width, :] = b[-width:, :] = 1.0
    b[:, :width] = b[:, -width:] = 1.0
    return b


def _threshold_volume(s, vol):
    """Binary 0/1 field with exactly round(vol * size) ones at the largest values of s."""
    flat = s.ravel()
    k = int(round(vol * flat.size))
    out = np.zeros(flat.size)
    out[np.argsort(-flat, kind="stable")[:k]] = 1.0
    return out.reshape(s.shape)


def _connected_threshold(s, vol, seed_mask):
    """Binary 0/1 field with exactly round(vol * size) ones, grown from ``seed_mask`` through
    4-connected cells in decreasing order of s (a priority flood), so every solid cell is connected
    to the seed: no floating solid islands."""
    import heapq
    ny, nx = s.shape
    k = int(round(vol * s.size))
    out = np.zeros(s.size, dtype=bool)
    flat = s.ravel()
    heap = [(-flat[i], int(i)) for i in np.flatnonzero(seed_mask.ravel())]
    heapq.heapify(heap)
    queued = np.zeros(s.size, dtype=bool)
    queued[[i for _, i in heap]] = True
    count = 0
    while heap and count < k:
        _, i = heapq.heappop(heap)
        out[i] = True
        count += 1
        y, x = divmod(i, nx)
        for yy, xx in ((y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)):
            if 0 <= yy < ny and 0 <= xx < nx:
                j = yy * nx + xx
                if not queued[j]:
                    queued[j] = True
                    heapq.heappush(heap, (-flat[j], j))
    return out.reshape(s.shape).astype(np.float64)


def _sigmoid_volume(s, vol, width=0.35, floor=1e-3):
    """Smooth densities in [floor, 1]: a logistic of s with its offset chosen so the mean is ``vol``.

    The offset is bisected on a strided 1/97 subsample of the cells, then refined by Newton steps
    on the whole field (the mean is smooth and monotone in the offset) until the step falls below
    1e-15."""
    es = np.exp(-s / width).ravel()     # exp(-(s - t)/w) = exp(-s/w) exp(t/w): one exponential per cell

    def dens(t, e):
        r = 1.0 / (1.0 + e * np.exp(t / width))
        return np.clip(r, floor, 1.0), r

    sub = es[::97]
    lo, hi = -10.0, 10.0
    for _ in range(64):   # the interval of 20 is below one ulp after ~60 halvings
        t = 0.5 * (lo + hi)
        if dens(t, sub)[0].mean() > vol:
            lo = t
        else:
            hi = t
    t = 0.5 * (lo + hi)
    for _ in range(12):
        rc, r = dens(t, es)
        g = rc.mean() - vol
        # d r / d t = -r (1 - r) / w where the clip is inactive
        dg = -np.mean(np.where((r > floor) & (r < 1.0), r * (1.0 - r), 0.0)) / width
        step = g / dg
        t -= step
        if abs(step) < 1e-15:
            break
    return dens(t, es)[0].reshape(s.shape)


def cantilever_small(nelx=20, nely=10, p=2, d=4, seed_index=1):
    """20 x 10 Q2, 4 x 4 design points, uniform 0.5 + U(-0.1, 0.1) densities; cantilever load."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    nel = nelx * nely
    rho = 0.5 + rng.uniform(-0.1, 0.1, nel * d * d)
    return Problem(f"cantilever_{nelx}x{nely}_p{p}_d{d}", nelx, nely, np.full(nel, p, np.int32),
                   np.full(nel, d, np.int32), rho, CANTILEVER)


def mbb_binary(nelx=160, nely=80, p=3, d=8, vol=0.3, sigma=8.0, seed_index=2, connected=True):
    """MBB half-beam, uniform order and design count, a Gaussian-smoothed white-noise field
    (std sigma design cells) thresholded to exactly ``vol`` material (0/1 densities).  A solid frame
    one element wide (at least 1/20 of the height) is selected first, so the load path exists.
    ``connected``: the threshold is a priority flood from the frame (every solid cell connected to
    it); otherwise a plain threshold, which leaves floating solid islands held only by void."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    s = _smooth_noise(rng, nely * d, nelx * d, sigma)
    frame = _frame_bias(nely * d, nelx * d, max(d, (nely * d) // 20))
    s = s + 100.0 * frame
    field = _connected_threshold(s, vol, frame > 0) if connected else _threshold_volume(s, vol)
    rho = pack_uniform(field, nelx, nely, d)
    nel = nelx * nely
    return Problem(f"mbb_{nelx}x{nely}_p{p}_d{d}_binary{vol}", nelx, nely, np.full(nel, p, np.int32),
                   np.full(nel, d, np.int32), rho, MBB)


def mbb_smooth(nelx=1024, nely=512, p=3, d=8, vol=0.2, sigma=8.0, seed_index=5):
    """MBB half-beam with smooth densities in [1e-3, 1] at mean ``vol`` (a logistic of smoothed noise)."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    s = _smooth_noise(rng, nely * d, nelx * d, sigma)
    s = s + 4.0 * _frame_bias(nely * d, nelx * d, max(d, (nely * d) // 40))
    rho = pack_uniform(_sigmoid_volume(s, vol), nelx, nely, d)
    nel = nelx * nely
    return Problem(f"mbb_{nelx}x{nely}_p{p}_d{d}_smooth{vol}", nelx, nely, np.full(nel, p, np.int32),
                   np.full(nel, d, np.int32), rho, MBB)


def mbb_tiled(tx=3, ty=3):
    """tx x ty copies of the 160 x 80 binary beam's design side by side (each tile keeps its solid
    frame, so the lattice is connected): a larger instance of the same structure."""
    base = mbb_binary()
    d = int(base.d[0])
    fine = unpack_uniform(base.rho, base.nelx, base.nely, d)
    big = np.tile(fine, (ty, tx))
    nelx, nely = base.nelx * tx, base.nely * ty
    nel = nelx * nely
    return Problem(f"mbb_{nelx}x{nely}_p3_d{d}_tiled", nelx, nely, np.full(nel, int(base.p[0]), np.int32),
                   np.full(nel, d, np.int32), pack_uniform(big, nelx, nely, d), MBB)


def _brace_bias(ny, nx, width):
    """1 within ``width`` cells of the two diagonals of an ny x nx grid, else 0: the X bracing of a
    truss-like cantilever (without it a thin frame alone is a near-mechanism)."""
    y, x = np.mgrid[0:ny, 0:nx] + 0.5
    b = np.zeros((ny, nx))
    for (x0, y0, x1, y1) in ((0.0, 0.0, nx, ny), (0.0, ny, nx, 0.0)):
        dx, dy = x1 - x0, y1 - y0
        dist = np.abs(dy * (x - x0) - dx * (y - y0)) / np.hypot(dx, dy)
        b[dist <= width] = 1.0
    return b


def dp_cantilever(nelx=320, nely=160, vol=0.1, seed_index=3, p_levels=(1, 2, 3, 4), d_levels=(1, 2, 4, 8)):
    """dp-adaptive cantilever: smooth random order and design maps with refined bands where the
    density gradient is large; smooth densities at mean ``vol`` on a braced frame (a frame of one
    element and X bracing, so the structure carries the load like an optimized truss).

    Orders: a smoothed field quantised to p_levels, +1 (capped) where |grad rho| is above its 80th
    percentile.  Design counts: an independent smoothed field quantised to d_levels, raised to the
    largest level inside the same bands.  Neighbouring orders differ by at most 2 by construction
    (checked)."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    r = 8
    s = _smooth_noise(rng, nely * r, nelx * r, 3.0 * r)
    s = s + 4.0 * np.maximum(_frame_bias(nely * r, nelx * r, max(r, (nely * r) // 80)),
                             _brace_bias(nely * r, nelx * r, max(r, (nely * r) // 80)))
    fine = _sigmoid_volume(s, vol)
    # per-element gradient magnitude of the element-mean density
    em = fine.reshape(nely, r, nelx, r).mean(axis=(1, 3))
    gy, gx = np.gradient(em)
    band = np.hypot(gx, gy) > np.percentile(np.hypot(gx, gy), 80)
    sp = _smooth_noise(rng, nely, nelx, 6.0)
    qp = np.clip(np.floor((sp + 2.0) / 4.0 * len(p_levels)), 0, len(p_levels) - 1).astype(int)
    P = np.array(p_levels)[qp] + band.astype(int)
    P = np.minimum(P, max(p_levels))
    sd = _smooth_noise(rng, nely, nelx, 6.0)
    qd = np.clip(np.floor((sd + 2.0) / 4.0 * len(d_levels)), 0, len(d_levels) - 1).astype(int)
    D = np.array(d_levels)[qd]
    D[band] = max(d_levels)
    jump = max(np.abs(np.diff(P, axis=0)).max(initial=0), np.abs(np.diff(P, axis=1)).max(initial=0))
    assert jump <= 2, "order map has a jump above 2"
    rho = pack_mixed(fine, nelx, nely, D.ravel(), r)
    return Problem(f"dp_cantilever_{nelx}x{nely}_vol{vol}", nelx, nely, P.ravel().astype(np.int32),
                   D.ravel().astype(np.int32), rho, CANTILEVER)


def batched(n_instances=64, seed_index=4, sizes=((40, 20), (80, 40), (160, 80), (320, 160)),
            p_levels=(1, 2, 3, 4), d_levels=(2, 4, 8)):
    """Independent instances of uneven sizes with per-instance uniform p and d, alternating
    cantilever and MBB loads, binary densities at volume 0.3 - 0.5."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    out = []
    for k in range(n_instances):
        nelx, nely = sizes[rng.integers(len(sizes))]
        p = int(rng.choice(p_levels))
        d = int(rng.choice(d_levels))
        vol = float(rng.uniform(0.3, 0.5))
        s = _smooth_noise(rng, nely * d, nelx * d, 2.0 * d)
        s = s + 100.0 * _frame_bias(nely * d, nelx * d, max(d, (nely * d) // 20))
        rho = pack_uniform(_threshold_volume(s, vol), nelx, nely, d)
        nel = nelx * nely
        out.append(Problem(f"inst{k}_{nelx}x{nely}_p{p}_d{d}", nelx, nely, np.full(nel, p, np.int32),
                           np.full(nel, d, np.int32), rho, CANTILEVER if k % 2 == 0 else MBB))
    return out


def named(name):
    """The named workloads used by tests and the bench."""
    table = {
        "cantilever_20x10_p2_d4": lambda: cantilever_small(),
        "mbb_160x80_p3_d8": lambda: mbb_binary(),
        "mbb_40x20_p3_d8": lambda: mbb_binary(40, 20, sigma=4.0, seed_index=12),
        "mbb_40x20_p3_d8_islands": lambda: mbb_binary(40, 20, sigma=4.0, seed_index=12, connected=False),
        "dp_cantilever_320x160": lambda: dp_cantilever(),
        "dp_cantilever_40x20": lambda: dp_cantilever(40, 20, vol=0.3, seed_index=13),
        "mbb_1024x512_p3_d8": lambda: mbb_smooth(),
        # the same recipe on a 64 x 32 mesh: the bounded sample the CPU oracle is timed on
        "mbb_64x32_p3_d8": lambda: mbb_smooth(64, 32, seed_index=15),
        # 3 x 3 tiles of the 160 x 80 binary beam: element matrices (~1 GB for both storages) above
        # L2, for hardware-counter captures of one operator launch
        "mbb_480x240_p3_d8": lambda: mbb_tiled(3, 3),
    }
    return table[name]()
