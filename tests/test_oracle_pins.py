"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
lattice-point counts, the analytic point-lens magnification, conservation and
symmetry invariants, the truncation bound of the Taylor series, values
printed in the paper (tests/golden/table1.json) and finite differences.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NO = np.zeros(0)


def _geom(kappa, gamma, ks, lx, ly, sheet, map_box, map_n, **kw):
    return oracle.derive_geometry(kappa, gamma, ks, lx, ly, sheet, map_box, map_n, **kw)


# -- P1: no lenses, no sheet: the map is an affine image of the lattice ------

def test_uniform_map_dyadic_exact():
    """kappa = gamma = 1/4: beta = (theta_x / 2, theta_y); with dyadic spacings
    every pixel receives exactly 8 x 4 = 32 rays and mu = 1/det = 2 (Eq. 12)."""
    g = _geom(0.25, 0.25, 0.0, [], [], (0, 0, 1), (-1, -1, 1, 1), (32, 32),
              ray_box=(-2, -1, 2, 1), ray_n=(256, 128))
    counts, stats = oracle.shoot_direct(g, NO, NO, NO)
    assert np.all(counts == 32)
    assert list(stats) == [256 * 128, 0, 0]
    mu = oracle.magnification(g, counts)
    assert np.all(mu == 2.0)


def _lattice_count_1d(a, r0, l3, n, m0, d, nb):
    """Number of lattice points i in [0, n) with m0 + k d <= a (r0 + (i+1/2) l3)
    < m0 + (k+1) d, for each bin k, by inverting the affine map (a > 0)."""
    edges = m0 + np.arange(nb + 1) * d
    first = np.ceil((edges / a - r0) / l3 - 0.5)          # first i at or past each edge
    first = np.clip(first, 0, n)
    return np.diff(first).astype(np.int64)


def test_uniform_map_lattice_count():
    """Non-dyadic macro model: each pixel count equals the product of the
    numbers of lattice columns and rows whose images fall in it."""
    kappa, gamma = 0.3, 0.17
    a, b = 1 - kappa - gamma, 1 - kappa + gamma
    g = _geom(kappa, gamma, 0.0, [], [], (0, 0, 1), (-1.0, -0.7, 0.9, 0.8), (37, 23),
              ray_box=(-2.2, -1.1, 2.1, 1.0), ray_n=(731, 419))
    counts, stats = oracle.shoot_direct(g, NO, NO, NO)
    cx = _lattice_count_1d(a, g.rx0, g.l3x, g.n3x, g.mx0, g.dpx, g.mnx)
    cy = _lattice_count_1d(b, g.ry0, g.l3y, g.n3y, g.my0, g.dpy, g.mny)
    assert np.array_equal(counts.astype(np.int64), np.outer(cy, cx))
    assert stats[0] == counts.sum() and stats[0] + stats[1] == g.n_rays


# -- P2: single point lens, kappa = gamma = kappa_* = 0 ---------------------

def test_point_lens_magnification():
    """Pixel means of the analytic point-lens magnification
    mu(u) = (u^2 + 2) / (u sqrt(u^2 + 4)) (Gauss-Legendre 16 x 16 per pixel)
    against mu_ij = N_ij S_I / S_S.  Pixels within 2 of the lens are skipped."""
    g = _geom(0.0, 0.0, 0.0, [0.0], [0.0], (0, 0, 1), (-1, -1, 1, 1), (32, 32),
              ray_box=(-2.5, -2.5, 2.5, 2.5), ray_n=(4000, 4000))
    counts, _ = oracle.shoot_direct(g, [0.0], [0.0], [1.0])
    mu = oracle.magnification(g, counts)
    xg, wg = np.polynomial.legendre.leggauss(16)
    W = np.outer(wg, wg) / 4.0
    ref = np.zeros((32, 32))
    for iy in range(32):
        for ix in range(32):
            X = -1 + (ix + (xg + 1) / 2) * g.dpx
            Y = -1 + (iy + (xg + 1) / 2) * g.dpy
            XX, YY = np.meshgrid(X, Y)
            u = np.hypot(XX, YY)
            ref[iy, ix] = np.sum(W * (u * u + 2) / (u * np.sqrt(u * u + 4)))
    ii, jj = np.meshgrid(np.arange(32), np.arange(32))
    keep = (np.abs(ii - 15.5) > 2.5) | (np.abs(jj - 15.5) > 2.5)
    rel = ((mu - ref) / ref)[keep]
    # lattice-sampling error: ~2500 rays per unit magnification per pixel
    assert np.abs(rel).max() < 0.015
    assert np.abs(rel).mean() < 0.003
    assert abs(rel.mean()) < 0.001


# -- P3, P4: ray conservation and split invariance ---------------------------

def test_conservation_and_dropped_ray():
    lf = inputs.lens_disc(30, 4.0, 5, "lognormal")
    x, y, m = lf.x.copy(), lf.y.copy(), lf.m.copy()
    g = _geom(0.4, 0.3, 0.02, x, y, (0, 0, 4.0), (-1, -1, 1, 1), (40, 40),
              ray_box=(-3, -2, 3, 2), ray_n=(300, 200))
    # put lens 0 exactly on ray (i, j) = (17, 9)
    tx, ty = oracle.ray_position(g, [9 * 300 + 17])
    x[0], y[0] = tx[0], ty[0]
    counts, stats = oracle.shoot_direct(g, x, y, m)
    assert stats[2] == 1
    assert int(stats.sum()) == g.n_rays
    assert int(counts.sum()) == int(stats[0])


def test_split_invariance():
    lf = inputs.lens_disc(25, 4.0, 6, "unit")
    g = _geom(0.4, 0.3, 0.02, lf.x, lf.y, (0, 0, 4.0), (-1, -1, 1, 1), (40, 40),
              ray_box=(-3, -2, 3, 2), ray_n=(300, 200))
    full, s_full = oracle.shoot_direct(g, lf.x, lf.y, lf.m)
    k = 12345
    a, s_a = oracle.shoot_direct(g, lf.x, lf.y, lf.m, 0, k)
    b, s_b = oracle.shoot_direct(g, lf.x, lf.y, lf.m, k, g.n_rays)
    assert np.array_equal(full, a + b)
    assert np.array_equal(s_full, s_a + s_b)


# -- P5: mirror symmetry fixes the signs of both deflection components -------

@pytest.mark.parametrize("axis", [0, 1])
def test_mirror_symmetry(axis):
    """Lenses mirrored across an axis, with a lattice and map symmetric about
    it, give the mirrored map.  Spacings are dyadic so that mirrored rays sit
    at exactly negated positions."""
    lf = inputs.lens_disc(20, 3.0, 9, "lognormal")
    x, y = lf.x, lf.y
    kw = dict(ray_box=(-2.0, -2.0, 2.0, 2.0), ray_n=(512, 512))
    g = _geom(0.35, 0.25, 0.03, x, y, (0, 0, 3.0), (-1, -1, 1, 1), (64, 64), **kw)
    c1, _ = oracle.shoot_direct(g, x, y, lf.m)
    mx, my = (-x, y) if axis == 0 else (x, -y)
    c2, _ = oracle.shoot_direct(g, mx, my, lf.m)
    flipped = c2[:, ::-1] if axis == 0 else c2[::-1, :]
    assert np.array_equal(c1, flipped)
    assert c1.sum() > 1000


# -- P6: the far-field Taylor series against the direct sum ------------------

@pytest.mark.parametrize("p,l2y", [(1, 20), (2, 20), (3, 20), (5, 20), (3, 7), (4, 40)])
def test_interp_within_truncation_bound(p, l2y):
    """|beta_interp - beta_direct| <= sum_far m rho^{p+1} / (r^{p+1} (r - rho)),
    the tail of the geometric series of 1/(z_k - z), for every sampled ray;
    the bound is nearly attained, so a wrong coefficient would break it."""
    lf = inputs.lens_disc(40, 6.0, 3, "lognormal")
    g = _geom(0.3, 0.2, 0.05, lf.x, lf.y, (0, 0, 6.0), (-2, -2, 2, 2), (64, 64),
              ray_box=(-4, -3, 4, 3), ray_n=(400, 300), p=p, l2_sub_y=l2y)
    assert g.n1y == l2y * g.n2y
    idx = np.arange(0, g.n_rays, 61)
    bd, fd = oracle.beta_direct(g, lf.x, lf.y, lf.m, idx)
    bi, fi = oracle.beta_interp(g, lf.x, lf.y, lf.m, idx)
    rb = oracle.remainder_bound(g, lf.x, lf.y, lf.m, idx)
    err = np.hypot(*(bd - bi).T)
    assert np.all(np.isfinite(rb))
    assert np.all(err <= rb * (1 + 1e-9) + 1e-13)
    assert np.max(err / rb) > 0.5          # the bound is tight, not vacuous
    assert np.array_equal(fd, fi)


def test_interp_converges_to_direct():
    lf = inputs.lens_disc(40, 6.0, 3, "lognormal")
    g = _geom(0.3, 0.2, 0.05, lf.x, lf.y, (0, 0, 6.0), (-2, -2, 2, 2), (64, 64),
              ray_box=(-4, -3, 4, 3), ray_n=(400, 300), p=14)
    idx = np.arange(0, g.n_rays, 211)
    bd, _ = oracle.beta_direct(g, lf.x, lf.y, lf.m, idx)
    bi, _ = oracle.beta_interp(g, lf.x, lf.y, lf.m, idx)
    assert np.max(np.abs(bd - bi)) < 1e-12


def test_node_coefficients_are_taylor_coefficients():
    """c_n at a node equals the n-th Taylor coefficient of the far field,
    checked by a complex-step-free route: a discrete Cauchy integral of the
    far deflection sampled on a small circle around the node."""
    lf = inputs.lens_disc(30, 5.0, 4, "unit")
    g = _geom(0.3, 0.2, 0.05, lf.x, lf.y, (0, 0, 5.0), (-2, -2, 2, 2), (32, 32),
              ray_box=(-4, -3, 4, 3), ray_n=(400, 300), p=4)
    c2x, c2y = 7, 5
    c = oracle.node_coeffs(g, lf.x, lf.y, lf.m, [c2x], [c2y])[0]
    zx, zy = oracle.node_position(g, c2x, c2y)
    z0 = complex(zx, zy)
    c1x, c1y = c2x * g.n2x // g.n1x, c2y * g.n2y // g.n1y
    l1x, l1y = g.n1x * g.l3x, g.n1y * g.l3y
    cx = np.floor((lf.x - g.rx0) / l1x)
    cy = np.floor((lf.y - g.ry0) / l1y)
    far = ~((np.abs(cx - c1x) <= 1) & (np.abs(cy - c1y) <= 1))
    zk = (lf.x + 1j * lf.y)[far]
    mk = lf.m[far]
    K, rad = 64, 0.2
    zs = z0 + rad * np.exp(2j * np.pi * np.arange(K) / K)
    f = np.array([np.sum(mk / (z - zk)) for z in zs])      # conj(alpha_far)
    for n in range(5):
        cauchy = np.mean(f * np.exp(-2j * np.pi * n * np.arange(K) / K)) / rad ** n
        assert abs(cauchy - c[n]) <= 1e-10 * max(1.0, abs(c[0]))


# -- P7: linearity of the deflection in the lens set --------------------------

def test_linearity_in_lens_set():
    lf = inputs.lens_disc(30, 4.0, 11, "lognormal")
    g = _geom(0.4, 0.3, 0.02, lf.x, lf.y, (0, 0, 4.0), (-1, -1, 1, 1), (40, 40),
              ray_box=(-3, -2, 3, 2), ray_n=(300, 200))
    idx = np.arange(0, g.n_rays, 37)
    ball, _ = oracle.beta_direct(g, lf.x, lf.y, lf.m, idx)
    ba, _ = oracle.beta_direct(g, lf.x[:13], lf.y[:13], lf.m[:13], idx)
    bb, _ = oracle.beta_direct(g, lf.x[13:], lf.y[13:], lf.m[13:], idx)
    b0, _ = oracle.beta_direct(g, NO, NO, NO, idx)
    assert np.allclose(ball, ba + bb - b0, rtol=0, atol=1e-11)


# -- P8: the compensating sheet keeps the mean magnification -----------------

def test_mean_magnification_with_compensating_sheet():
    """With kappa_* = N m / R^2 and the sheet on the lens disc, the mean
    magnification over the map is 1/|(1-kappa)^2 - gamma^2| (the protection
    band of §3.1 is quoted as ~98% accurate).  Averaged over 16 fields."""
    kappa, gamma, R = 0.3, 0.1, 38.0
    mus = []
    for seed in range(16):
        n = int(round(0.05 * R * R))
        lf = inputs.lens_disc(n, R, 100 + seed, "unit")
        g = _geom(kappa, gamma, n / R ** 2, lf.x, lf.y, (0, 0, R), (-10, -10, 10, 10),
                  (64, 64), n_av=100)
        counts, _ = oracle.shoot_direct(g, lf.x, lf.y, lf.m)
        mus.append(oracle.magnification(g, counts).mean())
    expect = 1.0 / abs((1 - kappa) ** 2 - gamma ** 2)
    assert abs(np.mean(mus) / expect - 1) < 0.03


# -- P9: numbers printed in the paper ----------------------------------------

def test_table1_and_figure2_values():
    gold = json.load(open(os.path.join(GOLDEN, "table1.json")))
    t = gold["table1"]
    kc = oracle.kappa_c(t["theta_e_arcsec"], t["d_per_arcmin"])
    assert float(f"{kc:.{t['kappa_c_printed_digits']}g}") == t["kappa_c"]
    assert t["kappa_star"] > 10 * kc                 # "kappa_* >> kappa_c"
    w = oracle.protection_width(t["kappa_star"])
    assert round(-w, 6) == gold["fig2"]["beta_x_lower_edge"]
    sx, sy = gold["section4_1"]["source_region"]
    nx, ny = gold["section4_1"]["n_pix"]
    assert abs(sx / nx - 5.5e-4) < 0.02 * 5.5e-4 and abs(sy / ny - 5.5e-4) < 0.02 * 5.5e-4
    # N_* = L_ix L_iy kappa_* / pi inverts to the image-plane area of Table 1
    area = math.pi * t["n_star"] / t["kappa_star"]
    assert abs(oracle.n_star_from_area(area, t["kappa_star"]) - t["n_star"]) < 1e-9


def test_level_grids_follow_eq10():
    """Eq. 10: L1 = min(L0, L_i / 10), so at least ten level-1 cells per side;
    level 2 is 1/20 of level 1."""
    w = inputs.paper_map(0, n_rays=1e9, map_px=1024)
    g = oracle.geometry_of(w)
    assert g.N1x >= 10 and g.N1y >= 10
    assert g.n1x == 20 * g.n2x and g.n1y == 20 * g.n2y
    l1x = g.n1x * g.l3x
    assert abs(l1x / g.l0 - 1) < 0.01                 # many lenses: L1 = L0 in x
    # the uniform image of the ray rectangle is the widened source region
    a = 1 - g.kappa - g.gamma
    assert abs(a * g.rx0 - (w.map_box[0] - oracle.protection_width(g.kappa_star) / 2)) < 1e-9


# -- Cloud-in-cell and its adjoint --------------------------------------------

def test_cic_conserves_rays_in_interior():
    """Without lenses every ray whose four neighbouring pixel centres lie in
    the map deposits total weight 1."""
    g = _geom(0.25, 0.25, 0.0, [], [], (0, 0, 1), (-1, -1, 1, 1), (32, 32),
              ray_box=(-1.5, -0.75, 1.5, 0.75), ray_n=(300, 150))
    M = oracle.cic_forward(g, NO, NO, NO)
    # the lattice images into [-0.75, 0.75]^2, whose rays all have four in-map centres
    assert abs(M.sum() - g.n_rays) < 1e-8


def _one_ray_cic(bx, by):
    """CIC map of a single ray placed at source position (bx, by): no lenses,
    kappa = gamma = kappa_* = 0 (beta = theta), one lattice ray at the centre
    of its ray box, an 8 x 8 map of unit pixels over [0, 8]^2."""
    g = _geom(0.0, 0.0, 0.0, [], [], (0, 0, 1), (0.0, 0.0, 8.0, 8.0), (8, 8),
              ray_box=(bx - 0.25, by - 0.25, bx + 0.25, by + 0.25), ray_n=(1, 1))
    return oracle.cic_forward(g, NO, NO, NO)


@pytest.mark.parametrize("bx, by, want", [
    # pixel (i, j) has its centre at (i + 1/2, j + 1/2); a ray at x shares
    # 1 - |x - centre| with each of the two nearest centres along x, by hand:
    # x = 2.75 -> centres 2.5 (0.75) and 3.5 (0.25); y = 3.25 -> 2.5 (0.25), 3.5 (0.75)
    (2.75, 3.25, {(2, 2): 0.75 * 0.25, (3, 2): 0.25 * 0.25, (2, 3): 0.75 * 0.75, (3, 3): 0.25 * 0.75}),
    # x = 5.125 -> 4.5 (0.375), 5.5 (0.625); y = 1.625 -> 1.5 (0.875), 2.5 (0.125)
    (5.125, 1.625, {(4, 1): 0.375 * 0.875, (5, 1): 0.625 * 0.875, (4, 2): 0.375 * 0.125,
                    (5, 2): 0.625 * 0.125}),
    # a corner ray: only centre (0.5, 0.5) is in the map, weight 0.75 * 0.75;
    # the other three centres lie outside and their weights are dropped
    (0.25, 0.25, {(0, 0): 0.75 * 0.75}),
    # on the last column's centre line: all of x goes to column 7
    (7.5, 4.0, {(7, 3): 0.5, (7, 4): 0.5}),
])
def test_cic_single_ray_weights_by_hand(bx, by, want):
    """The four bilinear weights of one ray against hand-computed values:
    pixel centres at half-integers, and the weight along x going to the
    nearer centre (a dropped -1/2 or swapped neighbours fail here)."""
    M = _one_ray_cic(bx, by)
    expect = np.zeros((8, 8))
    for (i, j), v in want.items():
        expect[j, i] = v
    assert np.array_equal(M, expect), np.argwhere(M != expect)


def _tent_weights_1d(centres, positions, spacing):
    """Sum over positions of the tent kernel max(0, 1 - |p - c| / spacing) at
    each centre, in exact rational arithmetic."""
    from fractions import Fraction
    out = []
    for c in centres:
        s = Fraction(0)
        for p in positions:
            s += max(Fraction(0), 1 - abs(Fraction(p) - Fraction(c)) / Fraction(spacing))
        out.append(s)
    return np.array([float(v) for v in out])


def test_cic_dyadic_lattice_is_the_tent_kernel_sum():
    """No lenses, kappa = gamma = 1/4 (beta = (theta_x / 2, theta_y)): every
    lattice ray lands at a dyadic fraction of a pixel, and the CIC map equals,
    pixel by pixel, the outer product of the per-axis sums of the tent kernel
    over the rays' source positions (the definition of cloud-in-cell
    weights), computed exactly.  Interior pixels get exactly the rays per
    pixel (16); edge pixels lose the weight of centres outside the map."""
    g = _geom(0.25, 0.25, 0.0, [], [], (0, 0, 1), (-1.0, -0.5, 1.0, 0.5), (16, 8),
              ray_box=(-2.0, -0.5, 2.0, 0.5), ray_n=(64, 32))
    M = oracle.cic_forward(g, NO, NO, NO)
    dp = 0.125
    bx = [0.5 * (-2.0 + (i + 0.5) * 4.0 / 64) for i in range(64)]    # beta_x = theta_x / 2
    by = [-0.5 + (j + 0.5) / 32 for j in range(32)]                  # beta_y = theta_y
    wx = _tent_weights_1d([-1.0 + (i + 0.5) * dp for i in range(16)], bx, dp)
    wy = _tent_weights_1d([-0.5 + (j + 0.5) * dp for j in range(8)], by, dp)
    assert np.array_equal(M, np.outer(wy, wx))
    # 4 source positions per pixel along each axis: interior 4, edges 3.5
    assert np.all(wx[1:-1] == 4.0) and np.all(wy[1:-1] == 4.0)
    assert wx[0] == wx[-1] == 3.5 and wy[0] == wy[-1] == 3.5


def test_cic_gradient_refuses_the_strip_sheet():
    """dbeta/dkappa_* in the oracle's adjoint is the disc sheet's; a strip
    sheet is refused rather than given the disc's derivative."""
    lf = inputs.lens_disc(4, 3.0, 7, "lognormal")
    g = _geom(0.3, 0.2, 0.05, lf.x, lf.y, (0, 0, 3.0, "strip"), (-1.0, -1.0, 1.0, 1.0), (8, 8),
              ray_box=(-2, -2, 2, 2), ray_n=(40, 40))
    assert g.sheet_shape == 1
    with pytest.raises(ValueError):
        oracle.cic_grad_dM(g, lf.x, lf.y, lf.m, np.ones((8, 8)))
    g.sheet_shape = 0
    oracle.cic_grad_dM(g, lf.x, lf.y, lf.m, np.ones((8, 8)))


def test_cic_gradient_matches_finite_differences():
    lf = inputs.lens_disc(6, 5.0, 7, "lognormal")
    lt = inputs.lens_disc(6, 5.0, 8, "lognormal")
    g = _geom(0.3, 0.2, 0.05, lf.x, lf.y, (0, 0, 5.0), (-1.5, -1.5, 1.5, 1.5), (24, 24),
              ray_box=(-3, -2, 3, 2), ray_n=(600, 400))
    _, T = oracle.cic_loss(g, lt.x, lt.y, lt.m, np.zeros((24, 24)))
    gl, gp = oracle.cic_grad(g, lf.x, lf.y, lf.m, T)
    h = 1e-4
    for k in range(4):
        for c in range(3):
            arr = [lf.x.copy(), lf.y.copy(), lf.m.copy()]
            arr[c][k] += h
            lp, _ = oracle.cic_loss(g, *arr, T)
            arr[c][k] -= 2 * h
            lm, _ = oracle.cic_loss(g, *arr, T)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gl[k, c]) <= 0.01 * abs(gl[k, c]) + 1e-3 * np.abs(gl).max()
    for q, name in enumerate(("kappa", "gamma", "kappa_star")):
        lp, _ = oracle.cic_loss(dataclasses.replace(g, **{name: getattr(g, name) + h}),
                                lf.x, lf.y, lf.m, T)
        lm, _ = oracle.cic_loss(dataclasses.replace(g, **{name: getattr(g, name) - h}),
                                lf.x, lf.y, lf.m, T)
        assert abs((lp - lm) / (2 * h) - gp[q]) <= 0.01 * abs(gp[q])


# -- Light curves -------------------------------------------------------------

def test_gaussian_taps():
    w = oracle.gaussian_taps(0.5)
    assert len(w) == 5 and abs(w.sum() - 1) < 1e-15
    assert abs(w[1] / w[2] - math.exp(-2.0)) < 1e-15


def test_light_curves_pins():
    """A constant map stays constant away from the edge; a single bright
    pixel reproduces the source profile; a linear ramp is sampled exactly."""
    mu = np.full((40, 50), 3.5)
    tr = np.array([[10.0, 10.0, 40.0, 30.0]])
    lc = oracle.light_curves(mu, tr, 33, 0.5)
    assert np.allclose(lc, 3.5, rtol=0, atol=1e-14)

    delta = np.zeros((21, 21))
    delta[10, 10] = 1.0
    w = oracle.gaussian_taps(0.5)
    tr = np.array([[8.5, 10.5, 12.5, 10.5]])                # along the centre row
    lc = oracle.light_curves(delta, tr, 5, 0.5)
    assert np.allclose(lc[0], w[2] * w, rtol=0, atol=1e-15)

    yy, xx = np.mgrid[0:30, 0:30]
    ramp = 0.25 * xx - 0.5 * yy + 3.0
    tr = np.array([[6.3, 7.1, 21.7, 19.9]])
    lc = oracle.light_curves(ramp, tr, 17, 0.5)
    t = np.linspace(0, 1, 17)
    u = 6.3 + t * (21.7 - 6.3) - 0.5
    v = 7.1 + t * (19.9 - 7.1) - 0.5
    assert np.allclose(lc[0], 0.25 * u - 0.5 * v + 3.0, rtol=0, atol=1e-12)


def test_light_curves_sampled_equals_whole_map_convolution():
    """The per-sample convolution (for production-size maps) against the
    whole-map one, on tracks that run into the map's edges and corners and
    past them, at two source sizes: identical to the last bit, since the
    sums are taken in the same order; and the pins above hold for it too."""
    rng = np.random.default_rng(4)
    mu = rng.uniform(0.0, 5.0, (37, 53))
    tr = np.array([[-3.0, -2.0, 60.0, 41.0], [0.0, 36.9, 52.9, 0.2], [0.4, 0.4, 0.6, 36.6],
                   [25.0, 18.0, 25.0, 18.0], [52.5, 10.0, 40.0, 36.5]])
    for sigma in (0.5, 1.3):
        a = oracle.light_curves(mu, tr, 101, sigma)
        b = oracle.light_curves_sampled(mu, tr, 101, sigma)
        assert np.array_equal(a, b)
    delta = np.zeros((21, 21))
    delta[10, 10] = 1.0
    w = oracle.gaussian_taps(0.5)
    lc = oracle.light_curves_sampled(delta, np.array([[8.5, 10.5, 12.5, 10.5]]), 5, 0.5)
    assert np.allclose(lc[0], w[2] * w, rtol=0, atol=1e-15)


# -- Fold macro model (Eq. 4-6) --------------------------------------------------

FOLD = ("fold", 0.83, 0.05, -0.047)   # kappa_0 of Table 1, d scaled up so that the image plane is small


def _fold_geom(map_box, map_n, ray_box=None, ray_n=None, n_av=0.0, kappa_star=0.0, sheet=(0, 0, 1e6)):
    return oracle.derive_geometry(0.0, 0.0, kappa_star, [], [], sheet, map_box, map_n,
                                  ray_box=ray_box, ray_n=ray_n, n_av=n_av, macro=FOLD)


def test_fold_jacobian_is_eq4():
    """Central differences of the oracle's beta (no lenses) at lattice
    neighbours: for the quadratic map they are exact up to rounding.  Eq. 4
    fixes A_11 = theta . d, A_21 = 0, A_22 = 2 (1 - kappa_0) and so the
    determinant; A_12 = d_y theta_x is what integrating Eq. 5 as printed gives."""
    _, k0, dx, dy = FOLD
    h = 1e-2
    for tx, ty in [(3.0, 1.0), (-7.5, 2.0), (12.0, -4.0), (0.3, 0.2)]:
        g = _fold_geom((0, 0, 1, 1), (4, 4), ray_box=(tx - 1.5 * h, ty - 1.5 * h, tx + 1.5 * h, ty + 1.5 * h),
                       ray_n=(3, 3))
        b, _ = oracle.beta_direct(g, NO, NO, NO, np.arange(9))
        b = b.reshape(3, 3, 2)                      # [j][i]
        A11 = (b[1, 2, 0] - b[1, 0, 0]) / (2 * h)
        A12 = (b[2, 1, 0] - b[0, 1, 0]) / (2 * h)
        A21 = (b[1, 2, 1] - b[1, 0, 1]) / (2 * h)
        A22 = (b[2, 1, 1] - b[0, 1, 1]) / (2 * h)
        assert abs(A11 - (dx * tx + dy * ty)) <= 1e-9
        assert abs(A21) <= 1e-9 and abs(A22 - 2 * (1 - k0)) <= 1e-9
        assert abs(A12 - dy * tx) <= 1e-9
        assert abs((A11 * A22 - A12 * A21) - 2 * (1 - k0) * (dx * tx + dy * ty)) <= 1e-8


def test_fold_ray_box_holds_every_image_and_is_tight():
    box = (0.2, -1.0, 3.0, 1.5)
    x0, y0, x1, y1 = oracle.fold_ray_box(*FOLD[1:], box)
    # map a lattice over a larger rectangle with the oracle (no lenses)
    wide = (x0 - 3, y0 - 1, x1 + 3, y1 + 1)
    g = _fold_geom((0, 0, 1, 1), (4, 4), ray_box=wide, ray_n=(1200, 300))
    b, _ = oracle.beta_direct(g, NO, NO, NO, np.arange(g.n_rays))
    tx, ty = oracle.ray_position(g, np.arange(g.n_rays))
    inside = (b[:, 0] >= box[0]) & (b[:, 0] <= box[2]) & (b[:, 1] >= box[1]) & (b[:, 1] <= box[3])
    assert inside.sum() > 1000
    assert np.all((tx[inside] >= x0) & (tx[inside] <= x1) & (ty[inside] >= y0) & (ty[inside] <= y1))
    # tight: images come within two lattice spacings of every side
    assert tx[inside].min() - x0 < 2 * g.l3x and x1 - tx[inside].max() < 2 * g.l3x
    assert ty[inside].min() - y0 < 2 * g.l3y and y1 - ty[inside].max() < 2 * g.l3y


def test_fold_map_without_lenses_is_the_two_image_magnification():
    """No lenses, no sheet: every source point above the caustic has two images
    with |det A| = 2 (1 - kappa_0) d_x s each, s = |theta_x - theta_*| (Eq. 4),
    so mu(beta) = 1 / ((1 - kappa_0) d_x s(beta)),
    s = sqrt(2 beta_x / d_x + (d_y theta_y / d_x)^2), theta_y = beta_y / (2 (1 - kappa_0)).
    Pixel means of that closed form by Gauss-Legendre quadrature against the
    oracle's ray counts."""
    _, k0, dx, dy = FOLD
    box, n = (0.5, -1.0, 3.5, 1.0), (24, 16)
    g = _fold_geom(box, n, n_av=30000.0)
    counts, st = oracle.shoot_direct(g, NO, NO, NO)
    mu = counts * oracle.cic_mu_scale(g)
    xg, wg = np.polynomial.legendre.leggauss(8)
    ref = np.zeros(n[::-1])
    for j in range(n[1]):
        for i in range(n[0]):
            bx = g.mx0 + (i + 0.5 + 0.5 * xg) * g.dpx
            by = g.my0 + (j + 0.5 + 0.5 * xg) * g.dpy
            BX, BY = np.meshgrid(bx, by)
            ty = BY / (2 * (1 - k0))
            s = np.sqrt(2 * BX / dx + (dy * ty / dx) ** 2)
            ref[j, i] = (np.outer(wg, wg) * (1.0 / ((1 - k0) * dx * s))).sum() / 4.0
    rel = np.abs(mu - ref) / ref
    assert abs(mu.sum() / ref.sum() - 1) < 1e-4          # the map's total
    assert rel.mean() < 0.006, rel.mean()                 # lattice sampling: 0.3 % here
    assert rel.max() < 0.02, rel.max()


def test_strip_sheet_cancels_the_mean_field_of_a_long_lens_strip():
    """A long strip of lenses of density kappa_* (a regular grid, unit
    spacing cells of mass kappa_* a^2 / pi) and the strip sheet of the same
    density: far from the strip's ends the two fields cancel, so with a macro
    term theta (kappa = gamma = 0) beta = theta.  Pins the strip sheet's
    factor 2 (Gauss: a slab's field is 2 kappa_* (theta_y - c_y)) and sign."""
    a, h, L, ks = 0.1, 1.0, 100.0, 0.1
    xs = np.arange(-L + a / 2, L, a)
    ys = np.arange(-h + a / 2, h, a)
    X, Y = np.meshgrid(xs, ys)
    m = np.full(X.size, ks * a * a / math.pi)
    for tx, ty in [(0.0, 0.5), (3.0, -0.3), (-10.0, 0.9)]:
        g = _geom(0.0, 0.0, ks, X.ravel(), Y.ravel(), (0.0, 0.0, h, "strip"), (-1, -1, 1, 1), (8, 8),
                  ray_box=(tx - 0.5 * a, ty - 0.5 * a, tx + 0.5 * a, ty + 0.5 * a), ray_n=(1, 1))
        b, _ = oracle.beta_direct(g, X.ravel(), Y.ravel(), m, np.array([0]))
        # the strip's finite ends leave an x field of (kappa_* / pi) 2h ln((L + x)/(L - x))
        ends = ks / math.pi * 2 * h * abs(math.log((L + tx) / (L - tx)))
        assert abs(b[0, 0] - tx) <= 1.1 * ends + 1e-5, (b[0], tx, ends)
        assert abs(b[0, 1] - ty) <= 0.02 * 2 * ks * abs(ty) + 1e-4, (b[0], tx, ty)
        # without the sheet the lens strip alone deflects by about 2 kappa_* theta_y
        g0 = _geom(0.0, 0.0, 0.0, X.ravel(), Y.ravel(), (0.0, 0.0, h, "strip"), (-1, -1, 1, 1), (8, 8),
                   ray_box=(tx - 0.5 * a, ty - 0.5 * a, tx + 0.5 * a, ty + 0.5 * a), ray_n=(1, 1))
        b0, _ = oracle.beta_direct(g0, X.ravel(), Y.ravel(), m, np.array([0]))
        assert abs((ty - b0[0, 1]) - 2 * ks * ty) <= 0.02 * 2 * ks * abs(ty)


# -- Peak identification (§4.2) ---------------------------------------------------

def test_peaks_ridge_spike_and_threshold():
    """A ridge crossing five curves at one position: candidates on all five,
    true peaks on the inner three (each has candidate neighbours on both
    sides); an isolated spike is a candidate only; a bump below 5 sigma is
    nothing.  Along y the transposed map gives the transposed mask."""
    N = np.full((9, 12), 1000, np.int64)
    N[2:7, 5] = 1300            # h = 200 > 5 sqrt(1100) = 165.8
    N[1, 9] = 1400              # isolated
    N[7, 2] = 1200              # h = 133 < 5 sqrt(1067) = 163.3
    m = oracle.peaks(N)
    assert np.array_equal(np.nonzero(m & 1)[0], [1, 2, 3, 4, 5, 6])
    assert set(zip(*np.nonzero(m & 1))) == {(1, 9), (2, 5), (3, 5), (4, 5), (5, 5), (6, 5)}
    assert set(zip(*np.nonzero(m & 2))) == {(3, 5), (4, 5), (5, 5)}
    assert np.array_equal(oracle.peaks(N.T, along="y"), m.T)


def test_peaks_threshold_is_strict_and_exact():
    """The oracle's squared integer form of h > 5 sigma against the criterion
    as the paper states it (h = N - <N> against 5 sqrt(<N>)), by brute force
    over N for two neighbours of 1000: both switch at the same N, and the
    comparison is strict."""
    a = b = 1000
    first = None
    for c in range(1001, 1400):
        mean = (a + b + c) / 3.0
        if (c - mean) > 5.0 * math.sqrt(mean) + 1e-9:
            first = c
            break
    N = np.full((3, 3), a, np.int64)
    N[1, 1] = first - 1
    assert not (oracle.peaks(N)[1, 1] & 1)
    N[1, 1] = first
    assert oracle.peaks(N)[1, 1] & 1
    # ties are not peaks: N must exceed both neighbours
    N = np.array([[5, 5, 5], [1000, 5000, 5000], [5, 5, 5]])
    assert not (oracle.peaks(N)[1, 1] & 1)


def test_peaks_of_poisson_noise_are_rare():
    """A flat Poisson map (mean 1000): 5 sigma candidates occur with
    probability about 3e-7 per pixel, true peaks (three aligned) never."""
    N = np.random.default_rng(3).poisson(1000.0, (200, 300))
    m = oracle.peaks(N)
    assert (m & 1).sum() <= 2 and (m & 2).sum() == 0


def test_peak_statistics_by_hand():
    """The ridge map of the peak pins, binned by hand: the three true peaks sit
    at j = 5 (d = 5.5 with origin 0, step 1, caustic 0); the seven interior
    curves scan positions j = 1..10, four of them in [0, 5), one in [5, 6),
    five in [6, 12).  An edge at exactly d = 5.5 puts j = 5 in the upper bin."""
    N = np.full((9, 12), 1000, np.int64)
    N[2:7, 5] = 1300
    N[1, 9] = 1400
    N[7, 2] = 1200
    m = oracle.peaks(N)
    n, s, p = oracle.peak_statistics(N, m, "x", 0.0, 1.0, 0.0, [0.0, 5.0, 6.0, 12.0])
    assert list(n) == [0, 3, 0] and list(s) == [0, 3900, 0] and list(p) == [28, 7, 35]
    n, s, p = oracle.peak_statistics(N, m, "x", 0.0, 1.0, 0.0, [0.0, 5.5, 12.0])
    assert list(n) == [0, 3] and list(p) == [28, 42]
    # positions beyond the last edge, or before the first, fall in no bin
    n, s, p = oracle.peak_statistics(N, m, "x", 0.0, 1.0, 0.0, [6.0, 12.0])
    assert list(n) == [0] and list(p) == [35]
    # along y: the curves are the columns, the ridge crosses none of them as a peak
    n, s, p = oracle.peak_statistics(N, oracle.peaks(N, "y"), "y", 0.0, 1.0, 0.0, [0.0, 9.0])
    assert list(n) == [0] and list(p) == [10 * 7]


def test_peak_statistics_of_periodic_crossings():
    """Ridges across every curve at every fourth position: the crossings per
    unit length of curve are exactly 1/(4 step) in each bin spanning whole
    periods, the mean peak count is the ridge's, and a caustic in the middle of
    the map folds the two sides onto the same distances."""
    nx, ny, step = 42, 30, 0.25
    N = np.full((ny, nx), 1000, np.int64)
    N[:, 3:40:4] = 1400
    m = oracle.peaks(N)
    assert (m & 2).sum() // 2 == 10 * (ny - 2)
    edges = [1.0 * step, 21.0 * step, 41.0 * step]          # j = 1..20 and 21..40
    n, s, p = oracle.peak_statistics(N, m, "x", 0.0, step, 0.0, edges)
    assert list(n) == [5 * (ny - 2)] * 2 and list(p) == [20 * (ny - 2)] * 2
    assert np.all(n * 4 == p) and np.all(s == 1400 * n)
    # caustic at the map's centre (x = 21 step): positions j and 41 - j are
    # equidistant; the ridges at j = 3 + 4k map onto j = 38 - 4k, none of which
    # is a ridge, so every bin of half-width step gathers exactly one side's peaks
    c = 21.0 * step
    half = [k * step for k in range(0, 21)]
    n2, _, p2 = oracle.peak_statistics(N, m, "x", 0.0, step, c, half)
    assert int(n2.sum()) == 10 * (ny - 2)
    assert int(p2.sum()) == 40 * (ny - 2) and np.all(p2 == 2 * (ny - 2))


def test_peak_statistics_totals_on_a_noisy_map():
    """Bins that cover every distance add up to the whole mask: all true
    peaks, the sum of their counts, and (ny - 2)(nx - 2) positions, along
    either direction."""
    rng = np.random.default_rng(11)
    N = rng.poisson(900.0, (50, 70)).astype(np.int64)
    N[5:20, 30] += 500
    N[40, 10:30] += 500
    for along, (nc, ln) in (("x", (50, 70)), ("y", (70, 50))):
        m = oracle.peaks(N, along)
        n, s, p = oracle.peak_statistics(N, m, along, -3.0, 0.1, 1.0, [0.0, 0.5, 2.0, 10.0])
        tp = (m & 2).astype(bool)
        assert int(n.sum()) == int(tp.sum()) > 0
        assert int(s.sum()) == int(N[tp].sum())
        assert int(p.sum()) == (nc - 2) * (ln - 2)
