"""The seeded input generators shared by the CUDA path's tests and the oracle.

They hold none of the method's arithmetic; these checks pin them to their
published definitions and to the distributions the workloads state.
"""
import math

import numpy as np

from paper_2308_14278_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    """Seed 0, stream 0 starts from state 0, so its outputs are SplitMix64's
    first outputs from x = 0 (Steele, Lea & Flood 2014, in Vigna's reference
    form): e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f, f88bb8a8724c81ec."""
    got = [int(v) for v in inputs.splitmix64(0, 0, 4)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_is_counter_based():
    """Output k depends on (seed, stream, k) only: any window of a stream is
    the same slice of the whole stream, and streams and seeds differ."""
    whole = inputs.splitmix64(7, 3, 1000)
    assert np.array_equal(inputs.splitmix64(7, 3, 100, offset=450), whole[450:550])
    assert not np.array_equal(inputs.splitmix64(7, 4, 1000), whole)
    assert not np.array_equal(inputs.splitmix64(8, 3, 1000), whole)


def test_uniform01_takes_the_top_53_bits():
    z = inputs.splitmix64(5, 9, 10000)
    u = inputs.uniform01(5, 9, 10000)
    assert np.array_equal(u * 2.0 ** 53, (z >> np.uint64(11)).astype(np.float64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01


def test_std_normal_moments():
    z = inputs.std_normal(1, 40, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(np.abs(z) < 1.0) - 0.682689) < 0.005


def test_lens_disc_is_uniform_and_lognormal():
    """Uniform in the disc: every lens inside R, and the fraction inside R/2 is
    1/4; lognormal masses: median and log-spread as asked, mean by the closed
    form median exp(sigma^2 / 2)."""
    lf = inputs.lens_disc(100000, 30.0, seed=2, mass="lognormal", median=0.3, sigma_ln=0.5,
                          cx=1.0, cy=-2.0)
    r = np.hypot(lf.x - 1.0, lf.y + 2.0)
    assert r.max() <= 30.0 and abs(np.mean(r < 15.0) - 0.25) < 0.005
    assert abs(np.median(lf.m) - 0.3) < 0.005
    assert abs(np.std(np.log(lf.m)) - 0.5) < 0.005
    assert abs(lf.m.mean() / inputs.lognormal_mean(0.3, 0.5) - 1.0) < 0.01
    assert math.isclose(inputs.lognormal_mean(0.3, 0.5), 0.3 * math.exp(0.125))


def test_tracks_stay_inside_the_margin():
    tr = inputs.tracks(500, 8192, 4096, 3.0, seed=1)
    assert tr.shape == (500, 4)
    assert tr[:, [0, 2]].min() >= 3.0 and tr[:, [0, 2]].max() <= 8192 - 3.0
    assert tr[:, [1, 3]].min() >= 3.0 and tr[:, [1, 3]].max() <= 4096 - 3.0


def test_paper_map_workload_follows_its_recipe():
    """13,000 lenses in the disc R = sqrt(N <m> / kappa_*), kappa = 0.48,
    gamma = 0.50, kappa_* = 0.005, a 23.65 theta_E square map of 8192^2
    pixels and N_av = 1e11 / 8192^2."""
    w = inputs.paper_map(0, n_rays=1e11, map_px=8192)
    assert w.lenses.n == 13000
    assert (w.kappa, w.gamma, w.kappa_star) == (0.48, 0.50, 0.005)
    R = math.sqrt(13000 * inputs.lognormal_mean(0.3, 0.5) / 0.005)
    assert abs(w.lenses.radius - R) < 1e-9 * R and abs(R - 940.13) < 0.01
    x0, y0, x1, y1 = w.map_box
    assert abs((x1 - x0) - 23.65) < 0.01 and abs((y1 - y0) - (x1 - x0)) < 1e-12
    assert w.map_n == (8192, 8192) and math.isclose(w.n_av, 1e11 / 8192 ** 2)


def test_fold_field_follows_table1():
    """Table 1's fold field: kappa_0 = 0.83, d converted from arcmin^-1 to
    1/theta_E, kappa_* = 0.001, 13,745 unit masses uniform in the lens
    rectangle, a strip sheet over the rectangle's y range; the rectangle holds
    the image of the protected source region (the oracle's fold image box) and,
    at kappa_* = 0.001, about Table 1's N_* lenses (N_* = L_ix L_iy kappa_*/pi)."""
    import oracle
    w = inputs.fold_field(0, n_rays=1e11)
    assert w.macro[0] == "fold" and w.macro[1] == 0.83
    assert math.isclose(w.macro[2], 3.62 * 1e-6 / 60.0) and math.isclose(w.macro[3], -3.41 * 1e-6 / 60.0)
    assert w.lenses.n == 13745 and np.all(w.lenses.m == 1.0) and w.kappa_star == 0.001
    x0, y0, x1, y1 = inputs.TABLE1_LENS_RECT
    assert w.lenses.x.min() >= x0 and w.lenses.x.max() <= x1
    assert w.lenses.y.min() >= y0 and w.lenses.y.max() <= y1
    assert w.sheet[3] == "strip" and math.isclose(w.sheet[2], 0.5 * (y1 - y0))
    assert w.map_box == (0.0, 0.0, 40.0, 200.0) and w.map_n == (2048, 10240)
    band = 10.0 * math.sqrt(0.001)
    bx0, by0, bx1, by1 = oracle.fold_ray_box(*w.macro[1:], (-band, -band, 40.0 + band, 200.0 + band))
    assert x0 <= bx0 and y0 <= by0 and x1 >= bx1 and y1 >= by1
    n_star = (x1 - x0) * (y1 - y0) * 0.001 / math.pi
    assert abs(n_star / 13745 - 1.0) < 0.01


def test_batched_maps_follow_their_recipe():
    """80 maps: N uniform in 2,000..20,000, kappa_* from {0.002, 0.005,
    0.01}, gamma = 0.5 with kappa + gamma in [0.95, 0.99], rays log-uniform in
    [1e9, 1e10], 4096^2 maps, each disc 1.5 x the ray rectangle's half-diagonal."""
    ws = inputs.batched_maps(n_maps=80, seed=0)
    assert len(ws) == 80
    for w in ws:
        assert 2000 <= w.lenses.n <= 20000
        assert w.kappa_star in (0.002, 0.005, 0.01)
        assert w.gamma == 0.5 and 0.95 <= w.kappa + w.gamma <= 0.99
        rays = w.n_av * w.map_n[0] * w.map_n[1]
        assert 1e9 * (1 - 1e-12) <= rays <= 1e10 * (1 + 1e-12)
        assert w.map_n == (4096, 4096)
        R = math.sqrt(w.lenses.n * inputs.lognormal_mean(0.3, 0.5) / w.kappa_star)
        assert math.isclose(w.lenses.radius, R, rel_tol=1e-12)
    assert len({w.kappa_star for w in ws}) == 3
    assert len({w.lenses.n for w in ws}) > 70
    import oracle
    for w in ws[:8]:
        g = oracle.geometry_of(w)
        half_diagonal = 0.5 * math.hypot(g.rx1 - g.rx0, g.ry1 - g.ry0)
        assert math.isclose(w.lenses.radius, 1.5 * half_diagonal, rel_tol=1e-12)


def test_differentiable_field_follows_its_recipe():
    w = inputs.differentiable_field(0)
    assert w.lenses.n == 1000 and (w.kappa, w.gamma, w.kappa_star) == (0.48, 0.50, 0.005)
    assert w.map_n == (1024, 1024) and math.isclose(w.n_av * 1024 * 1024, 4e8)
    assert w.l1 == (2.5, 2.5) and w.l2 == (10, 10)
    R = math.sqrt(1000 * inputs.lognormal_mean(0.3, 0.5) / 0.005)
    assert math.isclose(w.sheet[2], R) and np.all(np.hypot(w.lenses.x, w.lenses.y) <= R)
    # the target of the loss is the same recipe from another seed
    t = inputs.differentiable_field(1000)
    assert not np.array_equal(t.lenses.x, w.lenses.x) and t.map_box == w.map_box
