"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (stated here, derived in the design notes):
  * FP64 modes: integer counts equal except for rays within 1e-5 px of a bin
    edge; source positions within 1e-10 theta_E of the oracle.
  * mixed mode: per-ray deflection within 1e-5 relative of the FP64 direct sum
    (denominator max(|alpha|, 0.01 theta_E)); map relative L1 error <= 1e-3;
    every pixel-decision mismatch comes from a ray whose oracle position lies
    within its own measured error of a bin edge.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_DEFLECTION = 1e-5
ALPHA_FLOOR = 1e-2
MAP_L1 = 1e-3


def _field(ml, w, **kw):
    return ml.Field(w, **kw)


def _geometry(w, f):
    """Oracle geometry with the Taylor order the library chose."""
    return oracle.geometry_of(w, p=max(1, f.info["taylor_p"]))


def _alpha_ref(g, idx, beta_ref):
    tx, ty = oracle.ray_position(g, idx)
    ax = (1 - g.kappa - g.gamma) * tx + g.kappa_star * (tx - g.sheet_cx) - beta_ref[:, 0]
    ay = (1 - g.kappa + g.gamma) * ty + g.kappa_star * (ty - g.sheet_cy) - beta_ref[:, 1]
    return np.hypot(ax, ay)


def _edge_distance_px(g, beta):
    fx = (beta[:, 0] - g.mx0) / g.dpx
    fy = (beta[:, 1] - g.my0) / g.dpy
    return np.minimum(np.abs(fx - np.round(fx)), np.abs(fy - np.round(fy)))


def _check_geometry(f, g):
    info = f.info
    for k in ("n_rays_x", "n_rays_y", "n1x", "n1y", "n2x", "n2y", "N1x", "N1y"):
        ok = {"n_rays_x": g.n3x, "n_rays_y": g.n3y}.get(k, getattr(g, k, None))
        assert info[k] == ok, k
    assert info["n_star_in"] == g.n_star_in
    for k, v in (("ray_x0", g.rx0), ("ray_y0", g.ry0), ("ray_x1", g.rx1), ("ray_y1", g.ry1),
                 ("l3x", g.l3x), ("l3y", g.l3y), ("dpx", g.dpx), ("dpy", g.dpy)):
        assert info[k] == pytest.approx(v, rel=1e-15, abs=1e-15), k


# ---------------------------------------------------------------------------
# FP64 modes
# ---------------------------------------------------------------------------

def test_small_map_direct64_counts(ml):
    """100 lenses, 2000^2 rays, 256^2 map, FP64 direct sum: counts equal the
    oracle's except for rays within 1e-5 px of a bin edge."""
    w = inputs.small_map(0)
    f = _field(ml, w, precision=ml.PREC_DIRECT64)
    g = _geometry(w, f)
    _check_geometry(f, g)
    f.shoot()
    got = f.counts().cpu().numpy().astype(np.int64)
    st = f.stats()
    ref, rst = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m)
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == g.n_rays
    idx = np.arange(g.n_rays)
    beta, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    n_edge = int(np.sum(_edge_distance_px(g, beta) < 1e-5))
    diff = int(np.abs(got - ref.astype(np.int64)).sum())
    assert diff <= 2 * n_edge
    assert st["rays_in"] == int(got.sum())
    f.close()


@pytest.mark.parametrize("precision", ["direct64", "nearfar64"])
def test_fp64_trace_matches_oracle(ml, precision):
    lf = inputs.lens_disc(60, 8.0, 3, "lognormal")
    w = inputs.Workload("t", lf, 0.42, 0.31, 0.03, (0.0, 0.0, 8.0), (-1.5, -1.2, 1.7, 1.4),
                        (96, 80), ray_box=(-5.0, -3.0, 5.5, 3.5), ray_n=(1201, 777))
    prec = ml.PREC_DIRECT64 if precision == "direct64" else ml.PREC_NEARFAR64
    f = _field(ml, w, precision=prec, taylor_p=5, build=ml.BUILD_DIRECT)
    g = _geometry(w, f)
    _check_geometry(f, g)
    idx = np.unique(np.linspace(0, g.n_rays - 1, 5000).astype(np.int64))
    beta, pix = f.trace(idx)
    beta = beta.cpu().numpy()
    if precision == "direct64":
        ref, flag = oracle.beta_direct(g, lf.x, lf.y, lf.m, idx)
    else:
        ref, flag = oracle.beta_interp(g, lf.x, lf.y, lf.m, idx)
    assert np.max(np.abs(beta - ref)) < 1e-10
    px, py = oracle.pixel_of(g, ref)
    inside = (px >= 0) & (px < g.mnx) & (py >= 0) & (py < g.mny)
    pix = pix.cpu().numpy()
    near_edge = _edge_distance_px(g, ref) < 1e-6
    ok = near_edge | (inside & (pix[:, 0] == px) & (pix[:, 1] == py)) | (~inside & (pix[:, 0] == -1))
    assert ok.all()
    f.close()


@pytest.mark.parametrize("case", ["small", "paper", "table1"])
def test_hierarchical_build_matches_direct(ml, case):
    """The hierarchical coefficient build (box and sub-block expansions
    shifted to the nodes) against the direct sum at every node, through FP64
    near/far traces: the two differ only by series truncation and rounding.
    The paper-scale map has most lenses outside the binning ring (the outer
    lenses' box index); the Table-1 fold field fills its lattice with lenses
    (a strip sheet), on a coarse level-2 grid so that the direct sum stays
    quick."""
    kw = {}
    if case == "small":
        lf = inputs.lens_disc(60, 8.0, 3, "lognormal")
        w = inputs.Workload("t", lf, 0.42, 0.31, 0.03, (0.0, 0.0, 8.0), (-1.5, -1.2, 1.7, 1.4),
                            (96, 80), ray_box=(-5.0, -3.0, 5.5, 3.5), ray_n=(1201, 777))
    elif case == "paper":
        w = inputs.paper_map(0, n_rays=1e10, map_px=2048)
    else:
        w = inputs.fold_field(0, n_rays=2e9, map_px=(512, 2560))
        kw = dict(l2_sub=(4, 4))
    fd = _field(ml, w, precision=ml.PREC_NEARFAR64, taylor_p=8, build=ml.BUILD_DIRECT, **kw)
    fh = _field(ml, w, precision=ml.PREC_NEARFAR64, taylor_p=8, build=ml.BUILD_HIERARCHICAL, **kw)
    assert fd.info["build"] == ml.BUILD_DIRECT and fh.info["build"] == ml.BUILD_HIERARCHICAL
    n = fd.n_rays
    idx = np.unique(np.random.default_rng(2).integers(0, n, 20000))
    bd, _ = fd.trace(idx)
    bh, _ = fh.trace(idx)
    assert float((bd - bh).abs().max()) < 1e-9
    fd.close()
    fh.close()


@pytest.mark.parametrize("case", ["paper", "table1"])
def test_hierarchical_build_matches_interp_oracle(ml, case):
    """The default hierarchical build traced in the FP64 near/far mode against
    the oracle's near/far scheme (oracle.beta_interp: the node series of each
    ray from a direct sum over the far lenses, §3.2 Level 2), on the
    paper-scale field and on the Table-1 fold field: both evaluate the same
    truncated series, so they agree to FP64 rounding of the sums."""
    if case == "paper":
        w = inputs.paper_map(0, n_rays=1e10, map_px=2048)
        kw = {}
    else:
        w = inputs.fold_field(0, n_rays=2e9, map_px=(512, 2560))
        kw = dict(l2_sub=(4, 4))
    f = _field(ml, w, precision=ml.PREC_NEARFAR64, taylor_p=8, build=ml.BUILD_HIERARCHICAL, **kw)
    info = f.info
    assert info["build"] == ml.BUILD_HIERARCHICAL and info["taylor_p"] == 8
    g = oracle.geometry_of(w, p=8, l2_sub=info["l2_sub_x"], l2_sub_y=info["l2_sub_y"],
                           l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))
    _check_geometry(f, g)
    idx = np.unique(np.random.default_rng(4).integers(0, g.n_rays, 20000))
    beta, _ = f.trace(idx)
    ref, flag = oracle.beta_interp(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    assert not flag.any()
    err = np.abs(beta.cpu().numpy() - ref).max()
    assert err <= 1e-9, err
    f.close()


def test_nearfar64_map_matches_interp_oracle_stripe(ml):
    lf = inputs.lens_disc(60, 8.0, 4, "lognormal")
    w = inputs.Workload("t", lf, 0.42, 0.31, 0.03, (0.0, 0.0, 8.0), (-1.5, -1.2, 1.7, 1.4),
                        (96, 80), ray_box=(-5.0, -3.0, 5.5, 3.5), ray_n=(1201, 777))
    f = _field(ml, w, precision=ml.PREC_NEARFAR64, taylor_p=8)
    g = _geometry(w, f)
    r0, r1 = 123457, 123457 + 300001
    f.shoot(r0, r1)
    got = f.counts().cpu().numpy().astype(np.int64)
    ref, rst = oracle.shoot_direct(g, lf.x, lf.y, lf.m, r0, r1)
    l1 = np.abs(got - ref.astype(np.int64)).sum() / max(1, ref.sum())
    assert l1 <= MAP_L1
    st = f.stats()
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == r1 - r0
    f.close()


# ---------------------------------------------------------------------------
# Mixed precision: the hot path
# ---------------------------------------------------------------------------

def test_mixed_uniform_map_exact(ml):
    """No lenses, dyadic spacings: every pixel receives exactly 32 rays, as the
    oracle's exact lattice count says; mu = 1/det = 2 (Eq. 12)."""
    lf = inputs.LensField(np.zeros(0), np.zeros(0), np.zeros(0))
    w = inputs.Workload("uniform", lf, 0.25, 0.25, 0.0, (0.0, 0.0, 10.0), (-1, -1, 1, 1), (32, 32),
                        ray_box=(-2.0, -1.0, 2.0, 1.0), ray_n=(256, 128))
    f = _field(ml, w, precision=ml.PREC_MIXED, taylor_p=3)
    f.shoot()
    counts = f.counts().cpu().numpy()
    ref, _ = oracle.shoot_direct(oracle.geometry_of(w), lf.x, lf.y, lf.m)
    assert np.array_equal(counts.astype(np.uint64), ref)
    mu = f.mu("f64").cpu().numpy()
    assert np.all(mu == 2.0)
    st = f.stats()
    assert st["rays_in"] == 256 * 128 and st["rays_out"] == 0
    f.close()


def _mixed_case(seed=5, kappa=0.40, gamma=0.45, ks=0.05, n_av=60):
    """A consistent field near the critical line: lognormal lenses in a disc
    1.5 times the ray rectangle's half-diagonal, kappa_* = N <m> / R^2."""
    box, npx = (-1.0, -0.75, 1.0, 0.75), (200, 150)
    g0 = oracle.derive_geometry(kappa, gamma, ks, [], [], (0, 0, 1), box, npx, n_av=n_av)
    r = 1.5 * math.hypot(max(abs(g0.rx0), abs(g0.rx1)), max(abs(g0.ry0), abs(g0.ry1)))
    n = int(round(ks * r * r / inputs.lognormal_mean(0.3, 0.5)))
    lf = inputs.lens_disc(n, r, seed, "lognormal")
    ks = n * inputs.lognormal_mean(0.3, 0.5) / r ** 2
    return inputs.Workload("mixed", lf, kappa, gamma, ks, (0.0, 0.0, r), box, npx, n_av=n_av)


@pytest.mark.parametrize("l2_sub", [(20, 20), (60, 20), (20, 40)])
def test_mixed_trace_deflection_and_bins(ml, l2_sub):
    w = _mixed_case()
    f = _field(ml, w, precision=ml.PREC_MIXED, l2_sub=l2_sub)
    assert (f.info["l2_sub_x"], f.info["l2_sub_y"]) == l2_sub
    g = oracle.geometry_of(w, p=f.info["taylor_p"], l2_sub=l2_sub[0], l2_sub_y=l2_sub[1])
    _check_geometry(f, g)
    assert f.info["far_bound"] <= 1e-7
    idx = np.unique(np.random.default_rng(1).integers(0, g.n_rays, 40000))
    beta, pix = f.trace(idx)
    beta, pix = beta.cpu().numpy(), pix.cpu().numpy()
    ref, flag = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    alpha = _alpha_ref(g, idx, ref)
    err = np.hypot(*(beta - ref).T)
    rel = err / np.maximum(alpha, ALPHA_FLOOR)
    assert np.max(rel) <= REL_DEFLECTION, np.max(rel)
    px, py = oracle.pixel_of(g, ref)
    inside = (px >= 0) & (px < g.mnx) & (py >= 0) & (py < g.mny)
    same = np.where(inside, (pix[:, 0] == px) & (pix[:, 1] == py), pix[:, 0] == -1)
    dist = _edge_distance_px(g, ref)
    err_px = np.maximum(np.abs(beta - ref)[:, 0] / g.dpx, np.abs(beta - ref)[:, 1] / g.dpy)
    assert np.all(same | (dist <= err_px * (1 + 1e-6) + 1e-9))
    f.close()


def _traced_counts(ml, f, r0, r1, chunk=1 << 22):
    """Histogram of the pixels ml_trace_rays gives every ray of [r0, r1),
    with the number of rays outside the map and of dropped rays."""
    import torch
    nx, ny = f.info["map_nx"], f.info["map_ny"]
    counts = torch.zeros(nx * ny, dtype=torch.int64, device="cuda")
    n_out = n_drop = 0
    for a in range(r0, r1, chunk):
        idx = torch.arange(a, min(r1, a + chunk), dtype=torch.int64, device="cuda")
        beta = torch.empty((idx.numel(), 2), dtype=torch.float64, device="cuda")
        pix = torch.empty((idx.numel(), 2), dtype=torch.int32, device="cuda")
        ml.ml_trace_rays(f.h, idx, beta, pix)
        inside = pix[:, 0] >= 0
        flat = pix[inside, 1].to(torch.int64) * nx + pix[inside, 0].to(torch.int64)
        counts += torch.bincount(flat, minlength=nx * ny)
        n_out += int((pix[:, 0] == -1).sum())
        n_drop += int((pix[:, 0] == -2).sum())
    return counts.view(ny, nx).cpu().numpy(), n_out, n_drop


def _shot_equals_traced(ml, f, r0, r1):
    f.clear()
    f.shoot(r0, r1)
    shot = f.counts().cpu().numpy().view(np.uint32).astype(np.int64)
    st = f.stats()
    traced, n_out, n_drop = _traced_counts(ml, f, r0, r1)
    assert np.array_equal(shot, traced), int(np.abs(shot - traced).sum())
    assert (st["rays_in"], st["rays_out"], st["rays_dropped"]) == (int(traced.sum()), n_out, n_drop)
    return st


@pytest.mark.parametrize("l2_sub", [(20, 20), (60, 20)])
def test_shot_map_is_the_histogram_of_traced_pixels(ml, l2_sub):
    """The shooting kernel's counts equal, pixel for pixel, the histogram of
    the pixels the tracing kernel gives each ray one by one.  The tracer's
    per-ray pixels are the ones the edge criterion above checks against the
    oracle, so this carries that criterion over to every ray the shooting
    kernel deposits (its two-lane Horner chains, raw-bit pixel comparisons
    and run lengths included)."""
    w = _mixed_case()
    f = _field(ml, w, precision=ml.PREC_MIXED, l2_sub=l2_sub)
    n = f.n_rays
    st = _shot_equals_traced(ml, f, 0, n)
    assert st["rays_in"] > 0.05 * n and st["near_pairs"] > 0
    # ragged ranges: a partial first and last row, and a range inside one row
    nx3 = f.info["n_rays_x"]
    _shot_equals_traced(ml, f, 5 * nx3 + 17, 70 * nx3 + 3)
    _shot_equals_traced(ml, f, 40 * nx3 + 100, 40 * nx3 + 900)
    f.close()


@pytest.mark.parametrize("case", ["paper", "table1"])
def test_shot_stripe_is_the_histogram_of_traced_pixels(ml, case):
    """The same on 41 lattice rows of the paper-scale field (1e11-ray
    lattice, autotuned grid, as the benchmark runs it) and 64 rows of the
    Table-1 fold field (2.3 near lenses per ray: long near lists and close
    passes), both from a ragged start."""
    if case == "paper":
        w, rows = inputs.paper_map(0), 40
    else:
        w, rows = inputs.fold_field(0, n_rays=2e10, map_px=(1024, 5120)), 64
    f = _field(ml, w, precision=ml.PREC_MIXED, tune=True)
    nx3, ny3 = f.info["n_rays_x"], f.info["n_rays_y"]
    r0 = (ny3 // 2) * nx3 + 777
    r1 = r0 + rows * nx3 + 12345
    st = _shot_equals_traced(ml, f, r0, r1)
    assert st["rays_in"] > 0.5 * (r1 - r0) and st["near_pairs"] > 0
    f.close()


@pytest.mark.parametrize("case", ["mixed", "paper", "table1"])
def test_certified_walk_equals_per_ray_walk(ml, case):
    """The certified walk (rays between two evaluated rays counted without
    being evaluated when a bound proves they share the pixel) gives the same
    count map, bit for bit, and the same in/out/dropped totals as the walk
    that evaluates every ray, on the same grid; on the paper-scale lattice it
    evaluates fewer than half of the rays."""
    if case == "mixed":
        w, kw = _mixed_case(), dict(l2_sub=(40, 20))
    elif case == "paper":
        w, kw = inputs.paper_map(0), dict(tune=True)
    else:
        w, kw = inputs.fold_field(0, n_rays=2e10, map_px=(1024, 5120)), dict(tune=True)
    fc = _field(ml, w, precision=ml.PREC_MIXED, walk=ml.WALK_CERTIFIED, **kw)
    info = fc.info
    grid = dict(l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]),
                l2_sub=(info["l2_sub_x"], info["l2_sub_y"]))
    fp = _field(ml, w, precision=ml.PREC_MIXED, walk=ml.WALK_PER_RAY, **grid)
    for k in ("n1x", "n1y", "n2x", "n2y", "taylor_p"):
        assert fp.info[k] == info[k], k
    n = fc.n_rays
    nx3 = info["n_rays_x"]
    ranges = [(0, n)] if case == "mixed" else [
        ((info["n_rays_y"] // 2) * nx3 + 777, (info["n_rays_y"] // 2 + 64) * nx3 + 12345),
        (n // 7, n // 7 + 3 * nx3 + 5)]
    for r0, r1 in ranges:
        fc.clear()
        fp.clear()
        fc.shoot(r0, r1)
        fp.shoot(r0, r1)
        a = fc.counts().cpu().numpy()
        b = fp.counts().cpu().numpy()
        assert np.array_equal(a, b), int(np.abs(a.astype(np.int64) - b.astype(np.int64)).sum())
        sa, sb = fc.stats(), fp.stats()
        for k in ("rays_in", "rays_out", "rays_dropped", "near_pairs"):
            assert sa[k] == sb[k], k
        assert sb["rays_evaluated"] == r1 - r0
        assert 0 < sa["rays_evaluated"] <= r1 - r0
        if case == "paper":
            # two thirds of its rays lie in columns without near lenses
            assert sa["rays_evaluated"] < 0.5 * (r1 - r0), sa["rays_evaluated"] / (r1 - r0)
            assert sa["spans"] > 0
    fc.close()
    fp.close()


def test_mixed_map_matches_oracle_and_split_invariance(ml):
    w = _mixed_case(6)
    f = _field(ml, w, precision=ml.PREC_MIXED)
    g = _geometry(w, f)
    n = g.n_rays
    f.shoot()
    full = f.counts().cpu().numpy().astype(np.int64)
    st = f.stats()
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == n
    assert st["rays_in"] == int(full.sum())
    ref, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m)
    l1 = np.abs(full - ref.astype(np.int64)).sum() / ref.sum()
    assert l1 <= MAP_L1, l1
    # accumulation over ragged, out-of-order sub-ranges is bit-identical
    f.clear()
    cuts = [0, 7, n // 3 + 11, n // 2 - 5, n - 1, n]
    for a, b in reversed(list(zip(cuts[:-1], cuts[1:]))):
        f.shoot(a, b)
    f.shoot(17, 17)                      # empty range: no-op
    again = f.counts().cpu().numpy().astype(np.int64)
    assert np.array_equal(full, again)
    f.close()


def test_mixed_light_curves_and_mu(ml):
    w = _mixed_case(7)
    f = _field(ml, w, precision=ml.PREC_MIXED)
    g = _geometry(w, f)
    f.shoot()
    counts = f.counts().cpu().numpy().astype(np.float64)
    mu64 = f.mu("f64").cpu().numpy()
    assert np.allclose(mu64, oracle.magnification(g, counts), rtol=1e-15, atol=0)
    mu32 = f.mu("f32").cpu().numpy()
    assert np.allclose(mu32, mu64, rtol=2e-7, atol=0)
    tr = inputs.tracks(6, g.mnx, g.mny, 4 * 0.5 + 1, seed=3)
    lc = f.light_curves(tr, 257, 0.5).cpu().numpy()
    ref = oracle.light_curves(oracle.magnification(g, counts), tr, 257, 0.5)
    assert np.allclose(lc, ref, rtol=2e-6, atol=1e-6 * np.abs(ref).max())
    # host-output path of the same calls
    host = np.zeros((len(tr), 257), np.float32)
    import paper_2308_14278_gb300 as mlmod
    mlmod.ml_light_curves(f.h, tr, 257, 0.5, host)
    assert np.array_equal(host, lc)
    # the map into host memory: page-locked (written by the kernel over the
    # host link) and pageable (through a device buffer), both bit-equal to the
    # device map; a host buffer of the wrong type or size is refused
    import torch
    for want, dt, dev in ((mlmod.MAP_MU_F32, np.float32, mu32), (mlmod.MAP_MU_F64, np.float64, mu64),
                          (mlmod.MAP_COUNTS_U32, np.uint32, counts.astype(np.uint32))):
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.uint32: torch.int32}[dt]
        pinned = torch.zeros((g.mny, g.mnx), dtype=tdt).pin_memory().numpy().view(dt)
        pageable = np.zeros((g.mny, g.mnx), dt)
        for out in (pinned, pageable):
            mlmod.ml_magnification_map(f.h, want, out)
            assert np.array_equal(out, dev)
    with pytest.raises(ValueError):
        mlmod.ml_magnification_map(f.h, mlmod.MAP_MU_F64, np.zeros((g.mny, g.mnx), np.float32))
    with pytest.raises(ValueError):
        mlmod.ml_magnification_map(f.h, mlmod.MAP_MU_F32, np.zeros((g.mny, g.mnx - 1), np.float32))
    f.close()


def test_mixed_dropped_and_abort(ml):
    w = _mixed_case(8)
    f = _field(ml, w, precision=ml.PREC_MIXED)
    f.abort(True)
    f.shoot()
    import paper_2308_14278_gb300 as mlmod
    st, status = mlmod.ml_field_stats(f.h, check=False)
    assert status == 4 and st["flags"] & 2            # ML_ERR_ABORTED
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] < f.n_rays
    f.abort(False)
    f.clear()
    f.shoot()
    st = f.stats()
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == f.n_rays
    f.close()


def test_paper_scale_sampled_parity(ml):
    """13,000 lognormal lenses, 1e11-ray lattice, 8192^2 map: sampled rays
    against the FP64 direct sum, and a 1e6-ray stripe map against the
    oracle's map of the same stripe."""
    w = inputs.paper_map(0)
    f = _field(ml, w, precision=ml.PREC_MIXED)
    g = _geometry(w, f)
    _check_geometry(f, g)
    assert f.info["far_bound"] <= 1e-7
    rng = np.random.default_rng(11)
    idx = np.unique(rng.integers(0, g.n_rays, 20000))
    beta, pix = f.trace(idx)
    beta = beta.cpu().numpy()
    ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    rel = np.hypot(*(beta - ref).T) / np.maximum(_alpha_ref(g, idx, ref), ALPHA_FLOOR)
    assert np.max(rel) <= REL_DEFLECTION, np.max(rel)
    # a stripe in the middle of the lattice, ragged at both ends
    r0 = (g.n3y // 2) * g.n3x + 1234567
    r1 = r0 + 1_000_003
    f.shoot(r0, r1)
    got = f.counts().cpu().numpy().astype(np.int64)
    ref_map, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r1)
    l1 = np.abs(got - ref_map.astype(np.int64)).sum() / max(1, ref_map.sum())
    assert l1 <= MAP_L1, l1
    st = f.stats()
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == r1 - r0
    f.close()


def test_wrapped_count_is_reported(ml):
    """Counts are added without reading them back; a wrapped uint32 pixel
    must still be reported by ml_field_stats (map sum against in-map rays)."""
    import torch
    w = _mixed_case()
    f = _field(ml, w, precision=ml.PREC_MIXED)
    f.shoot()
    counts = f.counts()
    assert f.stats()["rays_in"] == int(counts.to(torch.int64).sum())
    # preset the busiest pixel just below 2^32 and shoot the same rays again
    flat = counts.view(-1)
    k = int(torch.argmax(flat))
    assert int(flat[k]) > 0
    preset = torch.zeros_like(counts)
    preset.view(-1)[k] = -1                   # 0xFFFFFFFF as uint32
    ml.ml_field_set_counts(f.h, preset)
    f.shoot()
    d, st = ml.ml_field_stats(f.h, None, check=False)
    assert st == 5 and d["flags"] & 1          # ML_ERR_OVERFLOW
    # without the preset the same run is clean
    f.clear()
    f.shoot()
    assert f.stats()["rays_in"] == int(f.counts().to(torch.int64).sum())
    f.close()


def test_production_map_1e13_rays(ml):
    """The full production configuration: 13,000 lognormal lenses, 1e13 rays,
    a 16384^2 map and the autotuned grid.  Sampled rays and a 1e6-ray stripe
    against the FP64 oracle; then every ray of the lattice is shot and
    accounted for (in + out + dropped = 1e13; the map's 64-bit sum equals
    the in-map count, checked by ml_field_stats); and 10 light curves of 4096
    samples (Gaussian source, sigma 0.5 px) against the oracle's from the same
    map."""
    w = inputs.paper_map(0, n_rays=1e13, map_px=16384)
    f = _field(ml, w, precision=ml.PREC_MIXED, tune=True)
    info = f.info
    g = oracle.geometry_of(w, p=info["taylor_p"], l2_sub=info["l2_sub_x"], l2_sub_y=info["l2_sub_y"],
                           l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))
    _check_geometry(f, g)
    assert info["far_bound"] <= 1e-7
    assert abs(g.n_rays - 1e13) <= 1e-5 * 1e13
    idx = np.unique(np.random.default_rng(13).integers(0, g.n_rays, 20000))
    beta, _ = f.trace(idx)
    ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    rel = np.hypot(*(beta.cpu().numpy() - ref).T) / np.maximum(_alpha_ref(g, idx, ref), ALPHA_FLOOR)
    assert np.max(rel) <= REL_DEFLECTION, np.max(rel)
    r0 = (g.n3y // 2) * g.n3x + 4321
    r1 = r0 + 1_000_000
    f.shoot(r0, r1)
    got = f.counts().cpu().numpy().astype(np.int64)
    ref_map, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r1)
    l1 = np.abs(got - ref_map.astype(np.int64)).sum() / max(1, ref_map.sum())
    assert l1 <= MAP_L1, l1
    del got, ref_map
    f.clear()
    f.shoot()
    st = f.stats()
    assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == g.n_rays
    tracks = inputs.tracks(10, g.mnx, g.mny, 4 * 0.5 + 1, seed=21)
    lc = f.light_curves(tracks, 4096, 0.5).cpu().numpy()
    counts = f.counts().cpu().numpy().view(np.uint32)
    assert int(counts.sum(dtype=np.uint64)) == st["rays_in"]
    f.close()
    ref_lc = oracle.light_curves_sampled(oracle.magnification(g, counts), tracks, 4096, 0.5)
    assert np.allclose(lc, ref_lc, rtol=2e-6, atol=1e-6 * np.abs(ref_lc).max())
