"""The fold macro model near the critical curve (Eq. 5 as printed in Eq. 6)
on the GPU against the FP64 oracle: geometry, FP64 direct counts, the mixed
path's deflections and map."""
import math

import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs

pytestmark = pytest.mark.gpu

FOLD = ("fold", 0.83, 0.01, -0.0094)  # kappa_0 of Table 1, d scaled up so that the image plane is small


def _fold_case(seed=3, ks=0.1, box=(0.5, -2.0, 6.5, 2.0), n=(64, 48), n_av=120.0, sheet="disc"):
    w_half = 10 * math.sqrt(ks)
    rect = oracle.fold_ray_box(*FOLD[1:], (box[0] - w_half, box[1] - w_half, box[2] + w_half, box[3] + w_half))
    area = (rect[2] - rect[0]) * (rect[3] - rect[1])
    nl = int(round(area * ks / math.pi))
    u = inputs.uniform01(seed, 41, nl)
    v = inputs.uniform01(seed, 42, nl)
    lf = inputs.LensField(rect[0] + (rect[2] - rect[0]) * u, rect[1] + (rect[3] - rect[1]) * v,
                          np.ones(nl))
    cx, cy = 0.5 * (rect[0] + rect[2]), 0.5 * (rect[1] + rect[3])
    sh = (cx, cy, 1e4) if sheet == "disc" else (cx, cy, 0.5 * (rect[3] - rect[1]) + 1e-9, "strip")
    return inputs.Workload("fold", lf, 0.0, 0.0, ks, sh, box, n, n_av=n_av, macro=FOLD)


def _geom(w, f):
    info = f.info
    return oracle.geometry_of(w, p=max(1, info["taylor_p"]), l2_sub=info["l2_sub_x"],
                              l2_sub_y=info["l2_sub_y"],
                              l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))


def test_fold_geometry_matches_oracle(ml):
    w = _fold_case()
    f = ml.Field(w, precision=ml.PREC_MIXED)
    g = _geom(w, f)
    info = f.info
    assert (info["n_rays_x"], info["n_rays_y"]) == (g.n3x, g.n3y)
    for k in ("n1x", "n1y", "n2x", "n2y", "N1x", "N1y"):
        assert info[k] == getattr(g, k), k
    for k, v in (("ray_x0", g.rx0), ("ray_y0", g.ry0), ("ray_x1", g.rx1), ("ray_y1", g.ry1)):
        assert info[k] == pytest.approx(v, rel=1e-14, abs=1e-12), k
    assert info["taylor_p"] >= 2 and info["far_bound"] <= 1e-7
    f.close()


@pytest.mark.parametrize("sheet", ["disc", "strip"])
def test_fold_direct64_counts_match_oracle(ml, sheet):
    w = _fold_case(sheet=sheet)
    f = ml.Field(w, precision=ml.PREC_DIRECT64)
    g = _geom(w, f)
    f.shoot()
    got = f.counts().cpu().numpy().astype(np.int64)
    ref, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m)
    beta, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, np.arange(g.n_rays))
    fx = (beta[:, 0] - g.mx0) / g.dpx
    fy = (beta[:, 1] - g.my0) / g.dpy
    n_edge = int(np.sum(np.minimum(np.abs(fx - np.round(fx)), np.abs(fy - np.round(fy))) < 1e-5))
    assert int(np.abs(got - ref.astype(np.int64)).sum()) <= 2 * n_edge
    assert int(ref.sum()) > 0.1 * g.n_rays           # 16 % of this rectangle maps into the map
    f.close()


@pytest.mark.parametrize("sheet", ["disc", "strip"])
def test_fold_mixed_deflection_and_map(ml, sheet):
    w = _fold_case(sheet=sheet)
    f = ml.Field(w, precision=ml.PREC_MIXED)
    g = _geom(w, f)
    idx = np.unique(np.random.default_rng(2).integers(0, g.n_rays, 30000))
    beta, _ = f.trace(idx)
    beta = beta.cpu().numpy()
    ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    tx, ty = oracle.ray_position(g, idx)
    # deflection = macro + sheet - beta; the macro is the fold term
    mx = 0.5 * g.d_x * tx * tx + g.d_y * tx * ty
    my = 2 * (1 - g.kappa0) * ty
    kx, ky = (0.0, 2 * g.kappa_star) if g.sheet_shape == 1 else (g.kappa_star, g.kappa_star)
    ax = mx + kx * (tx - g.sheet_cx) - ref[:, 0]
    ay = my + ky * (ty - g.sheet_cy) - ref[:, 1]
    rel = np.hypot(*(beta - ref).T) / np.maximum(np.hypot(ax, ay), 1e-2)
    assert rel.max() <= 1e-5, rel.max()
    f.shoot()
    got = f.counts().cpu().numpy().astype(np.int64)
    ref_map, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m)
    l1 = np.abs(got - ref_map.astype(np.int64)).sum() / ref_map.sum()
    assert l1 <= 1e-3, l1
    f.close()


def test_fold_nearfar64_trace_matches_oracle_interp(ml):
    w = _fold_case()
    f = ml.Field(w, precision=ml.PREC_NEARFAR64, taylor_p=6, build=ml.BUILD_DIRECT)
    g = _geom(w, f)
    idx = np.unique(np.linspace(0, g.n_rays - 1, 4000).astype(np.int64))
    beta, _ = f.trace(idx)
    ref, _ = oracle.beta_interp(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    assert np.max(np.abs(beta.cpu().numpy() - ref)) < 1e-10
    f.close()


def test_table1_field_sampled_parity(ml):
    """The Table-1 fold field (13,745 lenses, kappa_* = 0.001) on a reduced
    lattice: sampled rays against the FP64 direct sum."""
    w = inputs.fold_field(0, n_rays=2e9, map_px=(512, 2560))
    f = ml.Field(w, precision=ml.PREC_MIXED, tune=True)
    info = f.info
    assert info["far_bound"] <= 1e-7
    g = _geom(w, f)
    assert (info["n_rays_x"], info["n_rays_y"]) == (g.n3x, g.n3y)
    idx = np.unique(np.random.default_rng(7).integers(0, g.n_rays, 3000))
    beta, _ = f.trace(idx)
    ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    tx, ty = oracle.ray_position(g, idx)
    assert g.sheet_shape == 1
    ax = 0.5 * g.d_x * tx * tx + g.d_y * tx * ty - ref[:, 0]
    ay = 2 * (1 - g.kappa0) * ty + 2 * g.kappa_star * (ty - g.sheet_cy) - ref[:, 1]
    rel = np.hypot(*(beta.cpu().numpy() - ref).T) / np.maximum(np.hypot(ax, ay), 1e-2)
    assert rel.max() <= 1e-5, rel.max()
    f.close()


def test_fold_field_rejects_the_adjoint(ml):
    import torch
    w = _fold_case()
    f = ml.Field(w, precision=ml.PREC_MIXED, deposit=ml.DEPOSIT_CIC)
    G = torch.zeros(w.map_n[::-1], dtype=torch.float32, device="cuda")
    gl = torch.zeros((w.lenses.n, 3), dtype=torch.float64, device="cuda")
    gp = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ml.MLError):
        ml.ml_cic_backward(f.h, G, gl, gp)
    f.close()
