"""Batched maps (one persistent launch over many maps, CUDA graph replay)
and the level-2 grid autotuner.

Integer counts make the batch checkable exactly: every map of a batch must
equal, bit for bit, the same map shot alone with the same Taylor order and
level-2 grid; the single-map path is itself checked against the FP64 oracle
in test_gpu_parity.py, and a tuned field is checked against it here.
"""
import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs

pytestmark = pytest.mark.gpu


def _small_batch(ml, n_maps=5, tune=False):
    ws = inputs.batched_maps(n_maps=n_maps, seed=3, map_px=256, ray_range=(2e6, 2e7),
                             tracks_per_map=4)
    descs = [ml.make_desc(w, precision=ml.PREC_MIXED, tune=tune) for w in ws]
    tracks = np.stack([inputs.tracks(4, 256, 256, 3.0, seed=50 + i) for i in range(n_maps)])
    return ws, descs, tracks


def test_batch_matches_single_maps_bitwise(ml):
    ws, descs, tracks = _small_batch(ml)
    b = ml.Batch(descs, tracks=tracks, n_samples=200, sigma_px=0.5)
    b.run(use_graph=True)
    curves = b.curves().cpu().numpy()
    for i, w in enumerate(ws):
        info = b.info(i)
        P = info["taylor_p"]                              # each map keeps its own order
        st = b.stats(i)
        n = info["n_rays_x"] * info["n_rays_y"]
        assert st["rays_in"] + st["rays_out"] + st["rays_dropped"] == n
        counts = b.counts(i).cpu().numpy()
        assert st["rays_in"] == int(counts.astype(np.int64).sum())
        f = ml.Field(w, precision=ml.PREC_MIXED, taylor_p=P,
                     l2_sub=(info["l2_sub_x"], info["l2_sub_y"]))
        f.shoot()
        alone = f.counts().cpu().numpy()
        assert np.array_equal(counts, alone), i
        mu = b.mu(i).cpu().numpy()
        assert np.array_equal(mu, f.mu("f32").cpu().numpy())
        lc = f.light_curves(tracks[i], 200, 0.5).cpu().numpy()
        assert np.allclose(curves[i], lc, rtol=2e-6, atol=1e-6 * np.abs(lc).max())
        f.close()
    b.close()


def test_tuned_batch_groups_orders_and_matches_single_maps(ml):
    """Tuned maps may need different Taylor orders: each runs with its own in
    the launch of its order, bit for bit as the same map shot alone."""
    ws, descs, tracks = _small_batch(ml, n_maps=6, tune=True)
    b = ml.Batch(descs)
    b.run(use_graph=True)
    for i, w in enumerate(ws):
        info = b.info(i)
        assert info["tuned"] == 1 and info["far_bound"] <= 1e-7
        f = ml.Field(w, precision=ml.PREC_MIXED, taylor_p=info["taylor_p"],
                     l2_sub=(info["l2_sub_x"], info["l2_sub_y"]),
                     l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))
        f.shoot()
        assert np.array_equal(b.counts(i).cpu().numpy(), f.counts().cpu().numpy()), i
        f.close()
    b.close()


def test_batch_graph_replay_and_direct_launch_agree(ml):
    ws, descs, tracks = _small_batch(ml, n_maps=4)
    b = ml.Batch(descs, tracks=tracks, n_samples=64, sigma_px=0.5)
    b.run(use_graph=False)
    first = [b.counts(i).cpu().numpy() for i in range(b.n)]
    for _ in range(2):                    # replays clear and reshoot every map
        b.run(use_graph=True)
        again = [b.counts(i).cpu().numpy() for i in range(b.n)]
        assert all(np.array_equal(x, y) for x, y in zip(first, again))
    b.close()


def test_batch_maps_match_oracle_on_sampled_rays(ml):
    ws, descs, tracks = _small_batch(ml, n_maps=3)
    b = ml.Batch(descs)
    b.run()
    for i, w in enumerate(ws):
        info = b.info(i)
        g = oracle.geometry_of(w, p=info["taylor_p"], l2_sub=info["l2_sub_x"],
                               l2_sub_y=info["l2_sub_y"])
        assert (info["n_rays_x"], info["n_rays_y"]) == (g.n3x, g.n3y)
        idx = np.unique(np.random.default_rng(i).integers(0, g.n_rays, 3000))
        import torch
        tidx = torch.as_tensor(idx).cuda()
        beta = torch.empty((len(idx), 2), dtype=torch.float64, device="cuda")
        pix = torch.empty((len(idx), 2), dtype=torch.int32, device="cuda")
        ml.ml_trace_rays(b.fields[i], tidx, beta, pix)
        ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
        tx, ty = oracle.ray_position(g, idx)
        ax = (1 - g.kappa - g.gamma) * tx + g.kappa_star * (tx - g.sheet_cx) - ref[:, 0]
        ay = (1 - g.kappa + g.gamma) * ty + g.kappa_star * (ty - g.sheet_cy) - ref[:, 1]
        rel = np.hypot(*(beta.cpu().numpy() - ref).T) / np.maximum(np.hypot(ax, ay), 1e-2)
        assert rel.max() <= 1e-5, (i, rel.max())
    b.close()


def test_tuned_field_meets_bound_and_matches_oracle(ml):
    w = inputs.paper_map(0, n_rays=4e9, map_px=2048)
    f = ml.Field(w, precision=ml.PREC_MIXED, tune=True)
    info = f.info
    assert info["tuned"] == 1
    assert info["far_bound"] <= 1e-7
    g = oracle.geometry_of(w, p=info["taylor_p"], l2_sub=info["l2_sub_x"],
                           l2_sub_y=info["l2_sub_y"],
                           l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))
    assert (info["n1x"], info["n2x"], info["n1y"], info["n2y"]) == (g.n1x, g.n2x, g.n1y, g.n2y)
    idx = np.unique(np.random.default_rng(5).integers(0, g.n_rays, 10000))
    beta, _ = f.trace(idx)
    ref, _ = oracle.beta_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, idx)
    tx, ty = oracle.ray_position(g, idx)
    ax = (1 - g.kappa - g.gamma) * tx + g.kappa_star * (tx - g.sheet_cx) - ref[:, 0]
    ay = (1 - g.kappa + g.gamma) * ty + g.kappa_star * (ty - g.sheet_cy) - ref[:, 1]
    rel = np.hypot(*(beta.cpu().numpy() - ref).T) / np.maximum(np.hypot(ax, ay), 1e-2)
    assert rel.max() <= 1e-5
    # a second identical field reuses the tuner's decision
    f2 = ml.Field(w, precision=ml.PREC_MIXED, tune=True)
    assert (f2.info["l2_sub_x"], f2.info["l2_sub_y"], f2.info["n1x"], f2.info["n1y"]) == \
        (info["l2_sub_x"], info["l2_sub_y"], info["n1x"], info["n1y"])
    f.close()
    f2.close()
