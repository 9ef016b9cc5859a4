"""The allocation-free light-curve entry point against the allocating one.

ml_light_curves_noalloc serves callers that must not allocate device memory
once running (a fixed memory budget reserved at start-up, or a loop where an
allocation's implicit synchronisation or out-of-memory risk is unacceptable).
Its scratch is a fixed array inside the library shared by all calls, so the
test makes two calls in a row with different tracks and compares each with
ml_light_curves on the same inputs.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2308_14278_gb300 import inputs

pytestmark = pytest.mark.gpu


def _workload():
    """Lognormal lenses in a disc 1.5 times the ray rectangle's half-diagonal
    (kappa = 0.40, gamma = 0.45, kappa_* = 0.05 = N <m> / R^2)."""
    kappa, gamma, ks = 0.40, 0.45, 0.05
    box = (-1.0, -0.75, 1.0, 0.75)
    w = 10.0 * np.sqrt(ks)
    hx = (box[2] + w) / (1.0 - kappa - gamma)
    hy = (box[3] + w) / (1.0 - kappa + gamma)
    r = 1.5 * np.hypot(hx, hy)
    n = int(round(ks * r * r / inputs.lognormal_mean(0.3, 0.5)))
    lf = inputs.lens_disc(n, r, 4, "lognormal")
    ks = n * inputs.lognormal_mean(0.3, 0.5) / r ** 2
    return inputs.Workload("no-alloc check", lf, kappa, gamma, ks, (0.0, 0.0, r), box,
                           (160, 120), n_av=40)


def _field(ml):
    f = ml.Field(_workload(), precision=ml.PREC_MIXED)
    f.shoot()
    return f


def test_light_curves_noalloc_matches_allocating_entry_point(ml):
    import torch
    f = _field(ml)
    nx, ny = f.info["map_nx"], f.info["map_ny"]
    # the last call fills the whole scratch: the widest source (sigma = 16 px,
    # 129 taps) and ML_NOALLOC_MAX_TRACKS tracks
    calls = ((5, 257, 0.5, 1), (9, 130, 1.5, 2), (ml.NOALLOC_MAX_TRACKS, 4, 16.0, 3))
    for call, (n_tracks, n_samples, sigma, seed) in enumerate(calls):
        tr = inputs.tracks(n_tracks, nx, ny, 4 * sigma + 1 if sigma < 4 else 2.0, seed=seed)
        ref = f.light_curves(tr, n_samples, sigma)          # allocating entry point
        out = torch.full((n_tracks, n_samples), float("nan"), dtype=torch.float32, device="cuda")
        ml.ml_light_curves_noalloc(f.h, tr, n_samples, sigma, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        # both entry points run the same kernel on the same taps and tracks
        assert np.array_equal(o, r), call
    f.close()


def test_light_curves_noalloc_rejects_too_many_tracks(ml):
    import torch
    f = _field(ml)
    n = ml.NOALLOC_MAX_TRACKS + 1
    tr = np.tile(np.array([[10.0, 10.0, 20.0, 20.0]]), (n, 1))
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ml.MLError) as err:
        ml.ml_light_curves_noalloc(f.h, tr, 4, 0.5, out)
    assert err.value.status == 1 and "ML_NOALLOC_MAX_TRACKS" in str(err.value)
    f.close()
