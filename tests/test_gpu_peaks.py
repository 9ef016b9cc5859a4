"""Peak identification (§4.2) on the GPU against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2308_14278_gb300 import inputs

pytestmark = pytest.mark.gpu


def _blank_field(ml, nx, ny):
    w = inputs.Workload("blank", inputs.LensField(np.zeros(0), np.zeros(0), np.zeros(0)), 0.25, 0.25,
                        0.0, (0.0, 0.0, 100.0), (-1.0, -1.0, 1.0, 1.0), (nx, ny),
                        ray_box=(-2.0, -1.5, 2.0, 1.5), ray_n=(64, 48))
    return ml.Field(w, precision=ml.PREC_DIRECT64)


def _gpu_peaks(ml, f, along, nsigma=5.0, capacity=4096):
    import torch
    info = f.info
    mask = torch.zeros(info["map_ny"] * info["map_nx"] + 4, dtype=torch.uint8, device="cuda")
    n, peaks = ml.ml_find_peaks(f.h, along, nsigma, mask, capacity)
    m = mask[:-4].view(info["map_ny"], info["map_nx"]).cpu().numpy()
    return n, peaks.cpu().numpy(), m


@pytest.mark.parametrize("along", ["x", "y"])
def test_synthetic_ridges_match_oracle(ml, along):
    import torch
    rng = np.random.default_rng(5)
    N = rng.poisson(1000.0, (60, 80)).astype(np.int64)
    N[10:15, 20] += 400                        # ridge across five rows (curves along x)
    N[30, 40:46] += 400                        # ridge across six columns (curves along y)
    N[50, 60] += 500                           # isolated spike
    f = _blank_field(ml, 80, 60)
    ml.ml_field_set_counts(f.h, torch.as_tensor(N.astype(np.int32)).cuda())
    a = ml.ALONG_X if along == "x" else ml.ALONG_Y
    n, peaks, m = _gpu_peaks(ml, f, a)
    ref = oracle.peaks(N, along)
    assert np.array_equal(m, ref)
    assert n == int((ref & 2).astype(bool).sum()) and n > 0
    assert {tuple(p) for p in peaks} == {(x, y) for y, x in zip(*np.nonzero(ref & 2))}
    f.close()


def test_peaks_of_a_shot_map_match_oracle(ml):
    """A fold-model map shot on the GPU: its own count map through both
    implementations (the oracle reads the GPU's counts: the check is of the
    peak step alone)."""
    from test_gpu_fold import _fold_case
    w = _fold_case(n_av=400.0, n=(128, 96))
    f = ml.Field(w, precision=ml.PREC_MIXED)
    f.shoot()
    counts = f.counts().cpu().numpy().astype(np.int64)
    for along in ("x", "y"):
        n, _, m = _gpu_peaks(ml, f, ml.ALONG_X if along == "x" else ml.ALONG_Y, nsigma=3.0)
        ref = oracle.peaks(counts, along, nsigma=3.0)
        assert np.array_equal(m, ref)
        assert n == int((ref & 2).astype(bool).sum())
    f.close()


def test_peak_list_capacity(ml):
    import torch
    N = np.full((20, 30), 1000, np.int64)
    for c in range(3, 27, 3):
        N[4:9, c] = 1400
    f = _blank_field(ml, 30, 20)
    ml.ml_field_set_counts(f.h, torch.as_tensor(N.astype(np.int32)).cuda())
    n_all, peaks, _ = _gpu_peaks(ml, f, ml.ALONG_X, capacity=1000)
    n_few, few, _ = _gpu_peaks(ml, f, ml.ALONG_X, capacity=5)
    assert n_all == n_few == 8 * 3 and len(peaks) == 24 and len(few) == 5
    assert {tuple(p) for p in few} <= {tuple(p) for p in peaks}
    f.close()


def _device_mask(ml, f, along, nsigma):
    import torch
    info = f.info
    mask = torch.zeros(info["map_ny"] * info["map_nx"] + 4, dtype=torch.uint8, device="cuda")
    ml.ml_find_peaks(f.h, along, nsigma, mask, 0)
    return mask


def _axis(g, along):
    return (g.mx0, g.dpx) if along == "x" else (g.my0, g.dpy)


@pytest.mark.parametrize("along", ["x", "y"])
def test_peak_statistics_of_synthetic_ridges_match_oracle(ml, along):
    """Per-bin true peaks, their count sums and the scanned positions, bit for
    bit against the oracle: with the caller's mask, and with the peaks found
    inside the call.  The caustic lies inside the map (distances fold), and
    one edge is exactly the distance of a pixel centre (the tie goes up)."""
    import torch
    rng = np.random.default_rng(8)
    N = rng.poisson(1000.0, (60, 80)).astype(np.int64)
    for c in range(4, 76, 7):
        N[3:57, c] += 400                      # ridges across the rows (curves along x)
    for r in range(5, 55, 6):
        N[r, 2:78] += 400                      # ridges across the columns (curves along y)
    f = _blank_field(ml, 80, 60)
    ml.ml_field_set_counts(f.h, torch.as_tensor(N.astype(np.int32)).cuda())
    w = inputs.Workload("blank", inputs.LensField(np.zeros(0), np.zeros(0), np.zeros(0)), 0.25, 0.25,
                        0.0, (0.0, 0.0, 100.0), (-1.0, -1.0, 1.0, 1.0), (80, 60),
                        ray_box=(-2.0, -1.5, 2.0, 1.5), ray_n=(64, 48))
    g = oracle.geometry_of(w)
    origin, step = _axis(g, along)
    caustic = 0.1
    tie = abs(origin + (37 + 0.5) * step - caustic)
    edges = sorted(set([0.0, 0.05, 0.2, tie, 0.5, 0.75, 0.9, 1.2]))
    a = ml.ALONG_X if along == "x" else ml.ALONG_Y
    ref = oracle.peak_statistics(N, oracle.peaks(N, along), along, origin, step, caustic, edges)
    assert int(ref[0].sum()) > 100
    got = ml.ml_peak_statistics(f.h, edges, a, caustic, mask=_device_mask(ml, f, a, 5.0))
    got_inline = ml.ml_peak_statistics(f.h, edges, a, caustic, nsigma=5.0)
    for r, x, y in zip(ref, got, got_inline):
        assert np.array_equal(r, x) and np.array_equal(r, y)
    f.close()


def test_peak_statistics_of_a_shot_fold_map_match_oracle(ml):
    """A fold-model map shot on the GPU, binned by the distance beta_x from the
    caustic (beta_x = 0) on a log grid as in Figs. 4-5: the oracle reads the
    GPU's counts, so the check is of the peak and statistics steps alone."""
    from test_gpu_fold import _fold_case
    w = _fold_case(n_av=400.0, n=(128, 96))
    f = ml.Field(w, precision=ml.PREC_MIXED)
    f.shoot()
    counts = f.counts().cpu().numpy().astype(np.int64)
    g = oracle.geometry_of(w)
    edges = list(np.geomspace(0.4, 8.0, 9))
    ref = oracle.peak_statistics(counts, oracle.peaks(counts, "x", nsigma=3.0), "x", g.mx0, g.dpx, 0.0, edges)
    assert int(ref[0].sum()) > 0
    got = ml.ml_peak_statistics(f.h, edges, ml.ALONG_X, 0.0, nsigma=3.0)
    for r, x in zip(ref, got):
        assert np.array_equal(r, x)
    f.close()


def test_peak_statistics_rejects_bad_arguments(ml):
    f = _blank_field(ml, 30, 20)
    for edges in ([0.0], [0.0, 0.0, 1.0], [1.0, 0.5], [0.0, float("nan")], [0.0, float("inf")]):
        with pytest.raises(ml.MLError):
            ml.ml_peak_statistics(f.h, edges)
    with pytest.raises(ml.MLError):
        ml.ml_peak_statistics(f.h, [0.0, 1.0], caustic=float("nan"))
    with pytest.raises(ml.MLError):
        ml.ml_peak_statistics(f.h, [0.0, 1.0], nsigma=0.0)
    with pytest.raises(ml.MLError):
        ml.ml_peak_statistics(f.h, np.arange(2050.0))
    f.close()
