"""GB300 microlensing ray-shooting library: thin Python binding.

The work happens in the CUDA library built from csrc/ (include/ml.h is its C
ABI).  This module only marshals arguments: the functions below carry the
ABI's names (ml_field_create, ml_shoot_rays, ml_magnification_map,
ml_light_curves, ...), take torch device tensors or numpy host arrays, and
pass their pointers and the current CUDA stream through ctypes.  There is no
CPU fallback: every call fails loudly if the library is missing.

Yang, Chen, Zheng & Luo, "Simulation of the microlensing effect near the
critical curve of the galaxy cluster": lens equation Eq. 6 / Eq. 9, the
parameters of §3.1, the three-level grid of §3.2, magnification Eq. 12.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic inputs, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libml.so")

ABI_VERSION = 4
PREC_DIRECT64, PREC_NEARFAR64, PREC_MIXED = 0, 1, 2
DEPOSIT_NGP, DEPOSIT_CIC = 0, 1
MACRO_LINEAR, MACRO_FOLD = 0, 1
SHEET_DISC, SHEET_STRIP = 0, 1
BUILD_AUTO, BUILD_DIRECT, BUILD_HIERARCHICAL = 0, 1, 2
MAP_COUNTS_U32, MAP_MU_F32, MAP_MU_F64 = 0, 1, 2
STAT_NAMES = ("rays_in", "rays_out", "rays_dropped", "near_pairs", "tasks", "launches",
              "flags", "rays_asked", "rays_evaluated", "spans")
WALK_CERTIFIED, WALK_PER_RAY = 0, 1
STATUS = {0: "ML_OK", 1: "ML_ERR_INVALID_ARG", 2: "ML_ERR_OOM", 3: "ML_ERR_CUDA",
          4: "ML_ERR_ABORTED", 5: "ML_ERR_OVERFLOW", 6: "ML_ERR_STATE", 7: "ML_ERR_UNSUPPORTED"}

# every symbol include/ml.h declares
EXPORTS = ("ml_abi_version", "ml_last_error", "ml_field_create", "ml_shoot_rays",
           "ml_magnification_map", "ml_light_curves", "ml_trace_rays", "ml_field_clear",
           "ml_field_stats", "ml_field_info", "ml_field_abort", "ml_field_destroy",
           "ml_light_curves_noalloc", "ml_batch_create", "ml_batch_run", "ml_batch_field",
           "ml_batch_mu", "ml_batch_curves", "ml_batch_abort", "ml_batch_destroy",
           "ml_cic_forward", "ml_cic_backward", "ml_cic_backward_ex", "ml_map_light_curves",
           "ml_map_light_curves_backward", "ml_field_set_counts", "ml_find_peaks",
           "ml_peak_statistics", "ml_fp32_fma_peak")
NOALLOC_MAX_TRACKS = 16384


class MLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class FieldDesc(C.Structure):
    """ml_field_desc of include/ml.h."""
    _fields_ = [
        ("abi_version", C.c_int32), ("precision", C.c_int32), ("deposit", C.c_int32),
        ("build", C.c_int32),
        ("kappa", C.c_double), ("gamma", C.c_double), ("kappa_star", C.c_double),
        ("lens_x", C.c_void_p), ("lens_y", C.c_void_p), ("lens_m", C.c_void_p),
        ("n_lens", C.c_int64), ("lens_mem_is_device", C.c_int32), ("taylor_p", C.c_int32),
        ("sheet_cx", C.c_double), ("sheet_cy", C.c_double), ("sheet_radius", C.c_double),
        ("ray_x0", C.c_double), ("ray_y0", C.c_double), ("ray_x1", C.c_double),
        ("ray_y1", C.c_double),
        ("n_rays_x", C.c_int64), ("n_rays_y", C.c_int64), ("n_av", C.c_double),
        ("map_x0", C.c_double), ("map_y0", C.c_double), ("map_x1", C.c_double),
        ("map_y1", C.c_double), ("map_nx", C.c_int32), ("map_ny", C.c_int32),
        ("l1_x", C.c_double), ("l1_y", C.c_double), ("l2_sub_x", C.c_int32),
        ("l2_sub_y", C.c_int32), ("far_tol", C.c_double), ("max_launch_rays", C.c_uint64),
        ("tune", C.c_int32), ("walk", C.c_int32),
        ("macro_mode", C.c_int32), ("sheet_shape", C.c_int32),
        ("kappa0", C.c_double), ("d_x", C.c_double), ("d_y", C.c_double),
        ("span_far", C.c_double),
    ]


class FieldParams(C.Structure):
    """ml_field_params of include/ml.h."""
    _fields_ = [
        ("ray_x0", C.c_double), ("ray_y0", C.c_double), ("ray_x1", C.c_double),
        ("ray_y1", C.c_double), ("l3x", C.c_double), ("l3y", C.c_double),
        ("n_rays_x", C.c_int64), ("n_rays_y", C.c_int64),
        ("map_x0", C.c_double), ("map_y0", C.c_double), ("dpx", C.c_double), ("dpy", C.c_double),
        ("map_nx", C.c_int32), ("map_ny", C.c_int32),
        ("n_star_in", C.c_int64), ("l0", C.c_double),
        ("n1x", C.c_int64), ("n1y", C.c_int64), ("n2x", C.c_int64), ("n2y", C.c_int64),
        ("N1x", C.c_int64), ("N1y", C.c_int64), ("N2x", C.c_int64), ("N2y", C.c_int64),
        ("taylor_p", C.c_int32), ("l2_sub_x", C.c_int32), ("l2_sub_y", C.c_int32),
        ("precision", C.c_int32), ("deposit", C.c_int32), ("max_near", C.c_int32),
        ("build", C.c_int32), ("tuned", C.c_int32),
        ("far_bound", C.c_double), ("mu_per_count", C.c_double), ("span_far", C.c_double),
        ("spans", C.c_int32), ("reserved", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str | None = None):
    """Load the CUDA library (built by build.build_library or __graft_entry__.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    P, V = C.POINTER, C.c_void_p
    st = C.c_int
    sig = {
        "ml_abi_version": ([], C.c_int32),
        "ml_last_error": ([], C.c_char_p),
        "ml_field_create": ([P(FieldDesc), V, P(V)], st),
        "ml_shoot_rays": ([V, C.c_uint64, C.c_uint64, V], st),
        "ml_magnification_map": ([V, C.c_int32, V, C.c_int32, V], st),
        "ml_light_curves": ([V, V, C.c_int32, C.c_int32, C.c_double, V, C.c_int32, V], st),
        "ml_trace_rays": ([V, V, C.c_int64, V, V, V], st),
        "ml_light_curves_noalloc": ([V, V, C.c_int32, C.c_int32, C.c_double, V, V], st),
        "ml_batch_create": ([P(FieldDesc), C.c_int32, C.c_int32, V, C.c_int32, C.c_double, V,
                             P(V)], st),
        "ml_batch_run": ([V, C.c_int32, V], st),
        "ml_batch_field": ([V, C.c_int32, P(V)], st),
        "ml_batch_mu": ([V, C.c_int32, V, C.c_int32, V], st),
        "ml_batch_curves": ([V, V, C.c_int32, V], st),
        "ml_batch_abort": ([V, C.c_int32], st),
        "ml_batch_destroy": ([V], st),
        "ml_cic_forward": ([V, V, V], st),
        "ml_cic_backward": ([V, V, V, V, V], st),
        "ml_cic_backward_ex": ([V, V, V, V, C.c_int32, V], st),
        "ml_field_set_counts": ([V, V, C.c_int32, V], st),
        "ml_find_peaks": ([V, C.c_int32, C.c_double, V, V, C.c_int64, P(C.c_int64), V], st),
        "ml_peak_statistics": ([V, C.c_int32, C.c_double, V, C.c_double, V, C.c_int32, V, V, V, V], st),
        "ml_map_light_curves": ([V, C.c_int32, C.c_int32, V, C.c_int32, C.c_int32, C.c_double, V, V], st),
        "ml_map_light_curves_backward": ([C.c_int32, C.c_int32, V, C.c_int32, C.c_int32, C.c_double, V, V, V], st),
        "ml_fp32_fma_peak": ([C.c_int32, C.c_int32, C.c_int64, V, P(C.c_double), V], st),
        "ml_field_clear": ([V, V], st),
        "ml_field_stats": ([V, P(C.c_uint64), V], st),
        "ml_field_info": ([V, P(FieldParams)], st),
        "ml_field_abort": ([V, C.c_int32], st),
        "ml_field_destroy": ([V], st),
    }
    for name, (argt, rest) in sig.items():
        f = getattr(lib, name)
        f.argtypes = argt
        f.restype = rest
    if lib.ml_abi_version() != ABI_VERSION:
        raise RuntimeError("libml.so ABI version mismatch")
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise MLError(status, load().ml_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    """Device pointer of a torch tensor (must be contiguous, on CUDA)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


# ---- functions with the ABI's names ------------------------------------------

def ml_field_create(desc: FieldDesc, stream=None):
    h = C.c_void_p()
    _check(load().ml_field_create(C.byref(desc), _stream(stream), C.byref(h)))
    return h


def ml_shoot_rays(field, ray_begin: int, ray_end: int, stream=None):
    _check(load().ml_shoot_rays(field, int(ray_begin), int(ray_end), _stream(stream)))


_MAP_ITEMSIZE = {MAP_COUNTS_U32: 4, MAP_MU_F32: 4, MAP_MU_F64: 8}


def ml_magnification_map(field, want: int, out, stream=None):
    """out: torch CUDA tensor (device) or numpy array (host) of the map's
    map_ny x map_nx elements of the kind's type (host arrays are checked:
    C-contiguous, its element size and at least that many elements)."""
    if isinstance(out, np.ndarray):
        info = ml_field_info(field)
        npix = info["map_nx"] * info["map_ny"]
        kind = {MAP_COUNTS_U32: "ui", MAP_MU_F32: "f", MAP_MU_F64: "f"}.get(want)
        if kind is None:
            raise ValueError(f"unknown map kind {want}")
        if (out.dtype.kind not in kind or out.dtype.itemsize != _MAP_ITEMSIZE[want]
                or not out.flags.c_contiguous or out.size < npix):
            raise ValueError(f"host map needs {npix} contiguous elements of "
                             f"{_MAP_ITEMSIZE[want]} bytes ({'integer' if kind == 'ui' else 'float'}), "
                             f"got {out.dtype} {out.shape}")
        _check(load().ml_magnification_map(field, want, out.ctypes.data, 0, _stream(stream)))
    else:
        _check(load().ml_magnification_map(field, want, _dptr(out), 1, _stream(stream)))


def _check_curves_out(out, n_tracks: int, n_samples: int):
    """The light-curve kernels write n_tracks x n_samples float32 values."""
    import torch
    if out.dtype != torch.float32:
        raise ValueError(f"light curves are float32, got {out.dtype}")
    if out.numel() < n_tracks * n_samples:
        raise ValueError(f"out holds {out.numel()} values, {n_tracks} x {n_samples} needed")


def ml_light_curves(field, tracks, n_samples: int, sigma_px: float, out, stream=None):
    tr = np.ascontiguousarray(tracks, np.float64).reshape(-1, 4)
    if isinstance(out, np.ndarray):
        if out.dtype != np.float32 or out.size < len(tr) * n_samples or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float32 array of n_tracks x n_samples")
        _check(load().ml_light_curves(field, tr.ctypes.data, len(tr), n_samples, sigma_px,
                                      out.ctypes.data, 0, _stream(stream)))
    else:
        _check_curves_out(out, len(tr), n_samples)
        _check(load().ml_light_curves(field, tr.ctypes.data, len(tr), n_samples, sigma_px,
                                      _dptr(out), 1, _stream(stream)))


def ml_light_curves_noalloc(field, tracks, n_samples: int, sigma_px: float, out, stream=None):
    """Light curves into a device tensor without any allocation in the
    library (for callers that must not allocate device memory; see ml.h)."""
    tr = np.ascontiguousarray(tracks, np.float64).reshape(-1, 4)
    _check_curves_out(out, len(tr), n_samples)
    _check(load().ml_light_curves_noalloc(field, tr.ctypes.data, len(tr), n_samples, sigma_px,
                                          _dptr(out), _stream(stream)))


def ml_cic_forward(field, mu, stream=None):
    """Differentiable CIC magnification map into a device float32 tensor (see ml.h)."""
    _check(load().ml_cic_forward(field, _dptr(mu), _stream(stream)))


ADJOINT_NEARFAR, ADJOINT_DIRECT = 0, 1


def _tracks_host(tracks):
    tr = np.ascontiguousarray(tracks, np.float64).reshape(-1, 4)
    return tr, tr.ctypes.data


ALONG_X, ALONG_Y = 0, 1


def ml_find_peaks(field, along=ALONG_X, nsigma=5.0, mask=None, capacity=0, stream=None):
    """Peak identification of §4.2 (see ml.h).  Returns (n_found, peaks) with
    peaks a device int32 tensor (min(n_found, capacity), 2) of (ix, iy)."""
    import torch
    peaks = torch.empty((max(capacity, 1), 2), dtype=torch.int32, device="cuda")
    n = C.c_int64()
    _check(load().ml_find_peaks(field, along, float(nsigma), _dptr(mask) if mask is not None else None,
                                _dptr(peaks) if capacity > 0 else None, capacity, C.byref(n),
                                _stream(stream)))
    return n.value, peaks[:min(n.value, capacity)]


def ml_peak_statistics(field, edges, along=ALONG_X, caustic=0.0, mask=None, nsigma=5.0, stream=None):
    """Peak statistics of §4.2 by distance to the caustic (see ml.h).
    Returns (n_peaks, sum_counts, n_positions), uint64 arrays of len(edges) - 1."""
    e = np.ascontiguousarray(edges, np.float64)
    nb = len(e) - 1
    out = [np.zeros(max(nb, 1), np.uint64) for _ in range(3)]
    _check(load().ml_peak_statistics(field, along, float(nsigma), _dptr(mask) if mask is not None else None,
                                     float(caustic), e.ctypes.data, nb, *(o.ctypes.data for o in out),
                                     _stream(stream)))
    return tuple(o[:nb] for o in out)


def ml_field_set_counts(field, counts, stream=None):
    """Replace the field's count map with a device int32/uint32 tensor (see ml.h)."""
    _check(load().ml_field_set_counts(field, _dptr(counts), 1, _stream(stream)))


def ml_map_light_curves(mu, tracks, n_samples, sigma_px, out, stream=None):
    """Light curves of a device float32 map (see ml.h)."""
    tr, ptr = _tracks_host(tracks)
    ny, nx = mu.shape
    _check_curves_out(out, len(tr), n_samples)
    _check(load().ml_map_light_curves(_dptr(mu), nx, ny, ptr, len(tr), n_samples, sigma_px,
                                      _dptr(out), _stream(stream)))


def ml_map_light_curves_backward(dL_dcurves, tracks, n_samples, sigma_px, dL_dmu, stream=None):
    """Transpose of ml_map_light_curves into dL_dmu (device float32, overwritten)."""
    tr, ptr = _tracks_host(tracks)
    ny, nx = dL_dmu.shape
    _check(load().ml_map_light_curves_backward(nx, ny, ptr, len(tr), n_samples, sigma_px,
                                               _dptr(dL_dcurves), _dptr(dL_dmu), _stream(stream)))


def ml_cic_backward(field, dL_dM, grad_lens, grad_params, stream=None, method=ADJOINT_NEARFAR):
    """Adjoint of the CIC magnification map (see ml.h); device tensors."""
    _check(load().ml_cic_backward_ex(field, _dptr(dL_dM), _dptr(grad_lens), _dptr(grad_params),
                                     method, _stream(stream)))


def ml_trace_rays(field, ray_idx, beta, pix, stream=None):
    _check(load().ml_trace_rays(field, _dptr(ray_idx), ray_idx.numel(), _dptr(beta), _dptr(pix),
                                _stream(stream)))


def ml_fp32_fma_peak(two_lane: bool, blocks_per_sm: int, iters: int, sink, stream=None) -> float:
    """One launch of the FP32 FMA throughput probe (see ml.h); returns its flop count."""
    flop = C.c_double()
    _check(load().ml_fp32_fma_peak(1 if two_lane else 0, blocks_per_sm, int(iters), _dptr(sink),
                                   C.byref(flop), _stream(stream)))
    return flop.value


def ml_field_clear(field, stream=None):
    _check(load().ml_field_clear(field, _stream(stream)))


def ml_field_stats(field, stream=None, check=True):
    out = (C.c_uint64 * len(STAT_NAMES))()
    st = load().ml_field_stats(field, out, _stream(stream))
    d = dict(zip(STAT_NAMES, list(out)))
    if check:
        _check(st)
    return d, st


def ml_field_info(field) -> dict:
    p = FieldParams()
    _check(load().ml_field_info(field, C.byref(p)))
    return p.as_dict()


def ml_field_abort(field, on: bool):
    _check(load().ml_field_abort(field, 1 if on else 0))


def ml_field_destroy(field):
    _check(load().ml_field_destroy(field))


# ---- convenience wrapper -------------------------------------------------------

def make_desc(workload, precision=PREC_MIXED, deposit=DEPOSIT_NGP, build=BUILD_AUTO,
              taylor_p=0, far_tol=0.0, l1=None, l2_sub=(0, 0), max_launch_rays=0, lens_arrays=None,
              tune=False, walk=WALK_CERTIFIED, span_far=0.0):
    """ml_field_desc for an inputs.Workload (lens arrays from host numpy)."""
    w = workload
    lx, ly, lm = lens_arrays if lens_arrays is not None else (w.lenses.x, w.lenses.y, w.lenses.m)
    lx = np.ascontiguousarray(lx, np.float64)
    ly = np.ascontiguousarray(ly, np.float64)
    lm = np.ascontiguousarray(lm, np.float64)
    d = FieldDesc()
    d.abi_version = ABI_VERSION
    d.precision, d.deposit, d.build = precision, deposit, build
    d.kappa, d.gamma, d.kappa_star = w.kappa, w.gamma, w.kappa_star
    d.lens_x, d.lens_y, d.lens_m = lx.ctypes.data, ly.ctypes.data, lm.ctypes.data
    d.n_lens = len(lx)
    d.lens_mem_is_device = 0
    d.taylor_p = taylor_p
    d.sheet_cx, d.sheet_cy, d.sheet_radius = w.sheet[:3]
    if len(w.sheet) > 3 and w.sheet[3] == "strip":
        d.sheet_shape = SHEET_STRIP
    if w.ray_box is not None:
        d.ray_x0, d.ray_y0, d.ray_x1, d.ray_y1 = w.ray_box
    if w.ray_n is not None:
        d.n_rays_x, d.n_rays_y = w.ray_n
    d.n_av = w.n_av
    d.map_x0, d.map_y0, d.map_x1, d.map_y1 = w.map_box
    d.map_nx, d.map_ny = w.map_n
    if l1 is None:
        l1 = getattr(w, "l1", None)
    if l1 is not None:
        d.l1_x, d.l1_y = l1
    if tuple(l2_sub) == (0, 0) and getattr(w, "l2", None):
        l2_sub = w.l2
    d.l2_sub_x, d.l2_sub_y = l2_sub
    d.tune = 1 if tune else 0
    d.walk = walk
    d.span_far = span_far
    macro = getattr(w, "macro", None)
    if macro is not None:
        d.macro_mode = MACRO_FOLD
        d.kappa0, d.d_x, d.d_y = macro[1], macro[2], macro[3]
    d.far_tol = far_tol
    d.max_launch_rays = max_launch_rays
    d._keep = (lx, ly, lm)       # keep the arrays alive until create returns
    return d


class Field:
    """One magnification map on the current CUDA device."""

    def __init__(self, workload=None, desc: FieldDesc | None = None, stream=None, **kw):
        if desc is None:
            desc = make_desc(workload, **kw)
        self.desc = desc
        self.h = ml_field_create(desc, stream)
        self.info = ml_field_info(self.h)

    @property
    def n_rays(self) -> int:
        return self.info["n_rays_x"] * self.info["n_rays_y"]

    def shoot(self, ray_begin=0, ray_end=None, stream=None):
        ml_shoot_rays(self.h, ray_begin, self.n_rays if ray_end is None else ray_end, stream)

    def counts(self, stream=None):
        import torch
        out = torch.empty((self.info["map_ny"], self.info["map_nx"]), dtype=torch.int32,
                          device="cuda")
        ml_magnification_map(self.h, MAP_COUNTS_U32, out, stream)
        return out

    def mu(self, dtype="f32", stream=None):
        import torch
        td = torch.float32 if dtype == "f32" else torch.float64
        out = torch.empty((self.info["map_ny"], self.info["map_nx"]), dtype=td, device="cuda")
        ml_magnification_map(self.h, MAP_MU_F32 if dtype == "f32" else MAP_MU_F64, out, stream)
        return out

    def light_curves(self, tracks, n_samples, sigma_px, stream=None):
        import torch
        out = torch.empty((len(tracks), n_samples), dtype=torch.float32, device="cuda")
        ml_light_curves(self.h, tracks, n_samples, sigma_px, out, stream)
        return out

    def trace(self, idx, stream=None):
        import torch
        idx = torch.as_tensor(np.asarray(idx, np.int64)).cuda()
        beta = torch.empty((idx.numel(), 2), dtype=torch.float64, device="cuda")
        pix = torch.empty((idx.numel(), 2), dtype=torch.int32, device="cuda")
        ml_trace_rays(self.h, idx, beta, pix, stream)
        return beta, pix

    def stats(self, stream=None, check=True):
        return ml_field_stats(self.h, stream, check)[0]

    def clear(self, stream=None):
        ml_field_clear(self.h, stream)

    def abort(self, on=True):
        ml_field_abort(self.h, on)

    def close(self):
        if self.h is not None:
            ml_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many maps shot in one persistent launch (ml_batch_*); fields are views."""

    def __init__(self, descs, tracks=None, n_samples=0, sigma_px=0.5, stream=None):
        arr = (FieldDesc * len(descs))(*descs)
        self._descs = descs
        tpm = 0
        tr_ptr = None
        if tracks is not None:
            tr = np.ascontiguousarray(tracks, np.float64)
            tpm = tr.shape[1]
            self._tracks = tr
            tr_ptr = tr.ctypes.data
        h = C.c_void_p()
        _check(load().ml_batch_create(arr, len(descs), tpm, tr_ptr, n_samples, sigma_px,
                                      _stream(stream), C.byref(h)))
        self.h = h
        self.n = len(descs)
        self.tpm = tpm
        self.n_samples = n_samples
        self.fields = []
        for i in range(self.n):
            fh = C.c_void_p()
            _check(load().ml_batch_field(h, i, C.byref(fh)))
            self.fields.append(fh)

    def run(self, use_graph=True, stream=None):
        _check(load().ml_batch_run(self.h, 1 if use_graph else 0, _stream(stream)))

    def info(self, i):
        return ml_field_info(self.fields[i])

    def stats(self, i, stream=None):
        return ml_field_stats(self.fields[i], stream)[0]

    def counts(self, i, stream=None):
        import torch
        inf = self.info(i)
        out = torch.empty((inf["map_ny"], inf["map_nx"]), dtype=torch.int32, device="cuda")
        ml_magnification_map(self.fields[i], MAP_COUNTS_U32, out, stream)
        return out

    def mu(self, i, stream=None):
        import torch
        inf = self.info(i)
        out = torch.empty((inf["map_ny"], inf["map_nx"]), dtype=torch.float32, device="cuda")
        _check(load().ml_batch_mu(self.h, i, _dptr(out), 1, _stream(stream)))
        return out

    def curves(self, stream=None):
        import torch
        out = torch.empty((self.n, self.tpm, self.n_samples), dtype=torch.float32, device="cuda")
        _check(load().ml_batch_curves(self.h, _dptr(out), 1, _stream(stream)))
        return out

    def abort(self, on=True):
        _check(load().ml_batch_abort(self.h, 1 if on else 0))

    def close(self):
        if self.h is not None:
            _check(load().ml_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
