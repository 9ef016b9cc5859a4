"""FP64 oracle for the microlensing ray-shooting path.

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this package; the product library
never does.  It shares no code with the CUDA path: its geometry, binning,
magnification and light-curve code below, and the per-ray arithmetic in
`oracle.c`, are written separately from the paper.

Every function names the part of the paper it follows (Yang, Chen, Zheng &
Luo, "Simulation of the microlensing effect near the critical curve of the
galaxy cluster").  Readings of points the paper leaves open are stated where
they are used.

Parity status: every function here is pinned by a test in
tests/test_oracle_pins.py against closed forms, invariants, brute force or
values printed in the paper; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (FP64, no FMA contraction) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [("kappa", C.c_double), ("gamma", C.c_double), ("kappa_star", C.c_double),
                ("sheet_cx", C.c_double), ("sheet_cy", C.c_double), ("sheet_r", C.c_double),
                ("rx0", C.c_double), ("ry0", C.c_double), ("l3x", C.c_double), ("l3y", C.c_double),
                ("n3x", C.c_int64), ("n3y", C.c_int64),
                ("mx0", C.c_double), ("my0", C.c_double), ("dpx", C.c_double), ("dpy", C.c_double),
                ("mnx", C.c_int64), ("mny", C.c_int64),
                ("macro_mode", C.c_int64), ("kappa0", C.c_double), ("d_x", C.c_double),
                ("d_y", C.c_double), ("sheet_shape", C.c_int64)]


class _Grid(C.Structure):
    _fields_ = [("n1x", C.c_int64), ("n1y", C.c_int64), ("n2x", C.c_int64), ("n2y", C.c_int64),
                ("N1x", C.c_int64), ("N1y", C.c_int64), ("p", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int32, C.c_uint64
        pd, pi64, pi32, pu64 = P(d), P(i64), P(i32), P(u64)
        g, gr = P(_Geom), P(_Grid)
        sig = {
            "orc_shoot_direct": [g, pd, pd, pd, i64, i64, i64, pu64, pu64, C.c_int],
            "orc_beta_direct": [g, pd, pd, pd, i64, pi64, i64, pd, pi32, C.c_int],
            "orc_beta_interp": [g, gr, pd, pd, pd, i64, pi64, i64, pd, pi32, C.c_int],
            "orc_node_coeffs": [g, gr, pd, pd, pd, i64, pi64, pi64, i64, pd],
            "orc_remainder_bound": [g, gr, pd, pd, pd, i64, pi64, i64, pd],
            "orc_cic_forward": [g, pd, pd, pd, i64, i64, i64, pd, C.c_int],
            "orc_cic_grad": [g, pd, pd, pd, i64, i64, i64, pd, d, pd, pd, C.c_int],
        }
        for name, argt in sig.items():
            f = getattr(_lib, name)
            f.argtypes = argt
            f.restype = C.c_int
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# Geometry: §3.1 (source region, protection band, N_*) and §3.2 (Eqs. 8, 10,
# 11 and the level-2 spacing).
# ---------------------------------------------------------------------------

@dataclass
class Geometry:
    kappa: float
    gamma: float
    kappa_star: float
    sheet_cx: float
    sheet_cy: float
    sheet_r: float
    rx0: float
    ry0: float
    rx1: float
    ry1: float
    l3x: float
    l3y: float
    n3x: int
    n3y: int
    mx0: float
    my0: float
    dpx: float
    dpy: float
    mnx: int
    mny: int
    n_star_in: int = 0       # lenses inside the ray rectangle (N_* of §3.1)
    l0: float = math.inf     # mean spacing per lens, L_0 of Eq. 10
    n1x: int = 0             # rays per level-1 cell, x
    n1y: int = 0
    n2x: int = 0             # rays per level-2 cell, x
    n2y: int = 0
    N1x: int = 0             # level-1 cells across the lattice
    N1y: int = 0
    p: int = 3
    macro_mode: int = 0      # 0: constant (kappa, gamma), Eq. 1; 1: fold, Eq. 5
    kappa0: float = 0.0      # fold: convergence on the critical curve
    d_x: float = 0.0         # fold: d = -(grad kappa)_0 - (grad gamma)_0, in 1/theta_E
    d_y: float = 0.0
    sheet_shape: int = 0     # 0: disc (centre, radius); 1: strip along x (centre line y, half-width)

    @property
    def n_rays(self) -> int:
        return self.n3x * self.n3y

    def c_geom(self) -> _Geom:
        return _Geom(self.kappa, self.gamma, self.kappa_star, self.sheet_cx, self.sheet_cy,
                     self.sheet_r, self.rx0, self.ry0, self.l3x, self.l3y, self.n3x, self.n3y,
                     self.mx0, self.my0, self.dpx, self.dpy, self.mnx, self.mny,
                     self.macro_mode, self.kappa0, self.d_x, self.d_y, self.sheet_shape)

    def c_grid(self) -> _Grid:
        return _Grid(self.n1x, self.n1y, self.n2x, self.n2y, self.N1x, self.N1y, self.p)


def protection_width(kappa_star: float) -> float:
    """Total widening of each source-plane side, 20 sqrt(kappa_*) (§3.1):
    a band of 10 sqrt(kappa_*) on each side of the target region."""
    return 20.0 * math.sqrt(kappa_star)


def n_star_from_area(area: float, kappa_star: float) -> float:
    """Number of unit-mass microlenses in an image-plane area (§3.1):
    N_* = L_ix L_iy kappa_* / pi."""
    return area * kappa_star / math.pi


def kappa_c(theta_e_arcsec: float, d_per_arcmin) -> float:
    """Stellar-density threshold kappa_c = (theta_E |d|)^(2/3) (§4.1, Table 1),
    with theta_E converted from arcsec to arcmin to match d in arcmin^-1."""
    dx, dy = d_per_arcmin
    return (theta_e_arcsec / 60.0 * math.hypot(dx, dy)) ** (2.0 / 3.0)


def _round_half_up(v: float) -> int:
    return int(math.floor(v + 0.5))


def fold_ray_box(kappa0, d_x, d_y, src_box):
    """Bounding box of the pre-image of the source box src_box = (x0, y0, x1,
    y1) under the fold map of Eq. 5, beta_x = d_x theta_x^2 / 2 + d_y theta_x
    theta_y, beta_y = 2 (1 - kappa_0) theta_y (reading: the image plane is the
    smallest rectangle holding every image of s').

    theta_y = beta_y / (2 (1 - kappa_0)).  For fixed theta_y (and d_x > 0; the
    map is mirrored in beta_x otherwise) the images of beta_x <= x1 are
    |theta_x - t*| <= s1 with t* = -d_y theta_y / d_x and
    s1 = sqrt(2 x1 / d_x + (d_y theta_y / d_x)^2); t* + s1 is convex and
    t* - s1 concave in theta_y, so the extremes lie at the ends of the
    theta_y range.  Requires images (x1 > 0 after mirroring)."""
    x0, y0, x1, y1 = src_box
    a = 2.0 * (1.0 - kappa0)
    if a == 0.0 or d_x == 0.0:
        raise ValueError("fold map is singular")
    ty = sorted((y0 / a, y1 / a))
    if d_x < 0.0:
        x0, x1, d_x, d_y = -x1, -x0, -d_x, -d_y
    if x1 <= 0.0:
        raise ValueError("the source box has no images under the fold map")
    lo, hi = math.inf, -math.inf
    for t in ty:
        c = -d_y * t / d_x
        s1 = math.sqrt(2.0 * x1 / d_x + (d_y * t / d_x) ** 2)
        lo, hi = min(lo, c - s1), max(hi, c + s1)
    return lo, ty[0], hi, ty[1]


def derive_geometry(kappa, gamma, kappa_star, lens_x, lens_y, sheet, map_box, map_n,
                    ray_box=None, ray_n=None, n_av=0.0, l1=None, l2_sub=20, p=3,
                    l2_sub_y=None, macro=None) -> Geometry:
    """The parameters of §3.1-§3.2 for one map.

    Readings: the ray rectangle is the pre-image of the widened source region
    s' under the macro map diag(1-kappa-gamma, 1-kappa+gamma) (§3.1: "from the
    lens equation, one can obtain the image plane"); L_1y follows L_1x's rule
    on the y side; N_* in L_0 counts the lenses inside the ray rectangle; the
    level grids are laid on the ray lattice, a level-2 cell holding
    round(L_2 / L_3) rays per side and a level-1 cell l2_sub (x) or l2_sub_y (y,
    default l2_sub) times that; the paper's L_2 = L_1 / 20 is l2_sub = 20.
    """
    mx0, my0, mx1, my1 = map_box
    mnx, mny = map_n
    dpx = (mx1 - mx0) / mnx
    dpy = (my1 - my0) / mny
    if ray_box is None and macro is not None:
        w = 0.5 * protection_width(kappa_star)
        rx0, ry0, rx1, ry1 = fold_ray_box(macro[1], macro[2], macro[3],
                                          (mx0 - w, my0 - w, mx1 + w, my1 + w))
    elif ray_box is None:
        w = 0.5 * protection_width(kappa_star)
        a = 1.0 - kappa - gamma
        b = 1.0 - kappa + gamma
        if a == 0.0 or b == 0.0:
            raise ValueError("macro map is singular: no pre-image of the source region")
        xs = sorted(((mx0 - w) / a, (mx1 + w) / a))
        ys = sorted(((my0 - w) / b, (my1 + w) / b))
        rx0, rx1, ry0, ry1 = xs[0], xs[1], ys[0], ys[1]
    else:
        rx0, ry0, rx1, ry1 = ray_box
    lix = rx1 - rx0
    liy = ry1 - ry0
    if ray_n is None:
        n_rays = n_av * mnx * mny                      # Eq. 8
        l3 = math.sqrt(lix * liy / n_rays)             # Eq. 11
        n3x = max(1, _round_half_up(lix / l3))
        n3y = max(1, _round_half_up(liy / l3))
    else:
        n3x, n3y = ray_n
    l3x = lix / n3x
    l3y = liy / n3y
    lx = np.asarray(lens_x)
    ly = np.asarray(lens_y)
    n_in = int(np.count_nonzero((lx >= rx0) & (lx < rx1) & (ly >= ry0) & (ly < ry1)))
    l0 = math.sqrt(lix * liy / n_in) if n_in > 0 else math.inf
    if l1 is None:
        l1x = min(l0, lix / 10.0)                      # Eq. 10
        l1y = min(l0, liy / 10.0)
    else:
        l1x, l1y = l1
    l2sy = l2_sub if l2_sub_y is None else l2_sub_y
    l2x = l1x / l2_sub                                 # §3.2, Level 2
    l2y = l1y / l2sy
    n2x = max(1, _round_half_up(l2x / l3x))
    n2y = max(1, _round_half_up(l2y / l3y))
    n1x = l2_sub * n2x
    n1y = l2sy * n2y
    g = Geometry(kappa, gamma, kappa_star, sheet[0], sheet[1], sheet[2],
                 rx0, ry0, rx1, ry1, l3x, l3y, n3x, n3y, mx0, my0, dpx, dpy, mnx, mny,
                 n_in, l0, n1x, n1y, n2x, n2y, -(-n3x // n1x), -(-n3y // n1y), p)
    if macro is not None:
        g.macro_mode, g.kappa0, g.d_x, g.d_y = 1, float(macro[1]), float(macro[2]), float(macro[3])
    if len(sheet) > 3 and sheet[3] == "strip":
        g.sheet_shape = 1
    return g


def geometry_of(w, **kw) -> Geometry:
    """derive_geometry for a paper_2308_14278_gb300.inputs.Workload."""
    if getattr(w, "l1", None) is not None and "l1" not in kw:
        kw["l1"] = w.l1
    if getattr(w, "macro", None) is not None and "macro" not in kw:
        kw["macro"] = w.macro
    return derive_geometry(w.kappa, w.gamma, w.kappa_star, w.lenses.x, w.lenses.y, w.sheet,
                           w.map_box, w.map_n, ray_box=w.ray_box, ray_n=w.ray_n,
                           n_av=w.n_av, **kw)


# ---------------------------------------------------------------------------
# Ray shooting and per-ray source positions (oracle.c)
# ---------------------------------------------------------------------------

def _lens_arrays(x, y, m):
    return (np.ascontiguousarray(x, np.float64), np.ascontiguousarray(y, np.float64),
            np.ascontiguousarray(m, np.float64))


def shoot_direct(g: Geometry, x, y, m, ray_begin=0, ray_end=None, threads=None):
    """Counts N_ij (uint64, mny x mnx) of rays [ray_begin, ray_end) by direct
    summation, and stats (in map, out of map, dropped): the plain definition
    the near/far scheme approximates -- every lattice ray (§3.2 Level 3)
    through the lens equation with the deflection of all lenses (Eq. 6, or
    Eq. 5's fold term), binned by the nearest grid point into the source-plane
    pixels whose counts Eq. 12 turns into magnification."""
    x, y, m = _lens_arrays(x, y, m)
    if ray_end is None:
        ray_end = g.n_rays
    counts = np.zeros((g.mny, g.mnx), np.uint64)
    stats = np.zeros(3, np.uint64)
    gg = g.c_geom()
    rc = lib().orc_shoot_direct(C.byref(gg), _ptr(x, C.c_double), _ptr(y, C.c_double),
                                _ptr(m, C.c_double), len(x), int(ray_begin), int(ray_end),
                                _ptr(counts, C.c_uint64), _ptr(stats, C.c_uint64),
                                threads or default_threads())
    assert rc == 0
    return counts, stats


def beta_direct(g: Geometry, x, y, m, idx, threads=None):
    """Source positions (n, 2) of rays idx by Eq. 6 summed over all lenses;
    also a dropped flag per ray."""
    x, y, m = _lens_arrays(x, y, m)
    idx = np.ascontiguousarray(idx, np.int64)
    beta = np.zeros((len(idx), 2))
    flag = np.zeros(len(idx), np.int32)
    gg = g.c_geom()
    lib().orc_beta_direct(C.byref(gg), _ptr(x, C.c_double), _ptr(y, C.c_double),
                          _ptr(m, C.c_double), len(x), _ptr(idx, C.c_int64), len(idx),
                          _ptr(beta, C.c_double), _ptr(flag, C.c_int32),
                          threads or default_threads())
    return beta, flag


def beta_interp(g: Geometry, x, y, m, idx, threads=None):
    """Source positions of rays idx by the near/far scheme of Eq. 9, with
    far-field Taylor coefficients summed brute force at each level-2 node."""
    x, y, m = _lens_arrays(x, y, m)
    idx = np.ascontiguousarray(idx, np.int64)
    beta = np.zeros((len(idx), 2))
    flag = np.zeros(len(idx), np.int32)
    gg, gr = g.c_geom(), g.c_grid()
    rc = lib().orc_beta_interp(C.byref(gg), C.byref(gr), _ptr(x, C.c_double),
                               _ptr(y, C.c_double), _ptr(m, C.c_double), len(x),
                               _ptr(idx, C.c_int64), len(idx), _ptr(beta, C.c_double),
                               _ptr(flag, C.c_int32), threads or default_threads())
    assert rc == 0
    return beta, flag


def node_coeffs(g: Geometry, x, y, m, c2x, c2y):
    """Complex far-field Taylor coefficients c_0..c_p at level-2 nodes
    (c2x, c2y): array (nnodes, p+1) complex128.  §3.2 Level 2: the far
    lenses' deflection expanded in a Taylor series about each level-2 grid
    point, evaluated per ray by Eq. 9."""
    x, y, m = _lens_arrays(x, y, m)
    c2x = np.ascontiguousarray(c2x, np.int64)
    c2y = np.ascontiguousarray(c2y, np.int64)
    out = np.zeros((len(c2x), g.p + 1, 2))
    gg, gr = g.c_geom(), g.c_grid()
    rc = lib().orc_node_coeffs(C.byref(gg), C.byref(gr), _ptr(x, C.c_double),
                               _ptr(y, C.c_double), _ptr(m, C.c_double), len(x),
                               _ptr(c2x, C.c_int64), _ptr(c2y, C.c_int64), len(c2x),
                               _ptr(out, C.c_double))
    assert rc == 0
    return out[..., 0] + 1j * out[..., 1]


def node_position(g: Geometry, c2x, c2y):
    """Centre of level-2 cell (c2x, c2y), the expansion point of its series
    (§3.2 Level 2; the paper's "grid point where the ray is located" read as
    the centre of the ray's level-2 cell)."""
    l2x = g.n2x * g.l3x
    l2y = g.n2y * g.l3y
    return g.rx0 + (np.asarray(c2x) + 0.5) * l2x, g.ry0 + (np.asarray(c2y) + 0.5) * l2y


def remainder_bound(g: Geometry, x, y, m, idx):
    """Upper bound of the far-series truncation error at each ray of idx: the
    tail of Eq. 9's series beyond order p, summed over the far lenses
    (sum_k m_k rho^(p+1) / (r_k^(p+1) (r_k - rho)), rho the ray's distance from
    its node, r_k the lens's).  The paper states the accuracy it reaches
    (§3.2) but no bound; this is the geometric-series bound of the
    expansion."""
    x, y, m = _lens_arrays(x, y, m)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.zeros(len(idx))
    gg, gr = g.c_geom(), g.c_grid()
    lib().orc_remainder_bound(C.byref(gg), C.byref(gr), _ptr(x, C.c_double),
                              _ptr(y, C.c_double), _ptr(m, C.c_double), len(x),
                              _ptr(idx, C.c_int64), len(idx), _ptr(out, C.c_double))
    return out


def ray_position(g: Geometry, idx):
    """Lattice position of rays idx: centre of level-3 pixel (i, j), §3.2."""
    idx = np.asarray(idx, np.int64)
    i = idx % g.n3x
    j = idx // g.n3x
    return g.rx0 + (i + 0.5) * g.l3x, g.ry0 + (j + 0.5) * g.l3y


def pixel_of(g: Geometry, beta):
    """Nearest-grid-point pixel (ix, iy) of source positions (Eq. 12 binning),
    as floats: floor((beta - map origin) / pixel size)."""
    return (np.floor((beta[:, 0] - g.mx0) / g.dpx), np.floor((beta[:, 1] - g.my0) / g.dpy))


# ---------------------------------------------------------------------------
# Magnification (Eq. 12) and light curves (§4.1)
# ---------------------------------------------------------------------------

def magnification(g: Geometry, counts):
    """mu_ij = N_ij S_I / S_S (Eq. 12): S_I the level-3 pixel area, S_S the
    source-pixel area."""
    return np.asarray(counts, np.float64) * ((g.l3x * g.l3y) / (g.dpx * g.dpy))


def gaussian_taps(sigma_px: float):
    """Discrete Gaussian source profile: taps at integer offsets |t| <= 4 sigma
    (reading: truncated at 4 sigma), normalised to sum 1."""
    h = int(math.floor(4.0 * sigma_px))
    t = np.arange(-h, h + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma_px) ** 2)
    return w / w.sum()


def convolve_gaussian(mu, sigma_px: float):
    """Finite-source map: mu convolved with the Gaussian taps along each axis,
    zero outside the map (the Gaussian source of §4.1)."""
    w = gaussian_taps(sigma_px)
    h = len(w) // 2
    ny, nx = mu.shape
    pad = np.zeros((ny + 2 * h, nx + 2 * h))
    pad[h:h + ny, h:h + nx] = mu
    tmp = np.zeros((ny + 2 * h, nx))
    for q, wq in enumerate(w):
        tmp += wq * pad[:, q:q + nx]
    out = np.zeros((ny, nx))
    for q, wq in enumerate(w):
        out += wq * tmp[q:q + ny, :]
    return out


def bilinear(img, u, v):
    """Bilinear value at map coordinates (u, v) between pixel centres
    (pixel (i, j) has its centre at (i + 1/2, j + 1/2)); zero outside.  The
    light curves of §4.1 sample the finite-source map this way between
    pixels (the paper does not state its interpolation)."""
    ny, nx = img.shape
    fx = np.asarray(u) - 0.5
    fy = np.asarray(v) - 0.5
    i0 = np.floor(fx).astype(np.int64)
    j0 = np.floor(fy).astype(np.int64)
    wx = fx - i0
    wy = fy - j0
    out = np.zeros(np.shape(fx))
    for di, wi in ((0, 1.0 - wx), (1, wx)):
        for dj, wj in ((0, 1.0 - wy), (1, wy)):
            ii = i0 + di
            jj = j0 + dj
            ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)
            val = np.where(ok, img[np.clip(jj, 0, ny - 1), np.clip(ii, 0, nx - 1)], 0.0)
            out = out + wi * wj * val
    return out


def light_curves(mu, tracks, n_samples: int, sigma_px: float):
    """Light curves of a Gaussian source (§4.1, Fig. 3): the magnification of
    the convolved map sampled at n_samples equally spaced points from
    (x0, y0) to (x1, y1), endpoints included, for each track."""
    conv = convolve_gaussian(np.asarray(mu, np.float64), sigma_px)
    tr = np.asarray(tracks, np.float64)
    t = np.linspace(0.0, 1.0, n_samples) if n_samples > 1 else np.zeros(1)
    out = np.zeros((len(tr), n_samples))
    for q, (x0, y0, x1, y1) in enumerate(tr):
        out[q] = bilinear(conv, x0 + t * (x1 - x0), y0 + t * (y1 - y0))
    return out


def light_curves_sampled(mu, tracks, n_samples: int, sigma_px: float):
    """light_curves (§4.1) for a map too large to convolve whole: the convolved map
    is evaluated only at the pixels that the bilinear samples read, with the
    same taps, the same zero outside the map and the same order of the sums
    (along x, then along y; then the four bilinear terms), so the two agree
    exactly."""
    mu = np.asarray(mu)
    w = gaussian_taps(sigma_px)
    h = len(w) // 2
    ny, nx = mu.shape

    def conv_at(ii, jj):
        val = np.zeros(np.shape(ii))
        for b in range(2 * h + 1):
            r = jj + b - h
            row = np.zeros(np.shape(ii))
            for a in range(2 * h + 1):
                c = ii + a - h
                ok = (r >= 0) & (r < ny) & (c >= 0) & (c < nx)
                v = np.where(ok, mu[np.clip(r, 0, ny - 1), np.clip(c, 0, nx - 1)], 0.0)
                row = row + w[a] * v
            val = val + w[b] * row
        return val

    tr = np.asarray(tracks, np.float64)
    t = np.linspace(0.0, 1.0, n_samples) if n_samples > 1 else np.zeros(1)
    out = np.zeros((len(tr), n_samples))
    for q, (x0, y0, x1, y1) in enumerate(tr):
        fx = (x0 + t * (x1 - x0)) - 0.5
        fy = (y0 + t * (y1 - y0)) - 0.5
        i0 = np.floor(fx).astype(np.int64)
        j0 = np.floor(fy).astype(np.int64)
        wx = fx - i0
        wy = fy - j0
        acc = np.zeros(np.shape(fx))
        for di, wi in ((0, 1.0 - wx), (1, wx)):
            for dj, wj in ((0, 1.0 - wy), (1, wy)):
                ii = i0 + di
                jj = j0 + dj
                ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)
                acc = acc + wi * wj * np.where(ok, conv_at(ii, jj), 0.0)
        out[q] = acc
    return out


# ---------------------------------------------------------------------------
# Cloud-in-cell map and its gradient (the differentiable variant)
# ---------------------------------------------------------------------------

def cic_forward(g: Geometry, x, y, m, ray_begin=0, ray_end=None, threads=None):
    """Cloud-in-cell ray map (FP64, mny x mnx, units of rays): every lattice
    ray's Eq. 6 source position shared bilinearly among the four nearest
    pixel centres, the differentiable counterpart of Eq. 12's binning (the
    paper has no differentiable form; weights of centres outside the map are
    dropped)."""
    x, y, m = _lens_arrays(x, y, m)
    if ray_end is None:
        ray_end = g.n_rays
    out = np.zeros((g.mny, g.mnx))
    gg = g.c_geom()
    lib().orc_cic_forward(C.byref(gg), _ptr(x, C.c_double), _ptr(y, C.c_double),
                          _ptr(m, C.c_double), len(x), int(ray_begin), int(ray_end),
                          _ptr(out, C.c_double), threads or default_threads())
    return out


def cic_mu_scale(g: Geometry) -> float:
    """S_I / S_S, turning a CIC ray map into magnification (Eq. 12)."""
    return (g.l3x * g.l3y) / (g.dpx * g.dpy)


def cic_loss(g: Geometry, x, y, m, target, ray_begin=0, ray_end=None, threads=None):
    """L = sum_ij (M_ij - T_ij)^2 with M = S_I/S_S * CIC map (Eq. 12 scaling of
    the cloud-in-cell map)."""
    M = cic_mu_scale(g) * cic_forward(g, x, y, m, ray_begin, ray_end, threads)
    return float(np.sum((M - target) ** 2)), M


def cic_grad_dM(g: Geometry, x, y, m, dL_dM, ray_begin=0, ray_end=None, threads=None):
    """FP64 gradient of any loss of the CIC magnification map M given its
    dL/dM (mny x mnx): (dL/dlens (n, 3), dL/d(kappa, gamma, kappa_*)), by
    differentiating Eq. 6 (macro term, point-mass sum and sheet) and the
    bilinear weights ray by ray, over all lenses."""
    x, y, m = _lens_arrays(x, y, m)
    if ray_end is None:
        ray_end = g.n_rays
    G = np.ascontiguousarray(dL_dM, np.float64)
    gl = np.zeros((len(x), 3))
    gp = np.zeros(3)
    gg = g.c_geom()
    rc = lib().orc_cic_grad(C.byref(gg), _ptr(x, C.c_double), _ptr(y, C.c_double),
                            _ptr(m, C.c_double), len(x), int(ray_begin), int(ray_end),
                            _ptr(G, C.c_double), cic_mu_scale(g), _ptr(gl, C.c_double),
                            _ptr(gp, C.c_double), threads or default_threads())
    if rc != 0:
        raise ValueError("the oracle's CIC gradient covers the constant-(kappa, gamma) macro "
                         "with a disc sheet only")
    return gl, gp


def cic_grad(g: Geometry, x, y, m, target, ray_begin=0, ray_end=None, threads=None):
    """FP64 reference gradient of cic_loss: (dL/dlens (n, 3), dL/d(kappa,
    gamma, kappa_*)), Eq. 6 differentiated as in cic_grad_dM."""
    x, y, m = _lens_arrays(x, y, m)
    if ray_end is None:
        ray_end = g.n_rays
    _, M = cic_loss(g, x, y, m, target, ray_begin, ray_end, threads)
    G = np.ascontiguousarray(2.0 * (M - target))
    gl = np.zeros((len(x), 3))
    gp = np.zeros(3)
    gg = g.c_geom()
    rc = lib().orc_cic_grad(C.byref(gg), _ptr(x, C.c_double), _ptr(y, C.c_double),
                            _ptr(m, C.c_double), len(x), int(ray_begin), int(ray_end),
                            _ptr(G, C.c_double), cic_mu_scale(g), _ptr(gl, C.c_double),
                            _ptr(gp, C.c_double), threads or default_threads())
    if rc != 0:
        raise ValueError("the oracle's CIC gradient covers the constant-(kappa, gamma) macro "
                         "with a disc sheet only")
    return gl, gp


# ---------------------------------------------------------------------------
# Peak identification on light curves (§4.2)
# ---------------------------------------------------------------------------

def peaks(counts, along: str = "x", nsigma: float = 5.0):
    """The two-step peak identification of §4.2 on a count map (ny x nx).

    Light curves run along `along` ("x": each map row is a curve and the
    neighbouring curves are the rows above and below; "y": each column).
    Step 1, candidate at position j of curve i: N_ij > max(N_i,j-1, N_i,j+1)
    and h_ij = N_ij - <N> > nsigma sigma_ij, <N> = (N_i,j-1 + N_ij + N_i,j+1)/3,
    sigma_ij = sqrt(<N>).  Squared (both sides positive), with a, b the two
    neighbours: (2 N - a - b)^2 > 3 nsigma^2 (a + N + b), compared in FP64.
    Positions at the ends of a curve have no candidate.
    Step 2, a candidate is a true peak when one of positions j-1, j, j+1 of
    curve i-1 and one of curve i+1 are candidates; the first and last curves
    have no true peaks.
    Returns the uint8 mask: bit 0 candidate, bit 1 true peak."""
    N = np.asarray(counts)
    if along == "y":
        return peaks(N.T, "x", nsigma).T.copy()
    ny, nx = N.shape
    mask = np.zeros((ny, nx), np.uint8)
    k2x3 = 3.0 * nsigma * nsigma
    for i in range(ny):
        for j in range(1, nx - 1):
            a, c, b = int(N[i, j - 1]), int(N[i, j]), int(N[i, j + 1])
            if c > a and c > b and float((2 * c - a - b) ** 2) > k2x3 * float(a + c + b):
                mask[i, j] |= 1
    cand = (mask & 1).astype(bool)
    for i in range(1, ny - 1):
        for j in range(1, nx - 1):
            if cand[i, j] and cand[i - 1, j - 1:j + 2].any() and cand[i + 1, j - 1:j + 2].any():
                mask[i, j] |= 2
    return mask


def peak_statistics(counts, mask, along: str, origin: float, step: float, caustic: float, edges):
    """The statistics of §4.2 (Figs. 4 and 5) over the true peaks of a map:
    the number of micro-caustic crossings and the peak magnification, both
    as functions of the source's distance from the macro caustic.

    The distance of position j along a curve is that of its pixel centre,
    d = |origin + (j + 1/2) step - caustic| (origin and step the map's origin
    and pixel size along the curves; the caustic a line across them, as in a
    local region of the critical curve, §2).  Position j lies in bin b when
    edges[b] <= d < edges[b+1]; positions outside [edges[0], edges[-1]) lie in
    none.  Per bin:
      n_peaks     true peaks (mask bit 1) in the bin;
      sum_counts  the sum of their counts N_ij, so that the mean peak
                  magnification is sum_counts S_I/S_S / n_peaks (Eq. 12);
      n_positions the positions where a true peak can occur (curves other than
                  the first and last, positions other than the two ends), so
                  that the crossings per unit length of curve are
                  n_peaks / (n_positions step).
    The three are integers, returned as uint64 arrays of len(edges) - 1."""
    N = np.asarray(counts)
    M = np.asarray(mask)
    if along == "y":
        return peak_statistics(N.T, M.T, "x", origin, step, caustic, edges)
    e = [float(v) for v in edges]
    nb = len(e) - 1
    ny, nx = N.shape
    n_peaks = np.zeros(nb, np.uint64)
    sums = np.zeros(nb, np.uint64)
    n_pos = np.zeros(nb, np.uint64)

    def bin_of(j):
        centre = origin + (j + 0.5) * step
        d = abs(centre - caustic)
        for b in range(nb):
            if e[b] <= d < e[b + 1]:
                return b
        return -1

    bins = [bin_of(j) if 0 < j < nx - 1 else -1 for j in range(nx)]
    for j in range(nx):
        if bins[j] >= 0:
            n_pos[bins[j]] += max(ny - 2, 0)
    for i in range(ny):
        for j in range(nx):
            if (int(M[i, j]) & 2) and bins[j] >= 0:
                n_peaks[bins[j]] += 1
                sums[bins[j]] += int(N[i, j])
    return n_peaks, sums, n_pos
