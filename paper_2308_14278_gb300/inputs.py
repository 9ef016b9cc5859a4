"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds random numbers and workload parameters only: it draws lens
fields, light-curve tracks and target fields, and lists the workload shapes.
It contains none of the ray-shooting arithmetic (no lens equation, no
geometry derivation, no binning), so both sides of a parity test can take
their inputs from here without sharing any of the method's code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output k of stream s under seed S is mix(S * 2^32 + s * 2^48 + (k+1) * phi)
where phi = 0x9E3779B97F4A7C15 and mix is the SplitMix64 finaliser.  Doubles
in [0, 1) take the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_PHI = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of SplitMix64 stream `stream` under `seed`."""
    with np.errstate(over="ignore"):
        base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) ^ (
            np.uint64(stream & 0xFFFF) << np.uint64(48))
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = base + k * _PHI
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, stream, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def std_normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform (FP64)."""
    u1 = uniform01(seed, stream, n)
    u2 = uniform01(seed, stream + 1, n)
    u1 = np.where(u1 <= 0.0, 2.0 ** -53, u1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class LensField:
    """Point lenses (angles in Einstein radii, masses in units of M)."""
    x: np.ndarray
    y: np.ndarray
    m: np.ndarray
    cx: float = 0.0          # centre of the disc they were drawn in
    cy: float = 0.0
    radius: float = 0.0      # radius of that disc

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def lens_disc(n: int, radius: float, seed: int, mass: str = "unit",
              median: float = 0.3, sigma_ln: float = 0.5,
              cx: float = 0.0, cy: float = 0.0) -> LensField:
    """n lenses uniform in a disc: r = R sqrt(u), phi = 2 pi v.

    mass="unit" gives m = 1; mass="lognormal" gives m = median * exp(sigma_ln z)
    with z standard normal.
    """
    u = uniform01(seed, 1, n)
    v = uniform01(seed, 2, n)
    r = radius * np.sqrt(u)
    phi = 2.0 * np.pi * v
    x = cx + r * np.cos(phi)
    y = cy + r * np.sin(phi)
    if mass == "unit":
        m = np.ones(n)
    elif mass == "lognormal":
        m = median * np.exp(sigma_ln * std_normal(seed, 3, n))
    else:
        raise ValueError(f"unknown mass distribution {mass!r}")
    return LensField(np.ascontiguousarray(x), np.ascontiguousarray(y),
                     np.ascontiguousarray(m), cx, cy, radius)


def lognormal_mean(median: float, sigma_ln: float) -> float:
    """Mean of median * exp(sigma_ln z): median * exp(sigma_ln^2 / 2)."""
    return median * math.exp(0.5 * sigma_ln * sigma_ln)


def tracks(n_tracks: int, nx: int, ny: int, margin_px: float, seed: int) -> np.ndarray:
    """Straight tracks with both endpoints uniform in the map shrunk by margin_px.

    Returns an (n_tracks, 4) float64 array of (x0, y0, x1, y1) in map pixel
    coordinates (pixel i spans [i, i+1)).
    """
    u = uniform01(seed, 11, 4 * n_tracks).reshape(n_tracks, 4)
    out = np.empty((n_tracks, 4))
    out[:, 0] = margin_px + u[:, 0] * (nx - 2 * margin_px)
    out[:, 1] = margin_px + u[:, 1] * (ny - 2 * margin_px)
    out[:, 2] = margin_px + u[:, 2] * (nx - 2 * margin_px)
    out[:, 3] = margin_px + u[:, 3] * (ny - 2 * margin_px)
    return out


@dataclass
class Workload:
    """One synthetic map: lens field, macro model, map and ray budget."""
    name: str
    lenses: LensField
    kappa: float
    gamma: float
    kappa_star: float
    sheet: tuple            # (cx, cy, radius) of the compensating sheet's disc
    map_box: tuple          # (x0, y0, x1, y1) in Einstein radii
    map_n: tuple            # (nx, ny) pixels
    ray_box: tuple | None = None    # explicit ray rectangle, or None to derive it
    ray_n: tuple | None = None      # explicit (n3x, n3y), or None to use n_av
    n_av: float = 0.0
    l1: tuple | None = None         # explicit level-1 cell size, or None for Eq. 10's rule
    l2: tuple | None = None         # explicit level-2 subdivisions, or None for the library's
    macro: tuple | None = None      # ("fold", kappa0, d_x, d_y) for the fold model, else None
    n_tracks: int = 0
    track_samples: int = 4096
    sigma_px: float = 0.5
    extra: dict = field(default_factory=dict)


def small_map(seed: int = 0) -> Workload:
    """100 unit-mass lenses in a disc of radius 15; kappa=0.45, gamma=0.50,
    kappa_*=0.01; a 2000 x 2000 ray grid over [-5, 5]^2; a 256^2 map of
    [-1, 1]^2.  Taken literally: the lens density (0.44) does not match
    kappa_* (0.01), which only drives the sheet."""
    lf = lens_disc(100, 15.0, seed, "unit")
    return Workload("small map: 100 lenses, 2000^2 rays, 256^2 map", lf,
                    0.45, 0.50, 0.01, (0.0, 0.0, 15.0),
                    (-1.0, -1.0, 1.0, 1.0), (256, 256),
                    ray_box=(-5.0, -5.0, 5.0, 5.0), ray_n=(2000, 2000))


def small_map_consistent(seed: int = 0) -> Workload:
    """As small_map but kappa_* = N m / R^2 = 100/225, so that the sheet
    cancels the lenses' mean convergence; smooth part kappa - kappa_*."""
    w = small_map(seed)
    w.name = "small map, consistent sheet"
    w.kappa_star = 100.0 / 225.0
    w.kappa = 0.45 + w.kappa_star - 0.01
    return w


# Paper-scale geometry.  The lens disc radius follows from kappa_* = N <m> / R^2.
# The map side 23.65 makes that disc 1.5 times the half-diagonal of the ray
# rectangle, the pre-image of the map plus its protection band under the
# macro model (1 - kappa - gamma = 0.02, 1 - kappa + gamma = 1.02).
PAPER_N_LENS = 13000
PAPER_MAP_SIDE = 23.65


def paper_map(seed: int = 0, n_rays: float = 1e11, map_px: int = 8192,
              n_tracks: int = 10) -> Workload:
    """13,000 lognormal lenses (median 0.3, sigma_ln 0.5) in a disc,
    kappa=0.48, gamma=0.50, kappa_*=0.005, 1e11 rays, 8192^2 map."""
    ks = 0.005
    r = math.sqrt(PAPER_N_LENS * lognormal_mean(0.3, 0.5) / ks)
    lf = lens_disc(PAPER_N_LENS, r, seed, "lognormal", 0.3, 0.5)
    h = 0.5 * PAPER_MAP_SIDE
    return Workload(f"paper-scale map: 13000 lenses, {n_rays:.0e} rays, {map_px}^2 map",
                    lf, 0.48, 0.50, ks, (0.0, 0.0, r), (-h, -h, h, h),
                    (map_px, map_px), n_av=n_rays / (map_px * map_px),
                    n_tracks=n_tracks)


def differentiable_field(seed: int = 0, n_lens: int = 1000, n_rays: float = 4e8,
                         map_px: int = 1024) -> Workload:
    """1,000 lognormal lenses, kappa=0.48, gamma=0.5, kappa_*=0.005, 4e8 rays,
    1024^2 float map (cloud-in-cell).  The ray rectangle is a strip about
    350 x 7 Einstein radii.  Eq. 10's rule per axis would make level-1 cells
    24 x 0.7, whose far series converges too slowly at the cells' edges, so
    they are set square: 2.5 x 2.5 with level-2 cells of a tenth of that,
    the fastest forward + adjoint step measured over 2.5 to 12 (0.1 near
    lenses per ray; 4.4 ms against 8.9 ms for 12 x 12 cells, whose near
    sums of 5.5 lenses per ray dominate both kernels)."""
    ks = 0.005
    r = math.sqrt(n_lens * lognormal_mean(0.3, 0.5) / ks)
    lf = lens_disc(n_lens, r, seed, "lognormal", 0.3, 0.5)
    # Same construction as the paper-scale map: disc = 1.5 x half-diagonal.
    # 1.5 * 0.5 * L' * sqrt(50^2 + (1/1.02)^2) = r  ->  L' = r / 37.507
    lp = r / (0.75 * math.hypot(50.0, 1.0 / 1.02))
    h = 0.5 * (lp - 20.0 * math.sqrt(ks))
    return Workload(f"differentiable: {n_lens} lenses, {n_rays:.0e} rays, {map_px}^2 CIC",
                    lf, 0.48, 0.50, ks, (0.0, 0.0, r), (-h, -h, h, h),
                    (map_px, map_px), n_av=n_rays / (map_px * map_px), l1=(2.5, 2.5), l2=(10, 10))


# Table 1 (§4.1): the fold field of MACS J1149.5+2223, theta_E = 1e-6 arcsec.
TABLE1_KAPPA0 = 0.83
TABLE1_D_PER_ARCMIN = (3.62, -3.41)
TABLE1_THETA_E_ARCSEC = 1e-6
TABLE1_KAPPA_STAR = 0.001
TABLE1_N_STAR = 13745
# Image-plane rectangle of the 40 x 200 theta_E^2 source region of §4.1 widened
# by the protection band, under the fold map (rounded outward): holds 13,839
# lenses at kappa_* = 0.001 by N_* = L_ix L_iy kappa_* / pi (Table 1: 13,745).
TABLE1_LENS_RECT = (-36560.0, -1.0, 37120.0, 589.2)


def fold_field(seed: int = 0, n_rays: float = 1e11, map_px=(2048, 10240),
               n_tracks: int = 10) -> Workload:
    """The Table-1 fold field at reduced resolution: kappa_0 = 0.83,
    d = (3.62, -3.41) arcmin^-1 in units of 1/theta_E, kappa_* = 0.001,
    13,745 unit-mass lenses uniform in the image-plane rectangle, the sheet a
    strip over the same y range (the rectangle is 125 times longer than it is
    wide, so its field is a slab's); the source region
    beta_x in [0, 40], beta_y in [0, 200] (the 200 x 40 theta_E^2 of §4.1) on
    map_px pixels, n_rays rays."""
    arcmin_in_theta_e = 60.0 / TABLE1_THETA_E_ARCSEC
    dx = TABLE1_D_PER_ARCMIN[0] / arcmin_in_theta_e
    dy = TABLE1_D_PER_ARCMIN[1] / arcmin_in_theta_e
    x0, y0, x1, y1 = TABLE1_LENS_RECT
    u = uniform01(seed, 31, TABLE1_N_STAR)
    v = uniform01(seed, 32, TABLE1_N_STAR)
    lf = LensField(x0 + (x1 - x0) * u, y0 + (y1 - y0) * v, np.ones(TABLE1_N_STAR),
                   0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.0)
    nx, ny = map_px
    return Workload(f"fold field (Table 1): {TABLE1_N_STAR} lenses, {n_rays:.0e} rays, {nx}x{ny} map",
                    lf, 0.0, 0.0, TABLE1_KAPPA_STAR, (0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (y1 - y0), "strip"),
                    (0.0, 0.0, 40.0, 200.0), (nx, ny), n_av=n_rays / (nx * ny),
                    n_tracks=n_tracks, macro=("fold", TABLE1_KAPPA0, dx, dy))


def batched_maps(n_maps: int = 80, seed: int = 0, map_px: int = 4096,
                 ray_range=(1e9, 1e10), tracks_per_map: int = 10):
    """Heterogeneous maps: N ~ U{2000..20000}, kappa_* in {0.002, 0.005, 0.01},
    kappa + gamma ~ U[0.95, 0.99] with gamma = 0.5, rays log-uniform."""
    u = uniform01(seed, 21, 4 * n_maps).reshape(n_maps, 4)
    out = []
    for i in range(n_maps):
        n = 2000 + int(u[i, 0] * 18001)
        ks = (0.002, 0.005, 0.01)[min(2, int(u[i, 1] * 3))]
        s = 0.95 + 0.04 * u[i, 2]
        kappa, gamma = s - 0.5, 0.5
        rays = math.exp(math.log(ray_range[0]) + u[i, 3] * math.log(ray_range[1] / ray_range[0]))
        r = math.sqrt(n * lognormal_mean(0.3, 0.5) / ks)
        lf = lens_disc(n, r, seed * 1000 + 100 + i, "lognormal", 0.3, 0.5)
        a, b = 1.0 - kappa - gamma, 1.0 - kappa + gamma
        lp = r / (0.75 * math.hypot(1.0 / a, 1.0 / b))
        h = 0.5 * (lp - 20.0 * math.sqrt(ks))
        out.append(Workload(f"batched map {i}", lf, kappa, gamma, ks, (0.0, 0.0, r),
                            (-h, -h, h, h), (map_px, map_px),
                            n_av=rays / (map_px * map_px), n_tracks=tracks_per_map))
    return out
