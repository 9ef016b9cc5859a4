"""Differentiable cloud-in-cell magnification map and light curves.

CICMagnification.apply(x, y, m, kappa, gamma, kappa_star, spec) returns the
float32 magnification map M = (S_I / S_S) * CIC ray weights of a lens field
(Eq. 6 lens equation, Eq. 12 scaling), and its backward calls the library's
hand-written adjoint (ml_cic_backward): gradients for every lens position and
mass and for kappa, gamma and kappa_*.  Deflections are recomputed in the
backward, not stored.  Forward (ml_cic_forward) and backward run in the CUDA
library; this module only marshals tensors.
"""
from __future__ import annotations

import torch

import numpy as np

from . import (DEPOSIT_CIC, PREC_MIXED, Field, make_desc, ml_cic_backward, ml_cic_forward,
               ml_map_light_curves, ml_map_light_curves_backward)
from .inputs import LensField, Workload


def _desc(x, y, m, kappa, gamma, kappa_star, spec):
    """Descriptor of the field.  Lens tensors on the current CUDA device are
    passed to the library as device pointers (no copy to the host); others
    as host arrays."""
    w = Workload("differentiable", LensField(None, None, None), float(kappa), float(gamma),
                 float(kappa_star), spec["sheet"], spec["map_box"], spec["map_n"],
                 ray_box=spec.get("ray_box"), ray_n=spec.get("ray_n"), n_av=spec.get("n_av", 0.0))
    dev = torch.device("cuda", torch.cuda.current_device())
    on_dev = all(t.device == dev for t in (x, y, m))
    if on_dev:
        lens = [t.detach().to(torch.float64).contiguous() for t in (x, y, m)]
        host = [np.zeros(0)] * 3
    else:
        host = [t.detach().cpu().numpy() for t in (x, y, m)]
    d = make_desc(w, precision=PREC_MIXED, deposit=DEPOSIT_CIC, taylor_p=spec.get("taylor_p", 0),
                  l1=spec.get("l1"), l2_sub=spec.get("l2_sub", (0, 0)), lens_arrays=host)
    if on_dev:
        d.lens_x, d.lens_y, d.lens_m = (t.data_ptr() for t in lens)
        d.n_lens = lens[0].numel()
        d.lens_mem_is_device = 1
        d._keep = lens           # alive until the field is created
    return d


class CICMagnification(torch.autograd.Function):
    """M(x, y, m, kappa, gamma, kappa_*) with a hand-written adjoint.

    spec: dict of the fixed geometry: sheet (cx, cy, R), map_box, map_n, and
    either ray_box + ray_n or n_av; optionally taylor_p, l1, l2_sub.  Fixing
    ray_box, l1 and taylor_p keeps the lattice and the level grids independent
    of the differentiated inputs (otherwise they move with kappa and gamma).
    """

    @staticmethod
    def forward(ctx, x, y, m, kappa, gamma, kappa_star, spec):
        d = _desc(x, y, m, kappa, gamma, kappa_star, spec)
        f = Field(desc=d)
        mu = torch.empty((f.info["map_ny"], f.info["map_nx"]), dtype=torch.float32, device="cuda")
        ml_cic_forward(f.h, mu)
        ctx.field = f
        ctx.n = x.numel()
        ctx.devices = (x.device, kappa.device if torch.is_tensor(kappa) else None)
        return mu

    @staticmethod
    def backward(ctx, grad_mu):
        f = ctx.field
        glens = torch.zeros((ctx.n, 3), dtype=torch.float64, device="cuda")
        gpar = torch.zeros(3, dtype=torch.float64, device="cuda")
        ml_cic_backward(f.h, grad_mu.detach().contiguous().float(), glens, gpar)
        f.close()
        dev_lens, dev_par = ctx.devices
        gl = glens.to(dev_lens)
        gp = gpar.to(dev_par) if dev_par is not None else gpar
        return gl[:, 0], gl[:, 1], gl[:, 2], gp[0], gp[1], gp[2], None


class LightCurves(torch.autograd.Function):
    """Gaussian-source light curves of a map (ml_map_light_curves), with the
    transpose (ml_map_light_curves_backward) as backward.  Composes with
    CICMagnification for a light-curve loss:
        mu = CICMagnification.apply(x, y, m, kappa, gamma, kappa_star, spec)
        curves = LightCurves.apply(mu, tracks, n_samples, sigma_px)
    tracks: n x (x0, y0, x1, y1) in map pixel coordinates (host array)."""

    @staticmethod
    def forward(ctx, mu, tracks, n_samples, sigma_px):
        tr = np.ascontiguousarray(tracks, np.float64).reshape(-1, 4)
        mu = mu.detach().contiguous().float()
        out = torch.empty((len(tr), n_samples), dtype=torch.float32, device=mu.device)
        ml_map_light_curves(mu, tr, n_samples, sigma_px, out)
        ctx.args = (tr, n_samples, sigma_px, tuple(mu.shape))
        return out

    @staticmethod
    def backward(ctx, grad_curves):
        tr, n_samples, sigma_px, shape = ctx.args
        g = torch.empty(shape, dtype=torch.float32, device=grad_curves.device)
        ml_map_light_curves_backward(grad_curves.detach().contiguous().float(), tr, n_samples,
                                     sigma_px, g)
        return g, None, None, None
