"""Seeded synthetic visibilities for the imager (stand-ins for DSA-110 core data).

Input recipes only, none of the imaging arithmetic:

* core_layout: 82 antennas in a T, 48 on an east-west arm over +-230 m and 34 on
  a north-south arm from 12 m to 400 m, each position jittered by N(0, 0.3 m)
  (the real DSA-110 core positions are not available here).
* baseline_uv: every antenna pair i < j, (u, v) = (dE, dN cos(dec - lat)) metres:
  the baseline seen from a source on the meridian at declination dec (71.6 deg,
  the survey declination) from latitude lat (37.23 deg), w neglected.
* channel_freqs: n_sub subbands of equal width over [lo, hi] MHz, each split
  into n_chan equal channels; the centre of each channel.
* visibilities: point sources at pixel offsets (dx, dy) from the phase centre
  (l = dx * pixel, m = dy * pixel), V = sum_src flux / 2 * exp(-2 pi i (u l + v m) f / c)
  in each of two polarisations, plus complex Gaussian noise (sigma per real
  component).  flux is per (sample, subband): a dispersed pulse is a flux that
  is nonzero on subband-dependent samples.  Layout [n_t][n_sub][n_chan][n_base][2]
  complex64.
"""
from __future__ import annotations

import math

import numpy as np
import torch

C_LIGHT = 299792458.0


def core_layout(seed: int = 0, n_ew: int = 48, n_ns: int = 34) -> np.ndarray:
    rng = np.random.default_rng(seed)
    ew = np.stack([np.linspace(-230.0, 230.0, n_ew), np.zeros(n_ew)], axis=1)
    ns = np.stack([np.zeros(n_ns), np.linspace(12.0, 400.0, n_ns)], axis=1)
    ant = np.concatenate([ew, ns])
    return ant + rng.normal(0.0, 0.3, ant.shape)


def baseline_uv(ant: np.ndarray, dec_deg: float = 71.6, lat_deg: float = 37.23) -> np.ndarray:
    i, j = np.triu_indices(len(ant), k=1)
    d = ant[j] - ant[i]
    return np.stack([d[:, 0], d[:, 1] * math.cos(math.radians(dec_deg - lat_deg))], axis=1)


def channel_freqs(n_sub: int = 16, n_chan: int = 8, lo_mhz: float = 1311.0, hi_mhz: float = 1498.0) -> np.ndarray:
    bw = (hi_mhz - lo_mhz) / n_sub
    return lo_mhz + bw * np.arange(n_sub)[:, None] + bw / n_chan * (np.arange(n_chan)[None, :] + 0.5)


def visibilities(uv_m: np.ndarray, chan_mhz: np.ndarray, n_t: int, sources=(), pixel_arcsec: float = 10.3,
                 noise: float = 1.0, seed: int = 0, device="cpu") -> torch.Tensor:
    """complex64 tensor [n_t][n_sub][n_chan][n_base][2]; sources: iterable of (dx, dy, flux[n_t][n_sub])."""
    chan = torch.as_tensor(np.asarray(chan_mhz, float), dtype=torch.float64, device=device)
    uv = torch.as_tensor(np.asarray(uv_m, float), dtype=torch.float64, device=device)
    n_sub, n_chan = chan.shape
    n_base = uv.shape[0]
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = (n_t, n_sub, n_chan, n_base, 2, 2)
    v = torch.randn(shape, generator=g, device=device, dtype=torch.float32) * noise
    vis = torch.view_as_complex(v)
    pix = pixel_arcsec * math.pi / 648000.0
    for dx, dy, flux in sources:
        flux = torch.as_tensor(np.broadcast_to(np.asarray(flux, float), (n_t, n_sub)).copy(), dtype=torch.float64,
                               device=device)
        l, m = dx * pix, dy * pix
        # phase per (subband, channel, baseline)
        ph = -2.0 * math.pi * (uv[None, None, :, 0] * l + uv[None, None, :, 1] * m) * (chan[:, :, None] * 1.0e6 / C_LIGHT)
        e = torch.polar(torch.ones_like(ph), ph)                          # [n_sub][n_chan][n_base]
        add = (flux[:, :, None, None] / 2.0) * e[None]                      # [n_t][n_sub][n_chan][n_base]
        vis += add.to(torch.complex64)[..., None]
    return vis
