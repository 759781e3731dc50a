"""Seeded synthetic inputs for the search (stand-ins for DSA-110 dirty-image cubes).

This module holds the input recipes only -- noise fields, beam profiles,
injection parameters and the placement of injected pulses -- and none of the
search arithmetic.  Dispersion delays of injected pulses are *inputs* here:
callers pass each injection's integer per-subband shifts, computed by
whichever side builds the inputs.  Both the CUDA path and the oracle read the
cubes built here.

Recipes (cube layout is pixel-major [ny*nx, n_sub, n_t], pixel (r, c) = r*nx + c):

* plain:    i.i.d. N(0, 1) per pixel, subband and sample.
* psf:      per (subband, sample) image, N(0, 1) convolved (circularly) with a
            peak-normalised 5x5 Gaussian PSF of FWHM 2 px; per-pixel noise
            sigma_pix = ||PSF||_2 (about 1.508).
* beam:     per-pixel sigma(r) = 4**((r/r_e)**2), clamped at 4, r_e = half
            side; Student-t (nu = 5) noise scaled to unit variance.
* injections: boxcar pulses of width w starting at t0 + s_k in subband k,
            amplitude A per subband (PSF-shaped around the pixel for psf noise).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

FWHM_PX = 2.0


def band_centres(n_sub: int = 16, lo_mhz: float = 1311.0, hi_mhz: float = 1498.0) -> np.ndarray:
    """Subband centres when lo/hi are the band edges: lo + (k + 1/2) * (hi - lo)/n_sub."""
    bw = (hi_mhz - lo_mhz) / n_sub
    return lo_mhz + (np.arange(n_sub, dtype=np.float64) + 0.5) * bw


def pow2_widths(max_w: int = 1024, extra=(1200,)) -> np.ndarray:
    w = [1 << i for i in range(int(math.log2(max_w)) + 1)]
    return np.array(w + list(extra), dtype=np.int32)


@dataclass
class SearchConfig:
    """Plain description of one search configuration (all sizes explicit)."""
    ny: int
    nx: int
    n_sub: int = 16
    n_t: int = 1200
    t_samp_ms: float = 134.2
    k_dm_ms: float = 4.149
    freq_mhz: np.ndarray = field(default_factory=band_centres)
    dm: np.ndarray = field(default_factory=lambda: np.linspace(0.0, 2000.0, 64))
    widths: np.ndarray = field(default_factory=pow2_widths)
    threshold: float = 6.0

    @property
    def n_pix(self) -> int:
        return self.ny * self.nx

    @property
    def n_trials(self) -> int:
        return self.n_pix * len(self.dm) * len(self.widths)


def config_small(ny=64, nx=64) -> SearchConfig:
    """64x64 px, 16 subbands 1311-1498 MHz, 25 samples of 134.2 ms, 16 DM 0-2000, widths 1..16."""
    return SearchConfig(ny=ny, nx=nx, n_t=25, dm=np.linspace(0.0, 2000.0, 16),
                        widths=np.array([1, 2, 4, 8, 16], dtype=np.int32))


def config_full_window(ny=301, nx=301, n_t=1200) -> SearchConfig:
    """301x301 px, 1200 samples, 64 DM 0-2000, widths 1..1024 (powers of 2) + 1200."""
    return SearchConfig(ny=ny, nx=nx, n_t=n_t, dm=np.linspace(0.0, 2000.0, 64),
                        widths=pow2_widths())


def config_stress(ny=512, nx=512, n_t=1200) -> SearchConfig:
    """512x512 px, 1200 samples, 256 DM 0-4000, widths as the full-window config."""
    return SearchConfig(ny=ny, nx=nx, n_t=n_t, dm=np.linspace(0.0, 4000.0, 256),
                        widths=pow2_widths())


# ----------------------------------------------------------------------------- noise

def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian_psf(size: int = 5, fwhm_px: float = FWHM_PX) -> np.ndarray:
    """Peak-normalised (centre tap = 1) 2-D Gaussian PSF."""
    sg = fwhm_px / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    r = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-0.5 * (r / sg) ** 2)
    return np.outer(g, g)


def psf_sigma(psf: np.ndarray | None = None) -> float:
    """Noise of unit white noise after convolution with the PSF (its L2 norm)."""
    psf = gaussian_psf() if psf is None else psf
    return float(np.sqrt((psf ** 2).sum()))


def plain_noise(cfg: SearchConfig, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """i.i.d. N(0,1) cube [n_pix, n_sub, n_t]."""
    g = _gen(seed, device)
    return torch.randn((cfg.n_pix, cfg.n_sub, cfg.n_t), generator=g, device=device,
                       dtype=torch.float32).to(dtype)


def psf_noise(cfg: SearchConfig, seed: int, device="cpu", dtype=torch.float32,
              t_chunk: int = 200) -> torch.Tensor:
    """Per-image N(0,1) convolved circularly with the 5x5 PSF; cube [n_pix, n_sub, n_t]."""
    g = _gen(seed, device)
    psf = torch.tensor(gaussian_psf(), dtype=torch.float32, device=device)[None, None]
    half = psf.shape[-1] // 2
    out = torch.empty((cfg.n_pix, cfg.n_sub, cfg.n_t), dtype=dtype, device=device)
    for k in range(cfg.n_sub):
        for t0 in range(0, cfg.n_t, t_chunk):
            nt = min(t_chunk, cfg.n_t - t0)
            img = torch.randn((nt, 1, cfg.ny, cfg.nx), generator=g, device=device,
                              dtype=torch.float32)
            img = torch.nn.functional.pad(img, (half, half, half, half), mode="circular")
            img = torch.nn.functional.conv2d(img, psf)          # [nt, 1, ny, nx]
            out[:, k, t0:t0 + nt] = img.reshape(nt, cfg.n_pix).T.to(dtype)
    return out


def beam_sigma(cfg: SearchConfig) -> np.ndarray:
    """Per-pixel sigma(r) = 4**((r/r_e)**2), clamped at 4; r_e = half of the smaller side."""
    r_e = min(cfg.ny, cfg.nx) / 2.0
    yy, xx = np.meshgrid(np.arange(cfg.ny) - (cfg.ny - 1) / 2.0,
                         np.arange(cfg.nx) - (cfg.nx - 1) / 2.0, indexing="ij")
    r = np.sqrt(yy ** 2 + xx ** 2).reshape(-1)
    return np.minimum(4.0 ** ((r / r_e) ** 2), 4.0)


def beam_student_noise(cfg: SearchConfig, seed: int, nu: float = 5.0, device="cpu",
                       dtype=torch.bfloat16, pix_chunk: int = 16384) -> torch.Tensor:
    """Student-t (nu) noise of unit variance times the per-pixel beam sigma."""
    g = _gen(seed, device)
    sig = torch.tensor(beam_sigma(cfg), dtype=torch.float32, device=device)
    out = torch.empty((cfg.n_pix, cfg.n_sub, cfg.n_t), dtype=dtype, device=device)
    unit = math.sqrt(nu / (nu - 2.0))
    for p0 in range(0, cfg.n_pix, pix_chunk):
        n = min(pix_chunk, cfg.n_pix - p0)
        z = torch.randn((n, cfg.n_sub, cfg.n_t), generator=g, device=device)
        # chi-square with nu dof as a sum of nu squared normals (nu integer here)
        chi = torch.zeros_like(z)
        for _ in range(int(nu)):
            chi += torch.randn((n, cfg.n_sub, cfg.n_t), generator=g, device=device) ** 2
        t = z / torch.sqrt(chi / nu) / unit
        out[p0:p0 + n] = (t * sig[p0:p0 + n, None, None]).to(dtype)
    return out


# ----------------------------------------------------------------------------- injections

@dataclass
class Injections:
    """Truth table of injected pulses (one row per pulse)."""
    row: np.ndarray
    col: np.ndarray
    dm: np.ndarray
    width: np.ndarray
    snr: np.ndarray
    t0: np.ndarray
    amp: np.ndarray

    def __len__(self):
        return int(self.row.size)


def draw_injections(cfg: SearchConfig, n: int, seed: int, dm_range=(0.0, 2000.0),
                    snr_range=(6.0, 30.0), min_sep: int = 3, max_width: int = 1200,
                    edge: int = 0) -> dict:
    """Draw DM ~ U, width ~ log-U(1, max_width) rounded, S/N ~ U and pixels >= min_sep apart.

    Returns raw parameters; ``place_injections`` finishes them once the caller has
    the per-injection shifts.
    """
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    tries = 0
    while len(rows) < n and tries < 100000:
        tries += 1
        r = int(rng.integers(edge, cfg.ny - edge))
        c = int(rng.integers(edge, cfg.nx - edge))
        if all(max(abs(r - r2), abs(c - c2)) >= min_sep for r2, c2 in zip(rows, cols)):
            rows.append(r)
            cols.append(c)
    dm = rng.uniform(dm_range[0], dm_range[1], size=n)
    width = np.rint(np.exp(rng.uniform(0.0, math.log(max_width), size=n))).astype(np.int64)
    snr = rng.uniform(snr_range[0], snr_range[1], size=n)
    u = rng.uniform(0.0, 1.0, size=n)
    return {"row": np.array(rows), "col": np.array(cols), "dm": dm,
            "width": np.maximum(width, 1), "snr": snr, "u": u}


def place_injections(raw: dict, shifts: np.ndarray, n_t: int, n_sub: int,
                     sigma_pix) -> Injections:
    """Clamp widths to the window left by the largest shift and draw t0 uniformly.

    shifts: [n_inj, n_sub] integer shifts of each injection's own DM.
    sigma_pix: noise per pixel/subband/sample (scalar or per-injection array);
    the matched-filter amplitude is A = S/N * sigma_pix / (sqrt(n_sub) sqrt(w)).
    """
    shifts = np.asarray(shifts)
    smax = shifts.max(axis=1)
    w = np.minimum(raw["width"], np.maximum(n_t - smax, 1))
    span = np.maximum(n_t - smax - w + 1, 1)
    t0 = np.floor(raw["u"] * span).astype(np.int64)
    sp = np.broadcast_to(np.asarray(sigma_pix, dtype=np.float64), w.shape)
    amp = raw["snr"] * sp / (math.sqrt(n_sub) * np.sqrt(w))
    return Injections(row=raw["row"], col=raw["col"], dm=raw["dm"], width=w,
                      snr=raw["snr"], t0=t0, amp=amp)


def add_injections(cube: torch.Tensor, cfg: SearchConfig, inj: Injections,
                   shifts: np.ndarray, psf: np.ndarray | None = None) -> None:
    """Add each pulse in place: +A (times the PSF around the pixel, circular) on
    samples [t0 + s_k, t0 + s_k + w) of subband k, clipped to the window."""
    taps = [(0, 0, 1.0)]
    if psf is not None:
        h = psf.shape[0] // 2
        taps = [(dy - h, dx - h, float(psf[dy, dx])) for dy in range(psf.shape[0])
                for dx in range(psf.shape[1])]
    for i in range(len(inj)):
        for dy, dx, wgt in taps:
            r = (int(inj.row[i]) + dy) % cfg.ny
            c = (int(inj.col[i]) + dx) % cfg.nx
            p = r * cfg.nx + c
            for k in range(cfg.n_sub):
                a = int(inj.t0[i]) + int(shifts[i][k])
                b = min(a + int(inj.width[i]), cfg.n_t)
                if a < cfg.n_t:
                    cube[p, k, a:b] += float(inj.amp[i] * wgt)


def add_pulse(cube: torch.Tensor, cfg: SearchConfig, row: int, col: int, t0: int, width: int,
              amp: float, shifts) -> None:
    """Single boxcar pulse at one pixel (no PSF)."""
    p = row * cfg.nx + col
    for k in range(cfg.n_sub):
        a = t0 + int(shifts[k])
        b = min(a + width, cfg.n_t)
        if a < cfg.n_t:
            cube[p, k, a:b] += amp
