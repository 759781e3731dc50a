"""Plain statement of the NSFRB imager (Sec. 2.1), test infrastructure only.

Per subband and 134 ms sample, each of the subband's channels is imaged on its
own and the channel images are summed:

* baselines are kept when b_min < |b| < b_max, |b| the length of the baseline's
  (u, v) in metres (the core is taken as coplanar: no w term);
* the two polarisations are summed into one visibility per (channel, baseline)
  with natural weight 1;
* a visibility falls in the uv-grid cell k = rint(u f / c * N * dtheta) (u in
  metres, f in Hz, dtheta the image pixel in radians, N the grid side; cell
  size 1 / (N dtheta) wavelengths), and its complex conjugate in the cell -k;
  cells with |k| > (N - 1) // 2 on either axis are outside the grid and
  dropped together with their mirror;
* Briggs weighting with robustness R: W_cell = sum of natural weights in the
  cell (mirrors included), f^2 = (5 * 10^-R)^2 / (sum_cells W^2 / sum w), and
  each visibility (and its mirror) is weighted 1 / (1 + W_cell f^2); R = -2 is
  close to uniform weighting;
* the weighted visibilities are accumulated on the grid (zero frequency at
  index N // 2), and the image is ifftshift(ifft2(ifftshift(grid))).real, the
  inverse FFT with numpy's 1 / N^2 normalisation and the shift applied before
  and after as the paper states; no further normalisation.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0   # m/s


def pixel_radians(pixel_arcsec: float) -> float:
    return pixel_arcsec * math.pi / 648000.0


def baseline_kept(uv_m: np.ndarray, b_min: float, b_max: float) -> np.ndarray:
    """b_min < |b| < b_max on the (u, v) length in metres."""
    b = np.sqrt(uv_m[:, 0] * uv_m[:, 0] + uv_m[:, 1] * uv_m[:, 1])
    return (b > b_min) & (b < b_max)


def cells(uv_m: np.ndarray, freq_mhz: float, n_grid: int, pixel_arcsec: float):
    """Integer cell (ku, kv) of each baseline at one channel frequency.

    The product is evaluated left to right in FP64: u * f_MHz * 1e6 / c * N * dtheta,
    then rounded to nearest (ties to even)."""
    dth = pixel_radians(pixel_arcsec)
    ku = np.rint(uv_m[:, 0] * freq_mhz * 1.0e6 / C_LIGHT * n_grid * dth).astype(np.int64)
    kv = np.rint(uv_m[:, 1] * freq_mhz * 1.0e6 / C_LIGHT * n_grid * dth).astype(np.int64)
    return ku, kv


def channel_weights(uv_m, freq_mhz, n_grid, pixel_arcsec, robust, b_min, b_max) -> np.ndarray:
    """Briggs weight of every baseline at one channel (0 for dropped baselines)."""
    ku, kv = cells(uv_m, freq_mhz, n_grid, pixel_arcsec)
    h = (n_grid - 1) // 2
    ok = baseline_kept(uv_m, b_min, b_max) & (np.abs(ku) <= h) & (np.abs(kv) <= h)
    c = n_grid // 2
    W = np.zeros((n_grid, n_grid))
    for i in np.nonzero(ok)[0]:
        W[c + kv[i], c + ku[i]] += 1.0
        W[c - kv[i], c - ku[i]] += 1.0
    sum_w = 2.0 * ok.sum()
    w = np.zeros(len(uv_m))
    if sum_w == 0:
        return w
    f2 = (5.0 * 10.0 ** (-robust)) ** 2 / (np.sum(W * W) / sum_w)
    for i in np.nonzero(ok)[0]:
        w[i] = 1.0 / (1.0 + W[c + kv[i], c + ku[i]] * f2)
    return w


def weights(uv_m, chan_mhz, n_grid, pixel_arcsec, robust=-2.0, b_min=20.0, b_max=485.0) -> np.ndarray:
    """[n_sub][n_chan][n_base] Briggs weights."""
    chan_mhz = np.asarray(chan_mhz, float)
    out = np.zeros(chan_mhz.shape + (len(uv_m),))
    for s in range(chan_mhz.shape[0]):
        for ch in range(chan_mhz.shape[1]):
            out[s, ch] = channel_weights(uv_m, chan_mhz[s, ch], n_grid, pixel_arcsec, robust, b_min, b_max)
    return out


def grid_channel(vis: np.ndarray, uv_m, freq_mhz, w, n_grid, pixel_arcsec) -> np.ndarray:
    """Full complex uv-grid of one channel; vis[n_base] (polarisations already summed)."""
    ku, kv = cells(uv_m, freq_mhz, n_grid, pixel_arcsec)
    c = n_grid // 2
    G = np.zeros((n_grid, n_grid), np.complex128)
    for i in np.nonzero(w)[0]:
        G[c + kv[i], c + ku[i]] += w[i] * vis[i]
        G[c - kv[i], c - ku[i]] += w[i] * np.conj(vis[i])
    return G


def image_of_grid(G: np.ndarray, keep_imag: bool = False):
    """ifftshift -> 2-D inverse FFT -> ifftshift, as the paper's imager does."""
    z = np.fft.ifftshift(np.fft.ifft2(np.fft.ifftshift(G)))
    return (z.real, z.imag) if keep_imag else z.real


def image(vis: np.ndarray, uv_m, chan_mhz, n_grid: int, pixel_arcsec: float, robust: float = -2.0,
          b_min: float = 20.0, b_max: float = 485.0) -> np.ndarray:
    """Dirty images [n_t][n_sub][N][N] (float64) from vis[n_t][n_sub][n_chan][n_base][2 pol] (complex)."""
    vis = np.asarray(vis)
    uv_m = np.asarray(uv_m, float)
    chan_mhz = np.asarray(chan_mhz, float)
    n_t, n_sub, n_chan = vis.shape[:3]
    wt = weights(uv_m, chan_mhz, n_grid, pixel_arcsec, robust, b_min, b_max)
    out = np.zeros((n_t, n_sub, n_grid, n_grid))
    for t in range(n_t):
        for s in range(n_sub):
            for ch in range(n_chan):
                v = vis[t, s, ch, :, 0].astype(np.complex128) + vis[t, s, ch, :, 1].astype(np.complex128)
                out[t, s] += image_of_grid(grid_channel(v, uv_m, chan_mhz[s, ch], wt[s, ch], n_grid, pixel_arcsec))
    return out
