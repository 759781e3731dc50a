"""Pins of the imager oracle (Sec. 2.1) against closed forms, brute force and limits."""
import math

import numpy as np
import pytest

from oracle import imager as oi
from paper_2510_18136_gb300 import synth_vis as sv

N = 175
PIX = 10.3


def _one_baseline_uv(ku, kv, f_mhz, n=N, pix=PIX):
    """(u, v) metres that land exactly on cell (ku, kv) at f_mhz."""
    scale = f_mhz * 1.0e6 / oi.C_LIGHT * n * oi.pixel_radians(pix)
    return np.array([[ku / scale, kv / scale]])


@pytest.mark.parametrize("ku,kv,robust", [(3, -5, -2.0), (7, 2, 0.5), (0, 4, -2.0)])
def test_single_baseline_fringe_closed_form(ku, kv, robust):
    """One visibility V = 1 and its mirror: a cosine fringe of amplitude 2w/N^2 with the
    phase origin at pixel N//2 + 1 (ifftshift before and after the transform)."""
    f = 1400.0
    uv = _one_baseline_uv(ku, kv, f)
    vis = np.ones((1, 1, 1, 1, 2), np.complex128) * 0.5          # two polarisations sum to 1
    img = oi.image(vis, uv, [[f]], N, PIX, robust=robust, b_min=0.0, b_max=1e9)[0, 0]
    # Briggs: both cells hold weight 1 (distinct cells unless ku = kv = 0) -> sum W^2 / sum w = 1
    w = 1.0 / (1.0 + (5.0 * 10.0 ** (-robust)) ** 2)
    h = N // 2
    y, x = np.mgrid[0:N, 0:N]
    expect = 2.0 * w / N**2 * np.cos(2.0 * math.pi * (ku * (x + h) + kv * (y + h)) / N)
    np.testing.assert_allclose(img, expect, rtol=0, atol=1e-12 * w)


def test_brute_force_dft_small_grid():
    """Random baselines on a 9x9 grid: the image equals the direct double sum
    (1/N^2) sum_{k} G_k exp(+2 pi i (ku (x + N//2) + kv (y + N//2)) / N), real part."""
    n = 9
    rng = np.random.default_rng(3)
    f = 1350.0
    scale = f * 1.0e6 / oi.C_LIGHT * n * oi.pixel_radians(PIX)
    ks = rng.integers(-4, 5, size=(12, 2))
    uv = ks / scale + rng.uniform(-0.2, 0.2, size=ks.shape) / scale
    vis = (rng.normal(size=(1, 1, 1, 12, 2)) + 1j * rng.normal(size=(1, 1, 1, 12, 2)))
    img = oi.image(vis, uv, [[f]], n, PIX, robust=-2.0, b_min=0.0, b_max=1e9)[0, 0]
    w = oi.channel_weights(uv, f, n, PIX, -2.0, 0.0, 1e9)
    ku = np.rint(uv[:, 0] * scale).astype(int)
    kv = np.rint(uv[:, 1] * scale).astype(int)
    V = vis[0, 0, 0, :, 0] + vis[0, 0, 0, :, 1]
    h = n // 2
    ref = np.zeros((n, n))
    for y in range(n):
        for x in range(n):
            acc = 0j
            for i in range(12):
                for sgn in (1, -1):
                    val = V[i] if sgn == 1 else np.conj(V[i])
                    acc += w[i] * val * np.exp(2j * math.pi * sgn * (ku[i] * (x + h) + kv[i] * (y + h)) / n)
            ref[y, x] = acc.real / n**2
    np.testing.assert_allclose(img, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_hermitian_grid_gives_real_image():
    ant = sv.core_layout(1)
    uv = sv.baseline_uv(ant)
    ch = sv.channel_freqs(2, 2)
    rng = np.random.default_rng(0)
    w = oi.channel_weights(uv, ch[0, 0], N, PIX, -2.0, 20.0, 485.0)
    v = rng.normal(size=len(uv)) + 1j * rng.normal(size=len(uv))
    G = oi.grid_channel(v, uv, ch[0, 0], w, N, PIX)
    re, im = oi.image_of_grid(G, keep_imag=True)
    assert np.abs(im).max() < 1e-12 * np.abs(re).max()


def test_point_source_at_phase_centre():
    """V = S on every baseline: the peak is at (N//2 + 1, N//2 + 1) and equals
    sum over channels of 2 S sum_i w_i / N^2."""
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    ch = sv.channel_freqs(1, 3)
    S = 2.5
    vis = np.full((1, 1, 3, len(uv), 2), S / 2.0, np.complex128)
    img = oi.image(vis, uv, ch, N, PIX)[0, 0]
    wt = oi.weights(uv, ch, N, PIX)
    assert np.unravel_index(np.argmax(img), img.shape) == (N // 2 + 1, N // 2 + 1)
    assert img[N // 2 + 1, N // 2 + 1] == pytest.approx(2.0 * S * wt.sum() / N**2, rel=1e-12)


def test_offset_source_lands_on_its_pixel():
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    ch = sv.channel_freqs(1, 8)
    vis = sv.visibilities(uv, ch, 1, [(5, -3, 4.0)], pixel_arcsec=PIX, noise=0.0).numpy()
    img = oi.image(vis, uv, ch, N, PIX)[0, 0]
    c = N // 2 + 1
    assert np.unravel_index(np.argmax(img), img.shape) == (c - 3, c + 5)


def test_briggs_limits():
    """R -> +inf: natural weights (all 1).  R -> -inf: uniform weighting, every occupied
    cell carries the same total weight 1/f^2."""
    ant = sv.core_layout(2)
    uv = sv.baseline_uv(ant)
    f = 1400.0
    wn = oi.channel_weights(uv, f, N, PIX, 8.0, 20.0, 485.0)
    kept = oi.baseline_kept(uv, 20.0, 485.0)
    np.testing.assert_allclose(wn[kept], 1.0, rtol=0, atol=1e-9)
    assert np.all(wn[~kept] == 0)
    wu = oi.channel_weights(uv, f, N, PIX, -8.0, 20.0, 485.0)
    ku, kv = oi.cells(uv, f, N, PIX)
    tot = {}
    for i in np.nonzero(kept)[0]:
        for key in ((ku[i], kv[i]), (-ku[i], -kv[i])):
            tot[key] = tot.get(key, 0.0) + wu[i]
    vals = np.array(list(tot.values()))
    np.testing.assert_allclose(vals, vals[0], rtol=1e-6)


def test_baseline_selection_and_grid_edge():
    """Strict b_min < |b| < b_max; cells beyond (N-1)//2 are dropped with their mirror."""
    f = 1400.0
    n = 11
    scale = f * 1.0e6 / oi.C_LIGHT * n * oi.pixel_radians(PIX)
    uv = np.array([[5.0 / scale, 0.0], [6.0 / scale, 0.0], [0.0, 3.0 / scale]])
    w = oi.channel_weights(uv, f, n, PIX, 0.0, 0.0, 1e9)
    assert w[0] > 0 and w[1] == 0 and w[2] > 0
    b = np.hypot(uv[:, 0], uv[:, 1])
    w2 = oi.channel_weights(uv, f, n, PIX, 0.0, b[2], 1e9)      # |b| == b_min is dropped
    assert w2[2] == 0 and w2[0] > 0


def test_paper_geometry_support():
    """At the paper's grid (175 px of 10.3 arcsec) and b_max = 485 m the occupied uv
    cells lie within |k| <= 21 even at the top channel: far inside the grid."""
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    ch = sv.channel_freqs()
    ku, kv = oi.cells(uv, ch.max(), N, PIX)
    kept = oi.baseline_kept(uv, 20.0, 485.0)
    assert np.abs(ku[kept]).max() <= 21 and np.abs(kv[kept]).max() <= 21
    # 485 m at the top channel, in cells of 1/(N dtheta) wavelengths
    assert 485.0 * ch.max() * 1e6 / oi.C_LIGHT * N * oi.pixel_radians(PIX) < 21.5
