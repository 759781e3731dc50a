"""GPU imager (Sec. 2.1) vs the FP64 imager oracle, and imager -> serving search.

Tolerance.  Each pixel is inv_n2 (A_0 + 2 sum_u Re(A_u t_u)), A_u = sum_v G t,
G = sum of weighted visibilities; every quantity is a sum of at most
n = m + n_chan + 2V + 2U + 8 FP32 roundings (m the most entries in one half-plane
cell over all channels, n_chan for adding the channels' partial grids, plus the
weight, twiddle and 1/N^2 roundings), so
|gpu - oracle| <= gamma_n * 2 * sum_i w_i |V_i| / N^2 with gamma_n = n u / (1 - n u),
u = 2^-24 (summed over the subband's channels).  That worst case is loose, so the
rms error is also held to 1e-5 of the image rms: one dropped visibility moves
the rms by about 1 / sqrt(number of visibilities) ~ 5e-3 of it.
"""
import math

import numpy as np
import pytest
import torch

from oracle import imager as oi
from paper_2510_18136_gb300 import synth, synth_vis as sv

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _max_cell_entries(uv, chan_row, n, pix, b_min, b_max):
    keys = []
    for f in chan_row:
        w = oi.channel_weights(uv, f, n, pix, -2.0, b_min, b_max)
        ku, kv = oi.cells(uv, f, n, pix)
        for i in np.nonzero(w)[0]:
            if ku[i] > 0:
                keys.append((ku[i], kv[i]))
            elif ku[i] < 0:
                keys.append((-ku[i], -kv[i]))
            else:
                keys += [(0, kv[i]), (0, -kv[i])]
    if not keys:
        return 0
    _, cnt = np.unique(np.array(keys), axis=0, return_counts=True)
    return int(cnt.max())


def _compare(native, uv, chan, n, pix, vis_c, t_s=None, b_min=20.0, b_max=485.0, robust=-2.0):
    """GPU images of vis_c (complex64 [n_t][n_sub][n_chan][n_base][2]) vs the oracle, for the
    (t, s) pairs t_s (all if None)."""
    im = native.Imager(uv, chan, n_grid=n, pixel_arcsec=pix, robust=robust, b_min_m=b_min, b_max_m=b_max)
    gpu = im.image(vis_c.cuda()).cpu().numpy()
    im.status()
    U, V, _ = im.info()
    wt = oi.weights(uv, chan, n, pix, robust, b_min, b_max)
    # weights: same FP64 expressions on both sides, rounded to FP32 by the library
    np.testing.assert_array_equal(im.weights(), wt.astype(np.float32))
    vis = vis_c.numpy()
    n_t, n_sub = vis.shape[:2]
    pairs = t_s if t_s is not None else [(t, s) for t in range(n_t) for s in range(n_sub)]
    worst = 0.0
    for t, s in pairs:
        ref = oi.image(vis[t:t + 1, s:s + 1], uv, chan[s:s + 1], n, pix, robust, b_min, b_max)[0, 0]
        m = _max_cell_entries(uv, chan[s], n, pix, b_min, b_max)
        nr = m + chan.shape[1] + 2 * V + 2 * U + 8
        gam = nr * U32 / (1 - nr * U32)
        vsum = np.abs(vis[t, s, :, :, 0].astype(np.complex128) + vis[t, s, :, :, 1])
        tol = gam * 2.0 * float((wt[s] * vsum).sum()) / n**2
        err = np.abs(gpu[t, s] - ref)
        assert err.max() <= tol, (t, s, err.max(), tol)
        rms_ref = math.sqrt(float((ref**2).mean()))
        rel = math.sqrt(float((err**2).mean())) / rms_ref
        assert rel <= 1e-5, (t, s, rel)
        worst = max(worst, rel)
    im.close()
    return worst


def test_weights_and_images_small(native):
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs(2, 3)
    vis = sv.visibilities(uv, chan, 2, [(5, -3, 3.0), (-20, 11, 1.0)], noise=1.0, seed=4)
    _compare(native, uv, chan, 175, 10.3, vis)


@pytest.mark.parametrize("n,pix", [(64, 10.3), (33, 25.0), (9, 120.0)])
def test_other_grid_sizes_and_edges(native, n, pix):
    """Even and small odd grids; at 120" pixels on a 9-cell grid most baselines fall
    outside the grid and are dropped with their mirror."""
    ant = sv.core_layout(5)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs(3, 2)
    vis = sv.visibilities(uv, chan, 1, [(2, 1, 2.0)], pixel_arcsec=pix, noise=0.5, seed=6)
    _compare(native, uv, chan, n, pix, vis)


def test_zero_spacing_and_u0_column(native):
    """Baselines on the ku = 0 column (and one at the origin cell) enter the grid twice."""
    n, pix, f = 21, 60.0, 1400.0
    scale = f * 1.0e6 / oi.C_LIGHT * n * oi.pixel_radians(pix)
    uv = np.array([[0.0, 3.0], [0.0, -5.0], [0.1, 0.0], [4.0, 2.0], [-6.0, 1.0]]) / scale
    chan = np.array([[f]])
    rng = np.random.default_rng(0)
    v = (rng.normal(size=(1, 1, 1, 5, 2)) + 1j * rng.normal(size=(1, 1, 1, 5, 2))).astype(np.complex64)
    _compare(native, uv, chan, n, pix, torch.from_numpy(v), b_min=0.0, b_max=1e9)


def test_paper_block_sampled(native):
    """The paper's block: 25 samples x 16 subbands x 8 channels, 82-antenna core, 175 px,
    10.3", R = -2; the oracle checks a sample of the 400 images."""
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs()
    vis = sv.visibilities(uv, chan, 25, [(10, 4, 5.0)], noise=1.0, seed=9)
    pairs = [(0, 0), (7, 5), (13, 11), (24, 15)]
    _compare(native, uv, chan, 175, 10.3, vis, t_s=pairs)


def test_deterministic(native):
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs(4, 8)
    vis = sv.visibilities(uv, chan, 3, noise=1.0, seed=1, device="cuda")
    with native.Imager(uv, chan) as im:
        a = im.image(vis)
        b = im.image(vis)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_bad_arguments(native):
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs(1, 2)
    with pytest.raises(native.NsfrbError):
        native.Imager(uv, chan, n_grid=2)
    with pytest.raises(native.NsfrbError):
        native.Imager(uv, chan, b_min_m=500.0, b_max_m=485.0)
    with pytest.raises(native.NsfrbError):
        native.Imager(uv, -chan)
    with native.Imager(uv, chan) as im:
        vis = torch.zeros((0, 1, 2, len(uv), 2, 2), device="cuda")
        assert im.image(vis).shape == (0, 1, 175, 175)
        raw = torch.zeros(2 * 2 * len(uv) * 4 + 1, device="cuda")
        mis = raw[1:1 + 8 * len(uv)].view(1, 1, 2, len(uv), 2, 2)                 # 4-byte offset: not 16-byte aligned
        with pytest.raises(native.NsfrbError):
            native._check(native.lib.nsfrb_image(im._h, native._ptr(mis), 1, native._ptr(raw), None), "x")


def test_imager_feeds_serving_search(native):
    """A dispersed pulse from a point source: visibilities -> GPU images written into the
    stream's device block -> masked serving search.  The strongest candidate is the
    source's pixel with the injected DM trial and width."""
    n, pix = 64, 10.3
    cfg = synth.SearchConfig(ny=n, nx=n, n_t=100, dm=np.linspace(0, 2000, 16),
                             widths=np.array([1, 2, 4, 8, 16], np.int32), threshold=6.0)
    ant = sv.core_layout(0)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs(cfg.n_sub, 2)
    plan = native.Plan(cfg)
    plan.stream_open(25)
    sh = plan.delays()
    d_true, w_true, t0, amp = 9, 4, 30, 1.0
    dx, dy = 7, -5
    n_blocks = 4
    flux = np.zeros((25 * n_blocks, cfg.n_sub))
    for s in range(cfg.n_sub):
        flux[t0 + sh[d_true, s]: t0 + sh[d_true, s] + w_true, s] = amp
    with native.Imager(uv, chan, n_grid=n, pixel_arcsec=pix) as im:
        w = im.weights().astype(np.float64)
        # visibility noise giving unit image noise per subband: var = 8 sigma^2 sum w^2 / N^4
        sig = n**2 / math.sqrt(8.0 * float((w**2).sum(axis=(1, 2)).mean()))
        # source flux giving a peak of 3 noise units per subband image: peak = 2 F sum w / N^2
        f_src = 3.0 * n**2 / (2.0 * float(w.sum(axis=(1, 2)).mean()))
        best = None
        for b in range(n_blocks):
            vis = sv.visibilities(uv, chan, 25, [(dx, dy, flux[25 * b: 25 * (b + 1)] * f_src)],
                                  pixel_arcsec=pix, noise=sig, seed=100 + b, device="cuda")
            blk = plan.stream_block()
            im.image(vis, out=blk)
            plan.stream_push_device()
            cands, _ = plan.stream_poll(timeout_ms=20000)
            if len(cands):
                top = cands[np.argmax(cands["snr"])]
                if best is None or top["snr"] > best["snr"]:
                    best = top
    plan.close()
    c = n - n // 2          # phase centre after the two ifftshifts (N//2 + 1 for odd N, N/2 for even N)
    assert best is not None
    assert (int(best["row"]), int(best["col"])) == (c + dy, c + dx)
    assert abs(int(best["dm_idx"]) - d_true) <= 1 and int(cfg.widths[best["w_idx"]]) == w_true
    assert best["snr"] > 10.0
