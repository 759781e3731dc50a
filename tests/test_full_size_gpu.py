"""Full-size workloads, in the launch configuration the benchmark times, against the FP64 oracle
on a seeded sample of pixels (every injected pixel and random others).

The oracle searches each sampled pixel on its own, which is exact for that pixel whatever the cube
size, so the whole cube runs through the GPU path and only the sample through the oracle.  The
candidate lists are also checked for what holds at any size: pixel order, every S/N above the
threshold, and agreement with the per-pixel records.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_18136_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _sample(cfg, inj_pix, n_random, seed):
    rng = np.random.default_rng(seed)
    extra = rng.choice(cfg.n_pix, size=n_random, replace=False)
    return np.unique(np.concatenate([np.asarray(inj_pix, np.int64), extra]))


def _check_records_and_candidates(cfg, cand, snr, idx, best, pix):
    parity.compare_best(snr[pix], idx[pix], best)
    parity.compare_candidates(cand, best, cfg.threshold, pix, cfg.nx)
    # the whole list: pixel order, S/N above the threshold, the same pixels as the records
    g_pix = cand["row"].astype(np.int64) * cfg.nx + cand["col"]
    assert np.all(np.diff(g_pix) > 0)
    assert np.all(cand["snr"] > cfg.threshold)
    np.testing.assert_array_equal(np.sort(g_pix), np.nonzero(snr > cfg.threshold)[0])
    np.testing.assert_array_equal(cand["snr"], snr[g_pix])


def _full_window_cube(cfg, seed):
    """The benchmark's recipe: PSF-convolved noise and 50 injected bursts."""
    cube = synth.psf_noise(cfg, seed, device="cuda")
    raw = synth.draw_injections(cfg, 50, seed + 1000, max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    return cube, inj


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_window_301_sampled(native, dtype):
    """301 x 301 px x 16 sub x 1200 samples, 64 DM 0-2000, 12 widths (the benchmark workload)."""
    cfg = synth.config_full_window()
    cube, inj = _full_window_cube(cfg, 0)
    if dtype == "bf16":
        cube = cube.to(torch.bfloat16)
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0, device="cuda")
    with native.Plan(cfg, dtype=dtype) as plan:
        plan.search(cube, sigma)
        cand = plan.candidates()
        snr, idx = plan.best()
    pix = _sample(cfg, inj.row * cfg.nx + inj.col, 64, 1)
    x = cube[torch.from_numpy(pix).cuda()].float().cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    _, best, _ = oracle.search_cube(x, tab, cfg.widths, sigma=synth.psf_sigma() * 4.0)
    _check_records_and_candidates(cfg, cand, snr, idx, best, pix)
    # the bright injections are found at their pixels
    assert np.mean(snr[inj.row * cfg.nx + inj.col] > cfg.threshold) > 0.6


def test_stress_512_bf16_mad_sampled(native):
    """512 x 512 px BF16, 256 DM 0-4000, beam-scaled Student-t noise, MAD normalisation,
    500 injected bursts."""
    cfg = synth.config_stress()
    cube = synth.beam_student_noise(cfg, 5, device="cuda", dtype=torch.float32)
    raw = synth.draw_injections(cfg, 500, 6, dm_range=(0.0, 4000.0), max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    cube = cube.to(torch.bfloat16)
    with native.Plan(cfg, dtype="bf16", noise="mad") as plan:
        plan.search(cube)
        cand = plan.candidates()
        snr, idx = plan.best()
    pix = _sample(cfg, (inj.row * cfg.nx + inj.col)[:120], 48, 2)
    x = cube[torch.from_numpy(pix).cuda()].float().cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    _, best, bad = oracle.search_cube(x, tab, cfg.widths, mad=True)
    assert bad == 0
    _check_records_and_candidates(cfg, cand, snr, idx, best, pix)


def test_serving_301_field_sampled(native):
    """One 301 x 301 field of the serving workload (BF16 window of 1200 samples, 25-sample blocks):
    after each block the streamed candidates of the sampled pixels equal the oracle's search of
    the window restricted to the trials that end in the newest block."""
    cfg = synth.config_full_window()
    n_blk, n_blocks = 25, 3
    n_total = n_blk * n_blocks
    long_cfg = synth.SearchConfig(ny=cfg.ny, nx=cfg.nx, n_t=n_total, freq_mhz=cfg.freq_mhz, dm=cfg.dm,
                                  widths=cfg.widths)
    series = synth.plain_noise(long_cfg, 8, device="cuda")
    raw = synth.draw_injections(long_cfg, 40, 9, dm_range=(0.0, 2000.0), snr_range=(8.0, 20.0), max_width=16)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, n_total, cfg.n_sub, 1.0)
    synth.add_injections(series, long_cfg, inj, sh)
    series = series.to(torch.bfloat16).float()          # the window holds BF16 values
    pix = _sample(cfg, inj.row * cfg.nx + inj.col, 48, 3)
    xs = series[torch.from_numpy(pix).cuda()].cpu().numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    smax = tab.max(axis=1)
    t_lo = np.array([[cfg.n_t - n_blk - int(w) + 1 - int(s) for w in cfg.widths] for s in smax], np.int32)
    with native.Plan(cfg, dtype="bf16") as plan:
        plan.stream_open(n_blk)
        found = 0
        for b in range(n_blocks):
            blk = series[:, :, b * n_blk:(b + 1) * n_blk].permute(2, 1, 0).reshape(n_blk, cfg.n_sub, cfg.ny, cfg.nx)
            plan.stream_push(blk.contiguous().cpu().pin_memory())
            cand, _ = plan.stream_poll(timeout_ms=30000)
            end = (b + 1) * n_blk
            window = np.zeros((pix.size, cfg.n_sub, cfg.n_t), np.float32)
            window[:, :, cfg.n_t - end:] = xs[:, :, :end]
            _, best, _ = oracle.search_cube(window, tab, cfg.widths, sigma=4.0, t_lo=t_lo)
            parity.compare_candidates(cand, best, cfg.threshold, pix, cfg.nx)
            found += int(np.isin(cand["row"].astype(np.int64) * cfg.nx + cand["col"], pix).sum())
        assert found > 0
