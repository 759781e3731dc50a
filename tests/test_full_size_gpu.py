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


# ----------------------------------------------------------------------------- BF16 storage error and re-score

def _bf16_vs_fp32(native, cfg, cube32, sigma, noise, sample_pix):
    """The stored-BF16 search against the FP32 search of the same cube (whole cube) and against the
    FP64 oracle of the FP32 input (sampled pixels); then the re-scored BF16 search, whose candidate
    set must equal the FP32 one.  Returns the measured maxima."""
    kw = {} if noise == "known" else {"noise": "mad"}
    with native.Plan(cfg, **kw) as p:
        p.search(cube32, sigma)
        c32 = p.candidates()
        s32, i32 = p.best()
    cube16 = cube32.to(torch.bfloat16)
    with native.Plan(cfg, dtype="bf16", **kw) as p:
        p.search(cube16, sigma)
        s16, _ = p.best()
    fin = np.isfinite(s32)
    assert (np.isfinite(s16) == fin).all()
    err = np.abs(s16[fin].astype(np.float64) - s32[fin])
    # the FP32 search is within the FP32 tolerance of the FP64 oracle
    bound = parity.bf16_bound(s32[fin], noise) - parity.tol(s32[fin])
    assert (err <= bound).all(), f"worst {np.max(err / bound):.3f} x bound"
    eps = float(parity.bf16_bound(cfg.threshold, noise))
    with native.Plan(cfg, dtype="bf16", rescore_eps=eps, **kw) as p:
        p.search(cube16, sigma, cube_f32=cube32)
        cr = p.candidates()
        sr, ir = p.best()
    # the library's selection, in its FP32 arithmetic: thr - eps <= S/N <= thr + eps
    thr32, eps32 = np.float32(cfg.threshold), np.float32(eps)
    near = (s16 >= thr32 - eps32) & (s16 <= thr32 + eps32)
    # re-scored pixels carry the FP32 search's result (the re-score may group the DM rows over the
    # warps differently from the whole-cube search, which changes the FP32 summation order only)
    assert (np.abs(sr[near].astype(np.float64) - s32[near]) <= parity.tol(s32[near])).all()
    np.testing.assert_array_equal(sr[~near], s16[~near])
    g_r = cr["row"].astype(np.int64) * cfg.nx + cr["col"]
    g_32 = c32["row"].astype(np.int64) * cfg.nx + c32["col"]
    band32 = np.abs(s32.astype(np.float64) - cfg.threshold) <= parity.tol(s32)
    assert set(g_r.tolist()) - set(np.nonzero(band32)[0].tolist()) == \
        set(g_32.tolist()) - set(np.nonzero(band32)[0].tolist())
    # against the FP64 oracle of the FP32 input: sampled pixels and every re-scored pixel
    pix = np.unique(np.concatenate([sample_pix, np.nonzero(near)[0][:256]]))
    x = cube32[torch.from_numpy(pix).cuda()].cpu().numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    if noise == "known":
        _, best, _ = oracle.search_cube(x, tab, cfg.widths, sigma=float(sigma[0].item()))
    else:
        _, best, bad = oracle.search_cube(x, tab, cfg.widths, mad=True)
        assert bad == 0
    o = best["snr"]
    e16 = np.abs(s16[pix].astype(np.float64) - o)
    assert (e16 <= parity.bf16_bound(o, noise)).all()
    # after re-score the sampled candidates are the oracle's (outside the FP32 tolerance band)
    o_set = set(int(p) for p, s in zip(pix, o) if s > cfg.threshold + parity.tol(s))
    band = set(int(p) for p, s in zip(pix, o) if abs(s - cfg.threshold) <= parity.tol(s))
    assert (set(int(p) for p in g_r) & set(int(p) for p in pix)) - band == o_set - band
    return {"max_abs": float(err.max()), "rel_max": float(np.max(err / np.maximum(1.0, np.abs(s32[fin])))),
            "rescored": int(near.sum()), "oracle_max_abs": float(e16.max()), "candidates": int(len(c32))}


def test_bf16_error_bound_and_rescore_full_window(native):
    """301 x 301 full window: BF16 storage within 0.03 in S/N of the FP32 input's FP64 search; after
    re-scoring the pixels within 0.03 of the threshold, the candidate set is the FP32 one."""
    cfg = synth.config_full_window()
    cube, inj = _full_window_cube(cfg, 0)
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0, device="cuda")
    pix = _sample(cfg, inj.row * cfg.nx + inj.col, 64, 5)
    r = _bf16_vs_fp32(native, cfg, cube, sigma, "known", pix)
    print("full window BF16:", r)


def test_bf16_error_bound_and_rescore_stress_mad(native):
    """512 x 512, 256 DM, beam-scaled Student-t noise, MAD normalisation: BF16 within
    0.03 + 2^-7 |S/N| of the FP32 input's FP64 search; re-scored candidate set = FP32 set."""
    cfg = synth.config_stress()
    cube = synth.beam_student_noise(cfg, 5, device="cuda", dtype=torch.float32)
    raw = synth.draw_injections(cfg, 500, 6, dm_range=(0.0, 4000.0), max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    pix = _sample(cfg, (inj.row * cfg.nx + inj.col)[:64], 32, 6)
    r = _bf16_vs_fp32(native, cfg, cube, None, "mad", pix)
    print("stress BF16 MAD:", r)
    del cube
    torch.cuda.empty_cache()


def test_serving_301_field_bf16_rescore(native):
    """One 301 x 301 serving field stored in BF16 with re-scoring from the pinned FP32 window: after
    every block its candidate set equals that of the same stream stored in FP32, and the sampled
    pixels' candidates equal the FP64 oracle's masked-window search of the FP32 values."""
    cfg = synth.config_full_window()
    n_blk, n_blocks = 25, 3
    n_total = n_blk * n_blocks
    long_cfg = synth.SearchConfig(ny=cfg.ny, nx=cfg.nx, n_t=n_total, freq_mhz=cfg.freq_mhz, dm=cfg.dm,
                                  widths=cfg.widths)
    series = synth.plain_noise(long_cfg, 18, device="cuda")
    raw = synth.draw_injections(long_cfg, 40, 19, dm_range=(0.0, 2000.0), snr_range=(5.0, 9.0), max_width=16)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, n_total, cfg.n_sub, 1.0)
    synth.add_injections(series, long_cfg, inj, sh)
    pix = _sample(cfg, inj.row * cfg.nx + inj.col, 48, 7)
    xs = series[torch.from_numpy(pix).cuda()].cpu().numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    smax = tab.max(axis=1)
    t_lo = np.array([[cfg.n_t - n_blk - int(w) + 1 - int(s) for w in cfg.widths] for s in smax], np.int32)
    eps = float(parity.bf16_bound(cfg.threshold, "known"))
    p16 = native.Plan(cfg, dtype="bf16", rescore_eps=eps)
    p32 = native.Plan(cfg)
    p16.stream_open(n_blk)
    p32.stream_open(n_blk)
    try:
        for b in range(n_blocks):
            blk = series[:, :, b * n_blk:(b + 1) * n_blk].permute(2, 1, 0).reshape(n_blk, cfg.n_sub, cfg.ny, cfg.nx)
            host = blk.contiguous().cpu().pin_memory()
            p16.stream_push(host)
            p32.stream_push(host)
            c16, _ = p16.stream_poll(timeout_ms=30000)
            c32, _ = p32.stream_poll(timeout_ms=30000)
            np.testing.assert_array_equal(c16["row"] * cfg.nx + c16["col"], c32["row"] * cfg.nx + c32["col"])
            end = (b + 1) * n_blk
            window = np.zeros((pix.size, cfg.n_sub, cfg.n_t), np.float32)
            window[:, :, cfg.n_t - end:] = xs[:, :, :end]
            _, best, _ = oracle.search_cube(window, tab, cfg.widths, sigma=4.0, t_lo=t_lo)
            o_set = set(int(p) for p, s in zip(pix, best["snr"]) if s > cfg.threshold + parity.tol(s))
            band = set(int(p) for p, s in zip(pix, best["snr"]) if abs(s - cfg.threshold) <= parity.tol(s))
            g = set(int(p) for p in c16["row"].astype(np.int64) * cfg.nx + c16["col"]) & set(int(p) for p in pix)
            assert g - band == o_set - band
    finally:
        p16.close()
        p32.close()
