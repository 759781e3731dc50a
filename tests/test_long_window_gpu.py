"""Windows longer than the register path (1248..4096 samples): the long-window kernel against the
FP64 oracle, element by element, in every mode the search offers (needs a GPU).

The boundary takes windows of 1..4096 samples; windows up to 1247 samples run the register-chunked
kernels tested in test_search_gpu.py, longer ones the long-window kernel (cube read in place,
sample-interleaved lanes, prefix and boxcars from shared memory)."""
import ctypes
import math

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


TDT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def _cfg(n_t, ny=3, nx=5, n_dm=23, dm_hi=3000.0, seed=0, widths=None, threshold=4.5):
    rng = np.random.default_rng(seed + n_t)
    if widths is None:
        widths = sorted({1, 2, 3, 4, 8, 16, 32, 100, 256, 512, 1024, 2048, n_t - 200, n_t} & set(range(1, n_t + 1)))
    return synth.SearchConfig(ny=ny, nx=nx, n_t=n_t, dm=np.sort(rng.uniform(0, dm_hi, n_dm)),
                              widths=np.array(widths[:16], np.int32), threshold=threshold)


def _cube(cfg, seed, n_inj=4):
    cube = synth.psf_noise(cfg, seed)
    raw = synth.draw_injections(cfg, n_inj, seed + 100, dm_range=(0.0, float(cfg.dm[-1])), max_width=cfg.n_t,
                                min_sep=1)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    return cube


def _check_full(native, cfg, cube, sigma, dtype="f32", noise="known"):
    plan = native.Plan(cfg, dtype=dtype, noise=noise, out="full")
    sg = None if sigma is None else torch.as_tensor(sigma, dtype=torch.float32).cuda()
    plan.search(cube.cuda(), sg)
    cand = plan.candidates()
    snr, idx = plan.best()
    f_snr, f_t = plan.full()
    plan.close()
    x = cube.float().numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    res, best, bad = oracle.search_cube(x, tab, cfg.widths, sigma=sigma, mad=(noise == "mad"))
    assert bad == 0
    xs = oracle.mad_normalise(x)[0] if noise == "mad" else x
    sgo = math.sqrt(cfg.n_sub) if (sigma is None or noise == "mad") else sigma
    parity.compare_full(f_snr, f_t, res, x=xs, sigma=sgo, shifts=tab, widths=cfg.widths)
    parity.compare_best(snr, idx, best)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
    return cand, best


@pytest.mark.parametrize("n_t", [1248, 2000, 3333, 4096])
def test_long_window_full_fp32(native, n_t):
    """Every (pixel, DM, width) S/N and TOA of FP32 windows just past the register path up to the
    longest window, widths from 1 sample to the whole window, DMs up to 3000."""
    cfg = _cfg(n_t)
    cube = _cube(cfg, n_t)
    sig = np.random.default_rng(n_t).uniform(4.0, 8.0, cfg.n_pix).astype(np.float32)
    cand, best = _check_full(native, cfg, cube, sig)
    assert len(cand) > 0


def test_long_window_rows_without_trials(native):
    """DM rows whose largest shift reaches the window end have no trials (-inf, -1), and the
    whole-window width only has trials on rows without dispersion delay."""
    cfg = synth.SearchConfig(ny=2, nx=3, n_t=1300, dm=np.array([0.0, 500.0, 200000.0, 400000.0]),
                             widths=np.array([1, 64, 1299, 1300], np.int32))
    cube = _cube(cfg, 3, n_inj=2)
    plan = native.Plan(cfg, out="full")
    plan.search(cube.cuda())
    f_snr, f_t = plan.full()
    plan.close()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    assert tab[3].max() >= cfg.n_t
    assert np.all(f_snr[:, 3] == -np.inf) and np.all(f_t[:, 3] == -1)
    assert np.all(np.isfinite(f_snr[:, 0, 3])) and np.all(f_snr[:, 1, 3] == -np.inf)
    _check_full(native, cfg, cube, None)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_long_window_16bit(native, dtype):
    """16-bit storage: FP32 sums of the widened values against the oracle on the stored values."""
    cfg = _cfg(2500, ny=4, nx=4, seed=5)
    cube = _cube(cfg, 6).to(TDT[dtype])
    sig = np.full(cfg.n_pix, synth.psf_sigma() * 4.0, np.float32)
    _check_full(native, cfg, cube, sig, dtype=dtype)


@pytest.mark.parametrize("out", ["candidates", "full"])
def test_long_window_mad(native, out):
    """MAD normalisation (the normalisation pass into FP32 slabs, then the long-window kernel) in
    both output modes, beam-scaled Student-t noise; a zero-MAD pixel is reported and flagged."""
    cfg = synth.config_stress(4, 5, n_t=3000)
    cfg.widths = np.array([1, 2, 8, 64, 512, 2048, 3000], np.int32)
    cube = synth.beam_student_noise(cfg, 9, dtype=torch.float32)
    raw = synth.draw_injections(cfg, 3, 10, dm_range=(0.0, 4000.0), max_width=cfg.n_t, min_sep=1)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    cube = cube.to(torch.bfloat16)
    if out == "full":
        _check_full(native, cfg, cube, None, dtype="bf16", noise="mad")
    bad = cube.clone()
    bad[7, 2, :] = 0.75
    plan = native.Plan(cfg, dtype="bf16", noise="mad", out=out)
    plan.search(bad.cuda())
    with pytest.raises(native.NsfrbError) as e:
        plan.candidates()
    assert e.value.status == native.EINVAL
    snr, idx = plan.best()
    assert snr[7] == -np.inf and (idx[7] == -1).all()
    plan.search(cube.cuda())
    cand = plan.candidates()
    snr, idx = plan.best()
    plan.close()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    res, best, nbad = oracle.search_cube(cube.float().numpy(), tab, cfg.widths, mad=True)
    assert nbad == 0
    parity.compare_best(snr, idx, best)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)


def test_long_window_host_path_and_rescore(native):
    """The host-buffer search equals the device search; BF16 storage re-scored from the FP32 cube
    gives the FP32 results on the pixels near the threshold."""
    cfg = _cfg(2048, ny=5, nx=6, seed=11, threshold=5.0)
    cube = _cube(cfg, 12, n_inj=6)
    sig = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0)
    plan = native.Plan(cfg)
    plan.search(cube.cuda(), sig.cuda())
    a = plan.candidates()
    s32, i32 = plan.best()
    plan.search_host(cube.pin_memory(), sig)
    b = plan.candidates()
    s_b, i_b = plan.best()
    plan.close()
    np.testing.assert_array_equal(s32, s_b)
    np.testing.assert_array_equal(i32, i_b)
    assert a.tobytes() == b.tobytes()
    eps = 1.0
    p16 = native.Plan(cfg, dtype="bf16", rescore_eps=eps)
    p16.search(cube.to(torch.bfloat16).cuda(), sig.cuda())
    s16, _ = p16.best()
    p16.search(cube.to(torch.bfloat16).cuda(), sig.cuda(), cube.cuda())
    sr, ir = p16.best()
    p16.close()
    near = np.abs(s16 - cfg.threshold) <= eps
    assert near.any()
    np.testing.assert_array_equal(sr[near], s32[near])
    np.testing.assert_array_equal(ir[near], i32[near])


def _window_oracle(cfg, window, n_blk, tab):
    smax = tab.max(axis=1)
    t_lo = np.array([[cfg.n_t - n_blk - int(w) + 1 - int(s) for w in cfg.widths] for s in smax], np.int32)
    res, best, _ = oracle.search_cube(window, tab, cfg.widths, sigma=4.0, t_lo=t_lo)
    return best


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_long_window_serving(native, dtype):
    """Serving a 1600-sample window in 25-sample blocks: after each block the streamed candidates
    equal the oracle's search of the window restricted to trials ending in the newest block."""
    cfg = synth.SearchConfig(ny=3, nx=4, n_t=1600, dm=np.linspace(0, 2000, 12),
                             widths=np.array([1, 2, 4, 16, 64, 256, 1024, 1600], np.int32), threshold=5.0)
    n_blk, n_blocks = 25, 70
    n_total = n_blk * n_blocks
    long_cfg = synth.SearchConfig(ny=cfg.ny, nx=cfg.nx, n_t=n_total, freq_mhz=cfg.freq_mhz, dm=cfg.dm,
                                  widths=cfg.widths)
    x = synth.plain_noise(long_cfg, 21)
    raw = synth.draw_injections(long_cfg, 4, 22, dm_range=(0.0, 2000.0), snr_range=(8.0, 20.0), max_width=64,
                                min_sep=1)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, n_total, cfg.n_sub, 1.0)
    synth.add_injections(x, long_cfg, inj, sh)
    if dtype == "bf16":
        x = x.to(torch.bfloat16).to(torch.float32)
    xn = x.numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    plan = native.Plan(cfg, dtype=dtype)
    plan.stream_open(n_blk)
    total = 0
    for b in range(n_blocks):
        blk = torch.from_numpy(xn[:, :, b * n_blk:(b + 1) * n_blk].transpose(2, 1, 0).copy())
        plan.stream_push(blk.reshape(n_blk, cfg.n_sub, cfg.ny, cfg.nx).contiguous())
        cand, _ = plan.stream_poll(timeout_ms=10000)
        if b % 7 != 6 and b != n_blocks - 1:
            continue       # the oracle checks every 7th block and the last
        end = (b + 1) * n_blk
        window = np.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t), np.float32)
        lo = max(0, end - cfg.n_t)
        window[:, :, cfg.n_t - (end - lo):] = xn[:, :, lo:end]
        best = _window_oracle(cfg, window, n_blk, tab)
        parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
        total += len(cand)
    plan.close()
    assert total > 0


def test_long_window_static_search(native):
    """The search without device allocation runs long windows too (known noise), with the results
    of nsfrb_search; MAD normalisation of long windows needs nsfrb_search's workspace (EINVAL)."""
    cfg = _cfg(1800, ny=4, nx=5, seed=31)
    cube = _cube(cfg, 32).cuda()
    sig = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0, device="cuda")
    plan = native.Plan(cfg)
    plan.search(cube, sig)
    ref = plan.candidates()
    cap = cfg.n_pix
    out = torch.zeros((cap, 6), dtype=torch.int32, device="cuda")
    n = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    for _ in range(2):
        st = native.lib.nsfrb_search_static(plan.handle, ctypes.c_void_p(cube.data_ptr()),
                                            ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(out.data_ptr()), cap,
                                            ctypes.c_void_p(n.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == native.OK, native.lib.nsfrb_last_error()
        torch.cuda.synchronize()
        total = int(n.item())
        assert total == len(ref)
        rows = out[:total].cpu().numpy()
        for i, name in enumerate(["row", "col", "dm_idx", "w_idx", "t_idx"]):
            np.testing.assert_array_equal(rows[:, i], ref[name])
        np.testing.assert_array_equal(rows[:, 5].view(np.float32), ref["snr"])
    plan.close()
    pm = native.Plan(cfg, noise="mad")
    st = native.lib.nsfrb_search_static(pm.handle, ctypes.c_void_p(cube.data_ptr()), None,
                                        ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(n.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == native.EINVAL
    pm.close()


@pytest.mark.parametrize("n_sub", [5, 24])
def test_long_window_subband_counts(native, n_sub):
    """Subband counts other than 16 (first rows read past the first 16 subbands; few subbands)."""
    rng = np.random.default_rng(n_sub)
    n_t = 1500
    cfg = synth.SearchConfig(ny=3, nx=4, n_sub=n_sub, n_t=n_t, freq_mhz=synth.band_centres(n_sub),
                             dm=np.sort(rng.uniform(0, 4000, 17)),
                             widths=np.array([1, 2, 5, 16, 64, 300, 1024, 1500], np.int32), threshold=4.0)
    cube = torch.from_numpy(rng.standard_normal((cfg.n_pix, n_sub, n_t)).astype(np.float32))
    cube[5, :, 700:740] += 1.0
    sig = np.full(cfg.n_pix, math.sqrt(n_sub), np.float32)
    _check_full(native, cfg, cube, sig)
