"""CUDA search vs the FP64 oracle, element by element (needs a GPU)."""
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


def _run(native, cfg, cube, sigma=None, dtype="f32", noise="known", out="full", cube_f32=None, eps=0.0):
    plan = native.Plan(cfg, dtype=dtype, noise=noise, out=out, rescore_eps=eps)
    dev = cube.cuda()
    sg = None if sigma is None else torch.as_tensor(sigma, dtype=torch.float32).cuda().contiguous()
    plan.search(dev, sg, None if cube_f32 is None else cube_f32.cuda())
    cand = plan.candidates()
    snr, idx = plan.best()
    full = plan.full() if out == "full" else None
    plan.close()
    return cand, snr, idx, full


def _oracle(cfg, cube_f32_np, sigma=None, mad=False, pix=None):
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    res, best, bad = oracle.search_cube(cube_f32_np, tab, cfg.widths, sigma=sigma, pix=pix, mad=mad)
    return tab, res, best, bad


def _check_all(native, cfg, cube, sigma=None, dtype="f32", noise="known", rel=parity.REL):
    cand, snr, idx, (f_snr, f_t) = _run(native, cfg, cube, sigma, dtype=dtype, noise=noise)
    x = cube.float().numpy()
    tab, res, best, bad = _oracle(cfg, x, sigma=sigma, mad=(noise == "mad"))
    assert bad == 0
    xs = oracle.mad_normalise(x)[0] if noise == "mad" else x
    sg = math.sqrt(cfg.n_sub) if (sigma is None or noise == "mad") else sigma
    st = parity.compare_full(f_snr, f_t, res, rel, x=xs, sigma=sg, shifts=tab, widths=cfg.widths)
    parity.compare_best(snr, idx, best, rel)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx, rel)
    return st, cand, best


# ----------------------------------------------------------------------------- closed forms

def test_small_cube_closed_form(native):
    """Noise-free 64x64x16x25 cube with the DM-500, width-2, amplitude-3 pulse at (20, 37)."""
    cfg = synth.config_small()
    inj = oracle.delay_table(cfg.freq_mhz, [500.0])[0]
    cube = torch.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t))
    synth.add_pulse(cube, cfg, 20, 37, 10, 2, 3.0, inj)
    cand, snr, idx, _ = _run(native, cfg, cube, sigma=np.full(cfg.n_pix, 4.0, np.float32), out="candidates")
    assert len(cand) == 1
    c = cand[0]
    assert (c["row"], c["col"], c["dm_idx"], c["w_idx"], c["t_idx"]) == (20, 37, 4, 1, 10)
    assert c["snr"] == pytest.approx(3 * 16 * 2 / (4 * math.sqrt(2)), rel=1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_small_cube_with_noise(native, seed):
    cfg = synth.config_small()
    inj = oracle.delay_table(cfg.freq_mhz, [500.0])[0]
    cube = synth.plain_noise(cfg, seed)
    synth.add_pulse(cube, cfg, 20, 37, 10, 2, 3.0, inj)
    st, cand, best = _check_all(native, cfg, cube, sigma=np.full(cfg.n_pix, 4.0, np.float32))
    p = 20 * cfg.nx + 37
    assert p in [int(r) * cfg.nx + int(c) for r, c in zip(cand["row"], cand["col"])]


# ----------------------------------------------------------------------------- full-window shapes

def _psf_cube(cfg, seed, n_inj, dm_range=(0.0, 2000.0), dtype=torch.float32):
    cube = synth.psf_noise(cfg, seed)
    raw = synth.draw_injections(cfg, n_inj, seed + 100, dm_range=dm_range, max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    return cube.to(dtype)


def test_full_window_fp32(native):
    """11x13 px, 1200 samples, 64 DM 0-2000, widths 1..1024 + 1200, PSF noise + injections."""
    cfg = synth.config_full_window(11, 13)
    cube = _psf_cube(cfg, 5, 6)
    sig = np.full(cfg.n_pix, synth.psf_sigma() * 4.0, np.float32)
    st, cand, best = _check_all(native, cfg, cube, sigma=sig)
    assert len(cand) >= 3


@pytest.mark.parametrize("n_t,widths", [
    (37, [1, 2, 3, 5, 8, 13, 21, 37]),
    (100, [1, 4, 16, 17, 31, 32, 64, 96, 100]),
    (333, [2, 7, 9, 24, 32, 33, 160, 320, 333]),
    (700, [1, 3, 5, 9, 16, 64, 100, 512, 640, 699]),
    # the sample-pair chunk (38 per lane): its shortest and longest windows
    (801, [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 800, 801]),
    (1215, [1, 2, 3, 4, 8, 16, 32, 48, 64, 96, 128, 256, 512, 1024, 1215]),
    (1247, [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 1216, 1247]),
    (1, [1]),
    (31, [1, 31]),
])
def test_random_shapes(native, n_t, widths):
    """Window lengths of every kernel chunk size, widths of every class, ragged pixel counts."""
    rng = np.random.default_rng(n_t)
    cfg = synth.SearchConfig(ny=3, nx=7, n_t=n_t, dm=np.sort(rng.uniform(0, 3000, 23)),
                             widths=np.array(widths, np.int32))
    cube = torch.from_numpy(rng.standard_normal((cfg.n_pix, cfg.n_sub, n_t)).astype(np.float32))
    sig = rng.uniform(2.0, 6.0, cfg.n_pix).astype(np.float32)
    _check_all(native, cfg, cube, sigma=sig)


def test_dm_beyond_window_has_no_trials(native):
    """DM rows whose largest shift reaches the window end have no trials (-inf, -1)."""
    cfg = synth.SearchConfig(ny=2, nx=2, n_t=40, dm=np.array([0.0, 1000.0, 9000.0, 20000.0]),
                             widths=np.array([1, 4, 30], np.int32))
    rng = np.random.default_rng(1)
    cube = torch.from_numpy(rng.standard_normal((cfg.n_pix, 16, 40)).astype(np.float32))
    _, _, _, (f_snr, f_t) = _run(native, cfg, cube)
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    assert tab[3].max() >= 40
    assert np.all(f_snr[:, 3] == -np.inf) and np.all(f_t[:, 3] == -1)
    _check_all(native, cfg, cube)


def test_single_pixel_and_threshold_edges(native):
    cfg = synth.SearchConfig(ny=1, nx=1, n_t=64, dm=np.array([0.0]), widths=np.array([1, 2], np.int32),
                             threshold=2.0)
    cube = torch.zeros((1, 16, 64))
    cube[0, :, 5] = 0.5   # S/N at w=1: 16*0.5/4 = 2.0 exactly -> not above a threshold of 2.0
    cand, snr, idx, _ = _run(native, cfg, cube, out="candidates")
    assert snr[0] == pytest.approx(2.0) and len(cand) == 0


# ----------------------------------------------------------------------------- reduced precision

@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_16bit_storage_parity(native, dtype):
    """16-bit storage: FP32 accumulation parity against the oracle on the rounded values."""
    cfg = synth.config_full_window(9, 10)
    cube = _psf_cube(cfg, 9, 5).to(torch.bfloat16 if dtype == "bf16" else torch.float16)
    sig = np.full(cfg.n_pix, synth.psf_sigma() * 4.0, np.float32)
    _check_all(native, cfg, cube, sigma=sig, dtype=dtype)


def test_bf16_error_bound_and_rescore(native):
    """BF16 vs FP32 input: S/N differences stay within the stated bound; re-scored
    pixels near the threshold carry the FP32 result exactly."""
    cfg = synth.config_full_window(12, 12)
    cfg.threshold = 5.0
    cube = _psf_cube(cfg, 21, 8)
    sig = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0)
    _, s32, i32, _ = _run(native, cfg, cube, sigma=sig, out="candidates")
    cb = cube.to(torch.bfloat16)
    _, s16, i16, _ = _run(native, cfg, cb, sigma=sig, dtype="bf16", out="candidates")
    assert np.max(np.abs(s16 - s32)) < 0.02
    eps = 1.0
    cand, sr, ir, _ = _run(native, cfg, cb, sigma=sig, dtype="bf16", out="candidates", cube_f32=cube, eps=eps)
    near = np.abs(s16 - cfg.threshold) <= eps
    assert near.any()
    np.testing.assert_array_equal(sr[near], s32[near])
    np.testing.assert_array_equal(ir[near], i32[near])
    np.testing.assert_array_equal(sr[~near], s16[~near])


# ----------------------------------------------------------------------------- robust noise

def test_mad_mode_parity(native):
    """Per-(pixel, subband) median/MAD normalisation on beam-scaled Student-t noise."""
    cfg = synth.config_stress(8, 9)
    cube = synth.beam_student_noise(cfg, 3, dtype=torch.float32)
    raw = synth.draw_injections(cfg, 4, 7, dm_range=(0.0, 4000.0))
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    _check_all(native, cfg, cube, noise="mad")
    _check_all(native, cfg, cube.to(torch.bfloat16), noise="mad", dtype="bf16")


def test_mad_zero_is_reported(native):
    cfg = synth.SearchConfig(ny=2, nx=2, n_t=50, dm=np.array([0.0, 100.0]), widths=np.array([1, 3], np.int32))
    cube = torch.randn((4, 16, 50))
    cube[2, 5] = 1.0    # constant row: MAD = 0
    plan = native.Plan(cfg, noise="mad")
    plan.search(cube.cuda())
    with pytest.raises(native.NsfrbError) as e:
        plan.candidates()
    assert e.value.status == native.EINVAL
    snr, idx = plan.best()
    assert snr[2] == -np.inf and np.isfinite(snr[[0, 1, 3]]).all()


@pytest.mark.parametrize("n_t", [48, 50])
def test_mad_zero_full_arrays(native, n_t):
    """FULL arrays with a zero-MAD pixel: that pixel has no trial at any (DM, width) (-inf, -1);
    every other pixel's entries equal the oracle's (windows of whole 16-byte units take the
    barrier-free kernel on the normalised slabs, others the staged kernel)."""
    cfg = synth.SearchConfig(ny=2, nx=3, n_t=n_t, dm=np.array([0.0, 100.0, 400.0, 30000.0]),
                             widths=np.array([1, 3, 8], np.int32))
    rng = np.random.default_rng(n_t)
    cube = torch.from_numpy(rng.standard_normal((cfg.n_pix, cfg.n_sub, n_t)).astype(np.float32))
    cube[2, 5] = 1.0    # constant row: MAD = 0
    plan = native.Plan(cfg, noise="mad", out="full")
    plan.search(cube.cuda())
    with pytest.raises(native.NsfrbError):
        plan.candidates()
    f_snr, f_t = plan.full()
    plan.close()
    assert np.all(f_snr[2] == -np.inf) and np.all(f_t[2] == -1)
    keep = np.array([0, 1, 3, 4, 5])
    tab, res, best, bad = _oracle(cfg, cube.numpy(), mad=True, pix=keep)
    assert bad == 0
    xs = oracle.mad_normalise(cube.numpy()[keep])[0]
    parity.compare_full(f_snr[keep], f_t[keep], res, x=xs, sigma=math.sqrt(cfg.n_sub), shifts=tab,
                        widths=cfg.widths)


# ----------------------------------------------------------------------------- host entry point

def test_search_host_matches_device(native):
    cfg = synth.config_full_window(10, 10)
    cube = _psf_cube(cfg, 2, 4)
    sig = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0)
    plan = native.Plan(cfg)
    plan.search(cube.cuda(), sig.cuda())
    a = plan.candidates()
    s_a, i_a = plan.best()
    plan.search_host(cube.pin_memory(), sig)
    b = plan.candidates()
    s_b, i_b = plan.best()
    np.testing.assert_array_equal(s_a, s_b)
    np.testing.assert_array_equal(i_a, i_b)
    assert a.tobytes() == b.tobytes()


def test_candidate_capacity_truncation(native):
    cfg = synth.SearchConfig(ny=4, nx=4, n_t=32, dm=np.array([0.0]), widths=np.array([1], np.int32),
                             threshold=-100.0)
    plan = native.Plan(cfg)
    plan.search(torch.randn((16, 16, 32)).cuda())
    with pytest.raises(native.NsfrbError) as e:
        plan.candidates(cap=5)
    assert e.value.status == native.ETRUNC


# ----------------------------------------------------------------------------- records mode (barrier-free kernel)

@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n_t", [801, 1000, 1001, 1200, 1215])
def test_records_mode_parity(native, dtype, n_t):
    """Per-pixel records and candidates without FULL arrays: the barrier-free kernel for FP32 rows
    and for 16-bit rows read in place (even chunks; window lengths that are not a multiple of the
    16-byte sample count take the staged kernel), against the FP64 oracle on the stored values."""
    rng = np.random.default_rng(n_t + len(dtype))
    widths = [1, 2, 3, 4, 8, 16, 32, 64, 96, 128, 256, 512, 800]
    cfg = synth.SearchConfig(ny=5, nx=9, n_t=n_t, dm=np.sort(rng.uniform(0, 2500, 37)),
                             widths=np.array(widths, np.int32), threshold=4.5)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    cube = _psf_cube(cfg, n_t, 5, dm_range=(0.0, 2500.0)).to(tdt)
    sig = rng.uniform(4.0, 8.0, cfg.n_pix).astype(np.float32)
    cand, snr, idx, _ = _run(native, cfg, cube, sig, dtype=dtype, out="candidates")
    tab, res, best, bad = _oracle(cfg, cube.float().numpy(), sigma=sig)
    parity.compare_best(snr, idx, best)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
    assert len(cand) > 0


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n_t", [840, 1200])
def test_records_mode_mad_parity(native, dtype, n_t):
    """MAD normalisation with per-pixel records: the normalisation pass into FP32 slabs and the
    barrier-free search of them, against the FP64 oracle's median / MAD normalisation of the stored
    values; a pixel with a constant subband row (zero MAD) is reported and gets no record."""
    cfg = synth.config_stress(6, 7, n_t=n_t)
    cfg.widths = np.array([w for w in cfg.widths if w <= n_t], np.int32)
    cube = synth.beam_student_noise(cfg, 17, dtype=torch.float32)
    raw = synth.draw_injections(cfg, 5, 18, dm_range=(0.0, 4000.0), max_width=n_t, min_sep=2)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    cube = cube.to(tdt)
    good = cube.clone()
    cube[11, 4, :] = 1.5                                   # zero MAD in one row of pixel 11
    plan = native.Plan(cfg, dtype=dtype, noise="mad")
    plan.search(cube.cuda())
    with pytest.raises(native.NsfrbError) as e:
        plan.candidates()
    assert e.value.status == native.EINVAL
    snr, idx = plan.best()
    assert snr[11] == -np.inf and (idx[11] == -1).all()
    plan.search(good.cuda())
    cand = plan.candidates()
    snr, idx = plan.best()
    plan.close()
    tab, res, best, bad = _oracle(cfg, good.float().numpy(), mad=True)
    assert bad == 0
    parity.compare_best(snr, idx, best)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)


@pytest.mark.parametrize("kind", ["ties", "sorted", "spikes"])
def test_records_mode_mad_order_statistics(native, kind):
    """Rows that stress the exact median / MAD selection of the normalisation pass: few distinct
    values (long runs of ties), sorted rows, and constant rows with a few spikes (MAD from the
    ties of a single value), against the FP64 oracle's sort-based median and MAD."""
    cfg = synth.SearchConfig(ny=4, nx=5, n_t=1000, dm=np.linspace(0.0, 3000.0, 40),
                             widths=np.array([1, 2, 4, 8, 32, 100, 640], np.int32), threshold=4.0)
    rng = np.random.default_rng({"ties": 1, "sorted": 2, "spikes": 3}[kind])
    shape = (cfg.n_pix, cfg.n_sub, cfg.n_t)
    if kind == "ties":
        x = rng.integers(-3, 4, shape).astype(np.float32) * 0.5
    elif kind == "sorted":
        x = np.sort(rng.standard_normal(shape).astype(np.float32), axis=2)
        x[::2] = x[::2, :, ::-1]
    else:
        x = np.full(shape, 1.25, np.float32) + rng.integers(0, 4, shape).astype(np.float32) * 0.5
        x[:, :, rng.integers(0, cfg.n_t, 40)] += 9.0
    cube = torch.from_numpy(x).to(torch.bfloat16)
    plan = native.Plan(cfg, dtype="bf16", noise="mad")
    plan.search(cube.cuda())
    cand = plan.candidates()
    snr, idx = plan.best()
    plan.close()
    tab, res, best, bad = _oracle(cfg, cube.float().numpy(), mad=True)
    assert bad == 0
    parity.compare_best(snr, idx, best)
    parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)


# ----------------------------------------------------------------------------- pixel x DM tiles

@pytest.mark.parametrize("dtype,noise,n_t", [("f32", "known", 1200), ("f32", "known", 640),
                                             ("bf16", "known", 1200), ("f16", "known", 1000),
                                             ("bf16", "mad", 840)])
def test_every_tile_matches_oracle(native, dtype, noise, n_t):
    """Every (teams, buffers) tile of the barrier-free kernel that fits gives the oracle's per-pixel
    records and candidates; the autotuner keeps the fastest of them and leaves the plan's results
    those of that tile."""
    rng = np.random.default_rng(n_t + 7 * len(dtype))
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    if noise == "mad":
        cfg = synth.config_stress(7, 9, n_t=n_t)
        cfg.widths = np.array([w for w in cfg.widths if w <= n_t], np.int32)
        cube = synth.beam_student_noise(cfg, 3, dtype=torch.float32).to(tdt)
        sig = None
    else:
        widths = [1, 2, 3, 4, 8, 16, 32, 64, 128, 256, 512]
        cfg = synth.SearchConfig(ny=7, nx=11, n_t=n_t, dm=np.sort(rng.uniform(0, 2500, 41)),
                                 widths=np.array(widths, np.int32), threshold=4.5)
        cube = _psf_cube(cfg, n_t, 6, dm_range=(0.0, 2500.0)).to(tdt)
        sig = rng.uniform(4.0, 8.0, cfg.n_pix).astype(np.float32)
    dev = cube.cuda()
    sg = None if sig is None else torch.as_tensor(sig).cuda()
    tab, res, best, bad = _oracle(cfg, cube.float().numpy(), sigma=sig, mad=(noise == "mad"))
    assert bad == 0
    plan = native.Plan(cfg, dtype=dtype, noise=noise, out="candidates")
    chosen, ms = plan.autotune(dev, sg, reps=2)
    st = native.F32 if noise == "mad" else plan.dtype      # MAD slabs are searched as FP32
    assert chosen in ms and ms[chosen] == min(ms.values()) and plan.get_tile(st) == chosen
    assert 12 in ms and len(ms) >= 2                       # one team of two buffers always fits
    checked = []
    for tile in [chosen] + [t for t in ms if t != chosen]:
        if tile != chosen:
            plan.set_tile(st, tile)
            plan.search(dev, sg)
        cand = plan.candidates()
        snr, idx = plan.best()
        parity.compare_best(snr, idx, best)
        parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
        checked.append(tile)
    plan.close()
    assert sorted(checked) == sorted(ms)


@pytest.mark.parametrize("dtype,n_t", [("f32", 1200), ("bf16", 1200), ("f32", 100)])
def test_every_tile_full_arrays(native, dtype, n_t):
    """FULL arrays from every (teams, buffers) tile of the barrier-free kernel equal the oracle's."""
    rng = np.random.default_rng(n_t + 3 * len(dtype))
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    widths = [w for w in [1, 2, 3, 4, 8, 16, 32, 64, 100, 128, 256, 512, 1024] if w <= n_t]
    cfg = synth.SearchConfig(ny=5, nx=7, n_t=n_t, dm=np.sort(rng.uniform(0, 2500, 29)),
                             widths=np.array(widths, np.int32), threshold=4.5)
    cube = _psf_cube(cfg, n_t, 4, dm_range=(0.0, 2500.0)).to(tdt)
    sig = rng.uniform(4.0, 8.0, cfg.n_pix).astype(np.float32)
    dev, sg = cube.cuda(), torch.as_tensor(sig).cuda()
    x = cube.float().numpy()
    tab, res, best, bad = _oracle(cfg, x, sigma=sig)
    plan = native.Plan(cfg, dtype=dtype, out="full")
    _, ms = plan.autotune(dev, sg, reps=1)
    assert 12 in ms and len(ms) >= 2
    for tile in ms:
        plan.set_tile(plan.dtype, tile)
        plan.search(dev, sg)
        f_snr, f_t = plan.full()
        parity.compare_full(f_snr, f_t, res, x=x, sigma=sig, shifts=tab, widths=cfg.widths)
        snr, idx = plan.best()
        parity.compare_best(snr, idx, best)
    plan.close()
