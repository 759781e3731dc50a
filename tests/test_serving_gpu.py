"""Serving loop (rolling window, block push, masked search, CUDA graph) vs the oracle.

After each pushed block the streamed candidates must equal the oracle's search
of the current window restricted to the trials that end in the newest block
(t + w - 1 + smax_d >= n_t - n_blk).
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


def _series(cfg, n_total, seed, n_inj=5):
    """A long pixel-major series [n_pix, n_sub, n_total] with pulses spread over time."""
    long_cfg = synth.SearchConfig(ny=cfg.ny, nx=cfg.nx, n_t=n_total, freq_mhz=cfg.freq_mhz, dm=cfg.dm,
                                  widths=cfg.widths)
    x = synth.plain_noise(long_cfg, seed)
    raw = synth.draw_injections(long_cfg, n_inj, seed + 1, dm_range=(0.0, float(cfg.dm[-1])),
                                snr_range=(8.0, 20.0), max_width=32, min_sep=1)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, n_total, cfg.n_sub, 1.0)
    synth.add_injections(x, long_cfg, inj, sh)
    return x


def _window_oracle(cfg, window, n_blk, tab):
    smax = tab.max(axis=1)
    t_lo = np.array([[cfg.n_t - n_blk - int(w) + 1 - int(s) for w in cfg.widths] for s in smax], np.int32)
    res, best, _ = oracle.search_cube(window, tab, cfg.widths, sigma=4.0, t_lo=t_lo)
    return best


@pytest.mark.parametrize("dtype,n_blk", [("f32", 12), ("bf16", 12), ("f32", 25), ("bf16", 25)])
def test_stream_equals_masked_window_search(native, dtype, n_blk):
    """n_blk = 25 (the paper's block) moves the window start by 100 bytes per FP32 block: the
    search must not take the 16-byte-aligned bulk-copy path there."""
    cfg = synth.SearchConfig(ny=5, nx=7, n_t=96, dm=np.linspace(0, 1500, 20),
                             widths=np.array([1, 2, 4, 8, 16, 32, 50], np.int32), threshold=5.0)
    n_blocks = 14
    x = _series(cfg, n_blk * n_blocks, 3)
    if dtype == "bf16":
        x = x.to(torch.bfloat16).to(torch.float32)
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    plan = native.Plan(cfg, dtype=dtype)
    plan.stream_open(n_blk)
    xn = x.numpy()
    total = 0
    for b in range(n_blocks):
        blk = torch.from_numpy(xn[:, :, b * n_blk:(b + 1) * n_blk].transpose(2, 1, 0).copy())
        blk = blk.reshape(n_blk, cfg.n_sub, cfg.ny, cfg.nx).contiguous()
        plan.stream_push(blk)
        cand, lat = plan.stream_poll(timeout_ms=10000)
        assert lat > 0.0
        end = (b + 1) * n_blk
        window = np.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t), np.float32)
        lo = max(0, end - cfg.n_t)
        window[:, :, cfg.n_t - (end - lo):] = xn[:, :, lo:end]
        best = _window_oracle(cfg, window, n_blk, tab)
        parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
        total += len(cand)
    assert total > 0
    assert plan.stream_blocks() == n_blocks
    plan.close()


def test_stream_missing_subband_is_zero_filled(native):
    cfg = synth.SearchConfig(ny=3, nx=4, n_t=48, dm=np.linspace(0, 1000, 9),
                             widths=np.array([1, 2, 4, 8], np.int32), threshold=3.0)
    n_blk = 8
    x = _series(cfg, n_blk * 8, 11, n_inj=3).numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    plan = native.Plan(cfg)
    plan.stream_open(n_blk)
    seen = x.copy()
    for b in range(8):
        mask = (1 << 16) - 1
        if b == 6:
            mask &= ~(1 << 3)
            seen[:, 3, b * n_blk:(b + 1) * n_blk] = 0.0
        blk = torch.from_numpy(x[:, :, b * n_blk:(b + 1) * n_blk].transpose(2, 1, 0).copy())
        plan.stream_push(blk.reshape(n_blk, 16, cfg.ny, cfg.nx).contiguous(), present_mask=mask)
        cand, _ = plan.stream_poll(timeout_ms=10000)
        end = (b + 1) * n_blk
        window = np.zeros((cfg.n_pix, 16, cfg.n_t), np.float32)
        lo = max(0, end - cfg.n_t)
        window[:, :, cfg.n_t - (end - lo):] = seen[:, :, lo:end]
        best = _window_oracle(cfg, window, n_blk, tab)
        parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
    plan.close()


def test_stream_admission_and_protocol_errors(native):
    cfg = synth.SearchConfig(ny=4, nx=4, n_t=64, dm=np.array([0.0, 500.0]), widths=np.array([1, 4], np.int32))
    plan = native.Plan(cfg)
    with pytest.raises(native.NsfrbError) as e:
        plan.stream_open(8, hbm_reserve=1 << 60)    # admission: more than the device has
    assert e.value.status == native.ENOMEM
    plan.stream_open(8)
    with pytest.raises(native.NsfrbError) as e:
        plan.stream_poll(timeout_ms=10)              # nothing pushed yet
    assert e.value.status == native.ENOTREADY
    blk = torch.randn((8, 16, 4, 4))
    plan.stream_push(blk)
    with pytest.raises(native.NsfrbError) as e:
        plan.stream_push(blk)                        # previous block not polled
    assert e.value.status == native.ENOTREADY
    plan.stream_poll(timeout_ms=10000)
    assert plan.stream_bytes(8) > 0
    plan.close()


@pytest.mark.parametrize("n_blk,where", [(12, "device"), (25, "device"), (25, "host")])
def test_stream_bf16_rescore_from_fp32_window(native, n_blk, where):
    """BF16 window with re-scoring from the FP32 window: pixels whose best over the new trials
    lies within eps of the threshold carry the FP32 result (FP64 oracle of the FP32 values within
    the FP32 tolerance), the rest the BF16 one, and the candidate set is the FP32 oracle's.  A
    block with a missing subband checks that the FP32 window is zero-filled too.  The window sits
    in device memory when the admission budget allows, else in pinned host memory: a reserve that
    leaves room for the ring but not the window forces the host placement."""
    cfg = synth.SearchConfig(ny=6, nx=7, n_t=96, dm=np.linspace(0, 1500, 20),
                             widths=np.array([1, 2, 4, 8, 16, 32, 50], np.int32), threshold=5.0)
    eps = 1.0
    n_blocks = 12
    xn = _series(cfg, n_blk * n_blocks, 5).numpy()
    seen = xn.copy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    plan = native.Plan(cfg, dtype="bf16", rescore_eps=eps)
    reserve = 0
    if where == "host":
        plan.search(torch.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t), dtype=torch.bfloat16, device="cuda"))
        plan.candidates()                              # the plan's device state exists from here on
        free0 = torch.cuda.mem_get_info()[0]
        fbytes = cfg.n_pix * cfg.n_sub * cfg.n_t * 4
        reserve = free0 - plan.stream_bytes(n_blk) - fbytes // 2
    plan.stream_open(n_blk, hbm_reserve=reserve)
    assert plan.stream_window_info() == (1 if where == "device" else 2)
    n_rescored = 0
    for b in range(n_blocks):
        mask = (1 << 16) - 1
        if b == 7:
            mask &= ~(1 << 5)
            seen[:, 5, b * n_blk:(b + 1) * n_blk] = 0.0
        blk = torch.from_numpy(xn[:, :, b * n_blk:(b + 1) * n_blk].transpose(2, 1, 0).copy())
        plan.stream_push(blk.reshape(n_blk, cfg.n_sub, cfg.ny, cfg.nx).contiguous(), present_mask=mask)
        cand, _ = plan.stream_poll(timeout_ms=10000)
        end = (b + 1) * n_blk
        lo = max(0, end - cfg.n_t)
        window = np.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t), np.float32)
        window[:, :, cfg.n_t - (end - lo):] = seen[:, :, lo:end]
        best32 = _window_oracle(cfg, window, n_blk, tab)
        best16 = _window_oracle(cfg, oracle.bf16_round(window), n_blk, tab)
        near = np.abs(best16["snr"] - cfg.threshold) <= eps - 1e-3   # clear of the selection edge
        far = np.abs(best16["snr"] - cfg.threshold) > eps + 1e-3
        n_rescored += int(near.sum())
        g_pix = cand["row"].astype(np.int64) * cfg.nx + cand["col"]
        got = dict(zip(g_pix.tolist(), cand["snr"].tolist()))
        for p in range(cfg.n_pix):
            s32, s16 = best32["snr"][p], best16["snr"][p]
            if near[p] and abs(s32 - cfg.threshold) > parity.tol(s32):
                assert (p in got) == (s32 > cfg.threshold)
                if p in got:
                    assert abs(got[p] - s32) <= parity.tol(s32)
            elif far[p]:
                assert (p in got) == (s16 > cfg.threshold)
                if p in got:
                    assert abs(got[p] - s16) <= parity.tol(s16)
    assert n_rescored > 0
    plan.close()


@pytest.mark.parametrize("dtype,n_blk", [("f32", 25), ("bf16", 25), ("f16", 12), ("bf16", 7)])
def test_stream_long_window(native, dtype, n_blk):
    """A window of 832 samples (the sample-pair chunk): the window start moves by n_blk per block,
    so the barrier-free kernel reads every row from an offset below a 16-byte boundary and sets the
    de-dispersed samples past the valid range to -inf."""
    cfg = synth.SearchConfig(ny=3, nx=5, n_t=832, dm=np.linspace(0, 1500, 24),
                             widths=np.array([1, 2, 4, 8, 16, 32, 64, 100, 128, 256], np.int32), threshold=5.0)
    n_blocks = max(6, 160 // n_blk)
    start = (cfg.n_t // n_blk - 2) * n_blk       # check from a nearly full window on
    total = start + n_blk * n_blocks
    x = _series(cfg, total, 13, n_inj=6)
    if dtype != "f32":
        tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
        x = x.to(tdt).to(torch.float32)
    xn = x.numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    plan = native.Plan(cfg, dtype=dtype)
    plan.stream_open(n_blk)
    pushed = 0
    n_cand = 0
    while pushed < total:
        nb = n_blk
        blk = torch.from_numpy(xn[:, :, pushed:pushed + nb].transpose(2, 1, 0).copy())
        plan.stream_push(blk.reshape(nb, cfg.n_sub, cfg.ny, cfg.nx).contiguous())
        cand, _ = plan.stream_poll(timeout_ms=10000)
        pushed += nb
        if pushed >= start:
            lo = max(0, pushed - cfg.n_t)
            window = np.zeros((cfg.n_pix, cfg.n_sub, cfg.n_t), np.float32)
            window[:, :, cfg.n_t - (pushed - lo):] = xn[:, :, lo:pushed]
            best = _window_oracle(cfg, window, n_blk, tab)
            parity.compare_candidates(cand, best, cfg.threshold, np.arange(cfg.n_pix), cfg.nx)
            n_cand += len(cand)
    assert n_cand > 0
    plan.close()
