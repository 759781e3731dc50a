"""nsfrb_search_static: the search for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they search (another allocator owns
the free device memory, or a real-time loop cannot afford an allocation that
may synchronise the device).  nsfrb_search_static keeps its scratch in a fixed
array inside the library and writes the candidates into a device buffer the
caller provides.  This test calls it through the C ABI and checks that it
returns what nsfrb_search + nsfrb_candidates return, on two calls in a row
(the second call must not see the first call's leftovers).
"""
import ctypes

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


def _cube(cfg, seed):
    cube = synth.psf_noise(cfg, seed)
    raw = synth.draw_injections(cfg, 6, seed + 7, max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    return cube


def _launch(native, plan, cube, sigma, out, n):
    st = native.lib.nsfrb_search_static(plan.handle, ctypes.c_void_p(cube.data_ptr()),
                                        None if sigma is None else ctypes.c_void_p(sigma.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), out.shape[0], ctypes.c_void_p(n.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == native.OK, native.lib.nsfrb_last_error()


def _static_call(native, plan, cube, sigma, cap):
    out = torch.zeros((cap, 6), dtype=torch.int32, device="cuda")
    n = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    _launch(native, plan, cube, sigma, out, n)
    torch.cuda.synchronize()
    total = int(n.item())
    rows = out[:min(total, cap)].cpu().numpy()
    rec = np.zeros(rows.shape[0], dtype=native.CANDIDATE_DTYPE)
    for i, name in enumerate(["row", "col", "dm_idx", "w_idx", "t_idx"]):
        rec[name] = rows[:, i]
    rec["snr"] = rows[:, 5].view(np.float32)
    return total, rec


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_static_search_matches_allocating_search(native, dtype):
    cfg = synth.config_full_window(13, 17)
    cfg.threshold = 5.0
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0, device="cuda")
    plan = native.Plan(cfg, dtype=dtype)
    ref = native.Plan(cfg, dtype=dtype)
    for seed in (3, 4):   # two calls in a row through the same scratch array
        cube = _cube(cfg, seed).to(torch.bfloat16 if dtype == "bf16" else torch.float32).cuda()
        ref.search(cube, sigma)
        want = ref.candidates()
        total, got = _static_call(native, plan, cube, sigma, cap=cfg.n_pix)
        assert total == len(want) and total > 0
        for name in ["row", "col", "dm_idx", "w_idx", "t_idx"]:
            np.testing.assert_array_equal(got[name], want[name])
        tol = parity.tol(want["snr"].astype(np.float64))
        assert (np.abs(got["snr"].astype(np.float64) - want["snr"]) <= tol).all()
    plan.close()
    ref.close()


def test_static_search_capacity_and_limits(native):
    cfg = synth.SearchConfig(ny=4, nx=4, n_t=32, dm=np.array([0.0]), widths=np.array([1], np.int32),
                             threshold=-100.0)
    plan = native.Plan(cfg)
    cube = torch.randn((16, 16, 32), device="cuda")
    sigma = torch.full((16,), 4.0, device="cuda")
    total, got = _static_call(native, plan, cube, sigma, cap=5)
    assert total == 16 and len(got) == 5
    assert list(got["row"] * 4 + got["col"]) == [0, 1, 2, 3, 4]
    big = synth.SearchConfig(ny=513, nx=512, n_t=32, dm=np.array([0.0]), widths=np.array([1], np.int32))
    bplan = native.Plan(big)
    st = native.lib.nsfrb_search_static(bplan.handle, ctypes.c_void_p(cube.data_ptr()), None,
                                        ctypes.c_void_p(cube.data_ptr()), 1, ctypes.c_void_p(cube.data_ptr()),
                                        None)
    assert st == native.EINVAL


def test_static_search_mad_mode_and_zero_mad_code(native):
    """Median/MAD normalisation through the fixed scratch equals nsfrb_search's; a constant
    (pixel, subband) row (zero MAD) is reported as a count of -1."""
    cfg = synth.config_full_window(9, 11)
    cfg.threshold = 4.5
    plan = native.Plan(cfg, dtype="bf16", noise="mad")
    ref = native.Plan(cfg, dtype="bf16", noise="mad")
    for seed in (5, 6):
        cube = _cube(cfg, seed).to(torch.bfloat16).cuda()
        ref.search(cube)
        want = ref.candidates()
        total, got = _static_call(native, plan, cube, None, cap=cfg.n_pix)
        assert total == len(want) and total > 0
        for name in ["row", "col", "dm_idx", "w_idx", "t_idx"]:
            np.testing.assert_array_equal(got[name], want[name])
        assert (np.abs(got["snr"].astype(np.float64) - want["snr"]) <= parity.tol(want["snr"])).all()
    bad = _cube(cfg, 7).to(torch.bfloat16).cuda()
    bad[17, 3, :] = 2.0
    total, _ = _static_call(native, plan, bad, None, cap=cfg.n_pix)
    assert total == -1
    # the next call starts from cleared counters
    total, got = _static_call(native, plan, _cube(cfg, 5).to(torch.bfloat16).cuda(), None, cap=cfg.n_pix)
    assert total > 0
    plan.close()
    ref.close()


def test_static_search_allocates_nothing(native):
    """Repeated calls leave the device's free memory unchanged (the scratch array is reserved
    by the first call on the device, before the measurement)."""
    cfg = synth.config_full_window(13, 17)
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * 4.0, device="cuda")
    cube = _cube(cfg, 8).cuda()
    out = torch.zeros((cfg.n_pix, 6), dtype=torch.int32, device="cuda")
    n = torch.zeros((1,), dtype=torch.int32, device="cuda")
    plan = native.Plan(cfg)
    _launch(native, plan, cube, sigma, out, n)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _launch(native, plan, cube, sigma, out, n)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(n.item()) >= 0
    plan.close()
