"""The classifier's 3x3x3 convolution kernels through the C ABI (Sec. 2.3): the tcgen05 kernel
(accumulator in tensor memory) and the mma.sync halo kernel, each against a
float64 convolution of the same BF16 operands, and their per-brick batch-norm column sums
against sums of their own output."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _run(native, path, x, w, part):
    B, D, H, W, CI = x.shape
    CO = w.shape[0]
    y = torch.full((B, D, H, W, CO), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    used = ctypes.c_int32(0)
    st = native.lib.nsfrb_dbg_conv3(path, B, D, H, W, CI, CO, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    ctypes.c_void_p(part.data_ptr() if part is not None else 0),
                                    ctypes.c_void_p(err.data_ptr()), ctypes.byref(used), None)
    torch.cuda.synchronize()
    return st, y, int(err.item()), used.value


def _reference(x, w):
    """float64 cross-correlation with zero padding 1 of the BF16 values, and the same over |.|."""
    xd = x.double().cpu().permute(0, 4, 1, 2, 3)                      # [B][CI][D][H][W]
    CO, _, CI = w.shape
    wd = w.double().cpu().reshape(CO, 3, 3, 3, CI).permute(0, 4, 1, 2, 3)   # [CO][CI][dz][dy][dx]
    ref = torch.nn.functional.conv3d(xd, wd, padding=1).permute(0, 2, 3, 4, 1)
    mag = torch.nn.functional.conv3d(xd.abs(), wd.abs(), padding=1).permute(0, 2, 3, 4, 1)
    return ref.numpy(), mag.numpy()


def _brick_sums(y, brick):
    """Column sums of y and y^2 per brick (bz, by, bx), bricks numbered b, z, y, x-fastest."""
    B, D, H, W, CO = y.shape
    bz, by, bx = brick
    t = y.reshape(B, D // bz, bz, H // by, by, W // bx, bx, CO).transpose(0, 1, 3, 5, 2, 4, 6, 7)
    t = t.reshape(-1, bz * by * bx, CO)
    return t.sum(axis=1), (t * t).sum(axis=1)


CASES = [  # B, D, H, W, CI, CO
    (2, 8, 32, 32, 16, 32),     # the first layer of the classifier on 32^3 cutouts (fewer planes)
    (1, 16, 16, 16, 32, 32),
    (1, 6, 16, 24, 16, 16),     # bricks that do not fill a CTA's pipeline evenly
    (2, 4, 16, 16, 32, 64),
    (1, 4, 16, 16, 64, 16),
    (1, 4, 32, 16, 16, 64),
]


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("B,D,H,W,CI,CO", CASES)
def test_conv3_against_float64(native, path, B, D, H, W, CI, CO):
    g = torch.Generator().manual_seed(B * 1000 + D * 100 + CI + CO)
    x = torch.randn((B, D, H, W, CI), generator=g).to(torch.bfloat16)
    w = (torch.randn((CO, 27, CI), generator=g) / np.sqrt(27 * CI)).to(torch.bfloat16)
    xd, wd = x.cuda(), w.cuda()
    n_bricks = B * D * H * W // 128
    part = torch.full((n_bricks, 2, CO), float("nan"), dtype=torch.float32, device="cuda")
    st, y, err, used = _run(native, path, xd, wd, part)
    if path == 1 and D % 2:
        assert st != native.OK
        return
    assert st == native.OK, native.lib.nsfrb_last_error()
    assert err == 0 and used == path
    ref, mag = _reference(x, w)
    got = y.cpu().numpy().astype(np.float64)
    K = 27 * CI
    bound = K * 2.0 ** -23 * mag + 1e-6          # twice the worst case of FP32 summation
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    s, q = _brick_sums(got, (1, 16, 8) if path == 2 else (2, 8, 8))
    p = part.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(p[:, 0], s, rtol=1e-5, atol=1e-4 * np.sqrt(128))
    np.testing.assert_allclose(p[:, 1], q, rtol=1e-5, atol=1e-4 * np.sqrt(128))


def test_conv3_paths_agree_and_are_deterministic(native):
    g = torch.Generator().manual_seed(7)
    x = torch.randn((2, 8, 32, 32, 16), generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn((32, 27, 16), generator=g) / 20.0).to(torch.bfloat16).cuda()
    part = torch.empty((2 * 8 * 32 * 32 // 128, 2, 32), dtype=torch.float32, device="cuda")
    st1, y1, _, _ = _run(native, 2, x, w, part)
    p1 = part.clone()
    st2, y2, _, _ = _run(native, 2, x, w, part)
    assert st1 == st2 == native.OK
    assert torch.equal(y1, y2) and torch.equal(p1, part)
    st3, y3, _, used = _run(native, 0, x, w, None)
    assert st3 == native.OK and used == 2 and torch.equal(y1, y3)
    st4, y4, _, _ = _run(native, 1, x, w, None)
    assert st4 == native.OK
    assert (y1 - y4).abs().max().item() <= 1e-4 * y4.abs().max().item()


def test_conv3_tc_declines_shapes_it_cannot_tile(native):
    x = torch.zeros((1, 4, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((32, 27, 16), dtype=torch.bfloat16, device="cuda")
    st, _, _, _ = _run(native, 2, x, w, None)          # H = 8 does not divide into 16-row bricks
    assert st == native.EINVAL
    st, y, _, used = _run(native, 0, x, w, None)       # the library falls back to the halo kernel
    assert st == native.OK and used == 1 and torch.count_nonzero(y).item() == 0


def test_conv3_tc_wait_timeout_is_reported_and_recovers(native):
    """With its halo producers stalled, the tcgen05 kernel's bounded waits run out: it latches
    the error bit, frees its tensor memory and returns, y untouched; the next launch is normal."""
    g = torch.Generator().manual_seed(11)
    x = torch.randn((1, 4, 16, 16, 16), generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn((32, 27, 16), generator=g) / 20.0).to(torch.bfloat16).cuda()
    st, y, err, used = _run(native, 3, x, w, None)
    assert st == native.OK and used == 2
    assert err & 4
    assert torch.isnan(y).all()                       # the epilogue never ran
    st, y, err, _ = _run(native, 2, x, w, None)
    assert st == native.OK and err == 0
    ref, mag = _reference(x.cpu(), w.cpu())
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 27 * 16 * 2.0 ** -23 * mag + 1e-6)
