"""The MAD normalisation pass (Sec. 2.2, robust reading) on its own, row by row: every normalised
sample equals the FP32 evaluation of the same formula from the exact order statistics (numpy sort),
and lies within the FP32 rounding bound of the FP64 oracle.  Rows are chosen to stress the
counting selection: ties, clusters far apart, signed zeros, huge dynamic range, sorted rows,
spikes, zero MAD, and every row length class (scalar and 16-byte paths, one sample to 4096)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _rows(kind, n_rows, n_t, rng):
    shape = (n_rows, n_t)
    if kind == "gauss":
        x = rng.standard_normal(shape) * rng.uniform(0.1, 50.0, (n_rows, 1)) + rng.uniform(-20, 20, (n_rows, 1))
    elif kind == "student":
        x = rng.standard_t(5, shape) * 3.0
    elif kind == "ties":
        x = rng.integers(-3, 4, shape) * 0.5
    elif kind == "clusters":                        # two clusters 30 decades apart
        x = np.where(rng.random(shape) < rng.uniform(0.3, 0.7, (n_rows, 1)), 1.0, 1e30)
        x = x * (1.0 + 1e-3 * rng.standard_normal(shape))
    elif kind == "zeros":                           # +0, -0 and a few small values
        x = rng.choice(np.array([0.0, -0.0, 1e-3, -2e-3]), size=shape, p=[0.4, 0.4, 0.1, 0.1])
    elif kind == "range":                           # log-uniform magnitudes, random signs
        x = np.exp(rng.uniform(-80, 80, shape)) * rng.choice([-1.0, 1.0], size=shape)
    elif kind == "sorted":
        x = np.sort(rng.standard_normal(shape), axis=1)
        x[::2] = x[::2, ::-1]
    elif kind == "spikes":                          # nearly constant with spikes: MAD from ties
        x = np.full(shape, 1.25) + rng.integers(0, 4, shape) * 0.5
        x[:, rng.integers(0, n_t, max(1, n_t // 25))] += 9.0
    elif kind == "constant":                        # MAD 0 (bad rows), half of them
        x = rng.standard_normal(shape)
        x[::2] = 2.5
    else:
        raise ValueError(kind)
    return x


def _expected_f32(xs):
    """The FP32 formula from exact order statistics: median (mean of the two middle values for even
    n, in FP32), MAD likewise, y = (x - m) * (1 / (1.4826 MAD)); MAD 0 -> zeros, bad."""
    n = xs.shape[1]
    h = np.float32(0.5)

    def med(v):
        s = np.sort(v, axis=1)
        if n % 2:
            return s[:, n // 2]
        return (h * (s[:, n // 2 - 1] + s[:, n // 2])).astype(np.float32)

    m = med(xs)
    dev = np.abs(xs - m[:, None]).astype(np.float32)
    mad = med(dev)
    bad = mad == 0
    with np.errstate(divide="ignore"):
        inv = (np.float32(1.0) / (np.float32(1.4826) * mad)).astype(np.float32)
    y = ((xs - m[:, None]) * inv[:, None]).astype(np.float32)
    y[bad] = 0.0
    return y, bad, m, mad


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n_t", [1, 2, 3, 31, 32, 33, 64, 100, 999, 1000, 1200, 1246, 1247, 2001, 4096])
def test_mad_normalise_rows(native, dtype, n_t):
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    kinds = ["gauss", "student", "ties", "clusters", "zeros", "range", "sorted", "spikes", "constant"]
    if dtype == "f16":                              # FP16 holds neither 1e30 nor e^80
        kinds = [k for k in kinds if k not in ("clusters", "range")]
    rng = np.random.default_rng(1000 * n_t + len(dtype))
    blocks = [_rows(k, 24, n_t, rng) for k in kinds]
    x = torch.from_numpy(np.concatenate(blocks).astype(np.float32)).to(tdt)
    xs = x.float().numpy()                          # the stored values
    n_rows = xs.shape[0]
    d_in = x.cuda().contiguous()
    d_out = torch.full((n_rows, n_t), float("nan"), device="cuda")
    d_bad = torch.full((n_rows,), 7, dtype=torch.uint8, device="cuda")
    st = native.lib.nsfrb_dbg_mad_normalise(ctypes.c_void_p(d_in.data_ptr()), {"f32": 0, "bf16": 1, "f16": 2}[dtype],
                                            n_rows, n_t, ctypes.c_void_p(d_out.data_ptr()),
                                            ctypes.c_void_p(d_bad.data_ptr()), None)
    assert st == native.OK
    torch.cuda.synchronize()
    y = d_out.cpu().numpy()
    bad = d_bad.cpu().numpy().astype(bool)
    with np.errstate(over="ignore", invalid="ignore"):
        y_ref, bad_ref, m, mad = _expected_f32(xs)
    np.testing.assert_array_equal(bad, bad_ref)
    np.testing.assert_array_equal(y, y_ref)         # bit for bit (signed zeros compare equal)
    # the FP64 oracle: same rows flagged, and every sample within the FP32 rounding bound
    y64, nbad = oracle.mad_normalise(xs)
    assert nbad == int(bad_ref.sum())
    good = ~bad_ref
    # FP32 roundings: the median (|dm| <= eps |m|), the deviations and with them the MAD (relative
    # error <= eps (1 + |m| / MAD)), the difference x - m and the product (which may be subnormal:
    # absolute error up to 2^-149)
    mad_s = np.where(good, mad, 1.0)[:, None].astype(np.float64)
    scale = (np.abs(xs) + np.abs(m[:, None])) / (1.4826 * mad_s)
    bound = 8 * EPS32 * (np.abs(y64) * (1.0 + np.abs(m[:, None]) / mad_s) + scale) + 2.0 ** -148
    err = np.abs(y.astype(np.float64) - y64)
    cmp = good[:, None] & (np.abs(y64) < 1e37)      # normalised values inside the FP32 range
    assert (err[cmp] <= bound[cmp]).all(), float(np.max(err[cmp] / bound[cmp]))


def test_mad_normalise_rejects_bad_sizes(native):
    d = torch.zeros(16, device="cuda")
    b = torch.zeros(4, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    for n_rows, n_t, dt in ((0, 4, 0), (4, 0, 0), (1, 4097, 0), (4, 4, 3)):
        assert native.lib.nsfrb_dbg_mad_normalise(p, dt, n_rows, n_t, p, ctypes.c_void_p(b.data_ptr()),
                                                  None) == native.EINVAL
