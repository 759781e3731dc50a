"""Pins of the FP64 classifier oracle (Sec. 2.3 classifier) against library
routines (torch float64 autograd), central finite differences and published
Philox known-answer vectors."""
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle  # noqa: F401  (builds the library)
from oracle import cnn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DIMS = cnn.CnnDims(B=3, D=16, H=16, W=32, C0=2, C=(2, 3, 3, 4), F=3)


def _params(dims, seed):
    rng = np.random.default_rng(seed)
    p = np.empty(cnn.n_params(dims))
    for name, o, shape in cnn.layout(dims):
        n = int(np.prod(shape))
        if name.endswith("gamma"):
            p[o:o + n] = rng.uniform(0.5, 1.5, n)
        else:
            p[o:o + n] = rng.normal(0.0, 0.4, n)
    return p


def _torch_model(dims, params, x, labels, keep=None, p=0.0):
    """The same network written with torch.nn.functional in float64 (NCDHW)."""
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    t = {name: P[o:o + int(np.prod(shape))].reshape(shape) for name, o, shape in cnn.layout(dims)}
    h = torch.tensor(x, dtype=torch.float64).permute(0, 4, 1, 2, 3)
    for l in range(4):
        w = t[f"conv{l}.w"].permute(0, 4, 1, 2, 3)          # [Co, Ci, kz, ky, kx]
        h = F.conv3d(h, w, padding=1)
        h = F.batch_norm(h, None, None, t[f"bn{l}.gamma"], t[f"bn{l}.beta"], training=True, eps=1e-5)
        h = F.max_pool3d(F.relu(h), 2)
    feat = h.permute(0, 2, 3, 4, 1).reshape(dims.B, -1)       # flatten (d, h, w, c)
    h1 = F.relu(feat @ t["fc1.w"].T + t["fc1.b"])
    if keep is not None:
        h1 = h1 * torch.tensor(keep, dtype=torch.float64) / (1.0 - p)
    z = h1 @ t["fc2.w"] + t["fc2.b"]
    loss = F.binary_cross_entropy_with_logits(z, torch.tensor(labels, dtype=torch.float64))
    loss.backward()
    return loss.item(), z.detach().numpy(), P.grad.numpy()


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(s, 16) for s in line.split()]
            np.testing.assert_array_equal(cnn.philox4x32_10(v[0:4], v[4:6]), np.array(v[6:10], np.uint32))


def test_dropout_mask_rate():
    keep = cnn.dropout_mask(64, 128, 0.5, 7, 12345)
    assert abs(keep.mean() - 0.5) < 0.02
    assert (keep != cnn.dropout_mask(64, 128, 0.5, 8, 12345)).any()


@pytest.mark.parametrize("with_dropout", [False, True])
def test_forward_and_gradients_match_torch_float64(with_dropout):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    labels = np.array([0.0, 1.0, 1.0])
    params = _params(DIMS, 1)
    keep = cnn.dropout_mask(DIMS.B, DIMS.F, 0.3, 3, 99) if with_dropout else None
    p = 0.3 if with_dropout else 0.0
    out = cnn.forward_backward(DIMS, params, x, labels, keep=keep, p=p)
    l_ref, z_ref, g_ref = _torch_model(DIMS, params, x, labels, keep, p)
    assert out["loss"] == pytest.approx(l_ref, rel=1e-10)
    np.testing.assert_allclose(out["logits"], z_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(out["grads"], g_ref, rtol=1e-8, atol=1e-11)


def test_gradients_by_central_differences():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    labels = np.array([1.0, 0.0, 1.0])
    params = _params(DIMS, 2)
    g = cnn.forward_backward(DIMS, params, x, labels)["grads"]
    h = 1e-6
    for i in rng.choice(params.size, size=25, replace=False):
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        num = (cnn.forward_backward(DIMS, pp, x, labels, grads=False)["loss"] -
               cnn.forward_backward(DIMS, pm, x, labels, grads=False)["loss"]) / (2 * h)
        assert num == pytest.approx(g[i], rel=1e-4, abs=1e-7), i


def test_eval_mode_uses_running_statistics():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    params = _params(DIMS, 3)
    nc = sum(DIMS.C)
    rm, rv = rng.normal(0, 0.2, nc), rng.uniform(0.5, 2.0, nc)
    out = cnn.forward_backward(DIMS, params, x, train=False, run_mean=rm, run_var=rv, grads=False)
    P = torch.tensor(params)
    t = {name: P[o:o + int(np.prod(shape))].reshape(shape) for name, o, shape in cnn.layout(DIMS)}
    h = torch.tensor(x).permute(0, 4, 1, 2, 3)
    c0 = 0
    for l in range(4):
        h = F.conv3d(h, t[f"conv{l}.w"].permute(0, 4, 1, 2, 3), padding=1)
        c = DIMS.C[l]
        h = F.batch_norm(h, torch.tensor(rm[c0:c0 + c]), torch.tensor(rv[c0:c0 + c]), t[f"bn{l}.gamma"],
                         t[f"bn{l}.beta"], training=False, eps=1e-5)
        h = F.max_pool3d(F.relu(h), 2)
        c0 += c
    feat = h.permute(0, 2, 3, 4, 1).reshape(DIMS.B, -1)
    z = F.relu(feat @ t["fc1.w"].T + t["fc1.b"]) @ t["fc2.w"] + t["fc2.b"]
    np.testing.assert_allclose(out["logits"], z.numpy(), rtol=1e-10, atol=1e-12)


def test_batch_statistics_returned_unbiased():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    params = _params(DIMS, 4)
    out = cnn.forward_backward(DIMS, params, x, labels=np.zeros(3), grads=False)
    P = torch.tensor(params)
    w0 = P[:DIMS.C[0] * 27 * DIMS.C0].reshape(DIMS.C[0], 3, 3, 3, DIMS.C0).permute(0, 4, 1, 2, 3)
    y = F.conv3d(torch.tensor(x).permute(0, 4, 1, 2, 3), w0, padding=1)
    np.testing.assert_allclose(out["run_mean"][:DIMS.C[0]], y.mean(dim=(0, 2, 3, 4)).numpy(), rtol=1e-10)
    np.testing.assert_allclose(out["run_var"][:DIMS.C[0]], y.var(dim=(0, 2, 3, 4), unbiased=True).numpy(),
                               rtol=1e-10)


def test_adam_matches_torch():
    rng = np.random.default_rng(1)
    p0 = rng.standard_normal(50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        cnn.adam(p, g, m, v, t, lr=1e-2)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_cutout_hand_example():
    """One bright sample: cube 6x5 px, 2 subbands, 40 samples; candidate at (row 3, col 1),
    width 2, largest shift 2 -> span 4, bin b = 1 for D = 16 (span <= 8), window start
    ts = t_idx + 2 - 8.  With t_idx = 20: ts = 14, so sample t = 21 of subband 1 at pixel
    (2, 2) lands at z = 7, y = 2 - 3 + 8 = 7, x = 2 - 1 + 8 = 9."""
    cube = np.zeros((30, 2, 40))
    cube[2 * 5 + 2, 1, 21] = 8.0
    cands = np.zeros(1, dtype=[("row", "<i4"), ("col", "<i4"), ("dm_idx", "<i4"), ("w_idx", "<i4"),
                               ("t_idx", "<i4"), ("snr", "<f4")])
    cands[0] = (3, 1, 0, 0, 20, 9.0)
    out = cnn.cutouts_grid(cube, 6, 5, cands, smax=np.array([2]), widths=np.array([2]), D=16, H=16, W=16,
                           sigma=np.full(30, 2.0 * np.sqrt(2.0)))
    assert out.shape == (1, 16, 16, 16, 2)
    nz = np.argwhere(out != 0)
    assert nz.tolist() == [[0, 7, 7, 9, 1]]
    assert out[0, 7, 7, 9, 1] == 8.0 / 2.0
    # a wide pulse: width 64, shift 0 -> span 64, b = 8, window start 20 + 32 - 64 = -12;
    # bin z averages samples -12 + 8z .. -5 + 8z, so sample 21 falls in z = 4
    cube2 = np.zeros((30, 2, 40))
    cube2[3 * 5 + 1, 0, 21] = 8.0
    out2 = cnn.cutouts_grid(cube2, 6, 5, cands, smax=np.array([0]), widths=np.array([64]), D=16, H=16, W=16)
    assert np.argwhere(out2 != 0).tolist() == [[0, 4, 8, 8, 0]]
    assert out2[0, 4, 8, 8, 0] == 1.0


def test_bf16_storage_mode_rounds_only_storage():
    """bf16_storage changes results by about the bfloat16 unit roundoff, no more."""
    rng = np.random.default_rng(21)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    labels = np.array([1.0, 0.0, 1.0])
    params = _params(DIMS, 6)
    a = cnn.forward_backward(DIMS, params, x, labels)
    b = cnn.forward_backward(DIMS, params, x, labels, bf16_storage=True)
    assert b["loss"] == pytest.approx(a["loss"], rel=2e-2)
    assert b["loss"] != a["loss"]
    rounded = torch.tensor(b["logits"], dtype=torch.float32)
    assert torch.isfinite(rounded).all()


def _torch_magnitudes(dims, params, x, labels, keep=None, p=0.0):
    """Sum of the magnitudes of the terms of every gradient entry, from torch float64 autograd's
    intermediate gradients: conv weights sum |dy| |a| over voxels (torch's conv3d weight gradient
    of the absolute values), BN gamma / beta sum |dz yhat| / |dz| over voxels, the head's entries
    sum over samples."""
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    t = {name: P[o:o + int(np.prod(shape))].reshape(shape) for name, o, shape in cnn.layout(dims)}
    h = torch.tensor(x, dtype=torch.float64).permute(0, 4, 1, 2, 3)
    keep_t = []
    for l in range(4):
        w = t[f"conv{l}.w"].permute(0, 4, 1, 2, 3)
        a = h
        y = F.conv3d(a, w, padding=1)
        y.retain_grad()
        mu = y.mean(dim=(0, 2, 3, 4), keepdim=True)
        var = y.var(dim=(0, 2, 3, 4), unbiased=False, keepdim=True)
        yhat = (y - mu) / torch.sqrt(var + 1e-5)
        z = t[f"bn{l}.gamma"].view(1, -1, 1, 1, 1) * yhat + t[f"bn{l}.beta"].view(1, -1, 1, 1, 1)
        z.retain_grad()
        keep_t.append((a, w, y, yhat, z))
        h = F.max_pool3d(F.relu(z), 2)
    feat = h.permute(0, 2, 3, 4, 1).reshape(dims.B, -1)
    pre = feat @ t["fc1.w"].T + t["fc1.b"]
    pre.retain_grad()
    h1 = F.relu(pre)
    if keep is not None:
        h1 = h1 * torch.tensor(keep, dtype=torch.float64) / (1.0 - p)
    zl = h1 @ t["fc2.w"] + t["fc2.b"]
    zl.retain_grad()
    F.binary_cross_entropy_with_logits(zl, torch.tensor(labels, dtype=torch.float64)).backward()
    mag = np.zeros_like(params)
    lay = {name: (o, shape) for name, o, shape in cnn.layout(dims)}

    def put(name, v):
        o, shape = lay[name]
        mag[o:o + int(np.prod(shape))] = v.detach().reshape(-1).numpy()

    for l, (a, w, y, yhat, z) in enumerate(keep_t):
        gw = torch.nn.grad.conv3d_weight(a.abs(), w.shape, y.grad.abs(), padding=1)   # [Co, Ci, kz, ky, kx]
        put(f"conv{l}.w", gw.permute(0, 2, 3, 4, 1))
        put(f"bn{l}.gamma", (z.grad * yhat).abs().sum(dim=(0, 2, 3, 4)))
        put(f"bn{l}.beta", z.grad.abs().sum(dim=(0, 2, 3, 4)))
    put("fc1.w", pre.grad.abs().T @ feat.abs())
    put("fc1.b", pre.grad.abs().sum(dim=0))
    put("fc2.w", zl.grad.abs() @ h1.abs())
    put("fc2.b", zl.grad.abs().sum())
    return mag


@pytest.mark.parametrize("with_dropout", [False, True])
def test_gradient_term_magnitudes_match_torch(with_dropout):
    """The oracle's per-entry sum of term magnitudes (the scale of the GPU comparison's bound)
    equals the one built from torch's intermediate gradients, and bounds |gradient|."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0))
    labels = np.array([1.0, 0.0, 1.0])
    params = _params(DIMS, 6)
    keep = cnn.dropout_mask(DIMS.B, DIMS.F, 0.3, 1, 7) if with_dropout else None
    p = 0.3 if with_dropout else 0.0
    out = cnn.forward_backward(DIMS, params, x, labels, keep=keep, p=p)
    ref = _torch_magnitudes(DIMS, params, x, labels, keep, p)
    np.testing.assert_allclose(out["grad_mag"], ref, rtol=1e-9, atol=1e-12)
    assert (out["grad_mag"] >= np.abs(out["grads"]) * (1 - 1e-12) - 1e-15).all()
    assert (out["grad_mag"] > np.abs(out["grads"]) * 1.5).any()     # cancellations exist
