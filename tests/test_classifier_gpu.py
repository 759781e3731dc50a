"""CUDA classifier kernels vs the FP64 classifier oracle (needs a GPU).

The network is defined with its pooled activations and the back-propagated gradients at the
convolution outputs stored in bfloat16 (the classifier's BF16 training kernels); the oracle
computes that network in FP64 (``bf16_storage``), on the same BF16 input and conv weights.

Gradients are compared entry by entry: |g_gpu - g_oracle| <= TAU (M + M_rms), M the sum of the
magnitudes of the entry's terms (from the oracle) and M_rms the root mean square of M over the
entry's tensor.  A term is a product of two stored values (or of a stored value and an FP32 one);
the GPU stores the same BF16 value as the oracle except where its FP32 value and the oracle's FP64
value fall on two sides of a rounding boundary, and then they differ by one BF16 unit in the last
place (at most 2^-7 relative): a term moves by at most 2^-6 of its magnitude.  Such one-unit
differences of the stored inputs of a layer, summed over its 27 C taps, give its outputs an
absolute error on the scale of typical values, not of the output itself; small values (near the
ReLU kink, small pooled maxima) therefore carry errors relative to the typical term, which M_rms
stands for.  A max-pool arg-max taken differently at a near-tie moves one gradient between two
voxels of a window, a change bounded by those terms' magnitudes.  TAU = 2^-5 covers these;
FP32 accumulation adds at most K 2^-23 M (K the number of terms), far below.
Loss and logits are also compared with the plain FP64 network (no storage rounding): the GPU
must be as close to it as three times the storage rounding's own effect, measured by the oracle.
"""
import math
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
from oracle import cnn
from paper_2510_18136_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = cnn.CnnDims(B=4, D=16, H=16, W=16, C0=16, C=(8, 8, 16, 16), F=8)
# 16- and 32-channel layers on 16^3 and 8^3 volumes run the halo-tile convolution and
# weight-gradient kernels (2 x 8 x 8 bricks); the 4^3 and 2^3 layers the gathering GEMM
DIMS_HALO = cnn.CnnDims(B=2, D=16, H=16, W=16, C0=16, C=(32, 32, 16, 16), F=8)
# the production network: 32^3 cutouts x 16 subbands, 32-32-64-64 channels, 32 hidden units
DIMS_PROD = cnn.CnnDims(B=2, D=32, H=32, W=32, C0=16, C=(32, 32, 64, 64), F=32)
TAU = 2.0 ** -5


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _init(dims, seed):
    rng = np.random.default_rng(seed)
    p = np.empty(cnn.n_params(dims))
    for name, o, shape in cnn.layout(dims):
        n = int(np.prod(shape))
        if name.endswith("gamma"):
            p[o:o + n] = rng.uniform(0.5, 1.5, n)
        elif name.endswith("beta") or name.endswith(".b"):
            p[o:o + n] = rng.normal(0.0, 0.1, n)
        else:
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else shape[0]
            p[o:o + n] = rng.normal(0.0, 1.0 / math.sqrt(fan_in), n)
    return p.astype(np.float32)


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _as_oracle_params(dims, p32):
    """Conv weights as the GPU uses them (BF16); everything else FP32."""
    q = p32.astype(np.float64).copy()
    for name, o, shape in cnn.layout(dims):
        if name.startswith("conv"):
            n = int(np.prod(shape))
            q[o:o + n] = _bf16(p32[o:o + n])
    return q


def _make(native, dims, dropout=0.0, seed=3, lr=1e-3):
    return native.Classifier(batch=dims.B, d=dims.D, h=dims.H, w=dims.W, c0=dims.C0, c=dims.C, f=dims.F,
                             dropout=dropout, seed=seed, lr=lr)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("dims,dropout", [(DIMS, 0.0), (DIMS, 0.4), (DIMS_HALO, 0.0), (DIMS_PROD, 0.0),
                                          (DIMS_PROD, 0.5)])
def test_loss_and_gradients_match_oracle(native, dims, dropout):
    rng = np.random.default_rng(11)
    x = rng.standard_normal((dims.B, dims.D, dims.H, dims.W, dims.C0)).astype(np.float32)
    labels = np.array([0.0, 1.0, 1.0, 0.0][:dims.B], np.float32)
    p = _init(dims, 2)
    clf = _make(native, dims, dropout=dropout, seed=1234)
    clf.set_params(p)
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    loss = clf.train_step(xb, torch.from_numpy(labels).cuda(), update=False)
    g = clf.grads().astype(np.float64)
    keep = cnn.dropout_mask(dims.B, dims.F, dropout, 0, 1234) if dropout > 0 else None
    q = _as_oracle_params(dims, p)
    ref = cnn.forward_backward(dims, q, _bf16(x), labels, keep=keep, p=dropout, bf16_storage=True)
    plain = cnn.forward_backward(dims, q, _bf16(x), labels, keep=keep, p=dropout, grads=False)
    # every gradient entry
    mag = ref["grad_mag"]
    floor = np.empty_like(mag)
    for name, o, shape in cnn.layout(dims):
        n = int(np.prod(shape))
        floor[o:o + n] = np.sqrt(np.mean(mag[o:o + n] ** 2))
    bound = TAU * (mag + floor)
    err = np.abs(g - ref["grads"])
    worst = {}
    for name, o, shape in cnn.layout(dims):
        n = int(np.prod(shape))
        worst[name] = float(np.max(err[o:o + n] / bound[o:o + n]))
    if not (err <= bound).all():
        bad = np.nonzero(err > bound)[0]
        names = [next(nm for nm, o, sh in cnn.layout(dims) if o <= i < o + int(np.prod(sh))) for i in bad[:8]]
        print("violations", len(bad), list(zip(names, g[bad[:8]], ref["grads"][bad[:8]], ref["grad_mag"][bad[:8]])))
    assert (err <= bound).all(), sorted(worst.items(), key=lambda kv: -kv[1])[:4]
    # the bound is not vacuous: the terms' magnitudes are within a factor of the gradients'
    assert np.median(ref["grad_mag"] / np.maximum(np.abs(ref["grads"]), 1e-30)) < 200.0
    # loss against both networks
    k_loss = 2.0 ** -8 * abs(ref["loss"]) + 1e-6
    assert abs(loss - ref["loss"]) <= k_loss
    assert abs(loss - plain["loss"]) <= 3.0 * abs(ref["loss"] - plain["loss"]) + k_loss
    # running statistics: momentum 0.1 towards the batch mean / unbiased variance
    m, v = clf.bn_stats()
    np.testing.assert_allclose(m, 0.1 * ref["run_mean"], rtol=3e-2, atol=3e-3)
    np.testing.assert_allclose(v, 0.9 + 0.1 * ref["run_var"], rtol=3e-2, atol=3e-3)
    clf.close()
    print(f"{dims.C} {dims.D}^3 dropout {dropout}: worst |err| / bound per tensor", worst)


@pytest.mark.parametrize("dims", [DIMS, DIMS_HALO, DIMS_PROD])
def test_inference_matches_oracle_eval_mode(native, dims):
    DIMS = dims
    rng = np.random.default_rng(12)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0)).astype(np.float32)
    p = _init(DIMS, 4)
    nc = sum(DIMS.C)
    rm = rng.normal(0.0, 0.2, nc).astype(np.float32)
    rv = rng.uniform(0.5, 2.0, nc).astype(np.float32)
    clf = _make(native, DIMS)
    clf.set_params(p)
    clf.set_bn_stats(rm, rv)
    z = clf.infer(torch.from_numpy(x).to(torch.bfloat16).cuda()).cpu().numpy()
    q = _as_oracle_params(DIMS, p)
    ref = cnn.forward_backward(DIMS, q, _bf16(x), train=False, run_mean=rm, run_var=rv, grads=False,
                               bf16_storage=True)
    plain = cnn.forward_backward(DIMS, q, _bf16(x), train=False, run_mean=rm, run_var=rv, grads=False)
    # logits: within one BF16 unit of the storage network's (plus 1e-3 for FP32 sums over the head),
    # and as close to the plain FP64 network as three times the storage rounding's effect
    tol = 2.0 ** -7 * np.abs(ref["logits"]) + 1e-3
    assert (np.abs(z - ref["logits"]) <= tol).all(), np.max(np.abs(z - ref["logits"]) / tol)
    assert (np.abs(z - plain["logits"]) <= 3.0 * np.abs(ref["logits"] - plain["logits"]) + tol).all()
    clf.close()


def test_adam_step_matches_oracle(native):
    rng = np.random.default_rng(13)
    x = rng.standard_normal((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0)).astype(np.float32)
    labels = torch.tensor([1.0, 0.0, 0.0, 1.0]).cuda()
    p0 = _init(DIMS, 5)
    clf = _make(native, DIMS, lr=1e-2)
    clf.set_params(p0)
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    m, v = np.zeros(p0.size), np.zeros(p0.size)
    for t in range(1, 4):
        before = clf.params().astype(np.float64)
        clf.train_step(xb, labels, update=True)
        g = clf.grads().astype(np.float64)           # the gradient this update used
        cnn.adam(before, g, m, v, t, lr=1e-2)
        np.testing.assert_allclose(clf.params(), before, rtol=1e-5, atol=1e-7)
    clf.close()


@pytest.mark.parametrize("tn,M,N,K", [(0, 300, 8, 432), (0, 1000, 32, 216), (0, 4096, 64, 1728),
                                      (1, 8, 432, 16384), (1, 16, 216, 4096), (1, 64, 1728, 512)])
def test_gemm_against_torch(native, tn, M, N, K):
    import ctypes
    g = torch.Generator().manual_seed(M + N + K)
    if tn:
        a = torch.randn((K, M), generator=g).to(torch.bfloat16)
        b = torch.randn((K, N), generator=g).to(torch.bfloat16)
        ref = a.double().T @ b.double()
    else:
        a = torch.randn((M, K), generator=g).to(torch.bfloat16)
        b = torch.randn((N, K), generator=g).to(torch.bfloat16)
        ref = a.double() @ b.double().T
    ad, bd = a.cuda(), b.cuda()
    c = torch.empty((M, N), dtype=torch.float32, device="cuda")
    st = native.lib.nsfrb_dbg_gemm(tn, M, N, K, ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(bd.data_ptr()),
                                   ctypes.c_void_p(c.data_ptr()), None)
    assert st == native.OK
    torch.cuda.synchronize()
    err = (c.double().cpu() - ref).abs().max().item()
    assert err <= 1e-4 * math.sqrt(K) * ref.abs().max().item() + 1e-3, err


def test_checkpoint_roundtrip(native):
    clf = _make(native, DIMS)
    clf.set_params(_init(DIMS, 6))
    x = torch.randn((DIMS.B, DIMS.D, DIMS.H, DIMS.W, DIMS.C0)).to(torch.bfloat16).cuda()
    lab = torch.tensor([0.0, 1.0, 0.0, 1.0]).cuda()
    for _ in range(3):
        clf.train_step(x, lab)
    path = os.path.join(tempfile.mkdtemp(), "clf.bin")
    clf.save(path)
    other = _make(native, DIMS)
    other.load(path)
    np.testing.assert_array_equal(other.params(), clf.params())
    np.testing.assert_array_equal(other.bn_stats()[1], clf.bn_stats()[1])
    a = clf.train_step(x, lab)
    b = other.train_step(x, lab)
    # same state, same step counter: the same update bit for bit (every reduction of a training
    # step runs in a fixed order)
    assert a == b
    np.testing.assert_array_equal(other.params(), clf.params())
    clf.close()
    other.close()


def test_training_reduces_loss(native):
    """Two separable classes (a bright dispersed streak vs a bright single-subband line)."""
    torch.manual_seed(0)
    dims = cnn.CnnDims(B=16, D=16, H=16, W=16, C0=16, C=(8, 8, 16, 16), F=8)
    clf = _make(native, dims, dropout=0.0, lr=3e-3)
    clf.set_params(_init(dims, 7))
    losses = []
    for step in range(60):
        x = torch.randn((16, 16, 16, 16, 16))
        lab = (torch.arange(16) % 2).float()
        for i in range(16):
            if lab[i] == 0:
                for k in range(16):
                    x[i, 4 + k // 4, 7:9, 7:9, k] += 3.0
            else:
                x[i, 3:13, 7:9, 7:9, 5] += 3.0
        losses.append(clf.train_step(x.to(torch.bfloat16).cuda().contiguous(), lab.cuda()))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
    clf.close()


def test_cutouts_match_oracle(native):
    cfg = synth.SearchConfig(ny=20, nx=24, n_t=120, dm=np.linspace(0, 2000, 9),
                             widths=np.array([1, 4, 16, 64], np.int32))
    rng = np.random.default_rng(3)
    cube = torch.from_numpy(rng.standard_normal((cfg.n_pix, 16, 120)).astype(np.float32))
    sigma = torch.from_numpy(rng.uniform(2, 6, cfg.n_pix).astype(np.float32))
    plan = native.Plan(cfg)
    cands = np.zeros(6, dtype=native.CANDIDATE_DTYPE)
    rows = [(0, 0, 0, 0, 0), (19, 23, 8, 3, 60), (10, 12, 4, 1, 50), (5, 20, 8, 2, 100), (15, 2, 2, 3, 1),
            (9, 9, 6, 0, 119)]
    for i, (r, c, d, w, t) in enumerate(rows):
        cands[i] = (r, c, d, w, t, 7.0)
    dc = native.candidates_to_device(cands)
    out = native.cutouts(plan, cube.cuda(), dc, d=16, h=16, w=16, sigma=sigma.cuda()).float().cpu().numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    ref = cnn.cutouts_grid(cube.numpy(), cfg.ny, cfg.nx, cands, tab.max(axis=1), cfg.widths, 16, 16, 16,
                           sigma=sigma.numpy())
    ref_b = _bf16(ref.astype(np.float32))
    # one BF16 unit in the last place of slack for FP32-vs-FP64 rounding before the BF16 store
    np.testing.assert_allclose(out, ref_b, rtol=2 ** -7, atol=1e-6)
    plan.close()
