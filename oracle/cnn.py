"""Python side of the FP64 classifier oracle (test infrastructure only).

Marshals numpy arrays to ``cnn_oracle.c``: forward/backward of the candidate
classifier (Sec. 2.3 of arXiv 2510.18136: conv blocks with batch norm, ReLU
and max-pooling, FC head with dropout, BCE, Adam) and the Philox4x32-10
generator used for dropout masks.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from .oracle import _load, _p


class _Dims(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("D", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("C0", ctypes.c_int), ("C", ctypes.c_int * 4), ("F", ctypes.c_int)]


@dataclass
class CnnDims:
    B: int
    D: int = 32
    H: int = 32
    W: int = 32
    C0: int = 16
    C: tuple = (32, 32, 64, 64)
    F: int = 32

    def c(self):
        d = _Dims(self.B, self.D, self.H, self.W, self.C0, (ctypes.c_int * 4)(*self.C), self.F)
        return d


def n_params(dims: CnnDims) -> int:
    d = dims.c()
    return int(_load().orc_cnn_n_params(ctypes.byref(d)))


def forward_backward(dims: CnnDims, params, x, labels=None, keep=None, p: float = 0.0, train: bool = True,
                     run_mean=None, run_var=None, grads: bool = True, bf16_storage: bool = False):
    """x: [B, D, H, W, C0] (channels last). Returns dict(loss, logits, grads, grad_mag, run_mean,
    run_var); grad_mag[i] is the sum of the magnitudes of the terms of gradient entry i.

    bf16_storage: the network with its pooled activations and the back-propagated
    gradients at the convolution outputs stored in bfloat16 (round to nearest even)."""
    d = dims.c()
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(x, dtype=np.float64)
    assert X.shape == (dims.B, dims.D, dims.H, dims.W, dims.C0)
    L = None if labels is None else np.ascontiguousarray(labels, dtype=np.float64)
    K = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    nc = sum(dims.C)
    rm = np.zeros(nc) if run_mean is None else np.ascontiguousarray(run_mean, dtype=np.float64).copy()
    rv = np.ones(nc) if run_var is None else np.ascontiguousarray(run_var, dtype=np.float64).copy()
    logits = np.empty(dims.B)
    G = np.empty_like(P) if (grads and train and L is not None) else None
    M = np.empty_like(P) if G is not None else None
    loss = _load().orc_cnn_forward_backward_mag(ctypes.byref(d), _p(P), _p(X), _p(L), _p(K), float(p),
                                                int(bool(train)), _p(rm), _p(rv), _p(logits), _p(G),
                                                int(bool(bf16_storage)), _p(M))
    return {"loss": loss, "logits": logits, "grads": G, "grad_mag": M, "run_mean": rm, "run_var": rv}


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def dropout_mask(B: int, F: int, p: float, step: int, seed: int):
    keep = np.empty((B, F), dtype=np.uint8)
    _load().orc_dropout_mask(B, F, float(p), int(step), int(seed), _p(keep))
    return keep


def adam(params, grads, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    _load().orc_adam(params.size, _p(params), _p(np.ascontiguousarray(grads, dtype=np.float64)), _p(m), _p(v),
                     int(t), lr, b1, b2, eps)


def layout(dims: CnnDims):
    """Slices of the flat parameter vector: list of (name, offset, shape)."""
    out, o, cin = [], 0, dims.C0
    for l in range(4):
        n = dims.C[l] * 27 * cin
        out.append((f"conv{l}.w", o, (dims.C[l], 3, 3, 3, cin)))
        o += n
        out.append((f"bn{l}.gamma", o, (dims.C[l],)))
        o += dims.C[l]
        out.append((f"bn{l}.beta", o, (dims.C[l],)))
        o += dims.C[l]
        cin = dims.C[l]
    fin = (dims.D // 16) * (dims.H // 16) * (dims.W // 16) * dims.C[3]
    for name, shape in [("fc1.w", (dims.F, fin)), ("fc1.b", (dims.F,)), ("fc2.w", (dims.F,)), ("fc2.b", (1,))]:
        out.append((name, o, shape))
        o += int(np.prod(shape))
    return out


def cutouts_grid(cube, ny, nx, cands, smax, widths, D, H, W, sigma=None):
    """As ``cutouts`` with the image shape given explicitly."""
    n_pix, n_sub, n_t = cube.shape
    out = np.zeros((len(cands), D, H, W, n_sub))
    for i, c in enumerate(cands):
        w = int(widths[int(c["w_idx"])])
        sm = int(smax[int(c["dm_idx"])])
        span = w + sm
        b = max(1, -(-span // (D // 2)))
        ts = int(c["t_idx"]) + span // 2 - (D * b) // 2
        pc = int(c["row"]) * nx + int(c["col"])
        sg = 1.0 if sigma is None else float(sigma[pc]) / np.sqrt(n_sub)
        for y in range(H):
            r = int(c["row"]) - H // 2 + y
            if r < 0 or r >= ny:
                continue
            for x in range(W):
                cc = int(c["col"]) - W // 2 + x
                if cc < 0 or cc >= nx:
                    continue
                p = r * nx + cc
                for z in range(D):
                    t0 = ts + z * b
                    lo, hi = max(t0, 0), min(t0 + b, n_t)
                    s = cube[p, :, lo:hi].astype(np.float64).sum(axis=1) if hi > lo else np.zeros(n_sub)
                    out[i, z, y, x, :] = s / b / sg
    return out
