"""Python side of the FP64 oracle (test infrastructure only).

The arithmetic lives in ``nsfrb_oracle.c`` (built here with gcc, OpenMP);
this module marshals numpy arrays and derives the per-pixel results:

* ``delay_table``      -- Sec. 2.2 pre-computed integer shifts, cold-plasma law.
* ``mad_normalise``    -- Sec. 2.2 median subtraction + robust noise scaling.
* ``search``           -- Sec. 2.2 de-disperse -> boxcar -> S/N -> max over t.
* ``pixel_best``       -- maximum over DM and width with the (d, w, t)
                          lexicographic tie rule, and its near-tie margin.
* ``candidates``       -- Sec. 2.2 / Fig. 1 threshold: S/N strictly above thr.
* ``brute_force_search`` -- pure-Python direct sums for tiny cubes.

Nothing here imports the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsfrb_oracle.c")
_SRC_CNN = os.path.join(_HERE, "cnn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "delay_table", "mad_normalise", "search", "pixel_best",
    "candidates", "brute_force_search", "search_cube", "unique_row_ids",
    "bf16_round", "f16_round",
]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_CNN))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off",
                               _SRC, _SRC_CNN, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_delay_table.argtypes = [ctypes.c_int, P, ctypes.c_int, P,
                                            ctypes.c_double, ctypes.c_double, P]
            lib.orc_delay_table.restype = ctypes.c_int
            lib.orc_mad_normalise.argtypes = [ctypes.c_int64, ctypes.c_int, P, P]
            lib.orc_mad_normalise.restype = ctypes.c_int64
            lib.orc_search.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P,
                                       ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int,
                                       P, P, P]
            lib.orc_search.restype = None
            lib.orc_cnn_n_params.argtypes = [P]
            lib.orc_cnn_n_params.restype = ctypes.c_int64
            lib.orc_cnn_forward_backward.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_int,
                                                     P, P, P, P]
            lib.orc_cnn_forward_backward.restype = ctypes.c_double
            lib.orc_cnn_forward_backward_ex.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_int,
                                                        P, P, P, P, ctypes.c_int]
            lib.orc_cnn_forward_backward_ex.restype = ctypes.c_double
            lib.orc_cnn_forward_backward_mag.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_int,
                                                         P, P, P, P, ctypes.c_int, P]
            lib.orc_cnn_forward_backward_mag.restype = ctypes.c_double
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_dropout_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint32,
                                             ctypes.c_uint64, P]
            lib.orc_dropout_mask.restype = None
            lib.orc_adam.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.orc_adam.restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def delay_table(freq_mhz, dm, k_dm_ms: float = 4.149, t_samp_ms: float = 134.2) -> np.ndarray:
    """Integer shift table [n_dm, n_sub] (Sec. 2.2; cold-plasma delay law)."""
    f = np.ascontiguousarray(freq_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dm, dtype=np.float64)
    out = np.empty((d.size, f.size), dtype=np.int32)
    rc = _load().orc_delay_table(f.size, _p(f), d.size, _p(d), float(k_dm_ms),
                                 float(t_samp_ms), _p(out))
    if rc != 0:
        raise ValueError("invalid delay-table arguments")
    return out


def mad_normalise(x: np.ndarray):
    """Per-(pixel, subband) (x - median) / (1.4826 MAD) over time, FP64.

    x: [..., n_t].  Returns (y float64, number of rows with MAD == 0).
    """
    x64 = np.ascontiguousarray(x, dtype=np.float64)
    n_t = x64.shape[-1]
    y = np.empty_like(x64)
    nbad = _load().orc_mad_normalise(x64.size // n_t, n_t, _p(x64), _p(y))
    return y, int(nbad)


def search(x, sigma, shifts, widths, t_lo=None, direct: bool = False):
    """De-disperse, boxcar, S/N and max over time for every (pixel, DM, width).

    x: [n, n_sub, n_t] (any float dtype; widened to FP64), sigma: [n] noise of
    the de-dispersed series.  Returns dict of snr/tidx/snr2 arrays [n, n_dm, n_w].
    """
    x64 = np.ascontiguousarray(x, dtype=np.float64)
    n, n_sub, n_t = x64.shape
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n,)))
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    ws = np.ascontiguousarray(widths, dtype=np.int32)
    n_dm, n_w = sh.shape[0], ws.size
    assert sh.shape[1] == n_sub
    tl = None if t_lo is None else np.ascontiguousarray(t_lo, dtype=np.int32).reshape(n_dm, n_w)
    snr = np.empty((n, n_dm, n_w), dtype=np.float64)
    tidx = np.empty((n, n_dm, n_w), dtype=np.int32)
    snr2 = np.empty((n, n_dm, n_w), dtype=np.float64)
    _load().orc_search(n, n_sub, n_t, _p(x64), _p(sg), n_dm, _p(sh), n_w, _p(ws),
                       _p(tl), int(bool(direct)), _p(snr), _p(tidx), _p(snr2))
    return {"snr": snr, "tidx": tidx, "snr2": snr2}


def unique_row_ids(shifts) -> np.ndarray:
    """For each DM trial, the index of the first trial with an identical shift row."""
    sh = np.asarray(shifts)
    ids = np.empty(sh.shape[0], dtype=np.int64)
    seen = {}
    for d in range(sh.shape[0]):
        key = sh[d].tobytes()
        ids[d] = seen.setdefault(key, d)
    return ids


def pixel_best(res, shifts):
    """Per-pixel maximum over (DM, width) with the (d, w, t) lexicographic tie rule.

    Returns dict with snr, dm_idx, w_idx, t_idx and margin: the best S/N minus
    the best S/N of any trial that is not the same trial (trials of DM rows
    with identical shift tables are the same trial).
    """
    snr, tidx, snr2 = res["snr"], res["tidx"], res["snr2"]
    n, n_dm, n_w = snr.shape
    flat = snr.reshape(n, -1)
    # argmax returns the first occurrence in (d, w) row-major order -> smallest d, then w
    k = np.argmax(flat, axis=1)
    best = flat[np.arange(n), k]
    bd, bw = k // n_w, k % n_w
    bt = tidx[np.arange(n), bd, bw]
    rows = unique_row_ids(shifts)
    margin = np.empty(n, dtype=np.float64)
    for p in range(n):
        same = (rows == rows[bd[p]])
        mask = np.ones((n_dm, n_w), dtype=bool)
        mask[same, bw[p]] = False
        other = snr[p][mask].max() if mask.any() else -np.inf
        other = max(other, snr2[p, bd[p], bw[p]])
        margin[p] = best[p] - other
    return {"snr": best, "dm_idx": bd.astype(np.int32), "w_idx": bw.astype(np.int32),
            "t_idx": bt.astype(np.int32), "margin": margin}


def candidates(best, threshold: float, pix=None):
    """Pixels whose best S/N is strictly above the threshold, ordered by pixel index."""
    sel = np.nonzero(best["snr"] > threshold)[0]
    pix = np.arange(best["snr"].size) if pix is None else np.asarray(pix)
    return {"pix": pix[sel], "snr": best["snr"][sel], "dm_idx": best["dm_idx"][sel],
            "w_idx": best["w_idx"][sel], "t_idx": best["t_idx"][sel],
            "margin": best["margin"][sel]}


def search_cube(cube, shifts, widths, sigma=None, pix=None, mad: bool = False,
                t_lo=None, direct: bool = False):
    """Full oracle on (a subset of) a pixel-major cube [n_pix, n_sub, n_t].

    sigma: per-pixel noise of the de-dispersed series (array or scalar); for
    mad=True it is sqrt(n_sub) after normalisation.  Returns (res, best, bad)
    where bad counts rows with zero MAD.
    """
    cube = np.asarray(cube)
    n_pix, n_sub, n_t = cube.shape
    pix = np.arange(n_pix) if pix is None else np.asarray(pix, dtype=np.int64)
    x = np.asarray(cube[pix], dtype=np.float64)
    bad = 0
    if mad:
        x, bad = mad_normalise(x)
        sg = np.full(pix.size, np.sqrt(n_sub))
    elif sigma is None:
        sg = np.full(pix.size, np.sqrt(n_sub))
    else:
        s = np.asarray(sigma, dtype=np.float64)
        sg = np.full(pix.size, float(s)) if s.ndim == 0 else s[pix]
    res = search(x, sg, shifts, widths, t_lo=t_lo, direct=direct)
    return res, pixel_best(res, shifts), bad


def brute_force_search(x, sigma, shifts, widths):
    """Pure-Python enumeration of every (pixel, d, w, t) trial; tiny cubes only.

    Returns snr [n, n_dm, n_w] and tidx with the same conventions as ``search``.
    """
    x = np.asarray(x, dtype=np.float64)
    n, n_sub, n_t = x.shape
    n_dm, n_w = len(shifts), len(widths)
    snr = np.full((n, n_dm, n_w), -np.inf)
    tidx = np.full((n, n_dm, n_w), -1, dtype=np.int32)
    for p in range(n):
        sg = float(np.broadcast_to(sigma, (n,))[p])
        for d in range(n_dm):
            s = [int(v) for v in shifts[d]]
            L = n_t - max(s)
            for wi, w in enumerate(widths):
                for t in range(0, L - w + 1):
                    b = 0.0
                    for u in range(t, t + w):
                        for k in range(n_sub):
                            b += float(x[p, k, u + s[k]])
                    v = b / (sg * float(w) ** 0.5)
                    if v > snr[p, d, wi]:
                        snr[p, d, wi] = v
                        tidx[p, d, wi] = t
    return snr, tidx


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def f16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to IEEE half (nearest-even); returned as float32."""
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float32)
