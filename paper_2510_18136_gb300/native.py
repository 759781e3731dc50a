"""Thin ctypes binding of libnsfrb (include/nsfrb.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels; this module only
checks tensor shapes/devices, passes pointers and sizes, and converts status
codes to exceptions.  The function names follow the C ABI; ``Plan`` wraps them.
If the compiled library is missing this module raises at import: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int16, c_int32, c_int64, c_size_t, c_uint32, c_void_p

import numpy as np
import torch

from . import build as _build

F32, BF16, F16 = 0, 1, 2
NOISE_KNOWN, NOISE_MAD = 0, 1
OUT_CANDIDATES, OUT_FULL = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ETRUNC, ENOTREADY = range(7)

_DTYPES = {"f32": F32, "bf16": BF16, "f16": F16}
_TORCH = {F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}
# pixel x DM tiles of the search kernel, 10 * teams + buffers per team (NSFRB_TILES)
TILES = (12, 22, 21, 31, 41)
N_TILES = len(TILES)


class nsfrb_config(ctypes.Structure):
    _fields_ = [("ny", c_int32), ("nx", c_int32), ("n_sub", c_int32), ("n_t", c_int32),
                ("t_samp_ms", c_double), ("k_dm_ms", c_double), ("freq_mhz", POINTER(c_double)),
                ("n_dm", c_int32), ("dm", POINTER(c_double)), ("n_w", c_int32),
                ("widths", POINTER(c_int32)), ("threshold", c_float), ("dtype", c_int32),
                ("noise_mode", c_int32), ("out_mode", c_int32), ("rescore_eps", c_float)]


class nsfrb_candidate(ctypes.Structure):
    _fields_ = [("row", c_int32), ("col", c_int32), ("dm_idx", c_int32), ("w_idx", c_int32),
                ("t_idx", c_int32), ("snr", c_float)]


class nsfrb_clf_config(ctypes.Structure):
    _fields_ = [("batch", c_int32), ("d", c_int32), ("h", c_int32), ("w", c_int32), ("c0", c_int32),
                ("c", c_int32 * 4), ("f", c_int32), ("dropout", c_float), ("seed", ctypes.c_uint64),
                ("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("bn_momentum", c_float)]


class nsfrb_imager_config(ctypes.Structure):
    _fields_ = [("n_grid", c_int32), ("pixel_arcsec", c_double), ("robust", c_double), ("b_min_m", c_double),
                ("b_max_m", c_double), ("n_base", c_int32), ("uv_m", POINTER(c_double)), ("n_sub", c_int32),
                ("n_chan", c_int32), ("chan_mhz", POINTER(c_double))]


CANDIDATE_DTYPE = np.dtype([("row", "<i4"), ("col", "<i4"), ("dm_idx", "<i4"), ("w_idx", "<i4"),
                            ("t_idx", "<i4"), ("snr", "<f4")])


class NsfrbError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {lib.nsfrb_strerror(status).decode()} "
                         f"({lib.nsfrb_last_error().decode()})")
        self.status = status


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libnsfrb is not built ({path}); run paper_2510_18136_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "nsfrb_plan": ([POINTER(nsfrb_config), POINTER(c_void_p)], c_int32),
        "nsfrb_plan_delays": ([P, P], c_int32),
        "nsfrb_plan_info": ([P, POINTER(c_int32), P], c_int32),
        "nsfrb_search": ([P, P, P, P, P], c_int32),
        "nsfrb_search_host": ([P, P, P, P], c_int32),
        "nsfrb_candidates": ([P, P, c_int32, POINTER(c_int32)], c_int32),
        "nsfrb_best": ([P, P, P], c_int32),
        "nsfrb_full": ([P, P, P], c_int32),
        "nsfrb_last_timing": ([P, POINTER(c_float), POINTER(c_float)], c_int32),
        "nsfrb_plan_set_tile": ([P, c_int32, c_int32], c_int32),
        "nsfrb_plan_get_tile": ([P, c_int32, POINTER(c_int32)], c_int32),
        "nsfrb_plan_autotune": ([P, P, P, c_int32, P, POINTER(c_int32), POINTER(c_float)], c_int32),
        "nsfrb_search_static": ([P, P, P, P, c_int32, P, P], c_int32),
        "nsfrb_stream_open": ([P, c_int32, c_size_t], c_int32),
        "nsfrb_stream_bytes": ([P, c_int32, POINTER(c_size_t)], c_int32),
        "nsfrb_stream_push": ([P, P, c_uint32], c_int32),
        "nsfrb_stream_poll": ([P, c_int32, P, c_int32, POINTER(c_int32), POINTER(c_float)], c_int32),
        "nsfrb_stream_blocks": ([P, POINTER(c_int64)], c_int32),
        "nsfrb_stream_window_info": ([P, POINTER(c_int32)], c_int32),
        "nsfrb_stream_block": ([P, POINTER(c_void_p)], c_int32),
        "nsfrb_stream_push_device": ([P, c_uint32, P], c_int32),
        "nsfrb_imager_create": ([POINTER(nsfrb_imager_config), POINTER(c_void_p)], c_int32),
        "nsfrb_imager_weights": ([P, P], c_int32),
        "nsfrb_imager_info": ([P, POINTER(c_int32), POINTER(c_int32), POINTER(c_int64)], c_int32),
        "nsfrb_image": ([P, P, c_int32, P, P], c_int32),
        "nsfrb_imager_status": ([P], c_int32),
        "nsfrb_imager_destroy": ([P], None),
        "nsfrb_clf_create": ([POINTER(nsfrb_clf_config), POINTER(c_void_p)], c_int32),
        "nsfrb_clf_n_params": ([P, POINTER(c_int64)], c_int32),
        "nsfrb_clf_set_params": ([P, P], c_int32),
        "nsfrb_clf_get_params": ([P, P], c_int32),
        "nsfrb_clf_get_grads": ([P, P], c_int32),
        "nsfrb_clf_get_bn_stats": ([P, P, P], c_int32),
        "nsfrb_clf_set_bn_stats": ([P, P, P], c_int32),
        "nsfrb_clf_train_step": ([P, P, P, c_int32, c_int32, POINTER(c_float), P], c_int32),
        "nsfrb_clf_infer": ([P, P, c_int32, P, P], c_int32),
        "nsfrb_clf_cutouts": ([P, P, P, P, c_int32, c_int32, c_int32, c_int32, P, P], c_int32),
        "nsfrb_clf_save": ([P, ctypes.c_char_p], c_int32),
        "nsfrb_clf_load": ([P, ctypes.c_char_p], c_int32),
        "nsfrb_clf_destroy": ([P], None),
        "nsfrb_bin_time": ([P, c_int32, c_int64, c_int32, c_int32, P, P], c_int32),
        "nsfrb_psf_cluster": ([P, c_int32, c_int32, P, c_int32, c_int32, c_float, c_int32, c_int32, P, P, P],
                              c_int32),
        "nsfrb_dbg_gemm": ([c_int32, c_int32, c_int32, c_int32, P, P, P, P], c_int32),
        "nsfrb_dbg_conv3": ([c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, P, P, P, P, P, P, P],
                            c_int32),
        "nsfrb_dbg_wait_timeout": ([c_int32], c_int32),
        "nsfrb_dbg_mad_normalise": ([P, c_int32, c_int64, c_int32, P, P, P], c_int32),
        "nsfrb_destroy": ([P], None),
        "nsfrb_strerror": ([c_int32], ctypes.c_char_p),
        "nsfrb_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()
LIB_PATH = _build.LIB


def _check(status: int, what: str, allow=()):
    if status != OK and status not in allow:
        raise NsfrbError(status, what)
    return status


def _ptr(t: torch.Tensor | None):
    return None if t is None else c_void_p(t.data_ptr())


def _stream_handle(stream) -> c_void_p | None:
    if stream is None:
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


class Plan:
    """One search configuration (``nsfrb_plan``) and its device workspace."""

    def __init__(self, cfg, dtype: str = "f32", noise: str = "known", out: str = "candidates",
                 rescore_eps: float = 0.0):
        self.cfg = cfg
        self.dtype = _DTYPES[dtype]
        self._freq = np.ascontiguousarray(cfg.freq_mhz, dtype=np.float64)
        self._dm = np.ascontiguousarray(cfg.dm, dtype=np.float64)
        self._w = np.ascontiguousarray(cfg.widths, dtype=np.int32)
        c = nsfrb_config()
        c.ny, c.nx, c.n_sub, c.n_t = cfg.ny, cfg.nx, cfg.n_sub, cfg.n_t
        c.t_samp_ms, c.k_dm_ms = cfg.t_samp_ms, cfg.k_dm_ms
        c.freq_mhz = self._freq.ctypes.data_as(POINTER(c_double))
        c.n_dm = self._dm.size
        c.dm = self._dm.ctypes.data_as(POINTER(c_double))
        c.n_w = self._w.size
        c.widths = self._w.ctypes.data_as(POINTER(c_int32))
        c.threshold = float(cfg.threshold)
        c.dtype = self.dtype
        c.noise_mode = NOISE_MAD if noise == "mad" else NOISE_KNOWN
        c.out_mode = OUT_FULL if out == "full" else OUT_CANDIDATES
        c.rescore_eps = float(rescore_eps)
        self.noise_mode = c.noise_mode
        self.out_mode = c.out_mode
        h = c_void_p()
        _check(lib.nsfrb_plan(ctypes.byref(c), ctypes.byref(h)), "nsfrb_plan")
        self._h = h

    # ------------------------------------------------------------------ plan info
    @property
    def handle(self):
        return self._h

    def delays(self) -> np.ndarray:
        out = np.empty((self._dm.size, self.cfg.n_sub), dtype=np.int32)
        _check(lib.nsfrb_plan_delays(self._h, out.ctypes.data_as(c_void_p)), "nsfrb_plan_delays")
        return out

    def info(self):
        n_u = c_int32()
        smax = np.empty(self._dm.size, dtype=np.int32)
        _check(lib.nsfrb_plan_info(self._h, ctypes.byref(n_u), smax.ctypes.data_as(c_void_p)),
               "nsfrb_plan_info")
        return int(n_u.value), smax

    # ------------------------------------------------------------------ search
    def _check_cube(self, cube: torch.Tensor, dtype: int, device: str):
        cfg = self.cfg
        if tuple(cube.shape) != (cfg.n_pix, cfg.n_sub, cfg.n_t):
            raise ValueError(f"cube shape {tuple(cube.shape)} != {(cfg.n_pix, cfg.n_sub, cfg.n_t)}")
        if cube.dtype != _TORCH[dtype]:
            raise ValueError(f"cube dtype {cube.dtype} != {_TORCH[dtype]}")
        if not cube.is_contiguous():
            raise ValueError("cube must be contiguous")
        if (cube.device.type == "cuda") != (device == "cuda"):
            raise ValueError(f"cube must be on {device}")

    def search(self, cube: torch.Tensor, sigma: torch.Tensor | None = None,
               cube_f32: torch.Tensor | None = None, stream=None) -> None:
        """``nsfrb_search`` on a device cube [n_pix, n_sub, n_t] (asynchronous)."""
        self._check_cube(cube, self.dtype, "cuda")
        if sigma is not None:
            assert sigma.is_cuda and sigma.dtype == torch.float32 and sigma.numel() == self.cfg.n_pix
            assert sigma.is_contiguous()
        if cube_f32 is not None:
            self._check_cube(cube_f32, F32, "cuda")
        _check(lib.nsfrb_search(self._h, _ptr(cube), _ptr(sigma), _ptr(cube_f32),
                                _stream_handle(stream)), "nsfrb_search")

    def search_host(self, cube: torch.Tensor, sigma: torch.Tensor | None = None, stream=None) -> None:
        """``nsfrb_search_host`` on a host cube (pinned for full copy speed)."""
        self._check_cube(cube, self.dtype, "cpu")
        if sigma is not None:
            assert not sigma.is_cuda and sigma.dtype == torch.float32 and sigma.is_contiguous()
        _check(lib.nsfrb_search_host(self._h, _ptr(cube), _ptr(sigma), _stream_handle(stream)),
               "nsfrb_search_host")

    def candidates(self, cap: int | None = None) -> np.ndarray:
        """``nsfrb_candidates``: structured array (row, col, dm_idx, w_idx, t_idx, snr)."""
        n = c_int32()
        cap = self.cfg.n_pix if cap is None else int(cap)
        out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
        st = lib.nsfrb_candidates(self._h, out.ctypes.data_as(c_void_p), cap, ctypes.byref(n))
        _check(st, "nsfrb_candidates")
        return out[: n.value]

    def best(self):
        """``nsfrb_best``: per-pixel S/N [n_pix] and (dm_idx, w_idx, t_idx) [n_pix, 3]."""
        snr = np.empty(self.cfg.n_pix, dtype=np.float32)
        idx = np.empty((self.cfg.n_pix, 3), dtype=np.int32)
        _check(lib.nsfrb_best(self._h, snr.ctypes.data_as(c_void_p), idx.ctypes.data_as(c_void_p)),
               "nsfrb_best")
        return snr, idx

    def full(self):
        """``nsfrb_full``: S/N and t_idx [n_pix, n_dm, n_w] as numpy arrays."""
        shape = (self.cfg.n_pix, self._dm.size, self._w.size)
        snr = np.empty(shape, dtype=np.float32)
        t = np.empty(shape, dtype=np.int16)
        _check(lib.nsfrb_full(self._h, snr.ctypes.data_as(c_void_p), t.ctypes.data_as(c_void_p)),
               "nsfrb_full")
        return snr, t

    def last_timing(self):
        """``nsfrb_last_timing``: (search-kernel ms, total queued ms) of the last search."""
        a, b = c_float(), c_float()
        _check(lib.nsfrb_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)), "nsfrb_last_timing")
        return float(a.value), float(b.value)

    # ------------------------------------------------------------------ kernel tile
    def set_tile(self, dtype: int, tile: int) -> None:
        """``nsfrb_plan_set_tile``: preferred (10 * teams + buffers) tile for rows stored as dtype."""
        _check(lib.nsfrb_plan_set_tile(self._h, int(dtype), int(tile)), "nsfrb_plan_set_tile")

    def get_tile(self, dtype: int) -> int:
        t = c_int32()
        _check(lib.nsfrb_plan_get_tile(self._h, int(dtype), ctypes.byref(t)), "nsfrb_plan_get_tile")
        return int(t.value)

    def autotune(self, cube: torch.Tensor, sigma: torch.Tensor | None = None, reps: int = 3, stream=None):
        """``nsfrb_plan_autotune``: (chosen tile, {tile: median search ms} of the tiles that fit)."""
        self._check_cube(cube, self.dtype, "cuda")
        if sigma is not None:
            assert sigma.is_cuda and sigma.dtype == torch.float32 and sigma.numel() == self.cfg.n_pix
        tile = c_int32()
        ms = (c_float * N_TILES)()
        _check(lib.nsfrb_plan_autotune(self._h, _ptr(cube), _ptr(sigma), int(reps), _stream_handle(stream),
                                       ctypes.byref(tile), ms), "nsfrb_plan_autotune")
        return int(tile.value), {t: float(m) for t, m in zip(TILES, ms) if m >= 0}

    # ------------------------------------------------------------------ serving
    def stream_bytes(self, n_blk: int) -> int:
        b = c_size_t()
        _check(lib.nsfrb_stream_bytes(self._h, int(n_blk), ctypes.byref(b)), "nsfrb_stream_bytes")
        return int(b.value)

    def stream_open(self, n_blk: int, hbm_reserve: int = 0) -> None:
        _check(lib.nsfrb_stream_open(self._h, int(n_blk), int(hbm_reserve)), "nsfrb_stream_open")
        self._n_blk = int(n_blk)

    def stream_push(self, block: torch.Tensor, present_mask: int | None = None) -> None:
        """Push one block [n_blk, n_sub, ny, nx] FP32 (host memory)."""
        cfg = self.cfg
        assert not block.is_cuda and block.dtype == torch.float32 and block.is_contiguous()
        assert block.shape[1:] == (cfg.n_sub, cfg.ny, cfg.nx)
        mask = (1 << cfg.n_sub) - 1 if present_mask is None else int(present_mask)
        _check(lib.nsfrb_stream_push(self._h, _ptr(block), c_uint32(mask)), "nsfrb_stream_push")

    def stream_poll(self, timeout_ms: int = 3350, cap: int | None = None):
        """Returns (candidates, latency_ms) or raises NsfrbError(ETIMEOUT)."""
        n = c_int32()
        lat = c_float()
        cap = self.cfg.n_pix if cap is None else int(cap)
        out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
        _check(lib.nsfrb_stream_poll(self._h, int(timeout_ms), out.ctypes.data_as(c_void_p), cap,
                                     ctypes.byref(n), ctypes.byref(lat)), "nsfrb_stream_poll")
        return out[: n.value], float(lat.value)

    def stream_window_info(self) -> int:
        """``nsfrb_stream_window_info``: 1 re-score FP32 window in device memory, 2 in pinned host
        memory, 0 none."""
        v = c_int32()
        _check(lib.nsfrb_stream_window_info(self._h, ctypes.byref(v)), "nsfrb_stream_window_info")
        return int(v.value)

    def stream_blocks(self) -> int:
        n = c_int64()
        _check(lib.nsfrb_stream_blocks(self._h, ctypes.byref(n)), "nsfrb_stream_blocks")
        return int(n.value)

    def stream_block(self) -> torch.Tensor:
        """The stream's device block buffer [n_blk, n_sub, ny, nx] FP32 (a view; owned by the plan)."""
        ptr = c_void_p()
        _check(lib.nsfrb_stream_block(self._h, ctypes.byref(ptr)), "nsfrb_stream_block")
        c = self.cfg
        return _device_view(ptr.value, (self._n_blk, c.n_sub, c.ny, c.nx))

    def stream_push_device(self, present_mask: int | None = None, stream=None) -> None:
        """Queue the block already written into ``stream_block()`` by work on ``stream``."""
        m = (1 << self.cfg.n_sub) - 1 if present_mask is None else int(present_mask)
        _check(lib.nsfrb_stream_push_device(self._h, c_uint32(m), _stream_handle(stream)),
               "nsfrb_stream_push_device")

    # ------------------------------------------------------------------ lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.nsfrb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Classifier:
    """Candidate classifier (``nsfrb_clf_*``): BF16 CNN trained and run by the library's kernels."""

    def __init__(self, batch: int, d: int = 32, h: int = 32, w: int = 32, c0: int = 16,
                 c=(32, 32, 64, 64), f: int = 32, dropout: float = 0.5, seed: int = 1, lr: float = 1e-3,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, bn_momentum: float = 0.1):
        cfg = nsfrb_clf_config()
        cfg.batch, cfg.d, cfg.h, cfg.w, cfg.c0 = batch, d, h, w, c0
        cfg.c = (c_int32 * 4)(*c)
        cfg.f, cfg.dropout, cfg.seed = f, dropout, seed
        cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, cfg.bn_momentum = lr, beta1, beta2, eps, bn_momentum
        self.shape = (d, h, w, c0)
        self.batch = batch
        self.n_bn = int(sum(c))
        hd = c_void_p()
        _check(lib.nsfrb_clf_create(ctypes.byref(cfg), ctypes.byref(hd)), "nsfrb_clf_create")
        self._h = hd
        n = c_int64()
        _check(lib.nsfrb_clf_n_params(self._h, ctypes.byref(n)), "nsfrb_clf_n_params")
        self.n_params = int(n.value)

    def set_params(self, p: np.ndarray) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(lib.nsfrb_clf_set_params(self._h, p.ctypes.data_as(c_void_p)), "nsfrb_clf_set_params")

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib.nsfrb_clf_get_params(self._h, out.ctypes.data_as(c_void_p)), "nsfrb_clf_get_params")
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib.nsfrb_clf_get_grads(self._h, out.ctypes.data_as(c_void_p)), "nsfrb_clf_get_grads")
        return out

    def bn_stats(self):
        m = np.empty(self.n_bn, dtype=np.float32)
        v = np.empty(self.n_bn, dtype=np.float32)
        _check(lib.nsfrb_clf_get_bn_stats(self._h, m.ctypes.data_as(c_void_p), v.ctypes.data_as(c_void_p)),
               "nsfrb_clf_get_bn_stats")
        return m, v

    def set_bn_stats(self, m, v) -> None:
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        _check(lib.nsfrb_clf_set_bn_stats(self._h, m.ctypes.data_as(c_void_p), v.ctypes.data_as(c_void_p)),
               "nsfrb_clf_set_bn_stats")

    def train_step(self, x: torch.Tensor, labels: torch.Tensor, update: bool = True, stream=None,
                   want_loss: bool = True) -> float | None:
        """x: [B, d, h, w, c0] bf16 (device); labels [B] float32 (device)."""
        assert x.is_cuda and x.dtype == torch.bfloat16 and x.is_contiguous() and tuple(x.shape[1:]) == self.shape
        assert labels.is_cuda and labels.dtype == torch.float32 and labels.numel() == x.shape[0]
        loss = c_float()
        _check(lib.nsfrb_clf_train_step(self._h, _ptr(x), _ptr(labels), int(x.shape[0]), int(bool(update)),
                                        ctypes.byref(loss) if want_loss else None, _stream_handle(stream)),
               "nsfrb_clf_train_step")
        return float(loss.value) if want_loss else None

    def infer(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        """Logits [B] (device float32); p_rfi = sigmoid(logit)."""
        assert x.is_cuda and x.dtype == torch.bfloat16 and x.is_contiguous() and tuple(x.shape[1:]) == self.shape
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(lib.nsfrb_clf_infer(self._h, _ptr(x), int(x.shape[0]), _ptr(out), _stream_handle(stream)),
               "nsfrb_clf_infer")
        return out

    def save(self, path: str) -> None:
        _check(lib.nsfrb_clf_save(self._h, path.encode()), "nsfrb_clf_save")

    def load(self, path: str) -> None:
        _check(lib.nsfrb_clf_load(self._h, path.encode()), "nsfrb_clf_load")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.nsfrb_clf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cutouts(plan: "Plan", cube: torch.Tensor, cands: torch.Tensor, d: int = 32, h: int = 32, w: int = 32,
            sigma: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """``nsfrb_clf_cutouts``: cands is a device int32 tensor [n, 6] in nsfrb_candidate layout."""
    n = int(cands.shape[0])
    out = torch.empty((n, d, h, w, plan.cfg.n_sub), dtype=torch.bfloat16, device=cube.device)
    _check(lib.nsfrb_clf_cutouts(plan.handle, _ptr(cube), _ptr(sigma), _ptr(cands), n, d, h, w, _ptr(out),
                                 _stream_handle(stream)), "nsfrb_clf_cutouts")
    return out


class _CudaArray:
    """Minimal __cuda_array_interface__ holder: lets torch view library-owned device memory."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape), "typestr": "<f4",
                                         "version": 3, "strides": None}


def _device_view(ptr: int, shape) -> torch.Tensor:
    return torch.as_tensor(_CudaArray(ptr, shape), device="cuda")


class Imager:
    """``nsfrb_imager_*``: Briggs-weighted gridding + shifted inverse FFT (Sec. 2.1) on the GPU."""

    def __init__(self, uv_m: np.ndarray, chan_mhz: np.ndarray, n_grid: int = 175, pixel_arcsec: float = 10.3,
                 robust: float = -2.0, b_min_m: float = 20.0, b_max_m: float = 485.0):
        self._uv = np.ascontiguousarray(uv_m, dtype=np.float64)
        self._ch = np.ascontiguousarray(chan_mhz, dtype=np.float64)
        self.n_sub, self.n_chan = self._ch.shape
        self.n_base = self._uv.shape[0]
        self.n_grid = int(n_grid)
        c = nsfrb_imager_config(self.n_grid, float(pixel_arcsec), float(robust), float(b_min_m), float(b_max_m),
                                self.n_base, self._uv.ctypes.data_as(POINTER(c_double)), self.n_sub, self.n_chan,
                                self._ch.ctypes.data_as(POINTER(c_double)))
        h = c_void_p()
        _check(lib.nsfrb_imager_create(ctypes.byref(c), ctypes.byref(h)), "nsfrb_imager_create")
        self._h = h

    def weights(self) -> np.ndarray:
        out = np.empty((self.n_sub, self.n_chan, self.n_base), np.float32)
        _check(lib.nsfrb_imager_weights(self._h, out.ctypes.data_as(c_void_p)), "nsfrb_imager_weights")
        return out

    def info(self):
        u, v, n = c_int32(), c_int32(), c_int64()
        _check(lib.nsfrb_imager_info(self._h, ctypes.byref(u), ctypes.byref(v), ctypes.byref(n)), "nsfrb_imager_info")
        return int(u.value), int(v.value), int(n.value)

    def image(self, vis: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """vis: complex64 [n_t, n_sub, n_chan, n_base, 2] (or its float32 view [..., 2, 2]) on the GPU."""
        if vis.is_complex():
            vis = torch.view_as_real(vis)
        shape = (self.n_sub, self.n_chan, self.n_base, 2, 2)
        if vis.dtype != torch.float32 or not vis.is_cuda or not vis.is_contiguous() or tuple(vis.shape[1:]) != shape:
            raise ValueError(f"visibilities must be contiguous CUDA float32 [n_t, {shape}]")
        n_t = vis.shape[0]
        N = self.n_grid
        if out is None:
            out = torch.empty((n_t, self.n_sub, N, N), dtype=torch.float32, device=vis.device)
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() != n_t * self.n_sub * N * N:
            raise ValueError("out must be contiguous CUDA float32 [n_t, n_sub, N, N]")
        _check(lib.nsfrb_image(self._h, _ptr(vis), n_t, _ptr(out), _stream_handle(stream)), "nsfrb_image")
        return out

    def status(self) -> None:
        """Synchronous: raises NsfrbError(ETIMEOUT) if a kernel's bulk copy timed out."""
        _check(lib.nsfrb_imager_status(self._h), "nsfrb_imager_status")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.nsfrb_imager_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def candidates_to_device(cand: np.ndarray, device="cuda") -> torch.Tensor:
    """Structured candidate array -> device int32 [n, 6] in nsfrb_candidate layout."""
    raw = np.ascontiguousarray(cand).view(np.int32).reshape(-1, 6)
    return torch.from_numpy(raw.copy()).to(device)


CLUSTER_DTYPE = np.dtype([("row", "<i4"), ("col", "<i4"), ("dm_idx", "<i4"), ("w_idx", "<i4"), ("t_idx", "<i4"),
                          ("snr", "<f4"), ("weighted_snr", "<f4"), ("n_top", "<i4"), ("final_rank", "<i4"),
                          ("members", "<u4")])


CLUSTER_SCORES = {"psf_mean": 0, "lsq": 1}


def psf_cluster(cand: np.ndarray, nx: int, psf: np.ndarray, percentile: float = 90.0, top_k: int = 10,
                score: str = "psf_mean", device="cuda", stream=None):
    """``nsfrb_psf_cluster`` on a candidate list: returns (top list, result record).
    score: "psf_mean" (sum psf snr / sum psf) or "lsq" (sum psf snr / sum psf^2)."""
    d_cand = candidates_to_device(cand, device) if len(cand) else torch.zeros((1, 6), dtype=torch.int32,
                                                                               device=device)
    d_psf = torch.as_tensor(np.ascontiguousarray(psf, dtype=np.float32)).to(device)
    d_top = torch.zeros((top_k, 6), dtype=torch.int32, device=device)
    d_res = torch.zeros(10, dtype=torch.int32, device=device)
    _check(lib.nsfrb_psf_cluster(_ptr(d_cand), len(cand), int(nx), _ptr(d_psf), psf.shape[0], psf.shape[1],
                                 float(percentile), int(top_k), CLUSTER_SCORES[score], _ptr(d_top), _ptr(d_res),
                                 _stream_handle(stream)),
           "nsfrb_psf_cluster")
    torch.cuda.synchronize()
    res = d_res.cpu().numpy().view(CLUSTER_DTYPE)[0]
    n_top = int(res["n_top"])
    top = d_top[:n_top].cpu().numpy().copy().view(CANDIDATE_DTYPE).reshape(-1)
    return top, res
