"""Search at the paper's three timescales (arXiv 2510.18136 Sec. 2.2).

* 134 ms: the cube as given;
* 0.67 s: 5 samples summed, DM grid x5 (the same integer shifts apply, Sec. 2.2 footnote);
* 10.05 s: 75 samples summed, DM 0 only (the delay of DM < ~20000 stays within one sample).

Each scale is an ordinary search (``nsfrb_search``) of a time-binned cube
(``nsfrb_bin_time``); the noise of a binned sample grows by sqrt(factor).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import replace

import numpy as np
import torch

from . import native, synth


def bin_time(cube: torch.Tensor, factor: int, stream=None) -> torch.Tensor:
    """[n_pix, n_sub, n_t] (f32/bf16/f16, device) -> FP32 [n_pix, n_sub, n_t // factor] sums."""
    assert cube.is_cuda and cube.is_contiguous()
    dtype = {torch.float32: native.F32, torch.bfloat16: native.BF16, torch.float16: native.F16}[cube.dtype]
    n_pix, n_sub, n_t = cube.shape
    out = torch.empty((n_pix, n_sub, n_t // factor), dtype=torch.float32, device=cube.device)
    native._check(native.lib.nsfrb_bin_time(native._ptr(cube), dtype, n_pix * n_sub, n_t, factor, native._ptr(out),
                                            native._stream_handle(stream)), "nsfrb_bin_time")
    return out


def paper_timescales(cfg: synth.SearchConfig, widths=(1, 2, 4, 8, 16)):
    """(factor, config) for 134 ms, 0.67 s and 10.05 s with the native config's band and DM grid."""
    w = np.array(widths, np.int32)
    out = [(1, replace(cfg, widths=w[w <= cfg.n_t]))]
    for factor, dm in ((5, np.asarray(cfg.dm) * 5.0), (75, np.array([0.0]))):
        n_t = cfg.n_t // factor
        if n_t < 1:
            continue
        out.append((factor, replace(cfg, n_t=n_t, t_samp_ms=cfg.t_samp_ms * factor, dm=dm, widths=w[w <= n_t])))
    return out


def search_timescales(cube: torch.Tensor, cfg: synth.SearchConfig, sigma: torch.Tensor | None = None,
                      scales=None, dtype: str = "f32"):
    """Candidates at every timescale: list of dicts (factor, config, candidates)."""
    scales = scales or paper_timescales(cfg)
    results = []
    for factor, c in scales:
        if factor == 1:
            x, d = cube, dtype
            sg = sigma
        else:
            x, d = bin_time(cube, factor), "f32"
            sg = None if sigma is None else sigma * math.sqrt(factor)
        with native.Plan(c, dtype=d) as plan:
            plan.search(x, sg if sg is not None else torch.full((c.n_pix,), math.sqrt(c.n_sub) * math.sqrt(factor),
                                                                device=cube.device))
            results.append({"factor": factor, "config": c, "candidates": plan.candidates()})
    return results
