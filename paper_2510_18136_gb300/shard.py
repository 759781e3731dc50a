"""Data parallelism of the search over several GPUs (one process per GPU).

Pixels are independent, so the image is split into contiguous bands of pixel rows, one per rank;
each rank searches its band as a cube of its own (a plan with ny = band rows) and the candidate
lists are gathered on the host and merged in pixel order.  There is no device collective: the
search has no exchange step, and the gather is O(candidates).
"""
from __future__ import annotations

import numpy as np

from . import synth


def row_bands(ny: int, world: int):
    """Contiguous row bands [(r0, r1)] covering 0..ny-1 once, sizes differing by at most one."""
    if world < 1 or ny < 1:
        raise ValueError("need ny >= 1 and world >= 1")
    return [(ny * r // world, ny * (r + 1) // world) for r in range(world)]


def band_config(cfg: synth.SearchConfig, band) -> synth.SearchConfig:
    """The search configuration of one band (same subbands, DM trials, widths and threshold)."""
    r0, r1 = band
    if not 0 <= r0 < r1 <= cfg.ny:
        raise ValueError(f"band {band} outside 0..{cfg.ny}")
    return synth.SearchConfig(ny=r1 - r0, nx=cfg.nx, n_sub=cfg.n_sub, n_t=cfg.n_t, freq_mhz=cfg.freq_mhz, dm=cfg.dm,
                              widths=cfg.widths, threshold=cfg.threshold, k_dm_ms=cfg.k_dm_ms,
                              t_samp_ms=cfg.t_samp_ms)


def merge_candidates(lists, bands, nx: int) -> np.ndarray:
    """Band-local candidate lists (rows relative to their band) -> one list in image pixel order."""
    parts = []
    for cand, (r0, _) in zip(lists, bands):
        c = np.array(cand, copy=True)
        c["row"] += r0
        parts.append(c)
    if not parts:
        raise ValueError("no candidate lists")
    out = np.concatenate(parts)
    order = np.argsort(out["row"].astype(np.int64) * nx + out["col"], kind="stable")
    return out[order]


def gather_candidates(local: np.ndarray, band, nx: int, group=None, dst: int | None = None):
    """Gather every rank's band-local candidates (torch.distributed, any backend) and merge them.

    Returns the merged list on every rank (dst None) or on rank dst only (None elsewhere)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    payload = (np.ascontiguousarray(local), tuple(band))
    if dst is None:
        got = [None] * world
        dist.all_gather_object(got, payload, group=group)
    else:
        got = [None] * world if dist.get_rank(group) == dst else None
        dist.gather_object(payload, got, dst=dst, group=group)
        if got is None:
            return None
    return merge_candidates([g[0] for g in got], [g[1] for g in got], nx)


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
