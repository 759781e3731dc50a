"""Multi-GPU host logic on the CPU: row bands, per-band search configurations and the candidate
gather, with two gloo ranks.  The per-band searches are the FP64 oracle's, so the merged list
must equal the oracle's list for the whole image."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2510_18136_gb300 import shard, synth

CAND = np.dtype([("row", "<i4"), ("col", "<i4"), ("dm_idx", "<i4"), ("w_idx", "<i4"), ("t_idx", "<i4"),
                 ("snr", "<f4")])


def _cube(cfg, seed):
    x = synth.plain_noise(cfg, seed)
    raw = synth.draw_injections(cfg, 6, seed + 1, dm_range=(0.0, 2000.0), snr_range=(9.0, 15.0), max_width=16,
                                min_sep=1)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, 1.0)
    synth.add_injections(x, cfg, inj, sh)
    return x.numpy()


def _oracle_candidates(cfg, cube):
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    _, best, _ = oracle.search_cube(cube, tab, cfg.widths, sigma=4.0)
    c = oracle.candidates(best, cfg.threshold)
    out = np.zeros(len(c["pix"]), CAND)
    out["row"], out["col"] = c["pix"] // cfg.nx, c["pix"] % cfg.nx
    out["dm_idx"], out["w_idx"], out["t_idx"], out["snr"] = c["dm_idx"], c["w_idx"], c["t_idx"], c["snr"]
    return out


def _config():
    return synth.SearchConfig(ny=11, nx=6, n_t=64, dm=np.linspace(0.0, 1500.0, 12),
                              widths=np.array([1, 2, 4, 8, 16], np.int32), threshold=6.0)


@pytest.mark.parametrize("ny,world", [(1, 1), (7, 2), (301, 8), (9, 4), (5, 5)])
def test_row_bands_cover_every_row_once(ny, world):
    bands = shard.row_bands(ny, world)
    assert len(bands) == world and bands[0][0] == 0 and bands[-1][1] == ny
    assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
    sizes = [r1 - r0 for r0, r1 in bands]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def test_band_searches_merge_to_the_whole_image():
    cfg = _config()
    cube = _cube(cfg, 3)
    whole = _oracle_candidates(cfg, cube)
    bands = shard.row_bands(cfg.ny, 3)
    lists = [_oracle_candidates(shard.band_config(cfg, b), cube[b[0] * cfg.nx:b[1] * cfg.nx]) for b in bands]
    merged = shard.merge_candidates(lists, bands, cfg.nx)
    assert len(whole) > 0
    np.testing.assert_array_equal(merged, whole)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = _config()
        cube = _cube(cfg, 3)
        band = shard.row_bands(cfg.ny, world)[rank]
        local = _oracle_candidates(shard.band_config(cfg, band), cube[band[0] * cfg.nx:band[1] * cfg.nx])
        merged = shard.gather_candidates(local, band, cfg.nx)
        on_dst = shard.gather_candidates(local, band, cfg.nx, dst=0)
        slowest = shard.max_over_ranks(1.0 + rank)
        q.put((rank, merged.tobytes(), None if on_dst is None else on_dst.tobytes(), slowest))
    finally:
        dist.destroy_process_group()


def test_gather_candidates_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = _config()
    whole = _oracle_candidates(cfg, _cube(cfg, 3)).tobytes()
    for rank, merged, on_dst, slowest in got:
        assert merged == whole
        assert slowest == 2.0
        assert (on_dst == whole) if rank == 0 else (on_dst is None)
