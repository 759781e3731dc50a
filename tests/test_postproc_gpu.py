"""Longer timescales (Sec. 2.2) and PSF clustering (Sec. 2.3) on the GPU vs plain statements."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import postproc
from paper_2510_18136_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("factor", [1, 5, 75])
def test_bin_time_matches_numpy(native, dtype, factor):
    from paper_2510_18136_gb300 import multiscale
    g = torch.Generator().manual_seed(factor)
    x = torch.randn((37, 16, 1203), generator=g).to(dtype)
    got = multiscale.bin_time(x.cuda(), factor).cpu().numpy()
    n = 1203 // factor
    ref = x.float().numpy()[:, :, :n * factor].astype(np.float64).reshape(37, 16, n, factor).sum(axis=3)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-6 * math.sqrt(factor))


def test_timescales_parity_and_wide_pulse(native):
    """A 300-sample (40 s) DM-0 pulse is best seen at the 10.05 s timescale; each scale's search of
    the binned cube equals the oracle's search of the numpy-binned cube."""
    from paper_2510_18136_gb300 import multiscale
    cfg = synth.config_full_window(6, 7, n_t=1200)
    cfg.dm = np.linspace(171.0, 4000.0, 16)
    cube = synth.plain_noise(cfg, 4)
    z = oracle.delay_table(cfg.freq_mhz, [0.0])[0]
    synth.add_pulse(cube, cfg, 3, 3, 450, 300, 0.4, z)
    res = multiscale.search_timescales(cube.cuda(), cfg)
    assert [r["factor"] for r in res] == [1, 5, 75]
    for r in res:
        c, f = r["config"], r["factor"]
        x = cube.numpy()[:, :, :c.n_t * f].astype(np.float64).reshape(cfg.n_pix, 16, c.n_t, f).sum(axis=3)
        tab = oracle.delay_table(c.freq_mhz, c.dm, c.k_dm_ms, c.t_samp_ms)
        _, best, _ = oracle.search_cube(x.astype(np.float32), tab, c.widths, sigma=4.0 * math.sqrt(f))
        parity.compare_candidates(r["candidates"], best, c.threshold, np.arange(cfg.n_pix), cfg.nx)
    wide = {r["factor"]: [float(s) for s, rr, cc in zip(r["candidates"]["snr"], r["candidates"]["row"],
                                                         r["candidates"]["col"]) if (rr, cc) == (3, 3)]
            for r in res}
    # matched: 0.4 * 16 * 300 / (4 sqrt(300)) = 27.7 in the full window; binned x75 sees 4 bins
    assert wide[75] and wide[75][0] > 20.0
    assert not wide[1] or wide[1][0] < wide[75][0]
    # the x5 timescale reuses the native shift table (DM x5, sampling x5)
    t1 = oracle.delay_table(cfg.freq_mhz, res[0]["config"].dm, cfg.k_dm_ms, res[0]["config"].t_samp_ms)
    t5 = oracle.delay_table(cfg.freq_mhz, res[1]["config"].dm, cfg.k_dm_ms, res[1]["config"].t_samp_ms)
    assert (t1 == t5).all()


@pytest.mark.parametrize("score", ["psf_mean", "lsq"])
@pytest.mark.parametrize("seed", range(6))
def test_psf_cluster_matches_plain_statement(native, seed, score):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 40))
    c = np.zeros(n, dtype=native.CANDIDATE_DTYPE)
    pix = rng.choice(64 * 64, size=n, replace=False)
    c["row"], c["col"] = pix // 64, pix % 64
    c["snr"] = np.round(rng.uniform(6, 30, n), 1)          # rounded: exact ties occur
    c["dm_idx"], c["w_idx"], c["t_idx"] = rng.integers(0, 16, n), rng.integers(0, 5, n), rng.integers(0, 25, n)
    ph, pw = (int(rng.integers(1, 20)) * 2 + 1 for _ in range(2))
    yy, xx = np.mgrid[:ph, :pw]
    psf = np.exp(-0.5 * (((yy - ph // 2) / 1.5) ** 2 + ((xx - pw // 2) / 1.5) ** 2))
    psf += 0.3 * np.exp(-0.5 * ((np.hypot(yy - ph // 2, xx - pw // 2) - 6.0) / 1.0) ** 2)   # a sidelobe ring
    psf = (psf / psf.max()).astype(np.float32)
    top, res = native.psf_cluster(c, 64, psf, percentile=90.0, top_k=10, score=score)
    rtop, best, want, mask = postproc.psf_cluster(c, 64, psf.astype(np.float64), 90.0, 10, score=score)
    assert len(top) == len(rtop)
    np.testing.assert_array_equal(top["row"] * 64 + top["col"], rtop["row"] * 64 + rtop["col"])
    assert int(res["final_rank"]) == best
    if best >= 0:
        assert float(res["weighted_snr"]) == pytest.approx(want, rel=1e-5)
        assert int(res["members"]) == mask
        assert (int(res["row"]), int(res["col"])) == (int(rtop["row"][best]), int(rtop["col"][best]))


def test_psf_cluster_picks_central_lobe(native):
    """A bright source seen through a PSF with a sidelobe ring: the search finds the main lobe and
    sidelobe pixels; the least-squares score names the main lobe, and both scores equal the plain
    statement on the searched candidates."""
    cfg = synth.SearchConfig(ny=48, nx=48, n_t=64, dm=np.array([0.0]), widths=np.array([1, 2, 4], np.int32))
    R = 10
    yy, xx = np.mgrid[-R:R + 1, -R:R + 1]
    rr = np.hypot(yy, xx)
    psf = np.exp(-0.5 * (rr / 1.0) ** 2) + 0.45 * np.exp(-0.5 * ((rr - 6.0) / 0.7) ** 2)
    psf = (psf / psf.max()).astype(np.float32)
    cube = synth.plain_noise(cfg, 2)
    r0, c0 = 24, 20
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            cube[(r0 + dy) * cfg.nx + c0 + dx, :, 30:32] += 2.0 * float(psf[dy + R, dx + R])
    with native.Plan(cfg) as plan:
        plan.search(cube.cuda())
        cand = plan.candidates()
    assert len(cand) > 3
    top, res = native.psf_cluster(cand, cfg.nx, psf, percentile=90.0, top_k=10, score="lsq")
    assert (int(res["row"]), int(res["col"])) == (r0, c0)
    for score in ("psf_mean", "lsq"):
        top, res = native.psf_cluster(cand, cfg.nx, psf, percentile=90.0, top_k=10, score=score)
        rtop, best, want, mask = postproc.psf_cluster(cand, cfg.nx, psf.astype(np.float64), 90.0, 10, score=score)
        assert int(res["final_rank"]) == best and int(res["members"]) == mask
        assert float(res["weighted_snr"]) == pytest.approx(want, rel=1e-5)
