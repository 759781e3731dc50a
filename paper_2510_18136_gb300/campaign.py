"""Injection campaigns of arXiv 2510.18136 Sec. 3.1-3.2, run through the GPU search.

* Threshold optimisation (Sec. 3.1): boxcar pulses with DM U(0, 4000), widths
  1-16 samples (0.134-2.14 s) and matched S/N U(0, 10), and noise-only
  realisations; the false-negative rate (missed injections) and the
  false-positive rate (noise realisations with any candidate) as functions of
  the threshold; the optimum minimises their sum.
* Detection rate (Sec. 3.2): a fixed number of injections per S/N bin at random
  trial DMs and widths; the fraction recovered above the threshold, and, with
  the classifier, the fraction also passed by it (p_rfi below a cut).

A realisation is a small image (``side`` x ``side`` pixels) of a longer cube:
many realisations are searched at once as one cube and split per pixel block.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import native, synth


def campaign_config(side: int = 32, n_real: int = 1, n_t: int = 64) -> synth.SearchConfig:
    """n_real realisations of side x side pixels stacked along rows; 16 DM on 0-4000, widths 1-16."""
    return synth.SearchConfig(ny=side * n_real, nx=side, n_t=n_t, dm=np.linspace(0.0, 4000.0, 16),
                              widths=np.array([1, 2, 4, 8, 16], np.int32), threshold=6.0)


def _shifts(cfg, dms):
    order = np.argsort(dms)
    c = synth.SearchConfig(ny=1, nx=1, n_t=cfg.n_t, freq_mhz=cfg.freq_mhz, dm=np.asarray(dms, float)[order],
                           widths=np.array([1], np.int32))
    with native.Plan(c) as p:
        sh = p.delays()
    out = np.empty_like(sh)
    out[order] = sh
    return out


def _inject(cube, cfg, rows, cols, snr, rng):
    """Boxcar pulses of matched S/N at (rows, cols); DM U(0, 4000), width log-U(1, 16)."""
    n = len(rows)
    dm = rng.uniform(0.0, 4000.0, n)
    w = np.clip(np.rint(np.exp(rng.uniform(0.0, math.log(16.0), n))).astype(int), 1, 16)
    sh = _shifts(cfg, dm)
    smax = sh.max(axis=1)
    t0 = np.array([int(rng.integers(0, max(cfg.n_t - smax[i] - w[i], 1))) for i in range(n)])
    amp = np.asarray(snr) / (math.sqrt(cfg.n_sub) * np.sqrt(w))      # unit noise per subband and sample
    idx_p, idx_k, idx_t, val = [], [], [], []
    for i in range(n):
        p = int(rows[i]) * cfg.nx + int(cols[i])
        t = t0[i] + sh[i][:, None] + np.arange(w[i])[None, :]
        ok = t < cfg.n_t
        K = np.broadcast_to(np.arange(cfg.n_sub)[:, None], t.shape)
        idx_p.append(np.full(int(ok.sum()), p)); idx_k.append(K[ok]); idx_t.append(t[ok])
        val.append(np.full(int(ok.sum()), amp[i], np.float32))
    if n:
        dev = cube.device
        cube.index_put_((torch.from_numpy(np.concatenate(idx_p)).to(dev), torch.from_numpy(np.concatenate(idx_k)).to(dev),
                         torch.from_numpy(np.concatenate(idx_t)).to(dev)),
                        torch.from_numpy(np.concatenate(val)).to(dev), accumulate=True)
    return {"dm": dm, "width": w, "t0": t0}


def _best_snr(cfg, cube):
    """Per-pixel best S/N of the GPU search (sigma_D = sqrt(n_sub): unit noise per subband)."""
    with native.Plan(cfg) as plan:
        plan.search(cube)
        snr, _ = plan.best()
    return snr


def threshold_curves(n_inj: int = 200, n_noise: int = 2000, side: int = 32, n_t: int = 64, seed: int = 0,
                     thresholds=np.linspace(0.0, 20.0, 81), batch: int = 250, device="cuda"):
    """FN and FP rates versus threshold (Sec. 3.1).  Injection S/N U(0, 10) at each realisation's
    centre pixel; its detection S/N is the best S/N of that pixel.  Noise realisations count as
    false positives when any pixel exceeds the threshold."""
    rng = np.random.default_rng(seed)
    inj_snr, det_snr, noise_max = [], [], []
    done = 0
    s = seed
    while done < n_inj:
        nb = min(batch, n_inj - done)
        cfg = campaign_config(side, nb, n_t)
        cube = synth.plain_noise(cfg, s, device=device)
        s += 1
        snr_in = rng.uniform(0.0, 10.0, nb)
        rows = np.arange(nb) * side + side // 2
        cols = np.full(nb, side // 2)
        _inject(cube, cfg, rows, cols, snr_in, rng)
        best = _best_snr(cfg, cube)
        inj_snr.append(snr_in)
        det_snr.append(best[rows * cfg.nx + cols])
        done += nb
    done = 0
    while done < n_noise:
        nb = min(batch, n_noise - done)
        cfg = campaign_config(side, nb, n_t)
        cube = synth.plain_noise(cfg, s, device=device)
        s += 1
        best = _best_snr(cfg, cube).reshape(nb, side * side)
        noise_max.append(best.max(axis=1))
        done += nb
    det = np.concatenate(det_snr)
    nmax = np.concatenate(noise_max)
    thr = np.asarray(thresholds)
    fn = np.array([(det <= t).mean() for t in thr])
    fp = np.array([(nmax > t).mean() for t in thr])
    k = int(np.argmin(fn + fp))
    return {"thresholds": thr, "fn": fn, "fp": fp, "optimum": float(thr[k]), "inj_snr": np.concatenate(inj_snr),
            "det_snr": det, "noise_max": nmax}


def detection_curve(snr_bins=np.arange(1, 41), n_per_bin: int = 50, side: int = 32, n_t: int = 64,
                    threshold: float = 6.0, seed: int = 1, device="cuda"):
    """Fraction of injections recovered with S/N above the threshold per input S/N bin (Sec. 3.2)."""
    rng = np.random.default_rng(seed)
    bins = np.asarray(snr_bins, float)
    n = len(bins) * n_per_bin
    cfg = campaign_config(side, n, n_t)
    cube = synth.plain_noise(cfg, seed + 7, device=device)
    snr_in = np.repeat(bins, n_per_bin)
    rows = np.arange(n) * side + side // 2
    cols = np.full(n, side // 2)
    _inject(cube, cfg, rows, cols, snr_in, rng)
    best = _best_snr(cfg, cube)[rows * cfg.nx + cols]
    rate = (best > threshold).reshape(len(bins), n_per_bin).mean(axis=1)
    return {"snr_bins": bins, "rate": rate, "det_snr": best}


def detection_curve_classified(clf: native.Classifier, snr_bins=np.arange(2, 41, 2), cubes_per_bin: int = 3,
                               taus=(0.15, 0.5), seed: int = 2, device="cuda"):
    """Detection rate per S/N bin for the threshold alone and with the classifier (Sec. 3.2, Fig. of
    the detection rate): bursts only, PSF-shaped on PSF noise, in the classifier's data cubes."""
    from . import clfdata
    cfg = clfdata.search_config()
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * math.sqrt(cfg.n_sub), device=device)
    out = {"snr_bins": np.asarray(snr_bins, float), "threshold": [], **{f"p<{t}": [] for t in taus}}
    with native.Plan(cfg) as plan:
        for b, s_in in enumerate(snr_bins):
            det, p = [], []
            for k in range(cubes_per_bin):
                cube, truth = clfdata.make_cube(cfg, seed * 100000 + b * 100 + k, device=device,
                                                snr=(float(s_in), float(s_in)), kinds_allowed=(clfdata.KIND_BURST,))
                plan.search(cube, sigma)
                cand = plan.candidates()
                m = clfdata.match_sources(cand, truth, cfg.nx)
                pr = np.full(len(m), np.nan)
                hit = np.nonzero(m >= 0)[0]
                if hit.size:
                    x = native.cutouts(plan, cube, native.candidates_to_device(cand[m[hit]]), 32, 32, 32, sigma=sigma)
                    pr[hit] = clfdata.p_rfi(clf, x)
                det.append(m >= 0)
                p.append(pr)
                del cube
            det, p = np.concatenate(det), np.concatenate(p)
            out["threshold"].append(float(det.mean()))
            for t in taus:
                out[f"p<{t}"].append(float((det & (np.nan_to_num(p, nan=1.0) < t)).mean()))
    return out
