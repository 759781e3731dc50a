"""Comparison helpers: CUDA results against the FP64 oracle.

Tolerance (FP32 arithmetic): |S/N_gpu - S/N_oracle| <= REL * max(1, |S/N_oracle|).
Indices must be identical wherever the oracle's near-tie margin exceeds twice
that tolerance; inside the margin the GPU choice must itself reach the
maximum within tolerance (checked with a direct FP64 sum).
"""
import math

import numpy as np

REL = 1e-5

# Stated S/N error of the 16-bit (BF16) storage form against the FP64 search of the FP32 input,
# |S/N_bf16 - S/N_fp64| <= EPS_ABS + EPS_REL * |S/N|.  Rounding each stored sample to 8
# significand bits (unit roundoff 2^-8) adds noise of about 2^-8 rms(x) / sqrt(3) per sample to the
# sums, i.e. about 2e-3 in S/N per trial for unit noise; its maximum over a full-size cube is about
# 1e-2, and EPS_ABS = 0.03 covers that three times.  With MAD normalisation the median and MAD are
# taken from the rounded samples, so the normalisation scale, and with it every S/N of the pixel,
# carries up to about one unit roundoff of relative error: EPS_REL = 2^-7 there.
BF16_EPS = {"known": (0.03, 0.0), "mad": (0.03, 2.0 ** -7)}


def bf16_bound(snr, noise="known"):
    a, r = BF16_EPS[noise]
    return a + r * np.abs(np.asarray(snr, dtype=np.float64))


def tol(snr, rel=REL):
    return rel * np.maximum(1.0, np.abs(snr))


def direct_snr(x, sigma, shifts_row, w, t):
    """FP64 S/N of one trial by a direct sum (used only to validate near-tie choices)."""
    n_sub = x.shape[0]
    b = 0.0
    for k in range(n_sub):
        b += float(np.asarray(x[k, t + shifts_row[k]: t + shifts_row[k] + w], dtype=np.float64).sum())
    return b / (sigma * math.sqrt(w))


def compare_full(g_snr, g_t, res, rel=REL, x=None, sigma=None, shifts=None, widths=None):
    """FULL-mode arrays [n, n_dm, n_w] vs oracle ``search`` output. Returns stats."""
    o_snr, o_t, o_2 = res["snr"], res["tidx"], res["snr2"]
    fin = np.isfinite(o_snr)
    assert (np.isfinite(g_snr) == fin).all(), "finite pattern differs"
    assert (g_t[~fin] == -1).all()
    t = tol(o_snr, rel)
    err = np.abs(g_snr.astype(np.float64) - o_snr)
    err[~fin] = 0.0
    bad = err > t
    assert not bad.any(), f"{bad.sum()} S/N beyond tolerance; worst {np.max(err / np.where(fin, t, 1))} x tol"
    clear = fin & ((o_snr - o_2) > 2 * t)
    mism = clear & (g_t != o_t)
    assert not mism.any(), f"{mism.sum()} t_idx differ where the margin is clear"
    amb = fin & ~clear & (g_t != o_t)
    if amb.any() and x is not None:
        for p, d, wi in zip(*np.nonzero(amb)):
            s = direct_snr(x[p], float(np.broadcast_to(sigma, (x.shape[0],))[p]), shifts[d], int(widths[wi]),
                           int(g_t[p, d, wi]))
            assert abs(s - o_snr[p, d, wi]) <= 2 * t[p, d, wi]
    return {"max_err_over_tol": float(np.max(err / np.where(fin, t, 1.0))), "ambiguous": int(amb.sum()),
            "max_abs_err": float(err.max())}


def compare_best(g_snr, g_idx, best, rel=REL):
    """Per-pixel best (S/N, (dm, w, t)) vs oracle ``pixel_best``."""
    o = best["snr"]
    fin = np.isfinite(o)
    assert (np.isfinite(g_snr) == fin).all()
    t = tol(o, rel)
    err = np.abs(g_snr.astype(np.float64) - o)
    err[~fin] = 0
    assert (err <= t).all(), f"worst {np.max(err / t)} x tol"
    clear = fin & (best["margin"] > 2 * t)
    o_idx = np.stack([best["dm_idx"], best["w_idx"], best["t_idx"]], axis=1)
    mism = clear & (g_idx != o_idx).any(axis=1)
    assert not mism.any(), f"{mism.sum()} pixels with differing indices (clear margin): " \
                           f"{np.nonzero(mism)[0][:5]} gpu {g_idx[mism][:3]} oracle {o_idx[mism][:3]}"
    return {"max_err_over_tol": float(np.max(err / t)), "near_ties": int((fin & ~clear).sum())}


def compare_candidates(g_cand, best, threshold, pix, nx, rel=REL):
    """Candidate lists: same pixels (outside the threshold band), same S/N, same indices."""
    o = best["snr"]
    t = tol(o, rel)
    band = np.abs(o - threshold) <= t
    o_pix = set(int(p) for p, s, b in zip(pix, o, band) if s > threshold and not b)
    band_pix = set(int(p) for p, b in zip(pix, band) if b)
    g_pix = [int(r) * nx + int(c) for r, c in zip(g_cand["row"], g_cand["col"])]
    assert g_pix == sorted(g_pix), "candidate list not ordered by pixel"
    g_set = set(g_pix) & set(int(p) for p in pix)
    assert g_set - band_pix == o_pix, f"candidate sets differ: gpu-only {sorted(g_set - band_pix - o_pix)[:5]}," \
                                      f" oracle-only {sorted(o_pix - g_set)[:5]}"
    where = {int(p): i for i, p in enumerate(pix)}
    for c, gp in zip(g_cand, g_pix):
        if gp not in where:
            continue
        i = where[gp]
        assert abs(float(c["snr"]) - o[i]) <= t[i]
        if best["margin"][i] > 2 * t[i]:
            assert (int(c["dm_idx"]), int(c["w_idx"]), int(c["t_idx"])) == \
                   (int(best["dm_idx"][i]), int(best["w_idx"][i]), int(best["t_idx"][i]))
    return {"n": len(o_pix), "band": len(band_pix)}
