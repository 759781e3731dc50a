"""Plain statement of the PSF-based candidate clustering (Sec. 2.3), test infrastructure only.

Top `top_k` candidates by S/N (ties: smaller pixel index first); the PSF is
thresholded at its `percentile`-th percentile (numpy's linear interpolation) to
a binary mask; centred on each top candidate in turn, the top candidates inside
the mask form its cluster; the cluster's score is a weighted mean of the
members' S/N; the central candidate of the highest score (first on ties) is
the final candidate.  psf_j is the PSF value at member j's offset from the
central candidate (1 for the central one of a peak-normalised PSF).

Score (the paper says only "weighted mean S/N" over the central and sidelobe
candidates):
  score="psf_mean": the PSF-weighted mean  sum_j psf_j snr_j / sum_j psf_j
                    (the weights are the PSF values at the members);
  score="lsq":      the members' S/N referred to the central lobe (snr_j / psf_j)
                    averaged with inverse-variance weights psf_j^2,
                    sum_j psf_j snr_j / sum_j psf_j^2.
"""
from __future__ import annotations

import numpy as np


def psf_cluster(cands, nx: int, psf: np.ndarray, percentile: float = 90.0, top_k: int = 10,
                score: str = "psf_mean"):
    if score not in ("psf_mean", "lsq"):
        raise ValueError(score)
    n = len(cands)
    order = sorted(range(n), key=lambda i: (-float(cands["snr"][i]),
                                            int(cands["row"][i]) * nx + int(cands["col"][i])))[:top_k]
    top = cands[order] if n else cands[:0]
    thr = float(np.percentile(psf, percentile))
    ph, pw = psf.shape
    cy, cx = ph // 2, pw // 2

    def members(i):
        out = []
        for j in range(len(top)):
            y = cy + int(top["row"][j]) - int(top["row"][i])
            x = cx + int(top["col"][j]) - int(top["col"][i])
            if 0 <= y < ph and 0 <= x < pw and psf[y, x] >= thr:
                out.append((j, float(psf[y, x])))
        return out

    scores = []
    for i in range(len(top)):
        m = members(i)
        if score == "psf_mean":
            weights = [w for _, w in m]                       # weight psf_j on snr_j
            values = [float(top["snr"][j]) for j, _ in m]
        else:
            weights = [w * w for _, w in m]                   # weight psf_j^2 on snr_j / psf_j
            values = [float(top["snr"][j]) / w for j, w in m]
        den = sum(weights)
        scores.append(sum(a * v for a, v in zip(weights, values)) / den if den > 0 else -np.inf)
    if not scores:
        return top, -1, -np.inf, 0
    best = int(np.argmax(scores))
    mask = 0
    for j, _ in members(best):
        mask |= 1 << j
    return top, best, float(scores[best]), mask
