"""Plain statement of the PSF-based candidate clustering (Sec. 2.3), test infrastructure only.

Top `top_k` candidates by S/N (ties: smaller pixel index first); the PSF is
thresholded at its `percentile`-th percentile (numpy's linear interpolation) to
a binary mask; centred on each top candidate in turn, the top candidates inside
the mask form its cluster; the cluster's score is the mean of the members'
S/N referred to the central lobe (snr_j / psf_j) with inverse-variance
weights psf_j^2, i.e. sum_j psf_j snr_j / sum_j psf_j^2; the central
candidate of the highest score (first on ties) is the final candidate.
"""
from __future__ import annotations

import numpy as np


def psf_cluster(cands, nx: int, psf: np.ndarray, percentile: float = 90.0, top_k: int = 10):
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
        den = sum(w * w for _, w in m)
        scores.append(sum(w * w * (float(top["snr"][j]) / w) for j, w in m) / den if den > 0 else -np.inf)
    if not scores:
        return top, -1, -np.inf, 0
    best = int(np.argmax(scores))
    mask = 0
    for j, _ in members(best):
        mask |= 1 << j
    return top, best, float(scores[best]), mask
