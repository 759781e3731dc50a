"""What the trained classifier adds to the plain S/N threshold (Sec. 3.2: the
classifier trades some completeness for rejecting RFI; p_rfi < 15 % nominal,
< 50 % looser).

The classifier is trained on cutouts that the search itself produces from
injected bursts and simulated artefacts (zero-DM broadband steps, single-subband
spikes, PSF-sidelobe ghosts).  On fresh cubes, the threshold-only detections are
taken from the FP64 oracle (a source is detected when the oracle's best S/N over
the 3x3 pixels around it exceeds the threshold); the classifier's are the GPU
candidates it passes.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2510_18136_gb300 import clfdata, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def _oracle_detect(cfg, seed, truth):
    cube, _ = clfdata.make_cube(cfg, seed, device="cuda")
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    sg = synth.psf_sigma() * math.sqrt(cfg.n_sub)
    det = np.zeros(len(truth.kind), bool)
    for i in range(len(truth.kind)):
        pix = [((truth.row[i] + dy) % cfg.ny) * cfg.nx + (truth.col[i] + dx) % cfg.nx
               for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        x = cube[torch.tensor(pix, device=cube.device)].cpu().numpy()
        _, best, _ = oracle.search_cube(x, tab, cfg.widths, sigma=sg)
        det[i] = bool((best["snr"] > cfg.threshold).any())
    return det


@pytest.fixture(scope="module")
def trained(native):
    x, y, _ = clfdata.dataset(6000, seed=100)
    clf = native.Classifier(batch=64, dropout=0.5, seed=7, lr=1e-3)
    clfdata.init_params(clf, seed=3)
    losses = clfdata.train(clf, x, y, epochs=4)
    yield clf, losses
    clf.close()


def test_classifier_rejects_artefacts_at_small_recall_cost(native, trained):
    cfg = clfdata.search_config()
    clf, losses = trained
    assert losses[-1] < losses[0]
    ev = clfdata.evaluate(clf, cfg, range(9000, 9012))
    det_oracle = np.concatenate([_oracle_detect(cfg, s, t) for s, t in ev["cubes"]])
    thr = clfdata.rates(ev["label"], det_oracle)
    c50 = clfdata.rates(ev["label"], ev["detected"], ev["p_rfi"], 0.5)
    c15 = clfdata.rates(ev["label"], ev["detected"], ev["p_rfi"], 0.15)
    print("threshold", thr, "p<0.5", c50, "p<0.15", c15, "losses", losses)
    # the GPU search finds what the oracle finds (same sources detected)
    assert (ev["detected"] == det_oracle).mean() > 0.98
    # gain: at p_rfi < 0.5 most artefacts that pass the threshold are rejected, most bursts kept
    assert thr["fpr"] > 0.8
    assert c50["fpr"] < 0.5 * thr["fpr"]
    assert c50["recall"] > 0.7 * thr["recall"]
    assert c15["fpr"] <= c50["fpr"] and c15["recall"] <= c50["recall"]
    lo, hi = c50["recall_95"]
    assert lo <= c50["recall"] <= hi and c50["n_real"] == int((ev["label"] == 0).sum())


def test_detection_curve_with_classifier(native, trained):
    """Sec. 3.2 detection rate per S/N bin, threshold alone and behind the classifier (bursts only):
    the classifier passes a subset of the threshold detections, most of them at high S/N, and the
    rate rises with S/N."""
    from paper_2510_18136_gb300 import campaign
    clf, _ = trained
    bins = np.array([4, 8, 12, 20, 30, 40])
    r = campaign.detection_curve_classified(clf, snr_bins=bins, cubes_per_bin=2, seed=5)
    thr, c15, c50 = np.array(r["threshold"]), np.array(r["p<0.15"]), np.array(r["p<0.5"])
    print("threshold", thr, "p<0.15", c15, "p<0.5", c50)
    assert (c15 <= c50 + 1e-12).all() and (c50 <= thr + 1e-12).all()
    assert thr[0] < thr[2] and thr[-1] >= 0.95
    assert c50[3:].min() >= 0.6 * thr[3:].min()
