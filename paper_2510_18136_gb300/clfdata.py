"""Training and evaluation data for the candidate classifier, produced by the search itself.

Stand-ins for the paper's training sets (Sec. 2.3: simulated point sources,
simulated near- and far-field RFI, field data; the field data are not
available): seeded sky cubes with PSF-convolved noise carry

* bursts (label 0): dispersed boxcar pulses, PSF-shaped, matched S/N U(lo, hi);
* bright bursts (label 0) with a PSF-sidelobe ghost (label 1): a copy at 0.1 of
  the amplitude, offset 6-12 px;
* zero-DM broadband steps (label 1): all subbands, no dispersion, spread over a
  wide Gaussian blob (near-field RFI appears at all spatial scales);
* single-subband spikes (label 1): 50 sigma in one subband for 1-2 samples.

Each cube is searched by the library (``nsfrb_search``); every source is
matched to the strongest candidate within 1 px of it, and the cutout around
that candidate (``nsfrb_clf_cutouts``) becomes one labelled sample.  Dispersion
shifts of the injected pulses come from the library's planner.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import native, synth

KIND_BURST, KIND_BRIGHT, KIND_GHOST, KIND_STEP, KIND_SPIKE = range(5)
LABEL = {KIND_BURST: 0, KIND_BRIGHT: 0, KIND_GHOST: 1, KIND_STEP: 1, KIND_SPIKE: 1}
KIND_NAMES = {KIND_BURST: "burst", KIND_BRIGHT: "bright burst", KIND_GHOST: "sidelobe ghost",
              KIND_STEP: "zero-DM step", KIND_SPIKE: "subband spike"}


def search_config(ny=128, nx=128, n_t=256) -> synth.SearchConfig:
    """Cube used to make classifier samples: 16 subbands, 64 DM on 0-2000, widths 1..128."""
    return synth.SearchConfig(ny=ny, nx=nx, n_t=n_t, dm=np.linspace(0.0, 2000.0, 64),
                              widths=np.array([1, 2, 4, 8, 16, 32, 64, 128], np.int32), threshold=6.0)


@dataclass
class Truth:
    kind: np.ndarray
    row: np.ndarray
    col: np.ndarray
    t0: np.ndarray
    width: np.ndarray
    dm: np.ndarray
    snr: np.ndarray

    @property
    def label(self):
        return np.array([LABEL[int(k)] for k in self.kind], np.int64)


def _shifts(plan_cache, cfg, dms):
    order = np.argsort(dms)
    c = synth.SearchConfig(ny=1, nx=1, n_t=cfg.n_t, freq_mhz=cfg.freq_mhz, dm=np.asarray(dms, float)[order],
                           widths=np.array([1], np.int32))
    with native.Plan(c) as p:
        sh = p.delays()
    out = np.empty_like(sh)
    out[order] = sh
    return out


def make_cube(cfg: synth.SearchConfig, seed: int, device="cuda", snr=(6.0, 30.0), spacing: int = 32,
              kinds_allowed=(KIND_BURST, KIND_BURST, KIND_BRIGHT, KIND_STEP, KIND_SPIKE)):
    """One cube with sources on a jittered grid (one source per spacing x spacing cell), each of a
    kind drawn from kinds_allowed.  Returns (cube FP32 [n_pix, n_sub, n_t] on device, Truth)."""
    rng = np.random.default_rng(seed)
    cube = synth.psf_noise(cfg, seed, device=device)
    sig_pix = synth.psf_sigma()
    psf = synth.gaussian_psf()
    cells = [(r, c) for r in range(spacing // 2, cfg.ny - spacing // 2 + 1, spacing)
             for c in range(spacing // 2, cfg.nx - spacing // 2 + 1, spacing)]
    rng.shuffle(cells)
    kinds, rows, cols, t0s, ws, dms, snrs = [], [], [], [], [], [], []
    for (r0, c0) in cells:
        kind = int(rng.choice(list(kinds_allowed)))
        r = r0 + int(rng.integers(-3, 4))
        c = c0 + int(rng.integers(-3, 4))
        if kind == KIND_BRIGHT:
            # the parent sits off-centre in its cell so that its ghost stays in the same cell
            r, c = r0 - 4, c0 - 4
        kinds.append(kind); rows.append(r); cols.append(c)
        dms.append(0.0 if kind in (KIND_STEP, KIND_SPIKE) else float(rng.uniform(0.0, 2000.0)))
        ws.append(int(rng.integers(1, 3)) if kind == KIND_SPIKE else
                  int(np.rint(np.exp(rng.uniform(0.0, math.log(64.0))))))
        snrs.append(float(rng.uniform(100.0, 250.0)) if kind == KIND_BRIGHT else float(rng.uniform(*snr)))
        t0s.append(0)
        if kind == KIND_BRIGHT:
            off = rng.uniform(6.0, 12.0)
            ang = rng.uniform(0.0, 2 * math.pi)
            kinds.append(KIND_GHOST)
            rows.append(int(round(r + off * math.sin(ang))) % cfg.ny)
            cols.append(int(round(c + off * math.cos(ang))) % cfg.nx)
            dms.append(dms[-1]); ws.append(ws[-1]); snrs.append(snrs[-1] * 0.1); t0s.append(0)
    dms = np.array(dms)
    sh = _shifts(None, cfg, dms)
    smax = sh.max(axis=1)
    # start times: the pulse (plus its dispersion) inside the window
    for i in range(len(kinds)):
        if kinds[i] == KIND_GHOST:
            t0s[i] = t0s[i - 1]
            continue
        span = max(cfg.n_t - int(smax[i]) - ws[i], 1)
        t0s[i] = int(rng.integers(0, span))
    # injection: per source its spatial taps (pixel, weight) and its valid (subband, sample) cells;
    # every (tap, cell) pair of a source is one entry of the cube, built on the device from the
    # concatenated tables and added by one index_add
    taps_p, taps_a, cells, n_cell = [], [], [], []
    psf_dy, psf_dx = np.meshgrid(np.arange(5) - 2, np.arange(5) - 2, indexing="ij")
    psf_taps = (psf_dy.ravel(), psf_dx.ravel(), psf.ravel())
    plane = cfg.n_sub * cfg.n_t
    for i, kind in enumerate(kinds):
        w = ws[i]
        if kind == KIND_SPIKE:
            amp = 50.0 * sig_pix
            k_sel = np.array([int(rng.integers(0, cfg.n_sub))])
            dy, dx, wt = psf_taps
        elif kind == KIND_STEP:
            s_blob = float(rng.uniform(4.0, 10.0))
            rad = int(2.5 * s_blob)
            gy, gx = np.meshgrid(np.arange(-rad, rad + 1), np.arange(-rad, rad + 1), indexing="ij")
            dy, dx = gy.ravel(), gx.ravel()
            wt = np.exp(-0.5 * (dy * dy + dx * dx) / s_blob ** 2)
            amp = snrs[i] * sig_pix / (math.sqrt(cfg.n_sub) * math.sqrt(w))
            k_sel = np.arange(cfg.n_sub)
        else:
            amp = snrs[i] * sig_pix / (math.sqrt(cfg.n_sub) * math.sqrt(w))
            k_sel = np.arange(cfg.n_sub)
            dy, dx, wt = psf_taps
        pix = ((rows[i] + dy) % cfg.ny) * cfg.nx + (cols[i] + dx) % cfg.nx          # [taps]
        t = t0s[i] + sh[i][k_sel][:, None] + np.arange(w)[None, :]                   # [k, w]
        kk, ww = np.nonzero(t < cfg.n_t)
        c = k_sel[kk] * cfg.n_t + t[kk, ww]                                          # [valid (k, t)]
        taps_p.append(pix.astype(np.int64) * plane)
        taps_a.append((amp * wt).astype(np.float32))
        cells.append(c.astype(np.int64))
        n_cell.append(np.full(pix.size, c.size, np.int64))
    if taps_p:
        tp = torch.from_numpy(np.concatenate(taps_p)).to(device)     # [taps of all sources]
        ta = torch.from_numpy(np.concatenate(taps_a)).to(device)
        nc = np.concatenate(n_cell)                                   # cells of each tap's source
        # first cell of each tap's source in the concatenated cell table
        starts = np.cumsum([0] + [x.size for x in cells[:-1]])
        c0 = np.concatenate([np.full(x.size, st, np.int64) for x, st in zip(taps_p, starts)])
        cl = torch.from_numpy(np.concatenate(cells)).to(device)
        ncd = torch.from_numpy(nc).to(device)
        n_ent = int(nc.sum())
        tap_of = torch.repeat_interleave(torch.arange(tp.numel(), device=device), ncd, output_size=n_ent)
        seg0 = torch.cumsum(ncd, 0) - ncd                             # first entry of each tap
        cell = torch.arange(n_ent, device=device) - seg0[tap_of] + torch.from_numpy(c0).to(device)[tap_of]
        cube.view(-1).index_add_(0, tp[tap_of] + cl[cell], ta[tap_of])
    truth = Truth(kind=np.array(kinds), row=np.array(rows), col=np.array(cols), t0=np.array(t0s),
                  width=np.array(ws), dm=dms, snr=np.array(snrs))
    return cube, truth


def match_sources(cand: np.ndarray, truth: Truth, nx: int, radius: int = 1):
    """Index of the strongest candidate within `radius` px of each source, or -1."""
    out = np.full(len(truth.kind), -1, np.int64)
    if len(cand) == 0:
        return out
    cr, cc, cs = cand["row"].astype(int), cand["col"].astype(int), cand["snr"]
    for i in range(len(truth.kind)):
        m = np.nonzero((np.abs(cr - truth.row[i]) <= radius) & (np.abs(cc - truth.col[i]) <= radius))[0]
        if m.size:
            out[i] = m[np.argmax(cs[m])]
    return out


def samples_from_cube(plan: native.Plan, cfg, cube: torch.Tensor, truth: Truth, sigma: torch.Tensor,
                      d=32, h=32, w=32):
    """Search the cube, match sources, cut out.  Returns (x bf16 [n, d, h, w, n_sub], labels, kinds, cands)."""
    plan.search(cube, sigma)
    cand = plan.candidates()
    m = match_sources(cand, truth, cfg.nx)
    keep = np.nonzero(m >= 0)[0]
    sel = cand[m[keep]]
    if len(sel) == 0:
        return None
    x = native.cutouts(plan, cube, native.candidates_to_device(sel), d, h, w, sigma=sigma)
    return x, truth.label[keep], truth.kind[keep], sel, keep


def dataset(n_target: int, seed: int, cfg=None, device="cuda", balance: bool = True, snr=(6.0, 30.0)):
    """About n_target labelled cutouts (50/50 if balance) from as many cubes as needed."""
    cfg = cfg or search_config()
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * math.sqrt(cfg.n_sub), device=device)
    plan = native.Plan(cfg)
    xs, ys, ks = [], [], []
    n, s = 0, seed
    n_pos = n_neg = 0
    while (min(n_pos, n_neg) * 2 if balance else n) < n_target:
        cube, truth = make_cube(cfg, s, device=device, snr=snr)
        s += 1
        got = samples_from_cube(plan, cfg, cube, truth, sigma)
        del cube
        if got is None:
            continue
        x, lab, kind, _, _ = got
        xs.append(x); ys.append(lab); ks.append(kind)
        n += len(lab)
        n_pos += int((lab == 1).sum()); n_neg += int((lab == 0).sum())
    plan.close()
    x = torch.cat(xs)
    y = np.concatenate(ys)
    k = np.concatenate(ks)
    if balance:
        rng = np.random.default_rng(seed)
        i1, i0 = np.nonzero(y == 1)[0], np.nonzero(y == 0)[0]
        m = min(len(i1), len(i0), n_target // 2)
        sel = np.sort(np.concatenate([rng.choice(i1, m, replace=False), rng.choice(i0, m, replace=False)]))
        x, y, k = x[torch.from_numpy(sel).to(x.device)], y[sel], k[sel]
    return x.contiguous(), torch.from_numpy(y.astype(np.float32)).to(device), k


def train(clf: native.Classifier, x: torch.Tensor, y: torch.Tensor, epochs: int, seed: int = 0,
          loss_every: int = 1):
    """Mini-batch training (shuffled each epoch); returns the per-epoch mean losses.  The loss is
    read back (a wait for the step) every loss_every steps and at the last step of an epoch, and
    each epoch's mean is over the steps read; the other steps queue without waiting."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    B = clf.batch
    n = x.shape[0] // B * B
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(x.shape[0], generator=g)[:n].to(x.device)
        tot, n_read = 0.0, 0
        for j, i in enumerate(range(0, n, B)):
            idx = perm[i:i + B]
            want = (j + 1) % loss_every == 0 or i + B >= n
            loss = clf.train_step(x[idx].contiguous(), y[idx].contiguous(), want_loss=want)
            if want:
                tot += loss
                n_read += 1
        losses.append(tot / max(1, n_read))
    return losses


def train_streaming(clf: native.Classifier, n_total: int, chunk: int = 4000, seed: int = 0, cfg=None,
                    device="cuda"):
    """Training on data made on the fly: balanced chunks of about `chunk` cutouts from fresh cubes
    (cube seeds never reused), each chunk seen once, until n_total cutouts have been trained on.
    Returns (per-chunk mean losses, cutouts trained on, seconds spent making data)."""
    import time
    losses, seen, t_data = [], 0, 0.0
    k = 0
    while seen < n_total:
        t0 = time.perf_counter()
        x, y, _ = dataset(min(chunk, n_total - seen), seed=seed + 1000003 * k, cfg=cfg, device=device)
        torch.cuda.synchronize()
        t_data += time.perf_counter() - t0
        losses += train(clf, x, y, epochs=1, seed=seed + k)
        seen += x.shape[0] // clf.batch * clf.batch
        k += 1
        del x, y
    return losses, seen, t_data


def wilson(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n (None for n = 0)."""
    if n == 0:
        return None
    p = k / n
    d = 1.0 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [max(0.0, c - h), min(1.0, c + h)]


def p_rfi(clf: native.Classifier, x: torch.Tensor) -> np.ndarray:
    """Sigmoid of the classifier logit for every cutout (inference mode)."""
    B = clf.batch
    out = []
    for i in range(0, x.shape[0], B):
        xb = x[i:i + B].contiguous()
        out.append(torch.sigmoid(clf.infer(xb)).cpu().numpy())
    return np.concatenate(out) if out else np.zeros(0)


def init_params(clf: native.Classifier, c=(32, 32, 64, 64), c0: int = 16, f: int = 32, fin: int = 512,
                seed: int = 0) -> np.ndarray:
    """Seeded starting point: conv and FC weights N(0, 2/fan_in), BN gamma 1, beta 0, biases 0
    (flat layout of nsfrb_clf_set_params)."""
    rng = np.random.default_rng(seed)
    out, cin = [], c0
    for co in c:
        out.append(rng.normal(0.0, math.sqrt(2.0 / (27 * cin)), co * 27 * cin))
        out.append(np.ones(co))
        out.append(np.zeros(co))
        cin = co
    out.append(rng.normal(0.0, math.sqrt(2.0 / fin), f * fin))
    out.append(np.zeros(f))
    out.append(rng.normal(0.0, math.sqrt(1.0 / f), f))
    out.append(np.zeros(1))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == clf.n_params, (p.size, clf.n_params)
    clf.set_params(p)
    return p


def evaluate(clf: native.Classifier, cfg, seeds, device="cuda", taus=(0.15, 0.5)):
    """Per-source results on fresh cubes: GPU detection (candidate within 1 px), its p_rfi,
    and the truth.  Returns a dict of arrays (one entry per source)."""
    sigma = torch.full((cfg.n_pix,), synth.psf_sigma() * math.sqrt(cfg.n_sub), device=device)
    plan = native.Plan(cfg)
    kinds, det, prob, cubes = [], [], [], []
    for s in seeds:
        cube, truth = make_cube(cfg, s, device=device)
        plan.search(cube, sigma)
        cand = plan.candidates()
        m = match_sources(cand, truth, cfg.nx)
        p = np.full(len(m), np.nan)
        hit = np.nonzero(m >= 0)[0]
        if hit.size:
            x = native.cutouts(plan, cube, native.candidates_to_device(cand[m[hit]]), 32, 32, 32, sigma=sigma)
            p[hit] = p_rfi(clf, x)
        kinds.append(truth.kind); det.append(m >= 0); prob.append(p)
        cubes.append((s, truth))
        del cube
    plan.close()
    kind = np.concatenate(kinds)
    return {"kind": kind, "label": np.array([LABEL[int(k)] for k in kind]), "detected": np.concatenate(det),
            "p_rfi": np.concatenate(prob), "cubes": cubes}


def rates(label, detected, p_rfi=None, tau=None):
    """Recall on astrophysical sources and false-positive rate on artefacts, with their counts and
    95 % Wilson intervals."""
    ok = detected.copy()
    if tau is not None:
        ok = ok & (np.nan_to_num(p_rfi, nan=1.0) < tau)
    real, art = label == 0, label == 1
    k_r, k_a = int(ok[real].sum()), int(ok[art].sum())
    return {"recall": float(ok[real].mean()) if real.any() else float("nan"),
            "fpr": float(ok[art].mean()) if art.any() else float("nan"),
            "n_real": int(real.sum()), "n_artefact": int(art.sum()), "recovered": k_r, "passed_artefacts": k_a,
            "recall_95": wilson(k_r, int(real.sum())), "fpr_95": wilson(k_a, int(art.sum()))}
