"""The stated S/N error bound of BF16 storage, pinned on the FP64 oracle alone (no GPU).

The oracle searches the same seeded cube twice: once on the FP32 values and once on the same
values rounded to BF16 (nearest, ties to even).  Every trial's S/N difference is the
quantisation error of the storage form by itself, free of FP32 summation order; it must stay
inside ``parity.bf16_bound`` for the recipes of the full-window workload (PSF-convolved noise,
known sigma, bursts of S/N 6-30) and of the 512x512 workload (beam-scaled Student-t noise, MAD
normalisation, 256 DM), here on small images of the same recipes.
"""
import numpy as np
import torch

import oracle
from paper_2510_18136_gb300 import synth
from tests import parity


def _check(res32, res16, noise):
    s32, s16 = res32["snr"], res16["snr"]
    fin = np.isfinite(s32)
    assert (np.isfinite(s16) == fin).all()
    err = np.abs(s16[fin] - s32[fin])
    bound = parity.bf16_bound(s32[fin], noise)
    assert (err <= bound).all(), f"worst {np.max(err / bound):.3f} x bound"
    # the bound is not vacuous: rounding moves the S/N by about 2^-8 rms per trial
    assert 1e-4 < np.sqrt(np.mean(err ** 2)) < 1e-2
    return float(err.max())


def test_bf16_bound_full_window_recipe():
    cfg = synth.config_full_window(40, 40)
    cube = synth.psf_noise(cfg, 11)
    raw = synth.draw_injections(cfg, 40, 12, max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    x = cube.numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    sg = synth.psf_sigma() * 4.0
    r32, b32, _ = oracle.search_cube(x, tab, cfg.widths, sigma=sg)
    r16, b16, _ = oracle.search_cube(oracle.bf16_round(x), tab, cfg.widths, sigma=sg)
    _check(r32, r16, "known")
    assert b32["snr"].max() > 15.0        # bright bursts are part of the sample


def test_bf16_bound_stress_recipe_mad():
    cfg = synth.config_stress(28, 28)
    cube = synth.beam_student_noise(cfg, 13, dtype=torch.float32)
    raw = synth.draw_injections(cfg, 20, 14, dm_range=(0.0, 4000.0), max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    x = cube.numpy()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    r32, b32, bad32 = oracle.search_cube(x, tab, cfg.widths, mad=True)
    r16, b16, bad16 = oracle.search_cube(oracle.bf16_round(x), tab, cfg.widths, mad=True)
    assert bad32 == bad16 == 0
    _check(r32, r16, "mad")
    assert b32["snr"].max() > 15.0
