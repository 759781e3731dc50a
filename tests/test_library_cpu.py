"""Host-side checks of libnsfrb that need no GPU: the library loads, exports
every entry point the header declares, validates configurations, and its
delay planner matches the oracle bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2510_18136_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    return nat


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"\b(nsfrb_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(native):
    names = _declared("nsfrb.h") + _declared("nsfrb_debug.h")
    assert len(names) >= 16 and "nsfrb_dbg_conv3" in names
    lib = ctypes.CDLL(native.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("make", [synth.config_small, lambda: synth.config_full_window(8, 8),
                                  lambda: synth.config_stress(8, 8)])
def test_delay_table_bit_exact(native, make):
    cfg = make()
    plan = native.Plan(cfg)
    ref = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    np.testing.assert_array_equal(plan.delays(), ref)
    n_u, smax = plan.info()
    assert n_u == len({r.tobytes() for r in ref})
    np.testing.assert_array_equal(smax, ref.max(axis=1))


def test_delay_table_random_grids(native):
    rng = np.random.default_rng(4)
    for _ in range(20):
        n_sub = int(rng.integers(1, 33))
        f = np.sort(rng.uniform(300, 2000, size=n_sub))
        if np.any(np.diff(f) <= 0):
            continue
        dm = np.sort(rng.uniform(0, 3000, size=int(rng.integers(1, 300))))
        cfg = synth.SearchConfig(ny=2, nx=3, n_sub=n_sub, n_t=1000, freq_mhz=f, dm=dm,
                                 t_samp_ms=float(rng.uniform(1, 500)), widths=np.array([1, 5], np.int32))
        try:
            plan = native.Plan(cfg)
        except native.NsfrbError as e:
            assert e.status == native.EINVAL   # shifts beyond the supported range
            continue
        np.testing.assert_array_equal(plan.delays(),
                                      oracle.delay_table(f, dm, cfg.k_dm_ms, cfg.t_samp_ms))


@pytest.mark.parametrize("field,value", [("n_t", 0), ("n_t", 5000), ("n_sub", 33), ("ny", 0)])
def test_invalid_configs_rejected(native, field, value):
    cfg = synth.config_small()
    setattr(cfg, field, value)
    if field == "n_sub":
        cfg.freq_mhz = synth.band_centres(33)
    with pytest.raises(native.NsfrbError) as e:
        native.Plan(cfg)
    assert e.value.status == native.EINVAL


@pytest.mark.parametrize("n_t", [1247, 1248, 4096])
def test_window_lengths_up_to_4096_accepted(native, n_t):
    """Windows of 1..4096 samples make plans (up to 1247 the register path, beyond it the
    long-window kernel); 4097 is refused."""
    cfg = synth.config_full_window(2, 2, n_t=n_t)
    cfg.widths = np.array([1, 2, 1024, n_t], np.int32)
    with native.Plan(cfg) as p:
        assert p.delays().shape == (64, 16)
    cfg.n_t = 4097
    cfg.widths = np.array([1, 4097], np.int32)
    with pytest.raises(native.NsfrbError) as e:
        native.Plan(cfg)
    assert e.value.status == native.EINVAL and "4096" in native.lib.nsfrb_last_error().decode()


def test_unsorted_dm_and_widths_rejected(native):
    cfg = synth.config_small()
    cfg.dm = cfg.dm[::-1].copy()
    with pytest.raises(native.NsfrbError):
        native.Plan(cfg)
    cfg = synth.config_small()
    cfg.widths = np.array([2, 1], np.int32)
    with pytest.raises(native.NsfrbError):
        native.Plan(cfg)


def test_search_without_results_is_not_ready(native):
    plan = native.Plan(synth.config_small())
    with pytest.raises(native.NsfrbError) as e:
        plan.candidates()
    assert e.value.status == native.ENOTREADY


def test_tile_codes_and_preference(native):
    """The binding's tile list is the header's; the preference is host state, validated."""
    txt = open(os.path.join(ROOT, "include", "nsfrb.h")).read()
    codes = tuple(int(x) for x in re.search(r"#define NSFRB_TILES ([\d, ]+)", txt).group(1).split(","))
    assert codes == native.TILES
    assert int(re.search(r"#define NSFRB_N_TILES (\d+)", txt).group(1)) == native.N_TILES
    plan = native.Plan(synth.config_small())
    assert plan.get_tile(native.F32) == 0
    plan.set_tile(native.BF16, 41)
    assert plan.get_tile(native.BF16) == 41 and plan.get_tile(native.F32) == 0
    for dtype, tile in ((native.F32, 23), (native.F32, 11), (3, 12)):
        with pytest.raises(native.NsfrbError) as e:
            plan.set_tile(dtype, tile)
        assert e.value.status == native.EINVAL
