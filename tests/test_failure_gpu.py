"""Bounded device waits (failure detection without a GPU fault): a kernel waiting on an
mbarrier that nothing completes gives up after its limit, the host reads the latched bit as
NSFRB_ETIMEOUT, and the device keeps working."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_18136_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2510_18136_gb300 import build
    build.build()
    from paper_2510_18136_gb300 import native as nat
    assert torch.cuda.is_available()
    return nat


def test_stalled_wait_reports_timeout_and_device_stays_usable(native):
    assert native.lib.nsfrb_dbg_wait_timeout(50) == native.ETIMEOUT
    assert native.lib.nsfrb_dbg_wait_timeout(0) == native.EINVAL
    # a search right after it is normal
    cfg = synth.config_small(8, 8)
    cube = synth.plain_noise(cfg, 4)
    with native.Plan(cfg, out="full") as plan:
        plan.search(cube.cuda(), torch.full((cfg.n_pix,), 4.0, device="cuda"))
        f_snr, _ = plan.full()
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    res, _, _ = oracle.search_cube(cube.numpy(), tab, cfg.widths, sigma=4.0)
    fin = np.isfinite(res["snr"])
    assert np.abs(f_snr[fin] - res["snr"][fin]).max() <= 1e-5 * max(1.0, np.abs(res["snr"][fin]).max())
