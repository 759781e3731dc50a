"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the one-line JSON
contract, run on a tiny grid so that it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ny", "6",
                          "--nx", "6", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "trials/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["steps"] == 2 and d["warmup"] == 1
    # a step is the measured oracle run on its pixel sample
    assert d["sample_pixels_per_step"] > 0 and d["config"]["injections"] > 0
    assert d["value"] * d["ms_per_step"] / 1e3 == __import__("pytest").approx(d["sample_trials_per_step"], rel=0.5)


def test_search_kernel_name_follows_the_chunk_rule():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.search_kernel_name(1200, "f32") == "search_kernel_pipe<38, 0, T, B, 0>"
    assert bench.search_kernel_name(1200, "bf16") == "search_kernel_pipe<38, 1, T, B, 0>"
    assert bench.search_kernel_name(1200, "bf16", "mad", 21) == \
        "mad_normalise_kernel + search_kernel_pipe<38, 0, 2, 1, 0> (FP32 slabs)"
    assert bench.search_kernel_name(1200, "bf16", tile=41) == "search_kernel_pipe<38, 1, 4, 1, 0>"
    assert bench.search_kernel_name(1200, "f32", tile=21, out="full") == "search_kernel_pipe<38, 0, 2, 1, 1>"
    assert bench.search_kernel_name(1247, "f32") == "search_kernel_pipe<39, 0, T, B, 0>"
    assert bench.search_kernel_name(4096, "bf16") == "search_kernel_long<1, 0>"
    assert bench.search_kernel_name(4096, "f32", out="full") == "search_kernel_long<0, 1>"
    assert bench.search_kernel_name(64, "f32") == "search_kernel_pipe<3, 0, T, B, 0>"
    assert bench.search_kernel_name(1001, "bf16") == "search_kernel<38, 0>"


def test_alg_ops_counts_the_definition():
    """The roofline's numerator (bench.alg_ops) against an explicit count of the definition's FP32
    operations on a tiny grid: per pixel and distinct shift row u with L = n_t - max shift, each
    valid de-dispersed sample costs n_sub - 1 adds and one prefix add, each boxcar trial of each
    width a difference and a running maximum; rows without samples cost nothing.  Identical DMs
    are one row; the distinct rows come from the oracle's delay table."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2510_18136_gb300 import build, synth
    build.build()
    from paper_2510_18136_gb300 import native

    cfg = synth.SearchConfig(ny=2, nx=3, n_t=40, dm=np.array([0.0, 0.0, 300.0, 900.0, 2500.0, 30000.0]),
                             widths=np.array([1, 3, 8, 40], np.int32))
    with native.Plan(cfg) as plan:
        ops, n_u = bench.alg_ops(cfg, plan)
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    rows = {tuple(int(s) for s in r) for r in tab}
    assert max(max(r) for r in rows) >= cfg.n_t          # one row has no sample at all
    want = 0
    for r in rows:
        L = cfg.n_t - max(r)
        for _ in range(max(L, 0)):
            want += (cfg.n_sub - 1) + 1
        for w in cfg.widths:
            for _ in range(max(L - int(w) + 1, 0)):
                want += 2
    assert n_u == len(rows) == len(cfg.dm) - 1
    assert ops == want * cfg.n_pix
