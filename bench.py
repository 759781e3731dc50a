#!/usr/bin/env python
"""Benchmark of the image-plane single-pulse search on one or more GB300s.

Workload (per GPU): 301 x 301 pixels, 16 subbands (1311-1498 MHz), 1200
samples of 134.2 ms, 64 DM trials on 0..2000 pc cm^-3, boxcar widths
1, 2, 4, ..., 1024 and 1200; PSF-convolved Gaussian noise with 50 injected
bursts, FP32 storage (--dtype bf16 for 16-bit storage).  One step = one
nsfrb_search over the whole cube plus the candidate list read back.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded pixel sample per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pixel·DM·width S/N trials/s; % of GB300 HBM peak; p99 block latency (ms)"
WORKLOAD = "full-window search 301x301 px x 16 sub x 1200 samples, 64 DM 0-2000, 12 widths 1..1024+1200"


def workload_name(cfg) -> str:
    """The workload's name with its sizes (the default is WORKLOAD)."""
    return (f"full-window search {cfg.ny}x{cfg.nx} px x {cfg.n_sub} sub x {cfg.n_t} samples, "
            f"{len(cfg.dm)} DM 0-2000, {len(cfg.widths)} widths 1..1024+1200")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--out", default="candidates", choices=["candidates", "full"],
                    help="full: also S/N and TOA for every (pixel, DM, width) on the device")
    ap.add_argument("--ny", type=int, default=301)
    ap.add_argument("--nx", type=int, default=301)
    ap.add_argument("--n-t", type=int, default=1200,
                    help="window length in samples (1200 is the workload; up to 4096)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-blocks", type=int, default=40,
                    help="blocks per field of the 4-field serving latency run (0: skip)")
    ap.add_argument("--serving-minutes", type=float, default=30.0,
                    help="simulated minutes of the 4-field injection run (device-written blocks, unpaced)")
    ap.add_argument("--serving-paced-blocks", type=int, default=6,
                    help="blocks per field pushed at the 3.355 s cadence (0: skip)")
    ap.add_argument("--bf16-steps", type=int, default=5,
                    help="timed BF16 searches of the bench cube, with and without re-score (0: skip)")
    ap.add_argument("--classifier-samples", type=int, default=200000,
                    help="cutouts made on the fly and trained on once each in the classifier section (the "
                         "classifier workload's 200k; 0: skip)")
    ap.add_argument("--classifier-eval-cubes", type=int, default=60,
                    help="fresh cubes the trained classifier is scored on")
    ap.add_argument("--campaigns", type=int, default=1,
                    help="injection campaigns (FN/FP versus threshold, detection rate with and without the "
                         "classifier) after the classifier section (0: skip)")
    ap.add_argument("--only", default="all", choices=["all", "imager"],
                    help="imager: run only the imager section (one JSON object) and exit")
    ap.add_argument("--imager-steps", type=int, default=20,
                    help="timed launches of the imager section, one 25-sample block each (0: skip)")
    ap.add_argument("--stress-steps", type=int, default=5,
                    help="timed searches of the 512x512 BF16 MAD stress workload (0: skip)")
    ap.add_argument("--timescale-steps", type=int, default=5,
                    help="timed 0.67 s and 10.05 s searches of the bench cube and PSF clusterings (0: skip)")
    ap.add_argument("--stress-size", type=int, default=512,
                    help="side of the stress image (512 is the stress workload; smaller for profiling)")
    ap.add_argument("--serving-fields", default="301x301,257x257,193x193,129x129",
                    help="comma-separated field grids of the serving section (the four fields are the "
                         "serving workload; smaller for profiling)")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ----------------------------------------------------------------------------- workload

def injection_shifts(native, synth, cfg, dms):
    """Integer shifts of each injection's own DM, from the library's planner."""
    order = np.argsort(dms)
    c = synth.SearchConfig(ny=1, nx=1, n_t=cfg.n_t, freq_mhz=cfg.freq_mhz, dm=np.asarray(dms)[order],
                           widths=np.array([1], np.int32), t_samp_ms=cfg.t_samp_ms, k_dm_ms=cfg.k_dm_ms)
    with native.Plan(c) as p:
        sh = p.delays()
    out = np.empty_like(sh)
    out[order] = sh
    return out


def make_cube(native, synth, cfg, seed, device, dtype):
    import torch
    cube = synth.psf_noise(cfg, seed, device=device)
    raw = synth.draw_injections(cfg, 50, seed + 1000, max_width=cfg.n_t)
    sh = injection_shifts(native, synth, cfg, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(cube, cfg, inj, sh, psf=synth.gaussian_psf())
    if dtype == "bf16":
        cube = cube.to(torch.bfloat16)
    return cube, inj


# DRAM bytes (read + write) per 301x301 FP32 launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of a 128x128 launch, 1262.8 MB, scaled by 90601 / 16384 pixels), valid for the
# kernel source with this sha256 prefix.
NCU_TRAFFIC = {"sha256_16": "09ea857acd409e8f", "bytes": 6.981e9, "workload": (301, 301, "f32")}


# DRAM bytes of one imager call (grid_kernel + transform_kernel) from the ncu launch list of the
# committed kernels (paper block: 25 x 16 x 8 x 3321 x 2 pol, 175 px); ncu flushes the caches
# before each kernel, so the transform re-reads the 15.6 MB of partial grids from DRAM there.
IMG_NCU_TRAFFIC = {"sha256_16": "efc27e98ac335103", "bytes": 181822464 + 6787328 + 15642112 + 203264}


def imager_traffic():
    import hashlib
    with open(os.path.join(ROOT, "paper_2510_18136_gb300", "csrc", "imager.cu"), "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()[:16]
    return IMG_NCU_TRAFFIC["bytes"] if digest == IMG_NCU_TRAFFIC["sha256_16"] else None


def measured_traffic(ny, nx, dtype):
    """ncu traffic per launch if it was taken on the current kernel source, else None."""
    import hashlib
    src = os.path.join(ROOT, "paper_2510_18136_gb300", "csrc", "search_impl.cuh")
    with open(src, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()[:16]
    if digest != NCU_TRAFFIC["sha256_16"] or (ny, nx, dtype) != NCU_TRAFFIC["workload"]:
        return None
    return NCU_TRAFFIC["bytes"]


def search_kernel_name(n_t, dtype, noise="known", tile=None, out="candidates"):
    """The kernels the library launches for this window: chunks of C samples per lane, the smallest
    compiled C with 32 C > n_t.  With known noise the barrier-free kernel runs (FP32 rows; 16-bit
    rows read in place when C is even and the rows fill whole 16-byte units), with the pixel x DM
    tile (teams T, buffers per team B) the plan chose; MAD normalisation is a pass of its own into
    FP32 slabs that the barrier-free kernel then searches.  The last template argument is FULL."""
    st = {"f32": 0, "bf16": 1, "f16": 2}[dtype]
    full = 1 if out == "full" else 0     # bool template arguments as ncu prints them
    if n_t > 1247:   # beyond the register path: the long-window kernel (MAD slabs are FP32)
        return f"search_kernel_long<{0 if noise == 'mad' else st}, {full}>"
    c = next(c for c in (1, 3, 5, 9, 17, 25, 38, 39) if 32 * c >= n_t + 1)
    tt = ", T, B" if tile is None else f", {int(tile) // 10}, {int(tile) % 10}"
    if noise == "mad":
        return f"mad_normalise_kernel + search_kernel_pipe<{c}, 0{tt}, {full}> (FP32 slabs)"
    if st == 0 or (c % 2 == 0 and n_t % 8 == 0):
        return f"search_kernel_pipe<{c}, {st}{tt}, {full}>"
    return f"search_kernel<{c}, {full}>"


def alg_ops(cfg, plan):
    """FP32 operations per search launch: for every pixel and distinct shift row u with
    L = n_t - smax_u samples: (n_sub - 1) L de-dispersion adds, L prefix adds, and for
    every width 2 (L - w + 1) (boxcar difference and running maximum)."""
    tab = plan.delays()
    seen = set()
    per_pix = 0
    for d in range(tab.shape[0]):
        key = tab[d].tobytes()
        if key in seen:
            continue
        seen.add(key)
        L = cfg.n_t - int(tab[d].max())
        if L <= 0:
            continue
        per_pix += (cfg.n_sub - 1) * L + L
        for w in cfg.widths:
            if w <= L:
                per_pix += 2 * (L - int(w) + 1)
    return per_pix * cfg.n_pix, len(seen)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle legs

def oracle_sample_rate(cube_host, cfg, target_s: float, seed: int = 0, n_fixed: int = 0):
    """Time the FP64 oracle on a pixel sample sized for about target_s seconds (or of n_fixed
    pixels, one run)."""
    import oracle
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm, cfg.k_dm_ms, cfg.t_samp_ms)
    rng = np.random.default_rng(seed)
    sig = float(cfg.sigma_pix * math.sqrt(cfg.n_sub))

    def run(n):
        pix = np.sort(rng.choice(cfg.n_pix, size=n, replace=False))
        x = cube_host[pix].float().numpy()
        t0 = time.perf_counter()
        oracle.search_cube(x, tab, cfg.widths, sigma=sig)
        return time.perf_counter() - t0

    if n_fixed > 0:
        n = int(min(cfg.n_pix, n_fixed))
        t = run(n)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        return n * len(cfg.dm) * len(cfg.widths) / t, n, t, cores
    n = min(256, cfg.n_pix)
    t = run(n)
    for _ in range(2):   # calibrate the sample to about target_s seconds
        n = int(min(cfg.n_pix, max(16, n * target_s / max(t, 1e-3))))
        t = run(n)
        if t > 0.5 * target_s or n == cfg.n_pix:
            break
    trials = n * len(cfg.dm) * len(cfg.widths)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return trials / t, n, t, cores


def reference_arm(args):
    """The oracle as the reference implementation, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2510_18136_gb300 import synth
    cfg = synth.config_full_window(args.ny, args.nx, n_t=args.n_t)
    cfg.sigma_pix = synth.psf_sigma()
    import oracle
    host = synth.psf_noise(cfg, args.seed)          # CPU generation, same recipe
    # the same 50 bursts as the GPU arm's cube recipe, placed with the oracle's delay table
    raw = synth.draw_injections(cfg, 50, args.seed + 1000, max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"], cfg.k_dm_ms, cfg.t_samp_ms)
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub, synth.psf_sigma())
    synth.add_injections(host, cfg, inj, sh, psf=synth.gaussian_psf())
    # one sample size, calibrated once, then one oracle run per step: the whole run takes about
    # two minutes of host time whatever --steps and --warmup are
    per_step = min(20.0, 120.0 / max(1, args.steps + args.warmup))
    _, n_cal, _, _ = oracle_sample_rate(host, cfg, per_step)
    for k in range(args.warmup):
        oracle_sample_rate(host, cfg, per_step, seed=1000 + k, n_fixed=n_cal)
    rates, ns, secs = [], [], []
    for k in range(args.steps):
        r, n, t, cores = oracle_sample_rate(host, cfg, per_step, seed=k, n_fixed=n_cal)
        rates.append(r)
        ns.append(n)
        secs.append(t)
    value = statistics.median(rates)
    # a step is one oracle run on a sample of the cube's pixels (every DM and width): ms_per_step
    # is that measured time, and value the rate of trials it searched
    ms = statistics.median(secs) * 1e3
    line = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(cfg), "kind": "FP64 CPU oracle", "injections": len(inj),
                       "step": f"{int(np.median(ns))} random pixels of the cube searched per step"},
            "sample_pixels_per_step": int(np.median(ns)), "sample_trials_per_step": int(np.median(ns)) * 64 * 12,
            "cpu_baseline": {"value": value, "unit": "trials/s", "cores": cores, "kind": "oracle",
                             "sample": f"{int(np.median(ns))} random pixels per step, all 64 DM x 12 widths "
                                       f"({ms / 1e3:.1f} s per step)"},
            "e2e": {"value": value, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- serving

SERVING_FIELDS = ((301, 301), (257, 257), (193, 193), (129, 129))
SERVING_EPS = 0.03          # BF16 S/N error bound with known noise: re-score band around the threshold
CADENCE_S = 3.355


def _serving_fields(native, synth, seed):
    import torch
    fields = []
    for i, (ny, nx) in enumerate(SERVING_FIELDS):
        cfg = synth.config_full_window(ny, nx)
        plan = native.Plan(cfg, dtype="bf16", rescore_eps=SERVING_EPS)
        plan.stream_open(25)
        fields.append((cfg, plan))
    return fields


def serving_latency(native, synth, n_blocks: int, paced_blocks: int, seed: int = 0):
    """Four concurrent fields (one plan, stream and CUDA graph each), BF16 window of 1200 samples
    with re-scoring from the FP32 window (device memory where it fits), 25-sample blocks from pinned
    host memory:
    push -> candidates device latency, unpaced (back to back) and paced (one block per field every
    3.355 s)."""
    import torch
    fields = _serving_fields(native, synth, seed)
    blocks = []
    for i, (cfg, _) in enumerate(fields):
        g = torch.Generator().manual_seed(seed + i)
        blocks.append([torch.randn((25, cfg.n_sub, cfg.ny, cfg.nx), generator=g).pin_memory() for _ in range(2)])

    def run(n, paced):
        lat = []
        t0 = time.perf_counter()
        for b in range(n):
            if paced:
                time.sleep(max(0.0, t0 + b * CADENCE_S - time.perf_counter()))
            for (cfg, plan), blk in zip(fields, blocks):
                plan.stream_push(blk[b % 2])
            for cfg, plan in fields:
                _, ms = plan.stream_poll(timeout_ms=3350)
                lat.append(ms)
        return np.array(lat), time.perf_counter() - t0

    lat, wall = run(n_blocks, False)
    lat = lat[2 * len(fields):]                     # the first two blocks of each field are warm-up
    out = {"fields": [f"{ny}x{nx}" for ny, nx in SERVING_FIELDS], "storage": "bf16",
           "rescore_eps": SERVING_EPS,
           "rescore_from": ", ".join(sorted({{1: "device FP32 window", 2: "pinned host FP32 window"}.get(
               plan.stream_window_info(), "none") for _, plan in fields})), "block_samples": 25,
           "window_samples": 1200, "blocks_per_field": n_blocks, "paced": False,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "max_ms": float(lat.max()), "blocks_per_s": 4 * n_blocks / wall, "cadence_s": CADENCE_S}
    if paced_blocks > 0:
        plat, pwall = run(paced_blocks, True)
        out["paced_run"] = {"blocks_per_field": paced_blocks, "wall_s": pwall,
                            "p50_ms": float(np.percentile(plat, 50)), "p99_ms": float(np.percentile(plat, 99)),
                            "max_ms": float(plat.max())}
    for _, plan in fields:
        plan.close()
    return out


def serving_injections(native, synth, minutes: float, seed: int = 0):
    """Four concurrent BF16 fields with re-scoring, fed `minutes` of simulated sky in 25-sample
    blocks written on the device (unit Gaussian noise per pixel, subband and sample) with bursts
    arriving as a Poisson process at 1 per field-minute (pixel uniform, DM U(0, 2000), width
    log-U(1, 1200) clamped to the window, matched S/N U(6, 30)), searched unpaced.  A burst is
    recovered when a candidate lands on its pixel in the block that holds the end of its
    dispersed sweep or the next one."""
    import torch
    import oracle as _o
    fields = _serving_fields(native, synth, seed)
    n_blk, n_sub = 25, 16
    n_blocks = int(round(minutes * 60.0 / CADENCE_S))
    rng = np.random.default_rng(seed + 77)
    gen = torch.Generator(device="cuda").manual_seed(seed + 78)
    cfg0 = fields[0][0]
    injs = []
    for f, (cfg, _) in enumerate(fields):
        n_inj = rng.poisson(n_blocks * CADENCE_S / 60.0)
        t_arr = np.sort(rng.uniform(0.0, n_blocks * n_blk, n_inj))
        dm = rng.uniform(0.0, 2000.0, n_inj)
        sh = _o.delay_table(cfg.freq_mhz, dm) if n_inj else np.zeros((0, n_sub), np.int32)
        w = np.rint(np.exp(rng.uniform(0.0, math.log(1200.0), n_inj))).astype(np.int64)
        w = np.maximum(1, np.minimum(w, cfg.n_t - sh.max(axis=1) if n_inj else w))
        snr = rng.uniform(6.0, 30.0, n_inj)
        pix = rng.integers(0, cfg.n_pix, n_inj)
        for j in range(n_inj):
            t0 = int(t_arr[j])
            injs.append({"field": f, "pix": int(pix[j]), "t0": t0, "w": int(w[j]), "sh": sh[j], "snr": float(snr[j]),
                         "amp": float(snr[j]) / (math.sqrt(n_sub) * math.sqrt(float(w[j]))),
                         "end_blk": (t0 + int(w[j]) - 1 + int(sh[j].max())) // n_blk})
    found = [False] * len(injs)
    n_cand, lat = 0, []
    bufs = [plan.stream_block() for _, plan in fields]
    t_start = time.perf_counter()
    for b in range(n_blocks):
        a0, a1 = b * n_blk, (b + 1) * n_blk
        for f, (cfg, plan) in enumerate(fields):
            blk = bufs[f]
            torch.randn(blk.shape, generator=gen, device="cuda", out=blk)
            view = blk.view(n_blk, n_sub, cfg.n_pix)
            for j, inj in enumerate(injs):
                if inj["field"] != f:
                    continue
                for k in range(n_sub):
                    lo, hi = inj["t0"] + int(inj["sh"][k]), inj["t0"] + int(inj["sh"][k]) + inj["w"]
                    lo, hi = max(lo, a0), min(hi, a1)
                    if lo < hi:
                        view[lo - a0:hi - a0, k, inj["pix"]] += inj["amp"]
            plan.stream_push_device(stream=torch.cuda.current_stream())
        for f, (cfg, plan) in enumerate(fields):
            cand, ms = plan.stream_poll(timeout_ms=3350)
            lat.append(ms)
            n_cand += len(cand)
            got = set((cand["row"].astype(np.int64) * cfg.nx + cand["col"]).tolist())
            for j, inj in enumerate(injs):
                if inj["field"] == f and not found[j] and inj["end_blk"] <= b <= inj["end_blk"] + 1 \
                        and inj["pix"] in got:
                    found[j] = True
    wall = time.perf_counter() - t_start
    for _, plan in fields:
        plan.close()
    done = [j for j, inj in enumerate(injs) if inj["end_blk"] + 1 < n_blocks]
    snr = np.array([injs[j]["snr"] for j in done])
    hit = np.array([found[j] for j in done], bool)
    lat = np.array(lat)
    return {"simulated_minutes": minutes, "blocks_per_field": n_blocks, "injections": len(done),
            "recovered": int(hit.sum()), "recall": float(hit.mean()) if len(done) else None,
            "recall_interval_95": wilson(int(hit.sum()), len(done)),
            "recall_snr_gt_10": float(hit[snr > 10].mean()) if (snr > 10).any() else None,
            "candidates_total": int(n_cand), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall,
            "noise": "unit Gaussian per pixel, subband and sample (no PSF)", "threshold": 6.0}


def wilson(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return None
    p = k / n
    d = 1.0 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [max(0.0, c - h), min(1.0, c + h)]


def bf16_section(native, synth, cfg, cube32, sigma, steps: int, e2e_steps: int, s32):
    """BF16 storage of the bench cube: search time without and with re-scoring (pixels within
    0.03 of the threshold searched again from the FP32 cube), the largest |S/N| difference to the
    FP32 search over every pixel, the re-scored candidate set against the FP32 one, and the
    end-to-end rate from a pinned host BF16 cube (half the link bytes of FP32)."""
    import torch
    stream = torch.cuda.current_stream()
    cube16 = cube32.to(torch.bfloat16)
    eps = 0.03
    out = {"rescore_eps": eps}
    for name, kw, extra in (("plain", {}, {}), ("rescore", {"rescore_eps": eps}, {"cube_f32": cube32})):
        plan = native.Plan(cfg, dtype="bf16", **kw)
        tile, tile_ms = plan.autotune(cube16, sigma, reps=3, stream=stream)
        for _ in range(3):
            plan.search(cube16, sigma, stream=stream, **extra)
            cand = plan.candidates()
        ks = []
        for _ in range(steps):
            plan.search(cube16, sigma, stream=stream, **extra)
            cand = plan.candidates()
            ks.append(plan.last_timing()[0])
        snr, _ = plan.best()
        out[name] = {"kernel_ms": statistics.median(ks), "trials_per_s": cfg.n_trials / (statistics.median(ks) / 1e3),
                     "candidates": int(len(cand)), "tile": tile, "tile_ms": tile_ms}
        if name == "plain":
            fin = np.isfinite(s32)
            err = np.abs(snr[fin].astype(np.float64) - s32[fin])
            out["max_abs_dsnr_vs_fp32"] = float(err.max())
            thr32, e32 = np.float32(cfg.threshold), np.float32(eps)
            out["rescored_pixels"] = int(((snr >= thr32 - e32) & (snr <= thr32 + e32)).sum())
            plain_set = set((cand["row"].astype(np.int64) * cfg.nx + cand["col"]).tolist())
        else:
            out["rescore"]["candidate_set_equals_fp32"] = bool(
                set((cand["row"].astype(np.int64) * cfg.nx + cand["col"]).tolist()) ==
                set(np.nonzero(s32 > cfg.threshold)[0].tolist()))
        if name == "rescore":
            host = cube16.cpu().pin_memory()
            hs = sigma.cpu().pin_memory()
            plan.search_host(host, hs, stream=stream)
            plan.candidates()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p2 = native.Plan(cfg, dtype="bf16")
            p2.set_tile(native.BF16, tile)
            p2.search_host(host, hs, stream=stream)
            p2.candidates()
            e0.record(stream)
            for _ in range(e2e_steps):
                p2.search_host(host, hs, stream=stream)
                n_c = len(p2.candidates())
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3 / e2e_steps
            out["e2e_host_bf16"] = {"value": cfg.n_trials / t, "unit": "trials/s", "ms_per_step": t * 1e3,
                                    "h2d_bytes_per_step": host.numel() * 2 + hs.numel() * 4,
                                    "d2h_bytes_per_step": 8 + 24 * n_c, "rescore": False}
            p2.close()
            del host
        plan.close()
    del cube16
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- classifier

def clf_flops_per_sample(d=32, h=32, w=32, c0=16, c=(32, 32, 64, 64)):
    """Algorithmic FLOPs of the four conv blocks per cutout: forward 2 P Co 27 Ci per block;
    training adds the weight gradient (same) and the input gradient (same, blocks 1-3)."""
    fwd, dx = 0.0, 0.0
    cin, dd, hh, ww = c0, d, h, w
    for l, co in enumerate(c):
        f = 2.0 * dd * hh * ww * co * 27 * cin
        fwd += f
        if l > 0:
            dx += f
        cin, dd, hh, ww = co, dd // 2, hh // 2, ww // 2
    return fwd, 2 * fwd + dx


def classifier_section(native, n_samples: int, eval_cubes: int, seed: int = 0):
    """Train the candidate classifier on cutouts made on the fly by the search (each seen once),
    then score recall and artefact pass rate on fresh cubes; returns (JSON section, classifier)."""
    import torch
    from paper_2510_18136_gb300 import clfdata
    cfg = clfdata.search_config()
    gen_cfg = clfdata.search_config(256, 256)          # 64 sources per cube for the training stream
    clf = native.Classifier(batch=64, dropout=0.5, seed=7 + seed, lr=1e-3)
    clfdata.init_params(clf, seed=3 + seed)
    t0 = time.perf_counter()
    losses, seen, t_data = clfdata.train_streaming(clf, n_samples, chunk=6000, seed=100 + seed, cfg=gen_cfg)
    t_all = time.perf_counter() - t0
    # training throughput on one resident batch set (no data generation in the timed loop)
    x, y, _ = clfdata.dataset(2048, seed=77 + seed, cfg=gen_cfg)
    clfdata.train(clf, x, y, epochs=1, seed=seed, loss_every=1 << 30)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    # the loss is read back at the end of each epoch only (the steps queue without host waits)
    clfdata.train(clf, x, y, epochs=3, seed=seed + 1, loss_every=1 << 30)
    e1.record()
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1) / 1e3
    n_timed = 3 * (x.shape[0] // clf.batch) * clf.batch
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xb = x[:clf.batch].contiguous()
    clf.infer(xb)
    i0.record()
    for _ in range(20):
        clf.infer(xb)
    i1.record()
    torch.cuda.synchronize()
    t_inf = i0.elapsed_time(i1) / 1e3
    ev = clfdata.evaluate(clf, cfg, range(900000 + 1000 * seed, 900000 + 1000 * seed + eval_cubes))
    thr = clfdata.rates(ev["label"], ev["detected"])
    c15 = clfdata.rates(ev["label"], ev["detected"], ev["p_rfi"], 0.15)
    c50 = clfdata.rates(ev["label"], ev["detected"], ev["p_rfi"], 0.5)
    fwd, train_f = clf_flops_per_sample()
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    train_tflops = n_timed * train_f / t_train / 1e12
    return {"cutout": "32x32 px x 16 subbands x 32 samples (bf16)", "net": "4 conv (16-32-32-64-64) + FC 32 + FC 1",
            "trained_on": int(seen), "data": "made on the fly, each cutout seen once (256x256 cubes, 50/50 bursts "
            "and artefacts)", "first_loss": losses[0], "final_loss": losses[-1], "data_gen_s": t_data,
            "stream_wall_s": t_all, "train_samples_per_s": n_timed / t_train, "train_conv_tflops": train_tflops,
            "train_tensor_frac_of_bf16_peak": train_tflops / float(pk["bf16_tflops"]),
            "infer_cutouts_per_s": 20 * clf.batch / t_inf, "eval_cubes": eval_cubes,
            "threshold_only": thr, "with_classifier_p_lt_0.15": c15, "with_classifier_p_lt_0.5": c50,
            "threshold_method": "GPU search (parity with the FP64 oracle is a test)"}, clf


def campaigns_section(native, clf, seed: int = 0):
    """Sec. 3.1-3.2 injection campaigns through the GPU search: FN / FP rates against the threshold
    0-20 and its optimum; detection rate per input S/N 1-40 (50 per bin); and with the trained
    classifier at p_rfi < 0.15 and < 0.5 (bursts only, PSF noise)."""
    from paper_2510_18136_gb300 import campaign
    t0 = time.perf_counter()
    th = campaign.threshold_curves(n_inj=1000, n_noise=2000, seed=10 + seed)
    det = campaign.detection_curve(snr_bins=np.arange(1, 41), n_per_bin=50, seed=11 + seed)
    out = {"threshold_scan": {"thresholds": [float(t) for t in th["thresholds"][::4]],
                              "fn": [float(v) for v in th["fn"][::4]], "fp": [float(v) for v in th["fp"][::4]],
                              "optimum": th["optimum"], "injections": 1000, "noise_realisations": 2000,
                              "injection_snr": "U(0, 10)", "image": "32x32 px x 64 samples, 16 DM 0-4000, widths 1-16"},
           "detection_rate": {"snr_bins": [float(v) for v in det["snr_bins"]], "rate": [float(v) for v in det["rate"]],
                              "per_bin": 50, "threshold": 6.0}}
    if clf is not None:
        dc = campaign.detection_curve_classified(clf, snr_bins=np.arange(2, 41, 2), cubes_per_bin=3, seed=12 + seed)
        out["detection_rate_classified"] = {k: (list(map(float, v)) if not isinstance(v, str) else v)
                                            for k, v in dc.items()}
    out["wall_s"] = time.perf_counter() - t0
    return out


# ----------------------------------------------------------------------------- imager

def imager_section(native, steps: int, seed: int = 0):
    """Image one 25-sample block (16 subbands x 8 channels, 82-antenna core, 175 px, R = -2) per
    launch; HBM roofline on the visibilities read and images written; the FP64 oracle timed on
    a few images of the same block."""
    import torch
    from oracle import imager as oi
    from paper_2510_18136_gb300 import synth_vis as sv
    n_t, N, pix = 25, 175, 10.3
    ant = sv.core_layout(seed)
    uv = sv.baseline_uv(ant)
    chan = sv.channel_freqs()
    n_sub, n_chan = chan.shape
    vis = sv.visibilities(uv, chan, n_t, [(12, -7, 5.0)], pixel_arcsec=pix, noise=1.0, seed=seed, device="cuda")
    vis_f = torch.view_as_real(vis).contiguous()
    im = native.Imager(uv, chan, n_grid=N, pixel_arcsec=pix)
    u_max, v_max, n_entries = im.info()
    out = torch.empty((n_t, n_sub, N, N), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()
    for _ in range(3):
        im.image(vis_f, out=out, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        im.image(vis_f, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(times)
    vis_bytes = vis_f.numel() * 4
    img_bytes = out.numel() * 4
    alg = vis_bytes + img_bytes + 8 * n_entries
    pk = peaks()
    # oracle on a few images of the same block
    vh = vis.cpu().numpy()
    pairs = [(0, 0), (12, 7), (24, 15)]
    c0 = time.perf_counter()
    for tt, ss in pairs:
        oi.image(vh[tt:tt + 1, ss:ss + 1], uv, chan[ss:ss + 1], N, pix)
    t_cpu = (time.perf_counter() - c0) / len(pairs)
    im.close()
    return {"workload": f"{n_t} samples x {n_sub} subbands x {n_chan} channels x {len(uv)} baselines x 2 pol "
                        f"-> {n_t * n_sub} images {N}x{N} (10.3 arcsec, Briggs R=-2, b 20-485 m)",
            "uv_support": [u_max, v_max], "gridding_entries": n_entries,
            "ms_per_block": t * 1e3, "images_per_s": n_t * n_sub / t,
            "visibilities_per_s": n_t * n_sub * n_chan * len(uv) * 2 / t,
            "roofline": {"bound": "hbm", "achieved": alg / t / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": alg / t / 1e9 / pk["hbm_gbs"], "bytes_per_launch": alg,
                         "kernel": "grid_kernel + transform_kernel (one nsfrb_image call)",
                         "traffic": imager_traffic()},
            "l2": "256 MB buffer written between launches",
            "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "images/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(pairs)} images of the block, FP64 numpy"}}


def timescales_section(native, synth, cube, cfg, sigma, cand, steps: int):
    """The 0.67 s and 10.05 s searches of the bench cube (Sec. 2.2 and its footnote): per scale the
    time binning (nsfrb_bin_time, HBM-bound: the cube read once, 1/factor of it written) and the
    search of the binned cube (widths 1..16, DM x5 on the same integer shifts, or DM 0), both timed
    with CUDA events on the launching stream; and the PSF clustering of the full-resolution
    candidate list (Sec. 2.3, nsfrb_psf_cluster), timed per call with its copies."""
    import torch
    from paper_2510_18136_gb300 import multiscale
    pk = peaks()
    stream = torch.cuda.current_stream()
    in_bytes = cube.numel() * cube.element_size()
    out = {"cube": f"{cfg.ny}x{cfg.nx} px x {cfg.n_sub} sub x {cfg.n_t} samples ({cube.dtype})", "scales": []}
    for factor, c in multiscale.paper_timescales(cfg)[1:]:
        sg = sigma * math.sqrt(factor)
        plan = native.Plan(c, dtype="f32")
        for _ in range(2):   # warm-up (allocates the binned cube, loads the kernels)
            xb = multiscale.bin_time(cube, factor, stream=stream)
            plan.search(xb, sg, stream=stream)
            plan.candidates()
        bin_ms, search_ms, n_c = [], [], 0
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xb = multiscale.bin_time(cube, factor, stream=stream)
            e1.record(stream)
            plan.search(xb, sg, stream=stream)
            n_c = len(plan.candidates())
            bin_ms.append(e0.elapsed_time(e1))
            search_ms.append(plan.last_timing()[0])
        plan.close()
        b_ms, k_ms = statistics.median(bin_ms), statistics.median(search_ms)
        bin_bytes = in_bytes + xb.numel() * 4
        out["scales"].append({
            "factor": factor, "t_samp_ms": c.t_samp_ms, "n_t": c.n_t, "n_dm": len(c.dm),
            "widths": [int(w) for w in c.widths], "bin_ms": b_ms, "search_ms": k_ms,
            "trials_per_s": c.n_trials / ((b_ms + k_ms) / 1e3), "candidates": n_c,
            "bin_roofline": {"bound": "hbm", "achieved": bin_bytes / (b_ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                             "unit": "GB/s", "frac": bin_bytes / (b_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                             "bytes_per_launch": bin_bytes}})
    psf = synth.gaussian_psf(15).astype(np.float32)
    native.psf_cluster(cand, cfg.nx, psf)
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        top, res = native.psf_cluster(cand, cfg.nx, psf)
        t.append(time.perf_counter() - t0)
    out["psf_cluster"] = {"candidates_in": int(len(cand)), "top_k": 10, "psf": "15x15 Gaussian",
                          "ms_per_call": statistics.median(t) * 1e3, "n_top": int(res["n_top"]),
                          "timing": "host wall clock per call: candidate list to the device, kernel, result back"}
    return out


def stress_section(native, synth, steps: int, seed: int = 0, size: int = 512):
    """The stress workload: 512x512 px x 16 sub x 1200 samples stored in BF16, beam-scaled
    Student-t noise, MAD normalisation per (pixel, subband), 500 injections, 256 DM 0-4000,
    12 widths; search kernel time by CUDA events, ALU roofline on the definition's operations
    (the MAD normalisation's own work is not counted)."""
    import torch
    import oracle
    cfg = synth.config_stress(size, size)
    cube = synth.beam_student_noise(cfg, seed + 5, device="cuda", dtype=torch.float32)
    n_inj = max(8, round(500 * cfg.n_pix / (512 * 512)))    # 500 on the 512x512 image
    raw = synth.draw_injections(cfg, n_inj, seed + 6, dm_range=(0.0, 4000.0), max_width=cfg.n_t)
    sh = oracle.delay_table(cfg.freq_mhz, raw["dm"])
    inj = synth.place_injections(raw, sh, cfg.n_t, cfg.n_sub,
                                 synth.beam_sigma(cfg)[raw["row"] * cfg.nx + raw["col"]])
    synth.add_injections(cube, cfg, inj, sh)
    cube = cube.to(torch.bfloat16)
    torch.cuda.empty_cache()
    plan = native.Plan(cfg, dtype="bf16", noise="mad")
    stream = torch.cuda.current_stream()
    tile, tile_ms = plan.autotune(cube, reps=2, stream=stream)   # tile of the FP32 slab search
    ops, n_unique = alg_ops(cfg, plan)
    for _ in range(2):
        plan.search(cube, stream=stream)
        cand = plan.candidates()
    times, kern = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.search(cube, stream=stream)
        e1.record(stream)
        cand = plan.candidates()
        times.append(e0.elapsed_time(e1) / 1e3)
        kern.append(plan.last_timing()[0] / 1e3)
    t, tk = statistics.median(times), statistics.median(kern)
    snr_best, idx_best = plan.best()
    pk = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = n_sm * 128 * pk["sm_max_mhz"] * 1e6
    alg_bytes = cfg.n_pix * cfg.n_sub * cfg.n_t * 2 + cfg.n_pix * 16
    plan.close()
    # injections recovered at their pixel with the DM trial nearest their DM (+-2 trials), and
    # candidates elsewhere (false alarms).  Under Student-t (nu = 5) noise 1.4826 MAD is 0.834 of
    # the standard deviation, so the threshold of 6 in MAD units sits at 5.0 standard deviations;
    # 6 / 0.834 = 7.2 is the threshold that corresponds to 6 standard deviations.
    # An injection counts as recovered when its pixel's best trial is above the threshold, its
    # boxcar overlaps the injected one and its largest dispersion shift is within 2 samples of
    # the injected DM's (DM trials with equal shift rows report the lowest DM).
    inj_pix = inj.row * cfg.nx + inj.col
    tab = oracle.delay_table(cfg.freq_mhz, cfg.dm)
    smax_rep = tab.max(axis=1)[np.maximum(idx_best[inj_pix, 0], 0)]
    smax_true = sh.max(axis=1)[:len(inj)]
    t_rep = idx_best[inj_pix, 2]
    w_rep = cfg.widths[np.maximum(idx_best[inj_pix, 1], 0)]
    overlap = (t_rep < inj.t0 + inj.width) & (inj.t0 < t_rep + w_rep)
    hit = (snr_best[inj_pix] > cfg.threshold) & overlap & (np.abs(smax_rep - smax_true) <= 2)
    bright = inj.snr > 15.0
    is_inj = np.zeros(cfg.n_pix, bool)
    is_inj[inj_pix] = True
    fa = int(((snr_best > cfg.threshold) & ~is_inj).sum())
    fa72 = int(((snr_best > cfg.threshold / 0.834) & ~is_inj).sum())
    del cube
    torch.cuda.empty_cache()
    return {"workload": f"{cfg.ny}x{cfg.nx} px x {cfg.n_sub} sub x {cfg.n_t} samples BF16, MAD normalisation, "
                        f"{len(cfg.dm)} DM 0-4000 ({n_unique} distinct rows), {len(cfg.widths)} widths, {n_inj} injections",
            "ms_per_search": t * 1e3, "trials_per_s": cfg.n_trials / t, "candidates": int(len(cand)),
            "injections_recovered": int(hit.sum()), "injection_recall": float(hit.mean()),
            "recall_interval_95": wilson(int(hit.sum()), len(inj)),
            "injection_recall_snr_gt_15": float(hit[bright].mean()),
            "false_alarm_pixels": fa, "false_alarm_fraction": fa / float(cfg.n_pix - len(inj)),
            "false_alarm_pixels_above_7.2": fa72,
            "roofline": {"bound": "alu", "achieved": ops / tk / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                         "frac": ops / tk / peak_ops, "kernel": search_kernel_name(cfg.n_t, 'bf16', 'mad', tile),
                         "kernel_ms": tk * 1e3, "ops_per_launch": ops, "tile": tile, "tile_ms": tile_ms},
            "hbm": {"achieved_gbs": alg_bytes / tk / 1e9, "frac": alg_bytes / tk / 1e9 / pk["hbm_gbs"],
                    "bytes_per_launch": alg_bytes},
            "l2": f"inputs larger than L2 (cube {alg_bytes / 1e9:.1f} GB)"}


# ----------------------------------------------------------------------------- GPU arm

def main():
    global SERVING_FIELDS
    args = parse()
    SERVING_FIELDS = tuple(tuple(int(v) for v in f.split("x")) for f in args.serving_fields.split(","))
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist
    from paper_2510_18136_gb300 import native, synth

    if args.only == "imager":
        print(json.dumps({"imager": imager_section(native, args.imager_steps, seed=args.seed)}), flush=True)
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    cfg = synth.config_full_window(args.ny, args.nx, n_t=args.n_t)
    cfg.sigma_pix = synth.psf_sigma()
    cube, inj = make_cube(native, synth, cfg, args.seed + rank, dev, args.dtype)
    sigma = torch.full((cfg.n_pix,), cfg.sigma_pix * math.sqrt(cfg.n_sub), device=dev)
    plan = native.Plan(cfg, dtype=args.dtype, out=args.out)
    stream = torch.cuda.current_stream()
    # pixel x DM tile of the search kernel: each tile that fits timed on this cube, the fastest kept
    tile, tile_ms = plan.autotune(cube, sigma, reps=3, stream=stream)
    ops, n_unique = alg_ops(cfg, plan)
    elem = 4 if args.dtype == "f32" else 2
    cube_bytes = cfg.n_pix * cfg.n_sub * cfg.n_t * elem
    full_bytes = cfg.n_pix * len(cfg.dm) * len(cfg.widths) * 6 if args.out == "full" else 0
    # cube and sigma read, one 16-byte record per pixel written, and in FULL mode the S/N (f32) and
    # TOA (i16) of every (pixel, DM, width)
    alg_bytes = cube_bytes + cfg.n_pix * 4 + cfg.n_pix * 16 + full_bytes

    # N ranks: the image is N 301-row bands (shard.row_bands of an (N ny) x nx field), one per GPU,
    # each band's candidates gathered to rank 0 and merged in pixel order every step (weak scaling)
    from paper_2510_18136_gb300 import shard
    band = shard.row_bands(cfg.ny * world, world)[rank]

    def step():
        plan.search(cube, sigma, stream=stream)
        c = plan.candidates()
        if world > 1:
            shard.gather_candidates(c, band, cfg.nx, dst=0)
        return c

    for _ in range(max(3, args.warmup)):
        cand = step()

    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    search_ms = []
    ev0.record(stream)
    for _ in range(args.steps):
        cand = step()
        search_ms.append(plan.last_timing()[0])
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    t = torch.tensor([elapsed], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_max = float(t.item())
    value = world * args.steps * cfg.n_trials / elapsed_max

    # end to end: host cube (pinned) -> device -> search -> candidates (and in FULL mode the FULL
    # arrays) back to the host
    host_cube = cube.cpu().pin_memory()
    host_sigma = sigma.cpu().pin_memory()
    plan.search_host(host_cube, host_sigma, stream=stream)
    plan.candidates()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_c = 0
    for _ in range(args.e2e_steps):
        plan.search_host(host_cube, host_sigma, stream=stream)
        n_c = len(plan.candidates())
        if args.out == "full":
            plan.full()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_t = torch.tensor([e2e_s], device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * args.e2e_steps * cfg.n_trials / float(e2e_t.item())

    bf16 = None
    if args.bf16_steps > 0 and rank == 0 and args.dtype == "f32":
        s32, _ = plan.best()
        bf16 = bf16_section(native, synth, cfg, cube, sigma, args.bf16_steps, args.e2e_steps, s32)
    serving = None
    if args.serving_blocks > 0 and rank == 0:
        serving = serving_latency(native, synth, args.serving_blocks, args.serving_paced_blocks, seed=args.seed)
        if args.serving_minutes > 0:
            serving["injection_run"] = serving_injections(native, synth, args.serving_minutes, seed=args.seed)
    classifier, campaigns, clf = None, None, None
    if args.classifier_samples > 0 and rank == 0:
        classifier, clf = classifier_section(native, args.classifier_samples, args.classifier_eval_cubes,
                                             seed=args.seed)
    if args.campaigns and rank == 0:
        campaigns = campaigns_section(native, clf, seed=args.seed)
    if clf is not None:
        clf.close()

    imager = None
    if args.imager_steps > 0 and rank == 0:
        imager = imager_section(native, args.imager_steps, seed=args.seed)
    timescales = None
    if args.timescale_steps > 0 and rank == 0 and args.out == "candidates":
        timescales = timescales_section(native, synth, cube, cfg, sigma, cand, args.timescale_steps)
    stress = None
    if args.stress_steps > 0 and rank == 0:
        stress = stress_section(native, synth, args.stress_steps, seed=args.seed, size=args.stress_size)

    pk = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    kern_s = statistics.mean(search_ms) / 1e3
    achieved = ops / kern_s
    peak_ops = n_sm * 128 * pk["sm_max_mhz"] * 1e6
    hbm_gbs = alg_bytes / kern_s / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": workload_name(cfg), "ny": cfg.ny, "nx": cfg.nx, "n_sub": cfg.n_sub, "n_t": cfg.n_t,
                   "n_dm": len(cfg.dm), "n_unique_dm_rows": n_unique, "widths": [int(w) for w in cfg.widths],
                   "storage": args.dtype, "noise": "known sigma", "output": args.out,
                   "l2": "inputs larger than L2 (cube "
                   f"{cube_bytes / 1e9:.2f} GB)",
                   "parallelism": (f"row bands x{world}: a {cfg.ny * world}x{cfg.nx} image, one {cfg.ny}-row band "
                                   "per GPU, candidate lists gathered to rank 0 each step" if world > 1 else
                                   "one GPU")},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / peak_ops,
                     "traffic": measured_traffic(cfg.ny, cfg.nx, args.dtype),
                     "kernel": search_kernel_name(cfg.n_t, args.dtype, tile=tile, out=args.out),
                     "kernel_ms": kern_s * 1e3, "tile": tile, "tile_ms": tile_ms,
                     "ops_per_launch": ops, "peak_basis": f"{n_sm} SM x 128 FP32 lanes x "
                     f"{pk['sm_max_mhz']:.0f} MHz ({pk['source']} max clock)"},
        "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": pk["hbm_gbs"], "frac": hbm_gbs / pk["hbm_gbs"],
                "bytes_per_launch": alg_bytes, "peak_source": pk["source"]},
        "e2e": {"value": e2e_value, "unit": "trials/s", "h2d_bytes_per_step": cube_bytes + cfg.n_pix * 4,
                "d2h_bytes_per_step": 8 + 24 * n_c + full_bytes},
        "gpu_launches": 3 * args.steps,
        "candidates": int(len(cand)), "injections": int(len(inj)),
        "p99_block_latency_ms": None if serving is None else serving["p99_ms"],
        "bf16": bf16,
        "serving": serving,
        "classifier": classifier,
        "campaigns": campaigns,
        "imager": imager,
        "stress": stress,
        "timescales": timescales,
        "clocks": ck,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, n, t_cpu, cores = oracle_sample_rate(host_cube, cfg, 12.0)
        line["cpu_baseline"] = {"value": r, "unit": "trials/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n} random pixels of the cube, all 64 DM x 12 widths ({t_cpu:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
