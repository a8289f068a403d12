#!/usr/bin/env python
"""Benchmark of the TRED hot path on B300: deposits/s to pixel currents.

One step = drift -> blockbin -> effq -> convolve -> gather -> readout (all hot-path
stages) over one synthetic event already resident in HBM: the module-plane
workload (512 x 512 pixels x 6,400 ticks, tracks drawn until >= 1e6 deposits,
9 x 9 pixel x 100 impact x 200 tick response, 8 x 8 pixel x 256 tick blocks, FFT
16 x 16 x 512, GL-2).  The response spectrum (computed once per response) is timed
separately.  Under torchrun each rank simulates its own independent event (weak
scaling; no collective on the data path, a barrier and a max-reduce for timing).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tred|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "depos/s to pixel currents at <=1e-5 rel L2 vs FP64 oracle; % of HBM/TC roofline"
WORKLOAD = "module1M"
# Algorithmic FLOPs of one block's convolution: 50 packed forward 3-D FFTs of
# N = 16*16*lt points at 5 N log2 N, 50 spectrum products at 8 N, one inverse FFT.
def conv_flop_per_block(lt=512, npairs=50, lp=16):
    import math
    n = lp * lp * lt
    return npairs * 5 * n * math.log2(n) + npairs * 8 * n + 5 * n * math.log2(n)


CONV_FLOP_PER_BLOCK = conv_flop_per_block()
# FP32 ALU peak from unit counts and the maximum clock: 148 SMs x 128 FP32 lanes x
# 2 flop (FMA) x 2.032 GHz.  The measured one (an FMA loop over every SM, tred_fp32_peak)
# is reported beside it.
SMS, FP32_LANES, SM_MAX_GHZ = 148, 128, 2.032
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_GHZ / 1e3


def _profile_figures():
    """Per-block figures of the committed ncu capture of the convolution on module20
    (profiles/conv_traffic_module20.txt) with the source hashes they were taken at."""
    path = os.path.join(ROOT, "profiles", "conv_traffic_module20.txt")
    kv = {}
    try:
        for line in open(path):
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if len(parts) >= 3 and parts[1] == "sha256":
                kv[parts[0]] = parts[2]
            elif len(parts) >= 2:
                kv[parts[0]] = float(parts[1])
    except OSError:
        pass
    return kv


CONV_SOURCES = ("k_conv.cu", "conv_item.cuh", "tred_internal.cuh")


def _source_sha(names=CONV_SOURCES):
    """sha256 over the convolution's source files (the kernels and the headers they use)."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_2602_12052_b300", "csrc", name), "rb").read())
    return h.hexdigest()


def conv_traffic(blocks):
    """DRAM bytes of one tred_convolve call over `blocks` active blocks: the per-block
    read + write bytes of an ncu capture (profiles/conv_traffic_module20.txt), scaled by
    the blocks, or None when the convolution source changed since the capture."""
    kv = _profile_figures()
    if kv.get("conv_sources") != _source_sha() or "conv_dram_bytes_per_block" not in kv:
        return None, "capture predates the current convolution sources"
    per = kv["conv_dram_bytes_per_block"]
    return per * blocks, ("ncu dram__bytes_read+write of module20 (255 blocks), "
                          f"{per:.4g} B per block, scaled to {blocks} blocks")


def conv_counters():
    """Executed FP32 FLOPs per block (2 FFMA + FADD + FMUL thread instructions) and the
    FMA-pipe share of the spectral kernel, from the same capture, or {} when stale."""
    kv = _profile_figures()
    if kv.get("conv_sources") != _source_sha():
        return {}
    out = {}
    for k in ("conv_executed_flop_per_block", "conv_spec_fma_pipe_pct", "conv_spec_issue_active_pct"):
        if k in kv:
            out[k] = kv[k]
    return out


DIRECT_SOURCES = ("k_direct.cu", "tred_internal.cuh")


def _direct_figures():
    """Per-row / per-block DRAM bytes of the direct form's kernels from the committed ncu
    capture on module20 (profiles/direct_kernels_module20.txt) and its source hash."""
    path = os.path.join(ROOT, "profiles", "direct_kernels_module20.txt")
    kv = {}
    try:
        for line in open(path):
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if len(parts) >= 3 and parts[1] == "sha256":
                kv[parts[0]] = parts[2]
            elif len(parts) >= 2:
                kv[parts[0]] = float(parts[1])
    except OSError:
        pass
    return kv


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def direct_rooflines(cfg, rows, cols, blocks, kms, clocks, pixels=0):
    """Roofline objects of the direct form's kernels (conv_mode 4) and of the effective
    charge, each from its algorithmic work per step over its CUDA-event time (kms: kernel
    name -> ms per step); the dominant (longest) one first.
      k_dx_gemm  tensor: 3 split-BF16 products x 8 real FLOPs per complex MAC over
                 rows x n_sub^2 impacts x kp^2 taps x (lt/2 + 1) bins
      k_dx_fwd   HBM: the rows' non-empty Q^eff columns read (bt x 4 B each), their
                 spectra written (rows x (lt/2 + 1) bins x kq x 2 parts x 2 B)
      k_dx_inv   HBM: the block spectra read (blocks x bins x 256 x 8 B), the block
                 outputs written (blocks x 256 x lt x 4 B)
      k_dx_wave  HBM: the block spectra read (blocks x bins x 256 x 8 B), the pixel
                 waveforms written (pixels x nt x 4 B)"""
    pk = _peaks()
    hbm = pk.get("hbm_gbs", 6400.0)
    bf16 = pk.get("bf16_tflops_sustained", 1400.0)
    src = "measured (MEASURED_PEAKS.json)" if pk else "fallback"
    nch, ntap, nbins = cfg.n_sub ** 2, cfg.kp ** 2, cfg.lt // 2 + 1
    kq = 32 * ((nch + 15) // 16)
    figs = _direct_figures()
    fresh = figs.get("direct_sources") == _source_sha(DIRECT_SOURCES)
    out = {}
    if kms.get("k_dx_gemm"):
        fl = 3.0 * 8.0 * rows * nch * ntap * nbins
        a = fl / (kms["k_dx_gemm"] / 1e3) / 1e12
        out["k_dx_gemm"] = {"bound": "tensor", "achieved": a, "peak": bf16, "unit": "TFLOP/s", "frac": a / bf16,
                            "flop_per_step": fl, "ms": kms["k_dx_gemm"],
                            "peak_source": f"bf16 dense, sustained (kernel timed inside the step), {src}"}
    if kms.get("k_dx_fwd"):
        by = cols * cfg.bt * 4.0 + rows * nbins * kq * 4.0
        a = by / (kms["k_dx_fwd"] / 1e3) / 1e9
        out["k_dx_fwd"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                           "bytes_per_step": by, "ms": kms["k_dx_fwd"], "peak_source": f"copy bandwidth, {src}"}
    if kms.get("k_dx_inv"):
        by = blocks * (nbins * 256 * 8.0 + 256 * cfg.lt * 4.0)
        a = by / (kms["k_dx_inv"] / 1e3) / 1e9
        out["k_dx_inv"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                           "bytes_per_step": by, "ms": kms["k_dx_inv"], "peak_source": f"copy bandwidth, {src}"}
    if kms.get("k_dx_wave"):
        by = blocks * nbins * 256 * 8.0 + pixels * cfg.nt * 4.0
        a = by / (kms["k_dx_wave"] / 1e3) / 1e9
        out["k_dx_wave"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                            "bytes_per_step": by, "ms": kms["k_dx_wave"], "peak_source": f"copy bandwidth, {src}"}
    for k, r in out.items():
        r["kernel"] = k
        unit = "row" if k in ("k_dx_fwd", "k_dx_gemm") else "block"
        per = figs.get(f"{k}_dram_bytes_per_{unit}")
        rd, wr = figs.get(f"{k}_dram_read_bytes_per_block"), figs.get(f"{k}_dram_write_bytes_per_pixel")
        if fresh and rd and wr:   # reads scale with the blocks, writes with the pixels
            r["traffic"] = rd * blocks + wr * pixels
            r["traffic_source"] = (f"ncu dram__bytes_read of module20 per block ({rd:.4g} B) x {blocks} blocks + "
                                   f"dram__bytes_write per pixel ({wr:.4g} B) x {pixels} pixels")
        elif fresh and per:
            n_units = rows if unit == "row" else blocks
            r["traffic"] = per * n_units
            r["traffic_source"] = (f"ncu dram__bytes_read+write of module20, {per:.4g} B per {unit}, "
                                   f"scaled to {n_units} {unit}s")
        else:
            r["traffic"] = None
            r["traffic_source"] = "no capture at the current sources"
        if clocks and clocks.get("sm_mhz") and r["bound"] == "tensor":
            r["frac_at_observed_clock"] = r["achieved"] / (r["peak"] * clocks["sm_mhz"] / 2032.0)
    order = sorted(out, key=lambda k: -out[k]["ms"])
    return {k: out[k] for k in order}


def measured_fp32_peak():
    """FP32 FMA TFLOP/s and SM count measured on this device (tred_fp32_peak)."""
    from paper_2602_12052_b300 import tred
    tf, sms = tred.tred_fp32_peak(iters=32768)
    return tf, sms


def alu_roofline(kernel, flop_per_block, blocks, ms, clocks, peak_meas=None):
    """The FP32-ALU roofline object of a convolution-dominated form: algorithmic FLOPs
    (unpruned 5 N log2 N count) per launch over its CUDA-event time, against the
    unit-count peak and the measured FMA-loop peak."""
    achieved = flop_per_block * blocks / (ms / 1e3) / 1e12
    r = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
         "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
         "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz (unit counts, max clock)",
         "flop_per_block": flop_per_block, "blocks": blocks, "ms": ms}
    if peak_meas:
        r["peak_measured"] = peak_meas
        r["frac_vs_measured"] = achieved / peak_meas
    if clocks and clocks.get("sm_mhz"):
        r["frac_at_observed_clock"] = achieved / (FP32_PEAK_TFLOPS * clocks["sm_mhz"] / 2032.0)
    return r


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tred", choices=["tred", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--cpu-sample", type=int, default=12000,
                    help="deposits of the workload timed through the CPU oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", default="step",
                    choices=["step", "batched", "adjoint", "spill", "accuracy", "chunking", "lines", "binsize", "sizes"],
                    help="step: one event (default); batched: 64 uneven events, autotuned, CUDA graph; "
                         "adjoint: forward + backward; spill: 35 planes in sequence")
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--chunk-blocks", type=int, default=8192,
                    help="batched mode: slots per effective-charge / convolution chunk (the dense Q^eff chunk "
                         "takes 6.55 MB per slot at 8x8x256 blocks)")
    ap.add_argument("--graph", action="store_true",
                    help="step mode: time the step replayed from a CUDA graph (the launch sequence is "
                         "fixed and every count stays on the device); the per-stage times come from "
                         "the eager steps")
    ap.add_argument("--readout-mode", type=int, default=0, choices=[0, 1, 2],
                    help="0: trigger-reset (default); 1: successive digitisations without resets "
                         "(--n-samples per trigger); 2: fixed-charge integration")
    ap.add_argument("--n-samples", type=int, default=3, help="digitisations per trigger in readout mode 1")
    ap.add_argument("--fuse-gather", type=int, default=1, choices=[0, 1],
                    help="conv_mode 4: the inverse time DFT fused with the electrode gather "
                         "(tred_convolve_gather_readout) where the block shape allows it")
    ap.add_argument("--fused", type=int, default=0, choices=[0, 1],
                    help="step mode: 1 = the effective charge and the convolution as one persistent launch "
                         "over the active-block queue (tred_effq_convolve)")
    ap.add_argument("--conv-mode", type=int, default=4, choices=[0, 1, 2, 3, 4],
                    help="4: time DFT by FFT, impacts x taps per bin as a split-BF16 tcgen05 GEMM (default); "
                         "0: FP32 FFT convolution; 1: time DFT as a tcgen05 GEMM in TF32; "
                         "2: the same in split TF32 (three products); 3: the same in split BF16 (three products)")
    return ap.parse_args()


def replica_seed(cfg, rank: int) -> int:
    """Seed of rank `rank`'s independent event (replicas: every rank simulates its own)."""
    return cfg.seed + 7919 * rank


def aggregate_replicas(n_local: float, ms_local: float, world: int, device=None):
    """Whole-job totals of independent replicas: the units all ranks processed and the
    slowest rank's time (max over ranks).  The only collectives of the multi-GPU path;
    nothing on the data path."""
    if world <= 1:
        return float(n_local), float(ms_local)
    import torch
    import torch.distributed as dist
    n_t = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    m_t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(n_t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m_t, op=dist.ReduceOp.MAX)
    return float(n_t.item()), float(m_t.item())


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(cfg, dep, resp, sample: int):
    """The FP64 oracle as it stands, on the first `sample` deposits of the workload."""
    import oracle
    sub = {k: v[:sample] for k, v in dep.items()}
    t = time.perf_counter()
    r = oracle.simulate(cfg, sub, resp)
    dt = time.perf_counter() - t
    return {"value": sample / dt, "unit": "depos/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"first {sample} deposits of the {cfg.name} event, full path to pixel currents "
                       f"({len(r['block_ids'])} blocks, {len(r['pixel_ids'])} pixels), {dt:.1f} s")}


def probe_capacities(cfg, dep, dev):
    """Active blocks of this event (drift + blockbin through the ABI, untimed set-up)
    so that the device buffers are sized to the workload."""
    import torch
    from paper_2602_12052_b300 import tred
    n = len(dep["x"])
    h = tred.Handle(tred.geometry(cfg), tred.params(cfg), n, cfg.n_blocks, 1)
    deps = tred.DepositBuffers(n, dev)
    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    ids = torch.zeros(cfg.n_blocks, dtype=torch.int32, device=dev)
    cnt = torch.zeros_like(ids)
    off = torch.zeros(cfg.n_blocks + 1, dtype=torch.int32, device=dev)
    idx = torch.zeros(8 * n, dtype=torch.int32, device=dev)
    nbd = torch.zeros(1, dtype=torch.int32, device=dev)
    tred.tred_drift(h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], deps)
    tred.tred_blockbin(h, n, deps, ids, cnt, off, idx, nbd)
    nb = int(nbd.item())
    h.close()
    side = cfg.bp + cfg.kp - 1
    return max(nb, 1) + 8, min(cfg.npx * cfg.npx, max(nb, 1) * side * side)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import synth
    cfg = synth.get_config(args.config)
    dep, resp = synth.make_event(cfg)
    sample = max(1000, args.cpu_sample // 3)
    times = []
    for k in range(args.warmup + args.steps):
        off = (k * sample) % max(1, len(dep["x"]) - sample)
        sub = {kk: v[off:off + sample] for kk, v in dep.items()}
        import oracle
        t = time.perf_counter()
        oracle.simulate(cfg, sub, resp)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    import oracle
    ms = 1e3 * statistics.mean(times)
    value = sample / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "depos/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{cfg.name}: 512x512 px x 6400 ticks, {len(dep['x'])} deposits",
                   "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "depos/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{sample} consecutive deposits of the {cfg.name} event per step"},
        "e2e": {"value": value, "unit": "depos/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _line(metric, value, unit, ms, args, cfg_extra, **kw):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": kw.pop("dtype", "f32"), "data": "synthetic", "config": cfg_extra}
    line.update(kw)
    print(json.dumps(line), flush=True)


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def run_batched(args):
    """Config 3: uneven events (deposit counts log-uniform in [1e3, 1e6]) in one pass
    per kernel over the global active-block list, captured in a CUDA graph, with the
    block shape and FFT length picked by the autotuner; against one event at a time."""
    import torch
    import synth
    from paper_2602_12052_b300 import autotune, tred
    torch.cuda.set_device(0)
    base = synth.get_config("module200")
    resp = torch.from_numpy(synth.make_response(base))
    events = synth.make_events(base, args.events, 1000, 1_000_000, seed=3003)
    ntot = sum(len(e["x"]) for e in events)
    t = time.perf_counter()
    cm = args.conv_mode if args.conv_mode in (0, 4) else 0
    best, timings = autotune.autotune(base, events, resp, sample=8, conv_mode=cm)
    tune_s = time.perf_counter() - t
    cfg = base.with_(bp=best[0], bt=best[1], lt=best[2])
    sim = autotune.make_batch(cfg, events, resp, chunk_blocks=args.chunk_blocks, conv_mode=cm)
    sim.step()
    torch.cuda.synchronize()
    st = sim.status()
    if st[0] != 0:
        raise RuntimeError(f"device status {st}")
    nb, npix, nh = (int(v) for v in sim.counts[:3].cpu())
    sim.capture()
    with ClockSampler(0) as clk:
        ms_graph = _timed(sim.replay, args.steps, 1)
    clocks = clk.summary()
    # the convolution's own time, from an eager step with events around its launches (and
    # the library's per-kernel events)
    cev = []
    tred.tred_set_kernel_timing(sim.h, True)
    tred.tred_direct_counts(sim.h)
    sim.step(conv_events=cev)
    torch.cuda.synchronize()
    conv_ms = sum(a.elapsed_time(b) for a, b in cev)
    kernel_ms = {}
    for cls, name in tred.KT_NAMES.items():
        kt, kn = tred.tred_kernel_time(sim.h, cls)
        if kn:
            kernel_ms[name] = kt
    tred.tred_set_kernel_timing(sim.h, False)
    rows_dx, cols_dx = tred.tred_direct_counts(sim.h)
    peak_meas, sms = measured_fp32_peak()
    if cm == 4:
        kr = direct_rooflines(cfg, rows_dx, cols_dx, nb, kernel_ms, clocks, npix)
        roof = dict(kr[next(iter(kr))])
        roof.update({"kernels": kr, "kernel_ms_per_step": kernel_ms, "rows": rows_dx, "nonempty_columns": cols_dx,
                     "convolution_ms": conv_ms})
    else:
        roof = alu_roofline("tred_convolve_range (k_conv_spec + inverse time transform), all chunks of one step",
                            conv_flop_per_block(cfg.lt), nb, conv_ms, clocks, peak_meas)
    batch_fused = sim.fuse_gather
    del sim
    torch.cuda.empty_cache()
    # one event at a time through the same kernels (no graph, one launch sequence each)
    nmax = max(len(e["x"]) for e in events)
    bmax = max(autotune.probe_blocks(cfg, [e], resp)[0] for e in events)
    one = tred.BatchSimulator(cfg, resp, [events[0]], max_blocks=bmax + 8,
                              max_pixels=min(cfg.npx * cfg.npx, (bmax + 8) * (cfg.bp + cfg.kp - 1) ** 2),
                              chunk_blocks=args.chunk_blocks, n_events=1, max_deposits=nmax, conv_mode=cm,
                              fuse_gather=batch_fused)
    per_event = []
    for e in events:
        one.load([e])
        per_event.append(_timed(one.step, 1, 1))
        st = one.status()
        if st[0] != 0:
            raise RuntimeError(f"device status {st} on a single event of {len(e['x'])} deposits")
    ms_single = sum(per_event)
    _line("events/s and depos/s, 64 uneven events batched in one CUDA graph vs one at a time",
          ntot / (ms_graph / 1e3), "depos/s", ms_graph, args,
          {"workload": f"{args.events} events, deposits log-uniform in [1e3, 1e6] (total {ntot}), "
                       "512x512 px x 6400 ticks each, 9x9x10x10x200 response",
           "active_blocks": nb, "active_pixels": npix, "hits": nh,
           "autotuned_shape": {"bp": best[0], "bt": best[1], "lt": best[2]},
           "autotune_ms_per_kdepos": {f"{k[0]}x{k[0]}x{k[1]}/lt{k[2]}": 1e3 * v for k, v in timings.items()},
           "autotune_s": tune_s,
           "convolution": {0: "FFT form, persistent effective charge + convolution over the block queue",
                           4: f"direct spatial form (tensor-core GEMM per frequency bin), chunks of {args.chunk_blocks} blocks"
                              + (" up to the output spectra (kept for every slot), then the inverse time DFT "
                                 "fused with the gather per 8x8 pixel tile" if batch_fused else "")}[cm]},
          dtype={0: "f32", 4: "f32+bf16x3"}[cm],
          events_per_s=args.events / (ms_graph / 1e3),
          per_event={"ms_total": ms_single, "depos_per_s": ntot / (ms_single / 1e3),
                     "events_per_s": args.events / (ms_single / 1e3)},
          speedup_vs_per_event=ms_single / ms_graph, clocks=clocks, roofline=roof)


def run_lines(args):
    """Line-shape track segments (Sec. II-C, Eq. qline): a 200-track module plane in
    3 mm segments through segment transport, binning, the segments' effective charge,
    convolution, gather and readout; segments/s with per-stage times."""
    import torch
    import synth
    from paper_2602_12052_b300 import tred
    torch.cuda.set_device(0)
    cfg = synth.get_config("module_lines")
    seg = synth.make_segments(cfg, synth.SEG_CM["module_lines"])
    resp = torch.from_numpy(synth.make_response(cfg))
    n = len(seg["x0"])
    cm = args.conv_mode if args.conv_mode in (0, 4) else 0
    fg = cm == 4 and tred.fused_gather_shape_ok(cfg, cm)   # the inverse time DFT fused with the gather
    sim = tred.LineSimulator(cfg, resp, max_segments=n, max_blocks=6000, max_pixels=300000, effq_skip_empty=1,
                             conv_mode=cm, fuse_gather=fg)
    x = {k: torch.from_numpy(v).cuda() for k, v in seg.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def stages(ev):
        h = sim.h
        ev[0].record()
        tred.tred_drift_lines(h, n, x["x0"], x["y0"], x["z0"], x["x1"], x["y1"], x["z1"], x["t0"], x["ne"],
                              sim.deps, sim.half)
        tred.tred_blockbin(h, n, sim.deps, sim.block_ids, sim.block_counts, sim.dep_offsets, sim.dep_index,
                           sim.n_blocks_dev)
        ev[1].record()
        tred.tred_effq_lines(h, n, sim.deps, sim.half, sim.block_ids, sim.dep_offsets, sim.dep_index,
                             sim.n_blocks_dev, sim.qeff)
        ev[2].record()
        if fg:   # spectra, then the inverse time DFT per pixel tile into the waves, readout (one stage)
            tred.tred_convolve_gather_readout(h, sim.block_ids, sim.n_blocks_dev, sim.qeff, sim.pixel_ids,
                                              sim.waveforms, sim.n_pixels_dev, sim.rp, sim.hit_pixel, sim.hit_tick,
                                              sim.hit_charge, sim.n_hits_dev)
            ev[3].record()
            ev[4].record()
            return
        tred.tred_convolve(h, sim.block_ids, sim.n_blocks_dev, sim.qeff, sim.out_blocks)
        ev[3].record()
        tred.tred_gather_readout(h, sim.block_ids, sim.n_blocks_dev, sim.out_blocks, sim.pixel_ids, sim.waveforms,
                                 sim.n_pixels_dev, sim.rp, sim.hit_pixel, sim.hit_tick, sim.hit_charge,
                                 sim.n_hits_dev)
        ev[4].record()
    for _ in range(args.warmup):
        stages([torch.cuda.Event(enable_timing=True) for _ in range(5)])
    torch.cuda.synchronize()
    st = sim.status()
    if st[0] != 0:
        raise RuntimeError(f"device status {st}")
    rows = []
    tred.tred_set_kernel_timing(sim.h, True)
    tred.tred_direct_counts(sim.h)
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            stages(ev)
            torch.cuda.synchronize()
            rows.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    kernel_ms = {}
    for cls, name in tred.KT_NAMES.items():
        kt, kn = tred.tred_kernel_time(sim.h, cls)
        if kn:
            kernel_ms[name] = kt / args.steps
    tred.tred_set_kernel_timing(sim.h, False)
    rows_dx, cols_dx = (v // args.steps for v in tred.tred_direct_counts(sim.h))
    m = [statistics.mean(r[i] for r in rows) for i in range(4)]
    ms = sum(m)
    nb, npix, nh = (int(v) for v in sim.counts[:3].cpu())
    clocks = clk.summary()
    peak_meas, _ = measured_fp32_peak()
    if cm == 4:
        kr = direct_rooflines(cfg, rows_dx, cols_dx, nb, kernel_ms, clocks, npix)
        roof = dict(kr[next(iter(kr))])
        roof.update({"kernels": kr, "kernel_ms_per_step": kernel_ms, "rows": rows_dx, "nonempty_columns": cols_dx})
    else:
        roof = alu_roofline("tred_convolve (k_conv_spec + k_conv_itime_mp)", conv_flop_per_block(cfg.lt), nb, m[2],
                            clocks, peak_meas)
    _line("line segments/s to pixel currents (Eq. qline effective charge)", n / (ms / 1e3), "segments/s", ms, args,
          {"workload": f"module_lines: {n} segments of 3 mm from 200 tracks, 512x512 px x 6400 ticks, GL-2, "
                       "9x9x10x10x200 response, 8x8x256 blocks"
                       + (", inverse time DFT fused with the gather per 8x8 pixel tile" if fg else ""),
           "active_blocks": nb, "active_pixels": npix, "hits": nh,
           "l2": "flushed between timed steps"},
          stages_ms=({"drift+blockbin": m[0], "effq_lines": m[1], "convolve+gather+readout": m[2] + m[3]} if fg else
                     {"drift+blockbin": m[0], "effq_lines": m[1], "convolve": m[2], "gather+readout": m[3]}),
          clocks=clocks, roofline=roof, dtype={0: "f32", 4: "f32+bf16x3"}[cm],
          cpu_baseline=None if args.no_cpu_baseline else _lines_cpu(cfg, seg, resp.numpy()))


def _lines_cpu(cfg, seg, resp, k=400):
    """The FP64 oracle on the first k segments of the workload (every pixel they
    reach), on the host cores."""
    import oracle
    sub = {kk: v[:k] for kk, v in seg.items()}
    t = time.perf_counter()
    r = oracle.simulate_lines(cfg, sub, resp)
    dt = time.perf_counter() - t
    return {"value": k / dt, "unit": "segments/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {k} segments of module_lines, full path to pixel currents "
                      f"({len(r['block_ids'])} blocks, {len(r['pixel_ids'])} pixels), {dt:.1f} s"}


def run_adjoint(args):
    """Config 4: forward + backward (adjoint) deposits/s and peak device memory."""
    import torch
    import synth
    from paper_2602_12052_b300 import tred
    torch.cuda.set_device(0)
    cfg = synth.get_config("module200")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    dev = torch.device("cuda")
    max_blocks, max_pixels = probe_capacities(cfg, dep, dev)
    max_blocks = int(max_blocks * 1.3) + 8
    max_pixels = min(cfg.npx * cfg.npx, int(max_pixels * 1.3))
    free0, total = torch.cuda.mem_get_info()
    # the forward in the FP32 FFT form: the gradients meet the 1e-4 bar against the oracle
    # (with the direct form's split-BF16 products they come within 3e-4)
    cm = 0
    sim = tred.Simulator(cfg, torch.from_numpy(resp), max_deposits=n, max_blocks=max_blocks,
                         max_pixels=max_pixels, device=dev, conv_mode=cm, effq_skip_empty=1 if cm == 4 else 0,
                         fuse_gather=tred.fused_gather_shape_ok(cfg, cm))
    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"], readout=False)
    npix = int(sim.counts[1].item())
    tid, twave = sim.pixel_ids[:npix].clone(), sim.waveforms[:npix].clone()
    st = tred.DiffState(sim)
    p = [torch.tensor(v * 1.3, requires_grad=True) for v in (cfg.DL_cm2_per_s, cfg.DT_cm2_per_s, cfg.lifetime_us)]

    def fwd_bwd():
        loss = tred.TredLoss.apply(st, tid, twave, x["x"], x["y"], x["z"], x["t0"], x["ne"], *p)
        loss.backward()

    with ClockSampler(0) as clk:
        ms = _timed(fwd_bwd, args.steps, args.warmup)
        # the backward's dominant call alone: tred_adjoint (correlation with the response,
        # inverse transforms, chain rule) after one forward
        loss = tred.TredLoss.apply(st, tid, twave, x["x"], x["y"], x["z"], x["t0"], x["ne"], *p)

        def adj():
            tred.tred_adjoint(sim.h, n, sim.deps, sim.block_ids, sim.dep_offsets, sim.dep_index, sim.n_blocks_dev,
                              sim.pixel_ids, sim.n_pixels_dev, st.resid, sim.qeff, st.grad7)
        adj_ms = _timed(adj, args.steps, 1)
    clocks = clk.summary()
    free1, _ = torch.cuda.mem_get_info()
    nb = int(sim.counts[0].item())
    peak_meas, _ = measured_fp32_peak()
    roof = alu_roofline("tred_adjoint (k_adj_spec + k_adj_itime512 + k_adj_chain); the backward correlation "
                        "counted as one convolution's FLOPs", conv_flop_per_block(cfg.lt), nb, adj_ms, clocks,
                        peak_meas)
    stored_gb = nb * cfg.n_sub ** 2 * cfg.bp ** 2 * cfg.bt * 4 * (1 + 2 * cfg.gl_order ** 3) / 1e9
    _line("forward+backward depos/s (gradients of an L2 loss w.r.t. deposit x/y/t0/ne, DL, DT, lifetime)",
          n / (ms / 1e3), "depos/s", ms, args,
          {"workload": f"module200 event: {n} deposits, 512x512 px x 6400 ticks, GL-2, starts at 1.3x truth",
           "active_blocks": nb,
           "forward": {0: "FFT form", 4: "direct spatial form"}[cm]
                      + (", the inverse time DFT fused with the gather" if sim.fuse_gather else "")},
          memory={"device_bytes_in_use": int(total - free1), "before_handle": int(total - free0),
                  "note": "quadrature recomputed in the backward; dL/dQeff reuses the forward's Q^eff buffer",
                  "stored_quadrature_estimate_gb": stored_gb},
          clocks=clocks, roofline=roof, adjoint_call_ms=adj_ms)


def run_spill(args):
    """Config 5: ~1e7 deposits over 35 module planes, processed one plane after the
    other on one GPU; GL-3, 13x13x10x10x400 response, 4x4x256 blocks, FFT 16x16x768."""
    import torch
    import synth
    from paper_2602_12052_b300 import autotune, tred
    torch.cuda.set_device(0)
    cfg = synth.get_config("spill_plane")
    resp = torch.from_numpy(synth.make_response(cfg))
    planes = [synth.make_deposits(cfg, seed=cfg.seed * 100 + k) for k in range(35)]
    ntot = sum(len(p["x"]) for p in planes)
    nmax = max(len(p["x"]) for p in planes)
    bmax = max(autotune.probe_blocks(cfg, [p], resp)[0] for p in planes[:6]) * 2
    free0, total = torch.cuda.mem_get_info()
    one = tred.BatchSimulator(cfg, resp, [planes[0]], max_blocks=bmax,
                              max_pixels=min(cfg.npx * cfg.npx, bmax * (cfg.bp + cfg.kp - 1) ** 2),
                              chunk_blocks=4096, n_events=1, max_deposits=nmax)
    dev_planes = [{k: torch.from_numpy(v).cuda() for k, v in p.items()} for p in planes]

    def all_planes():
        for p in dev_planes:
            n = p["x"].numel()
            for k in ("x", "y", "z", "t0", "ne"):
                one.inputs[k][:n].copy_(p[k])
            one.n = n
            one.step()

    with ClockSampler(0) as clk:
        ms = _timed(all_planes, max(1, args.steps // 2), 1)
        # the convolution's own time over all planes (events around its launches) and the
        # planes' active blocks, from one more pass
        cev, nbs = [], 0
        for pl in dev_planes:
            nn = pl["x"].numel()
            for k in ("x", "y", "z", "t0", "ne"):
                one.inputs[k][:nn].copy_(pl[k])
            one.n = nn
            one.step(conv_events=cev)
            nbs += int(one.counts[0].item())
        torch.cuda.synchronize()
        conv_ms = sum(a.elapsed_time(b) for a, b in cev)
    clocks = clk.summary()
    free1, _ = torch.cuda.mem_get_info()
    st = one.status()
    peak_meas, _ = measured_fp32_peak()
    npairs = cfg.n_sub * cfg.n_sub // 2
    roof = alu_roofline("tred_convolve_range over the 35 planes (k_conv_spec + k_conv_itime)",
                        conv_flop_per_block(cfg.lt, npairs), nbs, conv_ms, clocks, peak_meas)
    roof["note"] = ("4 x 4-pixel blocks: each 16 x 16 spatial plane holds a 4 x 4 input, whose zero rows and "
                    "columns the kernel's half-zero stages skip; the unpruned 5 N log2 N count credits that "
                    "padding, so the fraction can exceed 1 (it is a count, not executed FLOPs)")
    dense = 35 * cfg.npx * cfg.npx * cfg.nt * 4
    _line("depos/s over 35 module planes in sequence (spill scale)", ntot / (ms / 1e3), "depos/s", ms, args,
          {"workload": f"35 planes x 512x512 px x 6400 ticks, {ntot} deposits, GL-3, 13x13x10x10x400 response, "
                       "4x4x256 blocks, FFT 16x16x768"},
          memory={"device_bytes_in_use": int(total - free1),
                  "dense_pixel_current_estimate_bytes": dense,
                  "dense_subpixel_qeff_estimate_bytes": dense * cfg.n_sub ** 2},
          status=st[:2], clocks=clocks, roofline=roof)


def run_accuracy(args):
    """The paper's accuracy study (Sec. IV-B): maximum deviation, per pixel, of the
    charge accumulated in 100 ns windows, for grid-point sampling (GL-1) and the
    2-point rule, each against the 4-point rule; module-plane event."""
    import numpy as np
    import torch
    import synth
    from paper_2602_12052_b300 import tred
    torch.cuda.set_device(0)
    base = synth.get_config("module200")
    dep, resp = synth.make_event(base)
    dev = torch.device("cuda")
    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    n = len(dep["x"])
    max_blocks, max_pixels = probe_capacities(base, dep, dev)
    out = {}
    clk = ClockSampler(0).__enter__()
    for gl in (1, 2, 4):
        cfg = base.with_(gl_order=gl)
        sim = tred.Simulator(cfg, torch.from_numpy(resp), max_deposits=n, max_blocks=max_blocks,
                             max_pixels=max_pixels, device=dev)
        sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"], readout=False)
        npix = int(sim.counts[1].item())
        w = sim.waveforms[:npix].double()
        ticks_per_window = int(round(0.1 / cfg.tick_us))                # 100 ns
        q = w[:, : cfg.nt // ticks_per_window * ticks_per_window].reshape(npix, -1, ticks_per_window).sum(-1)
        out[gl] = (sim.pixel_ids[:npix].cpu().numpy(), q)
        del sim
        torch.cuda.empty_cache()
    clk.__exit__(None, None, None)
    assert all(np.array_equal(out[1][0], out[k][0]) for k in (2, 4))
    res = {}
    for gl in (1, 2):
        dev_max = (out[gl][1] - out[4][1]).abs().max(dim=1).values.cpu().numpy()
        res[f"GL-{gl}"] = {p: float(np.percentile(dev_max, p)) for p in (50, 90, 99, 100)}
    _line("max deviation of accumulated charge per pixel per 100 ns vs the 4-point rule (electrons)",
          res["GL-2"][100], "e-", 0.0, args,
          {"workload": f"module200 event, {n} deposits, {len(out[4][0])} pixels", "noise_scale_e": 500},
          percentiles=res, higher_is_better=False, clocks=clk.summary())


def run_chunking(args):
    """Sub-dimensional chunking (Sec. III-B-2): peak device memory and time of one
    module-plane step vs the number of active blocks per effective-charge chunk."""
    import torch
    import synth
    from paper_2602_12052_b300 import autotune, tred
    torch.cuda.set_device(0)
    cfg = synth.get_config("module1M")
    dep, resp = synth.make_event(cfg)
    resp = torch.from_numpy(resp)
    nb, npix = autotune.probe_blocks(cfg, [dep], resp)
    rows = []
    clk = ClockSampler(0).__enter__()
    for chunk in (256, 1024, 4096, nb + 8):
        torch.cuda.empty_cache()
        free0, total = torch.cuda.mem_get_info()
        sim = tred.BatchSimulator(cfg, resp, [dep], max_blocks=nb + 8, max_pixels=npix, chunk_blocks=chunk)
        ms = _timed(sim.step, 2, 1)
        free1, _ = torch.cuda.mem_get_info()
        rows.append({"chunk_blocks": chunk, "device_bytes": int(free0 - free1), "ms": ms,
                     "qeff_bytes": sim.qeff.numel() * 4})
        del sim
    clk.__exit__(None, None, None)
    _line("device memory of one module-plane step vs effective-charge chunk size", rows[0]["device_bytes"],
          "bytes", rows[0]["ms"], args, {"workload": f"module1M event, {len(dep['x'])} deposits, {nb} blocks"},
          rows=rows, higher_is_better=False, clocks=clk.summary())


def run_binsize(args):
    """The paper's bin-size study (Sec. IV-B): the block-sparse binning's time and the
    whole step's time on the module-plane event for time-bin (block) lengths of 64 to 640
    ticks, each with the smallest supported FFT length at or above bt + nr - 1."""
    import torch
    import synth
    from paper_2602_12052_b300 import tred
    torch.cuda.set_device(0)
    base = synth.get_config("module1M")
    dep, resp = synth.make_event(base)
    n = len(dep["x"])
    dev = torch.device("cuda")
    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    rows = []
    cm = args.conv_mode if args.conv_mode in (0, 4) else 0
    clk = ClockSampler(0).__enter__()
    for bt, lt in ((64, 384), (128, 384), (256, 512), (320, 768), (640, 1024)):
        if cm == 4 and lt not in (384, 512):
            continue   # the direct form's time DFT lengths
        cfg = base.with_(bt=bt, lt=lt)
        max_blocks, max_pixels = probe_capacities(cfg, dep, dev)
        fg = tred.fused_gather_shape_ok(cfg, cm)   # the fused inverse + gather where the shape allows it
        sim = tred.Simulator(cfg, torch.from_numpy(resp), max_deposits=n, max_blocks=max_blocks,
                             max_pixels=max_pixels, effq_skip_empty=1, device=dev, conv_mode=cm, fuse_gather=fg)

        def binning():
            tred.tred_drift(sim.h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], sim.deps)
            tred.tred_blockbin(sim.h, n, sim.deps, sim.block_ids, sim.block_counts, sim.dep_offsets,
                               sim.dep_index, sim.n_blocks_dev)

        def step():
            sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"])

        bin_ms = _timed(binning, args.steps, args.warmup)
        step_ms = _timed(step, args.steps, args.warmup)
        st = sim.status()
        if st[0] != 0:
            raise RuntimeError(f"device status {st} at bt={bt}")
        nb = int(sim.counts[0].item())
        rows.append({"bt": bt, "lt": lt, "active_blocks": nb, "binning_ms": bin_ms, "step_ms": step_ms,
                     "depos_per_s": n / (step_ms / 1e3), "fused_gather": fg})
        del sim
        torch.cuda.empty_cache()
    clk.__exit__(None, None, None)
    best = min(rows, key=lambda r: r["step_ms"])
    _line("depos/s vs time-bin (block) length, module-plane event (bin-size study)", best["depos_per_s"],
          "depos/s", best["step_ms"], args,
          {"workload": f"module1M event, {n} deposits, 8x8-pixel blocks, bt = 64 ... 640 ticks"},
          rows=rows, clocks=clk.summary(), dtype={0: "f32", 4: "f32+bf16x3"}[cm],
          convolution={0: "FFT form", 4: "direct spatial form (tensor-core GEMM per frequency bin)"}[cm])


def run_sizes(args):
    """Runtime against input size (the paper's runtime-per-batch study, Sec. IV-B): one
    module-plane event of 10^3 .. 10^6 deposits at a time through the standard step, the
    step recorded in a CUDA graph and replayed (latency floor for small events, then the
    linear regime once the GPU is full)."""
    import torch
    import synth
    from paper_2602_12052_b300 import tred
    torch.cuda.set_device(0)
    base = synth.get_config("module200")
    resp = synth.make_response(base)
    dev = torch.device("cuda")
    rows = []
    cm = args.conv_mode if args.conv_mode in (0, 4) else 0
    clk = ClockSampler(0).__enter__()
    for n_target in (1000, 3000, 10000, 30000, 100000, 300000, 1000000):
        cfg = base.with_(n_tracks=0, min_deposits=n_target)
        dep = synth.make_deposits(cfg, seed=base.seed + n_target)
        dep = {k: v[:n_target] for k, v in dep.items()}
        n = len(dep["x"])
        max_blocks, max_pixels = probe_capacities(cfg, dep, dev)
        sim = tred.Simulator(cfg, torch.from_numpy(resp), max_deposits=n, max_blocks=max_blocks,
                             max_pixels=max_pixels, effq_skip_empty=1, device=dev, conv_mode=cm,
                             fuse_gather=tred.fused_gather_shape_ok(cfg, cm))
        x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
        sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"])
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"])
        torch.cuda.current_stream().wait_stream(side)
        ms = _timed(graph.replay, args.steps, args.warmup)
        st = sim.status()
        if st[0] != 0:
            raise RuntimeError(f"device status {st} at {n} deposits")
        nb = int(sim.counts[0].item())
        rows.append({"deposits": n, "active_blocks": nb, "ms": ms, "depos_per_s": n / (ms / 1e3),
                     "us_per_block": 1e3 * ms / max(nb, 1)})
        del sim, graph
        torch.cuda.empty_cache()
    clk.__exit__(None, None, None)
    big = rows[-1]
    _line("step time vs event size, module plane, CUDA graph replay (runtime vs input size)", big["depos_per_s"],
          "depos/s", big["ms"], args,
          {"workload": "one module-plane event (512x512 px x 6400 ticks) of 1e3 .. 1e6 deposits, 8x8x256 blocks"},
          rows=rows, clocks=clk.summary(), dtype={0: "f32", 4: "f32+bf16x3"}[cm],
          convolution={0: "FFT form", 4: "direct spatial form (tensor-core GEMM per frequency bin), the inverse time DFT fused with the gather"}[cm])


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode != "step":
        {"batched": run_batched, "adjoint": run_adjoint, "spill": run_spill, "accuracy": run_accuracy,
         "chunking": run_chunking, "lines": run_lines, "binsize": run_binsize,
         "sizes": run_sizes}[args.mode](args)
        return
    import numpy as np
    import torch

    import synth
    from paper_2602_12052_b300 import build as lib_build
    from paper_2602_12052_b300 import tred

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib_build.build()
    cfg = synth.get_config(args.config)
    if args.readout_mode:
        cfg = cfg.with_(readout_mode=args.readout_mode, n_samples=args.n_samples if args.readout_mode == 1 else 1)
    dep = synth.make_deposits(cfg, seed=replica_seed(cfg, rank))
    resp = synth.make_response(cfg)
    n = len(dep["x"])
    dev = torch.device("cuda", local)
    max_blocks, max_pixels = probe_capacities(cfg, dep, dev)
    max_hits = 4 * max_pixels
    fused = bool(args.fused) and args.conv_mode == 0

    def make(fuse_gather):
        return tred.Simulator(cfg, torch.from_numpy(resp), max_deposits=n, max_blocks=max_blocks,
                              max_pixels=max_pixels, max_hits=max_hits, conv_mode=args.conv_mode,
                              effq_skip_empty=1 if args.conv_mode in (0, 4) else 0, device=dev, fused=fused,
                              fuse_gather=fuse_gather)
    # conv_mode 4: the inverse time DFT fused with the gather when the shape allows it
    fg = bool(args.fuse_gather) and args.conv_mode == 4
    try:
        sim = make(fg)
    except ValueError:
        fg = False
        sim = make(False)
    # response spectrum, timed separately (once per response)
    torch.cuda.synchronize()
    t = time.perf_counter()
    tred.tred_set_response(sim.h, sim.resp)
    torch.cuda.synchronize()
    set_response_ms = 1e3 * (time.perf_counter() - t)

    x = {k: torch.from_numpy(v).to(dev) for k, v in dep.items()}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)

    stage_names = ["drift", "blockbin", "effq", "convolve", "gather+readout"]
    if fused:
        stage_names = ["drift", "blockbin", "effq_weights", "effq+convolve", "gather+readout"]
    if fg:
        stage_names = ["drift", "blockbin", "effq", "convolve+gather+readout"]
    n_ev = len(stage_names) + 1

    def step(events=None):
        h = sim.h
        ev = events or [None] * n_ev

        def rec(i):
            if ev[i] is not None:
                ev[i].record(stream)
        rec(0)
        tred.tred_drift(h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], sim.deps)
        rec(1)
        tred.tred_blockbin(h, n, sim.deps, sim.block_ids, sim.block_counts, sim.dep_offsets,
                           sim.dep_index, sim.n_blocks_dev)
        rec(2)
        if fused:   # one persistent launch (its per-deposit weights kernel first, inside the call)
            rec(3)
            tred.tred_effq_convolve(h, n, sim.deps, sim.block_ids, sim.dep_offsets, sim.dep_index,
                                    sim.n_blocks_dev, sim.qeff, sim.out_blocks)
        else:
            tred.tred_effq(h, n, sim.deps, sim.block_ids, sim.dep_offsets, sim.dep_index,
                           sim.n_blocks_dev, sim.qeff)
            rec(3)
            if fg:   # a4 + a5 + a6: spectra, pixel list, inverse DFT per pixel tile into the waves, readout
                tred.tred_convolve_gather_readout(h, sim.block_ids, sim.n_blocks_dev, sim.qeff, sim.pixel_ids,
                                                  sim.waveforms, sim.n_pixels_dev, sim.rp, sim.hit_pixel,
                                                  sim.hit_tick, sim.hit_charge, sim.n_hits_dev)
                rec(4)
                return
            tred.tred_convolve(h, sim.block_ids, sim.n_blocks_dev, sim.qeff, sim.out_blocks)
        rec(4)
        # a5 + a6: the electrode gather and the readout in one call (the readout skips the
        # pixels whose positive current cannot reach the threshold)
        tred.tred_gather_readout(h, sim.block_ids, sim.n_blocks_dev, sim.out_blocks, sim.pixel_ids,
                                 sim.waveforms, sim.n_pixels_dev, sim.rp, sim.hit_pixel, sim.hit_tick,
                                 sim.hit_charge, sim.n_hits_dev)
        rec(5)

    tred.tred_reset_status(sim.h)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = tred.tred_sync_status(sim.h)
    if status[0] != 0:
        raise RuntimeError(f"device status after warm-up: {status}")
    nb, npix, nh = (int(v) for v in sim.counts[:3].cpu())

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    launches0 = tred.tred_launch_count(sim.h)
    # per-kernel CUDA events on the launching stream (library-side) over the timed steps
    tred.tred_set_kernel_timing(sim.h, True)
    tred.tred_direct_counts(sim.h)   # resets the row and column sums
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.zero_()                       # L2 flushed between timed steps (outside events)
            step(evs[k])
        torch.cuda.synchronize()
    launches = tred.tred_launch_count(sim.h) - launches0
    kernel_ms = {}
    for cls, name in tred.KT_NAMES.items():
        kt, kn = tred.tred_kernel_time(sim.h, cls)
        if kn:
            kernel_ms[name] = kt / args.steps
    tred.tred_set_kernel_timing(sim.h, False)
    rows_dx, cols_dx = (v // args.steps for v in tred.tred_direct_counts(sim.h))
    clocks = clk.summary()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [evs[k][0].elapsed_time(evs[k][n_ev - 1]) for k in range(args.steps)]
    stage_ms = {nm: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
                for i, nm in enumerate(stage_names)}
    ms = statistics.mean(step_ms)

    # the same step recorded once in a CUDA graph and replayed: no host launch overhead
    graph = None
    if args.graph:
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            step()
        stream.wait_stream(side)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        g_ms = []
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            g_ms.append(a.elapsed_time(b))
        status = tred.tred_sync_status(sim.h)
        if status[0] != 0:
            raise RuntimeError(f"device status after the graph replays: {status}")
        eager_ms, ms = ms, statistics.mean(g_ms)

    n_job, ms = aggregate_replicas(n, ms, world, dev)
    value = n_job / (ms / 1e3)

    # end to end through the public API: pinned host inputs -> device, step,
    # counts + hit list -> pinned host, every step inside the timed region
    e2e = None
    if not args.no_e2e and graph is None:
        # the public streaming API: each event's deposits copied from pinned host memory,
        # its counts and hit list read back, both on side streams overlapped with the
        # neighbouring events' computation (tred.StreamRunner); every copy of every step
        # lies inside the timed region
        host = {k: torch.from_numpy(v).pin_memory() for k, v in dep.items()}
        runner = tred.StreamRunner(sim, n, timing=True)
        for _ in range(args.warmup):
            runner.submit(host, n)
        runner.drain()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_e2e:
            time.sleep(0.3)
            a.record(stream)
            runner.s_in.wait_event(a)
            got = []
            for k in range(args.steps):
                r = runner.submit(host, n, tag=k)
                if r is not None:
                    got.append(r)
            b.record(runner.s_out)
            b.synchronize()
        got += runner.drain()
        if any(r[1]["n_hits"] != nh or r[1]["n_pixels"] != npix for r in got):
            raise RuntimeError("streamed events disagree with the device-timed steps")
        em = a.elapsed_time(b) / args.steps
        step_in_stream = statistics.mean(r[1]["step_ms"] for r in got)
        n_e2e, em = aggregate_replicas(n, em, world, dev)
        e2e = {"value": n_e2e / (em / 1e3), "unit": "depos/s", "h2d_bytes_per_step": runner.h2d_bytes,
               "d2h_bytes_per_step": runner.d2h_bytes, "ms_per_step": em,
               "step_ms_in_stream": step_in_stream, "clocks": clk_e2e.summary(),
               "h2d_what": "the event's deposits (x, y, z, t0, n_e float32) from pinned host memory",
               "d2h_what": ("the device counts and the capacity-sized hit lists (pixel, tick, charge); "
                            "the pixel waveforms stay in device memory"),
               "pipeline": ("tred.StreamRunner: copies on two side streams overlapped with the neighbouring "
                            "events' steps (double-buffered inputs and hit staging); no L2 flush between "
                            "events, whose working set is far larger than L2")}
    elif not args.no_e2e:
        # graph replay: each step's copies and the replayed step one after another
        host = {k: torch.from_numpy(v).pin_memory() for k, v in dep.items()}
        h_counts = torch.empty(4, dtype=torch.int32).pin_memory()
        h_hp = torch.empty(max_hits, dtype=torch.int32).pin_memory()
        h_ht = torch.empty(max_hits, dtype=torch.int32).pin_memory()
        h_hc = torch.empty(max_hits, dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = h_counts.numel() * 4 + 12 * max_hits
        e_ms = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for kk in x:
                x[kk].copy_(host[kk], non_blocking=True)
            graph.replay()
            h_counts.copy_(sim.counts, non_blocking=True)
            h_hp.copy_(sim.hit_pixel, non_blocking=True)
            h_ht.copy_(sim.hit_tick, non_blocking=True)
            h_hc.copy_(sim.hit_charge, non_blocking=True)
            b.record(stream)
            b.synchronize()
            if k >= args.warmup:
                e_ms.append(a.elapsed_time(b))
        em = statistics.mean(e_ms)
        n_e2e, em = aggregate_replicas(n, em, world, dev)
        e2e = {"value": n_e2e / (em / 1e3), "unit": "depos/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": em,
               "h2d_what": "the event's deposits (x, y, z, t0, n_e float32)",
               "d2h_what": ("the device counts and the capacity-sized hit lists (pixel, tick, charge); "
                            "the pixel waveforms stay in device memory")}

    # the FP32 FMA peak after the timed legs (its burst would warm the part before them)
    peak_meas, sms = measured_fp32_peak()
    conv_ms = stage_ms["effq+convolve" if fused else "convolve+gather+readout" if fg else "convolve"]
    if args.conv_mode == 4:
        kr = direct_rooflines(cfg, rows_dx, cols_dx, nb, kernel_ms, clocks, npix)
        dom = next(iter(kr))
        roofline = dict(kr[dom])
        roofline["kernels"] = kr
        roofline["kernel_ms_per_step"] = kernel_ms
        roofline["rows"], roofline["nonempty_columns"] = rows_dx, cols_dx
        roofline["conv_alu_frac_unpruned"] = (conv_flop_per_block(cfg.lt) * nb / (conv_ms / 1e3) / 1e12
                                              / FP32_PEAK_TFLOPS)
    flop_blk = conv_flop_per_block(cfg.lt)
    if args.conv_mode != 4:
        roofline = alu_roofline("tred_effq_convolve (k_block_pipeline: effective charge + convolution, one "
                                "persistent launch)" if fused else "tred_convolve (k_conv_spec + k_conv_itime_mp)",
                                flop_blk, nb, conv_ms, clocks, peak_meas)
        roofline["traffic"], roofline["traffic_source"] = conv_traffic(nb) if not fused else (None, "no capture")
    roofline["sms"] = sms
    cc = conv_counters() if not fused and args.conv_mode == 0 else {}
    if "conv_executed_flop_per_block" in cc:
        ex = cc["conv_executed_flop_per_block"]
        roofline["executed_flop_per_block"] = ex
        roofline["frac_executed_vs_measured"] = ex * nb / (conv_ms / 1e3) / 1e12 / peak_meas
        roofline["executed_source"] = ("ncu 2*FFMA + FADD + FMUL thread instructions of the convolution's "
                                       "kernels on module20, per block")
    if "conv_spec_fma_pipe_pct" in cc:
        roofline["ncu_fma_pipe_pct"] = cc["conv_spec_fma_pipe_pct"]
        roofline["ncu_issue_active_pct"] = cc.get("conv_spec_issue_active_pct")
    if args.conv_mode in (1, 2, 3):
        # the time DFT on the tensor cores: per block 50 pairs x 128 x 512 x bt MACs, one
        # product (TF32) or three (split TF32); its tensor-pipe share is in profiles/
        products = 1 if args.conv_mode == 1 else 3   # TF32; split TF32 or split BF16
        roofline["dft_gemm_flop_per_block"] = 2 * 50 * 128 * 512 * cfg.bt * products
        roofline["traffic"], roofline["traffic_source"] = None, "no capture of this form"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "depos/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f32", 1: "tf32", 2: "tf32x3", 3: "bf16x3", 4: "f32+bf16x3"}[args.conv_mode],
            "data": "synthetic",
            "config": {"workload": (f"{cfg.name}: one event of {n} point deposits on a "
                                    f"{cfg.npx}x{cfg.npx} pixel plane x {cfg.nt} ticks, GL-{cfg.gl_order}, "
                                    f"{cfg.kp}x{cfg.kp}x{cfg.n_sub}x{cfg.n_sub}x{cfg.nr} response, "
                                    f"{cfg.bp}x{cfg.bp}x{cfg.bt} blocks"
                                    + (f", time DFT length {cfg.lt}" if args.conv_mode == 4 else
                                       f", FFT 16x16x{cfg.lt}, MPCP")
                                    + {0: ", effective charge written for covered columns only",
                                       1: ", time DFT as a TF32 tcgen05 GEMM (tolerance 1e-4)",
                                       2: ", time DFT as a split-TF32 tcgen05 GEMM",
                                       3: ", time DFT as a split-BF16 tcgen05 GEMM (tolerance 1e-4)",
                                       4: (", effective charge written for covered columns only; time DFT by FFT, "
                                           "impacts x taps per bin as a split-BF16 tcgen05 GEMM over the block "
                                           "pixels that hold charge")}[args.conv_mode]
                                    + {0: "", 1: f", readout: {cfg.n_samples} successive digitisations per trigger",
                                       2: ", readout: fixed-charge quanta"}[args.readout_mode]
                                    + (", inverse time DFT per 8x8 pixel tile straight into the pixel "
                                       "waveforms (no per-block output buffer)" if fg else "")
                                    + (", effective charge and convolution in one persistent launch over the "
                                       "active-block queue (Q^eff in per-CTA ring rows)" if fused else "")),
                       "deposits": n, "active_blocks": nb, "active_pixels": npix, "hits": nh,
                       **({"deposits_all_ranks": int(n_job)} if world > 1 else {}),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       **({"launch": f"CUDA graph replay (eager step {eager_ms:.3f} ms)"} if graph is not None else {}),
                       "l2": "flushed between timed steps (256 MB write, outside the step events)"},
            "stages_ms": stage_ms, "set_response_ms": set_response_ms,
            "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg, dep, resp, args.cpu_sample)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
