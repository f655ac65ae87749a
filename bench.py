#!/usr/bin/env python3
"""Throughput of the FFT-beamforming hot path on the CHIME-like 4x256 workload.

One step = the whole hot path over one integration block of the workload:
  49152 samples x 1024 channels x 2 pols of a 4x256 int4+4 lattice (1.03e11 antenna
  samples), as 16 fftbf_execute calls of 3072 samples (8 windows of 384) over a
  device-resident block, then fftbf_tied_beams for 2048 pointings over the 128 windows.
The 3072-sample device block (6.4 GB, far above the 129 MB L2) is 4 copies of a seeded
768-sample host block; every call re-reads it from HBM.

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WL = dict(nx=4, ny=256, pad_x=4, pad_y=512, npol=2, nfreq=1024, T=49152, n_int=384,
          n_tied=2048, seed=2, n_src=3, amp=1.5, sigma=2.5)
T_HOST = 768          # seeded host block (2 windows)
T_DEV = 3072          # device block per fftbf_execute call (8 windows)
METRIC = "antenna-samples/s at 4x256 int4 lattice"
UNIT = "antenna-samples/s"
# Algorithmic FP32 work of the plain form per snapshot (one pol, one t, one f), counted
# with 5 N log2 N per complex FFT: N-S 512-point transform of 256 inputs as two 256-point
# FFTs plus 256 twiddle products (6 flops) per E-W beam, E-W 4-point DFT at 5 N log2 N per
# column, apodisation 2 flops per sample (real weights), detection + accumulation 4 flops
# per beam: 108,544 flops (106 per antenna-sample).
FLOPS_PER_SNAPSHOT = 4 * (2 * 5 * 256 * 8 + 6 * 256) + 5 * 4 * 2 * 256 + 2 * 1024 + 4 * 2048
# Tensor-core form as specified: E-W 4x4 DFT on 256 columns (4096 complex MACs) plus the
# N-S 512 = 32 x 16 stages (4 x 16384 complex MACs), 8 real flops per complex MAC as
# real-embedded GEMMs: 544 flops per antenna-sample. As executed (E-W on the CUDA cores):
# 512 flops per antenna-sample of GEMM.
TC_FLOPS_SPEC, TC_FLOPS_EXEC = 544.0, 512.0
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def flops_per_snapshot(nx, ny, mx, my):
    """The same count for any lattice with 2x zero-padded N-S axis and real weights:
    apodisation 2/sample, E-W DFT per column (5 M log2 M for M = nx a power of two, 8 nx M
    for a DFT matrix), N-S transform of my/2 inputs as two my/2-point FFTs plus my/2 twiddle
    products per E-W beam, detection + accumulation 4 flops per beam."""
    import math
    if mx == 1:
        ew = 0
    elif mx == nx and mx & (mx - 1) == 0:
        ew = 5 * mx * int(math.log2(mx))
    else:
        ew = 8 * nx * mx
    h = my // 2
    ns = 2 * 5 * h * int(math.log2(h)) + 6 * h if h > 1 else 6
    return 2 * nx * ny + ew * ny + mx * ns + 4 * mx * my


# DRAM bytes (read + write) of one beam-kernel launch, from an ncu capture of the
# 256-channel profile case scaled by snapshots to the 3072 x 1024 launch; set to None
# whenever the kernel changes until it is captured again.
TRAFFIC_FP32 = 16 * (402.845440e6 + 3.619840e6)
# The same for the FP16 tensor-core form's beam kernel (`--profile-case --form tc_fp16`).
TRAFFIC_TCW = 16 * (402.823680e6 + 6.055680e6)
# The beam kernel each tensor-core form launches on the 4x256 lattice
TC_KERNEL = {"tc_fp16": "beams_tcg_kernel<true, false>", "tc_bf16": "beams_tcg_kernel<true, true>",
             "tc_fp16x3": "beams_tc_kernel<0, 1, 1>"}
# The same for one batched step (one batch_kernel launch over 8192 samples), from the
# 512-sample profile case (`--workload batched --profile-case`) scaled x16.
TRAFFIC_BATCH = 16 * (2184.573696e6 + 36.063232e6)


def samples_per_step():
    return WL["T"] * WL["nfreq"] * WL["npol"] * WL["nx"] * WL["ny"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ clocks ----------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.fh = None

    def start(self):
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.flush()
        self.fh.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.fh.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.fh.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- CPU oracle ---------
def host_block(rank=0):
    """The seeded 768-sample block of `rank`'s channel band (rank 0: the band every
    parity test uses)."""
    from paper_1710_08591_gb300 import multirank
    seed = multirank.band_seed(WL["seed"], rank)
    src = synth.seeded_sources(WL["seed"] + 100, WL["n_src"], WL["amp"])
    return synth.volts(T_HOST, WL["nfreq"], WL["npol"], WL["nx"], WL["ny"], seed=seed,
                       sigma=WL["sigma"], sources=src)


def oracle_sample(block, n_chan, chan0=0):
    """FP64 oracle on window 0 x n_chan channels x 2 pols; returns (samples, seconds,
    beams [n_chan][pad_x][pad_y])."""
    import oracle
    w = synth.separable_weights(synth.half_sine(WL["nx"]), synth.half_sine(WL["ny"]))
    v = np.ascontiguousarray(block[:WL["n_int"], chan0:chan0 + n_chan])
    t0 = time.perf_counter()
    P = oracle.beams(v, WL["nx"], WL["ny"], WL["pad_x"], WL["pad_y"], WL["npol"], n_chan,
                     WL["n_int"], weights=w.astype(np.complex128))
    dt = time.perf_counter() - t0
    return v.size, dt, P[0]


def cpu_cores():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max((i.get("num_threads", 1) for i in info), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(block, budget_s=12.0):
    """The oracle timed on window 0 of the workload, channel by channel from 0, for about
    budget_s seconds. Returns the baseline line and the oracle's beams of the channels it
    covered (window 0), against which every GPU form's beams are then compared."""
    n_chan, tot_s, tot_n, used = 2, 0.0, 0, 0
    chan = 0
    ref = []
    while tot_s < budget_s and chan + n_chan <= WL["nfreq"]:
        n, dt, P = oracle_sample(block, n_chan, chan)
        ref.append(P)
        tot_s += dt
        tot_n += n
        chan += n_chan
        used += n_chan
        n_chan = min(n_chan * 2, 32)
    line = {"value": tot_n / tot_s, "unit": UNIT, "cores": cpu_cores(), "cpu_model": cpu_model(),
            "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"1 window of 384 samples x {used} channels x 2 pols of the 4x256 "
                      f"workload ({tot_n:.3g} antenna-samples, {tot_s:.1f} s), FP64 numpy "
                      "separable direct DFT"}
    return line, np.concatenate(ref, axis=0)


def form_errors(got, ref):
    """Per-beam relative error |P - P_ref| / P_ref of a form's window-0 beams against the
    oracle's, over the channels the oracle covered: max and rms."""
    n = min(got.shape[0], ref.shape[0])
    rel = np.abs(got[:n].astype(np.float64) - ref[:n]) / ref[:n]
    return {"max_rel_err_vs_oracle": float(rel.max()),
            "rms_rel_err_vs_oracle": float(np.sqrt(np.mean(rel ** 2))),
            "checked": f"window 0, channels 0-{n - 1}, {rel.size} beams"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    block = host_block()
    n_chan = 4
    for _ in range(args.warmup):
        oracle_sample(block, n_chan)
    times, ns = [], 0
    for k in range(args.steps):
        n, dt, _ = oracle_sample(block, n_chan, (k * n_chan) % WL["nfreq"])
        times.append(dt)
        ns += n
    val = ns / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4x256 lattice, 2 pols, 1024 channels, 49152 samples, "
                                   "N-S padded to 512, n_int 384, half-sine weights",
                       "step_sample": f"1 window x {n_chan} channels x 2 pols per step"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"1 window x {n_chan} channels x 2 pols per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm ---------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1710_08591_gb300 as fb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    fb.build()
    fb.lib()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    t_gen = time.perf_counter()
    block = host_block(rank)
    t_gen = time.perf_counter() - t_gen
    nx, ny, mx, my = WL["nx"], WL["ny"], WL["pad_x"], WL["pad_y"]
    npol, nfreq, n_int, n_tied = WL["npol"], WL["nfreq"], WL["n_int"], WL["n_tied"]
    w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
    u, v = synth.tied_pointings(WL["seed"] + 1, nfreq, n_tied, nx, ny, mx, my)

    hb = torch.from_numpy(block.reshape(-1))
    dvol = torch.empty(T_DEV * hb.numel() // T_HOST, dtype=torch.uint8, device=dev)
    for c in range(T_DEV // T_HOST):
        dvol[c * hb.numel():(c + 1) * hb.numel()].copy_(hb)
    nwin = WL["T"] // n_int
    wpc = T_DEV // n_int                               # windows per execute call
    ncall = WL["T"] // T_DEV
    beams = torch.empty((nwin, nfreq, mx, my), device=dev)
    tied = torch.empty((nwin, nfreq, n_tied), device=dev)
    plan = fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w)
    if args.form != "fp32":
        fb.plan_set_precision(plan, {"tc_fp16": fb.PREC_TC_FP16, "tc_bf16": fb.PREC_TC_BF16,
                                     "tc_fp16x3": fb.PREC_TC_FP16X3}[args.form])
    stream = torch.cuda.current_stream(dev)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(ncall)] for _ in range(args.steps)]

    def step(k=None):
        for c in range(ncall):
            if k is not None:
                ev[k][c][0].record(stream)
            fb.execute(plan, dvol, T_DEV, beams[c * wpc:(c + 1) * wpc], stream)
            if k is not None:
                ev[k][c][1].record(stream)
        fb.tied_beams(plan, beams, nwin, n_tied, u, v, tied, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for k in range(args.steps):
        step(k)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    kern_ms = [a.elapsed_time(b) for row in ev for a, b in row]
    clk = clocks.stop()
    from paper_1710_08591_gb300 import multirank
    total_ms, job_samples = multirank.aggregate(t0.elapsed_time(t1), samples_per_step() * args.steps,
                                                device=dev)
    ms_step = total_ms / args.steps
    value = multirank.throughput(total_ms, job_samples)

    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        hvol = torch.empty(T_DEV * hb.numel() // T_HOST, dtype=torch.uint8, pin_memory=True)
        for c in range(T_DEV // T_HOST):
            hvol[c * hb.numel():(c + 1) * hb.numel()].copy_(hb)
        hbeams = torch.empty((nwin, nfreq, mx, my), pin_memory=True)
        htied = torch.empty((nwin, nfreq, n_tied), pin_memory=True)
        hv, hbn, htn = hvol.numpy(), hbeams.numpy(), htied.numpy()

        def e2e_step():
            for c in range(ncall):
                fb.execute_host(plan, hv, T_DEV, hbn[c * wpc:(c + 1) * wpc], n_tied, u, v,
                                htn[c * wpc:(c + 1) * wpc], stream)
            torch.cuda.synchronize(dev)

        for _ in range(2):
            e2e_step()
        if dist:
            dist.barrier()
        # each step timed on the host clock around its calls and the final synchronize;
        # the median step is reported (the host link is shared with the other GPUs of the
        # node, so single steps can be slow), every step is listed
        e_steps = max(3, min(args.steps, 7))
        step_s = []
        for _ in range(e_steps):
            t0e = time.perf_counter()
            e2e_step()
            step_s.append(time.perf_counter() - t0e)
        te = float(np.median(step_s))
        if dist:
            tt = torch.tensor([te], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": samples_per_step() * world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(ncall * hv.nbytes),
               "d2h_bytes_per_step": int(hbn.nbytes + htn.nbytes),
               "ms_per_step": 1e3 * te, "step_ms": [round(1e3 * x, 1) for x in step_s],
               "statistic": "median over steps",
               "api": "fftbf_execute_host (pinned host buffers)"}

    # ---- window-0 beams of the first channels, kept for the error check against the
    # oracle beams that the CPU-baseline leg computes
    n_chk = 64
    kept = {args.form: beams[0, :n_chk].cpu().numpy()}

    # ---- measured FP32 peak: FFMA and packed FFMA2 probes at full occupancy
    peaks, src = measured_peaks()
    fp32 = fp32_peak(fb, torch, dev, stream)
    fp32_pk = max(fp32["ffma_tflops"], fp32["ffma2_tflops"])

    # ---- roofline of the dominant kernel (the fused beam kernel)
    k_ms = sum(kern_ms) / len(kern_ms)
    samples_launch = T_DEV * nfreq * npol * nx * ny
    snaps_launch = T_DEV * nfreq * npol
    bytes_launch = samples_launch + wpc * nfreq * mx * my * 4
    flops = FLOPS_PER_SNAPSHOT * snaps_launch
    achieved = flops / (k_ms / 1e3) / 1e12
    tpk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    tpk_src = (src + " bf16 sustained (a seconds-long loop under the power cap; FP16 runs at "
               "the same rate); the beam kernel runs inside a seconds-long step")
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_pk, "unit": "TFLOP/s",
            "frac": achieved / fp32_pk, "traffic": TRAFFIC_FP32,
            "kernel": "beams_fp32_4x256_kernel<true>", "ms_per_launch": k_ms,
            "flops_per_snapshot": FLOPS_PER_SNAPSHOT,
            "peak_source": "measured: " + fp32["source"],
            "fp32_probe": fp32,
            "frac_of_nominal": achieved / FP32_PEAK_NOMINAL,
            "nominal_peak": FP32_PEAK_NOMINAL,
            "hbm": {"achieved_gbs": bytes_launch / (k_ms / 1e3) / 1e9,
                    "peak_gbs": peaks["hbm_gbs"],
                    "frac": bytes_launch / (k_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                    "peak_source": src}}

    if args.form != "fp32":
        rate = samples_launch / (k_ms / 1e3)
        tfl = TC_FLOPS_SPEC * rate / 1e12
        roof = {"bound": "tensor", "achieved": tfl, "peak": tpk, "unit": "TFLOP/s",
                "frac": tfl / tpk, "traffic": TRAFFIC_TCW if args.form == "tc_fp16" else None,
                "kernel": TC_KERNEL[args.form],
                "ms_per_launch": k_ms, "flops_per_sample": TC_FLOPS_SPEC, "peak_source": tpk_src,
                "hbm": {"achieved_gbs": bytes_launch / (k_ms / 1e3) / 1e9,
                        "peak_gbs": peaks["hbm_gbs"],
                        "frac": bytes_launch / (k_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "peak_source": src}}

    # ---- the other forms on the same workload (same step, fewer timed steps); each beam
    # launch is bracketed by CUDA events on the launching stream, as the main form's
    forms = {args.form: {"value": value, "ms_per_step": ms_step, "beam_ms_per_launch": k_ms,
                         "beam_antenna_samples_per_s": samples_launch / (k_ms / 1e3)}}
    if not args.no_forms:
        for form, prec in (("tc_fp16", fb.PREC_TC_FP16), ("tc_bf16", fb.PREC_TC_BF16),
                           ("tc_fp16x3", fb.PREC_TC_FP16X3)):
            if form == args.form:
                continue
            fplan = fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w)
            fb.plan_set_precision(fplan, prec)
            fsteps = max(2, min(args.steps, 5))
            fev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    for _ in range(ncall)] for _ in range(fsteps)]

            def fstep(k=None):
                for c in range(ncall):
                    if k is not None:
                        fev[k][c][0].record(stream)
                    fb.execute(fplan, dvol, T_DEV, beams[c * wpc:(c + 1) * wpc], stream)
                    if k is not None:
                        fev[k][c][1].record(stream)
                fb.tied_beams(fplan, beams, nwin, n_tied, u, v, tied, stream)

            for _ in range(max(3, args.warmup)):
                fstep()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            f0.record(stream)
            for k in range(fsteps):
                fstep(k)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            fms = f0.elapsed_time(f1) / fsteps
            b_ms = float(np.mean([a_.elapsed_time(b_) for row in fev for a_, b_ in row]))
            rate = samples_launch / (b_ms / 1e3)
            spec = TC_FLOPS_SPEC * rate / 1e12
            exe = TC_FLOPS_EXEC * rate / 1e12
            gb = bytes_launch / (b_ms / 1e3) / 1e9
            forms[form] = {
                "value": samples_per_step() * world / (fms / 1e3), "ms_per_step": fms,
                "beam_ms_per_launch": b_ms, "beam_antenna_samples_per_s": rate,
                "roofline": {
                    "kernel": TC_KERNEL[form], "bound": "tensor", "ms_per_launch": b_ms,
                    "traffic": TRAFFIC_TCW if form == "tc_fp16" else None,
                    "timing": "CUDA events around each beam launch on its stream",
                    "tensor_as_specified": {"flops_per_sample": TC_FLOPS_SPEC, "achieved": spec,
                                            "peak": tpk, "unit": "TFLOP/s", "frac": spec / tpk,
                                            "peak_source": tpk_src},
                    "tensor_as_executed": {"flops_per_sample": TC_FLOPS_EXEC, "achieved": exe,
                                           "peak": tpk, "unit": "TFLOP/s", "frac": exe / tpk,
                                           "note": "E-W DFT on the CUDA cores; useful flops"
                                                   + ("; the split form issues 3 products per "
                                                      "MAC (1536 tensor flops per sample)"
                                                      if form == "tc_fp16x3" else "")},
                    "hbm": {"achieved": gb, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": gb / peaks["hbm_gbs"], "peak_source": src}}}
            kept[form] = beams[0, :n_chk].cpu().numpy()
            fplan.close()
        # the step's FP32 beams back in the buffer for the tied-beam variants below
        for c in range(ncall):
            fb.execute(plan, dvol, T_DEV, beams[c * wpc:(c + 1) * wpc], stream)
        torch.cuda.synchronize(dev)

    # ---- tied-beam variants on the step's 128 windows: plain (Dirichlet, GEMM over the 512
    # N-S beams), optimal half-sine window (GEMM), the same window truncated to 5 taps
    tied_forms = None
    if not args.no_forms:
        tied_forms = {}
        ref_dense = None
        for name, hy, trunc in (("plain_gemm", None, 0), ("window_gemm", synth.half_sine(ny), 0),
                                ("window_5tap", synth.half_sine(ny), 5),
                                ("window_9tap", synth.half_sine(ny), 9)):
            fb.tied_set_window(plan, None, hy, 0, trunc)
            fb.tied_beams(plan, beams, nwin, n_tied, u, v, tied, stream)     # builds the tables
            torch.cuda.synchronize(dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(3):
                fb.tied_beams(plan, beams, nwin, n_tied, u, v, tied, stream)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            tms = a0.elapsed_time(a1) / 3
            # algorithmic flops: 2 per (tied beam, FFT beam used); E-W one FFT-beam column
            # (pad_x < 2 nx - 1), N-S all pad_y beams or the truncated taps
            k_ns = trunc if trunc else my
            tfl = 2.0 * nwin * nfreq * n_tied * k_ns / (tms / 1e3) / 1e12
            if trunc:                      # the gather kernel, on the CUDA cores
                tied_forms[name] = {"ms": tms, "tflops": tfl, "path": "CUDA cores",
                                    "frac_fp32_peak": tfl / fp32_pk}
            else:                          # split-FP16 GEMM: 3 tensor-core products per MAC
                pk, _ = measured_peaks()
                tied_forms[name] = {"ms": tms, "tflops": tfl,
                                    "path": "tensor cores, split FP16 (3 products per MAC)",
                                    "frac_tensor_peak_issued": 3.0 * tfl / pk["bf16_tflops"],
                                    "frac_tensor_peak_useful": tfl / pk["bf16_tflops"],
                                    "peak_source": "measured bf16 burst (a few-ms kernel timed alone)"}
            if name == "window_gemm":
                ref_dense = tied.clone()
            if name.endswith("tap"):
                # truncation error, normalised by the mean |tied beam| of each (window, channel)
                scale = ref_dense.abs().mean(dim=-1, keepdim=True).clamp_min(1e-30)
                rel = (tied - ref_dense).abs() / scale
                tied_forms[name]["max_err_vs_all_beams"] = float(rel.max())
                tied_forms[name]["rms_err_vs_all_beams"] = float(rel.pow(2).mean().sqrt())
        fb.tied_set_window(plan)
        # redundancy-stacked visibilities from the same FFT beams (N-S lags, E-W beams kept)
        sdx, sdy = fb.stacked_shape(plan)
        vis = torch.empty((nwin, nfreq, sdx, sdy), dtype=torch.complex64, device=dev)
        fb.stacked_visibilities(plan, beams, nwin, vis, stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a0.record(stream)
        for _ in range(3):
            fb.stacked_visibilities(plan, beams, nwin, vis, stream)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        vms = a0.elapsed_time(a1) / 3
        vbytes = nwin * nfreq * (mx * my * 4 + sdx * sdy * 8)          # beams in, visibilities out
        tied_forms["stacked_visibilities"] = {
            "ms": vms, "shape": [sdx, sdy], "gbs": vbytes / (vms / 1e3) / 1e9,
            "frac_hbm": vbytes / (vms / 1e3) / 1e9 / peaks["hbm_gbs"]}
        del vis
        # point-source localisation in every (window, channel) from the same FFT beams
        loc = torch.empty((nwin, nfreq, 3), dtype=torch.float32, device=dev)
        fb.localise(plan, beams, nwin, loc, 5, 10, stream)
        torch.cuda.synchronize(dev)
        a0.record(stream)
        for _ in range(3):
            fb.localise(plan, beams, nwin, loc, 5, 10, stream)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        lms = a0.elapsed_time(a1) / 3
        lbytes = nwin * nfreq * (mx * my * 4 + 12)
        tied_forms["localise"] = {"ms": lms, "n_iter": 5, "n_taps": 10,
                                  "gbs": lbytes / (lms / 1e3) / 1e9,
                                  "frac_hbm": lbytes / (lms / 1e3) / 1e9 / peaks["hbm_gbs"]}
        del loc

    # ---- the batched uneven-lattice configuration (12 arrays, one persistent launch)
    batched = None
    if not args.no_forms and world == 1:
        batched = batched_form(fb, torch, dev, steps=max(3, min(args.steps, 10)),
                               warmup=max(3, args.warmup), fp32_pk=fp32_pk)

    serving = None
    if not args.no_serving:
        serving = run_serving(fb, torch, dev, frames_total=args.serve_frames, rate=SERVE["rate"])
        sweep = []
        for rate in SERVE["sweep"]:
            r = run_serving(fb, torch, dev, frames_total=args.serve_frames, rate=rate)
            sweep.append({k: r[k] for k in ("offered_rate_fps", "achieved_fps", "frames",
                                            "antenna_samples_per_s", "p50_ms", "p99_ms",
                                            "max_ms", "frames_per_launch",
                                            "max_frames_per_launch", "peak_inflight")})
        serving["sweep"] = sweep

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu, ref = cpu_baseline(block)
        for form, got in kept.items():
            forms[form].update(form_errors(got, ref))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.form == "fp32" else args.form.split("_")[1],
            "data": "synthetic",
            "config": {"workload": "4x256 lattice (E-W x N-S), 2 pols, 1024 channels, 49152 "
                                   "samples per step, int4+4 voltages (sigma 2.5 noise + 3 "
                                   "plane-wave sources), E-W 4-point DFT, N-S padded to 512, "
                                   "half-sine weights, n_int 384, 2048 tied beams",
                       "form": args.form,
                       "l2": "inputs larger than L2 (6.4 GB block re-read from HBM per call)",
                       "calls_per_step": f"{ncall} x fftbf_execute(T={T_DEV}) + fftbf_tied_beams",
                       "host_block_gen_s": round(t_gen, 2),
                       "parallelism": f"{world} GPU(s), independent channel bands per GPU"},
            "gpu_launches": (ncall + 1) * args.steps,
            "roofline": roof, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
            "forms": forms, "batched": batched, "tied_beams": tied_forms, "serving": serving}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


SERVE = dict(lattices=[(4, 256), (8, 64), (16, 16)], nfreq=16, n_int=384, npol=2, streams=64,
             rate=2000.0, sweep=[8000.0, 16000.0, 32000.0], budget=40 << 30, seed=5)


def fp32_peak(fb, torch, dev, stream):
    """Measured FP32 peak: the FFMA and packed FFMA2 probes at full occupancy (8 CTAs of 256
    threads per SM), each about 12 ms, best of 3 launches, CUDA events on the stream; the SM
    clock sampled meanwhile."""
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = nsm * 8
    out = torch.empty(blocks * 256, device=dev)
    res = {}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    for packed in (False, True):
        fb.probe_fp32(packed, 2000, blocks, out, stream)
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = fb.probe_fp32(packed, 200000, blocks, out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            best = max(best, fl / (e0.elapsed_time(e1) / 1e3) / 1e12)
        res["ffma2_tflops" if packed else "ffma_tflops"] = best
    time.sleep(0.25)
    clk = clocks.stop()
    res["sm_mhz"] = clk.get("sm_mhz")
    res["source"] = ("FFMA2 (packed fma.rn.f32x2) probe" if res["ffma2_tflops"] > res["ffma_tflops"]
                     else "FFMA probe") + f", {blocks} CTAs x 256 threads x 8 chains, best of 3"
    return res


def run_serving(fb, torch, dev, frames_total=10000, rate=2000.0):
    """Poisson arrivals (mean `rate` frames/s) from 64 streams, each on a lattice drawn
    (seeded) from 4x256, 8x64, 16x16; one frame = 384 samples x 16 channels x 2 pols. Frames
    come from a pool of distinct seeded frames in pinned memory; beams land in pinned
    buffers. Returns throughput and latency percentiles of the continuous-batching server."""
    cfg = SERVE
    rng = np.random.default_rng(cfg["seed"])
    plans, pools = [], []
    for k, (lx, ly) in enumerate(cfg["lattices"]):
        wts = synth.separable_weights(synth.half_sine(lx), synth.half_sine(ly))
        plans.append(fb.plan_create(lx, ly, lx, 2 * synth.next_pow2(ly), cfg["npol"], cfg["nfreq"],
                                    cfg["n_int"], weights=wts))
        pool = []
        for j in range(4):
            buf = torch.empty(cfg["n_int"] * cfg["nfreq"] * cfg["npol"] * lx * ly,
                              dtype=torch.uint8, pin_memory=True).numpy()
            synth.volts(cfg["n_int"], cfg["nfreq"], cfg["npol"], lx, ly, seed=cfg["seed"] * 100 + 10 * k + j,
                        sources=synth.seeded_sources(cfg["seed"] + k, 2, 1.5), out=buf)
            pool.append(buf)
        pools.append(pool)
    stream_lat = rng.integers(0, len(cfg["lattices"]), cfg["streams"])
    gaps = rng.exponential(1.0 / rate, frames_total)
    streams = rng.integers(0, cfg["streams"], frames_total)
    nout = 4096
    outs = [torch.empty((cfg["nfreq"], p.pad_x, p.pad_y), dtype=torch.float32, pin_memory=True).numpy()
            for p in plans]
    ring = [torch.empty(max(o.size for o in outs), dtype=torch.float32, pin_memory=True).numpy()
            for _ in range(nout)]
    samples = 0
    with fb.server_create(plans, cfg["budget"]) as sv:
        # warm-up: one frame per lattice (excluded from the statistics below)
        for k in range(len(plans)):
            t = fb.server_submit(sv, k, pools[k][0], ring[k][:outs[k].size].reshape(outs[k].shape))
            fb.server_wait(sv, t, 30.0)
        st0 = fb.server_stats(sv)
    with fb.server_create(plans, cfg["budget"]) as sv:
        t0 = time.perf_counter()
        due = t0
        for i in range(frames_total):
            due += gaps[i]
            while time.perf_counter() < due:
                pass
            k = int(stream_lat[streams[i]])
            fb.server_submit(sv, k, pools[k][i % 4], ring[i % nout][:outs[k].size].reshape(outs[k].shape))
            lx, ly = cfg["lattices"][k]
            samples += cfg["n_int"] * cfg["nfreq"] * cfg["npol"] * lx * ly
        t_sub = time.perf_counter() - t0
        fb.server_wait(sv, -1, 120.0)
        elapsed = time.perf_counter() - t0
        st = fb.server_stats(sv)
    for p in plans:
        p.close()
    return {"frames": frames_total, "offered_rate_fps": rate, "streams": cfg["streams"],
            "submitted_fps": frames_total / t_sub,
            "achieved_fps": frames_total / elapsed, "antenna_samples_per_s": samples / elapsed,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "mean_ms": st["mean_ms"], "frames_per_launch": st["frames_per_launch"],
            "max_frames_per_launch": st["max_frames_per_launch"],
            "peak_inflight": st["peak_inflight"], "launches": st["launches"],
            "warmup_server_p50_ms": st0["p50_ms"],
            "hbm_budget_gb": cfg["budget"] / 2 ** 30, "slots": st["slots"],
            "note": "latency = completion - submission on the host clock (taken before the "
                    "server lock), frames submitted at Poisson arrival times; a fresh server "
                    "after a warm-up server"}


BATCH_T, BATCH_NINT, BATCH_TBLK = 8192, 256, 256


def batched_setup(torch, dev, T):
    """The batched workload: twelve arrays drawn (seed 4) from the six lattice shapes, 64-512
    channels each, T samples, 2 pols, n_int 256, half-sine weights; device voltages are
    copies of a seeded 256-sample block per array."""
    import paper_1710_08591_gb300 as fb
    rng = np.random.default_rng(4)
    npol = 2
    picks = rng.integers(0, len(synth.BATCH_LATTICES), 12)
    nfs = rng.integers(64, 513, 12)
    plans, dvs, outs, samples, flops = [], [], [], 0, 0.0
    for i, (li, nf) in enumerate(zip(picks, nfs)):
        lx, ly = synth.BATCH_LATTICES[li]
        lmx, lmy = lx, 2 * synth.next_pow2(ly)
        wts = synth.separable_weights(synth.half_sine(lx), synth.half_sine(ly))
        plans.append(fb.plan_create(lx, ly, lmx, lmy, npol, int(nf), BATCH_NINT, weights=wts))
        blk = synth.volts(BATCH_TBLK, int(nf), npol, lx, ly, seed=400 + i,
                          sources=synth.seeded_sources(410 + i, 2, 1.5))
        hb = torch.from_numpy(blk.reshape(-1))
        dv = torch.empty(hb.numel() * (T // BATCH_TBLK), dtype=torch.uint8, device=dev)
        for c in range(T // BATCH_TBLK):
            dv[c * hb.numel():(c + 1) * hb.numel()].copy_(hb)
        dvs.append(dv)
        outs.append(torch.empty((T // BATCH_NINT, int(nf), lmx, lmy), device=dev))
        samples += T * int(nf) * npol * lx * ly
        flops += T * int(nf) * npol * flops_per_snapshot(lx, ly, lmx, lmy)
    arrays = [[int(synth.BATCH_LATTICES[li][0]), int(synth.BATCH_LATTICES[li][1]), int(nf)]
              for li, nf in zip(picks, nfs)]
    return plans, dvs, outs, samples, flops, arrays


def batched_form(fb, torch, dev, steps, warmup, fp32_pk):
    """Time the batched configuration: one fftbf_batch_execute (one persistent launch,
    CUDA-graph replay) per step, CUDA events on its stream."""
    T = BATCH_T
    plans, dvs, outs, samples, flops, arrays = batched_setup(torch, dev, T)
    stream = torch.cuda.Stream(dev)
    with fb.batch_create(plans) as b, torch.cuda.stream(stream):
        tiles = [fb.batch_tuned_steps(b, i) for i in range(len(plans))]
        grid = fb.batch_grid(b)
        for _ in range(warmup):
            fb.batch_execute(b, dvs, T, outs, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fb.batch_execute(b, dvs, T, outs, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
    byts = sum(d.numel() for d in dvs) + sum(o.numel() * 4 for o in outs)
    items = sum(o.shape[0] * o.shape[1] for o in outs)
    peaks, src = measured_peaks()
    for p in plans:
        p.close()
    del dvs, outs
    torch.cuda.empty_cache()
    return {"metric": "antenna-samples/s, batched uneven lattices", "value": samples / (ms / 1e3),
            "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "workload": "12 arrays from {4x256, 8x64, 16x16, 2x512, 1x1024, 3x128} (seed 4), "
                        "64-512 channels, 8192 samples, 2 pols, N-S padded to 2x next pow2, "
                        "n_int 256, half-sine weights",
            "arrays": arrays, "tuned_snapshots_per_step": tiles, "items": items, "grid": grid,
            "launch": "one persistent kernel per step (CUDA graph replay)",
            "l2": "inputs larger than L2",
            "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12,
                         "peak": fp32_pk, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / fp32_pk,
                         "traffic": TRAFFIC_BATCH, "kernel": "batch_kernel",
                         "peak_source": "measured FP32 probe",
                         "hbm": {"achieved_gbs": byts / (ms / 1e3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
                                 "frac": byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                 "peak_source": src}}}


def run_batched(args):
    """The batched configuration alone (--workload batched), or its small ncu case."""
    import torch
    import paper_1710_08591_gb300 as fb
    fb.build()
    dev = torch.device("cuda", 0)
    if args.profile_case:
        # small case for ncu: 512 samples (about 2.6 GB of voltages), many launches so that
        # one of the run's own launches follows the tuner's (at most ~110 launches)
        T = 512
        plans, dvs, outs, _, _, _ = batched_setup(torch, dev, T)
        stream = torch.cuda.Stream(dev)
        with fb.batch_create(plans) as b, torch.cuda.stream(stream):
            for _ in range(200):
                fb.batch_execute(b, dvs, T, outs, stream)
            torch.cuda.synchronize(dev)
        print("profile case done", flush=True)
        for p in plans:
            p.close()
        return 0
    stream = torch.cuda.current_stream(dev)
    fp32 = fp32_peak(fb, torch, dev, stream)
    r = batched_form(fb, torch, dev, args.steps, args.warmup,
                     max(fp32["ffma_tflops"], fp32["ffma2_tflops"]))
    line = {"metric": r["metric"], "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "arrays", "tuned_snapshots_per_step",
                                         "items", "grid", "launch", "l2")},
            "gpu_launches": args.steps, "roofline": r["roofline"], "fp32_probe": fp32}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """A small case of the timed kernels for ncu: 256 channels x 768 samples (400 MB of
    voltages, above L2), three fftbf_execute calls and one fftbf_tied_beams call."""
    import torch
    import paper_1710_08591_gb300 as fb
    fb.build()
    nx, ny, mx, my, npol, n_int = 4, 256, 4, 512, 2, 384
    nfreq, T, n_tied = 256, 768, 2048
    src = synth.seeded_sources(WL["seed"] + 100, WL["n_src"], WL["amp"])
    block = synth.volts(T, nfreq, npol, nx, ny, seed=WL["seed"], sigma=WL["sigma"], sources=src)
    w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
    u, v = synth.tied_pointings(WL["seed"] + 1, nfreq, n_tied, nx, ny, mx, my)
    if args.tied:
        # the tied-beam GEMM at the step's shape on 64 channels: 128 windows of positive
        # synthetic beams, 2048 pointings (weight tables 268 MB, above L2); twice
        nw, nf = 128, 64
        g = torch.Generator(device="cuda")
        g.manual_seed(WL["seed"] + 9)
        pb = torch.rand((nw, nf, mx, my), device="cuda", generator=g) + 1.0
        uu, vv = synth.tied_pointings(WL["seed"] + 1, nf, n_tied, nx, ny, mx, my)
        out = torch.empty((nw, nf, n_tied), device="cuda")
        with fb.plan_create(nx, ny, mx, my, npol, nf, n_int, weights=w) as plan:
            for _ in range(2):
                fb.tied_beams(plan, pb, nw, n_tied, uu, vv, out)
            fb.plan_sync(plan)
        print("profile case (tied) done")
        return 0
    if args.products:
        # the intensity-space products on 40 windows x 1024 channels of positive synthetic
        # beams (335 MB, above L2): stacked visibilities and localisation, twice each
        nw, nf = 40, 1024
        g = torch.Generator(device="cuda")
        g.manual_seed(WL["seed"] + 7)
        pb = torch.rand((nw, nf, mx, my), device="cuda", generator=g) + 1.0
        with fb.plan_create(nx, ny, mx, my, npol, nf, n_int, weights=w) as plan:
            dx, dy = fb.stacked_shape(plan)
            vis = torch.empty((nw, nf, dx, dy), dtype=torch.complex64, device="cuda")
            loc = torch.empty((nw, nf, 3), device="cuda")
            for _ in range(2):
                fb.stacked_visibilities(plan, pb, nw, vis)
            for _ in range(2):
                fb.localise(plan, pb, nw, loc, 5, 10)
            fb.plan_sync(plan)
        print("profile case (products) done")
        return 0
    dvol = torch.from_numpy(block.reshape(-1)).cuda()
    beams = torch.empty((T // n_int, nfreq, mx, my), device="cuda")
    tied = torch.empty((T // n_int, nfreq, n_tied), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        if args.form != "fp32":
            fb.plan_set_precision(plan, {"tc_fp16": fb.PREC_TC_FP16, "tc_bf16": fb.PREC_TC_BF16,
                                     "tc_fp16x3": fb.PREC_TC_FP16X3}[args.form])
        for _ in range(3):
            fb.execute(plan, dvol, T, beams)
        fb.tied_beams(plan, beams, T // n_int, n_tied, u, v, tied)
        fb.plan_sync(plan)
    print("profile case done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["fp32", "tc_fp16", "tc_bf16", "tc_fp16x3"], default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["chime", "batched"], default="chime")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-frames", type=int, default=10000)
    ap.add_argument("--profile-case", action="store_true",
                    help="run a small case of the timed kernels (for ncu) and exit")
    ap.add_argument("--tied", action="store_true",
                    help="with --profile-case: the tied-beam GEMM")
    ap.add_argument("--products", action="store_true",
                    help="with --profile-case: the stacked-visibility and localisation kernels")
    args = ap.parse_args()
    if args.profile_case and args.workload == "batched":
        return run_batched(args)
    if args.profile_case:
        return run_profile_case(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
