#!/usr/bin/env python3
"""Throughput benchmark of the GB300 F-engine hot path.

One step = one fengine_process_chunk call: every stage of the hot path over
one chunk of every stream of the workload (default: 4 antennas x 2 pols x
2^25 samples/pol, 8192 channels, 16 taps). Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 2] [--impl fengine|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (the
comparison arm): each step is a bounded sample of the same workload.
Under torchrun every rank runs an independent replica (no collective on the
data path: the streams are independent), timing is max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "input Gsample/s per GB300 (8K-ch, 16-tap), TC/batched vs FP32 plain; % HBM roofline"
UNIT = "Gsample/s"

# DRAM bytes (read + write) per input sample of each slab kernel, from ncu
# captures (profiles/) of 1 antenna x 2 pol x 2^24 samples/pol with the whole
# chunk in one slab (one launch of 2 x 1024 spectra = 33.5 M samples). ncu
# flushes the caches before each replay (cold cache). The bench scales them to
# its own launch by the input samples the launch processes. Valid only for the
# sources they were taken from (src = hash of the kernel's source files).
KERNEL_SOURCES = {
    "k_phase1": ['k_phase1.cuh', 'k_phase1_tile.inc', 'k_phase1_t1.cu', 'k_phase1_t2.cu', 'k_phase1_t4.cu', 'k_phase1_t8.cu', 'k_phase1_t16.cu', 'k_phase1_t32.cu', 'fe_device.cuh', 'fe_internal.cuh'],
    "k_phase2": ['k_phase2.cu', 'fe_device.cuh', 'fe_internal.cuh'],
    "k_phase2w": ['k_phase2w.cu', 'fe_device.cuh', 'fe_internal.cuh'],
    "k_phase1_tc": ['k_phase1_tc.cu', 'fe_device.cuh', 'fe_internal.cuh'],
    "k_unpack_cols": ['k_phase1_tc.cu', 'fe_device.cuh', 'fe_internal.cuh'],
}
_CAPTURED = 33554432   # input samples of the captured launch
NCU_TRAFFIC = {
    "k_phase1<16,16,32,0>": {"bytes_per_sample": (44702720 + 92542720) / _CAPTURED, "src": "17209441f63721c1"},
    "k_phase2w": {"bytes_per_sample": (170189312 + 22351616) / _CAPTURED, "src": "0ed9442a5b4bd850"},
    "k_phase2w<half>": {"bytes_per_sample": (94110976 + 22121728) / _CAPTURED, "src": "0ed9442a5b4bd850"},
    "k_phase1_tc<2,16,1>": {"bytes_per_sample": (96520704 + 48678144) / _CAPTURED, "src": "ea5cae1109eb0be7"},
    "k_unpack_cols": {"bytes_per_sample": (42592512 + 19993088) / _CAPTURED, "src": "ea5cae1109eb0be7"},
}


def _src_hash(kernel: str) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2303_09886_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the loop runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self, t0: float, t1: float):
        rows = [r for ts, r in self.rows if t0 - 0.15 <= ts <= t1 + 0.15 and len(r) >= 9]
        if not rows:
            rows = [r for ts, r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _max_over_ranks(x: float, ws: int, device: str) -> float:
    """The largest x over all ranks: the job takes as long as its slowest rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_throughput(samples_per_step: int, steps: int, ms: float, ws: int) -> float:
    """Whole-job Gsample/s: every rank (one independent replica per GPU)
    processes samples_per_step per step; ms is the slowest rank's time."""
    return ws * samples_per_step * steps / (ms / 1e3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, wl):
    """Comparison arm: the FP64 CPU oracle, as it stands, on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O

    cores = os.cpu_count() or 1
    # bounded sample of the workload: antenna 0, both pols, one full chunk
    n_spec = wl.chunk_samples // wl.N
    T = wl.n_taps
    w = O.pfb_weights(wl.N, T)
    dl = {(a, p): (d, r, ph, pr) for a, p, d, r, ph, pr in wl.delays()}
    g = wl.gains()
    from paper_2303_09886_gb300 import synth
    pk = [synth.pack10(wl.samples(0, p, wl.chunk_samples)) for p in range(2)]
    n_out = n_spec - T + 1          # spectra whose windows lie inside the chunk

    def step():
        q = []
        for p in range(2):
            s = O.unpack10(pk[p], wl.chunk_samples)
            d, r, ph, pr = dl[(0, p)]
            gains = np.ones(wl.n_channels) if g is None else g[0, p]
            _, qq, _ = O.channelize(s, 0, wl.N, T, w, O.DelayModel.constant(d, ph, r, pr), gains,
                                    0, n_out)
            q.append(qq)
        O.corner_turn(q[0], q[1], min(256, n_out))
        return 2 * n_out * wl.N

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    samples = 0
    for _ in range(args.steps):
        samples += step()
    dt = time.perf_counter() - t0
    value = samples / dt / 1e9
    sample_desc = (f"antenna 0 of {wl.n_antennas}, both pols, spectra 0..{n_out - 1} of one "
                   f"{wl.chunk_samples}-sample chunk per step (unpack + FIR + FFT + delay/gain + "
                   f"quantise + corner turn, FP64)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.description, "name": wl.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(wl, budget_s: float = 15.0):
    """The oracle as it stands on the host cores, on a bounded sample: antenna 0,
    pol 0, as many whole 64-spectrum blocks of the chunk as fit the budget."""
    from oracle import oracle as O
    from paper_2303_09886_gb300 import synth

    T, N = wl.n_taps, wl.N
    w = O.pfb_weights(N, T)
    d, r, ph, pr = [x[2:] for x in wl.delays() if x[0] == 0 and x[1] == 0][0]
    g = wl.gains()
    gains = np.ones(wl.n_channels) if g is None else g[0, 0]
    blk = 64
    n_spec = wl.chunk_samples // N
    s_all = wl.samples(0, 0, wl.chunk_samples)
    samples = 0
    t0 = time.perf_counter()
    q0 = 0
    while q0 + blk - 1 + T <= n_spec and time.perf_counter() - t0 < budget_s:
        lo = max(0, N * q0 - wl.max_delay)
        lo -= lo % 4
        hi = N * (q0 + blk - 1 + T)
        s = O.unpack10(synth.pack10(s_all[lo:hi]), hi - lo)
        O.channelize(s, lo, N, T, w, O.DelayModel.constant(d, ph, r, pr), gains, q0, blk)
        samples += blk * N
        q0 += blk
    dt = time.perf_counter() - t0
    return {"value": samples / dt / 1e9, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"antenna 0 pol 0, {samples // N} spectra ({samples} samples) of one chunk of "
                      f"{wl.name}: unpack + FIR + FFT + delay/gain + quantise, FP64, OpenMP over spectra"}


def _base_streams(seed: int, n: int, sigma: float = 32.0):
    """Packed 10-bit noise for benchmark inputs whose content does not matter
    for throughput (the parity tests cover the content)."""
    from paper_2303_09886_gb300 import synth
    return synth.pack10(synth.digitiser_samples(seed, n, sigma, [(0.123, 50.0, 0.0)]))


def _batched_launches(plans):
    """Kernel launches of one fengine_batch_process over FP32 plans: a delay
    table and a history-tail update per member (and the lost-data flags when
    its chunks are heap-aligned), then per group of members with the same
    (taps, N1, N2), one phase-1 and one phase-2 grid per slab round (at most
    64 members per grid)."""
    groups = {}
    for p in plans:
        groups.setdefault((p.n_taps, p.info.fft_n1, p.info.fft_n2), []).append(int(p.info.slabs_per_chunk))
    grids = 0
    for slabs in groups.values():
        for r in range(max(slabs)):
            k = sum(1 for s in slabs if s > r)
            grids += 2 * ((k + 63) // 64)
    small = sum(2 + (1 if p.chunk_samples % 4096 == 0 else 0) for p in plans)
    return small + grids


def run_batched(args):
    """Workload 4 as its own JSON line."""
    import torch
    from paper_2303_09886_gb300 import build as fe_build
    from paper_2303_09886_gb300 import fengine

    torch.cuda.set_device(0)
    fe_build.build()
    fengine.load()
    r = batched_result(args, fengine, torch)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "samples_per_step": r["samples_per_step"],
                       "pool_streams": args.pool},
            "sequential_single_stream": r["sequential_single_stream"], "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def batched_result(args, fengine, torch):
    """Workload 4: many uneven independent streams in one batched call.

    64 plans (1 antenna x 2 pols each) with channels drawn from {1024, 4096,
    8192, 32768}, taps from {4, 8, 16}, chunk lengths uniform in
    [2^20, 2^26] samples/pol truncated to a multiple of 2n, random delays and
    gains. One step = one fengine_batch_process over one chunk of every plan;
    the same members one call after another on one stream are timed beside it."""
    from paper_2303_09886_gb300 import synth

    g = synth.rng(synth.SEED_BASE + 4)
    n_plans = args.plans or 64
    base = _base_streams(synth.SEED_BASE + 4, 1 << 26)
    d_base = torch.from_numpy(base).cuda()
    plans, members = [], []
    total = 0
    for i in range(n_plans):
        n = int(g.choice([1024, 4096, 8192, 32768]))
        T = int(g.choice([4, 8, 16]))
        L = int(g.integers(1 << 20, (1 << 26) + 1)) // (2 * n) * (2 * n)
        L = max(L, 2 * n * 32)
        p = fengine.Plan(1, n, T, L, spectra_per_heap=0, max_delay_samples=2100)
        for pol in range(2):
            p.set_delay(0, pol, float(g.uniform(0, 2000)), 1e-9, float(g.uniform(0, 6.28)))
        gains = synth.random_gains(1000 + i, 2, n)
        p.set_gains(0, 0, gains[0])
        p.set_gains(0, 1, gains[1])
        nbytes = 2 * L * 5 // 4
        d_in = d_base[:nbytes].view(1, 2, -1) if nbytes <= d_base.numel() else \
            torch.from_numpy(np.resize(base, nbytes)).cuda().view(1, 2, -1)
        d_out = torch.empty(p.info.out_bytes, dtype=torch.int8, device="cuda")
        plans.append(p)
        members.append([p, d_in, 0, d_out])
        total += 2 * L
    batch = fengine.Batch(args.pool)
    stream = torch.cuda.current_stream()
    t = [0] * n_plans

    def step():
        for i, m in enumerate(members):
            m[2] = t[i]
            t[i] += m[0].chunk_samples
        batch.process([tuple(m) for m in members], stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the same plans one after another on a single stream, for comparison
    for _ in range(2):
        for m in members:
            m[0].process(m[1], t[members.index(m)], m[3], stream=stream)
            t[members.index(m)] += m[0].chunk_samples
    torch.cuda.synchronize()
    e0.record(stream)
    k2 = max(1, min(args.steps, 5))
    for _ in range(k2):
        for i, m in enumerate(members):
            m[0].process(m[1], t[i], m[3], stream=stream)
            t[i] += m[0].chunk_samples
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    value = total * args.steps / (ms / 1e3) / 1e9
    res = {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps, "steps": args.steps,
           "workload": f"batched uneven: {n_plans} independent dual-pol streams, channels in "
                       "{1024,4096,8192,32768}, taps in {4,8,16}, chunks U[2^20,2^26] samples/pol",
           "samples_per_step": total,
           "sequential_single_stream": {"value": total * k2 / (ms_seq / 1e3) / 1e9, "unit": UNIT,
                                        "ms_per_step": ms_seq / k2},
           "gpu_launches": args.steps * _batched_launches([m[0] for m in members])}
    batch.close()
    for p in plans:
        p.close()
    return res


def run_service(args):
    """Workload 5 as its own JSON line."""
    import torch
    from paper_2303_09886_gb300 import build as fe_build
    from paper_2303_09886_gb300 import fengine

    torch.cuda.set_device(0)
    fe_build.build()
    fengine.load()
    r = service_result(args, fengine, torch)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "steps": r["chunks_total"], "warmup": r["warmup_chunks"], "ms_per_step": r["ms_per_chunk"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"], "pool_streams": args.pool},
            "service": {k: v for k, v in r.items() if k not in ("value", "workload")}}
    print(json.dumps(line), flush=True)
    return 0


def service_result(args, fengine, torch):
    """Workload 5: streaming service. 16 plans (1 antenna x 2 pols, 8192
    channels, 16 taps), chunks of 2^24 samples/pol submitted from host memory
    by a Poisson process at `--load` times the rate the device sustains on
    resident input (measured first on the same plans), so that requests queue
    behind the host copies; delay updates every 2^22 samples; an HBM budget of
    `--budget-gb` for the buffers in flight, small enough that admission
    defers. Reports delivered Gsample/s, chunk latency p50/p99 (submit ->
    output in host memory) and the admitted / deferred counts."""
    from paper_2303_09886_gb300 import synth

    n_ant, n, T, L = 16, 8192, 16, 1 << 24
    chunks = args.chunks
    g = synth.rng(synth.SEED_BASE + 5)
    base = _base_streams(synth.SEED_BASE + 5, 2 * L)
    h_in = torch.from_numpy(base).pin_memory().numpy()
    plans = [fengine.Plan(1, n, T, L, max_delay_samples=2100) for _ in range(n_ant)]
    outs = [[torch.empty(p.info.out_bytes, dtype=torch.int8).pin_memory().numpy() for _ in range(2)]
            for p in plans]
    d0 = g.uniform(0, 2000, n_ant)
    budget = int(args.budget_gb * (1 << 30))
    # device-resident sustained rate of the same plans: resident input,
    # back-to-back calls on one stream
    d_in = torch.from_numpy(base).cuda()
    d_out = torch.empty(plans[0].info.out_bytes, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    for a, p in enumerate(plans):
        p.set_delay(0, 0, float(d0[a]), 1e-9)
        p.set_delay(0, 1, float(d0[a]), 1e-9)
        p.process(d_in, 0, d_out, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c in range(1, 3):
        for p in plans:
            p.process(d_in, c * L, d_out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sustained = 2 * n_ant * 2 * L / (e0.elapsed_time(e1) / 1e3)
    del d_in, d_out
    for p in plans:
        p.reset()
    # Poisson arrivals at load x sustained
    rate = args.load * sustained / (2 * L)          # chunks per second, all antennas
    svc = fengine.Service(n_streams=args.pool, hbm_budget_bytes=budget)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n_ant * chunks))
    order = [(k % n_ant, k // n_ant) for k in range(n_ant * chunks)]
    tickets = []
    t_start = time.perf_counter()
    for (a, c), at in zip(order, arrivals):
        while time.perf_counter() - t_start < at:
            time.sleep(0.0002)
        p = plans[a]
        for u in range(4):     # delay model refreshed every 2^22 samples
            t_apply = c * L + u * (1 << 22) - (T - 1) * 2 * n
            svc.set_delay(p, 0, 0, float(d0[a]) + 1e-9 * t_apply, 1e-9, t_apply=t_apply, t_ref=t_apply)
            svc.set_delay(p, 0, 1, float(d0[a]) + 1e-9 * t_apply, 1e-9, t_apply=t_apply, t_ref=t_apply)
        tickets.append(svc.submit(p, h_in, c * L, outs[a][c % 2]))
    lat = [svc.wait(x) for x in tickets]
    wall = time.perf_counter() - t_start
    st = svc.stats()
    svc.close()
    res = {"value": n_ant * chunks * 2 * L / wall / 1e9, "unit": UNIT,
           "workload": f"streaming service: {n_ant} ant x 2 pol, 8192 ch, 16 taps, chunks 2^24 samples/pol "
                       f"from host memory, Poisson arrivals at {args.load}x the device-resident rate, delay "
                       f"updates every 2^22 samples, HBM budget {args.budget_gb:g} GiB, {chunks} chunks per antenna",
           "chunks_total": n_ant * chunks, "warmup_chunks": n_ant, "ms_per_chunk": wall * 1e3 / (n_ant * chunks),
           "device_resident_Gsps": sustained / 1e9, "offered_Gsps": args.load * sustained / 1e9,
           "latency_p50_ms": float(np.percentile(lat, 50)) / 1e3,
           "latency_p99_ms": float(np.percentile(lat, 99)) / 1e3,
           "service_p50_ms": st["latency_p50_us"] / 1e3, "service_p99_ms": st["latency_p99_us"] / 1e3,
           "admitted": st["admitted"], "deferred": st["deferred"], "failed": st["failed"],
           "peak_bytes": st["peak_bytes"], "budget_bytes": budget}
    for p in plans:
        p.close()
    return res


def narrowband_result(args, fengine, torch, wl, d_in):
    """Narrow-band mode on the headline workload's input: the down-converter
    (D = 8, 16 taps per phase, band centred at 0.2 cycles/sample) and an
    8192-channel, 16-tap plan over its 10-bit output, one call each per
    step, timed with CUDA events on the same stream; Gsample/s of wide-band
    input."""
    D, Th, fc = 8, 16, 0.2
    L = wl.chunk_samples
    ddc = fengine.DDC(wl.n_antennas, D, Th, L, fc, 1.0)
    Lo = ddc.out_samples
    plan = fengine.Plan(wl.n_antennas, 8192, 16, Lo, max_delay_samples=0)
    d_nb = torch.empty((wl.n_antennas, 2, Lo * 5 // 4), dtype=torch.uint8, device="cuda")
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    t = [0]

    def step(with_plan):
        ddc.process(d_in, t[0], d_nb, stream=stream)
        if with_plan:
            plan.process(d_nb, t[0] * 2 // D, d_out, stream=stream)
        t[0] += L

    res = {}
    k = max(3, min(args.steps, 20))
    for name, with_plan in (("ddc_only", False), ("ddc_and_plan", True)):
        ddc.reset()
        plan.reset()
        t[0] = 0
        for _ in range(3):
            step(with_plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            step(with_plan)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        res[name] = {"ms_per_step": ms, "value": wl.samples_per_step / (ms / 1e3) / 1e9}
    ddc.close()
    plan.close()
    return {"value": res["ddc_and_plan"]["value"], "unit": UNIT,
            "config": {"decimation": D, "taps_per_phase": Th, "center_frequency": fc,
                       "narrow_band_channels": 8192, "narrow_band_taps": 16},
            "ddc_only": res["ddc_only"], "ddc_and_plan": res["ddc_and_plan"]}


def run_narrowband(args, wl):
    """Workload 6: the narrow-band mode alone as its own JSON line (the
    down-converter and an 8192-channel plan over its output on the given
    workload's input)."""
    import torch
    from paper_2303_09886_gb300 import build as fe_build
    from paper_2303_09886_gb300 import fengine

    torch.cuda.set_device(0)
    fe_build.build()
    fengine.load()
    d_in = torch.from_numpy(wl.packed_chunk()).cuda()
    r = narrowband_result(args, fengine, torch, wl, d_in)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": max(3, min(args.steps, 20)),
            "warmup": 3, "ms_per_step": r["ddc_and_plan"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "narrow-band mode on " + wl.description, **r["config"]},
            # per step: the down-converter and its history tail, then the plan's delay table,
            # lost-data flags, phase 1, phase 2 and history tail
            "ddc_only": r["ddc_only"], "gpu_launches": 7 * max(3, min(args.steps, 20))}
    print(json.dumps(line), flush=True)
    return 0


def _tuned_split(fengine, wl, prec, args):
    """The work split of the plan: the autotuner's pick (fengine_autotune) unless --no-autotune."""
    if args.split:
        n1, sl = (int(v) for v in args.split.split(","))
        return {"fft_n1": n1, "slab_spectra": sl, "autotuned": False}
    if args.no_autotune:
        return {"fft_n1": 0, "slab_spectra": 0, "autotuned": False}
    if args.tune_cache:
        best, hit = fengine.autotune_cached(args.tune_cache, wl.n_antennas, wl.n_channels, wl.n_taps,
                                            wl.chunk_samples, spectra_per_heap=wl.spectra_per_heap,
                                            max_delay_samples=wl.max_delay, precision=prec, calls=3)
        return {**best, "autotuned": True, "from_cache": hit}
    best, table = fengine.autotune(wl.n_antennas, wl.n_channels, wl.n_taps, wl.chunk_samples,
                                   spectra_per_heap=wl.spectra_per_heap, max_delay_samples=wl.max_delay,
                                   precision=prec, calls=3)
    return {**best, "autotuned": True, "from_cache": False,
            "candidates_ms_per_call": {f"n1={a},slab={b}": round(ms, 4) for a, b, ms in table}}


def _time_form(fengine, torch, wl, name, d_in, args):
    """Device time of `args.steps` calls of one precision form on the resident input."""
    prec = {"fp32": fengine.FP32, "fp16": fengine.TC_FP16, "bf16": fengine.TC_BF16}[name]
    split = _tuned_split(fengine, wl, prec, args)
    plan = fengine.Plan(wl.n_antennas, wl.n_channels, wl.n_taps, wl.chunk_samples,
                        spectra_per_heap=wl.spectra_per_heap, max_delay_samples=wl.max_delay, precision=prec,
                        fft_n1=split["fft_n1"], slab_spectra=split["slab_spectra"])
    for a, p, d, r, ph, pr in wl.delays():
        plan.set_delay(a, p, d, r, ph, pr)
    g = wl.gains()
    if g is not None:
        for a in range(wl.n_antennas):
            for p in range(2):
                plan.set_gains(a, p, g[a, p])
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    t = 0
    for _ in range(args.warmup):
        plan.process(d_in, t, d_out, stream=stream)
        t += wl.chunk_samples
    plan.set_profiling(True)
    plan.stage_times()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.process(d_in, t, d_out, stream=stream)
        t += wl.chunk_samples
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stage_ms, calls = plan.stage_times()
    plan_n1, plan_sl = plan.info.fft_n1, plan.info.slab_spectra
    plan.close()
    return {"value": wl.samples_per_step * args.steps / (ms / 1e3) / 1e9, "ms_per_step": ms / args.steps,
            "stage_ms_per_step": {k: v / max(calls, 1) for k, v in stage_ms.items()},
            "split": {"fft_n1": int(plan_n1), "slab_spectra": int(plan_sl), "autotuned": split["autotuned"]}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--impl", default="fengine", choices=["fengine", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--antennas", type=int, default=0, help="override the workload's antenna count")
    ap.add_argument("--chunk-samples", type=int, default=0, help="override the chunk length")
    ap.add_argument("--plans", type=int, default=0, help="workload 4: number of plans (default 64)")
    ap.add_argument("--pool", type=int, default=8, help="workloads 4/5: internal CUDA streams")
    ap.add_argument("--chunks", type=int, default=64, help="workload 5: chunks per antenna")
    ap.add_argument("--budget-gb", type=float, default=4.0, help="workload 5: HBM budget of the service (GiB)")
    ap.add_argument("--load", type=float, default=1.5, help="workload 5: offered load / sustained rate")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other precision forms")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (workload 4) and service (workload 5) keys of the default line")
    ap.add_argument("--no-autotune", action="store_true", help="use the built-in work split instead of the autotuner's")
    ap.add_argument("--tune-cache", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                         "paper_2303_09886_gb300", "autotune_cache.jsonl"),
                    help="JSON Lines file of autotuned splits ('' = always tune)")
    ap.add_argument("--split", default="", help="fixed work split 'N1,SLAB' (fft_n1, slab_spectra) instead of tuning")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="fp32 plain form, or the tensor-core forms (FP16/BF16 operands, FP32 accumulation)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)

    if args.workload == 4 and args.impl == "fengine":
        return run_batched(args)
    if args.workload == 5 and args.impl == "fengine":
        return run_service(args)
    from paper_2303_09886_gb300.workloads import WORKLOADS
    wl = WORKLOADS[min(args.workload, 3) if args.workload in (1, 2, 3) else 2]
    if args.antennas or args.chunk_samples:
        import dataclasses
        wl = dataclasses.replace(wl, n_antennas=args.antennas or wl.n_antennas,
                                 chunk_samples=args.chunk_samples or wl.chunk_samples)
        wl.description += f" [scaled: {wl.n_antennas} ant, {wl.chunk_samples} samples/pol]"
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.workload == 6:
        return run_narrowband(args, wl)

    import torch
    import torch.distributed as dist
    from paper_2303_09886_gb300 import build as fe_build
    from paper_2303_09886_gb300 import fengine

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fe_build.build() if rank == 0 else None
    if ws > 1:
        dist.barrier()
    fengine.load()

    prec = {"fp32": fengine.FP32, "fp16": fengine.TC_FP16, "bf16": fengine.TC_BF16}[args.precision]
    split = _tuned_split(fengine, wl, prec, args)
    plan = fengine.Plan(wl.n_antennas, wl.n_channels, wl.n_taps, wl.chunk_samples,
                        spectra_per_heap=wl.spectra_per_heap, max_delay_samples=wl.max_delay,
                        precision=prec, fft_n1=split["fft_n1"], slab_spectra=split["slab_spectra"])
    for a, p, d, r, ph, pr in wl.delays():
        plan.set_delay(a, p, d, r, ph, pr)
    g = wl.gains()
    if g is not None:
        for a in range(wl.n_antennas):
            for p in range(2):
                plan.set_gains(a, p, g[a, p])
    h_in = torch.from_numpy(wl.packed_chunk()).pin_memory()
    d_in = h_in.cuda()
    d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    L = wl.chunk_samples
    t_next = [0]

    def step():
        plan.process(d_in, t_next[0], d_out, stream=stream)
        t_next[0] += L

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    plan.set_profiling(True)
    plan.stage_times()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    stage_ms, calls = plan.stage_times()
    plan.set_profiling(False)
    ms_max = _max_over_ranks(ms, ws, "cuda")
    value = _job_throughput(wl.samples_per_step, args.steps, ms_max, ws)

    # end to end through the public API with host buffers: H2D of the packed
    # chunk from pinned memory, the call, D2H of the 8-bit output, every step
    e2e = None
    if not args.no_e2e:
        # End to end through the public API with host buffers, pipelined the
        # way a streaming receiver runs: two device input and output buffers,
        # the H2D copy of step k + 1 and the D2H copy of step k - 1 on their
        # own streams while step k computes. Every step's copies lie inside
        # the timed region (it opens before the first H2D and closes after
        # the last D2H).
        d_ins = [d_in, torch.empty_like(d_in)]
        d_outs = [d_out, torch.empty_like(d_out)]
        h_outs = [torch.empty(plan.info.out_bytes, dtype=torch.int8).pin_memory() for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def run_e2e(k_steps):
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            ev_out = [torch.cuda.Event() for _ in range(2)]
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)
            with torch.cuda.stream(s_in):
                d_ins[0].copy_(h_in, non_blocking=True)
            ev_in[0].record(s_in)
            for k in range(k_steps):
                b = k & 1
                if k + 1 < k_steps:
                    if k >= 1:
                        s_in.wait_event(ev_done[1 - b])      # compute k - 1 has read that buffer
                    with torch.cuda.stream(s_in):
                        d_ins[1 - b].copy_(h_in, non_blocking=True)
                    ev_in[1 - b].record(s_in)
                stream.wait_event(ev_in[b])
                if k >= 2:
                    stream.wait_event(ev_out[b])             # D2H of step k - 2 has drained d_outs[b]
                plan.process(d_ins[b], t_next[0], d_outs[b], stream=stream)
                t_next[0] += L
                ev_done[b].record(stream)
                s_out.wait_event(ev_done[b])
                with torch.cuda.stream(s_out):
                    h_outs[b].copy_(d_outs[b], non_blocking=True)
                ev_out[b].record(s_out)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)

        run_e2e(3)
        torch.cuda.synchronize()
        k2 = max(3, min(args.steps, 50))   # steady state: the first H2D and last D2H are not overlapped
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        run_e2e(k2)
        e3.record(stream)
        torch.cuda.synchronize()
        ems = _max_over_ranks(e2.elapsed_time(e3), ws, "cuda")
        e2e = {"value": _job_throughput(wl.samples_per_step, k2, ems, ws), "unit": UNIT,
               "h2d_bytes_per_step": int(h_in.numel()), "d2h_bytes_per_step": int(h_outs[0].numel()),
               "steps": k2, "pipelined": "H2D of step k+1 and D2H of step k-1 overlap step k"}
    # the other precision forms on the same input, same timing (context for
    # the FP32-plain vs tensor-core comparison; 8192-channel shapes only)
    forms = None
    if ws == 1 and not args.no_forms and wl.n_channels == 8192:
        forms = {args.precision: {"value": value, "ms_per_step": ms_max / args.steps,
                                  "stage_ms_per_step": {k: v / max(calls, 1) for k, v in stage_ms.items()}}}
        for name in ("fp32", "fp16", "bf16"):
            if name != args.precision:
                forms[name] = _time_form(fengine, torch, wl, name, d_in, args)
    clocks.stop()
    # workloads 4 (batched uneven streams) and 5 (service) on the same GPU,
    # after the headline's timed region, as extra keys of the line
    extra = {}
    if ws == 1 and not args.no_extra and args.workload == 2:
        import copy
        ab = copy.copy(args)
        ab.steps, ab.warmup = min(args.steps, 10), 3
        extra["batched"] = batched_result(ab, fengine, torch)
        extra["service"] = service_result(args, fengine, torch)
        extra["narrowband"] = narrowband_result(args, fengine, torch, wl, d_in)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel: the method's algorithmic bytes (1.25 B
    # packed in + 1 B out per input sample) of the samples one launch covers,
    # over that kernel's mean launch duration (CUDA events on its stream)
    N1 = plan.info.fft_n1
    tc = args.precision != "fp32"
    # bytes of intermediate per input sample (FP32 pairs; FP16 pairs in the FP16 form)
    inter = (N1 // 2 + 1) / N1 * (4.0 if args.precision == "fp16" else 8.0)
    spl = wl.samples_per_step
    # bytes each kernel itself must move per input sample (with the intermediates)
    kernel_bytes = {"phase1": (2.0 if tc else 1.25) + inter, "phase2": inter + 1.0, "unpack": 1.25 + 2.0}
    stages = [k for k in ("phase1", "phase2", "unpack") if stage_ms.get(k, 0.0) > 0.0]
    dom = max(stages, key=lambda k: stage_ms[k])
    slabs = max(int(plan.info.slabs_per_chunk), 1)
    launches = 1 if dom == "unpack" else slabs             # the unpack runs once per call
    kernel_ms_per_step = stage_ms[dom] / max(calls, 1)
    launch_ms = kernel_ms_per_step / launches
    peak, peak_kind = _peaks()
    samples_per_launch = spl / launches
    achieved = 2.25 * samples_per_launch / (launch_ms / 1e3) / 1e9
    achieved_kernel = kernel_bytes[dom] * samples_per_launch / (launch_ms / 1e3) / 1e9
    N2 = plan.info.fft_n2
    R_tc = N1 // 8
    kname = {"phase1": (f"k_phase1<{wl.n_taps},{N1},{min(512 // N1, N2)},0>" if not tc
                        else f"k_phase1_tc<{R_tc},{wl.n_taps},{1 if args.precision == 'fp16' else 2}>"),
             "phase2": ("k_phase2w" if N2 == 1024 else f"k_phase2<{N2}>")
             + ("" if args.precision != "fp16" else "<half>"),
             "unpack": "k_unpack_cols"}[dom]
    tr = NCU_TRAFFIC.get(kname)
    # scaled from the captured launch to this launch by its input samples
    # (the kernels' DRAM traffic grows in proportion to the samples processed)
    traffic = (tr["bytes_per_sample"] * samples_per_launch
               if tr and tr.get("src") == _src_hash(kname.split("<")[0]) else None)
    step_ms = ms_max / args.steps
    path_alg = 2.25 * spl / (step_ms / 1e3) / 1e9
    path_all = (2.25 + 2 * inter) * spl / (step_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": wl.description, "name": wl.name, "n_antennas": wl.n_antennas,
                   "n_channels": wl.n_channels, "n_taps": wl.n_taps, "chunk_samples": wl.chunk_samples,
                   "precision": args.precision, "parallelism": f"replicas x{ws}",
                   "split": {**split, "fft_n1": int(plan.info.fft_n1), "slab_spectra": int(plan.info.slab_spectra)},
                   "l2": f"inputs larger than L2: {h_in.numel() >> 20} MiB packed in + "
                         f"{plan.info.out_bytes >> 20} MiB out per step"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_sample": 2.25, "samples_per_launch": samples_per_launch,
                     "launch_ms": launch_ms, "launches_per_step": launches,
                     "with_intermediates": {"bytes_per_sample": kernel_bytes[dom], "achieved": achieved_kernel,
                                            "frac": achieved_kernel / peak}},
        "path": {"stage_ms_per_step": {k: v / max(calls, 1) for k, v in stage_ms.items()},
                 "algorithmic_GBps": path_alg, "frac_algorithmic": path_alg / peak,
                 "with_intermediates_GBps": path_all, "frac_with_intermediates": path_all / peak,
                 "bytes_per_sample": {"algorithmic": 2.25, "with_intermediates": 2.25 + 2 * inter}},
        "e2e": e2e,
        # delay table, history tail, lost-data flags (heap-aligned chunks),
        # the column unpack (tensor-core forms), a phase-1 / phase-2 pair per slab
        "gpu_launches": (2 + (1 if wl.chunk_samples % 4096 == 0 else 0) + (1 if tc else 0) + 2 * slabs)
        * args.steps,
        "forms": forms,
        "clocks": clocks.summary(w0, w1),
        **extra,
    }
    if not args.no_cpu and ws == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
