"""Shared machinery of the GPU parity tests: run a multi-chunk stream through
the CUDA path (via the C ABI binding) and through the FP64 oracle on the same
seeded bytes, and compare.

Parity bars (element by element, per stream):
  * window tap (unpacked, coarse-delayed integers): bit-exact;
  * pre-quantisation spectra: relative RMS <= 1e-5 for the FP32 form;
  * 8-bit output: |GPU - oracle| <= 1 LSB everywhere (exact fraction reported).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import oracle as O
from paper_2303_09886_gb300 import fengine, synth

REL_RMS_FP32 = 1e-5
REL_RMS_REDUCED = 2e-3     # FP16 / BF16 tensor-core forms


@dataclasses.dataclass
class Seg:
    delay: float = 0.0
    rate: float = 0.0
    phase: float = 0.0
    phase_rate: float = 0.0
    t_apply: int = -(2 ** 62)
    t_ref: int = 0


def streams(seed, n_ant, total, sigma, tones=(), chirp=None):
    """int16 [n_ant, 2, total]; each stream its own seed."""
    out = np.empty((n_ant, 2, total), np.int16)
    for a in range(n_ant):
        for p in range(2):
            out[a, p] = synth.digitiser_samples(seed + 101 * a + 7 * p, total, sigma, tones, chirp)
    return out


def run_gpu(samples, n_ch, T, L, n_chunks, delays, gains, S=0, D=0, weights=None, start=0,
            taps=True, prequant=True, precision=fengine.FP32, fft_n1=0, slab_spectra=0, Dmin=0,
            valids=None, flags=False, in_offset=0):
    """Process consecutive chunks of `samples` (starting at absolute `start`).
    delays[a][p]: list of Seg; gains[a][p]: complex array, a list of
    (t_apply, complex array) gain sets, or None. valids: per call a uint8
    [ant, pol, L/4096] array of received-heap flags (or None); flags: read
    back the output-heap flags; in_offset: place the packed chunk this many
    bytes (a multiple of 4) into a larger device buffer. Returns list of dicts
    per call (numpy copies of every output)."""
    import torch
    n_ant = samples.shape[0]
    plan = fengine.Plan(n_ant, n_ch, T, L, spectra_per_heap=S, max_delay_samples=D, weights=weights,
                        precision=precision, fft_n1=fft_n1, slab_spectra=slab_spectra, min_delay_samples=Dmin)
    for a in range(n_ant):
        for p in range(2):
            for sg in delays[a][p]:
                plan.set_delay(a, p, sg.delay, sg.rate, sg.phase, sg.phase_rate, sg.t_apply, sg.t_ref)
            if gains is not None and gains[a][p] is not None:
                if isinstance(gains[a][p], list):
                    for t_apply, g in gains[a][p]:
                        plan.set_gains(a, p, g, t_apply)
                else:
                    plan.set_gains(a, p, gains[a][p])
    M, N = plan.M, 2 * n_ch
    res = []
    for c in range(n_chunks):
        lo = c * L
        chunk = samples[:, :, lo:lo + L]
        packed = np.stack([np.stack([synth.pack10(chunk[a, p]) for p in range(2)]) for a in range(n_ant)])
        d_in = torch.from_numpy(packed).cuda()
        if in_offset:
            buf = torch.zeros(d_in.numel() + in_offset, dtype=torch.uint8, device="cuda")
            buf[in_offset:].copy_(d_in.reshape(-1))
            d_in = buf[in_offset:]
        d_out = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
        d_pre = torch.empty(n_ant * 2 * M * n_ch * 2, dtype=torch.float32, device="cuda") if prequant else None
        d_tap = torch.empty(n_ant * 2 * M * N, dtype=torch.int32, device="cuda") if taps else None
        d_valid = (torch.from_numpy(np.ascontiguousarray(valids[c], np.uint8)).cuda()
                   if valids is not None and valids[c] is not None else None)
        d_flags = torch.full((n_ant, plan.heaps), 7, dtype=torch.uint8, device="cuda") if flags else None
        m0 = plan.process(d_in, start + lo, d_out, d_pre, d_tap, valid=d_valid, heap_flags=d_flags)
        torch.cuda.synchronize()
        res.append(dict(
            m0=m0, out=d_out.cpu().numpy(), flags=(d_flags.cpu().numpy() if flags else None),
            pre=(d_pre.cpu().numpy().view(np.complex64).reshape(n_ant, 2, M, n_ch) if prequant else None),
            tap=(d_tap.cpu().numpy().reshape(n_ant, 2, M, N) if taps else None)))
    plan.device_status()          # raises if a kernel recorded a timeout or a clamped delay
    plan.close()
    return res, M, plan.S


def oracle_model(segs):
    return O.DelayModel([(s.t_apply, s.t_ref, s.delay, s.rate, s.phase, s.phase_rate) for s in segs])


def run_oracle(samples, n_ch, T, delays, gains, m0, M, weights=None, start=0):
    """Oracle for spectra [m0, m0 + M) of every stream: (pre, q, coarse)."""
    N = 2 * n_ch
    w = O.pfb_weights(N, T) if weights is None else np.asarray(weights, np.float64)
    n_ant = samples.shape[0]
    pre = np.empty((n_ant, 2, M, n_ch), np.complex128)
    q = np.empty((n_ant, 2, M, n_ch, 2), np.int8)
    co = np.empty((n_ant, 2, M), np.int64)
    for a in range(n_ant):
        for p in range(2):
            g = np.ones(n_ch) if gains is None or gains[a][p] is None else gains[a][p]
            if isinstance(g, list):
                g = [(t, np.asarray(x)) for t, x in g]
            dm = oracle_model(delays[a][p]) if delays[a][p] else O.DelayModel()
            pr, qq, cc = O.channelize(samples[a, p].astype(np.int32), start, N, T, w, dm, g, m0, M)
            pre[a, p], q[a, p], co[a, p] = pr, qq, cc
    return pre, q, co


def default_delays(n_ant, segs=None):
    return [[list(segs or [Seg()]) for _ in range(2)] for _ in range(n_ant)]


def compare_call(samples, call, M, S, n_ch, T, delays, gains, weights=None, start=0,
                 rel_rms=REL_RMS_FP32):
    """Compare one GPU call with the oracle. Returns a dict of statistics."""
    N = 2 * n_ch
    n_ant = samples.shape[0]
    pre_o, q_o, co = run_oracle(samples, n_ch, T, delays, gains, call["m0"], M, weights, start)
    stats = {}
    # window tap: bit-exact unpack + coarse delay
    if call["tap"] is not None:
        for a in range(n_ant):
            for p in range(2):
                s = samples[a, p].astype(np.int64)
                for qi in range(M):
                    i = N * (call["m0"] + qi) - co[a, p, qi] + np.arange(N) - start
                    expect = np.where(i >= 0, s[np.clip(i, 0, None)], 0)
                    np.testing.assert_array_equal(call["tap"][a, p, qi], expect,
                                                  err_msg=f"window tap a={a} p={p} q={qi}")
    # pre-quantisation spectra
    if call["pre"] is not None:
        worst = 0.0
        for a in range(n_ant):
            for p in range(2):
                ref = pre_o[a, p]
                err = np.sqrt(np.sum(np.abs(call["pre"][a, p] - ref) ** 2) / np.sum(np.abs(ref) ** 2))
                worst = max(worst, err)
        stats["rel_rms"] = worst
        assert worst <= rel_rms, f"pre-quant relative RMS {worst:.3g} > {rel_rms}"
    # 8-bit output in the heap layout
    exact = total = 0
    for a in range(n_ant):
        ref = O.corner_turn(q_o[a, 0], q_o[a, 1], S)
        got = call["out"][a * M * n_ch * 4:(a + 1) * M * n_ch * 4]
        d = np.abs(got.astype(np.int16) - ref.astype(np.int16))
        assert d.max() <= 1, f"int8 output differs by {d.max()} LSB (antenna {a})"
        exact += int(np.sum(d == 0))
        total += d.size
        # the requantiser itself: the 8-bit output is exactly R7 (round half
        # away from zero, saturate to +-127) of the GPU's own FP32 spectra
        if call["pre"] is not None:
            pre = call["pre"][a].astype(np.complex128)          # [pol][m][k]
            comp = np.stack([pre.real, pre.imag], axis=-1)      # [pol][m][k][2]
            r = np.where(comp >= 0, np.floor(comp + 0.5), -np.floor(-comp + 0.5))
            qq = np.clip(r, -127, 127).astype(np.int8)
            np.testing.assert_array_equal(got, O.corner_turn(qq[0], qq[1], S),
                                          err_msg=f"requantiser (antenna {a})")
    stats["exact_fraction"] = exact / total
    return stats
