"""The allocation-free entry point (fengine_process_chunk_noalloc) against the
plan-based fengine_process_chunk, through the C ABI, on two consecutive
chunks. It is for callers that cannot allocate device memory (their memory
belongs to another allocator, or cudaMalloc's implicit synchronisation is
not acceptable in their loop); its working storage is a fixed device array
inside the library. Collected last so that a run stopping at the first
failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2303_09886_gb300 import fengine, synth
from tests.fe_harness import streams

pytestmark = pytest.mark.gpu


class NoAllocArgs(ctypes.Structure):
    _fields_ = [("n_antennas", ctypes.c_int32), ("n_channels", ctypes.c_int32),
                ("n_taps", ctypes.c_int32), ("spectra_per_heap", ctypes.c_int32),
                ("chunk_samples", ctypes.c_int64), ("max_delay_samples", ctypes.c_int64),
                ("first_sample", ctypes.c_int64)]


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_09886_gb300 import build
    build.build()
    lib = fengine.load()
    f = lib.fengine_process_chunk_noalloc
    f.argtypes = [ctypes.POINTER(NoAllocArgs), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib


def _pack(s):
    return np.stack([np.stack([synth.pack10(s[a, p]) for p in range(2)]) for a in range(s.shape[0])])


@pytest.mark.parametrize("n_ant,n,T,M,D,S", [
    (2, 1024, 16, 48, 40, 16),     # one slab, N2 = 256
    (1, 32768, 16, 128, 40, 20),   # N1 = 64, N2 = 1024 (persistent second stage); its working storage
                                   # holds 96 spectra, so a call is two slabs through one intermediate,
                                   # and heaps of 20 spectra straddle the slab boundary
])
def test_noalloc_matches_plan_on_two_calls(lib, n_ant, n, T, M, D, S):
    import torch
    N = 2 * n
    L = N * M
    H = (N * (T - 1) + D + 15) // 16 * 16
    s = streams(synth.SEED_BASE + 90, n_ant, 2 * L, 35.0, tones=[(0.17, 70.0, 0.2)])
    models = np.array([[[3.7 + 11 * a + 0.4 * p, 2e-6, 0.3 * a - 0.2 * p, 1e-5, 0.0] for p in range(2)]
                       for a in range(n_ant)], np.float64)
    gains = synth.random_gains(91, 2 * n_ant, n).reshape(n_ant, 2, n)

    plan = fengine.Plan(n_ant, n, T, L, spectra_per_heap=S, max_delay_samples=D)
    for a in range(n_ant):
        for p in range(2):
            d, r, ph, pr, tref = models[a, p]
            plan.set_delay(a, p, d, r, ph, pr, t_ref=int(tref))
            plan.set_gains(a, p, gains[a, p])
    d_w = torch.from_numpy(fengine.default_weights(n, T)).cuda()
    d_g = torch.from_numpy(np.ascontiguousarray(gains).view(np.float32).reshape(-1)).cuda()
    dm = np.ascontiguousarray(models.reshape(-1))
    stream = torch.cuda.current_stream()
    for c in range(2):
        t_in = c * L
        d_in = torch.from_numpy(_pack(s[:, :, t_in:t_in + L])).cuda()
        ref = torch.empty(plan.info.out_bytes, dtype=torch.int8, device="cuda")
        plan.process(d_in, t_in, ref)
        # history: samples [t_in - H, t_in), zeros before the stream start
        hist = np.zeros((n_ant, 2, H), np.int16)
        lo = max(0, t_in - H)
        hist[:, :, H - (t_in - lo):] = s[:, :, lo:t_in]
        d_hist = torch.from_numpy(_pack(hist)).cuda()
        out = torch.full((plan.info.out_bytes,), 99, dtype=torch.int8, device="cuda")
        args = NoAllocArgs(n_ant, n, T, S, L, D, t_in)
        st = lib.fengine_process_chunk_noalloc(
            ctypes.byref(args), d_hist.data_ptr(), d_in.data_ptr(), d_w.data_ptr(), d_g.data_ptr(),
            dm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.data_ptr(), stream.cuda_stream)
        assert st == 0, fengine.STATUS.get(st, st)
        torch.cuda.synchronize()
        a_ref, a_out = ref.cpu().numpy().astype(np.int16), out.cpu().numpy().astype(np.int16)
        diff = np.abs(a_ref - a_out)
        print(f"[no-alloc] n={n} call {c}: exact fraction {np.mean(diff == 0):.6f}")
        assert diff.max() <= 1
    plan.close()


def test_noalloc_refuses_shapes_beyond_its_storage(lib):
    import torch
    dummy = torch.zeros(64, dtype=torch.uint8, device="cuda")
    w = torch.zeros(16, dtype=torch.float32, device="cuda")
    dm = np.zeros(5 * 200, np.float64)
    for args in (NoAllocArgs(40, 1024, 16, 0, 2048 * 4, 0, 0),          # 80 streams > 64
                 NoAllocArgs(32, 32768, 16, 0, 65536 * 4096, 0, 0)):    # working storage > array
        st = lib.fengine_process_chunk_noalloc(
            ctypes.byref(args), dummy.data_ptr(), dummy.data_ptr(), w.data_ptr(), w.data_ptr(),
            dm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dummy.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert st == 1


def test_noalloc_refuses_non_finite_or_fractional_models(lib):
    import torch
    n, T, L = 1024, 4, 2048 * 8
    dummy = torch.zeros(2 * L, dtype=torch.uint8, device="cuda")
    w = torch.zeros(2 * n * T, dtype=torch.float32, device="cuda")
    g = torch.zeros(4 * n, dtype=torch.float32, device="cuda")
    out = torch.zeros(n * 8 * 4, dtype=torch.int8, device="cuda")
    args = NoAllocArgs(1, n, T, 0, L, 10, 0)
    for bad in ([1.0, float("nan"), 0, 0, 0], [1.0, 0, float("inf"), 0, 0], [1.0, 0, 0, 0, 0.5]):
        dm = np.array(bad + [1.0, 0, 0, 0, 0], np.float64)
        st = lib.fengine_process_chunk_noalloc(
            ctypes.byref(args), dummy.data_ptr(), dummy.data_ptr(), w.data_ptr(), g.data_ptr(),
            dm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert st == 1, bad
