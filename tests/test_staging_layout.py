"""Host checks of the phase-1 staged-input layout (no GPU): the shared-memory
segment size SEG that k_phase1.cuh declares holds, for every alignment of a
tile's first sample, the two bytes of each of the segment's W 10-bit samples
after the copy start has been rounded down to 16 bytes; and the FIR output
tile plus the staging ring of every staged shape leave room for two CTAs per
SM. The constants are read from the header itself, so a change there is
checked here."""
import os
import re

import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2303_09886_gb300", "csrc", "k_phase1.cuh")
SMEM_PER_SM = 228 * 1024      # shared memory of one SM
RESERVED_PER_CTA = 1024       # reserved by the system for each resident CTA


def _const(name):
    src = open(HDR).read()
    m = re.search(r"static constexpr int " + name + r" = ([^;]+);", src)
    assert m, name
    return m.group(1)


def _eval(expr, **env):
    # the header's integer arithmetic on non-negative values: C division is floor division
    py = expr.replace("/", "//")
    return eval(py, {}, env)


def _byte(s):
    """First byte of 10-bit sample s of an MSB-first packed stream (bits [10 s, 10 s + 10))."""
    return (s >> 2) * 5 + (((s & 3) * 5) >> 2)


def test_byte_of_sample_is_floor_of_ten_bits():
    for s in range(4096):
        assert _byte(s) == (10 * s) // 8


@pytest.mark.parametrize("W", [4, 8, 16, 32, 64])
def test_segment_holds_every_sample_for_every_alignment(W):
    seg = _eval(_const("SEG"), W=W)
    assert seg % 16 == 0
    for s0 in range(512):                        # every byte alignment of the first sample, many times over
        a0 = _byte(s0) & ~15                      # copy start, rounded down to 16 bytes
        for w in range(W):
            b = _byte(s0 + w)
            assert b - a0 + 1 < seg, (W, s0, w)   # both bytes of the field are inside the segment


@pytest.mark.parametrize("N1,W", [(8, 64), (16, 32), (32, 16), (64, 8)])
def test_two_staged_ctas_fit_on_an_sm(N1, W):
    R, SG = 32, int(_const("SG"))
    seg = _eval(_const("SEG"), W=W)
    m = re.fullmatch(r"\(N1 \* SEG <= (\d+)\) \? (\d+) : (\d+)", _const("NGRING"))
    assert m, _const("NGRING")
    ngring = int(m.group(2)) if N1 * seg <= int(m.group(1)) else int(m.group(3))
    gs = R * N1 * (W + 1) * 4                     # FIR output g
    ring = ngring * SG * N1 * seg                 # staged input rows
    static = (N1 // 2 + 1) * W * 8 + R * 4 + 256  # twiddles, delays, a grouped launch's parameters
    per_cta = gs + ring + static + RESERVED_PER_CTA
    assert 2 * per_cta <= SMEM_PER_SM, (N1, W, per_cta)
    # group g + NGRING - 1 is copied into the slot of group g - 1, which every
    # thread has finished with at g's barrier: at least two groups in the ring
    assert ngring >= 2
