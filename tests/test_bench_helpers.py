"""Host-side helpers of bench.py that shape its JSON line, checked without a GPU: the counted flops of an
overlap-save float64 pass for either FFT length, and the batch planner's per-class summary."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fft_pass_flops_per_length():
    # a product pass: tiles of N - pad16(p + 1) rows, two real N-point transforms of 2.5 N log2 N each per tile
    m, p = 1_000_000, 500
    for N in (2048, 4096):
        tiles = math.ceil(m / (N - 512))
        assert bench.fft_pass_flops("fft", m, p, False, N) == tiles * 2 * 2.5 * N * math.log2(N)
    # per row the long tiles count fewer flops at this order (the reason they were tried)
    assert bench.fft_pass_flops("fft", m, p, False, 4096) < bench.fft_pass_flops("fft", m, p, False, 2048)
    # a Gram pass of a small order: one transform plus pad16(p + 1) (p + 1) edge multiply-adds per tile
    q = 20
    tiles = math.ceil(m / (2048 - 32))
    assert bench.fft_pass_flops("fft", m, q, True) == tiles * (2.5 * 2048 * 11 + 2.0 * 32 * 21)


class _T:
    TOLS_PRODUCT_DIRECT, TOLS_PRODUCT_FFT = 1, 2


def test_batch_plan_mix_groups_by_order_class():
    ps = [5, 14, 15, 40, 47, 48, 200]
    infos = [{"product_used": 1}, {"product_used": 1}, {"product_used": 2}, {"product_used": 2},
             {"product_used": 2}, {"product_used": 2}, {"product_used": 1}]
    mix = bench.batch_plan_mix(_T, ps, infos)
    assert mix["fft_series"] == 4 and mix["direct_series"] == 3
    # pad16(p + 1): 5, 14 -> 16; 15 -> 16; 40 -> 48; 47 -> 48; 48 -> 64; 200 -> 208
    assert mix["by_pad16_p_plus_1"] == {"16": "direct/fft", "48": "fft", "64": "fft", "208": "direct"}
