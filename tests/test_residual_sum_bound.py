"""The error bound behind the column-strip sweep's residual sums (CPU only).

In the strip sweep each lane adds the squared stage-1 brackets of up to 256
cells (one per row of its strip) with compensated (Kahan) FP32 summation and
hands the lane's total to FP64 for every sum above the lane (Alg. 1's
stopping test reads these norms).  The claim is that the compensated lane
total is within about two FP32 roundings of the exact sum of the same FP32
squares, whatever the strip height, where a plain FP32 running sum drifts by
up to one rounding per term.  This checks both statements with the same
operations in numpy float32 (each add and subtract rounded to FP32, in the
kernel's order) against math.fsum of the values in FP64, on squares spread
over many orders of magnitude and on sorted worst-case orders.
"""
import math

import numpy as np

U32 = 2.0 ** -24   # unit roundoff of FP32


def kahan_f32(values):
    s = np.float32(0.0)
    c = np.float32(0.0)
    for q in values:
        y = np.float32(q - c)
        t = np.float32(s + y)
        c = np.float32(np.float32(t - s) - y)
        s = t
    return float(s) - float(c)   # the compensation folded in FP64, as the kernel does


def plain_f32(values):
    s = np.float32(0.0)
    for q in values:
        s = np.float32(s + q)
    return float(s)


def squares(rng, n, spread):
    b = rng.standard_normal(n) * 10.0 ** rng.uniform(-spread, spread, n)
    return (b.astype(np.float32) * b.astype(np.float32)).astype(np.float32)


def test_compensated_lane_sum_within_two_roundings():
    rng = np.random.default_rng(2108)
    worst = 0.0
    for n in (16, 64, 256):
        for spread in (0.0, 1.0, 3.0):
            for order in ("random", "ascending", "descending"):
                q = squares(rng, n, spread)
                if order == "ascending":
                    q = np.sort(q)
                elif order == "descending":
                    q = np.sort(q)[::-1]
                exact = math.fsum(float(x) for x in q)
                err = abs(kahan_f32(q) - exact) / exact
                worst = max(worst, err)
    assert worst <= 2.0 * U32, worst


def test_plain_fp32_running_sum_drifts_past_that_bound():
    # long runs of equal-sized squares: the plain running sum's roundings
    # accumulate with the number of terms, the compensated one's do not
    worst_plain, worst_comp = 0.0, 0.0
    for seed in range(5):
        rng = np.random.default_rng(seed)
        q = (1.0 + 0.1 * rng.random(4096)).astype(np.float32) * np.float32(1.1)
        exact = math.fsum(float(x) for x in q)
        worst_plain = max(worst_plain, abs(plain_f32(q) - exact) / exact)
        worst_comp = max(worst_comp, abs(kahan_f32(q) - exact) / exact)
    assert worst_comp <= 2.0 * U32, worst_comp
    assert worst_plain > 8.0 * U32, worst_plain
