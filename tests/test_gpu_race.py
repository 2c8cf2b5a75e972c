"""The move race's FP32 screen never drops the winner (Sec. II B, first-reaction form).

The walk draws an exponential clock t = -ln(u)/Gamma for every neighbour and moves to the
smallest.  It evaluates the exact FP64 clock only for candidates whose FP32 clock is within a
1e-4 margin of the best so far, so the FP32 clock (formed exactly as the walk forms it, from the
FP32 image of Gamma) must track the FP64 one to well under 1e-4 for every u, including u near 0
(k small) and near 1 (k near 2^53), and must be 0 - never screened out - wherever FP32 cannot
hold it: rates outside [1e-30, 1e30] and clocks below the normal FP32 range.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KS = [0, 1, 2, 1 << 20, (1 << 28) - 1, 1 << 28, 1 << 36, 1 << 45, (1 << 52) - 2, (1 << 52) - 1, 1 << 52,
      (1 << 52) + 1, 1 << 51, (1 << 53) - 2, (1 << 53) - 1]
RATES = [1e-29, 1e-10, 3.7e-3, 1.0, 42.0, 1e10, 1e29]


def _clocks(k, r):
    import paper_1909_06935_gb300 as P
    with P.Context() as ctx:
        return ctx.race_clocks(k, r)


def test_screen_tracks_the_exact_clock_for_every_u():
    rng = np.random.default_rng(5)
    ks = np.array(KS + list(rng.integers(0, 1 << 53, 2000, dtype=np.uint64)), np.uint64)
    k, r = np.meshgrid(ks, np.array(RATES))
    k, r = k.ravel(), r.ravel()
    scr, ex = _clocks(k, r)
    u = (k.astype(np.float64) + 1.0) * 2.0 ** -53          # exact: k + 1 <= 2^53
    ref = -np.log(u) / r
    assert np.allclose(ex, ref, rtol=1e-15, atol=0.0)
    assert np.all(np.isfinite(scr)) and np.all(np.isfinite(ex)) and np.all(scr >= 0.0)
    # the safety property: the screen never exceeds the exact clock by more than 1e-6
    assert np.all(scr.astype(np.float64) <= ex * (1.0 + 1e-6))
    # 0 only where FP32 cannot hold the clock (u = 1, or a clock below the normal FP32 range)
    zero = scr == 0.0
    assert np.all((ex[zero] == 0.0) | (ex[zero] < 1.2e-37))
    rel = np.abs(scr[~zero].astype(np.float64) / ex[~zero] - 1.0)
    assert rel.max() < 1e-6, (rel.max(), k[~zero][rel.argmax()], r[~zero][rel.argmax()])
    # the screen is exercised, not bypassed: almost every pair gets a finite FP32 clock
    assert (~zero).mean() > 0.99


def test_rates_outside_the_fp32_range_are_never_screened_out():
    k = np.array([0, 1 << 30, (1 << 53) - 2, 12345, 1 << 52], np.uint64)
    r = np.array([1e-300, 1e-40, 1e-31, 1e31, 1e300])
    scr, ex = _clocks(k, r)
    assert np.all(scr == 0.0)
    assert np.allclose(ex, -np.log((k.astype(np.float64) + 1.0) * 2.0 ** -53) / r, rtol=1e-15)
