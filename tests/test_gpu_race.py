"""The move race's FP32 screen never drops the winner (Sec. II B, first-reaction form).

The walk draws an exponential clock t = -ln(u)/Gamma for every neighbour and moves to the
smallest.  It takes the exact FP64 clock only for candidates that pass an FP32 screen against the
lane's best clock so far (u > exp(-Gamma t_best), tested as 1 - u < -expm1(-y) with a 1e-4 margin
on y).  The screen must let through every candidate whose exact clock beats the best, for every u
(u near 0 and near 1 included), and must reject clear losers, so that it does its job.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KS = [0, 1, 2, 1 << 20, (1 << 28) - 1, 1 << 28, 1 << 36, 1 << 45, (1 << 51), (1 << 52) - 2, (1 << 52) - 1,
      1 << 52, (1 << 52) + 1, (1 << 53) - 2, (1 << 53) - 1]
RATES = [1e-29, 1e-10, 3.7e-3, 1.0, 42.0, 1e10, 1e29]
FACTORS = [0.25, 0.5, 0.9, 0.999, 0.99999, 1.00001, 1.0001, 1.001, 1.1, 2.0, 10.0, 1e6]


def _screen(k, r, tb):
    import paper_1909_06935_gb300 as P
    with P.Context() as ctx:
        return ctx.race_screen(k, r, tb)


def _grid():
    rng = np.random.default_rng(5)
    ks = np.array(KS + list(rng.integers(0, 1 << 53, 600, dtype=np.uint64)), np.uint64)
    k, r = np.meshgrid(ks, np.array(RATES))
    k, r = k.ravel(), r.ravel()
    exact = -np.log((k.astype(np.float64) + 1.0) * 2.0 ** -53) / r
    return k, r, exact


def test_screen_never_rejects_a_winner():
    k, r, exact = _grid()
    kk, rr, tb = [], [], []
    for f in FACTORS:
        kk.append(k)
        rr.append(r)
        tb.append(np.where(exact > 0, exact * f, 1e-300 * f))
    kk, rr, tb = np.concatenate(kk), np.concatenate(rr), np.concatenate(tb)
    ok, ex = _screen(kk, rr, tb)
    assert np.allclose(ex, -np.log((kk.astype(np.float64) + 1.0) * 2.0 ** -53) / rr, rtol=1e-15, atol=0.0)
    wins = ex < tb
    assert wins.sum() > 1000
    assert np.all(ok[wins]), (kk[wins & ~ok][:5], rr[wins & ~ok][:5], tb[wins & ~ok][:5])
    # clear losers (clock at least 10 % above the best) are rejected wherever the screen is active:
    # rate, best clock and their product in the normal FP32 range, Gamma t_best <= 3.9
    active = (rr >= 1e-29) & (rr <= 1e29) & (tb >= 1e-29) & (tb <= 1e29) & (rr * tb >= 1e-29) & (rr * tb <= 3.9)
    losers = active & (ex > 1.1 * tb)
    assert losers.sum() > 1000
    assert not np.any(ok[losers])


def test_no_best_yet_and_rates_outside_the_fp32_range_always_pass():
    k, r, exact = _grid()
    ok, _ = _screen(k, r, np.full(len(k), np.inf))
    assert np.all(ok)
    k2 = np.array([0, 1 << 30, (1 << 53) - 2, 12345, 1 << 52], np.uint64)
    r2 = np.array([1e-300, 1e-40, 1e-31, 1e31, 1e300])
    ok2, _ = _screen(k2, r2, np.full(5, 1.0))
    assert np.all(ok2)
