"""Repeat-run check of the CUDA path's jackknife error bars (the Results section's check: the
spread of independent runs against the quoted error bar, their mean against the deterministic
value).  K = 32 independent `mrq_sample` runs (distinct Philox seeds, G = 16 walker groups each)
on the 12-orbital workload:

  * the sample standard deviation of E^(2), E_var and a0^2 over the runs agrees with the root mean
    square of the sigma each run reports (ratio in [0.65, 1.4]: about 3 standard deviations of the
    chi^2 spread with K - 1 = 31 degrees of freedom; a jackknife missing its (G - 1)/G factor is
    off by a factor of about 4);
  * the mean of the K estimates lies within 3 standard errors of the brute-force value;
  * the blocking analysis of one walk's time series of block sums agrees with its jackknife.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

K = 32


@pytest.fixture(scope="module")
def runs():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    orc = O.Oracle.from_system(s)
    ex = O.exact_from_brute(orc.brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    ctx = P.Context.from_system(s)
    try:
        fin = [ctx.sample(ctx.params(512, 500, burn_in=100, seed=9001 + 7 * k, n_groups=16)) for k in range(K)]
    finally:
        ctx.close()
    return fin, ex


@pytest.mark.parametrize("q", ["e2", "e_var", "a0sq"])
def test_spread_of_independent_runs_matches_the_jackknife_sigma(runs, q):
    fin, _ = runs
    v = np.array([f[q] for f in fin])
    sig = np.array([f[q + "_sigma"] for f in fin])
    assert np.all(sig > 0)
    ratio = v.std(ddof=1) / np.sqrt(np.mean(sig ** 2))
    assert 0.65 <= ratio <= 1.4, ratio


@pytest.mark.parametrize("q", ["e2", "e_var", "a0sq"])
def test_mean_of_independent_runs_is_unbiased(runs, q):
    fin, ex = runs
    v = np.array([f[q] for f in fin])
    se = v.std(ddof=1) / np.sqrt(K)
    assert abs(v.mean() - ex[q]) < 3.0 * se, (v.mean(), ex[q], se)


def test_blocking_analysis_agrees_with_the_jackknife():
    """The cross-check of the error bars: one walk advanced in 256 blocks of 8 steps, its per-block
    sums of w E_L, w and w delta_CAS (all walkers) reblocked (Flyvbjerg-Petersen) give errors of
    E_var and a0^2 that agree with the jackknife over walker groups of the same walk."""
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    ctx = P.Context.from_system(s)
    G, nw, burn, nb, bs = 16, 512, 100, 256, 8
    try:
        ctx.walkers_init(ctx.params(nw, 0, burn_in=burn, seed=424, n_groups=G))
        ctx.walkers_advance(burn)
        prev = ctx.accumulators(G)
        E, Wt, N0 = [], [], []
        for _ in range(nb):
            ctx.walkers_advance(bs)
            a = ctx.accumulators(G)
            E.append(a["E"].sum() - prev["E"].sum())
            Wt.append(a["W"].sum() - prev["W"].sum())
            N0.append(a["N"][:, 0].sum() - prev["N"][:, 0].sum())
            prev = a
        res = ctx.finalize()
    finally:
        ctx.close()
    r_e = P.reblock_ratio(E, Wt)
    r_a = P.reblock_ratio(s.c[0] ** 2 * np.array(N0), Wt)
    assert abs(r_e["R"] - res["e_var"]) < 1e-10 * abs(res["e_var"])
    assert abs(r_a["R"] - res["a0sq"]) < 1e-10
    assert 0.6 <= r_e["sigma"] / res["e_var_sigma"] <= 1.6, (r_e["sigma"], res["e_var_sigma"])
    assert 0.6 <= r_a["sigma"] / res["a0sq_sigma"] <= 1.6, (r_a["sigma"], res["a0sq_sigma"])
