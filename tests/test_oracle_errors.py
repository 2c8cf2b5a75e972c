"""Repeat-run pin of the oracle's jackknife error bars (no GPU).

The Results section checks SC-NEVPT2(s) error bars the same way: many independent runs, whose
spread is compared with the quoted error bar and whose mean is compared with the deterministic
value.  Here K = 64 independent runs (each with G = 16 walker groups) come out of one oracle walk
with K * G groups: the groups of run k are k*G ... k*G + G - 1, and walker w sits in group w mod KG,
so every run has its own walkers and shares nothing with the others.  Then

  * the sample standard deviation of a run's estimate over the K runs must agree with the root
    mean square of the jackknife sigma each run reports: for K = 64 the ratio of the two lies in
    [0.75, 1.3] with overwhelming probability (chi^2 with K - 1 degrees of freedom, plus the
    sigma estimates' own scatter); a jackknife that drops its (G - 1)/G factor, or uses the
    leave-one-out spread without it, is off by a factor of about 4 and fails;
  * the mean of the K estimates must lie within 3 standard errors of the brute-force value over
    the whole first-order interacting space (the nonlinear bias of E^(2) is below the noise).

The same holds for the sampled SC-MRCI(s) gradient (Eq. 8-9) on labels the walk visits often.
"""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle import SYSTEMS, tiny

K, G = 64, 16
RUNS = {"1c2a2v": (32, 600, 2024), "1c3a2v_open": (32, 400, 8)}   # walkers per run, steps, seed


@pytest.fixture(scope="module", params=list(RUNS))
def runs(request):
    name = request.param
    nw, ns, seed = RUNS[name]
    s = tiny(**SYSTEMS[name])
    o = O.Oracle.from_system(s)
    br = o.brute(label_matrix=True)
    ex = O.exact_from_brute(br, o.e0, o.c, s.n_core, s.n_virt)
    gx, _ = O.exact_gradient(br, o.c)
    acc = o.sample(K * nw, ns, 100, seed=seed, n_groups=K * G)
    fin, grads, gsig = [], [], []
    for k in range(K):
        sl = slice(k * G, (k + 1) * G)
        a = {q: acc[q][sl] for q in ("N", "U", "W", "E", "A", "B")}
        fin.append(o.finalize(a))
        g, sg = O.mrci_gradient_groups(a)
        grads.append(g)
        gsig.append(sg)
    return dict(fin=fin, ex=ex, gx=gx, grads=np.array(grads), gsig=np.array(gsig))


@pytest.mark.parametrize("q", ["e2", "e_var", "a0sq"])
def test_spread_of_independent_runs_matches_the_jackknife_sigma(runs, q):
    v = np.array([f[q] for f in runs["fin"]])
    sig = np.array([f[q + "_sigma"] for f in runs["fin"]])
    assert np.all(sig > 0)
    ratio = v.std(ddof=1) / np.sqrt(np.mean(sig ** 2))
    assert 0.75 <= ratio <= 1.3, ratio


@pytest.mark.parametrize("q", ["e2", "e_var", "a0sq"])
def test_mean_of_independent_runs_is_unbiased(runs, q):
    v = np.array([f[q] for f in runs["fin"]])
    z = (v.mean() - runs["ex"][q]) / (v.std(ddof=1) / np.sqrt(K))
    assert abs(z) < 3.0, z


def test_gradient_spread_matches_its_jackknife_sigma(runs):
    g, sg, gx = runs["grads"], runs["gsig"], runs["gx"]
    # labels visited by almost every group of every run (the jackknife needs each group's sum)
    ok = np.isfinite(sg).all(0) & (sg > 0).all(0) & (np.abs(gx) > 0)
    assert ok.sum() >= 1
    ratio = np.sqrt(np.mean(g[:, ok].var(0, ddof=1)) / np.mean(sg[:, ok] ** 2))
    assert 0.75 <= ratio <= 1.3, ratio
    z = (g[:, ok].mean(0) - gx[ok]) / (g[:, ok].std(0, ddof=1) / np.sqrt(K))
    assert np.abs(z).max() < 3.5, z
