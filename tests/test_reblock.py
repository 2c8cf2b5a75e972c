"""The blocking analysis (Flyvbjerg and Petersen) that cross-checks the jackknife error bars,
pinned on series whose error of the mean is known in closed form: independent samples (the plain
standard error) and a stationary AR(1) process x_t = phi x_(t-1) + e_t, whose mean has the variance
(s2 / n) [(1 + phi) / (1 - phi) - 2 phi (1 - phi^n) / (n (1 - phi)^2)], s2 = var(e) / (1 - phi^2).
A ratio of block sums is checked against the delta method on independent blocks."""
import numpy as np

import paper_1909_06935_gb300 as P


def _ar1(n, phi, rng):
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1.0 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x


def test_independent_samples_give_the_plain_standard_error():
    rng = np.random.default_rng(3)
    x = rng.normal(2.0, 3.0, 1 << 14)
    r = P.reblock(x)
    assert r["levels"][0][1] == np.sqrt(np.mean((x - x.mean()) ** 2) / (len(x) - 1))
    assert abs(r["sigma"] / (3.0 / np.sqrt(len(x))) - 1.0) < 0.1


def test_ar1_plateau_matches_the_closed_form():
    rng = np.random.default_rng(11)
    n, phi = 1 << 18, 0.9
    x = _ar1(n, phi, rng)
    s2 = 1.0 / (1.0 - phi * phi)
    var = s2 / n * ((1 + phi) / (1 - phi) - 2 * phi * (1 - phi ** n) / (n * (1 - phi) ** 2))
    r = P.reblock(x)
    assert r["level"] >= 4                                 # the correlated series needs blocking
    assert abs(r["sigma"] / np.sqrt(var) - 1.0) < 0.15
    assert r["levels"][0][1] < 0.4 * np.sqrt(var)           # the unblocked estimate is far too small


def test_ratio_of_block_sums_matches_the_delta_method():
    rng = np.random.default_rng(5)
    nb = 4096
    den = rng.uniform(0.5, 1.5, nb)
    num = 2.5 * den + rng.normal(0.0, 0.2, nb)
    r = P.reblock_ratio(num, den)
    R = num.sum() / den.sum()
    y = (num - R * den) / den.mean()
    assert r["R"] == R
    assert abs(r["sigma"] / (y.std() / np.sqrt(nb)) - 1.0) < 0.1
