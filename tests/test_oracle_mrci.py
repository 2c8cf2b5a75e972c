"""Pins of the oracle's SC-MRCI(s) optimisation pieces (Sec. II B, Eq. 8-9) against things other
than themselves (no GPU):

* the label Hamiltonian H_ll' = <v_l|H|v_l'> against the independent operator applier on whole
  determinant spaces;
* the exact gradient against central finite differences of the brute-force energy
  <psi|H|psi>/<psi|psi> (a different code path: the scalar sum over determinant pairs);
* the sampled gradient sums against exact identities (sum_l c_l A_l = sum w E_L,
  sum_l c_l B_l = sum w) and, statistically, against the exact gradient;
* the SC-MRCI eigenpair: variational bounds (full CI below, the reference and the sampling
  function above), zero gradient, and the energy of its vector through the brute-force scalar path;
* AMSGrad: the closed form of its first step, and convergence on a convex quadratic.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from tests import secondq as Q
from tests.test_oracle import SYSTEMS, eri4_of, label_of, phi0_dict, tiny


@pytest.fixture(scope="module", params=list(SYSTEMS))
def full(request):
    s = tiny(**SYSTEMS[request.param])
    o = O.Oracle.from_system(s)
    H = Q.Hamiltonian(s.h1, eri4_of(s), s.e_nuc)
    return s, o, H


def _sc_basis(s, H):
    """v_0 = phi0 and v_l = P_l H phi0 as dictionaries, from the operator applier."""
    phi = phi0_dict(s)
    basis = {0: dict(phi)}
    for m, a in H.apply(phi).items():
        l = label_of(m, s)
        if l > 0:
            basis.setdefault(l, {})[m] = a
    return basis


def test_label_hamiltonian_vs_operator_algebra(full):
    s, o, H = full
    br = o.brute(label_matrix=True)
    basis = _sc_basis(s, H)
    Hv = {l: H.apply(v) for l, v in basis.items()}
    ref = np.zeros_like(br["H"])
    for l, vl in basis.items():
        for k, hk in Hv.items():
            ref[l, k] = sum(a * hk.get(m, 0.0) for m, a in vl.items())
    scale = np.abs(ref).max()
    assert np.abs(br["H"] - ref).max() < 1e-11 * scale
    assert np.abs(br["H"] - br["H"].T).max() < 1e-11 * scale
    for l, vl in basis.items():                 # overlap: diag(N_l)
        assert br["N"][l] == pytest.approx(sum(a * a for a in vl.values()), rel=1e-12)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_exact_gradient_is_half_the_finite_difference(name):
    s = tiny(**SYSTEMS[name])
    o = O.Oracle.from_system(s)
    g, E = O.exact_gradient(o.brute(label_matrix=True), o.c)
    br = o.brute()
    assert E == pytest.approx(br["psi_H_psi"] / br["psi_norm"], rel=1e-12)
    visited = np.nonzero(br["N"] > 0)[0]
    rng = np.random.default_rng(5)
    for l in rng.choice(visited, min(6, len(visited)), replace=False):
        h = 1e-5 * max(1.0, abs(o.c[l]))
        e = []
        for sgn in (1, -1):
            c = o.c.copy()
            c[l] += sgn * h
            b = O.Oracle.from_system(s, c=c).brute()
            e.append(b["psi_H_psi"] / b["psi_norm"])
        fd = (e[0] - e[1]) / (2 * h)
        assert 2 * g[l] == pytest.approx(fd, rel=1e-5, abs=1e-9), l


def test_sampled_gradient_sums_identities():
    """sum_l c_l A_l = sum w E_L and sum_l c_l B_l = sum w in every group, for any sample: a
    wrong power of c_l, a lost label or a misplaced group breaks them."""
    s = S.workload("tiny_12o_cas4")
    o = O.Oracle.from_system(s)
    acc = o.sample(32, 60, 5, seed=3, n_groups=4)
    np.testing.assert_allclose(acc["A"] @ o.c, acc["E"], rtol=1e-12)
    np.testing.assert_allclose(acc["B"] @ o.c, acc["W"], rtol=1e-12)
    g, E = O.mrci_gradient(acc)
    assert abs(g @ o.c) < 1e-12 * np.abs(g * o.c).sum()          # <E_L - E> = 0
    assert E == pytest.approx(acc["E"].sum() / acc["W"].sum(), rel=1e-15)


def test_sampled_gradient_matches_exact_gradient():
    s = tiny(**SYSTEMS["1c2a2v"])
    o = O.Oracle.from_system(s)
    br = o.brute(label_matrix=True)
    gx, _ = O.exact_gradient(br, o.c)
    acc = o.sample(64, 2000, 100, seed=11, n_groups=16)
    g, sig = O.mrci_gradient_groups(acc)
    ok = sig > 0
    z = (g[ok] - gx[ok]) / sig[ok]
    assert ok.sum() >= 10
    assert np.abs(z).max() < 5.0
    assert np.sqrt(np.mean(z ** 2)) < 2.0
    # empty labels (N_l = 0) are never visited and carry no gradient, sampled or exact
    empty = br["N"] == 0
    assert np.all(acc["B"].sum(0)[empty] == 0) and np.all(gx[empty] == 0)


def test_sc_mrci_eigenpair(full):
    s, o, H = full
    br = o.brute(label_matrix=True)
    E, c = O.sc_mrci(br)
    # below the reference energy and below the sampling function's energy ...
    assert E <= o.e0 + 1e-12
    assert E <= br["psi_H_psi"] / br["psi_norm"] + 1e-12
    # ... and above full CI in the whole determinant space
    space = Q.full_space(s.n_orb, s.n_alpha, s.n_beta)
    idx = {d: i for i, d in enumerate(space)}
    Hf = np.zeros((len(space), len(space)))
    for d in space:
        for m, a in H.apply({d: 1.0}).items():
            Hf[idx[m], idx[d]] += a
    e_fci = np.linalg.eigvalsh(Hf)[0]
    assert E >= e_fci - 1e-10
    # a stationary point of the energy, whose value the brute-force scalar path reproduces
    g, E2 = O.exact_gradient(br, c)
    assert E2 == pytest.approx(E, rel=1e-12)
    assert np.abs(g).max() < 1e-9 * max(1.0, abs(E))
    b = O.Oracle.from_system(s, c=c).brute()
    assert b["psi_H_psi"] / b["psi_norm"] == pytest.approx(E, rel=1e-11)


def test_amsgrad_first_step_closed_form():
    rng = np.random.default_rng(0)
    c = rng.normal(size=7)
    g = rng.normal(size=7)
    lr, b1, b2, eps = 0.05, 0.9, 0.999, 1e-8
    c1 = O.amsgrad(c, g, O.amsgrad_state(7), lr, b1, b2, eps)
    step = lr * (1 - b1) * g[1:] / (np.sqrt(1 - b2) * np.abs(g[1:]) + eps)
    np.testing.assert_allclose(c1[1:], c[1:] - step, rtol=1e-14)
    assert c1[0] == c[0]


def test_amsgrad_minimises_a_convex_quadratic():
    rng = np.random.default_rng(1)
    n = 12
    a = rng.uniform(0.5, 4.0, n)
    xs = rng.normal(size=n)
    x = np.zeros(n)
    x[0] = xs[0]
    st = O.amsgrad_state(n)
    for it in range(4000):
        lr = 0.05 / np.sqrt(1 + it / 50)
        x = O.amsgrad(x, a * (x - xs), st, lr)
    assert np.abs(x - xs).max() < 1e-3
