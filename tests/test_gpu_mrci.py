"""SC-MRCI(s) optimisation on the device (Sec. II B, Eq. 8-9) against the oracle.

Bar: the per-group gradient sums and the gradient within 1e-10 relative of the oracle's on the
same (bit-identical) trajectories; AMSGrad updates within 1e-12 of the oracle's update of the
same gradient; and an optimisation run that takes the exact energy of its coefficients most of
the way down to the SC-MRCI eigenvalue of the oracle's label Hamiltonian.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def close(a, b, rtol=1e-10, atol=1e-14):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= atol + rtol * np.maximum(np.abs(a), np.abs(b)))


@pytest.fixture(scope="module")
def tiny():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    return s, P.Context.from_system(s)


def test_gradient_sums_and_gradient_match_oracle(tiny):
    s, ctx = tiny
    ctx.set_coeffs(s.c)
    orc = O.Oracle.from_system(s)
    nw, ns, burn, G, seed = 96, 60, 10, 8, 4242
    acc = orc.sample(nw, ns, burn, seed, G)
    ctx.sample(ctx.params(nw, ns, burn_in=burn, seed=seed, n_groups=G))
    A, B = ctx.gradient_sums(G)
    assert close(A, acc["A"]) and close(B, acc["B"])
    g, E = ctx.mrci_gradient()
    go, Eo = O.mrci_gradient(acc)
    assert close(E, Eo, 1e-12)
    scale = np.abs(acc["A"]).sum(0) / acc["W"].sum()       # size of the sums g is a difference of
    assert np.all(np.abs(g - go) <= 1e-10 * (scale + np.abs(go)) + 1e-15)


def test_amsgrad_steps_match_oracle(tiny):
    """Two walk-gradient-update iterations; the second walks with the updated coefficients and
    uses the moment estimates of the first."""
    s, ctx = tiny
    ctx.set_coeffs(s.c)
    c = s.c.copy()
    st = O.amsgrad_state(len(c))
    nw, ns, burn, G = 64, 40, 5, 4
    for it, lr in enumerate((0.02, 0.01)):
        acc = O.Oracle.from_system(s, c=c).sample(nw, ns, burn, 77 + it, G)
        ctx.sample(ctx.params(nw, ns, burn_in=burn, seed=77 + it, n_groups=G))
        g, _ = ctx.mrci_gradient()
        go, _ = O.mrci_gradient(acc)
        scale = np.abs(acc["A"]).sum(0) / acc["W"].sum()
        assert np.all(np.abs(g - go) <= 1e-10 * (scale + np.abs(go)) + 1e-15), it
        ctx.amsgrad_step(lr)
        c = O.amsgrad(c, g, st, lr)                          # the oracle's update of the same g
        cg = ctx.coeffs()
        assert close(cg, c, 1e-12), it
        assert cg[0] == s.c[0]
    # set_coeffs starts a new optimisation: zero moments again
    ctx.set_coeffs(s.c)
    ctx.sample(ctx.params(nw, ns, burn_in=burn, seed=77, n_groups=G))
    g, _ = ctx.mrci_gradient()
    ctx.amsgrad_step(0.02)
    assert close(ctx.coeffs(), O.amsgrad(s.c, g, O.amsgrad_state(len(c)), 0.02), 1e-12)


def test_amsgrad_rejects_bad_arguments(tiny):
    import paper_1909_06935_gb300 as P
    s, ctx = tiny
    ctx.set_coeffs(s.c)
    ctx.sample(ctx.params(32, 10, burn_in=0, seed=1, n_groups=2))
    ctx.mrci_gradient()
    for kw in (dict(lr=0.0), dict(lr=0.01, beta1=1.0), dict(lr=0.01, beta2=-0.1), dict(lr=0.01, eps=0.0)):
        with pytest.raises(P.MRQError) as e:
            ctx.amsgrad_step(**kw)
        assert e.value.code == -1
    ctx.set_coeffs(s.c)


def test_optimisation_approaches_the_sc_mrci_eigenvalue(tiny):
    s, ctx = tiny
    orc = O.Oracle.from_system(s)
    br = orc.brute(label_matrix=True)
    e_mrci, _ = O.sc_mrci(br)
    _, e_start = O.exact_gradient(br, s.c)
    ctx.set_coeffs(s.c)
    hist = ctx.optimize_mrci(40, 2048, 200, burn_in=20, lr=0.01, seed=500, n_groups=16)
    c = ctx.coeffs()
    _, e_end = O.exact_gradient(br, c)
    assert e_end >= e_mrci - 1e-12                              # variational
    assert e_end - e_mrci < 0.1 * (e_start - e_mrci)
    assert len(hist) == 40 and hist[-1]["e_var"] < hist[0]["e_var"]
    # a walk with the optimised coefficients estimates their exact energy
    res = ctx.sample(ctx.params(4096, 400, burn_in=50, seed=9001, n_groups=32))
    assert abs(res["e_var"] - e_end) < 4 * res["e_var_sigma"]
    ctx.set_coeffs(s.c)
