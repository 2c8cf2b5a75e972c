"""Pins of the oracle's heat-bath cutoff (Sec. II D: excitations are generated by the heat-bath
algorithm; with a positive cutoff eps a double excitation whose element |<ab||ij>| is below eps is
not generated).  The screened oracle is checked against the independent second-quantised
operator applier (tests/secondq.py) whose H and H_D rows are screened here, element by element:
double-excitation elements below eps are dropped, singles and diagonals kept.  The cutoff sits in
the middle of a gap between two consecutive element magnitudes, so rounding cannot move an
element across it."""
import numpy as np
import pytest

import oracle as O
from tests import secondq as Q
from tests.test_oracle import SYSTEMS, eri4_of, label_of, phi0_dict, tiny


class Screened:
    """An operator's rows with the double-excitation elements below eps dropped."""

    def __init__(self, op, eps):
        self.op, self.eps = op, eps
        self.dropped = 0

    def apply(self, vec):
        out = {}
        for det, amp in vec.items():
            for d2, h in self.op.apply({det: 1.0}).items():
                if d2 != det and len(set(det) - set(d2)) == 2 and abs(h) < self.eps:
                    self.dropped += 1
                    continue
                out[d2] = out.get(d2, 0.0) + h * amp
        return out


def _double_magnitudes(H, space):
    mags = set()
    for det in space:
        for d2, h in H.apply({det: 1.0}).items():
            if d2 != det and len(set(det) - set(d2)) == 2 and abs(h) > 1e-14:
                mags.add(abs(h))
    return np.array(sorted(mags))


def _cutoff(mags, q=0.5):
    """eps in the middle of the widest gap between consecutive magnitudes near quantile q."""
    i0 = int(q * (len(mags) - 1))
    lo, hi = max(0, i0 - 5), min(len(mags) - 1, i0 + 5)
    k = max(range(lo, hi), key=lambda i: mags[i + 1] - mags[i])
    assert mags[k + 1] - mags[k] > 1e-9 * mags[k + 1]
    return 0.5 * (mags[k] + mags[k + 1])


@pytest.fixture(scope="module", params=list(SYSTEMS))
def screened(request):
    s = tiny(**SYSTEMS[request.param])
    o = O.Oracle.from_system(s)
    eri4 = eri4_of(s)
    H = Q.Hamiltonian(s.h1, eri4, s.e_nuc)
    space = Q.full_space(s.n_orb, s.n_alpha, s.n_beta)
    eps = _cutoff(_double_magnitudes(H, space))
    o.set_hb_eps(eps)
    Hs = Screened(H, eps)
    e, heff, e_core, _ = Q.dyall_inputs(s.h1, eri4, s.n_core, s.n_act, s.meta["gamma"], s.e_nuc)
    HDs = Screened(Q.DyallHamiltonian(s.n_core, s.n_act, s.n_virt, e, heff, eri4, e_core), eps)
    return s, o, Hs, HDs, space, eps


def _buckets(s, Hs):
    phi = phi0_dict(s)
    v = Hs.apply(phi)
    out = {}
    for m, amp in v.items():
        l = label_of(m, s)
        if l > 0:
            out.setdefault(l, {})[m] = amp
    return phi, out


def test_screened_brute_force_vs_operator_algebra(screened):
    s, o, Hs, HDs, space, eps = screened
    phi, buckets = _buckets(s, Hs)
    assert Hs.dropped > 0                                 # the cutoff removes elements
    br = o.brute()
    for l, vl in buckets.items():
        Nl = sum(a * a for a in vl.values())
        hv = HDs.apply(vl)
        Dl = sum(a * hv.get(m, 0.0) for m, a in vl.items())
        assert abs(br["N"][l] - Nl) < 1e-12 * max(1, Nl)
        assert abs(br["D"][l] - Dl) < 1e-11 * max(1, abs(Dl))
    assert {int(x) for x in np.nonzero(br["N"][1:])[0] + 1} == {l for l, b in buckets.items()
                                                               if sum(a * a for a in b.values()) > 0}
    # and the cutoff changes the answer: the exact method's norms differ
    o0 = O.Oracle.from_system(s)
    assert not np.allclose(o0.brute()["N"], br["N"], rtol=1e-6, atol=1e-14)
    assert o0.e0 == o.e0                                  # E0 stays exact


def test_screened_local_quantities_vs_operator_algebra(screened):
    s, o, Hs, HDs, space, eps = screened
    n = s.n_orb
    phi, buckets = _buckets(s, Hs)
    psi = {m: s.c[0] * a for m, a in phi.items()}
    for l, vl in buckets.items():
        for m, a in vl.items():
            psi[m] = psi.get(m, 0.0) + s.c[l] * a
    hp = Hs.apply(psi)
    checked = 0
    for det, amp in psi.items():
        if abs(amp) < 1e-8:
            continue
        r = o.local(Q.to_words(det, n), max_nb=4096)
        assert r["psi"] == pytest.approx(amp, rel=1e-12)
        assert r["EL"] == pytest.approx(hp.get(det, 0.0) / amp, rel=1e-10, abs=1e-10)
        hrow = Hs.apply({det: 1.0})
        S_ref = sum(abs(hrow.get(m, 0.0) * psi.get(m, 0.0) / amp) for m in psi if m != det)
        assert r["S"] == pytest.approx(S_ref, rel=1e-10)
        l = label_of(det, s)
        if l > 0:
            hv = HDs.apply(buckets[l])
            assert r["num"] == pytest.approx(hv[det] / buckets[l][det], rel=1e-10, abs=1e-10)
        checked += 1
    assert checked > 10


def test_cutoff_zero_is_the_exact_method():
    s = tiny(**SYSTEMS["1c2a2v"])
    o, ref = O.Oracle.from_system(s), O.Oracle.from_system(s)
    o.set_hb_eps(0.05)
    o.set_hb_eps(0.0)
    a, b = o.brute(), ref.brute()
    assert np.array_equal(a["N"], b["N"]) and np.array_equal(a["D"], b["D"])
