"""Pins of the CPU oracle against things other than itself (no GPU).

* an independent second-quantised operator applier (tests/secondq.py) on whole determinant
  spaces of tiny systems: matrix elements, neighbour sets, reach-back overlaps <m|H|phi0>
  (Eq. 6-7), perturber norms and H_D energies (Eq. 2, 14), local energies (Eq. 5);
* the generator's own string-driven CAS-CI solver (E0, 1-RDM);
* closed forms and invariants: zero variance for an exact eigenvector, the MP2 limit of
  SC-NEVPT2 with an empty active space, size consistency (Table 4), Philox known answers.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from tests import secondq as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def tiny(n_core, n_act, n_virt, n_alpha, n_beta, seed, rank=12, chol_sigma=0.12, c_seed=None):
    return S.make_system(n_core, n_act, n_virt, n_alpha, n_beta, rank=rank, seed=seed, chol_sigma=chol_sigma,
                         c_seed=c_seed)


def eri4_of(s):
    L = s.meta["L"]
    return np.einsum("kpq,krs->pqrs", L, L)


def label_of(det, s):
    """Label of a tuple determinant, ranked independently of the oracle."""
    n, nc, na, nv = s.n_orb, s.n_core, s.n_act, s.n_virt
    hs = [sg * nc + i for sg in range(2) for i in range(nc) if sg * n + i not in det]
    ps = [sg * nv + a for sg in range(2) for a in range(nv) if sg * n + nc + na + a in det]
    if len(hs) > 2 or len(ps) > 2:
        return -1

    def rank(x, m):
        if not x:
            return 0
        if len(x) == 1:
            return 1 + x[0]
        return 1 + m + x[1] * (x[1] - 1) // 2 + x[0]

    nps = 1 + 2 * nv + (2 * nv) * (2 * nv - 1) // 2
    return rank(hs, 2 * nc) * nps + rank(ps, 2 * nv)


def phi0_dict(s):
    return {Q.from_words(d, s.n_orb): c for d, c in zip(s.dets, s.coeffs)}


SYSTEMS = {
    "1c2a2v": dict(n_core=1, n_act=2, n_virt=2, n_alpha=2, n_beta=2, seed=31),
    "1c3a2v_open": dict(n_core=1, n_act=3, n_virt=2, n_alpha=3, n_beta=2, seed=32),
    "2c2a1v": dict(n_core=2, n_act=2, n_virt=1, n_alpha=3, n_beta=3, seed=33),
}


@pytest.fixture(scope="module", params=list(SYSTEMS))
def full(request):
    s = tiny(**SYSTEMS[request.param])
    o = O.Oracle.from_system(s)
    eri4 = eri4_of(s)
    H = Q.Hamiltonian(s.h1, eri4, s.e_nuc)
    space = Q.full_space(s.n_orb, s.n_alpha, s.n_beta)
    return s, o, eri4, H, space


# ------------------------------------------------------------------ golden / setup

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert list(O.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


@pytest.mark.parametrize("name", ["tiny_12o_cas4"])
def test_e0_and_rdm_match_generator_casci(name):
    s = S.workload(name)
    o = O.Oracle.from_system(s)
    assert abs(o.e0 - s.e_cas) < 1e-10 * max(1.0, abs(s.e_cas))
    np.testing.assert_allclose(o.gamma, s.meta["gamma"], atol=1e-11)
    assert abs(np.trace(o.gamma) - (s.n_alpha + s.n_beta - 2 * s.n_core)) < 1e-10


def test_setup_matches_definitions(full):
    s, o, eri4, H, space = full
    eps, heff, e_core, F = Q.dyall_inputs(s.h1, eri4, s.n_core, s.n_act, s.meta["gamma"], s.e_nuc)
    np.testing.assert_allclose(o.eps, eps, atol=1e-11)
    np.testing.assert_allclose(o.heff[:s.n_act, :s.n_act], heff, atol=1e-11)
    assert abs(o.e_core - e_core) < 1e-11
    # semicanonical inputs: core-core and virtual-virtual Fock blocks are diagonal
    nc, na = s.n_core, s.n_act
    Fc, Fv = F[:nc, :nc], F[nc + na:, nc + na:]
    assert np.abs(Fc - np.diag(np.diag(Fc))).max() < 1e-10
    assert np.abs(Fv - np.diag(np.diag(Fv))).max() < 1e-10


# ------------------------------------------------------------------ whole-space pins

def test_matrix_elements_vs_operator_algebra(full):
    s, o, eri4, H, space = full
    n = s.n_orb
    for det in space:
        hv = H.apply({det: 1.0})
        x = Q.to_words(det, n)
        for m in space:
            deg = len(set(det) - set(m))
            if deg > 2:
                continue
            ref = hv.get(m, 0.0)
            got = o.h(x, Q.to_words(m, n))
            assert abs(got - ref) < 1e-12, (det, m, got, ref)


def test_neighbour_sets_brute_force(full):
    s, o, eri4, H, space = full
    n = s.n_orb
    for det in space:
        if label_of(det, s) < 0:
            continue
        r = o.local(Q.to_words(det, n), max_nb=4096)
        got = sorted(Q.from_words(x, n) for x in r["dets"])
        want = sorted(m for m in space if m != det and len(set(det) - set(m)) <= 2 and label_of(m, s) >= 0)
        assert got == want
        assert r["label"] == label_of(det, s)


def test_neighbour_list_entries_reproduce_local(full):
    """The list-only enumeration and the per-neighbour evaluation of a given list (used for the
    large-system parity checks) give exactly what local() gives: same ids in the same order, the
    same values bit for bit (the same arithmetic)."""
    s, o, eri4, H, space = full
    n = s.n_orb
    dets = [d for d in space if label_of(d, s) >= 0][:12]
    for det in dets:
        x = Q.to_words(det, n)
        r = o.local(x, max_nb=4096)
        ids = o.neighbour_ids(x)
        assert np.array_equal(ids, r["exc"])
        got = o.neighbours(x, ids[::-1])
        for k in ("dets", "H", "HD", "O", "psi_m", "Gamma"):
            assert np.array_equal(got[k], r[k][::-1]), k
    with pytest.raises(ValueError):
        o.neighbours(Q.to_words(dets[0], n), np.array([0], np.uint32) | np.uint32(1 << 16))


def test_reach_back_overlap_is_H_phi0(full):
    s, o, eri4, H, space = full
    n = s.n_orb
    phi = phi0_dict(s)
    v = H.apply(phi)
    for m in space:
        l = label_of(m, s)
        if l < 0:
            continue
        ps, ov = o.psi(Q.to_words(m, n))
        if l == 0:
            assert ov == pytest.approx(phi.get(m, 0.0), abs=1e-14)
            assert ps == pytest.approx(s.c[0] * phi.get(m, 0.0), abs=1e-14)
        else:
            assert abs(ov - v.get(m, 0.0)) < 1e-12
            assert abs(ps - s.c[l] * v.get(m, 0.0)) < 1e-12


def _sc_vectors(s, H):
    phi = phi0_dict(s)
    v = H.apply(phi)
    buckets = {}
    for m, amp in v.items():
        l = label_of(m, s)
        if l > 0:
            buckets.setdefault(l, {})[m] = amp
    return phi, buckets


def test_brute_force_sc_quantities_vs_operator_algebra(full):
    s, o, eri4, H, space = full
    eps, heff, e_core, _ = Q.dyall_inputs(s.h1, eri4, s.n_core, s.n_act, s.meta["gamma"], s.e_nuc)
    HD = Q.DyallHamiltonian(s.n_core, s.n_act, s.n_virt, eps, heff, eri4, e_core)
    phi, buckets = _sc_vectors(s, H)
    br = o.brute()
    nz = np.nonzero(br["N"][1:])[0] + 1
    assert set(nz) == {l for l, b in buckets.items() if sum(a * a for a in b.values()) > 0}
    for l, vl in buckets.items():
        Nl = sum(a * a for a in vl.values())
        hv = HD.apply(vl)
        Dl = sum(a * hv.get(m, 0.0) for m, a in vl.items())
        assert abs(br["N"][l] - Nl) < 1e-12 * max(1, Nl)
        assert abs(br["D"][l] - Dl) < 1e-11 * max(1, abs(Dl))
        # H_D keeps the label: the orthogonal SC states stay orthogonal under H_D (Sec. II A)
        assert all(label_of(m, s) == l for m, a in hv.items() if abs(a) > 0)
    # sampling function psi_s = c0 phi0 + sum_l c_l v_l (Eq. 17)
    psi = {m: s.c[0] * a for m, a in phi.items()}
    for l, vl in buckets.items():
        for m, a in vl.items():
            psi[m] = psi.get(m, 0.0) + s.c[l] * a
    hp = H.apply(psi)
    assert br["psi_norm"] == pytest.approx(sum(a * a for a in psi.values()), rel=1e-12)
    assert br["psi_H_psi"] == pytest.approx(sum(a * hp.get(m, 0.0) for m, a in psi.items()), rel=1e-11)


def test_local_quantities_vs_operator_algebra(full):
    s, o, eri4, H, space = full
    n = s.n_orb
    eps, heff, e_core, _ = Q.dyall_inputs(s.h1, eri4, s.n_core, s.n_act, s.meta["gamma"], s.e_nuc)
    HD = Q.DyallHamiltonian(s.n_core, s.n_act, s.n_virt, eps, heff, eri4, e_core)
    phi, buckets = _sc_vectors(s, H)
    psi = {m: s.c[0] * a for m, a in phi.items()}
    for l, vl in buckets.items():
        for m, a in vl.items():
            psi[m] = psi.get(m, 0.0) + s.c[l] * a
    hp = H.apply(psi)
    checked = 0
    for det, amp in psi.items():
        if abs(amp) < 1e-8:
            continue
        r = o.local(Q.to_words(det, n), max_nb=4096)
        assert r["psi"] == pytest.approx(amp, rel=1e-12)
        assert r["EL"] == pytest.approx(hp.get(det, 0.0) / amp, rel=1e-10, abs=1e-10)
        hrow = H.apply({det: 1.0})
        S_ref = sum(abs(hrow.get(m, 0.0) * psi.get(m, 0.0) / amp) for m in psi if m != det)
        assert r["S"] == pytest.approx(S_ref, rel=1e-10)
        l = label_of(det, s)
        if l > 0:
            hv = HD.apply(buckets[l])
            assert r["num"] == pytest.approx(hv[det] / buckets[l][det], rel=1e-10, abs=1e-10)
        else:
            assert r["HDnn"] == pytest.approx(r["Hnn"], rel=1e-13)
        checked += 1
    assert checked > 20


# ------------------------------------------------------------------ closed forms and invariants

def test_zero_variance_exact_eigenvector():
    """Whole space = CAS (no core, no virtuals): psi_s = c0 phi0 is an exact eigenvector, so the
    local energy (Eq. 5) equals the eigenvalue at every determinant."""
    s = tiny(0, 6, 0, 3, 3, seed=41, rank=16, chol_sigma=0.15)
    o = O.Oracle.from_system(s)
    assert abs(o.e0 - s.e_cas) < 1e-10
    big = np.abs(s.coeffs) > 1e-4
    assert big.sum() > 50
    for d in s.dets[big]:
        r = o.local(d)
        assert abs(r["EL"] - o.e0) < 1e-9


def test_mp2_limit_empty_active_space():
    """n_act = 0 and a single-determinant reference: every SC perturber is one determinant and
    SC-NEVPT2 (Eq. 15) reduces to closed-shell MP2 with non-Brillouin singles."""
    s = tiny(3, 0, 5, 3, 3, seed=43, rank=20, chol_sigma=0.1)
    o = O.Oracle.from_system(s)
    eri4 = eri4_of(s)
    eps, _, e_core, F = Q.dyall_inputs(s.h1, eri4, 3, 0, np.zeros((0, 0)), s.e_nuc)
    nc = 3
    ei, ea = eps[:nc], eps[nc:]
    ovov = eri4[:nc, nc:, :nc, nc:]                             # (ia|jb)
    den = ei[:, None, None, None] - ea[None, :, None, None] + ei[None, None, :, None] - ea[None, None, None, :]
    e_d = np.sum(ovov * (2 * ovov - ovov.transpose(0, 3, 2, 1)) / den)
    e_s = 2.0 * np.sum(F[:nc, nc:] ** 2 / (ei[:, None] - ea[None, :]))
    br = o.brute()
    ex = O.exact_from_brute(br, o.e0, o.c, 3, 5)
    assert abs(o.e0 - e_core) < 1e-12
    assert ex["e2"] == pytest.approx(e_d + e_s, rel=1e-11)
    assert abs(e_s) > 1e-6            # the singles really contribute


def _embed(sa, sb):
    """Two non-interacting fragments in one orbital space ordered core|active|virtual."""
    nca, naa, nva = sa.n_core, sa.n_act, sa.n_virt
    ncb, nab, nvb = sb.n_core, sb.n_act, sb.n_virt
    nc, na, nv = nca + ncb, naa + nab, nva + nvb
    n = nc + na + nv
    mapA = list(range(nca)) + [nc + t for t in range(naa)] + [nc + na + a for a in range(nva)]
    mapB = [nca + i for i in range(ncb)] + [nc + naa + t for t in range(nab)] + [nc + na + nva + a for a in range(nvb)]
    h1 = np.zeros((n, n))
    h1[np.ix_(mapA, mapA)] = sa.h1
    h1[np.ix_(mapB, mapB)] = sb.h1
    LA, LB = sa.meta["L"], sb.meta["L"]
    L = np.zeros((LA.shape[0] + LB.shape[0], n, n))
    for k in range(LA.shape[0]):
        L[k][np.ix_(mapA, mapA)] = LA[k]
    for k in range(LB.shape[0]):
        L[LA.shape[0] + k][np.ix_(mapB, mapB)] = LB[k]
    return h1, L, (nc, na, nv)


def test_size_consistency_noninteracting_fragments():
    """SC-NEVPT2 is exactly size consistent (Table 4): E2(A+B) = E2(A) + E2(B)."""
    sa = tiny(1, 2, 2, 2, 2, seed=51)
    sb = tiny(1, 2, 3, 2, 2, seed=52)
    h1, L, (nc, na, nv) = _embed(sa, sb)
    e, Cm, s_a, s_b, gamma = S.casci(h1, L, nc, na, 2, 2)
    assert abs(e - (sa.e_cas + sb.e_cas)) < 1e-10
    dets, coeffs = S._to_dets(Cm, s_a, s_b, nc, nc + na + nv)
    c = S.psi_s_coeffs(S.n_labels(nc, nv), 5)
    o = O.Oracle(nc, na, nv, sa.n_alpha + sb.n_alpha, sa.n_beta + sb.n_beta, h1, S.pack_eri(L), 0.0,
                 dets, coeffs, c)
    res = {}
    for key, sys_ in (("A", sa), ("B", sb)):
        oo = O.Oracle.from_system(sys_)
        res[key] = O.exact_from_brute(oo.brute(), oo.e0, oo.c, sys_.n_core, sys_.n_virt)["e2"]
    e2ab = O.exact_from_brute(o.brute(), o.e0, c, nc, nv)["e2"]
    assert abs(e2ab - (res["A"] + res["B"])) < 1e-11
    assert abs(res["A"]) > 1e-5 and abs(res["B"]) > 1e-5


def test_hermiticity_on_workload():
    s = S.workload("tiny_12o_cas4")
    o = O.Oracle.from_system(s)
    d = s.dets[o.start]
    r = o.local(d, max_nb=4096)
    rng = np.random.default_rng(0)
    for k in rng.choice(len(r["dets"]), 200, replace=False):
        m = r["dets"][k]
        assert o.h(d, m) == pytest.approx(o.h(m, d), rel=1e-14, abs=1e-15)
        rm = o.local(m, max_nb=4096)
        j = [i for i, x in enumerate(rm["dets"]) if np.array_equal(x, d)]
        assert len(j) == 1 and rm["H"][j[0]] == pytest.approx(r["H"][k], rel=1e-13, abs=1e-15)


# ------------------------------------------------------------------ the walk

def test_race_picks_moves_with_probability_gamma_over_S():
    """First-reaction form of the rejection-free walk: P(move to m) = Gamma_m / S."""
    s = tiny(1, 2, 2, 2, 2, seed=31)
    o = O.Oracle.from_system(s)
    d = s.dets[o.start]
    r = o.local(d, max_nb=4096)
    p = r["Gamma"] / r["S"]
    idx = {int(e): i for i, e in enumerate(r["exc"])}
    counts = np.zeros(len(p))
    K = 20000
    for step in range(K):
        _, exc, _ = o.move(d, seed=99, step=step, walker=3)
        counts[idx[exc]] += 1
    big = p * K > 20
    chi2 = np.sum((counts[big] - K * p[big]) ** 2 / (K * p[big]))
    dof = big.sum() - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)


def test_walk_matches_exact_expectations():
    """Time-weighted averages (Eq. 4, 16) against brute-force expectations under |psi_s|^2."""
    s = tiny(1, 2, 2, 2, 2, seed=31)
    o = O.Oracle.from_system(s)
    br = o.brute()
    ex = O.exact_from_brute(br, o.e0, o.c, 1, 2)
    acc = o.sample(64, 2000, 100, seed=7, n_groups=16)
    f = o.finalize(acc)
    assert abs(f["e_var"] - ex["e_var"]) < 4 * f["e_var_sigma"] + 1e-12
    assert abs(f["a0sq"] - ex["a0sq"]) < 4 * f["a0sq_sigma"]
    assert abs(f["e2"] - ex["e2"]) < 4 * f["e2_sigma"]
    # per-label residence against rho_l = c_l^2 N_l / <psi_s|psi_s>
    W = acc["W"].sum()
    occ = acc["N"].sum(0) * o.c ** 2 / W
    big = ex["rho_label"] > 1e-3
    np.testing.assert_allclose(occ[big], ex["rho_label"][big], rtol=0.15)


def test_frozen_core_variant_is_the_core_free_part_of_the_sum():
    """Zero coefficients on core-hole labels (the paper's frozen-core implementation): the walk never
    visits a core-excited class, and E^(2) is the brute-force sum over the core-free labels, which
    equals the brute force restricted to those labels (N_l and E_l do not depend on c)."""
    import paper_1909_06935_gb300 as P
    s = tiny(1, 2, 2, 2, 2, seed=31)
    types = O.label_types(1, 2)
    cf = np.where(types >= 3, 0.0, s.c)
    assert np.array_equal(P.frozen_core_coeffs(s.c, 1, 2), cf)     # the binding's helper (plain numpy)
    o = O.Oracle.from_system(s)
    of = O.Oracle.from_system(s, c=cf)
    full = O.exact_from_brute(o.brute(), o.e0, o.c, 1, 2)
    e2_frozen = full["type_e2"][:3].sum()          # types 3h + p with h = 0
    acc = of.sample(64, 1500, 100, seed=5, n_groups=16)
    assert np.all(acc["type_steps"][3:] == 0)
    f = of.finalize(acc)
    assert np.all(f["type_e2"][3:] == 0)
    assert abs(f["e2"] - e2_frozen) < 4 * f["e2_sigma"]
    assert abs(f["e2"] - full["e2"]) > 4 * f["e2_sigma"]          # core correlation is not small here


def test_e2_does_not_depend_on_the_sampling_coefficients():
    """The sampling coefficients c_l only shape |psi_s|^2 (Eq. 17): N_l, E_l and E^(2) are the same
    for any choice, and walks with two different c vectors agree with that one value."""
    base = tiny(1, 2, 2, 2, 2, seed=31, c_seed=101)
    other = tiny(1, 2, 2, 2, 2, seed=31, c_seed=202)
    assert not np.allclose(base.c, other.c)
    oa, ob = O.Oracle.from_system(base), O.Oracle.from_system(other)
    ba, bb = oa.brute(), ob.brute()
    np.testing.assert_allclose(ba["N"], bb["N"], rtol=1e-12)
    np.testing.assert_allclose(ba["D"], bb["D"], rtol=1e-12, atol=1e-14)
    e2 = O.exact_from_brute(ba, oa.e0, oa.c, 1, 2)["e2"]
    for o in (oa, ob):
        f = o.finalize(o.sample(64, 1500, 100, seed=9, n_groups=16))
        assert abs(f["e2"] - e2) < 4 * f["e2_sigma"]
