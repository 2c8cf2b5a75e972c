"""The selected-CI reference built on the device (heat-bath selection of Sec. II D, Davidson, the
semicanonical rotation of Sec. II C) against independent definitions:

* with every string selected the product space is the whole CAS, and the device energy is the
  lowest eigenvalue of the oracle's Hamiltonian matrix over all CAS determinants;
* for a proper selection the device energy is the lowest eigenvalue of the oracle's Hamiltonian
  over the selected product space, and the loaded reference's E0 = <phi0|H|phi0> agrees;
* on the 78-orbital generator recipe the device selects the same strings as the host generator
  and reaches its energy and coefficients;
* the rotated integrals equal the host generator's semicanonical ones up to orbital signs, and
  the generalised Fock matrix is diagonal in the core and virtual blocks.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def _ctx(nc, na, nv, nel, h1, L, e_nuc=0.0):
    import paper_1909_06935_gb300 as P
    ctx = P.Context()
    ctx.load_hamiltonian(nc, na, nv, nel, nel, h1, S.pack_eri(L), e_nuc)
    return ctx


def _product_dets(strings, nc, n):
    W = (n + 63) // 64
    out = np.zeros((len(strings) ** 2, 2 * W), np.uint64)
    for a, sa in enumerate(strings):
        for b, sb in enumerate(strings):
            for sp, s in enumerate((int(sa), int(sb))):
                bits = ((1 << nc) - 1) | (s << nc)
                for w in range(W):
                    out[a * len(strings) + b, sp * W + w] = np.uint64((bits >> (64 * w)) & ((1 << 64) - 1))
    return out


def _dense_h(orc, dets):
    N = len(dets)
    Hm = np.zeros((N, N))
    for i in range(N):
        for j in range(i, N):
            Hm[i, j] = Hm[j, i] = orc.h(dets[i], dets[j])
    return Hm


def _oracle(nc, na, nv, nel, h1, L, dets, e_nuc=0.0):
    coeffs = np.ones(len(dets))
    return O.Oracle(nc, na, nv, nel, nel, h1, S.pack_eri(L), e_nuc, dets, coeffs,
                    np.full(S.n_labels(nc, nv), 0.1))


def test_every_string_selected_gives_the_cas_ci_energy():
    nc, na, nv, nel = 2, 6, 10, 5
    h1, L = S.make_integrals(nc, na, nv, 36, 5, chol_sigma=0.05)
    ctx = _ctx(nc, na, nv, nel, h1, L, e_nuc=0.7)
    try:
        r = ctx.sci_reference(20, n_seed_strings=6, tol=1e-10, max_iter=200, semicanonical=False)
    finally:
        ctx.close()
    assert r["n_strings"] == 20 and r["n_det"] == 400
    dets = _product_dets(r["strings"], nc, nc + na + nv)
    Hm = _dense_h(_oracle(nc, na, nv, nel, h1, L, dets, e_nuc=0.7), dets)
    w, U = np.linalg.eigh(Hm)
    assert abs(r["energy"] - w[0]) < 1e-9 * max(1.0, abs(w[0]))
    e_cas = S.casci(h1, L, nc, na, nel - nc, nel - nc, e_nuc=0.7)[0]
    assert abs(r["energy"] - e_cas) < 1e-9 * max(1.0, abs(e_cas))
    # the eigenvector, up to its sign convention (largest |c| positive)
    u = U[:, 0] * np.sign(U[np.argmax(np.abs(U[:, 0])), 0])
    assert np.allclose(r["coeffs"].ravel(), u, atol=1e-6)


def test_selected_space_energy_is_its_lowest_eigenvalue_and_the_loaded_e0():
    nc, na, nv, nel = 2, 8, 12, 6
    h1, L = S.make_integrals(nc, na, nv, 44, 17, chol_sigma=0.05)
    ctx = _ctx(nc, na, nv, nel, h1, L)
    try:
        r = ctx.sci_reference(24, n_seed_strings=8, tol=1e-10, max_iter=300, semicanonical=False)
        e0 = ctx.setup_info()["e0"]
    finally:
        ctx.close()
    assert r["n_det"] == 576 and len(set(r["strings"].tolist())) == 24
    dets = _product_dets(r["strings"], nc, nc + na + nv)
    w = np.linalg.eigvalsh(_dense_h(_oracle(nc, na, nv, nel, h1, L, dets), dets))
    assert abs(r["energy"] - w[0]) < 1e-9 * max(1.0, abs(w[0]))
    assert abs(e0 - w[0]) < 1e-9 * max(1.0, abs(w[0]))
    # a selection is variational: above the CAS-CI energy, below the seed space's
    e_cas = S.casci(h1, L, nc, na, nel - nc, nel - nc)[0]
    assert e_cas - 1e-10 <= r["energy"] <= r["seed_energy"] + 1e-12


def test_selection_matches_the_host_generator_on_the_78_orbital_recipe():
    nc, na, nv, nel = 2, 6, 70, 5
    h1, L = S.make_integrals(nc, na, nv, 24, 9, chol_sigma=0.05)
    e_h, C_h, sa_h, _, gamma_h = S.sci(h1, L, nc, na, nel - nc, 12, 8, tol=1e-10)
    ctx = _ctx(nc, na, nv, nel, h1, L)
    try:
        r = ctx.sci_reference(12, n_seed_strings=8, tol=1e-10, max_iter=300, semicanonical=False)
    finally:
        ctx.close()
    assert r["strings"].tolist() == sa_h.tolist()
    assert abs(r["energy"] - e_h) < 1e-9 * max(1.0, abs(e_h))
    assert np.allclose(r["coeffs"], C_h, atol=1e-6)


def test_semicanonical_rotation_matches_the_host_up_to_orbital_signs():
    nc, na, nv, nel = 3, 6, 9, 6
    h1, L = S.make_integrals(nc, na, nv, 36, 21, chol_sigma=0.05)
    e_h, C_h, sa_h, _, gamma_h = S.sci(h1, L, nc, na, nel - nc, 20, 20, tol=1e-11)
    h1_ref, L_ref = S.semicanonicalize(h1, L, nc, na, gamma_h)
    ctx = _ctx(nc, na, nv, nel, h1, L)
    try:
        r = ctx.sci_reference(20, n_seed_strings=20, tol=1e-11, max_iter=300, semicanonical=True)
        h1r, erir = ctx.read_hamiltonian()
        info = ctx.setup_info()
    finally:
        ctx.close()
    assert r["fock_offdiag"] > 1e-3                       # the input orbitals were not semicanonical
    assert np.allclose(np.abs(h1r), np.abs(h1_ref), atol=1e-9)
    assert np.allclose(np.abs(erir), np.abs(S.pack_eri(L_ref)), atol=1e-9)
    # F of the rotated integrals (with the reference's gamma) is diagonal in the core and virtual blocks
    n = nc + na + nv
    eri4 = S.unpack_eri(erir, n)
    c, a = slice(0, nc), slice(nc, nc + na)
    F = h1r + 2.0 * np.einsum("pqii->pq", eri4[:, :, c, c]) - np.einsum("piiq->pq", eri4[:, c, c, :])
    F += np.einsum("tu,pqtu->pq", info["gamma"], eri4[:, :, a, a]) - 0.5 * np.einsum("tu,ptuq->pq", info["gamma"],
                                                                                       eri4[:, a, a, :])
    for blk in (slice(0, nc), slice(nc + na, n)):
        B = F[blk, blk]
        assert np.max(np.abs(B - np.diag(np.diag(B)))) < 1e-9
        assert np.all(np.diff(np.diag(B)) >= 0)           # ascending, as the eigenvalues come
    assert np.allclose(info["eps"][: nc], np.diag(F)[:nc], atol=1e-10)
    assert np.allclose(info["gamma"], gamma_h, atol=1e-8)


def test_edge_cases_of_the_string_space():
    """A full active space (one string per spin, no opposite-spin lists), an empty one (no active
    electrons), a request for more strings than exist (clamped), and invalid requests."""
    import paper_1909_06935_gb300 as P
    h1, L = S.make_integrals(2, 3, 4, 18, 3, chol_sigma=0.05)
    for nel, nstr in ((5, 1), (2, 1), (3, 3)):
        ctx = _ctx(2, 3, 4, nel, h1, L)
        try:
            r = ctx.sci_reference(50, n_seed_strings=50, tol=1e-10, max_iter=100, semicanonical=True)
            e0 = ctx.setup_info()["e0"]
        finally:
            ctx.close()
        assert r["n_strings"] == nstr and r["n_det"] == nstr * nstr
        dets = _product_dets(r["strings"], 2, 9)
        w = np.linalg.eigvalsh(_dense_h(_oracle(2, 3, 4, nel, h1, L, dets), dets))
        assert abs(r["energy"] - w[0]) < 1e-9 * max(1.0, abs(w[0]))
        assert abs(e0 - w[0]) < 1e-8 * max(1.0, abs(w[0]))
    ctx = _ctx(2, 3, 4, 3, h1, L)
    try:
        for bad in (dict(n_strings=2, n_seed_strings=3), dict(n_strings=3, n_seed_strings=0),
                    dict(n_strings=3, n_seed_strings=1, tol=0.0), dict(n_strings=3, n_seed_strings=1, max_sub=1)):
            with pytest.raises(P.MRQError) as e:
                ctx.sci_reference(**bad)
            assert e.value.code == -1
    finally:
        ctx.close()
    ctx = P.Context()
    try:
        ctx.load_hamiltonian(2, 3, 4, 3, 2, h1, S.pack_eri(L))      # open shell: Sz != 0
        with pytest.raises(P.MRQError) as e:
            ctx.sci_reference(3, n_seed_strings=1)
        assert e.value.code == -1
    finally:
        ctx.close()
