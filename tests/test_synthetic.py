"""The input generator's selected-CI reference (the 104-orbital workload's recipe) against its exact
CAS-CI solver: the full string space reproduces CAS-CI, a selection is variational, and the
product-space determinants are well formed."""
import numpy as np

import synthetic as S


def test_selected_ci_with_every_string_is_cas_ci():
    h1, L = S.make_integrals(2, 6, 4, 36, 5, chol_sigma=0.05)
    e_sci, C, sa, sb, g = S.sci(h1, L, 2, 6, 3, n_strings=20, n_seed_strings=20, tol=1e-9)
    e_cas, Cc, *_ = S.casci(h1, L, 2, 6, 3, 3)
    assert abs(e_sci - e_cas) < 1e-8 * max(1.0, abs(e_cas))
    assert abs(np.trace(g) - 6.0) < 1e-10


def test_selected_ci_is_variational():
    h1, L = S.make_integrals(2, 6, 4, 36, 5, chol_sigma=0.05)
    e_cas, *_ = S.casci(h1, L, 2, 6, 3, 3)
    e_small, C, sa, sb, g = S.sci(h1, L, 2, 6, 3, n_strings=10, n_seed_strings=6, tol=1e-9)
    assert e_small >= e_cas - 1e-10
    assert C.shape == (10, 10) and len(sa) == 10


def test_selected_ci_system_layout():
    s = S.make_sci_system(2, 6, 70, 5, 5, rank=24, seed=9, n_strings=12, n_seed_strings=8, chol_sigma=0.05)
    assert s.W == 2 and len(s.coeffs) == 144
    assert len(np.unique(s.dets, axis=0)) == 144
    core = np.uint64(0b11)
    for sg in range(2):
        w0 = s.dets[:, sg * s.W]
        assert np.all(w0 & core == core)                            # full core
        assert np.all(s.dets[:, sg * s.W + 1] == 0)                 # empty virtuals in the second word
        assert np.all([bin(int(x)).count("1") == 5 for x in w0])    # 5 electrons per spin
