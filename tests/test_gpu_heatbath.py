"""The heat-bath cutoff (mrq_set_heat_bath_cutoff; Sec. II D) against the oracle with the same
cutoff: local quantities element by element (the screened double excitations carry zero
elements, their O(m) lose the screened terms), bit-exact trajectories, accumulators within
1e-10, and the stochastic E^(2) within 3 sigma of the screened brute force.  A cutoff of zero
gives back the exact method bit for bit; the CAS path (physicists' tables) and the FOIS path
(integrals) are both exercised on the 56-orbital workload's start determinant."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from tests.test_gpu_parity import close, compare_local

pytestmark = pytest.mark.gpu

EPS = 0.004


@pytest.fixture(scope="module")
def pair():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    ctx.set_heat_bath_cutoff(EPS)
    orc.set_hb_eps(EPS)
    yield s, ctx, orc
    ctx.close()


def test_local_parity_with_cutoff(pair):
    s, ctx, orc = pair
    start = s.dets[orc.start]
    r = orc.local(start, max_nb=4096)
    rng = np.random.default_rng(7)
    pick = rng.choice(r["nnb"], 24, replace=False)
    dets = np.vstack([start[None], s.dets[:8], r["dets"][pick]])
    r2 = orc.local(r["dets"][pick[0]], max_nb=8192)
    dets = np.vstack([dets, r2["dets"][rng.choice(r2["nnb"], 24, replace=False)]])
    compare_local(ctx, orc, dets, s.W)
    # the cutoff acts: some neighbours of the start determinant carry a zero element now
    exact = O.Oracle.from_system(s).local(start, max_nb=4096)
    assert np.sum((r["H"] == 0.0) & (exact["H"] != 0.0)) > 0


def test_walk_with_cutoff_matches_oracle(pair):
    s, ctx, orc = pair
    nw, ns, burn, G, seed = 96, 60, 10, 8, 77
    acc_o = orc.sample(nw, ns, burn, seed, G, trajectory=True)
    ctx.sample(ctx.params(nw, ns, burn_in=burn, seed=seed, n_groups=G))
    dets, _ = ctx.walkers(nw)
    assert np.array_equal(dets, acc_o["trajectory"][:, -1, :])
    acc_g = ctx.accumulators(G)
    for k in ("N", "U", "W", "E"):
        assert close(acc_g[k], acc_o[k], 1e-10, 1e-14), k


def test_stochastic_energy_with_cutoff_within_3_sigma_of_its_brute_force(pair):
    s, ctx, orc = pair
    ex = O.exact_from_brute(orc.brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    exact = O.exact_from_brute(O.Oracle.from_system(s).brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    res = ctx.sample(ctx.params(2048, 1600, burn_in=100, seed=78, n_groups=32))
    assert res["e2_sigma"] <= 1e-4
    assert abs(res["e2"] - ex["e2"]) < 3 * res["e2_sigma"]
    assert abs(ex["e2"] - exact["e2"]) > 1e-7                  # the cutoff changes the answer


def test_zero_cutoff_restores_the_exact_walk():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    a, b = P.Context.from_system(s), P.Context.from_system(s)
    try:
        a.set_heat_bath_cutoff(0.05)
        a.set_heat_bath_cutoff(0.0)
        for c in (a, b):
            c.sample(c.params(128, 40, burn_in=5, seed=5, n_groups=4))
        assert np.array_equal(a.walkers(128)[0], b.walkers(128)[0])
        assert np.array_equal(a.accumulators(4)["N"], b.accumulators(4)["N"])
    finally:
        a.close()
        b.close()


def test_cutoff_on_the_56_orbital_start_determinant():
    """The CAS path's table screening and the FOIS path's integral screening at full size: all
    neighbour records of the start determinant and of one FOIS neighbour."""
    import paper_1909_06935_gb300 as P
    s = S.workload("cas10_56o")
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    try:
        ctx.set_heat_bath_cutoff(0.002)
        orc.set_hb_eps(0.002)
        start = s.dets[orc.start]
        r = orc.local(start, max_nb=400000)
        fois = r["dets"][np.argmax(np.abs(r["psi_m"]) * (r["O"] != r["psi_m"]))]
        compare_local(ctx, orc, np.vstack([start[None], fois[None]]), s.W)
    finally:
        ctx.close()
