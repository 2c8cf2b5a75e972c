"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Bar: excitation sets bit-exact; H_nm, H_D, O(m), psi_s(m), Gamma, S, E_L and the H_D numerator
within 1e-10 relative (FP64 on both sides, different summation orders); walker trajectories
bit-exact (first-reaction clocks are keyed on the excitation, so enumeration order does not
matter); accumulators within 1e-10 relative.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from tests import secondq as Q

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _mrq():
    import paper_1909_06935_gb300 as P
    return P


def close(a, b, rtol=RTOL, atol=1e-13):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= atol + rtol * np.maximum(np.abs(a), np.abs(b)))


def compare_local(ctx, orc, dets, W):
    loc, nb = ctx.debug_local(dets, max_nb=0)
    maxnb = int(loc["n_neighbours"].max()) if len(loc) else 0
    loc, nb = ctx.debug_local(dets, max_nb=max(maxnb, 1))
    for i, d in enumerate(dets):
        r = orc.local(d, max_nb=max(maxnb, 1))
        assert loc["label"][i] == r["label"]
        assert loc["type"][i] == r["type"]
        assert loc["n_neighbours"][i] == r["nnb"]
        assert loc["n_terms"][i] == r["terms"]            # the roofline's algorithmic count
        for key_g, key_o in (("S", "S"), ("e_local", "EL"), ("num", "num"), ("h_nn", "Hnn"), ("hd_nn", "HDnn"),
                             ("psi", "psi")):
            assert close(loc[key_g][i], r[key_o]), (i, key_g, loc[key_g][i], r[key_o])
        k = r["nnb"]
        g = nb[i, :k]
        og = np.argsort(g["exc"], kind="stable")
        oo = np.argsort(r["exc"], kind="stable")
        assert np.array_equal(g["exc"][og], r["exc"][oo])                        # bit-exact sets
        assert np.array_equal(g["det"][og][:, :2 * W], r["dets"][oo])            # bit-exact images
        for fg, fo in (("h", "H"), ("hd", "HD"), ("o", "O"), ("psi", "psi_m"), ("gamma", "Gamma")):
            assert close(g[fg][og], r[fo][oo]), (i, fg)


@pytest.fixture(scope="module")
def tiny_pair():
    P = _mrq()
    s = S.workload("tiny_12o_cas4")
    return s, P.Context.from_system(s), O.Oracle.from_system(s)


def test_setup_parity(tiny_pair):
    s, ctx, orc = tiny_pair
    info = ctx.setup_info()
    assert close(info["e0"], orc.e0, 1e-12)
    assert close(info["norm0"], orc.norm0, 1e-12)
    assert close(info["e_core"], orc.e_core, 1e-12)
    assert close(info["eps"], orc.eps, 1e-11)
    assert close(info["gamma"], orc.gamma[:s.n_act, :s.n_act], 1e-11, 1e-13)
    assert info["start"] == orc.start


def test_local_parity_tiny_workload(tiny_pair):
    s, ctx, orc = tiny_pair
    start = s.dets[orc.start]
    r = orc.local(start, max_nb=4096)
    rng = np.random.default_rng(1)
    pick = rng.choice(r["nnb"], 24, replace=False)
    dets = np.vstack([start[None], s.dets[:8], r["dets"][pick]])
    # second layer: neighbours of FOIS neighbours (all classes)
    r2 = orc.local(r["dets"][pick[0]], max_nb=8192)
    dets = np.vstack([dets, r2["dets"][rng.choice(r2["nnb"], 24, replace=False)]])
    compare_local(ctx, orc, dets, s.W)


@pytest.mark.parametrize("spec", [
    dict(n_core=1, n_act=2, n_virt=2, n_alpha=2, n_beta=2, seed=31),
    dict(n_core=1, n_act=3, n_virt=2, n_alpha=3, n_beta=2, seed=32),
    dict(n_core=2, n_act=2, n_virt=1, n_alpha=3, n_beta=3, seed=33),
    dict(n_core=0, n_act=6, n_virt=0, n_alpha=3, n_beta=3, seed=41),
    dict(n_core=3, n_act=0, n_virt=5, n_alpha=3, n_beta=3, seed=43),
])
def test_local_parity_whole_spaces(spec):
    """Every determinant of a tiny space (all classes, ragged list sizes, empty core/active/virtual)."""
    P = _mrq()
    s = S.make_system(**spec, rank=12, chol_sigma=0.12)
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    space = Q.full_space(s.n_orb, s.n_alpha, s.n_beta)
    dets = np.array([Q.to_words(d, s.n_orb) for d in space])
    keep = [i for i, d in enumerate(dets) if orc.label(d)[0] >= 0 and orc.psi(d)[0] != 0.0]
    compare_local(ctx, orc, dets[keep], s.W)


def test_two_word_determinants_and_straddling_active_block():
    """n > 64 (two words per spin) with the active block across the word boundary."""
    P = _mrq()
    s = S.make_system(62, 4, 4, 64, 64, rank=8, seed=61, chol_sigma=0.05)
    assert s.W == 2
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    r = orc.local(s.dets[orc.start], max_nb=400000)
    rng = np.random.default_rng(2)
    dets = np.vstack([s.dets[orc.start][None], r["dets"][rng.choice(r["nnb"], 6, replace=False)]])
    compare_local(ctx, orc, dets, s.W)


def test_trajectories_and_accumulators_match_oracle(tiny_pair):
    s, ctx, orc = tiny_pair
    nw, ns, burn, G, seed = 96, 60, 10, 8, 4242
    acc_o = orc.sample(nw, ns, burn, seed, G, trajectory=True)
    p = ctx.params(nw, ns, burn_in=burn, seed=seed, n_groups=G)
    res = ctx.sample(p)
    dets, psi = ctx.walkers(nw)
    assert np.array_equal(dets, acc_o["trajectory"][:, -1, :])
    acc_g = ctx.accumulators(G)
    assert np.array_equal(acc_g["type_steps"], acc_o["type_steps"])
    for k in ("N", "U", "W", "E"):
        assert close(acc_g[k], acc_o[k], 1e-10, 1e-14), k
    # finalize on the device against the oracle's finalize of the same accumulators
    f = O.finalize(acc_g, orc.e0, orc.c, s.n_core, s.n_virt, 1e-10)
    for k in ("e2", "e2_sigma", "e_var", "e_var_sigma", "a0sq", "a0sq_sigma", "e_mrci_q", "screened_norm"):
        assert close(res[k], f[k], 1e-9, 1e-14), k
    for k in ("type_norm", "type_e2", "type_e2_sigma", "type_norm_sigma", "type_screened"):
        assert close(res[k], f[k], 1e-9, 1e-14), k
    assert res["walker_steps"] == nw * (ns - burn)
    assert res["status"] == 0


def test_chunked_advance_equals_one_launch(tiny_pair):
    s, ctx, orc = tiny_pair
    p = ctx.params(64, 40, burn_in=5, seed=9, n_groups=4)
    ctx.walkers_init(p)
    ctx.walkers_advance(40)
    a = ctx.walkers(64)[0]
    ctx.walkers_init(p)
    for _ in range(4):
        ctx.walkers_advance(10)
    b = ctx.walkers(64)[0]
    assert np.array_equal(a, b)


def test_stochastic_energy_within_3_sigma_of_brute_force(tiny_pair):
    s, ctx, orc = tiny_pair
    ex = O.exact_from_brute(orc.brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    p = ctx.params(2048, 1600, burn_in=100, seed=77, n_groups=32)
    res = ctx.sample(p)
    assert res["e2_sigma"] <= 1e-4
    assert abs(res["e2"] - ex["e2"]) < 3 * res["e2_sigma"]
    assert abs(res["e_var"] - ex["e_var"]) < 3 * res["e_var_sigma"]
    assert abs(res["a0sq"] - ex["a0sq"]) < 3 * res["a0sq_sigma"]


def test_errors_are_reported():
    P = _mrq()
    s = S.workload("tiny_12o_cas4")
    ctx = P.Context()
    with pytest.raises(P.MRQError) as e:
        ctx.load_reference(s.dets, s.coeffs)
    assert e.value.code == -2
    ctx.load_hamiltonian(s.n_core, s.n_act, s.n_virt, s.n_alpha, s.n_beta, s.h1, s.eri, s.e_nuc)
    bad = s.dets.copy()
    bad[0, 0] ^= np.uint64(1)          # a core hole
    with pytest.raises(P.MRQError) as e:
        ctx.load_reference(bad, s.coeffs)
    assert e.value.code == -3
    dup = s.dets.copy()
    dup[1] = dup[0]
    with pytest.raises(P.MRQError) as e:
        ctx.load_reference(dup, s.coeffs)
    assert e.value.code == -3
    ctx.load_reference(s.dets, s.coeffs)
    with pytest.raises(P.MRQError) as e:
        ctx.set_coeffs(s.c[:-1])
    assert e.value.code == -1
    with pytest.raises(P.MRQError):
        ctx.walkers_advance(3)


def test_full_size_launch_sampled_walkers_and_dets():
    """56-orbital CAS(10e,10o) workload in the benchmark's launch configuration (4096 walkers, one
    walker step per launch): sampled walkers' trajectories, and every per-neighbour record at the
    start determinant and at one determinant of each class the walkers reached, against the oracle."""
    P = _mrq()
    s = S.workload("cas10_56o")
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    nw, steps, seed = 4096, 2, 1000
    p = ctx.params(nw, steps, burn_in=0, seed=seed, n_groups=16)
    ctx.walkers_init(p)
    for _ in range(steps):
        ctx.walkers_advance(1)
        ctx.finalize()
    dets, _ = ctx.walkers(nw)
    for w in (0, 4095):
        traj = orc.walk_one(w, steps, seed)
        assert np.array_equal(dets[w], traj[-1]), w
    # every neighbour record, element by element, at the start determinant (3.45e5 neighbours)
    # and at one walker determinant of each class the walk has reached
    loc, _ = ctx.debug_local(dets)
    picks, seen = [s.dets[orc.start]], {0}
    for i in range(nw):
        t = int(loc["type"][i])
        if t not in seen:
            seen.add(t)
            picks.append(dets[i])
    assert len(picks) >= 3
    compare_local(ctx, orc, np.array(picks), s.W)


def test_target_sigma_stops_early_and_equals_a_fixed_length_run(tiny_pair):
    s, ctx, orc = tiny_pair
    ctx.set_coeffs(s.c)
    p = ctx.params(512, 4000, burn_in=20, seed=31, n_groups=16, target_sigma=2e-3, steps_per_check=40)
    res = ctx.sample(p)
    steps = res["total_steps"] // 512
    assert res["e2_sigma"] <= 2e-3 and steps < 4000 and steps % 40 == 0
    ref = ctx.sample(ctx.params(512, steps, burn_in=20, seed=31, n_groups=16, warps_per_walker=2))
    for k in ("e2", "e2_sigma", "e_var", "a0sq"):
        assert close(res[k], ref[k], 1e-9), k
    ctx.walkers_init(ctx.params(32, 0, warps_per_walker=4))


def test_frozen_core_variant_within_3_sigma_of_brute_force(tiny_pair):
    """c_l = 0 on core-hole labels: only the (0,1) and (0,2) classes are sampled, and E^(2) hits the
    brute-force sum over the core-free labels."""
    import paper_1909_06935_gb300 as P
    s, ctx, orc = tiny_pair
    ex = O.exact_from_brute(orc.brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    e2_frozen = ex["type_e2"][:3].sum()                 # types 3h + p with h = 0
    ctx.set_coeffs(P.frozen_core_coeffs(s.c, s.n_core, s.n_virt))
    try:
        res = ctx.sample(ctx.params(2048, 800, burn_in=100, seed=78, n_groups=32))
    finally:
        ctx.set_coeffs(s.c)
    assert np.all(res["type_steps"][3:] == 0) and np.all(res["type_e2"][3:] == 0)
    assert abs(res["e2"] - e2_frozen) < 3 * res["e2_sigma"]


def test_l2_window_changes_nothing(tiny_pair):
    """The persisting-L2 window on the integral tables is a cache hint: the same trajectories and
    the same accumulators, bit for bit."""
    s, ctx, orc = tiny_pair
    ctx.set_coeffs(s.c)
    out = []
    for frac in (0.0, 1.0):
        ctx.set_l2_window(frac)
        ctx.walkers_init(ctx.params(256, 0, burn_in=2, seed=17, n_groups=4))
        ctx.walkers_advance(12)
        out.append((ctx.walkers(256)[0], ctx.accumulators(4)))
    ctx.set_l2_window(0.0)
    assert np.array_equal(out[0][0], out[1][0])
    for key in ("N", "U", "W", "E", "type_steps"):
        assert np.array_equal(out[0][1][key], out[1][1][key]), key
