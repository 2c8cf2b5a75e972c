"""104-orbital workload at full size: 10 core, 14 active, 80 virtual orbitals, 34 electrons, a
1,000,000-determinant selected-CI reference (two words per spin; the hash table, labels and
integral tables live in HBM).  Set-up, local quantities at CAS and FOIS determinants of every
class type, and 16,384-walker trajectories against the oracle (the oracle's sums over the
3.2 million neighbours of a CAS determinant run in parallel, so values agree to rounding)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def close(a, b, rtol=RTOL, atol=1e-13):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= atol + rtol * np.maximum(np.abs(a), np.abs(b)))


@pytest.fixture(scope="module")
def c3():
    import paper_1909_06935_gb300 as P
    s = S.workload("sci_104o_cas14")
    assert s.W == 2 and len(s.coeffs) == 1_000_000
    return s, P.Context.from_system(s), O.Oracle.from_system(s)


def _move(det, W, n, moves):
    """Apply (spin, from, to) electron moves to a determinant (alpha words, then beta words)."""
    d = det.copy()
    for sg, p, q in moves:
        for orb, on in ((p, False), (q, True)):
            w, b = sg * W + orb // 64, np.uint64(1) << np.uint64(orb % 64)
            assert bool(d[w] & b) != on, (sg, orb)
            d[w] = (d[w] | b) if on else (d[w] & ~b)
    return d


def test_setup_parity(c3):
    s, ctx, orc = c3
    info = ctx.setup_info()
    assert close(info["e0"], orc.e0, 1e-11)
    assert close(info["norm0"], orc.norm0, 1e-11)
    assert close(info["eps"], orc.eps, 1e-10)
    assert close(info["gamma"], orc.gamma[:s.n_act, :s.n_act], 1e-10, 1e-12)
    assert info["start"] == orc.start


def _class_dets(s, orc):
    """The CAS start determinant and one FOIS determinant of each of the eight classes."""
    n, W, nc, na = s.n_orb, s.W, s.n_core, s.n_act
    start = s.dets[orc.start]

    def occupied(sg, lo, hi):
        return [p for p in range(lo, hi) if (int(start[sg * W + p // 64]) >> (p % 64)) & 1]

    def empty(sg, lo, hi):
        return [p for p in range(lo, hi) if not (int(start[sg * W + p // 64]) >> (p % 64)) & 1]

    aocc, aemp = occupied(0, nc, nc + na), empty(0, nc, nc + na)
    bocc, bemp = occupied(1, nc, nc + na), empty(1, nc, nc + na)
    v0 = nc + na
    dets = [start]
    for moves in (
        [(0, nc - 1, aemp[0])],                                  # (1,0)
        [(1, bocc[0], v0 + 3)],                                  # (0,1)
        [(0, 4, v0 + 50)],                                       # (1,1), virtual in word 1
        [(0, nc - 2, aemp[0]), (1, nc - 1, bemp[1])],           # (2,0)
        [(0, aocc[0], v0), (1, bocc[1], v0 + 41)],              # (0,2)
        [(0, 3, v0 + 60), (1, 7, n - 1)],                        # (2,2), both virtuals in word 1
        [(1, 2, v0 + 5), (1, bocc[2], v0 + 9)],                  # (1,2) same spin
        [(0, 1, aemp[1]), (0, 6, v0 + 70)],                      # (2,1)
    ):
        dets.append(_move(start, W, n, moves))
    return np.array(dets)


def test_local_quantities_every_class(c3):
    s, ctx, orc = c3
    dets = _class_dets(s, orc)
    loc, _ = ctx.debug_local(dets)
    types = []
    for i, d in enumerate(dets):
        r = orc.local(d)
        types.append(r["type"])
        assert loc["label"][i] == r["label"] and loc["type"][i] == r["type"]
        assert loc["n_neighbours"][i] == r["nnb"] and loc["n_terms"][i] == r["terms"], i
        for kg, ko in (("S", "S"), ("e_local", "EL"), ("num", "num"), ("h_nn", "Hnn"), ("hd_nn", "HDnn"),
                       ("psi", "psi")):
            assert close(loc[kg][i], r[ko]), (i, kg, loc[kg][i], r[ko])
    assert sorted(types) == [0, 1, 2, 3, 4, 5, 6, 7, 8]


def test_per_neighbour_records_at_every_class(c3):
    """Every neighbour record at full size: at the CAS start determinant (3.2 million neighbours)
    and one determinant of each FOIS class, the set of excitations is bit-exact against the
    oracle's enumeration, and a seeded random sample of up to 50,000 records per determinant
    (images, H_nm, (H_D)_nm, O(m), psi_s(m), Gamma) matches the oracle's evaluation of the same
    neighbours within 1e-10."""
    s, ctx, orc = c3
    dets = _class_dets(s, orc)
    rng = np.random.default_rng(104)
    loc, _ = ctx.debug_local(dets)
    for i, d in enumerate(dets):
        nnb = int(loc["n_neighbours"][i])
        _, nb = ctx.debug_local(d[None], max_nb=nnb)
        g = nb[0]
        ids = orc.neighbour_ids(d)
        assert len(ids) == nnb, i
        assert np.array_equal(np.sort(g["exc"]), np.sort(ids)), i
        pick = np.sort(rng.choice(nnb, min(nnb, 50_000), replace=False))
        r = orc.neighbours(d, g["exc"][pick])
        assert np.array_equal(g["det"][pick][:, :2 * s.W], r["dets"]), i
        for fg, fo in (("h", "H"), ("hd", "HD"), ("o", "O"), ("psi", "psi_m"), ("gamma", "Gamma")):
            assert close(g[fg][pick], r[fo]), (i, fg)


def test_walk_16384_walkers_sampled_trajectories(c3):
    s, ctx, orc = c3
    nw, steps, seed = 16384, 2, 4711
    ctx.walkers_init(ctx.params(nw, steps, burn_in=0, seed=seed, n_groups=16))
    for _ in range(steps):
        ctx.walkers_advance(1)
    res = ctx.finalize()
    assert res["status"] == 0 and res["walker_steps"] == nw * steps
    dets, _ = ctx.walkers(nw)
    for w in (0, nw - 1):
        traj = orc.walk_one(w, steps, seed)
        assert np.array_equal(dets[w], traj[-1]), w


def test_device_selected_ci_reproduces_the_host_reference(c3):
    """The device generator (mrq_sci_reference) on the raw 104-orbital integrals selects the host
    generator's 1,000 strings and reaches its energy; the semicanonical rotation it loads gives the
    same E0 and core/virtual orbital energies as the host's rotated integrals."""
    import time
    import paper_1909_06935_gb300 as P
    s, ctx_host, _ = c3
    h1, L = S.make_integrals(10, 14, 80, 312, 2309, chol_sigma=0.05)
    alpha = np.unique((s.dets[:, 0] >> np.uint64(10)) & np.uint64((1 << 14) - 1)).astype(np.int64)
    ctx = P.Context()
    try:
        ctx.load_hamiltonian(10, 14, 80, 17, 17, h1, S.pack_eri(L), s.e_nuc)
        t0 = time.perf_counter()
        r = ctx.sci_reference(1000, n_seed_strings=256, tol=1e-5, max_iter=80, max_sub=24, semicanonical=True)
        dt = time.perf_counter() - t0
        info = ctx.setup_info()
    finally:
        ctx.close()
    print(f"device selected CI: {dt:.2f} s, E = {r['energy']:.12f}, iterations {r['iters_seed']} + {r['iters']}")
    assert r["n_det"] == 1_000_000
    assert sorted(r["strings"].tolist()) == alpha.tolist()
    assert abs(r["energy"] - s.e_cas) < 1e-7
    ref = ctx_host.setup_info()
    assert abs(info["e0"] - ref["e0"]) < 1e-7
    assert np.allclose(info["eps"], ref["eps"], atol=1e-7)
