"""Batched form: several independent systems walked in one launch give the same result as each
system walked alone, bit for bit (every walker's step is evaluated by the same block code, and the
accumulation adds each group's walkers in walker order), and the same as the oracle's walk
(trajectories bit-identical, accumulators within 1e-10)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def _systems():
    return [
        S.workload("tiny_12o_cas4"),
        S.make_system(1, 3, 4, 3, 3, rank=12, seed=71, chol_sigma=0.1),
        S.make_system(62, 4, 4, 64, 64, rank=8, seed=61, chol_sigma=0.05),     # two words per spin
        S.make_system(2, 4, 10, 4, 4, rank=16, seed=72, chol_sigma=0.08),
    ]


def _close(a, b, rtol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= 1e-14 + rtol * np.maximum(np.abs(a), np.abs(b)))


def test_batch_equals_alone():
    import paper_1909_06935_gb300 as P
    systems = _systems()
    walkers = [128, 64, 32, 96]
    seeds = [11, 12, 13, 14]
    steps, G = 12, 8
    alone = []
    for s, nw, seed in zip(systems, walkers, seeds):
        ctx = P.Context.from_system(s)
        res = ctx.sample(ctx.params(nw, steps, burn_in=2, seed=seed, n_groups=G))
        alone.append((ctx.walkers(nw)[0], ctx.accumulators(G), res))
        ctx.close()
    ctxs = [P.Context.from_system(s) for s in systems]
    params = [c.params(nw, steps, burn_in=2, seed=seed, n_groups=G) for c, nw, seed in zip(ctxs, walkers, seeds)]
    results = P.sample_batch(ctxs, params)
    for k, (c, nw) in enumerate(zip(ctxs, walkers)):
        dets_a, acc_a, res_a = alone[k]
        dets_b = c.walkers(nw)[0]
        assert np.array_equal(dets_a, dets_b), k
        acc_b = c.accumulators(G)
        assert np.array_equal(acc_a["type_steps"], acc_b["type_steps"])
        for key in ("N", "U", "W", "E"):
            assert np.array_equal(acc_a[key], acc_b[key]), (k, key)
        for key in ("e2", "e_var", "a0sq", "e2_sigma"):
            assert res_a[key] == results[k][key], (k, key)
        assert results[k]["walker_steps"] == nw * (steps - 2)
        # and the oracle's walk of the same system, walkers and seed
        orc = O.Oracle.from_system(systems[k])
        acc_o = orc.sample(nw, steps, 2, seeds[k], G, trajectory=True)
        assert np.array_equal(dets_b, acc_o["trajectory"][:, -1, :]), k
        assert np.array_equal(acc_b["type_steps"], acc_o["type_steps"]), k
        for key in ("N", "U", "W", "E"):
            assert _close(acc_b[key], acc_o[key], 1e-10), (k, key)
        fo = orc.finalize(acc_o)
        for key in ("e2", "e_var", "a0sq", "e2_sigma"):
            assert _close(results[k][key], fo[key], 1e-9), (k, key)


def test_batch_advance_in_chunks_matches_single_launch():
    import paper_1909_06935_gb300 as P
    systems = _systems()[:2]
    ctxs = [P.Context.from_system(s) for s in systems]
    for c in ctxs:
        c.walkers_init(c.params(64, 0, seed=5, n_groups=4))
    P.batch_advance(ctxs, 9)
    a = [c.walkers(64)[0] for c in ctxs]
    for c in ctxs:
        c.walkers_init(c.params(64, 0, seed=5, n_groups=4))
    for _ in range(3):
        P.batch_advance(ctxs, 3)
    b = [c.walkers(64)[0] for c in ctxs]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_batch_rejects_bad_lists():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    c = P.Context.from_system(s)
    c.walkers_init(c.params(32, 0, seed=1, n_groups=4))
    with pytest.raises(P.MRQError):
        P.batch_advance([c, c], 1)
    d = P.Context.from_system(s)               # no walkers yet
    with pytest.raises(P.MRQError):
        P.batch_advance([c, d], 1)


def _run_batch(ctxs, walkers, seeds, steps, G, launch):
    import paper_1909_06935_gb300 as P
    for c in ctxs:
        c.set_launch(*launch)
    for c, nw, seed in zip(ctxs, walkers, seeds):
        c.walkers_init(c.params(nw, steps, burn_in=2, seed=seed, n_groups=G))
    P.batch_advance(ctxs, steps)
    out = [(c.walkers(nw)[0], c.accumulators(G)) for c, nw in zip(ctxs, walkers)]
    for c in ctxs:
        c.set_launch()
    return out


@pytest.mark.parametrize("launch", [(1, 1, False), (2, 4, True), (8, 16, True), (1, 7, True), (2, 0, False),
                                    (0, 3, True)])
def test_launch_configuration_leaves_results_unchanged(launch):
    """Warps per walker, steps per launch (re-ordering the slots between launches) and CUDA-graph
    replay change the schedule only: every walker's units form the same fixed partition whatever
    the warps, and the accumulation adds each group's walkers in id order, so trajectories and
    accumulators are bit-identical."""
    import paper_1909_06935_gb300 as P
    systems = _systems()
    walkers, seeds, steps, G = [128, 64, 32, 96], [21, 22, 23, 24], 40, 4
    ctxs = [P.Context.from_system(s) for s in systems]
    ref = _run_batch(ctxs, walkers, seeds, steps, G, (4, 0, False))
    got = _run_batch(ctxs, walkers, seeds, steps, G, launch)
    got2 = _run_batch(ctxs, walkers, seeds, steps, G, launch)          # graph reuse
    for k in range(len(systems)):
        for g in (got, got2):
            assert np.array_equal(ref[k][0], g[k][0]), (k, launch)
            assert np.array_equal(ref[k][1]["type_steps"], g[k][1]["type_steps"])
            for key in ("N", "U", "W", "E"):
                assert np.array_equal(ref[k][1][key], g[k][1][key]), (k, key, launch)
    for c in ctxs:
        c.close()


def test_tuner_leaves_state_unchanged_and_sets_a_tried_configuration():
    import paper_1909_06935_gb300 as P
    systems = _systems()
    walkers, G = [128, 64, 32, 96], 4
    ctxs = [P.Context.from_system(s) for s in systems]
    for c, nw in zip(ctxs, walkers):
        c.walkers_init(c.params(nw, 0, burn_in=0, seed=3, n_groups=G))
    P.batch_advance(ctxs, 5)
    before = [(c.walkers(nw)[0], c.accumulators(G)) for c, nw in zip(ctxs, walkers)]
    t = P.tune_batch(ctxs, trial_steps=16)
    assert len(t["tried"]) == 9 and all(ms > 0 for _, _, ms in t["tried"])
    assert (t["warps_per_walker"], t["steps_per_launch"]) in [(w, s) for w, s, _ in t["tried"]]
    after = [(c.walkers(nw)[0], c.accumulators(G)) for c, nw in zip(ctxs, walkers)]
    for (da, aa), (db, ab) in zip(before, after):
        assert np.array_equal(da, db)
        for key in ("N", "U", "W", "E", "type_steps"):
            assert np.array_equal(aa[key], ab[key])
    # the tuned configuration continues the same trajectories
    for c in ctxs:
        c.set_launch(t["warps_per_walker"], t["steps_per_launch"], True)
    P.batch_advance(ctxs, 10)
    tuned = [c.walkers(nw)[0] for c, nw in zip(ctxs, walkers)]
    for c, nw in zip(ctxs, walkers):
        c.set_launch()
        c.walkers_init(c.params(nw, 0, burn_in=0, seed=3, n_groups=G))
    P.batch_advance(ctxs, 15)
    for x, c, nw in zip(tuned, ctxs, walkers):
        assert np.array_equal(x, c.walkers(nw)[0])
    with pytest.raises(P.MRQError):
        P.tune_batch(ctxs, trial_steps=0)
    for c in ctxs:
        c.close()
