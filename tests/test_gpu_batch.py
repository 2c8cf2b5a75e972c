"""Batched form: several independent systems walked in one launch give the same result as each
system walked alone (trajectories bit-identical; accumulators and energies to rounding, because the
group sums are FP64 atomics whose order differs)."""
import numpy as np
import pytest

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
            assert _close(acc_a[key], acc_b[key], 1e-12), (k, key)
        for key in ("e2", "e_var", "a0sq", "e2_sigma"):
            assert _close(res_a[key], results[k][key], 1e-10), (k, key)
        assert results[k]["walker_steps"] == nw * (steps - 2)


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
