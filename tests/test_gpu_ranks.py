"""The cross-rank reduction through the C ABI (mrq_load_accumulators): two independent walks
stand in for two ranks; their groups, concatenated in rank order, are loaded into one context
and finalized.  The combined estimates equal the oracle's finalize of the same sums (1e-10),
and the combined E^(2) lies within 3 sigma of the brute force."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def test_union_of_two_walks_finalizes_like_the_oracle():
    import bench
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    orc = O.Oracle.from_system(s)
    G = bench.groups_per_rank(2)
    accs = []
    for rank in range(2):
        ctx = P.Context.from_system(s)
        try:
            res = ctx.sample(ctx.params(1024, 800, burn_in=100, seed=bench.rank_seed(rank), n_groups=G))
            acc = ctx.accumulators(G)
            acc["A"], acc["B"] = ctx.gradient_sums(G)
            acc["total_steps"] = int(res["total_steps"])
        finally:
            ctx.close()
        accs.append(acc)
    merged = bench.merge_rank_accumulators(accs)
    ctx = P.Context.from_system(s)
    try:
        ctx.load_accumulators(merged, merged["total_steps"])
        got = ctx.finalize()
        with pytest.raises(P.MRQError):
            ctx.walkers_advance(1)               # the walkers no longer match the loaded groups
    finally:
        ctx.close()
    want = orc.finalize(merged)
    for q in ("e2", "e2_sigma", "e_var", "e_var_sigma", "a0sq", "a0sq_sigma"):
        assert abs(got[q] - want[q]) <= 1e-10 * max(1.0, abs(want[q])), (q, got[q], want[q])
    assert int(got["total_steps"]) == merged["total_steps"] == 2 * 1024 * 800
    ex = O.exact_from_brute(orc.brute(), orc.e0, orc.c, s.n_core, s.n_virt)
    assert abs(got["e2"] - ex["e2"]) < 3 * got["e2_sigma"]
