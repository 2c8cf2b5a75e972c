"""The largest shapes the boundary accepts, against the oracle: 128 spatial orbitals (two full
words per spin, the last virtual orbital in bit 63 of the second word) and a 32-orbital active
space (the active block fills a whole 32-bit half of the combined active masks).  Local
quantities element by element at the start determinant (3.4e5 neighbours at 128 orbitals), at
reference determinants and at sampled FOIS neighbours, and bit-exact trajectories of a short
walk."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from tests.test_gpu_parity import close, compare_local

pytestmark = pytest.mark.gpu

SHAPES = {
    "n128": dict(n_core=2, n_act=4, n_virt=122, n_alpha=4, n_beta=4, rank=12, seed=71, chol_sigma=0.05),
    "act32": dict(n_core=1, n_act=32, n_virt=4, n_alpha=2, n_beta=2, rank=10, seed=72, chol_sigma=0.05),
}


@pytest.mark.parametrize("name", list(SHAPES))
def test_largest_shapes_match_the_oracle(name):
    import paper_1909_06935_gb300 as P
    s = S.make_system(**SHAPES[name])
    ctx = P.Context.from_system(s)
    orc = O.Oracle.from_system(s)
    try:
        info = ctx.setup_info()
        assert close(info["e0"], orc.e0, 1e-12)
        start = s.dets[orc.start]
        r = orc.local(start, max_nb=400000)
        rng = np.random.default_rng(9)
        fois = r["dets"][r["O"] != r["psi_m"]]
        pick = fois[rng.choice(len(fois), min(6, len(fois)), replace=False)]
        dets = np.vstack([start[None], s.dets[rng.choice(len(s.dets), 4, replace=False)], pick])
        compare_local(ctx, orc, dets, s.W)
        nw, ns, burn, G, seed = 64, 12, 2, 4, 31
        acc_o = orc.sample(nw, ns, burn, seed, G, trajectory=True)
        ctx.sample(ctx.params(nw, ns, burn_in=burn, seed=seed, n_groups=G))
        got, _ = ctx.walkers(nw)
        assert np.array_equal(got, acc_o["trajectory"][:, -1, :])
        acc_g = ctx.accumulators(G)
        for k in ("N", "U", "W", "E"):
            assert close(acc_g[k], acc_o[k], 1e-10, 1e-14), k
    finally:
        ctx.close()
