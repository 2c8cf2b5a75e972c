"""Host-side logic of the benchmark (no GPU): the clock record built from nvidia-smi samples, the
whole-job rate of weak scaling, and the merge of several ranks' walker groups."""
import numpy as np

import bench


def test_clock_summary_from_samples():
    c = bench.ClockSampler(0)
    c.rows = [
        ["0", "1965", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "2070", "2070", "1100.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2070", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "[N/A]", "2070"],                       # a malformed line is ignored
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    c.rows.append(["0", "1500", "2070", "1300", "0x8", "Active", "Not Active", "Active", "Not Active"])
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_job_rate_is_all_ranks_over_the_slowest():
    assert bench.job_rate(4096, 1, 250.0) == 4096 / 0.25
    assert bench.job_rate(4096, 8, 500.0) == 8 * 4096 / 0.5


def test_merge_keeps_rank_order_and_adds_counts():
    G, L = 4, 7
    rng = np.random.default_rng(1)
    accs = []
    for r in range(3):
        a = {k: rng.random((G, L)) for k in ("N", "U", "A", "B")}
        a.update(W=rng.random(G), E=rng.random(G), type_steps=np.arange(9) + r, total_steps=100 * (r + 1))
        accs.append(a)
    m = bench.merge_rank_accumulators(accs)
    assert m["N"].shape == (3 * G, L) and m["W"].shape == (3 * G,)
    for r in range(3):
        for k in ("N", "U", "A", "B", "W", "E"):
            assert np.array_equal(m[k][r * G:(r + 1) * G], accs[r][k])
    assert np.array_equal(m["type_steps"], 3 * np.arange(9) + 3) and m["total_steps"] == 600
    # ranks without gradient sums merge without them
    for a in accs:
        del a["A"]
    assert "A" not in bench.merge_rank_accumulators(accs)
