"""Serving form: requests for different systems admitted by a device-memory budget and advanced
together (continuous batching) give the same results as each request run alone (bit for bit) and
as the oracle's walk of the same request (within 1e-10)."""
import time

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def _systems():
    return [S.workload("tiny_12o_cas4"),
            S.make_system(1, 3, 4, 3, 3, rank=12, seed=71, chol_sigma=0.1),
            S.make_system(2, 4, 10, 4, 4, rank=16, seed=72, chol_sigma=0.08)]


def _close(a, b, rtol=1e-10):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= 1e-14 + rtol * np.maximum(np.abs(a), np.abs(b)))


def test_served_results_equal_alone():
    import paper_1909_06935_gb300 as P
    systems = _systems()
    walkers, seeds, steps = [128, 64, 96], [21, 22, 23], 10
    alone = []
    for s, nw, seed in zip(systems, walkers, seeds):
        ctx = P.Context.from_system(s)
        alone.append(ctx.sample(ctx.params(nw, steps, burn_in=2, seed=seed, n_groups=8)))
        ctx.close()
    srv = P.Server(max_active=8, steps_per_round=2)
    tickets = [srv.submit(s, nw, steps, burn_in=2, seed=seed, n_groups=8)
               for s, nw, seed in zip(systems, walkers, seeds)]
    for _ in range(100):
        srv.step()
        if all(srv.poll(t)["state"] in ("done", "failed") for t in tickets):
            break
    for t, ref, s, nw, seed in zip(tickets, alone, systems, walkers, seeds):
        st = srv.poll(t)
        assert st["state"] == "done" and st["steps_done"] == steps
        res = st["result"]
        assert np.array_equal(res["type_steps"], ref["type_steps"])
        for k in ("e2", "e2_sigma", "e_var", "a0sq"):
            assert res[k] == ref[k], k
        orc = O.Oracle.from_system(s)
        fo = orc.finalize(orc.sample(nw, steps, 2, seed, 8))
        assert np.array_equal(res["type_steps"], fo["type_steps"])
        for k in ("e2", "e2_sigma", "e_var", "a0sq"):
            assert _close(res[k], fo[k], 1e-9), k
    assert srv.info()["active"] == 0 and srv.info()["bytes"] == 0
    srv.close()


def test_admission_waits_for_budget_and_cancel():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    probe = P.Server(max_active=8, hbm_budget_bytes=1 << 40, steps_per_round=1)
    t0 = probe.submit(s, 64, 4)
    probe.step()
    one = probe.info()["bytes"]
    probe.close()
    assert one > 0
    srv = P.Server(max_active=8, hbm_budget_bytes=int(1.5 * one), steps_per_round=1)   # room for one
    a = srv.submit(s, 64, 3, seed=1)
    b = srv.submit(s, 64, 3, seed=2)
    c = srv.submit(s, 64, 3, seed=3)
    srv.step()
    assert srv.poll(a)["state"] == "running" and srv.poll(b)["state"] == "queued"
    srv.cancel(c)
    assert srv.poll(c)["state"] == "cancelled"
    for _ in range(20):
        srv.step()
    assert srv.poll(a)["state"] == "done" and srv.poll(b)["state"] == "done"
    assert srv.poll(b)["queue_seconds"] > 0.0
    big = srv.submit(S.workload("cas10_56o"), 64, 3)            # larger than the whole budget
    st = srv.poll(big)
    assert st["state"] == "failed" and st["status"] == -9
    srv.close()


def test_background_loop_serves_requests_arriving_while_busy():
    import paper_1909_06935_gb300 as P
    systems = _systems()
    srv = P.Server(max_active=4, steps_per_round=2)
    srv.start()
    tickets = []
    for k in range(6):
        s = systems[k % len(systems)]
        tickets.append(srv.submit(s, 64, 8, seed=100 + k, n_groups=4))
        time.sleep(0.01)
    deadline = time.time() + 120
    while time.time() < deadline and not all(srv.poll(t)["state"] == "done" for t in tickets):
        time.sleep(0.05)
    srv.stop()
    for t in tickets:
        st = srv.poll(t)
        assert st["state"] == "done" and st["result"]["status"] == 0 and st["total_seconds"] > 0
    srv.close()
