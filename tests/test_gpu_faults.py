"""Failure detection without a GPU fault: every bound runs out on purpose and is reported.

* a host wait with a 1 ms deadline on a walk of about a second returns MRQ_DEVICE_TIMEOUT, the
  kernels finish on their own, and the context gives the full result afterwards;
* a hash-probe bound lowered to one slot runs out on the reference table's collisions and the
  finalize reports MRQ_HASH_OVERFLOW; restoring the bound restores the walk;
* a candidate-list capacity lowered to one entry is exceeded by the grouped CAS-walker path and
  reported as MRQ_TOO_LARGE.
No kernel traps, asserts or spins without a limit; the walk always ends.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TIMEOUT, HASH_OVERFLOW, TOO_LARGE = -6, -5, -9


@pytest.fixture(scope="module")
def tiny_ctx():
    import paper_1909_06935_gb300 as P
    s = S.workload("tiny_12o_cas4")
    ctx = P.Context.from_system(s)
    yield P, s, ctx
    ctx.close()


def test_deadline_returns_timeout_and_the_context_recovers(tiny_ctx):
    P, s, ctx = tiny_ctx
    ctx.walkers_init(ctx.params(4096, 0, burn_in=0, seed=3, n_groups=8))
    ctx.walkers_advance(200)
    ctx.set_deadline(1e-3)
    try:
        with pytest.raises(P.MRQError) as e:
            ctx.finalize()
        assert e.value.code == TIMEOUT
    finally:
        ctx.set_deadline(0.0)
    res = ctx.finalize()
    assert res["status"] == 0 and res["walker_steps"] == 4096 * 200
    # a generous deadline does not fire
    ctx.set_deadline(600.0)
    try:
        ctx.walkers_advance(2)
        assert ctx.finalize()["walker_steps"] == 4096 * 202
    finally:
        ctx.set_deadline(0.0)


def test_hash_probe_bound_runs_out_and_is_reported(tiny_ctx):
    P, s, ctx = tiny_ctx
    ctx.debug_set_limits(max_probe=1)
    try:
        ctx.walkers_init(ctx.params(256, 0, burn_in=0, seed=4, n_groups=4))
        ctx.walkers_advance(20)
        with pytest.raises(P.MRQError) as e:
            ctx.finalize()
        assert e.value.code == HASH_OVERFLOW
    finally:
        ctx.debug_set_limits(0, 0)
    ctx.walkers_init(ctx.params(256, 0, burn_in=0, seed=4, n_groups=4))
    ctx.walkers_advance(20)
    assert ctx.finalize()["status"] == 0


def test_candidate_capacity_runs_out_and_is_reported(tiny_ctx):
    P, s, ctx = tiny_ctx
    ctx.debug_set_limits(cand_cap=1)
    try:
        ctx.walkers_init(ctx.params(256, 0, burn_in=0, seed=6, n_groups=4))
        ctx.walkers_advance(5)
        with pytest.raises(P.MRQError) as e:
            ctx.finalize()
        assert e.value.code == TOO_LARGE
    finally:
        ctx.debug_set_limits(0, 0)
    ctx.walkers_init(ctx.params(256, 0, burn_in=0, seed=6, n_groups=4))
    ctx.walkers_advance(5)
    assert ctx.finalize()["status"] == 0


def test_limits_reject_bad_arguments(tiny_ctx):
    P, s, ctx = tiny_ctx
    for mp, cap in ((-1, 0), (65, 0), (0, -3)):
        with pytest.raises(P.MRQError) as e:
            ctx.debug_set_limits(mp, cap)
        assert e.value.code == -1
    with pytest.raises(P.MRQError):
        ctx.set_deadline(-1.0)
