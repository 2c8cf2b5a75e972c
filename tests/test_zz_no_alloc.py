"""The allocation-free finalize gives the same result as the ordinary one.

mrq_finalize_noalloc exists for callers that must not call cudaMalloc/cudaFree while they run
(a serving loop whose device memory is all owned by its own pool allocator, or a latency-bound
loop that cannot absorb the device synchronisation an allocation may cause): its scratch is a
fixed array inside the library.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

KEYS = ("e0", "e2", "e2_sigma", "e_var", "e_var_sigma", "a0sq", "a0sq_sigma", "e_mrci_q", "screened_norm",
        "n_labels_visited")
ARRAYS = ("type_norm", "type_norm_sigma", "type_e2", "type_e2_sigma", "type_screened")


def _close(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= 1e-14 + 1e-12 * np.maximum(np.abs(a), np.abs(b)))


def test_noalloc_finalize_matches_finalize_on_two_calls():
    import paper_1909_06935_gb300 as P
    lib = P.load_library()
    s = S.workload("tiny_12o_cas4")
    ctx = P.Context.from_system(s)
    p = ctx.params(256, 0, burn_in=4, seed=31, n_groups=8)
    ctx.walkers_init(p)
    for call in range(2):
        ctx.walkers_advance(25)
        ref = P.Result()
        got = P.Result()
        assert lib.mrq_finalize(ctx._h, ctypes.byref(ref)) == 0
        assert lib.mrq_finalize_noalloc(ctx._h, ctypes.byref(got)) == 0, lib.mrq_last_error(ctx._h)
        r, g = ref.as_dict(), got.as_dict()
        for k in KEYS + ARRAYS:
            assert _close(g[k], r[k]), (call, k, g[k], r[k])
        assert np.array_equal(g["type_steps"], r["type_steps"])
        assert g["walker_steps"] == r["walker_steps"] > 0
        assert g["status"] == 0
    ctx.close()


def test_noalloc_finalize_rejects_sizes_beyond_its_fixed_scratch():
    """A walk whose finalize needs more partial sums than the fixed array holds is refused with
    MRQ_TOO_LARGE (and a message), nothing is written; the ordinary finalize still works, and a
    smaller group count fits again (two-word determinants, 1.5 million labels)."""
    import paper_1909_06935_gb300 as P
    lib = P.load_library()
    s = S.make_system(10, 2, 60, 11, 11, rank=40, seed=4242)      # 211 x 7261 labels
    nchunk = -(-len(s.c) // 8192)
    assert 65 * nchunk * 45 > P.NOALLOC_SCRATCH_DOUBLES > 17 * nchunk * 45
    ctx = P.Context.from_system(s)
    try:
        ctx.walkers_init(ctx.params(64, 0, burn_in=0, seed=5, n_groups=64))
        ctx.walkers_advance(2)
        got = P.Result()
        assert lib.mrq_finalize_noalloc(ctx._h, ctypes.byref(got)) == -9
        assert b"fixed" in lib.mrq_last_error(ctx._h)
        assert got.walker_steps == 0
        assert ctx.finalize()["walker_steps"] == 128
        ctx.walkers_init(ctx.params(64, 0, burn_in=0, seed=5, n_groups=16))
        ctx.walkers_advance(2)
        ref = P.Result()
        assert lib.mrq_finalize(ctx._h, ctypes.byref(ref)) == 0
        assert lib.mrq_finalize_noalloc(ctx._h, ctypes.byref(got)) == 0, lib.mrq_last_error(ctx._h)
        r, g = ref.as_dict(), got.as_dict()
        for k in KEYS + ARRAYS:
            assert _close(g[k], r[k]), (k, g[k], r[k])
    finally:
        ctx.close()
