"""The inner product entry point that allocates nothing, for callers that
cannot allocate memory while they call it: it must give the same <a, b> as
qtt_tt_dot (FP64 transfer matrices in both), call after call, with its
temporaries in the library's fixed device array. This file is collected last
so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from oracle import qtt as oq
from tests._helpers import random_tt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_dot_matches_dot_twice(Q, precision):
    prec = Q.QTT_FP64 if precision == "fp64" else Q.QTT_FP32
    ctx = Q.Context(0, prec, 1 << 28, seed=7)
    rng = np.random.default_rng(11)
    dims = [6] + [2] * 9
    ranks = [1, 6, 12, 24, 48, 64, 40, 16, 8, 4, 1]
    ac = random_tt(rng, dims, ranks)
    bc = random_tt(rng, dims, [1, 5, 10, 20, 40, 64, 32, 16, 8, 2, 1])
    if precision == "fp32":  # the values the FP32 context holds
        ac = [c.astype(np.complex64).astype(np.complex128) for c in ac]
        bc = [c.astype(np.complex64).astype(np.complex128) for c in bc]
    a, b = ctx.tt(ac), ctx.tt(bc)
    tol = 1e-11 if precision == "fp64" else 1e-9
    ref = Q.qtt_tt_dot(ctx, a, b)
    exact = np.vdot(oq.tt_full(ac).reshape(-1), oq.tt_full(bc).reshape(-1))
    assert abs(ref - exact) <= tol * abs(exact)
    for _ in range(2):  # two calls in a row: the shared array keeps old data
        got = Q.qtt_tt_dot_noalloc(ctx, a, b)
        assert abs(got - ref) <= tol * abs(ref)
        assert abs(got - exact) <= tol * abs(exact)
    # self inner product, then a different pair: no state leaks between calls
    assert abs(Q.qtt_tt_dot_noalloc(ctx, a, a) - Q.qtt_tt_dot(ctx, a, a)) <= tol * abs(
        Q.qtt_tt_dot(ctx, a, a))
    ctx.close()


def test_noalloc_dot_rejects_rank_above_limit(Q):
    ctx = Q.Context(0, Q.QTT_FP64, 1 << 28, seed=7)
    rng = np.random.default_rng(12)
    dims = [2] * 8
    big = ctx.tt(random_tt(rng, dims, [1, 2, 4, 8, 16, 65, 4, 2, 1]))
    with pytest.raises(Q.QttError, match="maximum 64"):
        Q.qtt_tt_dot_noalloc(ctx, big, big)
    ctx.close()
