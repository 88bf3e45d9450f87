"""fhe_rescale_noalloc: the rescale for callers that cannot let the library
allocate device memory while they run (an application that manages all device
memory itself, or a latency-critical loop that cannot absorb a cudaMalloc).
It must give exactly the result of the ordinary fhe_rescale, call after call,
although its scratch lives in one static array shared by every call."""
import numpy as np
import pytest

from tests.gpu_common import ct_slice, gpu_ctx, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("preset", ["t11a2", "paper"])
def test_noalloc_rescale_matches_rescale_twice(preset):
    ctx = gpu_ctx(preset, 5)
    rng = np.random.default_rng(3)
    cts = ctx.empty_ct(2)
    for t in range(2):
        ctx.encrypt(rng.normal(size=ctx.slots), ctx.top, 10 + t, ct_slice(ctx, cts, t))
    for t, level in enumerate([ctx.top, ctx.top - 1]):   # two calls in a row, different inputs and levels
        src = ct_slice(ctx, cts, t)
        want = ctx.empty_ct()
        got = ctx.empty_ct()
        ctx.rescale(src, want, 1, level)
        ctx.rescale_noalloc(src, got, level)
        torch.cuda.synchronize()
        lw = (ctx.top + 1) * ctx.n
        for p in range(2):   # limbs 0..level-1 of both components are the result
            a = want[p * lw: p * lw + level * ctx.n]
            b = got[p * lw: p * lw + level * ctx.n]
            assert torch.equal(a, b), f"call {t}: component {p} differs"


def test_noalloc_rescale_rejects_oversized_and_level_zero():
    from paper_2509_03024_gb300.capi import FheError
    ctx = gpu_ctx("large", 5)   # N = 2^16, top level 19: 2 N (level + 1) exceeds the static scratch
    ct, out = ctx.empty_ct(), ctx.empty_ct()
    with pytest.raises(FheError, match="INVALID_ARG"):
        ctx.rescale_noalloc(ct, out, ctx.top)
    with pytest.raises(FheError, match="LEVEL_EXHAUSTED"):
        ctx.rescale_noalloc(ct, out, 0)
    ctx.rescale_noalloc(ct, out, 7)   # within the limit at N = 2^16
