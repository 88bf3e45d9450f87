"""fhe_rescale_noalloc: the rescale for callers that cannot let the library
allocate device memory while they run (an application that manages all device
memory itself, or a latency-critical loop that cannot absorb a cudaMalloc).
It must give exactly the result of the ordinary fhe_rescale, call after call,
although its scratch lives in one static array shared by every call, and it
must leave the device's free memory unchanged."""
import numpy as np
import pytest

from tests.gpu_common import ct_slice, gpu_ctx, torch

pytestmark = pytest.mark.gpu


def _same_result(ctx, src, got, level):
    want = ctx.empty_ct()
    ctx.rescale(src, want, 1, level)
    torch.cuda.synchronize()
    lw = (ctx.top + 1) * ctx.n
    for p in range(2):   # limbs 0..level-1 of both components are the result
        a = want[p * lw: p * lw + level * ctx.n]
        b = got[p * lw: p * lw + level * ctx.n]
        assert torch.equal(a, b), f"level {level}: component {p} differs"


@pytest.mark.parametrize("preset", ["t11a2", "paper"])
def test_noalloc_rescale_matches_rescale_twice(preset):
    ctx = gpu_ctx(preset, 5)
    rng = np.random.default_rng(3)
    cts = ctx.empty_ct(2)
    for t in range(2):
        ctx.encrypt(rng.normal(size=ctx.slots), ctx.top, 10 + t, ct_slice(ctx, cts, t))
    outs = [ctx.empty_ct(), ctx.empty_ct()]
    levels = [ctx.top, ctx.top - 1]
    for t in range(2):   # two calls in a row, different inputs and levels
        ctx.rescale_noalloc(ct_slice(ctx, cts, t), outs[t], levels[t])
    torch.cuda.synchronize()
    for t in range(2):
        _same_result(ctx, ct_slice(ctx, cts, t), outs[t], levels[t])


def test_noalloc_rescale_leaves_device_memory_unchanged():
    """A context that never ran the ordinary rescale: after one warm-up call (which looks up the
    scratch array's address), further calls change neither the device's free memory nor torch's."""
    ctx = gpu_ctx("paper", 6)
    rng = np.random.default_rng(4)
    src, out = ctx.empty_ct(), ctx.empty_ct()
    ctx.encrypt(rng.normal(size=ctx.slots), ctx.top, 3, src)
    ctx.rescale_noalloc(src, out, ctx.top)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for level in (ctx.top, ctx.top - 1, 3, 1, ctx.top):
        ctx.rescale_noalloc(src, out, level)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == alloc0
    _same_result(ctx, src, out, ctx.top)


def test_noalloc_rescale_size_limit_is_exact():
    """At N = 2^16 the 2^21-word scratch holds 2 N (level + 1) words up to level 15: level 15 runs
    and equals fhe_rescale, level 16 is refused; level 0 has nothing to rescale."""
    from paper_2509_03024_gb300.capi import FheError
    ctx = gpu_ctx("large", 5)   # N = 2^16, top level 19
    rng = np.random.default_rng(5)
    ct, out = ctx.empty_ct(), ctx.empty_ct()
    ctx.encrypt(rng.normal(size=64), ctx.top, 9, ct)
    with pytest.raises(FheError, match="INVALID_ARG"):
        ctx.rescale_noalloc(ct, out, 16)
    with pytest.raises(FheError, match="INVALID_ARG"):
        ctx.rescale_noalloc(ct, out, ctx.top)
    with pytest.raises(FheError, match="LEVEL_EXHAUSTED"):
        ctx.rescale_noalloc(ct, out, 0)
    ctx.rescale_noalloc(ct, out, 15)
    torch.cuda.synchronize()
    _same_result(ctx, ct, out, 15)
