"""Every launch variant the autotuner chooses between gives the same bits: the key inner products
of a hoisted rotate-and-sum, a relinearisation, a rotation and an epoch (tree fan-out included) are
compared across variants, and fhe_autotune keeps exactly one variant per family."""
import numpy as np
import pytest

from paper_2509_03024_gb300 import capi
from paper_2509_03024_gb300 import workloads as W
from tests.gpu_common import ct_slice, gpu_ctx, torch

pytestmark = pytest.mark.gpu

VARIANTS = ["v0", "c1", "p1", "s1", "s2", "s2l"]


@pytest.mark.parametrize("preset", ["t11a2", "paper"])
def test_inner_variants_bit_identical(preset):
    ctx = gpu_ctx(preset, 21, list(range(1, 16)))
    rng = np.random.default_rng(1)
    count = 5                                    # odd: the multi-item variants have a ragged tail
    a, b = ctx.empty_ct(count), ctx.empty_ct(count)
    for t in range(count):
        ctx.encrypt(rng.normal(size=64), ctx.top, 100 + t, ct_slice(ctx, a, t))
        ctx.encrypt(rng.normal(size=64), ctx.top, 200 + t, ct_slice(ctx, b, t))
    ref = {}
    for v in VARIANTS:
        ctx.set_variant("ks_hoist_inner", v)
        ctx.set_variant("ks_inner", v)
        assert ctx.get_variant("ks_inner") == v
        rs, pr, ro = ctx.empty_ct(count), ctx.empty_ct(count), ctx.empty_ct(count)
        ctx.rotate_sum(a.clone(), rs, count, ctx.top - 1, 16)
        ctx.mul_relin_rescale(a, b, pr, count, ctx.top)
        ctx.rotate(a, ro, count, ctx.top, 3)
        torch.cuda.synchronize()
        got = (rs, pr, ro)
        if not ref:
            ref = got
        for name, x, y in zip(("rotate_sum", "mul_relin_rescale", "rotate"), got, ref):
            assert torch.equal(x, y), f"{preset}: variant {v} changes {name}"


def test_epoch_identical_under_every_variant():
    csr = W.uniform_ratings(60, 200, 0.04, 9)
    rng = np.random.default_rng(2)
    k = 10
    U, V = rng.normal(0, 0.1, (csr.n, k)), rng.normal(0, 0.1, (csr.m, k))
    ctx = gpu_ctx("t11a2", 23)
    ctx.add_rotation_keys(ctx.mf_rotation_steps(k))
    plan = capi.MfPlan(ctx, csr.n, csr.m, k, csr.row_ptr, csr.col_idx, csr.vals)
    U0, V0 = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, U0)
    plan.encrypt_factors(1, V, V0)
    ref = None
    for v in ("v0", "s2", "c1", "p1", "s2l"):
        ctx.set_variant("ks_hoist_inner", v)
        ctx.set_variant("ks_inner", v)
        UD, VD = U0.clone(), V0.clone()
        plan.sgd_epoch(UD, VD, ctx.top, 0.01, 0.02)
        torch.cuda.synchronize()
        if ref is None:
            ref = (UD, VD)
        assert torch.equal(UD, ref[0]) and torch.equal(VD, ref[1]), f"variant {v} changes the epoch"


def test_autotune_keeps_one_variant_per_family():
    ctx = gpu_ctx("t11a2", 24)
    res = ctx.autotune()
    fams = {r["family"] for r in res}
    assert fams == {"ks_hoist_inner", "ks_inner"}             # N = 2^11: one-pass NTT, no tile shapes
    for f in fams:
        rows = [r for r in res if r["family"] == f]
        assert sorted(r["variant"] for r in rows) == sorted(VARIANTS)
        chosen = [r for r in rows if r["chosen"]]
        assert len(chosen) == 1 and all(r["ms"] > 0 for r in rows)
        assert chosen[0]["ms"] == min(r["ms"] for r in rows)
        assert ctx.get_variant(f) == chosen[0]["variant"]
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        ctx.set_variant("ks_inner", "nope")


def test_autotune_cache_sets_stored_choices(tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = gpu_ctx("t11a2", 24)
    first = {r["family"]: r["variant"] for r in ctx.autotune(cache=path) if r["chosen"]}
    other = gpu_ctx("t11a2", 25)                              # a fresh context on the same ring
    hit = other.autotune(cache=path)
    assert all(r.get("cached") for r in hit)
    assert {r["family"]: r["variant"] for r in hit} == first
    for f, v in first.items():
        assert other.get_variant(f) == v


@pytest.mark.parametrize("preset", ["paper", "t16a3"])
def test_ntt_tile_shapes_bit_identical(preset):
    """Every tile shape of the two-pass NTT gives the same transform (N = 2^15 and 2^16)."""
    ctx = gpu_ctx(preset, 25)
    L1 = ctx.top + 1
    rng = np.random.default_rng(6)
    a = np.stack([rng.integers(0, q, (3, ctx.n), dtype=np.uint64) for q in ctx.primes[:L1]], axis=1)
    base = torch.from_numpy(a.view(np.int64).copy()).cuda()
    ref = None
    for v in ("r16b4", "r8b4", "r32b4", "r16b3"):
        ctx.set_variant("ntt", v)
        t = base.clone()
        ctx.ntt_forward(t, 3, L1)
        torch.cuda.synchronize()
        if ref is None:
            ref = t.clone()
        assert torch.equal(t, ref), f"tile shape {v} changes the forward transform"
        ctx.ntt_inverse(t, 3, L1)
        torch.cuda.synchronize()
        assert torch.equal(t, base), f"tile shape {v}: inverse does not undo the forward transform"
    res = ctx.autotune()
    rows = [r for r in res if r["family"] == "ntt"]
    assert sorted(r["variant"] for r in rows) == ["r16b3", "r16b4", "r32b4", "r8b4"]
    assert sum(r["chosen"] for r in rows) == 1
    rows = [r for r in res if r["family"] == "ks_pass"]
    assert sorted(r["variant"] for r in rows) == ["r16", "r8", "r8x"] and sum(r["chosen"] for r in rows) == 1


@pytest.mark.parametrize("preset", ["paper", "t16a3"])
def test_ks_pass_tile_shapes_bit_identical(preset):
    """Every tile shape of the fused key-switch / rescale passes gives the same rotation, product and
    rescale (N = 2^15 and 2^16)."""
    ctx = gpu_ctx(preset, 26, [1, 5])
    rng = np.random.default_rng(7)
    count = 3
    a, b = ctx.empty_ct(count), ctx.empty_ct(count)
    for t in range(count):
        ctx.encrypt(rng.normal(size=64), ctx.top, 300 + t, ct_slice(ctx, a, t))
        ctx.encrypt(rng.normal(size=64), ctx.top, 400 + t, ct_slice(ctx, b, t))
    ref = None
    for v in ("r16", "r8", "r8x"):
        ctx.set_variant("ks_pass", v)
        ro, pr, rs = ctx.empty_ct(count), ctx.empty_ct(count), ctx.empty_ct(count)
        ctx.rotate(a, ro, count, ctx.top, 5)
        ctx.mul_relin_rescale(a, b, pr, count, ctx.top)
        ctx.rescale(a, rs, count, ctx.top)
        torch.cuda.synchronize()
        got = (ro, pr, rs)
        if ref is None:
            ref = got
        for name, x, y in zip(("rotate", "mul_relin_rescale", "rescale"), got, ref):
            assert torch.equal(x, y), f"{preset}: tile shape {v} changes {name}"


def test_conv_cost_probe():
    """The conversion-cost probe times both pass sets over the key switch's conversion rows."""
    ctx = gpu_ctx("t11a2", 27)
    lv = ctx.top
    r = ctx.probe_conv_cost(lv, 4)
    l1, a = lv + 1, ctx.alpha
    dn = -(-l1 // a)
    want_rows = 4 * sum(l1 + a - min(a, l1 - j * a) for j in range(dn))
    assert r["rows"] == want_rows and r["roundtrip_bytes"] == 16.0 * want_rows * ctx.n
    assert r["conv_ms"] > 0 and r["plain_ms"] > 0
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        ctx.probe_conv_cost(0, 4)
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        ctx.probe_conv_cost(lv, 0)
