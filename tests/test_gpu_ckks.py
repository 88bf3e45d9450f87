"""GPU parity of the RNS-CKKS primitives against the CPU oracle (bit-exact in coefficient form).

Covers the ring sizes of the single-pass NTT (N = 2^10, 2^13) and of the
two-pass NTT (N = 2^15, 2^16), one and several special primes, every level.
"""
import numpy as np
import pytest

from tests.gpu_common import (assert_ct_equal, ct_slice, gpu_ctx, oracle_ctx, tensor3_to_coeff, to_coeff,
                              torch)
from oracle import ckks

pytestmark = pytest.mark.gpu

SEED = 20250903


def _slots(n, seed, scale=1.0):
    return np.random.default_rng(seed).normal(0, scale, n)


@pytest.mark.parametrize("preset", ["t10", "t11a2", "tiny"])
def test_primes_match_oracle(preset):
    ctx = gpu_ctx(preset, SEED)
    he = oracle_ctx(preset, SEED)
    assert ctx.primes == he.prm.q + he.prm.p


@pytest.mark.parametrize("preset", ["t10", "tiny", "paper", "large"])
def test_ntt_roundtrip_and_product(preset):
    """INTT(NTT(a)) = a at every limb, for single-pass and two-pass rings. (The NTT-domain product is
    checked against the oracle's negacyclic product by test_add_sub_mul_plain_tensor, whose mul_plain
    and tensor go through these transforms.)"""
    ctx = gpu_ctx(preset, SEED)
    n, L1 = ctx.n, ctx.top + 1
    rng = np.random.default_rng(1)
    a = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.primes[:L1]])
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    ctx.ntt_forward(t, 1, L1)
    assert not np.array_equal(t.cpu().numpy().view(np.uint64), a)
    ctx.ntt_inverse(t, 1, L1)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), a)
    # empty batch is a no-op
    ctx.ntt_forward(t, 0, L1)


@pytest.mark.parametrize("preset", ["t10", "t11a2", "tiny", "paper"])
def test_encode_matches_oracle_exactly(preset):
    ctx = gpu_ctx(preset, SEED)
    he = oracle_ctx(preset, SEED)
    for z in (_slots(ctx.slots, 2), _slots(37, 3, 4.0), np.zeros(5), np.array([0.0, 1.5, 0.0, -2.25])):
        out = torch.zeros(ctx.n, dtype=torch.int64, device="cuda")
        ctx.encode(z, out)
        got = out.cpu().numpy()
        want = he.enc.encode(z)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("preset", ["t10", "t11a2", "tiny", "large"])
def test_encrypt_bit_exact_and_decrypt(preset):
    ctx = gpu_ctx(preset, SEED)
    he = oracle_ctx(preset, SEED)
    z = _slots(ctx.slots, 4)
    for level in sorted({ctx.top, 1, 0}):
        ct = ctx.empty_ct()
        ctx.encrypt(z, level, 77 + level, ct)
        ora = he.encrypt(z, level, 77 + level)
        assert_ct_equal(to_coeff(ctx, ct, level)[0], ora, f"encrypt level {level}")
        dec = ctx.decrypt(ct, level)
        tol = 1e-6 if ctx.log_scale >= 40 else 1e-3
        if level >= 1 or ctx.log_scale <= 40:
            assert np.abs(dec - z).max() < tol


@pytest.mark.parametrize("preset", ["t10", "t11a2", "paper"])
def test_add_sub_mul_plain_tensor(preset):
    ctx = gpu_ctx(preset, SEED)
    he = oracle_ctx(preset, SEED)
    L = ctx.top
    x, y = _slots(ctx.slots, 5), _slots(ctx.slots, 6)
    a, b = ctx.empty_ct(2), None
    ctx.encrypt(x, L, 1, ct_slice(ctx, a, 0))
    ctx.encrypt(y, L, 2, ct_slice(ctx, a, 1))
    oa, ob = he.encrypt(x, L, 1), he.encrypt(y, L, 2)
    A, B = ct_slice(ctx, a, 0), ct_slice(ctx, a, 1)
    for level in (L, 1):
        out = ctx.empty_ct()
        ctx.add(A, B, out, 1, level)
        assert_ct_equal(to_coeff(ctx, out, level)[0], he.add(he.drop(oa, level), he.drop(ob, level)), "add")
        ctx.sub(A, B, out, 1, level)
        assert_ct_equal(to_coeff(ctx, out, level)[0], he.sub(he.drop(oa, level), he.drop(ob, level)), "sub")
        pt = torch.zeros(ctx.n, dtype=torch.int64, device="cuda")
        zp = _slots(ctx.slots, 7)
        ctx.encode(zp, pt)
        ctx.mul_plain(A, pt, out, 1, level)
        assert_ct_equal(to_coeff(ctx, out, level)[0], he.mul_plain(he.drop(oa, level), he.enc.encode(zp)),
                        "mul_plain")
        t3 = ctx.empty_ct(1, parts=3)
        ctx.tensor(A, B, t3, 1, level)
        assert_ct_equal(tensor3_to_coeff(ctx, t3, level), he.tensor(he.drop(oa, level), he.drop(ob, level)),
                        "tensor")
    # several ciphertexts in one call
    out2 = ctx.empty_ct(2)
    ctx.add(a, a, out2, 2, L)
    got = to_coeff(ctx, out2, L, 2)
    assert_ct_equal(got[0], he.add(oa, oa), "batched add 0")
    assert_ct_equal(got[1], he.add(ob, ob), "batched add 1")


@pytest.mark.parametrize("preset", ["t10", "t11a2", "tiny", "paper"])
def test_rescale_relin_mul_bit_exact(preset):
    ctx = gpu_ctx(preset, SEED)
    he = oracle_ctx(preset, SEED)
    L = ctx.top
    x, y = _slots(ctx.slots, 8), _slots(ctx.slots, 9)
    a = ctx.empty_ct(2)
    ctx.encrypt(x, L, 11, ct_slice(ctx, a, 0))
    ctx.encrypt(y, L, 12, ct_slice(ctx, a, 1))
    oa, ob = he.encrypt(x, L, 11), he.encrypt(y, L, 12)
    A, B = ct_slice(ctx, a, 0), ct_slice(ctx, a, 1)
    levels = [L] if preset == "paper" else sorted({L, 1})
    for level in levels:
        out = ctx.empty_ct()
        ctx.rescale(A, out, 1, level)
        assert_ct_equal(to_coeff(ctx, out, level - 1)[0], he.rescale(he.drop(oa, level)), "rescale")
        t3 = ctx.empty_ct(1, parts=3)
        ctx.tensor(A, B, t3, 1, level)
        ctx.relinearize(t3, out, 1, level)
        relin = he.relinearize(he.tensor(he.drop(oa, level), he.drop(ob, level)))
        assert_ct_equal(to_coeff(ctx, out, level)[0], relin, "relinearize")
        ctx.mul_relin_rescale(A, B, out, 1, level)
        prod = he.relin_rescale(he.tensor(he.drop(oa, level), he.drop(ob, level)))
        assert_ct_equal(to_coeff(ctx, out, level - 1)[0], prod, "mul_relin_rescale (fused)")
        dec = ctx.decrypt(out, level - 1)
        assert np.abs(dec - x * y).max() < 1e-4


@pytest.mark.parametrize("preset,steps", [("t10", [1, -1, 5, 64]), ("t11a2", [3, -8]), ("tiny", [1, -16]),
                                          ("paper", [32])])
def test_rotate_bit_exact(preset, steps):
    ctx = gpu_ctx(preset, SEED, steps)
    he = oracle_ctx(preset, SEED, steps)
    L = ctx.top
    x = _slots(ctx.slots, 10)
    a = ctx.empty_ct()
    ctx.encrypt(x, L, 21, a)
    oa = he.encrypt(x, L, 21)
    for r in steps:
        for level in sorted({L, 0 if preset != "paper" else L}):
            out = ctx.empty_ct()
            ctx.rotate(a, out, 1, level, r)
            assert_ct_equal(to_coeff(ctx, out, level)[0], he.rotate(he.drop(oa, level), r), f"rotate {r}")
        dec = ctx.decrypt(out, level)
        if level >= 1:
            assert np.abs(dec - np.roll(x, -r)).max() < 1e-5
    # rotation by the slot count is the identity and needs no key
    out = ctx.empty_ct()
    ctx.rotate(a, out, 1, L, ctx.slots)
    assert_ct_equal(to_coeff(ctx, out, L)[0], oa, "rotate by N/2")


@pytest.mark.parametrize("preset,kp,level_off", [("t10", 4, 0), ("t10", 16, 1), ("t11a2", 3, 0), ("t11a2", 8, 2),
                                                  ("t11a2", 32, 0), ("paper", 16, 1)])
def test_rotate_sum_bit_exact(preset, kp, level_off):
    """sum_{r < kp} rot(ct, r) over two ciphertexts: hoisted for kp <= 16, rotate-and-adds above."""
    from oracle import mf
    steps = mf.rotsum_steps(kp)
    ctx = gpu_ctx(preset, SEED, steps)
    he = oracle_ctx(preset, SEED, steps)
    level = ctx.top - level_off
    xs = [_slots(ctx.slots, 40 + i) for i in range(2)]
    a = ctx.empty_ct(2)
    for i, x in enumerate(xs):
        ctx.encrypt(x, ctx.top, 50 + i, ct_slice(ctx, a, i))
    want = [mf.block_sum(he, he.drop(he.encrypt(x, he.prm.top, 50 + i), level), kp) for i, x in enumerate(xs)]
    out = ctx.empty_ct(2)
    keep = a.clone()
    ctx.rotate_sum(a, out, 2, level, kp)
    got = to_coeff(ctx, out, level, 2)
    for i in range(2):
        assert_ct_equal(got[i], want[i], f"rotate_sum kp={kp} item {i}")
        dec = ctx.decrypt(ct_slice(ctx, out, i), level)
        ref = sum(np.roll(xs[i], -r) for r in range(kp))
        assert np.abs(dec - ref).max() < 1e-4
    if kp <= 16:   # in place gives the same bits
        ctx.rotate_sum(keep, keep, 2, level, kp)
        assert (to_coeff(ctx, keep, level, 2) == got).all()


@pytest.mark.parametrize("preset,level_off", [("t10", 0), ("t11a2", 1)])
def test_rotate_fanin_bit_exact(preset, level_off):
    """acc_g += sum_i rot(ct_i, s_i) with one ModDown per group; groups of 3, 1, 0 and 4 children."""
    steps = [1, -3, 5, 2, -1, 7, 1, -3]
    first = [0, 3, 4, 4, 8]
    keys = sorted(set(steps))
    ctx = gpu_ctx(preset, SEED, keys)
    he = oracle_ctx(preset, SEED, keys)
    level = ctx.top - level_off
    G, C = len(first) - 1, len(steps)
    xs = [_slots(ctx.slots, 70 + i) for i in range(G + C)]
    acc, ch = ctx.empty_ct(G), ctx.empty_ct(C)
    for i, x in enumerate(xs):
        ctx.encrypt(x, ctx.top, 300 + i, ct_slice(ctx, acc, i) if i < G else ct_slice(ctx, ch, i - G))
    o = [he.drop(he.encrypt(x, he.prm.top, 300 + i), level) for i, x in enumerate(xs)]
    ctx.rotate_fanin(acc, first, ch, steps, level)
    got = to_coeff(ctx, acc, level, G)
    for g in range(G):
        kids = range(first[g], first[g + 1])
        want = o[g]
        if len(kids):
            want = he.add(want, he.rotate_fanin([o[G + i] for i in kids], [steps[i] for i in kids]))
        assert_ct_equal(got[g], want, f"fan-in group {g}")
        dec = ctx.decrypt(ct_slice(ctx, acc, g), level)
        ref = xs[g] + sum((np.roll(xs[G + i], -steps[i]) for i in kids), np.zeros(ctx.slots))
        assert np.abs(dec - ref).max() < 1e-4


def test_rotate_fanin_group_across_sub_batches():
    """A group whose children span two key-switch sub-batches (about 54 children of a top-level
    N = 2^16, 20 + 3 prime ciphertext fit the 6 GiB work area): the second sub-batch adds to the
    first one's group sums. Checked by decryption against the sum of rotated slot vectors."""
    steps_set = [1, 2, 3, -1, 5, 7, -4, 9]
    ctx = gpu_ctx("large", SEED, steps_set)
    level = ctx.top
    first = [0, 70, 73]
    steps = [steps_set[i % len(steps_set)] for i in range(first[-1])]
    G, C = len(first) - 1, first[-1]
    xs = [_slots(ctx.slots, 500 + i) for i in range(G + C)]
    acc, ch = ctx.empty_ct(G), ctx.empty_ct(C)
    for i, x in enumerate(xs):
        ctx.encrypt(x, level, 900 + i, ct_slice(ctx, acc, i) if i < G else ct_slice(ctx, ch, i - G))
    ctx.rotate_fanin(acc, first, ch, steps, level)
    for g in range(G):
        ref = xs[g] + sum(np.roll(xs[G + i], -steps[i]) for i in range(first[g], first[g + 1]))
        dec = ctx.decrypt(ct_slice(ctx, acc, g), level)
        assert np.abs(dec - ref).max() < 1e-4, f"group {g}"


def test_errors_are_reported_and_context_survives():
    ctx = gpu_ctx("t10", SEED, [1])
    from paper_2509_03024_gb300.capi import FheError
    a = ctx.empty_ct()
    ctx.encrypt(_slots(ctx.slots, 1), ctx.top, 1, a)
    out = ctx.empty_ct()
    with pytest.raises(FheError, match="MISSING_KEY"):
        ctx.rotate(a, out, 1, ctx.top, 2)
    with pytest.raises(FheError, match="LEVEL_EXHAUSTED"):
        ctx.rescale(a, out, 1, 0)
    with pytest.raises(FheError, match="INVALID_ARG"):
        ctx.add(a, a, out, 1, ctx.top + 1)
    with pytest.raises(FheError, match="INVALID_ARG"):
        ctx.rotate(a, a, 1, ctx.top, 1)
    # still usable
    ctx.rotate(a, out, 1, ctx.top, 1)
    assert np.abs(ctx.decrypt(out, ctx.top) - np.roll(_slots(ctx.slots, 1), -1)).max() < 1e-5


def test_key_switches_bit_exact_at_n_2_16():
    """The N = 2^16 instantiations of the fused key-switch passes (the ring of the batched, served and
    large workloads) with three special primes and a one-limb last digit at the top level: rotation
    both ways, the fused product, the rescale and the hoisted rotate-and-sum at kp = 16 (the block of
    the k = 16 workloads) at two levels, bit for bit. Sparse slot vectors keep the oracle's encoding
    short."""
    from oracle import mf
    steps = mf.rotsum_steps(16) + [32, -32]
    ctx = gpu_ctx("t16a3", SEED, steps)
    he = oracle_ctx("t16a3", SEED, steps)
    L = ctx.top
    xs = []
    for i in range(2):
        rng = np.random.default_rng(60 + i)
        x = np.zeros(ctx.slots)
        x[rng.choice(ctx.slots, 64, replace=False)] = rng.uniform(-1, 1, 64)
        xs.append(x)
    a = ctx.empty_ct(2)
    for i, x in enumerate(xs):
        ctx.encrypt(x, L, 70 + i, ct_slice(ctx, a, i))
    oa = [he.encrypt(x, L, 70 + i) for i, x in enumerate(xs)]
    A, B = ct_slice(ctx, a, 0), ct_slice(ctx, a, 1)
    assert_ct_equal(to_coeff(ctx, A, L)[0], oa[0], "encrypt")
    out = ctx.empty_ct()
    for r in (32, -32):
        ctx.rotate(A, out, 1, L, r)
        assert_ct_equal(to_coeff(ctx, out, L)[0], he.rotate(oa[0], r), f"rotate {r}")
    ctx.mul_relin_rescale(A, B, out, 1, L)
    assert_ct_equal(to_coeff(ctx, out, L - 1)[0], he.relin_rescale(he.tensor(oa[0], oa[1])), "fused product")
    assert np.abs(ctx.decrypt(out, L - 1) - xs[0] * xs[1]).max() < 1e-4
    ctx.rescale(A, out, 1, L)
    assert_ct_equal(to_coeff(ctx, out, L - 1)[0], he.rescale(oa[0]), "rescale")
    ref = sum(np.roll(xs[0], -r) for r in range(16))
    for level in (L, L - 1):
        src = A.clone()
        ctx.rotate_sum(src, out, 1, level, 16)
        assert_ct_equal(to_coeff(ctx, out, level)[0], mf.block_sum(he, he.drop(oa[0], level), 16),
                        f"rotate_sum kp=16 at level {level}")
        assert np.abs(ctx.decrypt(out, level) - ref).max() < 1e-4
