"""Pins of the oracle's served fold-in + predict (CPU)."""
import numpy as np

from oracle import ckks, mf, serve


def test_fold_in_fp64_hand_checked():
    V = np.array([[1.0, 0.0], [0.0, 2.0], [1.0, 1.0]])
    u0 = np.array([0.5, 0.0])
    items, ratings = [0, 1], [1.0, 2.0]
    # e = (1 - 0.5, 2 - 0) = (0.5, 2); u <- u (1 - .1 * .5 * 2) + .1 (0.5 v0 + 2 v1) = (0.45, 0) + (0.05, 0.4)
    u, pred = serve.fold_in_fp64(u0, V, items, ratings, 1, 0.1, 0.5)
    assert np.allclose(u, [0.5, 0.4], atol=1e-15)
    assert np.allclose(pred, V @ np.array([0.5, 0.4]), atol=1e-15)


def test_fold_in_fp64_is_the_mf_user_update_with_items_fixed():
    rng = np.random.default_rng(1)
    V = rng.normal(size=(9, 3))
    u0 = rng.normal(size=3)
    items = np.array([1, 4, 7])
    ratings = np.array([3.0, 5.0, 1.0])
    u, _ = serve.fold_in_fp64(u0, V, items, ratings, 1, 0.05, 0.1)
    U2, _ = mf.mf_epoch_fp64(u0[None], V, [0, 0, 0], items, ratings, 0.05, 0.1)
    assert np.allclose(u, U2[0], atol=1e-14)


def test_encrypted_request_matches_fp64():
    prm = ckks.Params(9, (50,) * 8, (60, 60), 50)
    he = ckks.Ckks(prm)
    k, m = 3, 90
    kp, w, B = serve.layout(k, prm.slots)
    n_vb = -(-m // B)
    steps = serve.rotation_steps(k, prm.slots)
    rounds = serve.block_sum_rounds(k, prm.slots)
    assert sorted(steps) == sorted({1, 2, 3} | {x for r in rounds for x in r if x != 0})
    he.keygen(3, steps)
    rng = np.random.default_rng(2)
    V = rng.normal(0, 0.3, (m, k))
    dummy = mf.build_plan(1, m, k, [0], [0], [1.0], prm.slots)
    VD = [he.encrypt(mf.pack_factors(V, dummy, c), prm.top, 1000 + c) for c in range(n_vb)]
    items = np.sort(rng.choice(m, 12, replace=False))
    ratings = rng.integers(1, 6, 12).astype(float)
    u0 = rng.normal(0, 0.1, k)
    UR, R = serve.encrypt_request(he, u0, items, ratings, k, n_vb, 77)
    Uf, P = serve.serve_request(he, UR, R, VD, items, k, 3, 0.05, 0.02)
    assert Uf.level == prm.top - 6 and P[0].level == prm.top - 7
    u_ref, pred_ref = serve.fold_in_fp64(u0, V, items, ratings, 3, 0.05, 0.02)
    z = he.decrypt(Uf)
    for a in (0, B // 2, B - 1):   # every block holds the doubled user vector
        assert np.abs(z[a * w: a * w + k] - u_ref).max() < 1e-6
        assert np.abs(z[a * w + kp: a * w + kp + k] - u_ref).max() < 1e-6
    pred = np.concatenate([he.decrypt(P[c])[::w][:B] for c in range(n_vb)])[:m]
    assert np.abs(pred - pred_ref).max() < 1e-6


def test_row_layout_hand_example():
    """The served request's ROW layout written out by hand for k = 3 (kp = 4, w = 8) in 32 slots
    (B = 4 blocks): u in every block, twice; item j = 4c + d rated in block d of batch c; the mask
    on the first k slots of the rated blocks; the rotation amounts of a step."""
    u = np.array([1.0, 2.0, 3.0])
    z = serve.replicate_user(u, 3, 32)
    want = np.zeros(32)
    for a in range(4):
        want[8 * a: 8 * a + 3] = want[8 * a + 4: 8 * a + 7] = u
    assert np.array_equal(z, want)
    items, ratings = [1, 6, 7], [4.0, 2.0, 5.0]        # item 1: batch 0 block 1; items 6, 7: batch 1 blocks 2, 3
    R = serve.rating_batches(items, ratings, 3, 32, 2)
    want0, want1 = np.zeros(32), np.zeros(32)
    want0[8:11] = 4.0
    want1[16:19], want1[24:27] = 2.0, 5.0
    assert np.array_equal(R[0], want0) and np.array_equal(R[1], want1)
    assert serve.rated_batches(items, 3, 32) == [0, 1]
    m1 = serve.mask_batch(items, 1, 3, 32, 0.5)
    want = np.zeros(32)
    want[16:19] = want[24:27] = 0.5
    assert np.array_equal(m1, want)
    # in-block sums by 1, 2, 3 (hoisted, kp = 4); B = 4 blocks: one radix-4 round over the block
    # offsets 0, 8, 16, 24 with the half-fill by -4 merged into it
    assert serve.block_sum_rounds(3, 32) == [[0, 8, 16, 24, -4, 4, 12, 20]]
    assert serve.rotation_steps(3, 32) == [1, 2, 3, 8, 16, 24, -4, 4, 12, 20]


def test_block_sum_rounds_cover_every_block_once():
    """One step per round, summed, hits every block offset a*w (a < B) exactly once, and every one of
    them again shifted by the half-fill -kp: the rounds are the block sum followed by the half-fill."""
    from collections import Counter
    from itertools import product
    for k, slots in ((3, 32), (3, 64), (16, 1 << 15), (1, 1 << 9), (10, 1 << 14), (8, 16)):
        kp, w, B = serve.layout(k, slots)
        rounds = serve.block_sum_rounds(k, slots)
        sums = Counter(sum(c) % slots for c in product(*rounds))
        want = Counter([(a * w) % slots for a in range(B)] + [(a * w - kp) % slots for a in range(B)])
        assert sums == want, (k, slots)
        assert all(len(r) in (2, 4) for r in rounds[:-1]) and len(rounds[-1]) in (2, 4, 8)
        assert len(rounds) == max(1, (mf.highest_bit(B) + 1) // 2)


def test_hoisted_block_sum_rounds_equal_the_doubling_sums():
    """Decrypted, the hoisted rounds give the block sum and half-fill of the doubling definition
    G + rot(G, 2^t w) (t < log2 B) followed by G + rot(G, -kp), within the key-switch noise."""
    prm = ckks.Params(9, (50,) * 4, (60,), 40)
    he = ckks.Ckks(prm)
    k = 3
    kp, w, B = serve.layout(k, prm.slots)
    doubling = [(1 << t) * w for t in range(mf.highest_bit(B))] + [-kp]
    he.keygen(5, sorted(set(serve.rotation_steps(k, prm.slots) + doubling)))
    z = np.random.default_rng(4).normal(0, 1, prm.slots)
    G = he.encrypt(z, prm.top, 9)
    H = G
    for steps in serve.block_sum_rounds(k, prm.slots):
        H = he.rotate_sum_hoisted(H, steps)
    D = G
    for s in doubling:
        D = he.add(D, he.rotate(D, s))
    want = sum(np.roll(z, -a * w) for a in range(B))
    want = want + np.roll(want, kp)
    assert np.abs(he.decrypt(D) - want).max() < 1e-6
    assert np.abs(he.decrypt(H) - want).max() < 1e-6
