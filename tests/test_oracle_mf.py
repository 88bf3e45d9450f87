"""Pins of the oracle MF: the paper's batch-pair example, FP64 update algebra, plan, encrypted epoch."""
import json
import os

import numpy as np
import pytest

from oracle import ckks, mf
from paper_2509_03024_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_batch_pair_example_from_paper():
    g = json.load(open(os.path.join(GOLD, "batch_pairs.json")))
    rows = [r for r, _ in g["ratings"]]
    cols = [c for _, c in g["ratings"]]
    pairs = mf.batch_pairs(rows, cols, g["batch_size"])
    counts = {f"{b},{c}": len(v) for (b, c), v in pairs.items()}
    assert counts == g["pair_counts"]
    local0 = [i % g["batch_size"] for i, _ in pairs[(0, 0)]].count(0)
    assert local0 == g["user_local_0_count_in_pair_0_0"]


def test_plan_groups_partition_ratings():
    csr, _, _ = W.tiny_workload(3)
    rows, cols, vals = csr.triples()
    for slots in (512, 4096):
        plan = mf.build_plan(csr.n, csr.m, 4, rows, cols, vals, slots)
        seen = set()
        for g in plan.groups:
            assert len(set(g.a.tolist())) == len(g.a)  # one rating per block per group
            for a in g.a.tolist():
                i = g.b * plan.B + a
                j = g.c * plan.B + (a + g.delta) % plan.B
                assert (i, j) not in seen
                seen.add((i, j))
        assert seen == set(zip(rows.tolist(), cols.tolist()))
        assert len(plan.groups) <= plan.n_ub * plan.n_vb * plan.B
        # the groups refine the paper's batch pairs
        pairs = mf.batch_pairs(rows, cols, plan.B)
        for (b, c), lst in pairs.items():
            assert sum(len(g.a) for g in plan.groups if g.b == b and g.c == c) == len(lst)
        for c, nodes in enumerate(plan.closure):
            for d in nodes:
                assert d == 0 or mf.tree_parent(d, plan.baby)[0] in nodes


def test_fp64_epoch_hand_checked_2x2():
    U = np.array([[1.0, 0.0], [0.0, 1.0]])
    V = np.array([[1.0, 1.0], [2.0, 0.0]])
    rows, cols, vals = [0, 0, 1], [0, 1, 0], [3.0, 1.0, 2.0]
    lr, lam = 0.1, 0.5
    # e00 = 3 - 1 = 2; e01 = 1 - 2 = -1; e10 = 2 - 1 = 1
    # u0 <- u0 (1 - .1*.5*2) + .1 (2 v0 - 1 v1) = (0.9, 0) + .1 (0, 2) = (0.9, 0.2)
    # u1 <- u1 (1 - .05) + .1 (1 v0) = (0, .95) + (.1, .1) = (0.1, 1.05)
    # v0 <- v0 (1 - .1) + .1 (2 u0 + 1 u1) = (.9, .9) + (.2, .1) = (1.1, 1.0)
    # v1 <- v1 (1 - .05) + .1 (-1 u0) = (1.9, 0) + (-.1, 0) = (1.8, 0)
    U2, V2 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    assert np.allclose(U2, [[0.9, 0.2], [0.1, 1.05]], atol=1e-15)
    assert np.allclose(V2, [[1.1, 1.0], [1.8, 0.0]], atol=1e-15)
    # RMSE, Eq. 10
    assert abs(mf.rmse(U, V, rows, cols, vals) - np.sqrt((4 + 1 + 1) / 3)) < 1e-15


def test_fp64_epoch_equals_per_rating_accumulation():
    """Alg. 2 with the accumulators applied once: the sum of per-rating Alg. 1 gradients."""
    rng = np.random.default_rng(0)
    n, m, k = 7, 5, 3
    U, V = rng.normal(size=(n, k)), rng.normal(size=(m, k))
    pairs = [(i, j) for i in range(n) for j in range(m) if rng.random() < 0.5]
    rows = [p[0] for p in pairs]; cols = [p[1] for p in pairs]
    vals = rng.integers(1, 6, size=len(pairs)).astype(float)
    lr, lam = 0.05, 0.1
    accU, accV = np.zeros_like(U), np.zeros_like(V)
    for (i, j), r in zip(pairs, vals):
        e = r - U[i] @ V[j]
        accU[i] += lr * (e * V[j] - lam * U[i])
        accV[j] += lr * (e * U[i] - lam * V[j])
    U2, V2 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    assert np.allclose(U2, U + accU, atol=1e-12) and np.allclose(V2, V + accV, atol=1e-12)


@pytest.mark.parametrize("slots,k", [(512, 4), (4096, 4), (512, 3), (1024, 10), (256, 1)])
def test_simulated_plan_equals_fp64(slots, k):
    rng = np.random.default_rng(slots + k)
    csr = W.uniform_ratings(150, 110, 0.05, slots)
    rows, cols, vals = csr.triples()
    U, V = rng.normal(0, 0.1, (csr.n, k)), rng.normal(0, 0.1, (csr.m, k))
    plan = mf.build_plan(csr.n, csr.m, k, rows, cols, vals, slots)
    Us, Vs = mf.simulate_epoch_slots(U, V, plan, 0.01, 0.02)
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, 0.01, 0.02)
    assert np.abs(Us - U1).max() < 1e-12 and np.abs(Vs - V1).max() < 1e-12


def _small_he(log_n=9, data=(60, 40, 40), special=(60,), ls=40, seed=5, steps=()):
    he = ckks.Ckks(ckks.Params(log_n, data, special, ls))
    he.keygen(seed, steps)
    return he


def test_encrypted_epoch_matches_fp64():
    csr = W.uniform_ratings(40, 30, 0.08, 4)
    rows, cols, vals = csr.triples()
    rng = np.random.default_rng(1)
    U, V = rng.normal(0, 0.1, (csr.n, 4)), rng.normal(0, 0.1, (csr.m, 4))
    he = ckks.Ckks(ckks.Params(9, (60, 40, 40), (60,), 40))
    plan = mf.build_plan(csr.n, csr.m, 4, rows, cols, vals, he.prm.slots)
    he.keygen(5, plan.rotation_steps())
    emf = mf.EncryptedMF(he, plan)
    emf.encrypt_ratings()
    UD, VD = emf.encrypt_factors(U, V)
    U2, V2 = emf.epoch(UD, VD, 0.01, 0.02)
    assert U2[0].level == he.prm.top - 2
    Ud, Vd = emf.decrypt_factors(U2, V2)
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, 0.01, 0.02)
    assert np.abs(Ud - U1).max() < 1e-3 and np.abs(Vd - V1).max() < 1e-3
    # the reachable accuracy at 40-bit scale is far below the 1e-3 bar
    assert np.abs(Ud - U1).max() < 1e-6


def test_encrypted_epoch_group_order_independent():
    """Modular accumulation is order-free: permuting the group order gives identical ciphertexts."""
    csr = W.uniform_ratings(24, 20, 0.1, 6)
    rows, cols, vals = csr.triples()
    rng = np.random.default_rng(2)
    U, V = rng.normal(0, 0.1, (csr.n, 2)), rng.normal(0, 0.1, (csr.m, 2))
    he = ckks.Ckks(ckks.Params(7, (60, 40, 40), (60,), 40))
    plan = mf.build_plan(csr.n, csr.m, 2, rows, cols, vals, he.prm.slots)
    he.keygen(8, plan.rotation_steps())
    emf = mf.EncryptedMF(he, plan)
    emf.encrypt_ratings()
    UD, VD = emf.encrypt_factors(U, V)
    U2, V2 = emf.epoch(UD, VD, 0.01, 0.02)
    perm = np.random.default_rng(3).permutation(len(plan.groups))
    plan.groups = [plan.groups[t] for t in perm]
    plan.bin_of = [plan.bin_of[t] for t in perm]   # the bins (and R) stay; each group keeps its bin
    U3, V3 = emf.epoch(UD, VD, 0.01, 0.02)
    for a, b in zip(U2 + V2, U3 + V3):
        assert (a.c == b.c).all()


def test_rating_bins_first_fit_hand_example():
    """B = 4 user blocks, one item batch; groups (delta order) with user sets {0,1}, {2}, {1,2}, {3}:
    first fit puts them in bins 0, 0, 1, 0."""
    # delta = (d - a) mod B: ratings (a, d) -> delta 0: (0,0),(1,1); 1: (2,3); 2: (1,3),(2,0); 3: (3,2)
    rows = [0, 1, 2, 1, 2, 3]
    cols = [0, 1, 3, 3, 0, 2]
    plan = mf.build_plan(4, 4, 1, rows, cols, [1.0] * 6, slots=8)   # k = 1: w = 2, B = 4
    assert plan.B == 4
    assert [(g.delta, g.a.tolist()) for g in plan.groups] == [(0, [0, 1]), (1, [2]), (2, [1, 2]), (3, [3])]
    assert plan.bin_of == [0, 0, 1, 0] and plan.bin_batch == [0, 0]


def test_rating_bins_invariants():
    """Every group lies in one bin; a bin holds each user block at most once; bins per user batch
    are at least the most ratings of one user (every rating of a user needs its own bin)."""
    train, _, _, _ = W.paper_workload(seed=2)
    rows, cols, vals = train.triples()
    plan = mf.build_plan(train.n, train.m, 10, rows, cols, vals, 1 << 14)
    assert len(plan.bin_of) == len(plan.groups)
    for t in range(len(plan.bin_batch)):
        users = [a for g, bt in zip(plan.groups, plan.bin_of) if bt == t for a in g.a.tolist()]
        assert len(users) == len(set(users))
        assert all(plan.groups[i].b == plan.bin_batch[t] for i, bt in enumerate(plan.bin_of) if bt == t)
    for b in range(plan.n_ub):
        nb = sum(1 for x in plan.bin_batch if x == b)
        lb = int(plan.nnz_u[b * plan.B:(b + 1) * plan.B].max())
        assert lb <= nb <= 2 * lb
    # the bin slot vectors carry every rating exactly once
    total = sum(mf.bin_slots(t, plan).sum() for t in range(len(plan.bin_batch)))
    assert abs(total - plan.k * vals.sum()) < 1e-6


def test_slot_layouts_hand_example():
    """The doubled-block layout (Sec. III-C's u_L0 || ... || u_Lk-1 padded to kp and written twice),
    the rating, mask and regulariser slot vectors, written out by hand for k = 3 (kp = 4, w = 8) in
    a ring of 32 slots (B = 4 entities per batch)."""
    rows, cols, vals = [0, 0, 5], [1, 2, 1], [4.0, 2.0, 5.0]     # users 0, 0, 5; items 1, 2, 1
    plan = mf.build_plan(6, 3, 3, rows, cols, vals, 32)
    assert (plan.kp, plan.w, plan.B, plan.n_ub, plan.n_vb) == (4, 8, 4, 2, 1)
    X = np.arange(1.0, 19.0).reshape(6, 3)                        # entity e holds 3e+1, 3e+2, 3e+3
    z = mf.pack_factors(X, plan, 1)                               # entities 4, 5 in blocks 0, 1
    want = np.zeros(32)
    want[0:3] = want[4:7] = [13, 14, 15]
    want[8:11] = want[12:15] = [16, 17, 18]
    assert np.array_equal(z, want)
    # group (b=0, c=0, delta=1): user 0 (a=0) rated item 1 (d=1); its rating sits in user 0's block
    g = next(g for g in plan.groups if (g.b, g.c, g.delta) == (0, 0, 1))
    assert g.a.tolist() == [0]
    r = mf.rating_slots(g, plan)
    want = np.zeros(32)
    want[0:3] = 4.0
    assert np.array_equal(r, want)
    m = mf.mask_slots(g, plan, 0.5)
    want = np.zeros(32)
    want[0:3] = 0.5
    assert np.array_equal(m, want)
    # regulariser of user batch 0: user 0 has 2 ratings, users 1-3 none
    reg = mf.reg_slots(plan.nnz_u, plan, 0, 0.1, 0.5)
    want = np.ones(32)
    want[0:8] = 1.0 - 0.1 * 0.5 * 2
    assert np.array_equal(reg, want)
    # user batch 1 holds users 4, 5 then two empty blocks (no entity: regulariser 1, factors 0)
    reg1 = mf.reg_slots(plan.nnz_u, plan, 1, 0.1, 0.5)
    assert np.array_equal(reg1[8:16], np.full(8, 1.0 - 0.05)) and np.array_equal(reg1[16:], np.ones(16))


def test_encrypted_predict_matches_fp64_row():
    """EncryptedMF.predict (the encrypted row of R-hat = U V^T, Alg. 1) decrypts to u_user . v_j for
    every item j of every item batch. The user sits in the second user batch at a block other than 0,
    and there are two item batches, so a mask on the wrong block, a missing replication round (some
    blocks left empty) or a swapped batch index all change the row. (The replication sums all B
    cyclic shifts of the masked block, so its rotation direction does not change the values.)"""
    n, m, k = 40, 50, 4
    csr = W.uniform_ratings(n, m, 0.08, 11)
    rows, cols, vals = csr.triples()
    rng = np.random.default_rng(12)
    U, V = rng.normal(0, 0.3, (n, k)), rng.normal(0, 0.3, (m, k))
    he = ckks.Ckks(ckks.Params(9, (60, 40, 40), (60,), 40))
    plan = mf.build_plan(n, m, k, rows, cols, vals, he.prm.slots)
    assert (plan.B, plan.n_ub, plan.n_vb) == (32, 2, 2)
    he.keygen(13, plan.rotation_steps())
    emf = mf.EncryptedMF(he, plan)
    UD, VD = emf.encrypt_factors(U, V)
    for user in (37, 3):            # (b, a) = (1, 5) and (0, 3)
        out = emf.predict(UD, VD, user)
        assert len(out) == plan.n_vb and out[0].level == he.prm.top - 2
        got = np.concatenate([he.decrypt(ct)[::plan.w][:plan.B] for ct in out])[:m]
        want = V @ U[user]
        assert np.abs(got - want).max() < 1e-6


def test_delta_tree_baby_step_giant_step():
    """Every delta d < B is reached from 0 along its parents by rotations summing to d; a baby hangs
    off its giant, a giant off a giant; the tree's rotation amounts are the baby steps 1..beta-1 and
    the giant steps 2^t beta; a full tree needs only about 3B/(2 beta) parents (ModUps) instead of B/2."""
    for B in (2, 4, 8, 32, 512, 1024, 2048):
        beta = mf.baby_range(B)
        assert beta * beta <= B < 4 * beta * beta
        parents = set()
        for d in range(1, B):
            total, x, depth = 0, d, 0
            while x:
                par, step = mf.tree_parent(x, beta)
                assert par < x and step > 0 and step in mf.tree_steps(B)
                parents.add(par)
                total += step
                x = par
                depth += 1
            assert total == d and depth == mf.tree_depth(d, beta)
            g, r = divmod(d, beta)
            assert (mf.tree_parent(d, beta)[0] == g * beta) if r else (mf.tree_parent(d, beta)[0] % beta == 0)
        assert sorted(mf.tree_steps(B)) == sorted(set(range(1, min(beta, B))) |
                                                  {beta << t for t in range(16) if (beta << t) < B})
        assert len(parents) <= 3 * B // (2 * beta) + 1
    assert mf.delta_closure([37], 16) == [0, 32, 37]            # 37 = 2*16 + 5: giant 32 = 0 + 2*16, then + 5
    assert mf.delta_closure([53], 16) == [0, 16, 48, 53]        # 53 = 3*16 + 5: giants 16, 48 = 16 + 2*16
