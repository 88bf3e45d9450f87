"""GPU parity of the encrypted CSR matrix factorisation against the CPU oracle.

Bit-exact: the plan's groups, the encrypted factors, every U and V ciphertext
after an epoch, and the prediction row. Approximate (1e-3, the bar stated for
decrypted factors): decrypted factors against the FP64 plaintext epoch.
"""
import numpy as np
import pytest

from oracle import mf
from paper_2509_03024_gb300 import capi
from paper_2509_03024_gb300 import workloads as W
from tests.gpu_common import assert_ct_equal, ct_slice, gpu_ctx, oracle_ctx, to_coeff, torch

pytestmark = pytest.mark.gpu

SEED = 99


def _setup(preset, csr, k, U, V, chunk=None):
    ctx = gpu_ctx(preset, SEED)
    ctx.add_rotation_keys(ctx.mf_rotation_steps(k))
    plan = capi.MfPlan(ctx, csr.n, csr.m, k, csr.row_ptr, csr.col_idx, csr.vals)
    if chunk:
        plan.set_chunk(chunk)
    rows, cols, vals = csr.triples()
    he = oracle_ctx(preset, SEED)
    oplan = mf.build_plan(csr.n, csr.m, k, rows, cols, vals, he.prm.slots)
    for r in oplan.rotation_steps():
        he.add_rotation_key(r)
    emf = mf.EncryptedMF(he, oplan)
    emf.encrypt_ratings()
    UD = ctx.empty_ct(plan.n_ub)
    VD = ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, UD)
    plan.encrypt_factors(1, V, VD)
    oUD, oVD = emf.encrypt_factors(U, V)
    return ctx, plan, he, oplan, emf, UD, VD, oUD, oVD


def _small_case(seed=4, n=40, m=30, density=0.08, k=4):
    csr = W.uniform_ratings(n, m, density, seed)
    rng = np.random.default_rng(seed)
    return csr, rng.normal(0, 0.1, (n, k)), rng.normal(0, 0.1, (m, k))


def test_rotation_steps_match_oracle():
    ctx = gpu_ctx("t10", SEED)
    csr, U, V = _small_case()
    rows, cols, vals = csr.triples()
    for k in (1, 3, 4, 10):
        p = mf.build_plan(csr.n, csr.m, k, rows, cols, vals, ctx.slots)
        assert sorted(ctx.mf_rotation_steps(k)) == sorted(p.rotation_steps())


def test_plan_groups_and_factor_encryption_bit_exact():
    csr, U, V = _small_case()
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup("t10", csr, 4, U, V)
    b, c, d, cnt = plan.groups()
    assert list(zip(b, c, d, cnt)) == [(g.b, g.c, g.delta, len(g.a)) for g in oplan.groups]
    assert plan.info.n_tree_nodes == sum(len(x) for x in oplan.closure)
    assert plan.bins().tolist() == oplan.bin_of and plan.info.n_bins == len(oplan.bin_batch)
    got = to_coeff(ctx, UD, ctx.top, plan.n_ub)
    for t, o in enumerate(oUD):
        assert_ct_equal(got[t], o, f"UD[{t}]")
    got = to_coeff(ctx, VD, ctx.top, plan.n_vb)
    for t, o in enumerate(oVD):
        assert_ct_equal(got[t], o, f"VD[{t}]")
    Ud = plan.decrypt_factors(0, UD, ctx.top, csr.n)
    assert np.abs(Ud - U).max() < 1e-6


@pytest.mark.parametrize("preset,n,m,density,k,chunk", [
    ("t10", 40, 30, 0.08, 4, None),       # one user batch, one item batch
    ("t10", 150, 70, 0.05, 2, 7),         # several user batches (B = 128), ragged chunks of 7 groups
    ("t10", 60, 200, 0.04, 3, None),      # k < kp, several item batches
    ("t11a2", 90, 50, 0.06, 10, 5),       # k = 10 (kp = 16), alpha = 2, dnum > 1
    ("t10", 30, 20, 0.1, 1, None),        # k = 1: no rotate-and-sum at all
    ("t10", 12, 10, 0.2, 17, None),       # k = 17 (kp = 32): rotate-and-adds instead of hoisting, B = 8
])
def test_epoch_bit_exact_and_fp64(preset, n, m, density, k, chunk):
    csr, U, V = _small_case(seed=n + m, n=n, m=m, density=density, k=k)
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup(preset, csr, k, U, V, chunk)
    lr, lam = 0.01, 0.02
    plan.sgd_epoch(UD, VD, ctx.top, lr, lam)
    oU2, oV2 = emf.epoch(oUD, oVD, lr, lam)
    lv = ctx.top - 2
    got = to_coeff(ctx, UD, lv, plan.n_ub)
    for t, o in enumerate(oU2):
        assert_ct_equal(got[t], o, f"U'[{t}]")
    got = to_coeff(ctx, VD, lv, plan.n_vb)
    for t, o in enumerate(oV2):
        assert_ct_equal(got[t], o, f"V'[{t}]")
    rows, cols, vals = csr.triples()
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    Ud = plan.decrypt_factors(0, UD, lv, csr.n)
    Vd = plan.decrypt_factors(1, VD, lv, csr.m)
    assert np.abs(Ud - U1).max() < 1e-3 and np.abs(Vd - V1).max() < 1e-3
    e_gpu = mf.rmse(Ud, Vd, rows, cols, vals)
    e_ref = mf.rmse(U1, V1, rows, cols, vals)
    assert abs(e_gpu - e_ref) < 1e-4


def test_epoch_in_item_batch_waves_bit_exact():
    """One item batch per wave of the node workspace (the large-workload memory mode): the same bits."""
    csr, U, V = _small_case(seed=260, n=60, m=200, density=0.04, k=3)
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup("t10", csr, 3, U, V, 5)
    assert plan.n_vb > 1
    plan.set_wave_budget(1)
    lr, lam = 0.01, 0.02
    plan.sgd_epoch(UD, VD, ctx.top, lr, lam)
    oU2, oV2 = emf.epoch(oUD, oVD, lr, lam)
    lv = ctx.top - 2
    for got, want, name in ((to_coeff(ctx, UD, lv, plan.n_ub), oU2, "U"), (to_coeff(ctx, VD, lv, plan.n_vb), oV2, "V")):
        for t, o in enumerate(want):
            assert_ct_equal(got[t], o, f"{name}'[{t}]")


def test_two_epochs_and_level_exhaustion():
    csr, U, V = _small_case(seed=8, n=50, m=40, density=0.06, k=2)
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup("t11a2", csr, 2, U, V)
    lr, lam = 0.02, 0.01
    lv = ctx.top
    rows, cols, vals = csr.triples()
    Ur, Vr = U, V
    for ep in range(2):
        plan.sgd_epoch(UD, VD, lv, lr, lam)
        oUD, oVD = emf.epoch(oUD, oVD, lr, lam)
        lv -= 2
        Ur, Vr = mf.mf_epoch_fp64(Ur, Vr, rows, cols, vals, lr, lam)
        got = to_coeff(ctx, UD, lv, plan.n_ub)
        for t, o in enumerate(oUD):
            assert_ct_equal(got[t], o, f"epoch {ep} U[{t}]")
    assert np.abs(plan.decrypt_factors(0, UD, lv, csr.n) - Ur).max() < 1e-3
    with pytest.raises(capi.FheError, match="LEVEL_EXHAUSTED"):
        plan.sgd_epoch(UD, VD, 1, lr, lam)


def test_predict_bit_exact():
    csr, U, V = _small_case(seed=5, n=40, m=140, density=0.05, k=3)
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup("t10", csr, 3, U, V)
    for user in (0, 17, csr.n - 1):
        out = ctx.empty_ct(plan.n_vb)
        plan.predict(UD, VD, ctx.top, user, out)
        want = emf.predict(oUD, oVD, user)
        got = to_coeff(ctx, out, ctx.top - 2, plan.n_vb)
        for t, o in enumerate(want):
            assert_ct_equal(got[t], o, f"predict user {user} batch {t}")
        # slot d*w holds <u_user, v_(cB+d)>
        for cb in range(plan.n_vb):
            z = ctx.decrypt(ct_slice(ctx, out, cb), ctx.top - 2)
            for d in range(plan.B):
                j = cb * plan.B + d
                if j < csr.m:
                    assert abs(z[d * plan.w] - U[user] @ V[j]) < 1e-4


def test_tiny_config_epoch_bit_exact():
    """The tiny configuration end to end: N = 2^13, 60/40/40-bit data primes, 64 x 48 at 6 %, k = 4."""
    csr, U, V = W.tiny_workload(1)
    ctx, plan, he, oplan, emf, UD, VD, oUD, oVD = _setup("tiny", csr, 4, U, V)
    lr, lam = 0.01, 0.02
    plan.sgd_epoch(UD, VD, ctx.top, lr, lam)
    oU2, oV2 = emf.epoch(oUD, oVD, lr, lam)
    got = to_coeff(ctx, UD, 0, plan.n_ub)
    for t, o in enumerate(oU2):
        assert_ct_equal(got[t], o, f"U'[{t}]")
    got = to_coeff(ctx, VD, 0, plan.n_vb)
    for t, o in enumerate(oV2):
        assert_ct_equal(got[t], o, f"V'[{t}]")
    rows, cols, vals = csr.triples()
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    assert np.abs(plan.decrypt_factors(0, UD, 0, csr.n) - U1).max() < 1e-3
    assert np.abs(plan.decrypt_factors(1, VD, 0, csr.m) - V1).max() < 1e-3


def test_rating_bins_match_oracle_at_paper_scale():
    """The bin assignment of the paper-scale workload (943 x 1682, 90k ratings, k = 10) is the oracle's;
    about half as many rating ciphertexts as groups."""
    train, _, _, _ = W.paper_workload(seed=2)
    ctx = gpu_ctx("paper", SEED)
    plan = capi.MfPlan(ctx, train.n, train.m, 10, train.row_ptr, train.col_idx, train.vals)
    rows, cols, vals = train.triples()
    oplan = mf.build_plan(train.n, train.m, 10, rows, cols, vals, ctx.slots)
    assert plan.bins().tolist() == oplan.bin_of
    assert plan.info.n_bins == len(oplan.bin_batch) < plan.info.n_groups


def test_csr_pack_rejects_bad_input():
    ctx = gpu_ctx("t10", SEED)
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        capi.MfPlan(ctx, 2, 2, 1, [0, 2, 2], [1, 1], [1.0, 2.0])   # duplicate (0, 1)
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        capi.MfPlan(ctx, 2, 2, 1, [0, 1, 2], [0, 5], [1.0, 2.0])   # column out of range
    # an empty matrix is a valid plan with no groups
    p = capi.MfPlan(ctx, 3, 3, 2, [0, 0, 0, 0], [], [])
    assert p.info.n_groups == 0


def test_refresh_then_epoch_bit_exact():
    """epoch, epoch, key-holder refresh, epoch: every ciphertext equals the oracle's."""
    from paper_2509_03024_gb300 import train as T
    csr, U, V = _small_case(seed=9, n=45, m=35, density=0.07, k=3)
    ctx, plan, he, oplan, emf, UD0, VD0, oUD, oVD = _setup("t11a2", csr, 3, U, V)
    lr, lam = 0.02, 0.01
    UD, VD, level, times, refreshes = T.run(ctx, plan, U, V, 3, lr, lam)
    assert refreshes == 1 and level == ctx.top - 2
    per = plan.n_ub + plan.n_vb
    lv = he.prm.top
    for ep in range(3):
        if lv < 2:
            base = T.REFRESH_NONCE_BASE + 1 * per
            oUD = [he.refresh(c, base + b) for b, c in enumerate(oUD)]
            oVD = [he.refresh(c, base + plan.n_ub + j) for j, c in enumerate(oVD)]
            lv = he.prm.top
        oUD, oVD = emf.epoch(oUD, oVD, lr, lam)
        lv -= 2
    got = to_coeff(ctx, UD, level, plan.n_ub)
    for t, o in enumerate(oUD):
        assert_ct_equal(got[t], o, f"U[{t}] after refresh")
    got = to_coeff(ctx, VD, level, plan.n_vb)
    for t, o in enumerate(oVD):
        assert_ct_equal(got[t], o, f"V[{t}] after refresh")
    rows, cols, vals = csr.triples()
    Ur, Vr = U, V
    for _ in range(3):
        Ur, Vr = mf.mf_epoch_fp64(Ur, Vr, rows, cols, vals, lr, lam)
    assert np.abs(plan.decrypt_factors(0, UD, level, csr.n) - Ur).max() < 1e-3


def test_checkpoint_resume_bit_identical(tmp_path):
    """Three epochs straight (one refresh on the way) equal two epochs, a checkpoint written and read
    back, and the third epoch."""
    from paper_2509_03024_gb300 import train as T
    csr, U, V = _small_case(seed=12, n=45, m=35, density=0.07, k=3)
    ctx, plan, he, oplan, emf, UD0, VD0, oUD, oVD = _setup("t11a2", csr, 3, U, V)
    lr, lam = 0.02, 0.01
    UDa, VDa, la, _, ra = T.run(ctx, plan, U, V, 3, lr, lam)
    path = str(tmp_path / "ck.npz")

    def save(t, UD, VD, level, refreshes):
        if t == 1:
            T.save_checkpoint(path, ctx, UD, VD, level, t + 1, refreshes)

    T.run(ctx, plan, U, V, 2, lr, lam, on_epoch=save)
    st = T.load_checkpoint(path, ctx)
    assert st["epoch"] == 2
    UDb, VDb, lb, _, rb = T.run(ctx, plan, U, V, 3, lr, lam, state=st)
    assert (la, ra) == (lb, rb) == (ctx.top - 2, 1)
    assert torch.equal(UDa, UDb) and torch.equal(VDa, VDb)


def test_paper_scale_epoch_properties():
    """The paper-scale epoch as the bench runs it (943 x 1682, 89,893 training ratings, k = 10,
    N = 2^15): every output residue is reduced below its prime, and the decrypted factors are
    within 1e-3 of the FP64 epoch with a held-out RMSE gap below 1e-4."""
    train, test, U, V = W.paper_workload(seed=2)
    ctx = gpu_ctx("paper", SEED)
    ctx.add_rotation_keys(ctx.mf_rotation_steps(10))
    plan = capi.MfPlan(ctx, train.n, train.m, 10, train.row_ptr, train.col_idx, train.vals)
    UD, VD = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, UD)
    plan.encrypt_factors(1, V, VD)
    lr, lam = 0.005, 0.02
    plan.sgd_epoch(UD, VD, ctx.top, lr, lam)
    lv = ctx.top - 2
    primes = torch.tensor([int(q) for q in ctx.primes[: lv + 1]], dtype=torch.int64, device=UD.device)
    for buf, cnt in ((UD, plan.n_ub), (VD, plan.n_vb)):
        x = buf.view(cnt, 2, ctx.top + 1, ctx.n)[:, :, : lv + 1, :]
        assert bool((x >= 0).all()) and bool((x < primes.view(1, 1, -1, 1)).all())
    rows, cols, vals = train.triples()
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    Ud = plan.decrypt_factors(0, UD, lv, train.n)
    Vd = plan.decrypt_factors(1, VD, lv, train.m)
    assert max(np.abs(Ud - U1).max(), np.abs(Vd - V1).max()) < 1e-3
    trow, tcol, tval = test.triples()
    assert abs(mf.rmse(Ud, Vd, trow, tcol, tval) - mf.rmse(U1, V1, trow, tcol, tval)) < 1e-4


def test_epoch_of_an_empty_matrix_keeps_the_factors():
    """No ratings: no groups, no rating bins; the epoch only rescales by reg = 1, so the decrypted
    factors come back unchanged (and every residue stays reduced)."""
    ctx = gpu_ctx("t10", SEED)
    k = 3
    ctx.add_rotation_keys(ctx.mf_rotation_steps(k))
    plan = capi.MfPlan(ctx, 20, 15, k, np.zeros(21, dtype=np.int64), np.zeros(0, dtype=np.int32),
                       np.zeros(0, dtype=np.float64))
    assert plan.info.n_groups == 0 and plan.info.n_bins == 0
    rng = np.random.default_rng(1)
    U, V = rng.normal(0, 0.1, (20, k)), rng.normal(0, 0.1, (15, k))
    UD, VD = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, UD)
    plan.encrypt_factors(1, V, VD)
    plan.sgd_epoch(UD, VD, ctx.top, 0.01, 0.02)
    lv = ctx.top - 2
    assert np.abs(plan.decrypt_factors(0, UD, lv, 20) - U).max() < 1e-6
    assert np.abs(plan.decrypt_factors(1, VD, lv, 15) - V).max() < 1e-6
