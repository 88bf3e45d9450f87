"""Bit-exact parity at the ring sizes the benchmark times.

* The paper-scale ring (N = 2^15, eight 50-bit data primes, two 60-bit special primes, k = 10 so
  kp = 16 and the in-block rotate-and-sum is hoisted): one whole encrypted epoch on a small CSR whose
  ratings sit on two diagonals of two item batches and two user batches, so that the two-pass NTT,
  the fused ModUp / ModDown / relinearise-rescale passes, the plaintext-product rescale, the seeded
  rating ciphertexts (c1 regenerated on the device), the hoisted tree fan-out along a multi-node
  delta-tree path (0 -> 32 -> 37) and the cached masks all run at the benchmark's instantiation. Every
  output ciphertext is compared with the oracle's in coefficient form.
* The served ring (N = 2^16, thirteen 50-bit data primes, three 60-bit special primes, k = 16): one
  request through the server (one fold-in step, then the prediction row over two item batches),
  compared with the oracle's served request.

The oracle's rotation keys and dense encodings are computed by a spawn pool (tests/oracle_pool.py);
the arithmetic is the oracle's own.
"""
import numpy as np
import pytest

from oracle import mf, serve
from paper_2509_03024_gb300 import capi
from paper_2509_03024_gb300 import workloads as W
from tests.gpu_common import assert_ct_equal, ct_slice, gpu_ctx, to_coeff, torch
from tests.oracle_pool import oracle_setup

pytestmark = pytest.mark.gpu


def _paper_case():
    """Users 0..39 rate items i, i + 37 (item batch 0) and 512 + i, 512 + i + 37 (item batch 1);
    users 512..529 (user batch 1) rate item i - 512. B = 512 at N = 2^15 with k = 10, so the groups
    are (b, c, delta) = (0,0,0), (0,0,37), (0,1,0), (0,1,37), (1,0,0), and each item batch's delta
    tree (baby steps below 16) is 0 -> 32 -> 37: a giant step, then a baby step."""
    rows, cols = [], []
    for i in range(40):
        for j in (i, (i + 37) % 512, 512 + i, 512 + i + 37):
            rows.append(i)
            cols.append(j)
    for i in range(512, 530):
        rows.append(i)
        cols.append(i - 512)
    rng = np.random.default_rng(7)
    vals = rng.integers(1, 6, len(rows)).astype(float)
    return W.csr_from_triples(530, 600, rows, cols, vals)


def test_paper_preset_epoch_bit_exact():
    seed, k, lr, lam = 99, 10, 0.005, 0.02
    csr = _paper_case()
    rows, cols, vals = csr.triples()
    rng = np.random.default_rng(3)
    U, V = rng.normal(0, 0.1, (csr.n, k)), rng.normal(0, 0.1, (csr.m, k))

    ctx = gpu_ctx("paper", seed)
    ctx.add_rotation_keys(ctx.mf_rotation_steps(k))
    plan = capi.MfPlan(ctx, csr.n, csr.m, k, csr.row_ptr, csr.col_idx, csr.vals)
    assert (plan.B, plan.n_ub, plan.n_vb, plan.info.n_groups, plan.info.n_tree_nodes) == (512, 2, 2, 5, 6)
    UD, VD = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, UD)
    plan.encrypt_factors(1, V, VD)
    plan.sgd_epoch(UD, VD, ctx.top, lr, lam)
    torch.cuda.synchronize()

    oplan = mf.build_plan(csr.n, csr.m, k, rows, cols, vals, ctx.slots)
    he, _ = oracle_setup("paper", seed, oplan.rotation_steps())
    emf = mf.EncryptedMF(he, oplan)
    emf.encrypt_ratings()
    oUD, oVD = emf.encrypt_factors(U, V)
    oU2, oV2 = emf.epoch(oUD, oVD, lr, lam)
    lv = ctx.top - 2
    got = to_coeff(ctx, UD, lv, plan.n_ub)
    for t, o in enumerate(oU2):
        assert_ct_equal(got[t], o, f"U'[{t}]")
    got = to_coeff(ctx, VD, lv, plan.n_vb)
    for t, o in enumerate(oV2):
        assert_ct_equal(got[t], o, f"V'[{t}]")
    U1, V1 = mf.mf_epoch_fp64(U, V, rows, cols, vals, lr, lam)
    Ud = plan.decrypt_factors(0, UD, lv, csr.n)
    Vd = plan.decrypt_factors(1, VD, lv, csr.m)
    assert np.abs(Ud - U1).max() < 1e-3 and np.abs(Vd - V1).max() < 1e-3


def test_served_preset_request_bit_exact():
    seed, k, m, steps, lr, lam = 31, 16, 1100, 1, 0.005, 0.02
    rng = np.random.default_rng(5)
    V = rng.normal(0, 0.3, (m, k))
    items = np.array([1030, 1041, 1077, 1099], dtype=np.int32)      # all in the ragged item batch 1
    ratings = np.array([4.0, 5.0, 3.0, 1.0])
    u0 = rng.normal(0, 0.1, k)
    nonce = 5000

    ctx = gpu_ctx("served", seed)
    ctx.add_rotation_keys(ctx.serve_rotation_steps(k))
    kp, w, B = serve.layout(k, ctx.slots)
    n_vb = -(-m // B)
    assert (B, n_vb) == (1024, 2)
    plan = capi.MfPlan(ctx, 1, m, k, [0, 1], [0], [1.0])   # the item packing of the resident factors
    VD = ctx.empty_ct(n_vb)
    plan.encrypt_factors(1, V, VD)
    UR, R = ctx.empty_ct(1), ctx.empty_ct(n_vb)
    ctx.encrypt_request(m, k, u0, items, ratings, nonce, UR, R)
    server = capi.Server(ctx, VD, m, k, steps, lr, lam, max_slots=2)
    assert server.submit(7, items, UR, R)
    for _ in range(steps + 1):
        server.tick()
    torch.cuda.synchronize()              # ticks only enqueue; poll reports completed device work
    assert server.poll() == [7]
    buf = ctx.empty_ct(n_vb)
    lv = server.take(7, buf)
    server.close()
    got = to_coeff(ctx, buf, lv, n_vb)

    dummy = mf.build_plan(1, m, k, [0], [0], [1.0], ctx.slots)
    zV = [mf.pack_factors(V, dummy, c) for c in range(n_vb)]
    zR = serve.rating_batches(items, ratings, k, ctx.slots, n_vb)
    he, enc = oracle_setup("served", seed, serve.rotation_steps(k, ctx.slots),
                           zV + [serve.replicate_user(u0, k, ctx.slots)] + zR)
    top = he.prm.top
    oVD = [he.encrypt_coeffs(enc[c], top, mf.V_NONCE_BASE + c) for c in range(n_vb)]
    oUR = he.encrypt_coeffs(enc[n_vb], top, nonce)
    oR = [he.encrypt_coeffs(enc[n_vb + 1 + c], top, nonce + 1 + c) for c in range(n_vb)]
    _, P = serve.serve_request(he, oUR, oR, oVD, items, k, steps, lr, lam)
    assert lv == P[0].level == top - 2 * steps - 1
    for c in range(n_vb):
        assert_ct_equal(got[c], P[c], f"prediction batch {c}")
    _, pred_ref = serve.fold_in_fp64(u0, V, items, ratings, steps, lr, lam)
    pred = np.concatenate([ctx.decrypt(ct_slice(ctx, buf, c), lv)[::w][:B] for c in range(n_vb)])[:m]
    assert np.abs(pred - pred_ref).max() < 1e-3
