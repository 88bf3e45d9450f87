"""GPU parity of the continuous-batching server against the oracle; a request's
result is bit-identical alone and in a mix of staggered requests."""
import numpy as np
import pytest

from oracle import mf, serve
from paper_2509_03024_gb300 import capi
from tests.gpu_common import assert_ct_equal, ct_slice, gpu_ctx, oracle_ctx, to_coeff, torch

pytestmark = pytest.mark.gpu

SEED = 31
K, M, STEPS, LR, LAM = 3, 140, 3, 0.05, 0.02


def _fixture():
    ctx = gpu_ctx("t10s", SEED)
    ctx.add_rotation_keys(ctx.serve_rotation_steps(K))
    kp, w, B = serve.layout(K, ctx.slots)
    n_vb = -(-M // B)
    rng = np.random.default_rng(0)
    V = rng.normal(0, 0.3, (M, K))
    plan = capi.MfPlan(ctx, 1, M, K, [0, 1], [0], [1.0])   # any plan over M items gives the item packing
    VD = ctx.empty_ct(n_vb)
    plan.encrypt_factors(1, V, VD)
    reqs = []
    for r in range(5):
        nnz = [1, 7, 20, 3, 12][r]
        items = np.sort(rng.choice(M, nnz, replace=False)).astype(np.int32)
        ratings = rng.integers(1, 6, nnz).astype(np.float64)
        reqs.append((items, ratings, rng.normal(0, 0.1, K)))
    return ctx, V, VD, n_vb, reqs


def _encrypt(ctx, n_vb, req, nonce):
    items, ratings, u0 = req
    UR, R = ctx.empty_ct(1), ctx.empty_ct(n_vb)
    ctx.encrypt_request(M, K, u0, items, ratings, nonce, UR, R)
    return UR, R


def _run(server, ctx, n_vb, reqs, schedule):
    """schedule: list of (tick index, request index) submissions."""
    enc = {i: _encrypt(ctx, n_vb, reqs[i], 1000 * (i + 1)) for _, i in schedule}
    out, tick, pending = {}, 0, sorted(schedule)
    while pending or len(out) < len(schedule):
        for t, i in list(pending):
            if t <= tick and server.submit(i, reqs[i][0], *enc[i]):
                pending.remove((t, i))
        server.tick()
        for rid in server.poll():
            buf = ctx.empty_ct(n_vb)
            lv = server.take(rid, buf)
            out[rid] = (buf, lv)
        tick += 1
        assert tick < 100
    return out


def test_rotation_steps_match_oracle():
    ctx = gpu_ctx("t10s", SEED)
    for k in (1, 2, 3, 8, 16, 20):
        assert sorted(ctx.serve_rotation_steps(k)) == sorted(serve.rotation_steps(k, ctx.slots))


def test_single_request_bit_exact_with_oracle():
    ctx, V, VD, n_vb, reqs = _fixture()
    server = capi.Server(ctx, VD, M, K, STEPS, LR, LAM, max_slots=4)
    out = _run(server, ctx, n_vb, reqs, [(0, 1)])
    buf, lv = out[1]
    he = oracle_ctx("t10s", SEED, serve.rotation_steps(K, ctx.slots))
    kp, w, B = serve.layout(K, ctx.slots)
    dummy = mf.build_plan(1, M, K, [0], [0], [1.0], he.prm.slots)
    oVD = [he.encrypt(mf.pack_factors(V, dummy, c), he.prm.top, mf.V_NONCE_BASE + c) for c in range(n_vb)]
    items, ratings, u0 = reqs[1]
    UR, R = serve.encrypt_request(he, u0, items, ratings, K, n_vb, 2000)
    _, P = serve.serve_request(he, UR, R, oVD, items, K, STEPS, LR, LAM)
    assert lv == P[0].level
    got = to_coeff(ctx, buf, lv, n_vb)
    for c in range(n_vb):
        assert_ct_equal(got[c], P[c], f"prediction batch {c}")
    _, pred_ref = serve.fold_in_fp64(u0, V, items, ratings, STEPS, LR, LAM)
    pred = np.concatenate([ctx.decrypt(ct_slice(ctx, buf, c), lv)[::w][:B] for c in range(n_vb)])[:M]
    assert np.abs(pred - pred_ref).max() < 1e-3


def test_result_same_alone_and_in_the_mix():
    ctx, V, VD, n_vb, reqs = _fixture()
    alone = {}
    for i in range(len(reqs)):
        server = capi.Server(ctx, VD, M, K, STEPS, LR, LAM, max_slots=1)
        alone.update(_run(server, ctx, n_vb, reqs, [(0, i)]))
        server.close()
    # staggered arrivals, 3 slots: requests join while others are mid-flight, one waits for a slot
    server = capi.Server(ctx, VD, M, K, STEPS, LR, LAM, max_slots=3)
    mixed = _run(server, ctx, n_vb, reqs, [(0, 0), (0, 1), (1, 2), (2, 3), (2, 4)])
    for i in range(len(reqs)):
        a, la = alone[i]
        b, lb = mixed[i]
        assert la == lb
        assert torch.equal(a, b), f"request {i} differs between alone and mixed"


def test_admission_is_bounded_by_slots():
    ctx, V, VD, n_vb, reqs = _fixture()
    server = capi.Server(ctx, VD, M, K, STEPS, LR, LAM, max_slots=2)
    assert server.n_slots == 2 and server.free_slots() == 2
    enc = [_encrypt(ctx, n_vb, reqs[i], 50 + i) for i in range(3)]
    assert server.submit(0, reqs[0][0], *enc[0])
    assert server.submit(1, reqs[1][0], *enc[1])
    assert not server.submit(2, reqs[2][0], *enc[2])        # no free slot: refused, nothing changed
    with pytest.raises(capi.FheError):
        server.submit(0, reqs[0][0], *enc[0])               # duplicate id in flight
    for _ in range(STEPS + 1):
        server.tick()
    torch.cuda.synchronize()               # ticks only enqueue; poll reports completed device work
    done = server.poll()
    assert sorted(done) == [0, 1]
    buf = ctx.empty_ct(n_vb)
    server.take(0, buf)
    assert server.free_slots() == 1
    assert server.submit(2, reqs[2][0], *enc[2])
    # a memory budget smaller than one slot still gives one slot; a tiny budget caps the count
    s2 = capi.Server(ctx, VD, M, K, STEPS, LR, LAM, max_slots=64, memory_budget_bytes=1)
    assert s2.n_slots == 1
