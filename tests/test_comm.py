"""The communication report's counts for small hand-checkable cases (host arithmetic only)."""
from paper_2509_03024_gb300 import comm


def test_ct_and_key_sizes():
    assert comm.ct_bytes(8, 2) == 2 * 3 * 8 * 8
    k = comm.key_bytes(8, top=3, alpha=2)          # 4 data limbs, 2 digits, 6 extended limbs
    assert k == {"public_key": 2 * 4 * 8 * 8, "eval_key_each": 2 * 2 * 6 * 8 * 8}


def test_training_refresh_schedule():
    # top = 7: epochs start at levels 7, 5, 3, then a refresh (level 1 < 2), 7, 5 ...
    r = comm.mf_training(n=16, top=7, alpha=2, n_rot_keys=3, n_bins=10, n_ub=2, n_vb=4, epochs=5)
    assert r["refreshes"] == 1 and r["final_level"] == 3
    per_ct = lambda l: 2 * (l + 1) * 16 * 8
    assert r["refresh_bytes"] == 6 * (per_ct(1) + per_ct(7))
    assert r["setup"]["rating_bytes"] == 10 * (7 * 16 * 8 + 16)   # c0 at level 6 and a seed reference
    assert r["final_decrypt_bytes"] == 6 * per_ct(3)


def test_served_request_levels():
    r = comm.served_request(n=16, top=13, n_vb=4, rated_batches=2, steps=5)
    assert r["out_level"] == 2 and r["up_cts"] == 3 and r["down_cts"] == 4
    assert r["total_bytes"] == 3 * 2 * 14 * 16 * 8 + 4 * 2 * 3 * 16 * 8
