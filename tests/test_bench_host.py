"""Host-side arithmetic of the bench line: per-class rooflines and the oracle worker count."""
import bench


def test_butterfly_count_of_a_full_transform():
    # a full negacyclic transform of one row does (N/2) log2(N) butterflies; the library accounts
    # 16 N algorithmic bytes per row and pass (one pass up to 2^13, two above)
    for log_n in (10, 13, 14, 15, 16):
        n = 1 << log_n
        passes = 1 if log_n <= 13 else 2
        rows = 7
        stats = {"ntt_forward": (passes, 1.0, 16.0 * n * rows * passes)}
        rec = bench.class_rooflines(stats, log_n, 100.0, 1000.0)["ntt_forward"]
        want = (n // 2) * log_n * rows / 1e-3 / 1e9        # Gbfly/s over 1 ms
        assert abs(rec["alu"]["achieved_gbfly"] - want) < 1e-9 * want
        assert abs(rec["alu"]["frac"] - want / 100.0) < 1e-12 * want


def test_class_rooflines_shares_and_bounds():
    stats = {"ntt_forward": (10, 30.0, 3e9), "ks_inner": (4, 10.0, 1e9), "tensor": (2, 10.0, 2e9),
             "rescale": (0, 0.0, 0.0)}
    out = bench.class_rooflines(stats, 15, None, 5000.0)
    assert set(out) == {"ntt_forward", "ks_inner", "tensor"}          # classes without launches dropped
    assert abs(sum(r["share"] for r in out.values()) - 1.0) < 1e-12
    assert out["tensor"]["bound"] == "hbm" and out["ks_inner"]["bound"] == "alu"
    assert abs(out["tensor"]["hbm_view"]["achieved_gbs"] - 200.0) < 1e-9     # 2 GB in 10 ms
    assert abs(out["tensor"]["hbm_view"]["frac"] - 0.04) < 1e-12
    assert "alu" not in out["ntt_forward"]                              # no measured butterfly rate given


def test_oracle_workers_bounds():
    n = bench.oracle_workers(cap=3)
    assert 1 <= n <= 3
    assert bench.oracle_workers(cap=64, bytes_per_worker=float(1 << 62)) == 1   # memory caps it


def test_oracle_epoch_extrapolation():
    st = {"groups": 100, "nodes": 10}
    assert bench.oracle_epoch_s(st, 2.0, 0.5) == 100 * 2.0 + 30 * 0.5
    assert bench.oracle_epoch_s(st, 2.0, 0.5, cores=5) == (100 * 2.0 + 30 * 0.5) / 5
