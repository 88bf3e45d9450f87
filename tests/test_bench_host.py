"""Host-side arithmetic of the bench line: per-class rooflines and the oracle worker count."""
import bench


def test_class_rooflines_integer_views():
    # a full negacyclic transform of one row does (N/2) log2(N) butterflies; the library reports them
    # as each class's work, and the rate is checked against the butterfly ceiling
    ceil = {"butterfly_gbfly": 100.0, "probe_butterfly_gbfly": 50.0, "mac_gmacs": 400.0}
    for log_n in (10, 13, 15, 16):
        n = 1 << log_n
        rows = 7
        work = (n // 2) * log_n * rows
        stats = {"ntt_forward": (2, 1.0, 16.0 * n * rows * 2, float(work))}
        rec = bench.class_rooflines(stats, ceil, 1000.0)["ntt_forward"]
        want = work / 1e-3 / 1e9        # Gbfly/s over 1 ms
        assert abs(rec["alu"]["achieved_gbfly"] - want) < 1e-9 * want
        assert abs(rec["alu"]["frac"] - want / 100.0) < 1e-12 * want
        assert abs(rec["alu"]["frac_of_probe"] - want / 50.0) < 1e-12 * want
    stats = {"ks_inner": (3, 2.0, 1e9, 8e9)}                        # 8e9 MACs in 2 ms = 4000 GMAC/s
    rec = bench.class_rooflines(stats, ceil, 1000.0)["ks_inner"]
    assert abs(rec["alu"]["achieved_gmacs"] - 4000.0) < 1e-6 and abs(rec["alu"]["frac"] - 10.0) < 1e-9


def test_class_rooflines_shares_and_bounds():
    stats = {"ntt_forward": (10, 30.0, 3e9, 0.0), "ks_inner": (4, 10.0, 1e9, 0.0), "tensor": (2, 10.0, 2e9, 0.0),
             "rescale": (0, 0.0, 0.0, 0.0)}
    out = bench.class_rooflines(stats, None, 5000.0)
    assert set(out) == {"ntt_forward", "ks_inner", "tensor"}          # classes without launches dropped
    assert abs(sum(r["share"] for r in out.values()) - 1.0) < 1e-12
    assert out["tensor"]["bound"] == "hbm" and out["ks_inner"]["bound"] == "alu"
    assert abs(out["tensor"]["hbm_view"]["achieved_gbs"] - 200.0) < 1e-9     # 2 GB in 10 ms
    assert abs(out["tensor"]["hbm_view"]["frac"] - 0.04) < 1e-12
    assert "alu" not in out["ntt_forward"]                              # no ceilings given


def test_roofline_of_the_dominant_class():
    ceil = {"butterfly_gbfly": 2000.0, "probe_butterfly_gbfly": 900.0, "mac_gmacs": 5000.0, "source": "x"}
    stats = {"ntt_forward": (4, 8.0, 4 * 16.0 * 2**15 * 10, 4 * 1e9), "tensor": (2, 1.0, 1e9, 0.0)}
    r = bench.roofline_of(stats, ceil, 6000.0, True, 1000.0, 15)
    assert r["kernel"] == "ntt_forward" and r["bound"] == "alu" and r["unit"] == "Gbfly/s"
    assert abs(r["achieved"] - 1e9 / 2e-3 / 1e9) < 1e-9                # 1e9 butterflies per 2 ms launch
    assert abs(r["frac"] - r["achieved"] / 2000.0) < 1e-12
    assert abs(r["traffic"] - 1000.0 * 10) < 1e-9                      # 10 rows per launch
    stats = {"ks_inner": (1, 5.0, 1e9, 2e10)}
    r = bench.roofline_of(stats, ceil, 6000.0, True, None, 15)
    assert r["unit"] == "GMAC/s" and abs(r["achieved"] - 4000.0) < 1e-6


def test_served_request_seconds_model():
    ops = {"ip": 10.0, "mask": 1.0, "relin": 2.0, "rot": 3.0, "reg": 0.5}
    top, B, n_vb = 12, 1024, 4
    got = bench.served_request_seconds(ops, 2, top, n_vb, B, steps=1, alpha=3)
    scale = lambda lv: (lv + 1 + 3) / (top + 1 + 3)
    want = 2 * (10 + 1) + 2 * scale(11) + 11 * 3 * scale(10) + 0.5 + 4 * 10 * scale(10)
    assert abs(got - want) < 1e-12


def test_oracle_workers_bounds():
    n = bench.oracle_workers(cap=3)
    assert 1 <= n <= 3
    assert bench.oracle_workers(cap=64, bytes_per_worker=float(1 << 62)) == 1   # memory caps it


def test_oracle_epoch_extrapolation():
    st = {"groups": 100, "nodes": 10}
    assert bench.oracle_epoch_s(st, 2.0, 0.5) == 100 * 2.0 + 30 * 0.5
    assert bench.oracle_epoch_s(st, 2.0, 0.5, cores=5) == (100 * 2.0 + 30 * 0.5) / 5
