"""The synthetic input recipe: shapes, laws and seeding of the workload generators."""
import numpy as np

from paper_2509_03024_gb300 import workloads as W


def test_paper_workload_shape_and_laws():
    train, test, U, V = W.paper_workload(seed=2)
    assert (train.n, train.m) == (943, 1682) and train.nnz + test.nnz == 100_000
    assert 0.08 < test.nnz / 100_000 < 0.12                      # 10 % held out
    rows, cols, vals = train.triples()
    trow, tcol, _ = test.triples()
    pairs = set(zip(rows.tolist(), cols.tolist()))
    assert len(pairs) == rows.size                               # no duplicates
    assert not pairs & set(zip(trow.tolist(), tcol.tolist()))    # train and test disjoint
    per_user = np.bincount(np.concatenate([rows, trow]), minlength=943)
    assert per_user.min() >= 20                                  # >= 20 ratings per user
    counts = np.bincount(vals.astype(int), minlength=6)[1:] / vals.size
    assert np.abs(counts - np.array(W.RATING_PROBS)).max() < 0.01
    # Zipf(1.0) by rank: the most rated item gets far more than the median one
    per_item = np.sort(np.bincount(np.concatenate([cols, tcol]), minlength=1682))[::-1]
    assert per_item[0] > 20 * max(per_item[840], 1)
    assert U.shape == (943, 10) and V.shape == (1682, 10) and abs(U.std() - 0.1) < 0.01


def test_generators_are_seeded():
    a, b = W.paper_workload(seed=2), W.paper_workload(seed=2)
    assert np.array_equal(a[0].col_idx, b[0].col_idx) and np.array_equal(a[2], b[2])
    c = W.paper_workload(seed=3)
    assert not np.array_equal(a[0].col_idx[:100], c[0].col_idx[:100])


def test_batched_instances_ranges():
    inst = W.batched_instances(16)
    for csr, U, V in inst:
        assert 50 <= csr.n <= 2000 and 40 <= csr.m <= 3000
        d = csr.nnz / (csr.n * csr.m)
        assert 0.009 < d < 0.061
        assert U.shape == (csr.n, 8) and V.shape == (csr.m, 8)


def test_served_requests_laws():
    reqs = W.served_requests(400, 100.0, 3706, 16, 7)
    t = np.array([r.arrival_s for r in reqs])
    assert (np.diff(t) > 0).all() and 2.5 < t[-1] < 6.0          # Poisson at 100 req/s
    nnz = np.array([r.items.size for r in reqs])
    assert nnz.min() >= 5 and nnz.max() <= 300
    assert 0.2 < np.mean(np.log(nnz) < np.log(np.sqrt(5 * 300))) < 0.8   # log-uniform: median near sqrt(5*300)
    for r in reqs[:50]:
        assert (np.diff(r.items) > 0).all() and r.u0.shape == (16,)
