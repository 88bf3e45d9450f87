"""The library's plan layout (batch-pair groups, rating bins, delta-tree nodes; Alg. 2, Fig. 5) run
on the host through the C ABI without a GPU, integer-equal to the oracle's plan."""
import numpy as np
import pytest

from oracle import mf
from paper_2509_03024_gb300 import build, capi
from paper_2509_03024_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _compare(csr, k, slots):
    got = capi.mf_layout(slots, csr.n, csr.m, k, csr.row_ptr, csr.col_idx, csr.vals)
    rows, cols, vals = csr.triples()
    plan = mf.build_plan(csr.n, csr.m, k, rows, cols, vals, slots)
    want = np.array([(g.b, g.c, g.delta, len(g.a)) for g in plan.groups], dtype=np.int32).reshape(-1, 4)
    assert np.array_equal(got["groups"], want)
    assert got["bins"].tolist() == plan.bin_of and got["n_bins"] == len(plan.bin_batch)
    nodes = [(c, d) for c, cl in enumerate(plan.closure) for d in cl]
    assert got["nodes"].tolist() == [list(x) for x in nodes]
    return got, plan


@pytest.mark.parametrize("n,m,density,k,slots", [
    (64, 48, 0.06, 4, 4096),       # the tiny configuration: one user and one item batch
    (150, 70, 0.05, 2, 512),       # several user batches (B = 128)
    (90, 300, 0.04, 3, 512),       # several item batches, k not a power of two
    (40, 30, 0.2, 1, 256),         # k = 1 (a block of two slots)
    (33, 41, 0.1, 17, 1024),       # k = 17 -> kp = 32, B = 16: ragged last batches on both sides
])
def test_layout_matches_oracle(n, m, density, k, slots):
    csr = W.uniform_ratings(n, m, density, seed=n + m + k)
    got, plan = _compare(csr, k, slots)
    assert int(got["groups"][:, 3].sum()) == csr.nnz      # every rating in exactly one group


def test_layout_matches_oracle_at_paper_scale():
    """943 x 1682, 90k training ratings, k = 10, N = 2^15: 4096 groups in 2017 bins, 2048 tree nodes."""
    train, _, _, _ = W.paper_workload(seed=2)
    got, _ = _compare(train, 10, 1 << 14)
    assert got["groups"].shape[0] == 4096 and got["n_bins"] == 2017 and got["nodes"].shape[0] == 2048


def test_layout_of_degenerate_inputs():
    empty = capi.mf_layout(256, 3, 3, 2, [0, 0, 0, 0], [], [])
    assert empty["groups"].shape == (0, 4) and empty["n_bins"] == 0
    assert empty["nodes"].tolist() == [[0, 0]]            # the root of the one item batch's tree
    one = capi.mf_layout(256, 1, 1, 1, [0, 1], [0], [5.0])
    assert one["groups"].tolist() == [[0, 0, 0, 1]] and one["bins"].tolist() == [0]


@pytest.mark.parametrize("args,why", [
    ((256, 2, 2, 1, [0, 2, 2], [1, 1], [1.0, 2.0]), "duplicate (0, 1)"),
    ((256, 2, 2, 1, [0, 1, 2], [0, 5], [1.0, 2.0]), "column out of range"),
    ((256, 2, 2, 1, [0, 1, 2], [0, 1], [1.0, np.nan]), "non-finite rating"),
    ((256, 2, 2, 1, [0, 2, 1], [0, 1], [1.0, 2.0]), "decreasing row_ptr"),
    ((256, 2, 2, 512, [0, 0, 0], [], []), "rank too large for the ring"),
    ((300, 2, 2, 1, [0, 0, 0], [], []), "slots not a power of two"),
])
def test_layout_rejects_bad_input(args, why):
    with pytest.raises(capi.FheError, match="INVALID_ARG"):
        capi.mf_layout(*args)


def test_layout_matches_oracle_at_the_large_shape():
    """6040 x 3706, 900k training ratings (Zipf 1.1), k = 16, N = 2^16: the largest plan the bench
    builds, 24,576 groups in 12,204 bins over 4096 tree nodes (about 40 s of oracle time)."""
    full = W.movielens_like(6040, 3706, 1_000_209, 1.1, 5)
    train, _ = W.split_holdout(full, 0.1, 12)
    got, _ = _compare(train, 16, 1 << 15)
    assert got["groups"].shape[0] == 24576 and got["n_bins"] == 12204 and got["nodes"].shape[0] == 4096


def test_layout_ignores_column_order_within_rows():
    """CSR rows need not be sorted: permuting each row's entries gives the same layout."""
    csr = W.uniform_ratings(150, 70, 0.05, seed=9)
    ref = capi.mf_layout(512, csr.n, csr.m, 2, csr.row_ptr, csr.col_idx, csr.vals)
    rng = np.random.default_rng(3)
    ci, va = csr.col_idx.copy(), csr.vals.copy()
    for i in range(csr.n):
        lo, hi = csr.row_ptr[i], csr.row_ptr[i + 1]
        p = rng.permutation(hi - lo) + lo
        ci[lo:hi], va[lo:hi] = ci[p], va[p]
    got = capi.mf_layout(512, csr.n, csr.m, 2, csr.row_ptr, ci, va)
    for key in ("groups", "bins", "nodes"):
        assert np.array_equal(got[key], ref[key])
