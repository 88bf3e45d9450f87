"""Seeded synthetic workloads shaped like the paper's MovieLens experiments.

This module draws inputs only: CSR rating matrices, initial factor matrices,
held-out splits, serving request streams and the CKKS parameter presets. It
contains none of the encrypted method's arithmetic, so both the CUDA path and
the CPU oracle may take their inputs from it.

The paper evaluates on MovieLens-100K (943 users, 1682 items, 100,000 ratings;
Sec. IV-A). That data set is not available here; the generators below produce
matrices of the same shape and rating law instead:
  * item popularity: Zipf(s) by item rank,
  * every user has at least 20 ratings; the remainder is spread over users by a
    multinomial with lognormal(0, 1) weights, capped at the item count,
  * rating values 1..5 with probabilities .06/.11/.27/.34/.22,
  * no duplicate (user, item) pairs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

RATING_PROBS = (0.06, 0.11, 0.27, 0.34, 0.22)


@dataclasses.dataclass(frozen=True)
class CkksPreset:
    """RNS-CKKS parameter set: ring degree 2^log_n, prime bit sizes, scale 2^log_scale."""
    name: str
    log_n: int
    data_bits: Tuple[int, ...]
    special_bits: Tuple[int, ...]
    log_scale: int
    sigma: float = 3.2


# Parameter sets of the five workloads (tiny, paper-scale, batched, served, large),
# and small ring sizes used for fast parity cases.
PRESETS = {
    "tiny": CkksPreset("tiny", 13, (60, 40, 40), (60,), 40),
    "paper": CkksPreset("paper", 15, (50,) * 8, (60, 60), 50),
    "batched": CkksPreset("batched", 16, (50,) * 12, (60, 60, 60), 50),
    "served": CkksPreset("served", 16, (50,) * 13, (60, 60, 60), 50),
    "large": CkksPreset("large", 16, (50,) * 20, (60, 60, 60), 50),
    # the paper's ring (N = 8192) at its two fractional precisions (22 and 32 bits): one epoch
    # (two levels) per refresh, 128-bit secure chains (log QP = 144 and 164)
    "sweep22": CkksPreset("sweep22", 13, (40, 22, 22), (60,), 22),
    "sweep32": CkksPreset("sweep32", 13, (40, 32, 32), (60,), 32),
    # test-only small rings
    "t10": CkksPreset("t10", 10, (60, 40, 40), (60,), 40),
    "t11a2": CkksPreset("t11a2", 11, (50,) * 5, (60, 60), 50),
    "t12": CkksPreset("t12", 12, (60, 40, 40, 40, 40), (60,), 40),
    "t10s": CkksPreset("t10s", 10, (50,) * 13, (60, 60, 60), 50),
    # the N = 2^16 ring of the batched, served and large workloads with a short chain: three special
    # primes, two key-switch digits at the top level (the second holding one limb)
    "t16a3": CkksPreset("t16a3", 16, (50,) * 4, (60, 60, 60), 50),
}


@dataclasses.dataclass
class Csr:
    """Rating matrix in CSR form (row = user, column = item), Sec. II-A.3 of the paper."""
    n: int
    m: int
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    vals: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def triples(self):
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        return rows, self.col_idx.astype(np.int64), self.vals


def csr_from_triples(n: int, m: int, rows, cols, vals) -> Csr:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Csr(n, m, row_ptr, cols.astype(np.int32), vals)


def uniform_ratings(n: int, m: int, density: float, seed: int) -> Csr:
    """Uniform positions at the given density, integer ratings uniform in 1..5."""
    rng = np.random.default_rng(seed)
    nnz = int(round(density * n * m))
    flat = rng.choice(n * m, size=nnz, replace=False)
    vals = rng.integers(1, 6, size=nnz).astype(np.float64)
    return csr_from_triples(n, m, flat // m, flat % m, vals)


def movielens_like(n: int, m: int, nnz: int, zipf_s: float, seed: int,
                   min_per_user: int = 20) -> Csr:
    """Zipf item popularity, >= min_per_user ratings per user, MovieLens rating law."""
    rng = np.random.default_rng(seed)
    nnz = min(nnz, n * m)
    base = min(min_per_user, m)
    counts = np.full(n, base, dtype=np.int64)
    rest = nnz - base * n
    if rest > 0:
        w = rng.lognormal(0.0, 1.0, size=n)
        extra = rng.multinomial(rest, w / w.sum())
        counts = np.minimum(counts + extra, m)
        # re-spread what the cap removed, onto users with room, largest weight first
        short = nnz - int(counts.sum())
        order = np.argsort(-w)
        while short > 0:
            for u in order:
                if short == 0:
                    break
                if counts[u] < m:
                    counts[u] += 1
                    short -= 1
    ranks = np.arange(1, m + 1, dtype=np.float64)
    pop = ranks ** (-zipf_s)
    pop /= pop.sum()
    item_of_rank = rng.permutation(m)
    rows, cols = [], []
    for u in range(n):
        c = int(counts[u])
        picked = rng.choice(m, size=c, replace=False, p=pop)
        rows.append(np.full(c, u, dtype=np.int64))
        cols.append(item_of_rank[picked])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.choice(np.arange(1, 6), size=rows.size, p=RATING_PROBS).astype(np.float64)
    return csr_from_triples(n, m, rows, cols, vals)


def split_holdout(csr: Csr, frac: float, seed: int) -> Tuple[Csr, Csr]:
    """Uniform random held-out split of the non-zeros: (train, test)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = csr.triples()
    test = rng.random(rows.size) < frac
    tr = csr_from_triples(csr.n, csr.m, rows[~test], cols[~test], vals[~test])
    te = csr_from_triples(csr.n, csr.m, rows[test], cols[test], vals[test])
    return tr, te


def init_factors(count: int, k: int, seed: int, std: float = 0.1) -> np.ndarray:
    """Initial latent factors ~ N(0, std^2), float64 [count, k]."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, size=(count, k))


def tiny_workload(seed: int = 1):
    """64 users x 48 items at 6 % density, ratings 1..5 uniform, k = 4."""
    csr = uniform_ratings(64, 48, 0.06, seed)
    U = init_factors(64, 4, seed + 100)
    V = init_factors(48, 4, seed + 200)
    return csr, U, V


def paper_workload(seed: int = 2, n: int = 943, m: int = 1682, nnz: int = 100_000, k: int = 10):
    """943 x 1682, 100,000 ratings, Zipf(1.0); 90/10 train/test split; k = 10."""
    full = movielens_like(n, m, nnz, 1.0, seed)
    train, test = split_holdout(full, 0.1, seed + 7)
    U = init_factors(n, k, seed + 100)
    V = init_factors(m, k, seed + 200)
    return train, test, U, V


def batched_instances(count: int = 64, seed: int = 3, k: int = 8,
                      users=(50, 2000), items=(40, 3000), density=(0.01, 0.06)):
    """Independent uneven MF instances: users/items uniform, density log-uniform, Zipf(1.0)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(rng.integers(users[0], users[1] + 1))
        m = int(rng.integers(items[0], items[1] + 1))
        dens = math.exp(rng.uniform(math.log(density[0]), math.log(density[1])))
        nnz = max(1, int(round(dens * n * m)))
        per_user = max(1, min(20, nnz // n))
        csr = movielens_like(n, m, nnz, 1.0, seed * 1000 + t, min_per_user=per_user)
        U = init_factors(n, k, seed * 1000 + t + 100)
        V = init_factors(m, k, seed * 1000 + t + 200)
        out.append((csr, U, V))
    return out


@dataclasses.dataclass
class Request:
    """One served request: a user's CSR rating row over the resident item set."""
    arrival_s: float
    items: np.ndarray    # int32 [nnz]
    ratings: np.ndarray  # float64 [nnz]
    u0: np.ndarray       # float64 [k] initial user factor


def served_requests(count: int, rate_per_s: float, m: int, k: int, seed: int,
                    nnz_range=(5, 300), zipf_s: float = 1.0) -> List[Request]:
    """Poisson arrivals; nnz log-uniform in nnz_range; Zipf item choice; MovieLens rating law."""
    rng = np.random.default_rng(seed)
    ranks = np.arange(1, m + 1, dtype=np.float64)
    pop = ranks ** (-zipf_s)
    pop /= pop.sum()
    t = 0.0
    reqs = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        nnz = int(round(math.exp(rng.uniform(math.log(nnz_range[0]), math.log(nnz_range[1])))))
        nnz = max(1, min(nnz, m))
        items = np.sort(rng.choice(m, size=nnz, replace=False, p=pop)).astype(np.int32)
        ratings = rng.choice(np.arange(1, 6), size=nnz, p=RATING_PROBS).astype(np.float64)
        reqs.append(Request(t, items, ratings, rng.normal(0.0, 0.1, size=k)))
    return reqs
