"""Pins of the oracle's ring arithmetic against definitions computed with Python integers."""
import math
import random

import numpy as np
import pytest
import sympy

from oracle import ckks, ring


def _rand_poly(rng, n, q):
    return np.array([rng.randrange(q) for _ in range(n)], dtype=np.uint64)


@pytest.mark.parametrize("log_n,bits", [(3, 30), (4, 40), (5, 60), (6, 50)])
def test_ntt_product_equals_schoolbook(log_n, bits):
    n = 1 << log_n
    q = ckks.gen_primes(log_n, [bits])[0]
    rng = random.Random(log_n * 100 + bits)
    for _ in range(3):
        a, b = _rand_poly(rng, n, q), _rand_poly(rng, n, q)
        assert (ring.polymul(a, b, q) == ring.schoolbook(a, b, q)).all()


def test_schoolbook_is_negacyclic_definition():
    # X^(N-1) * X = X^N = -1 in Z_q[X]/(X^N+1)
    n, q = 8, 97
    a = np.zeros(n, dtype=np.uint64); a[n - 1] = 1
    b = np.zeros(n, dtype=np.uint64); b[1] = 1
    out = ring.schoolbook(a, b, q)
    assert out[0] == q - 1 and (out[1:] == 0).all()
    # direct big-int definition on random data
    rng = random.Random(5)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    want = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                want[k] += a[i] * b[j]
            else:
                want[k - n] -= a[i] * b[j]
    got = ring.schoolbook(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64), q)
    assert [int(x) for x in got] == [w % q for w in want]


def test_polydot_linearity():
    n = 32
    q = ckks.gen_primes(5, [50])[0]
    rng = random.Random(9)
    A = np.stack([_rand_poly(rng, n, q) for _ in range(3)])
    B = np.stack([_rand_poly(rng, n, q) for _ in range(3)])
    want = np.zeros(n, dtype=object)
    for t in range(3):
        want = want + np.array([int(x) for x in ring.schoolbook(A[t], B[t], q)], dtype=object)
    assert [int(x) for x in ring.polydot(A, B, q)] == [int(x) % q for x in want]


def test_ntt_of_one_and_identity():
    # 1 * a = a, and the product is commutative
    n = 64
    q = ckks.gen_primes(6, [60])[0]
    rng = random.Random(2)
    a = _rand_poly(rng, n, q)
    one = np.zeros(n, dtype=np.uint64); one[0] = 1
    assert (ring.polymul(a, one, q) == a).all()
    b = _rand_poly(rng, n, q)
    assert (ring.polymul(a, b, q) == ring.polymul(b, a, q)).all()


def test_find_psi_is_primitive_2n_root():
    for log_n, bits in [(4, 40), (10, 60), (13, 40)]:
        n = 1 << log_n
        q = ckks.gen_primes(log_n, [bits])[0]
        psi = ring.find_psi(n, q)
        assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1


def test_automorphism_definition_and_composition():
    n = 16
    q = ckks.gen_primes(4, [40])[0]
    rng = random.Random(11)
    a = [rng.randrange(q) for _ in range(n)]
    for g in (3, 5, 7, 25, 31):
        want = [0] * n
        for j, v in enumerate(a):
            e = j * g % (2 * n)
            if e < n:
                want[e] = (want[e] + v) % q
            else:
                want[e - n] = (want[e - n] - v) % q
        got = ring.automorphism(np.array(a, dtype=np.uint64), g, q)
        assert [int(x) for x in got] == want
    A = np.array(a, dtype=np.uint64)
    for g, h in [(5, 25), (3, 7), (5, 5 ** 7 % 32)]:
        lhs = ring.automorphism(ring.automorphism(A, h, q), g, q)
        rhs = ring.automorphism(A, g * h % (2 * n), q)
        assert (lhs == rhs).all()
    # the automorphism is a ring homomorphism
    b = np.array([rng.randrange(q) for _ in range(n)], dtype=np.uint64)
    lhs = ring.automorphism(ring.polymul(A, b, q), 5, q)
    rhs = ring.polymul(ring.automorphism(A, 5, q), ring.automorphism(b, 5, q), q)
    assert (lhs == rhs).all()


def test_fast_base_conversion_is_x_plus_uQ():
    n = 16
    src = ckks.gen_primes(4, [50, 50, 50])
    dst = ckks.gen_primes(4, [60, 60])[:2]
    Q = math.prod(src)
    rng = random.Random(3)
    xs = [rng.randrange(Q) for _ in range(n)]
    res = np.array([[x % q for x in xs] for q in src], dtype=np.uint64)
    out = ring.fast_base_conv(res, src, dst)
    for k, x in enumerate(xs):
        # find u with 0 <= u < len(src) such that out = x + u Q modulo every dst prime
        ok = [u for u in range(len(src)) if all(int(out[d][k]) == (x + u * Q) % p for d, p in enumerate(dst))]
        assert ok, (k, x)
    # converting to the source primes themselves returns the input residues
    back = ring.fast_base_conv(res, src, src)
    assert (back == res).all()


def test_rescale_is_exact_rounding():
    n = 16
    primes = ckks.gen_primes(4, [50, 40, 40, 40])
    Q = math.prod(primes)
    rng = random.Random(4)
    xs = [rng.randrange(Q) for _ in range(n)]
    res = np.array([[x % q for x in xs] for q in primes], dtype=np.uint64)
    out = ring.rescale(res, primes)
    ql = primes[-1]
    for k, x in enumerate(xs):
        r = (2 * x + ql) // (2 * ql)   # round(x / ql), ql odd so no ties
        for i, q in enumerate(primes[:-1]):
            assert int(out[i][k]) == r % q


def test_is_prime_matches_sympy():
    rng = random.Random(7)
    nums = [rng.randrange(1 << 62) | 1 for _ in range(300)] + [2, 3, 4, 1, 0, 561, 1105, 2 ** 61 - 1]
    for x in nums:
        assert ring.is_prime(x) == sympy.isprime(x) == ckks._is_prime_py(x)


@pytest.mark.parametrize("log_n,bits", [(13, [60, 40, 40, 60]), (15, [50] * 8 + [60, 60]), (16, [50] * 4 + [60] * 3)])
def test_prime_chain(log_n, bits):
    primes = ckks.gen_primes(log_n, bits)
    two_n = 1 << (log_n + 1)
    assert len(set(primes)) == len(primes)
    for i, (p, b) in enumerate(zip(primes, bits)):
        assert sympy.isprime(p) and p % two_n == 1 and p < (1 << b)
        # p is the largest candidate below 2^b not already used by an earlier entry
        c = (1 << b) + 1 - two_n
        while c > p:
            assert (not sympy.isprime(c)) or c in primes[:i]
            c -= two_n
