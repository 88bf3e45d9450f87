"""Pins of the oracle RNS-CKKS (sampling, encoding, encryption, homomorphic operations)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ckks, ring

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(log_n=6, data=(60, 40, 40), special=(60,), ls=40):
    return ckks.Params(log_n, data, special, ls)


def test_splitmix64_published_sequence():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    assert [int(x) for x in ckks.draws(g["seed"], 0, len(g["outputs"]))] == g["outputs"]


def test_sampler_distributions():
    h = ckks.stream_key(42, ckks.P_PK_E)
    e = ckks.sample_gaussian(h, 200000, 3.2)
    assert np.abs(e).max() <= 19
    assert abs(e.std() - 3.2) < 0.05 and abs(e.mean()) < 0.05
    t = ckks.sample_ternary(ckks.stream_key(42, ckks.P_SECRET), 90000)
    assert set(np.unique(t).tolist()) == {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs((t == v).mean() - 1 / 3) < 0.01
    q = ckks.gen_primes(10, [60])[0]
    u = ckks.sample_uniform(ckks.stream_key(42, ckks.P_PK_A), 100000, q)
    assert (u < np.uint64(q)).all()
    # mean of a uniform residue is ~ q/2
    assert abs(float(np.mean(u.astype(np.float64))) / q - 0.5) < 0.01
    # the streams differ between purposes and objects
    assert ckks.stream_key(1, 2, 3) != ckks.stream_key(1, 2, 4) != ckks.stream_key(1, 3, 3)


def test_gaussian_table_is_a_cdf():
    T = ckks.gaussian_table(3.2)
    assert all(a < b for a, b in zip(T, T[1:])) and T[-1] <= (1 << 63)
    # P(|e| = 0) = rho(0) / (rho(0) + 2 sum rho(x))
    rho = [math.exp(-x * x / (2 * 3.2 ** 2)) for x in range(20)]
    assert abs(T[0] / 2 ** 63 - 1 / (1 + 2 * sum(rho[1:]))) < 1e-12


def test_slot_count_matches_paper():
    g = json.load(open(os.path.join(GOLD, "slots.json")))
    prm = ckks.Params(g["log_n"], (60, 40, 40), (60,), 40)
    assert prm.slots == g["slots"]


def test_encode_is_canonical_embedding():
    prm = _params(log_n=5)
    enc = ckks.Encoder(prm)
    rng = np.random.default_rng(0)
    z = rng.normal(size=prm.slots)
    m = enc.encode(z)
    # evaluate the integer polynomial at zeta^(5^t) directly
    zeta = np.exp(1j * np.pi / prm.n)
    for t in range(prm.slots):
        root = zeta ** pow(5, t, 2 * prm.n)
        val = sum(int(m[j]) * root ** j for j in range(prm.n)) / prm.delta
        assert abs(val - z[t]) < 1e-9
    # round trip via decode
    assert np.abs(enc.decode(m) - z).max() < 2 ** -30 * np.abs(z).max() * prm.n


def test_encode_constant_is_constant_polynomial():
    prm = _params(log_n=8)
    enc = ckks.Encoder(prm)
    for c in (0.5, 3.0, -2.0):
        m = enc.encode(np.full(prm.slots, c))
        assert m[0] == round(c * prm.delta) and (m[1:] == 0).all()


def _int_negacyclic(a, b):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return out


def test_encrypt_decrypt_exact_error_polynomial():
    """decrypt(encrypt(m)) = m + v*e_pk + e0 + e1*s exactly (integer ring identity)."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(7)
    rng = np.random.default_rng(1)
    m = rng.integers(-(1 << 45), 1 << 45, size=prm.n)
    nonce = 3
    ct = he.encrypt_coeffs(m, prm.top, nonce)
    got = he.decrypt_coeffs(ct)
    n = prm.n
    v = ckks.sample_ternary(ckks.stream_key(7, ckks.P_ENC_V, nonce), n).tolist()
    e0 = ckks.sample_gaussian(ckks.stream_key(7, ckks.P_ENC_E0, nonce), n, 3.2).tolist()
    e1 = ckks.sample_gaussian(ckks.stream_key(7, ckks.P_ENC_E1, nonce), n, 3.2).tolist()
    epk = ckks.sample_gaussian(ckks.stream_key(7, ckks.P_PK_E), n, 3.2).tolist()
    s = he.s.tolist()
    ve = _int_negacyclic(v, epk)
    e1s = _int_negacyclic(e1, s)
    want = [int(m[j]) + ve[j] + e0[j] + e1s[j] for j in range(n)]
    assert got == want


def test_decrypt_slots_and_add_sub():
    prm = _params(log_n=7)
    he = ckks.Ckks(prm)
    he.keygen(11)
    rng = np.random.default_rng(2)
    x, y = rng.normal(size=prm.slots), rng.normal(size=prm.slots)
    cx, cy = he.encrypt(x, prm.top, 1), he.encrypt(y, prm.top, 2)
    assert np.abs(he.decrypt(cx) - x).max() < 1e-6
    assert np.abs(he.decrypt(he.add(cx, cy)) - (x + y)).max() < 1e-6
    assert np.abs(he.decrypt(he.sub(cx, cy)) - (x - y)).max() < 1e-6


def test_tensor_decrypts_to_product_exactly():
    """(d0 + d1 s + d2 s^2) = (a0 + a1 s)(b0 + b1 s) in R_Q: the tensor is the ring product."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(5)
    rng = np.random.default_rng(3)
    a = he.encrypt(rng.normal(size=prm.slots), prm.top, 1)
    b = he.encrypt(rng.normal(size=prm.slots), prm.top, 2)
    t = he.tensor(a, b)
    for i, q in enumerate(prm.q):
        s = ckks.to_rns(he.s, [q])[0]
        s2 = ring.polymul(s, s, q)
        lhs = (t.c[0][i].astype(object) + ring.polymul(t.c[1][i], s, q).astype(object)
               + ring.polymul(t.c[2][i], s2, q).astype(object)) % q
        pa = (a.c[0][i].astype(object) + ring.polymul(a.c[1][i], s, q).astype(object)) % q
        pb = (b.c[0][i].astype(object) + ring.polymul(b.c[1][i], s, q).astype(object)) % q
        rhs = ring.polymul(np.array(pa, dtype=np.uint64), np.array(pb, dtype=np.uint64), q)
        assert [int(x) for x in lhs] == [int(x) for x in rhs]


def test_relinearize_and_rescale():
    prm = _params(log_n=8)
    he = ckks.Ckks(prm)
    he.keygen(13)
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=prm.slots), rng.normal(size=prm.slots)
    cx, cy = he.encrypt(x, prm.top, 1), he.encrypt(y, prm.top, 2)
    r = he.mul_relin_rescale(cx, cy)
    assert r.level == prm.top - 1
    assert np.abs(he.decrypt(r) - x * y).max() < 1e-5


def test_keyswitch_multi_digit_alpha2():
    prm = ckks.Params(7, (50,) * 5, (60, 60), 50)
    he = ckks.Ckks(prm)
    he.keygen(17, [3])
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=prm.slots), rng.normal(size=prm.slots)
    cx, cy = he.encrypt(x, prm.top, 1), he.encrypt(y, prm.top, 2)
    for lv in (prm.top, 2, 1):
        a, b = he.drop(cx, lv), he.drop(cy, lv)
        r = he.mul_relin_rescale(a, b)
        assert np.abs(he.decrypt(r) - x * y).max() < 1e-6
        assert np.abs(he.decrypt(he.rotate(a, 3)) - np.roll(x, -3)).max() < 1e-6


def test_rotation_identities():
    prm = _params(log_n=7)
    he = ckks.Ckks(prm)
    he.keygen(19, [1, 2, -1, 5])
    rng = np.random.default_rng(6)
    x = rng.normal(size=prm.slots)
    cx = he.encrypt(x, prm.top, 1)
    for r in (1, 2, -1, 5):
        assert np.abs(he.decrypt(he.rotate(cx, r)) - np.roll(x, -r)).max() < 1e-6
    # rotation by the slot count is the identity (5 has order N/2 modulo 2N)
    assert prm.galois(prm.slots) == 1
    # rot(rot(x, 1), 1) = rot(x, 2)
    assert np.abs(he.decrypt(he.rotate(he.rotate(cx, 1), 1)) - np.roll(x, -2)).max() < 1e-6


def test_rotation_key_switches_from_rotated_secret():
    """decrypt under phi_g(s) of (phi_g(c0), phi_g(c1)) equals phi_g applied to the plaintext."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(23, [1])
    g = prm.galois(1)
    rng = np.random.default_rng(7)
    cx = he.encrypt(rng.normal(size=prm.slots), prm.top, 1)
    q = prm.q[0]
    s = ckks.to_rns(he.s, [q])[0]
    m = (cx.c[0][0].astype(object) + ring.polymul(cx.c[1][0], s, q).astype(object)) % q
    m_g = ring.automorphism(np.array(m, dtype=np.uint64), g, q)
    c0g = ring.automorphism(cx.c[0][0], g, q)
    c1g = ring.automorphism(cx.c[1][0], g, q)
    s_g = ring.automorphism(s, g, q)
    lhs = (c0g.astype(object) + ring.polymul(c1g, s_g, q).astype(object)) % q
    assert [int(v) for v in lhs] == [int(v) for v in m_g]


def _int_automorphism(a, g):
    """a(X^g) in Z[X]/(X^N + 1), written out from the definition: X^i -> (+/-) X^(g i mod N)."""
    n = len(a)
    out = [0] * n
    for i, v in enumerate(a):
        e = (g * i) % (2 * n)
        if e < n:
            out[e] += v
        else:
            out[e - n] -= v
    return out


def _hoist_setup(log_n=6, steps=range(1, 8), seed=29):
    prm = ckks.Params(log_n, (50,) * 4, (60, 60), 50)   # alpha = 2: two digits at the top level
    he = ckks.Ckks(prm)
    he.keygen(seed, list(steps))
    rng = np.random.default_rng(seed)
    x = rng.normal(size=prm.slots)
    return prm, he, x, he.encrypt(x, prm.top, 1)


def test_hoisted_rotate_sum_is_sum_of_automorphisms_plus_small_noise():
    """decrypt(rotate_sum_hoisted(ct, 0..7)) = sum_r phi_(5^r)(decrypt(ct)) + key-switch noise, in Z[X]/(X^N+1).

    A wrong permutation, key, digit or ModDown term leaves an error of the order of the modulus."""
    prm, he, x, ct = _hoist_setup()
    steps = list(range(8))
    m = he.decrypt_coeffs(ct)
    want = [0] * prm.n
    for r in steps:
        for i, v in enumerate(_int_automorphism(m, pow(5, r, 2 * prm.n))):
            want[i] += v
    for lv in (prm.top, 2):
        got = he.decrypt_coeffs(he.rotate_sum_hoisted(he.drop(ct, lv), steps))
        err = max(abs(a - b) for a, b in zip(got, want))
        assert err < (1 << 16), (lv, err)


def test_hoisted_rotate_sum_slots_and_special_cases():
    prm, he, x, ct = _hoist_setup()
    S = he.rotate_sum_hoisted(ct, range(8))
    want = sum(np.roll(x, -r) for r in range(8))
    assert np.abs(he.decrypt(S) - want).max() < 1e-6
    # step 0 alone is the ciphertext itself, bit for bit
    I = he.rotate_sum_hoisted(ct, [0])
    assert (I.c == ct.c).all()
    # one step: the same plaintext as rotate() (the bits differ: phi is applied after ModUp)
    one = he.rotate_sum_hoisted(ct, [3])
    assert np.abs(he.decrypt(one) - np.roll(x, -3)).max() < 1e-6
    # the sum is order-free: modular additions commute exactly
    perm = he.rotate_sum_hoisted(ct, [5, 0, 7, 2, 1, 6, 3, 4])
    assert (perm.c == S.c).all()
    # hoisting changes only noise: against sequential rotate-and-adds
    seq = ct
    for t in range(3):
        seq = he.add(seq, he.rotate(seq, 1 << t))
    assert np.abs(he.decrypt(seq) - he.decrypt(S)).max() < 1e-6


def test_relin_rescale_without_d2_is_floor_rescale():
    """With d2 = 0 the fused relinearise-rescale is the floor division of (c0, c1) by q_l, exactly
    (big-integer CRT over Q_l, then floor(c / q_l) reduced modulo each q_i, i < l)."""
    prm = ckks.Params(5, (50,) * 4, (60, 60), 50)
    he = ckks.Ckks(prm)
    he.keygen(31)
    rng = np.random.default_rng(9)
    lv = prm.top
    c = np.stack([np.stack([rng.integers(0, q, prm.n, dtype=np.uint64) for q in prm.q]) for _ in range(2)])
    t = ckks.Ciphertext(np.concatenate([c, np.zeros((1, lv + 1, prm.n), dtype=np.uint64)]), lv)
    got = he.relin_rescale(t)
    Q = math.prod(prm.q[: lv + 1])
    for h in range(2):
        for k in range(prm.n):
            x = 0
            for i, q in enumerate(prm.q[: lv + 1]):
                qi_hat = Q // q
                x += int(c[h][i][k]) * qi_hat * pow(qi_hat, -1, q)
            x %= Q
            f = x // prm.q[lv]
            assert [int(got.c[h][i][k]) for i in range(lv)] == [f % q for q in prm.q[:lv]]


def test_relin_rescale_matches_two_step_up_to_conversion_error():
    """decrypt(relin_rescale(a (x) b)) differs from decrypt(rescale(relinearize(a (x) b))) by
    e0 + e1 s with |e0|, |e1| <= alpha + 1 per coefficient; slots hold the product."""
    for prm in (ckks.Params(6, (50,) * 4, (60, 60), 50), ckks.Params(6, (60, 40, 40), (60,), 40)):
        he = ckks.Ckks(prm)
        he.keygen(37)
        rng = np.random.default_rng(10)
        x, y = rng.normal(size=prm.slots), rng.normal(size=prm.slots)
        cx, cy = he.encrypt(x, prm.top, 1), he.encrypt(y, prm.top, 2)
        for lv in sorted({prm.top, 1}):
            t = he.tensor(he.drop(cx, lv), he.drop(cy, lv))
            fused = he.relin_rescale(t)
            two = he.rescale(he.relinearize(t))
            assert fused.level == two.level == lv - 1
            d = [a - b for a, b in zip(he.decrypt_coeffs(fused), he.decrypt_coeffs(two))]
            assert max(abs(v) for v in d) <= (prm.alpha + 1) * (prm.n + 1)
            assert np.abs(he.decrypt(fused) - x * y).max() < 1e-5


def test_uniform_indexed_sampler():
    """Uniform residues, each coefficient from its own draws: the first-try value is the SplitMix64
    output x_k mod q whenever x_k is below floor(2^64/q) q."""
    q = ckks.gen_primes(10, [50])[0]
    h = ckks.stream_key(5, ckks.P_SEEDED_A, 3, 0, 1)
    u = ckks.sample_uniform_indexed(h, 4096, q)
    assert (u < np.uint64(q)).all()
    assert abs(float(np.mean(u.astype(np.float64))) / q - 0.5) < 0.02
    x = ckks.draws(h, 0, 4096)
    ok = x < np.uint64(((1 << 64) // q) * q)
    assert (u[ok] == x[ok] % np.uint64(q)).all()
    # just above 2^63 the bound is q itself, so about half the first draws are rejected; the
    # retries keep the values uniform
    q3 = 9223372036854775837   # the first prime above 2^63
    v = ckks.sample_uniform_indexed(h, 20000, q3)
    x = ckks.draws(h, 0, 20000)
    assert 0.45 < float(np.mean(x >= np.uint64(q3))) < 0.55
    assert (v < np.uint64(q3)).all() and abs(float(np.mean(v.astype(np.float64))) / q3 - 0.5) < 0.02


def test_encrypt_seeded_exact_error_and_regenerable_c1():
    """decrypt(encrypt_seeded(m)) = m + e exactly, with e the seeded Gaussian stream; c1 is the
    uniform stream of (seed, object) and nothing else."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(41)
    rng = np.random.default_rng(4)
    m = rng.integers(-(1 << 40), 1 << 40, size=prm.n)
    ct = he.encrypt_seeded(m, prm.top - 1, 77)
    e = ckks.sample_gaussian(ckks.stream_key(41, ckks.P_SEEDED_E, 77), prm.n, 3.2)
    assert he.decrypt_coeffs(ct) == [int(a) + int(b) for a, b in zip(m, e)]
    for i, q in enumerate(prm.q[: prm.top]):
        a = ckks.sample_uniform_indexed(ckks.stream_key(41, ckks.P_SEEDED_A, 77, 0, i), prm.n, q)
        assert (ct.c[1][i] == a).all()


def _centred_plaintext(he, ct):
    """c0 + c1 s over the ciphertext's two lowest limbs, lifted to Z_{q0 q1} by CRT and centred,
    with the secret product taken in the integers (the decryption definition, written out)."""
    q0, q1 = he.prm.q[0], he.prm.q[1]
    Q, inv = q0 * q1, pow(q0, -1, q1)

    def lift(comp):
        x0, x1 = ct.c[comp][0].tolist(), ct.c[comp][1].tolist()
        return [a + q0 * (((b - a) * inv) % q1) for a, b in zip(x0, x1)]
    c0, c1s = lift(0), _int_negacyclic(lift(1), he.s.tolist())
    out = []
    for a, b in zip(c0, c1s):
        v = (a + b) % Q
        out.append(v - Q if v > Q // 2 else v)
    return out


def test_refresh_is_a_fresh_encryption_of_the_exact_plaintext():
    """refresh(ct) = Enc_top(c0 + c1 s; nonce): encryption is (v pk0 + e0 + m, v pk1 + e1), so it
    differs from the same nonce's encryption of zero by (m, 0) exactly, m the centred integer
    plaintext of the level-1 input."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(13)
    rng = np.random.default_rng(5)
    m0 = rng.integers(-(1 << 38), 1 << 38, size=prm.n)
    ct = he.drop(he.encrypt_coeffs(m0, prm.top, 5), 1)
    pt = _centred_plaintext(he, ct)
    assert max(abs(p - int(a)) for p, a in zip(pt, m0)) < 1 << 12      # m0 plus a fresh error
    r = he.refresh(ct, 9)
    z = he.encrypt_coeffs(np.zeros(prm.n, dtype=np.int64), prm.top, 9)
    assert r.level == prm.top
    for i, q in enumerate(prm.q[: prm.top + 1]):
        assert all((int(x) - int(y) - p) % q == 0 for x, y, p in zip(r.c[0][i], z.c[0][i], pt))
        assert (r.c[1][i] == z.c[1][i]).all()


def test_mul_plain_multiplies_the_integer_plaintext():
    """Eq. 9: the integer plaintext of ct (.) p is p times that of ct in Z[X]/(X^N + 1), exactly,
    while it stays below q0 q1 / 2."""
    prm = _params(log_n=5)
    he = ckks.Ckks(prm)
    he.keygen(17)
    rng = np.random.default_rng(6)
    ct = he.drop(he.encrypt_coeffs(rng.integers(-(1 << 30), 1 << 30, size=prm.n), prm.top, 3), 1)
    p = np.zeros(prm.n, dtype=np.int64)
    p[[0, 3, prm.n - 1]] = [1000, -7, 1 << 20]
    got = _centred_plaintext(he, he.mul_plain(ct, p))
    assert got == _int_negacyclic(p.tolist(), _centred_plaintext(he, ct))


def test_rotate_fanin_is_the_sum_of_rotations_plus_small_noise():
    """decrypt(rotate_fanin(cts, steps)) = sum_i phi_(5^r_i)(decrypt(cts[i])) in Z[X]/(X^N+1) up to the
    key-switch noise, and the slots are the sum of the rotated slot vectors; one input reduces to one
    rotation (same plaintext), and the order of the inputs does not change the bits."""
    prm = ckks.Params(8, (50, 40, 40), (60,), 40)
    he = ckks.Ckks(prm)
    steps = [3, -5, 7]
    he.keygen(21, steps)
    rng = np.random.default_rng(22)
    zs = [rng.normal(0, 1, prm.slots) for _ in steps]
    cts = [he.encrypt(z, prm.top, 40 + i) for i, z in enumerate(zs)]
    out = he.rotate_fanin(cts, steps)
    want = sum(np.roll(z, -r) for z, r in zip(zs, steps))
    assert np.abs(he.decrypt(out) - want).max() < 1e-6
    seq = he.add(he.add(he.rotate(cts[0], 3), he.rotate(cts[1], -5)), he.rotate(cts[2], 7))
    d_out = he.decrypt_coeffs(out)
    d_seq = he.decrypt_coeffs(seq)
    assert max(abs(a - b) for a, b in zip(d_out, d_seq)) < 2 ** 20          # noise, far below Delta = 2^40
    assert (out.c != seq.c).any()                                           # one ModDown, other bits
    perm = he.rotate_fanin([cts[2], cts[0], cts[1]], [7, 3, -5])
    assert (perm.c == out.c).all()
    one = he.rotate_fanin([cts[1]], [-5])
    assert (one.c == he.rotate(cts[1], -5).c).all()                         # one input: the plain key switch
    assert np.abs(he.decrypt(one) - np.roll(zs[1], 5)).max() < 1e-6
