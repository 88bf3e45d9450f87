"""Oracle RNS-CKKS — TEST INFRASTRUCTURE ONLY.

A plain, slow, exact CPU implementation of the leveled CKKS scheme the paper
runs its encrypted matrix factorisation on (Sec. II-A.2, Eq. 6-9; Sec. IV-A:
CKKS, N = 8192, 128-bit security). Only tests/, the smoke check and the
benchmark's CPU-baseline leg may import it; the CUDA library never does, and
the two share no code.

Everything is kept in COEFFICIENT form: a ring element modulo q_i is a
length-N uint64 array of residues; an RNS polynomial at level l is [l+1, N].
Ring products use oracle/ring.c (a textbook NTT pinned to the schoolbook
definition). Where the paper is silent the scheme follows the published
literature (Cheon-Kim-Kim-Song 2017; full-RNS CKKS of Cheon-Han-Kim-Kim-Song
2018; hybrid key switching of Han-Ki 2020; fast base conversion of Bajard et
al. 2016), with these fixed readings:

  * primes: per bit size b in list order (data primes q_0.., then special
    primes p_0..), the largest unused prime below 2^b that is 1 mod 2N;
  * randomness: one master seed; SplitMix64 (Steele-Lea-Flood 2014) streams
    keyed by (purpose, object, poly, limb); uniform residues and ternary
    values by rejection; rounded Gaussian (sigma 3.2, |e| <= 19) by a
    cumulative table;
  * encoding: slot t <-> evaluation at zeta^(5^t), zeta = exp(i*pi/N); real
    slots only; coefficient j = rint((2*Delta/N) * sum_t z_t cos(pi*(j*5^t mod 2N)/N)),
    the sum taken in ascending t over non-zero slots in IEEE double;
  * rescale: exact round(c / q_l) with the centred representative;
  * key switching: digits of alpha consecutive limbs from limb 0, fast
    (uncorrected) conversion in ModUp and ModDown, one key for all levels.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import ring

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# sampling purposes (the first field of every stream key)
P_SECRET, P_PK_A, P_PK_E, P_EVK_A, P_EVK_E, P_ENC_V, P_ENC_E0, P_ENC_E1 = 1, 2, 3, 4, 5, 6, 7, 8
P_SEEDED_A, P_SEEDED_E = 9, 10   # key-holder encryption with a regenerable c1 (object = the ciphertext's id)
SEEDED_TRIES = 16
RELIN_OBJECT = 0


# ----------------------------------------------------------------------------- primes

def gen_primes(log_n: int, bits: Sequence[int]) -> List[int]:
    """Largest unused primes q < 2^b with q = 1 mod 2N, one per entry of bits, in order."""
    two_n = 1 << (log_n + 1)
    chosen: List[int] = []
    for b in bits:
        c = (1 << b) + 1 - two_n
        while True:
            if c < two_n:
                raise ValueError(f"no {b}-bit prime = 1 mod {two_n}")
            if c not in chosen and _is_prime_py(c):
                chosen.append(c)
                break
            c -= two_n
    return chosen


def _is_prime_py(n: int) -> bool:
    """Deterministic Miller-Rabin with the first 12 prime bases (exact for n < 3.3e24)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


# ----------------------------------------------------------------------------- parameters

@dataclasses.dataclass
class Params:
    log_n: int
    data_bits: Tuple[int, ...]
    special_bits: Tuple[int, ...]
    log_scale: int
    sigma: float = 3.2

    def __post_init__(self):
        self.n = 1 << self.log_n
        self.slots = self.n // 2
        allp = gen_primes(self.log_n, tuple(self.data_bits) + tuple(self.special_bits))
        self.q = allp[: len(self.data_bits)]
        self.p = allp[len(self.data_bits):]
        self.alpha = len(self.p)
        self.top = len(self.q) - 1          # top level L
        self.ext = self.q + self.p          # extended basis Q_L u P
        self.P = math.prod(self.p)
        self.delta = 1 << self.log_scale

    @classmethod
    def from_preset(cls, preset) -> "Params":
        return cls(preset.log_n, tuple(preset.data_bits), tuple(preset.special_bits),
                   preset.log_scale, preset.sigma)

    def dnum(self, level: int) -> int:
        return -(-(level + 1) // self.alpha)

    def digit(self, j: int, level: int) -> List[int]:
        return list(range(j * self.alpha, min((j + 1) * self.alpha, level + 1)))

    def galois(self, r: int) -> int:
        """Galois element of a left slot rotation by r: 5^(r mod N/2) mod 2N."""
        return pow(5, r % self.slots, 2 * self.n)


# ----------------------------------------------------------------------------- SplitMix64 sampling

def _mix64_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def stream_key(master: int, purpose: int, obj: int = 0, poly: int = 0, limb: int = 0) -> int:
    """h <- mix64((h xor f) + gamma) for f in (purpose, object, poly, limb), from h = master."""
    h = master & MASK64
    for f in (purpose, obj, poly, limb):
        h = _mix64_int(((h ^ (f & MASK64)) + GAMMA) & MASK64)
    return h


def draws(h: int, start: int, count: int) -> np.ndarray:
    """SplitMix64 outputs number start..start+count-1 of the stream with state h:
    x_c = mix64(h + (c + 1) * gamma)."""
    ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64_np(np.uint64(h) + ctr * np.uint64(GAMMA))


def _rejection(h: int, n: int, bound: int) -> np.ndarray:
    out = np.empty(0, dtype=np.uint64)
    start = 0
    while out.size < n:
        chunk = max(64, (n - out.size) * 2)
        x = draws(h, start, chunk)
        start += chunk
        out = np.concatenate([out, x[x < np.uint64(bound)]])
    return out[:n]


def sample_uniform(h: int, n: int, q: int) -> np.ndarray:
    """n residues uniform mod q: accept x < floor(2^64/q)*q, value x mod q."""
    bound = ((1 << 64) // q) * q
    return _rejection(h, n, bound) % np.uint64(q)


def sample_uniform_indexed(h: int, n: int, q: int, tries: int = SEEDED_TRIES) -> np.ndarray:
    """n residues uniform mod q, coefficient k drawn on its own: the first of the stream outputs
    x_{jn + k}, j = 0..tries-1, below floor(2^64/q)*q, reduced mod q (x_{(tries-1)n + k} mod q if
    none is). Any coefficient can thus be regenerated without the others."""
    bound = np.uint64(((1 << 64) // q) * q)
    out = np.zeros(n, dtype=np.uint64)
    done = np.zeros(n, dtype=bool)
    for j in range(tries):
        x = draws(h, j * n, n)
        take = ~done & ((x < bound) | (j == tries - 1))
        out[take] = x[take] % np.uint64(q)
        done |= take
    return out


def sample_ternary(h: int, n: int) -> np.ndarray:
    """n values uniform in {-1, 0, 1}: accept x < floor(2^64/3)*3, value (x mod 3) - 1."""
    bound = ((1 << 64) // 3) * 3
    return (_rejection(h, n, bound) % np.uint64(3)).astype(np.int64) - 1


def gaussian_table(sigma: float) -> List[int]:
    """T[k] = floor(2^63 * P(|e| <= k)), k = 0..18, for the rounded Gaussian on |e| <= 19."""
    two_sigma_sq = 2.0 * sigma * sigma
    rho = [math.exp(-(x * x) / two_sigma_sq) for x in range(20)]
    tail = 0.0
    for x in range(1, 20):
        tail = tail + rho[x]
    norm = rho[0] + 2.0 * tail
    cdf = 0.0
    table = []
    for k in range(19):
        pk = rho[0] / norm if k == 0 else 2.0 * rho[k] / norm
        cdf = cdf + pk
        table.append(int(cdf * 9223372036854775808.0))
    return table


def sample_gaussian(h: int, n: int, sigma: float) -> np.ndarray:
    """One draw per value: sign = bit 0, u = x >> 1, |e| = #{k : u >= T[k]}."""
    x = draws(h, 0, n)
    u = x >> np.uint64(1)
    mag = np.zeros(n, dtype=np.int64)
    for t in gaussian_table(sigma):
        mag += (u >= np.uint64(t)).astype(np.int64)
    sign = (x & np.uint64(1)).astype(np.int64)
    return np.where(sign == 1, -mag, mag)


def to_rns(coeffs: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    """Signed integer coefficients -> [len(primes), N] residues."""
    c = np.asarray(coeffs)
    out = np.empty((len(primes), c.shape[-1]), dtype=np.uint64)
    for i, q in enumerate(primes):
        if c.dtype == object:
            out[i] = np.array([int(v) % q for v in c], dtype=np.uint64)
        else:
            out[i] = np.mod(c.astype(np.int64), np.int64(q)).astype(np.uint64)
    return out


# ----------------------------------------------------------------------------- encoding

class Encoder:
    """Canonical-embedding encoder for real slot vectors (definition-level O(N * N/2) sums)."""

    def __init__(self, params: Params):
        self.prm = params
        n = params.n
        self.cos_tab = np.array([math.cos(math.pi * e / n) for e in range(2 * n)], dtype=np.float64)
        self.pow5 = np.array([pow(5, t, 2 * n) for t in range(params.slots)], dtype=np.int64)
        self.j = np.arange(n, dtype=np.int64)

    def encode(self, z, log_scale: Optional[int] = None) -> np.ndarray:
        """Real slots z (len <= N/2) -> int64 coefficients of round(Delta * m(X))."""
        prm = self.prm
        ls = prm.log_scale if log_scale is None else log_scale
        z = np.asarray(z, dtype=np.float64)
        if z.size > prm.slots:
            raise ValueError("too many slots")
        two_n = 2 * prm.n
        acc = np.zeros(prm.n, dtype=np.float64)
        for t in range(z.size):
            zt = z[t]
            if zt != 0.0:
                acc = acc + zt * self.cos_tab[(self.j * self.pow5[t]) % two_n]
        factor = 2.0 ** (ls + 1 - prm.log_n)   # 2*Delta/N, a power of two
        return np.rint(acc * factor).astype(np.int64)

    def decode(self, m_coeffs, log_scale: Optional[int] = None, count: Optional[int] = None) -> np.ndarray:
        """Centred integer coefficients -> real parts of the first `count` slots / Delta."""
        prm = self.prm
        ls = prm.log_scale if log_scale is None else log_scale
        count = prm.slots if count is None else count
        m = np.array([float(int(v)) for v in m_coeffs], dtype=np.float64)
        two_n = 2 * prm.n
        out = np.empty(count, dtype=np.float64)
        step = 128
        for t0 in range(0, count, step):
            t = np.arange(t0, min(count, t0 + step))
            idx = (self.j[None, :] * self.pow5[t][:, None]) % two_n
            out[t] = self.cos_tab[idx] @ m
        return out / float(1 << ls)


# ----------------------------------------------------------------------------- keys and ciphertexts

@dataclasses.dataclass
class Ciphertext:
    """Components [k, level+1, N] (k = 2, or 3 after a tensor product), coefficient form."""
    c: np.ndarray
    level: int

    def copy(self) -> "Ciphertext":
        return Ciphertext(self.c.copy(), self.level)


@dataclasses.dataclass
class EvalKey:
    """Hybrid key-switching key: b, a of shape [dnum_top, L+1+alpha, N]."""
    b: np.ndarray
    a: np.ndarray


class Ckks:
    def __init__(self, params: Params):
        self.prm = params
        self.enc = Encoder(params)
        self.seed: Optional[int] = None
        self.s: Optional[np.ndarray] = None
        self.pk: Optional[np.ndarray] = None
        self.rlk: Optional[EvalKey] = None
        self.rot: Dict[int, EvalKey] = {}

    # ---- primitive ring helpers (per-limb, coefficient form)

    def _add(self, a, b, primes):
        out = np.empty_like(a)
        for i, q in enumerate(primes):
            s = a[i] + b[i]
            out[i] = np.where(s >= np.uint64(q), s - np.uint64(q), s)
        return out

    def _sub(self, a, b, primes):
        out = np.empty_like(a)
        for i, q in enumerate(primes):
            out[i] = np.where(a[i] >= b[i], a[i] - b[i], a[i] + (np.uint64(q) - b[i]))
        return out

    def _neg(self, a, primes):
        out = np.empty_like(a)
        for i, q in enumerate(primes):
            out[i] = np.where(a[i] == 0, a[i], np.uint64(q) - a[i])
        return out

    def _mul(self, a, b, primes):
        return np.stack([ring.polymul(a[i], b[i], q) for i, q in enumerate(primes)])

    # ---- key generation

    def keygen(self, seed: int, rot_steps: Iterable[int] = ()) -> None:
        prm = self.prm
        self.seed = seed & MASK64
        n = prm.n
        self.s = sample_ternary(stream_key(seed, P_SECRET), n)
        s_q = to_rns(self.s, prm.q)
        a = np.stack([sample_uniform(stream_key(seed, P_PK_A, 0, 0, i), n, q)
                      for i, q in enumerate(prm.q)])
        e = to_rns(sample_gaussian(stream_key(seed, P_PK_E), n, prm.sigma), prm.q)
        pk0 = self._add(self._neg(self._mul(a, s_q, prm.q), prm.q), e, prm.q)
        self.pk = np.stack([pk0, a])
        s_ext = to_rns(self.s, prm.ext)
        s2 = self._mul(s_ext, s_ext, prm.ext)
        self.rlk = self._evk(s2, RELIN_OBJECT)
        for r in rot_steps:
            self.add_rotation_key(r)

    def add_rotation_key(self, r: int) -> None:
        prm = self.prm
        g = prm.galois(r)
        if g in self.rot:
            return
        s_g = np.stack([ring.automorphism(x, g, q) for x, q in zip(to_rns(self.s, prm.ext), prm.ext)])
        self.rot[g] = self._evk(s_g, g)

    def _evk(self, s_prime: np.ndarray, obj: int) -> EvalKey:
        """evk_j = (-a_j s + e_j + [i in D_j] (P mod q_i) s', a_j) over Q_L u P, j < dnum(L)."""
        prm = self.prm
        n = prm.n
        s_ext = to_rns(self.s, prm.ext)
        dn = prm.dnum(prm.top)
        B = np.empty((dn, len(prm.ext), n), dtype=np.uint64)
        A = np.empty_like(B)
        for j in range(dn):
            a = np.stack([sample_uniform(stream_key(self.seed, P_EVK_A, obj, j, t), n, q)
                          for t, q in enumerate(prm.ext)])
            e = to_rns(sample_gaussian(stream_key(self.seed, P_EVK_E, obj, j, 0), n, prm.sigma), prm.ext)
            b = self._add(self._neg(self._mul(a, s_ext, prm.ext), prm.ext), e, prm.ext)
            for i in prm.digit(j, prm.top):
                q = prm.q[i]
                term = ring.scalar_mul(s_prime[i], prm.P % q, q)
                b[i] = self._add(b[i][None], term[None], [q])[0]
            B[j], A[j] = b, a
        return EvalKey(B, A)

    # ---- encryption / decryption

    def encrypt_coeffs(self, m: np.ndarray, level: int, nonce: int) -> Ciphertext:
        """ct = (v*pk0 + e0 + m, v*pk1 + e1) mod Q_level."""
        prm = self.prm
        n = prm.n
        primes = prm.q[: level + 1]
        v = to_rns(sample_ternary(stream_key(self.seed, P_ENC_V, nonce), n), primes)
        e0 = to_rns(sample_gaussian(stream_key(self.seed, P_ENC_E0, nonce), n, prm.sigma), primes)
        e1 = to_rns(sample_gaussian(stream_key(self.seed, P_ENC_E1, nonce), n, prm.sigma), primes)
        mm = to_rns(m, primes)
        c0 = self._add(self._add(self._mul(v, self.pk[0][: level + 1], primes), e0, primes), mm, primes)
        c1 = self._add(self._mul(v, self.pk[1][: level + 1], primes), e1, primes)
        return Ciphertext(np.stack([c0, c1]), level)

    def encrypt_seeded(self, m: np.ndarray, level: int, obj: int) -> Ciphertext:
        """Key-holder (symmetric) encryption whose c1 is regenerable from (seed, obj):
        c1 = a with a_i = sample_uniform_indexed(stream_key(seed, P_SEEDED_A, obj, 0, i), N, q_i)
        (coefficient form), e from stream_key(seed, P_SEEDED_E, obj), c0 = -a s + m + e mod Q_level.
        A holder of the seed stores c0 only."""
        prm = self.prm
        n = prm.n
        primes = prm.q[: level + 1]
        a = np.stack([sample_uniform_indexed(stream_key(self.seed, P_SEEDED_A, obj, 0, i), n, q)
                      for i, q in enumerate(primes)])
        e = to_rns(sample_gaussian(stream_key(self.seed, P_SEEDED_E, obj), n, prm.sigma), primes)
        s_q = to_rns(self.s, primes)
        c0 = self._add(self._add(self._neg(self._mul(a, s_q, primes), primes), e, primes), to_rns(m, primes), primes)
        return Ciphertext(np.stack([c0, a]), level)

    def encrypt(self, z, level: int, nonce: int) -> Ciphertext:
        return self.encrypt_coeffs(self.enc.encode(z), level, nonce)

    def decrypt_coeffs(self, ct: Ciphertext) -> List[int]:
        """m = c0 + c1*s mod Q_l, lifted to the centred integer modulo q_0 q_1 (q_0 at level 0)."""
        prm = self.prm
        lv = min(ct.level, 1)
        primes = prm.q[: lv + 1]
        s_q = to_rns(self.s, primes)
        m = self._add(ct.c[0][: lv + 1], self._mul(ct.c[1][: lv + 1], s_q, primes), primes)
        Q = math.prod(primes)
        out = []
        if lv == 0:
            q0 = primes[0]
            for v in m[0]:
                v = int(v)
                out.append(v - q0 if v > q0 // 2 else v)
        else:
            q0, q1 = primes
            inv = pow(q0, -1, q1)
            for x0, x1 in zip(m[0], m[1]):
                x0, x1 = int(x0), int(x1)
                v = x0 + q0 * (((x1 - x0) * inv) % q1)
                out.append(v - Q if v > Q // 2 else v)
        return out

    def refresh(self, ct: Ciphertext, nonce: int) -> Ciphertext:
        """Key-holder refresh: the exact integer plaintext m = c0 + c1 s (centred, from the
        lowest two limbs as in decryption) re-encrypted at the top level with `nonce`."""
        m = np.array(self.decrypt_coeffs(ct), dtype=object)
        return self.encrypt_coeffs(m, self.prm.top, nonce)

    def decrypt(self, ct: Ciphertext, count: Optional[int] = None) -> np.ndarray:
        return self.enc.decode(self.decrypt_coeffs(ct), count=count)

    # ---- homomorphic operations (Eq. 6-9)

    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        lv = min(a.level, b.level)
        pr = self.prm.q[: lv + 1]
        k = max(a.c.shape[0], b.c.shape[0])
        out = np.zeros((k, lv + 1, self.prm.n), dtype=np.uint64)
        for t in range(k):
            x = a.c[t][: lv + 1] if t < a.c.shape[0] else np.zeros_like(out[0])
            y = b.c[t][: lv + 1] if t < b.c.shape[0] else np.zeros_like(out[0])
            out[t] = self._add(x, y, pr)
        return Ciphertext(out, lv)

    def sub(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        lv = min(a.level, b.level)
        pr = self.prm.q[: lv + 1]
        out = np.stack([self._sub(a.c[t][: lv + 1], b.c[t][: lv + 1], pr) for t in range(2)])
        return Ciphertext(out, lv)

    def drop(self, a: Ciphertext, level: int) -> Ciphertext:
        return Ciphertext(a.c[:, : level + 1].copy(), level)

    def mul_plain(self, a: Ciphertext, m: np.ndarray) -> Ciphertext:
        """ct (.) pt: each component times the plaintext polynomial (Eq. 9)."""
        pr = self.prm.q[: a.level + 1]
        mm = to_rns(m, pr)
        return Ciphertext(np.stack([self._mul(a.c[t], mm, pr) for t in range(a.c.shape[0])]), a.level)

    def tensor(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        """(a0 b0, a0 b1 + a1 b0, a1 b1)."""
        lv = min(a.level, b.level)
        pr = self.prm.q[: lv + 1]
        A, B = a.c[:, : lv + 1], b.c[:, : lv + 1]
        d0 = self._mul(A[0], B[0], pr)
        d1 = np.stack([ring.polydot(np.stack([A[0][i], A[1][i]]), np.stack([B[1][i], B[0][i]]), q)
                       for i, q in enumerate(pr)])
        d2 = self._mul(A[1], B[1], pr)
        return Ciphertext(np.stack([d0, d1, d2]), lv)

    def rescale(self, a: Ciphertext) -> Ciphertext:
        pr = self.prm.q[: a.level + 1]
        out = np.stack([ring.rescale(a.c[t], pr) for t in range(a.c.shape[0])])
        return Ciphertext(out, a.level - 1)

    def _key_rows(self, level: int) -> List[int]:
        """Rows of a key (stored over Q_L u P) that belong to the basis Q_level u P."""
        prm = self.prm
        return list(range(level + 1)) + [prm.top + 1 + k for k in range(prm.alpha)]

    def _modup(self, d: np.ndarray, level: int) -> np.ndarray:
        """ModUp_j(d) for every digit j: fast conversion of the digit-j residues of d to every
        prime of Q_level u P (Bajard et al. 2016). Shape [dnum, |basis|, N]."""
        prm = self.prm
        basis = prm.q[: level + 1] + prm.p
        ups = []
        for j in range(prm.dnum(level)):
            Dj = prm.digit(j, level)
            ups.append(ring.fast_base_conv(d[Dj], [prm.q[i] for i in Dj], basis))
        return np.stack(ups)

    def _moddown(self, acc: np.ndarray, level: int) -> np.ndarray:
        """ModDown(x) = (x_Q - Conv_{P->Q}(x_P)) * P^{-1} mod each q_i."""
        prm = self.prm
        qs = prm.q[: level + 1]
        xq, xp = acc[: level + 1], acc[level + 1:]
        conv = ring.fast_base_conv(xp, prm.p, qs)
        diff = self._sub(xq, conv, qs)
        out = np.empty_like(diff)
        for i, q in enumerate(qs):
            out[i] = ring.scalar_mul(diff[i], pow(prm.P % q, -1, q), q)
        return out

    def keyswitch(self, d: np.ndarray, level: int, key: EvalKey) -> Tuple[np.ndarray, np.ndarray]:
        """Hybrid key switch of one polynomial d (level l, [l+1, N]) under key (Han-Ki 2020).

        ModUp_j(d) = fast conversion of the digit-j residues to every prime of Q_l u P;
        acc = sum_j ModUp_j(d) * evk_j; ModDown(x) = (x_Q - Conv_{P->Q}(x_P)) * P^{-1}.
        """
        prm = self.prm
        basis = prm.q[: level + 1] + prm.p
        rows = self._key_rows(level)
        dn = prm.dnum(level)
        ups = self._modup(d, level)  # [dnum, |basis|, N]
        halves = []
        for K in (key.b, key.a):
            Kx = K[:dn][:, rows]  # [dnum, |basis|, N]
            acc = ring.polydot_rows(np.ascontiguousarray(ups.transpose(1, 0, 2)),
                                    np.ascontiguousarray(Kx.transpose(1, 0, 2)), basis)
            halves.append(self._moddown(acc, level))
        return halves[0], halves[1]

    def relinearize(self, t: Ciphertext) -> Ciphertext:
        pr = self.prm.q[: t.level + 1]
        k0, k1 = self.keyswitch(t.c[2], t.level, self.rlk)
        return Ciphertext(np.stack([self._add(t.c[0], k0, pr), self._add(t.c[1], k1, pr)]), t.level)

    def relin_rescale(self, t: Ciphertext) -> Ciphertext:
        """Relinearise and rescale in one step (level l -> l - 1): the key switch's ModDown divides
        by P q_l instead of P. With acc_h = sum_j ModUp_j(d2) evk_j[h] over Q_l u P and
        X_h = acc_h + P c_h (c_h the tensor's component h, which is zero on the P limbs):
            out_h = (X_h - Conv_{P u {q_l} -> Q_{l-1}}(X_h)) (P q_l)^{-1}  mod q_i, i < l,
        Conv being the fast (non-centred) base conversion. It equals floor(X_h / (P q_l)) - u with
        0 <= u <= alpha, where rescale(relinearize(t)) rounds in two steps."""
        prm = self.prm
        lv = t.level
        if lv < 1:
            raise ValueError("relin_rescale needs level >= 1")
        qs = prm.q[: lv + 1]
        basis = qs + prm.p
        rows = self._key_rows(lv)
        dn = prm.dnum(lv)
        ups = self._modup(t.c[2][: lv + 1], lv)
        src_primes = [qs[lv]] + list(prm.p)
        dst = qs[:lv]
        Mp = prm.P * qs[lv]
        out = []
        for h, K in enumerate((self.rlk.b, self.rlk.a)):
            Kx = K[:dn][:, rows]
            acc = ring.polydot_rows(np.ascontiguousarray(ups.transpose(1, 0, 2)),
                                    np.ascontiguousarray(Kx.transpose(1, 0, 2)), basis)
            X = acc.copy()
            for i, q in enumerate(qs):
                X[i] = self._add(acc[i][None], ring.scalar_mul(t.c[h][i], prm.P % q, q)[None], [q])[0]
            src = np.stack([X[lv]] + [X[lv + 1 + k] for k in range(prm.alpha)])
            conv = ring.fast_base_conv(src, src_primes, dst)
            diff = self._sub(X[:lv], conv, dst)
            res = np.empty_like(diff)
            for i, q in enumerate(dst):
                res[i] = ring.scalar_mul(diff[i], pow(Mp % q, -1, q), q)
            out.append(res)
        return Ciphertext(np.stack(out), lv - 1)

    def rotate(self, a: Ciphertext, r: int) -> Ciphertext:
        """Left slot rotation by r: phi_g on both components, then key switch phi_g(c1) (g = 5^r)."""
        prm = self.prm
        g = prm.galois(r)
        if g == 1:
            return a.copy()
        if g not in self.rot:
            raise KeyError(f"missing rotation key for step {r}")
        pr = prm.q[: a.level + 1]
        c0 = np.stack([ring.automorphism(a.c[0][i], g, q) for i, q in enumerate(pr)])
        c1 = np.stack([ring.automorphism(a.c[1][i], g, q) for i, q in enumerate(pr)])
        k0, k1 = self.keyswitch(c1, a.level, self.rot[g])
        return Ciphertext(np.stack([self._add(c0, k0, pr), k1]), a.level)

    def rotate_sum_hoisted(self, a: Ciphertext, steps: Sequence[int]) -> Ciphertext:
        """sum over r in steps of rot(a, r), with the key switches hoisted (Halevi-Shoup 2018).

        ModUp of c1 is computed once; rotation r applies phi_g (g = 5^r) to the raised digits
        instead of raising phi_g(c1); the inner products with every rotation key are summed in
        Q_l u P and one ModDown ends the sum:
          out0 = sum_r phi_g(c0) + ModDown(sum_r sum_j phi_g(ModUp_j(c1)) * b_{r,j}),
          out1 = [0 in steps] c1 + ModDown(sum_r sum_j phi_g(ModUp_j(c1)) * a_{r,j}),
        where a step with g = 1 contributes (c0, c1) itself and no key switch. phi_g of a raised
        digit differs from the digit of phi_g(c1) by multiples of the digit modulus (the fast
        conversion is not odd), which the key switch tolerates like the conversion's own
        overflow; the result is therefore not bit-identical to summing rotate()."""
        prm = self.prm
        lv = a.level
        pr = prm.q[: lv + 1]
        basis = pr + prm.p
        rows = self._key_rows(lv)
        dn = prm.dnum(lv)
        c0 = np.zeros((lv + 1, prm.n), dtype=np.uint64)
        c1 = np.zeros_like(c0)
        ups = None
        terms, kb, ka = [], [], []
        for r in steps:
            g = prm.galois(r)
            if g == 1:
                c0 = self._add(c0, a.c[0][: lv + 1], pr)
                c1 = self._add(c1, a.c[1][: lv + 1], pr)
                continue
            if g not in self.rot:
                raise KeyError(f"missing rotation key for step {r}")
            if ups is None:
                ups = self._modup(a.c[1][: lv + 1], lv)
            c0 = self._add(c0, np.stack([ring.automorphism(a.c[0][i], g, q) for i, q in enumerate(pr)]), pr)
            key = self.rot[g]
            for j in range(dn):
                terms.append(np.stack([ring.automorphism(ups[j][x], g, q) for x, q in enumerate(basis)]))
                kb.append(key.b[j][rows])
                ka.append(key.a[j][rows])
        if terms:
            T = np.ascontiguousarray(np.stack(terms).transpose(1, 0, 2))  # [|basis|, terms, N]
            for h, K in enumerate((kb, ka)):
                acc = ring.polydot_rows(T, np.ascontiguousarray(np.stack(K).transpose(1, 0, 2)), basis)
                part = self._moddown(acc, lv)
                if h == 0:
                    c0 = self._add(c0, part, pr)
                else:
                    c1 = self._add(c1, part, pr)
        return Ciphertext(np.stack([c0, c1]), lv)

    def rotate_fanin(self, cts: Sequence[Ciphertext], steps: Sequence[int]) -> Ciphertext:
        """sum_i rot(cts[i], steps[i]) with one ModDown for the whole sum.

        Every input keeps its own ModUp: phi_g of its c1 is raised (ModUp) and multiplied with the
        rotation key of its step; the inner products of all inputs are summed in Q_l u P and a
        single ModDown ends the sum, which the phi_g of every c0 joins:
          out0 = sum_i phi_gi(c0_i) + ModDown(sum_i sum_j ModUp_j(phi_gi(c1_i)) * b_{gi,j}),
          out1 = ModDown(sum_i sum_j ModUp_j(phi_gi(c1_i)) * a_{gi,j}).
        ModDown is linear up to its conversion error, so this equals the sum of rotate() results
        within the key-switch noise but is not bit-identical to it. All inputs share one level."""
        prm = self.prm
        lv = cts[0].level
        if any(ct.level != lv for ct in cts) or len(cts) != len(steps):
            raise ValueError("fan-in rotation: inputs at one level, one step each")
        pr = prm.q[: lv + 1]
        basis = pr + prm.p
        rows = self._key_rows(lv)
        dn = prm.dnum(lv)
        c0 = np.zeros((lv + 1, prm.n), dtype=np.uint64)
        terms, kb, ka = [], [], []
        for ct, r in zip(cts, steps):
            g = prm.galois(r)
            if g == 1:
                raise ValueError("fan-in rotation: a step that is a multiple of the slot count")
            if g not in self.rot:
                raise KeyError(f"missing rotation key for step {r}")
            c0 = self._add(c0, np.stack([ring.automorphism(ct.c[0][i], g, q) for i, q in enumerate(pr)]), pr)
            c1g = np.stack([ring.automorphism(ct.c[1][i], g, q) for i, q in enumerate(pr)])
            ups = self._modup(c1g, lv)
            key = self.rot[g]
            for j in range(dn):
                terms.append(ups[j])
                kb.append(key.b[j][rows])
                ka.append(key.a[j][rows])
        T = np.ascontiguousarray(np.stack(terms).transpose(1, 0, 2))  # [|basis|, terms, N]
        halves = []
        for K in (kb, ka):
            acc = ring.polydot_rows(T, np.ascontiguousarray(np.stack(K).transpose(1, 0, 2)), basis)
            halves.append(self._moddown(acc, lv))
        return Ciphertext(np.stack([self._add(c0, halves[0], pr), halves[1]]), lv)

    def mul_relin_rescale(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        """Ciphertext product (Eq. 8) followed by the fused relinearise-rescale."""
        return self.relin_rescale(self.tensor(a, b))

    def zero(self, level: int, parts: int = 2) -> Ciphertext:
        return Ciphertext(np.zeros((parts, level + 1, self.prm.n), dtype=np.uint64), level)
