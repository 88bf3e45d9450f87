"""Oracle for a served request: encrypted fold-in of one user's factor against
resident encrypted item factors, then the encrypted predicted-rating row —
TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's
CPU-baseline leg may use it; the CUDA library does not).

Layout (one request): the user's k-vector u is written in EVERY slot block
(block a, slots a*w + x and a*w + kp + x, x < k); item j = c*B + d sits in
block d of item batch c (the item-batch packing of the MF plan). One fold-in
step at level l applies Alg. 1's error and gradient lines to all of the
user's ratings at once and the accumulated update of Alg. 2:

  for every item batch c holding a rated item:
      S_c = rotsum_kp(rescale(relin(UR (x) V_c)))        <u, v_(cB+d)> in block d
      E_c = R_c - S_c                                   e_j = r_j - <u, v_j>
      T  += E_c (x) rescale(V_c|l (.) mask_c)           mask_c = lr on the first k slots of rated blocks
  G = rescale(relin(T))                                 block d: lr e_j v_j
  G = sum_{a < B} rot(G, a w)                           every block: lr sum_j e_j v_j
  G = G + rot(G, -kp)                                   doubled block layout
  UR = drop(rescale(UR * round((1 - lr*lambda*nnz) * Delta))) + G

The block sum and the half-fill run as hoisted rounds (``block_sum_rounds``):
radix-4 rotate-and-sums with strides w, 4w, 16w, ..., the half-fill merged into
the last round.

two levels per step. The prediction pass computes S_c for every item batch
(one level). ``fold_in_fp64`` is the same update in float64.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from .ckks import Ciphertext, Ckks
from .mf import block_sum, highest_bit, next_pow2, rotsum_steps

REQ_NONCE_STRIDE = 64


def layout(k: int, slots: int):
    kp = next_pow2(k)
    w = 2 * kp
    return kp, w, slots // w


def block_sum_rounds(k: int, slots: int) -> List[List[int]]:
    """The gradient's block sum over the B slot blocks followed by the half-fill, as rounds of
    hoisted rotate-and-sums (each round: G <- sum over its steps r of rot(G, r), step 0 = G itself).

    Mathematically the block sum is G <- sum_{a < B} rot(G, a w) and the half-fill G <- G + rot(G, -kp);
    the rounds factor the block offsets a w as sums of one step per round: radix-4 rounds with strides
    w, 4 w, 16 w, ... (steps 0, s, 2 s, 3 s), then a radix-2 round when log2 B is odd, and the last round
    also carries the half-fill (its steps r and r - kp), since rot(sum_r rot(G', r), -kp) is
    sum_r rot(G', r - kp). Every round is one hoisted key switch (one ModUp, one inner product per
    non-zero step, one ModDown) instead of one full key switch per doubling."""
    kp, w, B = layout(k, slots)
    lb = highest_bit(B)
    rounds, stride, t = [], w, 0
    while t < lb:
        r = 4 if lb - t >= 2 else 2
        rounds.append([j * stride for j in range(r)])
        stride *= r
        t += 2 if r == 4 else 1
    last = rounds.pop() if rounds else [0]
    rounds.append(last + [x - kp for x in last])
    return rounds


def rotation_steps(k: int, slots: int) -> List[int]:
    """Every left-rotation amount a request uses: the in-block sum, then the non-zero steps of the
    block-sum rounds (block sum and half-fill) in round order."""
    kp, _, _ = layout(k, slots)
    steps = rotsum_steps(kp)
    for rnd in block_sum_rounds(k, slots):
        steps += [x for x in rnd if x != 0 and x not in steps]
    return steps


def replicate_user(u: np.ndarray, k: int, slots: int) -> np.ndarray:
    kp, w, B = layout(k, slots)
    z = np.zeros(B * w)
    for a in range(B):
        z[a * w: a * w + k] = u
        z[a * w + kp: a * w + kp + k] = u
    return z


def rating_batches(items, ratings, k: int, slots: int, n_vb: int) -> List[np.ndarray]:
    kp, w, B = layout(k, slots)
    out = [np.zeros(B * w) for _ in range(n_vb)]
    for j, r in zip(np.asarray(items).tolist(), np.asarray(ratings).tolist()):
        c, d = divmod(j, B)
        out[c][d * w: d * w + k] = r
    return out


def rated_batches(items, k: int, slots: int) -> List[int]:
    _, _, B = layout(k, slots)
    return sorted({int(j) // B for j in items})


def mask_batch(items, c: int, k: int, slots: int, lr: float) -> np.ndarray:
    kp, w, B = layout(k, slots)
    z = np.zeros(B * w)
    for j in np.asarray(items).tolist():
        cj, d = divmod(int(j), B)
        if cj == c:
            z[d * w: d * w + k] = lr
    return z


def const_mul(he: Ckks, ct: Ciphertext, value: float) -> Ciphertext:
    """ct times the integer round(value * Delta) (the constant polynomial encoding a constant vector)."""
    cint = int(np.rint(value * float(he.prm.delta)))
    out = np.empty_like(ct.c)
    for t in range(ct.c.shape[0]):
        for i in range(ct.level + 1):
            q = he.prm.q[i]
            from . import ring
            out[t][i] = ring.scalar_mul(ct.c[t][i], cint % q, q)
    return Ciphertext(out, ct.level)


def encrypt_request(he: Ckks, u0, items, ratings, k: int, n_vb: int, nonce_base: int):
    """Client side: UR (u in every block) and one rating ciphertext per item batch, top level."""
    top = he.prm.top
    UR = he.encrypt(replicate_user(u0, k, he.prm.slots), top, nonce_base)
    Rz = rating_batches(items, ratings, k, he.prm.slots, n_vb)
    R = [he.encrypt(Rz[c], top, nonce_base + 1 + c) for c in range(n_vb)]
    return UR, R


def inner_products(he: Ckks, UR: Ciphertext, V: Sequence[Ciphertext], batches, kp: int) -> List[Ciphertext]:
    out = []
    for c in batches:
        out.append(block_sum(he, he.mul_relin_rescale(UR, V[c]), kp))
    return out


def fold_in_step(he: Ckks, UR: Ciphertext, R: Sequence[Ciphertext], V: Sequence[Ciphertext], items,
                 k: int, lr: float, lam: float) -> Ciphertext:
    slots = he.prm.slots
    kp, w, B = layout(k, slots)
    batches = rated_batches(items, k, slots)
    S = inner_products(he, UR, V, batches, kp)
    T = None
    for c, Sc in zip(batches, S):
        E = he.sub(he.drop(R[c], Sc.level), Sc)
        Vc = he.drop(V[c], UR.level)   # the resident top-level factors, read at the request's level
        MV = he.rescale(he.mul_plain(Vc, he.enc.encode(mask_batch(items, c, k, slots, lr))))
        t3 = he.tensor(E, MV)
        T = t3 if T is None else he.add(T, t3)
    out_lv = UR.level - 2
    G = he.zero(out_lv) if T is None else he.relin_rescale(T)
    for steps in block_sum_rounds(k, slots):     # block sum over the B blocks, then the half-fill
        G = he.rotate_sum_hoisted(G, steps)
    base = he.drop(he.rescale(const_mul(he, UR, 1.0 - lr * lam * len(items))), out_lv)
    return he.add(base, G)


def serve_request(he: Ckks, UR: Ciphertext, R, V, items, k: int, steps: int, lr: float, lam: float):
    for _ in range(steps):
        UR = fold_in_step(he, UR, R, V, items, k, lr, lam)
    kp, _, _ = layout(k, he.prm.slots)
    return UR, inner_products(he, UR, V, list(range(len(V))), kp)


def fold_in_fp64(u0, V: np.ndarray, items, ratings, steps: int, lr: float, lam: float) -> Tuple[np.ndarray, np.ndarray]:
    """Float64 reference: u <- u (1 - lr lam nnz) + lr sum_j (r_j - <u, v_j>) v_j; returns (u, V u)."""
    u = np.asarray(u0, dtype=np.float64).copy()
    items = np.asarray(items)
    ratings = np.asarray(ratings, dtype=np.float64)
    for _ in range(steps):
        e = ratings - V[items] @ u
        u = u * (1.0 - lr * lam * items.size) + lr * (e @ V[items])
    return u, V @ u
