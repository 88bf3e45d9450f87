"""Oracle for encrypted CSR matrix factorisation — TEST INFRASTRUCTURE ONLY.

Three independent pieces (only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this module):

1. ``mf_epoch_fp64``: plaintext MF in float64. The epoch follows Alg. 2 with
   the accumulators applied once per epoch: every error e_ij = r_ij - <u_i, v_j>
   uses the epoch-start factors, the per-rating gradients of Alg. 1 (grad_u =
   e v - lambda u, grad_v = e u - lambda v, lambda applied per rating) are
   summed, and
       u_i <- u_i (1 - a lambda nnz_i) + a sum_j e_ij v_j,
       v_j <- v_j (1 - a lambda nnz_j) + a sum_i e_ij u_i.
   RMSE is Eq. 10.

2. ``build_plan``: the batch-pair grouping of Sec. III-D (Fig. 5, Alg. 2) made
   SIMD. Users and items are cut into batches of B = N/2 / w entities; entity a
   of a batch owns the slot block [a w, a w + w) with w = 2 kp, kp =
   next_pow2(k), and holds its k-vector twice: x_0..x_{k-1}, 0.., x_0..x_{k-1}, 0...
   A rating (i, j) with a = i mod B, b = i div B, d = j mod B, c = j div B lies in
   group (b, c, delta = (d - a) mod B); one rotation of item batch c by delta*w
   lines up every (a, a + delta) pair of the group at once.

3. ``EncryptedMF.epoch``: the encrypted epoch on the oracle CKKS, operation by
   operation (Alg. 1 error and gradient lines, Alg. 2 accumulators).
   ``simulate_epoch_slots`` runs the same slot arithmetic in float64 (no
   encryption) and pins the plan against (1).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .ckks import Ciphertext, Ckks


# ----------------------------------------------------------------------------- (1) FP64 reference

def mf_epoch_fp64(U: np.ndarray, V: np.ndarray, rows, cols, vals, lr: float, lam: float):
    """One accumulated (Jacobi) epoch of Alg. 2 with per-rating lambda, in float64."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    e = vals - np.einsum("tk,tk->t", U[rows], V[cols])
    gU = np.zeros_like(U)
    gV = np.zeros_like(V)
    np.add.at(gU, rows, e[:, None] * V[cols])
    np.add.at(gV, cols, e[:, None] * U[rows])
    nnz_u = np.bincount(rows, minlength=U.shape[0]).astype(np.float64)
    nnz_v = np.bincount(cols, minlength=V.shape[0]).astype(np.float64)
    U2 = U * (1.0 - lr * lam * nnz_u)[:, None] + lr * gU
    V2 = V * (1.0 - lr * lam * nnz_v)[:, None] + lr * gV
    return U2, V2


def rmse(U: np.ndarray, V: np.ndarray, rows, cols, vals) -> float:
    """Eq. 10: sqrt(mean over the given ratings of (<u_i, v_j> - r_ij)^2)."""
    pred = np.einsum("tk,tk->t", U[np.asarray(rows)], V[np.asarray(cols)])
    return float(np.sqrt(np.mean((pred - np.asarray(vals)) ** 2)))


# ----------------------------------------------------------------------------- (2) plan

def next_pow2(x: int) -> int:
    p = 1
    while p < x:
        p <<= 1
    return p


def highest_bit(x: int) -> int:
    return x.bit_length() - 1


@dataclasses.dataclass
class Group:
    b: int
    c: int
    delta: int
    a: np.ndarray        # int64 [cnt] user slot blocks (ascending)
    r: np.ndarray        # float64 [cnt] ratings


@dataclasses.dataclass
class Plan:
    n: int
    m: int
    k: int
    kp: int
    w: int
    B: int
    n_ub: int
    n_vb: int
    groups: List[Group]
    closure: List[List[int]]   # per item batch c: sorted delta tree nodes (0 included)
    nnz_u: np.ndarray
    nnz_v: np.ndarray
    bin_of: List[int]          # rating bin of each group
    bin_batch: List[int]       # user batch of each bin

    @property
    def baby(self) -> int:
        return baby_range(self.B)

    def rotation_steps(self) -> List[int]:
        """Every left-rotation amount an epoch uses (negative = right): the in-block sum, the
        delta tree's baby steps r w (r < beta) and giant steps 2^t beta w in both directions, the
        half-fill."""
        tree = tree_steps(self.B)
        steps = rotsum_steps(self.kp)
        steps += [x * self.w for x in tree]
        steps += [-x * self.w for x in tree]
        steps += [-self.kp]
        return steps


# The in-block rotate-and-sum over kp slots is hoisted (one ModUp, kp - 1 key inner products,
# one ModDown) for 2 <= kp <= HOIST_MAX_KP; wider blocks use log2(kp) rotate-and-adds.
HOIST_MAX_KP = 16


def rotsum_steps(kp: int) -> List[int]:
    """Rotation amounts of the rotate-and-sum over kp slots."""
    if 2 <= kp <= HOIST_MAX_KP:
        return list(range(1, kp))
    return [1 << t for t in range(highest_bit(kp))]


def block_sum(he: Ckks, P: Ciphertext, kp: int) -> Ciphertext:
    """S = sum_{j < kp} rot(P, j): every slot x < kp of a doubled block gets the block's sum."""
    if 2 <= kp <= HOIST_MAX_KP:
        return he.rotate_sum_hoisted(P, range(kp))
    S = P
    for t in range(highest_bit(kp)):
        S = he.add(S, he.rotate(S, 1 << t))
    return S


# The delta tree (the Vr chain of Alg. 2's rotated item batches): every needed delta d is reached
# from 0 by rotations of the item batch by multiples of w. Baby-step giant-step form with beta =
# baby_range(B): write d = g beta + r (r < beta). A baby (r > 0) hangs off its giant g beta and is
# one rotation by r w away; a giant g beta (g > 0) hangs off (g - 2^hb(g)) beta, one rotation by
# 2^hb(g) beta w away. Rotations of one parent share its ModUp (hoisted fan-out), so the ModUps
# per item batch fall from about B/2 (a binary tree over d) to about 3 B / (2 beta).

def baby_range(B: int) -> int:
    """beta = 2^floor(log2(B) / 2): the baby steps of the delta tree."""
    return 1 << (highest_bit(B) // 2)


def tree_parent(d: int, beta: int) -> Tuple[int, int]:
    """(parent, rotation in blocks) of delta d > 0 in the baby-step giant-step delta tree."""
    g, r = divmod(int(d), beta)
    if r:
        return g * beta, r
    step = 1 << highest_bit(g)
    return (g - step) * beta, step * beta


def tree_depth(d: int, beta: int) -> int:
    """Rotations from 0 to d: popcount of the giant index, plus one for a baby."""
    g, r = divmod(int(d), beta)
    return bin(g).count("1") + (1 if r else 0)


def tree_steps(B: int) -> List[int]:
    """Rotation amounts (in blocks) of the delta tree: baby steps 1..beta-1, giant steps 2^t beta < B."""
    beta = baby_range(B)
    steps = list(range(1, min(beta, B)))
    t = beta
    while t < B:
        steps.append(t)
        t <<= 1
    return steps


def delta_closure(deltas, beta: int) -> List[int]:
    """The deltas plus all their ancestors in the delta tree, plus 0."""
    nodes = {0}
    for d in deltas:
        d = int(d)
        while d and d not in nodes:
            nodes.add(d)
            d = tree_parent(d, beta)[0]
    return sorted(nodes)


def assign_bins(groups: Sequence[Group], n_ub: int) -> Tuple[List[int], List[int]]:
    """Rating bins: the ciphertexts that store the ratings (the paper packs L ratings per
    ciphertext, Sec. III-C). Within each user batch, groups in plan order go to the first bin
    (in creation order) that holds none of their users; if every bin does, a new bin opens. A
    bin therefore holds at most one rating per user block, and a group's ratings all lie in
    one bin. Bins are numbered batch by batch. Returns (bin of each group, batch of each bin)."""
    bin_of = [0] * len(groups)
    bin_batch: List[int] = []
    for b in range(n_ub):
        first = len(bin_batch)
        users_in: List[set] = []
        for t, g in enumerate(groups):
            if g.b != b:
                continue
            users = set(int(a) for a in g.a)
            for i, taken in enumerate(users_in):
                if not (taken & users):
                    taken |= users
                    bin_of[t] = first + i
                    break
            else:
                users_in.append(users)
                bin_batch.append(b)
                bin_of[t] = first + len(users_in) - 1
    return bin_of, bin_batch


def batch_pairs(rows, cols, B: int) -> Dict[Tuple[int, int], List[Tuple[int, int]]]:
    """Alg. 2 / Fig. 5 grouping: ratings keyed by (user batch i div B, item batch j div B)."""
    out: Dict[Tuple[int, int], List[Tuple[int, int]]] = {}
    for i, j in zip(np.asarray(rows).tolist(), np.asarray(cols).tolist()):
        out.setdefault((i // B, j // B), []).append((i, j))
    return out


def build_plan(n: int, m: int, k: int, rows, cols, vals, slots: int) -> Plan:
    kp = next_pow2(k)
    w = 2 * kp
    B = slots // w
    if B < 1:
        raise ValueError("rank too large for the ring")
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    n_ub = -(-n // B)
    n_vb = -(-m // B)
    groups: Dict[Tuple[int, int, int], List[Tuple[int, float]]] = {}
    for i, j, r in zip(rows.tolist(), cols.tolist(), vals.tolist()):
        a, b = i % B, i // B
        d, c = j % B, j // B
        delta = (d - a) % B
        groups.setdefault((b, c, delta), []).append((a, r))
    glist = []
    for key in sorted(groups):
        items = sorted(groups[key])
        glist.append(Group(key[0], key[1], key[2], np.array([x[0] for x in items], dtype=np.int64),
                           np.array([x[1] for x in items], dtype=np.float64)))
    closure = []
    for c in range(n_vb):
        closure.append(delta_closure([g.delta for g in glist if g.c == c], baby_range(B)))
    nnz_u = np.bincount(rows, minlength=n).astype(np.int64)
    nnz_v = np.bincount(cols, minlength=m).astype(np.int64)
    bin_of, bin_batch = assign_bins(glist, n_ub)
    return Plan(n, m, k, kp, w, B, n_ub, n_vb, glist, closure, nnz_u, nnz_v, bin_of, bin_batch)


def pack_factors(X: np.ndarray, plan: Plan, batch: int) -> np.ndarray:
    """Slot vector of one batch: entity a's k-vector at [a w, a w + k) and [a w + kp, a w + kp + k)."""
    z = np.zeros(plan.B * plan.w, dtype=np.float64)
    for a in range(plan.B):
        e = batch * plan.B + a
        if e >= X.shape[0]:
            break
        z[a * plan.w: a * plan.w + plan.k] = X[e]
        z[a * plan.w + plan.kp: a * plan.w + plan.kp + plan.k] = X[e]
    return z


def unpack_factors(z: np.ndarray, plan: Plan, batch: int, count: int) -> np.ndarray:
    """Inverse of pack_factors (first copy), for the entities of one batch."""
    out = []
    for a in range(plan.B):
        e = batch * plan.B + a
        if e >= count:
            break
        out.append(z[a * plan.w: a * plan.w + plan.k])
    return np.array(out).reshape(-1, plan.k)


def rating_slots(g: Group, plan: Plan) -> np.ndarray:
    """R_g: rating r_(a, a+delta) in the first k slots of block a."""
    z = np.zeros(plan.B * plan.w)
    for a, r in zip(g.a.tolist(), g.r.tolist()):
        z[a * plan.w: a * plan.w + plan.k] = r
    return z


def bin_slots(t: int, plan: Plan) -> np.ndarray:
    """Slot vector of rating bin t: every group of the bin in its own user blocks."""
    z = np.zeros(plan.B * plan.w)
    for g, bt in zip(plan.groups, plan.bin_of):
        if bt == t:
            z += rating_slots(g, plan)
    return z


def mask_slots(g: Group, plan: Plan, lr: float) -> np.ndarray:
    """mask_g: the learning rate in the first k slots of each rated block, 0 elsewhere."""
    z = np.zeros(plan.B * plan.w)
    for a in g.a.tolist():
        z[a * plan.w: a * plan.w + plan.k] = lr
    return z


def reg_slots(nnz: np.ndarray, plan: Plan, batch: int, lr: float, lam: float) -> np.ndarray:
    """Regulariser of one batch: 1 - lr*lambda*nnz_e on every slot of entity e's block."""
    z = np.zeros(plan.B * plan.w)
    for a in range(plan.B):
        e = batch * plan.B + a
        cnt = int(nnz[e]) if e < nnz.size else 0
        z[a * plan.w: (a + 1) * plan.w] = 1.0 - lr * lam * cnt
    return z


# ----------------------------------------------------------------------------- slot-level simulation

def _rot(z: np.ndarray, r: int) -> np.ndarray:
    return np.roll(z, -r)


def simulate_epoch_slots(U: np.ndarray, V: np.ndarray, plan: Plan, lr: float, lam: float):
    """The encrypted epoch's slot arithmetic in float64 (no encryption), returning new U, V."""
    UD = [pack_factors(U, plan, b) for b in range(plan.n_ub)]
    VD = [pack_factors(V, plan, c) for c in range(plan.n_vb)]
    Vr = []
    beta = plan.baby
    for c in range(plan.n_vb):
        t = {0: VD[c]}
        for d in sorted(plan.closure[c], key=lambda x: (tree_depth(x, beta), x)):
            if d:
                par, step = tree_parent(d, beta)
                t[d] = _rot(t[par], step * plan.w)
        Vr.append(t)
    TU = [np.zeros_like(UD[0]) for _ in range(plan.n_ub)]
    TV: Dict[Tuple[int, int], np.ndarray] = {}
    for g in plan.groups:
        vr = Vr[g.c][g.delta]
        S = UD[g.b] * vr
        for t in range(highest_bit(plan.kp)):
            S = S + _rot(S, 1 << t)
        E = rating_slots(g, plan) - S
        msk = mask_slots(g, plan, lr)
        TU[g.b] = TU[g.b] + E * (vr * msk)
        key = (g.c, g.delta)
        TV[key] = TV.get(key, 0.0) + E * (UD[g.b] * msk)
    newU, newV = [], []
    for b in range(plan.n_ub):
        acc = TU[b] + _rot(TU[b], -plan.kp)
        z = UD[b] * reg_slots(plan.nnz_u, plan, b, lr, lam) + acc
        newU.append(unpack_factors(z, plan, b, plan.n))
    for c in range(plan.n_vb):
        H = {d: TV.get((c, d), np.zeros_like(VD[0])) for d in plan.closure[c]}
        for d in sorted(plan.closure[c], key=lambda x: (tree_depth(x, beta), x), reverse=True):
            if d:
                par, step = tree_parent(d, beta)
                H[par] = H[par] + _rot(H[d], -step * plan.w)
        acc = H[0] + _rot(H[0], -plan.kp)
        z = VD[c] * reg_slots(plan.nnz_v, plan, c, lr, lam) + acc
        newV.append(unpack_factors(z, plan, c, plan.m))
    return np.concatenate(newU)[: plan.n], np.concatenate(newV)[: plan.m]


# ----------------------------------------------------------------------------- (3) encrypted epoch

R_NONCE_BASE = 1 << 40
U_NONCE_BASE = 1 << 41
V_NONCE_BASE = (1 << 41) + (1 << 40)


class EncryptedMF:
    """Encrypted MF state on the oracle CKKS: U/V batch ciphertexts and the rating ciphertexts."""

    def __init__(self, he: Ckks, plan: Plan):
        self.he = he
        self.plan = plan
        self.R: List[Ciphertext] = []

    def encrypt_ratings(self) -> None:
        """The CSP's EncryptCsrMatrix step (Alg. 1): one ciphertext per rating bin, encrypted by the
        key holder with a regenerable c1 (object R_NONCE_BASE + bin) at level top - 1, the highest
        level at which an epoch reads it."""
        he = self.he
        lv = he.prm.top - 1
        self.R = [he.encrypt_seeded(he.enc.encode(bin_slots(t, self.plan)), lv, R_NONCE_BASE + t)
                  for t in range(len(self.plan.bin_batch))]

    def encrypt_factors(self, U: np.ndarray, V: np.ndarray):
        top = self.he.prm.top
        UD = [self.he.encrypt(pack_factors(U, self.plan, b), top, U_NONCE_BASE + b)
              for b in range(self.plan.n_ub)]
        VD = [self.he.encrypt(pack_factors(V, self.plan, c), top, V_NONCE_BASE + c)
              for c in range(self.plan.n_vb)]
        return UD, VD

    def decrypt_factors(self, UD: Sequence[Ciphertext], VD: Sequence[Ciphertext]):
        p = self.plan
        U = np.concatenate([unpack_factors(self.he.decrypt(ct, p.B * p.w), p, b, p.n)
                            for b, ct in enumerate(UD)])[: p.n]
        V = np.concatenate([unpack_factors(self.he.decrypt(ct, p.B * p.w), p, c, p.m)
                            for c, ct in enumerate(VD)])[: p.m]
        return U, V

    # the per-group part of the epoch: returns E (*) M and E (*) MU tensors
    def group_terms(self, t: int, UD_b: Ciphertext, vr: Ciphertext, lr: float):
        he, p = self.he, self.plan
        g = p.groups[t]
        S = block_sum(he, he.mul_relin_rescale(UD_b, vr), p.kp)
        E = he.sub(he.drop(self.R[p.bin_of[t]], S.level), S)   # exact on g's blocks; the mask kills the rest
        mask = he.enc.encode(mask_slots(g, p, lr))
        M = he.rescale(he.mul_plain(vr, mask))
        MU = he.rescale(he.mul_plain(UD_b, mask))
        return he.tensor(E, M), he.tensor(E, MU)

    def epoch(self, UD: List[Ciphertext], VD: List[Ciphertext], lr: float, lam: float):
        """One encrypted epoch at level l -> level l - 2 (Alg. 1 error/gradient, Alg. 2 accumulators)."""
        he, p = self.he, self.plan
        lv = UD[0].level
        if lv < 2:
            raise ValueError("level exhausted")
        # Vr chain: rotations of each item batch by delta*w along the delta tree
        Vr: List[Dict[int, Ciphertext]] = []
        beta = p.baby
        for c in range(p.n_vb):
            t = {0: VD[c]}
            for d in sorted(p.closure[c], key=lambda x: (tree_depth(x, beta), x)):
                if d:
                    par, step = tree_parent(d, beta)
                    # hoisted: the children of a node share the ModUp of its c1
                    t[d] = he.rotate_sum_hoisted(t[par], [step * p.w])
            Vr.append(t)
        TU: List[Optional[Ciphertext]] = [None] * p.n_ub
        TV: Dict[Tuple[int, int], Ciphertext] = {}
        for t, g in enumerate(p.groups):
            tu, tv = self.group_terms(t, UD[g.b], Vr[g.c][g.delta], lr)
            TU[g.b] = tu if TU[g.b] is None else he.add(TU[g.b], tu)
            key = (g.c, g.delta)
            TV[key] = tv if key not in TV else he.add(TV[key], tv)
        return self.finish_epoch(UD, VD, TU, TV, lr, lam, lv)

    def finish_epoch(self, UD, VD, TU, TV, lr, lam, lv):
        he, p = self.he, self.plan
        out_lv = lv - 2
        newU = []
        for b in range(p.n_ub):
            acc = he.zero(out_lv) if TU[b] is None else he.relin_rescale(TU[b])
            acc = he.add(acc, he.rotate(acc, -p.kp))
            reg = he.enc.encode(reg_slots(p.nnz_u, p, b, lr, lam))
            base = he.drop(he.rescale(he.mul_plain(UD[b], reg)), out_lv)
            newU.append(he.add(base, acc))
        newV = []
        for c in range(p.n_vb):
            H: Dict[int, Ciphertext] = {}
            for d in p.closure[c]:
                H[d] = he.relin_rescale(TV[(c, d)]) if (c, d) in TV else he.zero(out_lv)
            # back-rotation, deepest nodes first: every parent takes the sum of its children rotated
            # back with one ModDown (the children of a node all lie one level deeper)
            nodes = [d for d in p.closure[c] if d]
            for dep in sorted({tree_depth(d, p.baby) for d in nodes}, reverse=True):
                kids: Dict[int, List[int]] = {}
                for d in sorted(x for x in nodes if tree_depth(x, p.baby) == dep):
                    kids.setdefault(tree_parent(d, p.baby)[0], []).append(d)
                for par, ds in kids.items():
                    back = he.rotate_fanin([H[d] for d in ds], [-tree_parent(d, p.baby)[1] * p.w for d in ds])
                    H[par] = he.add(H[par], back)
            acc = H[0]
            acc = he.add(acc, he.rotate(acc, -p.kp))
            reg = he.enc.encode(reg_slots(p.nnz_v, p, c, lr, lam))
            base = he.drop(he.rescale(he.mul_plain(VD[c], reg)), out_lv)
            newV.append(he.add(base, acc))
        return newU, newV

    def predict(self, UD: Sequence[Ciphertext], VD: Sequence[Ciphertext], user: int) -> List[Ciphertext]:
        """Encrypted row `user` of R-hat = U V^T (Alg. 1): slot d*w of output c holds <u_user, v_(cB+d)>.

        The user's block is isolated by a 0/1 mask, copied into every block by
        log2(B) rotate-and-adds, multiplied with each item batch and summed over
        the kp slots of each block."""
        he, p = self.he, self.plan
        b, a = divmod(user, p.B)
        mask = np.zeros(p.B * p.w)
        mask[a * p.w: a * p.w + p.k] = 1.0
        X = he.rescale(he.mul_plain(UD[b], he.enc.encode(mask)))
        for t in range(highest_bit(p.B)):
            X = he.add(X, he.rotate(X, (1 << t) * p.w))
        out = []
        for c in range(p.n_vb):
            out.append(block_sum(he, he.mul_relin_rescale(X, VD[c]), p.kp))
        return out
