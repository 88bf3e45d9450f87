"""Communication between the parties of the encrypted MF protocol (Sec. III-B), in ciphertexts
and bytes.

The key holder (CSP) generates the keys and publishes the public and evaluation keys; the ratings
(encrypted by the key holder, c0 and a seed for c1) and the initial factors reach the recommender
(RS) encrypted; the RS runs the
epochs on its GPU; when the modulus chain runs out the RS sends U and V to the key holder, which
returns them re-encrypted at the top level (refresh); at the end the factors go to the key holder
for decryption. A served request uploads the user's encrypted vector and ratings and downloads the
encrypted predicted-rating row. Counts follow the library's layout (one ciphertext per user or
item batch, per rating bin, per item batch of a request); a ciphertext at level l is
2 (l + 1) N words of 8 bytes.
"""
from __future__ import annotations

from typing import Dict


def ct_bytes(n: int, level: int) -> int:
    return 2 * (level + 1) * n * 8


def key_bytes(n: int, top: int, alpha: int) -> Dict[str, int]:
    dnum = -(-(top + 1) // alpha)
    return {"public_key": 2 * (top + 1) * n * 8, "eval_key_each": dnum * 2 * (top + 1 + alpha) * n * 8}


def mf_training(n: int, top: int, alpha: int, n_rot_keys: int, n_bins: int, n_ub: int, n_vb: int,
                epochs: int, levels_per_epoch: int = 2) -> Dict[str, object]:
    """Ciphertexts and bytes of one training run of `epochs` epochs starting at the top level,
    refreshing U and V through the key holder whenever fewer than `levels_per_epoch` levels remain
    (the refreshed factors travel at the level they reached: out at that level, back at the top)."""
    keys = key_bytes(n, top, alpha)
    # rating bins: encrypted by the key holder with a regenerable c1, so c0 at level top - 1 plus a
    # 16-byte seed reference per bin travel
    setup = {"public_key": keys["public_key"], "eval_keys": keys["eval_key_each"] * (1 + n_rot_keys),
             "rating_cts": n_bins, "rating_bytes": n_bins * (top * n * 8 + 16),
             "factor_cts": n_ub + n_vb, "factor_bytes": (n_ub + n_vb) * ct_bytes(n, top)}
    level, refreshes, refresh_bytes = top, 0, 0
    for _ in range(epochs):
        if level < levels_per_epoch:
            refreshes += 1
            refresh_bytes += (n_ub + n_vb) * (ct_bytes(n, level) + ct_bytes(n, top))
            level = top
        level -= levels_per_epoch
    final = (n_ub + n_vb) * ct_bytes(n, level)
    total = (setup["public_key"] + setup["eval_keys"] + setup["rating_bytes"] + setup["factor_bytes"]
             + refresh_bytes + final)
    return {"setup": setup, "refreshes": refreshes, "refresh_bytes": refresh_bytes,
            "final_decrypt_bytes": final, "final_level": level, "total_bytes": total,
            "per_epoch_bytes_excluding_setup": (refresh_bytes + final) / max(epochs, 1)}


def served_request(n: int, top: int, n_vb: int, rated_batches: int, steps: int,
                   levels_per_step: int = 2) -> Dict[str, int]:
    """One request: up the replicated user vector and the rated batches' rating ciphertexts at the
    top level, down the predicted-rating row (n_vb ciphertexts) after `steps` fold-in steps and the
    one-level prediction pass."""
    out_level = top - levels_per_step * steps - 1
    up = (1 + rated_batches) * ct_bytes(n, top)
    down = n_vb * ct_bytes(n, out_level)
    return {"up_cts": 1 + rated_batches, "up_bytes": up, "down_cts": n_vb, "down_bytes": down,
            "out_level": out_level, "total_bytes": up + down}
