"""Shared helpers of the GPU parity tests: build the library, create matching
CUDA and oracle contexts, and move ciphertexts between them in coefficient form."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ckks  # noqa: E402
from paper_2509_03024_gb300 import build, capi  # noqa: E402
from paper_2509_03024_gb300.workloads import PRESETS  # noqa: E402


@functools.lru_cache(maxsize=None)
def built():
    return build.build()


def gpu_ctx(preset_name: str, seed: int, steps=()):
    built()
    pre = PRESETS[preset_name]
    ctx = capi.Context.from_preset(pre)
    ctx.keygen(seed, steps)
    return ctx


def oracle_ctx(preset_name: str, seed: int, steps=()):
    he = ckks.Ckks(ckks.Params.from_preset(PRESETS[preset_name]))
    he.keygen(seed, steps)
    return he


def to_coeff(ctx, ct, level: int, count: int = 1) -> np.ndarray:
    """GPU ciphertexts -> numpy uint64 [count, 2, level+1, N] coefficient form (library INTT)."""
    out = torch.zeros(count * 2 * (level + 1) * ctx.n, dtype=torch.int64, device="cuda")
    ctx.ct_to_coeff(ct, count, level, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(count, 2, level + 1, ctx.n)


def ct_slice(ctx, buf, t: int, parts: int = 2):
    w = parts * (ctx.top + 1) * ctx.n
    return buf[t * w:(t + 1) * w]


def tensor3_to_coeff(ctx, buf, level: int) -> np.ndarray:
    """One 3-component tensor buffer [3][L+1][N] -> [3, level+1, N] coefficient form."""
    tmp = buf.clone()
    ctx.ntt_inverse(tmp, 3, ctx.top + 1)
    torch.cuda.synchronize()
    return tmp.cpu().numpy().view(np.uint64).reshape(3, ctx.top + 1, ctx.n)[:, : level + 1]


def assert_ct_equal(gpu: np.ndarray, ora, what=""):
    """Bit-exact equality of a GPU coefficient-form ciphertext with an oracle Ciphertext."""
    o = ora.c if hasattr(ora, "c") else ora
    assert gpu.shape == o.shape, (what, gpu.shape, o.shape)
    bad = np.argwhere(gpu != o)
    assert bad.size == 0, f"{what}: {len(bad)} residues differ, first at {bad[:3].tolist()}"
