"""Thin ctypes binding over the C ABI in include/ckks_mf.h (argument marshalling only).

Device buffers are torch tensors on the context's CUDA device (int64 storage
viewed as uint64 words); host buffers are numpy arrays. Streams are
``torch.cuda.Stream`` objects (or None for the legacy default stream). Every
computation runs in the CUDA library; if the library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libckks_mf.so")

FHE_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "LEVEL_EXHAUSTED", -3: "SCALE_MISMATCH", -4: "MISSING_KEY",
    -5: "OOM", -6: "DEVICE_TIMEOUT", -7: "CUDA", -8: "STATE",
}

# every entry point declared in include/ckks_mf.h
EXPORTS = [
    "fhe_ctx_create", "fhe_ctx_destroy", "fhe_last_error", "fhe_ctx_get_info", "fhe_ctx_get_primes",
    "fhe_keygen_from_seed", "fhe_add_rotation_keys", "fhe_encode", "fhe_encrypt", "fhe_encrypt_coeffs",
    "fhe_decrypt", "fhe_refresh", "fhe_ntt_forward", "fhe_ntt_inverse", "fhe_ct_to_coeff", "fhe_add", "fhe_sub",
    "fhe_mul_plain", "fhe_mul_relin_rescale", "fhe_tensor", "fhe_relinearize", "fhe_rescale", "fhe_rescale_noalloc",
    "fhe_rotate", "fhe_rotate_sum", "fhe_rotate_fanin", "fhe_probe_butterfly_rate", "fhe_probe_int_pipe", "fhe_probe_conv_cost", "fhe_autotune", "fhe_set_variant", "fhe_get_variant", "fhe_profile_begin", "fhe_profile_end", "fhe_mf_rotation_steps", "fhe_csr_pack", "fhe_mf_layout", "fhe_mf_plan_destroy",
    "fhe_mf_plan_get_info", "fhe_mf_plan_get_groups", "fhe_mf_plan_get_bins", "fhe_mf_plan_set_chunk", "fhe_mf_plan_set_wave_budget", "fhe_mf_encrypt_factors",
    "fhe_mf_decrypt_factors", "fhe_mf_sgd_epoch", "fhe_predict", "fhe_serve_rotation_steps",
    "fhe_serve_create", "fhe_serve_destroy", "fhe_serve_slots", "fhe_serve_submit", "fhe_serve_tick",
    "fhe_serve_poll", "fhe_serve_encrypt_request", "fhe_serve_take",
]


class FheError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int32), ("n_data_primes", ctypes.c_int32),
                ("data_prime_bits", ctypes.POINTER(ctypes.c_int32)), ("n_special_primes", ctypes.c_int32),
                ("special_prime_bits", ctypes.POINTER(ctypes.c_int32)), ("log_scale", ctypes.c_int32),
                ("sigma", ctypes.c_double), ("device", ctypes.c_int32)]


class CtxInfo(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int32), ("n", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("top_level", ctypes.c_int32), ("n_special", ctypes.c_int32), ("log_scale", ctypes.c_int32),
                ("ct_words", ctypes.c_size_t)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("device_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("work", ctypes.c_double)]


class IntPipeRates(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int32), ("imad_lo_gops", ctypes.c_double), ("imad_hi_gops", ctypes.c_double),
                ("imad_wide_gops", ctypes.c_double), ("mac_c_gmacs", ctypes.c_double),
                ("mac_ptx64_gmacs", ctypes.c_double), ("mac_ptx32_gmacs", ctypes.c_double),
                ("mac_wide_gmacs", ctypes.c_double)]


def tune_cache_key(device_name: str, n: int, primes: Sequence[int], level: int) -> str:
    """Key of a stored autotuner choice: the GPU model, and the ring and level it was timed on."""
    return f"{device_name}|N={n}|q={','.join(str(int(p)) for p in primes)}|level={level}"


def load_tune_cache(path: str) -> dict:
    """The stored choices ({key: {family: variant}}); empty when the file is absent."""
    import json
    try:
        with open(path) as f:
            data = json.load(f)
    except FileNotFoundError:
        return {}
    if not isinstance(data, dict):
        raise ValueError(f"{path}: not an autotuner cache")
    return data


def store_tune_cache(path: str, key: str, choices: dict) -> None:
    """Adds or replaces one key's choices; the file is replaced atomically."""
    import json
    data = load_tune_cache(path)
    data[key] = dict(choices)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class ConvCost(ctypes.Structure):
    _fields_ = [("conv_ms", ctypes.c_double), ("plain_ms", ctypes.c_double), ("rows", ctypes.c_int32),
                ("roundtrip_bytes", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("family", ctypes.c_char_p), ("variant", ctypes.c_char_p), ("chosen", ctypes.c_int32),
                ("ms", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_users", ctypes.c_int32), ("n_items", ctypes.c_int32), ("k", ctypes.c_int32),
                ("kp", ctypes.c_int32), ("w", ctypes.c_int32), ("B", ctypes.c_int32),
                ("n_user_batches", ctypes.c_int32), ("n_item_batches", ctypes.c_int32),
                ("n_ratings", ctypes.c_int64), ("n_groups", ctypes.c_int64),
                ("n_tree_nodes", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2509_03024_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, i32, i64, sz, dbl = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_size_t, ctypes.c_double)
        sig = {
            "fhe_ctx_create": [ctypes.POINTER(Params), ctypes.POINTER(vp)],
            "fhe_ctx_destroy": [vp],
            "fhe_last_error": [vp],
            "fhe_ctx_get_info": [vp, ctypes.POINTER(CtxInfo)],
            "fhe_ctx_get_primes": [vp, vp, sz],
            "fhe_keygen_from_seed": [vp, u64, vp, sz],
            "fhe_add_rotation_keys": [vp, vp, sz],
            "fhe_encode": [vp, vp, sz, vp, vp],
            "fhe_encrypt": [vp, vp, sz, i32, u64, vp, vp],
            "fhe_encrypt_coeffs": [vp, vp, i32, u64, vp, vp],
            "fhe_decrypt": [vp, vp, i32, vp, sz, vp],
            "fhe_refresh": [vp, vp, i32, i32, u64, vp, vp],
            "fhe_ntt_forward": [vp, vp, i32, i32, vp],
            "fhe_ntt_inverse": [vp, vp, i32, i32, vp],
            "fhe_ct_to_coeff": [vp, vp, i32, i32, vp, vp],
            "fhe_add": [vp, vp, vp, vp, i32, i32, vp],
            "fhe_sub": [vp, vp, vp, vp, i32, i32, vp],
            "fhe_mul_plain": [vp, vp, vp, vp, i32, i32, vp],
            "fhe_mul_relin_rescale": [vp, vp, vp, vp, i32, i32, vp],
            "fhe_tensor": [vp, vp, vp, vp, i32, i32, vp],
            "fhe_relinearize": [vp, vp, vp, i32, i32, vp],
            "fhe_rescale": [vp, vp, vp, i32, i32, vp],
            "fhe_rescale_noalloc": [vp, vp, vp, i32, vp],
            "fhe_rotate": [vp, vp, vp, i32, i32, i32, vp],
            "fhe_rotate_sum": [vp, vp, vp, i32, i32, i32, vp],
            "fhe_rotate_fanin": [vp, vp, i32, vp, vp, vp, i32, vp],
            "fhe_probe_butterfly_rate": [vp, i32, vp],
            "fhe_probe_int_pipe": [vp, i32, ctypes.POINTER(IntPipeRates)],
            "fhe_probe_conv_cost": [vp, i32, i32, ctypes.POINTER(ConvCost)],
            "fhe_autotune": [vp, i32, ctypes.POINTER(TuneResult), i32],
            "fhe_set_variant": [vp, ctypes.c_char_p, ctypes.c_char_p],
            "fhe_get_variant": [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_char_p)],
            "fhe_profile_begin": [vp, i32],
            "fhe_profile_end": [vp, vp, i32],
            "fhe_mf_rotation_steps": [vp, i32, vp, sz],
            "fhe_csr_pack": [vp, i32, i32, i32, vp, vp, vp, ctypes.POINTER(vp)],
            "fhe_mf_layout": [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, i64],
            "fhe_mf_plan_destroy": [vp],
            "fhe_mf_plan_get_info": [vp, ctypes.POINTER(PlanInfo)],
            "fhe_mf_plan_get_groups": [vp, vp, vp, vp, vp],
            "fhe_mf_plan_get_bins": [vp, vp],
            "fhe_mf_plan_set_wave_budget": [vp, ctypes.c_uint64],
            "fhe_mf_plan_set_chunk": [vp, i32],
            "fhe_mf_encrypt_factors": [vp, vp, i32, vp, i32, vp, vp],
            "fhe_mf_decrypt_factors": [vp, vp, i32, vp, i32, vp, i32, vp],
            "fhe_mf_sgd_epoch": [vp, vp, vp, vp, i32, dbl, dbl, vp],
            "fhe_predict": [vp, vp, vp, vp, i32, i32, vp, vp],
            "fhe_serve_rotation_steps": [vp, i32, vp, sz],
            "fhe_serve_create": [vp, vp, i32, i32, i32, dbl, dbl, i32, sz, ctypes.POINTER(vp)],
            "fhe_serve_destroy": [vp],
            "fhe_serve_slots": [vp, vp, vp],
            "fhe_serve_submit": [vp, i64, vp, i32, vp, vp, vp],
            "fhe_serve_tick": [vp, vp],
            "fhe_serve_poll": [vp, vp, i32],
            "fhe_serve_encrypt_request": [vp, i32, i32, vp, vp, vp, i32, u64, vp, vp, vp],
            "fhe_serve_take": [vp, i64, vp, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fhe_ctx_destroy.restype = None
        L.fhe_mf_plan_destroy.restype = None
        L.fhe_serve_destroy.restype = None
        L.fhe_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(x) -> Optional[int]:
    """Device (torch) or host (numpy) buffer -> address."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return x.data_ptr()
    return int(x)


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def mf_layout(slots: int, n: int, m: int, k: int, row_ptr, col_idx, vals):
    """The plan layout fhe_csr_pack computes for a ring of `slots` slots, on the host alone (no
    context, no GPU): {"groups": int32 [G, 4] (b, c, delta, ratings), "bins": int32 [G],
    "nodes": int32 [nodes, 2] (item batch, delta), "n_bins": int}."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    counts = np.zeros(3, dtype=np.int64)
    L = lib()

    def call(arrays, gcap, ncap):
        rc = L.fhe_mf_layout(slots, n, m, k, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, counts.ctypes.data,
                             *[None if a is None else a.ctypes.data for a in arrays[:5]], gcap,
                             *[None if a is None else a.ctypes.data for a in arrays[5:]], ncap)
        if rc != FHE_OK:
            raise FheError(rc, "fhe_mf_layout rejected its input")
    call([None] * 7, 0, 0)
    G, NB, ND = (int(x) for x in counts)
    g = [np.zeros(G, dtype=np.int32) for _ in range(5)]
    nd = [np.zeros(ND, dtype=np.int32) for _ in range(2)]
    call(g + nd, G, ND)
    return {"groups": np.stack(g[:4], axis=1), "bins": g[4], "nodes": np.stack(nd, axis=1), "n_bins": NB}


class Context:
    """Owns one fhe_ctx (primes, tables, keys and scratch on one CUDA device)."""

    def __init__(self, log_n: int, data_bits: Sequence[int], special_bits: Sequence[int], log_scale: int,
                 sigma: float = 3.2, device: int = 0):
        L = lib()
        self._db = (ctypes.c_int32 * len(data_bits))(*data_bits)
        self._sb = (ctypes.c_int32 * len(special_bits))(*special_bits)
        p = Params(log_n, len(data_bits), self._db, len(special_bits), self._sb, log_scale, sigma, device)
        h = ctypes.c_void_p()
        rc = L.fhe_ctx_create(ctypes.byref(p), ctypes.byref(h))
        if rc != FHE_OK:
            raise FheError(rc, "fhe_ctx_create failed")
        self.h = h
        self.device = device
        info = CtxInfo()
        self._check(L.fhe_ctx_get_info(self.h, ctypes.byref(info)))
        self.log_n, self.n, self.slots = info.log_n, info.n, info.slots
        self.top, self.alpha, self.log_scale = info.top_level, info.n_special, info.log_scale
        self.ct_words = info.ct_words
        pr = np.zeros(self.top + 1 + self.alpha, dtype=np.uint64)
        self._check(L.fhe_ctx_get_primes(self.h, pr.ctypes.data, pr.size))
        self.primes = [int(x) for x in pr]

    @classmethod
    def from_preset(cls, preset, device: int = 0) -> "Context":
        return cls(preset.log_n, preset.data_bits, preset.special_bits, preset.log_scale, preset.sigma, device)

    def close(self):
        if getattr(self, "h", None):
            lib().fhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return (lib().fhe_last_error(self.h) or b"").decode()

    def _check(self, rc: int):
        if rc != FHE_OK:
            raise FheError(rc, self.last_error())

    # ---- buffers
    def empty_ct(self, count: int = 1, parts: int = 2):
        import torch
        return torch.zeros(count * parts * (self.top + 1) * self.n, dtype=torch.int64,
                           device=f"cuda:{self.device}")

    # ---- keys, encode, encrypt
    def keygen(self, seed: int, rot_steps: Sequence[int] = ()):
        arr = np.array(list(rot_steps), dtype=np.int32)
        self._check(lib().fhe_keygen_from_seed(self.h, seed, arr.ctypes.data if arr.size else None, arr.size))

    def add_rotation_keys(self, rot_steps: Sequence[int]):
        arr = np.array(list(rot_steps), dtype=np.int32)
        self._check(lib().fhe_add_rotation_keys(self.h, arr.ctypes.data if arr.size else None, arr.size))

    def encode(self, slots, out, stream=None):
        z = np.ascontiguousarray(slots, dtype=np.float64)
        self._check(lib().fhe_encode(self.h, z.ctypes.data if z.size else None, z.size, _ptr(out), _stream(stream)))

    def encrypt(self, slots, level: int, nonce: int, out, stream=None):
        z = np.ascontiguousarray(slots, dtype=np.float64)
        self._check(lib().fhe_encrypt(self.h, z.ctypes.data if z.size else None, z.size, level, nonce,
                                      _ptr(out), _stream(stream)))

    def encrypt_coeffs(self, coeffs_dev, level: int, nonce: int, out, stream=None):
        self._check(lib().fhe_encrypt_coeffs(self.h, _ptr(coeffs_dev), level, nonce, _ptr(out), _stream(stream)))

    def decrypt(self, ct, level: int, n_slots: Optional[int] = None, stream=None) -> np.ndarray:
        n_slots = self.slots if n_slots is None else n_slots
        out = np.zeros(n_slots, dtype=np.float64)
        self._check(lib().fhe_decrypt(self.h, _ptr(ct), level, out.ctypes.data, n_slots, _stream(stream)))
        return out

    def refresh(self, ct, count: int, level: int, nonce_base: int, out, stream=None):
        self._check(lib().fhe_refresh(self.h, _ptr(ct), count, level, nonce_base, _ptr(out), _stream(stream)))

    # ---- primitives
    def ntt_forward(self, polys, count: int, n_limbs: int, stream=None):
        self._check(lib().fhe_ntt_forward(self.h, _ptr(polys), count, n_limbs, _stream(stream)))

    def ntt_inverse(self, polys, count: int, n_limbs: int, stream=None):
        self._check(lib().fhe_ntt_inverse(self.h, _ptr(polys), count, n_limbs, _stream(stream)))

    def ct_to_coeff(self, ct, count: int, level: int, out, stream=None):
        self._check(lib().fhe_ct_to_coeff(self.h, _ptr(ct), count, level, _ptr(out), _stream(stream)))

    def add(self, a, b, out, count: int, level: int, stream=None):
        self._check(lib().fhe_add(self.h, _ptr(a), _ptr(b), _ptr(out), count, level, _stream(stream)))

    def sub(self, a, b, out, count: int, level: int, stream=None):
        self._check(lib().fhe_sub(self.h, _ptr(a), _ptr(b), _ptr(out), count, level, _stream(stream)))

    def mul_plain(self, ct, pt_dev, out, count: int, level: int, stream=None):
        self._check(lib().fhe_mul_plain(self.h, _ptr(ct), _ptr(pt_dev), _ptr(out), count, level, _stream(stream)))

    def tensor(self, a, b, out3, count: int, level: int, stream=None):
        self._check(lib().fhe_tensor(self.h, _ptr(a), _ptr(b), _ptr(out3), count, level, _stream(stream)))

    def relinearize(self, in3, out, count: int, level: int, stream=None):
        self._check(lib().fhe_relinearize(self.h, _ptr(in3), _ptr(out), count, level, _stream(stream)))

    def rescale(self, ct, out, count: int, level: int, stream=None):
        self._check(lib().fhe_rescale(self.h, _ptr(ct), _ptr(out), count, level, _stream(stream)))

    def rescale_noalloc(self, ct, out, level: int, stream=None):
        """Rescale one ciphertext using only the library's static scratch (no allocation)."""
        self._check(lib().fhe_rescale_noalloc(self.h, _ptr(ct), _ptr(out), level, _stream(stream)))

    def mul_relin_rescale(self, a, b, out, count: int, level: int, stream=None):
        self._check(lib().fhe_mul_relin_rescale(self.h, _ptr(a), _ptr(b), _ptr(out), count, level,
                                                _stream(stream)))

    def rotate(self, ct, out, count: int, level: int, step: int, stream=None):
        self._check(lib().fhe_rotate(self.h, _ptr(ct), _ptr(out), count, level, step, _stream(stream)))

    def rotate_sum(self, ct, out, count: int, level: int, kp: int, stream=None):
        """out = sum_{r < kp} rot(ct, r) (hoisted for kp <= 16)."""
        self._check(lib().fhe_rotate_sum(self.h, _ptr(ct), _ptr(out), count, level, kp, _stream(stream)))

    def rotate_fanin(self, acc, first, ct, steps, level: int, stream=None):
        """acc_g += sum_{first[g] <= i < first[g+1]} rot(ct_i, steps[i]), one ModDown per group."""
        fo = np.ascontiguousarray(first, dtype=np.int32)
        st = np.ascontiguousarray(steps, dtype=np.int32)
        self._check(lib().fhe_rotate_fanin(self.h, _ptr(acc), fo.size - 1, fo.ctypes.data, _ptr(ct) if st.size else None,
                                           st.ctypes.data if st.size else None, level, _stream(stream)))

    def serve_rotation_steps(self, k: int):
        buf = np.zeros(256, dtype=np.int32)
        rc = lib().fhe_serve_rotation_steps(self.h, k, buf.ctypes.data, buf.size)
        if rc < 0:
            self._check(rc)
        return [int(x) for x in buf[:rc]]

    def encrypt_request(self, m: int, k: int, u0, items, ratings, nonce_base: int, UR, R, stream=None):
        u = np.ascontiguousarray(u0, dtype=np.float64)
        it = np.ascontiguousarray(items, dtype=np.int32)
        rt = np.ascontiguousarray(ratings, dtype=np.float64)
        self._check(lib().fhe_serve_encrypt_request(self.h, m, k, u.ctypes.data, it.ctypes.data if it.size else None,
                                                    rt.ctypes.data if rt.size else None, it.size, nonce_base,
                                                    _ptr(UR), _ptr(R), _stream(stream)))

    # ---- launch accounting
    def probe_butterfly_rate(self, reps: int = 2000) -> float:
        """Register-only rate of the NTT butterfly arithmetic on this GPU, in 10^9 butterflies/s."""
        out = ctypes.c_double(0.0)
        self._check(lib().fhe_probe_butterfly_rate(self.h, reps, ctypes.byref(out)))
        return out.value

    def probe_int_pipe(self, reps: int = 500) -> dict:
        """Register-only issue rates of the 32-bit multiply instructions (10^9 instructions/s) and of
        four 64 x 64 -> 128-bit multiply-accumulate formulations (10^9 MACs/s) on this GPU."""
        out = IntPipeRates()
        self._check(lib().fhe_probe_int_pipe(self.h, reps, ctypes.byref(out)))
        return {name: getattr(out, name) for name, _ in IntPipeRates._fields_}

    def probe_conv_cost(self, level: int, sources: int = 64) -> dict:
        """Device time of the ModUp conversion pass set with and without the base conversion in its
        loads, the rows it transforms and the HBM bytes an unfused conversion would add."""
        out = ConvCost()
        self._check(lib().fhe_probe_conv_cost(self.h, level, sources, ctypes.byref(out)))
        return {name: getattr(out, name) for name, _ in ConvCost._fields_}

    def autotune(self, level: int = None, cache: Optional[str] = None) -> list:
        """Time every launch variant of each tunable kernel family at `level` (default: one below the
        top, the level of an epoch's per-group products) and keep the fastest. Returns
        [{family, variant, chosen, ms}]. With `cache` (a JSON file path), choices are stored under the
        GPU model and the ring (degree, primes, level), and a later call that finds its key sets the
        stored choices without timing (records then carry ms None and cached True)."""
        level = self.top - 1 if level is None else level
        key = None
        if cache:
            import torch
            key = tune_cache_key(torch.cuda.get_device_name(self.device), self.n, self.primes, level)
            hit = load_tune_cache(cache).get(key)
            if hit:
                for fam, var in hit.items():
                    self.set_variant(fam, var)
                return [{"family": f, "variant": v, "chosen": True, "ms": None, "cached": True}
                        for f, v in hit.items()]
        arr = (TuneResult * 64)()
        n = lib().fhe_autotune(self.h, level, arr, 64)
        if n < 0:
            self._check(n)
        res = [{"family": r.family.decode(), "variant": r.variant.decode(), "chosen": bool(r.chosen),
                "ms": r.ms} for r in arr[:min(n, 64)]]
        if key:
            store_tune_cache(cache, key, {r["family"]: r["variant"] for r in res if r["chosen"]})
        return res

    def set_variant(self, family: str, variant: str):
        self._check(lib().fhe_set_variant(self.h, family.encode(), variant.encode()))

    def get_variant(self, family: str) -> str:
        out = ctypes.c_char_p()
        self._check(lib().fhe_get_variant(self.h, family.encode(), ctypes.byref(out)))
        return out.value.decode()

    def profile_begin(self, time_kernels: bool = False):
        self._check(lib().fhe_profile_begin(self.h, 1 if time_kernels else 0))

    def profile_end(self):
        """-> {class name: (launches, device_ms, algorithmic_bytes, work)}; work is butterflies for the NTT
        classes and 64 x 64-bit multiply-accumulates for ks_inner."""
        arr = (KernelStat * 32)()
        rc = lib().fhe_profile_end(self.h, ctypes.cast(arr, ctypes.c_void_p), 32)
        if rc < 0:
            self._check(rc)
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].device_ms), float(arr[i].bytes),
                                       float(arr[i].work)) for i in range(rc)}

    # ---- matrix factorisation
    def mf_rotation_steps(self, k: int):
        buf = np.zeros(256, dtype=np.int32)
        rc = lib().fhe_mf_rotation_steps(self.h, k, buf.ctypes.data, buf.size)
        if rc < 0:
            self._check(rc)
        return [int(x) for x in buf[:rc]]


class MfPlan:
    """Owns one fhe_mf_plan (groups, delta trees and encrypted ratings on the device)."""

    def __init__(self, ctx: Context, n: int, m: int, k: int, row_ptr, col_idx, vals):
        self.ctx = ctx
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        vv = np.ascontiguousarray(vals, dtype=np.float64)
        h = ctypes.c_void_p()
        ctx._check(lib().fhe_csr_pack(ctx.h, n, m, k, rp.ctypes.data, ci.ctypes.data if ci.size else None,
                                      vv.ctypes.data if vv.size else None, ctypes.byref(h)))
        self.h = h
        info = PlanInfo()
        ctx._check(lib().fhe_mf_plan_get_info(self.h, ctypes.byref(info)))
        self.info = info
        self.n_ub, self.n_vb = info.n_user_batches, info.n_item_batches
        self.B, self.w, self.kp, self.k = info.B, info.w, info.kp, info.k

    def close(self):
        if getattr(self, "h", None):
            lib().fhe_mf_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self):
        g = int(self.info.n_groups)
        b, c, d, cnt = (np.zeros(g, dtype=np.int32) for _ in range(4))
        self.ctx._check(lib().fhe_mf_plan_get_groups(self.h, b.ctypes.data, c.ctypes.data, d.ctypes.data,
                                                     cnt.ctypes.data))
        return b, c, d, cnt

    def bins(self):
        """Rating bin of each group (int32 [n_groups])."""
        out = np.zeros(max(int(self.info.n_groups), 1), dtype=np.int32)
        self.ctx._check(lib().fhe_mf_plan_get_bins(self.h, out.ctypes.data))
        return out[: int(self.info.n_groups)]

    def set_wave_budget(self, nbytes: int):
        """Node-workspace budget per wave of item batches (results do not depend on it)."""
        self.ctx._check(lib().fhe_mf_plan_set_wave_budget(self.h, nbytes))

    def set_chunk(self, groups_per_chunk: int):
        self.ctx._check(lib().fhe_mf_plan_set_chunk(self.h, groups_per_chunk))

    def encrypt_factors(self, which: int, X, out, stream=None):
        X = np.ascontiguousarray(X, dtype=np.float64)
        self.ctx._check(lib().fhe_mf_encrypt_factors(self.ctx.h, self.h, which, X.ctypes.data, X.shape[0],
                                                     _ptr(out), _stream(stream)))

    def decrypt_factors(self, which: int, cts, level: int, count: int, stream=None) -> np.ndarray:
        X = np.zeros((count, self.k), dtype=np.float64)
        self.ctx._check(lib().fhe_mf_decrypt_factors(self.ctx.h, self.h, which, _ptr(cts), level,
                                                     X.ctypes.data, count, _stream(stream)))
        return X

    def sgd_epoch(self, U, V, level: int, lr: float, lam: float, stream=None):
        self.ctx._check(lib().fhe_mf_sgd_epoch(self.ctx.h, self.h, _ptr(U), _ptr(V), level, lr, lam,
                                               _stream(stream)))

    def predict(self, U, V, level: int, user: int, out, stream=None):
        self.ctx._check(lib().fhe_predict(self.ctx.h, self.h, _ptr(U), _ptr(V), level, user, _ptr(out),
                                          _stream(stream)))


class Server:
    """Owns one fhe_server: continuous-batching fold-in + predict over resident item factors."""

    def __init__(self, ctx: Context, V, m: int, k: int, steps: int, lr: float, lam: float, max_slots: int,
                 memory_budget_bytes: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(lib().fhe_serve_create(ctx.h, _ptr(V), m, k, steps, lr, lam, max_slots, memory_budget_bytes,
                                          ctypes.byref(h)))
        self.h = h
        tot, fr = ctypes.c_int32(), ctypes.c_int32()
        ctx._check(lib().fhe_serve_slots(self.h, ctypes.byref(tot), ctypes.byref(fr)))
        self.n_slots = tot.value

    def close(self):
        if getattr(self, "h", None):
            lib().fhe_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def free_slots(self) -> int:
        tot, fr = ctypes.c_int32(), ctypes.c_int32()
        self.ctx._check(lib().fhe_serve_slots(self.h, ctypes.byref(tot), ctypes.byref(fr)))
        return fr.value

    def submit(self, request_id: int, items, UR, R, stream=None) -> bool:
        """True if admitted; False if no slot is free (FHE_ERR_STATE)."""
        it = np.ascontiguousarray(items, dtype=np.int32)
        rc = lib().fhe_serve_submit(self.h, request_id, it.ctypes.data if it.size else None, it.size, _ptr(UR),
                                    _ptr(R), _stream(stream))
        if rc == -8:
            return False
        self.ctx._check(rc)
        return True

    def tick(self, stream=None) -> int:
        rc = lib().fhe_serve_tick(self.h, _stream(stream))
        if rc < 0:
            self.ctx._check(rc)
        return rc

    def poll(self):
        ids = np.zeros(4096, dtype=np.int64)
        n = lib().fhe_serve_poll(self.h, ids.ctypes.data, ids.size)
        if n < 0:
            self.ctx._check(n)
        return [int(x) for x in ids[:n]]

    def take(self, request_id: int, out, stream=None) -> int:
        lv = ctypes.c_int32()
        self.ctx._check(lib().fhe_serve_take(self.h, request_id, _ptr(out), ctypes.byref(lv), _stream(stream)))
        return lv.value
