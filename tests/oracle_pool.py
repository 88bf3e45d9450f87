"""Oracle set-up spread over host cores for the large-ring parity tests (test infrastructure).

At N = 2^15 and 2^16 the oracle spends most of a test's set-up on rotation keys and on encodings
(the definition-level encoder is O(N * slots)). The keys and encodings are independent, so a pool
of spawned processes (spawned, not forked: the test process already holds a CUDA context) computes
them at once, each worker on its own oracle context with the same parameters and seed. The results
are the oracle's own, computed by its own code; only the scheduling differs."""
from __future__ import annotations

import multiprocessing as mp
import os

_HE = None


def _init(preset_name: str, seed: int):
    global _HE
    from oracle import ckks
    from paper_2509_03024_gb300.workloads import PRESETS
    _HE = ckks.Ckks(ckks.Params.from_preset(PRESETS[preset_name]))
    _HE.keygen(seed, [])


def _task(job):
    kind, arg = job
    if kind == "rot":
        g = _HE.prm.galois(arg)
        _HE.add_rotation_key(arg)
        key = _HE.rot.pop(g)
        return kind, g, key
    if kind == "encode":
        return kind, None, _HE.enc.encode(arg)
    raise ValueError(kind)


def workers(cap: int = 16) -> int:
    cpus = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return max(1, min(cap, cpus))


def oracle_setup(preset_name: str, seed: int, rot_steps=(), encodings=()):
    """An oracle context keyed by `seed` with the rotation keys of `rot_steps`, and the encodings of
    the slot vectors in `encodings` (a list, in order), computed by a spawn pool."""
    from oracle import ckks
    from paper_2509_03024_gb300.workloads import PRESETS
    he = ckks.Ckks(ckks.Params.from_preset(PRESETS[preset_name]))
    he.keygen(seed, [])
    jobs, seen = [], set()
    for r in rot_steps:
        g = he.prm.galois(r)
        if g not in seen and g not in he.rot:
            seen.add(g)
            jobs.append(("rot", r))
    jobs += [("encode", z) for z in encodings]
    enc = []
    if jobs:
        ctx = mp.get_context("spawn")
        with ctx.Pool(min(workers(), len(jobs)), initializer=_init, initargs=(preset_name, seed)) as pool:
            for kind, g, val in pool.imap(_task, jobs):
                if kind == "rot":
                    he.rot[g] = val
                else:
                    enc.append(val)
    return he, enc
