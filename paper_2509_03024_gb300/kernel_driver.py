"""Run one batched kernel workload through the C ABI (for timing and ncu captures).

  python -m paper_2509_03024_gb300.kernel_driver ntt --preset paper --rows 1024 [--inverse] [--reps 3]
  python -m paper_2509_03024_gb300.kernel_driver keyswitch --preset paper --count 64 [--reps 3]
  python -m paper_2509_03024_gb300.kernel_driver rotsum --preset paper --count 64 --kp 16 [--reps 3]
  python -m paper_2509_03024_gb300.kernel_driver probe --preset paper [--reps 2000]
  python -m paper_2509_03024_gb300.kernel_driver tune --preset paper [--level L]
  python -m paper_2509_03024_gb300.kernel_driver convcost --preset paper [--level L] [--count 64]
  (any kind) --variants family=variant,...   sets autotuner families, e.g. ntt=r8b4,ks_pass=r8

`ntt` transforms `rows` limbs of N residues in place (rows / (L+1) polynomials
of L+1 limbs); `keyswitch` rotates `count` top-level ciphertexts by one slot
(automorphism + hybrid key switch); `rotsum` runs the in-block rotate-and-sum over kp
slots on `count` ciphertexts one level below the top (the level of the per-group
product in an epoch). Prints CUDA-event timings per repetition and, for the last
repetition, the device time of each kernel class; `probe` prints the register-only
butterfly rate of fhe_probe_butterfly_rate (`reps` loop trips) and the integer-pipe rates of
fhe_probe_int_pipe; `tune` runs the autotuner at `level` (default top - 1) and prints every
variant's time; `convcost` times the ModUp conversion pass set over `count` sources with and
without the base conversion in its loads (fhe_probe_conv_cost, at `level`, default the top).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch
    from paper_2509_03024_gb300 import build, capi
    from paper_2509_03024_gb300.workloads import PRESETS

    ap = argparse.ArgumentParser()
    ap.add_argument("kind", choices=["ntt", "keyswitch", "rotsum", "probe", "tune", "convcost"])
    ap.add_argument("--level", type=int, default=None)
    ap.add_argument("--variant", default=None, help="inner-product variant to use (ks_inner and ks_hoist_inner)")
    ap.add_argument("--variants", default="", help="family=variant,... of the autotuner families to set")
    ap.add_argument("--kp", type=int, default=16)
    ap.add_argument("--preset", default="paper")
    ap.add_argument("--rows", type=int, default=1024)
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--inverse", action="store_true")
    args = ap.parse_args()
    build.build()
    ctx = capi.Context.from_preset(PRESETS[args.preset])
    if args.kind == "probe":
        print(json.dumps({"kind": "probe", "preset": args.preset, "reps": args.reps,
                          "gbfly_per_s": ctx.probe_butterfly_rate(args.reps),
                          "int_pipe": ctx.probe_int_pipe(max(1, args.reps // 4))}))
        return
    if args.kind == "tune":
        print(json.dumps({"kind": "tune", "preset": args.preset, "results": ctx.autotune(args.level)}))
        return
    if args.kind == "convcost":
        lv = ctx.top if args.level is None else args.level
        print(json.dumps({"kind": "convcost", "preset": args.preset, "level": lv, "sources": args.count,
                          **ctx.probe_conv_cost(lv, args.count)}))
        return
    if args.variant:
        ctx.set_variant("ks_inner", args.variant)
        ctx.set_variant("ks_hoist_inner", args.variant)
    for fv in filter(None, args.variants.split(",")):
        fam, var = fv.split("=")
        ctx.set_variant(fam, var)
    if args.kind == "keyswitch":
        ctx.keygen(1, [1])
    elif args.kind == "rotsum":
        ctx.keygen(1, list(range(1, args.kp)) if args.kp <= 16 else [1 << t for t in range(args.kp.bit_length() - 1)])
    L1 = ctx.top + 1
    times = []
    if args.kind == "ntt":
        polys = max(1, args.rows // L1)
        rng = np.random.default_rng(0)
        host = np.stack([rng.integers(0, q, (polys, ctx.n), dtype=np.uint64) for q in ctx.primes[:L1]], axis=1)
        buf = torch.from_numpy(host.view(np.int64).copy()).cuda()
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if args.inverse:
                ctx.ntt_inverse(buf, polys, L1)
            else:
                ctx.ntt_forward(buf, polys, L1)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        alg = 16.0 * polys * L1 * ctx.n
    if args.kind != "ntt":
        cts = ctx.empty_ct(args.count)
        for t in range(args.count):
            w = 2 * L1 * ctx.n
            ctx.encrypt(np.random.default_rng(t).normal(size=16), ctx.top, t, cts[t * w:(t + 1) * w])
        out = ctx.empty_ct(args.count)
        for r in range(args.reps):
            last = r == args.reps - 1
            if last:
                ctx.profile_begin(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if args.kind == "keyswitch":
                ctx.rotate(cts, out, args.count, ctx.top, 1)
            else:
                ctx.rotate_sum(cts, out, args.count, ctx.top - 1, args.kp)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            if last:
                per_class = {k: v[1] for k, v in ctx.profile_end().items()}
        alg = None
    res = {"kind": args.kind, "preset": args.preset, "ms": times}
    if args.kind != "ntt":
        res["kernel_ms"] = per_class
    if alg:
        res["alg_gbs_best"] = alg / (min(times) / 1e3) / 1e9
    print(json.dumps(res))


if __name__ == "__main__":
    main()
