#!/usr/bin/env python
"""Served encrypted matrix factorisation on one GB300: ratings/s with p50/p99 latency, continuous
batching against one request at a time.

Headline workload (the served configuration): resident encrypted item factors, 3706 items x k = 16,
RNS-CKKS N = 2^16 with thirteen 50-bit data primes and three 60-bit special primes, scale 2^50.
Requests arrive as a Poisson stream; each carries one user's encrypted CSR rating row (nnz
log-uniform 5..300, Zipf(1.0) items, MovieLens rating law) and an initial user factor, and is
answered with the encrypted predicted-rating row over every item after 5 encrypted SGD fold-in
steps (lr 0.005, lambda 0.02). For every arrival rate in 50, 100, 200, 500, 1000, 2000 req/s the
same request stream (1000 requests) runs through the continuous-batching server (48 request slots
under a memory budget) and through the same server with one slot (one request at a time). The line's
`value`, p50_ms and p99_ms are the batched server's at the top rate; the one-by-one numbers and the
whole sweep sit beside them. `e2e` repeats the top rate with request ciphertexts uploaded from
page-locked host memory and predictions downloaded to host memory inside the timed loop.

Sub-record `epoch`: one encrypted SGD epoch of the paper-scale configuration (943 users x 1682
items, 100,000 synthetic MovieLens-shaped ratings, k = 10, N = 2^15, 8 x 50-bit + 2 x 60-bit primes)
per step, with its decrypted accuracy against FP64.

Each part carries the per-kernel-class rooflines: NTT classes in butterflies/s and the key inner
products in multiply-accumulates/s against integer ceilings from the integer-pipe rates measured in
the same run, every class in algorithmic bytes/s against the measured HBM bandwidth. Multi-GPU runs
are independent replicas (weak scaling). The CPU baseline is the oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload served|paper|large|batched] [--served-sweep R1,R2,...]
                  [--served-requests R] [--no-epoch] [--no-cpu-baseline]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "encrypted MF ratings/sec, served vs one-by-one on 1 GB300; p50/p99 latency"
# DRAM bytes per limb row of a forward NTT pass at N = 2^15, from the ncu capture (dram__bytes_read
# + write) of the fused ModUp passes of the current kernels (the hoisted rotate-and-sum of 64
# ciphertexts at level 6, 1856 rows per pass): (552.8 MB + 917.4 MB) / 2 passes / 1856 rows
NCU_FWD_DRAM_BYTES_PER_ROW = (552.8e6 + 917.4e6) / 2 / 1856
# the same for the served ring's forward passes (N = 2^16, 13 + 3 primes): ncu dram__bytes_read + write
# of the four forward passes (ModUp conversion and second pass, ModDown conversion and combine) of a
# key switch of 8 top-level ciphertexts, 1240 MB over 1488 limb-row passes (0.79 x the algorithmic 16 N)
NCU_SERVED_FWD_DRAM_BYTES_PER_ROW = 1239.7e6 / 1488
UNIT = "ratings/s"
SEED = 20250903
LR, LAM, K_RANK = 0.005, 0.02, 10
WORKLOAD = ("paper-scale encrypted MF epoch: 943 users x 1682 items, 100,000 synthetic MovieLens-shaped "
            "ratings (90,000 train), k=10; RNS-CKKS N=2^15, 8x50-bit data + 2x60-bit special primes, "
            "scale 2^50; one SGD epoch (lr 0.005, lambda 0.02) per step")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-kernel-timing", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variants", default="", help="family=variant,... to set instead of autotuning "
                                                   "(e.g. for a reproducible profile)")
    ap.add_argument("--served-requests", type=int, default=1000, help="requests per arrival rate")
    ap.add_argument("--served-pool", type=int, default=256, help="distinct pre-encrypted requests")
    ap.add_argument("--served-slots", type=int, default=48)
    ap.add_argument("--served-sweep", default="", help="comma-separated arrival rates (req/s); default "
                                                       "50,100,200,500,1000,2000 (the last one is the headline)")
    ap.add_argument("--e2e-requests", type=int, default=300)
    ap.add_argument("--epoch-steps", type=int, default=3, help="timed epochs of the epoch sub-record")
    ap.add_argument("--no-epoch", action="store_true")
    ap.add_argument("--workload", choices=["served", "paper", "large", "batched"], default="served",
                    help="served: the served fold-in + predict workload (headline) with the paper-scale epoch "
                         "as a sub-record; paper: the paper-scale epoch alone; large: the 6040 x 3706 workload "
                         "at N=2^16; batched: independent instances")
    ap.add_argument("--instances", type=int, default=64, help="instances of the batched workload")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def start_clocks(device: int):
    path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
    try:
        proc = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={CLOCK_FIELDS}",
                                 "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None, path
    return proc, path


def stop_clocks(proc, path):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workload

LARGE = ("large encrypted MF epoch: 6040 users x 3706 items, 1,000,209 synthetic MovieLens-1M-shaped ratings "
         "(Zipf 1.1, 90 % train), k=16; RNS-CKKS N=2^16, 20x50-bit data + 3x60-bit special primes, scale 2^50; "
         "one SGD epoch (lr 0.0002, lambda 0.02) per step")


BATCHED = ("batched encrypted MF: independent instances (users U[50, 2000], items U[40, 3000], density "
           "log-uniform 1-6 %, Zipf 1.0), k=8; RNS-CKKS N=2^16, 12x50-bit data + 3x60-bit special primes, "
           "scale 2^50; one SGD epoch (lr 0.005, lambda 0.02) of every instance, the instances one after "
           "another through one context and its keys (one warm-up epoch each, untimed)")


def run_batched(args):
    """The batched workload as consecutive plans: each instance's plan is built, warmed up with one
    epoch (which allocates its workspace), timed on a second epoch from the same start, checked
    against FP64 and released before the next. Reports training ratings / summed epoch time."""
    import torch
    from paper_2509_03024_gb300 import build as B
    B.build()
    from oracle import mf as omf
    from paper_2509_03024_gb300 import capi
    from paper_2509_03024_gb300 import workloads as W
    k = 8
    inst = W.batched_instances(args.instances)
    ctx = capi.Context.from_preset(W.PRESETS["batched"])
    ctx.keygen(SEED, ctx.mf_rotation_steps(k))
    stream = torch.cuda.Stream()
    ratings, epoch_ms, groups, bins, max_err = 0, 0.0, 0, 0, 0.0
    busy = []
    tuning = autotune(ctx, args)
    wall0 = time.perf_counter()
    for csr, U, V in inst:
        plan = capi.MfPlan(ctx, csr.n, csr.m, k, csr.row_ptr, csr.col_idx, csr.vals)
        UD0, VD0 = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
        plan.encrypt_factors(0, U, UD0)
        plan.encrypt_factors(1, V, VD0)
        UD, VD = UD0.clone(), VD0.clone()
        plan.sgd_epoch(UD, VD, ctx.top, LR, LAM, stream)
        with torch.cuda.stream(stream):
            UD.copy_(UD0)
            VD.copy_(VD0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.sgd_epoch(UD, VD, ctx.top, LR, LAM, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        epoch_ms += e0.elapsed_time(e1)
        # a third epoch from the same start with every launch timed: the share of the epoch's device
        # span covered by kernels (how much room merged launches of several instances could fill)
        with torch.cuda.stream(stream):
            UD.copy_(UD0)
            VD.copy_(VD0)
        torch.cuda.synchronize()
        ctx.profile_begin(time_kernels=True)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        plan.sgd_epoch(UD, VD, ctx.top, LR, LAM, stream)
        e3.record(stream)
        torch.cuda.synchronize()
        kern = sum(v[1] for v in ctx.profile_end().values())
        busy.append(kern / e2.elapsed_time(e3))
        rows, cols, vals = csr.triples()
        U1, V1 = omf.mf_epoch_fp64(U, V, rows, cols, vals, LR, LAM)
        Ud = plan.decrypt_factors(0, UD, ctx.top - 2, csr.n)
        Vd = plan.decrypt_factors(1, VD, ctx.top - 2, csr.m)
        max_err = max(max_err, float(np.abs(Ud - U1).max()), float(np.abs(Vd - V1).max()))
        ratings += csr.nnz
        groups += int(plan.info.n_groups)
        bins += int(plan.info.n_bins)
        plan.close()
        del UD, VD, UD0, VD0
    return {"metric": METRIC, "value": ratings / (epoch_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": epoch_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": BATCHED, "instances": len(inst), "ratings_per_step": ratings,
                       "groups": groups, "rating_bins": bins, "parallelism": "replicas"},
            "accuracy": {"max_abs_vs_fp64": max_err}, "wall_s": time.perf_counter() - wall0,
            "device_busy_fraction": {"min": min(busy), "median": statistics.median(busy), "max": max(busy),
                                     "note": "per instance: summed kernel time / the epoch's device span "
                                             "(a separate epoch with every launch timed)"},
            "tuning": tuning}


def workload_spec(name):
    """(preset, rank, learning rate, description) of a bench workload."""
    if name == "large":   # lr 0.0002: the largest stable rate of the accumulated update at this shape
        return "large", 16, 0.0002, LARGE
    return "paper", K_RANK, LR, WORKLOAD


def workload(name="paper"):
    from paper_2509_03024_gb300 import workloads as W
    if name == "large":
        full = W.movielens_like(6040, 3706, 1_000_209, 1.1, 5)
        train, test = W.split_holdout(full, 0.1, 12)
        return train, test, W.init_factors(6040, 16, 105), W.init_factors(3706, 16, 205)
    train, test, U, V = W.paper_workload(seed=2)
    return train, test, U, V


def measured_peaks():
    try:
        return json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------------------------- CPU oracle baseline

def oracle_setup(train, U, V, groups_sampled: int = 1, only=None):
    """Keys, plan and the sampled groups' ciphertexts on the oracle (not timed). The sample is
    `groups_sampled` groups spread evenly over the plan; `only` keeps one of them."""
    from oracle import ckks, mf
    from paper_2509_03024_gb300.workloads import PRESETS
    rows, cols, vals = train.triples()
    he = ckks.Ckks(ckks.Params.from_preset(PRESETS["paper"]))
    plan = mf.build_plan(train.n, train.m, K_RANK, rows, cols, vals, he.prm.slots)
    steps = mf.rotsum_steps(plan.kp) + [plan.w]
    he.keygen(SEED, steps)
    emf = mf.EncryptedMF(he, plan)
    top = he.prm.top
    pick = list(range(0, len(plan.groups), max(1, len(plan.groups) // groups_sampled)))[:groups_sampled]
    if only is not None:
        pick = [pick[only]]
    emf.R = [None] * len(plan.bin_batch)
    for t in pick:
        bt = plan.bin_of[t]
        emf.R[bt] = he.encrypt_seeded(he.enc.encode(mf.bin_slots(bt, plan)), top - 1, mf.R_NONCE_BASE + bt)
    UD = {g.b: None for g in (plan.groups[t] for t in pick)}
    for b in UD:
        UD[b] = he.encrypt(mf.pack_factors(U, plan, b), top, mf.U_NONCE_BASE + b)
    VDc = {}
    for t in pick:
        c = plan.groups[t].c
        if c not in VDc:
            VDc[c] = he.encrypt(mf.pack_factors(V, plan, c), top, mf.V_NONCE_BASE + c)
    return {"he": he, "plan": plan, "emf": emf, "pick": pick, "UD": UD, "VDc": VDc, "ratings": rows.size,
            "groups": len(plan.groups), "nodes": sum(len(c) for c in plan.closure)}


def oracle_measure(st):
    """Seconds the oracle (as it stands) takes for one sampled group's work (product,
    relinearise-rescale, rotate-and-sum, masks, tensors; averaged over the sample) and for one
    delta-tree rotation."""
    he, plan, emf, pick = st["he"], st["plan"], st["emf"], st["pick"]
    t0 = time.perf_counter()
    for t in pick:
        g = plan.groups[t]
        emf.group_terms(t, st["UD"][g.b], st["VDc"][g.c], LR)   # Vr of delta 0 stands in for the rotated copy
    t_group = (time.perf_counter() - t0) / len(pick)
    t1 = time.perf_counter()
    he.rotate(next(iter(st["VDc"].values())), plan.w)
    return t_group, time.perf_counter() - t1


def oracle_epoch_s(st, t_group, t_rot, cores=1):
    """Epoch time extrapolated from the sample: groups x t_group + 3 x tree nodes x t_rot (the
    rotation, relinearisation and back-rotation of every node), spread over `cores` processes
    (the groups and the nodes of one tree level are independent)."""
    return (t_group * st["groups"] + t_rot * 3 * st["nodes"]) / cores


def oracle_time(st):
    """One single-thread sample, extrapolated to an epoch. Returns (ratings/s, seconds measured,
    description)."""
    t0 = time.perf_counter()
    t_group, t_rot = oracle_measure(st)
    est = oracle_epoch_s(st, t_group, t_rot)
    desc = (f"oracle on {len(st['pick'])} of {st['groups']} groups + 1 rotation at N=2^15, single thread; "
            f"epoch extrapolated as groups x {t_group:.2f} s + {3 * st['nodes']} rotation-sized key switches x "
            f"{t_rot:.2f} s = {est:.0f} s")
    return st["ratings"] / est, time.perf_counter() - t0, desc


def oracle_sample(train, U, V, groups_sampled: int = 1):
    return oracle_time(oracle_setup(train, U, V, groups_sampled))


def _oracle_worker(index, n_workers, cmd, res):
    """One process of the all-core oracle baseline: sets up its own sampled group (group `index` of
    `n_workers` spread over the plan), then times that group and one rotation whenever told to."""
    try:
        train, _, U, V = workload()
        st = oracle_setup(train, U, V, groups_sampled=n_workers, only=index)
        res.put(("ready", index, {k: st[k] for k in ("ratings", "groups", "nodes")}))
        while cmd.get() == "go":
            res.put(("time", index, oracle_measure(st)))
    except Exception as e:   # reported to the parent, which then gives up on the all-core figure
        res.put(("error", index, repr(e)))


def oracle_workers(cap: int = 16, bytes_per_worker: float = 2.0 * 2**30) -> int:
    """Worker processes for the all-core baseline: the CPUs this process may run on, at most
    `cap`, and no more than available memory allows (about 1.3 GB peak per worker at N = 2^15)."""
    cpus = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        with open("/sys/fs/cgroup/memory.max") as f:
            lim = f.read().strip()
        if lim != "max":
            avail = min(avail or int(lim), int(lim))
    except (OSError, ValueError):
        pass
    n = min(cpus, cap)
    if avail is not None:
        n = min(n, max(1, int(avail // bytes_per_worker)))
    return max(1, n)


class OracleCores:
    """Independent single-threaded oracle processes (spawned, so no process inherits a CUDA
    context), one sampled group each, timed concurrently on the host's cores."""

    def __init__(self, n_workers: int, timeout_s: float = 900.0):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.n, self.timeout = n_workers, timeout_s
        self.cmds = [ctx.Queue() for _ in range(n_workers)]
        self.res = ctx.Queue()
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({v: "1" for v in saved})   # one thread per worker
        try:
            self.procs = [ctx.Process(target=_oracle_worker, args=(i, n_workers, self.cmds[i], self.res),
                                      daemon=True) for i in range(n_workers)]
            for p in self.procs:
                p.start()
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        self.info = self._collect(n_workers)[0]

    def _collect(self, count):
        out = {}
        while len(out) < count:
            kind, i, v = self.res.get(timeout=self.timeout)
            if kind == "error":
                raise RuntimeError(f"oracle worker {i}: {v}")
            out[i] = v
        return out

    def sample(self, workers):
        """Time the given workers' groups concurrently: {worker: (t_group, t_rot)}."""
        for i in workers:
            self.cmds[i].put("go")
        return self._collect(len(workers))

    def rate(self, times):
        """Ratings/s of an epoch spread over len(times) processes, from their concurrent samples."""
        tg = statistics.mean(t[0] for t in times.values())
        tr = statistics.mean(t[1] for t in times.values())
        est = oracle_epoch_s(self.info, tg, tr, cores=len(times))
        return self.info["ratings"] / est, tg, tr, est

    def close(self):
        for q in self.cmds:
            q.put("stop")
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)


def oracle_baseline():
    """The GPU line's cpu_baseline: the oracle on every available core (one process per core, each
    timing its own group concurrently), with the same sample on one core alone beside it."""
    t0 = time.perf_counter()
    pool = OracleCores(oracle_workers())
    try:
        one = pool.rate(pool.sample([0]))
        allc = pool.rate(pool.sample(range(pool.n)))
    finally:
        pool.close()
    G, nodes = pool.info["groups"], pool.info["nodes"]
    desc = (f"oracle at N=2^15, {pool.n} single-threaded processes at once, each on its own group (of "
            f"{G}) and one rotation; epoch extrapolated as (groups x {allc[1]:.2f} s + {3 * nodes} "
            f"rotation-sized key switches x {allc[2]:.2f} s) / {pool.n} = {allc[3]:.0f} s")
    return {"value": allc[0], "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": desc,
            "single_thread": {"value": one[0], "unit": UNIT, "cores": 1,
                              "sample": f"the same oracle on one group alone: groups x {one[1]:.2f} s + "
                                        f"{3 * nodes} x {one[2]:.2f} s = {one[3]:.0f} s"},
            "measured_s": round(time.perf_counter() - t0, 1)}


# ----------------------------------------------------------------------------- served workload

SERVED = ("served fold-in + predict: resident encrypted item factors 3706 x k=16 (N=2^16, 13x50-bit + "
          "3x60-bit primes, scale 2^50); Poisson arrivals at 50-2000 req/s; per request one user's encrypted "
          "CSR row (nnz log-uniform 5..300, Zipf(1.0) items, MovieLens rating law), 5 encrypted SGD fold-in "
          "steps (lr 0.005, lambda 0.02) then the encrypted predicted-rating row over all 3706 items; "
          "memory-based admission into request slots")
SERVED_M, SERVED_K, SERVED_STEPS, SERVED_LR, SERVED_LAM = 3706, 16, 5, 0.005, 0.02
SERVED_RATES = (50.0, 100.0, 200.0, 500.0, 1000.0, 2000.0)


class ServedSetup:
    """The served context (keys, resident item factors) and a pool of distinct client requests
    encrypted once before any timing (client-side work): request i of a stream uses pool entry
    i mod P, so a stream of any length keeps the same nnz mix without holding one ciphertext set
    per request. The pool is also copied to page-locked host memory for the end-to-end runs."""

    def __init__(self, args, dev):
        import torch
        from paper_2509_03024_gb300 import capi
        from paper_2509_03024_gb300 import workloads as W
        self.torch, self.capi = torch, capi
        m, k = SERVED_M, SERVED_K
        self.ctx = ctx = capi.Context.from_preset(W.PRESETS["served"], device=dev)
        ctx.keygen(SEED, ctx.serve_rotation_steps(k))
        self.tuning = autotune(ctx, args)
        V = W.init_factors(m, k, SEED + 5)
        plan = capi.MfPlan(ctx, 1, m, k, [0, 1], [0], [1.0])  # item packing of the resident factors
        self.n_vb, self.B = plan.n_vb, plan.B
        self.VD = ctx.empty_ct(self.n_vb)
        plan.encrypt_factors(1, V, self.VD)
        self.stream = torch.cuda.Stream(device=dev)
        self.reqs = W.served_requests(args.served_pool, 100.0, m, k, SEED + 6)
        self.pool = []
        for i, r in enumerate(self.reqs):
            UR, R = ctx.empty_ct(1), ctx.empty_ct(self.n_vb)
            ctx.encrypt_request(m, k, r.u0, r.items, r.ratings, (1 << 44) + 64 * i, UR, R)
            self.pool.append((UR, R))
        torch.cuda.synchronize()
        self.take_buf = ctx.empty_ct(self.n_vb)
        self.host_pool = None
        self.host_take = None

    def host_buffers(self):
        torch = self.torch
        if self.host_pool is None:
            self.host_pool = [(UR.cpu().pin_memory(), R.cpu().pin_memory()) for UR, R in self.pool]
            self.host_take = torch.empty(self.take_buf.numel(), dtype=torch.int64).pin_memory()
        return self.host_pool, self.host_take

    def server(self, slots, budget=48 << 30):
        return self.capi.Server(self.ctx, self.VD, SERVED_M, SERVED_K, SERVED_STEPS, SERVED_LR, SERVED_LAM,
                                max_slots=slots, memory_budget_bytes=budget)


def arrival_times(count, rate, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serve_loop(st, server, arrivals, host=False):
    """Wall-clock request loop: admit arrived requests FIFO while slots are free, tick (each tick only
    enqueues its work), collect completed requests and download their predictions. Request i carries
    pool entry i mod P. With host=True the request ciphertexts are uploaded from page-locked host
    memory at admission and the predictions downloaded to host memory (end to end)."""
    import collections
    torch = st.torch
    pool, take = (st.host_buffers() if host else (st.pool, st.take_buf))
    P = len(pool)
    n = len(arrivals)
    queue = collections.deque()
    done_at = [None] * n
    nxt, inflight, ticks, finished = 0, 0, 0, 0
    nnz = 0
    stream = st.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    while finished < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            queue.append(nxt)
            nxt += 1
        while queue:
            i = queue[0]
            UR, R = pool[i % P]
            if not server.submit(i, st.reqs[i % P].items, UR, R, stream):
                break
            queue.popleft()
            inflight += 1
        if inflight:
            server.tick(stream)
            ticks += 1
            for rid in server.poll():
                server.take(rid, take, stream)
                done_at[rid] = time.perf_counter() - t0
                nnz += int(st.reqs[rid % P].items.size)
                inflight -= 1
                finished += 1
        elif nxt < n:
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    e1.record(stream)
    torch.cuda.synchronize()
    lat = (np.array(done_at) - arrivals) * 1e3
    span = max(done_at) - arrivals[0]
    out = {"requests": n, "ratings": nnz, "ratings_per_s": nnz / span, "requests_per_s": n / span,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "ticks": ticks, "wall_s": span,
           "device_span_ms": e0.elapsed_time(e1), "slots": server.n_slots}
    return out


def run_served(args, st):
    """Every arrival rate of the served workload: continuous batching against the same server with one
    slot (one request at a time), args.served_requests requests each. Returns (sweep, headline)."""
    rates = [float(x) for x in args.served_sweep.split(",")] if args.served_sweep else list(SERVED_RATES)
    sweep = []
    for r_i, rate in enumerate(rates):
        arr = arrival_times(args.served_requests, rate, SEED + 100 + r_i)
        sv = st.server(args.served_slots)
        batched = serve_loop(st, sv, arr)
        sv.close()
        one_sv = st.server(1)
        one = serve_loop(st, one_sv, arr)
        one_sv.close()
        sweep.append({"rate_req_s": rate, "continuous_batching": batched, "one_by_one": one,
                      "speedup_vs_one_by_one": batched["ratings_per_s"] / one["ratings_per_s"]})
    return sweep


def served_profile(args, st, rate):
    """One more batched run at `rate` with every launch timed by CUDA events (for the per-kernel
    roofline; its own throughput is not reported): ({class: (launches, device_ms, bytes, work)},
    the fraction of the run's device span covered by kernel time)."""
    arr = arrival_times(min(args.served_requests, 200), rate, SEED + 99)
    sv = st.server(args.served_slots)
    st.ctx.profile_begin(time_kernels=True)
    r = serve_loop(st, sv, arr)
    stats = st.ctx.profile_end()
    sv.close()
    busy = sum(v[1] for v in stats.values()) / max(r["device_span_ms"], 1e-9)
    return stats, busy


# ----------------------------------------------------------------------------- GPU arm

def job_throughput(elapsed_ms, ratings, steps, world, dist, device):
    """Whole-job rate: every rank processed `ratings` x `steps` (weak scaling, independent
    replicas); the job time is the slowest rank's (max over ranks). Returns (max ms, ratings/s)."""
    if dist is not None:
        import torch
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, world * ratings * steps / (elapsed_ms / 1e3)


def job_rate(ratings, seconds, dist, device):
    """Whole-job served rate: ratings summed over ranks / the slowest rank's wall time."""
    if dist is None:
        return ratings / seconds
    import torch
    t = torch.tensor([float(ratings), float(seconds)], dtype=torch.float64, device=device)
    r = t[:1].clone()
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    m = t[1:].clone()
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(r.item()) / float(m.item())


def init_dist(world, dev):
    import torch
    if world <= 1:
        return None
    import torch.distributed as dist_mod
    dist_mod.init_process_group("nccl", device_id=torch.device("cuda", dev))
    return dist_mod


def run_gpu(args, rank, world, local_rank):
    """The served workload (the headline), then the paper-scale training epoch as a sub-record."""
    import torch
    from paper_2509_03024_gb300 import build as B
    B.build()
    dev = local_rank
    torch.cuda.set_device(dev)
    dist = init_dist(world, dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.workload != "served":
        out = run_epoch(args, rank, world, dev, dist, barrier)
        if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "paper":
            out["cpu_baseline"] = cpu_baseline_epoch()
        if dist is not None:
            dist.destroy_process_group()
        return out

    st = ServedSetup(args, dev)
    for w in range(args.warmup):          # untimed: short bursts through a fresh server
        sv = st.server(args.served_slots)
        serve_loop(st, sv, arrival_times(16, SERVED_RATES[-1], SEED + 50 + w))
        sv.close()
    torch.cuda.synchronize()
    barrier()
    clk, clk_path = start_clocks(dev)
    torch.cuda.nvtx.range_push("served_timed")      # lets an ncu launch list select the timed region
    sweep = run_served(args, st)
    torch.cuda.nvtx.range_pop()
    clocks = stop_clocks(clk, clk_path)
    barrier()
    head = sweep[-1]
    hb = head["continuous_batching"]
    value = job_rate(hb["ratings"], hb["wall_s"], dist, f"cuda:{dev}")
    one_value = job_rate(head["one_by_one"]["ratings"], head["one_by_one"]["wall_s"], dist, f"cuda:{dev}")

    # end to end: the same request stream with the ciphertexts uploaded from page-locked host memory at
    # admission and the predictions downloaded to host memory, inside the timed loop
    e2e = None
    if args.e2e_requests > 0:
        sv = st.server(args.served_slots)
        r = serve_loop(st, sv, arrival_times(args.e2e_requests, head["rate_req_s"], SEED + 77), host=True)
        sv.close()
        ct_bytes = st.take_buf.numel() // st.n_vb * 8
        pool_up = sum((UR.numel() + R.numel()) * 8 for UR, R in st.pool) / len(st.pool)
        e2e = {"value": job_rate(r["ratings"], r["wall_s"], dist, f"cuda:{dev}"), "unit": UNIT,
               "h2d_bytes_per_step": int(pool_up), "d2h_bytes_per_step": int(st.n_vb * ct_bytes * 2 // (st.ctx.top + 1)),
               "step": "one request: its user and rating ciphertexts up, its prediction ciphertexts (limbs 0..1) down",
               "requests": r["requests"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "rate_req_s": head["rate_req_s"]}

    stats, busy = served_profile(args, st, head["rate_req_s"])
    ceil = int_ceilings(st.ctx)
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    roofline = roofline_of(stats, ceil, hbm_peak, peaks is not None, NCU_SERVED_FWD_DRAM_BYTES_PER_ROW, st.ctx.log_n)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": hb["wall_s"] * 1e3 / max(1, hb["ticks"]),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "p50_ms": hb["p50_ms"], "p99_ms": hb["p99_ms"],
           "one_by_one": {"value": one_value, "unit": UNIT, "p50_ms": head["one_by_one"]["p50_ms"],
                          "p99_ms": head["one_by_one"]["p99_ms"]},
           "speedup_vs_one_by_one": value / one_value,
           "config": {"workload": SERVED, "arrival_rate_req_s": head["rate_req_s"],
                      "requests_per_rate": args.served_requests, "distinct_requests": len(st.pool),
                      "slots": hb["slots"], "parallelism": "replicas",
                      "step": "one server tick (every admitted request advances one fold-in step or its "
                              "prediction); ms_per_step = wall time per tick of the headline run",
                      "steps_warmup": "warm-up = that many untimed 16-request bursts; the timed region is "
                                      "the request stream at every arrival rate",
                      "l2": "inputs larger than L2 (resident item factors 4 x 13 MiB, every request 65 MiB of "
                            "ciphertexts, evaluation keys 2.1 GB)",
                      "tuning": st.tuning},
           "roofline": roofline, "e2e": e2e, "gpu_launches": int(sum(v[0] for v in stats.values())),
           "gpu_launches_scope": "the profiled served run (" + str(min(args.served_requests, 200)) + " requests)",
           "clocks": clocks,
           "kernels": class_rooflines(stats, ceil, hbm_peak),
           "device_busy_fraction": busy,
           "int_pipe": ceil,
           "served": {"sweep": [{"rate_req_s": x["rate_req_s"],
                                 "continuous_batching": {k: x["continuous_batching"][k] for k in
                                                         ("ratings_per_s", "requests_per_s", "p50_ms", "p99_ms",
                                                          "mean_ms", "ticks", "wall_s", "device_span_ms",
                                                          "slots", "requests")},
                                 "one_by_one": {k: x["one_by_one"][k] for k in
                                                ("ratings_per_s", "requests_per_s", "p50_ms", "p99_ms", "mean_ms",
                                                 "ticks", "wall_s", "requests")},
                                 "speedup_vs_one_by_one": x["speedup_vs_one_by_one"]} for x in sweep]}}
    from paper_2509_03024_gb300 import comm
    per_req = [comm.served_request(st.ctx.n, st.ctx.top, st.n_vb, len(set((r.items // st.B).tolist())),
                                   SERVED_STEPS) for r in st.reqs]
    out["served"]["communication"] = {"mean_up_bytes": sum(x["up_bytes"] for x in per_req) / len(per_req),
                                      "down_bytes": per_req[0]["down_bytes"], "down_level": per_req[0]["out_level"]}
    del st
    if not args.no_epoch:
        out["epoch"] = run_epoch(args, rank, world, dev, dist, barrier, sub=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = served_cpu_baseline(rounds=1)
        except Exception as e:
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "kind": "oracle", "error": repr(e)}
    if dist is not None:
        dist.destroy_process_group()
    return out


def run_epoch(args, rank, world, dev, dist, barrier, sub=False):
    """The encrypted SGD epoch of the paper-scale (or large) workload: W warm-up epochs, K timed epochs
    from the same top-level factors; decrypted accuracy against FP64; per-class rooflines."""
    import torch
    from paper_2509_03024_gb300 import capi
    from paper_2509_03024_gb300.workloads import PRESETS
    wl = "paper" if args.workload == "served" else args.workload
    preset, k_rank, lr, desc = workload_spec(wl)
    train, test, U, V = workload(wl)
    ctx = capi.Context.from_preset(PRESETS[preset], device=dev)
    ctx.keygen(SEED + rank, ctx.mf_rotation_steps(k_rank))
    tuning = autotune(ctx, args)
    plan = capi.MfPlan(ctx, train.n, train.m, k_rank, train.row_ptr, train.col_idx, train.vals)
    U0, V0 = ctx.empty_ct(plan.n_ub), ctx.empty_ct(plan.n_vb)
    plan.encrypt_factors(0, U, U0)
    plan.encrypt_factors(1, V, V0)
    UD, VD = torch.empty_like(U0), torch.empty_like(V0)
    stream = torch.cuda.Stream(device=dev)
    ratings = train.nnz
    top = ctx.top
    steps = args.epoch_steps if sub else args.steps

    def step():
        with torch.cuda.stream(stream):
            UD.copy_(U0)
            VD.copy_(V0)
        plan.sgd_epoch(UD, VD, top, lr, LAM, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk, clk_path = (None, None) if sub else start_clocks(dev)
    ctx.profile_begin(time_kernels=not args.no_kernel_timing)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("epoch_timed")
    for _ in range(steps):
        step()
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    stats = ctx.profile_end()
    clocks = None if sub else stop_clocks(clk, clk_path)
    barrier()
    elapsed_ms, value = job_throughput(ev0.elapsed_time(ev1), ratings, steps, world, dist, f"cuda:{dev}")

    # decrypted accuracy of the last step against the FP64 epoch (sanity, not timed)
    from oracle import mf as omf
    rows, cols, vals = train.triples()
    U1, V1 = omf.mf_epoch_fp64(U, V, rows, cols, vals, lr, LAM)
    Ud = plan.decrypt_factors(0, UD, top - 2, train.n)
    Vd = plan.decrypt_factors(1, VD, top - 2, train.m)
    err = max(float(np.abs(Ud - U1).max()), float(np.abs(Vd - V1).max()))
    trow, tcol, tval = test.triples()
    rmse_gap = abs(omf.rmse(Ud, Vd, trow, tcol, tval) - omf.rmse(U1, V1, trow, tcol, tval))

    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(args, torch, dist, plan, U0, V0, UD, VD, stream, ratings, top, world, dev, barrier, lr)
    ceil = int_ceilings(ctx)
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    traffic_row = NCU_FWD_DRAM_BYTES_PER_ROW if wl == "paper" else None
    out = {"metric": METRIC if not sub else "encrypted MF training ratings/sec (one SGD epoch per step)",
           "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": desc, "ratings_per_step": ratings, "parallelism": "replicas",
                      "l2": "inputs larger than L2 (the rating ciphertexts alone are %.1f GiB)" % (
                          plan.info.n_bins * ctx.top * ctx.n * 8 / 2 ** 30),
                      "rating_bins": int(plan.info.n_bins),
                      "groups": int(plan.info.n_groups), "tree_nodes": int(plan.info.n_tree_nodes),
                      "plan_device_gib": plan.info.device_bytes / 2 ** 30, "tuning": tuning},
           "roofline": roofline_of(stats, ceil, hbm_peak, peaks is not None, traffic_row, ctx.log_n),
           "e2e": e2e, "gpu_launches": int(sum(v[0] for v in stats.values())),
           "accuracy": {"max_abs_vs_fp64": err, "rmse_gap_test": rmse_gap},
           "kernels": class_rooflines(stats, ceil, hbm_peak)}
    if clocks is not None:
        out["clocks"] = clocks
    from paper_2509_03024_gb300 import comm
    out["communication"] = {
        "training_10_epochs": comm.mf_training(ctx.n, ctx.top, ctx.alpha, len(ctx.mf_rotation_steps(k_rank)),
                                               int(plan.info.n_bins), plan.n_ub, plan.n_vb, epochs=10),
        "note": "bytes between the parties (key holder, data owners, recommender); the epochs themselves move "
                "nothing off the GPU"}
    del plan, ctx
    return out


def autotune(ctx, args):
    """Run the library's autotuner (untimed) unless --no-autotune; returns the chosen variant per
    kernel family and every variant's time, for the bench line."""
    if args.variants:
        for fv in args.variants.split(","):
            fam, var = fv.split("=")
            ctx.set_variant(fam.strip(), var.strip())
        return {"autotuned": False, "set": args.variants}
    if args.no_autotune:
        return {"autotuned": False}
    res = ctx.autotune()
    out = {"autotuned": True, "level": ctx.top - 1}
    for r in res:
        fam = out.setdefault(r["family"], {"chosen": None, "ms": {}})
        fam["ms"][r["variant"]] = round(r["ms"], 4)
        if r["chosen"]:
            fam["chosen"] = r["variant"]
    return out


def run_e2e(args, torch, dist, plan, U0, V0, UD, VD, stream, ratings, top, world, dev, barrier, lr):
    hU = torch.empty(U0.numel(), dtype=torch.int64, pin_memory=True)
    hV = torch.empty(V0.numel(), dtype=torch.int64, pin_memory=True)
    hU.copy_(U0.cpu())
    hV.copy_(V0.cpu())
    oU = torch.empty_like(hU, pin_memory=True)
    oV = torch.empty_like(hV, pin_memory=True)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            UD.copy_(hU, non_blocking=True)
            VD.copy_(hV, non_blocking=True)
        plan.sgd_epoch(UD, VD, top, lr, LAM, stream)
        with torch.cuda.stream(stream):
            oU.copy_(UD, non_blocking=True)
            oV.copy_(VD, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_value = job_throughput(e0.elapsed_time(e1), ratings, args.e2e_steps, world, dist, f"cuda:{dev}")
    bytes_h2d = (hU.numel() + hV.numel()) * 8
    return {"value": e2e_value, "unit": UNIT,
            "h2d_bytes_per_step": bytes_h2d, "d2h_bytes_per_step": bytes_h2d}


# the bound of each kernel class: the NTT passes (fused rescales and conversions included) and the
# key inner products run on the integer pipes, the element-wise classes stream HBM
CLASS_BOUND = {"ntt_forward": "alu", "ntt_inverse": "alu", "ks_inner": "alu", "tensor": "hbm",
               "elementwise": "hbm"}

# Minimum 32-bit multiply instructions (each a 32 x 32 (+ 64) -> 64-bit mad.wide or a 32-bit mad.lo on
# the integer multiply pipe) of one lazy Shoup butterfly on 64-bit residues: the high half of y ws (four
# partial products), the low halves of y w and of qhat q (one wide and two low products each) = 10; and
# of one 64 x 64 -> 128-bit multiply-accumulate: four partial products. Additions and carries run on the
# ALU pipe alongside.
BFLY_MIN_IMAD = 10
MAC_MIN_IMAD = 4


def int_ceilings(ctx):
    """Integer ceilings from the integer-pipe rates measured now on this GPU: butterflies/s = multiply
    issue rate / BFLY_MIN_IMAD, multiply-accumulates/s = rate / MAC_MIN_IMAD (the slower of mad.wide and
    mad.lo counts), with the register-only rate of this library's own butterfly code beside it."""
    r = ctx.probe_int_pipe(500)
    rate = min(r["imad_wide_gops"], r["imad_lo_gops"])
    return {"butterfly_gbfly": rate / BFLY_MIN_IMAD, "mac_gmacs": rate / MAC_MIN_IMAD,
            "probe_butterfly_gbfly": ctx.probe_butterfly_rate(2000), "rates_gops": r,
            "source": "fhe_probe_int_pipe: mad.lo / mad.hi / mad.wide.u32 issue rates on register operands "
                      "(152 SMs x 4 CTAs of 256 threads); ceilings = the mad rate / %d per butterfly and / %d "
                      "per 64 x 64 -> 128-bit multiply-accumulate" % (BFLY_MIN_IMAD, MAC_MIN_IMAD)}


def class_rooflines(stats, ceil, hbm_peak: float):
    """Per kernel class: launches, device time, algorithmic bytes, share of the device time, its
    algorithmic bytes/s against the HBM peak, and for the integer classes the arithmetic rate against
    the integer ceiling: butterflies/s (NTT classes) or multiply-accumulates/s (ks_inner).
    stats: {name: (launches, device_ms, bytes, work)}."""
    total = sum(v[1] for v in stats.values()) or 1.0
    out = {}
    for name, v in stats.items():
        launches, dev_ms, alg_bytes = v[0], v[1], v[2]
        work = v[3] if len(v) > 3 else 0.0
        if not launches:
            continue
        rec = {"launches": launches, "device_ms": round(dev_ms, 3), "alg_gb": round(alg_bytes / 1e9, 3),
               "share": dev_ms / total, "bound": CLASS_BOUND.get(name, "hbm")}
        if dev_ms > 0:
            secs = dev_ms / 1e3
            gbs = alg_bytes / secs / 1e9
            rec["hbm_view"] = {"achieved_gbs": gbs, "frac": gbs / hbm_peak}
            if ceil and work > 0 and name.startswith("ntt"):
                g = work / secs / 1e9
                rec["alu"] = {"achieved_gbfly": g, "frac": g / ceil["butterfly_gbfly"],
                              "frac_of_probe": g / ceil["probe_butterfly_gbfly"]}
            elif ceil and work > 0 and name == "ks_inner":
                g = work / secs / 1e9
                rec["alu"] = {"achieved_gmacs": g, "frac": g / ceil["mac_gmacs"]}
        out[name] = rec
    return out


def roofline_of(stats, ceil, hbm_peak, measured, traffic_per_row, log_n):
    """The bench line's roofline object for the dominant kernel class (longest summed device time)."""
    name, v = max(stats.items(), key=lambda kv: kv[1][1])
    launches, dev_ms, alg_bytes, work = v[0], v[1], v[2], (v[3] if len(v) > 3 else 0.0)
    avg_s = (dev_ms / launches) / 1e3
    hbm_achieved = (alg_bytes / launches) / avg_s / 1e9
    hbm_view = {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if measured else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": alg_bytes / launches}
    rows_per_launch = (alg_bytes / launches) / (16.0 * 2 ** log_n)
    base = {"kernel": name, "launches": launches, "avg_launch_us": avg_s * 1e6,
            "share_of_timed_device_time": dev_ms / sum(x[1] for x in stats.values())}
    if name.startswith("ntt") and work > 0:
        achieved = (work / launches) / avg_s / 1e9
        traffic = traffic_per_row * rows_per_launch if (traffic_per_row and name == "ntt_forward") else None
        return {"bound": "alu", "achieved": achieved, "peak": ceil["butterfly_gbfly"], "unit": "Gbfly/s",
                "frac": achieved / ceil["butterfly_gbfly"], "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read+write per limb row of this workload's forward passes, "
                                  "scaled by the rows of the average launch" if traffic else None,
                "peak_source": ceil["source"],
                "probe_peak": {"value": ceil["probe_butterfly_gbfly"], "frac": achieved / ceil["probe_butterfly_gbfly"],
                               "source": "fhe_probe_butterfly_rate: this library's lazy Shoup butterfly code on "
                                         "register-resident values (no memory traffic)"},
                "butterflies_per_launch": work / launches, "hbm_view": hbm_view, **base}
    if name == "ks_inner" and work > 0:
        achieved = (work / launches) / avg_s / 1e9
        return {"bound": "alu", "achieved": achieved, "peak": ceil["mac_gmacs"], "unit": "GMAC/s",
                "frac": achieved / ceil["mac_gmacs"], "traffic": None, "peak_source": ceil["source"],
                "macs_per_launch": work / launches, "hbm_view": hbm_view, **base}
    return {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": hbm_achieved / hbm_peak, "traffic": None, "peak_source": hbm_view["peak_source"],
            "alg_bytes_per_launch": alg_bytes / launches, **base}


def cpu_baseline_epoch():
    """The epoch workload's oracle baseline: every available core, with one core alone beside it."""
    try:
        return oracle_baseline()
    except Exception as e:   # the worker pool failed: the single-thread sample in this process
        train, _, U, V = workload()
        rps, secs, desc = oracle_sample(train, U, V)
        return {"value": rps, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                "measured_s": round(secs, 1), "all_cores_error": repr(e)}


# ----------------------------------------------------------------------------- served CPU baseline

# Operations of a served request, as the oracle runs them (oracle/serve.py), timed at the top level:
#   ip     one item batch's inner products: mul_relin_rescale(UR, V_c) then the hoisted rotate-and-sum
#   mask   E = R_c - S, MV = rescale(V_c (.) mask), E (x) MV
#   relin  relin_rescale of the summed three-component tensor
#   rot    one block-sum rotation and its addition
#   reg    the regulariser: constant product, rescale, addition
SERVED_OPS = ("ip", "mask", "relin", "rot", "reg")


def _served_oracle_worker(index, cmd, res):
    try:
        from oracle import ckks, mf, serve
        from paper_2509_03024_gb300 import workloads as W
        he = ckks.Ckks(ckks.Params.from_preset(W.PRESETS["served"]))
        k = SERVED_K
        kp, w, B = serve.layout(k, he.prm.slots)
        he.keygen(SEED, mf.rotsum_steps(kp) + [w, -kp])
        top = he.prm.top
        z = np.zeros(he.prm.slots)
        z[: 4 * w] = 0.25                       # sparse slot vectors: fast to encode, full-size ciphertexts
        UR = he.encrypt(z, top, 1)
        Vc = he.encrypt(z, top, 2)
        Rc = he.encrypt(z, top, 3)
        mask = he.enc.encode(z)
        t3 = he.tensor(UR, Vc)
        res.put(("ready", index, None))

        def timed(op):
            t0 = time.perf_counter()
            if op == "ip":
                mf.block_sum(he, he.mul_relin_rescale(UR, Vc), kp)
            elif op == "mask":
                S = he.drop(Rc, top - 1)
                E = he.sub(he.drop(Rc, top - 1), S)
                MV = he.rescale(he.mul_plain(Vc, mask))
                he.tensor(E, MV)
            elif op == "relin":
                he.relin_rescale(t3)
            elif op == "rot":
                G = he.drop(UR, top - 2)
                he.add(G, he.rotate(G, w))
            else:
                base = he.rescale(serve.const_mul(he, UR, 0.99))
                he.add(he.drop(base, top - 2), he.drop(UR, top - 2))
            return time.perf_counter() - t0

        while True:
            c = cmd.get()
            if c == "stop":
                break
            res.put(("time", index, {op: timed(op) for op in c}))
    except Exception as e:
        res.put(("error", index, repr(e)))


class ServedOracleCores:
    """Single-threaded oracle processes (spawned), one per core, each with its own served-ring context
    and keys; a round times every served operation on every process at once."""

    def __init__(self, n_workers, timeout_s=1800.0):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.n, self.timeout = n_workers, timeout_s
        self.cmds = [ctx.Queue() for _ in range(n_workers)]
        self.res = ctx.Queue()
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({v: "1" for v in saved})
        try:
            self.procs = [ctx.Process(target=_served_oracle_worker, args=(i, self.cmds[i], self.res), daemon=True)
                          for i in range(n_workers)]
            for p in self.procs:
                p.start()
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        self._collect(n_workers)

    def _collect(self, count):
        out = {}
        while len(out) < count:
            kind, i, v = self.res.get(timeout=self.timeout)
            if kind == "error":
                raise RuntimeError(f"oracle worker {i}: {v}")
            out[i] = v
        return out

    def round(self):
        """Every worker times every operation, all workers at once: {op: mean seconds}."""
        for q in self.cmds:
            q.put(SERVED_OPS)
        times = self._collect(self.n)
        return {op: statistics.mean(t[op] for t in times.values()) for op in SERVED_OPS}

    def close(self):
        for q in self.cmds:
            q.put("stop")
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)


def served_request_seconds(op_s, nnz_batches, top, n_vb, B, steps=SERVED_STEPS, alpha=3):
    """Oracle seconds of one served request, from the top-level operation times: step s runs at level
    l = top - 2 s (every rated batch: ip + mask; then relin at l - 1, log2(B) + 1 rotations at l - 2 and
    the regulariser at l), the prediction runs ip on every batch at top - 2 steps; an operation at level
    l is taken to cost its top-level time scaled by the extended limbs (l + 1 + alpha) / (top + 1 + alpha)."""
    def at(op, lv):
        return op_s[op] * (lv + 1 + alpha) / (top + 1 + alpha)
    beta = int(math.log2(B))
    total = 0.0
    for s in range(steps):
        lv = top - 2 * s
        total += nnz_batches * (at("ip", lv) + at("mask", lv)) + at("relin", lv - 1)
        total += (beta + 1) * at("rot", lv - 2) + at("reg", lv)
    total += n_vb * at("ip", top - 2 * steps)
    return total


def served_cpu_rate(op_s, cores):
    """Ratings/s of the served request mix on `cores` independent single-threaded oracle processes."""
    from paper_2509_03024_gb300 import workloads as W
    reqs = W.served_requests(256, 100.0, SERVED_M, SERVED_K, SEED + 6)
    top, B = len(W.PRESETS["served"].data_bits) - 1, (1 << 15) // (2 * SERVED_K)
    n_vb = -(-SERVED_M // B)
    secs = sum(served_request_seconds(op_s, len(set((r.items // B).tolist())), top, n_vb, B) for r in reqs)
    nnz = sum(int(r.items.size) for r in reqs)
    return nnz / secs * cores, secs / len(reqs)


def served_cpu_baseline(rounds=1, budget_s=None):
    t0 = time.perf_counter()
    pool = ServedOracleCores(oracle_workers(bytes_per_worker=2.5 * 2**30))
    setup_s = time.perf_counter() - t0
    vals = []
    try:
        while True:
            op_s = pool.round()
            rate, per_req = served_cpu_rate(op_s, pool.n)
            vals.append((rate, per_req, op_s))
            if len(vals) >= rounds or (budget_s is not None and time.perf_counter() - t0 > budget_s):
                break
    finally:
        pool.close()
    vals.sort(key=lambda v: v[0])
    rate, per_req, op_s = vals[(len(vals) - 1) // 2]
    desc = (f"{pool.n} single-threaded oracle processes at once on the served ring (N=2^16, 13+3 primes), each "
            f"timing every operation of a served request at the top level ({', '.join(f'{k} {v:.2f} s' for k, v in op_s.items())}); "
            f"per-request seconds extrapolated over the 5 fold-in steps and the prediction with the level's limb "
            f"count (mean {per_req:.0f} s per request over 256 requests of the served mix); rate = ratings / "
            f"request seconds x {pool.n} processes; extrapolated, {len(vals)} round(s)")
    return {"value": rate, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": desc,
            "rounds": len(vals), "setup_s": round(setup_s, 1), "measured_s": round(time.perf_counter() - t0, 1)}


def run_reference(args, rank, world):
    """The oracle (CPU, as it stands) on the served workload and metric; rank 0 only. The W warm-up
    steps are not repeated on the CPU (nothing there warms up); timed rounds run until K are done or
    about three minutes have passed, whichever comes first."""
    if rank != 0:
        return None
    if args.workload != "served":
        return run_reference_epoch(args)
    cb = served_cpu_baseline(rounds=max(1, args.steps), budget_s=180.0)
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world,
            "steps": cb["rounds"], "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": SERVED, "arrival_rate_req_s": SERVED_RATES[-1]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_epoch(args):
    """The oracle (CPU, as it stands) on the epoch workload; extrapolated from sampled groups."""
    pool = OracleCores(oracle_workers())
    vals, per_step = [], []
    try:
        for i in range(args.warmup + args.steps):
            rps, tg, tr, est = pool.rate(pool.sample(range(pool.n)))
            if i >= args.warmup:
                vals.append(rps)
                per_step.append((tg, tr, est))
    finally:
        pool.close()
    v = statistics.median_low(vals)
    tg, tr, est = per_step[vals.index(v)]
    desc = (f"each step: {pool.n} single-threaded oracle processes at once at N=2^15, each on its own group "
            f"(of {pool.info['groups']}) and one rotation; epoch extrapolated as (groups x {tg:.2f} s + "
            f"{3 * pool.info['nodes']} rotation-sized key switches x {tr:.2f} s) / {pool.n} = {est:.0f} s; "
            f"value = median over the timed steps")
    return {"impl": "reference", "metric": "encrypted MF training ratings/sec", "value": v, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batched":
        out = run_batched(args) if rank == 0 else None
    else:
        out = run_gpu(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
