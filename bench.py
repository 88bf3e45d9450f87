#!/usr/bin/env python
"""Throughput of the encrypted CSR matrix-factorisation epoch on one GB300.

Workload (the paper-scale configuration): 943 users x 1682 items with 100,000
synthetic ratings shaped like MovieLens-100K (Zipf(1.0) item popularity, >= 20
ratings per user, MovieLens rating law), a 10 % held-out split, rank k = 10;
RNS-CKKS with N = 2^15, eight 50-bit data primes, two 60-bit special primes,
scale 2^50. One step = one encrypted SGD epoch (lr 0.005, lambda 0.02) over the
90 % training split, starting from top-level encrypted factors (restored from a
resident copy at the start of each step; the chain holds three epochs).

Metric: training ratings processed per second (whole job over all ranks).
Multi-GPU runs are independent replicas (one per rank, weak scaling). The same
line carries the served section (continuous batching of fold-in + predict
requests against one-at-a-time execution, p50/p99 latency), the roofline of
the dominant kernel class, the end-to-end rate with host copies, the
communication report and the oracle's CPU rate (all host cores, and one core alone).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload paper|large|batched] [--served-rate R] [--served-sweep R1,R2,...]
"""
from __future__ import annotations

import argparse
import json
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
# nominal integer-issue ceiling of the NTT butterfly, reported beside the measured one: 152 SMs x 4
# schedulers x 32 lanes x 2.07 GHz issue slots at 20 32-bit instructions per lazy 64-bit Shoup
# butterfly (product high half 5, two low halves 6, subtraction 2, range reduction 4, sum and
# difference 3), assuming full issue
ALU_PEAK_GBFLY = 152 * 128 * 2.07 / 20.0
# DRAM bytes per limb row of a forward NTT pass at N = 2^15, from the ncu capture (dram__bytes_read
# + write) of the fused ModUp passes of the current kernels (64 rotations at level 7, 2048 rows per
# pass): (615 MB + 1020 MB) / 2 passes / 2048 rows
NCU_FWD_DRAM_BYTES_PER_ROW = (615.0e6 + 1020.0e6) / 2 / 2048
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
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-requests", type=int, default=96)
    ap.add_argument("--served-rate", type=float, default=100.0)
    ap.add_argument("--served-slots", type=int, default=48)
    ap.add_argument("--served-sweep", default="", help="comma-separated arrival rates (req/s) to sweep")
    ap.add_argument("--workload", choices=["paper", "large", "batched"], default="paper",
                    help="paper: the headline paper-scale epoch; large: the 6040 x 3706 workload at N=2^16; "
                         "batched: independent instances one after another")
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
            "accuracy": {"max_abs_vs_fp64": max_err}, "wall_s": time.perf_counter() - wall0}


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
          "3x60-bit primes); Poisson arrivals; per request one user's encrypted CSR row (nnz log-uniform "
          "5..300, MovieLens rating law), 5 encrypted SGD fold-in steps (lr 0.005, lambda 0.02) then the "
          "encrypted predicted-rating row over all items")


def serve_loop(server, reqs, enc, take_buf):
    """Wall-clock request loop: admit arrived requests FIFO while slots are free, tick, collect."""
    import collections
    queue = collections.deque()
    arrivals = [r.arrival_s for r in reqs]
    done_at = [None] * len(reqs)
    nxt = 0
    t0 = time.perf_counter()
    inflight = 0
    ticks = 0
    while any(d is None for d in done_at):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            queue.append(nxt)
            nxt += 1
        while queue and server.submit(queue[0], reqs[queue[0]].items, *enc[queue[0]]):
            queue.popleft()
            inflight += 1
        if inflight:
            server.tick()
            ticks += 1
            now = time.perf_counter() - t0
            for rid in server.poll():
                server.take(rid, take_buf)
                done_at[rid] = now
                inflight -= 1
        elif nxt < len(reqs):
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    lat = np.array([d - a for d, a in zip(done_at, arrivals)]) * 1e3
    span = max(done_at) - arrivals[0]
    nnz = sum(int(r.items.size) for r in reqs)
    return {"ratings_per_s": nnz / span, "requests_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "ticks": ticks,
            "wall_s": span}


def run_served(args, dev):
    """Served fold-in + predict at --served-rate (and at every rate of --served-sweep): continuous
    batching against the same server with one slot (one request at a time)."""
    import torch
    from paper_2509_03024_gb300 import capi
    from paper_2509_03024_gb300 import workloads as W
    m, k, steps, lr, lam = 3706, 16, 5, 0.005, 0.02
    ctx = capi.Context.from_preset(W.PRESETS["served"], device=dev)
    ctx.keygen(SEED, ctx.serve_rotation_steps(k))
    V = W.init_factors(m, k, SEED + 5)
    plan = capi.MfPlan(ctx, 1, m, k, [0, 1], [0], [1.0])  # item packing of the resident factors
    n_vb = plan.n_vb
    VD = ctx.empty_ct(n_vb)
    plan.encrypt_factors(1, V, VD)
    take_buf = ctx.empty_ct(n_vb)

    def at_rate(rate):
        reqs = W.served_requests(args.served_requests, rate, m, k, SEED + 6)
        enc = []
        for i, r in enumerate(reqs):  # client-side encryption, before the timed loop
            UR, R = ctx.empty_ct(1), ctx.empty_ct(n_vb)
            ctx.encrypt_request(m, k, r.u0, r.items, r.ratings, (1 << 44) + 64 * i, UR, R)
            enc.append((UR, R))
        server = capi.Server(ctx, VD, m, k, steps, lr, lam, max_slots=args.served_slots,
                             memory_budget_bytes=48 << 30)
        batched = serve_loop(server, reqs, enc, take_buf)
        batched["slots"] = server.n_slots
        server.close()
        single = capi.Server(ctx, VD, m, k, steps, lr, lam, max_slots=1)
        one = serve_loop(single, reqs, enc, take_buf)
        single.close()
        return len(reqs), batched, one

    n, batched, one = at_rate(args.served_rate)
    from paper_2509_03024_gb300 import comm
    B = plan.B
    reqs = W.served_requests(args.served_requests, args.served_rate, m, k, SEED + 6)
    per_req = [comm.served_request(ctx.n, ctx.top, n_vb, len(set((r.items // B).tolist())), steps) for r in reqs]
    out_comm = {"mean_up_bytes": sum(x["up_bytes"] for x in per_req) / len(per_req),
                "down_bytes": per_req[0]["down_bytes"], "down_level": per_req[0]["out_level"]}
    out = {"workload": SERVED, "requests": n, "arrival_rate_req_s": args.served_rate, "communication": out_comm,
           "value": batched["ratings_per_s"], "unit": UNIT, "p50_ms": batched["p50_ms"],
           "p99_ms": batched["p99_ms"], "continuous_batching": batched, "one_by_one": one,
           "speedup_vs_one_by_one": batched["ratings_per_s"] / one["ratings_per_s"]}
    if args.served_sweep:
        sweep = []
        for rate in (float(x) for x in args.served_sweep.split(",")):
            _, b, o = at_rate(rate)
            sweep.append({"rate_req_s": rate,
                          "batched": {k2: b[k2] for k2 in ("ratings_per_s", "p50_ms", "p99_ms")},
                          "one_by_one": {k2: o[k2] for k2 in ("ratings_per_s", "p50_ms", "p99_ms")}})
        out["sweep"] = sweep
    return out


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


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2509_03024_gb300 import build as B
    B.build()
    from paper_2509_03024_gb300 import capi
    from paper_2509_03024_gb300.workloads import PRESETS

    dev = local_rank
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", dev))
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    preset, k_rank, lr, _ = workload_spec(args.workload)
    train, test, U, V = workload(args.workload)
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
    clk, clk_path = start_clocks(dev)
    ctx.profile_begin(time_kernels=not args.no_kernel_timing)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    stats = ctx.profile_end()
    clocks = stop_clocks(clk, clk_path)
    barrier()
    elapsed_ms, value = job_throughput(ev0.elapsed_time(ev1), ratings, args.steps, world, dist, f"cuda:{dev}")

    # decrypted accuracy of the last step against the FP64 epoch (sanity, not timed)
    from oracle import mf as omf
    rows, cols, vals = train.triples()
    U1, V1 = omf.mf_epoch_fp64(U, V, rows, cols, vals, lr, LAM)
    Ud = plan.decrypt_factors(0, UD, top - 2, train.n)
    Vd = plan.decrypt_factors(1, VD, top - 2, train.m)
    err = max(float(np.abs(Ud - U1).max()), float(np.abs(Vd - V1).max()))
    trow, tcol, tval = test.triples()
    rmse_gap = abs(omf.rmse(Ud, Vd, trow, tcol, tval) - omf.rmse(U1, V1, trow, tcol, tval))

    # end to end through the C ABI with host buffers: H2D of the encrypted factors, epoch, D2H
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(args, torch, dist, plan, U0, V0, UD, VD, stream, ratings, top, world, dev, barrier, lr)
    out = finish(args, ctx, plan, stats, clocks, elapsed_ms, value, ratings, world, rank, e2e, err, rmse_gap,
                 train, U, V, dist)
    out["config"]["tuning"] = tuning
    return out


def autotune(ctx, args):
    """Run the library's autotuner (untimed) unless --no-autotune; returns the chosen variant per
    kernel family and every variant's time, for the bench line."""
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


def torch_device_of(ctx):
    return ctx.device


# the bound of each kernel class: the NTT passes (fused rescales and conversions included) and the
# key inner products run on the integer pipes, the element-wise classes stream HBM
CLASS_BOUND = {"ntt_forward": "alu", "ntt_inverse": "alu", "ks_inner": "alu", "tensor": "hbm",
               "elementwise": "hbm"}


def butterflies_per_residue_pass(log_n: int) -> float:
    """Butterflies per residue in one NTT pass: rings up to 2^13 run the log2(N) stages in one pass,
    larger rings split them over two passes; a stage does N/2 butterflies."""
    passes = 1 if log_n <= 13 else 2
    return log_n / passes / 2.0


def class_rooflines(stats, log_n: int, bfly_peak, hbm_peak: float):
    """Per kernel class: launches, device time, algorithmic bytes, share of the device time and the
    achieved fraction of the class's roofline: for NTT classes butterflies/s against the measured
    butterfly rate (each pass reads and writes 16 bytes per residue), and for every class its
    algorithmic bytes/s against the HBM peak. stats: {name: (launches, device_ms, bytes)}."""
    total = sum(v[1] for v in stats.values()) or 1.0
    out = {}
    for name, (launches, dev_ms, alg_bytes) in stats.items():
        if not launches:
            continue
        rec = {"launches": launches, "device_ms": round(dev_ms, 3), "alg_gb": round(alg_bytes / 1e9, 3),
               "share": dev_ms / total, "bound": CLASS_BOUND.get(name, "hbm")}
        if dev_ms > 0:
            secs = dev_ms / 1e3
            gbs = alg_bytes / secs / 1e9
            rec["hbm_view"] = {"achieved_gbs": gbs, "frac": gbs / hbm_peak}
            if name.startswith("ntt") and bfly_peak:
                gbfly = alg_bytes / 16.0 * butterflies_per_residue_pass(log_n) / secs / 1e9
                rec["alu"] = {"achieved_gbfly": gbfly, "frac": gbfly / bfly_peak}
        out[name] = rec
    return out


def finish(args, ctx, plan, stats, clocks, elapsed_ms, value, ratings, world, rank, e2e, err, rmse_gap,
           train, U, V, dist):
    # roofline of the dominant kernel class (longest summed device time)
    peaks = measured_peaks()
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    name, (launches, dev_ms, alg_bytes) = dom
    avg_s = (dev_ms / launches) / 1e3
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    hbm_achieved = (alg_bytes / launches) / avg_s / 1e9
    hbm_view = {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": alg_bytes / launches}
    # the butterfly rate on register-resident values, measured now on this GPU: the NTT classes' peak
    bfly_peak = (ctx.probe_butterfly_rate(2000)
                 if any(k.startswith("ntt") and v[0] for k, v in stats.items()) else None)
    if name.startswith("ntt"):
        # one NTT pass sweeps every row once (16 bytes per residue)
        log_n = ctx.log_n
        bfly = (alg_bytes / launches) / 16.0 * butterflies_per_residue_pass(log_n)
        achieved = bfly / avg_s / 1e9
        rows_per_launch = (alg_bytes / launches) / (16.0 * 2 ** log_n)
        traffic = (NCU_FWD_DRAM_BYTES_PER_ROW * rows_per_launch
                   if name == "ntt_forward" and args.workload == "paper" else None)
        peak = bfly_peak
        roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "Gbfly/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "traffic_source": "ncu dram__bytes_read+write per row of the fused forward passes, scaled "
                                      "by the rows of the average launch",
                    "peak_source": ("measured by fhe_probe_butterfly_rate: the forward transform's lazy Shoup "
                                    "butterflies on register-resident values (no shared-memory, twiddle or HBM "
                                    "traffic), 152 SMs x 3 CTAs of 256 threads"),
                    "nominal_peak": {"value": ALU_PEAK_GBFLY, "frac": achieved / ALU_PEAK_GBFLY,
                                     "source": "152 SMs x 128 lanes x 2.07 GHz / 20 32-bit instructions per "
                                               "butterfly at full issue (not reached: the probe issues 23.8 "
                                               "instructions per butterfly at 53 % issue)"},
                    "launches": launches, "avg_launch_us": avg_s * 1e6, "butterflies_per_launch": bfly,
                    "hbm_view": hbm_view}
    else:
        roofline = {"bound": "hbm", "kernel": name, "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": None, "peak_source": hbm_view["peak_source"],
                    "launches": launches, "avg_launch_us": avg_s * 1e6,
                    "alg_bytes_per_launch": alg_bytes / launches}
    roofline["share_of_timed_device_time"] = dev_ms / sum(v[1] for v in stats.values())
    gpu_launches = sum(v[0] for v in stats.values())

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": workload_spec(args.workload)[3], "ratings_per_step": ratings, "parallelism": "replicas",
                      "l2": "inputs larger than L2 (the rating ciphertexts alone are %.1f GiB)" % (
                          plan.info.n_bins * ctx.top * ctx.n * 8 / 2 ** 30),
                      "rating_bins": int(plan.info.n_bins),
                      "groups": int(plan.info.n_groups), "tree_nodes": int(plan.info.n_tree_nodes),
                      "plan_device_gib": plan.info.device_bytes / 2 ** 30},
           "roofline": roofline, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
           "accuracy": {"max_abs_vs_fp64": err, "rmse_gap_test": rmse_gap},
           "kernels": class_rooflines(stats, ctx.log_n, bfly_peak, hbm_peak)}
    from paper_2509_03024_gb300 import comm
    out["communication"] = {
        "training_10_epochs": comm.mf_training(ctx.n, ctx.top, ctx.alpha,
                                               len(ctx.mf_rotation_steps(workload_spec(args.workload)[1])),
                                               int(plan.info.n_bins), plan.n_ub, plan.n_vb, epochs=10),
        "note": "bytes between the parties (key holder, data owners, recommender) for the paper-scale workload; "
                "the epochs themselves move nothing off the GPU"}
    if not args.no_served:
        out["served"] = run_served(args, torch_device_of(ctx))
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "paper":
        try:
            out["cpu_baseline"] = oracle_baseline()
        except Exception as e:   # the worker pool failed: the single-thread sample in this process
            rps, secs, desc = oracle_sample(train, U, V)
            out["cpu_baseline"] = {"value": rps, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                   "measured_s": round(secs, 1), "all_cores_error": repr(e)}
    if dist is not None:
        dist.destroy_process_group()
    return out


def run_reference(args, rank, world):
    """The oracle (CPU, as it stands) on the same workload and metric; rank 0 only."""
    if rank != 0:
        return None
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
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
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
