#!/usr/bin/env python
"""Benchmark of the RLT2 dual ascent on GB300: passes (iterations) per second.

One step = one pass of the loop of Algorithm 1 (fused spread/complementary pass
over D, N^2 (N-1)^2 D->C Hungarian LAPs, complementary C + C->B, B->LB) on the
30-facility clustered workload (the paper's QAPLIB shapes stand-in; synthetic
data).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank bounds its own replica of
the workload (independent instances, no collective on the data path): weak
scaling; the reported value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RLT2 dual-ascent iters/sec at N=30"
OPS_PER_RELAXATION = 9   # textbook int ops of one relaxation: 2 subtractions, compare with the
                         # label, its 2 conditional updates, compare with the minimum, its 2
                         # conditional updates, the label decrement
ALU_LANES_PER_SM = 64    # integer ALU pipe: 16 lanes per scheduler, 4 schedulers
# DRAM bytes per launch of the D->C and fused-pass kernels on the 30-facility
# workload (tile store), from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum;
# reported only while the kernel's sources hash to the captured version.
DLAP_TRAFFIC = {"workload": "clustered_n30", "bytes": 2713529600 + 2654458624,
                "files": ("lap_kernels.cu", "device.cuh", "kernels.h"),
                "sources_sha1": "eed19020147e72a9c5d3269774b4da331ab575e7"}
P1_TRAFFIC = {"workload": "clustered_n30", "bytes": 2741044736 + 2655430400,
              "files": ("sweep_kernels.cu", "device.cuh", "kernels.h"),
              "sources_sha1": "7effb6ceb3bb7a07c31ea1e7936c36abb2fcd5ea"}


def captured_traffic(rec, workload, store):
    """rec["bytes"] if the workload and the kernel sources match the capture."""
    if workload != rec["workload"] or store != "tiles":
        return None
    import hashlib
    h = hashlib.sha1()
    for f in rec["files"]:
        with open(os.path.join(ROOT, "paper_1510_02065_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest() == rec["sources_sha1"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered_n30")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work for the cpu_baseline sample (0: skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-nodes", type=int, default=256,
                    help="B&B nodes of the batched-bounding measurement (0: skip)")
    ap.add_argument("--batch-iters", type=int, default=100)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests of the serving measurement (0: skip)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="lanes per D->C LAP (4, 8, 16, 32); 0: autotuned")
    ap.add_argument("--cta-warps", type=int, default=0, help="warps per D->C CTA; 0: chosen")
    ap.add_argument("--store", default="tiles", choices=["tiles", "classes"],
                    help="store of D for the headline run (results are identical)")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="passes of the FP64 form timed on the workload (0: skip)")
    ap.add_argument("--n35-steps", type=int, default=30,
                    help="timed passes of the 35-facility root bound (0: skip)")
    return ap.parse_args()


def serve_measure(instances, torch, count, passes=50, rate=50.0):
    """Continuous-batching server on a Poisson stream of bound requests.

    Arrivals: Poisson (rate/s, exponential gaps from default_rng(7)); request r
    is the clustered instance of size N_r uniform in [12, 30] with seed r, 50
    passes.  Admission by device memory (budget 64 GB).  If the measured
    throughput is below the offered rate (saturation), the stream is served
    again at 0.8x the measured capacity (its first min(count, 500) requests)
    and both runs are reported.
    """
    from paper_1510_02065_gb300.serve import BoundServer, Request

    def run(r, count):
        arr, Ns = instances.poisson_requests(count, rate=r)
        reqs = []
        for rid in range(count):
            F, D = instances.clustered_euclid(int(Ns[rid]), seed=rid)
            reqs.append(Request(rid=rid, F=F, D=D, iters=passes, arrival=float(arr[rid])))
        s = torch.cuda.Stream()
        srv = BoundServer(mem_budget=64 << 30, max_slots=64, passes_per_round=5, stream=s.cuda_stream)
        st = srv.serve(reqs, realtime=True)
        st["offered_rate"] = r
        return st

    first = run(rate, count)
    out = {"metric": "served RLT2 bound requests", "unit": "requests/s", "passes": passes,
           "N_range": [12, 30], "offered": first}
    if first["throughput"] is not None and first["throughput"] < 0.95 * rate:
        out["at_0.8_capacity"] = run(0.8 * first["throughput"], min(count, 500))
    return out


def n35_measure(rlt2, instances, torch, steps, store, warmup=3, workload="clustered_n35"):
    """Root bound of one clustered instance (the 35-facility one by default)."""
    F, D, _ = instances.instance(workload)
    N = F.shape[0]
    s = torch.cuda.Stream()
    with rlt2.Context(F, D, profile=True, max_iters=steps + warmup + 1, stream=s.cuda_stream,
                      store=store) as c:
        c.iterate(warmup)
        torch.cuda.synchronize()
        rlt2.rlt2_reset_stage_times(c.ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        c.iterate(steps)
        e1.record(s)
        torch.cuda.synchronize()
        ms, n = c.stage_times()
        lb = c.bound()[1]
    t = e0.elapsed_time(e1)
    return {"metric": "RLT2 dual-ascent iters/sec at N=%d" % N, "unit": "iters/s",
            "value": steps / (t / 1000.0), "steps": steps, "LB": lb,
            "stages_ms": {"spread_complementary_D": ms[0] / n, "concentrate_D_to_C": ms[1] / n,
                          "complementary_C_concentrate_C_to_B": ms[2] / n,
                          "concentrate_B_to_LB": ms[3] / n},
            "store": "%s (%.2f GB on the device)" % (
                {rlt2.RLT2_STORE_CLASSES: "class sums", rlt2.RLT2_STORE_PAIRS: "pairs (Sec. 6)"}.get(store, "tiles"),
                rlt2.rlt2_state_bytes(N, store=store) / 1e9)}


# DRAM bytes of one f64_dlap_kernel launch at N=20 (one ncu capture of the DRAM byte counters)
# per tile coefficient read (n x N per tile) and written (n x n), valid while
# the FP64 sources hash to the captured version; other sizes scale by those units
F64_DLAP_TRAFFIC = {"N": 20, "read": 417091840, "write": 358182400, "files": ("f64.cu", "device.cuh"),
                    "sources_sha1": "852ad019743ca0a1dda6930a9a37adf640d44899"}


def f64_traffic(N):
    import hashlib
    rec = F64_DLAP_TRAFFIC
    h = hashlib.sha1()
    for f in rec["files"]:
        with open(os.path.join(ROOT, "paper_1510_02065_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sources_sha1"]:
        return None
    M = rec["N"]
    tiles = lambda K: K * K * (K - 1) ** 2
    rd = rec["read"] / (tiles(M) * (M - 2) * M) * tiles(N) * (N - 2) * N
    wr = rec["write"] / (tiles(M) * (M - 2) ** 2) * tiles(N) * (N - 2) ** 2
    return int(rd + wr)


def fp64_measure(rlt2, instances, torch, steps, workload="clustered_n30", warmup=3):
    """The FP64 form (the paper's real division) on the headline workload, with
    the roofline of its D->C kernel on the FP64 pipe: the additions the method
    needs per Hungarian step (2 per reduced distance, 1 per label or potential
    moved) over GB300's nominal FP64 rate (1.25 TFLOP/s = 625 G additions/s)."""
    F, D, _ = instances.instance(workload)
    N = F.shape[0]
    n = N - 2
    s = torch.cuda.Stream()
    with rlt2.ContextF64(F, D, profile=True, max_iters=warmup + 2, stream=s.cuda_stream) as c:
        c.iterate(warmup)
        w0 = c.work()
        st0, n0 = c.stage_times()
        c.iterate(2)
        st1, n1 = c.stage_times()
        w1 = c.work()
    ms = (st1 - st0) / (n1 - n0)
    dsteps = (w1[4] - w0[4]) / 2.0
    drelax = (w1[5] - w0[5]) / 2.0
    adds = drelax + (2 * n + 1) * dsteps
    with rlt2.ContextF64(F, D, max_iters=warmup + steps, stream=s.cuda_stream) as c:
        c.iterate(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        c.iterate(steps)
        e1.record(s)
        torch.cuda.synchronize()
        lb = c.bound()[0]
    t = e0.elapsed_time(e1)
    achieved = adds / (ms[1] / 1e3) / 1e9
    return {"metric": "RLT2 dual-ascent iters/sec at N=%d, FP64 form" % N, "unit": "iters/s",
            "value": steps / (t / 1000.0), "steps": steps, "LB": lb, "dtype": "f64",
            "stages_ms": {"spread_complementary_D": ms[0], "concentrate_D_to_C": ms[1],
                          "complementary_C_concentrate_C_to_B": ms[2], "concentrate_B_to_LB": ms[3]},
            "roofline": {"bound": "fp64", "kernel": "f64_dlap_kernel (concentration D->C)",
                         "achieved": achieved, "peak": 625.0, "unit": "Gadd/s", "frac": achieved / 625.0,
                         "traffic": f64_traffic(N),
                         "traffic_kind": "ncu DRAM bytes of the N=20 launch, scaled per tile coefficient",
                         "peak_kind": "nominal FP64 1.25 TFLOP/s (an FMA = 2 flops; one addition per FMA slot)",
                         "work": {"steps": dsteps, "relaxations": drelax, "fp64_adds": adds}}}


def bnb_measure(instances, torch):
    """Branch-and-bound to proven optimality on the 12-facility grid workload:
    every node's children bounded by one batched RLT2 call (12 passes),
    strong branching on RLT1 at the root, local-search incumbent."""
    from paper_1510_02065_gb300 import bnb
    F, D, _ = instances.instance("grid_n12")
    torch.cuda.synchronize()
    r = bnb.BranchAndBound(F, D, iters=12, root_iters=30, strong_depth=1).solve()
    r.pop("perm", None)
    r["workload"] = "grid_n12"
    return r


def lap_methods_measure(rlt2, instances, torch, count=100000):
    """LAPs/s of the Hungarian kernel (the dual ascent's) and of the auction
    method (the paper's GPU LAP) on the same real D tiles: `count` random
    tiles of the 30-facility clustered instance after one pass, 28 x 28 (the
    tile's own two locations dropped), exported through the C ABI."""
    F, D, _ = instances.instance("clustered_n30")
    N, n, m = 30, 28, 29
    with rlt2.Context(F, D) as c:
        c.iterate(1)
        z = c.state(2).reshape(-1, n, n)             # compact tiles on the host
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(z.shape[0], size=count, replace=False))
    M = torch.from_numpy(np.ascontiguousarray(z[pick])).cuda()
    del z
    s = torch.cuda.Stream()
    S1 = torch.empty(count, dtype=torch.int64, device="cuda")
    S2 = torch.empty(count, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    out = {}
    for name, call in (("hungarian", lambda: rlt2.rlt2_lap_batch(M.data_ptr(), n, count, S1.data_ptr(),
                                                                 stream=s.cuda_stream)),
                       ("auction", lambda: rlt2.rlt2_lap_batch_auction(M.data_ptr(), n, count, S2.data_ptr(),
                                                                       stream=s.cuda_stream))):
        call()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        rc = call()
        e1.record(s)
        torch.cuda.synchronize()
        out[name] = {"laps_per_s": count / (e0.elapsed_time(e1) / 1000.0), "rc": rc}
    out["identical_optima"] = bool(torch.equal(S1, S2))
    out["problems"] = "%d D tiles (28 x 28) of clustered N=30 after one pass" % count
    return out


def batch_measure(rlt2, instances, torch, nodes_count, iters):
    """Batched B&B bounding against the plain one-node-at-a-time path.

    Nodes of one 25-facility clustered instance, node s fixing 1-15 random
    facilities (residual sizes 10-24), `iters` passes each.  Batched: one
    rlt2_batch_bound call (tuning passes, then one captured graph for all
    nodes and the remaining passes).  Plain: per node rlt2_subproblem,
    rlt2_create, rlt2_iterate, rlt2_bound, rlt2_destroy.  Both wall-clock,
    both including every allocation and copy, both after an untimed warm-up
    of their own on four nodes (module loading, first graph capture); the
    bounds must be identical.  By residual size: the same two arms on the
    nodes of each range of N' (batched: one call per range).
    """
    F, D = instances.clustered_euclid(25, seed=0)
    nodes = instances.subproblem_nodes(25, nodes_count)
    s = torch.cuda.Stream()

    def plain_one(fac, loc):
        Fp, Dp, Bl, cst = rlt2.rlt2_subproblem(F, D, fac, loc)
        with rlt2.Context(Fp, Dp, B_lin=Bl, lb_const=cst, max_iters=iters + 1, stream=s.cuda_stream) as c:
            c.iterate(iters)
            return c.bound()[1]

    # untimed warm-up of both arms
    rlt2.rlt2_batch_bound(F, D, nodes[:4], 3)
    for fac, loc in nodes[:4]:
        plain_one(fac, loc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbs, dev_ms, shapes = rlt2.rlt2_batch_bound(F, D, nodes, iters, return_lanes=True)
    t_batch = time.perf_counter() - t0
    plain, t_node = [], []
    t0 = time.perf_counter()
    for fac, loc in nodes:
        t1 = time.perf_counter()
        plain.append(plain_one(fac, loc))
        t_node.append(time.perf_counter() - t1)
    t_plain = time.perf_counter() - t0
    sizes = [25 - len(f) for f, _ in nodes]
    by_size = []
    for lo, hi in ((10, 14), (15, 19), (20, 24)):
        idx = [i for i, n in enumerate(sizes) if lo <= n <= hi]
        if not idx:
            continue
        t0 = time.perf_counter()
        rlt2.rlt2_batch_bound(F, D, [nodes[i] for i in idx], iters)
        tb = time.perf_counter() - t0
        tp = sum(t_node[i] for i in idx)
        by_size.append({"residual_N": [lo, hi], "nodes": len(idx), "batched_nodes_per_s": len(idx) / tb,
                        "plain_nodes_per_s": len(idx) / tp, "speedup": tp / tb})
    return {"metric": "batched B&B nodes/sec vs plain", "unit": "nodes/s",
            "batched": nodes_count / t_batch, "plain": nodes_count / t_plain,
            "speedup": t_plain / t_batch, "identical_bounds": list(plain) == [int(x) for x in lbs],
            "nodes": nodes_count, "iters": iters, "residual_N": [min(sizes), max(sizes)],
            "batched_device_ms": dev_ms, "graph_launches": 1,
            "dlap_shape_after_tuning": {"N_gt_16": {"lanes": shapes[0][0], "cta_warps": shapes[0][1]},
                                        "N_le_16": {"lanes": shapes[1][0], "cta_warps": shapes[1][1]}},
            "by_residual_size": by_size,
            "config": "clustered N=25 seed 0, node s fixes 1-15 pairs from default_rng(1000+s)"}


def batch_sharded_measure(rlt2, instances, torch, dist, nodes_count, iters):
    """The same nodes dealt round-robin over the ranks (one GPU each), each
    rank bounding its share with one rlt2_batch_bound call; wall clock from a
    barrier to the gathered bounds, the maximum over the ranks."""
    from paper_1510_02065_gb300 import distributed
    F, D = instances.clustered_euclid(25, seed=0)
    nodes = instances.subproblem_nodes(25, nodes_count)
    rlt2.rlt2_batch_bound(F, D, nodes[:4], 3)   # warm-up
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    lbs = distributed.bound_nodes_sharded(F, D, nodes, iters)
    t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")   # NCCL: device tensors
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return {"metric": "batched B&B nodes/sec, nodes sharded over the ranks", "unit": "nodes/s",
            "value": nodes_count / float(t.item()), "nodes": nodes_count, "iters": iters,
            "ranks": dist.get_world_size(), "scaling": "strong", "lb_sum": int(sum(lbs)),
            "config": "clustered N=25 seed 0, node s fixes 1-15 pairs from default_rng(1000+s)"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- CPU oracle

def oracle_sample(F, D, budget_s, steps=None):
    """Time the CPU oracle (single thread) on a bounded sample of one pass.

    The fused spread/complementary operations and the C/B concentrations are
    timed in full; the D->C concentration (the bulk of a pass) is timed on
    facility slices i (the tiles D_ijkn with that first facility), each on the
    true pass-1 input (the slice is restored after timing), and extrapolated
    to all N slices.  With `steps`, returns one extrapolated pass time per step
    (one slice each) instead.
    """
    from oracle import oracle as O
    N = F.shape[0]
    st = O.State(F, D)
    t0 = time.perf_counter()
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    t_sc = time.perf_counter() - t0
    d, c = st.d, st.c
    slice_times = []
    per_step = []
    k = 0
    tb = time.perf_counter()
    while True:
        i = k % N
        dsave, csave = d[i].copy(), c[i].copy()
        t1 = time.perf_counter()
        st.concentrate_D_to_C_range(i, i + 1)
        dt = time.perf_counter() - t1
        d[i] = dsave
        c[i] = csave
        slice_times.append(dt)
        per_step.append(dt)
        k += 1
        if steps is not None:
            if k >= steps:
                break
        elif time.perf_counter() - tb >= budget_s and k >= 2:
            break
    # the C/B operations of the pass on the true state after D->C is not
    # available without the full concentration; time them on the current state
    t2 = time.perf_counter()
    st.complementary_C()
    st.concentrate_C_to_B()
    st.add_LB(st.concentrate_B_to_LB())
    t_cb = time.perf_counter() - t2
    st.close()
    rest = t_sc + t_cb
    if steps is not None:
        return [N * s + rest for s in per_step], rest
    t_pass = N * float(np.mean(slice_times)) + rest
    return t_pass, len(slice_times), rest


def oracle_all_cores(F, D):
    """One full pass (pass 1, all seven operations) of the CPU oracle with its
    operations over D split by facility over every host core
    (State.iterate_threaded; the same result as the sequential pass)."""
    from oracle import oracle as O
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    st = O.State(F, D)
    t0 = time.perf_counter()
    st.iterate_threaded(threads)
    t = time.perf_counter() - t0
    st.close()
    return t, threads


def reference_arm(args):
    """--impl reference: the CPU oracle as it stands, one sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1510_02065_gb300 import instances
    F, D, _ = instances.instance(args.workload)
    N = F.shape[0]
    t0 = time.perf_counter()
    times, rest = oracle_sample(F, D, 0, steps=args.warmup + args.steps)
    wall = time.perf_counter() - t0
    timed = times[args.warmup:]
    t_pass = float(np.mean(timed))
    value = 1.0 / t_pass
    sample = ("each step: D->C concentration of one facility slice (N*(N-1)^2 = %d LAPs of size %d, "
              "true pass-1 input) x N slices, plus the pass's spread, complementary and C/B "
              "operations timed once (%.1f s); single thread" % (N * (N - 1) ** 2, N - 2, rest))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_pass, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "seed": 0},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours

def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1510_02065_gb300 import build, instances, rlt2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(rlt2.LIB_PATH):
        build.build()
    rlt2.lib()

    F, D, _ = instances.instance(args.workload)
    N = F.shape[0]
    K, W = args.steps, args.warmup
    # a stream of our own: the library launches on it and the events time it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    peaks, peaks_kind = load_peaks()
    props = torch.cuda.get_device_properties(local)

    store = rlt2.RLT2_STORE_CLASSES if args.store == "classes" else rlt2.RLT2_STORE_TILES
    ctx = rlt2.Context(F, D, profile=True, use_graph=True, max_iters=K + W + 24,
                       stream=stream.cuda_stream, store=store, lanes=args.lanes, cta_warps=args.cta_warps)
    ctx.iterate(W)
    # the D->C shape is tuned on a context's first passes (see rlt2.h): should
    # W be shorter than that, the remaining tuning passes run here, untimed
    extra = 0
    while ctx.dlap_shape()[2] and extra < 8:
        ctx.iterate(1)
        extra += 1
    torch.cuda.synchronize()
    rlt2.rlt2_reset_stage_times(ctx.ctx)
    w0 = ctx.work()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.iterate(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    stage_ms, passes = ctx.stage_times()
    w1 = ctx.work()
    lb, lb_exact, iters = ctx.bound()
    shape = ctx.dlap_shape()
    ctx.close()

    ms_per_step = ms / K
    value = world * K / (ms / 1000.0)
    laps_per_pass = (w1["laps"] - w0["laps"]) / K
    d_relax = (w1["d_relaxations"] - w0["d_relaxations"]) / K
    d_steps = (w1["d_steps"] - w0["d_steps"]) / K
    d_laps = (w1["d_laps"] - w0["d_laps"]) / K
    t_p1 = stage_ms[0] / passes
    t_dlap = stage_ms[1] / passes
    t_clap = stage_ms[2] / passes
    t_xlap = stage_ms[3] / passes

    # roofline of the dominant kernel (D -> C concentration): integer ALU bound.
    # The ALU pipe (integer compare, select, add, logic, shift) takes one warp
    # instruction every two cycles per scheduler: 64 lanes per SM per clock
    # (ncu on this kernel: issue slots 85.8% busy, ALU pipe 85.7% of its peak,
    # FMA and MIO pipes about 22% each -- only a half-rate ALU pipe fits).
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = props.multi_processor_count * ALU_LANES_PER_SM * sm_max * 1e6 / 1e12   # Tops/s
    achieved = OPS_PER_RELAXATION * d_relax / (t_dlap / 1e3) / 1e12
    n_tiles = N * N * (N - 1) ** 2
    m = N - 2
    z_bytes = n_tiles * m * m * 4
    if args.store == "tiles":
        # D read and written once by each kernel (+ C and B read by the fused pass)
        dlap_bytes = 2 * z_bytes
        p1_bytes = 2 * z_bytes + n_tiles * 4 + N * N * 4
    else:
        # class sums (one per class) and per-tile duals (u: N-2, v: N-2 coefficients)
        classes = N * (N - 1) * (N - 2) // 6 * N * (N - 1) * (N - 2)
        duals = n_tiles * 2 * m * 4
        dlap_bytes = classes * 4 + duals                      # class sums read, duals written
        p1_bytes = 2 * classes * 4 + duals + n_tiles * 4 + N * N * 4
    dlap_hbm_gbs = dlap_bytes / (t_dlap / 1e3) / 1e9
    p1_gbs = p1_bytes / (t_p1 / 1e3) / 1e9
    traffic = captured_traffic(DLAP_TRAFFIC, args.workload, args.store)
    p1_traffic = captured_traffic(P1_TRAFFIC, args.workload, args.store)

    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "seed": 0, "tiles": n_tiles, "store": args.store,
                   "laps_per_iter": int(round(laps_per_pass)), "z_bytes": z_bytes,
                   "l2": "inputs larger than L2 (D %.2f GB of coefficients)" % (z_bytes / 1e9),
                   "parallelism": "replicas x%d" % world if world > 1 else "1 GPU"},
        "laps_per_s": world * laps_per_pass * K / (ms / 1000.0),
        "bound": {"LB": lb_exact, "iterations": iters},
        "stages_ms": {"spread_complementary_D": t_p1, "concentrate_D_to_C": t_dlap,
                      "complementary_C_concentrate_C_to_B": t_clap, "concentrate_B_to_LB": t_xlap},
        "roofline": {"bound": "alu", "kernel": "dlap_kernel (concentration D->C)",
                     "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "peak_kind": "%d SMs x %d ALU-pipe lanes x %.0f MHz (%s sm_max)" % (
                         props.multi_processor_count, ALU_LANES_PER_SM, sm_max, peaks_kind),
                     "work": {"laps": d_laps, "steps": d_steps, "relaxations": d_relax,
                              "ops_per_relaxation": OPS_PER_RELAXATION},
                     "hbm_gbs": dlap_hbm_gbs},
        "p1_roofline": {"bound": "hbm", "kernel": "p1_kernel (spread + complementary D)",
                        "achieved": p1_gbs, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                        "frac": p1_gbs / float(peaks["hbm_gbs"]), "bytes_per_launch": p1_bytes,
                        "traffic": p1_traffic,
                        "peak_kind": peaks_kind},
        "gpu_launches": 5 * K,
        "clocks": clk,
        "dlap_shape": {"lanes": shape[0], "cta_warps": shape[1], "tuning_passes_after_warmup": extra},
    }

    # end to end through the public API with host buffers: create (H2D of F, D
    # from pinned memory), then every step one pass and a D2H read of the bound
    if not args.no_e2e:
        Fp = torch.from_numpy(F).pin_memory().numpy()
        Dp = torch.from_numpy(D).pin_memory().numpy()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = rlt2.Context(Fp, Dp, max_iters=K + 4, stream=stream.cuda_stream, store=store)
        for _ in range(K):
            c2.iterate(1)
            c2.bound()
        c2.close()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        line["e2e"] = {"value": world * K / e2e_s, "unit": "iters/s",
                       "h2d_bytes_per_step": 2 * N * N * 4 / K, "d2h_bytes_per_step": 12,
                       "includes": "rlt2_create (alloc, H2D, init) + per step rlt2_iterate(1) + "
                                   "rlt2_bound + rlt2_destroy"}

    # the single-GPU measurements beside the metric run at N = 1 only (a
    # multi-GPU run times the replicas and does not hold its GPUs longer)
    solo = world == 1
    if args.batch_nodes > 0 and solo:
        line["batch"] = batch_measure(rlt2, instances, torch, args.batch_nodes, args.batch_iters)
    if args.batch_nodes > 0 and not solo:
        # B&B nodes shard naturally: each rank bounds its share (no collective
        # on the data path; the bounds are gathered once)
        line["batch_sharded"] = batch_sharded_measure(rlt2, instances, torch, dist, args.batch_nodes,
                                                      args.batch_iters)
    if args.n35_steps > 0 and solo:
        line["n35"] = n35_measure(rlt2, instances, torch, args.n35_steps, rlt2.RLT2_STORE_CLASSES)
        line["n35_tiles"] = n35_measure(rlt2, instances, torch, args.n35_steps, rlt2.RLT2_STORE_TILES)
        # the paired dual ascent of Sec. 6's complementary submatrices (another
        # arithmetic: half the D->C LAPs, its own bound), beside the metric
        line["pairs_n30"] = n35_measure(rlt2, instances, torch, 100, rlt2.RLT2_STORE_PAIRS,
                                        workload="clustered_n30")
        line["pairs_n35"] = n35_measure(rlt2, instances, torch, args.n35_steps, rlt2.RLT2_STORE_PAIRS)
    if args.fp64_steps > 0 and solo:
        line["fp64"] = fp64_measure(rlt2, instances, torch, args.fp64_steps, workload=args.workload)
    if args.serve_requests > 0 and solo:
        line["serve"] = serve_measure(instances, torch, args.serve_requests)
    if args.batch_nodes > 0 and solo:
        line["bnb"] = bnb_measure(instances, torch)
        line["lap_methods"] = lap_methods_measure(rlt2, instances, torch)

    if rank == 0 and world == 1 and args.cpu_budget > 0:
        t_pass, nslices, rest = oracle_sample(F, D, args.cpu_budget)
        line["cpu_baseline"] = {
            "value": 1.0 / t_pass, "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": "pass 1: spread/complementary and C/B operations in full (%.1f s), D->C "
                      "concentration on %d facility slices of %d LAPs each, extrapolated to %d "
                      "slices; single-threaded C oracle" % (rest, nslices, N * (N - 1) ** 2, N)}
        t_all, threads = oracle_all_cores(F, D)
        line["cpu_baseline_all_cores"] = {
            "value": 1.0 / t_all, "unit": "iters/s", "cores": threads, "kind": "oracle",
            "sample": "one full pass 1 (all seven operations, %.1f s), the operations over D split by "
                      "facility over %d host threads; C oracle as it stands" % (t_all, threads)}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
