#!/usr/bin/env python3
"""Benchmark of the SPOCK hot path on B300 GPUs.

One step = one cold-start SPOCK solve (Alg. 4 with Anderson directions) of the
large scenario-tree RAOCP (nx=50, nu=25, N=15, 3-way branching at stages 0-3,
1012 nodes, AV@R 0.3, box + ball constraints) until ||v - T(v)||_inf <= 1e-4.
The headline value is SPOCK iterations per second over the timed solves (the
iteration count of a solve is fixed by the data, so iterations/s and the
time to 1e-4 carry the same information); the FP64 iteration is reported
beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica of the problem (the
method has no data-parallel split of one problem): value = iterations of all
ranks / the slowest rank's time. --impl reference times the FP64 CPU oracle on
the same workload (rank 0 only).
"""
import os

# the CPU oracle runs single-threaded (set before numpy is imported)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPOCK iters/s & time-to-1e-4 residual; batched solves/s, p99 latency vs plain"
WORKLOAD = ("large_raocp: nx=50 nu=25 N=15, 3-way branching at stages 0-3 (81 scenarios, "
            "1012 nodes), AV@R 0.3, box on x and u + ||u||_2<=3, seed 2")
TOL = 1e-4


KSOLVE_SOURCES = ("spock_dev.cuh", "spock_internal.h", "spock_cta.cuh", "spock_solver_kernel.cuh",
                  "spock_solver_inst.cu")


def solver_source_hash():
    """Hash of the code (comment lines left out) of the sources that define the
    solve kernel: DRAM counters recorded for another build of it are not used."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2505_12078_b300", "csrc")
    for name in KSOLVE_SOURCES:
        for line in open(os.path.join(d, name)):
            if not line.strip().startswith("//"):
                h.update(line.encode())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def algorithmic_bytes(sizes, n_T, iters, word):
    """Bytes one solve must move at least, from the counting of the design notes:
    per T evaluation the per-node factor matrices (MB, MF per non-root node,
    MP, KT per non-leaf node, unpadded) once, plus 8 passes over v; per SPOCK
    iteration 21 passes over v for the Anderson memory and the direction."""
    n, n_nl, nx, nu = sizes["n"], sizes["n_nonleaf"], sizes["nx"], sizes["nu"]
    factors = (n - 1) * (nx * (nx + nu) + (nx + nu) * nx) + n_nl * (nu * (nx + nu) + nx * nu)
    nv = sizes["n_v"]
    per_T = word * (factors + 8 * nv)
    per_iter = word * 21 * nv
    return n_T * per_T + iters * per_iter, per_T


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(p, seconds=12.0):
    """The FP64 oracle as it stands, on the same workload, for a bounded sample."""
    from oracle.spock_oracle import Oracle
    o = Oracle(p)
    t = time.time()
    o.T(o.initial_v())
    per_T = time.time() - t
    iters = max(3, int(seconds / (2.3 * per_T)))
    t = time.time()
    r = o.solve(tol=0.0, max_iters=iters)
    el = time.time() - t
    return {"value": r["iters"] / el, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"{r['iters']} SPOCK iterations ({r['n_T']} T evaluations) of the same "
                      f"workload from a cold start, FP64 numpy oracle, {el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2505_12078_b300 import synth
    from oracle.spock_oracle import Oracle
    p = synth.large_raocp()
    o = Oracle(p)
    step_iters = 12
    for _ in range(args.warmup):
        o.solve(tol=0.0, max_iters=2)
    times, iters = [], 0
    for _ in range(args.steps):
        t = time.time()
        r = o.solve(tol=0.0, max_iters=step_iters)
        times.append(time.time() - t)
        iters += r["iters"]
    total = sum(times)
    value = iters / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": TOL,
                       "step": f"{step_iters} SPOCK iterations from a cold start (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} x {step_iters} SPOCK iterations of the workload"},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH_COUNT = 512
BATCH_FIXED_ITERS = 200      # fixed-work throughput on the whole draw
SMALL_COUNT = 64             # the draw's problems with the fewest nodes: solves to 1e-4 and serving
MAX_ITERS = 20000


def _gen(i):
    from paper_2505_12078_b300 import synth
    return synth.batch_problem(synth.batch_specs(BATCH_COUNT, seed=4)[i], i)


def batch_draw():
    """The uneven 512-problem draw (seed 4), generated by a pool of spawned
    host processes (before this process touches the GPU for the batch)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen, range(BATCH_COUNT), chunksize=8)


def _plain_fp64(spock, G, probs, idx, max_iters, tol, warm=False, x0s=None):
    t = time.time()
    conv = iters = 0
    for k in idx:
        r = G[k].solve(x0s[k] if x0s else probs[k].x0,
                       spock.opts(precision=64, tol=tol, max_iters=max_iters, warm_start=warm, fp64_check=False))
        conv += r["status"] == 0
        iters += r["info"]["iters"]
    return time.time() - t, int(conv), int(iters)


def bench_batched(spock, probs, G, small):
    """Batched FP32 (one persistent graph-captured launch, warps per team from
    the autotuner) against the plain single-problem FP64 method (one
    cooperative launch per problem, the whole GPU each): (1) fixed work,
    BATCH_FIXED_ITERS SPOCK iterations of every problem of the draw; (2) the
    SMALL_COUNT smallest problems solved to ||v - T(v)||_inf <= 1e-4. The plain
    method runs on every 8th problem (its time is linear in the number of
    problems)."""
    res = {"workload": "uneven draw of 512 problems (seed 4): nx~U{4..64}, nu=nx/2, N~U{5..20}, "
                       "b~U{2..4}-way branching at the first k~U{1..4} stages, AV@R~U[0.2,1], box + ball; "
                       f"{sum(len(p.anc) for p in probs)} nodes"}
    o = spock.opts(precision=32, tol=0.0, max_iters=BATCH_FIXED_ITERS)
    b = spock.Batch(G, precision=32)
    tw = b.autotune(iters=20)                   # warps per team of every problem's sweeps
    x0s = [p.x0 for p in probs]
    r = b.solve(x0s, o)
    b.close()
    res["autotuned_tw"] = {str(t): int((tw == t).sum()) for t in (1, 2, 4, 8)}
    it = sum(i["iters"] for i in r["info"])
    # algorithmic bytes of the launch (same counting as the single-problem roofline)
    alg = sum(algorithmic_bytes(g.sizes, i["n_T"], i["iters"], 4)[0] for g, i in zip(G, r["info"]))
    peak, peak_kind = measured_peak()
    achieved = alg / (r["total_ms"] / 1000.0) / 1e9
    pw, _, pit = _plain_fp64(spock, G, probs, range(0, len(probs), 8), BATCH_FIXED_ITERS, 0.0)
    res["fixed_work"] = {"iters_per_problem": BATCH_FIXED_ITERS,
                         "batched_fp32_iters_per_s": it / (r["total_ms"] / 1000.0),
                         "batched_device_ms": r["total_ms"],
                         "plain_fp64_iters_per_s": pit / pw,
                         "ratio": (it / (r["total_ms"] / 1000.0)) / (pit / pw),
                         "roofline": {"bound": "hbm", "kernel": "k_batch (one persistent launch, graph replay)",
                                      "algorithmic_bytes": alg, "achieved": achieved, "peak": peak,
                                      "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind}}
    sG = [G[k] for k in small]
    sp = [probs[k] for k in small]
    o = spock.opts(precision=32, tol=TOL, max_iters=MAX_ITERS)
    b = spock.Batch(sG, precision=32)
    b.autotune(iters=20)
    r = b.solve([p.x0 for p in sp], o)
    b.close()
    conv = sum(1 for i in r["info"] if i["status"] == 0)
    pw, pc, _ = _plain_fp64(spock, sG, sp, range(0, len(sp), 8), MAX_ITERS, TOL)
    res["to_tol"] = {"problems": f"the {SMALL_COUNT} problems of the draw with the fewest nodes "
                                 f"({sum(len(p.anc) for p in sp)} nodes)",
                     "tol": TOL, "max_iters": MAX_ITERS,
                     "batched_fp32_solves_per_s": conv / (r["total_ms"] / 1000.0), "converged": conv,
                     "batched_device_ms": r["total_ms"],
                     "plain_fp64_solves_per_s": pc / pw, "plain_converged": pc,
                     "plain_problems": len(range(0, len(sp), 8)),
                     "ratio": (conv / (r["total_ms"] / 1000.0)) / max(pc / pw, 1e-12)}
    return res


def bench_serving(spock, probs, G, rate=2000.0, seconds=0.2, seed=5):
    """MPC serving on the SMALL_COUNT smallest plants: Poisson arrivals at
    `rate` for `seconds`; a request carries the plant's next state (x1 = A x0 +
    B u0 at a child drawn by its probability, plus N(0, 0.01 I) noise, clipped
    into the state box) and is warm-started from the plant's resident iterate.
    Latency = submission to collection on the host."""
    import numpy as np
    o32 = spock.opts(precision=32, tol=TOL, max_iters=MAX_ITERS)
    srv = spock.Server(G, precision=32, o=o32)
    x = [p.x0.copy() for p in probs]
    u = [None] * len(probs)
    for k, p in enumerate(probs):             # one cold solve per plant first
        srv.submit(k, x[k], warm=False)
    for r in srv.drain(600):
        u[r["plant"]] = r["u0"]
    rng = np.random.default_rng(seed)

    def next_state(k):
        p = probs[k]
        ch = [c for c in range(1, len(p.anc)) if p.anc[c] == 0]
        pr = np.array([p.prob[c] for c in ch])
        c = ch[int(rng.choice(len(ch), p=pr / pr.sum()))]
        x1 = p.A[c - 1] @ x[k] + p.B[c - 1] @ u[k] + p.c[c - 1]
        return np.clip(x1 + 0.1 * rng.standard_normal(p.nx), -4.5, 4.5)

    got, sub = [], 0
    t0 = time.time()
    t_next = t0
    while time.time() - t0 < seconds:
        now = time.time()
        while t_next <= now:
            k = int(rng.integers(0, len(probs)))
            x[k] = next_state(k)
            srv.submit(k, x[k], warm=True)
            sub += 1
            t_next += rng.exponential(1.0 / rate)
        for r in srv.poll():
            got.append(r)
            u[r["plant"]] = r["u0"]
    got += srv.drain(600)
    wall = time.time() - t0
    srv.close()
    lat = np.array([r["latency_ms"] for r in got])
    dev = np.array([r["device_ms"] for r in got])
    conv = sum(1 for r in got if r["status"] == 0)
    # the plain FP64 method, one warm-started request at a time on a sample of plants
    pl = []
    for k in range(0, len(probs), 16):
        t = time.time()
        G[k].solve(x[k], spock.opts(precision=64, tol=TOL, max_iters=MAX_ITERS, warm_start=True,
                                     fp64_check=False))
        pl.append(1000 * (time.time() - t))
    return {"plants": f"the {SMALL_COUNT} problems of the draw with the fewest nodes",
            "arrival_rate_per_s": rate, "arrival_seconds": seconds, "submitted": sub, "completed": len(got),
            "converged": conv, "solves_per_s": len(got) / wall,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "device_ms_p50": float(np.percentile(dev, 50)), "device_ms_p99": float(np.percentile(dev, 99)),
            "plain_fp64_solve_ms_p50": float(np.percentile(pl, 50)),
            "plain_fp64_solve_ms_p99": float(np.percentile(pl, 99)),
            "note": "plain = the single-problem FP64 method on one warm-started request at a time "
                    "(solve time, no queueing)"}


def combine_ranks(dist, total_ms, iters, device):
    """Replicas: the slowest rank's time and the iterations of all ranks."""
    import torch
    t = torch.tensor([total_ms, float(iters)], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    n = t[1:].clone()
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(tmax.item()), int(n.item())


def run_ours(args, rank, world, local_rank, dist):
    # the batched draw is generated before this process touches the GPU
    bprobs = batch_draw() if (not args.no_batch and rank == 0) else None
    import torch

    from paper_2505_12078_b300 import spock, synth
    torch.cuda.set_device(local_rank)
    spock.load()
    p = synth.large_raocp()
    g = spock.Problem(p)
    sizes = g.sizes
    stream = torch.cuda.current_stream()
    x0 = torch.tensor(p.x0, dtype=torch.float64, device="cuda")
    xo = torch.empty(g.n * g.nx, dtype=torch.float64, device="cuda")
    uo = torch.empty(g.n_nl * g.nu, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(prec, timed):
        o = spock.opts(precision=prec, tol=TOL, max_iters=200000, fp64_check=True)
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = g.solve_device(x0, o, xo, uo, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), info, st

    prec = args.precision
    for _ in range(args.warmup):
        one(prec, False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, infos = [], []
    with ClockSampler(local_rank) as cs:
        for _ in range(args.steps):
            ms, info, st = one(prec, True)
            times.append(ms)
            infos.append(info)
    clocks = cs.summary()
    torch.cuda.synchronize()
    total_ms = sum(times)
    iters = sum(i["iters"] for i in infos)
    if dist:
        total_ms, iters = combine_ranks(dist, total_ms, iters, "cuda")
    if rank != 0:
        return
    value = iters / (total_ms / 1000.0)
    word = 4 if prec == 32 else 8
    inf0 = infos[0]
    kern_ms = statistics.mean(i["device_ms"] for i in infos)
    bytes_launch, per_T = algorithmic_bytes(sizes, inf0["n_T"], inf0["iters"], word)
    peak, peak_kind = measured_peak()
    achieved = bytes_launch / (kern_ms / 1000.0) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic_k_solve_large_raocp.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            if tr.get("precision") == prec and tr.get("source_hash") == solver_source_hash():
                traffic = tr["dram_bytes_per_T"] * inf0["n_T"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_solve (one persistent cooperative launch per solve)",
                "algorithmic_bytes_per_launch": bytes_launch, "algorithmic_bytes_per_T": per_T,
                "launch_ms": kern_ms}
    # the FP64 iteration on the same workload
    fp64 = None
    if prec == 32:
        ms64, info64, _ = one(64, True)
        fp64 = {"iters_per_s": info64["iters"] / (ms64 / 1000.0), "time_to_tol_ms": ms64,
                "iterations": info64["iters"], "T_evals": info64["n_T"],
                "res_inf": info64["res_inf"]}
    # end to end through the C ABI with host buffers (x0 in, x/u out)
    e2e_ms = []
    o = spock.opts(precision=prec, tol=TOL, max_iters=200000, fp64_check=True)
    for _ in range(1):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.time()
        r = g.solve(p.x0, o)
        e2e_ms.append(1000 * (time.time() - t))
    e2e_iters = r["info"]["iters"]
    e2e = {"value": e2e_iters / (statistics.mean(e2e_ms) / 1000.0), "unit": "iter/s",
           "h2d_bytes_per_step": 8 * g.nx,
           "d2h_bytes_per_step": 8 * (g.n * g.nx + g.n_nl * g.nu + 1),
           "time_to_tol_ms": statistics.mean(e2e_ms)}
    launches_per_step = 3 + (2 if prec == 32 else 0)   # x0 scaling, solve, unscale (+ FP64 check)
    cpu = cpu_baseline(p) if world == 1 else None
    batched = serving = None
    if bprobs is not None:
        # a failure here must not cost the headline line: it is reported in place
        try:
            bG = [spock.Problem(q) for q in bprobs]
            small = sorted(range(len(bprobs)), key=lambda k: (len(bprobs[k].anc), k))[:SMALL_COUNT]
            batched = bench_batched(spock, bprobs, bG, small)
            serving = bench_serving(spock, [bprobs[k] for k in small], [bG[k] for k in small])
        except Exception as e:   # noqa: BLE001
            err = {"error": f"{type(e).__name__}: {e}"}
            batched = batched or err
            serving = serving or err
    line = {"metric": METRIC, "value": value * 1.0, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == 32 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": TOL,
                       "precision": "FP32 iteration, FP64 factors and FP64 residual check" if prec == 32
                                    else "FP64",
                       "step": "one cold-start SPOCK solve to ||v - T(v)||_inf <= 1e-4",
                       "time_to_tol_ms": total_ms / args.steps,
                       "iterations_per_solve": inf0["iters"], "T_evals_per_solve": inf0["n_T"],
                       "final_res_inf": inf0["res_inf"], "final_res_inf_fp64": inf0["res_inf_fp64"],
                       "l2": "flushed (256 MB write) before every step",
                       "parallelism": f"replicas x{world}"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "fp64": fp64,
            "batched": batched, "serving": serving}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="run one batched launch of this many iterations on every 32nd problem of the "
                         "uneven draw and exit (for ncu captures)")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="run one solve of this many SPOCK iterations and exit (for ncu captures)")
    args = ap.parse_args()
    if args.profile_batch:
        from paper_2505_12078_b300 import spock, synth
        spock.load()
        specs = synth.batch_specs(BATCH_COUNT, seed=4)
        probs = [synth.batch_problem(specs[i], i) for i in range(0, BATCH_COUNT, 32)]
        G = [spock.Problem(q) for q in probs]
        b = spock.Batch(G, precision=32)
        r = b.solve([q.x0 for q in probs], spock.opts(precision=32, tol=0.0, max_iters=args.profile_batch))
        it = sum(i["iters"] for i in r["info"])
        nT = sum(i["n_T"] for i in r["info"])
        alg = sum(algorithmic_bytes(g.sizes, i["n_T"], i["iters"], 4)[0] for g, i in zip(G, r["info"]))
        print(json.dumps({"problems": len(probs), "nodes": sum(len(q.anc) for q in probs), "iters": it,
                          "n_T": nT, "algorithmic_bytes": alg, "device_ms": r["total_ms"],
                          "source_hash": solver_source_hash()}))
        return
    if args.profile_iters:
        import torch
        from paper_2505_12078_b300 import spock, synth
        spock.load()
        p = synth.large_raocp()
        g = spock.Problem(p)
        r = g.solve(p.x0, spock.opts(precision=args.precision, tol=0.0,
                                      max_iters=args.profile_iters, fp64_check=False))
        print(json.dumps({"n_T": r["info"]["n_T"], "iters": r["info"]["iters"],
                          "precision": args.precision, "source_hash": solver_source_hash()}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
