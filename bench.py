#!/usr/bin/env python
"""Benchmark of the elastance/mobility Nystrom-GMRES hot path on GB300.

One step = one complete elastance solve of 100 star curves x 256 nodes
(M = 25,600): geometry staging, right-hand side, GMRES with FP32 pair sums
inside FP64 iterative refinement down to a relative residual of 1e-12, and the
potentials at interior points.  Inputs are resident in HBM when the timed
region starts; the L2 is flushed (a 256 MB write) before every step, outside
the per-step CUDA events.

Printed (rank 0, one JSON line): solves/s (mixed precision, whole job), the
plain-FP64 solves/s beside it, pair interactions/s of the hot pair-sum kernel,
per-step latency percentiles, the end-to-end rate through the C ABI with host
buffers, the roofline of the dominant kernel and the CPU-oracle baseline.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun every rank solves its own replica (independent problems, no
collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "stars100_M25600"
METRIC = "elastance solves/s at 1e-12 relative residual (mixed precision: FP32 pair sums inside refinement)"
# algorithmic flops per pair interaction (FMA = 2): Laplace r (2), |r|^2 (3),
# q/|r|^2 (1), accumulate q r/|r|^2 (4); Stokes r (2), |r|^2 (3), r.mu (3),
# r.n (3), (r.mu)(r.n)/|r|^4 (3), accumulate (4)
FLOPS_PER_PAIR = {"laplace": 10.0, "stokes": 18.0}
# DRAM bytes (read + write) per launch of the 100-star pair sums, from one ncu
# capture of the current kernels (profiles/k_pair32s_laplace_stars100_M25600.md:
# the symmetric FP32 kernel); a kernel changed since its capture must be taken
# out of this table
DRAM_BYTES_PER_LAUNCH = {"laplace_fp32": 1.002e6}
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--precision", default="mixed_ff", choices=["mixed", "mixed_ff"],
                    help="headline path: FP32 pair sums in refinement with an FP64 (mixed) or a "
                         "float-float (mixed_ff) residual")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--four-disc-steps", type=int, default=100,
                    help="solves of the four-disc case (M = 512) per precision, host clock (0 = skip)")
    ap.add_argument("--splits", type=int, default=0,
                    help="--kernel: install this pair-sum split count instead of searching (0 = search, "
                         "negative = the symmetric FP32 Laplace plan)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the occupancy rule's pair-sum split counts (no bie_tune before the warm-up)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="served stream: mixed elastance/mobility requests (0 = skip)")
    ap.add_argument("--serve-workers", type=int, default=16)
    ap.add_argument("--serve-hbm-fraction", type=float, default=0.05,
                    help="served stream: admission cap as a fraction of the device's HBM")
    ap.add_argument("--cpu-1core", action="store_true",
                    help="also time the full oracle solve with one BLAS thread (about 8 minutes)")
    ap.add_argument("--serve-batch", type=int, default=8,
                    help="served stream again with up to this many queued requests solved together (<= 1: skip)")
    ap.add_argument("--fmm-order", type=int, default=36)
    ap.add_argument("--only-large", action="store_true",
                    help="run only the large mobility section (FMM), e.g. for ncu captures")
    ap.add_argument("--only-serving", action="store_true", help="run only the serving section")
    ap.add_argument("--only-batched", action="store_true", help="run only the batched-solves section")
    ap.add_argument("--batch-requests", type=int, default=1000,
                    help="batched solves: served-mix requests solved in batches of one kind (0 = skip the section)")
    ap.add_argument("--batch-size", type=int, default=16)
    ap.add_argument("--mobility-steps", type=int, default=5,
                    help="timed mobility solves of 400 ellipses x 128 nodes, direct pair sums (0 = skip)")
    ap.add_argument("--mobility-fmm-order", type=int, default=36,
                    help="the 400-ellipse solves again with FMM pair sums of this order (0 = skip)")
    ap.add_argument("--headline-fmm-order", type=int, default=30,
                    help="the 100-star solves again with FMM pair sums of this order, reported beside "
                         "the headline (0 = skip)")
    ap.add_argument("--large-steps", type=int, default=1,
                    help="timed mobility solves of 10,000 ellipses x 64 nodes with FMM pair sums (0 = skip)")
    ap.add_argument("--kernel", default=None,
                    choices=["laplace_fp32", "laplace_fp64", "laplace_ff", "laplace_fmm", "stokes_fp32",
                             "stokes_fp64", "stokes_ff", "stokes_fmm", "stokes_fmm_large", "stokes_fp32_large"],
                    help="time one operator application (pair sum + epilogue) instead of solves; "
                         "Laplace on the 100-star workload, Stokes on the 400-ellipse workload")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(rank: int):
    """Each rank solves its own replica: the 100-star workload with a rank seed."""
    return synth.star_grid(seed=1000 + rank)


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's (a no-op without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank did `steps` units in at most `seconds`."""
    return world * steps / seconds


# ---------------------------------------------------------------------------
# CPU oracle baseline: the full solve of the benchmark workload
# ---------------------------------------------------------------------------
def oracle_full_solve(n_stars: int = 100):
    """Time the FP64 oracle, as it stands, on the benchmark workload: one complete
    oracle.laplace.solve (dense Nystrom assembly, LU with partial pivoting,
    potentials at the interior points) of the 100-star problem (M = 25,600;
    n_stars < 100: the first rows of the same grid, used only to warm up)."""
    from oracle import laplace

    g = synth.star_grid(seed=1000) if n_stars >= 100 else synth.star_grid(seed=1000, rows=4, cols=n_stars // 4)
    t0 = time.perf_counter()
    res = laplace.solve(g, g["q"])
    return dict(seconds=time.perf_counter() - t0, M=int(g["x"].size), phi=res["phi"])


def oracle_single_core_seconds():
    """The same full oracle solve with one BLAS thread, in a child process (the
    thread count of OpenBLAS is fixed when numpy is first imported)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_full_solve(); print(json.dumps({'seconds': r['seconds']}))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["seconds"]


def stored_oracle(name: str):
    """The oracle's solution of a full-size workload as stored in tests/golden
    (written by tests/golden/make_fullsize.py, which calls only the oracle)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            try:
                rows.append([float(x) for x in line.split()])
            except ValueError:
                pass
    return np.array(rows).reshape(-1)


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def fmm_solves(bie, ctx, gd, kind, load, out, order, steps, tune, stream=None):
    """Float-float-refined solves with FMM pair sums of the given order: the
    default schedule (leaf population 24, inner order ceil(p/2)) and, with
    tune, the schedule bie_tune_fmm keeps; mean ms of `steps` solves each."""
    import torch

    fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
    opts = bie.make_opts(precision=bie.MIXED_FF, fmm_order=order)

    def timed():
        rc, info = fn(ctx, gd, load, out, opts=opts, stream=stream)
        assert rc == bie.OK, (rc, ctx.last_error())
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, info = fn(ctx, gd, load, out, opts=opts, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            assert rc == bie.OK
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms)), info, out.cpu().numpy()

    res = {"order": order}
    ms, info, x = timed()
    res["default_schedule"] = {"leaf_nodes": 24, "inner_order": (order + 1) // 2, "ms_per_solve": ms,
                               "iters": info["iters"]}
    if tune:
        rc, leaf, inner, _ = bie.tune_fmm(ctx, gd, kind, load, opts, stream=stream)
        assert rc == bie.OK, ctx.last_error()
        ms, info, x = timed()
        res["tuned_schedule"] = {"leaf_nodes": leaf, "inner_order": inner, "ms_per_solve": ms,
                                 "iters": info["iters"]}
    res["solves_per_s"] = 1e3 / ms
    return res, x


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=cpu_cores())
    except Exception:
        return cpu_cores()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def run_reference(args, rank, world):
    """The oracle arm: the FP64 CPU oracle, as it stands, on the host cores.  Every
    timed step is one complete oracle solve of the benchmark workload (about 43 s
    on 16 Grace cores); the warm-up steps solve the first 16 stars only (they
    load the libraries and start the BLAS threads)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_full_solve(16)
    secs = []
    for _ in range(args.steps):
        r = oracle_full_solve()
        secs.append(r["seconds"])
    value = len(secs) / sum(secs)
    ref = stored_oracle("stars100_M25600_elastance.txt")
    sample = ("the full workload every step: oracle.laplace.solve of the 100 stars (M = 25,600: dense "
              "Nystrom assembly, LU with partial pivoting, potentials), FP64, numpy/scipy")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "M": 25600, "N": 100, "nodes_per_body": 256,
                                        "tol": 1e-12, "precision": "f64 dense LU",
                                        "parallelism": f"replicas x{world}"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": blas_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_vs_stored_solution": rel_err(r["phi"], ref) if ref is not None else None,
    }))


def run_serving(args, rank, local):
    """Served stream: Poisson arrivals of mixed elastance/mobility requests
    (1..64 bodies of 64/128/256 nodes, ellipses or stars) through bie_server.
    Phase 1 queues every request at once (saturated solves/s); phase 2 submits
    at 80% of that rate with exponential gaps and reports latency percentiles
    (submit to completion, host clock)."""
    import threading

    import torch

    from paper_1507_05925_gb300 import bie

    rng = np.random.default_rng(3000 + rank)
    reqs = [synth.random_request(rng) for _ in range(args.serve_requests)]
    host = []
    for g in reqs:
        geom = {k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
        load = np.ascontiguousarray(g["q"] if g["kind"] == 0 else g["FT"].reshape(-1))
        n = g["body_start"].size - 1
        host.append((g["kind"], geom, load, np.empty(n if g["kind"] == 0 else 3 * n)))
    _, hbm_total = torch.cuda.mem_get_info(local)
    cap = int(args.serve_hbm_fraction * hbm_total)
    srv = bie.Server(local, workers=args.serve_workers, hbm_cap_bytes=cap)
    opts = bie.make_opts(precision=bie.MIXED_FF)

    def submit(i):
        kind, geom, load, out = host[i]
        t = srv.submit(kind, geom, load, out, opts=opts)
        if t <= 0:
            raise RuntimeError(f"request {i} rejected: {t}")
        return t

    for i in range(min(32, len(host))):  # warm-up
        srv.wait(submit(i))
    t0 = time.perf_counter()
    tickets = [submit(i) for i in range(len(host))]
    lat_sat = []
    for t in tickets:
        rc, _, sec = srv.wait(t)
        if rc < 0:
            raise RuntimeError(f"served solve failed: {rc}")
        lat_sat.append(sec)
    sat_s = time.perf_counter() - t0
    sat_rate = len(host) / sat_s

    def poisson(frac, seed):
        """Arrivals at frac x the saturated rate (exponential gaps); returns latencies."""
        rate = frac * sat_rate
        gaps = np.random.default_rng(seed).exponential(1.0 / rate, len(host))
        tickets = [None] * len(host)

        def producer():
            t_next = time.perf_counter()
            for i in range(len(host)):
                t_next += gaps[i]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = submit(i)

        th = threading.Thread(target=producer)
        t0 = time.perf_counter()
        th.start()
        lat = []
        for i in range(len(host)):
            while tickets[i] is None:
                time.sleep(0.0002)
            rc, _, sec = srv.wait(tickets[i])
            if rc < 0:
                raise RuntimeError(f"served solve failed: {rc}")
            lat.append(sec)
        th.join()
        wall = time.perf_counter() - t0
        return {"arrival_rate_per_s": rate, "solves_per_s": len(host) / wall,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99))}

    sweep = {f"poisson_{int(round(100 * f))}pct": poisson(f, 4000 + rank + int(100 * f)) for f in (0.5, 0.8, 0.95)}
    st = srv.stats()
    srv.close()
    batched = None
    if args.serve_batch > 1:
        # the same saturated stream with queued requests solved in batches
        srv = bie.Server(local, workers=args.serve_workers, hbm_cap_bytes=cap)
        srv.batching(args.serve_batch)
        for i in range(min(32, len(host))):  # warm-up
            srv.wait(submit(i))
        nb0 = srv.batching()
        t0 = time.perf_counter()
        tickets = [submit(i) for i in range(len(host))]
        lat_b = []
        for t in tickets:
            rc, _, sec = srv.wait(t)
            if rc < 0:
                raise RuntimeError(f"served solve failed: {rc}")
            lat_b.append(sec)
        bat_s = time.perf_counter() - t0
        batched = {"max_batch": args.serve_batch, "solves_per_s": len(host) / bat_s, "seconds": bat_s,
                   "batched_solves": srv.batching() - nb0, "p50_ms": 1e3 * float(np.percentile(lat_b, 50)),
                   "p99_ms": 1e3 * float(np.percentile(lat_b, 99)), "peak_inflight_bytes": srv.stats()["peak_inflight_bytes"]}
        srv.close()
    M = [g["x"].size for g in reqs]
    return {
        "requests": len(host), "workers": args.serve_workers, "hbm_cap_bytes": cap,
        "precision": "mixed_ff", "elastance": int(sum(1 for g in reqs if g["kind"] == 0)),
        "mobility": int(sum(1 for g in reqs if g["kind"] == 1)), "mean_nodes": float(np.mean(M)),
        "max_nodes": int(max(M)),
        "hbm_cap_fraction": args.serve_hbm_fraction,
        "saturated": {"solves_per_s": sat_rate, "seconds": sat_s,
                      "p50_ms": 1e3 * float(np.percentile(lat_sat, 50)),
                      "p99_ms": 1e3 * float(np.percentile(lat_sat, 99))},
        **sweep,
        "peak_inflight_bytes": st["peak_inflight_bytes"],
        "saturated_batched": batched,
    }


def run_batched(args, rank, local):
    """Batched solves (elastance_solve_batch / mobility_solve_batch): independent
    problems solved as one block-diagonal system.  (1) Four-disc problems (4
    discs x 128 nodes, M = 512), inputs resident on the device, batches of
    1..128; (2) the served request mix (1..64 bodies of 64/128/256 nodes),
    grouped by kind into batches of args.batch_size, inputs and outputs in host
    memory (copies inside the timed region, as for the server).  Host clock
    around synchronised calls: every batch call ends with a device-to-host read
    of its status."""
    import torch

    from paper_1507_05925_gb300 import bie

    dev = torch.device("cuda", local)
    ctx = bie.Context(local)
    opts = bie.make_opts(precision=bie.MIXED_FF)
    out = {"precision": "mixed_ff", "four_discs_M512": {}}
    rng = np.random.default_rng(5000 + rank)
    for kind, name in ((0, "elastance"), (1, "mobility")):
        fn = bie.elastance_solve_batch if kind == 0 else bie.mobility_solve_batch
        per = {}
        for P in (1, 8, 32, 128):
            geoms, loads, outs = [], [], []
            for i in range(P):
                g = synth.four_discs(seed=i)
                geoms.append({k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev)
                              for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")})
                ld = synth.charges(4, rng) if kind == 0 else synth.forces_torques(4, rng).reshape(-1)
                loads.append(torch.from_numpy(np.ascontiguousarray(ld)).to(dev))
                outs.append(torch.empty_like(loads[-1]))
            for _ in range(3):
                rc, infos, _ = fn(ctx, geoms, loads, outs, opts=opts)
                info = infos[0]
            reps = max(3, 512 // P)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                rc, infos, _ = fn(ctx, geoms, loads, outs, opts=opts)
                info = infos[0]
                if rc < 0:
                    raise RuntimeError(f"batched solve failed: {rc} {ctx.last_error()}")
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            per[str(P)] = {"solves_per_s": P / dt, "ms_per_batch": 1e3 * dt, "iters": info["iters"],
                           "refinements": info["refinements"]}
        out["four_discs_M512"][name] = per
    # the served request mix, in batches of one kind
    rng = np.random.default_rng(3000 + rank)
    reqs = [synth.random_request(rng) for _ in range(args.batch_requests)]
    t_all, n_all, iters = 0.0, 0, []
    for kind in (0, 1):
        fn = bie.elastance_solve_batch if kind == 0 else bie.mobility_solve_batch
        mine = [g for g in reqs if g["kind"] == kind]
        groups = [mine[i:i + args.batch_size] for i in range(0, len(mine), args.batch_size)]
        host = []
        for grp in groups:
            geoms = [{k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
                     for g in grp]
            loads = [np.ascontiguousarray(g["q"] if kind == 0 else g["FT"].reshape(-1)) for g in grp]
            host.append((geoms, loads, [np.empty(ld.size) for ld in loads]))
        fn(ctx, *host[0], opts=opts)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for geoms, loads, outs in host:
            rc, infos, _ = fn(ctx, geoms, loads, outs, opts=opts)
            info = infos[0]
            if rc < 0:
                raise RuntimeError(f"batched solve failed: {rc} {ctx.last_error()}")
            iters.append(info["iters"])
        torch.cuda.synchronize()
        t_all += time.perf_counter() - t0
        n_all += len(mine)
    out["served_mix"] = {"requests": n_all, "batch_size": args.batch_size, "solves_per_s": n_all / t_all,
                         "seconds": t_all, "median_iters": float(np.median(iters)),
                         "note": "same request generator and seed as the serving section; host inputs"}
    ctx.close()
    return out


def run_four_discs(args, rank, local):
    """The small elastance case (4 discs x 128 nodes, M = 512, GMRES tol 1e-12):
    solves/s one at a time with inputs on the device, FP64 GMRES (block-Jacobi
    preconditioned) and the mixed-precision paths; latency bound."""
    import torch

    from paper_1507_05925_gb300 import bie

    g = synth.four_discs(seed=0)
    dev = torch.device("cuda", local)
    gd = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev) for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    gd["body_start"] = torch.from_numpy(g["body_start"]).to(dev)
    q = torch.from_numpy(g["q"]).to(dev)
    phi = torch.empty(4, dtype=torch.float64, device=dev)
    ctx = bie.Context(local)
    stream = torch.cuda.Stream(device=dev)
    out = {}
    for name, prec in (("fp64", bie.FP64), ("mixed", bie.MIXED), ("mixed_ff", bie.MIXED_FF)):
        opts = bie.make_opts(precision=prec)
        for _ in range(3):
            rc, info = bie.elastance_solve(ctx, gd, q, phi, opts=opts, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.four_disc_steps):
            rc, info = bie.elastance_solve(ctx, gd, q, phi, opts=opts, stream=stream)
            assert rc == bie.OK
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.four_disc_steps
        out[name] = {"solves_per_s": 1.0 / dt, "ms_per_solve": 1e3 * dt, "iters": info["iters"],
                     "rel_residual": info["rel_residual"]}
    ctx.close()
    return out


def run_large(args, rank, local):
    """Mobility of 10,000 ellipses (M = 640,000): refinement with FMM pair sums
    (order fmm_order for residuals, half for the inner solves)."""
    import torch

    from paper_1507_05925_gb300 import bie

    g = synth.ellipse_lattice(seed=5000 + rank)
    dev = torch.device("cuda", local)
    gd = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev) for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    gd["body_start"] = torch.from_numpy(g["body_start"]).to(dev)
    N = g["body_start"].size - 1
    FT = torch.from_numpy(g["FT"].reshape(-1)).to(dev)
    UW = torch.empty(3 * N, dtype=torch.float64, device=dev)
    ctx = bie.Context(local)
    opts = bie.make_opts(precision=bie.MIXED_FF, fmm_order=args.fmm_order)
    stream = torch.cuda.Stream(device=dev)  # capturable: the GMRES iterations replay as CUDA graphs

    def timed_solves():
        rc, info = bie.mobility_solve(ctx, gd, FT, UW, opts=opts, stream=stream)
        assert rc == bie.OK, (rc, ctx.last_error())
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.large_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, info = bie.mobility_solve(ctx, gd, FT, UW, opts=opts, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            assert rc == bie.OK
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms)), info

    ms_default, info_default = timed_solves()
    out = {"workload": "ellipses10000_M640000 (hexagonal lattice, area fraction %.2f)" % g["area_fraction"],
           "M": int(g["x"].size), "fmm_order": args.fmm_order, "precision": "mixed_ff",
           "default_schedule": {"leaf_nodes": 24, "inner_order": (args.fmm_order + 1) // 2,
                                "seconds_per_solve": ms_default / 1e3, "info": info_default}}
    ms, info = ms_default, info_default
    if not args.no_tune:
        # the FMM schedule (leaf population, inner order) tuned by timing whole solves
        rc, leaf, inner, tms = bie.tune_fmm(ctx, gd, 1, FT, opts, stream=stream)
        assert rc == bie.OK, ctx.last_error()
        ms, info = timed_solves()
        out["tuned_schedule"] = {"leaf_nodes": leaf, "inner_order": inner, "seconds_per_solve": ms / 1e3,
                                 "info": info}
    ctx.close()
    out.update({"seconds_per_solve": ms / 1e3, "solves_per_s": 1e3 / ms, "info": info})
    return out


def run_mobility(args, rank, local):
    """Mobility of 400 ellipses (M = 51,200, direct pair sums): FP32 inner
    solves with a float-float residual (mixed_ff) and with FP64 residuals
    (mixed), split counts tuned first (bie_tune) unless --no-tune."""
    import torch

    from paper_1507_05925_gb300 import bie

    g = synth.ellipse_suspension(seed=2000 + rank)
    dev = torch.device("cuda", local)
    gd = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev) for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    gd["body_start"] = torch.from_numpy(g["body_start"]).to(dev)
    N = g["body_start"].size - 1
    FT = torch.from_numpy(np.ascontiguousarray(g["FT"].reshape(-1))).to(dev)
    UW = torch.empty(3 * N, dtype=torch.float64, device=dev)
    ctx = bie.Context(local)
    tuning = None
    if not args.no_tune:
        tuning = {}
        for name, prec in (("stokes_fp32", bie.MIXED), ("stokes_ff", bie.MIXED_FF)):
            rc, S, tms = bie.tune(ctx, gd, bie.STOKES, prec)
            assert rc == bie.OK, ctx.last_error()
            tuning[name] = {"splits": S, "ms_per_application": tms}
    out = {"workload": "ellipses400_M51200", "M": int(g["x"].size), "pair_sum_tuning": tuning}
    # the oracle's solution of this workload (seed 2000 only: rank 0)
    ref = stored_oracle("ellipses400_M51200_mobility.txt") if rank == 0 else None
    for name, prec, steps in (("mixed_ff", bie.MIXED_FF, args.mobility_steps), ("mixed", bie.MIXED, 1)):
        if steps <= 0:
            continue
        opts = bie.make_opts(precision=prec)
        rc, info = bie.mobility_solve(ctx, gd, FT, UW, opts=opts)  # warm-up
        assert rc == bie.OK, (rc, ctx.last_error())
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rc, info = bie.mobility_solve(ctx, gd, FT, UW, opts=opts)
            e1.record()
            torch.cuda.synchronize()
            assert rc == bie.OK
            ms.append(e0.elapsed_time(e1))
        out[name] = {"solves_per_s": 1e3 / float(np.mean(ms)), "ms_per_solve": float(np.mean(ms)), "steps": steps,
                     "info": info}
        if ref is not None:
            out[name]["oracle_rel_error"] = rel_err(UW.cpu().numpy(), ref)
    if args.mobility_fmm_order > 0:
        # the same workload with FMM pair sums (the quadtree's O(M) work wins at this size)
        res, x = fmm_solves(bie, ctx, gd, 1, FT, UW, args.mobility_fmm_order, args.mobility_steps, not args.no_tune)
        if ref is not None:
            res["oracle_rel_error"] = rel_err(x, ref)
        out["mixed_ff_fmm"] = res
    ctx.close()
    return out


def run_kernel(args, local):
    """Operator applications only (for kernel timing and ncu captures)."""
    import torch

    from paper_1507_05925_gb300 import bie, build

    build.build()
    parts = args.kernel.split("_")
    kind_name, prec_name = parts[0], parts[1]
    kind = bie.LAPLACE if kind_name == "laplace" else bie.STOKES
    fmm = prec_name == "fmm"
    prec = {"fp32": bie.MIXED, "fp64": bie.FP64, "ff": bie.MIXED_FF, "fmm": bie.FP64}[prec_name]
    if parts[-1] == "large":
        g = synth.ellipse_lattice(seed=5000)
    else:
        g = synth.star_grid(seed=1000) if kind == bie.LAPLACE else synth.ellipse_suspension(seed=2000)
    dev = torch.device("cuda", local)
    gd = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev) for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    gd["body_start"] = torch.from_numpy(g["body_start"]).to(dev)
    n = g["x"].size * (kind + 1)
    v = torch.randn(n, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    ctx = bie.Context(local)
    splits = None
    if not fmm and not args.no_tune:
        # the split count the solves use after tuning (--splits S: install S
        # untimed, so that no tuning launches come before the timed ones)
        rc, splits, _ = bie.tune(ctx, gd, kind, prec, splits=args.splits)
        assert rc == bie.OK, ctx.last_error()

    def apply():
        if fmm:
            rc = bie.apply_operator_fmm(ctx, gd, kind, args.fmm_order, v, out)
        else:
            rc = bie.apply_operator(ctx, gd, kind, prec, v, out)
        assert rc == bie.OK, ctx.last_error()

    for _ in range(args.warmup):
        apply()
    torch.cuda.synchronize()
    if fmm:  # whole operator application (tree build included), CUDA events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            apply()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        M = g["x"].size
        print(json.dumps({"kernel": args.kernel, "order": args.fmm_order, "M": M, "ms_per_apply": ms,
                          "equivalent_pairs_per_s": M * (M - 1) / (ms / 1e3)}))
        ctx.close()
        return
    ctx.profile(True)
    for _ in range(args.steps):
        apply()
    torch.cuda.synchronize()
    key = kind_name + "_" + prec_name
    prof = ctx.profile(False)[key]
    ms = prof["ms"] / max(prof["launches"], 1)
    flops = FLOPS_PER_PAIR[kind_name] * prof["pairs"] / max(prof["launches"], 1)
    print(json.dumps({"kernel": args.kernel, "M": g["x"].size, "launches": prof["launches"], "splits": splits,
                      "ms_per_launch": ms, "pairs_per_s": prof["pairs"] / (prof["ms"] / 1e3),
                      "tflops": flops / (ms / 1e3) / 1e12}))
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel:
        run_kernel(args, local)
        return
    if args.only_large or args.only_serving or args.only_batched:  # one section alone (profiling, tuning)
        from paper_1507_05925_gb300 import build
        build.build()
        if args.only_large:
            print(json.dumps({"large_mobility": run_large(args, rank, local)}))
        elif args.only_batched:
            print(json.dumps({"batched": run_batched(args, rank, local)}))
        else:
            print(json.dumps({"serving": run_serving(args, rank, local)}))
        return
    import torch

    from paper_1507_05925_gb300 import bie, build

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = workload(rank)
    N, M = g["body_start"].size - 1, g["x"].size
    gd = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(dev) for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    gd["body_start"] = torch.from_numpy(g["body_start"]).to(dev)
    q = torch.from_numpy(g["q"]).to(dev)
    phi = torch.empty(N, dtype=torch.float64, device=dev)
    ctx = bie.Context(local)
    # a stream of our own (the legacy default stream cannot be captured, so the
    # library would not replay its GMRES iterations as CUDA graphs there)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    head_prec = bie.MIXED_FF if args.precision == "mixed_ff" else bie.MIXED
    other_prec = bie.MIXED if head_prec == bie.MIXED_FF else bie.MIXED_FF
    mixed = bie.make_opts(precision=head_prec)
    other = bie.make_opts(precision=other_prec)
    fp64 = bie.make_opts(precision=bie.FP64)
    fp64_noprec = bie.make_opts(precision=bie.FP64, precond=bie.PRECOND_NONE)

    def solve(opts):
        rc, info = bie.elastance_solve(ctx, gd, q, phi, opts=opts, stream=stream)
        if rc != bie.OK:
            raise RuntimeError(f"solve failed: {rc} {ctx.last_error()} {info}")
        return info

    # measured arithmetic peaks of this GPU (the roofline denominators)
    peaks = bie.measure_alu_peaks(local)
    # split plans of the headline shape tuned by timing (bie_tune), before the
    # warm-up: the FP32 inner pair sums and the float-float residual
    tuning = None
    if not args.no_tune:
        tuning = {}
        for name, prec in (("laplace_fp32", bie.MIXED), ("laplace_ff", bie.MIXED_FF)):
            rc, S, tms = bie.tune(ctx, gd, bie.LAPLACE, prec, stream=stream)
            if rc != bie.OK:
                raise RuntimeError(f"bie_tune failed: {rc} {ctx.last_error()}")
            tuning[name] = {"splits": S, "ms_per_application": tms}
    # clocks are sampled from the warm-up through the timed region (a short
    # region alone would give nvidia-smi too few samples)
    cs = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        info = solve(mixed)
    torch.cuda.synchronize()

    def timed(opts, steps, profile):
        """Solves on `stream`, each bracketed by CUDA events recorded on it, the
        L2 flushed (on the same stream) before each, outside the events."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            ctx.profile(True)
        infos = []
        for e0, e1 in evs:
            with torch.cuda.stream(stream):
                flush.zero_()
            e0.record(stream)
            infos.append(solve(opts))
            e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile(False) if profile else None
        if dist is not None:
            dist.barrier()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        return ms, infos, prof

    # the headline: GMRES iterations replayed as CUDA graphs (no per-launch timing)
    ms, infos, _ = timed(mixed, args.steps, False)
    phi_mixed = phi.cpu().numpy()
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = job_rate(world, args.steps, total_ms / 1000.0)
    # the same solves again with per-launch pair-sum timing (no graphs): kernel
    # times for the roofline, launch count, shares of the step
    ms_p, _, prof = timed(mixed, args.steps, True)
    cs.__exit__(None, None, None)
    clocks = cs.summary()

    # the other mixed-precision residual and the FP64 GPU path on the same workload
    for _ in range(2):
        solve(other)
    ms_o, infos_o, _ = timed(other, args.steps, False)
    phi_other = phi.cpu().numpy()
    other_rate = len(ms_o) / (sum(ms_o) / 1000.0)
    ms64, infos64, prof64 = timed(fp64, args.fp64_steps, True)
    phi64 = phi.cpu().numpy()
    fp64_rate = len(ms64) / (sum(ms64) / 1000.0)
    ms64n, infos64n, _ = timed(fp64_noprec, 1, False)
    fp64_noprec_rate = len(ms64n) / (sum(ms64n) / 1000.0)
    ref_phi = stored_oracle("stars100_M25600_elastance.txt")
    oracle_err = None
    if ref_phi is not None and ref_phi.size == N and rank == 0:
        oracle_err = {args.precision: rel_err(phi_mixed, ref_phi),
                      ("mixed" if other_prec == bie.MIXED else "mixed_ff"): rel_err(phi_other, ref_phi),
                      "fp64": rel_err(phi64, ref_phi),
                      "note": "||phi - phi_oracle|| / ||phi_oracle||, oracle = dense LU of the same system "
                              "(tests/golden/stars100_M25600_elastance.txt)"}

    # the same workload with FMM pair sums (tuned schedule), beside the headline's direct pair sums
    fmm_alt = None
    if args.headline_fmm_order > 0:
        fmm_alt, x = fmm_solves(bie, ctx, gd, 0, q, phi, args.headline_fmm_order, max(3, min(args.steps, 10)),
                                not args.no_tune, stream)
        if ref_phi is not None and ref_phi.size == N and rank == 0:
            fmm_alt["oracle_rel_error"] = rel_err(x, ref_phi)

    # end to end through the C ABI with host (pinned) buffers (headline precision): the library copies
    # the geometry and charges in and the potentials out inside the timed call
    host = {k: torch.from_numpy(np.ascontiguousarray(g[k])).pin_memory() for k in
            ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
    qh = torch.from_numpy(g["q"]).pin_memory()
    phih = torch.empty(N, dtype=torch.float64).pin_memory()
    h2d = sum(int(t.numel() * t.element_size()) for t in host.values()) + qh.numel() * 8
    d2h = phih.numel() * 8
    bie.elastance_solve(ctx, host, qh, phih, opts=mixed, stream=stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        rc, _ = bie.elastance_solve(ctx, host, qh, phih, opts=mixed, stream=stream)
        assert rc == bie.OK
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_rate = job_rate(world, args.e2e_steps, e2e_s)
    assert np.array_equal(phih.numpy(), phi_mixed), "host and device paths disagree"

    # dominant kernel of the timed mixed-precision solves, against the measured
    # FP32 peak (the better of scalar and packed FMA)
    fp32_peak = max(peaks["fp32_ffma_tflops"], peaks["fp32_ffma2_tflops"])
    fp64_peak = peaks["fp64_dfma_tflops"]
    launches = prof.pop("kernel_launches")
    prof64.pop("kernel_launches")
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    kind = dname.split("_")[0]
    is32 = not dname.endswith("fp64")
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    pairs_per_launch = d["pairs"] / max(d["launches"], 1)
    achieved = FLOPS_PER_PAIR[kind] * pairs_per_launch / (per_launch_ms / 1e3) / 1e12
    peak = fp32_peak if is32 else fp64_peak

    def rate(p):
        return p["pairs"] / (p["ms"] / 1e3) if p["ms"] > 0 else None
    pair_rate32 = rate(prof["laplace_fp32"])
    pair_rate64 = rate(prof64["laplace_fp64"])
    pair_rate_ff = rate(prof["laplace_ff"])
    kernel_share = {k: round(v["ms"] / sum(ms_p), 4) for k, v in prof.items() if v["ms"] > 0}
    # the pair kernel's own ALU bound, from its far-pair loop: the directed kernel
    # needs 7 FP32 lane operations and one MUFU reciprocal a pair, the
    # symmetric one (tile pairs, one reciprocal for both directions) 5.5 and 0.5
    sym = bool(tuning and tuning["laplace_fp32"]["splits"] < 0) if tuning else M >= 8960
    ops_pair, mufu_pair = (5.5, 0.5) if sym else (7.0, 1.0)
    lane_ops = fp32_peak * 1e12 / 2.0
    pipe_bound_pairs = min(lane_ops / ops_pair, peaks["mufu_rcp_tops"] * 1e12 / mufu_pair)

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32 pair sums, float-float residual, f64 Krylov" if head_prec == bie.MIXED_FF
                  else "f32 pair sums, f64 residual, f64 Krylov"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": M, "N": N, "nodes_per_body": 256, "tol": 1e-12,
                   "precision": args.precision, "l2": "flushed (256 MB write) before every step, outside the events",
                   "graphs": "GMRES iterations replayed as CUDA graphs (a stream of its own)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "residual_certified_by": ("float-float pair sums (about 48 bits), then FP32 residual updates with "
                                  "their error bound" if head_prec == bie.MIXED_FF else "FP64 pair sums"),
        ("mixed_fp64_residual_solves_per_s" if other_prec == bie.MIXED else "mixed_ff_residual_solves_per_s"):
            other_rate,
        "fp64_solves_per_s": fp64_rate,
        "fp64_unpreconditioned_solves_per_s": fp64_noprec_rate,
        "mixed_over_fp64": value / world / fp64_rate,
        "oracle_rel_error": oracle_err,
        "fmm_alternative": fmm_alt,
        "pair_interactions_per_s": {"laplace_fp32": pair_rate32, "laplace_ff": pair_rate_ff,
                                    "laplace_fp64": pair_rate64},
        "solve_info": {args.precision: infos[-1], "other_mixed": infos_o[-1], "fp64": infos64[-1],
                       "fp64_unpreconditioned": infos64n[-1]},
        "kernel_share_of_step": kernel_share,
        "profiled_ms_per_step": sum(ms_p) / len(ms_p),
        "pair_sum_tuning": tuning,
        "gpu_launches": launches,
        "e2e": {"value": e2e_rate, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "measured_peaks": peaks,
        "roofline": {"bound": "alu", "kernel": f"pair sum {dname}", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": DRAM_BYTES_PER_LAUNCH.get(dname),
                     "traffic_note": "DRAM bytes per launch from ncu (inputs L2-resident)",
                     "peak_note": ("FP32: measured on this GPU by bie_measure_alu_peaks (FFMA/FFMA2 chains on "
                                   "every SM), FMA = 2 flop" if is32 else
                                   "FP64: measured on this GPU by bie_measure_alu_peaks (DFMA chains)"),
                     "flops_per_pair": FLOPS_PER_PAIR[kind], "launch_ms": per_launch_ms,
                     "pipe_bound_pairs_per_s": pipe_bound_pairs,
                     "frac_of_pipe_bound": (pairs_per_launch / (per_launch_ms / 1e3)) / pipe_bound_pairs,
                     "pair_kernel": "symmetric (k_pair32s)" if sym else "directed (k_pair32)",
                     "pipe_bound_note": (f"far pairs: {ops_pair} FP32 lane operations + {mufu_pair} MUFU rcp each, "
                                         "at the measured FFMA and MUFU rates")},
        "clocks": clocks,
    }
    if args.four_disc_steps > 0:
        out["four_discs_M512"] = run_four_discs(args, rank, local)
    if args.serve_requests > 0:
        out["serving"] = run_serving(args, rank, local)
    if args.batch_requests > 0:
        out["batched"] = run_batched(args, rank, local)
    if args.mobility_steps > 0:
        out["mobility_ellipses400"] = run_mobility(args, rank, local)
    if args.large_steps > 0:
        out["large_mobility"] = run_large(args, rank, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_full_solve()
        out["cpu_baseline"] = {"value": 1.0 / r["seconds"], "unit": "solves/s", "cores": blas_threads(),
                               "kind": "oracle",
                               "sample": ("the full workload: one oracle.laplace.solve of the 100 stars (M = 25,600: "
                                          f"dense assembly, LU, potentials) in {r['seconds']:.1f} s")}
        if args.cpu_1core:
            out["cpu_baseline"]["single_core_seconds"] = oracle_single_core_seconds()
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
