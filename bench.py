#!/usr/bin/env python
"""Benchmark of the hot path: one bilevel-hypergradient pass per step.

Workload (the FWI-step geometry): 128 x 128 unit square, omega in {5, 10, 15}, 16
top-row sources, 32 surface receivers, alpha = alpha0 = 1e-3, mu = 1e-6; training model
m' = 1/c'^2 with c' = 1 + 0.3 g (Gaussian random field, correlation length 0.1, seed 2 +
rank), lower-level reconstruction stood in for by m' smoothed with sigma = 4h.  One
step runs every row of the path: assemble, line factors of A(m_fwi) and A(m'),
point sources, data solves, forward solves, misfit, adjoint solves, gradient, PCG
with 10 iterations (11 Hessian products, 2 solve batches each) preconditioned by P2,
the tau solve and the hypergradient reductions.  Metric: Helmholtz right-hand-side
solves per second, every solve delivered at relative residual <= 1e-10 (mixed) or
by the FP64 factor (fp64).

Multi-GPU (torchrun): every rank owns its own training model (weak scaling); no
collective touches the data path, only the timing max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 128
N_CG = 10
METRIC = "Helmholtz RHS-solves/sec at 1e-8 rel. error (mixed vs FP64 GPU); p50/p99 solve latency"
UNIT = "RHS-solves/s"
WORKLOAD = "hypergrad_step_128: 128x128, omega {5,10,15}, 16 sources, 32 receivers, N_CG=10"

# FP32 SIMT peak of GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock)
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 nominal of GB300 (vendor figure; the measured cuBLAS DGEMM reached 1.05)
FP64_ALU_TFLOPS = 1.25
# DRAM bytes (read + write) per launch from an ncu capture of the same kernel build, on this
# workload (profiles/line_sweep_fp32_hypergrad_step_128.md); absent: not captured for the
# current kernel.
NCU_TRAFFIC_PER_LAUNCH: dict[str, float] = {"line_sweep_fp32": 56.67e6 + 0.75e6}


def workload(rank=0, n=N_GRID):
    import workloads as W
    return W.config_hyper_step(n, seed=2 + rank)


# ------------------------------------------------------------------ CPU oracle leg

def oracle_sample(n_cg, n=N_GRID):
    """Time the CPU oracle on one hypergradient pass of the workload (one core)."""
    from oracle import helmholtz as H
    w = workload(0, n)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    H.reset_solve_counter()
    t0 = time.perf_counter()
    H.hypergradient(g, w.m, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz, w.alpha, w.alpha, w.mu,
                    cg_fixed_iters=n_cg)
    dt = time.perf_counter() - t0
    return {"solves": H.SOLVE_COUNTER["solves"], "seconds": dt}


def run_oracle_subprocess(n_cg, reps=1, n=N_GRID):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_cg), "--oracle-reps", str(reps),
           "--n", str(n)]
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return [json.loads(l) for l in r.stdout.strip().splitlines() if l.startswith("{")]


# ------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- roofline

def kernel_cost(name, w, n_cols_per_solve):
    """Algorithmic (flops, bytes) of one launch of `name` in this workload.
    n_cols_per_solve = n_omega * n_src right-hand sides per solve batch."""
    nx, nz = w.nx, w.nz
    n_sys = len(w.omegas)
    nrhs = n_cols_per_solve // n_sys
    N = nx * nz
    if name.startswith("line_sweep"):
        esz = 8 if name.endswith("fp32") else 16
        flops = 16.0 * nx * nz * nz * nrhs * n_sys           # 2 sweeps x 8 flop per complex MAC
        # factor read twice; b read, y written and read back, result written
        byts = 2.0 * n_sys * nx * nz * nz * esz + n_sys * nrhs * N * 4.0 * esz
        return flops, byts
    if name.startswith("line_factor"):
        esz = 8 if name.endswith("fp32") else 16
        flops = 8.0 * nx * nz ** 3 * n_sys                   # one n_z^3 complex inverse per line
        byts = n_sys * nx * nz * nz * esz + n_sys * N * 16
        return flops, byts
    if name == "residual_fp64":
        return 40.0 * N * nrhs * n_sys, (48.0 * nrhs + 16.0) * N * n_sys
    if name == "refine_update":   # x', r from x, delta, b (FP32 pairs) and the diagonal
        return None, (64.0 * nrhs + 16.0) * N * n_sys
    return None, None


def roofline(name, trace, breakdown, w, peaks, prec):
    """name: the dominant kernel; trace: the timed region's trace (that kernel timed on every
    launch); breakdown: one fully traced step outside the timed region (for the share)."""
    cols = len(w.omegas) * w.acq.n_src
    st = trace.get(name)
    if not st or st["timed"] == 0:
        return None
    avg_s = st["total_ms"] / st["timed"] / 1e3
    flops, byts = kernel_cost(name, w, cols)
    total_ms = sum(v["total_ms"] for v in breakdown.values())
    st = dict(st, total_ms=breakdown[name]["total_ms"])
    out = {"kernel": name, "share": st["total_ms"] / total_ms if total_ms else None,
           "avg_launch_us": avg_s * 1e6, "launches": st["timed"]}
    traffic = NCU_TRAFFIC_PER_LAUNCH.get(name)
    if name.startswith("line_sweep") and byts is not None:
        # the solve phase streams the factor: HBM-bound at these right-hand-side counts (its
        # intensity, about nrhs/2 flop per byte, is far below the tensor ridge)
        ach = byts / avg_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": traffic,
                    "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else
                                    "fallback 6800 GB/s"),
                    "algorithmic_bytes_per_launch": byts, "algorithmic_flops_per_launch": flops,
                    "useful_tflops": flops / avg_s / 1e12})
    elif flops is not None and name.startswith("line_factor"):
        fp32 = name.endswith("fp32")
        peak = FP32_ALU_TFLOPS if fp32 else FP64_ALU_TFLOPS
        ach = flops / avg_s / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": traffic,
                    "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if fp32 else
                                    "nominal GB300 FP64 1.25 TFLOP/s"),
                    "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": byts})
    elif byts is not None:
        ach = byts / avg_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "algorithmic_bytes_per_launch": byts})
    return out


# ------------------------------------------------------------------------ main

def server_session(args):
    """Solve-server load (include/helm_server.h): a capacity run (all requests queued at
    once), then Poisson arrivals at 50 / 80 / 95 % of that capacity.  Requests: grids of the
    given sizes, 1..128 right-hand sides, 16 fixed frequencies per model in [5, 60], FP64 or
    mixed (workloads.server_requests).  Latency = submission -> X on the host, from the
    library.  Prints one JSON line."""
    import queue
    import threading
    import time

    import numpy as np
    import torch
    import workloads as W
    from paper_2301_10762_gb300 import helm as hm

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the library has no CPU path)")
    sizes = [int(x) for x in args.server_sizes.split(",")]
    cfg = W.config_server(seed=5, sizes=sizes)
    srv = hm.Server()   # 180 GiB budget, batches of up to 128 right-hand sides, 8 workers
    ids = {}
    for si, n in enumerate(sizes):
        for k, m in enumerate(cfg["m"][si]):
            ids[(si, k)] = srv.add_model(n, n, 1.0, 1.0, m)
    gen = torch.Generator().manual_seed(55)
    bpool = [torch.complex(torch.randn(128, n * n, dtype=torch.float64, generator=gen),
                           torch.randn(128, n * n, dtype=torch.float64, generator=gen)).pin_memory() for n in sizes]
    slots = [queue.Queue() for _ in sizes]   # pinned result blocks, reused
    for si, n in enumerate(sizes):
        for _ in range(12):
            slots[si].put(torch.empty(128, n * n, dtype=torch.complex128).pin_memory())

    def run(reqs, arrivals):
        done, lock, q = [], threading.Lock(), queue.Queue()

        def waiter():
            while True:
                item = q.get()
                if item is None:
                    return
                t, si, X, nrhs = item
                out = srv.wait(t)
                slots[si].put(X)
                out["nrhs"] = nrhs
                with lock:
                    done.append(out)

        ws = [threading.Thread(target=waiter) for _ in range(8)]
        for th in ws:
            th.start()
        t0 = time.perf_counter()
        for (si, k, om, prec, nrhs), ta in zip(reqs, arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            X = slots[si].get()
            t = srv.submit(ids[(si, k)], om, bpool[si][:nrhs], X[:nrhs], prec=prec, rtol=1e-10)
            q.put((t, si, X, nrhs))
        for _ in ws:
            q.put(None)
        for th in ws:
            th.join()
        wall = time.perf_counter() - t0
        lat = np.array([d["total_ms"] for d in done])
        rhs = sum(d["nrhs"] for d in done)
        return {"requests": len(done), "rhs": rhs, "seconds": round(wall, 3),
                "rhs_solves_per_s": rhs / wall, "requests_per_s": len(done) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "cache_hit_rate": float(np.mean([d["cache_hit"] for d in done])),
                "errors": sum(1 for d in done if "error" in d),
                "max_relres": float(max(d["max_relres"] for d in done))}

    cap_reqs = W.server_requests(cfg, args.server_requests, seed=50)
    cap = run(cap_reqs, np.zeros(len(cap_reqs)))
    sessions = []
    for j, load in enumerate((0.5, 0.8, 0.95)):
        rate = load * cap["requests_per_s"]
        count = max(1, int(rate * args.server_seconds))
        r = run(W.server_requests(cfg, count, seed=51 + j), W.poisson_arrivals(count, rate, seed=61 + j))
        r.update({"load": load, "rate_rps": rate})
        sessions.append(r)
    st = srv.stats()
    srv.close()
    print(json.dumps({
        "metric": "solve server: RHS-solves/s and p50/p99 request latency (arrival -> X on host) under Poisson "
                  "arrivals",
        "unit": "RHS-solves/s", "n_gpus": 1, "data": "synthetic (seeded Gaussian-random-field models)",
        "config": {"workload": "solve_server", "sizes": sizes, "models_per_size": 16, "frequencies_per_model": 16,
                   "rhs": "log-uniform 1..128", "precision": "FP64 or mixed (1/2 each), mixed refined to 1e-10",
                   "hbm_budget_GiB": 180, "max_batch_rhs": 128, "workers": 8},
        "capacity": cap, "sessions": sessions,
        "server": {k: st[k] for k in ("batches", "factor_builds", "cache_hits", "evictions", "entries",
                                      "bytes_peak", "refused")}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--ncg", type=int, default=N_CG)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--server", action="store_true",
                    help="solve-server session (Poisson arrivals) instead of the hypergradient step")
    ap.add_argument("--server-sizes", default="64,128,256")
    ap.add_argument("--server-seconds", type=float, default=10.0)
    ap.add_argument("--server-requests", type=int, default=200, help="requests of the capacity run")
    ap.add_argument("--oracle-sample", type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-reps", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_sample is not None:
        for _ in range(args.oracle_reps):
            print(json.dumps(oracle_sample(args.oracle_sample, args.n)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if args.server:
        if rank == 0:
            server_session(args)
        return

    import numpy as np
    import torch
    from paper_2301_10762_gb300 import helm as hm

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the library has no CPU path)")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    hm.load()
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))

    w = workload(rank, args.n)
    grid = (w.nx, w.nz, w.lx, w.lz)
    acq = hm.Acq(w.acq.src_xz, w.acq.rec_xz, rec_w=np.ones(w.acq.n_rec))
    mf = torch.tensor(w.m, device="cuda")
    mt = torch.tensor(w.m_true, device="cuda")
    prec = hm.HELM_MIXED if args.prec == "mixed" else hm.HELM_FP64
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(m_f, m_t, p=prec):
        return hm.bilevel_hypergrad([grid], [m_f], [m_t], acq, w.omegas, w.alpha, w.alpha, w.mu, prec=p,
                                    cg_fixed_iters=args.ncg, refine_rtol=1e-10)

    for _ in range(args.warmup):
        out = step(mf, mt)
    torch.cuda.synchronize()

    # ---- one fully traced step (outside the timed region): per-kernel device times, and the
    # dominant kernel, which alone is timed launch by launch inside the timed region (timing
    # every launch adds two event records per launch to the host's critical path)
    hm.helm_trace_reset()
    hm.helm_trace_select(None)
    hm.helm_trace_enable(True)
    step(mf, mt)
    hm.helm_trace_enable(False)
    breakdown = hm.helm_trace_read()
    dominant = max(breakdown.items(), key=lambda kv: kv[1]["total_ms"])[0]

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    sampler = ClockSampler(local_rank)
    hm.helm_trace_reset()
    hm.helm_trace_select(dominant)
    hm.helm_trace_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = hm.helm_launch_count()
    times, solves = [], 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = step(mf, mt)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        solves += out["solves"] + out["data_solves"]
    torch.cuda.synchronize()
    launches = hm.helm_launch_count() - launches0
    clocks = sampler.stop()
    hm.helm_trace_enable(False)
    trace = hm.helm_trace_read()
    hm.helm_trace_select(None)
    total = sum(times)
    if dist:
        t = torch.tensor([total, float(solves)], device="cuda", dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total, all_solves = float(tmax[0]), float(t[1])
    else:
        all_solves = float(solves)
    value = all_solves / total
    per_step_solves = solves / args.steps
    lat = sorted(times)

    # ---- end to end through the public call with host buffers (H2D + D2H in the region)
    e2e = None
    if not args.no_e2e:
        mf_h = torch.tensor(w.m).pin_memory()
        mt_h = torch.tensor(w.m_true).pin_memory()
        mf_d = torch.empty_like(mf)
        mt_d = torch.empty_like(mt)
        et, es = [], 0
        for it in range(args.warmup + max(1, args.steps)):   # the first W untimed, as in the main loop
            flush.fill_(2.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            mf_d.copy_(mf_h, non_blocking=True)
            mt_d.copy_(mt_h, non_blocking=True)
            o = step(mf_d, mt_d)           # results come back to host inside the call
            e1.record()
            e1.synchronize()
            if it >= args.warmup:
                et.append(e0.elapsed_time(e1) / 1e3)
                es += o["solves"] + o["data_solves"]
        e2e = {"value": es / sum(et), "unit": UNIT, "h2d_bytes_per_step": 2 * w.n_nodes * 8,
               "d2h_bytes_per_step": (2 + 3 * w.acq.n_rec) * 8}

    # ---- FP64 GPU path on the same workload (the comparison the metric names)
    fp64 = None
    if not args.no_fp64_compare and prec == hm.HELM_MIXED:
        step(mf, mt, hm.HELM_FP64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        o = step(mf, mt, hm.HELM_FP64)
        e1.record()
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": (o["solves"] + o["data_solves"]) / dt, "ms_per_step": dt * 1e3,
                "dpsi_dalpha_rel_diff_vs_mixed": abs(o["dpsi_dalpha"] - out["dpsi_dalpha"]) / abs(o["dpsi_dalpha"])}

    rl = roofline(dominant, trace, breakdown, w, peaks, args.prec)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            r = run_oracle_subprocess(args.ncg, 1, args.n)[0]
            cpu = {"value": r["solves"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"one full step of the workload ({r['solves']} solves, {r['seconds']:.1f} s) by the "
                             f"FP64 CPU oracle (SuperLU sparse LU), one thread"}
        except Exception as e:  # keep the GPU line even if the host leg fails
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if args.prec == "mixed" else "f64",
            "data": "synthetic (seeded Gaussian-random-field training model; Marmousi not available)",
            "config": {"workload": WORKLOAD, "precision": args.prec, "solves_per_step": per_step_solves,
                       "cg_iterations": args.ncg, "refine_rtol": 1e-10, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"one training model per GPU x{world}"},
            "latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "per": "hypergradient step"},
            "solve_latency_us": {"mean_per_rhs": 1e6 * total / max(1.0, all_solves / world)},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": rl, "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            # one fully traced step outside the timed region (every launch bracketed by events)
            "kernels_one_step": {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3)}
                                 for k, v in breakdown.items()},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args, world, rank):
    """The CPU oracle timed as the reference arm: every step is a bounded sample of the
    workload (one hypergradient pass with 2 PCG iterations, one core)."""
    if rank != 0:
        return
    n_cg = 2
    recs = run_oracle_subprocess(n_cg, args.warmup + args.steps, args.n)
    timed = recs[args.warmup:]
    tot = sum(r["seconds"] for r in timed)
    sol = sum(r["solves"] for r in timed)
    value = sol / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-random-field training model; Marmousi not available)",
        "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "sample": f"N_CG={n_cg} per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed steps, each one hypergradient pass with {n_cg} PCG "
                                   f"iterations ({timed[0]['solves']} solves), one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
