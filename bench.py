#!/usr/bin/env python
"""Benchmark of the hot path: batched Helmholtz right-hand-side solves, mixed precision
against FP64 on the GPU.

Default step (the mixed-precision workload): 256 x 256 nodes on the unit square, omega in
{5, 10, ..., 40} (8 values), 64 point sources on top-row nodes as right-hand sides, smooth
random velocity c = 1 + 2 (g - min) / (max - min) in [1, 3] (Gaussian random field,
correlation length 0.1, seed 3 + rank).  One step runs the solve path end to end on data
already in HBM: assemble A(m, w) for the 8 frequencies, factor them (block cyclic reduction,
its block products and Schur updates on the tensor cores in complex FP32), form the 64
point-source right-hand sides and solve all 512 columns, each refined with FP64-accurate
residuals to ||b - A x|| / ||b|| <= 1e-10.  Metric: right-hand-side
solves per second with the factor time included (512 per step).  The same step with FP64
factors is the comparison the metric names; the per-frequency error of sampled columns
against the CPU oracle is reported for both.

Also reported: per-solve latency (p50 / p99 of helm_solve calls on a resident factor, one
right-hand side per frequency and the full 64), the tensor-core GEMM alone at the workload's
product shapes, the bilevel-hypergradient step of the FWI-step geometry (128 x 128, omega in
{5, 10, 15}, 16 sources, 32 receivers, ten PCG iterations), the batched hypergradient over the
32 uneven training models (96^2 .. 256^2) and a short solve-server session (Poisson arrivals,
64^2 .. 256^2, FP64 and mixed).

Multi-GPU (torchrun): every rank solves its own velocity model (weak scaling); no collective
touches the data path, only the timing max over ranks and the solve count.
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

METRIC = "Helmholtz RHS-solves/sec at 1e-8 rel. error (mixed vs FP64 GPU); p50/p99 solve latency"
UNIT = "RHS-solves/s"
N_GRID = 256
REFINE_RTOL = 1e-10
SAMPLE_COLS = (0, 21, 42, 63)   # right-hand sides compared with the oracle, every frequency

# FP32 SIMT peak of GB300 from its unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop x
# 2.07 GHz (the peak of the CUDA-core line factor, which issues no tensor instructions)
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def workload(rank=0, n=N_GRID):
    import workloads as W
    return W.config_mixed(n, seed=3 + rank)


def workload_desc(w):
    return (f"mixed_{w.nx}: {w.nx}x{w.nz}, omega {{{', '.join(f'{o:g}' for o in w.omegas)}}}, "
            f"{w.acq.n_src} top-row point sources as right-hand sides, c in [1, 3] (GRF, l = 0.1), "
            f"refined to 1e-10")


# ------------------------------------------------------------------ CPU oracle leg

def _oracle_unit(args):
    """One frequency of the workload on one host core: the oracle's sparse LU of A(m, w) and
    its solve of every right-hand side.  Returns the time and the sampled columns."""
    n, seed, q, cols = args
    import numpy as np
    import workloads as W
    from oracle import helmholtz as H
    w = W.config_mixed(n, seed=seed)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    E = H.source_vectors(g, w.acq.src_xz)
    t0 = time.perf_counter()
    X = H.Factor(H.helmholtz_matrix(g, w.m, w.omegas[q])).solve(E)
    dt = time.perf_counter() - t0
    return q, dt, int(E.shape[0]), np.ascontiguousarray(X[list(cols)])


def oracle_pool_run(n, seed, reps, out_npy=None):
    """`reps` runs of the whole workload by the oracle: the frequencies are independent units,
    spread over a process pool of the allowed host cores (one thread each)."""
    import multiprocessing as mp
    import numpy as np
    import workloads as W
    n_om = len(W.config_mixed(n, seed=seed).omegas)
    cores = len(os.sched_getaffinity(0))
    procs = max(1, min(n_om, cores))
    recs = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for r in range(reps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_unit, [(n, seed, q, SAMPLE_COLS) for q in range(n_om)])
            wall = time.perf_counter() - t0
            solves = sum(x[2] for x in res)
            recs.append({"seconds": wall, "solves": solves, "cpu_seconds": sum(x[1] for x in res),
                         "procs": procs, "cores_allowed": cores})
            if out_npy and r == reps - 1:
                cols = np.stack([x[3] for x in sorted(res, key=lambda x: x[0])])   # [n_omega][len(SAMPLE_COLS)][N]
                np.save(out_npy, cols)
    return recs


def run_oracle_subprocess(n, seed, reps, out_npy=None):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-run", str(reps), "--n", str(n), "--seed", str(seed)]
    if out_npy:
        cmd += ["--oracle-out", out_npy]
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
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

def kernel_cost(name, nx, nz, n_sys, nrhs):
    """Algorithmic (flops, bytes) of one launch of `name` that covers n_sys systems of nrhs
    right-hand sides each (one factor launch covers every frequency of an operator)."""
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


# nominal dense TF32 / BF16 tensor rate of GB300 (1.1 / 2.25 PFLOP/s): the TF32 peak is the
# measured BF16 GEMM peak times this ratio
TF32_PER_BF16 = 1.1 / 2.25


def tensor_peak(peaks, sustained=True):
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    if key in peaks:
        return peaks[key] * TF32_PER_BF16, f"MEASURED_PEAKS.json {key} x 1.1/2.25 (TF32/BF16 nominal; of measured)"
    return (1700.0 if sustained else 1900.0) * TF32_PER_BF16, "fallback BF16 x 1.1/2.25 (of fallback)"


def matmul_peaks(torch):
    """cuBLAS dense matmul rates (2 n^3 flops per product) for the precisions the path touches:
    FP32 operands with TF32 tensor cores allowed, plain FP32, and FP64; best of 10 products after
    3 warm-up ones, CUDA events around each product."""
    out = {}
    cases = [("tf32", torch.float32, True, 8192), ("fp32", torch.float32, False, 8192),
             ("fp64", torch.float64, False, 4096)]
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, tf32, n in cases:
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            c = torch.empty(n, n, device="cuda", dtype=dt)
            best = float("inf")
            for it in range(13):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                if it >= 3:
                    best = min(best, e0.elapsed_time(e1))
            out[name] = {"n": n, "ms": best, "tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12}
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    return out


def roofline(name, trace, breakdown, dims, peaks):
    """name: the dominant kernel; trace: the timed region's trace (that kernel timed on every
    launch); breakdown: one fully traced step outside the timed region (for the share)."""
    st = trace.get(name)
    if not st or st["timed"] == 0:
        return None
    avg_s = st["total_ms"] / st["timed"] / 1e3
    flops, byts = kernel_cost(name, *dims)
    total_ms = sum(v["total_ms"] for v in breakdown.values())
    out = {"kernel": name, "share": breakdown[name]["total_ms"] / total_ms if total_ms else None,
           "avg_launch_us": avg_s * 1e6, "launches": st["timed"],
           # DRAM bytes of this kernel come from ncu captures committed beside the code; the bench
           # does not run under a profiler, so the live line carries none
           "traffic": None}
    hbm = peaks.get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else "fallback 6800 GB/s (of fallback)"
    if name == "zgemm_tf32x3" and st.get("flops"):
        # the tensor-core GEMM of the block-cyclic-reduction factor and solve: useful flops are
        # 8 M N K per complex product term (the library counts them per launch); the tensor pipe
        # issues three TF32 products per useful one (hi*hi + hi*lo + lo*hi)
        useful = st["flops"] / (st["total_ms"] / 1e3) / 1e12
        peak, src = tensor_peak(peaks, sustained=True)
        out.update({"bound": "tensor", "achieved": useful, "peak": peak, "unit": "TFLOP/s", "frac": useful / peak,
                    "peak_source": src, "issued_tflops": 3 * useful, "issued_frac": 3 * useful / peak,
                    "algorithmic_flops_per_launch": st["flops"] / st["timed"]})
    elif name.startswith("line_factor") and flops is not None:
        ach = flops / avg_s / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP32_ALU_TFLOPS,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                    "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": byts})
    elif byts is not None:
        ach = byts / avg_s / 1e9
        peak = hbm or 6800.0
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "peak_source": hbm_src, "algorithmic_bytes_per_launch": byts})
        if flops is not None:
            out.update({"algorithmic_flops_per_launch": flops, "useful_tflops": flops / avg_s / 1e12})
    return out


# --------------------------------------------------------------- solve server

def server_run(sizes, n_cap, seconds, loads):
    """Solve-server load (include/helm_server.h): a capacity run (n_cap requests queued at
    once), then Poisson arrivals at the given fractions of that capacity.  Requests: grids of
    the given sizes, 1..128 right-hand sides, 16 fixed frequencies per model in [5, 60], FP64
    or mixed (workloads.server_requests).  Latency = submission -> X on the host, from the
    library."""
    import queue
    import threading

    import numpy as np
    import torch
    import workloads as W
    from paper_2301_10762_gb300 import helm as hm

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

    cap_reqs = W.server_requests(cfg, n_cap, seed=50)
    cap = run(cap_reqs, np.zeros(len(cap_reqs)))
    sessions = []
    for j, load in enumerate(loads):
        rate = load * cap["requests_per_s"]
        count = max(1, int(rate * seconds))
        r = run(W.server_requests(cfg, count, seed=51 + j), W.poisson_arrivals(count, rate, seed=61 + j))
        r.update({"load": load, "rate_rps": rate})
        sessions.append(r)
    st = srv.stats()
    srv.close()
    return {"config": {"workload": "solve_server", "sizes": sizes, "models_per_size": 16, "frequencies_per_model": 16,
                       "rhs": "log-uniform 1..128", "precision": "FP64 or mixed (1/2 each), mixed refined to 1e-10",
                       "hbm_budget_GiB": 180, "max_batch_rhs": 128, "workers": 8},
            "capacity": cap, "sessions": sessions,
            "server": {k: st[k] for k in ("batches", "factor_builds", "cache_hits", "evictions", "entries",
                                          "bytes_peak", "refused")}}


def server_session(args):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the library has no CPU path)")
    sizes = [int(x) for x in args.server_sizes.split(",")]
    out = server_run(sizes, args.server_requests, args.server_seconds, (0.5, 0.8, 0.95))
    print(json.dumps(dict({"metric": "solve server: RHS-solves/s and p50/p99 request latency (arrival -> X on host) "
                                     "under Poisson arrivals", "unit": UNIT, "n_gpus": 1,
                           "data": "synthetic (seeded Gaussian-random-field models)"}, **out)), flush=True)


# ------------------------------------------------------ tensor-core GEMM alone

GEMM_SHAPES = {   # (batch, M, N, K): the two shapes of the mixed workload's block products
    "factor_256x256x256": (256, 256, 256, 256),     # Schur updates of a factor level
    "solve_256x64x256": (1024, 256, 64, 256),       # one level-0 pass of the solve: 8 freq x 128 lines
}


def gemm_kernel_bench(hm, torch, peaks, reps=10):
    """helm_zgemm_batched on its own at the workload's two product shapes (operands larger
    than L2): useful TFLOP/s (8 M N K per complex product), the tensor pipe's issued rate (three
    TF32 products per useful one) against the measured tensor peak, and the operand bytes'
    GB/s against the measured HBM bandwidth."""
    out = {}
    peak, src = tensor_peak(peaks, sustained=False)
    hbm = peaks.get("hbm_gbs", 6800.0)
    g = torch.Generator(device="cuda").manual_seed(7)
    for name, (b, M, N, K) in GEMM_SHAPES.items():
        A = torch.randn((b, M, K), dtype=torch.complex64, device="cuda", generator=g)
        Bt = torch.randn((b, N, K), dtype=torch.complex64, device="cuda", generator=g)
        C = torch.empty((b, M, N), dtype=torch.complex64, device="cuda")
        for _ in range(2):
            hm.helm_zgemm_batched(A, Bt, C=C)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hm.helm_zgemm_batched(A, Bt, C=C)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(ts)
        flops = 8.0 * M * N * K * b
        byts = 8.0 * b * (M * K + N * K + M * N)
        out[name] = {"batch": b, "M": M, "N": N, "K": K, "us": t * 1e6, "useful_tflops": flops / t / 1e12,
                     "issued_tflops": 3 * flops / t / 1e12, "issued_frac": 3 * flops / t / 1e12 / peak,
                     "gbs": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm}
        del A, Bt, C
    out["peak_tflops"] = peak
    out["peak_source"] = src
    return out


def zinv_kernel_bench(hm, torch, reps=10):
    """The batched inversion alone at the 256^2 factor's shapes: the 1024 line blocks of level 0
    (256 x 256, each through the 2 x 2 block inverse over two 128 x 128 base inversions and six
    tensor-core products) and a deep level's 8 blocks (latency of one chain).  Complex
    symmetric, diagonally dominant inputs; medians of `reps` calls, CUDA events."""
    out = {}
    g = torch.Generator(device="cuda").manual_seed(11)
    for name, (b, n) in {"level0_1024x256": (1024, 256), "deep_8x256": (8, 256), "base_1024x128": (1024, 128)}.items():
        A = torch.randn((b, n, n), dtype=torch.complex64, device="cuda", generator=g)
        A = 0.5 * (A + A.transpose(1, 2)) + 3.0 * n ** 0.5 * torch.eye(n, dtype=torch.complex64, device="cuda")
        X = torch.empty_like(A)
        for _ in range(2):
            hm.helm_zinv_batched(A, X)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hm.helm_zinv_batched(A, X)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(ts)
        flops = 8.0 * n ** 3 * b   # Gauss-Jordan inverse: ~2 n^3 complex multiply-adds
        out[name] = {"batch": b, "n": n, "us": t * 1e6, "tflops": flops / t / 1e12}
        del A, X
    return out


# -------------------------------------------------------- hypergradient step

def hypergrad_step(hm, torch, steps, warmup, rank):
    """The bilevel-hypergradient pass of the FWI-step geometry (every row of the path): time
    per step and RHS-solves per second, mixed refined to 1e-10, ten PCG iterations."""
    import numpy as np
    import workloads as W
    w = W.config_hyper_step(128, seed=2 + rank)
    grid = (w.nx, w.nz, w.lx, w.lz)
    acq = hm.Acq(w.acq.src_xz, w.acq.rec_xz, rec_w=np.ones(w.acq.n_rec))
    mf = torch.tensor(w.m, device="cuda")
    mt = torch.tensor(w.m_true, device="cuda")

    def step(p):
        return hm.bilevel_hypergrad([grid], [mf], [mt], acq, w.omegas, w.alpha, w.alpha, w.mu, prec=p,
                                    cg_fixed_iters=10, refine_rtol=REFINE_RTOL)

    out = {}
    for name, p, k in (("mixed", hm.HELM_MIXED, steps), ("fp64", hm.HELM_FP64, 1)):
        for _ in range(warmup if p == hm.HELM_MIXED else 1):
            step(p)
        torch.cuda.synchronize()
        ts, sol = [], 0
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            o = step(p)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
            sol += o["solves"] + o["data_solves"]
        out[name] = {"value": sol / sum(ts), "unit": UNIT, "ms_per_step": 1e3 * sum(ts) / len(ts), "steps": k,
                     "solves_per_step": sol // k, "dpsi_dalpha": o["dpsi_dalpha"]}
    out["workload"] = "hypergrad_step_128: 128x128, omega {5,10,15}, 16 sources, 32 receivers, N_CG=10"
    out["dpsi_dalpha_rel_diff_fp64_vs_mixed"] = abs(out["fp64"]["dpsi_dalpha"] - out["mixed"]["dpsi_dalpha"]) / abs(
        out["fp64"]["dpsi_dalpha"])
    return out


# ------------------------------------------------ batched hypergradient (C4)

def grid512_step(hm, torch, steps=2, warmup=1):
    """The metric's step on the largest grid of the solve server's workload: 512 x 512, the
    same 8 frequencies and 64 top-row sources, mixed (block cyclic reduction) refined to 1e-10,
    factor included; RHS-solves/s, per-phase times and the refinement sweeps."""
    import workloads as W
    w = W.config_mixed(512)
    acq = hm.Acq.from_workload(w.acq)
    m = torch.tensor(w.m, device="cuda")
    n_om, ns, N = len(w.omegas), w.acq.n_src, w.n_nodes
    B = torch.empty((n_om, ns, N), dtype=torch.complex128, device="cuda")
    X = torch.empty_like(B)

    def step(ev=None):
        op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, m, w.omegas)
        f = hm.helm_factor(op, hm.HELM_MIXED)
        if ev is not None:
            ev.record()
        hm.helm_sources(op, acq, B)
        _, info = hm.helm_solve(f, B, X, rtol=REFINE_RTOL, max_iter=40)
        f.close()
        op.close()
        return info

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ts, fs, its = [], [], []
    for _ in range(steps):
        e0, ef, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        info = step(ef)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
        fs.append(e0.elapsed_time(ef) / 1e3)
        its.append(info["iters"])
    t = statistics.median(ts)
    return {"workload": "mixed_512: 512x512, omega {5, 10, ..., 40}, 64 top-row point sources, refined to 1e-10",
            "value": n_om * ns / t, "unit": UNIT, "ms_per_step": 1e3 * t, "steps": steps,
            "factor_ms": 1e3 * statistics.median(fs), "refinement_sweeps": max(its),
            "max_relres": info["max_relres"]}


def hypergrad_batch(hm, torch, n_cg=20, concurrent=4):
    """The batched bilevel hypergradient of Algorithm alg:box over the uneven training set: 32
    layered-plus-inclusion models on grids n = 96 + 32 (k mod 6), omega in {3, 9, 18, 36}, 51
    sources in the well at x = 0.05 (on each model's own grid), 24 receivers at x = 0.95, fixed
    N_CG = 20, mixed, refined to 1e-10; models processed `concurrent` at a time (own streams).
    One timed pass after a warm-up pass on two models."""
    import workloads as W
    ms = W.config_hypergrad()
    grids = [(w.nx, w.nz, w.lx, w.lz) for w in ms]
    mf = [torch.tensor(w.m, device="cuda") for w in ms]
    mt = [torch.tensor(w.m_true, device="cuda") for w in ms]
    acqs = [hm.Acq.from_workload(w.acq) for w in ms]
    w0 = ms[0]
    kw = dict(prec=hm.HELM_MIXED, cg_fixed_iters=n_cg, refine_rtol=REFINE_RTOL, concurrent_models=concurrent)
    hm.bilevel_hypergrad(grids[:2], mf[:2], mt[:2], acqs[:2], w0.omegas, w0.alpha, w0.alpha, w0.mu, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = hm.bilevel_hypergrad(grids, mf, mt, acqs, w0.omegas, w0.alpha, w0.alpha, w0.mu, **kw)
    e1.record()
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    solves = out["solves"] + out["data_solves"]
    return {"workload": f"hypergrad_batch: {len(ms)} models, grids 96^2..256^2, omega {{3,9,18,36}}, "
                        f"{w0.acq.n_src} sources, 24 receivers, N_CG={n_cg}, mixed",
            "value": solves / dt, "unit": UNIT, "seconds": dt, "solves": solves, "concurrent_models": concurrent,
            "max_refine_iters": out["max_refine_iters"]}


def hypergrad_lower(hm, torch, n_models=2, n_cg=20):
    """The uneven set fed with true lower-level solutions: L-BFGS (Section 4, Wolfe line
    search) to ||grad phi|| <= 1e-10 on the first n_models models (96^2, 128^2), every phi /
    grad phi evaluation on the GPU (mixed, refined to 1e-12); then the hypergradient at those
    m_FWI (N_CG fixed).  Times the lower level (its evaluations are the method's dominant
    cost at this stage) and the hypergradient pass."""
    import workloads as W
    from paper_2301_10762_gb300 import bilevel as B
    ms = W.config_hypergrad()[:n_models]
    res = B.lower_level_set(ms)
    w0 = ms[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = hm.bilevel_hypergrad([(w.nx, w.nz, w.lx, w.lz) for w in ms], [torch.tensor(r["x"], device="cuda") for r in res],
                               [torch.tensor(w.m_true, device="cuda") for w in ms],
                               [hm.Acq.from_workload(w.acq) for w in ms], w0.omegas, w0.alpha, w0.alpha, w0.mu,
                               prec=hm.HELM_MIXED, cg_fixed_iters=n_cg, refine_rtol=REFINE_RTOL)
    e1.record()
    e1.synchronize()
    # one phi / grad phi evaluation: the forward and the adjoint solve of every (omega, source)
    lower_solves = sum(r["evals"] * 2 * len(w.omegas) * w.acq.n_src for w, r in zip(ms, res))
    lower_s = sum(r["seconds"] for r in res)
    return {"workload": f"hypergrad_lower: models 0..{n_models - 1} of the uneven set ({', '.join(f'{w.nx}^2' for w in ms)}), "
                        f"L-BFGS to ||grad phi|| <= 1e-10 from the smoothed model, then N_CG={n_cg}",
            "lower_level": [{"n": w.nx, "iters": r["iters"], "evals": r["evals"], "gnorm": r["gnorm"],
                             "seconds": r["seconds"]} for w, r in zip(ms, res)],
            "lower_rhs_solves_per_s": lower_solves / lower_s, "lower_seconds": lower_s,
            "hypergrad_seconds": e0.elapsed_time(e1) / 1e3, "unit": UNIT,
            "dpsi_dalpha": out["dpsi_dalpha"]}


# ------------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the hypergradient step and the server session")
    ap.add_argument("--server", action="store_true", help="long solve-server session instead of the solve step")
    ap.add_argument("--gemm-only", action="store_true", help="time the tensor-core GEMM alone and exit")
    ap.add_argument("--zinv-only", action="store_true", help="time the batched block inversion alone and exit")
    ap.add_argument("--matmul-peaks", action="store_true",
                    help="time torch.matmul (cuBLAS) in TF32, FP32 and FP64 and exit")
    ap.add_argument("--server-sizes", default="64,128,256")
    ap.add_argument("--server-seconds", type=float, default=10.0)
    ap.add_argument("--server-requests", type=int, default=200, help="requests of the capacity run")
    ap.add_argument("--oracle-run", type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-out", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_run is not None:
        for r in oracle_pool_run(args.n, args.seed, args.oracle_run, args.oracle_out):
            print(json.dumps(r), flush=True)
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
    if args.matmul_peaks:
        if rank == 0:
            print(json.dumps({"matmul_peaks": matmul_peaks(torch)}), flush=True)
        return
    if args.zinv_only:
        if rank == 0:
            print(json.dumps({"kernel_zinv": zinv_kernel_bench(hm, torch)}), flush=True)
        return
    if args.gemm_only:
        if rank == 0:
            print(json.dumps({"kernel_zgemm": gemm_kernel_bench(hm, torch, peaks)}), flush=True)
        return

    seed = args.seed + rank
    w = workload(rank, args.n) if args.seed == 3 else __import__("workloads").config_mixed(args.n, seed=seed)
    n_om, ns, N = len(w.omegas), w.acq.n_src, w.n_nodes
    acq = hm.Acq.from_workload(w.acq)
    m_dev = torch.tensor(w.m, device="cuda")
    prec = hm.HELM_MIXED if args.prec == "mixed" else hm.HELM_FP64
    B = torch.empty((n_om, ns, N), dtype=torch.complex128, device="cuda")
    X = torch.empty_like(B)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(p, ev=None, m=m_dev, Xout=None):
        """assemble + factor + sources + refined solve of all columns; ev: events after the factor"""
        op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, m, w.omegas)
        f = hm.helm_factor(op, p)
        if ev is not None:
            ev.record()
        hm.helm_sources(op, acq, B)
        _, info = hm.helm_solve(f, B, X if Xout is None else Xout, rtol=REFINE_RTOL, max_iter=40)
        f.close()
        op.close()
        return info

    for _ in range(args.warmup):
        step(prec)
    torch.cuda.synchronize()

    # ---- one fully traced step (outside the timed region): per-kernel device times, and the
    # dominant kernel, which alone is timed launch by launch inside the timed region
    hm.helm_trace_reset()
    hm.helm_trace_select(None)
    hm.helm_trace_enable(True)
    step(prec)
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
    times, fac_times, iters = [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, ef, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        info = step(prec, ef)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        fac_times.append(e0.elapsed_time(ef) / 1e3)
        iters.append(info["iters"])
    torch.cuda.synchronize()
    launches = hm.helm_launch_count() - launches0
    clocks = sampler.stop()
    hm.helm_trace_enable(False)
    trace = hm.helm_trace_read()
    hm.helm_trace_select(None)
    total = sum(times)
    solves = args.steps * n_om * ns
    if dist:
        t = torch.tensor([total, float(solves)], device="cuda", dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total, all_solves = float(tmax[0]), float(t[1])
    else:
        all_solves = float(solves)
    value = all_solves / total
    X_mixed_sample = X[:, list(SAMPLE_COLS)].cpu().numpy()

    # ---- end to end through the public calls with host buffers: each step copies the model from
    # pinned host memory to the device, forms the point sources from host positions and copies
    # every solution column back to pinned host memory.  As a serving loop would, the copy of step
    # k's solutions runs on a copy stream while step k + 1 computes (two result buffers); the
    # timed region spans the K steps and ends when the last copy has landed.
    e2e = None
    if not args.no_e2e:
        m_h = torch.tensor(w.m).pin_memory()
        X_d = [X, torch.empty_like(X)]
        X_h = [torch.empty(X.shape, dtype=X.dtype).pin_memory() for _ in range(2)]
        m_d = torch.empty_like(m_dev)
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_steps(k):
            for it in range(k):
                b = it % 2
                if it >= 2:   # the buffer's previous copy has landed before the step overwrites it
                    torch.cuda.current_stream().wait_event(copied[b])
                m_d.copy_(m_h, non_blocking=True)
                step(prec, m=m_d, Xout=X_d[b])
                ready = torch.cuda.Event()
                ready.record()
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(ready)
                    X_h[b].copy_(X_d[b], non_blocking=True)
                    copied[b].record(copy_stream)
            torch.cuda.current_stream().wait_stream(copy_stream)

        e2e_steps(args.warmup)   # untimed, as in the main loop
        torch.cuda.synchronize()
        flush.fill_(2.0)
        k = max(1, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        e2e_steps(k)
        e1.record()
        e1.synchronize()
        t_e2e = e0.elapsed_time(e1) / 1e3
        e2e = {"value": k * n_om * ns / t_e2e, "unit": UNIT, "ms_per_step": 1e3 * t_e2e / k,
               "h2d_bytes_per_step": N * 8 + ns * 2 * 8 + w.acq.n_rec * 3 * 8,
               "d2h_bytes_per_step": X.numel() * 16,
               "pipelining": "step k's solutions copied to the host while step k+1 computes"}

    # ---- FP64 GPU path on the same step (the comparison the metric names)
    fp64 = None
    X_fp64_sample = None
    if not args.no_fp64_compare and prec == hm.HELM_MIXED:
        step(hm.HELM_FP64)
        torch.cuda.synchronize()
        e0, ef, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        step(hm.HELM_FP64, ef)
        e1.record()
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        X_fp64_sample = X[:, list(SAMPLE_COLS)].cpu().numpy()
        fp64 = {"value": n_om * ns / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
                "factor_ms": e0.elapsed_time(ef), "solve_ms": ef.elapsed_time(e1),
                "mixed_speedup": value / world / (n_om * ns / dt)}

    # ---- per-solve latency on a resident factor: one right-hand side per frequency, and all
    latency = {}
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, m_dev, w.omegas)
    hm.helm_sources(op, acq, B)
    for name, p in (("mixed", hm.HELM_MIXED), ("fp64", hm.HELM_FP64)):
        f = hm.helm_factor(op, p)
        for nr, reps in ((1, 30), (ns, 10)):
            Bs = B[:, :nr].contiguous()
            Xs = torch.empty_like(Bs)
            hm.helm_solve(f, Bs, Xs, rtol=REFINE_RTOL, max_iter=40)
            lat = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                hm.helm_solve(f, Bs, Xs, rtol=REFINE_RTOL, max_iter=40)
                e1.record()
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
            latency[f"{name}_{nr}rhs"] = {"p50_ms": float(np.percentile(lat, 50)),
                                          "p99_ms": float(np.percentile(lat, 99)), "calls": reps,
                                          "columns_per_call": nr * n_om}
        f.close()
    op.close()

    rl = roofline(dominant, trace, breakdown, (w.nx, w.nz, n_om, ns), peaks)

    extras = {"kernel_zgemm": gemm_kernel_bench(hm, torch, peaks), "kernel_zinv": zinv_kernel_bench(hm, torch)} \
        if rank == 0 else {}
    if not args.no_extras and rank == 0:
        extras["hypergrad_step_128"] = hypergrad_step(hm, torch, 10, args.warmup, rank)
        try:
            extras["hypergrad_batch"] = hypergrad_batch(hm, torch)
        except Exception as e:  # keep the main line if the batch fails
            extras["hypergrad_batch"] = {"failed": str(e)[:300]}
        try:
            extras["hypergrad_lower"] = hypergrad_lower(hm, torch)
        except Exception as e:  # keep the main line if the lower level fails
            extras["hypergrad_lower"] = {"failed": str(e)[:300]}
        try:
            extras["mixed_512"] = grid512_step(hm, torch)
        except Exception as e:  # keep the main line if the large grid fails
            extras["mixed_512"] = {"failed": str(e)[:300]}
        try:
            extras["server"] = server_run([64, 128, 256], 40, 3.0, (0.8,))
        except Exception as e:  # keep the main line if the session fails
            extras["server"] = {"failed": str(e)[:300]}

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            fd, npy = tempfile.mkstemp(suffix=".npy")
            os.close(fd)
            r = run_oracle_subprocess(args.n, seed, 1, npy)[0]
            ref = np.load(npy)
            os.unlink(npy)
            cpu = {"value": r["solves"] / r["seconds"], "unit": UNIT, "cores": r["procs"], "kind": "oracle",
                   "cores_allowed": r["cores_allowed"],
                   "sample": f"the whole workload ({r['solves']} right-hand sides, {n_om} factors) by the FP64 CPU "
                             f"oracle (SciPy SuperLU), one frequency per process on {r['procs']} processes, "
                             f"{r['seconds']:.1f} s wall, {r['cpu_seconds']:.1f} s CPU"}

            def per_omega(Xs):
                e = np.linalg.norm(Xs - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
                return [float(v) for v in e.max(axis=1)]
            errors = {"columns": list(SAMPLE_COLS), "metric": "max over the sampled columns of ||x - x_oracle|| / "
                                                              "||x_oracle||, per frequency",
                      "mixed": per_omega(X_mixed_sample)}
            if X_fp64_sample is not None:
                errors["fp64"] = per_omega(X_fp64_sample)
        except Exception as e:  # keep the GPU line even if the host leg fails
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {e}"[:300]}

    if rank == 0:
        lat_steps = sorted(times)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if args.prec == "mixed" else "f64",
            "data": "synthetic (seeded Gaussian-random-field velocity; Marmousi not available)",
            "config": {"workload": workload_desc(w), "precision": args.prec, "solves_per_step": n_om * ns,
                       "refine_rtol": REFINE_RTOL, "factor_included": True,
                       "l2": "flushed between steps (256 MB write); the factors (1.1 GB) exceed L2",
                       "parallelism": f"one velocity model per GPU x{world}"},
            "phase_ms": {"factor": 1e3 * statistics.median(fac_times),
                         "solve": 1e3 * statistics.median([t - f for t, f in zip(times, fac_times)]),
                         "refinement_sweeps": max(iters)},
            "latency_ms": {"per": "helm_solve call on a resident factor (columns_per_call columns)", **latency,
                           "step_p50": 1e3 * lat_steps[len(lat_steps) // 2],
                           "step_p99": 1e3 * lat_steps[min(len(lat_steps) - 1, int(0.99 * len(lat_steps)))]},
            "error_vs_oracle": errors,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": rl, "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "kernels_one_step": {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3)}
                                 for k, v in breakdown.items()},
            **extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args, world, rank):
    """The CPU oracle timed as the reference arm on the same workload: every step is the whole
    workload (every frequency factored, every right-hand side solved), one frequency per
    process of a pool over the allowed host cores."""
    if rank != 0:
        return
    recs = run_oracle_subprocess(args.n, args.seed, args.warmup + args.steps)
    timed = recs[args.warmup:]
    tot = sum(r["seconds"] for r in timed)
    sol = sum(r["solves"] for r in timed)
    value = sol / tot
    import workloads as W
    w = W.config_mixed(args.n, seed=args.seed)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-random-field velocity; Marmousi not available)",
        "config": {"workload": workload_desc(w), "precision": "fp64 oracle (SciPy SuperLU)",
                   "solves_per_step": timed[0]["solves"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": timed[0]["procs"], "kind": "oracle",
                         "sample": f"{args.steps} timed steps, each the whole workload, one frequency per process on "
                                   f"{timed[0]['procs']} processes ({timed[0]['cores_allowed']} cores allowed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
