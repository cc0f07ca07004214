"""Benchmark of the stability hot path on GB300.

Default workload: the 256 x 512 compressible tanh mixing layer (524,288
complex unknowns, Ma 0.3, Re 1000).  One step is one application of the
matrix-free operator J(q0) v (cancellation-free epsilon-quotient, FP64),
the innermost and most-called operation of the method.  Prints one JSON line.

--impl reference times the CPU oracle (the plain C++ restatement, literal
double epsilon-quotient) on the host cores, on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import stab_inputs as si  # noqa: E402

METRIC = "J·v GB/s (% HBM peak); converged eigenpairs/s; p50/p99 solve latency"
JV_BYTES_PER_DOF = 32  # read v (16 B) + write J v (16 B); the y-only base tables stay in cache
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _workload(nx=256, ny=512):
    g, f = si.mixing_layer_2d(nx, ny)
    return g, f, si.tanh_base_flow(g, f)


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(g, f, q0, budget_s: float = 12.0) -> dict:
    """The oracle's literal epsilon-quotient J v, timed on the host cores."""
    import oracle
    oracle.build()
    P = oracle.Problem.from_inputs(g, f)
    v = si.random_complex(11, g.n)
    eps = oracle.core.knoll_keyes_eps(q0, v)
    oracle.core.jv(P, q0, v, "literal", eps)  # warm
    t0 = time.perf_counter()
    count = 0
    while True:
        oracle.core.jv(P, q0, v, "literal", eps)
        count += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / count
    return {"value": g.n * JV_BYTES_PER_DOF / dt / 1e9, "unit": "GB/s", "cores": oracle.core.num_threads(),
            "kind": "oracle",
            "sample": f"{count} literal double epsilon-quotient J v on the full {g.nx}x{g.ny} layer "
                      f"({dt * 1e3:.1f} ms each)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, f, q0 = _workload(args.nx, args.ny)
    import oracle
    oracle.build()
    P = oracle.Problem.from_inputs(g, f)
    v = si.random_complex(11, g.n)
    eps = oracle.core.knoll_keyes_eps(q0, v)
    for _ in range(args.warmup):
        oracle.core.jv(P, q0, v, "literal", eps)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.core.jv(P, q0, v, "literal", eps)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    val = g.n * JV_BYTES_PER_DOF / dt / 1e9
    cores = oracle.core.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"jv_mixing_layer_{g.nx}x{g.ny}", "nx": g.nx, "ny": g.ny, "Ma": f.Ma, "Re": f.Re},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} literal double epsilon-quotient J v on the full layer"},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1502_03701_gb300 import Stab, build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    g, f, q0 = _workload(args.nx, args.ny)
    stream = torch.cuda.current_stream()
    S = Stab(q0, g, f.Ma, f.Re, f.Pr)
    n = g.n
    v = torch.from_numpy(si.random_complex(11 + rank, n)).cuda()
    out = torch.empty_like(v)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 3)):
        S.apply_J(v, out)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    with sampler:
        for s in range(args.steps):
            flush.zero_()  # L2 flush between timed iterations (outside the events)
            ev[s][0].record(stream)
            S.apply_J(v, out)
            ev[s][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(ms) / 1e3
    t = torch.tensor([t_local], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    bytes_step = n * JV_BYTES_PER_DOF
    value = world * args.steps * bytes_step / t_max / 1e9

    # end to end through the same public call with host buffers (pinned), copies inside
    vh = torch.from_numpy(si.random_complex(11 + rank, n)).pin_memory()
    oh = torch.empty_like(vh).pin_memory()
    e2e_steps = max(3, args.steps)
    vd, od = torch.empty_like(v), torch.empty_like(v)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        vd.copy_(vh, non_blocking=True)
        S.apply_J(vd, od)
        oh.copy_(od, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_t = e0.elapsed_time(e1) / 1e3 / e2e_steps
    e2e_val = world * bytes_step / e2e_t / 1e9

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    achieved = bytes_step / (t_local / args.steps) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"jv_mixing_layer_{g.nx}x{g.ny}", "nx": g.nx, "ny": g.ny, "Ma": f.Ma, "Re": f.Re,
                   "eps_mode": "cancellation-free epsilon-quotient", "l2": "flushed between timed steps",
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if hbm else None, "traffic": None,
                     "kernel": "J v operator (one stab_apply_J call)",
                     "bytes_per_launch": bytes_step, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
        "clocks": sampler.summary(),
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 16},
        "gpu_launches": args.steps * 6,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, f, q0)
    if rank == 0:
        print(json.dumps(line))
    S.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=512)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
