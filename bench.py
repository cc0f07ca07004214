"""Benchmark of the stability hot path on GB300.  Prints one JSON line.

Default (--workload jv): the 3-D compressible tanh mixing layer at
128 x 256 x 64 points (10,485,760 complex unknowns, Ma 0.3, Re 1000), the
largest single-GPU configuration.  One timed step is one application of the
matrix-free operator J(q0) v through the C ABI (the cancellation-free
epsilon-quotient of the paper's Frechet derivative), the innermost and
most-called step of the method; value = GB/s of algorithmic traffic (32 B per
complex unknown: read v, write J v; the y-only base tables stay on chip),
and the roofline compares it with the measured HBM copy bandwidth, with the
FP64-pipe fraction of the line passes beside it.  Also reported, measured in
the same run:
  * "jv_pair_stencil": the same J v with the compact-scheme right-hand sides in
    FP32 pair arithmetic (stencil_prec 48), and its difference to the main step's;
  * "jv_2d_256x512": the J v of the 2-D 256 x 512 layer (524,288 unknowns);
  * "eigs": complete Cayley-IRAM solves of the 32 x 64 layer through stab_eigs
    (sigma 1, tau -1, nev 4, ncv 30, block-Jacobi over 16 x 16 tiles, FGMRES(50) to 1e-10,
    exact-tangent J v): converged eigenpairs per second (true residual
    < 1e-8), the p50 / p99 solve latency and the J v count per solve;
  * "gmres_256x512": preconditioned FGMRES(50) iterations per second on the
    256 x 512 layer (block-Jacobi over 8 x 8-point tiles, FP32 inverses; also
    BF16 inverses, and BF16 inverses with an FP32 Krylov basis);
  * "precond_build_256x512": the block-Jacobi build on the CUDA cores and with
    tensor-core GEMMs (BF16x9, TF32), 8 x 8 and 16 x 16 tiles;
  * "preconditioners_256x512": the inner solve to 1e-10 at sigma = 1 with exact
    8 x 32 blocks against reduced-operator blocks (block-tridiagonal factors)
    over taller tiles: iterations, time, build, factor bytes, apply time;
  * "jv_batch_64": J v and block-Jacobi apply of the 64 uneven instances of the batch
    configuration as one batched call (one launch per phase) against 64 single-problem calls;
  * "many_small": uneven small layers solved one at a time on the plain FP64
    path, as one mixed-precision batch (stab_eigs_batch), and as a Poisson
    stream through the continuous-batching server (p50 / p99 latency).
The line-pass launch shapes of the timed grid are autotuned first
(--tune-cache FILE reuses and stores the tuned shapes).

--workload eigs makes Cayley-IRAM solves of the 2-D 256 x 512 layer the timed step.

--impl reference times the CPU oracle (plain C++ restatement) on the host
cores on a bounded sample and scales it to the same metric.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import stab_inputs as si  # noqa: E402

METRIC = "J·v GB/s (% HBM peak); converged eigenpairs/s; p50/p99 solve latency"
JV_BYTES_PER_DOF = 32  # read v (16 B) + write J v (16 B); the y-only base tables stay on chip
L2_FLUSH_BYTES = 512 << 20
# 256 x 512 solves: the pole right of the spectrum (sigma 1, tau -1: the least stable modes have the largest
# |theta|); block-Jacobi over 8 x 32-point tiles (1,024 unknowns), the tile shape whose inner solves reach
# 1e-10 (measured: 3,776 FGMRES(50) iterations, against no convergence for 8 x 8 tiles)
EIG = dict(sigma=1.0, tau=-1.0, nev=10, ncv=60, tol=1e-10)
EIG_GRID = (256, 512)  # the 2-D layer of the --workload eigs solves
SOLVER_OPTS = dict(eps_mode=2, precond=1, tile=(8, 32), precond_prec=32, precond_factor=1, gmres_m=50,
                   gmres_tol=1e-10, gmres_max_restarts=400, max_restarts=40)
RESID_OK = 1e-8


def _jv_workload_name(g) -> str:
    return f"jv_mixing_layer_{g.nx}x{g.ny}" + (f"x{g.nz}" if g.dim == 3 else "")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _layer(nx, ny, Ma, nz=1):
    """The tanh mixing layer of the workloads: 2-D for nz = 1, else 3-D (x and z periodic, Lz = Lx)."""
    if nz > 1:
        g, f = si.mixing_layer_3d(nx, ny, nz, Ma=Ma)
    else:
        g, f = si.mixing_layer_2d(nx, ny, Ma=Ma)
    return g, f, si.tanh_base_flow(g, f)


def _jv_sample_grid(g):
    """Bounded CPU sample of a J v workload: 3-D layers keep their x-y planes and z spacing but only 8
    z planes (the oracle's cost is linear in the points), 2-D layers run whole."""
    if g.dim == 3 and g.nz > 8:
        return si.Grid(3, g.nx, g.ny, 8, g.lx, g.ly0, g.ly1, g.lz * 8 / g.nz, g.stretch)
    return g


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int, period_ms: int = 100):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.index = index
        self.period = period_ms

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def wait_first_sample(self, limit_s: float = 5.0):
        """Block until nvidia-smi has written its first row (its start-up takes a moment)."""
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < limit_s:
            try:
                if os.path.getsize(self.path) > 0:
                    return
            except OSError:
                pass
            time.sleep(0.02)

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

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timings (bounded samples)
# ---------------------------------------------------------------------------
def oracle_jv_seconds(g, f, q0, budget_s: float, mode: str = "tangent"):
    import oracle
    oracle.build()
    P = oracle.Problem.from_inputs(g, f)
    v = si.random_complex(11, g.n)
    eps = oracle.core.knoll_keyes_eps(q0, v) if mode != "tangent" else None
    oracle.core.jv(P, q0, v, mode, eps)  # warm
    t0 = time.perf_counter()
    count = 0
    while True:
        oracle.core.jv(P, q0, v, mode, eps)
        count += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return (time.perf_counter() - t0) / count, count, oracle.core.num_threads()


def cpu_baseline_eigs(g, f, q0, jv_calls: float, nconv: float, budget_s: float = 12.0) -> dict:
    """Oracle cost of one solve, lower bound: the solve's J v count times the
    oracle's J v time (orthogonalisation and preconditioner not counted)."""
    dt, count, cores = oracle_jv_seconds(g, f, q0, budget_s)
    t_solve = jv_calls * dt
    return {"value": nconv / t_solve if t_solve > 0 else None, "unit": "eigenpairs/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{count} oracle tangent J v on the full {g.nx}x{g.ny} layer ({dt * 1e3:.1f} ms each), "
                      f"scaled by the GPU solve's {jv_calls:.0f} J v per solve (lower bound on CPU time)"}


def _cpu_model() -> str:
    try:  # lscpu names Arm cores (Neoverse-...); /proc/cpuinfo only carries part numbers there
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_jv(g, f, budget_s: float = 12.0) -> dict:
    gs = _jv_sample_grid(g)
    dt, count, cores = oracle_jv_seconds(gs, f, si.tanh_base_flow(gs, f), budget_s, "literal")
    return {"value": gs.n * JV_BYTES_PER_DOF / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": f"{count} literal double epsilon-quotient J v of the oracle on a {gs.nx}x{gs.ny}x{gs.nz} "
                      f"layer ({gs.n} unknowns, {dt * 1e3:.1f} ms each; the workload's x-y planes and spacing), "
                      f"scaled per unknown to the {g.nx}x{g.ny}x{g.nz} workload"}


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "jv":
        g, f, q0 = _layer(args.nx, args.ny, 0.3, args.nz)
        import oracle
        oracle.build()
        gs = _jv_sample_grid(g)
        qs = si.tanh_base_flow(gs, f)
        P = oracle.Problem.from_inputs(gs, f)
        v = si.random_complex(11, gs.n)
        eps = oracle.core.knoll_keyes_eps(qs, v)
        for _ in range(max(args.warmup, 1)):
            oracle.core.jv(P, qs, v, "literal", eps)
        t0 = time.perf_counter()
        count = 0
        while count < args.steps and time.perf_counter() - t0 < 60.0:  # K steps, at most a minute
            oracle.core.jv(P, qs, v, "literal", eps)
            count += 1
        dt = (time.perf_counter() - t0) / count * g.n / gs.n  # per full-size J v
        cores = oracle.core.num_threads()
        val, unit, ms = g.n * JV_BYTES_PER_DOF / dt / 1e9, "GB/s", dt * 1e3
        sample = (f"{count} literal double epsilon-quotient J v of the oracle on a {gs.nx}x{gs.ny}x{gs.nz} layer "
                  f"(of {args.steps} steps), scaled per unknown to the {g.nx}x{g.ny}x{g.nz} workload; "
                  f"CPU {_cpu_model()}")
        wl = _jv_workload_name(g)
    else:
        g, f, q0 = _layer(EIG_GRID[0], EIG_GRID[1], 0.3)
        wl = f"eigs_mixing_layer_{g.nx}x{g.ny}"
        # bounded sample: the oracle's J v time scaled by the J v count of a solve of this workload
        # (recorded by the GPU arm in profiles/; 1 J v per GMRES iteration plus one per restart)
        jv_per_solve = args.ref_jv_per_solve
        dt, count, cores = oracle_jv_seconds(g, f, q0, max(1.0, 0.5 * args.steps))
        ms = jv_per_solve * dt * 1e3
        val, unit = EIG["nev"] / (ms / 1e3), "eigenpairs/s"
        sample = (f"{count} oracle tangent J v ({dt * 1e3:.1f} ms each) x {jv_per_solve} J v per solve "
                  f"(lower bound on the CPU solve time)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl, "nx": g.nx, "ny": g.ny, "nz": g.nz},
            "cpu_baseline": {"value": val, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# 32 x 64 layer; the pole sits right of the spectrum (inner solves converge), the four least-stable
# eigenvalues (two Kelvin-Helmholtz double eigenvalues) are wanted.
SMALL_EIG = dict(nx=32, ny=64, sigma=1.0, tau=-1.0, nev=4, ncv=30, tol=1e-10)
# On grids this small the solves are latency-bound, so larger blocks (16 x 16 points, 1,024 unknowns)
# pay: 78 instead of 197 FGMRES iterations per inner solve at the same cost per iteration (measured).
SMALL_TILE = (16, 16)


def small_layer_eigs(args, Stab, torch, rank):
    """Complete solves of the 32 x 64 layer: eigenpairs/s and latency."""
    g, f, q0 = _layer(SMALL_EIG["nx"], SMALL_EIG["ny"], 0.3)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=SMALL_TILE, precond_prec=32, gmres_m=50,
             gmres_tol=1e-10, gmres_max_restarts=100, max_restarts=40, seed=0x5EED + rank)
    S.autotune()
    args_e = (SMALL_EIG["sigma"], SMALL_EIG["tau"], SMALL_EIG["nev"], SMALL_EIG["ncv"], SMALL_EIG["tol"])
    S.eigs(*args_e)  # warm-up
    times, good, res = [], 0, []
    for _ in range(args.eig_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = S.eigs(*args_e)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        good += int(np.sum(r.resid[:r.nconv] < RESID_OK))
        res.append(r)
    S.close()
    lat = sorted(times)
    return {"value": good / sum(times), "unit": "eigenpairs/s", "workload": "eigs_mixing_layer_32x64",
            "sigma": [1.0, 0.0], "tau": [-1.0, 0.0], "nev": SMALL_EIG["nev"], "ncv": SMALL_EIG["ncv"],
            "tol": SMALL_EIG["tol"], "gmres": "FGMRES(50) to 1e-10, block-Jacobi 16x16 tiles FP32",
            "solves": len(times),
            "latency_ms": {"p50": statistics.median(lat) * 1e3, "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3},
            "nconv": [r.nconv for r in res], "max_resid": max(float(np.max(r.resid)) for r in res),
            "jv_per_solve": statistics.mean(r.stats["jv_calls"] for r in res),
            "gmres_iterations_per_solve": statistics.mean(r.stats["gmres_iterations"] for r in res),
            "restarts": [r.stats["restarts"] for r in res]}


def jv_extra(args, Stab, torch, flush, stream, nx, ny, nz=1) -> dict:
    """J v of another layer (autotuned, L2 flushed between steps) with its own roofline."""
    g, f, q0 = _layer(nx, ny, 0.3, nz)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr)
    tuned = S.autotune()
    St = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    v = torch.from_numpy(si.random_complex(21, g.n)).cuda()
    out = torch.empty_like(v)
    for _ in range(3):
        S.apply_J(v, out)
        St.apply_J(v, out)
    tan = _time_jv(St, v, out, 20, flush, stream, torch)
    S.timing(True)
    steps = _time_jv(S, v, out, args.steps_2d, flush, stream, torch)
    ph = S.timing_read()
    S.close()
    St.close()
    t = statistics.mean(steps)
    return {"workload": _jv_workload_name(g), "value": g.n * JV_BYTES_PER_DOF / t / 1e9, "unit": "GB/s",
            "ms_per_step": t * 1e3, "steps": args.steps_2d, "unknowns": g.n,
            "line_pass_shapes": {ax: {"C": c, "L": l, "kinds": k} for ax, (c, l, k, _) in tuned.items()},
            "roofline": jv_roofline(g, f, ph, t, _peaks().get("hbm_gbs"), statistics.mean(tan))}


def gmres_throughput(args, Stab, torch, q0, g, f):
    """Preconditioned FGMRES(50) on the 256 x 512 layer: iterations per second with FP32 and with BF16
    block inverses, each with the true relative residual reached after the same iteration budget."""
    out = {}
    sigma = 1.0
    b = torch.from_numpy(si.random_complex(1, g.n)).cuda()
    for prec, basis, key in ((32, 64, "fp32_inverses"), (16, 64, "bf16_inverses"), (16, 32, "bf16_inverses_fp32_basis")):
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=(8, 8), precond_prec=prec, gmres_m=50,
                 gmres_tol=1e-10, gmres_max_restarts=args.gmres_restarts, gmres_basis_prec=basis)
        S.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.precond_build(sigma)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        x = torch.zeros_like(b)
        S.solve(sigma, b, x)  # captures the cycle graph
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it = S.solve(sigma, b, x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ax = torch.empty_like(b)
        S.apply_J(x, ax, sigma)  # (J - sigma I) x with the operator the solve uses
        res = float(torch.linalg.vector_norm(b - ax) / torch.linalg.vector_norm(b))
        S.close()
        out[key] = {"value": it / dt, "unit": "iterations/s", "iterations": it, "seconds": dt,
                    "converged": st == 0, "true_rel_residual": res, "precond_build_s": t_build}
    r = dict(out["fp32_inverses"])
    r.update({"sigma": sigma, "tile": [8, 8], "block": 256, "precond": "FP32 inverses", "bf16": out["bf16_inverses"],
              "bf16_fp32_basis": out["bf16_inverses_fp32_basis"]})
    return r


def precond_build_256x512(args, Stab, torch) -> dict:
    """Block-Jacobi build on the 256 x 512 layer (assembly + inversion of every tile block, FP32
    inverses): Gauss-Jordan on the CUDA cores against the blocked sweep with tensor-core GEMMs
    (BF16x9-emulated FP32 and TF32), for 8 x 8 tiles (2,048 blocks of 256) and 16 x 16 tiles (512 of
    1,024).  Inversion work: b^3 complex multiply-adds per block = 8 b^3 real flops."""
    g, f, q0 = _layer(256, 512, 0.3)
    out = {}
    for tile in ((8, 8), (16, 16)):
        b = 4 * tile[0] * tile[1]
        nblk = g.npts // (tile[0] * tile[1])
        flops = 8.0 * b ** 3 * nblk
        row = {"block": b, "blocks": nblk, "inversion_flop": flops}
        for fac, key in ((0, "cuda_cores"), (1, "tensor_bf16x9"), (2, "tensor_tf32")):
            S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=tile, precond_prec=32, precond_factor=fac)
            S.precond_build(1.0)  # warm (cuBLAS handle, workspaces)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S.precond_build(1.0 + 1e-3j)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            S.close()
            row[key] = {"seconds": dt, "TFLOP_per_s": flops / dt / 1e12}
        out[f"{tile[0]}x{tile[1]}"] = row
    return out


def inner_solves(Stab, torch, g, f, q0, variants, sigma=1.0, max_restarts=120) -> dict:
    """FGMRES(50) to 1e-10 of (J - sigma I) x = b on one layer per preconditioner variant (name, options):
    iterations, J v calls, solve time, build time, factor bytes (FP32) and the time of one block apply
    (CUDA events, 20 applies)."""
    b = torch.from_numpy(si.random_complex(1, g.n)).cuda()
    out = {"sigma": sigma, "tol": 1e-10, "gmres": "FGMRES(50)", "unknowns": g.n}
    nv = g.dim + 2
    for key, o in variants:
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond_prec=32, gmres_m=50, gmres_tol=1e-10,
                 gmres_max_restarts=max_restarts, **o)
        S.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.precond_build(sigma)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        z = torch.empty_like(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        S.precond_apply(b, z)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            S.precond_apply(b, z)
        e1.record()
        torch.cuda.synchronize()
        apply_ms = e0.elapsed_time(e1) / 20
        x = torch.zeros_like(b)
        jv0 = S.stats()["jv_calls"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it = S.solve(sigma, b, x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        jv = S.stats()["jv_calls"] - jv0
        ax = torch.empty_like(b)
        S.apply_J(x, ax, sigma)
        res = float(torch.linalg.vector_norm(b - ax) / torch.linalg.vector_norm(b))
        tile = o["tile"]
        tz = tile[2] if g.dim == 3 else 1
        if o["precond"] == 1:
            nbytes = g.n * nv * tile[0] * tile[1] * tz * 8
        else:
            nbytes = g.n * 3 * (nv * 2 * tile[0] * tz) * 8
        S.close()
        out[key] = {"iterations": it, "jv_calls": jv, "converged": st == 0, "true_rel_residual": res, "solve_s": dt,
                    "ms_per_iteration": 1e3 * dt / max(it, 1), "build_s": t_build, "apply_ms": apply_ms,
                    "factor_bytes": nbytes, "apply_GB_per_s": nbytes / apply_ms / 1e6}
    return out


def preconditioners_256x512(args, Stab, torch) -> dict:
    """The 256 x 512 inner solve (FGMRES(50) to 1e-10 at sigma = 1) with exact tile blocks (block-Jacobi
    over 8 x 32 tiles, FP32 inverses factorised with TF32 tensor-core GEMMs) against the reduced-operator
    blocks (second-order explicit operator, block-tridiagonal FP32 factors) over taller tiles, and with
    LGMRES(50, 4) beside GMRES(50)."""
    g, f, q0 = _layer(256, 512, 0.3)
    variants = (("exact_8x32", dict(precond=1, tile=(8, 32), precond_factor=2)),
                ("exact_8x32_lgmres4", dict(precond=1, tile=(8, 32), precond_factor=2, lgmres_k=4)),
                ("reduced_8x64", dict(precond=2, tile=(8, 64))),
                ("reduced_8x512", dict(precond=2, tile=(8, 512))),
                ("reduced_8x512_lgmres4", dict(precond=2, tile=(8, 512), lgmres_k=4)),
                ("reduced_4x512", dict(precond=2, tile=(4, 512))))
    return inner_solves(Stab, torch, g, f, q0, variants)


def _parse_variants(spec: str, dim: int):
    """'exact:8x8x2,reduced:4x128x2:lg4' -> [(name, Stab options)]."""
    out = []
    for item in spec.split(","):
        parts = item.split(":")
        tile = tuple(int(t) for t in parts[1].split("x"))
        if dim == 2:
            tile = tile[:2]
        o = dict(precond=1 if parts[0] == "exact" else 2, tile=tile)
        if parts[0] == "exact":
            o["precond_factor"] = 2
        name = f"{parts[0]}_{parts[1]}"
        for extra in parts[2:]:
            if extra.startswith("lg"):
                o["lgmres_k"] = int(extra[2:])
                name += f"_lgmres{o['lgmres_k']}"
        out.append((name, o))
    return out


def run_mixed(args):
    """--workload mixed: Cayley-IRAM (sigma 1, tau -1, nev 4, ncv 20, tol 1e-10, exact-tangent J v) of the
    --nx x --ny x --nz layer with FP64 block inverses over --tile3 tiles (the plain path) against the
    mixed-precision variants (FP32 inverses factorised with BF16x9 or TF32 tensor-core GEMMs; BF16
    inverses with the FP32 Krylov basis; the nested FP32-basis inner GMRES(10); the reduced-operator
    blocks over --reduced-tile tiles with FP32 factors): per eigenvalue the relative difference to the
    FP64 path, true residuals, J v counts and times."""
    import numpy as np
    import torch
    from paper_1502_03701_gb300 import Stab, build
    build.build()
    g, f, q0 = _layer(args.nx, args.ny, 0.3, nz=args.nz)
    tile = tuple(args.tile3[:g.dim]) if g.dim == 3 else tuple(args.tile3[:2])
    rtile = tuple(args.reduced_tile[:g.dim]) if g.dim == 3 else tuple(args.reduced_tile[:2])
    v0 = torch.from_numpy(si.start_vector(0x5EED, g.n)).cuda()
    variants = [("fp64_inverses", dict(precond=1, tile=tile, precond_prec=64)),
                ("fp32_tensor_bf16x9", dict(precond=1, tile=tile, precond_prec=32, precond_factor=1)),
                ("fp32_tensor_tf32", dict(precond=1, tile=tile, precond_prec=32, precond_factor=2)),
                ("bf16_inverses_fp32_basis", dict(precond=1, tile=tile, precond_prec=16, precond_factor=1,
                                                  gmres_basis_prec=32)),
                ("nested_fp32_inner_gmres10", dict(precond=1, tile=tile, precond_prec=32, precond_factor=1,
                                                   gmres_inner_m=10, gmres_inner_tol=1e-3)),
                ("reduced_fp32_factors", dict(precond=2, tile=rtile, precond_prec=32))]
    ref, rows = None, {}
    for name, o in variants:
        gm = 20 if o.get("gmres_inner_m") else 50
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, gmres_m=gm, gmres_tol=1e-10, gmres_max_restarts=200,
                 max_restarts=30, **o)
        S.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = S.eigs(1.0, -1.0, nev=4, ncv=20, tol=1e-10, v0=v0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        S.close()
        row = {"status": r.status, "nconv": r.nconv, "seconds": dt, "lam": [[l.real, l.imag] for l in r.lam],
               "resid": [float(x) for x in r.resid], "jv_calls": r.stats["jv_calls"],
               "gmres_iterations": r.stats["gmres_iterations"], "tile": list(o["tile"])}
        if ref is None:
            ref = r.lam
        else:
            row["rel_diff_vs_fp64"] = [float(np.abs(ref - l).min() / abs(l)) for l in r.lam]
        rows[name] = row
    worst = max(max(v.get("rel_diff_vs_fp64", [0.0])) for v in rows.values())
    print(json.dumps({"metric": "largest relative eigenvalue difference to the FP64 path", "value": worst,
                      "unit": "relative", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
                      "config": {"workload": _jv_workload_name(g).replace("jv_", "mixed_"), "sigma": 1.0, "tau": -1.0,
                                 "nev": 4, "ncv": 20, "tol": 1e-10},
                      "variants": rows}))


def run_inner(args):
    """--workload inner: the inner solve of the --nx x --ny (x --nz) layer at sigma = 1 for each
    preconditioner variant of --variants (kind:TXxTYxTZ[:lgK], kind exact or reduced)."""
    import torch
    from paper_1502_03701_gb300 import Stab, build
    build.build()
    g, f, q0 = _layer(args.nx, args.ny, 0.3, nz=args.nz)
    r = inner_solves(Stab, torch, g, f, q0, _parse_variants(args.variants, g.dim), max_restarts=args.inner_restarts)
    best = min((v["solve_s"] for v in r.values() if isinstance(v, dict) and v["converged"]), default=None)
    print(json.dumps({"metric": "inner solve to 1e-10", "value": (1.0 / best) if best else None, "unit": "solves/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
                      "config": {"workload": _jv_workload_name(g).replace("jv_", "inner_"), "variants": args.variants},
                      "inner": r}))


# Algorithmic FP64 flops of the compact line pass per real output value (FMA = 2):
#   first derivative  : stencil a(f+1 - f-1) + b(f+2 - f-2)        5  + tridiagonal solve 5 = 10
#   second derivative : stencil a(f+1 - 2f + f-1) + b(f+2 - 2f + f-2) 9 + tridiagonal solve 5 = 14
# (solve: forward elimination one FMA, back substitution one FMA and one multiply).
LINE_FLOP_D1, LINE_FLOP_D2 = 10, 14
# FP64 FMA throughput measured on GB300 by the project's microbenchmark (tests/test_gpu_fp_throughput.py,
# profiles/fp_throughput.md); MEASURED_PEAKS.json carries no FP64 figure.
FP64_MEASURED_GFLOPS = 1197.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of all kernels of one J v, from one ncu capture
# per layer (see profiles/), keyed by workload; scaled by unknowns when the capture ran on a smaller case.
JV_TRAFFIC = {
    # ncu on the 128x256x16 layer (2,621,440 unknowns: the derivative slots, 310 MB, exceed L2): one
    # J v with the epsilon norm read 615.1 MB and wrote 155.9 MB; the z planes are independent, so the
    # 128x256x64 layer moves four times as much (profiles/jv_mixing_layer_128x256x64_launches.md)
    "jv_mixing_layer_128x256x64": {"bytes": 4 * (615.1e6 + 155.9e6),
                                   "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of all kernels of "
                                             "one J v on the 128x256x16 layer, scaled by 4 (z planes)"},
}


def line_pass_flops(g, visc: bool) -> dict:
    """Per-launch algorithmic FP64 flops of the y, z and x line passes."""
    d = g.dim
    nf1 = d + 3 if visc else d + 2          # p, u_i, s (and T) first derivatives
    nf2 = d + 1 if visc else 0              # u_i and T second derivatives
    base = 2 * (nf1 * LINE_FLOP_D1 + nf2 * LINE_FLOP_D2) * g.npts  # x2: real and imaginary parts
    mix_x = (2 if d == 2 else 4) if visc else 0
    mix_z = 2 if (d == 3 and visc) else 0
    out = {"line_y": base, "line_x": base + 2 * mix_x * LINE_FLOP_D1 * g.npts}
    if d == 3:
        out["line_z"] = base + 2 * mix_z * LINE_FLOP_D1 * g.npts
    return out


def jv_roofline(g, f, phases: dict, step_s: float, hbm, tangent_s: float) -> dict:
    """Roofline of the timed J v: the operator's algorithmic bytes (32 B per unknown) over its measured
    step time against the measured HBM copy bandwidth, with the line passes' FP64 rate (the unit that
    binds on GB300) beside it."""
    ms = {k: v[0] for k, v in phases.items() if k != "dropped"}
    cnt = {k: v[1] for k, v in phases.items() if k != "dropped"}
    total = sum(ms.values())
    line_keys = [k for k in ("line_y", "line_z", "line_x") if cnt.get(k)]
    line_ms = sum(ms[k] for k in line_keys)
    launches = sum(cnt[k] for k in line_keys)
    flops = line_pass_flops(g, f.Re > 0)
    line_flops = sum(flops[k] * cnt[k] for k in line_keys)
    avg_s = line_ms / 1e3 / launches
    fp64_achieved = line_flops / launches / avg_s / 1e9
    share = {k: (ms[k] / total if total else None) for k in ms if cnt[k]}
    achieved = g.n * JV_BYTES_PER_DOF / step_s / 1e9
    tr = JV_TRAFFIC.get(_jv_workload_name(g))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if hbm else None,
            "traffic": tr["bytes"] if tr else None,
            "kernel": "the J v operator (epsilon norm, temperature differences, y/z/x compact line passes, "
                      "pointwise assembly: one launch each), timed per step with CUDA events",
            "bytes_per_step": g.n * JV_BYTES_PER_DOF, "step_ms": step_s * 1e3, "tangent_step_ms": tangent_s * 1e3,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
            "traffic_source": tr["source"] if tr else "no ncu capture of the current kernels",
            "phase_share": share,
            "fp64_pipe": {"kernel": "k_line_pass / k_line_pass_compact (all axes)", "achieved": fp64_achieved,
                          "peak": FP64_MEASURED_GFLOPS, "unit": "GFLOP/s", "frac": fp64_achieved / FP64_MEASURED_GFLOPS,
                          "flop_per_launch": line_flops / launches, "launch_ms": avg_s * 1e3, "launches": launches,
                          "peak_source": "FP64 FMA microbenchmark on GB300 (of measured)"}}


# Many small problems (uneven 2-D instances drawn like the 64-instance batch
# configuration, with Nx in {16, 32}, Ny in {32, 64} so that the section ends
# in seconds): Cayley-IRAM sigma 1, tau -1, 2 of 12, tol 1e-10, FGMRES(30) to
# 1e-10 with block-Jacobi over 16 x 16 tiles, exact-tangent J v.
FLEET_SIZES = dict(nxs=(16, 32), nys=(32, 64))
FLEET_EIG = (1.0, -1.0, 2, 12, 1e-10)
FLEET_OPTS = dict(eps_mode=2, precond=1, tile=(16, 16), gmres_m=30, gmres_tol=1e-10, max_restarts=60)


def _fleet_problem(p):
    g, _ = si.mixing_layer_2d(p["nx"], p["ny"])
    f = si.Flow(float(p["Ma"]), float(p["Re"]))
    return g, f, si.tanh_base_flow(g, f)


def jv_batch_64(args, torch) -> dict:
    """J v of the 64 uneven instances of the batch configuration (Nx in {32..256}, Ny in {64..512}, Ma
    U[0.1, 0.9], Re log-U[500, 5000], seed 1234): one stab_jv_batch_apply per step (one launch per phase for
    all instances) against the 64 stab_apply_J calls of the plain path, both on one stream.  Inputs and
    outputs (236 MB) exceed L2, so no flush is needed between steps."""
    from paper_1502_03701_gb300 import JvBatch, Stab
    insts = si.batched_instances(64, 1234)
    hs = []
    for p in insts:
        g, f, q0 = _fleet_problem(p)
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, tile=(8, 8), precond_prec=32)
        S.autotune()
        hs.append(S)
    vs = [torch.from_numpy(si.random_complex(900 + i, S.n)).cuda() for i, S in enumerate(hs)]
    outs = [torch.empty_like(v) for v in vs]
    refs = [torch.empty_like(v) for v in vs]
    B = JvBatch(hs)
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps // 20, 100))

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    def plain():
        for S, v, o in zip(hs, vs, refs):
            S.apply_J(v, o)

    t_plain = timed(plain)
    t_batch = timed(lambda: B.apply(vs, outs))
    same = all(torch.equal(o, r) for o, r in zip(outs, refs))
    n_total = sum(S.n for S in hs)
    # block-Jacobi apply (8 x 8 tiles, FP32 inverses), batched against one call per instance
    for S in hs:
        S.precond_build(1.0)

    def plain_pc():
        for S, v, o in zip(hs, vs, refs):
            S.precond_apply(v, o)

    t_pc_plain = timed(plain_pc)
    t_pc_batch = timed(lambda: B.precond_apply(vs, outs))
    same_pc = all(torch.equal(o, r) for o, r in zip(outs, refs))
    inv_bytes = sum(S.n * 256 * 8 for S in hs)  # one 256-entry FP32 complex row per unknown
    B.close()
    for S in hs:
        S.close()
    return {"workload": "jv_batch_64_uneven_2d", "instances": 64, "unknowns": n_total, "steps": steps,
            "batched": {"value": 64 / t_batch, "unit": "instance J v/s", "ms_per_step": t_batch * 1e3,
                        "GB_per_s": n_total * JV_BYTES_PER_DOF / t_batch / 1e9, "launches_per_step": "5 to 9"},
            "plain_one_at_a_time": {"value": 64 / t_plain, "unit": "instance J v/s", "ms_per_step": t_plain * 1e3,
                                    "GB_per_s": n_total * JV_BYTES_PER_DOF / t_plain / 1e9},
            "speedup": t_plain / t_batch, "bitwise_equal_to_plain": same,
            "precond_apply": {"batched_ms": t_pc_batch * 1e3, "plain_ms": t_pc_plain * 1e3,
                              "batched_GB_per_s": inv_bytes / t_pc_batch / 1e9, "speedup": t_pc_plain / t_pc_batch,
                              "bitwise_equal_to_plain": same_pc,
                              "note": "block-Jacobi over 8 x 8 tiles, FP32 inverses (stored bytes per step)"}}


def gmres_batch_64(args, torch) -> dict:
    """Solver-level batching at the batch configuration's full sizes: two FGMRES(30) cycles (60 iterations)
    of (J - sigma I) x = b for each of the 64 uneven instances (block-Jacobi over 8 x 8 tiles, FP32 inverses),
    in lockstep (stab_jv_batch_solve: every phase one launch for all instances) against one instance at a
    time (stab_solve: one captured graph per cycle).  Instance iterations per second; the lockstep iterates
    equal the lone ones bit for bit below 16,384 unknowns (above, the lone solve reorthogonalises
    selectively), and agree to the solves' progress above."""
    from paper_1502_03701_gb300 import JvBatch, Stab
    insts = si.batched_instances(64, 1234)
    hs = []
    for p in insts:
        g, f, q0 = _fleet_problem(p)
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=(8, 8), precond_prec=32, precond_factor=1,
                 gmres_m=30, gmres_tol=1e-10, gmres_max_restarts=2)
        S.autotune()
        S.precond_build(1.0)
        hs.append(S)
    bs = [torch.from_numpy(si.random_complex(950 + i, S.n)).cuda() for i, S in enumerate(hs)]
    xs_plain = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_plain = [S.solve(1.0, b, x)[1] for S, b, x in zip(hs, bs, xs_plain)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    B = JvBatch(hs)
    xs = [torch.zeros_like(b) for b in bs]
    B.solve([1.0] * len(hs), bs, xs)  # warm (parameter images, workspaces)
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, it_lock = B.solve([1.0] * len(hs), bs, xs)
    torch.cuda.synchronize()
    t_lock = time.perf_counter() - t0
    B.close()
    small = [i for i, S in enumerate(hs) if S.n < 16384]
    same_small = all(torch.equal(xs[i], xs_plain[i]) for i in small)
    diff = max(float((x - y).norm() / y.norm()) for x, y in zip(xs, xs_plain))
    n_total = sum(S.n for S in hs)
    for S in hs:
        S.close()
    return {"workload": "gmres_batch_64_uneven_2d", "instances": 64, "unknowns": n_total,
            "iterations": {"lockstep": int(sum(it_lock)), "plain": int(sum(it_plain))},
            "lockstep": {"value": sum(it_lock) / t_lock, "unit": "instance iterations/s", "seconds": t_lock},
            "plain_one_at_a_time": {"value": sum(it_plain) / t_plain, "unit": "instance iterations/s",
                                    "seconds": t_plain},
            "speedup": (sum(it_lock) / t_lock) / (sum(it_plain) / t_plain),
            "bitwise_equal_below_16k": same_small, "instances_below_16k": len(small),
            "max_rel_diff_of_iterates": diff}


def fleet(args, torch) -> dict:
    """Plain one-at-a-time FP64 path vs batched mixed-precision path vs served Poisson stream."""
    from paper_1502_03701_gb300 import Server, Stab, eigs_batch
    insts = si.batched_instances(args.fleet, 1234, **FLEET_SIZES)
    probs = [_fleet_problem(p) for p in insts]
    nev = FLEET_EIG[2]

    def good(lam_res):
        return int(np.sum(lam_res[1] < RESID_OK))

    # plain: one instance at a time, FP64 block inverses
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain, n_plain = [], 0
    for g, f, q0 in probs:
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, precond_prec=64, **FLEET_OPTS)
        S.autotune()
        r = S.eigs(*FLEET_EIG)
        S.close()
        plain.append((r.lam, r.resid))
        n_plain += good((r.lam, r.resid)) if r.nconv == nev else 0
    t_plain = time.perf_counter() - t0
    # batched: FP32 block inverses (FP64 outer FGMRES, J v, Arnoldi, residuals), all side by side
    t0 = time.perf_counter()
    hs = [Stab(q0, g, f.Ma, f.Re, f.Pr, precond_prec=32, **FLEET_OPTS) for g, f, q0 in probs]
    for h in hs:
        h.autotune()
    res = eigs_batch(hs, [FLEET_EIG] * len(hs), concurrency=len(hs))
    for h in hs:
        h.close()
    t_batch = time.perf_counter() - t0
    n_batch = sum(good((r.lam, r.resid)) for r in res if r.nconv == nev)
    err = [float(np.max(np.abs(r.lam - p[0]) / np.abs(p[0]))) for r, p in zip(res, plain)]
    # lockstep: every phase of all instances' GMRES cycles and Arnoldi steps one launch (stab_jv_batch_eigs),
    # FP32 inverses factorised on the tensor cores
    from paper_1502_03701_gb300 import JvBatch
    t0 = time.perf_counter()
    hs = [Stab(q0, g, f.Ma, f.Re, f.Pr, precond_prec=32, precond_factor=1, **FLEET_OPTS) for g, f, q0 in probs]
    for h in hs:
        h.autotune()
    B = JvBatch(hs)
    res_l = B.eigs([FLEET_EIG] * len(hs))
    B.close()
    for h in hs:
        h.close()
    t_lock = time.perf_counter() - t0
    n_lock = sum(good((r.lam, r.resid)) for r in res_l if r.nconv == nev)
    err_l = [float(np.max(np.abs(r.lam - p[0]) / np.abs(p[0]))) for r, p in zip(res_l, plain)]
    # served: Poisson arrivals, continuous batching
    arrivals = si.poisson_arrivals(len(probs), args.rate, 4321)
    srv = Server(slots=args.slots, mem_budget_bytes=args.budget_gb << 30, autotune=True)
    t0 = time.perf_counter()
    ids = []
    for (g, f, q0), ta in zip(probs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(q0, g, f.Ma, f.Re, f.Pr, *FLEET_EIG, precond_prec=32, **FLEET_OPTS))
    lat, n_srv = [], 0
    for rid in ids:
        srv.wait(rid)
        lam, resid, info = srv.result(rid)
        lat.append(info["latency_s"])
        n_srv += good((lam, resid)) if info["nconv"] == nev else 0
    t_srv = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat.sort()
    return {"workload": f"{len(probs)} uneven 2-D layers, Nx in {FLEET_SIZES['nxs']}, Ny in {FLEET_SIZES['nys']}, "
                        "Ma U[0.1,0.9], Re log-U[500,5000], seed 1234",
            "eig": {"sigma": 1.0, "tau": -1.0, "nev": nev, "ncv": FLEET_EIG[3], "tol": FLEET_EIG[4],
                    "gmres": "FGMRES(30) to 1e-10, block-Jacobi 16x16"},
            "plain_fp64_one_at_a_time": {"value": n_plain / t_plain, "unit": "eigenpairs/s", "seconds": t_plain},
            "batched_mixed": {"value": n_batch / t_batch, "unit": "eigenpairs/s", "seconds": t_batch,
                              "speedup_vs_plain": (n_batch / t_batch) / (n_plain / t_plain) if n_plain else None,
                              "max_rel_diff_vs_plain_fp64": max(err),
                              "how": "stab_eigs_batch: host threads, one stream per instance"},
            "lockstep_mixed": {"value": n_lock / t_lock, "unit": "eigenpairs/s", "seconds": t_lock,
                               "speedup_vs_plain": (n_lock / t_lock) / (n_plain / t_plain) if n_plain else None,
                               "max_rel_diff_vs_plain_fp64": max(err_l),
                               "how": "stab_jv_batch_eigs: one launch per phase for all instances, FP32 inverses "
                                      "factorised with tensor-core GEMMs"},
            "served": {"value": n_srv / t_srv, "unit": "eigenpairs/s", "seconds": t_srv,
                       "arrivals_per_s": args.rate, "slots": args.slots,
                       "latency_ms": {"p50": lat[len(lat) // 2] * 1e3, "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3},
                       "peak_running": st["peak_running"], "peak_bytes": st["peak_bytes"]}}


# Served stream shaped like the serving configuration: Poisson arrivals (50/s, seed 4321); 95 % 2-D layers
# drawn like the 64-instance batch configuration with sizes scaled by a quarter per axis, 5 % 3-D layers
# scaled from 64 x 128 x 32; Cayley-IRAM sigma 1, tau -1, 2 of 12, FGMRES(30) with block-Jacobi.
SERVE_SIZES = dict(nxs=(16, 32, 64), nys=(32, 64, 128))
SERVE_3D = (16, 32, 8)


def serve_stream(args, torch) -> dict:
    """Continuous batching under a Poisson load: p50 / p99 latency and eigenpairs/s of the served stream
    (lockstep cohorts), the plain one-at-a-time FP64 path on the first requests, and each of those
    requests' eigenvalues alone against in the mix (1e-8)."""
    from paper_1502_03701_gb300 import Server, Stab
    count = args.requests
    insts = si.batched_instances(count, 1234, **SERVE_SIZES)
    u = si.splitmix64_uniform(777, count) + 0.5
    probs = []
    for i, p in enumerate(insts):
        if u[i] < 0.05:
            g, f = si.mixing_layer_3d(*SERVE_3D, Ma=float(p["Ma"]))
            f = si.Flow(float(p["Ma"]), float(p["Re"]))
            opts = dict(FLEET_OPTS, tile=(4, 4, 4))
        else:
            g, f, _ = _fleet_problem(p)
            opts = dict(FLEET_OPTS, tile=(min(16, p["nx"]), 16))
        probs.append((g, f, si.tanh_base_flow(g, f), opts))
    nev = FLEET_EIG[2]
    arrivals = si.poisson_arrivals(count, args.rate, 4321)
    srv = Server(slots=args.slots, mem_budget_bytes=args.budget_gb << 30, autotune=True, cohort=args.cohort)
    t0 = time.perf_counter()
    ids = []
    for (g, f, q0, opts), ta in zip(probs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(q0, g, f.Ma, f.Re, f.Pr, *FLEET_EIG, precond_prec=32, precond_factor=1, **opts))
    lat, served, n_srv = [], [], 0
    for rid in ids:
        srv.wait(rid)
        lam, resid, info = srv.result(rid)
        lat.append(info["latency_s"])
        served.append(lam)
        n_srv += int(np.sum(resid < RESID_OK)) if info["nconv"] == nev else 0
    t_srv = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    # the plain FP64 path, one request at a time, on the first requests
    k = min(args.plain_requests, count)
    torch.cuda.synchronize()
    tp = time.perf_counter()
    n_plain, diff = 0, []
    for (g, f, q0, opts), lam_s in zip(probs[:k], served[:k]):
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, precond_prec=64, **opts)
        S.autotune()
        r = S.eigs(*FLEET_EIG)
        S.close()
        n_plain += int(np.sum(r.resid < RESID_OK)) if r.nconv == nev else 0
        diff.append(float(np.max(np.abs(np.sort_complex(lam_s) - np.sort_complex(r.lam)) / np.abs(r.lam))))
    t_plain = time.perf_counter() - tp
    lat.sort()
    return {"workload": f"served stream of {count} requests: 95% 2-D layers Nx in {SERVE_SIZES['nxs']}, Ny in "
                        f"{SERVE_SIZES['nys']} (the batch configuration's sizes scaled by 1/4 per axis), 5% 3-D "
                        f"{SERVE_3D[0]}x{SERVE_3D[1]}x{SERVE_3D[2]}; Ma U[0.1,0.9], Re log-U[500,5000]",
            "arrivals_per_s": args.rate, "requests": count, "slots": args.slots, "cohort": args.cohort,
            "eig": {"sigma": 1.0, "tau": -1.0, "nev": nev, "ncv": FLEET_EIG[3], "tol": FLEET_EIG[4],
                    "gmres": "FGMRES(30) to 1e-10, block-Jacobi 16x16 (3-D 4x4x4), FP32 inverses on tensor cores"},
            "served": {"value": n_srv / t_srv, "unit": "eigenpairs/s", "seconds": t_srv,
                       "latency_ms": {"p50": lat[len(lat) // 2] * 1e3,
                                      "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3},
                       "peak_running": st["peak_running"], "peak_bytes": st["peak_bytes"]},
            "plain_fp64_one_at_a_time": {"value": n_plain / t_plain, "unit": "eigenpairs/s", "seconds": t_plain,
                                         "requests": k},
            "alone_vs_in_mix_max_rel_diff": max(diff) if diff else None}


def reduce_over_ranks(x: float, op: str, device: str) -> float:
    """All-reduce one scalar over the process group ("max" or "sum"); identity without one."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(local_units: float, local_seconds: float, device: str) -> tuple[float, float]:
    """Replicas only: units processed by all ranks over the slowest rank's time; returns (value, t_max)."""
    t_max = reduce_over_ranks(local_seconds, "max", device)
    total = reduce_over_ranks(local_units, "sum", device)
    return total / t_max, t_max


def pair_stencil_jv(args, Stab, torch, q0, g, f, v, out, flush, stream, bytes_jv):
    """The same J v with the compact-scheme right-hand sides in FP32 pair arithmetic
    (stencil_prec 48; sweeps, closures and the pointwise map unchanged), timed like
    the main step, with its largest difference to the FP64-stencil result."""
    from paper_1502_03701_gb300 import binding
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, stencil_prec=48)
    tuned = S.autotune()
    if args.tune_cache:
        binding.autotune_save(args.tune_cache)
    o2 = torch.empty_like(v)
    for _ in range(3):
        S.apply_J(v, o2)
    steps = min(args.steps, 500)
    t = _time_jv(S, v, o2, steps, flush, stream, torch)
    diff = float((o2 - out).abs().max() / out.abs().max())
    S.close()
    return {"value": bytes_jv / (sum(t) / steps) / 1e9, "unit": "GB/s", "ms_per_step": sum(t) / steps * 1e3,
            "steps": steps, "max_rel_diff_vs_fp64_stencil": diff,
            "line_pass_shapes": {ax: {"C": c, "L": l, "kinds": k} for ax, (c, l, k, _) in tuned.items()},
            "arith": "interior right-hand sides of the compact schemes in FP32 pairs (~2^-47 relative); "
                     "Thomas sweeps, closure rows and the pointwise map as in the main step"}


def _time_jv(S, v, out, steps, flush, stream, torch):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        S.apply_J(v, out)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in ev]


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1502_03701_gb300 import Stab, binding, build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()


    # J v on the Ma 0.3 layer (both forms)
    if args.workload == "jv":
        g, f, q0 = _layer(args.nx, args.ny, 0.3, args.nz)
    else:
        g, f, q0 = _layer(EIG_GRID[0], EIG_GRID[1], 0.3)
    n = g.n
    Sj = Stab(q0, g, f.Ma, f.Re, f.Pr)
    if args.tune_cache and os.path.exists(args.tune_cache):
        binding.autotune_load(args.tune_cache)
    tuned = Sj.autotune()                    # line-pass launch shapes for this grid (cached for St)
    if args.tune_cache:
        binding.autotune_save(args.tune_cache)
    St = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    v = torch.from_numpy(si.random_complex(11 + rank, n)).cuda()
    out = torch.empty_like(v)
    for _ in range(max(args.warmup, 3)):
        Sj.apply_J(v, out)
        St.apply_J(v, out)
    jv_tan = _time_jv(St, v, out, 20, flush, stream, torch)
    bytes_jv = n * JV_BYTES_PER_DOF

    if args.workload == "jv":
        sampler = ClockSampler(local, 50)
        barrier()
        with sampler:
            sampler.wait_first_sample()
            Sj.timing(True)
            steps_t = _time_jv(Sj, v, out, args.steps, flush, stream, torch)
            phases = Sj.timing_read()
            Sj.timing(False)
            barrier()
        clock_sum = sampler.summary()
        value, t_max = replica_throughput(args.steps * bytes_jv / 1e9, sum(steps_t), "cuda")
        unit = "GB/s"
        ms_step = t_max / args.steps * 1e3
        roofline = jv_roofline(g, f, phases, sum(steps_t) / args.steps, hbm, statistics.mean(jv_tan))
        config = {"workload": _jv_workload_name(g), "nx": g.nx, "ny": g.ny, "nz": g.nz, "unknowns": g.n,
                  "Ma": f.Ma, "Re": f.Re,
                  "line_pass_shapes": {ax: {"C": c, "L": l, "kinds": k} for ax, (c, l, k, _) in tuned.items()},
                  "eps_mode": "cancellation-free epsilon-quotient",
                  "l2": "flushed between timed steps (512 MB written)",
                  "parallelism": f"replicas{world}"}
        # end to end through the public API: every step copies its input from pinned host memory and
        # its result back; copies run on a second stream, double-buffered, so that step i+1's input
        # and step i-1's result move while step i computes (all inside the timed region)
        vh = [torch.from_numpy(si.random_complex(11 + rank + i, n)).pin_memory() for i in range(2)]
        oh = [torch.empty_like(vh[0]).pin_memory() for _ in range(2)]
        vd = [torch.empty_like(v) for _ in range(2)]
        od = [torch.empty_like(v) for _ in range(2)]
        cstream = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cstream.wait_event(e0)
        with torch.cuda.stream(cstream):
            vd[0].copy_(vh[0], non_blocking=True)
            ev_in[0].record(cstream)
        for i in range(args.steps):
            b = i & 1
            if i + 1 < args.steps:  # next input, once the buffer's previous step has been consumed
                with torch.cuda.stream(cstream):
                    if i >= 1:
                        cstream.wait_event(ev_free[1 - b])
                    vd[1 - b].copy_(vh[(i + 1) & 1], non_blocking=True)
                    ev_in[1 - b].record(cstream)
            stream.wait_event(ev_in[b])
            if i >= 2:
                stream.wait_event(ev_free[b])  # result buffer copied out
            Sj.apply_J(vd[b], od[b])
            ev_out[b].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(ev_out[b])
                oh[b].copy_(od[b], non_blocking=True)
                ev_free[b].record(cstream)
        stream.wait_stream(cstream)
        e1.record(stream)
        barrier()
        e2e_val, _ = replica_throughput(args.steps * bytes_jv / 1e9, e0.elapsed_time(e1) / 1e3, "cuda")
        # conservative single-call figure: L2 flushed before each call (untimed), then copy-in, J v and
        # copy-out timed one call at a time with nothing overlapped
        calls = min(args.steps, 200)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
        for i in range(calls):
            flush.zero_()
            evs[i][0].record(stream)
            vd[0].copy_(vh[i & 1], non_blocking=True)
            Sj.apply_J(vd[0], od[0])
            oh[0].copy_(od[0], non_blocking=True)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        call_s = statistics.mean(a.elapsed_time(b) / 1e3 for a, b in evs)
        e2e = {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 16,
               "overlap": "copies double-buffered on a second stream",
               "l2": "not flushed in this loop: every step's input is new data copied from the host"
                     + ("; the operator's derivative scratch (%.0f MB) exceeds L2" % (g.npts * 16 * 37 / 1e6)
                        if g.dim == 3 else "; the operator's scratch and tables stay in L2 between calls"),
               "single_call": {"value": bytes_jv / call_s / 1e9, "unit": "GB/s", "ms": call_s * 1e3,
                               "l2": "flushed before each call, copies and J v not overlapped"}}
        # every timed phase is one kernel launch of the library (k_norm2, k_temperature_fast,
        # k_line_pass per axis, k_point_fast); the L2 flush between steps is torch's, not counted
        extra = {"gpu_launches": int(sum(v[1] for k, v in phases.items() if k != "dropped"))}
        sampler_summary = clock_sum
        extra["jv_pair_stencil"] = pair_stencil_jv(args, Stab, torch, q0, g, f, v, out, flush, stream, bytes_jv)
        if args.eig_steps > 0:
            extra["eigs"] = small_layer_eigs(args, Stab, torch, rank)
        if args.steps_2d > 0:
            extra["jv_2d_256x512"] = jv_extra(args, Stab, torch, flush, stream, 256, 512)
        if args.gmres_restarts > 0:
            g2, f2, q2 = _layer(256, 512, 0.3)
            extra["gmres_256x512"] = gmres_throughput(args, Stab, torch, q2, g2, f2)
            extra["precond_build_256x512"] = precond_build_256x512(args, Stab, torch)
            extra["preconditioners_256x512"] = preconditioners_256x512(args, Stab, torch)
        if args.fleet > 0 and world == 1:
            extra["jv_batch_64"] = jv_batch_64(args, torch)
            extra["gmres_batch_64"] = gmres_batch_64(args, torch)
            extra["many_small"] = fleet(args, torch)
    else:
        # roofline of the J v kernels from a short phase-timed sample (the solves below are host-driven)
        Sj.timing(True)
        sample_t = _time_jv(Sj, v, out, 50, flush, stream, torch)
        roofline = jv_roofline(g, f, Sj.timing_read(), statistics.mean(sample_t), hbm, statistics.mean(jv_tan))
        Sj.timing(False)
        sweep = (0.3, 0.6, 0.9)
        solver_opts = dict(SOLVER_OPTS)
        if args.eig_precond == 2:  # reduced-operator blocks, block-tridiagonal factors
            solver_opts.update(precond=2, tile=tuple(args.eig_tile or (8, EIG_GRID[1])))
        elif args.eig_tile:
            solver_opts.update(tile=tuple(args.eig_tile))
        if args.eig_lgmres:
            solver_opts.update(lgmres_k=args.eig_lgmres)
        if args.eig_max_restarts:
            solver_opts.update(max_restarts=args.eig_max_restarts)
        handles = []
        for Ma in sweep:
            gg, ff, qq = _layer(EIG_GRID[0], EIG_GRID[1], Ma)
            handles.append(Stab(qq, gg, ff.Ma, ff.Re, ff.Pr, seed=0x5EED + rank, **solver_opts))
        vecs = torch.empty((EIG["nev"], n), dtype=torch.complex128, device="cuda")
        v0h = torch.from_numpy(si.start_vector(0x5EED + rank, n)).pin_memory()
        v0d = torch.empty(n, dtype=torch.complex128, device="cuda")
        vecs_h = torch.empty((EIG["nev"], n), dtype=torch.complex128).pin_memory()

        def solve(S, host_io):
            S.precond_build(EIG["sigma"])  # the build is part of every solve
            if host_io:
                v0d.copy_(v0h, non_blocking=True)
            r = S.eigs(EIG["sigma"], EIG["tau"], EIG["nev"], EIG["ncv"], EIG["tol"], v0=v0d if host_io else None,
                       vecs=vecs)
            if host_io:
                vecs_h.copy_(vecs, non_blocking=True)
            return r

        # warm-up (a full solve takes minutes): per handle the line-pass tuning, a preconditioner build and
        # one inner solve
        for S in handles[:max(1, min(args.warmup, 3))]:
            S.autotune()
            S.precond_build(EIG["sigma"])
            bw = torch.from_numpy(si.random_complex(3, n)).cuda()
            S.solve(EIG["sigma"], bw, torch.zeros_like(bw))
        barrier()
        sampler = ClockSampler(local)
        step_t, results = [], []
        with sampler:
            for s in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = solve(handles[s % 3], False)
                e1.record(stream)
                torch.cuda.synchronize()
                step_t.append(e0.elapsed_time(e1) / 1e3)
                results.append(r)
            barrier()
        sampler_summary = sampler.summary()
        good = [int(np.sum(r.resid[:r.nconv] < RESID_OK)) for r in results]
        value, t_max = replica_throughput(float(sum(good)), sum(step_t), "cuda")
        total_good = value * t_max
        unit = "eigenpairs/s"
        ms_step = t_max / args.steps * 1e3
        lat = sorted(step_t)
        # end to end: start vector from pinned host memory in, eigenvectors out, inside the timed region
        barrier()
        e2e = None
        if args.eig_e2e:
            te0 = time.perf_counter()
            e2e_good = 0
            for s in range(max(1, min(args.steps, 3))):
                r = solve(handles[s % 3], True)
                torch.cuda.synchronize()
                e2e_good += int(np.sum(r.resid[:r.nconv] < RESID_OK))
            te = (time.perf_counter() - te0)
            e2e = {"value": world * e2e_good / te, "unit": "eigenpairs/s", "h2d_bytes_per_step": n * 16,
                   "d2h_bytes_per_step": EIG["nev"] * n * 16 + EIG["nev"] * 24}
        st = [r.stats for r in results]
        jv_per_solve = statistics.mean(s_["jv_calls"] for s_ in st)
        config = {"workload": f"eigs_mixing_layer_{g.nx}x{g.ny}", "nx": g.nx, "ny": g.ny, "Re": f.Re,
                  "Ma_sweep": list(sweep), "sigma": [1.0, 0.0], "tau": [-1.0, 0.0], "nev": EIG["nev"],
                  "ncv": EIG["ncv"], "tol": EIG["tol"], "iram_max_restarts": solver_opts["max_restarts"],
                  "gmres": ("flexible GMRES(50) to 1e-10" if not args.eig_lgmres else
                            f"flexible LGMRES(50, {args.eig_lgmres}) to 1e-10"),
                  "precond": (f"block-Jacobi {solver_opts['tile'][0]}x{solver_opts['tile'][1]} tiles, FP32 inverses "
                              "factorised with tensor-core GEMMs") if solver_opts["precond"] == 1 else
                             (f"reduced-operator block-Jacobi {solver_opts['tile'][0]}x{solver_opts['tile'][1]} tiles, "
                              "FP32 block-tridiagonal factors"),
                  "jv": "exact tangent (FP64)", "warmup": "per handle: tuning, preconditioner build, one inner solve",
                  "l2": "flushed before each timed solve", "parallelism": f"replicas{world}"}
        extra = {"latency_ms": {"p50": statistics.median(lat) * 1e3, "p99": lat[min(len(lat) - 1,
                                                                                      int(0.99 * len(lat)))] * 1e3},
                 "per_step": [{"Ma": sweep[i % 3], "nconv": r.nconv, "good": good[i], "status": r.status,
                               "seconds": step_t[i], "jv_calls": r.stats["jv_calls"],
                               "gmres_iterations": r.stats["gmres_iterations"], "restarts": r.stats["restarts"],
                               "max_resid": float(np.max(r.resid[:max(r.nconv, 1)]))} for i, r in enumerate(results)],
                 # per FGMRES iteration: block apply, 4 J v kernels (tangent), 4 CGS2 kernels, Givens update,
                 # scaling = 11 graph nodes; other J v calls 4; per Arnoldi step about 8 more
                 "gpu_launches": int(sum(s_["gmres_iterations"] * 11 + (s_["jv_calls"] - s_["gmres_iterations"]) * 4
                                         + s_["arnoldi_steps"] * 8 for s_ in st))}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            extra["cpu_baseline"] = cpu_baseline_eigs(g, f, q0, jv_per_solve, total_good / max(args.steps, 1))
        for S in handles:
            S.close()

    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic tanh mixing layer)",
            "config": config, "roofline": roofline,
            "clocks": sampler_summary if sampler_summary else {"sm_mhz": None, "sm_max_mhz": None,
                                                                "reasons": ["short timed region"]},
            "e2e": e2e}
    line.update(extra)
    if args.workload == "jv" and rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_jv(g, f)
    if rank == 0:
        print(json.dumps(line))
    Sj.close()
    St.close()
    if world > 1:
        dist.destroy_process_group()


def run_precond(args):
    """--workload precond: block-Jacobi builds (assembly + inversion of every tile block, FP32 inverses) of
    the --nx x --ny layer with --tile tiles, by the factorisation --factor (0 CUDA cores, 1 tensor cores
    BF16x9, 2 tensor cores TF32), or (--precond 2) of the reduced-operator block-tridiagonal factors;
    --steps timed builds after --warmup builds, then 20 applies timed with CUDA events."""
    import torch
    from paper_1502_03701_gb300 import Stab, build
    build.build()
    g, f, q0 = _layer(args.nx, args.ny, 0.3)
    tile = tuple(args.tile)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=args.precond, tile=tile, precond_prec=32,
             precond_factor=args.factor)
    for i in range(args.warmup):
        S.precond_build(1.0 + 1e-3 * i)
    times = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.precond_build(2.0 + 1e-3 * i)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    q = torch.from_numpy(si.random_complex(1, g.n)).cuda()
    z = torch.empty_like(q)
    S.precond_apply(q, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        S.precond_apply(q, z)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 20
    S.close()
    t = statistics.median(times)
    if args.precond == 2:
        m = 4 * 2 * tile[0]
        nbytes = g.n * 3 * m * 8
        line = {"metric": "reduced-operator block-Jacobi build", "value": 1.0 / t, "unit": "builds/s",
                "config": {"workload": f"precond_reduced_{g.nx}x{g.ny}", "tile": list(tile), "level": m,
                           "levels_per_tile": tile[1] // 2}}
    else:
        b = 4 * tile[0] * tile[1]
        nblk = g.npts // (tile[0] * tile[1])
        nbytes = g.n * b * 8
        line = {"metric": "block-Jacobi build", "value": 8.0 * b ** 3 * nblk / t / 1e12, "unit": "TFLOP/s",
                "config": {"workload": f"precond_build_{g.nx}x{g.ny}", "tile": list(tile), "block": b,
                           "blocks": nblk, "factor": args.factor}}
    line.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                 "higher_is_better": True, "dtype": "f32",
                 "apply": {"ms": apply_ms, "factor_bytes": nbytes, "GB_per_s": nbytes / apply_ms / 1e6}})
    print(json.dumps(line))


def run_serve(args):
    """--workload serve: the served stream as the bench line (eigenpairs/s of the stream; p50/p99 beside)."""
    import torch
    from paper_1502_03701_gb300 import build
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with sampler:
        sampler.wait_first_sample()
        r = serve_stream(args, torch)
    line = {"metric": METRIC, "value": r["served"]["value"], "unit": "eigenpairs/s", "n_gpus": 1,
            "steps": r["requests"], "warmup": 0, "ms_per_step": r["served"]["seconds"] / r["requests"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 inverses)",
            "data": "synthetic (analytic tanh mixing layers)",
            "config": {"workload": "served_stream", "requests": r["requests"], "rate": args.rate},
            "clocks": sampler.summary(), "serve": r}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="jv", choices=["eigs", "jv", "serve", "precond", "inner", "mixed"])
    ap.add_argument("--tile3", type=int, nargs=3, default=[8, 8, 2], help="exact-block tile (--workload mixed)")
    ap.add_argument("--reduced-tile", type=int, nargs=3, default=[4, 64, 2],
                    help="reduced-operator tile (--workload mixed)")
    ap.add_argument("--variants", default="exact:8x8x2,reduced:4x128x2",
                    help="preconditioner variants of --workload inner: kind:TXxTYxTZ[:lgK], comma separated")
    ap.add_argument("--inner-restarts", type=int, default=80, help="FGMRES(50) restart limit (--workload inner)")
    ap.add_argument("--tile", type=int, nargs=2, default=[16, 16], help="block-Jacobi tile (--workload precond)")
    ap.add_argument("--factor", type=int, default=1, help="precond_factor (--workload precond)")
    ap.add_argument("--precond", type=int, default=1, choices=[1, 2], help="preconditioner (--workload precond)")
    ap.add_argument("--eig-lgmres", type=int, default=0, help="lgmres_k of the inner solves (--workload eigs)")
    ap.add_argument("--eig-e2e", type=int, default=1, help="0: skip the end-to-end solves (--workload eigs)")
    ap.add_argument("--eig-max-restarts", type=int, default=0,
                    help="IRAM restart limit of --workload eigs (0: the default 40); a capped solve reports nconv")
    ap.add_argument("--eig-precond", type=int, default=1, choices=[1, 2],
                    help="inner preconditioner of --workload eigs: 1 exact tile blocks, 2 reduced-operator blocks")
    ap.add_argument("--eig-tile", type=int, nargs=2, default=None,
                    help="tile of --workload eigs (default 8 x 32 exact, 8 x 512 reduced)")
    ap.add_argument("--requests", type=int, default=200, help="served stream length (--workload serve)")
    ap.add_argument("--plain-requests", type=int, default=16, help="requests also solved one at a time (serve)")
    ap.add_argument("--cohort", type=int, default=16, help="lockstep cohort size of the server (serve)")
    ap.add_argument("--eig-steps", type=int, default=2)
    ap.add_argument("--gmres-restarts", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--nz", type=int, default=64, help="z points of the J v layer (1: 2-D)")
    ap.add_argument("--ref-jv-per-solve", type=int, default=20000)
    ap.add_argument("--fleet", type=int, default=8, help="instances of the many-small-problems section (0: skip)")
    ap.add_argument("--rate", type=float, default=50.0, help="Poisson arrival rate of the served stream (1/s)")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-gb", type=int, default=64)
    ap.add_argument("--steps-2d", type=int, default=500, help="timed J v steps on the 2-D 256 x 512 layer (0: skip)")
    ap.add_argument("--tune-cache", default="", help="line-pass tuning cache file to load before and save after tuning")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precond":
        run_precond(args)
    elif args.workload == "inner":
        run_inner(args)
    elif args.workload == "mixed":
        run_mixed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
