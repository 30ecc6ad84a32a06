"""Benchmark: multigrid V-cycle throughput of the shifted-HSS Helmholtz solver on GB300.

One step = one full solve of the 2D 512^2 Q1 problem at k = 80 (delta = 0, delta_hat = k,
Sommerfeld on all sides, Gaussian source sigma = 0.05 at a seeded uniform centre), outer
FGMRES in FP64 to a relative residual of 1e-8 with complex-FP32 V-cycles inside the
shifted-HSS preconditioner.  The right side is resident in HBM before timing starts.

Printed (rank 0, one JSON line): V-cycle DoF/s = fine nodes x V-cycles / solve time,
summed over the K timed solves, plus end-to-end (host buffers), the dominant kernel's
roofline, the FP64-oracle CPU baseline, the FP64 V-cycle comparison and the clocks.

--impl reference times the FP64 CPU oracle on the same workload instead.
Under torchrun (N > 1) every rank solves its own copy (weak scaling, no collective on
the data path; one barrier and a max-reduction of the times).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle DoF/s & HBM roofline %; solves/s, p99 latency; mixed vs FP64 at 1e-8"
UNIT = "DoF*V-cycles/s"
WORKLOAD = "2d_n512_k80"
GRIDS = {"2d_n512_k80": "2D unit square, 512x512 Q1 cells (513^2 nodes), Sommerfeld on all sides",
         "3d_n128_k40": "3D unit cube, 128^3 Q1 cells (129^3 nodes), u=0 on z=0, Sommerfeld elsewhere"}
L2_FLUSH_BYTES = 256 << 20
SERVE_REQUESTS = [100]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--delta-hat", default="k")
    ap.add_argument("--workload", default=WORKLOAD, choices=["2d_n512_k80", "3d_n128_k40"],
                    help="2D 512^2 k=80 (default) or 3D 128^3 k=40 (FGMRES restart 60)")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 / roofline / CPU legs")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="requests of the serving workload replayed by the serving leg (its full size is 1000)")
    ap.add_argument("--serve-only", action="store_true", help="run the serving leg alone and print its line")
    ap.add_argument("--max-outer", type=int, default=0,
                    help="cap FGMRES iterations (profiling runs only; 0 = solve to tolerance)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples are kept next to the other run outputs when HH_CLOCKS_DIR names a folder
        folder = os.environ.get("HH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1].split()[0]))
                mx = float(parts[2].split()[0])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


# ----------------------------------------------------------------------------- CPU oracle leg
def host_cores():
    """Cores this process may run on (its affinity mask), and the machine's count."""
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count() or 1
    return usable, os.cpu_count() or usable


def oracle_problem(w):
    """The FP64 oracle's matrices for workload w (Python assembly) and its C OpenMP runner."""
    from oracle import hh_oracle as O
    from oracle import hss_omp as C
    from paper_2506_18694_gb300 import inputs

    g = O.Grid(w.dim, w.n, w.bc)
    prob = O.Problem(g, w.k, w.delta, w.delta_hat, O.Options())
    f = inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)
    r = prob.mats[0][1] @ f  # b = M f
    return g, C.COracle(prob), r, C


def oracle_vcycle_rate(w, seconds=8.0):
    """The oracle's HSS steps (one V-cycle each, FP64 CSR, OpenMP over rows) on the workload,
    on all usable host cores and on one core: DoF*V-cycles/s for each."""
    g, c, r, C = oracle_problem(w)
    usable, machine = host_cores()
    saved = C.COracle.threads()
    try:
        C.COracle.threads(usable)
        steps_all, dt_all = c.time_steps(r, seconds)
        C.COracle.threads(1)
        steps_one, dt_one = c.time_steps(r, seconds)
    finally:
        C.COracle.threads(saved)
    return {"value": g.N * steps_all / dt_all, "unit": UNIT, "cores": usable, "machine_cores": machine,
            "kind": "oracle",
            "sample": f"{steps_all} HSS steps (one V(2,2) cycle each) of the {w.name} workload in {dt_all:.1f} s "
                      f"on {usable} threads; FP64 CSR, plain C with OpenMP over rows (oracle/hss_omp.c)",
            "one_core": {"value": g.N * steps_one / dt_one, "cores": 1,
                         "sample": f"{steps_one} HSS steps in {dt_one:.1f} s on 1 thread"}}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return
    from paper_2506_18694_gb300 import inputs

    w = inputs.workload(args.workload, args.delta_hat)
    g, c, r, C = oracle_problem(w)
    usable, machine = host_cores()
    C.COracle.threads(usable)
    per_step = 4 if w.dim == 2 else 1  # one bounded sample per step: HSS steps (V-cycles)
    for _ in range(args.warmup):
        c.time_steps(r, 0.0, per_step)
    times = []
    for _ in range(args.steps):
        _, dt = c.time_steps(r, 0.0, per_step)
        times.append(dt)
    tot = sum(times)
    value = g.N * per_step * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "delta_hat": w.delta_hat, "nodes": g.N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": usable, "machine_cores": machine, "kind": "oracle",
                         "sample": f"{per_step} HSS steps (V-cycles) per step of the {w.name} workload, FP64 CSR, "
                                   f"plain C with OpenMP over rows on {usable} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- native arm
def max_over_ranks(x, device):
    """The largest of every rank's x (each rank passes its own; all get the maximum): the job
    takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nodes, vcycles_per_rank, total_s, world):
    """Whole-job DoF x V-cycles per second: every rank solves its own copy of the workload
    (replicas, weak scaling), timed by the slowest rank."""
    return world * nodes * vcycles_per_rank / total_s


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    from paper_2506_18694_gb300 import hh, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    SERVE_REQUESTS[0] = args.serve_requests
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": measure_serving(hh, inputs, torch, args.serve_requests)}), flush=True)
        return
    w = inputs.workload(args.workload, args.delta_hat)
    opts = hh.default_options(precision=hh.HH_C64, restart=60 if w.dim == 3 else 30)
    if args.max_outer > 0:
        opts.max_outer = args.max_outer
    prob = hh.Problem(w.dim, w.n, w.k, w.delta, w.delta_hat, w.bc, opts)
    N = prob.nodes()
    f = torch.from_numpy(inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)).cuda()
    b = prob.load_vector(f)
    u = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    infos = []
    for _ in range(args.warmup):
        _, info = prob.solve(b, w.tol, u=u)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        barrier()
        for s in range(args.steps):
            flush.zero_()  # evict L2 between steps (outside the timed pair)
            ev[s][0].record(stream)
            _, info = prob.solve(b, w.tol, u=u)
            ev[s][1].record(stream)
            infos.append(info)
        barrier()
    step_ms = [a.elapsed_time(z) for a, z in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        total_s = max_over_ranks(total_s, "cuda")
    vcycles = sum(i.vcycles for i in infos)
    value = job_value(N, vcycles, total_s, world)
    launches = sum(i.kernel_launches for i in infos)

    # end to end through the public API with host buffers (copies inside the timed region)
    rhs_host = torch.empty(N, dtype=torch.complex128).pin_memory()
    rhs_host.copy_(b.cpu())
    u_host = torch.empty(N, dtype=torch.complex128).pin_memory()
    e2e_ms, e2e_cycles = [], 0
    for s in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = prob.solve_host(rhs_host.numpy(), w.tol, out=u_host.numpy())
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_cycles += info.vcycles
    e2e_value = world * N * e2e_cycles / (sum(e2e_ms) / 1e3)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = measure_extras(hh, inputs, torch, w, prob, b, u, infos[-1], opts)
    prob.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 V-cycles / c128 FGMRES",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": GRIDS[w.name],
                       "k": w.k, "delta": w.delta, "delta_hat": w.delta_hat, "tol": w.tol,
                       "levels": opts.levels, "smoother": f"V({opts.nu_pre},{opts.nu_post}) Jacobi w={opts.omega or (0.5 if w.dim == 3 else 0.6)}",
                       "nu_coarse": opts.nu_coarse, "restart": opts.restart, "l2": "flushed between steps",
                       "per_rank": "one independent solve per step"},
            "solves_per_s": world * args.steps / total_s,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "per_solve": {"outer_its": infos[-1].outer_its, "vcycles": infos[-1].vcycles,
                          "rel_residual": infos[-1].rel_residual},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16,
                    "ms_per_step": float(np.mean(e2e_ms))},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def profiled_traffic(profile, source):
    """DRAM bytes per launch recorded in a committed ncu summary, if the kernel source is unchanged."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        sha = hashlib.sha1(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    traffic, recorded = None, None
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = int(line.split(":")[1])
        if line.startswith("kernel_source_sha1:"):
            recorded = line.split(":")[1].split()[0]
    return traffic if recorded == sha else None


def time_kernel(torch, fn, reps, flush=None):
    """Average device time of one fn() launch on the current stream (CUDA events).

    With flush: each launch timed alone after an L2 flush.  Without: reps launches back to
    back between one pair of events (inputs larger than L2 make every launch read HBM).
    """
    s = torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    if flush is None:
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            fn()
        z.record(s)
        z.synchronize()
        return a.elapsed_time(z) / reps / 1e3
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        z.record(s)
        z.synchronize()
        tot += a.elapsed_time(z)
    return tot / reps / 1e3


def sweep_roofline(hh, torch, w, prob, b, hbm, peak_src, flush):
    """HBM roofline of the scaled-Jacobi sweep (24 algorithmic bytes per node) on a grid whose
    vectors exceed L2 (2D 4097^2 or 3D 257^3), timed with CUDA events over back-to-back launches,
    and its effective rate at the workload's own size (L2-resident)."""
    N = prob.nodes()
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    b32 = b.to(torch.complex64)
    y = torch.empty_like(x)
    t_w = time_kernel(torch, lambda: prob.jacobi(0, b32, x, y), 50, flush)
    nbig = 4096 if w.dim == 2 else 256
    big = hh.Problem(w.dim, nbig, w.k, w.delta, w.delta_hat, w.bc, hh.default_options(precision=hh.HH_C64, levels=2,
                                                                                       restart=1))
    Nb = big.nodes()
    xb = torch.randn(Nb, dtype=torch.complex64, device="cuda")
    bb = torch.randn(Nb, dtype=torch.complex64, device="cuda")
    yb = torch.empty_like(xb)
    t_b = time_kernel(torch, lambda: big.jacobi(0, bb, xb, yb), 20)
    big.close()
    ach = 24 * Nb / t_b / 1e9
    if w.dim == 2:
        kname, prof, src = ("k_march2p<float, JACOBI, 8> (scaled-Jacobi sweep, persistent)", "jacobi_2d_4097sq_c64.md",
                            "paper_2506_18694_gb300/csrc/march2.cu")
        size = "4097^2 nodes (3 x 134 MB vectors > L2)"
    else:
        kname, prof, src = ("k_march3<float, JACOBI, 4> (scaled-Jacobi sweep)", "jacobi_3d_257cube_c64.md",
                            "paper_2506_18694_gb300/csrc/march3.cu")
        size = "257^3 nodes (3 x 136 MB vectors > L2)"
    return {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": profiled_traffic(prof, src), "size": size, "bytes_per_node": 24, "peak_source": peak_src,
            "at_workload": {"nodes": N, "us": t_w * 1e6, "effective_gbs": 24 * N / t_w / 1e9,
                            "note": "the workload's vectors are L2-resident"}}


def measure_c3(hh, inputs, torch, hbm, peak_src, flush, steps=2):
    """The 3D unit-cube workload: 128^3 Q1 cells, k = 40, delta_hat = k, u = 0 on z = 0, complex64
    V-cycles inside FGMRES(60) to 1e-8; device-resident solves timed with CUDA events (L2 flushed
    before each), one end-to-end solve through hh_solve_host, and the 3D sweep's roofline."""
    w = inputs.workload("3d_n128_k40")
    opts = hh.default_options(precision=hh.HH_C64, restart=60)
    stream = torch.cuda.current_stream()
    with hh.Problem(w.dim, w.n, w.k, w.delta, w.delta_hat, w.bc, opts) as p:
        N = p.nodes()
        f = torch.from_numpy(inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)).cuda()
        b = p.load_vector(f)
        u = torch.empty_like(b)
        p.solve(b, w.tol, u=u)  # warm-up (graph capture)
        ms, infos = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = p.solve(b, w.tol, u=u)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        rhs_host = b.cpu().numpy()
        out_host = np.empty_like(rhs_host)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ie = p.solve_host(rhs_host, w.tol, out=out_host)
        e2e_s = time.perf_counter() - t0
        roof = sweep_roofline(hh, torch, w, p, b, hbm, peak_src, flush)
    tot = sum(ms) / 1e3
    return {"workload": w.name, "grid": GRIDS[w.name], "k": w.k, "delta_hat": w.delta_hat, "tol": w.tol,
            "restart": 60, "value": N * sum(i.vcycles for i in infos) / tot, "unit": UNIT,
            "ms_per_solve": 1e3 * tot / steps,
            "per_solve": {"outer_its": infos[-1].outer_its, "vcycles": infos[-1].vcycles,
                          "rel_residual": infos[-1].rel_residual},
            "e2e": {"value": N * ie.vcycles / e2e_s, "unit": UNIT, "h2d_bytes_per_step": N * 16,
                    "d2h_bytes_per_step": N * 16, "ms_per_step": 1e3 * e2e_s},
            "roofline": roof}


def measure_extras(hh, inputs, torch, w, prob, b, u_mixed, info_mixed, opts):
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # dominant kernel: fine-level Jacobi sweep (c64).  24 algorithmic bytes per node
    # (read x, b; write x').  Timed at the workload size (L2-resident) and on a 4096^2
    # grid whose vectors (134 MB each) exceed L2, which is where the HBM roofline applies.
    out["roofline"] = sweep_roofline(hh, torch, w, prob, b, hbm, peak_src, flush)

    # the 3D 128^3, k = 40 workload (complex64 V-cycles, FGMRES(60) to 1e-8) with the roofline
    # of its sweep kernel on 257^3 nodes
    if w.dim == 2:
        try:
            out["c3"] = measure_c3(hh, inputs, torch, hbm, peak_src, flush)
        except Exception as e:
            out["c3"] = {"failed": str(e)}

    # FP64 V-cycles on the same workload (single solve), error vs the mixed result
    opts64 = hh.default_options(precision=hh.HH_C128, restart=opts.restart)
    with hh.Problem(w.dim, w.n, w.k, w.delta, w.delta_hat, w.bc, opts64) as p64:
        p64.solve(b, w.tol)  # warm (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u64, i64 = p64.solve(b, w.tol)
        t64 = time.perf_counter() - t0
    diff = float(torch.linalg.vector_norm(u64 - u_mixed) / torch.linalg.vector_norm(u64))
    out["fp64_vcycles"] = {"solve_ms": 1e3 * t64, "outer_its": i64.outer_its, "vcycles": i64.vcycles,
                           "rel_residual": i64.rel_residual, "value": prob.nodes() * i64.vcycles / t64,
                           "mixed_vs_fp64_rel_diff": diff}

    # the paper's delta_hat = 2 on the same grid and source (mixed precision).  One
    # V(2,2)-Jacobi cycle per HSS step is too inexact over ceil(k) = 80 steps (FGMRES
    # stagnates); two cycles per step converge.
    w2 = inputs.workload(w.name, 2.0)
    with hh.Problem(w2.dim, w2.n, w2.k, w2.delta, w2.delta_hat, w2.bc, hh.default_options(cycles_per_hss=2)) as p2:
        p2.solve(b, w.tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, i2 = p2.solve(b, w.tol)
        t2 = time.perf_counter() - t0
    out["delta_hat_2"] = {"cycles_per_hss": 2, "solve_ms": 1e3 * t2, "outer_its": i2.outer_its, "vcycles": i2.vcycles,
                          "rel_residual": i2.rel_residual, "value": prob.nodes() * i2.vcycles / t2}

    # the paper's preconditioned Richardson outer iteration on the same grid and source
    # (delta_hat = 2, two cycles per HSS step)
    try:
        with hh.Problem(w2.dim, w2.n, w2.k, w2.delta, w2.delta_hat, w2.bc,
                        hh.default_options(cycles_per_hss=2, outer=hh.HH_OUTER_RICHARDSON, max_outer=400)) as pr:
            pr.solve(b, w.tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ir = pr.solve(b, w.tol)
            tr = time.perf_counter() - t0
        out["richardson_delta_hat_2"] = {"cycles_per_hss": 2, "solve_ms": 1e3 * tr, "outer_its": ir.outer_its,
                                         "vcycles": ir.vcycles, "rel_residual": ir.rel_residual,
                                         "value": prob.nodes() * ir.vcycles / tr}
    except Exception as e:
        out["richardson_delta_hat_2"] = {"failed": str(e)}

    # the paper's cycle type: W-cycles, one per HSS step, delta_hat = 2
    try:
        with hh.Problem(w2.dim, w2.n, w2.k, w2.delta, w2.delta_hat, w2.bc,
                        hh.default_options(cycle_gamma=2, max_outer=400)) as pw:
            pw.solve(b, w.tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, iw = pw.solve(b, w.tol)
            tw = time.perf_counter() - t0
        out["w_cycle_delta_hat_2"] = {"cycle": "W(2,2)", "solve_ms": 1e3 * tw, "outer_its": iw.outer_its,
                                      "cycles": iw.vcycles, "rel_residual": iw.rel_residual}
    except Exception as e:
        out["w_cycle_delta_hat_2"] = {"failed": str(e)}

    # the paper's multigrid settings (Sec. 5.3): W-cycles with GMRES(5) and a Jacobi
    # preconditioner on every level, one cycle per HSS step, delta_hat = 2; on 2D 256^2 at
    # k = 20, where V(2,2)-Jacobi with two cycles per HSS step stagnates
    try:
        out["gmres_smoother"] = measure_gmres_smoother(hh, inputs, torch, w)
    except Exception as e:
        out["gmres_smoother"] = {"failed": str(e)}

    # the mixed formulation (Sec. 2) with the paper's multigrid for it (Sec. 5.3: two W-cycles
    # per HSS step, GMRES(4) with Jacobi on every level), delta_hat = 2, against the primal one
    try:
        out["mixed_formulation"] = measure_mixed(hh, inputs, torch, w)
    except Exception as e:
        out["mixed_formulation"] = {"failed": str(e)}

    # serving: Poisson arrivals of mixed 2D/3D requests through the solve server
    try:
        out["serving"] = measure_serving(hh, inputs, torch, SERVE_REQUESTS[0])
    except Exception as e:
        out["serving"] = {"failed": str(e)}

    # uneven grids: packed launches against one solve at a time and against worker streams
    try:
        out["pack_uneven"] = measure_pack(hh, inputs, torch)
    except Exception as e:
        out["pack_uneven"] = {"failed": str(e)}

    # batched: 64 right sides on 2D 256^2, k from {20, 40, 80}, one problem object
    try:
        out["batch64"] = measure_batch(hh, inputs, torch)
    except Exception as e:  # report, do not hide the other numbers
        out["batch64"] = {"failed": str(e)}

    # FP64 CPU oracle on a bounded sample of the same workload, all cores and one core
    try:
        out["cpu_baseline"] = oracle_vcycle_rate(w)
    except Exception as e:  # the CPU leg must not hide the GPU numbers
        out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": f"failed: {e}"}
    return out


def measure_gmres_smoother(hh, inputs, torch, w, n=256, k=20.0):
    f = torch.from_numpy(inputs.gaussian_source(2, n, tuple(w.centre)[:2], w.sigma)).cuda()
    legs = {
        "gmres5_w_cycle": dict(cycle_gamma=2, nu_pre=5, nu_post=5, nu_coarse=5, smoother=hh.HH_SMOOTH_GMRES),
        "jacobi_v22_two_cycles": dict(cycles_per_hss=2),
    }
    res = {"grid": f"2D {n}^2 Q1 cells, Sommerfeld", "k": k, "delta_hat": 2.0, "tol": w.tol, "levels": 4}
    for name, o in legs.items():
        with hh.Problem(2, n, k, 0.0, 2.0, [hh.SOMMERFELD] * 4, hh.default_options(max_outer=300, **o)) as p:
            b = p.load_vector(f)
            p.solve(b, w.tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = p.solve(b, w.tol)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        res[name] = {"solve_s": t, "outer_its": info.outer_its, "cycles": info.vcycles,
                     "rel_residual": info.rel_residual, "converged": info.rel_residual <= w.tol,
                     "kernel_launches": info.kernel_launches}
    return res


def measure_mixed(hh, inputs, torch, w, n=256, k=20.0):
    f = torch.from_numpy(inputs.gaussian_source(2, n, tuple(w.centre)[:2], w.sigma)).cuda()
    mg = dict(cycle_gamma=2, cycles_per_hss=2, nu_pre=4, nu_post=4, nu_coarse=4, smoother=hh.HH_SMOOTH_GMRES)
    res = {"grid": f"2D {n}^2 Q1 cells, Sommerfeld", "k": k, "delta_hat": 2.0, "tol": w.tol, "levels": 4,
           "multigrid": "two W-cycles per HSS step, GMRES(4) with Jacobi on every level"}
    for name, form in (("mixed", hh.HH_FORM_MIXED), ("primal", hh.HH_FORM_PRIMAL)):
        with hh.Problem(2, n, k, 0.0, 2.0, [hh.SOMMERFELD] * 4,
                        hh.default_options(max_outer=300, formulation=form, **mg)) as p:
            bu = p.load_vector(f)
            if form == hh.HH_FORM_MIXED:
                # (F_sigma, F_u) = (0, M f / (delta - i k)), delta = 0
                b = torch.cat([torch.zeros(p.system_size() - bu.numel(), dtype=bu.dtype, device=bu.device),
                               bu * (1j / k)])
            else:
                b = bu
            p.solve(b, w.tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = p.solve(b, w.tol)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        res[name] = {"solve_s": t, "outer_its": info.outer_its, "cycles": info.vcycles,
                     "rel_residual": info.rel_residual, "converged": info.rel_residual <= w.tol,
                     "unknowns": int(b.numel()), "kernel_launches": info.kernel_launches}
    return res


def serving_options(hh):
    """Options of the serving workload's first solve (V(2,2)-Jacobi cycles at delta_hat = k,
    FGMRES restart 60, given up once it stalls) and of the fallback solve for requests that do
    not converge with them (the paper's multigrid at delta_hat = 2: W-cycles with GMRES(5) and a
    Jacobi preconditioner on every level, Sec. 5.3)."""
    first = hh.default_options(precision=hh.HH_C64, restart=60, max_outer=3000, stall_cycles=4)
    fallback = hh.default_options(precision=hh.HH_C64, restart=30, max_outer=600, cycle_gamma=2, nu_pre=5,
                                  nu_post=5, nu_coarse=5, smoother=hh.HH_SMOOTH_GMRES)
    return first, fallback


def measure_serving(hh, inputs, torch, count, slots=4, load=0.8, tol=1e-8, pack=16, pack_max_hss=60):
    """The serving workload (mixed 2D/3D grids and wavenumbers, nodal Gaussian sources, tol 1e-8)
    through the solve server with the fallback policy of serving_options, every request on one of
    `slots` worker slots (its own stream; kernels of different requests overlap on the device).
    Pass 1 queues every request at once: the server's capacity (solves/s) and each request's
    service record.  Pass 2 replays them with the seeded Poisson arrival times rescaled to `load`
    times that capacity: latency p50/p99.  Pass 3 queues them all at once with the 2D requests of
    at most `pack_max_hss` HSS steps as members of one pack of `pack` slots (their V-cycle passes
    share launches), for comparison.  A request that ends above tol counts as failed and not in solves/s."""
    reqs = inputs.serving_requests(count)
    srcs = [r.source() for r in reqs]
    first, fallback = serving_options(hh)
    budget = int(torch.cuda.mem_get_info()[0] * 0.6)

    def run(arrivals, packed=False):
        with hh.Server(slots=slots, budget_bytes=budget, options=first) as srv:
            srv.set_fallback(fallback, 2.0)
            if packed and pack > 0:
                srv.set_pack(pack, pack_max_hss)
            t0 = time.perf_counter()
            tickets = []
            for r, f, a in zip(reqs, srcs, arrivals):
                now = time.perf_counter() - t0
                if a > now:
                    time.sleep(a - now)
                tickets.append(srv.submit(r.dim, r.n, r.k, r.delta, r.delta_hat, r.bc, f, tol, nodal=True))
            res = [srv.wait(t) for t in tickets]
            span = time.perf_counter() - t0
            st = srv.stats()
        return res, span, st

    sat, sat_span, sat_st = run([0.0] * len(reqs))
    ok_sat = [x[1].rel_residual <= tol for x in sat]
    cap = sum(ok_sat) / sat_span
    rate = load * len(reqs) / sat_span
    arr = [r.arrival / reqs[-1].arrival * (len(reqs) / rate) for r in reqs]  # seeded Poisson times, rescaled
    res, span, st = run(arr)
    ok = [x[1].rel_residual <= tol for x in res]
    unp, unp_span, unp_st = run([0.0] * len(reqs), packed=True)
    ok_unp = [x[1].rel_residual <= tol for x in unp]
    lat = [x[2] for x in res]
    work = sum(r.nodes * x[1].vcycles for r, x in zip(reqs, res))
    return {
        "workload": "serving: half 2D n in [64,1024], half 3D n in [32,96] (log-uniform, multiple of 8), "
                    "k uniform [10,160] capped at 2 pi n/10, tol 1e-8; first solve V(2,2)-Jacobi at delta_hat = k "
                    "(FGMRES(60), given up after 4 restart cycles without halving the residual), fallback the "
                    "paper's multigrid at delta_hat = 2 (W-cycles, GMRES(5) + Jacobi on every level)",
        "requests": len(reqs), "of_full": 1000, "slots": slots, "pack_slots": pack, "budget_bytes": budget,
        "capacity_solves_per_s": cap, "arrival_rate_per_s": rate, "load": load,
        "solves_per_s": sum(ok) / span, "failed": len(ok) - sum(ok), "failed_saturated": len(ok_sat) - sum(ok_sat),
        "fallbacks": sum(x[1].fallback for x in res),
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
        "queue_ms_p50": 1e3 * float(np.percentile([x[3] for x in res], 50)),
        "value": work / span, "unit": UNIT,
        "max_rel_residual": max(x[1].rel_residual for x in res),
        "max_concurrent": st["max_concurrent"], "peak_bytes": st["peak_bytes"],
        "problems_created": st["problems_created"], "problems_reused": st["problems_reused"],
        "problems_evicted": st["problems_evicted"],
        "saturated": {"solves_per_s": cap, "span_s": sat_span, "max_concurrent": sat_st["max_concurrent"]},
        "saturated_with_pack": {"solves_per_s": sum(ok_unp) / unp_span, "span_s": unp_span,
                                "failed": len(ok_unp) - sum(ok_unp), "max_concurrent": unp_st["max_concurrent"],
                                "pack_max_hss_steps": pack_max_hss,
                                "note": "2D requests of at most pack_max_hss_steps HSS steps in one pack (every "
                                        "member advances one FGMRES iteration per round, so a round lasts as "
                                        "long as the longest member's HSS loop); the others on worker slots"},
        "per_request": [[r.dim, r.n, round(r.k, 1), x[1].outer_its, x[1].rel_residual, round(x[1].seconds, 3),
                         x[1].fallback] for r, x in zip(reqs, sat)],
    }


def measure_pack(hh, inputs, torch, tol=1e-8):
    """Problems on uneven 2D grids (inputs.uneven_requests: 48 solves, n from 64 to 256, k 20 or
    40) through the solve server three ways, all queued at once: one at a time (1 worker slot),
    on 4 worker slots (their own streams), and as members of one pack (their V-cycle passes share
    launches; 1 worker slot for nothing else).  Each way must give the same solutions bit for
    bit; solves/s for each."""
    reqs = inputs.uneven_requests()
    srcs = [r.source() for r in reqs]
    opts = hh.default_options(precision=hh.HH_C64)
    budget = int(torch.cuda.mem_get_info()[0] * 0.6)

    def run(slots, pack):
        with hh.Server(slots=slots, budget_bytes=budget, options=opts) as srv:
            if pack:
                srv.set_pack(pack)
            t0 = time.perf_counter()
            tickets = [srv.submit(r.dim, r.n, r.k, r.delta, r.delta_hat, r.bc, f, tol, nodal=True)
                       for r, f in zip(reqs, srcs)]
            res = [srv.wait(t) for t in tickets]
            return res, time.perf_counter() - t0

    out = {"workload": "48 solves on 2D grids n in {64, 96, ..., 256} (seed 6), k in {20, 40}, delta_hat = k, "
                       "tol 1e-8, all queued at once", "requests": len(reqs)}
    ref = None
    for name, slots, pack in (("sequential", 1, 0), ("workers4", 4, 0), ("pack48", 1, 48)):
        res, span = run(slots, pack)
        us = [x[0] for x in res]
        if ref is None:
            ref = us
        out[name] = {"solves_per_s": len(reqs) / span, "span_s": span,
                     "max_rel_residual": max(x[1].rel_residual for x in res),
                     "equal_to_sequential_bitwise": all(np.array_equal(a, b) for a, b in zip(us, ref))}
    out["pack_vs_sequential"] = out["sequential"]["span_s"] / out["pack48"]["span_s"]
    out["pack_vs_workers4"] = out["workers4"]["span_s"] / out["pack48"]["span_s"]
    return out


def measure_batch(hh, inputs, torch):
    """The 64-problem batch solved at once (complex64 V-cycles, autotuned tile shapes) against
    solving the problems one after another, in mixed precision and in FP64.  The sequential
    times are estimated from one solo solve per k class (that problem's own right side),
    multiplied by the class size."""
    w = inputs.batch_workload()
    N = w.nodes
    f = torch.from_numpy(w.sources().reshape(-1)).cuda()
    ks = np.array(w.ks)
    opts = hh.default_options(precision=hh.HH_C64, autotune=1)
    t0 = time.perf_counter()
    pb = hh.Problem(2, w.n, ks, w.delta, np.array(w.delta_hats), w.bc, opts)
    create_s = time.perf_counter() - t0
    b = pb.load_vector(f)
    u = torch.empty_like(b)
    pb.solve(b, w.tol, u=u)  # graph capture
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    _, infos = pb.solve(b, w.tol, u=u)
    e1.record(s)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    shapes = pb.autotune()
    pb.close()
    its = [i.outer_its for i in infos]
    vcycles = sum(i.vcycles for i in infos)
    solo = {}
    for kk in sorted(set(w.ks)):
        i = list(w.ks).index(kk)
        bi = b[i * N:(i + 1) * N].clone()
        for name, prec in (("mixed", hh.HH_C64), ("fp64", hh.HH_C128)):
            with hh.Problem(2, w.n, kk, w.delta, w.delta_hats[i], w.bc, hh.default_options(precision=prec)) as p:
                p.solve(bi, w.tol)
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                _, info = p.solve(bi, w.tol)
                z.record(s)
                z.synchronize()
                solo[(kk, name)] = (a.elapsed_time(z) / 1e3, info.outer_its, info.rel_residual)
    count = {kk: list(w.ks).count(kk) for kk in set(w.ks)}
    seq = {name: sum(count[kk] * solo[(kk, name)][0] for kk in count) for name in ("mixed", "fp64")}
    return {
        "workload": w.name, "problems": w.count, "grid": "2D 256^2 Q1 cells (257^2 nodes) each, Sommerfeld",
        "k_counts": {str(k): c for k, c in sorted(count.items())}, "delta_hat": "k", "tol": w.tol,
        "solve_s": t_batch, "solves_per_s": w.count / t_batch, "value": N * vcycles / t_batch, "unit": UNIT,
        "outer_its": {"min": min(its), "max": max(its)},
        "max_rel_residual": max(i.rel_residual for i in infos),
        "create_s_with_autotune": create_s, "tuned_kernels": len(shapes),
        "solo": {f"k{int(kk)}_{name}": {"solve_s": v[0], "outer_its": v[1], "rel_residual": v[2]}
                 for (kk, name), v in sorted(solo.items())},
        "sequential_estimate_s": seq,
        "speedup_vs_sequential_mixed": seq["mixed"] / t_batch,
        "speedup_vs_sequential_fp64": seq["fp64"] / t_batch,
        "note": "sequential times = class size x one solo solve per k class",
    }


if __name__ == "__main__":
    main()
