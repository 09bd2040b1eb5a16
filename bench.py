#!/usr/bin/env python
"""RK45 cell-steps/s of the micromagnetic hot path on GB300.

One step = one accepted Dormand-Prince RK45 step of the whole path (demag FFT
convolution, exchange stencil, anisotropy, Zeeman, LL torque, stage updates,
error reduction and step control) over the whole grid.

Default workload: the 3-D ellipsoid, 128 x 128 x 32 cells of 3 nm (demag
convolution padded to 256 x 256 x 64), the configuration on which both the
cell-steps/s and the HBM-roofline fraction of the demag convolution are
quoted; the 256 x 256 x 1 grain film is reported beside it ("film").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the path does not shard (one simulation per GPU); N ranks run N
independent replicas ("replicas only", weak scaling), no collective on the
data path.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1406_7635_gb300.workloads import WORKLOADS  # noqa: E402

METRIC = "RK45 cell-steps/s at 256²×1 and 128²×32; demag FFT-conv % of HBM roofline"
DEFAULT_WORKLOAD = "ellipsoid_128x128x32"
SIDE_WORKLOAD = "grains_256x256x1"


def max_over_ranks(x, world, device):
    """The largest of the ranks' values of x (a time): every rank gets it.
    Replicas share nothing else; this is the only collective of a run."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Weak-scaling aggregate: the units every rank processed divided by the
    slowest rank's time."""
    return units_per_rank * world / seconds_max


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _pad(n):
    return 1 if n == 1 else 1 << (2 * n - 2).bit_length()


def algorithmic_demag_bytes(p):
    """Minimum HBM bytes of one demag convolution (50 B per cell at 128 x 128
    x 32): read m (3 x 4 B) and the mask/region bytes (2 B) per cell, the
    kernel spectrum octant (6 float32 per octant point), write B (3 x 4 B)
    per cell."""
    def half(n):
        return 1 if n == 1 else _pad(n) // 2 + 1
    octant = half(p.nx) * half(p.ny) * half(p.nz)
    return p.ncells * (12 + 2 + 12) + 6 * 4 * octant


def five_pass_demag_bytes(p):
    """HBM bytes of the unfused five-pass design (x R2C, y, z*K*z^-1, y^-1,
    x C2R, each pass through memory, pruned to the rows that carry data):
    340 B per cell at 128 x 128 x 32."""
    px, py, pz = _pad(p.nx), _pad(p.ny), _pad(p.nz)
    hx = px // 2 + 1 if px > 1 else 1
    c8 = 3 * 8
    x_out = c8 * hx * p.ny * p.nz
    y_out = c8 * hx * py * p.nz
    pass1 = p.ncells * (12 + 2) + x_out
    kern = algorithmic_demag_bytes(p) - p.ncells * 26
    if pz == 1:                                   # 2-D: y*K*y^-1 is one pass
        return pass1 + 2 * x_out + kern + x_out + 12 * p.ncells
    pass2 = x_out + y_out
    pass3 = 2 * y_out + kern                      # z pruned both ways, + kernel
    pass4 = y_out + x_out
    pass5 = x_out + 12 * p.ncells
    return pass1 + pass2 + pass3 + pass4 + pass5


def algorithmic_demag_flops(p):
    """Floating-point operations of one demag convolution, counted as 5 L
    log2 L per complex transform of length L and 2.5 L log2 L per real one,
    over the lines that carry data (x: ny*nz rows per component, y: hx*nz
    columns, z: hx*py columns), forward and inverse, plus the spectral
    product (30 flops per frequency point in 3-D, 14 in 2-D where Kxz = Kyz
    = 0).  823 MFLOP at 128 x 128 x 32."""
    from math import log2
    px, py, pz = _pad(p.nx), _pad(p.ny), _pad(p.nz)
    hx = px // 2 + 1 if px > 1 else 1
    f = 0.0
    if px > 1:
        f += 2 * 3 * p.ny * p.nz * 2.5 * px * log2(px)
    if py > 1:
        f += 2 * 3 * hx * p.nz * 5 * py * log2(py)
    if pz > 1:
        f += 2 * 3 * hx * py * 5 * pz * log2(pz)
    f += (30 if pz > 1 else 14) * hx * py * pz
    return f


# FP32 issue peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x
# 2.070 GHz maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12

CONV_SOURCES = ("paper_1406_7635_gb300/csrc/fft_fused.cu", "paper_1406_7635_gb300/csrc/fft.cuh")


def conv_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in CONV_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def conv_traffic(workload):
    """DRAM bytes of one convolution from the committed ncu summary of the
    same workload, or None when the convolution's sources changed since the
    counters were taken."""
    prof = os.path.join(ROOT, "profiles", f"demag_conv_{workload}.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        d = json.load(f)
    if d.get("src_sha256_16") != conv_sources_sha():
        return None
    return d.get("dram_bytes_per_conv")


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1406_7635_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    from paper_1406_7635_gb300 import mm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def bench_workload(name, steps, warmup):
        p = WORKLOADS[name]()
        ctx = mm.Context.from_problem(p, device=local_rank, stream=stream.cuda_stream)
        ctx.step(warmup)
        s0 = ctx.get_stats()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local_rank)
        clocks.start()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()                  # evict the previous step's data from L2
                starts[k].record(stream)
                ctx.step(1)
                ends[k].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if world > 1:
            torch.distributed.barrier()
        dev_s = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3
        s1 = ctx.get_stats()
        return p, ctx, dev_s, s0, s1, clk

    def reduce_max(x):
        return max_over_ranks(x, world, dev)

    K, W = args.steps, args.warmup
    p, ctx, dev_s, s0, s1, clk = bench_workload(args.workload, K, W)
    t_max = reduce_max(dev_s)
    value = whole_job_rate(p.ncells * K, world, t_max)
    attempts = (s1["accepted"] + s1["rejected"]) - (s0["accepted"] + s0["rejected"])
    launches = s1["launches"] - s0["launches"]

    # demag convolution alone (the dominant kernel sequence), events on the
    # context's stream, L2 flushed before each launch
    m_dev = torch.tensor(p.m0.astype(np.float32), device=dev).contiguous()
    b_dev = torch.empty_like(m_dev)
    R = 50
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(R)]
    for _ in range(3):
        ctx.demag_apply(m_dev, b_dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            ctx.demag_apply(m_dev, b_dev)
            b.record(stream)
    torch.cuda.synchronize()
    conv_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / R
    peaks, peak_kind = measured_peaks()
    alg = algorithmic_demag_bytes(p)
    flops = algorithmic_demag_flops(p)
    achieved = flops / conv_s / 1e12
    floor_gbs = alg / conv_s / 1e9
    five_gbs = five_pass_demag_bytes(p) / conv_s / 1e9
    roofline = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(FP32_PEAK_TFLOPS, 1),
                "unit": "TFLOP/s", "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                "traffic": conv_traffic(args.workload),
                "kernel": "demag FFT convolution (x R2C, fused y/z*K*z^-1/y^-1 cluster kernel, x C2R)",
                "algorithmic_flops": flops, "avg_launch_us": round(conv_s * 1e6, 2),
                "peak_kind": "derived FP32 issue peak (152 SM x 128 lanes x FMA x 2.07 GHz)",
                "hbm": {"peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
                        "floor_bytes": alg, "floor_gbs": round(floor_gbs, 1),
                        "floor_frac": round(floor_gbs / peaks["hbm_gbs"], 4),
                        "five_pass_bytes": five_pass_demag_bytes(p), "five_pass_equiv_gbs": round(five_gbs, 1),
                        "five_pass_equiv_frac": round(five_gbs / peaks["hbm_gbs"], 4)}}

    # end to end through the C ABI with pinned host buffers: m up, one step,
    # m down
    Ke = min(K, 50)
    host_m = torch.empty((3,) + ctx.shape, dtype=torch.float32, pin_memory=True).numpy()
    ctx.get_m(out=host_m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        ctx.set_m(host_m)
        ctx.step(1)
        ctx.get_m(out=host_m)
    e2e_s = reduce_max(time.perf_counter() - t0)
    e2e = {"value": p.ncells * Ke * world / e2e_s, "unit": "cell-steps/s",
           "h2d_bytes_per_step": 3 * 4 * p.ncells, "d2h_bytes_per_step": 3 * 4 * p.ncells, "steps": Ke}
    evals_per_step = 6.0 * attempts / K
    ctx.close()

    side = None
    if args.side and args.workload != SIDE_WORKLOAD:
        ps, cs, ds, a0, a1, _ = bench_workload(SIDE_WORKLOAD, K, W)
        side = {"workload": SIDE_WORKLOAD, "value": ps.ncells * K * world / reduce_max(ds), "unit": "cell-steps/s",
                "ms_per_step": ds / K * 1e3}
        cs.close()

    out = {
        "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_max / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [p.nx, p.ny, p.nz], "cells": p.ncells,
                   "cell_m": [p.dx, p.dy, p.dz], "magnetic_cells": int(p.magnetic().sum()),
                   "max_err": p.max_err, "parallelism": f"replicas{world}",
                   "l2": "flushed before every timed step (256 MB write)",
                   "evals_per_step": evals_per_step, "rejected_attempts": int(s1["rejected"] - s0["rejected"])},
        "cell_evals_per_s": value * evals_per_step,
        "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
    }
    if side:
        out["film"] = side
    if args.batch:
        out["batch"] = run_batch(args, local_rank)
    if args.surrogate:
        out["surrogate"] = run_surrogate(args, local_rank)
    return out


def run_batch(args, local_rank, t_end=0.1e-9, seq_per_shape=2):
    """The batched form: 512 independent instances of four grid sizes, each
    with its own adaptive step, advanced to t_end by one graph launch; against
    the plain single-instance path run one instance after another on a
    stratified sample (seq_per_shape instances of each grid size),
    extrapolated by the number of instances of each size."""
    import torch
    from paper_1406_7635_gb300 import mm
    from paper_1406_7635_gb300.workloads import batch_instances, problem_from_instance
    specs, m0s = batch_instances(512)
    b = mm.Batch(specs, device=local_rank)
    tiles = [b.class_info(c) for c in range(b.num_classes())]
    for i, m in enumerate(m0s):
        b.set_m(i, m)
    b.run(1e-15)                      # warm-up: builds and instantiates the graph
    for i, m in enumerate(m0s):
        b.set_m(i, m)
    b.set_solver()                    # restart the step-size controller
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(t_end + 1e-15)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stats = [b.get_stats(i) for i in range(len(specs))]
    b.close()
    cell_steps = sum(s["accepted"] * sp["nx"] * sp["ny"] * sp["nz"] for s, sp in zip(stats, specs))
    shapes = {}
    for i, sp in enumerate(specs):
        shapes.setdefault((sp["nx"], sp["ny"], sp["nz"]), []).append(i)
    seq_time = 0.0
    for key, idx in shapes.items():
        per = []
        for i in idx[:seq_per_shape]:
            p = problem_from_instance(specs[i], m0s[i])
            ctx = mm.Context.from_problem(p, device=local_rank)
            ctx.run(1e-15)
            ctx.set_m(p.m0)
            ctx.set_time(0.0, p.dt0)
            torch.cuda.synchronize()
            ts = time.perf_counter()
            ctx.run(t_end + 1e-15)
            torch.cuda.synchronize()
            per.append(time.perf_counter() - ts)
            ctx.close()
        seq_time += np.mean(per) * len(idx)
    return {"workload": "batch512 (32x32x1, 64x32x1, 128x64x2, 96x96x4; 4 nm cells)", "instances": len(specs),
            "t_end_s": t_end, "wall_s": wall, "instances_per_s": len(specs) / wall,
            "cell_steps_per_s": cell_steps / wall, "accepted_steps_mean": float(np.mean([s["accepted"] for s in stats])),
            "sequential_instances_per_s": len(specs) / seq_time,
            "speedup_vs_sequential": seq_time / wall,
            "sequential_sample": f"{seq_per_shape} instances per grid size, same t_end, extrapolated by count",
            "autotuned_tiles": tiles}


def run_surrogate(args, local_rank, steps=40):
    """The learned demag surrogate on the 512 x 512 x 1 film: trained on
    args.pairs (m, B_demag) pairs from the context's own exact trajectories,
    then `steps` RK45 steps timed with the exact convolution, with the guarded
    surrogate (exact check every 10 steps, fallback above 1e-3) and with the
    surrogate unguarded."""
    import torch
    from paper_1406_7635_gb300 import mm
    p = WORKLOADS["film_512x512x1"]()
    net = mm.FNO(p.ny, p.nx, width=32, layers=4, modes_x=24, modes_y=24, max_batch=4, seed=1, device=local_rank)
    ctx = mm.Context.from_problem(p, device=local_rank)
    t0 = time.perf_counter()
    loss = ctx.train_surrogate(net, p.msat[0], n_pairs=args.pairs, traj_len=16, steps_between=5,
                               field_max=50e-3, epochs=args.epochs, batch=4, lr=1e-3, seed=2)
    train_s = time.perf_counter() - t0
    ctx.close()
    # one surrogate evaluation (S = 1), wall time per synchronised call
    u = torch.randn(3 * p.ny * p.nx, device=f"cuda:{local_rank}") * 0.5
    yfno = torch.empty_like(u)
    for _ in range(3):
        net.forward(u, yfno, 1)
    ts = time.perf_counter()
    for _ in range(20):
        net.forward(u, yfno, 1)
    fwd_ms = (time.perf_counter() - ts) / 20 * 1e3

    def timed(setup):
        c = mm.Context.from_problem(p, device=local_rank)
        setup(c)
        c.step(2)                                  # warm-up
        c.set_m(p.m0)
        c.set_time(0.0, p.dt0)
        if setup is not plain:
            setup(c)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        c.step(steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - ts
        out = (c.get_m().astype(np.float64), p.ncells * steps / dt, c.surrogate_stats())
        c.close()
        return out

    def plain(c):
        pass
    m_exact, v_exact, _ = timed(plain)
    m_guard, v_guard, st_guard = timed(lambda c: c.set_demag_surrogate(net, p.msat[0], 10, 1e-3))
    m_free, v_free, st_free = timed(lambda c: c.set_demag_surrogate(net, p.msat[0], 10, 1e30))
    net.close()
    return {"workload": "film_512x512x1 (2 nm cells), FNO width 32, 4 layers, 24 modes per axis",
            "pairs": args.pairs, "epochs": args.epochs, "train_s": train_s, "final_train_loss": loss,
            "steps": steps, "forward_ms": fwd_ms, "exact_cell_steps_per_s": v_exact,
            "guarded_cell_steps_per_s": v_guard, "guarded_speedup": v_guard / v_exact,
            "guard": {k: st_guard[k] for k in ("checks", "fallbacks", "last_rel_err", "steps")},
            "unguarded_cell_steps_per_s": v_free, "unguarded_speedup": v_free / v_exact,
            "unguarded_field_rel_err_at_checks": st_free["last_rel_err"],
            "unguarded_final_m_max_err_vs_exact": float(np.abs(m_free - m_exact).max()),
            "guarded_final_m_max_err_vs_exact": float(np.abs(m_guard - m_exact).max())}


def oracle_cpu_run(name, budget_s, max_steps, warmup=0, warmup_budget_s=30.0):
    """The float64 oracle on the same workload: kernel set-up untimed, up to
    `warmup` untimed adaptive RK45 steps (within warmup_budget_s), then
    accepted steps until the time budget is spent.  Returns (problem, timed
    steps, seconds, warm-up steps done)."""
    from oracle.rk45 import RK45
    p = WORKLOADS[name]()
    s = RK45(p)
    s.k1 = s.field.torque(s.m, 0.0)   # first stage (untimed, like the GPU's warm-up)
    w0, done_w = time.perf_counter(), 0
    while done_w < warmup and time.perf_counter() - w0 < warmup_budget_s:
        s.adaptive_step()
        done_w += 1
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        s.adaptive_step()
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return p, steps, dt, done_w


def run_reference(args, rank, world):
    if rank != 0:
        return None
    budget = float(os.environ.get("MM_REF_BUDGET_S", 60))
    p, steps, dt, warm = oracle_cpu_run(args.workload, budget, max(args.steps, 1), warmup=args.warmup)
    v = p.ncells * steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "cell-steps/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [p.nx, p.ny, p.nz], "cells": p.ncells},
        "cpu_baseline": {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{steps} accepted RK45 steps of the full {args.workload} grid "
                                   f"(float64 numpy oracle, kernel set-up untimed, ~{budget:.0f} s budget)"},
        "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", dest="side", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-surrogate", dest="surrogate", action="store_false")
    ap.add_argument("--pairs", type=int, default=256, help="surrogate training pairs (the full recipe: 20000)")
    ap.add_argument("--epochs", type=int, default=2, help="surrogate training epochs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local_rank = env_rank()
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    out = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        budget = float(os.environ.get("MM_CPU_BUDGET_S", 20))
        p, steps, dt, _ = oracle_cpu_run(args.workload, budget, 1000)
        out["cpu_baseline"] = {"value": p.ncells * steps / dt, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"{steps} accepted RK45 steps of the full {args.workload} grid "
                                         f"(float64 numpy oracle, kernel set-up untimed)"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
