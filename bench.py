#!/usr/bin/env python
"""RK45 cell-steps/s of the micromagnetic hot path on GB300.

One step = one accepted Dormand-Prince RK45 step of the whole path (demag FFT
convolution, exchange stencil, anisotropy, Zeeman, LL torque, stage updates,
error reduction and step control) over the whole grid.

Default workload: the 3-D ellipsoid, 128 x 128 x 32 cells of 3 nm (demag
convolution padded to 256 x 256 x 64), the configuration on which both the
cell-steps/s and the HBM-roofline fraction of the demag convolution are
quoted; the 256 x 256 x 1 grain film is reported beside it ("film"), and the
contexts that step with the general kernels (spin-transfer torques, a
periodic x axis) beside that ("general_path").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the path does not shard (one simulation per GPU); N ranks run N
independent replicas ("replicas only", weak scaling), no collective on the
data path.

The reference arm (--impl reference) is the float64 oracle: one replica per
host core, each stepping the same workload, on rank 0 only.
"""
import argparse
import json
import os
import platform
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


def host_description():
    """Core count and CPU model of this host."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return {"nproc": cores, "cpu_model": model, "machine": platform.machine()}


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


# ---------------------------------------------------------------------------
# Algorithmic bytes and flops of the demag convolution (per evaluation)
# ---------------------------------------------------------------------------
def _pad(n):
    return 1 if n == 1 else 1 << (2 * n - 2).bit_length()


def _spectrum_rows_bytes(p):
    """Complex float32 bytes of the x-transformed spectrum rows that carry
    data: 3 components x (px/2 + 1) x ny x nz (12.68 MB at 128 x 128 x 32)."""
    px = _pad(p.nx)
    hx = px // 2 + 1 if px > 1 else 1
    return 3 * 8 * hx * p.ny * p.nz


def _octant_bytes(p):
    """The float32 kernel spectrum octant: 6 components (13.18 MB at 128 x
    128 x 32)."""
    def half(n):
        return 1 if n == 1 else _pad(n) // 2 + 1
    return 6 * 4 * half(p.nx) * half(p.ny) * half(p.nz)


def algorithmic_demag_bytes(p):
    """Minimum HBM bytes of one demag convolution (51 B per cell at 128 x 128
    x 32): read m (3 x 4 B) and the mask/region bytes (2 B) per cell, the
    kernel spectrum octant, write B (3 x 4 B) per cell."""
    return p.ncells * (12 + 2 + 12) + _octant_bytes(p)


def five_pass_passes(p):
    """HBM bytes of each pass of the unfused five-pass design (x R2C, y,
    z*K*z^-1, y^-1, x C2R, each pass through memory, pruned to the rows that
    carry data; 2-D: x, y*K*y^-1, x^-1): at 128 x 128 x 32 20.0 / 38.0 / 63.9 /
    38.0 / 19.0 MB, 341 B per cell in all."""
    py, pz = _pad(p.ny), _pad(p.nz)
    x_out = _spectrum_rows_bytes(p)
    y_out = x_out // p.ny * py
    kern = _octant_bytes(p)
    pass1 = p.ncells * (12 + 2) + x_out
    last = x_out + 12 * p.ncells
    if pz == 1:
        return [pass1, 2 * x_out + kern, last]
    return [pass1, x_out + y_out, 2 * y_out + kern, y_out + x_out, last]


def five_pass_demag_bytes(p):
    return sum(five_pass_passes(p))


def yz_kernel_bytes(p):
    """The (y, z) kernel's share of the five-pass bytes: the passes it fuses
    (y, z*K*z^-1, y^-1; in 2-D y*K*y^-1): 139.98 MB (267 B per cell) at 128 x
    128 x 32; and its own floor: read the spectrum rows and the octant, write
    the spectrum rows (38.5 MB)."""
    passes = five_pass_passes(p)
    fused = sum(passes[1:-1])
    floor = 2 * _spectrum_rows_bytes(p) + _octant_bytes(p)
    return fused, floor


# arrays the earlier-stage sums of the six row kernels read (m + the k's with
# a nonzero Dormand-Prince coefficient; the last: the error's 5 k's)
EARLIER_ARRAYS = [2, 3, 4, 5, 5, 5]


def row_kernel_bytes(p, partial=False):
    """Algorithmic HBM bytes of one row-stage kernel launch, the mean over the
    six launches of an attempt: read the demag spectrum rows and the stage
    input (its stencil neighbours are the same array) and the cell codes,
    read the earlier-stage sums' inputs (m and the earlier k's: 2, 3, 4, 5, 5
    arrays for stages 2..6, 5 k's for the error of the last; with `partial`
    the one array k_rs_partial made of them), write k_s, and the next stage
    input and its spectrum rows (stages 2..6) or the candidate m (the last):
    69 MB at 128 x 128 x 32, 51 MB with `partial`."""
    arr = 12 * p.ncells                      # one float32 3-vector field
    spec = _spectrum_rows_bytes(p)
    earlier = [1] * 6 if partial else EARLIER_ARRAYS
    per = [spec + arr + 4 * p.ncells + e * arr + arr + (arr + spec if i < 5 else arr) for i, e in enumerate(earlier)]
    return sum(per) / len(per)


def partial_kernel_bytes(p):
    """Algorithmic HBM bytes of one k_rs_partial launch, the mean over the six
    of an attempt: read m and the earlier k's, write one array."""
    arr = 12 * p.ncells
    return sum((e + 1) * arr for e in EARLIER_ARRAYS) / len(EARLIER_ARRAYS)


def algorithmic_demag_flops(p):
    """Floating-point operations of one demag convolution, counted as 5 L
    log2 L per complex transform of length L and 2.5 L log2 L per real one,
    over the lines that carry data (x: ny*nz rows per component, y: hx*nz
    columns, z: hx*py columns), forward and inverse, plus the spectral
    product (30 flops per frequency point in 3-D, 14 in 2-D where Kxz = Kyz
    = 0).  823 MFLOP at 128 x 128 x 32, of which the (y, z) kernel's share
    (y, z and the product) is 695 MFLOP."""
    return sum(demag_flops_parts(p))


def demag_flops_parts(p):
    """(x transforms, y and z transforms plus the product) flops."""
    from math import log2
    px, py, pz = _pad(p.nx), _pad(p.ny), _pad(p.nz)
    hx = px // 2 + 1 if px > 1 else 1
    fx = 2 * 3 * p.ny * p.nz * 2.5 * px * log2(px) if px > 1 else 0.0
    f = 0.0
    if py > 1:
        f += 2 * 3 * hx * p.nz * 5 * py * log2(py)
    if pz > 1:
        f += 2 * 3 * hx * py * 5 * pz * log2(pz)
    f += (30 if pz > 1 else 14) * hx * py * pz
    return fx, f


YZ_SOURCES = ("paper_1406_7635_gb300/csrc/fft_fused.cu", "paper_1406_7635_gb300/csrc/fft_yz3.cu",
              "paper_1406_7635_gb300/csrc/fft.cuh")


def sources_sha(files):
    """Hash of the code of `files`: line comments and blank lines are left
    out, so that a change of wording does not orphan counters taken on the
    same kernels."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def yz_traffic(workload):
    """DRAM bytes of one in-step (y, z) kernel launch from the committed ncu
    summary of the same workload, or None when the kernel's sources changed
    since the counters were taken."""
    prof = os.path.join(ROOT, "profiles", f"yz_kernel_{workload}.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        d = json.load(f)
    if d.get("src_sha256_16") != sources_sha(YZ_SOURCES):
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU oracle (float64 numpy): the cpu_baseline legs and the reference arm
# ---------------------------------------------------------------------------
def _oracle_worker(name, steps, warmup, budget_s, barrier, queue):
    """One oracle replica (a spawned process, one thread): kernel set-up and
    the first stage untimed, `warmup` untimed steps, then wait for the other
    replicas and time up to `steps` accepted RK45 steps (at least one) within
    budget_s."""
    try:
        from oracle.rk45 import RK45
        p = WORKLOADS[name]()
        s = RK45(p)
        s.k1 = s.field.torque(s.m, 0.0)
        for _ in range(warmup):
            s.adaptive_step()
        if barrier is not None:
            barrier.wait(timeout=3600)
        t0 = time.perf_counter()
        done = 0
        while done < steps:
            s.adaptive_step()
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        queue.put((done, time.perf_counter() - t0, p.ncells))
    except Exception as e:   # reported, never hangs the parent
        queue.put(("error", repr(e), 0))


class single_threaded_children:
    """While active, processes spawned from here run their numeric libraries
    on one thread each (the variables are inherited at spawn time)."""
    KEYS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __enter__(self):
        self.keep = {k: os.environ.get(k) for k in self.KEYS}
        for k in self.KEYS:
            os.environ[k] = "1"
        return self

    def __exit__(self, *exc):
        for k, v in self.keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_replicas(name, replicas, steps, warmup=0, budget_s=60.0):
    """`replicas` independent oracle processes (spawned, one thread each) on
    the same workload, timed together after a barrier.  Returns
    (aggregate cell-steps/s, per-replica steps, slowest replica's seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with single_threaded_children():
        q = ctx.Queue()
        bar = ctx.Barrier(replicas) if replicas > 1 else None
        procs = [ctx.Process(target=_oracle_worker, args=(name, steps, warmup, budget_s, bar, q), daemon=True)
                 for _ in range(replicas)]
        for pr in procs:
            pr.start()
        res = [q.get(timeout=3600) for _ in procs]
        for pr in procs:
            pr.join(timeout=60)
    bad = [r for r in res if r[0] == "error"]
    if bad:
        raise RuntimeError(f"oracle replica failed: {bad[0][1]}")
    seconds = max(r[1] for r in res)
    cell_steps = sum(r[0] * r[2] for r in res)
    return cell_steps / seconds, [r[0] for r in res], seconds


def cpu_baseline(name, steps, cores_all):
    """The oracle on this host: one replica (one core) and one replica per
    core (all cores, aggregate)."""
    v1, st1, s1 = oracle_replicas(name, 1, steps)
    vn, stn, sn = oracle_replicas(name, cores_all, steps)
    host = host_description()
    return {"value": vn, "unit": "cell-steps/s", "cores": cores_all, "kind": "oracle",
            "sample": f"{cores_all} independent float64 numpy oracle replicas (one thread each), "
                      f"{min(stn)}-{max(stn)} accepted RK45 steps each of the full {name} grid after untimed "
                      f"kernel set-up, timed together ({sn:.1f} s)",
            "one_core": {"value": v1, "cores": 1, "steps": st1[0], "seconds": s1},
            "host": host}


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------
def stt_variant(p):
    """The same problem with both spin-transfer torques switched on (a
    current of 1e11 A/m^2 along x and 5e10 A/m^2 through the film plane,
    P = 0.4, xi = 0.05, Lambda = 1, fixed layer along +z): the contexts that
    step with the general stage kernels."""
    for r in np.unique(p.region):
        p.jcur[r] = (1e11, 0.0, 5e10)
        p.xi[r] = 0.05
        p.pol[r] = 0.4
        p.lam[r] = 1.0
        p.tfree[r] = p.nz * p.dz
    p.zhang_li = True
    p.slonczewski = True
    return p


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

    def timed_steps(p, steps, warmup, clocks=False):
        ctx = mm.Context.from_problem(p, device=local_rank, stream=stream.cuda_stream)
        ctx.step(warmup)
        s0 = ctx.get_stats()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local_rank) if clocks else None
        if sampler:
            sampler.start()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()                  # evict the previous step's data from L2
                starts[k].record(stream)
                ctx.step(1)
                ends[k].record(stream)
        torch.cuda.synchronize()
        clk = sampler.stop() if sampler else None
        if world > 1:
            torch.distributed.barrier()
        dev_s = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3
        s1 = ctx.get_stats()
        return ctx, dev_s, s0, s1, clk

    def reduce_max(x):
        return max_over_ranks(x, world, dev)

    K, W = args.steps, args.warmup
    p = WORKLOADS[args.workload]()
    ctx, dev_s, s0, s1, clk = timed_steps(p, K, W, clocks=True)
    t_max = reduce_max(dev_s)
    value = whole_job_rate(p.ncells * K, world, t_max)
    attempts = (s1["accepted"] + s1["rejected"]) - (s0["accepted"] + s0["rejected"])
    launches = s1["launches"] - s0["launches"]

    # kernels of the step, one at a time with events between launches
    # (after the timed region, continuing the same trajectory; L2 not flushed)
    try:
        prof = ctx.profile_attempts(args.profile_attempts)
    except mm.MMError:   # a context outside the fused row-stage path
        prof = []
    kinds = {}
    for kind, us in prof:
        kinds.setdefault(kind, []).append(us)
    per_kind = {k: {"launches_per_attempt": len(v), "mean_us": float(np.mean(v)), "sum_us": float(np.sum(v))}
                for k, v in kinds.items()}
    peaks, peak_kind = measured_peaks()
    fp32_tflops, sms, sm_clock = mm.fp32_peak(local_rank)
    fused_bytes, floor_bytes = yz_kernel_bytes(p)
    _, yz_flops = demag_flops_parts(p)
    # the (y, z) part of one evaluation: the cluster kernel, or the three
    # kernels (y forward, column kernel, y inverse) together
    if "yz" in per_kind:
        t_yz, yz_name, yz_launches = per_kind["yz"]["mean_us"] * 1e-6, \
            "(y, z) cluster kernel k_yz2 (y, z*K*z^-1, y^-1 fused)", per_kind["yz"]["launches_per_attempt"]
    elif all(k in per_kind for k in ("yf", "zk", "yi")):
        t_yz = sum(per_kind[k]["mean_us"] for k in ("yf", "zk", "yi")) * 1e-6
        yz_name = "(y, z) kernels k_yf + k_zk + k_yi (y; z*K*z^-1 per column; y^-1), one evaluation"
        yz_launches = per_kind["zk"]["launches_per_attempt"]
    else:
        t_yz = None
    roofline = None
    if t_yz:
        ach = fused_bytes / t_yz / 1e9
        roofline = {
            "bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": yz_traffic(args.workload),
            "kernel": yz_name + " inside the RK45 step",
            "peak_kind": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes": fused_bytes,
            "algorithmic_basis": "five-pass bytes of the passes the kernel fuses (y, z*K*z^-1, y^-1), "
                                 f"{fused_bytes / p.ncells:.0f} B per cell x {p.ncells} cells",
            "avg_launch_us": round(t_yz * 1e6, 2),
            "timing": f"CUDA events between launches on the context's stream, {args.profile_attempts} attempts "
                      f"x {yz_launches} evaluations, L2 not flushed",
            "floor_bytes": floor_bytes, "floor_gbs": round(floor_bytes / t_yz / 1e9, 1),
            "floor_frac": round(floor_bytes / t_yz / 1e9 / peaks["hbm_gbs"], 4),
            "alu": {"flops": yz_flops, "achieved_tflops": round(yz_flops / t_yz / 1e12, 2),
                    "peak_tflops": round(fp32_tflops, 1),
                    "peak_kind": f"measured FP32 FMA throughput (mm_fp32_peak, {sms} SMs, max {sm_clock} MHz)",
                    "frac": round(yz_flops / t_yz / 1e12 / fp32_tflops, 4)},
        }
    roofline_row = None
    if "row" in per_kind:
        t_row = per_kind["row"]["mean_us"] * 1e-6
        branch = "part" in per_kind
        rb = row_kernel_bytes(p, partial=branch)
        roofline_row = {"bound": "hbm", "achieved": round(rb / t_row / 1e9, 1), "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": round(rb / t_row / 1e9 / peaks["hbm_gbs"], 4),
                        "kernel": "row-stage kernel k_rs_row (x C2R, field, torque, stage update, x R2C)"
                                  + (", earlier-stage sums read from k_rs_partial" if branch else ""),
                        "algorithmic_bytes": rb, "avg_launch_us": round(t_row * 1e6, 2)}
        if branch:
            t_part = per_kind["part"]["mean_us"] * 1e-6
            pb = partial_kernel_bytes(p)
            roofline_row["partial"] = {
                "kernel": "k_rs_partial (earlier-stage sums; a graph branch beside the (y, z) part)",
                "algorithmic_bytes": pb, "avg_launch_us": round(t_part * 1e6, 2),
                "achieved": round(pb / t_part / 1e9, 1),
                "frac": round(pb / t_part / 1e9 / peaks["hbm_gbs"], 4)}
    step_kernels = {"per_kind": per_kind,
                    "sum_us_per_attempt": round(sum(us for _, us in prof), 1),
                    "graph_us_per_attempt": round(t_max / max(attempts, 1) * 1e6, 1),
                    "note": "events between launches remove the programmatic-dependent-launch overlap of the graph"}

    # the whole convolution alone (x R2C, (y, z), x C2R kernels), L2 flushed
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
    five = five_pass_demag_bytes(p)
    convolution = {"kernels": "x R2C (k_fx_t) + the context's (y, z) part + x C2R (k_ix_t) "
                              "(mm_demag_apply), L2 flushed before each call",
                   "avg_us": round(conv_s * 1e6, 2), "five_pass_bytes": five,
                   "five_pass_equiv_gbs": round(five / conv_s / 1e9, 1),
                   "five_pass_equiv_frac": round(five / conv_s / 1e9 / peaks["hbm_gbs"], 4),
                   "floor_bytes": algorithmic_demag_bytes(p),
                   "floor_frac": round(algorithmic_demag_bytes(p) / conv_s / 1e9 / peaks["hbm_gbs"], 4),
                   "flops": algorithmic_demag_flops(p),
                   "alu_frac": round(algorithmic_demag_flops(p) / conv_s / 1e12 / fp32_tflops, 4)}

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
        "roofline": roofline, "roofline_row": roofline_row, "step_kernels": step_kernels,
        "convolution": convolution,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
    }

    # (side lines and the surrogate describe one GPU: measured at N = 1 only;
    # the batch is sharded over the ranks)
    if world > 1:
        args.side = args.surrogate = False
    if args.side and args.workload != SIDE_WORKLOAD:
        ps = WORKLOADS[SIDE_WORKLOAD]()
        cs, ds, _, _, _ = timed_steps(ps, K, W)
        out["film"] = {"workload": SIDE_WORKLOAD, "value": ps.ncells * K * world / reduce_max(ds),
                       "unit": "cell-steps/s", "ms_per_step": ds / K * 1e3}
        cs.close()
    if args.side:
        general = {}
        pg = stt_variant(WORKLOADS[DEFAULT_WORKLOAD]())
        cg, dg, _, _, _ = timed_steps(pg, K, W)
        general["ellipsoid_128x128x32_stt"] = {
            "value": pg.ncells * K * world / reduce_max(dg), "unit": "cell-steps/s", "ms_per_step": dg / K * 1e3,
            "what": "Zhang-Li + Slonczewski torques on: general stage kernels + three-kernel convolution"}
        cg.close()
        pf = WORKLOADS[SIDE_WORKLOAD]()
        pf.pbc = (4, 0, 0)
        cf, df, _, _, _ = timed_steps(pf, K, W)
        general["grains_256x256x1_pbc_x"] = {
            "value": pf.ncells * K * world / reduce_max(df), "unit": "cell-steps/s", "ms_per_step": df / K * 1e3,
            "what": "periodic x (4 images each side): general stage kernels + cyclic x transform"}
        cf.close()
        out["general_path"] = general
    if args.batch:
        out["batch"] = run_batch(args, local_rank, rank, world)
    if args.surrogate:
        out["surrogate"] = run_surrogate(args, local_rank)
    return out


def _replay_instance(spec, m0, dts, m_gpu):
    """Oracle replay of one batched instance's accepted steps (spawned
    process): (max |m_gpu - m_oracle|, the problem's own sensitivity: max
    |m_oracle' - m_oracle| for an oracle run from m0 perturbed by 1e-7
    (seeded Gaussian) with the same steps)."""
    from oracle.rk45 import RK45
    from paper_1406_7635_gb300.workloads import problem_from_instance
    p = problem_from_instance(spec, m0)
    m32 = p.m0.astype(np.float32).astype(np.float64)
    ora = RK45(p, m=m32)
    ora.run_fixed(dts)
    pert = RK45(p, m=m32 + 1e-7 * np.random.default_rng(1406).standard_normal(m32.shape))
    pert.run_fixed(dts)
    return float(np.abs(m_gpu.astype(np.float64) - ora.m).max()), float(np.abs(pert.m - ora.m).max())


def run_batch(args, local_rank, rank=0, world=1, t_end=0.1e-9, seq_per_shape=2, acc_per_shape=8,
              t_acc=(2e-12, 5e-12)):
    """The batched form: 512 independent instances of four grid sizes, each
    with its own adaptive step, advanced to t_end by one graph launch; against
    the plain single-instance path run one instance after another on a
    stratified sample (seq_per_shape instances of each grid size),
    extrapolated by the number of instances of each size.  Accuracy: a batch
    of acc_per_shape instances of each size run to each horizon of t_acc,
    replayed by the float64 oracle with their own step sizes.  With several ranks the 512
    instances are sharded round-robin (one batch per GPU, no collective while
    they run) and the per-instance stats all-gathered at the end; the
    sequential sample and the accuracy leg run on rank 0."""
    import multiprocessing as mp
    import torch
    from paper_1406_7635_gb300 import mm
    from paper_1406_7635_gb300.shard import gather_instance_stats, instance_shard
    from paper_1406_7635_gb300.workloads import batch_instances, problem_from_instance
    specs, m0s = batch_instances(512)
    ids = instance_shard(len(specs), rank, world)
    b = mm.Batch([specs[i] for i in ids], device=local_rank)
    tiles = [b.class_info(c) for c in range(b.num_classes())]
    for j, i in enumerate(ids):
        b.set_m(j, m0s[i])
    b.run(1e-15)                      # warm-up: builds and instantiates the graph
    for j, i in enumerate(ids):
        b.set_m(j, m0s[i])
    b.set_solver()                    # restart the step-size controller
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(t_end + 1e-15)
    torch.cuda.synchronize()
    wall = max_over_ranks(time.perf_counter() - t0, world, torch.device("cuda", local_rank))
    local_stats = [b.get_stats(j) for j in range(len(ids))]
    stats = gather_instance_stats(ids, local_stats, len(specs), world, device=f"cuda:{local_rank}")
    cell_steps = sum(s["accepted"] * sp["nx"] * sp["ny"] * sp["nz"] for s, sp in zip(stats, specs))
    shapes = {}
    for i, sp in enumerate(specs):
        shapes.setdefault((sp["nx"], sp["ny"], sp["nz"]), []).append(i)
    b.close()
    base = {"workload": "batch512 (32x32x1, 64x32x1, 128x64x2, 96x96x4; 4 nm cells)", "instances": len(specs),
            "t_end_s": t_end, "wall_s": wall, "instances_per_s": len(specs) / wall,
            "cell_steps_per_s": cell_steps / wall,
            "accepted_steps_mean": float(np.mean([s["accepted"] for s in stats])),
            "sharding": f"{world} rank(s), round-robin by instance, stats all-gathered at the end",
            "autotuned_tiles": tiles}
    if rank != 0:
        return base
    # accuracy: a batch of the stratified subsample from its initial state to
    # each horizon (its own autotuned tiles), each instance replayed by the
    # oracle with its accepted step sizes
    sample = [i for idx in shapes.values() for i in idx[:acc_per_shape]]
    ba = mm.Batch([specs[i] for i in sample], device=local_rank)
    for j, i in enumerate(sample):
        ba.set_m(j, m0s[i])
    jobs, horizons = [], []
    for t_h in t_acc:
        ba.run(t_h)
        horizons.append((t_h, [ba.get_stats(j)["accepted"] for j in range(len(sample))]))
        jobs += [(specs[i], m0s[i], ba.get_dt_history(j), ba.get_m(j)) for j, i in enumerate(sample)]
    ba.close()
    with single_threaded_children(), mp.get_context("spawn").Pool(min(len(jobs), host_description()["nproc"])) as pool:
        all_errs = pool.starmap(_replay_instance, jobs)
    acc = {"instances": len(sample), "bar": 1e-5,
           "method": f"a batch of the subsample ({acc_per_shape} instances per grid size, the first of each size) "
                     "run from its initial state to each horizon; the float64 oracle replays each instance's "
                     "accepted step sizes; max |m_gpu - m_oracle| per instance, beside the oracle's own change "
                     "when its initial m is perturbed by 1e-7 (the growth the dynamics give a rounding-sized "
                     "perturbation over the same steps)"}
    for h, (t_h, steps) in enumerate(horizons):
        part = all_errs[h * len(sample):(h + 1) * len(sample)]
        errs = [e for e, _ in part]
        sens = [q for _, q in part]
        acc[f"t_{t_h * 1e12:g}ps"] = {
            "accepted_steps_mean": float(np.mean(steps)), "max_abs_m_err": max(errs),
            "median_abs_m_err": float(np.median(errs)),
            "per_shape_max": {f"{k[0]}x{k[1]}x{k[2]}": max(e for i, e in zip(sample, errs) if i in idx[:acc_per_shape])
                              for k, idx in shapes.items()},
            "oracle_sensitivity_1e-7": {"max": max(sens), "median": float(np.median(sens))},
            "instances_within_bar_or_sensitivity": int(sum(e <= max(1e-5, 2 * q) for e, q in zip(errs, sens)))}
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
    base.update({"sequential_instances_per_s": len(specs) / seq_time,
                 "speedup_vs_sequential": seq_time / wall,
                 "sequential_sample": f"{seq_per_shape} instances per grid size on one GPU, same t_end, "
                                      f"extrapolated by count",
                 "accuracy_vs_oracle": acc})
    return base


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


def run_reference(args, rank, world):
    """The float64 oracle on the host cores: one replica per core (or
    MM_REF_CORES), each stepping the full workload, rank 0 only."""
    if rank != 0:
        return None
    budget = float(os.environ.get("MM_REF_BUDGET_S", 60))
    host = host_description()
    cores = int(os.environ.get("MM_REF_CORES", host["nproc"]))
    warm = min(args.warmup, int(os.environ.get("MM_REF_WARMUP", 2)))
    v, steps, secs = oracle_replicas(args.workload, cores, max(args.steps, 1), warmup=warm, budget_s=budget)
    p = WORKLOADS[args.workload]()
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "cell-steps/s", "n_gpus": world,
        "steps": min(steps), "warmup": args.warmup, "ms_per_step": secs / max(min(steps), 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [p.nx, p.ny, p.nz], "cells": p.ncells},
        "cpu_baseline": {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} float64 numpy oracle replicas (one thread each), {min(steps)}-"
                                   f"{max(steps)} accepted RK45 steps each of the full {args.workload} grid after "
                                   f"{warm} untimed warm-up steps and untimed kernel set-up (~{budget:.0f} s budget)",
                         "host": host},
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
    ap.add_argument("--cpu-steps", type=int, default=10, help="accepted oracle steps per replica (cpu_baseline)")
    ap.add_argument("--profile-attempts", type=int, default=10, help="attempts launched kernel by kernel")
    ap.add_argument("--no-side", dest="side", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-surrogate", dest="surrogate", action="store_false")
    ap.add_argument("--pairs", type=int, default=20000, help="surrogate training pairs (the recipe: 20000)")
    ap.add_argument("--epochs", type=int, default=1, help="surrogate training epochs")
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
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_steps, host_description()["nproc"])
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
