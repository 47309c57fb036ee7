#!/usr/bin/env python3
"""Throughput of the shift-free 2D FMM on one GB300 (particles / s at rel L2 error <= 1e-6).

One step = one full evaluation of the method (bin/sort, P2M for every level,
M2L, L2P for every level, P2P + final phi in input order) through the C ABI
call fmm_potential followed by fmm_sync, on inputs already resident in HBM.
The default workload is 1,048,576 particles uniform in [0,5]^2, q ~ U[-1,1],
a uniform quadtree of 8 levels and expansion order p = 20, computed in the
mixed-precision form with the BF16x2 tensor-core M2L (the fastest form that
meets the 1e-6 error bound); the plain FP64 GPU path is timed beside it.

Timing: W warm-up steps, then exactly K steps timed with CUDA events on the
plan's stream; between steps a 256 MB buffer is written to flush the 129 MB
L2 (outside the events).  The accuracy gate compares phi at 4096 sampled
targets with the FP64 direct sum (the library's FP64 direct-sum kernel, itself
tested against the CPU oracle).

--impl reference times the FP64 CPU oracle (the method's plain statement,
test infrastructure) on the host cores on a bounded sample of the workload.
Under torchrun each rank runs an independent replica (the single-system path
has no data-parallel split without a halo exchange); the value is the sum of
all ranks' particles over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/sec at rel L2 err <=1e-6 vs FP64 direct; mixed vs plain FP64, same GB300"
UNIT = "particles/s"
ERR_BOUND = 1e-6
N_SMS = 152
FP32_LANES_PER_SM = 128        # FP32 FMA lanes per SM (4 sub-partitions x 32)
MUFU_PER_SM = 16               # lg2 results per clock per SM: measured by the library's probe
                               # (fmm_probe_peak: 5.01e12 lg2/s on 152 SMs at 2.06 GHz)

WORKLOADS = {
    "uniform_1m_l8_p20": dict(n=1 << 20, levels=8, p=20, family="uniform", config=1),
    "uniform_4k_l4_p16": dict(n=4096, levels=4, p=16, family="uniform", config=0),
    "gmm32_16m_l10_p24": dict(n=1 << 24, levels=10, p=24, family="gmm", config=2),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform_1m_l8_p20", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16x2",
                    help="fp32 (CUDA-core M2L), 3xtf32 / tf32 or bf16x3 / bf16x2 / bf16 (tensor-core M2L from "
                         "level 6), fp64")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the plain FP64 GPU path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched form (1024 systems, N log-uniform in [1024, 262144], against a loop "
                         "of single-system launches)")
    ap.add_argument("--batched-systems", type=int, default=1024)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned (levels, p) selector's leg")
    ap.add_argument("--no-clustered", action="store_true",
                    help="skip the clustered leg (2^24 Gaussian-mixture particles, levels 10, p 24)")
    ap.add_argument("--clustered-steps", type=int, default=5)
    ap.add_argument("--lagrange-only", action="store_true",
                    help="run only the Lagrange-node leg (a profiling target); prints that leg's JSON")
    ap.add_argument("--lagrange-steps", type=int, default=20)
    ap.add_argument("--no-lagrange", action="store_true",
                    help="skip the leg of the paper's own Lagrange-node form (3D Coulomb workloads of its "
                         "Tables 1-3, the 2D comparison and the FP64-conditioning sweep)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the default process group (x itself without one): every
    rank's replica is timed alone and the job runs as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_per_rank, world_size, seconds):
    """Whole-job throughput: the particles of every rank's replica over the slowest rank's time."""
    return world_size * n_per_rank / seconds


def make_inputs(w, rank=0):
    from paper_2009_00767_gb300 import inputs
    gen = getattr(inputs, w["family"])
    return gen(w["n"], inputs.config_seed(w["config"], rank))


# ---------------------------------------------------------------- algorithmic work per launch

def m2l_pairs(levels, kmin=2):
    """(target, source) square pairs of the interaction lists of levels kmin..levels inside the box."""
    total = 0
    for k in range(kmin, levels + 1):
        side = 1 << k
        t = np.arange(side)
        cnt = np.zeros(side, dtype=np.int64)   # per-axis counts are not separable; count per offset
        tot_k = 0
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                if abs(dx) <= 1 and abs(dy) <= 1:
                    continue
                # target parity must admit the offset: d in [-2-p, 3-p] per axis
                okx = ((t & 1) == 0) & (dx >= -2) & (dx <= 3) | ((t & 1) == 1) & (dx >= -3) & (dx <= 2)
                oky = ((t & 1) == 0) & (dy >= -2) & (dy <= 3) | ((t & 1) == 1) & (dy >= -3) & (dy <= 2)
                inx = okx & (t + dx >= 0) & (t + dx < side)
                iny = oky & (t + dy >= 0) & (t + dy < side)
                tot_k += int(inx.sum()) * int(iny.sum())
        del cnt
        total += tot_k
    return total


TC_KMIN = 6   # the tensor-core M2L takes levels 6 and finer


TC_PRECISIONS = ("tf32", "3xtf32", "bf16", "bf16x2", "bf16x3")


def _tensor_peak(peaks, precision):
    bf = precision.startswith("bf16")
    peak = peaks.get("bf16_tflops", 1939.8) / (1.0 if bf else 2.0)
    basis = "measured bf16 dense (MEASURED_PEAKS.json)" + ("" if bf else " x the nominal TF32/BF16 ratio 1/2")
    return peak, basis


def roofline_for(stage, stats, ms, w, peaks, sm_clock_mhz, precision, traffic):
    """Roofline of one kernel (or stage) from its device time `ms`: algorithmic work per launch over
    the time, against the measured (or derived) peak of the unit that bounds it.  Particle stages
    (P2M, L2P) carry both their FP32-FMA fraction and their HBM fraction."""
    if ms <= 0:
        return None
    p1 = w["p"] + 1
    n, L = w["n"], w["levels"]
    fma_peak = N_SMS * FP32_LANES_PER_SM * 2 * sm_clock_mhz * 1e6 / 1e12
    fma_basis = f"FP32 FMA: {N_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_clock_mhz:.0f} MHz"
    hbm = peaks.get("hbm_gbs", 6800.0)
    sec = ms * 1e-3

    def out(kernel, bound, ach, peak, unit, work, **extra):
        d = {"kernel": kernel, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
             "traffic": traffic, "work_per_launch": work, "ms": ms}
        d.update(extra)
        return d

    def grid_bytes(k0, k1, per_cell):
        return sum(((1 << k) ** 2) * per_cell for k in range(max(2, k0), k1 + 1))

    if stage in ("m2l_tc", "m2l_fine") and precision in TC_PRECISIONS:
        flops = m2l_pairs(L, TC_KMIN) * 8 * p1 * p1
        peak, basis = _tensor_peak(peaks, precision)
        name = "k_m2l_tc" if stage == "m2l_tc" else "k_prep_tc + k_m2l_tc"
        return out(name, "tensor", flops / sec / 1e12, peak, "TFLOP/s",
                   f"{flops:.4g} flop = IL pairs of levels {TC_KMIN}..{L} x 8 (p+1)^2 (split products not counted)",
                   peak_basis=basis)
    if stage in ("m2l_coarse", "m2l_fine", "m2l"):
        k0, k1 = (2, min(L, 5)) if stage == "m2l_coarse" else ((6, L) if stage == "m2l_fine" else (2, L))
        flops = m2l_pairs(L, k0) * 8 * p1 * p1 - (m2l_pairs(L, k1 + 1) * 8 * p1 * p1 if k1 < L else 0)
        if precision == "fp64":
            return None
        return out({"m2l_coarse": "k_m2l_coarse", "m2l_fine": "k_m2l_f32", "m2l": "m2l"}[stage], "alu",
                   flops / sec / 1e12, fma_peak, "TFLOP/s", f"{flops:.4g} flop = IL pairs of levels {k0}..{k1} x 8 (p+1)^2",
                   peak_basis=fma_basis)
    if stage in ("p2p_kernel", "p2p"):
        pairs = stats["p2p_pairs"]
        peak = N_SMS * MUFU_PER_SM * sm_clock_mhz * 1e6 / 1e12   # Tlg2/s
        return out("k_p2p_mixed" if stage == "p2p_kernel" else "p2p", "alu", pairs / sec / 1e12, peak, "Tlg2/s",
                   f"{pairs} ordered pairs, one lg2 each (the survey's unit; the symmetric kernel evaluates the "
                   f"forward-neighbour pairs once for both sides, about 0.56 lg2 per ordered pair)",
                   peak_basis=f"MUFU lg2: {N_SMS} SMs x {MUFU_PER_SM}/clk x {sm_clock_mhz:.0f} MHz")
    if stage == "p2m_coarse" and precision != "fp64":
        # the upward pass: per parent of levels 2 .. l-3, coefficient m sums (m + 1) complex
        # multiply-adds (8 flop) for each of its four children
        parents = sum(4 ** k for k in range(2, L - 2))
        if parents == 0:
            return None
        flops = parents * 4 * 8 * sum(m + 1 for m in range(1, p1))
        nbytes = sum((4 ** (k + 1) + 4 ** k) * p1 * 8 for k in range(2, L - 2))
        ach_b = nbytes / sec / 1e9
        return out("k_m2m_f32", "alu", flops / sec / 1e12, fma_peak, "TFLOP/s",
                   f"{flops:.4g} flop = {parents} parents x 4 children x sum_m (m+1) complex MACs of 8 flop "
                   f"(levels 2..{L - 3})", peak_basis=fma_basis,
                   hbm={"achieved": ach_b, "peak": hbm, "unit": "GB/s", "frac": ach_b / hbm, "bytes": nbytes,
                        "what": "children's FP32 moment grids in, parents' out"})
    if stage in ("p2m_fine", "l2p", "p2m") and precision != "fp64":
        if stage == "p2m_fine":
            lev = range(max(2, L - 2), L + 1)
            nbytes = 16 * n + grid_bytes(L - 2, L, p1 * 8)
            what = "16 B particle in, FP32 moment grids out"
        elif stage == "l2p":
            lev = range(2, L + 1)
            nbytes = 36 * n + grid_bytes(2, L, p1 * 8)
            what = "16 B particle + 4 B key + 8 B near in, 8 B phi out, local grids in"
        else:
            lev = range(2, L + 1)
            nbytes = 20 * n
            what = "particles in"
        flops = 8 * w["p"] * n * len(lev)
        if flops == 0:
            return None
        ach_b = nbytes / sec / 1e9
        return out(stage, "alu", flops / sec / 1e12, fma_peak, "TFLOP/s",
                   f"{flops:.4g} flop = 8p per particle per level, {len(lev)} levels", peak_basis=fma_basis,
                   hbm={"achieved": ach_b, "peak": hbm, "unit": "GB/s", "frac": ach_b / hbm,
                        "bytes": nbytes, "what": what})
    # sort (and the FP64 path's P2M / L2P): HBM bytes per launch
    nbytes = {"sort": n * (24 + 4 + 4 + 4 + 4 + 16 + 4 + 24), "p2m": n * 20, "l2p": n * (20 + 8)}.get(stage)
    if nbytes is None:
        return None
    return out(stage, "hbm", nbytes / sec / 1e9, hbm, "GB/s", f"{nbytes} bytes")


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            import tempfile
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return res
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.seek(0)
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sms.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        self.out.close()
        res.update(sm_mhz=statistics.median(sms) if sms else None, sm_max_mhz=mx, reasons=sorted(reasons),
                   samples=len(sms))
        return res


# ---------------------------------------------------------------- our arm

def load_traffic(stage):
    """ncu DRAM bytes per launch for a kernel, if captured on the current source of its files."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(stage)
        if not rec:
            return None
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2009_00767_gb300", "csrc", f), "rb").read())
        return rec["bytes_per_launch"] if h.hexdigest()[:16] == rec["sha"] else None
    except Exception:
        return None


def time_plan(binding, torch, w, precision, xy_d, q_d, steps, warmup, flush, stream):
    plan = binding.Plan(w["n"], w["levels"], w["p"], 5.0, precision, stream)
    phi = torch.empty(w["n"], dtype=torch.float64, device=xy_d.device)
    for _ in range(warmup):
        binding.fmm_potential(plan.handle, xy_d, q_d, phi)
        plan.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage_ms = {k: [] for k in ("sort", "p2m", "m2l", "l2p", "p2p", "m2l_tc", "p2p_kernel", "p2m_fine", "p2m_coarse",
                                "m2l_fine", "m2l_coarse")}
    launches = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        flush.zero_()                        # evict L2 outside the timed events
        ev[i][0].record(stream)
        binding.fmm_potential(plan.handle, xy_d, q_d, phi)
        ev[i][1].record(stream)
        plan.sync()
        st = plan.stats()
        for k in stage_ms:
            stage_ms[k].append(st["ms_" + k])
        launches += st["kernel_launches"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = [a.elapsed_time(b) for a, b in ev]
    return plan, phi, ms, stage_ms, launches, wall, st


KERNELS_ALONE = ("sort", "p2m_fine", "p2m_coarse", "m2l_coarse", "m2l_fine", "m2l_tc", "p2p_kernel", "l2p")


def time_kernels_alone(binding, torch, plan, xy_d, q_d, phi, steps, warmup, flush, stream):
    """Each kernel's device time with the stages run one after the other on the plan's stream
    (fmm_set_concurrency(plan, 1)); the timed step overlaps them on three streams, where a kernel's
    own span also holds the time it waits for SMs the others hold.  Medians over `steps` calls, L2
    flushed before each."""
    binding.fmm_set_concurrency(plan.handle, 1)
    rec = {k: [] for k in KERNELS_ALONE + ("total",)}
    try:
        for i in range(warmup + steps):
            flush.zero_()
            binding.fmm_potential(plan.handle, xy_d, q_d, phi)
            plan.sync()
            if i < warmup:
                continue
            st = plan.stats()
            for k in KERNELS_ALONE:
                rec[k].append(st["ms_" + k])
            rec["total"].append(st["ms_total"])
    finally:
        binding.fmm_set_concurrency(plan.handle, 3)
    return {k: float(np.median(v)) for k, v in rec.items()}


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2009_00767_gb300 import binding, build
    build.build()
    w = WORKLOADS[args.workload]
    xy, q = make_inputs(w, rank)
    xy_d = torch.from_numpy(xy).to(dev)
    q_d = torch.from_numpy(q).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    plan, phi, ms, stage_ms, launches, wall, last = time_plan(binding, torch, w, args.precision, xy_d, q_d,
                                                              args.steps, args.warmup, flush, stream)
    barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(float(np.median(ms)), dev)   # the median step (mean reported beside it)
    value = job_rate(w["n"], ws, ms_step * 1e-3)

    # accuracy gate: FP64 direct sum at 4096 sampled targets (on the GPU)
    from paper_2009_00767_gb300 import inputs as inp
    S = min(4096, w["n"])
    idx = np.unique((inp.u01(4242, 0, S) * w["n"]).astype(np.int64))
    idx_d = torch.from_numpy(idx).to(dev)
    ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
    binding.fmm_direct_targets(xy_d, q_d, idx_d, ref)
    torch.cuda.synchronize()
    got = phi[idx_d]
    err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))

    # per-stage device times in the timed (overlapped) step, each kernel's time alone from a serial
    # pass, and the rooflines from the times alone (the dominant kernel: the longest alone)
    stage_avg = {k: float(np.mean(stage_ms[k])) for k in ("sort", "p2m", "m2l", "l2p", "p2p", "p2m_fine", "p2m_coarse",
                                                          "m2l_fine", "m2l_coarse")}
    kern_avg = {k: float(np.mean(stage_ms[k])) for k in ("m2l_tc", "p2p_kernel")}
    alone = None
    if args.precision != "fp64":
        alone = time_kernels_alone(binding, torch, plan, xy_d, q_d, phi, max(5, min(args.steps, 50)), 3, flush,
                                   stream)
        cands = {k: alone[k] for k in KERNELS_ALONE if alone[k] > 0}
    else:
        cands = {k: stage_avg[k] for k in ("sort", "p2m", "m2l", "l2p", "p2p")}
    # the dominant kernel: the longest single kernel timed alone (the sort, the upward pass, the fine
    # M2L stage and the L2P of the coarse and the fine levels are several kernels each)
    singles = [k for k in ("p2m_fine", "m2l_coarse", "m2l_tc", "p2p_kernel") if k in cands]
    dom = max(singles or [k for k in cands if k != "sort"], key=cands.get)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    in_step = dict(stage_avg, m2l_tc=kern_avg["m2l_tc"], p2p_kernel=kern_avg["p2p_kernel"], l2p=stage_avg["l2p"])
    roof_all = {}
    for k, v in cands.items():
        r = roofline_for(k, last, v, w, peaks, sm_max, args.precision, load_traffic(k))
        if r is not None:
            r["timing"] = "kernel alone (serial pass, CUDA events)" if alone else "stage in the timed step"
            if k in in_step:
                r["in_step_ms"] = in_step[k]
            roof_all[k] = r
    roof = roof_all.get(dom)
    # the arithmetic units measured by the library's own probes (a few ms, after the timed region),
    # beside the peaks derived from unit counts and the maximum clock
    probe = {"fp32_tflops": binding.fmm_probe_peak(binding.FMM_PROBE_FP32_FMA) / 1e12,
             "mufu_tlg2_per_s": binding.fmm_probe_peak(binding.FMM_PROBE_MUFU_LG2) / 1e12,
             "fp64_tflops": binding.fmm_probe_peak(binding.FMM_PROBE_FP64_FMA) / 1e12}
    for r in roof_all.values():
        if r and r.get("bound") == "alu":
            r["peak_probe"] = probe["mufu_tlg2_per_s"] if r["unit"] == "Tlg2/s" else probe["fp32_tflops"]

    # end to end through the host-buffer entry points: H2D of xy, q and D2H of phi every step, on
    # the host clock.  Pipelined: fmm_potential_host_async per step (its uploads overlap the previous
    # step's compute, its download the next one's), one fmm_sync at the end; and one call at a time
    # (fmm_potential_host, which waits) for comparison.
    xy_h = torch.from_numpy(xy).pin_memory()
    q_h = torch.from_numpy(q).pin_memory()
    phi_h = [torch.empty(w["n"], dtype=torch.float64).pin_memory() for _ in range(2)]
    # at least 100 calls (about 40 ms): the host clock's jitter and Python's call overhead average
    # out, where a few calls of 0.4 ms each gave rates that moved by 20% between runs
    e2e_steps = max(100, min(args.steps, 400))
    for _ in range(2):
        plan.potential_host(xy_h, q_h, phi_h[0])
    barrier()
    te = time.perf_counter()
    for i in range(e2e_steps):
        binding.fmm_potential_host_async(plan.handle, xy_h, q_h, phi_h[i & 1])
    plan.sync()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - te) / e2e_steps, dev)
    te = time.perf_counter()
    for _ in range(e2e_steps):
        plan.potential_host(xy_h, q_h, phi_h[0])
    barrier()
    e2e_sync_s = max_over_ranks((time.perf_counter() - te) / e2e_steps, dev)
    e2e = {"value": job_rate(w["n"], ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": w["n"] * 24,
           "d2h_bytes_per_step": w["n"] * 8, "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
           "call": "fmm_potential_host_async per step (pinned host buffers), fmm_sync after the last",
           "one_call_at_a_time": {"value": job_rate(w["n"], ws, e2e_sync_s), "ms_per_step": e2e_sync_s * 1e3,
                                  "call": "fmm_potential_host (waits every step)"}}

    # the plain FP64 GPU path on the same inputs
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        p64, phi64, ms64, st64, l64, _, _ = time_plan(binding, torch, w, "fp64", xy_d, q_d, args.fp64_steps, 2,
                                                      flush, stream)
        err64 = float(torch.linalg.norm(phi64[idx_d] - ref) / torch.linalg.norm(ref))
        m64 = max_over_ranks(float(np.median(ms64)), dev)
        fp64 = {"value": job_rate(w["n"], ws, m64 * 1e-3), "ms_per_step": m64, "rel_l2_err": err64,
                "stage_ms": {k: float(np.mean(v)) for k, v in st64.items()}}
        p64.close()
    plan.close()

    clustered = None
    if not args.no_clustered and rank == 0 and args.workload != "gmm32_16m_l10_p24":
        clustered = run_clustered(binding, torch, dev, args.precision, flush, args.clustered_steps, peaks)

    lagrange = None
    if not args.no_lagrange and rank == 0:
        lagrange = run_lagrange(binding, torch, dev, flush, peaks.get("sm_max_mhz", 2070.0),
                                steps=args.lagrange_steps)

    batched = None
    if not args.no_batched and args.precision != "fp64":
        batched = run_batched(binding, torch, dev, args.batched_systems, max(5, min(args.steps, 20)), 3,
                              args.precision)

    learned = None
    if not args.no_learned and args.precision != "fp64":
        learned = run_learned(binding, torch, dev, args.precision, flush)

    cpu = None
    if rank == 0 and not args.no_cpu and ws == 1:
        cpu = cpu_baseline(w, xy, q)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "ms_per_step_mean": max_over_ranks(float(np.mean(ms)), dev),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded SplitMix64: uniform positions in [0,5]^2, q ~ U[-1,1])",
            "config": {"workload": args.workload, "n": w["n"], "levels": w["levels"], "p": w["p"],
                       "precision": args.precision, "parallelism": f"replicas x{ws}",
                       "l2": "256 MB buffer written between timed steps (outside the events)"},
            "rel_l2_err": err, "meets_error_bound": err <= ERR_BOUND,
            "stage_ms": stage_avg, "kernel_ms": kern_avg, "kernel_ms_alone": alone, "roofline": roof,
            "roofline_stages": roof_all,
            "gpu_launches": launches, "e2e": e2e, "fp64_gpu": fp64, "alu_peaks_probe": probe,
            "speedup_vs_fp64_gpu": (value / fp64["value"]) if fp64 else None,
            "cpu_baseline": cpu, "batched": batched, "learned": learned, "lagrange": lagrange, "clustered": clustered, "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                                            "reasons": clk["reasons"], "samples": clk["samples"]},
            "wall_s_timed": wall,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- batched form

def batched_families(nsys, seed=20094767):
    """True for the systems batched_workload draws uniform (the rest are Gaussian mixtures)."""
    from paper_2009_00767_gb300 import inputs
    return inputs.u01(seed, 32, nsys) < 0.5


def batched_workload(nsys, seed=20094767):
    """1024 independent systems: N log-uniform in [1024, 262144], uniform or a Gaussian mixture
    per system (the clustered recipe: 32 Gaussians, sigma log-uniform in [0.01, 0.3]),
    q ~ U[-1, 1], depth round(log4(N / 16)) clamped to >= 2, p = 16."""
    from paper_2009_00767_gb300 import inputs
    u = inputs.u01(seed, 31, nsys)
    fam = inputs.u01(seed, 32, nsys)
    ns = np.exp(np.log(1024) + (np.log(262144) - np.log(1024)) * u).astype(np.int64)
    levels = np.maximum(2, np.rint(np.log(ns / 16.0) / np.log(4.0))).astype(np.int32)
    xys, qs = [], []
    for i in range(nsys):
        if fam[i] < 0.5:
            xy, q = inputs.uniform(int(ns[i]), seed + 17 * i)
        else:
            xy, q = inputs.gmm(int(ns[i]), seed + 17 * i)
        xys.append(xy)
        qs.append(q)
    return ns, levels, np.concatenate(xys), np.concatenate(qs)


def _time_batch(binding, torch, ns, levels, xy_d, q_d, steps, warmup, precision):
    """One batch over the systems (ns, levels), p = 16: autotuned, warmed up, then the median of
    `steps` graph replays timed with CUDA events."""
    phi = torch.empty(int(ns.sum()), dtype=torch.float64, device=xy_d.device)
    b = binding.Batch(ns, levels, 16, precision=precision)
    binding.fmm_batch_autotune_cached(b.handle, xy_d, q_d, phi, None)
    tuning = binding.fmm_batch_tuning(b.handle)
    for _ in range(warmup):
        binding.fmm_batch_potential(b.handle, xy_d, q_d, phi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms_steps = []
    for _ in range(steps):
        e0.record()
        binding.fmm_batch_potential(b.handle, xy_d, q_d, phi)
        e1.record()
        torch.cuda.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
    binding.fmm_batch_sync(b.handle)
    launches = binding.fmm_batch_launches(b.handle)
    b.close()
    return float(np.median(ms_steps)), phi, tuning, launches


def _batch_errors(binding, torch, ns, levels, xy_d, q_d, phi):
    """Relative L2 error of 8 systems spread over the size range, 256 sampled targets each, against
    the FP64 direct sum."""
    from paper_2009_00767_gb300 import inputs
    dev = xy_d.device
    off = np.concatenate([[0], np.cumsum(ns)])
    order = np.argsort(ns)
    errs = []
    for i in order[np.linspace(0, len(ns) - 1, 8).astype(int)]:
        n_i = int(ns[i])
        idx = np.unique((inputs.u01(5150 + int(i), 0, min(256, n_i)) * n_i).astype(np.int64))
        idx_d = torch.from_numpy(idx).to(dev)
        ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
        xs, qs_ = xy_d[off[i]:off[i + 1]].contiguous(), q_d[off[i]:off[i + 1]].contiguous()
        binding.fmm_direct_targets(xs, qs_, idx_d, ref)
        torch.cuda.synchronize()
        got = phi[off[i]:off[i + 1]][idx_d]
        errs.append({"system": int(i), "n": n_i, "levels": int(levels[i]),
                     "rel_l2_err": float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))})
    return errs


def run_batched(binding, torch, dev, nsys, steps, warmup, precision):
    """The batched form: one graph replay per step over all systems (launch shapes picked by the
    library's autotuner), against a loop of single-system plans of the same precision over the same
    systems; accuracy against the FP64 direct sum at sampled targets of sampled systems."""
    ns, levels, xy, q = batched_workload(nsys)
    total = int(ns.sum())
    xy_d = torch.from_numpy(xy).to(dev)
    q_d = torch.from_numpy(q).to(dev)
    ms_batch, phi, tuning, launches = _time_batch(binding, torch, ns, levels, xy_d, q_d, steps, warmup, precision)
    errs = _batch_errors(binding, torch, ns, levels, xy_d, q_d, phi)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the uniform half alone, as its own batch: the particles/s of the same form on the family of
    # the single-system workload (the Gaussian-mixture half fills its leaves unevenly at ~16
    # particles per leaf on average, so its near field dominates the mixed batch)
    uni = np.nonzero(batched_families(nsys))[0]
    off = np.concatenate([[0], np.cumsum(ns)])
    sel = np.concatenate([np.arange(off[i], off[i + 1]) for i in uni])
    xu, qu = xy_d[torch.from_numpy(sel).to(dev)].contiguous(), q_d[torch.from_numpy(sel).to(dev)].contiguous()
    ms_uni, phu, _, _ = _time_batch(binding, torch, ns[uni], levels[uni], xu, qu, steps, warmup, precision)
    uniform_subset = {"systems": int(uni.shape[0]), "particles": int(sel.shape[0]), "ms_per_step": ms_uni,
                      "value": sel.shape[0] / (ms_uni * 1e-3), "unit": UNIT}
    del xu, qu, phu
    # the same systems as a loop of single-system plans (one launch sequence per system)
    plans = [binding.Plan(int(ns[i]), int(levels[i]), 16, 5.0, precision) for i in range(nsys)]
    views = [(xy_d[off[i]:off[i + 1]], q_d[off[i]:off[i + 1]], phi[off[i]:off[i + 1]]) for i in range(nsys)]
    for _ in range(max(1, warmup // 2)):
        for pl, (x, qq, ph) in zip(plans, views):
            binding.fmm_potential(pl.handle, x, qq, ph)
    torch.cuda.synchronize()
    loop_steps = max(1, steps // 4)
    e0.record()
    for _ in range(loop_steps):
        for pl, (x, qq, ph) in zip(plans, views):
            binding.fmm_potential(pl.handle, x, qq, ph)
    e1.record()
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1) / loop_steps
    for pl in plans:
        pl.close()
    return {"systems": nsys, "particles": total, "ms_per_step": ms_batch, "value": total / (ms_batch * 1e-3),
            "unit": UNIT, "loop_ms_per_step": ms_loop, "loop_value": total / (ms_loop * 1e-3),
            "speedup_vs_loop": ms_loop / ms_batch, "graph_launches_per_step": launches, "tuning": tuning,
            "uniform_subset": uniform_subset,
            "precision": precision, "p": 16, "rel_l2_err_max": max(e["rel_l2_err"] for e in errs),
            "meets_error_bound": all(e["rel_l2_err"] <= ERR_BOUND for e in errs), "sampled_systems": errs,
            "timing": "CUDA events around each graph replay, median of the steps"}


# ---------------------------------------------------------------- learned selector

# held out (training seeds start at 700000, evaluation at 710000): two systems of each family --
# uniform (990001, 990007), Gaussian mixture (990005, 990006), annulus (990002, 990003)
LEARNED_SEEDS = (990001, 990007, 990005, 990006, 990002, 990003)


def run_learned(binding, torch, dev, precision, flush, steps=20):
    """The learned form: for held-out systems of the selector's family (N log-uniform in [2^16, 2^20],
    uniform / Gaussian mixture / annulus), the trained network's (levels, p) pick against the fixed
    (8, 20) and the no-network rule, each timed (median of `steps` calls, L2 flushed) and judged by
    the FP64 direct sum at 1024 sampled targets."""
    from paper_2009_00767_gb300 import inputs, selector
    model = os.path.join(ROOT, "paper_2009_00767_gb300", "selector_gb300.bin")
    if not os.path.exists(model):
        return None
    sel = binding.Selector(hidden=64, seed=1)
    sel.load(model)
    p_rule = selector.calibrate_p(ERR_BOUND, precision)   # the rule's p, calibrated live
    rows = []
    for sd in LEARNED_SEEDS:
        name, xy, q = selector.system(sd)
        n = int(q.shape[0])
        xy_d = torch.from_numpy(xy).to(dev)
        q_d = torch.from_numpy(q).to(dev)
        idx = np.unique((inputs.u01(sd, 78, 1024) * n).astype(np.int64))
        idx_d = torch.from_numpy(idx).to(dev)
        ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
        binding.fmm_direct_targets(xy_d, q_d, idx_d, ref)
        torch.cuda.synchronize()
        lev, p, fb = sel.select(xy_d, ERR_BOUND, 0.3)
        row = {"seed": sd, "family": name, "n": n, "pick": [lev, p], "fallback_used": fb}
        for key, (cl, cp) in (("pick", (lev, p)), ("fallback", selector.FALLBACK),
                              ("rule", (selector.heuristic_levels(n), p_rule))):
            phi = torch.empty(n, dtype=torch.float64, device=dev)
            with binding.Plan(n, cl, cp, 5.0, precision) as plan:
                for _ in range(3):
                    binding.fmm_potential(plan.handle, xy_d, q_d, phi)
                plan.sync()
                ms = []
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                for _ in range(steps):
                    flush.zero_()
                    e0.record()
                    binding.fmm_potential(plan.handle, xy_d, q_d, phi)
                    e1.record()
                    plan.sync()
                    ms.append(e0.elapsed_time(e1))
            row[f"ms_{key}"] = float(np.median(ms))
            row[f"err_{key}"] = float(torch.linalg.norm(phi[idx_d] - ref) / torch.linalg.norm(ref))
            if key == "rule":
                row["rule"] = [cl, cp]
        rows.append(row)
    sel.close()
    tot = {k: sum(r[f"ms_{k}"] for r in rows) for k in ("pick", "fallback", "rule")}
    total_n = sum(r["n"] for r in rows)
    return {"systems": rows, "precision": precision, "value": total_n / (tot["pick"] * 1e-3), "unit": UNIT,
            "ms_total": tot, "speedup_vs_fallback": tot["fallback"] / tot["pick"],
            "speedup_vs_rule": tot["rule"] / tot["pick"],
            "meets_error_bound": all(r["err_pick"] <= ERR_BOUND for r in rows),
            "rule_basis": f"no network: levels round(log4(N/16)), p {p_rule} = the smallest grid p meeting 1e-6 "
                          f"on a 2^18 uniform calibration system"}


# ---------------------------------------------------------------- clustered workload

def run_clustered(binding, torch, dev, precision, flush, steps, peaks):
    """The clustered configuration (2^24 particles, a mixture of 32 Gaussians, levels 10, p 24) in the
    benchmarked precision: median step, error against the FP64 direct sum at 4096 sampled targets,
    each stage's time alone and the near field's roofline.  On a uniform tree the clusters fill
    their leaves with thousands of particles, so the near field dominates."""
    w = WORKLOADS["gmm32_16m_l10_p24"]
    xy, q = make_inputs(w)
    xy_d, q_d = torch.from_numpy(xy).to(dev), torch.from_numpy(q).to(dev)
    stream = torch.cuda.current_stream(dev)
    plan, phi, ms, stage_ms, launches, wall, last = time_plan(binding, torch, w, precision, xy_d, q_d, steps, 2,
                                                              flush, stream)
    from paper_2009_00767_gb300 import inputs as inp
    idx = np.unique((inp.u01(4545, 0, 4096) * w["n"]).astype(np.int64))
    idx_d = torch.from_numpy(idx).to(dev)
    ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
    binding.fmm_direct_targets(xy_d, q_d, idx_d, ref)
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(phi[idx_d] - ref) / torch.linalg.norm(ref))
    alone = time_kernels_alone(binding, torch, plan, xy_d, q_d, phi, max(2, steps), 1, flush, stream)
    st = plan.stats()
    plan.close()
    med = float(np.median(ms))
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = N_SMS * MUFU_PER_SM * sm_max * 1e6 / 1e12
    ach = st["p2p_pairs"] / (alone["p2p_kernel"] * 1e-3) / 1e12 if alone["p2p_kernel"] > 0 else None
    return {"workload": "gmm32_16m_l10_p24", "n": w["n"], "levels": w["levels"], "p": w["p"],
            "precision": precision, "ms_per_step": med, "value": w["n"] / (med * 1e-3), "unit": UNIT,
            "rel_l2_err": err, "meets_error_bound": err <= ERR_BOUND, "kernel_ms_alone": alone,
            "max_leaf": st["max_leaf"], "p2p_pairs": st["p2p_pairs"],
            "roofline_p2p": None if ach is None else {
                "kernel": "k_p2p_mixed", "bound": "alu", "achieved": ach, "peak": peak, "unit": "Tlg2/s",
                "frac": ach / peak, "work_per_launch": f"{st['p2p_pairs']} ordered pairs, one lg2 each",
                "timing": "kernel alone (serial pass, CUDA events)"}}


# ---------------------------------------------------------------- Lagrange-node form (Appendix)

# The paper's own experiments (Sec. 3, Tables 1-3): +-1 charges uniform in a cube of side 5, 64
# nodes per cube, FP64 on one Core i7-9700; its total times are the context of these lines.
LAGRANGE_WORKLOADS = [
    {"name": "table1_3d_80k_l3", "dim": 3, "n": 80_000, "levels": 3, "paper_total_s": 9.4e-2, "paper_accuracy": 0.18e-2},
    {"name": "table2_3d_200k_l3", "dim": 3, "n": 200_000, "levels": 3, "paper_total_s": 1.1e-1, "paper_accuracy": 0.40e-2},
    {"name": "table3_3d_80k_l2", "dim": 3, "n": 80_000, "levels": 2, "paper_total_s": 1.4e-2, "paper_accuracy": 0.15e-2},
    {"name": "2d_1m_l7", "dim": 2, "n": 1 << 20, "levels": 7},
]


def run_lagrange(binding, torch, dev, flush, sm_max_mhz, steps=20, steps64=3):
    """The Lagrange-node form through include/fmm_lagrange.h: per workload each form's median step
    (L2 flushed between steps), its stage times alone (serial pass), its error against the FP64
    direct sum at sampled targets, and the near-field kernel's roofline; then, in 2D, the paper's
    literal form against the node form level by level (its FP64 conditioning, Sec. 4 (3))."""
    from paper_2009_00767_gb300 import inputs as inp
    out = []
    for wl in LAGRANGE_WORKLOADS:
        dim, n, L = wl["dim"], wl["n"], wl["levels"]
        pos, q = inp.paper_cube(n, inp.config_seed(30 + dim * 10 + L), dim)
        tp = torch.from_numpy(pos).to(dev)
        tq = torch.from_numpy(q).to(dev)
        S = min(4096, n)
        idx = np.unique((inp.u01(4343, 0, S) * n).astype(np.int64))
        idx_d = torch.from_numpy(idx).to(dev)
        ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
        binding.fmm_lag_direct_targets(tp, tq, idx_d, ref)
        torch.cuda.synchronize()
        forms = ("node_f32",) if dim == 2 else ("node_f32", "node_f64", "literal_f64")
        row = {"name": wl["name"], "dim": dim, "n": n, "levels": L, "forms": {}}
        for form in forms:
            k = steps if form == "node_f32" else steps64
            with binding.LagPlan(dim, n, L, 5.0, form) as plan:
                phi = torch.empty(n, dtype=torch.float64, device=dev)
                for _ in range(2):
                    plan.potential(tp, tq, phi)
                ms = []
                for _ in range(k):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    binding.fmm_lag_potential(plan.handle, tp, tq, n, phi)
                    e1.record()
                    plan.sync()
                    ms.append(e0.elapsed_time(e1))
                got = phi[idx_d]
                err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
                mean_rel = float(torch.mean(torch.abs((got - ref) / ref)))
                binding.fmm_lag_set_concurrency(plan.handle, 1)
                alone = []
                for _ in range(max(2, k // 2)):
                    flush.zero_()
                    plan.potential(tp, tq, phi)
                    alone.append(plan.stats())
                st = alone[-1]
            med = float(np.median(ms))
            stages = {key[3:]: float(np.median([a[key] for a in alone]))
                      for key in ("ms_sort", "ms_up", "ms_down", "ms_eval", "ms_p2p")}
            f = {"ms_per_step": med, "value": n / (med * 1e-3), "unit": UNIT, "rel_l2_vs_direct": err,
                 "mean_abs_rel_err_vs_direct": mean_rel, "stages_alone_ms": stages,
                 "p2p_pairs": st["p2p_pairs"], "m2l_pairs": st["m2l_pairs"],
                 "workspace_bytes": st["workspace_bytes"]}
            if form == "node_f32":
                # the near-field kernel, the longest stage: ordered pairs per second against the MUFU
                # rate (rsqrt in 3D, lg2 in 2D: 16 per clock per SM); the kernel evaluates each pair of
                # adjacent cells once for both sides (about 0.5 MUFU op per ordered pair)
                peak = N_SMS * MUFU_PER_SM * sm_max_mhz * 1e6 / 1e12
                ach = st["p2p_pairs"] / (stages["p2p"] * 1e-3) / 1e12
                f["roofline"] = {"kernel": "k_p2p32", "bound": "alu", "achieved": ach, "peak": peak,
                                 "unit": "Tpairs/s", "frac": ach / peak, "traffic": None,
                                 "work_per_launch": f"{st['p2p_pairs']} ordered pairs, one MUFU "
                                                    f"{'rsqrt' if dim == 3 else 'lg2'} each (the survey's unit)",
                                 "peak_basis": f"MUFU: {N_SMS} SMs x {MUFU_PER_SM}/clk x {sm_max_mhz:.0f} MHz",
                                 "timing": "kernel alone (serial pass, CUDA events)"}
            if "paper_total_s" in wl:
                f["speedup_vs_paper_total"] = wl["paper_total_s"] / (med * 1e-3)
            row["forms"][form] = f
        if "paper_total_s" in wl:
            row["paper"] = {"total_s": wl["paper_total_s"], "accuracy": wl["paper_accuracy"],
                            "machine": "FP64 Fortran, one Intel Core i7-9700 (Sec. 3)"}
        out.append(row)
        del tp, tq
    # FP64 conditioning of the literal form (2D, 2^16 charges): its error against the direct sum
    # next to the node form's, level by level
    cond = []
    pos, q = inp.paper_cube(1 << 16, inp.config_seed(39), 2)
    tp, tq = torch.from_numpy(pos).to(dev), torch.from_numpy(q).to(dev)
    idx = np.unique((inp.u01(4444, 0, 2048) * pos.shape[0]).astype(np.int64))
    idx_d = torch.from_numpy(idx).to(dev)
    ref = torch.empty(idx.shape[0], dtype=torch.float64, device=dev)
    binding.fmm_lag_direct_targets(tp, tq, idx_d, ref)
    torch.cuda.synchronize()
    for L in range(2, 8):
        r = {"levels": L}
        for form in ("node_f64", "literal_f64"):
            with binding.LagPlan(2, pos.shape[0], L, 5.0, form) as plan:
                phi = plan.potential(tp, tq)
                r[form] = float(torch.linalg.norm(phi[idx_d] - ref) / torch.linalg.norm(ref))
        cond.append(r)
    return {"workloads": out, "fp64_conditioning_2d_64k": cond,
            "data": "synthetic: +-1 charges uniform in a square/cube of side 5 (the paper's Sec. 3 setup)",
            "timing": "median step, CUDA events on the stream, 256 MB L2 flush between steps"}


# ---------------------------------------------------------------- CPU oracle

def cpu_model():
    """The host CPU's model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
        for line in out.splitlines():
            if line.startswith("Vendor ID"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_baseline(w, xy, q, max_runs=3, budget_s=30.0):
    """The oracle as it stands on the host cores: all threads, then one thread where a run fits the
    remaining budget (it reports `one_thread`, the same metric from a single core)."""
    import oracle
    oracle.build()
    runs, t_total = 0, 0.0
    while runs < max_runs and t_total < budget_s / 2:
        t = time.perf_counter()
        oracle.shiftfree(xy, q, w["levels"], w["p"])
        t_total += time.perf_counter() - t
        runs += 1
    cores = oracle.get_threads()
    res = {"value": runs * w["n"] / t_total, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"full workload (N={w['n']}, levels={w['levels']}, p={w['p']}), {runs} run(s) of the FP64 "
                     f"C oracle's shift-free FMM, OpenMP over independent outputs"}
    # one thread: expected about cores x the time of one all-core run
    if (t_total / runs) * cores <= budget_s / 2:
        oracle.set_threads(1)
        try:
            t = time.perf_counter()
            oracle.shiftfree(xy, q, w["levels"], w["p"])
            res["one_thread"] = {"value": w["n"] / (time.perf_counter() - t), "unit": UNIT, "cores": 1}
        finally:
            oracle.set_threads(cores)
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = WORKLOADS[args.workload]
    xy, q = make_inputs(w)
    # size one step so the whole run stays within about two minutes
    t = time.perf_counter()
    oracle.shiftfree(xy, q, w["levels"], w["p"])
    full = time.perf_counter() - t
    budget = 120.0 / max(1, args.steps + args.warmup)
    a = 0
    while full / (4 ** a) > budget and w["levels"] - a > 2:
        a += 1
    if a == 0:
        sx, sq, lev = xy, q, w["levels"]
        desc = f"full workload (N={w['n']}, levels={w['levels']}, p={w['p']})"
    else:
        side = 5.0 / (2 ** a)
        m = (xy[:, 0] < side) & (xy[:, 1] < side)
        sx, sq, lev = xy[m] * (2 ** a), q[m], w["levels"] - a   # the corner sub-square, rescaled to [0,5]^2
        desc = (f"corner 1/{4 ** a} of the workload ({int(m.sum())} particles, same density and p={w['p']}, "
                f"levels={lev}), FP64 C oracle shift-free FMM")
    for _ in range(args.warmup):
        oracle.shiftfree(sx, sq, lev, w["p"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.shiftfree(sx, sq, lev, w["p"])
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = sx.shape[0] / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": args.workload, "n": w["n"], "levels": w["levels"], "p": w["p"],
                       "precision": "fp64", "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_lagrange_only(args):
    import torch
    from paper_2009_00767_gb300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    res = run_lagrange(binding, torch, dev, flush, peaks.get("sm_max_mhz", 2070.0), steps=args.lagrange_steps,
                       steps64=max(1, min(3, args.lagrange_steps)))
    print(json.dumps({"lagrange": res}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.lagrange_only:
        run_lagrange_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
