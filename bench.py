#!/usr/bin/env python
"""Benchmark of the BlocKOA hot path on one GB300: verified sample pairs/s.

One step = the whole hot path on one synthetic chip (128 x 128 x 8 cells,
8 layers, s = 32 power maps, M = 5000 fields): assemble, right-hand sides,
two-step z-line-preconditioned mixed-precision block CG to a float64 relative
residual of 1e-6, bfloat16x3
tensor-core combination T = U C, operator action q = A T.  Inputs (power
maps and coefficients) are resident on the device when timing starts; L2 is
flushed (512 MB write) between timed steps, outside the timed events.  As a
serving loop would, the process creates one operator per precision for the
chip's shape and re-discretises it in place every step
(blockoa_reassemble: the assembly kernels run, allocations and the block-CG
graph are reused).

A pair (T_m, q_m) counts as verified when the basis it came from meets the
1e-6 relative residual (float64 true residual reported by the solver) and
||A T_m - q_m|| / ||q_m|| <= 1e-6 with A applied in float64 to the stored
T_m (blockoa_pair_check); verification runs after timing.

The JSON line also reports the plain float64 GPU form (unpreconditioned block
CG, as in the paper) on the same chip, the
end-to-end rate from pinned host buffers (host<->device copies timed; K
steps back to back, each step's pairs copied to the host while the next
step computes -- pipeline.PairStreamer), the
live roofline of the dominant kernel, sampled clocks, kernel launches, and
the FP64 CPU oracle timed on a bounded sample of the same workload.

Multi-GPU (torchrun): replicas -- each rank runs its own chip (seed offset by
rank) with no collective on the data path; value = pairs of all ranks / max
over ranks of the timed duration.

    python bench.py [--steps K] [--warmup W] [--impl reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "verified sample pairs/s at <=1e-6 rel err, chosen vs plain FP64, one GB300"
UNIT = "pairs/s"
RTOL = 1e-6
PAIR_TOL = 1e-6
# inner tolerance of the first float32 block-CG pass of the chosen (two-step
# z-line) form; the second pass is asked only for what the 1e-6 target still
# needs.  Measured on this chip: 1e-3 -> 89 iterations, 16.0 ms per solve;
# 1e-4 (the library default) -> 102 iterations, 17.1 ms; both two passes.
INNER_RTOL = 1e-3
# convergence polls of the chosen form: every 16 block-CG iterations (one
# CUDA graph of 16 iterations per poll; fewer host round trips)
CHECK_EVERY = 16
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070 / 1000   # SMs x FP32 lanes x 2 flop x max SM GHz
FP64_PEAK_TFLOPS = 1.25                      # GB300 float64 (vector and tensor), nominal


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--plain-steps", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=4)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(total_ms: float, verified: float, world: int, device=None):
    """Whole-job figures of a replicas run: the timed duration is the
    maximum over ranks and the verified pairs are summed over ranks (needs
    an initialised process group when world > 1)."""
    if world == 1:
        return total_ms, float(verified)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, float(verified)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def workload(rank: int):
    from paper_2510_23221_gb300 import synth
    # rank 0 is the 128x128x8 benchmark chip; other replicas draw their own chip
    return synth.single_chip_workload(cfg=2 if rank == 0 else 2000 + rank)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = self.summarize(f)
        os.unlink(self.path)
        return out

    @staticmethod
    def summarize(lines):
        """Median SM clock, maximum SM clock and the throttle reasons seen
        in nvidia-smi rows of FIELDS (csv, no header, no units); None when
        no row parses."""
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, v in enumerate(flags)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- our arm
def algorithmic(kernel: str, n: int, s: int, M: int, precond: str = "zline2"):
    """(bound, algorithmic units per launch, unit) of a kernel on an n-cell chip.

    Flop counts per cell (S = the padded block width, an FMA counted as 2):
    the 7-point stencil is 13 S, a tridiagonal z-line solve 5 S (forward
    elimination 3, back substitution 2), an S x S Gram or block update 2 S^2."""
    S = 8 if s <= 8 else 16 if s <= 16 else 32 if s <= 32 else 64
    Sp = (s + 15) // 16 * 16
    if precond == "zline2":
        # X and R updates, Z1 = M^-1 R and ||R_j||^2; W = Q^T Z is in zline_second
        update = n * (4 * S * S + 5 * S + 2 * S)
    elif precond == "zline":
        update = n * (6 * S * S + 5 * S + 2 * S)
    else:
        # X and R updates, W = Q^T (D^-1 R), column norms
        update = n * (6 * S * S + 3 * S)
    table = {
        # float32 SIMT: stencil + two S x S Grams (P^T Q, Q^T Q)
        "spmm_gram": ("alu", n * (13 * S + 4 * S * S), "flop"),
        "update_gram": ("alu", update, "flop"),
        # Y = 2 R - A Z1 (stencil + 2 S), z-line solve, W = Q^T Z
        "zline_second": ("alu", n * (13 * S + 2 * S + 5 * S + 2 * S * S), "flop"),
        "p_update": ("alu", n * 2 * S * S, "flop"),
        # operator action: read T, write q (float32)
        "apply_fields": ("hbm", 8 * n * M, "byte"),
        # combination: write T (float32), read the bf16x3 basis tiles
        "combine_tc": ("hbm", 4 * n * M + 2 * 3 * Sp * n, "byte"),
        "residual64": ("alu64", n * S * 14, "flop"),
    }
    return table.get(kernel)


def roofline(kt: dict, n: int, s: int, M: int, peaks: dict, precond: str = "zline2"):
    """Roofline entry of the dominant kernel from live event timings.

    Loop kernels are timed on one iteration per convergence poll; a kernel's
    share is its average timed launch times all its launches."""
    est = {name: (ms / cnt * nall if cnt else 0.0) for name, (ms, cnt, nall) in kt.items()}
    total_est = sum(est.values()) or 1.0
    ranked = sorted(((est[name], ms, name, cnt) for name, (ms, cnt, nall) in kt.items() if cnt > 0),
                    reverse=True)
    for _, ms, name, cnt in ranked:
        a = algorithmic(name, n, s, M, precond)
        if a is None:
            continue
        bound, units, kind = a
        avg_s = ms / cnt / 1e3
        if bound == "hbm":
            peak, unit, src = peaks.get("hbm_gbs", 6800.0), "GB/s", "measured copy (MEASURED_PEAKS.json)"
            achieved = units / avg_s / 1e9
        elif bound == "alu":
            peak, unit, src = FP32_PEAK_TFLOPS, "TFLOP/s", "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
            achieved = units / avg_s / 1e12
        else:
            peak, unit, src = FP64_PEAK_TFLOPS, "TFLOP/s", "nominal GB300 FP64"
            achieved = units / avg_s / 1e12
            bound = "alu"
        traffic = None
        tpath = os.path.join(ROOT, "profiles", "dram_traffic.json")
        if os.path.exists(tpath):
            traffic = json.load(open(tpath)).get(name)
        share = est[name] / total_est
        return {"kernel": name, "bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 1),
                "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": src, "avg_launch_us": round(avg_s * 1e6, 2),
                "timed_launches": int(cnt), "launches": int(kt[name][2]),
                "share_of_kernel_time": round(share, 3)}
    return None


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2510_23221_gb300 import blockoa as bo
    from paper_2510_23221_gb300 import build as bld
    from paper_2510_23221_gb300 import pipeline as pl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    bld.build()
    bo.library()
    dev = torch.device("cuda", local)
    w = workload(rank)
    n = w.chips[0].n
    s, M = w.s, w.M
    inputs = pl.upload(w)
    B = torch.empty(n * s, dtype=torch.float64, device=dev)
    U = torch.empty_like(B)
    T = torch.empty(n * M, dtype=torch.float32, device=dev)
    q = torch.empty_like(T)
    e_pair = torch.empty(M, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    CHOSEN_PRECOND = bo.PRECOND_ZLINE2   # two-step z-line
    ops = {}   # one long-lived operator per precision, re-discretised every step

    def operator(precision):
        if precision not in ops:
            ops[precision] = bo.assemble(w.chips)
        return bo.reassemble(ops[precision], w.chips)

    def step(precision, Tb, qb, precond=CHOSEN_PRECOND):
        op = operator(precision)
        bo.build_rhs(op, inputs.density, B, s)
        chosen = precision == bo.MIXED and precond == CHOSEN_PRECOND
        st = bo.block_solve(op, B, U, s, rtol=RTOL, precision=precision, precond=precond,
                            inner_rtol=INNER_RTOL if chosen else 0.0,
                            check_every=CHECK_EVERY if chosen else 0, raise_on_error=False)
        bo.combine(op, U, inputs.C, Tb, s, M, precision)
        bo.apply_operator(op, Tb, qb, M, precision)
        return op, st

    def verify(op, st, Tb, qb, precision):
        bo.pair_check(op, Tb, qb, M, precision, e_pair)
        ep = e_pair.cpu().numpy()
        ok_basis = st[0].status == bo.OK and st[0].relres_max <= RTOL
        return int(np.sum(ep <= PAIR_TOL)) if ok_basis else 0, float(ep.max()), st[0]

    for _ in range(args.warmup):
        op, st = step(bo.MIXED, T, q)
    torch.cuda.synchronize()
    bo.reset_kernel_times(op)

    clocks = ClockSampler(local)
    launches0 = bo.launch_count()
    kt_sum = {}
    step_ms, verified, worst_pair, solver = [], 0, 0.0, []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        op, st = step(bo.MIXED, T, q)
        ev1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for name, (ms, cnt, nall) in bo.kernel_times(op).items():
            a, b, c = kt_sum.get(name, (0.0, 0, 0))
            kt_sum[name] = (a + ms, b + cnt, c + nall)
        bo.reset_kernel_times(op)
        v, worst, st0 = verify(op, st, T, q, bo.MIXED)   # outside the timed events
        verified += v
        worst_pair = max(worst_pair, worst)
        solver.append(st0)
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - t_wall
    clk = clocks.stop()
    launches = bo.launch_count() - launches0
    total_ms = sum(step_ms)
    total_ms_max, verified_all = aggregate(total_ms, verified, world, dev)
    value = verified_all / (total_ms_max / 1e3)

    # ---- plain float64 GPU form on the same chip
    plain = None
    if args.plain_steps > 0:
        T64 = torch.empty(n * M, dtype=torch.float64, device=dev)
        q64 = torch.empty_like(T64)
        op, st = step(bo.FP64, T64, q64, bo.PRECOND_NONE)   # warm-up
        pms, pver = [], 0
        for _ in range(args.plain_steps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            op, st = step(bo.FP64, T64, q64, bo.PRECOND_NONE)
            ev1.record(stream)
            torch.cuda.synchronize()
            pms.append(ev0.elapsed_time(ev1))
            v, _, st0 = verify(op, st, T64, q64, bo.FP64)
            pver += v
        plain = {"value": round(pver / (sum(pms) / 1e3), 2), "unit": UNIT,
                 "ms_per_step": round(statistics.mean(pms), 3), "iters": st0.iters,
                 "verified_pairs_per_step": pver // len(pms)}
        del T64, q64

    # ---- end to end from pinned host buffers, host<->device copies timed.
    # K steps back to back through pipeline.PairStreamer: each step copies its
    # inputs in from pinned host memory, runs the hot path and streams its
    # pairs (T, q) back to pinned host memory on a copy stream while the next
    # step computes.  Timed from the first input copy to the last byte of the
    # last step on the host; afterwards every pair that reached host memory is
    # uploaded again and verified.
    e2e = None
    if args.e2e_steps > 0:
        K = args.e2e_steps
        dens_h, C_h = pl.host_inputs(w)
        dens_p = torch.from_numpy(dens_h).pin_memory()
        C_p = torch.from_numpy(C_h).pin_memory()
        outs = [(torch.empty(n * M, dtype=torch.float32, pin_memory=True),
                 torch.empty(n * M, dtype=torch.float32, pin_memory=True)) for _ in range(K)]
        dens_d = torch.empty_like(inputs.density)
        C_d = torch.empty_like(inputs.C)
        ps = pl.PairStreamer(operator(bo.MIXED), s, M, bo.MIXED)
        kw = dict(rtol=RTOL, precond=CHOSEN_PRECOND, inner_rtol=INNER_RTOL, check_every=CHECK_EVERY,
                  raise_on_error=False)
        for k in range(K):   # warm-up: every pinned output buffer written once (first touch)
            ps.step(w.chips, dens_p, C_p, dens_d, C_d, *outs[k], **kw)
        ps.finish()
        torch.cuda.synchronize()
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e2e_stats = [ps.step(w.chips, dens_p, C_p, dens_d, C_d, *outs[k], **kw) for k in range(K)]
        ps.finish()
        ev1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = ev0.elapsed_time(ev1)
        ever = 0
        for k in range(K):   # verify what reached the host
            ps.T[0].copy_(outs[k][0])
            ps.q[0].copy_(outs[k][1])
            ever += verify(ps.op, e2e_stats[k], ps.T[0], ps.q[0], bo.MIXED)[0]
        e2e = {"value": round(ever / (e2e_ms / 1e3), 2), "unit": UNIT,
               "ms_per_step": round(e2e_ms / K, 3), "steps": K,
               "h2d_bytes_per_step": int(dens_h.nbytes + C_h.nbytes),
               "d2h_bytes_per_step": int(outs[0][0].numel() * 4 + outs[0][1].numel() * 4),
               "overlap": "pairs of step k copied to host while step k+1 computes"}
        del ps, outs

    for o in ops.values():
        o.close()
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    roof = roofline(kt_sum, n, s, M, peaks, precond="zline2")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "cells": n, "s": s, "M": M, "precision": "mixed",
                       "precond": "zline2", "inner_rtol": INNER_RTOL, "check_every": CHECK_EVERY, "plain_fp64_precond": "none",
                       "rtol": RTOL, "pair_tol": PAIR_TOL,
                       "l2": "flushed between steps (512 MB write, outside timed events)",
                       "parallelism": f"replicas x{world}"},
            "verification": {"verified_pairs": int(verified_all),
                             "pairs": int(M * args.steps * world),
                             "max_e_pair": worst_pair,
                             "iters": [x.iters for x in solver],
                             "refine_steps": [x.refine_steps for x in solver],
                             "relres_max": max(x.relres_max for x in solver)},
            "plain_fp64": plain, "e2e": e2e, "gpu_launches": int(launches),
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "kernel_timing": {k: {"timed_ms": round(v[0], 3), "timed_launches": v[1], "launches": v[2],
                                  "avg_us": round(1e3 * v[0] / v[1], 2)}
                              for k, v in sorted(kt_sum.items()) if v[1] > 0},
            "wall_s_timed": round(wall_s, 3),
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- oracle (CPU)
def oracle_sample(w, seconds: float):
    """Time the FP64 oracle on a bounded sample of the workload and scale it
    to the whole workload: assembly in full, the first block-CG iterations
    (as many as fit in about half the budget), and combination + operator
    action for a subset of the fields.  The iteration count used for scaling
    is the oracle's own, recorded by oracle/record_iterations.py."""
    from oracle import blockoa_oracle as orc
    chip = w.chips[0]
    t0 = time.perf_counter()
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    t_asm = time.perf_counter() - t0
    # block CG iterations, timed as whole iterations from the start
    budget = 0.5 * seconds
    k = 4
    while True:
        t0 = time.perf_counter()
        orc.block_cg(A, B, rtol=0.0 + 1e-300, maxiter=k)
        dt = time.perf_counter() - t0
        if dt > budget / 4 or k >= 256:
            break
        k *= 2
    t_iter = dt / k
    rec = json.load(open(os.path.join(ROOT, "oracle", "recorded_iterations.json")))
    iters = rec.get("chip128x128x8_s32", {}).get("iters", 291)
    # combination + operator action on a field subset
    U = np.random.default_rng(0).standard_normal((chip.n, w.s))
    mf = 8
    t0 = time.perf_counter()
    while True:
        Tm = orc.combine(U, w.coeffs[0][:, :mf])
        orc.apply_operator(A, Tm)
        dt = time.perf_counter() - t0
        if dt > 0.25 * seconds or mf >= w.M:
            break
        mf *= 2
        t0 = time.perf_counter()
    t_field = dt / mf
    total = t_asm + t_iter * iters + t_field * w.M
    sample = (f"oracle on {w.name}: assembly, {k} block-CG iterations scaled to the oracle's "
              f"{iters}, combine+apply on {mf} of {w.M} fields scaled to {w.M}")
    return w.M / total, sample, total


def cpu_cores():
    try:
        import numpy.__config__  # noqa: F401
    except Exception:
        pass
    return os.cpu_count()


def cpu_baseline(w, seconds):
    v, sample, total = oracle_sample(w, seconds)
    return {"value": round(v, 4), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": sample, "estimated_s_per_step": round(total, 2)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(0)
    per_step = max(2.0, min(8.0, 90.0 / max(1, args.steps + args.warmup)))
    vals, totals = [], []
    sample = ""
    for k in range(args.warmup + args.steps):
        v, sample, total = oracle_sample(w, per_step)
        if k >= args.warmup:
            vals.append(v)
            totals.append(total)
    value = len(vals) * w.M / sum(totals)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * statistics.mean(totals), 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "cells": w.chips[0].n, "s": w.s, "M": w.M,
                      "precision": "fp64", "rtol": RTOL},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cpu_cores(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
