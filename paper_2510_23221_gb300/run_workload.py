"""Run one synthetic workload through the whole hot path and report it.

    python -m paper_2510_23221_gb300.run_workload --workload batch256
    python -m paper_2510_23221_gb300.run_workload --workload chip512 --chunk 1000

Workloads (seeded, see synth.py):
  chip128  -- one 128x128x8 chip, s = 32, M = 5000 (the benchmark chip)
  batch256 -- 256 uneven chips (sides 64..256, 4-12 layers), s = 16, M = 20
  chip512  -- one 512x512x16 chip, s = 64, M = 10,000 streamed in chunks
  paper3dic -- the 3-D IC of the paper's experiments (Sec. V-A) in its
              ablation setting (Sec. V-E): 5 floorplans of 92x92x12 cells
              (copper TSV columns, sources in the core and both cache
              layers), s = 50, M = 1000 per chip, Dirichlet faces (or
              --boundary robin / mixed), noise epsilon of amplitude 0.01

One pass: assemble, right-hand sides, block CG to the workload's relative
residual (1e-6), then per chunk of fields the combination T = U C and the
operator action q = A T.  Phases are timed with CUDA events on the current
stream (inputs resident on the device).  After timing every pair is checked
in float64 (blockoa_pair_check) and counted as verified when its chip's
basis met the tolerance and e_pair <= 1e-6.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

PAIR_TOL = 1e-6


def main():
    import torch

    from . import blockoa as bo
    from . import build, synth

    p = argparse.ArgumentParser()
    p.add_argument("--workload", choices=["chip128", "batch256", "chip512", "paper3dic"], default="batch256")
    p.add_argument("--boundary", choices=list(synth.PAPER_BOUNDARIES), default="dirichlet",
                   help="boundary scenario of the paper3dic workload")
    p.add_argument("--noise-amp", type=float, default=None,
                   help="noise epsilon of the combination (default 0.01 for paper3dic, else 0)")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--precond", choices=["none", "jacobi", "zline", "zline2"], default="jacobi")
    p.add_argument("--chunk", type=int, default=1000, help="fields per combine/apply pass")
    p.add_argument("--M", type=int, default=0, help="override the workload's field count")
    p.add_argument("--maxiter", type=int, default=20000)
    p.add_argument("--no-verify", action="store_true")
    p.add_argument("--autotune", action="store_true", help="tune the unit sizes before the timed pass")
    a = p.parse_args()
    build.build()
    if a.workload == "chip128":
        w = synth.single_chip_workload(M=a.M or 5000)
    elif a.workload == "batch256":
        w = synth.batched_workload(M=a.M or 20)
    elif a.workload == "chip512":
        w = synth.large_chip_workload(M=a.M or 10000)
    else:
        w = synth.paper_3dic_workload(M=a.M or 1000, boundary=a.boundary)
    amp = a.noise_amp if a.noise_amp is not None else (0.01 if a.workload == "paper3dic" else 0.0)
    prec = bo.MIXED if a.precision == "mixed" else bo.FP64
    pc = {"none": bo.PRECOND_NONE, "jacobi": bo.PRECOND_JACOBI, "zline": bo.PRECOND_ZLINE, "zline2": bo.PRECOND_ZLINE2}[a.precond]
    fdt = torch.float32 if prec == bo.MIXED else torch.float64
    dev = torch.device("cuda")
    s, M = w.s, w.M
    chunk = min(a.chunk, M)
    n_chunks = (M + chunk - 1) // chunk
    # inputs resident: densities (or volumetric sources), and C split into
    # per-chunk [chip][s][chunk] blocks
    src = w.sources if w.sources is not None else w.density
    dens = torch.from_numpy(np.concatenate([np.ascontiguousarray(d, np.float64).ravel()
                                            for d in src])).to(dev)
    C_chunks = []
    for q in range(n_chunks):
        m0, m1 = q * chunk, min(M, (q + 1) * chunk)
        C_chunks.append(torch.from_numpy(np.concatenate(
            [np.ascontiguousarray(c[:, m0:m1], np.float64).ravel() for c in w.coeffs])).to(dev))
    tuning = None
    if a.autotune:   # one-time, per operator shape; outside the timed pass
        op_t = bo.assemble(w.chips)
        tuning = bo.autotune(op_t, w.s, prec, pc)
        op_t.close()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    ev[0].record(stream)
    op = bo.assemble(w.chips)
    if tuning:
        bo.set_tuning(op, tuning["tiles_per_unit"], tuning["ztiles_per_unit"])
    n = op.n_total
    B = torch.empty(n * s, dtype=torch.float64, device=dev)
    U = torch.empty_like(B)
    if w.sources is not None:
        bo.build_rhs_volume(op, dens, B, s)
    else:
        bo.build_rhs(op, dens, B, s)
    ev[1].record(stream)
    stats = bo.block_solve(op, B, U, s, rtol=w.rtol, maxiter=a.maxiter, precision=prec, precond=pc,
                           raise_on_error=False)
    ev[2].record(stream)
    torch.cuda.synchronize()
    T = torch.empty(n * chunk, dtype=fdt, device=dev)
    q_ = torch.empty_like(T)
    e_pair = torch.empty(op.n_chips * chunk, dtype=torch.float64, device=dev)
    ok_basis = np.array([st.status == bo.OK and st.relres_max <= w.rtol for st in stats])
    comb_ms, apply_ms, verified, worst = [], [], 0, 0.0
    for qi in range(n_chunks):
        Mc = min(M, (qi + 1) * chunk) - qi * chunk
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        # noise counters restart per chunk: field index within the chunk, so
        # chunks use disjoint seeds
        bo.combine(op, U, C_chunks[qi], T, s, Mc, prec, noise_seed=1 + qi, noise_amp=amp)
        e1.record(stream)
        bo.apply_operator(op, T, q_, Mc, prec)
        e2.record(stream)
        torch.cuda.synchronize()
        comb_ms.append(e0.elapsed_time(e1))
        apply_ms.append(e1.elapsed_time(e2))
        if not a.no_verify:   # after the timed phases of this chunk
            bo.pair_check(op, T, q_, Mc, prec, e_pair)
            ep = e_pair[:op.n_chips * Mc].view(op.n_chips, Mc).cpu().numpy()
            verified += int(np.sum((ep <= PAIR_TOL) & ok_basis[:, None]))
            worst = max(worst, float(ep.max()))
    setup_ms = ev[0].elapsed_time(ev[1])
    solve_ms = ev[1].elapsed_time(ev[2])
    total_ms = setup_ms + solve_ms + sum(comb_ms) + sum(apply_ms)
    esz = 4 if prec == bo.MIXED else 8
    its = [st.iters for st in stats]
    kt = bo.kernel_times(op)
    out = {
        "workload": w.name, "chips": op.n_chips, "cells": n, "s": s, "M": M, "chunk": chunk,
        "precision": a.precision, "precond": a.precond, "noise_amp": amp,
        "ms": {"assemble_rhs": round(setup_ms, 3), "solve": round(solve_ms, 3),
               "combine": round(sum(comb_ms), 3), "apply": round(sum(apply_ms), 3),
               "total": round(total_ms, 3)},
        "pairs": op.n_chips * M, "verified_pairs": verified if not a.no_verify else None,
        "verified_pairs_per_s": round(verified / (total_ms / 1e3), 2) if not a.no_verify else None,
        "max_e_pair": worst if not a.no_verify else None,
        "iters": {"min": min(its), "median": statistics.median(its), "max": max(its)},
        "status_counts": {str(k): sum(1 for st in stats if st.status == k) for k in sorted({st.status for st in stats})},
        "relres_max": max(st.relres_max for st in stats),
        "apply_GBps": round(2 * esz * n * M / (sum(apply_ms) / 1e3) / 1e9, 1),
        "combine_GBps_T_writes": round(esz * n * M / (sum(comb_ms) / 1e3) / 1e9, 1),
        "kernels_avg_us": {k: round(1e3 * v[0] / v[1], 2) for k, v in kt.items() if v[1]},
        "tuning": tuning,
    }
    print(json.dumps(out), flush=True)
    op.close()


if __name__ == "__main__":
    main()
