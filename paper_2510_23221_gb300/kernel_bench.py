"""Microbenchmark of single C-ABI calls (operator action, combination, solve).

    python -m paper_2510_23221_gb300.kernel_bench --call apply --chip 512x512x16 --M 1000
    python -m paper_2510_23221_gb300.kernel_bench --call combine --chip 128x128x8 --s 32 --M 5000
    python -m paper_2510_23221_gb300.kernel_bench --call solve --chip 128x128x8 --s 32 --precond jacobi

Times `--reps` calls with CUDA events after `--warmup` calls and prints one
JSON line with the mean time and the algorithmic bandwidth (operator action:
read T + write q; combination: write T + read the bfloat16x3 basis images).
Inputs are random (solve: the chip's power-map right-hand sides, relative
residual 1e-6); no correctness check beyond the solver's status (the test
suite does that).
"""
from __future__ import annotations

import argparse
import dataclasses
import json

import numpy as np


def main():
    import torch

    from . import blockoa as bo
    from . import build, synth
    from . import pipeline as pl

    p = argparse.ArgumentParser()
    p.add_argument("--call", choices=["apply", "combine", "solve"], default="apply")
    p.add_argument("--chip", default="128x128x8")
    p.add_argument("--s", type=int, default=32)
    p.add_argument("--M", type=int, default=1000)
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--precond", choices=["none", "jacobi", "zline", "zline2"], default="jacobi")
    p.add_argument("--small", choices=["auto", "fp64-cholesky"], default="auto")
    p.add_argument("--deterministic", action="store_true", help="static schedules, ordered reductions")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--reps", type=int, default=10)
    a = p.parse_args()
    build.build()
    nx, ny, nl = (int(v) for v in a.chip.split("x"))
    w = synth.single_chip_workload(nx, ny, nl, s=a.s, M=a.M, cfg=7)
    op = bo.assemble(w.chips)
    n, M, s = op.n_total, a.M, a.s
    prec = bo.MIXED if a.precision == "mixed" else bo.FP64
    fdt = torch.float32 if prec == bo.MIXED else torch.float64
    T = torch.randn(n * M, dtype=fdt, device="cuda")
    q = torch.empty_like(T)
    U = torch.randn(n * s, dtype=torch.float64, device="cuda")
    C = torch.from_numpy(np.ascontiguousarray(w.coeffs[0].ravel())).cuda()
    stats = []
    if a.call == "solve":
        del T, q
        dens = pl.upload(w).density
        B = torch.empty(n * s, dtype=torch.float64, device="cuda")
        bo.build_rhs(op, dens, B, s)
        pc = {"none": bo.PRECOND_NONE, "jacobi": bo.PRECOND_JACOBI, "zline": bo.PRECOND_ZLINE, "zline2": bo.PRECOND_ZLINE2}[a.precond]

    def call():
        if a.call == "solve":
            stats[:] = bo.block_solve(op, B, U, s, rtol=1e-6, precision=prec, precond=pc,
                                      small_solve=bo.SMALL_AUTO if a.small == "auto" else bo.SMALL_FP64_CHOLESKY,
                                      deterministic=a.deterministic)
        elif a.call == "apply":
            bo.apply_operator(op, T, q, M, prec)
        else:
            bo.combine(op, U, C, T, s, M, prec)

    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    esz = 4 if prec == bo.MIXED else 8
    if a.call == "apply":
        nbytes = 2 * esz * n * M
    elif a.call == "solve":
        nbytes = 0
    else:
        nbytes = esz * n * M + (6 * ((s + 15) // 16 * 16) * n if prec == bo.MIXED else 8 * n * s)
    kt = bo.kernel_times(op)
    print(json.dumps({"call": a.call, "chip": a.chip, "cells": n, "s": s, "M": M, "small": a.small,
                      "precision": a.precision, "ms": round(ms, 4),
                      "GBps": round(nbytes / ms / 1e6, 1),
                      "solver": [dataclasses.asdict(st) for st in stats],
                      "kernels": {k: round(v[0] / v[1], 4) for k, v in kt.items() if v[1]}}))


if __name__ == "__main__":
    main()
