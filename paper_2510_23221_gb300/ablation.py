"""Block CG against independent single-right-hand-side CG on one chip, and
the per-sample direct method against the basis route.

    python -m paper_2510_23221_gb300.ablation [--chip 128x128x8] [--s 32]
        [--tols 1e-3,1e-5,1e-6,1e-7,1e-9] [--direct-batches 2]
    python -m paper_2510_23221_gb300.ablation --workload paper3dic [--tols 1e-6]

With ``--workload paper3dic`` only part 1 runs, on the paper's ablation
setting (Sec. V-E: five 3-D IC floorplans of ~1e5 cells batched, 50 basis
sources each, Dirichlet faces): iterations are the largest over the chips.

Part 1 (iterations): the chip's s power maps are solved with the s columns
coupled (block CG, one Krylov space) and with the columns independent
(s scalar CG solves: every off-diagonal Gram entry dropped), at each
tolerance, in the chosen form (mixed precision, two-step z-line preconditioning)
and in the plain float64 unpreconditioned form.  Reported: block
iterations, the largest single-column iteration count, and solve times
(CUDA events, device-resident inputs, warm operator).

Part 2 (throughput at 1e-6): the direct method makes each sample
(T_m, q_m) by solving A T_m = q_m for its own power map q_m, here in
batches of 64 independent columns (the widest block this library solves
at once); a sample is verified when its float64 true residual is <= 1e-6.
The basis route (assemble, s basis solves, T = U C, q = A T for M fields)
is timed on the same chip with the same verification rule applied to its
basis.  Both are reported as verified pairs per second.

Part 3 (q by linearity): on the basis of part 2, q = (A U) C
(blockoa_apply_basis + blockoa_combine) against q = A T on the float32 T
(blockoa_apply_operator): time, and the largest e_q of each against a
float64 reference (float64 combination and operator action of the same U);
and the cost of the combination's noise term on the same fields.

Prints one JSON line per measurement.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    from . import blockoa as bo
    from . import build, pipeline as pl, synth

    p = argparse.ArgumentParser()
    p.add_argument("--chip", default="128x128x8")
    p.add_argument("--s", type=int, default=32)
    p.add_argument("--M", type=int, default=5000)
    p.add_argument("--tols", default="1e-3,1e-5,1e-6,1e-7,1e-9")
    p.add_argument("--direct-batches", type=int, default=2)
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--workload", choices=["chip", "paper3dic"], default="chip")
    a = p.parse_args()
    build.build()
    dev = torch.device("cuda")
    if a.workload == "paper3dic":
        w = synth.paper_3dic_workload(M=8)
        a.chip = "paper3dic_5x92x92x12"
        op = bo.assemble(w.chips)
        n, s = op.n_total, w.s
        qv = torch.from_numpy(np.concatenate([q.ravel() for q in w.sources])).to(dev)
        B = torch.empty(n * s, dtype=torch.float64, device=dev)
        U = torch.empty_like(B)
        bo.build_rhs_volume(op, qv, B, s)
    else:
        nx, ny, nl = (int(v) for v in a.chip.split("x"))
        w = synth.single_chip_workload(nx, ny, nl, s=a.s, M=a.M)
        op = bo.assemble(w.chips)
        n, s = op.n_total, a.s
        inputs = pl.upload(w)
        B = torch.empty(n * s, dtype=torch.float64, device=dev)
        U = torch.empty_like(B)
        bo.build_rhs(op, inputs.density, B, s)
    forms = {"chosen": dict(precision=bo.MIXED, precond=bo.PRECOND_ZLINE2),
             "plain_fp64": dict(precision=bo.FP64, precond=bo.PRECOND_NONE)}

    def timed(fn):
        out = fn()   # warm (workspace and graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / a.reps

    # ---- part 1: iterations and time, block vs independent columns
    for tol in (float(t) for t in a.tols.split(",")):
        for fname, kw in forms.items():
            row = {"part": "iterations", "chip": a.chip, "s": s, "rtol": tol, "form": fname}
            for mode, indep in (("block", False), ("independent", True)):
                st, ms = timed(lambda: bo.block_solve(op, B, U, s, rtol=tol, independent=indep,
                                                      raise_on_error=False, **kw))
                row[mode] = {"iters": max(x.iters for x in st), "status": max(x.status for x in st),
                             "relres": max(x.relres_max for x in st), "ms": round(ms, 3)}
            row["iteration_ratio"] = round(row["independent"]["iters"] / max(row["block"]["iters"], 1), 3)
            print(json.dumps(row), flush=True)
    if a.workload == "paper3dic":
        op.close()
        return

    # ---- part 2: verified pairs/s at 1e-6, direct method vs the basis route
    tol, sd = 1e-6, 64
    rng = np.random.default_rng(31_000_000)
    dens = torch.from_numpy(np.ascontiguousarray(synth.power_maps(rng, nx, ny, sd, mix=True).ravel())).to(dev)
    Bd = torch.empty(n * sd, dtype=torch.float64, device=dev)
    Xd = torch.empty_like(Bd)
    kw = forms["chosen"]
    bo.build_rhs(op, dens, Bd, sd)
    bo.block_solve(op, Bd, Xd, sd, rtol=tol, independent=True, raise_on_error=False, **kw)   # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    verified, iters = 0, []
    e0.record()
    for _ in range(a.direct_batches):
        bo.build_rhs(op, dens, Bd, sd)
        st = bo.block_solve(op, Bd, Xd, sd, rtol=tol, independent=True, raise_on_error=False, **kw)
        iters.append(st[0].iters)
        verified += sd if (st[0].status == bo.OK and st[0].relres_max <= tol) else 0
    e1.record()
    torch.cuda.synchronize()
    dms = e0.elapsed_time(e1)
    direct = {"pairs_per_s": round(verified / (dms / 1e3), 2), "samples": sd * a.direct_batches,
              "verified": verified, "ms_per_batch_of_64": round(dms / a.direct_batches, 3),
              "iters_per_batch": iters}
    # the basis route on the same chip: s basis solves + combine + apply for M fields
    T = torch.empty(n * a.M, dtype=torch.float32, device=dev)
    q = torch.empty_like(T)

    def route():
        bo.reassemble(op, w.chips)
        bo.build_rhs(op, inputs.density, B, s)
        st = bo.block_solve(op, B, U, s, rtol=tol, raise_on_error=False, **kw)
        bo.combine(op, U, inputs.C, T, s, a.M, bo.MIXED)
        bo.apply_operator(op, T, q, a.M, bo.MIXED)
        return st

    st, rms = timed(route)
    ok = st[0].status == bo.OK and st[0].relres_max <= tol
    basis = {"pairs_per_s": round((a.M if ok else 0) / (rms / 1e3), 2), "pairs": a.M, "ms_per_step": round(rms, 3),
             "iters": st[0].iters, "note": "basis verified by its float64 true residual; per-pair checks in bench.py"}
    print(json.dumps({"part": "throughput", "chip": a.chip, "rtol": tol, "form": "chosen",
                      "direct_method": direct, "basis_route": basis,
                      "speedup": round(basis["pairs_per_s"] / max(direct["pairs_per_s"], 1e-9), 1)}), flush=True)

    # ---- part 3: q by linearity, q = (A U) C, against q = A T on the float32 T
    del T, q
    T = torch.empty(n * a.M, dtype=torch.float32, device=dev)
    q_apply = torch.empty_like(T)
    q_lin = torch.empty_like(T)
    AU = torch.empty(n * s, dtype=torch.float64, device=dev)
    bo.combine(op, U, inputs.C, T, s, a.M, bo.MIXED)
    _, ms_apply = timed(lambda: bo.apply_operator(op, T, q_apply, a.M, bo.MIXED))

    def linear():
        bo.apply_basis(op, U, AU, s)
        bo.combine(op, AU, inputs.C, q_lin, s, a.M, bo.MIXED)

    _, ms_lin = timed(linear)
    # float64 reference of the same basis: T64 = U C and q64 = A T64 in float64
    T64 = torch.empty(n * a.M, dtype=torch.float64, device=dev)
    q64 = torch.empty_like(T64)
    bo.combine(op, U, inputs.C, T64, s, a.M, bo.FP64)
    bo.apply_operator(op, T64, q64, a.M, bo.FP64)
    ref = q64.view(a.M, n)

    def e_q(x):
        d = torch.linalg.vector_norm(x.view(a.M, n).double() - ref, dim=1)
        return float((d / torch.linalg.vector_norm(ref, dim=1)).max())

    print(json.dumps({"part": "q_by_linearity", "chip": a.chip, "M": a.M,
                      "apply_ms": round(ms_apply, 3), "linearity_ms": round(ms_lin, 3),
                      "e_q_apply_max": e_q(q_apply), "e_q_linearity_max": e_q(q_lin)}), flush=True)
    # the epsilon term of Eq. 5 in the combination: its cost on M fields
    _, ms_plain = timed(lambda: bo.combine(op, U, inputs.C, T, s, a.M, bo.MIXED))
    _, ms_noise = timed(lambda: bo.combine(op, U, inputs.C, T, s, a.M, bo.MIXED, noise_seed=7, noise_amp=0.01))
    print(json.dumps({"part": "combine_noise", "chip": a.chip, "M": a.M, "combine_ms": round(ms_plain, 3),
                      "combine_with_noise_ms": round(ms_noise, 3)}), flush=True)
    op.close()


if __name__ == "__main__":
    main()
