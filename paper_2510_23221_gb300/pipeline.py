"""The whole hot path through the C ABI: assemble, right-hand sides, block
solve, combination and operator action for a synthetic workload.

Orchestration and argument marshalling only; every arithmetic step runs in
libblockoa.so.  Device buffers are torch CUDA tensors.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import blockoa as bo

# Solve options of the chosen form on the 128x128x8 benchmark chip: mixed
# precision (float32 block CG inside float64 refinement), two-step z-line
# preconditioning, the first float32 pass asked for a 1e-3 residual
# reduction (later passes only for what the target still needs), a
# convergence poll every 16 iterations, the s x s Gram systems factored
# by float64 pivoted Cholesky.  deterministic=True (static unit schedules,
# partial sums added in a fixed order: the same inputs give the same bits
# and iteration counts) measured 1-4% slower per step on this chip.
CHOSEN_SOLVE = dict(precision=bo.MIXED, precond=bo.PRECOND_ZLINE2, inner_rtol=1e-3,
                    check_every=16, small_solve=bo.SMALL_FP64_CHOLESKY, deterministic=False)


@dataclass
class DeviceInputs:
    density: "object"   # torch float64 [chip][s][ny][nx] concatenated
    C: "object"         # torch float64 [chip][s][M]


@dataclass
class Result:
    op: bo.Operator
    B: "object"
    U: "object"
    T: "object"
    q: "object"
    stats: List[bo.Stats]
    s: int
    M: int
    precision: int
    timings_ms: dict = field(default_factory=dict)


def fields(op, U, C, T, q, s: int, M: int, precision: int, stream=None, fused: bool = False):
    """The pairs of a solved basis: T = U C and q = A T.  ``fused`` takes the
    single pass of blockoa_combine_apply (mixed form only; T and q written
    once, T never read back), otherwise the two calls, which are the faster
    of the two on the 128 x 128 x 8, s = 32 chip."""
    if fused and precision == bo.MIXED:
        bo.combine_apply(op, U, C, T, q, s, M, stream=stream)
    else:
        bo.combine(op, U, C, T, s, M, precision, stream=stream)
        bo.apply_operator(op, T, q, M, precision, stream=stream)


def host_inputs(w):
    """Concatenated host arrays (float64) of a workload's density maps and C."""
    dens = np.concatenate([np.ascontiguousarray(d, np.float64).ravel() for d in w.density])
    C = np.concatenate([np.ascontiguousarray(c, np.float64).ravel() for c in w.coeffs])
    return dens, C


def upload(w, device="cuda", pin=False) -> DeviceInputs:
    import torch
    dens, C = host_inputs(w)
    return DeviceInputs(torch.from_numpy(dens).to(device), torch.from_numpy(C).to(device))


def field_dtype(precision: int):
    import torch
    return torch.float64 if precision == bo.FP64 else torch.float32


def run(w, precision: int, inputs: Optional[DeviceInputs] = None, rtol: Optional[float] = None,
        maxiter: int = 200000, stream=None, outputs=None, **solve_kw) -> Result:
    """One pass of the hot path on workload ``w``.

    ``outputs`` may hold preallocated (B, U, T, q) tensors to reuse.
    """
    import torch
    dev = torch.device("cuda")
    if inputs is None:
        inputs = upload(w)
    op = bo.assemble(w.chips, stream=stream)
    s, M = w.s, w.M
    if outputs is None:
        B = torch.empty(op.n_total * s, dtype=torch.float64, device=dev)
        U = torch.empty_like(B)
        T = torch.empty(op.n_total * M, dtype=field_dtype(precision), device=dev)
        q = torch.empty_like(T)
    else:
        B, U, T, q = outputs
    bo.build_rhs(op, inputs.density, B, s, stream=stream)
    stats = bo.block_solve(op, B, U, s, rtol=w.rtol if rtol is None else rtol, maxiter=maxiter,
                           precision=precision, stream=stream, **solve_kw)
    fields(op, U, inputs.C, T, q, s, M, precision, stream=stream)
    return Result(op, B, U, T, q, stats, s, M, precision)


def chip_fields(res: Result, chip: int, which: str):
    """View [M][n_c] of chip ``chip``'s fields in ``res.T`` or ``res.q``."""
    sz = res.op.sizes[chip]
    buf = getattr(res, which)
    return buf[sz["off"] * res.M:(sz["off"] + sz["n"]) * res.M].view(res.M, sz["n"])


def chip_block(res: Result, chip: int, which: str = "U"):
    """View [n_c][s] of chip ``chip``'s rows in a block vector."""
    sz = res.op.sizes[chip]
    buf = getattr(res, which)
    return buf[sz["off"] * res.s:(sz["off"] + sz["n"]) * res.s].view(sz["n"], res.s)


class PairStreamer:
    """The hot path over a stream of same-shaped inputs, with each step's
    pairs (T, q) copied to host memory while the next step computes.

    Each ``step`` copies its inputs from (pinned) host arrays, re-discretises
    the operator in place, solves, combines and applies into one of two
    device result buffers, then queues the device-to-host copy of that
    buffer on a copy stream; the step after next waits for that copy before
    reusing the buffer.  Compute runs on a stream of its own: work on the
    legacy default stream would wait for every pending copy.  Each step's
    copies are dealt in chunks over ``copy_streams`` streams so that several
    copy engines share the device-to-host traffic.  Host outputs must be
    pinned for the copies to overlap.  ``finish`` makes the caller's stream
    wait for all queued work.
    """

    def __init__(self, op: bo.Operator, s: int, M: int, precision: int, chunk_bytes: int = 64 << 20,
                 copy_streams: int = 4):
        import torch
        n = op.n_total
        dev = torch.device("cuda")
        self.op, self.s, self.M, self.precision = op, s, M, precision
        self.B = torch.empty(n * s, dtype=torch.float64, device=dev)
        self.U = torch.empty_like(self.B)
        fdt = field_dtype(precision)
        self.T = [torch.empty(n * M, dtype=fdt, device=dev) for _ in range(2)]
        self.q = [torch.empty(n * M, dtype=fdt, device=dev) for _ in range(2)]
        self.compute_stream = torch.cuda.Stream(device=dev)
        self.copy_streams = [torch.cuda.Stream(device=dev) for _ in range(max(1, copy_streams))]
        self.ready = [torch.cuda.Event() for _ in range(2)]
        self.freed = [[torch.cuda.Event() for _ in self.copy_streams] for _ in range(2)]
        self.chunk = max(1, chunk_bytes // self.T[0].element_size())
        self.k = 0

    def step(self, chips, dens_h, C_h, dens_d, C_d, T_h, q_h, **solve_kw):
        import torch
        b = self.k % 2
        cs = self.compute_stream
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            if self.k >= 2:
                for ev in self.freed[b]:
                    cs.wait_event(ev)
            dens_d.copy_(dens_h, non_blocking=True)
            C_d.copy_(C_h, non_blocking=True)
            bo.reassemble(self.op, chips)
            bo.build_rhs(self.op, dens_d, self.B, self.s)
            stats = bo.block_solve(self.op, self.B, self.U, self.s, precision=self.precision, **solve_kw)
            fields(self.op, self.U, C_d, self.T[b], self.q[b], self.s, self.M, self.precision)
            self.ready[b].record(cs)
        ncs = len(self.copy_streams)
        for c in self.copy_streams:
            c.wait_event(self.ready[b])
        q = 0
        for src, dst in ((self.T[b], T_h), (self.q[b], q_h)):
            for i in range(0, src.numel(), self.chunk):
                with torch.cuda.stream(self.copy_streams[q % ncs]):
                    dst[i:i + self.chunk].copy_(src[i:i + self.chunk], non_blocking=True)
                q += 1
        for c, ev in zip(self.copy_streams, self.freed[b]):
            ev.record(c)
        self.k += 1
        return stats

    def finish(self):
        import torch
        cur = torch.cuda.current_stream()
        cur.wait_stream(self.compute_stream)
        for c in self.copy_streams:
            cur.wait_stream(c)
