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
    bo.combine(op, U, inputs.C, T, s, M, precision, stream=stream)
    bo.apply_operator(op, T, q, M, precision, stream=stream)
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
