"""ctypes binding of libblockoa.so (the C ABI declared in include/blockoa.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Device arrays are torch CUDA tensors (PyTorch supplies device
memory and streams); their raw pointers cross the ABI.  If the library is
missing this module raises on first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblockoa.so")

OK = 0
ERR_INVALID = 1
ERR_CUDA = 2
ERR_BREAKDOWN = 3
ERR_NOT_CONVERGED = 4
ERR_TIMEOUT = 5
ERR_OOM = 6
FP64 = 0
MIXED = 1
PRECOND_NONE = 0
PRECOND_JACOBI = 1
PRECOND_ZLINE = 2
PRECOND_ZLINE2 = 3
SMALL_AUTO = 0
SMALL_FP64_CHOLESKY = 1

EXPORTED = (
    "blockoa_assemble", "blockoa_reassemble", "blockoa_operator_size", "blockoa_operator_total", "blockoa_build_rhs",
    "blockoa_build_rhs_volume",
    "blockoa_block_solve", "blockoa_combine", "blockoa_combine_ex", "blockoa_apply_basis", "blockoa_apply_operator", "blockoa_pair_check",
    "blockoa_export_conductances", "blockoa_destroy", "blockoa_status_string",
    "blockoa_last_error", "blockoa_kernel_times", "blockoa_reset_kernel_times",
    "blockoa_launch_count", "blockoa_autotune", "blockoa_set_tuning", "blockoa_get_tuning",
    "blockoa_pair_check_static", "blockoa_residual_ratio", "blockoa_inject_chip_status",
    "blockoa_combine_apply",
)

# Largest n_chips * M accepted by blockoa_pair_check_static (its fixed device array).
STATIC_PAIR_MAX = 32768


class ChipDesc(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("n_layers", ct.c_int),
                ("layer_nz", ct.POINTER(ct.c_int)), ("layer_dz", ct.POINTER(ct.c_double)),
                ("layer_k", ct.POINTER(ct.c_double)), ("k_cell", ct.POINTER(ct.c_double)),
                ("dx", ct.c_double), ("dy", ct.c_double), ("h_top", ct.c_double),
                ("h_bottom", ct.c_double), ("h_side", ct.c_double), ("t_ambient", ct.c_double)]


class Tuning(ct.Structure):
    _fields_ = [("tiles_per_unit", ct.c_int), ("ztiles_per_unit", ct.c_int), ("ms_per_iter", ct.c_double)]


class CombineOpts(ct.Structure):
    _fields_ = [("noise_seed", ct.c_uint64), ("noise_amp", ct.c_double), ("noise_kind", ct.c_int),
                ("normalize", ct.c_int), ("normalize_min", ct.c_double)]


NOISE_UNIFORM = 0
NOISE_GAUSSIAN = 1


class SolveOpts(ct.Structure):
    _fields_ = [("rtol", ct.c_double), ("maxiter", ct.c_int), ("precision", ct.c_int),
                ("inner_rtol", ct.c_double), ("max_refine", ct.c_int),
                ("deflate_tol", ct.c_double), ("x0", ct.c_void_p), ("check_every", ct.c_int),
                ("precond", ct.c_int),
                ("small_solve", ct.c_int), ("independent", ct.c_int), ("deterministic", ct.c_int)]


class SolveStats(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iters", ct.c_int), ("refine_steps", ct.c_int),
                ("deflated_cols", ct.c_int), ("relres_max", ct.c_double)]


class BlockoaError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = _lib()
        msg = lib.blockoa_status_string(code).decode()
        last = lib.blockoa_last_error().decode()
        super().__init__(f"{what}: {msg} ({code}){' -- ' + last if last else ''}")
        self.code = code


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libblockoa.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ct.CDLL(LIB_PATH)
        vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
        lib.blockoa_assemble.argtypes = [ct.POINTER(ChipDesc), i, vp, ct.POINTER(vp)]
        lib.blockoa_reassemble.argtypes = [vp, ct.POINTER(ChipDesc), i, vp]
        lib.blockoa_operator_size.argtypes = [vp, i, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                              ct.POINTER(i), ct.POINTER(i), ct.POINTER(i)]
        lib.blockoa_operator_total.argtypes = [vp, ct.POINTER(ct.c_int64), ct.POINTER(i)]
        lib.blockoa_build_rhs.argtypes = [vp, vp, vp, i, vp]
        lib.blockoa_build_rhs_volume.argtypes = [vp, vp, vp, i, vp]
        lib.blockoa_block_solve.argtypes = [vp, vp, vp, i, ct.POINTER(SolveOpts),
                                            ct.POINTER(SolveStats), vp]
        lib.blockoa_combine.argtypes = [vp, vp, vp, vp, i, i, i, vp]
        lib.blockoa_apply_operator.argtypes = [vp, vp, vp, i, i, vp]
        lib.blockoa_apply_basis.argtypes = [vp, vp, vp, i, vp]
        lib.blockoa_combine_ex.argtypes = [vp, vp, vp, vp, i, i, i, ct.POINTER(CombineOpts), vp]
        lib.blockoa_autotune.argtypes = [vp, i, i, i, ct.POINTER(Tuning), vp]
        lib.blockoa_set_tuning.argtypes = [vp, ct.POINTER(Tuning)]
        lib.blockoa_get_tuning.argtypes = [vp, ct.POINTER(Tuning)]
        lib.blockoa_pair_check.argtypes = [vp, vp, vp, i, i, vp, vp]
        lib.blockoa_pair_check_static.argtypes = [vp, vp, vp, i, i, vp, vp]
        lib.blockoa_residual_ratio.argtypes = [vp, vp, vp, i, vp, vp]
        lib.blockoa_inject_chip_status.argtypes = [vp, i, i, i]
        lib.blockoa_combine_apply.argtypes = [vp, vp, vp, vp, vp, i, i, vp]
        lib.blockoa_export_conductances.argtypes = [vp, i, vp, vp, vp, vp]
        lib.blockoa_destroy.argtypes = [vp]
        lib.blockoa_destroy.restype = None
        lib.blockoa_status_string.argtypes = [i]
        lib.blockoa_status_string.restype = ct.c_char_p
        lib.blockoa_last_error.argtypes = []
        lib.blockoa_last_error.restype = ct.c_char_p
        lib.blockoa_kernel_times.argtypes = [vp, i, ct.POINTER(ct.c_double),
                                             ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong),
                                             ct.POINTER(ct.c_char_p)]
        lib.blockoa_reset_kernel_times.argtypes = [vp]
        lib.blockoa_launch_count.argtypes = []
        lib.blockoa_launch_count.restype = ct.c_longlong
        for name in EXPORTED:
            if name not in ("blockoa_destroy", "blockoa_status_string", "blockoa_last_error",
                            "blockoa_launch_count"):
                getattr(lib, name).restype = ct.c_int
        _LIB = lib
    return _LIB


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _lib()


def _check(code: int, what: str, ok=(OK,)):
    if code not in ok:
        raise BlockoaError(code, what)
    return code


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t, dtype=None, name="tensor", need: int = 0):
    """Raw device pointer of a contiguous CUDA tensor (None passes NULL).

    ``need`` is the number of elements the call reads or writes through the
    pointer: a smaller tensor is refused here, before any launch, since the
    library sees only the pointer."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {need}")
    return t.data_ptr()


# ---------------------------------------------------------------- operator
class Operator:
    """Owns a blockoa_operator handle (freed by close() or garbage collection)."""

    def __init__(self, handle: int, chips: Sequence):
        self.handle = handle
        self.chips = list(chips)
        lib = _lib()
        n_total = ct.c_int64()
        n_chips = ct.c_int()
        _check(lib.blockoa_operator_total(handle, ct.byref(n_total), ct.byref(n_chips)), "operator_total")
        self.n_total = int(n_total.value)
        self.n_chips = int(n_chips.value)
        self.sizes = [operator_size(self, c) for c in range(self.n_chips)]

    def close(self):
        if self.handle:
            _lib().blockoa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(chip, keep: list) -> ChipDesc:
    lnz = np.ascontiguousarray(chip.layer_nz, np.int32)
    ldz = np.ascontiguousarray(chip.layer_dz, np.float64)
    lk = np.ascontiguousarray(chip.layer_k, np.float64)
    kc = None if chip.k_cell is None else np.ascontiguousarray(chip.k_cell, np.float64)
    keep.extend([lnz, ldz, lk, kc])
    d = ChipDesc()
    d.nx, d.ny, d.n_layers = int(chip.nx), int(chip.ny), int(len(lnz))
    d.layer_nz = lnz.ctypes.data_as(ct.POINTER(ct.c_int))
    d.layer_dz = ldz.ctypes.data_as(ct.POINTER(ct.c_double))
    d.layer_k = lk.ctypes.data_as(ct.POINTER(ct.c_double))
    d.k_cell = kc.ctypes.data_as(ct.POINTER(ct.c_double)) if kc is not None else None
    d.dx, d.dy = float(chip.dx), float(chip.dy)
    d.h_top, d.h_bottom, d.h_side = float(chip.h_top), float(chip.h_bottom), float(chip.h_side)
    d.t_ambient = float(chip.t_ambient)
    return d


def assemble(chips: Sequence, stream=None) -> Operator:
    """blockoa_assemble on a list of synth.Chip-like objects."""
    keep: list = []
    arr = (ChipDesc * len(chips))(*[_desc(c, keep) for c in chips])
    h = ct.c_void_p()
    _check(_lib().blockoa_assemble(arr, len(chips), _stream(stream), ct.byref(h)), "assemble")
    return Operator(h.value, chips)


def reassemble(op: Operator, chips: Sequence, stream=None) -> Operator:
    """blockoa_reassemble: new chips of the same geometry into `op` (kept
    arrays, solve workspace and graph); returns op."""
    keep: list = []
    arr = (ChipDesc * len(chips))(*[_desc(c, keep) for c in chips])
    _check(_lib().blockoa_reassemble(op.handle, arr, len(chips), _stream(stream)), "reassemble")
    op.chips = list(chips)
    return op


def autotune(op: Operator, s: int, precision: int = MIXED, precond: int = PRECOND_NONE, stream=None) -> dict:
    """blockoa_autotune: time candidate unit sizes, keep the fastest in `op`."""
    t = Tuning()
    _check(_lib().blockoa_autotune(op.handle, s, precision, precond, ct.byref(t), _stream(stream)), "autotune")
    return {"tiles_per_unit": t.tiles_per_unit, "ztiles_per_unit": t.ztiles_per_unit, "ms_per_iter": t.ms_per_iter}


def set_tuning(op: Operator, tiles_per_unit: int = 0, ztiles_per_unit: int = 0):
    t = Tuning(tiles_per_unit=tiles_per_unit, ztiles_per_unit=ztiles_per_unit, ms_per_iter=0.0)
    _check(_lib().blockoa_set_tuning(op.handle, ct.byref(t)), "set_tuning")


def get_tuning(op: Operator) -> dict:
    t = Tuning()
    _check(_lib().blockoa_get_tuning(op.handle, ct.byref(t)), "get_tuning")
    return {"tiles_per_unit": t.tiles_per_unit, "ztiles_per_unit": t.ztiles_per_unit}


def operator_size(op: Operator, chip: int):
    n, off = ct.c_int64(), ct.c_int64()
    nx, ny, nz = ct.c_int(), ct.c_int(), ct.c_int()
    _check(_lib().blockoa_operator_size(op.handle, chip, ct.byref(n), ct.byref(off), ct.byref(nx),
                                        ct.byref(ny), ct.byref(nz)), "operator_size")
    return {"n": n.value, "off": off.value, "nx": nx.value, "ny": ny.value, "nz": nz.value}


def build_rhs(op: Operator, density, B, s: int, stream=None):
    import torch
    top = sum(z["nx"] * z["ny"] for z in op.sizes)
    _check(_lib().blockoa_build_rhs(op.handle, _ptr(density, torch.float64, "density", s * top),
                                    _ptr(B, torch.float64, "B", op.n_total * s), s, _stream(stream)), "build_rhs")


def build_rhs_volume(op: Operator, qv, B, s: int, stream=None):
    """B[a][j] = qv[j][a] * dx dy dz(a): volumetric sources (W/m^3) of every cell."""
    import torch
    _check(_lib().blockoa_build_rhs_volume(op.handle, _ptr(qv, torch.float64, "qv", s * op.n_total),
                                           _ptr(B, torch.float64, "B", op.n_total * s), s, _stream(stream)),
           "build_rhs_volume")


@dataclass
class Stats:
    status: int
    iters: int
    refine_steps: int
    deflated_cols: int
    relres_max: float


def block_solve(op: Operator, B, X, s: int, rtol: float = 1e-12, maxiter: int = 100000,
                precision: int = FP64, inner_rtol: float = 0.0, max_refine: int = 0,
                deflate_tol: float = 0.0, x0=None, check_every: int = 0, precond: int = PRECOND_NONE,
                small_solve: int = SMALL_AUTO, independent: bool = False, deterministic: bool = False,
                stream=None, raise_on_error: bool = True) -> List[Stats]:
    import torch
    o = SolveOpts(rtol=rtol, maxiter=maxiter, precision=precision, inner_rtol=inner_rtol,
                  max_refine=max_refine, deflate_tol=deflate_tol,
                  x0=_ptr(x0, torch.float64, "x0", op.n_total * s), check_every=check_every, precond=precond,
                  small_solve=small_solve, independent=int(bool(independent)),
                  deterministic=int(deterministic))
    st = (SolveStats * op.n_chips)()
    code = _lib().blockoa_block_solve(op.handle, _ptr(B, torch.float64, "B", op.n_total * s),
                                      _ptr(X, torch.float64, "X", op.n_total * s), s, ct.byref(o), st,
                                      _stream(stream))
    stats = [Stats(x.status, x.iters, x.refine_steps, x.deflated_cols, x.relres_max) for x in st]
    if raise_on_error:
        _check(code, "block_solve")
    return stats


def combine(op: Operator, U, C, T, s: int, M: int, dtype: int, stream=None, noise_seed: int = 0,
            noise_amp: float = 0.0, noise_kind: int = NOISE_UNIFORM, normalize: bool = False,
            normalize_min: float = 0.0):
    """T = U C; with noise_amp > 0, plus the epsilon term of Eq. 5
    (blockoa_combine_ex: uniform in [-noise_amp, noise_amp) K, or Gaussian of
    standard deviation noise_amp, from Philox); with normalize, Eq. 5's
    weights C_jm / sum_i C_im."""
    import torch
    tdt = torch.float64 if dtype == FP64 else torch.float32
    pU = _ptr(U, torch.float64, "U", op.n_total * s)
    pC = _ptr(C, torch.float64, "C", op.n_chips * s * M)
    pT = _ptr(T, tdt, "T", op.n_total * M)
    if noise_amp == 0.0 and not normalize:
        _check(_lib().blockoa_combine(op.handle, pU, pC, pT, s, M, dtype, _stream(stream)), "combine")
        return
    o = CombineOpts(noise_seed=int(noise_seed) & ((1 << 64) - 1), noise_amp=float(noise_amp),
                    noise_kind=int(noise_kind), normalize=int(bool(normalize)),
                    normalize_min=float(normalize_min))
    _check(_lib().blockoa_combine_ex(op.handle, pU, pC, pT, s, M, dtype, ct.byref(o), _stream(stream)),
           "combine_ex")


def combine_apply(op: Operator, U, C, T, q, s: int, M: int, stream=None):
    """T = U C and q = A T in one pass (blockoa_combine_apply; float32 fields)."""
    import torch
    _check(_lib().blockoa_combine_apply(op.handle, _ptr(U, torch.float64, "U", op.n_total * s),
                                        _ptr(C, torch.float64, "C", op.n_chips * s * M),
                                        _ptr(T, torch.float32, "T", op.n_total * M),
                                        _ptr(q, torch.float32, "q", op.n_total * M), s, M, _stream(stream)),
           "combine_apply")


def apply_operator(op: Operator, T, q, M: int, dtype: int, stream=None):
    import torch
    tdt = torch.float64 if dtype == FP64 else torch.float32
    _check(_lib().blockoa_apply_operator(op.handle, _ptr(T, tdt, "T", op.n_total * M),
                                         _ptr(q, tdt, "q", op.n_total * M), M, dtype,
                                         _stream(stream)), "apply_operator")


def apply_basis(op: Operator, U, AU, s: int, stream=None):
    """AU = A U on a float64 [n][s] block (blockoa_apply_basis)."""
    import torch
    _check(_lib().blockoa_apply_basis(op.handle, _ptr(U, torch.float64, "U", op.n_total * s),
                                      _ptr(AU, torch.float64, "AU", op.n_total * s), s,
                                      _stream(stream)), "apply_basis")


def pair_check(op: Operator, T, q, M: int, dtype: int, e_pair, stream=None):
    import torch
    tdt = torch.float64 if dtype == FP64 else torch.float32
    _check(_lib().blockoa_pair_check(op.handle, _ptr(T, tdt, "T", op.n_total * M),
                                     _ptr(q, tdt, "q", op.n_total * M), M, dtype,
                                     _ptr(e_pair, torch.float64, "e_pair", op.n_chips * M), _stream(stream)),
           "pair_check")


def inject_chip_status(op: Operator, chip: int, status: int, after_polls: int = 1):
    """Test support: the next solve finds chip `chip` with `status` (inactive)
    before poll `after_polls` (blockoa_inject_chip_status)."""
    _check(_lib().blockoa_inject_chip_status(op.handle, chip, status, after_polls), "inject_chip_status")


def residual_ratio(op: Operator, B, X, s: int, ratio, stream=None):
    """ratio[c * s + j] = ||B_j - A X_j|| / ||B_j|| per chip and column
    (blockoa_residual_ratio, float64)."""
    import torch
    _check(_lib().blockoa_residual_ratio(op.handle, _ptr(B, torch.float64, "B", op.n_total * s),
                                         _ptr(X, torch.float64, "X", op.n_total * s), s,
                                         _ptr(ratio, torch.float64, "ratio", op.n_chips * s), _stream(stream)),
           "residual_ratio")


def pair_check_static(op: Operator, T, q, M: int, dtype: int, e_pair, stream=None):
    """blockoa_pair_check without device allocation (its accumulators live in
    a fixed library array; n_chips * M <= STATIC_PAIR_MAX)."""
    import torch
    tdt = torch.float64 if dtype == FP64 else torch.float32
    _check(_lib().blockoa_pair_check_static(op.handle, _ptr(T, tdt, "T", op.n_total * M),
                                            _ptr(q, tdt, "q", op.n_total * M), M, dtype,
                                            _ptr(e_pair, torch.float64, "e_pair", op.n_chips * M),
                                            _stream(stream)),
           "pair_check_static")


def export_conductances(op: Operator, chip: int):
    sz = op.sizes[chip]
    nx, ny, nz = sz["nx"], sz["ny"], sz["nz"]
    gx = np.zeros((nz, ny, max(nx - 1, 0)))
    gy = np.zeros((nz, max(ny - 1, 0), nx))
    gz = np.zeros((max(nz - 1, 0), ny, nx))
    gb = np.zeros((nz, ny, nx))
    _check(_lib().blockoa_export_conductances(op.handle, chip, gx.ctypes.data, gy.ctypes.data,
                                              gz.ctypes.data, gb.ctypes.data), "export_conductances")
    return {"gx": gx, "gy": gy, "gz": gz, "gb": gb}


def status_string(code: int) -> str:
    return _lib().blockoa_status_string(code).decode()


def kernel_times(op: Operator) -> dict:
    """Live per-kernel timing: {name: (timed_ms, timed_launches, launches)}."""
    lib = _lib()
    n = lib.blockoa_kernel_times(op.handle, 0, None, None, None, None)
    ms = (ct.c_double * n)()
    cnt = (ct.c_longlong * n)()
    allc = (ct.c_longlong * n)()
    names = (ct.c_char_p * n)()
    lib.blockoa_kernel_times(op.handle, n, ms, cnt, allc, names)
    return {names[k].decode(): (ms[k], cnt[k], allc[k]) for k in range(n)}


def reset_kernel_times(op: Operator):
    _check(_lib().blockoa_reset_kernel_times(op.handle), "reset_kernel_times")


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib().blockoa_launch_count())
