"""ctypes binding of the warm-start Fourier neural operator in libblockoa.so
(argument marshalling only; every step runs in the library's kernels).

The network, its parameter layout and the meaning of each call are
documented in include/blockoa.h (section "Learned warm start").
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import numpy as np

from . import blockoa as bo

FNO_EXPORTED = (
    "blockoa_fno_param_count", "blockoa_fno_create", "blockoa_fno_forward", "blockoa_fno_mse",
    "blockoa_fno_backward", "blockoa_fno_zero_grad", "blockoa_fno_adam_step",
    "blockoa_fno_get_params", "blockoa_fno_get_grads", "blockoa_fno_destroy", "blockoa_fno_basis",
)


class FnoShapeC(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("c_in", ct.c_int),
                ("width", ct.c_int), ("hidden", ct.c_int), ("layers", ct.c_int),
                ("mx", ct.c_int), ("my", ct.c_int), ("mz", ct.c_int), ("max_batch", ct.c_int)]


@dataclass
class FnoShape:
    nx: int
    ny: int
    nz: int
    c_in: int = 5
    width: int = 32
    hidden: int = 128
    layers: int = 4
    mx: int = 12
    my: int = 12
    mz: int = 4
    max_batch: int = 8

    def c(self) -> FnoShapeC:
        return FnoShapeC(self.nx, self.ny, self.nz, self.c_in, self.width, self.hidden, self.layers,
                         self.mx, self.my, self.mz, self.max_batch)


_READY = False


def _lib():
    global _READY
    lib = bo._lib()
    if not _READY:
        vp, i, f = ct.c_void_p, ct.c_int, ct.c_float
        lib.blockoa_fno_param_count.argtypes = [ct.POINTER(FnoShapeC), ct.POINTER(ct.c_int64)]
        lib.blockoa_fno_create.argtypes = [ct.POINTER(FnoShapeC), vp, ct.POINTER(vp)]
        lib.blockoa_fno_forward.argtypes = [vp, vp, vp, i, i, vp]
        lib.blockoa_fno_mse.argtypes = [vp, vp, vp, i, vp, vp, vp]
        lib.blockoa_fno_backward.argtypes = [vp, vp, i, vp]
        lib.blockoa_fno_zero_grad.argtypes = [vp, vp]
        lib.blockoa_fno_adam_step.argtypes = [vp, f, f, f, f, i, vp]
        lib.blockoa_fno_get_params.argtypes = [vp, vp]
        lib.blockoa_fno_get_grads.argtypes = [vp, vp]
        lib.blockoa_fno_basis.argtypes = [vp, vp, vp, i, vp, vp]
        lib.blockoa_fno_destroy.argtypes = [vp]
        lib.blockoa_fno_destroy.restype = None
        for name in FNO_EXPORTED:
            if name != "blockoa_fno_destroy":
                getattr(lib, name).restype = ct.c_int
        _READY = True
    return lib


def param_count(shape: FnoShape) -> int:
    n = ct.c_int64()
    sc = shape.c()
    bo._check(_lib().blockoa_fno_param_count(ct.byref(sc), ct.byref(n)), "fno_param_count")
    return int(n.value)


class Fno:
    """A network on the current device (see include/blockoa.h)."""

    def __init__(self, shape: FnoShape, params: np.ndarray):
        self.shape = shape
        self.n_params = param_count(shape)
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        h = ct.c_void_p()
        sc = shape.c()
        bo._check(_lib().blockoa_fno_create(ct.byref(sc), p.ctypes.data_as(ct.c_void_p), ct.byref(h)),
                  "fno_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            _lib().blockoa_fno_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cells(self, batch: int) -> int:
        return batch * self.shape.nx * self.shape.ny * self.shape.nz

    def forward(self, x, y, batch: int, keep: bool = False, stream=None):
        import torch
        n = self._cells(batch)
        bo._check(_lib().blockoa_fno_forward(self.handle, bo._ptr(x, torch.float32, "x", n * self.shape.c_in),
                                             bo._ptr(y, torch.float32, "y", n), batch, int(keep),
                                             bo._stream(stream)), "fno_forward")

    def mse(self, y, target, batch: int, dy, loss, stream=None):
        import torch
        n = self._cells(batch)
        bo._check(_lib().blockoa_fno_mse(self.handle, bo._ptr(y, torch.float32, "y", n),
                                         bo._ptr(target, torch.float32, "target", n), batch,
                                         bo._ptr(dy, torch.float32, "dy", n), bo._ptr(loss, torch.float32, "loss", 1),
                                         bo._stream(stream)), "fno_mse")

    def backward(self, dy, batch: int, stream=None):
        import torch
        bo._check(_lib().blockoa_fno_backward(self.handle, bo._ptr(dy, torch.float32, "dy", self._cells(batch)), batch,
                                              bo._stream(stream)), "fno_backward")

    def zero_grad(self, stream=None):
        bo._check(_lib().blockoa_fno_zero_grad(self.handle, bo._stream(stream)), "fno_zero_grad")

    def adam_step(self, lr: float, t: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  stream=None):
        bo._check(_lib().blockoa_fno_adam_step(self.handle, lr, beta1, beta2, eps, t, bo._stream(stream)),
                  "fno_adam_step")

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        bo._check(_lib().blockoa_fno_get_params(self.handle, out.ctypes.data_as(ct.c_void_p)), "fno_get_params")
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        bo._check(_lib().blockoa_fno_get_grads(self.handle, out.ctypes.data_as(ct.c_void_p)), "fno_get_grads")
        return out


def basis(op: bo.Operator, y, scale, s: int, X, stream=None):
    """blockoa_fno_basis: network outputs y [chip][s][n_c] (float32) times
    scale [chip * s] (float64) into the block vector X [n_total][s]."""
    import torch
    bo._check(_lib().blockoa_fno_basis(op.handle, bo._ptr(y, torch.float32, "y", op.n_total * s),
                                       bo._ptr(scale, torch.float64, "scale", op.n_chips * s), s,
                                       bo._ptr(X, torch.float64, "X", op.n_total * s), bo._stream(stream)),
              "fno_basis")


def pack(params: dict, layers: int) -> np.ndarray:
    """Flat parameter array in the library's order from named arrays
    P, bP, Wl, bl, Rr, Ri, Q1, c1, Q2, c2 (shapes as in the header)."""
    order = ("P", "bP", "Wl", "bl", "Rr", "Ri", "Q1", "c1", "Q2", "c2")
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k in order]).astype(np.float32)


def unpack(flat: np.ndarray, shapes: dict) -> dict:
    """Inverse of pack for the named shapes (an ordered mapping)."""
    order = ("P", "bP", "Wl", "bl", "Rr", "Ri", "Q1", "c1", "Q2", "c2")
    out, o = {}, 0
    for k in order:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(flat[o:o + n]).reshape(shapes[k])
        o += n
    return out
