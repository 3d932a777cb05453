"""Float64 reference of the Fourier neural operator used as a warm start.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

The network (a 3-D Fourier neural operator in the sense of the FNO
literature, with the sizes of the warm-start configuration: 4 Fourier
layers, width 32, 12 x 12 x 4 modes) maps per-cell input channels on an
(nz, ny, nx) grid to one output channel:

    v0 = P x + bP                                  (pointwise, c_in -> W)
    u_l = K_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(u_l)  (gelu skipped on the last layer)
    h = gelu(Q1 v_L + c1),  y = Q2 h + c2          (pointwise, W -> H -> 1)

with the spectral convolution over the truncated mode set
kx = a - MX/2 (a < MX), ky = b - MY/2 (b < MY), kz = c (c < MZ):

    Xh[c,b,a,i] = sum_{z,y,x} v[z,y,x,i] exp(-2 pi i (kx x/nx + ky y/ny + kz z/nz))
    Yh[c,b,a,o] = sum_i Xh[c,b,a,i] R[c,b,a,i,o]                    (complex R)
    K(v)[z,y,x,o] = 1/(nx ny nz) sum_{c,b,a} w_c Re(Yh[c,b,a,o] exp(+2 pi i (...)))

w_0 = 1, w_c = 2 for c > 0 (one half of the z spectrum).  gelu is the exact
x Phi(x).  The forward pass keeps what the backward pass needs; backward
is derived by hand (each step's adjoint) and checked by central finite
differences in tests/test_fno_oracle.py.  Weights enter as given; the GPU
uses bfloat16-rounded copies, which the tests pass here as well.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import erf, sqrt, pi
from typing import Dict

import numpy as np


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


def param_shapes(sh: FnoShape) -> Dict[str, tuple]:
    W, L, M = sh.width, sh.layers, sh.mx * sh.my * sh.mz
    return {
        "P": (W, sh.c_in), "bP": (W,),
        "Wl": (L, W, W), "bl": (L, W),
        "Rr": (L, M, W, W), "Ri": (L, M, W, W),   # R[l, mode, i, o]
        "Q1": (sh.hidden, W), "c1": (sh.hidden,),
        "Q2": (1, sh.hidden), "c2": (1,),
    }


def modes(sh: FnoShape):
    kx = np.arange(sh.mx) - sh.mx // 2
    ky = np.arange(sh.my) - sh.my // 2
    kz = np.arange(sh.mz)
    return kx, ky, kz


def dft_mats(sh: FnoShape):
    """E_x[a, x] = exp(-2 pi i kx_a x / nx), likewise for y and z."""
    kx, ky, kz = modes(sh)
    ex = np.exp(-2j * pi * np.outer(kx, np.arange(sh.nx)) / sh.nx)
    ey = np.exp(-2j * pi * np.outer(ky, np.arange(sh.ny)) / sh.ny)
    ez = np.exp(-2j * pi * np.outer(kz, np.arange(sh.nz)) / sh.nz)
    return ex, ey, ez


def forward_dft(v, sh: FnoShape):
    """v [B, nz, ny, nx, C] real -> Xh [B, mz, my, mx, C] complex."""
    ex, ey, ez = dft_mats(sh)
    return np.einsum("nzyxi,ax,by,cz->ncbai", v, ex, ey, ez)


def inverse_dft(Yh, sh: FnoShape, weighted: bool = True, scale: float = None):
    """Yh [B, mz, my, mx, C] -> real [B, nz, ny, nx, C]:
    scale * sum_m w_c Re(Yh_m exp(+i theta)); weighted=False uses w = 1."""
    ex, ey, ez = dft_mats(sh)
    w = np.ones(sh.mz)
    if weighted:
        w[1:] = 2.0
    if scale is None:
        scale = 1.0 / (sh.nx * sh.ny * sh.nz)
    Z = np.einsum("ncbao,c,ax,by,cz->nzyxo", Yh, w, np.conj(ex), np.conj(ey), np.conj(ez))
    return scale * Z.real


def spectral(v, Rr, Ri, sh: FnoShape):
    Xh = forward_dft(v, sh)                       # [B, mz, my, mx, W]
    B = v.shape[0]
    Xf = Xh.reshape(B, -1, sh.width)              # [B, M, W]
    R = Rr + 1j * Ri                              # [M, W, W]
    Yf = np.einsum("nmi,mio->nmo", Xf, R)
    Yh = Yf.reshape(Xh.shape)
    return inverse_dft(Yh, sh), Xh


def gelu(x):
    return x * 0.5 * (1.0 + _erf(x / sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / sqrt(2.0))) + x * np.exp(-0.5 * x * x) / sqrt(2.0 * pi)


_erf = np.vectorize(erf, otypes=[float])


def init_params(sh: FnoShape, seed: int) -> Dict[str, np.ndarray]:
    """Seeded initialisation (uniform fan-in scaling; spectral weights as in
    the FNO literature, scale 1 / (W W))."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(sh).items():
        if name in ("Rr", "Ri"):
            p[name] = rng.uniform(0.0, 1.0, shp) / (sh.width * sh.width)
        elif name in ("bP", "bl", "c1", "c2"):
            p[name] = np.zeros(shp)
        else:
            fan_in = shp[-1]
            lim = 1.0 / sqrt(fan_in)
            p[name] = rng.uniform(-lim, lim, shp)
    return p


def forward(params, x, sh: FnoShape):
    """x [B, nz, ny, nx, c_in] -> y [B, nz, ny, nx] and the saved tensors."""
    cache = {"x": x}
    v = x @ params["P"].T + params["bP"]
    cache["v"] = [v]
    cache["u"], cache["Xh"] = [], []
    for l in range(sh.layers):
        k, Xh = spectral(v, params["Rr"][l], params["Ri"][l], sh)
        u = k + v @ params["Wl"][l].T + params["bl"][l]
        cache["u"].append(u)
        cache["Xh"].append(Xh)
        v = gelu(u) if l < sh.layers - 1 else u
        cache["v"].append(v)
    a1 = v @ params["Q1"].T + params["c1"]
    h = gelu(a1)
    y = (h @ params["Q2"].T + params["c2"])[..., 0]
    cache["a1"], cache["h"] = a1, h
    return y, cache


def loss(y, target):
    """Mean squared error over all samples and cells."""
    return float(np.mean((y - target) ** 2))


def _outer_sum(a, b):
    """sum over all leading indices of a[..., o] b[..., i] -> [o, i]."""
    return a.reshape(-1, a.shape[-1]).T @ b.reshape(-1, b.shape[-1])


def _lead_sum(a):
    return a.reshape(-1, a.shape[-1]).sum(axis=0)


def backward(params, cache, dy, sh: FnoShape):
    """dy = dLoss/dy [B, nz, ny, nx] -> gradients of every parameter."""
    g = {k: np.zeros_like(v) for k, v in params.items()}
    h, a1 = cache["h"], cache["a1"]
    dyc = dy[..., None]                                     # [.., 1]
    g["Q2"] = _outer_sum(dyc, h)
    g["c2"] = _lead_sum(dyc)
    dh = dyc @ params["Q2"]
    da1 = dh * gelu_grad(a1)
    vL = cache["v"][-1]
    g["Q1"] = _outer_sum(da1, vL)
    g["c1"] = _lead_sum(da1)
    dv = da1 @ params["Q1"]
    B = dy.shape[0]
    N = sh.nx * sh.ny * sh.nz
    for l in reversed(range(sh.layers)):
        u = cache["u"][l]
        du = dv * gelu_grad(u) if l < sh.layers - 1 else dv
        vin = cache["v"][l]
        g["Wl"][l] = _outer_sum(du, vin)
        g["bl"][l] = _lead_sum(du)
        dv = du @ params["Wl"][l]
        # spectral branch: dYh = (w_c / N) * forward-DFT(du)
        w = np.ones(sh.mz)
        w[1:] = 2.0
        dYh = forward_dft(du, sh) * (w[None, :, None, None, None] / N)
        dYf = dYh.reshape(B, -1, sh.width)
        Xf = cache["Xh"][l].reshape(B, -1, sh.width)
        R = params["Rr"][l] + 1j * params["Ri"][l]
        dR = np.einsum("nmi,nmo->mio", np.conj(Xf), dYf)
        g["Rr"][l] = dR.real
        g["Ri"][l] = dR.imag
        dXf = np.einsum("nmo,mio->nmi", dYf, np.conj(R))
        dXh = dXf.reshape(cache["Xh"][l].shape)
        dv = dv + inverse_dft(dXh, sh, weighted=False, scale=1.0)
    g["P"] = _outer_sum(dv, cache["x"])
    g["bP"] = _lead_sum(dv)
    return g


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) in place; t counts from 1."""
    for k in params:
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
