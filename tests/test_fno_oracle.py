"""Pins of the float64 FNO reference (oracle/fno_oracle.py), no GPU.

The truncated transform is checked against numpy's FFT (a library routine
computed independently), its inverse against exact reconstruction of a
band-limited signal, the activation against its closed form, every
gradient of a small network against central finite differences, and the
Adam step against Algorithm 1 of Kingma & Ba written out for one step.
"""
import numpy as np
import pytest

from oracle import fno_oracle as fo

TINY = fo.FnoShape(nx=8, ny=6, nz=4, c_in=3, width=3, hidden=4, layers=2, mx=4, my=4, mz=2)


def test_forward_dft_matches_numpy_fft():
    sh = fo.FnoShape(nx=16, ny=12, nz=8, width=2, mx=6, my=4, mz=3)
    rng = np.random.default_rng(0)
    v = rng.standard_normal((2, sh.nz, sh.ny, sh.nx, 2))
    Xh = fo.forward_dft(v, sh)
    F = np.fft.fftn(v, axes=(1, 2, 3))
    kx, ky, kz = fo.modes(sh)
    for c in range(sh.mz):
        for b in range(sh.my):
            for a in range(sh.mx):
                ref = F[:, kz[c] % sh.nz, ky[b] % sh.ny, kx[a] % sh.nx, :]
                assert np.allclose(Xh[:, c, b, a, :], ref, atol=1e-10)


def test_inverse_dft_reconstructs_band_limited_signal():
    sh = fo.FnoShape(nx=16, ny=12, nz=8, width=1, mx=6, my=6, mz=3)
    rng = np.random.default_rng(1)
    x, y, z = np.meshgrid(np.arange(sh.nx), np.arange(sh.ny), np.arange(sh.nz), indexing="ij")
    v = np.zeros((sh.nz, sh.ny, sh.nx))
    # real signal with |kx| <= 2, |ky| <= 2, |kz| <= 2 (inside the symmetric part of the mode set)
    for kx_ in range(-2, 3):
        for ky_ in range(-2, 3):
            for kz_ in range(0, 3):
                ph = 2 * np.pi * (kx_ * x / sh.nx + ky_ * y / sh.ny + kz_ * z / sh.nz)
                v += (rng.standard_normal() * np.cos(ph) + rng.standard_normal() * np.sin(ph)).transpose(2, 1, 0)
    v = v[None, ..., None]
    back = fo.inverse_dft(fo.forward_dft(v, sh), sh)
    assert np.allclose(back, v, atol=1e-10)


def test_gelu_closed_form_and_derivative():
    from math import erf, sqrt
    xs = np.array([-3.0, -1.0, -0.25, 0.0, 0.5, 2.0, 6.0])
    ref = np.array([x * 0.5 * (1 + erf(x / sqrt(2))) for x in xs])
    assert np.allclose(fo.gelu(xs), ref, rtol=0, atol=1e-15)
    assert fo.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    fd = (fo.gelu(xs + h) - fo.gelu(xs - h)) / (2 * h)
    assert np.allclose(fo.gelu_grad(xs), fd, atol=1e-8)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_central_differences(seed):
    sh = TINY
    rng = np.random.default_rng(10 + seed)
    params = fo.init_params(sh, seed)
    for k in params:   # nonzero biases and larger spectral weights exercise every path
        params[k] = params[k] + 0.1 * rng.standard_normal(params[k].shape)
    x = rng.standard_normal((2, sh.nz, sh.ny, sh.nx, sh.c_in))
    target = rng.standard_normal((2, sh.nz, sh.ny, sh.nx))

    def L(p):
        y, _ = fo.forward(p, x, sh)
        return fo.loss(y, target)

    y, cache = fo.forward(params, x, sh)
    dy = 2.0 * (y - target) / y.size
    g = fo.backward(params, cache, dy, sh)
    h = 1e-6
    for name, val in params.items():
        flat = val.ravel()
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = L(params)
            flat[i] = old - h
            lm = L(params)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[i]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (name, i, fd, an)


def test_spectral_layer_is_linear_in_its_input():
    sh = TINY
    rng = np.random.default_rng(5)
    p = fo.init_params(sh, 3)
    a = rng.standard_normal((1, sh.nz, sh.ny, sh.nx, sh.width))
    b = rng.standard_normal((1, sh.nz, sh.ny, sh.nx, sh.width))
    ka, _ = fo.spectral(a, p["Rr"][0], p["Ri"][0], sh)
    kb, _ = fo.spectral(b, p["Rr"][0], p["Ri"][0], sh)
    kab, _ = fo.spectral(2 * a - 3 * b, p["Rr"][0], p["Ri"][0], sh)
    assert np.allclose(kab, 2 * ka - 3 * kb, atol=1e-12)


@pytest.mark.parametrize("shift", [(1, 0, 0), (0, 2, 0), (0, 0, 1), (3, 1, 2)])
def test_spectral_layer_commutes_with_circular_shifts(shift):
    """A shift of the input by (sx, sy, sz) cells multiplies every retained
    mode by the same phase, which the inverse transform turns back into the
    same shift: the spectral convolution is circular-shift equivariant in
    x, y and z (a sign or index slip in either transform breaks this)."""
    sh = TINY
    rng = np.random.default_rng(11)
    p = fo.init_params(sh, 4)
    v = rng.standard_normal((2, sh.nz, sh.ny, sh.nx, sh.width))
    sx, sy, sz = shift
    k, _ = fo.spectral(v, p["Rr"][1], p["Ri"][1], sh)
    vs = np.roll(v, (sz, sy, sx), axis=(1, 2, 3))
    ks, _ = fo.spectral(vs, p["Rr"][1], p["Ri"][1], sh)
    assert np.allclose(ks, np.roll(k, (sz, sy, sx), axis=(1, 2, 3)), atol=1e-12 * np.abs(k).max())
    # and a shift is not the identity on this input (the check has teeth)
    assert not np.allclose(ks, k)


def test_adam_first_step():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    fo.adam_step(p, g, m, v, t=1, lr=0.01)
    # step 1: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    ref = np.array([1.0, -2.0, 0.5]) - 0.01 * np.array([0.3, -4.0, 0.0]) / (np.abs([0.3, -4.0, 0.0]) + 1e-8)
    assert np.allclose(p["w"], ref, atol=1e-15)


def test_parameter_count_of_the_warm_start_network():
    sh = fo.FnoShape(nx=128, ny=128, nz=8)
    n = sum(int(np.prod(s)) for s in fo.param_shapes(sh).values())
    # spectral weights dominate: 4 layers x 576 modes x 32 x 32 complex
    assert n == 4 * 576 * 32 * 32 * 2 + 4 * (32 * 32 + 32) + 5 * 32 + 32 + 32 * 128 + 128 + 128 + 1
