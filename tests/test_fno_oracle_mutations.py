"""Planted mistakes in the FNO reference must each be caught by a pin of
tests/test_fno_oracle.py.  Every mutant is a plausible slip (a flipped
exponent sign, a dropped weight or term, a missing bias correction, a
channel mix left out); it replaces one function of the reference, the
pins run against it, and at least one must fail.  No GPU."""
import numpy as np
import pytest

from oracle import fno_oracle as fo
from tests import test_fno_oracle as pins

REAL = {name: getattr(fo, name) for name in ("forward_dft", "inverse_dft", "gelu_grad", "adam_step", "spectral")}


def _run_pins():
    checks = [
        ("fft", pins.test_forward_dft_matches_numpy_fft),
        ("inverse", pins.test_inverse_dft_reconstructs_band_limited_signal),
        ("gelu", pins.test_gelu_closed_form_and_derivative),
        ("gradients0", lambda: pins.test_gradients_match_central_differences(0)),
        ("gradients1", lambda: pins.test_gradients_match_central_differences(1)),
        ("linear", pins.test_spectral_layer_is_linear_in_its_input),
        ("shift_x", lambda: pins.test_spectral_layer_commutes_with_circular_shifts((1, 0, 0))),
        ("shift_xyz", lambda: pins.test_spectral_layer_commutes_with_circular_shifts((3, 1, 2))),
        ("adam", pins.test_adam_first_step),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(name)
    return failed


def test_unmutated_reference_passes_every_pin():
    assert _run_pins() == []


def _mut_dft_sign_x(v, sh):
    ex, ey, ez = fo.dft_mats(sh)
    return np.einsum("nzyxi,ax,by,cz->ncbai", v, np.conj(ex), ey, ez)


def _mut_inverse_unweighted(Yh, sh, weighted=True, scale=None):
    return REAL["inverse_dft"](Yh, sh, weighted=False, scale=scale)


def _mut_gelu_grad_no_pdf(x):
    return 0.5 * (1.0 + fo._erf(x / np.sqrt(2.0)))


def _mut_adam_no_bias_correction(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    for k in params:
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        params[k] = params[k] - lr * m[k] / (np.sqrt(v[k]) + eps)


def _mut_spectral_no_mix(v, Rr, Ri, sh):
    Xh = fo.forward_dft(v, sh)
    return fo.inverse_dft(Xh, sh), Xh


MUTANTS = {
    "dft_sign_x": ("forward_dft", _mut_dft_sign_x),
    "inverse_unweighted": ("inverse_dft", _mut_inverse_unweighted),
    "gelu_grad_no_pdf": ("gelu_grad", _mut_gelu_grad_no_pdf),
    "adam_no_bias_correction": ("adam_step", _mut_adam_no_bias_correction),
    "spectral_no_mix": ("spectral", _mut_spectral_no_mix),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(fo, attr, fn)
    assert _run_pins(), f"mutant {name} passed every pin"
