"""The seeded synthetic workloads against the configurations they stand in
for: grid, layer stack, boundary conditions, number of right-hand sides,
fields and tolerance, and the value ranges of every random draw.  No GPU."""
import numpy as np
import pytest

from paper_2510_23221_gb300 import synth


def _bf16_exact(x):
    x = np.asarray(x, np.float64)
    return np.array_equal(synth.round_to_bf16(x), x)


def test_reference_stack_chip_workload():
    """32x32x4: silicon 150 / TIM 5 / spreader 400 / substrate 20 W/m/K,
    100 x 100 x 50 um cells, top h = 1e4 at 300 K, other faces adiabatic,
    s = 8 rectangle maps, M = 64, relative residual 1e-12."""
    w = synth.small_fp64_workload()
    (c,) = w.chips
    assert (c.nx, c.ny, c.nz) == (32, 32, 4) and c.n == 4096
    assert list(c.layer_k) == [150.0, 5.0, 400.0, 20.0]
    assert np.all(c.layer_dz == 50e-6) and c.dx == 100e-6 and c.dy == 100e-6
    assert (c.h_top, c.h_bottom, c.h_side, c.t_ambient) == (1e4, 0.0, 0.0, 300.0)
    assert (w.s, w.M, w.rtol) == (8, 64, 1e-12)
    d = w.density[0]
    assert d.shape == (8, 32, 32) and np.all(d >= 0)
    for m in d:   # a sum of 1-5 uniform rectangles, each density in [1e5, 1e7]
        vals = np.unique(m[m > 0])
        assert 1e5 <= vals.min() and vals.max() <= 5e7
        assert 1 <= len(vals) <= 2 ** 5 - 1
    C = w.coeffs[0]
    assert C.shape == (8, 64) and _bf16_exact(C)


def test_benchmark_chip_workload():
    """128x128x8 with 8 layers of k log-uniform in [1, 400], the same
    boundary conditions, s = 32 block/hotspot maps, M = 5000, 1e-6."""
    w = synth.single_chip_workload()
    (c,) = w.chips
    assert (c.nx, c.ny, c.nz) == (128, 128, 8) and c.n == 131072
    assert np.all((c.layer_k >= 1.0) & (c.layer_k <= 400.0)) and len(np.unique(c.layer_k)) == 8
    assert (c.h_top, c.h_bottom, c.h_side) == (1e4, 0.0, 0.0)
    assert (w.s, w.M, w.rtol) == (32, 5000, 1e-6)
    assert w.density[0].shape == (32, 128, 128) and np.all(w.density[0] >= 0)
    C = w.coeffs[0]
    assert C.shape == (32, 5000) and _bf16_exact(C)
    # N(0, 1) draws, rounded to 8 significant bits
    assert abs(C.mean()) < 0.02 and abs(C.std() - 1.0) < 0.02


def test_batched_workload_draws():
    """Uneven chips: side in {64, 96, 128, 192, 256}, 4-12 layers, k in
    [1, 400], top h uniform in [1e3, 1e5], s = 16, M = 20, 1e-6; chip j
    is seeded on its own, so a prefix of the batch is the same chips."""
    w = synth.batched_workload(n_chips=10)
    assert (w.s, w.M, w.rtol) == (16, 20, 1e-6)
    for c in w.chips:
        assert c.nx == c.ny and c.nx in (64, 96, 128, 192, 256)
        assert 4 <= c.nz <= 12 and np.all(c.layer_nz == 1)
        assert np.all((c.layer_k >= 1.0) & (c.layer_k <= 400.0))
        assert 1e3 <= c.h_top <= 1e5 and c.h_bottom == 0.0 and c.h_side == 0.0
    w4 = synth.batched_workload(n_chips=4)
    for a, b in zip(w4.chips, w.chips):
        assert a.nx == b.nx and np.array_equal(a.layer_k, b.layer_k) and a.h_top == b.h_top


def test_large_chip_workload():
    """512x512x16, 16 layers, s = 64; M fields (10,000 streamed in chunks)."""
    w = synth.large_chip_workload(M=10)
    (c,) = w.chips
    assert (c.nx, c.ny, c.nz) == (512, 512, 16) and c.n == 4194304
    assert (w.s, w.M, w.rtol) == (64, 10, 1e-6)
    assert w.density[0].shape == (64, 512, 512)


def test_warm_start_chips_are_the_benchmark_distribution():
    chip, dens = synth.warm_start_chip(synth.FNO_TRAIN_SEED0)
    assert (chip.nx, chip.ny, chip.nz) == (128, 128, 8) and chip.h_top == 1e4
    assert dens.shape == (32, 128, 128)
    held, _ = synth.warm_start_chip(synth.FNO_HELDOUT_SEED0)
    assert not np.array_equal(chip.layer_k, held.layer_k)
    assert synth.FNO_HELDOUT_SEED0 - synth.FNO_TRAIN_SEED0 >= 512 * 1000


@pytest.mark.parametrize("make", [synth.gauss_power_map, synth.rect_power_map])
def test_power_maps_are_nonnegative_and_in_range(make):
    rng = np.random.default_rng(4)
    for _ in range(20):
        m = make(rng, 40, 30)
        assert m.shape == (30, 40) and np.all(m >= 0) and m.max() <= 5e7 and m.max() > 0
