"""The 3-D IC of the paper's experiments (Sec. V-A) as the input generator
builds it, checked against the values the paper prints
(``tests/golden/paper_3dic_setup.json``, transcribed with citations), and
the oracle on that stack under the paper's three boundary scenarios.
No GPU."""
import json
import os

import numpy as np
import pytest

from oracle import blockoa_oracle as orc
from paper_2510_23221_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_3dic_setup.json")))
P = synth.PAPER_3DIC


def test_generator_constants_are_the_printed_ones():
    g = GOLDEN["chip"]
    assert tuple(1e3 * v for v in P["die_m"]) == pytest.approx(tuple(g["size_mm"]), rel=1e-12)
    assert P["device_layers"] == g["device_layers"]
    assert 1e3 * P["device_dz_m"] == pytest.approx(g["device_layer_thickness_mm"], rel=1e-12)
    assert 1e3 * P["tim_dz_m"] == pytest.approx(g["tim_layer_thickness_mm"], rel=1e-12)
    k = g["conductivity_W_per_mK"]
    assert (P["k_silicon"], P["k_copper"], P["k_tim"]) == (k["silicon"], k["copper"], k["tim"])
    w = GOLDEN["power"]
    assert P["core_blocks"] == w["core_blocks"] and P["hot_blocks"] == w["hot_blocks"]
    assert tuple(P["hot_w_per_mm2"]) == tuple(w["hot_W_per_mm2"])
    assert tuple(P["cool_w_per_mm2"]) == tuple(w["other_W_per_mm2"])
    assert P["caches_per_l2_layer"] == w["caches_per_l2_layer"]
    assert P["device_layers"] - 1 == w["l2_layers"]
    assert tuple(P["l2_w_per_mm2"]) == tuple(w["cache_W_per_mm2"])
    b = GOLDEN["boundaries"]
    assert P["h_robin"] == b["robin_all_faces_htc_W_per_m2K"] == b["mixed_top_bottom_htc_W_per_m2K"]
    assert P["t_held_k"] - 273.15 == pytest.approx(b["dirichlet_all_faces_C"], abs=1e-12)
    assert b["mixed_sides_held_C"] == b["dirichlet_all_faces_C"]


def test_printed_stack_adds_up_and_the_grid_spans_it():
    g = GOLDEN["chip"]
    total = g["device_layers"] * (g["device_layer_thickness_mm"] + g["tim_layer_thickness_mm"])
    assert total == pytest.approx(g["size_mm"][2], rel=1e-12)
    assert synth.CORE_GRID[0] * synth.CORE_GRID[1] == GOLDEN["power"]["core_blocks"]
    for cells in (1, 3):
        chip = synth.paper_3dic_chip(0, nx=20, ny=30, device_cells=cells)
        assert 1e3 * chip.cell_dz().sum() == pytest.approx(g["size_mm"][2], rel=1e-12)
        assert 1e3 * chip.nx * chip.dx == pytest.approx(g["size_mm"][0], rel=1e-12)
        assert 1e3 * chip.ny * chip.dy == pytest.approx(g["size_mm"][1], rel=1e-12)
        # device layers silicon, TIM below each
        k = chip.cell_k()[:, 0, 0] if chip.k_cell is None else np.repeat(chip.layer_k, chip.layer_nz)
        assert list(np.unique(k)) == [P["k_tim"], P["k_silicon"]]


def test_workload_sizes_match_the_printed_dimensions():
    ab = GOLDEN["ablation"]
    w = synth.paper_3dic_workload(n_chips=2, s=3, M=4)
    n = w.chips[0].n
    assert abs(n - ab["matrix_dimension"]) / ab["matrix_dimension"] < 0.02
    assert ab["N_basis"] == 50 and ab["N_k"] == 5 and ab["N_data"] == 5 * 1000   # the workload's defaults
    lo, hi = GOLDEN["meshes"]["matrix_dimension_range"]
    # the printed mesh range is covered by square grids of 72 .. 150 cells a side
    assert lo <= synth.paper_3dic_chip(0, 72, 72).n and abs(synth.paper_3dic_chip(0, 150, 150).n - hi) / hi < 0.01
    # the volumetric sources replace the top-layer densities
    assert w.sources[0].shape == (3, w.chips[0].nz, w.chips[0].ny, w.chips[0].nx)


@pytest.mark.parametrize("seed", [0, 1])
def test_power_draws_follow_the_printed_ranges(seed):
    chip = synth.paper_3dic_chip(seed, nx=37, ny=41, device_cells=2)
    qv = synth.paper_3dic_sources(np.random.default_rng(seed), chip, 3)
    t_dev = P["device_dz_m"]
    ex = np.rint(np.linspace(0, chip.nx, synth.CORE_GRID[0] + 1)).astype(int)
    ey = np.rint(np.linspace(0, chip.ny, synth.CORE_GRID[1] + 1)).astype(int)
    for j in range(3):
        rows = qv[j]
        for d, z0 in enumerate((0, 3, 6)):
            assert np.array_equal(rows[z0], rows[z0 + 1])          # uniform through the layer
            assert np.all(rows[z0 + 2] == 0)                       # TIM below carries none
        core = rows[0] * t_dev / 1e6                               # W/mm^2
        dens = np.array([[core[ey[b]:ey[b + 1], ex[a]:ex[a + 1]] for a in range(synth.CORE_GRID[0])]
                         for b in range(synth.CORE_GRID[1])], dtype=object)
        vals = np.array([[blk.min(), blk.max()] for blk in dens.ravel()])
        assert np.all(vals[:, 0] == vals[:, 1])                    # one density per block
        hot = (vals[:, 0] >= 3.0) & (vals[:, 0] <= 6.0)
        cool = (vals[:, 0] >= 0.5) & (vals[:, 0] <= 1.0)
        assert hot.sum() == 6 and cool.sum() == 150
        for z0 in (3, 6):
            l2 = rows[z0] * t_dev / 1e6
            halves = (l2[:, :chip.nx // 2], l2[:, chip.nx // 2:])
            for h in halves:
                assert h.min() == h.max() and 0.02 <= h.min() <= 0.04


@pytest.mark.parametrize("boundary", synth.PAPER_BOUNDARIES)
def test_oracle_on_the_paper_boundaries(boundary):
    """SPD, and energy balance: the power injected in the three device
    layers leaves through the held or convective faces."""
    chip = synth.paper_3dic_chip(5, nx=6, ny=5, boundary=boundary, device_cells=1, tsv_bundles=2)
    assert chip.k_cell is not None and np.any(chip.k_cell == P["k_copper"])
    A = orc.assemble(chip)
    Ad = A.toarray()
    assert np.array_equal(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > 0
    qv = synth.paper_3dic_sources(np.random.default_rng(5), chip, 2)
    B = orc.rhs_volume(chip, qv)
    theta = np.linalg.solve(Ad, B)
    assert np.allclose(orc.boundary_loss(chip, theta), B.sum(axis=0), rtol=1e-10)
    U, info = orc.block_cg(A, B, rtol=1e-12)
    assert np.allclose(U, theta, rtol=1e-9, atol=1e-9 * np.abs(theta).max())


def _stack_continuous(zc, tops, k, g, h):
    """Exact theta(z) of -(k theta')' = g(z) through a stack of layers (z down
    from the cooled top, layer i on [tops[i], tops[i+1]) with constant k[i],
    g[i]), insulated bottom, h theta = k theta' at z = 0.  F(z), the heat
    crossing depth z upwards, is the source beneath it; theta is F(0)/h plus
    the integral of F/k from the top."""
    L = tops[-1]

    def F(z):
        return sum(g[i] * max(0.0, tops[i + 1] - max(z, tops[i])) for i in range(len(k)))

    out = np.empty(len(zc))
    for m, z in enumerate(zc):
        th = F(0.0) / h
        for i in range(len(k)):
            a, b = tops[i], min(tops[i + 1], z)
            if b <= a:
                break
            # F is linear on [a, b] inside one layer: trapezoid is exact
            th += (b - a) * (F(a) + F(b)) / (2.0 * k[i])
        out[m] = th
    assert L > 0
    return out


def test_oracle_converges_to_the_stack_solution_with_three_heated_layers():
    """The paper's six-layer stack with a volumetric source in each device
    layer, convective top, insulated elsewhere: refining every layer along z
    converges to the continuous solution at second order."""
    h = 3e4
    q = [4e9, 3e8, 2e8]                       # W/m^3 in the core and the two cache layers
    errs = []
    for r in (1, 2, 4, 8):
        chip = synth.paper_3dic_chip(0, nx=2, ny=2, device_cells=3 * r, tsv_bundles=0)
        chip.layer_nz = np.array([3 * r, r] * 3, np.int32)
        chip.layer_dz = np.array([P["device_dz_m"] / (3 * r), P["tim_dz_m"] / r] * 3)
        chip.h_top, chip.h_bottom, chip.h_side = h, 0.0, 0.0
        dz = chip.cell_dz()
        qrow = np.zeros(chip.nz)
        z0 = 0
        for d in range(3):
            qrow[z0:z0 + 3 * r] = q[d]
            z0 += 4 * r
        qv = np.broadcast_to(qrow[None, :, None, None], (1, chip.nz, chip.ny, chip.nx)).copy()
        B = orc.rhs_volume(chip, qv)
        theta = np.linalg.solve(orc.assemble(chip).toarray(), B)[:, 0].reshape(chip.nz, 2, 2)[:, 0, 0]
        tops = np.concatenate([[0.0], np.cumsum(chip.layer_dz * chip.layer_nz)])
        zc = np.cumsum(dz) - dz / 2
        g = [q[0], 0.0, q[1], 0.0, q[2], 0.0]
        exact = _stack_continuous(zc, tops, chip.layer_k, g, h)
        errs.append(np.abs(theta - exact).max() / np.abs(exact).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-4, errs
    assert all(rt > 1.8 for rt in rates), (errs, rates)
