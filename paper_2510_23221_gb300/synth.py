"""Seeded synthetic layered-chip workloads.

This module only draws inputs: chip geometry and materials, power-density
maps and combination coefficients.  It holds none of the method's arithmetic
(no conductances, no right-hand sides, no solves), so both the CUDA path and
the FP64 CPU oracle may use it.

The paper's own matrices come from FEM meshes of hand-made floorplans
(Sec. V-A) that are not available; these layered chips stand in for them.
Recipe (all distributions seeded through ``numpy.random.default_rng``):

* cell size 100 um x 100 um laterally, 50 um per layer, one cell per layer;
* 32x32x4 reference stack: silicon k=150, TIM k=5, spreader k=400,
  substrate k=20 W/m/K (top to bottom), top convective h=1e4 W/m^2/K at
  300 K, every other face adiabatic;
* other stacks draw each layer's k log-uniform in [1, 400] W/m/K;
* power maps live on the top (silicon) layer, in W/m^2: either a sum of 1-5
  rectangles of uniform density (sides uniform in 1..n/2 cells, density
  log-uniform in [1e5, 1e7]) or one Gaussian hotspot (amplitude log-uniform
  in [1e5, 1e7], sigma uniform in [2, 16] cells, centre uniform);
* combination coefficients C ~ N(0, 1), rounded to the nearest bfloat16
  value (round-half-even) so that every consumer sees the same exact operand.

The 3-D IC of the paper's experiments (Sec. V-A) is also available
(``paper_3dic_chip``, ``paper_3dic_sources``, ``paper_3dic_workload``):
10 mm x 10 mm x 0.51 mm; three 0.15 mm silicon device layers (core on top,
then two L2-cache layers), each above a 0.02 mm TIM layer; k = 150 (silicon),
40 (TIM), 413 (copper TSVs) W/m/K; 156 core blocks (6 at 3-6 W/mm^2, 150 at
0.5-1 W/mm^2) and two caches per L2 layer (0.02-0.04 W/mm^2); Dirichlet
(all faces at 50 C), Robin (h = 3e4 on every face) or mixed (Robin top and
bottom, held sides).  The paper's floorplans are hand-made and not
published; here the core blocks tile the die in a 12 x 13 grid, each cache
is half of its layer, TSV bundles are square copper columns through the
stack at seeded sites, and a device layer's areal power density is spread
evenly over its thickness.

Seeds: chip j of workload c uses ``1_000_000 * c + j``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

CELL_DX = 100e-6
CELL_DY = 100e-6
CELL_DZ = 50e-6
T_AMBIENT = 300.0


@dataclass
class Chip:
    """One layered chip on a structured nx x ny x nz grid (z = 0 is the top)."""

    nx: int
    ny: int
    layer_nz: np.ndarray          # int32 [n_layers]: cells per layer along z
    layer_dz: np.ndarray          # float64 [n_layers]: thickness of one cell, m
    layer_k: np.ndarray           # float64 [n_layers]: conductivity, W/m/K
    dx: float = CELL_DX
    dy: float = CELL_DY
    h_top: float = 1e4            # W/m^2/K, 0 = adiabatic
    h_bottom: float = 0.0
    h_side: float = 0.0
    t_ambient: float = T_AMBIENT
    k_cell: Optional[np.ndarray] = None   # float64 [nz][ny][nx] overrides layer_k

    @property
    def nz(self) -> int:
        return int(np.sum(self.layer_nz))

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def cell_dz(self) -> np.ndarray:
        """Thickness of every z-row of cells (float64 [nz])."""
        return np.repeat(np.asarray(self.layer_dz, np.float64),
                         np.asarray(self.layer_nz, np.int64))

    def cell_k(self) -> np.ndarray:
        """Per-cell conductivity as float64 [nz][ny][nx]."""
        if self.k_cell is not None:
            return np.asarray(self.k_cell, np.float64).reshape(self.nz, self.ny, self.nx)
        kz = np.repeat(np.asarray(self.layer_k, np.float64),
                       np.asarray(self.layer_nz, np.int64))
        return np.broadcast_to(kz[:, None, None], (self.nz, self.ny, self.nx)).copy()


@dataclass
class Workload:
    """Chips, their power maps and combination coefficients."""

    name: str
    chips: List[Chip]
    density: List[np.ndarray]     # per chip float64 [s][ny][nx], W/m^2 on the top layer
    coeffs: List[np.ndarray]      # per chip float64 [s][M], bfloat16-exact
    s: int
    M: int
    rtol: float
    extra: dict = field(default_factory=dict)
    # per chip float64 [s][nz][ny][nx], W/m^3: volumetric sources anywhere in
    # the stack; when set, the right-hand sides come from these (and
    # ``density`` is unused)
    sources: Optional[List[np.ndarray]] = None


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 value (ties to even).

    bfloat16 keeps 8 significant bits; frexp gives a mantissa in [0.5, 1),
    so scaling by 2**8 and rounding half-to-even keeps exactly 8 bits.
    """
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def rect_power_map(rng, nx: int, ny: int) -> np.ndarray:
    """Sum of 1-5 rectangles of uniform density (W/m^2), float64 [ny][nx]."""
    out = np.zeros((ny, nx), np.float64)
    for _ in range(int(rng.integers(1, 6))):
        w = int(rng.integers(1, max(1, nx // 2) + 1))
        h = int(rng.integers(1, max(1, ny // 2) + 1))
        x0 = int(rng.integers(0, nx - w + 1))
        y0 = int(rng.integers(0, ny - h + 1))
        out[y0:y0 + h, x0:x0 + w] += _log_uniform(rng, 1e5, 1e7)
    return out


def gauss_power_map(rng, nx: int, ny: int) -> np.ndarray:
    """One Gaussian hotspot (W/m^2), float64 [ny][nx], sampled at cell centres."""
    amp = _log_uniform(rng, 1e5, 1e7)
    sig = rng.uniform(2.0, 16.0)
    cx = rng.uniform(0.0, nx)
    cy = rng.uniform(0.0, ny)
    xs = np.arange(nx) + 0.5
    ys = np.arange(ny) + 0.5
    r2 = (xs[None, :] - cx) ** 2 + (ys[:, None] - cy) ** 2
    return amp * np.exp(-r2 / (2.0 * sig * sig))


def power_maps(rng, nx: int, ny: int, s: int, mix: bool) -> np.ndarray:
    """s power maps; with ``mix`` each map is a rectangle set or a hotspot (50/50)."""
    maps = []
    for _ in range(s):
        if mix and rng.uniform() < 0.5:
            maps.append(gauss_power_map(rng, nx, ny))
        else:
            maps.append(rect_power_map(rng, nx, ny))
    return np.stack(maps) if maps else np.zeros((0, ny, nx))


def coefficients(rng, s: int, M: int) -> np.ndarray:
    """C ~ N(0,1) of shape [s][M], rounded to bfloat16-exact float64."""
    return round_to_bf16(rng.standard_normal((s, M)))


def _layered_chip(rng, nx, ny, n_layers, h_top) -> Chip:
    return Chip(nx=nx, ny=ny,
                layer_nz=np.ones(n_layers, np.int32),
                layer_dz=np.full(n_layers, CELL_DZ),
                layer_k=_log_uniform(rng, 1.0, 400.0, n_layers),
                h_top=float(h_top))


def reference_stack_chip() -> Chip:
    """32x32x4 chip: silicon / TIM / spreader / substrate, top Robin h=1e4."""
    return Chip(nx=32, ny=32, layer_nz=np.ones(4, np.int32),
                layer_dz=np.full(4, CELL_DZ),
                layer_k=np.array([150.0, 5.0, 400.0, 20.0]), h_top=1e4)


def small_fp64_workload(M: int = 64) -> Workload:
    """32x32x4 reference stack, s=8 rectangle maps, M=64, solved to 1e-12."""
    rng = np.random.default_rng(1_000_000 * 1 + 0)
    chip = reference_stack_chip()
    dens = power_maps(rng, chip.nx, chip.ny, 8, mix=False)
    C = coefficients(rng, 8, M)
    return Workload("chip32x32x4_s8_M64_fp64", [chip], [dens], [C], s=8, M=M, rtol=1e-12)


def single_chip_workload(nx=128, ny=128, n_layers=8, s=32, M=5000,
                         cfg=2, rtol=1e-6, name=None) -> Workload:
    """One chip with log-uniform layer k, mixed rectangle/hotspot maps."""
    rng = np.random.default_rng(1_000_000 * cfg + 0)
    chip = _layered_chip(rng, nx, ny, n_layers, 1e4)
    dens = power_maps(rng, nx, ny, s, mix=True)
    C = coefficients(rng, s, M)
    name = name or f"chip{nx}x{ny}x{n_layers}_s{s}_M{M}"
    return Workload(name, [chip], [dens], [C], s=s, M=M, rtol=rtol)


def batched_workload(n_chips: int = 256, s: int = 16, M: int = 20,
                     sides=(64, 96, 128, 192, 256), cfg=3, rtol=1e-6, which=None) -> Workload:
    """Uneven chips: square side from ``sides``, 4-12 layers, h in [1e3, 1e5].

    Chip j draws from its own seed, so ``which`` (a list of chip indices)
    selects exactly those chips of the n_chips-chip batch."""
    chips, dens, Cs = [], [], []
    for j in (range(n_chips) if which is None else which):
        rng = np.random.default_rng(1_000_000 * cfg + j)
        side = int(rng.choice(np.asarray(sides)))
        nl = int(rng.integers(4, 13))
        h = rng.uniform(1e3, 1e5)
        chip = _layered_chip(rng, side, side, nl, h)
        chips.append(chip)
        dens.append(power_maps(rng, side, side, s, mix=True))
        Cs.append(coefficients(rng, s, M))
    name = f"batch{n_chips}_s{s}_M{M}" if which is None else f"batch{n_chips}_subset{len(chips)}_s{s}_M{M}"
    return Workload(name, chips, dens, Cs, s=s, M=M, rtol=rtol)


FNO_TRAIN_SEED0 = 10_000_000      # training chips of the warm-start network
FNO_HELDOUT_SEED0 = 20_000_000    # held-out evaluation chips (disjoint seeds)


def warm_start_chip(seed: int, nx: int = 128, ny: int = 128, n_layers: int = 8, s: int = 32):
    """One chip of the benchmark chip's distribution (8 layers, k log-uniform
    in [1, 400], top h = 1e4, s mixed rectangle/hotspot maps) from its own
    seed: (chip, density [s][ny][nx])."""
    rng = np.random.default_rng(seed)
    chip = _layered_chip(rng, nx, ny, n_layers, 1e4)
    return chip, power_maps(rng, nx, ny, s, mix=True)


def large_chip_workload(M: int = 10000, s: int = 64) -> Workload:
    """512x512x16 chip, 16 log-uniform layers, s=64, M fields."""
    return single_chip_workload(512, 512, 16, s=s, M=M, cfg=5,
                                name=f"chip512x512x16_s{s}_M{M}")


def random_small_chip(seed: int, nx: int, ny: int, n_layers: int,
                      h_top=1e4, h_bottom=0.0, h_side=0.0,
                      layer_nz=None) -> Chip:
    """Small chip for tests: random layer k and thickness jitter."""
    rng = np.random.default_rng(seed)
    lnz = np.ones(n_layers, np.int32) if layer_nz is None else np.asarray(layer_nz, np.int32)
    return Chip(nx=nx, ny=ny, layer_nz=lnz,
                layer_dz=CELL_DZ * rng.uniform(0.5, 2.0, n_layers),
                layer_k=_log_uniform(rng, 1.0, 400.0, n_layers),
                h_top=h_top, h_bottom=h_bottom, h_side=h_side)


# ---------------------------------------------------------------- the paper's 3-D IC (Sec. V-A)
PAPER_3DIC = {
    "die_m": (10e-3, 10e-3, 0.51e-3),
    "device_layers": 3,
    "device_dz_m": 0.15e-3,
    "tim_dz_m": 0.02e-3,
    "k_silicon": 150.0,
    "k_copper": 413.0,
    "k_tim": 40.0,
    "core_blocks": 156,
    "hot_blocks": 6,
    "hot_w_per_mm2": (3.0, 6.0),
    "cool_w_per_mm2": (0.5, 1.0),
    "caches_per_l2_layer": 2,
    "l2_w_per_mm2": (0.02, 0.04),
    "h_robin": 3e4,
    "t_held_k": 323.15,
}
CORE_GRID = (12, 13)          # core blocks along x and y (12 x 13 = 156)
PAPER_BOUNDARIES = ("dirichlet", "robin", "mixed")


def paper_3dic_chip(seed: int, nx: int = 92, ny: int = 92, boundary: str = "dirichlet",
                    device_cells: int = 3, tsv_bundles: int = 4, tsv_side: int = 2) -> Chip:
    """The paper's six-layer 3-D IC stack on an nx x ny x (3 (device_cells + 1))
    grid.  TSV bundles (``tsv_bundles`` squares of ``tsv_side`` cells, seeded
    sites) are copper through every layer, so the chip carries a per-cell k."""
    P = PAPER_3DIC
    if boundary not in PAPER_BOUNDARIES:
        raise ValueError(f"boundary must be one of {PAPER_BOUNDARIES}")
    nd = P["device_layers"]
    layer_nz = np.array([device_cells, 1] * nd, np.int32)
    layer_dz = np.array([P["device_dz_m"] / device_cells, P["tim_dz_m"]] * nd)
    layer_k = np.array([P["k_silicon"], P["k_tim"]] * nd)
    h = {"dirichlet": (np.inf, np.inf, np.inf),
         "robin": (P["h_robin"], P["h_robin"], P["h_robin"]),
         "mixed": (P["h_robin"], P["h_robin"], np.inf)}[boundary]
    chip = Chip(nx=nx, ny=ny, layer_nz=layer_nz, layer_dz=layer_dz, layer_k=layer_k,
                dx=P["die_m"][0] / nx, dy=P["die_m"][1] / ny,
                h_top=h[0], h_bottom=h[1], h_side=h[2], t_ambient=P["t_held_k"])
    if tsv_bundles > 0:
        rng = np.random.default_rng(seed)
        k = chip.cell_k()
        side = min(tsv_side, nx, ny)
        for _ in range(tsv_bundles):
            x0 = int(rng.integers(0, nx - side + 1))
            y0 = int(rng.integers(0, ny - side + 1))
            k[:, y0:y0 + side, x0:x0 + side] = P["k_copper"]
        chip.k_cell = k
    return chip


def _block_edges(n: int, parts: int) -> np.ndarray:
    return np.rint(np.linspace(0.0, n, parts + 1)).astype(np.int64)


def paper_3dic_sources(rng, chip: Chip, s: int) -> np.ndarray:
    """s floorplan power draws as volumetric sources, float64 [s][nz][ny][nx]
    (W/m^3): per draw, 6 of the 156 core blocks are hot (3-6 W/mm^2), the rest
    0.5-1 W/mm^2, and each of the two caches of both L2 layers 0.02-0.04
    W/mm^2 (all uniform); areal density / device-layer thickness."""
    P = PAPER_3DIC
    nd = P["device_layers"]
    dev_cells = int(chip.layer_nz[0])
    t_dev = P["device_dz_m"]
    gx, gy = CORE_GRID
    ex, ey = _block_edges(chip.nx, gx), _block_edges(chip.ny, gy)
    half = chip.nx // 2
    out = np.zeros((s, chip.nz, chip.ny, chip.nx))
    for j in range(s):
        core = np.zeros((chip.ny, chip.nx))
        hot = set(rng.choice(gx * gy, P["hot_blocks"], replace=False).tolist())
        for b in range(gx * gy):
            bx, by = b % gx, b // gx
            lo, hi = P["hot_w_per_mm2"] if b in hot else P["cool_w_per_mm2"]
            core[ey[by]:ey[by + 1], ex[bx]:ex[bx + 1]] = rng.uniform(lo, hi) * 1e6
        layers = [core]
        for _ in range(nd - 1):
            l2 = np.zeros((chip.ny, chip.nx))
            for c, (x0, x1) in enumerate(((0, half), (half, chip.nx))[:P["caches_per_l2_layer"]]):
                l2[:, x0:x1] = rng.uniform(*P["l2_w_per_mm2"]) * 1e6
            layers.append(l2)
        for d, areal in enumerate(layers):
            z0 = d * (dev_cells + 1)            # first z-row of device layer d
            out[j, z0:z0 + dev_cells] = areal / t_dev
    return out


def paper_3dic_workload(n_chips: int = 5, nx: int = 92, ny: int = 92, s: int = 50, M: int = 1000,
                        boundary: str = "dirichlet", cfg: int = 6, rtol: float = 1e-6) -> Workload:
    """N_k = n_chips floorplans of the 3-D IC (own TSV sites and power draws),
    N_basis = s sources each, M fields per chip: the paper's ablation setting
    (Sec. V-E: N_basis 50, N_k 5, N_data 5000, n ~ 1e5, Dirichlet) at the
    defaults (92 x 92 x 12 = 101,568 cells per chip)."""
    chips, srcs, Cs = [], [], []
    for j in range(n_chips):
        seed = 1_000_000 * cfg + j
        chip = paper_3dic_chip(seed, nx, ny, boundary)
        rng = np.random.default_rng(seed + 500_000)
        chips.append(chip)
        srcs.append(paper_3dic_sources(rng, chip, s))
        Cs.append(coefficients(rng, s, M))
    empty = [np.zeros((s, c.ny, c.nx)) for c in chips]
    return Workload(f"paper3dic_{boundary}_{n_chips}x{nx}x{ny}x{chips[0].nz}_s{s}_M{M}", chips, empty, Cs,
                    s=s, M=M, rtol=rtol, sources=srcs)
