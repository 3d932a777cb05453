"""Index geometry of the block-CG kernels, checked on the CPU for many chip
shapes: the cell units of the loop kernels and the column tiles of the
z-line kernels must cover every cell of every chip exactly once and never
address a cell outside its chip.  The formulas restate those of
csrc/blockcg.cu (BK tile sizes, ColGeom, make_units); the checks are
coverage and bounds properties, so a geometry change that breaks them
fails here before any GPU run.  No GPU."""
import itertools

import numpy as np
import pytest


def tile_cells(S: int, elem: int) -> int:
    """BK<T, S>::TC: four cells per thread, 256 threads, 16 bytes of columns per thread."""
    V = 16 // elem
    TPR = S // V
    return 4 * (256 // TPR)


def make_units(chips, cells):
    units, off = [], 0
    for c, (nx, ny, nz) in enumerate(chips):
        n = nx * ny * nz
        for b in range(0, n, cells):
            units.append((c, off + b, off + min(b + cells, n)))
        off += n
    return units, off


def column_tile_slots(nx, ny, nz, TC):
    """Global (chip-local) cell of every (tile, slot); -1 outside the chip."""
    xt = TC // nz
    tiles_x = (nx + xt - 1) // xt
    nt = ny * tiles_x
    sl = np.arange(TC)
    z, dx = sl // xt, sl % xt
    out = np.full((nt, TC), -1, np.int64)
    for t in range(nt):
        y = t // tiles_x
        xb = (t - y * tiles_x) * xt
        xin = nx - xb
        ok = (z < nz) & (dx < xin)
        out[t, ok] = z[ok] * nx * ny + y * nx + xb + dx[ok]
    return out, xt


SHAPES = [(92, 92, 12), (128, 128, 8), (24, 20, 9), (13, 14, 9), (3, 5, 2), (33, 17, 5), (1, 7, 4),
          (7, 1, 3), (11, 9, 4), (48, 40, 6), (64, 64, 16), (37, 21, 8)]


@pytest.mark.parametrize("S,elem", list(itertools.product((8, 16, 32, 64), (4, 8))))
def test_column_tiles_cover_every_cell_once(S, elem):
    TC = tile_cells(S, elem)
    for nx, ny, nz in SHAPES:
        if nz > TC:
            continue   # such chips cannot use the z-line forms (checked by the library)
        slots, xt = column_tile_slots(nx, ny, nz, TC)
        assert xt >= 1 and xt * nz <= TC
        got = slots[slots >= 0]
        assert got.min() >= 0 and got.max() < nx * ny * nz
        assert np.array_equal(np.sort(got), np.arange(nx * ny * nz)), (S, elem, nx, ny, nz)
        # the tridiagonal recurrences walk slot z * xt + dx, inside the tile
        assert (nz - 1) * xt + (xt - 1) < TC


@pytest.mark.parametrize("cells", [64, 128, 256, 512, 1024, 2048, 4096])
def test_cell_units_partition_the_chips(cells):
    chips = SHAPES
    units, n_total = make_units(chips, cells)
    covered = np.zeros(n_total, np.int32)
    off = 0
    offs = []
    for nx, ny, nz in chips:
        offs.append(off)
        off += nx * ny * nz
    for c, b, e in units:
        nx, ny, nz = chips[c]
        assert offs[c] <= b < e <= offs[c] + nx * ny * nz and e - b <= cells
        covered[b:e] += 1
    assert np.all(covered == 1)


def test_tile_sizes_match_the_kernels_comments():
    # float32 S = 32: 128-cell tiles (the tensor-core P update's M = 128);
    # float32 S = 64: 64; float64 S = 64: 32
    assert tile_cells(32, 4) == 128 and tile_cells(64, 4) == 64 and tile_cells(64, 8) == 32
    # every tile size is a multiple of 4 cells (four cells per thread) and of 8 16-byte units
    for S, elem in itertools.product((8, 16, 32, 64), (4, 8)):
        TC = tile_cells(S, elem)
        assert TC % 4 == 0 and (TC // (16 // elem)) % 8 == 0
