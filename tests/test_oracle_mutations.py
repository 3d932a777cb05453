"""Planted mistakes in the oracle must each be caught by at least one pin.

Every mutant below is a plausible slip (a dropped half-cell factor, a wrong
sign, a wrong operand or index).  The mutant replaces one oracle function,
the pins of ``test_oracle_pins`` run against it, and at least one of them
must fail.  Nothing here touches a GPU.
"""
import numpy as np
import pytest

from oracle import blockoa_oracle as orc
from paper_2510_23221_gb300 import synth
from tests import test_oracle_pins as pins


def _run_pins():
    """Run every pin once; return the names of the pins that failed."""
    failed = []
    checks = [
        ("slab_chain", lambda: pins.test_slab_resistor_chain_closed_form(2.5e4)),
        ("slab_chain_held", lambda: pins.test_slab_resistor_chain_closed_form(np.inf)),
        ("slab_continuous", lambda: pins.test_slab_converges_to_continuous_solution(1e4)),
        ("slab_continuous_held", lambda: pins.test_slab_converges_to_continuous_solution(np.inf)),
        ("ladder_x", lambda: pins.test_lateral_ladder_closed_form("x", 4e4)),
        ("ladder_y", lambda: pins.test_lateral_ladder_closed_form("y", 4e4)),
        ("ladder_x_held", lambda: pins.test_lateral_ladder_closed_form("x", np.inf)),
        ("rhs", pins.test_rhs_total_power_and_placement),
        ("rhs_volume_unit", pins.test_rhs_volume_unit_sources),
        ("rhs_volume_total", pins.test_rhs_volume_paper_stack_total_power),
        ("rhs_volume_chain", pins.test_rhs_volume_chain_closed_form),
        ("finite_termination", pins.test_finite_termination),
        ("textbook_cg", pins.test_single_column_equals_textbook_cg),
        ("deflation", pins.test_deflation_duplicate_and_zero_columns),
        ("combine_apply", pins.test_combine_and_apply_brute_force),
        ("linearity", pins.test_linearity_and_pair_consistency),
        ("pivoted_cholesky", pins.test_pivoted_cholesky_against_library),
        ("philox", pins.test_philox_matches_library_generator),
        ("noise", pins.test_noise_is_uniform_bounded_and_reproducible),
        ("normalised_weights", pins.test_normalised_weights_of_eq5),
    ]
    for chip in pins._chips():
        checks.append(("spd", lambda c=chip: pins.test_operator_symmetric_bitwise_and_spd(c)))
        checks.append(("energy", lambda c=chip: pins.test_energy_balance(c)))
        checks.append(("dense_direct", lambda c=chip: pins.test_block_cg_matches_dense_direct(c)))
    for name, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(name)
    return failed


REAL = {name: getattr(orc, name) for name in
        ("rhs", "rhs_volume", "block_cg", "face_conductances", "_gram_solve", "_series",
         "scaled_pivoted_cholesky", "noise", "combine_normalized")}
REAL_ROBIN = orc._robin


def test_unmutated_oracle_passes_every_pin():
    assert _run_pins() == []


def _mut_series_full_width(area, half_a, k_a, half_b, k_b):
    return area / (half_a / k_a + half_b / k_b)


def _mut_robin_no_half_cell(area, d, k, h):
    return area / (1.0 / h)


def _mut_robin_full_cell(area, d, k, h):
    return area / (d / k + 1.0 / h)


def _mut_robin_held_as_adiabatic(area, d, k, h):
    # a held face (h = inf) treated like an insulated one
    return 0.0 * area if np.isinf(h) else REAL_ROBIN(area, d, k, h)


def _mut_rhs_bottom_layer(chip, density):
    B = REAL["rhs"](chip, density)
    top = chip.nx * chip.ny
    out = np.zeros_like(B)
    out[chip.n - top:] = B[:top]
    return out


def _mut_rhs_volume_no_dz(chip, qv):
    # cell volume taken as dx * dy (the layer thickness dropped)
    B = REAL["rhs_volume"](chip, qv)
    return B / np.repeat(chip.cell_dz(), chip.nx * chip.ny)[:, None]


def _mut_rhs_volume_top_dz(chip, qv):
    # every row given the top row's thickness
    B = REAL["rhs_volume"](chip, qv)
    dz = np.repeat(chip.cell_dz(), chip.nx * chip.ny)[:, None]
    return B / dz * chip.cell_dz()[0]


def _mut_rhs_volume_rows_flipped(chip, qv):
    # z numbered from the bottom
    qv = np.asarray(qv)[:, ::-1].copy()
    return REAL["rhs_volume"](chip, qv)


def _mut_rhs_no_area(chip, density):
    # power density deposited as if it were power per cell
    return REAL["rhs"](chip, density) / (chip.dx * chip.dy)


def _mut_cholesky_no_pivoting(G, tol):
    # columns taken in index order instead of largest remaining pivot first
    s = G.shape[0]
    diag = np.diag(G).copy()
    usable = np.isfinite(diag) & (diag > 0)
    d = np.zeros(s)
    d[usable] = 1.0 / np.sqrt(diag[usable])
    W = d[:, None] * G * d[None, :]
    remaining = [j for j in range(s) if usable[j]]
    kept, cols = [], []
    while remaining:
        piv = remaining[0]
        w = W[piv, piv]
        if not (w > tol):
            break
        col = np.zeros(s)
        col[remaining] = W[remaining, piv] / np.sqrt(w)
        rem = np.ix_(remaining, remaining)
        W[rem] -= np.outer(col[remaining], col[remaining])
        kept.append(piv)
        cols.append(col)
        remaining.remove(piv)
    if not kept:
        return [], np.zeros((0, 0)), d
    return kept, np.stack(cols, axis=1)[kept, :], d


def _mut_noise_wrong_word(seed, cells, M, amp):
    # word index taken from the block number instead of the field
    out = np.empty((M, len(cells)))
    for i, a in enumerate(cells):
        for g in range((M + 3) // 4):
            w = orc.philox4x64_10((int(a), g, 0, 0), (seed, 0))
            for j in range(4):
                m = 4 * g + j
                if m < M:
                    out[m, i] = amp * (2.0 * ((w[g % 4] >> 11) * 2.0 ** -53) - 1.0)
    return out


def _mut_normalize_by_basis_sums(U, C):
    # weights divided by the sums over fields (the wrong axis)
    C = np.asarray(C, np.float64)
    return orc.combine(U, C / C.sum(axis=1, keepdims=True))


def _mut_normalize_by_magnitude(U, C):
    # weights divided by sum |mu| instead of sum mu
    C = np.asarray(C, np.float64)
    return orc.combine(U, C / np.abs(C).sum(axis=0, keepdims=True))


def _mut_combine_no_transpose(U, C):
    return np.asarray(U, np.float64) @ np.asarray(C, np.float64)


def _make_bcg_mutant(kind):
    real = REAL["block_cg"]

    def mutant(A, B, X0=None, rtol=1e-12, maxiter=10000, deflate_tol=1e-14, record=None):
        orig_solve = REAL["_gram_solve"]
        calls = {"n": 0}

        def solve(kept, L, d, Y):
            calls["n"] += 1
            z = orig_solve(kept, L, d, Y)
            if kind == "beta_sign" and calls["n"] % 2 == 0:
                return -z
            if kind == "alpha_scale" and calls["n"] % 2 == 1:
                return 0.5 * z
            return z

        orc._gram_solve = solve
        try:
            return real(A, B, X0, rtol, maxiter, deflate_tol, record)
        finally:
            orc._gram_solve = orig_solve

    return mutant


def _mut_gz_wrong_index(chip):
    f = REAL["face_conductances"](chip)
    k = chip.cell_k()
    dz = chip.cell_dz()[:, None, None]
    f["gz"] = REAL["_series"](chip.dx * chip.dy, dz[:-1], k[:-1], dz[:-1], k[1:])
    return f


MUTANTS = {
    "series_full_width": ("_series", _mut_series_full_width),
    "robin_no_half_cell": ("_robin", _mut_robin_no_half_cell),
    "robin_full_cell": ("_robin", _mut_robin_full_cell),
    "robin_held_as_adiabatic": ("_robin", _mut_robin_held_as_adiabatic),
    "rhs_bottom_layer": ("rhs", _mut_rhs_bottom_layer),
    "combine_no_transpose": ("combine", _mut_combine_no_transpose),
    "rhs_no_area": ("rhs", _mut_rhs_no_area),
    "cholesky_no_pivoting": ("scaled_pivoted_cholesky", _mut_cholesky_no_pivoting),
    "noise_wrong_word": ("noise", _mut_noise_wrong_word),
    "rhs_volume_no_dz": ("rhs_volume", _mut_rhs_volume_no_dz),
    "rhs_volume_top_dz": ("rhs_volume", _mut_rhs_volume_top_dz),
    "rhs_volume_rows_flipped": ("rhs_volume", _mut_rhs_volume_rows_flipped),
    "beta_sign": ("block_cg", _make_bcg_mutant("beta_sign")),
    "alpha_scale": ("block_cg", _make_bcg_mutant("alpha_scale")),
    "gz_wrong_index": ("face_conductances", _mut_gz_wrong_index),
    "normalize_by_basis_sums": ("combine_normalized", _mut_normalize_by_basis_sums),
    "normalize_by_magnitude": ("combine_normalized", _mut_normalize_by_magnitude),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(orc, attr, fn)
    assert _run_pins(), f"mutant {name} passed every pin"
