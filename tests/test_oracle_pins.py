"""Pins of the FP64 oracle against facts fixed by physics and mathematics.

Each test checks the oracle against something other than itself: resistor
networks with closed-form solutions, the continuous layered-slab solution,
dense direct solves, textbook CG, exact algebraic invariants of the
finite-volume operator, and library routines.
"""
import numpy as np
import pytest
import torch

from oracle import blockoa_oracle as orc
from paper_2510_23221_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _chips():
    return [
        synth.random_small_chip(11, 3, 4, 3),
        synth.random_small_chip(12, 5, 2, 4, h_top=3e4, h_bottom=1e3),
        synth.random_small_chip(13, 4, 4, 2, h_top=0.0, h_side=2e4),
        synth.random_small_chip(14, 2, 3, 3, h_top=1e4, h_bottom=5e3, h_side=1e3,
                                layer_nz=[2, 1, 3]),
        # Dirichlet faces (h = inf, held at the reference temperature): all
        # faces, and Robin top/bottom with Dirichlet sides
        synth.random_small_chip(15, 4, 3, 3, h_top=np.inf, h_bottom=np.inf, h_side=np.inf),
        synth.random_small_chip(16, 5, 4, 3, h_top=3e4, h_bottom=3e4, h_side=np.inf),
    ]


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("chip", _chips())
def test_operator_symmetric_bitwise_and_spd(chip):
    A = orc.assemble(chip)
    D = A.toarray()
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    np.linalg.cholesky(D)
    x = np.random.default_rng(0).standard_normal((chip.n, 16))
    assert np.all(np.einsum("ij,ij->j", x, A @ x) > 0)


@pytest.mark.parametrize("chip", _chips())
def test_energy_balance(chip):
    """Interior fluxes telescope: sum_a (A theta)_a equals the Robin heat loss."""
    theta = np.random.default_rng(1).standard_normal((chip.n, 5))
    q = orc.apply_operator(orc.assemble(chip), theta.T)
    loss = orc.boundary_loss(chip, theta)
    scale = np.abs(q).sum(axis=1)
    assert np.all(np.abs(q.sum(axis=1) - loss) <= 1e-13 * scale)


def test_row_sums_vanish_without_robin_faces():
    """With every face adiabatic a uniform temperature carries no flux."""
    chip = synth.random_small_chip(21, 4, 3, 3, h_top=0.0)
    A = orc.assemble(chip)
    assert np.max(np.abs(A @ np.ones(chip.n))) <= 1e-16 * abs(A).max()


def _cg_textbook(A, b, tol, maxiter, record=None):
    """Hestenes-Stiefel CG with rho = r.r (independent of the block form)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = r @ r
    it = 0
    while np.sqrt(rho) > tol * np.linalg.norm(b) and it < maxiter:
        Ap = A @ p
        a = rho / (p @ Ap)
        x = x + a * p
        r = r - a * Ap
        rho_new = r @ r
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
        if record is not None:
            record.append(x.copy())
    return x, it


@pytest.mark.parametrize("h_top", [2.5e4, np.inf])
def test_slab_resistor_chain_closed_form(h_top):
    """Power only in the bottom layer, adiabatic sides: the solution is the
    series resistor chain.  The thermal resistance of a slab of thickness t
    and conductivity k over area S is t / (k S); convection is 1 / (h S),
    zero for a top face held at the reference temperature (h = inf)."""
    chip = synth.Chip(nx=3, ny=2, layer_nz=np.ones(5, np.int32),
                      layer_dz=np.array([40e-6, 15e-6, 90e-6, 60e-6, 120e-6]),
                      layer_k=np.array([150.0, 4.0, 390.0, 25.0, 1.5]), h_top=h_top)
    S = chip.dx * chip.dy
    p = 0.0375  # W in every bottom cell
    B = np.zeros((chip.n, 1))
    B[-chip.nx * chip.ny:, 0] = p
    U, info = orc.block_cg(orc.assemble(chip), B, rtol=1e-15, maxiter=200)
    theta = U[:, 0].reshape(chip.nz, chip.ny, chip.nx)
    t, k = chip.layer_dz, chip.layer_k
    expect = np.empty(5)
    expect[0] = p * (t[0] / 2 / (k[0] * S) + 1.0 / (chip.h_top * S))
    for l in range(4):
        expect[l + 1] = expect[l] + p * (t[l] / 2 / (k[l] * S) + t[l + 1] / 2 / (k[l + 1] * S))
    assert np.allclose(theta, expect[:, None, None], rtol=1e-13, atol=0)


def _continuous_slab(z, tops, k, g, h):
    """Exact theta(z) of -(k theta')' = g in the bottom layer, adiabatic bottom,
    h theta = k theta' at z = 0 (z points down from the cooled surface)."""
    L, zb = tops[-1], tops[-2]
    F0 = g * (L - zb)          # upward flux through every plane above the heated layer
    out = np.empty_like(z)
    for i, zz in enumerate(z):
        th = F0 / h
        for l in range(len(k) - 1):          # unheated layers: linear profile
            th += F0 * (np.clip(zz, tops[l], tops[l + 1]) - tops[l]) / k[l]
        if zz > zb:                           # heated layer: quadratic profile
            th += g / k[-1] * ((L - zb) ** 2 / 2 - (L - zz) ** 2 / 2)
        out[i] = th
    return out


@pytest.mark.parametrize("h", [1e4, np.inf])
def test_slab_converges_to_continuous_solution(h):
    """Refining every layer along z must converge to the continuous
    piecewise-linear / quadratic slab profile at second order, with a
    convective top or a top held at the reference temperature (h = inf)."""
    t = np.array([150e-6, 20e-6, 150e-6, 200e-6])
    k = np.array([150.0, 5.0, 400.0, 20.0])
    g = 2e9                    # W/m^3 in the bottom layer
    tops = np.concatenate([[0.0], np.cumsum(t)])
    errs = []
    for N in (1, 2, 4, 8, 16):
        chip = synth.Chip(nx=1, ny=1, layer_nz=np.full(4, N, np.int32),
                          layer_dz=t / N, layer_k=k, h_top=h)
        dz = chip.cell_dz()
        zc = np.cumsum(dz) - dz / 2
        B = np.zeros((chip.n, 1))
        bottom = zc > tops[-2]
        B[bottom, 0] = g * chip.dx * chip.dy * dz[bottom]
        A = orc.assemble(chip)
        theta = np.linalg.solve(A.toarray(), B[:, 0])
        exact = _continuous_slab(zc, tops, k, g, h)
        errs.append(np.max(np.abs(theta - exact)) / np.max(exact))
    errs = np.array(errs)
    # the held top has the larger error constant (1.9e-3 at N = 8, 4.7e-4 at
    # N = 16); both converge at second order
    assert errs[-1] < (1e-4 if np.isfinite(h) else 1e-3)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order > 1.8), (errs, order)


@pytest.mark.parametrize("h", [4e4, np.inf])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_lateral_ladder_closed_form(axis, h):
    """One row of N cells cooled from the top, power p in the first cell:
    theta_i = c (r^i + r^(2N-1-i)) with r + 1/r = 2 + Gb/G (a top held at
    the reference temperature for h = inf)."""
    N, kk, p = 9, 120.0, 0.02
    nx, ny = (N, 1) if axis == "x" else (1, N)
    chip = synth.Chip(nx=nx, ny=ny, layer_nz=np.ones(1, np.int32),
                      layer_dz=np.array([70e-6]), layer_k=np.array([kk]), h_top=h,
                      dx=110e-6, dy=90e-6)
    dz = 70e-6
    S_top = chip.dx * chip.dy
    if axis == "x":
        G = kk * chip.dy * dz / chip.dx
    else:
        G = kk * chip.dx * dz / chip.dy
    Gb = 1.0 / (dz / 2 / (kk * S_top) + 1.0 / (h * S_top))
    a = 2 + Gb / G
    r = (a - np.sqrt(a * a - 4)) / 2
    c = p / (G * (1 - r) * (1 / r - r ** (2 * N - 1)))
    i = np.arange(N)
    expect = c * (r ** i + r ** (2 * N - 1 - i))
    B = np.zeros((N, 1))
    B[0, 0] = p
    U, info = orc.block_cg(orc.assemble(chip), B, rtol=1e-15, maxiter=500)
    assert np.allclose(U[:, 0], expect, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- right-hand side
def test_rhs_total_power_and_placement():
    chip = synth.random_small_chip(5, 6, 5, 3)
    rng = np.random.default_rng(3)
    dens = np.stack([synth.rect_power_map(rng, 6, 5), synth.gauss_power_map(rng, 6, 5)])
    B = orc.rhs(chip, dens)
    assert B.shape == (chip.n, 2)
    assert np.allclose(B.sum(axis=0), dens.sum(axis=(1, 2)) * chip.dx * chip.dy, rtol=1e-14)
    assert np.all(B[chip.nx * chip.ny:] == 0)
    # cell (x=2, y=3) of map 1
    assert B[3 * 6 + 2, 1] == dens[1, 3, 2] * (chip.dx * chip.dy)


def test_rhs_volume_unit_sources():
    """A volumetric source of P / V_a in one cell a (V_a = dx dy times the
    thickness of a's layer, taken from the layer table) is P watts in cell a
    and nothing elsewhere, for cells in layers of different thickness."""
    chip = synth.random_small_chip(9, 4, 3, 4, layer_nz=[2, 1, 3, 1])
    nxny = chip.nx * chip.ny
    layer_of_row = np.repeat(np.arange(4), chip.layer_nz)
    cells = [(0, 1, 2), (2, 0, 3), (3, 2, 1), (6, 1, 0)]   # (z, y, x)
    P = 0.125
    qv = np.zeros((len(cells), chip.nz, chip.ny, chip.nx))
    for j, (z, y, x) in enumerate(cells):
        qv[j, z, y, x] = P / (chip.dx * chip.dy * chip.layer_dz[layer_of_row[z]])
    B = orc.rhs_volume(chip, qv)
    assert B.shape == (chip.n, len(cells))
    for j, (z, y, x) in enumerate(cells):
        a = z * nxny + y * chip.nx + x
        assert B[a, j] == pytest.approx(P, rel=1e-15)
        assert np.count_nonzero(B[:, j]) == 1


def test_rhs_volume_paper_stack_total_power():
    """On the 3-D IC stack every draw's total power is the sum over device
    layers of areal density times cell area (the TIM layers carry none)."""
    chip = synth.paper_3dic_chip(3, nx=13, ny=14, device_cells=2)
    qv = synth.paper_3dic_sources(np.random.default_rng(3), chip, 2)
    B = orc.rhs_volume(chip, qv)
    t_dev = synth.PAPER_3DIC["device_dz_m"]
    first_rows = [0, 3, 6]                      # first z-row of each device layer
    areal = qv[:, first_rows] * t_dev           # W/m^2 per device layer
    expect = areal.sum(axis=(1, 2, 3)) * chip.dx * chip.dy
    assert np.allclose(B.sum(axis=0), expect, rtol=1e-13)
    tim_rows = [2, 5, 8]
    nxny = chip.nx * chip.ny
    for z in tim_rows:
        assert np.all(B[z * nxny:(z + 1) * nxny] == 0)


def test_rhs_volume_chain_closed_form():
    """Laterally uniform sources in all three device layers of the 3-D IC
    stack, Robin top, insulated elsewhere: the heat of every cell leaves
    through the top, so the flux through the face below row z is the power
    of the rows beneath it, and the solution is the series resistor chain
    (half-cell resistances dz / (2 k S), convection 1 / (h S))."""
    chip = synth.paper_3dic_chip(0, nx=3, ny=2, device_cells=2, tsv_bundles=0)
    chip.h_top, chip.h_bottom, chip.h_side = 2e4, 0.0, 0.0
    S = chip.dx * chip.dy
    qrow = np.zeros(chip.nz)
    qrow[[0, 1]] = 4e9
    qrow[[3, 4]] = 2e8
    qrow[[6, 7]] = 1.5e8
    qv = np.broadcast_to(qrow[None, :, None, None], (1, chip.nz, chip.ny, chip.nx)).copy()
    B = orc.rhs_volume(chip, qv)
    U, info = orc.block_cg(orc.assemble(chip), B, rtol=1e-15, maxiter=400)
    theta = U[:, 0].reshape(chip.nz, chip.ny, chip.nx)
    dz = np.repeat(chip.layer_dz, chip.layer_nz)
    k = np.repeat(chip.layer_k, chip.layer_nz)
    p = qrow * S * dz                          # W per cell of row z
    below = np.cumsum(p[::-1])[::-1]            # power of rows z .. bottom
    expect = np.empty(chip.nz)
    expect[0] = below[0] * (dz[0] / (2 * k[0] * S) + 1.0 / (chip.h_top * S))
    for z in range(chip.nz - 1):
        expect[z + 1] = expect[z] + below[z + 1] * (dz[z] / (2 * k[z] * S) + dz[z + 1] / (2 * k[z + 1] * S))
    assert np.allclose(theta, expect[:, None, None], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- block CG
@pytest.mark.parametrize("chip", _chips())
def test_block_cg_matches_dense_direct(chip):
    rng = np.random.default_rng(7)
    B = rng.uniform(0, 1e-2, (chip.n, 3))
    A = orc.assemble(chip)
    U, info = orc.block_cg(A, B, rtol=1e-13, maxiter=1000)
    assert info["status"] == orc.STATUS_OK
    ref = np.linalg.solve(A.toarray(), B)
    err = np.linalg.norm(U - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert np.all(err < 1e-11), err


def test_finite_termination():
    """Exact-arithmetic block CG ends after ceil(n/s) = 6 block steps: the
    residual collapses at step 6 and not before."""
    chip = synth.Chip(nx=4, ny=4, layer_nz=np.ones(3, np.int32),
                      layer_dz=np.full(3, 50e-6), layer_k=np.array([150.0, 40.0, 150.0]),
                      h_top=3e4)
    A = orc.assemble(chip)
    B = np.random.default_rng(8).standard_normal((chip.n, 8))

    def relres(iters):
        X, info = orc.block_cg(A, B, rtol=1e-30, maxiter=iters)
        return np.max(np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0))

    r5, r6 = relres(5), relres(6)
    assert r5 > 1e-1
    assert r6 < 1e-7 * r5


def test_single_column_equals_textbook_cg():
    chip = synth.reference_stack_chip()
    chip.nx = chip.ny = 8
    A = orc.assemble(chip)
    b = np.random.default_rng(9).uniform(0, 1e-3, chip.n)
    rec_b, rec_t = [], []
    orc.block_cg(A, b[:, None], rtol=1e-14, maxiter=30, record=rec_b)
    _cg_textbook(A, b, 1e-14, 30, record=rec_t)
    assert len(rec_b) == len(rec_t) == 30
    for xb, xt in zip(rec_b, rec_t):
        assert np.linalg.norm(xb[:, 0] - xt) <= 1e-9 * np.linalg.norm(xt)


def test_deflation_duplicate_and_zero_columns():
    chip = synth.random_small_chip(31, 6, 5, 3)
    A = orc.assemble(chip)
    rng = np.random.default_rng(10)
    B = rng.uniform(0, 1e-2, (chip.n, 5))
    B[:, 3] = B[:, 1]
    B[:, 4] = 0.0
    U, info = orc.block_cg(A, B, rtol=1e-12, maxiter=1000)
    assert info["status"] == orc.STATUS_OK
    assert info["deflated"] > 0
    assert np.all(U[:, 4] == 0.0)
    assert np.linalg.norm(U[:, 3] - U[:, 1]) <= 1e-12 * np.linalg.norm(U[:, 1])
    ref = np.linalg.solve(A.toarray(), B[:, :3])
    assert np.allclose(U[:, :3], ref, rtol=1e-10, atol=0)


def test_block_needs_fewer_iterations_than_single_cg():
    """Sharing one Krylov space across columns cuts iterations (Sec. V-E)."""
    chip = synth.reference_stack_chip()
    chip.nx = chip.ny = 16
    A = orc.assemble(chip)
    rng = np.random.default_rng(12)
    dens = np.stack([synth.rect_power_map(rng, 16, 16) for _ in range(8)])
    B = orc.rhs(chip, dens)
    _, info = orc.block_cg(A, B, rtol=1e-8, maxiter=5000)
    single = max(orc.block_cg(A, B[:, [j]], rtol=1e-8, maxiter=5000)[1]["iters"] for j in range(8))
    assert info["iters"] < single


def test_not_converged_and_breakdown_status():
    chip = synth.random_small_chip(41, 4, 4, 3)
    A = orc.assemble(chip)
    B = np.random.default_rng(1).uniform(0, 1, (chip.n, 2))
    _, info = orc.block_cg(A, B, rtol=1e-14, maxiter=2)
    assert info["status"] == orc.STATUS_NOT_CONVERGED and info["iters"] == 2
    B[0, 0] = np.nan
    _, info = orc.block_cg(A, B, rtol=1e-14, maxiter=10)
    assert info["status"] == orc.STATUS_BREAKDOWN


def test_pivoted_cholesky_against_library():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((6, 6))
    G = M @ M.T + 6 * np.eye(6)
    kept, L, d = orc.scaled_pivoted_cholesky(G, 1e-14)
    assert sorted(kept) == list(range(6))
    S = (d[:, None] * G * d[None, :])[np.ix_(kept, kept)]
    assert np.allclose(L @ L.T, S, rtol=0, atol=1e-13)
    assert np.allclose(np.tril(L), L)
    # pivots decrease (largest remaining diagonal first)
    assert np.all(np.diff(np.diag(L)) <= 1e-15)
    # rank-deficient: third column is a combination of the first two
    V = rng.standard_normal((10, 4))
    V[:, 2] = V[:, 0] - 2 * V[:, 1]
    kept, L, d = orc.scaled_pivoted_cholesky(V.T @ V, 1e-12)
    assert len(kept) == 3


# ---------------------------------------------------------------- combine / apply
def test_combine_and_apply_brute_force():
    chip = synth.random_small_chip(51, 3, 2, 2)
    A = orc.assemble(chip)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((chip.n, 3))
    C = synth.coefficients(rng, 3, 4)
    T = orc.combine(U, C)
    D = A.toarray()
    for m in range(4):
        for a in range(chip.n):
            ref = sum(C[i, m] * U[a, i] for i in range(3))
            assert abs(T[m, a] - ref) <= 1e-15 * max(1.0, abs(ref)) * 4
    q = orc.apply_operator(A, T)
    for m in range(4):
        for a in range(chip.n):
            ref = sum(D[a, b] * T[m, b] for b in range(chip.n))
            assert abs(q[m, a] - ref) <= 1e-13 * np.abs(D[a]).sum() * np.abs(T[m]).max()


def test_linearity_and_pair_consistency():
    """A (U C) = (A U) C, and q = A T reproduces B C up to the basis residual."""
    w = synth.small_fp64_workload(M=16)
    chip = w.chips[0]
    out = orc.generate(chip, w.density[0], w.coeffs[0], rtol=1e-12)
    A, U, C = out["A"], out["U"], w.coeffs[0]
    lin = ((A @ U) @ C).T
    assert np.allclose(out["q"], lin, rtol=0, atol=1e-12 * np.abs(lin).max())
    BC = (out["B"] @ C).T
    rel = np.linalg.norm(out["q"] - BC, axis=1) / np.linalg.norm(BC, axis=1)
    assert np.all(rel < 1e-10)
    e = orc.pair_errors(A, U, C, out["T"], out["q"])
    assert np.all(e["e_T"] == 0) and np.all(e["e_pair"] < 1e-15)
    # a planted error in one stored field shows in e_pair of that field only
    T2 = out["T"].copy()
    T2[3, 100] *= 1 + 1e-6
    e2 = orc.pair_errors(A, U, C, T2, out["q"])
    assert e2["e_pair"][3] > 1e-9 and np.all(np.delete(e2["e_pair"], 3) < 1e-15)


# ---------------------------------------------------------------- inputs
def test_philox_matches_library_generator():
    """The oracle's Philox4x64-10 block equals numpy's Philox bit generator,
    which draws block (counter + 1) first."""
    rng = np.random.default_rng(4)
    for t in range(40):
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2, dtype=np.uint64)]
        ctr = [int(x) for x in rng.integers(1, 2 ** 63, 4, dtype=np.uint64)]
        if t == 0:
            key, ctr = [0, 0], [1, 0, 0, 0]
        bg = np.random.Philox(counter=np.array([ctr[0] - 1] + ctr[1:], dtype=np.uint64),
                              key=np.array(key, dtype=np.uint64))
        assert [int(x) for x in bg.random_raw(4)] == orc.philox4x64_10(ctr, key)


def test_noise_is_uniform_bounded_and_reproducible():
    amp, M = 0.01, 64
    cells = np.arange(1000, 1600)
    e = orc.noise(77, cells, M, amp)
    assert e.shape == (M, len(cells))
    assert np.all(e >= -amp) and np.all(e < amp)
    N = e.size
    assert abs(e.mean()) < 4 * amp / np.sqrt(3 * N)             # mean 0, sd amp / sqrt(3)
    assert abs(e.var() / (amp * amp / 3) - 1) < 0.05
    assert np.array_equal(e, orc.noise(77, cells, M, amp))
    assert np.array_equal(e[:, 5:9], orc.noise(77, cells[5:9], M, amp))   # per cell, not per call
    assert not np.allclose(e, orc.noise(78, cells, M, amp))
    # 4 fields per generator block: fields 4g..4g+3 are one block's four words
    w = orc.philox4x64_10((int(cells[0]), 3, 0, 0), (77, 0))
    assert np.allclose(e[12:16, 0], [amp * (2 * ((x >> 11) * 2.0 ** -53) - 1) for x in w], rtol=0, atol=0)


def test_gaussian_noise_is_normal_reproducible_and_apart_from_the_uniform_stream():
    from scipy import stats
    sigma, M = 0.02, 32
    cells = np.arange(500, 1100)
    e = orc.noise_gaussian(91, cells, M, sigma)
    assert e.shape == (M, len(cells)) and np.all(np.isfinite(e))
    x = e.ravel() / sigma
    N = x.size
    assert abs(x.mean()) < 5 / np.sqrt(N) and abs(x.std() - 1) < 5 / np.sqrt(2 * N)
    assert stats.kstest(x, "norm").pvalue > 1e-3                 # the normal law, not just two moments
    assert abs(stats.kurtosis(x)) < 0.1
    assert np.array_equal(e[:, 7:11], orc.noise_gaussian(91, cells[7:11], M, sigma))
    u = orc.noise(91, cells, M, 1.0)                             # same seed, uniform stream
    assert abs(np.corrcoef(u.ravel(), x)[0, 1]) < 5 / np.sqrt(N)
    # one generator block per two fields: Box-Muller of words (0, 1) and (2, 3)
    w = orc.philox4x64_10((int(cells[3]), 5, 1, 0), (91, 0))
    u1, u2 = ((w[2] >> 11) + 0.5) * 2.0 ** -53, (w[3] >> 11) * 2.0 ** -53
    assert e[11, 3] == sigma * np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)


def test_normalised_weights_of_eq5():
    """Eq. 5's weights sum to one per field: (i) a basis whose columns are all
    the same field v combines to v for every field, whatever the
    coefficients (a normalisation by the wrong axis or by sum |mu| breaks
    this); (ii) scaling one field's coefficients leaves that field -- and
    every other field -- unchanged; (iii) weights that already sum to one
    give the plain combination."""
    rng = np.random.default_rng(12)
    n, s, M = 40, 6, 9
    v = rng.standard_normal(n)
    C = rng.standard_normal((s, M)) + 0.3
    T = orc.combine_normalized(np.repeat(v[:, None], s, axis=1), C)
    assert np.allclose(T, np.broadcast_to(v, (M, n)), rtol=1e-12, atol=1e-12)
    U = rng.standard_normal((n, s))
    T0 = orc.combine_normalized(U, C)
    C2 = C.copy()
    C2[:, 4] *= -3.5
    assert np.allclose(orc.combine_normalized(U, C2), T0, rtol=1e-12, atol=1e-12)
    A = C / C.sum(axis=0, keepdims=True)
    assert np.allclose(orc.combine_normalized(U, A), orc.combine(U, A), rtol=1e-12, atol=1e-12)
    assert not np.allclose(T0, orc.combine(U, C))


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(5).standard_normal(4096)
    ours = synth.round_to_bf16(x)
    lib = torch.tensor(x, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    # torch rounds float64 -> bfloat16 directly with round-half-even
    assert np.array_equal(ours, lib)


def test_workload_recipes_are_seeded():
    a = synth.small_fp64_workload()
    b = synth.small_fp64_workload()
    assert np.array_equal(a.density[0], b.density[0]) and np.array_equal(a.coeffs[0], b.coeffs[0])
    assert a.density[0].shape == (8, 32, 32) and a.coeffs[0].shape == (8, 64)
    w = synth.batched_workload(n_chips=6)
    assert len(w.chips) == 6 and all(c.nx in (64, 96, 128, 192, 256) for c in w.chips)
    assert all(4 <= c.nz <= 12 for c in w.chips)
